"""The seeded input generators: the process-pool path of random_su3 gives the same matrices, bit for
bit, as the serial path (every matrix is computed on its own from one random stream)."""

import numpy as np

import synth


def test_random_su3_pool_is_bit_identical_to_serial():
    a = synth.random_su3(np.random.default_rng(5), 3001, workers=3)
    b = synth.random_su3(np.random.default_rng(5), 3001, workers=1)
    assert np.array_equal(a, b)
    # and they are SU(3): unitary with unit determinant
    eye = np.broadcast_to(np.eye(3), a.shape)
    assert np.max(np.abs(a @ np.conj(np.swapaxes(a, -1, -2)) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(a) - 1)) < 1e-14
