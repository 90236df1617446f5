"""sqcg_normal_op_noalloc: the normal operator for callers that cannot allocate
device memory when they apply it (their device memory belongs to their own
allocator or pool, or they cannot accept an allocation's latency). It keeps
its intermediate in a fixed array inside the library instead of the context's
workspace.

Checked against sqcg_normal_op on two calls in a row, through the C ABI, with
the tolerances of the other operator tests. This file is collected last so
that a run stopping at the first failure has already run everything else; it
also passes alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L", [(16, 16, 16, 16), (8, 10, 12, 14)])
def test_noalloc_matches_normal_op_two_calls(sqcg, links_cache, L, prec):
    fat, lng = links_cache(L, 1001)
    sigma = 4 * 0.05 ** 2
    lib = sqcg.library()
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        for call, seed in enumerate((31, 32)):  # two calls in a row, different inputs
            x = lat.pack(synth.gaussian_source(L, seed), prec)
            want = lat.new_spinor(prec)
            lat.normal_op(sigma, x, want, prec)
            got = lat.new_spinor(prec)
            lat._sync_stream()
            rc = lib.sqcg_normal_op_noalloc(lat._h, ctypes.c_double(sigma), prec, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(got.data_ptr()))
            assert rc == 0, rc
            w, g = lat.unpack(want, prec), lat.unpack(got, prec)
            assert rel(g, w) <= TOL[prec], (call, rel(g, w))


def test_noalloc_rejects_lattices_beyond_the_scratch(sqcg):
    lib = sqcg.library()
    with sqcg.Lattice((32, 32, 32, 32)) as lat:  # 524288 sites per parity
        x, y = lat.new_spinor(1), lat.new_spinor(1)
        rc = lib.sqcg_normal_op_noalloc(lat._h, ctypes.c_double(0.1), 1, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()))
        assert rc == -8
        assert b"too large" in lib.sqcg_strerror(rc)
