"""Pins for the preconditioner-network oracle (oracle/nn.py), independent of its own code:

* gauge covariance N[U^G](G r) = G N[U](r) (colour-blind weights, invariant gates);
* a special case that reduces to the C oracle: with the gates open (sigmoid -> 1)
  and weights +1 / -1 on the forward / backward hops of layers 1 and 2 (identity
  layer 3), the network is D_fat D_fat, i.e. -(D_eo D_oe) with zero long links;
* scale covariance N(c r) = c N(r);
* finite-difference checks of the loss gradient (both loss norms) for weights of
  every layer, real and imaginary parts, and for the gate parameters;
* the A^2-norm loss equals |A N(r) - r|^2 / |r|^2 computed directly.
"""

import numpy as np
import pytest

import oracle
import oracle.nn as nn
import synth

L = (4, 4, 4, 6)


def test_gauge_covariance():
    fat, lng = synth.fat_long_links(L, 3)
    G = synth.random_gauge(L, 4)
    params = nn.init_params(1, scale=0.6)
    r = synth.gaussian_source(L, 5)
    z = nn.apply(L, fat, params, r)
    zg = nn.apply(L, synth.gauge_transform_links(L, fat, G, 1), params,
                  synth.gauge_transform_parity_field(L, r, G, 0))
    assert np.linalg.norm(zg - synth.gauge_transform_parity_field(L, z, G, 0)) <= 1e-12 * np.linalg.norm(z)


def test_hop_weights_reduce_to_fat_dslash_squared():
    fat, lng = synth.fat_long_links(L, 6)
    params = nn.init_params(0)
    for W in params["W"]:
        W[:] = 0
    for mu in range(4):
        params["W"][0][1 + 2 * mu, 0, 0] = 1.0
        params["W"][0][2 + 2 * mu, 0, 0] = -1.0
        params["W"][1][1 + 2 * mu, 0, 0] = 1.0
        params["W"][1][2 + 2 * mu, 0, 0] = -1.0
    params["W"][2][0, 0, 0] = 1.0
    params["gates"] = [(np.zeros(8), np.full(8, 60.0)), (np.zeros(8), np.full(8, 60.0))]
    r = synth.gaussian_source(L, 7)
    z = nn.apply(L, fat, params, r)
    want = -oracle.normal_op(L, fat, np.zeros_like(lng), 0.0, r)  # D_eo D_oe r with fat links only
    assert np.linalg.norm(z - want) <= 1e-12 * np.linalg.norm(want)


def test_scale_covariance():
    fat, _ = synth.fat_long_links(L, 8)
    params = nn.init_params(2, scale=0.8)
    r = synth.gaussian_source(L, 9)
    assert np.allclose(nn.apply(L, fat, params, 3.7 * r), 3.7 * nn.apply(L, fat, params, r), rtol=1e-12, atol=0)


def _perturbed(params, which, eps):
    p = {"W": [w.copy() for w in params["W"]], "gates": [(a.copy(), b.copy()) for a, b in params["gates"]]}
    kind, idx, part = which
    if kind == "W":
        l, tap, o, i = idx
        p["W"][l][tap, o, i] += eps * (1 if part == "re" else 1j)
    else:
        l, ab, c = idx
        p["gates"][l][ab][c] += eps
    return p


@pytest.mark.parametrize("norm", [1, 2])
@pytest.mark.parametrize("which", [
    ("W", (0, 0, 3, 0), "re"), ("W", (0, 5, 1, 0), "im"), ("W", (1, 2, 4, 6), "re"), ("W", (1, 7, 0, 3), "im"),
    ("W", (2, 0, 0, 5), "im"), ("W", (2, 8, 0, 2), "re"), ("G", (0, 0, 2), None), ("G", (0, 1, 5), None),
    ("G", (1, 0, 7), None), ("G", (1, 1, 1), None)])
def test_gradient_matches_finite_differences(which, norm):
    fat, lng = synth.fat_long_links(L, 10)
    sigma = 0.05
    params = nn.init_params(3, scale=0.7)
    r = synth.gaussian_source(L, 11)
    e = np.linalg.solve(oracle.dense_normal_matrix(L, fat, lng, sigma), r.ravel()).reshape(r.shape)
    loss, grads = nn.loss_and_grad(L, fat, lng, params, r, e, sigma, norm=norm)
    eps = 1e-6
    lp, _ = nn.loss_and_grad(L, fat, lng, _perturbed(params, which, eps), r, e, sigma, norm=norm)
    lm, _ = nn.loss_and_grad(L, fat, lng, _perturbed(params, which, -eps), r, e, sigma, norm=norm)
    fd = (lp - lm) / (2 * eps)
    kind, idx, part = which
    if kind == "W":
        l, tap, o, i = idx
        g = grads["W"][l][tap, o, i]
        an = g.real if part == "re" else g.imag
    else:
        l, ab, c = idx
        an = grads["gates"][l][ab][c]
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_residual_norm_loss_is_the_preconditioned_residual():
    fat, lng = synth.fat_long_links(L, 12)
    sigma = 0.05
    params = nn.init_params(4, scale=0.5)
    r = synth.gaussian_source(L, 13)
    e = np.linalg.solve(oracle.dense_normal_matrix(L, fat, lng, sigma), r.ravel()).reshape(r.shape)
    loss, _ = nn.loss_and_grad(L, fat, lng, params, r, e, sigma, norm=2)
    z = nn.apply(L, fat, params, r)
    want = np.linalg.norm(oracle.normal_op(L, fat, lng, sigma, z) - r) ** 2 / np.linalg.norm(r) ** 2
    assert abs(loss - want) <= 1e-10 * want


def test_bf16_rounding_of_the_rounded_oracle_test_is_round_to_nearest_even():
    """The tensor-core network test inserts BF16 rounding into the oracle with its own bit arithmetic;
    that rounding must be the conversion the GPU's cvt.rn.bf16x2 performs: round to nearest, ties to
    even (the same as PyTorch's float32 -> bfloat16 cast on the CPU), on random values and exact ties."""
    torch = pytest.importorskip("torch")
    from tests.test_gpu_nn import bf16c

    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(4096) * 10.0 ** rng.integers(-20, 20, 4096),
                        [0.0, -0.0, 1.0, -1.0, 3.0e38, -3.0e38, 1e-40]]).astype(np.float32)
    # exact ties: the 16 dropped bits are 0x8000; the kept upper halves (sign, exponent, 7 mantissa bits)
    # are drawn over both signs and exponents 2^-64 .. 2^63, so the kept last bit is even and odd
    upper = rng.integers(0x1F80, 0x5F00, 1024, dtype=np.uint32) | (rng.integers(0, 2, 1024, dtype=np.uint32) << 15)
    ties = ((upper << np.uint32(16)) | np.uint32(0x8000)).view(np.float32)
    assert np.all(np.isfinite(ties)) and len(set(upper & 1)) == 2
    for v in (x, ties):
        want = torch.from_numpy(v.copy()).to(torch.bfloat16).to(torch.float64).numpy()
        got = bf16c(v.astype(np.float64) + 0j).real
        assert np.array_equal(got, want)
        got_im = bf16c(1j * v.astype(np.float64)).imag
        assert np.array_equal(got_im, want)
