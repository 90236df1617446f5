"""Pins for the FP64 CPU oracle: facts fixed by the mathematics of the improved
staggered operator, independent of the oracle's own code.

The paper (arXiv:1611.00728) prints no formula, no worked example and no
residual history, so nothing numeric can come from it. Every check below is a
closed form, an invariant, or a brute-force dense solve:

* free field (unit links times c1, c3): D on a plane wave gives
  sum_mu eta_mu(n) 2i (c1 sin p_mu + c3 sin 3p_mu) times the wave, and
  -D_eo D_oe has eigenvalue 4 sum_mu (c1 sin p_mu + c3 sin 3p_mu)^2
  (phases cancel in D^2 because eta_nu flips under an odd hop in mu < nu);
* anti-Hermiticity D_eo^+ = -D_oe on random links;
* gauge covariance D[U^G] (G psi) = G D[U] psi;
* normal operator Hermitian and bounded below by sigma;
* CG solution equal to a dense LU solve (numpy) on 4^4;
* closed-form free-field solves for one and many shifts.
"""

import numpy as np
import pytest

import oracle
import synth

LATTICES = [(4, 4, 4, 4), (6, 8, 10, 12), (8, 10, 12, 14)]


def eta(mu, c):
    """eta_mu(n) in the MILC convention, x fastest."""
    return np.where(c[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0) if mu > 0 else np.ones(len(c))


def momenta(L, k, apbc):
    p = [2 * np.pi * k[mu] / L[mu] for mu in range(3)]
    p.append((2 * k[3] + (1 if apbc else 0)) * np.pi / L[3])
    return np.array(p)


def free_lambda(L, k, c1, c3, apbc):
    p = momenta(L, k, apbc)
    return 4.0 * np.sum((c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def random_parity_field(L, seed):
    return synth.gaussian_source(L, seed)


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("apbc", [True, False])
def test_free_field_single_hop_closed_form(L, apbc):
    c1, c3 = 1.125, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    rng = np.random.default_rng(7)
    for trial in range(3):
        k = tuple(int(v) for v in rng.integers(0, 8, size=4))
        colour = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        for out_par in (0, 1):
            psi = synth.plane_wave(L, k, 1 - out_par, colour, apbc)
            got = oracle.dslash(L, fat, lng, psi, out_par, apbc)
            c = synth.site_coords(L)[synth.parity_sites(L, out_par)]
            p = momenta(L, k, apbc)
            wave = synth.plane_wave(L, k, out_par, colour, apbc)
            coef = sum(eta(mu, c) * 2j * (c1 * np.sin(p[mu]) + c3 * np.sin(3 * p[mu])) for mu in range(4))
            want = coef[:, None] * wave
            # phases exp(i p.n) carry ~|p.n| ulp of rounding: relative 1e-12
            assert rel(got, want) < 1e-12


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("apbc", [True, False])
def test_free_field_normal_spectrum(L, apbc):
    c1, c3 = 0.9, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    sigma = 4 * 0.1**2
    for k in [(0, 0, 0, 0), (1, 2, 3, 1), (2, 1, 0, 3), (L[0] // 2 - 1, 1, L[2] - 1, 2)]:
        x = synth.plane_wave(L, k, 0, (0.3, -1.0, 0.5j), apbc)
        Ax = oracle.normal_op(L, fat, lng, sigma, x, apbc)
        lam = free_lambda(L, k, c1, c3, apbc)
        assert rel(Ax, (sigma + lam) * x) < 1e-13


@pytest.mark.parametrize("L", LATTICES)
def test_anti_hermiticity(L):
    fat, lng = synth.fat_long_links(L, seed=11)
    y_e = random_parity_field(L, 1)
    x_o = random_parity_field(L, 2)
    lhs = np.vdot(y_e, oracle.dslash(L, fat, lng, x_o, 0))  # <y_e, D_eo x_o>
    rhs = np.vdot(oracle.dslash(L, fat, lng, y_e, 1), x_o)  # <D_oe y_e, x_o>
    assert abs(lhs + rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("out_par", [0, 1])
def test_gauge_covariance(L, out_par):
    fat, lng = synth.fat_long_links(L, seed=12)
    G = synth.random_gauge(L, seed=13)
    fat_g = synth.gauge_transform_links(L, fat, G, 1)
    lng_g = synth.gauge_transform_links(L, lng, G, 3)
    psi = random_parity_field(L, 3)
    lhs = oracle.dslash(L, fat_g, lng_g, synth.gauge_transform_parity_field(L, psi, G, 1 - out_par), out_par)
    rhs = synth.gauge_transform_parity_field(L, oracle.dslash(L, fat, lng, psi, out_par), G, out_par)
    assert rel(lhs, rhs) < 1e-13


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 8, 10, 12)])
def test_normal_op_hermitian_positive(L):
    fat, lng = synth.fat_long_links(L, seed=21)
    sigma = 4 * 0.05**2
    x = random_parity_field(L, 4)
    y = random_parity_field(L, 5)
    Ax = oracle.normal_op(L, fat, lng, sigma, x)
    Ay = oracle.normal_op(L, fat, lng, sigma, y)
    assert abs(np.vdot(y, Ax) - np.vdot(Ay, x)) <= 1e-13 * abs(np.vdot(y, Ax))
    xAx = np.vdot(x, Ax)
    assert abs(xAx.imag) <= 1e-13 * abs(xAx)
    assert xAx.real >= sigma * np.vdot(x, x).real


def test_cg_matches_dense_lu_4444():
    L = (4, 4, 4, 4)
    fat, lng = synth.fat_long_links(L, seed=1001)
    sigma = 4 * 0.1**2
    A = oracle.dense_normal_matrix(L, fat, lng, sigma)
    assert np.max(np.abs(A - A.conj().T)) < 1e-13
    b = synth.gaussian_source(L, 2100)
    x_lu = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    x, it, res = oracle.cg(L, fat, lng, sigma, b, tol=1e-13, max_iter=2000)
    assert it > 0 and res < 1e-12
    assert rel(x, x_lu) < 1e-11
    # dense eigenvalues: A is Hermitian positive definite, bounded below by sigma
    w = np.linalg.eigvalsh(A)
    assert w.min() >= sigma * (1 - 1e-12)


def test_cg_initial_guess_and_breakdown():
    L = (4, 4, 4, 4)
    fat, lng = synth.fat_long_links(L, seed=1001)
    sigma = 0.04
    b = synth.gaussian_source(L, 2101)
    x, it, res = oracle.cg(L, fat, lng, sigma, b, tol=1e-12)
    # starting from the solution takes no iteration
    x2, it2, res2 = oracle.cg(L, fat, lng, sigma, b, tol=1e-10, x0=x)
    assert it2 == 0 and res2 < 1e-10
    # sigma = 0 on the free field with a zero-momentum source: A b = 0 -> breakdown
    f0, l0 = synth.unit_links(L, 1.0, 1.0)
    b0 = synth.plane_wave(L, (0, 0, 0, 0), 0, (1, 0, 0), antiperiodic_t=False)
    _, it0, _ = oracle.cg(L, f0, l0, 0.0, b0, tol=1e-10, antiperiodic_t=False)
    assert it0 == -1


@pytest.mark.parametrize("apbc", [True, False])
def test_free_field_solve_closed_form(apbc):
    L = (8, 8, 8, 8)
    c1, c3 = 0.9, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    m = 0.1
    sigma = 4 * m * m
    k = (1, 2, 0, 3)
    b = synth.plane_wave(L, k, 0, (1.0, 0.5, -0.25j), apbc)
    x, it, res = oracle.cg(L, fat, lng, sigma, b, tol=1e-13, max_iter=2000, antiperiodic_t=apbc)
    want = b / (sigma + free_lambda(L, k, c1, c3, apbc))
    assert rel(x, want) < 1e-12


def test_multishift_free_field_closed_form():
    L = (8, 8, 8, 8)
    c1, c3 = 0.9, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    shifts = np.logspace(-4, 0, 11)
    # sum of two plane waves with different eigenvalues
    k1, k2 = (1, 0, 0, 0), (2, 3, 1, 2)
    b = synth.plane_wave(L, k1, 0, (1, 0, 0)) + synth.plane_wave(L, k2, 0, (0, 1, 1j))
    sols = oracle.multishift_solutions(L, fat, lng, shifts, b, tol=1e-13, max_iter=5000)
    for s, (x, it, res) in zip(shifts, sols):
        want = (synth.plane_wave(L, k1, 0, (1, 0, 0)) / (s + free_lambda(L, k1, c1, c3, True))
                + synth.plane_wave(L, k2, 0, (0, 1, 1j)) / (s + free_lambda(L, k2, c1, c3, True)))
        assert rel(x, want) < 1e-11


def test_dslash_sites_matches_full():
    L = (6, 8, 10, 12)
    fat, lng = synth.fat_long_links(L, seed=31)
    psi = random_parity_field(L, 6)
    full = oracle.dslash(L, fat, lng, psi, 1)
    sites = synth.parity_sites(L, 1)
    pick = np.array([0, 5, 17, len(sites) - 1])
    got = oracle.dslash_sites(L, fat, lng, psi, 0, sites[pick])
    assert np.array_equal(got, full[pick])


def test_flop_count_bookkeeping():
    # 16 complex 3x3 mat-vecs (9 cmul = 54 flops, 6 cadd = 12 flops) + 15 colour-vector adds (6 flops)
    assert 16 * (9 * 6 + 6 * 2) + 15 * 6 == 1146


def test_parity_layout_roundtrip():
    L = (6, 8, 10, 12)
    f = random_parity_field(L, 9)
    assert np.array_equal(oracle.to_parity(L, oracle.to_full(L, f, 1), 1), f)
    # the oracle's parity order agrees with the generators' (lex order within a parity)
    assert np.array_equal(np.nonzero(oracle.parity_of_sites(L) == 1)[0], synth.parity_sites(L, 1))


def test_rational_apply_free_field_closed_form():
    """out = (a0 + sum_s a_s / (sigma_s + lambda(p))) b for a plane wave b (unit links)."""
    L = (8, 8, 8, 8)
    c1, c3 = 0.9, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    a0, a, beta = synth.inverse_sqrt_rational(9, 0.01, 64.0)
    m = 0.05
    shifts = 4 * m * m + beta
    k = (1, 2, 0, 3)
    b = synth.plane_wave(L, k, 0, (1.0, -0.5j, 0.25))
    got = oracle.rational_apply(L, fat, lng, shifts, a, 0.3, b, tol=1e-13, max_iter=5000)
    lam = free_lambda(L, k, c1, c3, True)
    want = (0.3 + np.sum(a / (shifts + lam))) * b
    assert rel(got, want) < 1e-11


def test_inverse_sqrt_rational_approximates_the_function():
    """The quadrature rational function approximates x^(-1/2) on the interval it was built for."""
    a0, a, beta = synth.inverse_sqrt_rational(9, 0.01, 64.0)
    x = np.logspace(-2, np.log10(64.0), 50)
    r = a0 + np.sum(a[None, :] / (x[:, None] + beta[None, :]), axis=1)
    assert np.max(np.abs(r * np.sqrt(x) - 1.0)) < 2e-2
    assert np.all(a > 0) and np.all(beta > 0)
