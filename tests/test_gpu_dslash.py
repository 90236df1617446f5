"""GPU Dslash and normal operator vs the FP64 CPU oracle, through the C ABI.

Bars (fixed by the build's target): relative L2 error <= 1e-12 for the FP64
Dslash and <= 1e-5 for the FP32 Dslash, element by element on seeded inputs.
Small lattices cover several thread blocks and a ragged tail (Vh not a
multiple of the 128-thread block); 32^4 (the single-mass benchmark lattice,
in the launch configuration the benchmark times) is checked on sampled sites
the oracle computes one by one, plus the free-field closed form at every site.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}  # F64, F32


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fold_phases(L, U, hop, apbc):
    """Multiply links by eta_mu(n) and the boundary sign (test-side, for PHASES_FOLDED)."""
    c = synth.site_coords(L)
    out = U.copy()
    for mu in range(4):
        s = np.where(c[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0) if mu else np.ones(len(c))
        if mu == 3 and apbc:
            s = np.where(c[:, 3] + hop >= L[3], -s, s)
        out[:, mu] *= s[:, None, None]
    return out


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 8, 10, 12), (8, 10, 12, 14)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("recon", [False, True])
def test_dslash_matches_oracle(sqcg, links_cache, L, prec, recon):
    fat, lng = links_cache(L, 1001)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng, recon12=recon)
        for out_par in (0, 1):
            psi = synth.gaussian_source(L, 2000 + out_par)
            d_in = lat.pack(psi, prec)
            d_out = lat.new_spinor(prec)
            lat.dslash(out_par, d_in, d_out, prec)
            got = lat.unpack(d_out, prec)
            want = oracle.dslash(L, fat, lng, psi, out_par)
            assert rel(got, want) <= TOL[prec], (L, prec, recon, out_par, rel(got, want))


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 8, 10, 12)])
@pytest.mark.parametrize("recon", [False, True])
@pytest.mark.parametrize("apbc", [False, True])
def test_dslash_eight_way_matches_oracle(sqcg, links_cache, L, recon, apbc):
    """8-way FP32 storage (backward links at the site that uses them) gives the same D."""
    fat, lng = links_cache(L, 1001)
    with sqcg.Lattice(L, antiperiodic_t=apbc) as lat:
        lat.load_links(fat, lng, recon12=recon, eight_way=True)
        for out_par in (0, 1):
            psi = synth.gaussian_source(L, 2000 + out_par)
            out = lat.new_spinor(1)
            lat.dslash(out_par, lat.pack(psi, 1), out, 1)
            want = oracle.dslash(L, fat, lng, psi, out_par, apbc)
            assert rel(lat.unpack(out, 1), want) <= TOL[1]
        # FP64 stays forward-only and exact
        out = lat.new_spinor(0)
        psi = synth.gaussian_source(L, 3)
        lat.dslash(0, lat.pack(psi), out)
        assert rel(lat.unpack(out), oracle.dslash(L, fat, lng, psi, 0, apbc)) <= TOL[0]


@pytest.mark.parametrize("apbc", [False, True])
def test_dslash_periodic_and_folded_phases(sqcg, links_cache, apbc):
    L = (6, 8, 10, 12)
    fat, lng = links_cache(L, 77)
    psi = synth.gaussian_source(L, 5)
    want = oracle.dslash(L, fat, lng, psi, 1, antiperiodic_t=apbc)
    with sqcg.Lattice(L, antiperiodic_t=apbc) as lat:
        lat.load_links(fat, lng)
        out = lat.new_spinor(0)
        lat.dslash(1, lat.pack(psi), out)
        assert rel(lat.unpack(out), want) <= 1e-12
    # the caller folds the phases itself
    with sqcg.Lattice(L, antiperiodic_t=apbc, phases_folded=True) as lat:
        lat.load_links(fold_phases(L, fat, 1, apbc), fold_phases(L, lng, 3, apbc), recon12=True)
        out = lat.new_spinor(0)
        lat.dslash(1, lat.pack(psi), out)
        assert rel(lat.unpack(out), want) <= 1e-12


def test_recon12_rejected_for_non_su3_long_links(sqcg, links_cache):
    L = (4, 4, 4, 6)
    fat, lng = links_cache(L, 3)
    bad = lng.copy()
    bad[17, 2] *= 1.001  # one link is no longer s * SU(3) with the global s
    with sqcg.Lattice(L) as lat:
        with pytest.raises(sqcg.SqcgError) as e:
            lat.load_links(fat, bad, recon12=True)
        assert e.value.name == "RECON_REJECTED"
        lat.load_links(fat, bad, recon12=False)  # full storage is always accepted


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (6, 8, 10, 12)])
@pytest.mark.parametrize("prec", [0, 1])
def test_normal_op_matches_oracle(sqcg, links_cache, L, prec):
    fat, lng = links_cache(L, 1001)
    sigma = 4 * 0.1**2
    x = synth.gaussian_source(L, 2100)
    want = oracle.normal_op(L, fat, lng, sigma, x)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        y = lat.new_spinor(prec)
        lat.normal_op(sigma, lat.pack(x, prec), y, prec)
        assert rel(lat.unpack(y, prec), want) <= TOL[prec]


def test_anti_hermiticity_on_gpu(sqcg, links_cache):
    L = (16, 16, 16, 16)
    fat, lng = links_cache(L, 1001)
    y_e = synth.gaussian_source(L, 1)
    x_o = synth.gaussian_source(L, 2)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        a, b = lat.new_spinor(), lat.new_spinor()
        lat.dslash(0, lat.pack(x_o), a)
        lat.dslash(1, lat.pack(y_e), b)
        lhs = np.vdot(y_e, lat.unpack(a))
        rhs = np.vdot(lat.unpack(b), x_o)
    assert abs(lhs + rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("prec", [0, 1])
def test_free_field_closed_form_32(sqcg, prec):
    """Unit links: D on a plane wave is sum_mu eta_mu 2i (c1 sin p + c3 sin 3p) times the wave, at every site."""
    L = (32, 32, 32, 32)
    c1, c3 = 0.9, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    k = (3, 1, 7, 5)
    colour = (0.6, -0.2 + 0.5j, 1.0j)
    psi = synth.plane_wave(L, k, 0, colour)
    p = np.array([2 * np.pi * k[m] / L[m] for m in range(3)] + [(2 * k[3] + 1) * np.pi / L[3]])
    c = synth.site_coords(L)[synth.parity_sites(L, 1)]
    coef = np.zeros(len(c), dtype=np.complex128)
    for mu in range(4):
        eta = np.where(c[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0) if mu else np.ones(len(c))
        coef += eta * 2j * (c1 * np.sin(p[mu]) + c3 * np.sin(3 * p[mu]))
    want = coef[:, None] * synth.plane_wave(L, k, 1, colour)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng, recon12=True)
        out = lat.new_spinor(prec)
        lat.dslash(1, lat.pack(psi, prec), out, prec)
        got = lat.unpack(out, prec)
    assert rel(got, want) <= (1e-12 if prec == 0 else 1e-5)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("recon", [False, True])
def test_dslash_32_sampled_sites(sqcg, links_cache, prec, recon):
    """Full benchmark lattice: GPU output at sampled sites (including every boundary) vs the oracle."""
    L = (32, 32, 32, 32)
    fat, lng = links_cache(L, 1002)
    psi = synth.gaussian_source(L, 2200)
    out_par = 1
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng, recon12=recon)
        out = lat.new_spinor(prec)
        lat.dslash(out_par, lat.pack(psi, prec), out, prec)
        got = lat.unpack(out, prec)
    sites = synth.parity_sites(L, out_par)
    c = synth.site_coords(L)[sites]
    rng = np.random.default_rng(0)
    edge = np.nonzero((c == 0).any(axis=1) | (c == 31).any(axis=1) | (c == 2).any(axis=1) | (c == 29).any(axis=1))[0]
    pick = np.unique(np.concatenate([rng.choice(len(sites), 600, replace=False), rng.choice(edge, 400, replace=False),
                                     [0, len(sites) - 1]]))
    want = oracle.dslash_sites(L, fat, lng, psi, 1 - out_par, sites[pick])
    assert rel(got[pick], want) <= TOL[prec]


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 8, 10, 12), (8, 10, 12, 14), (16, 16, 16, 16)])
@pytest.mark.parametrize("par", [0, 1])
def test_dslash_float_float_matches_oracle(sqcg, links_cache, L, par):
    """The float-float Dslash (hi + lo floats per real, error-free products and sums on the FP32 pipe)
    against the FP64 oracle at the FP64 bar, 1e-12, on cubic and ragged lattices and both parities."""
    fat, lng = links_cache(L, 1001)
    psi = synth.gaussian_source(L, 2001 + par)
    want = oracle.dslash(L, fat, lng, psi, par)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng, recon12=True)  # the float-float copy is always 18-real
        out = lat.new_spinor(sqcg.FF)
        lat.dslash(par, lat.pack(psi, sqcg.FF), out, sqcg.FF)
        got = lat.unpack(out, sqcg.FF)
        # and the FP64 kernel on the same input, for the record of how close the two arithmetics are
        out64 = lat.new_spinor(sqcg.F64)
        lat.dslash(par, lat.pack(psi, sqcg.F64), out64, sqcg.F64)
        got64 = lat.unpack(out64, sqcg.F64)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-12, err
    assert np.linalg.norm(got - got64) / np.linalg.norm(got64) <= 1e-12


def test_float_float_pack_round_trip_and_free_field(sqcg):
    """Packing splits each real into hi = fl32(v), lo = fl32(v - hi) (hi + lo = v to 2^-48 relative), and the
    float-float Dslash reproduces the free-field plane-wave eigenvalue of D to that precision."""
    L = (8, 8, 8, 8)
    c1, c3 = 0.9, -1.0 / 24.0
    fat, lng = synth.unit_links(L, c1, c3)
    psi = synth.gaussian_source(L, 77)
    with sqcg.Lattice(L) as lat:
        got = lat.unpack(lat.pack(psi, sqcg.FF), sqcg.FF)
        assert np.max(np.abs(got - psi)) <= 1e-14 * np.max(np.abs(psi))
        lat.load_links(fat, lng)
        k = (1, 2, 3, 1)
        pw = synth.plane_wave(L, k, 1, (1.0, 0.5j, -0.25))
        out = lat.new_spinor(sqcg.FF)
        lat.dslash(0, lat.pack(pw, sqcg.FF), out, sqcg.FF)
        got = lat.unpack(out, sqcg.FF)
    want = oracle.dslash(L, fat, lng, pw, 0)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-13
