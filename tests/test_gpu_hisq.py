"""GPU HISQ link construction vs the FP64 oracle (oracle/hisq.py), through the C ABI.

Bar: the GPU forms the staple products in float-float arithmetic (hi + lo
floats, a 48-bit significand: unit roundoff 2^-48 = 3.6e-15 per operation)
and the U(3) projection in FP64, so the GPU links must match the FP64
oracle's element by element to 1e-12 of the largest link entry: a fat link
sums a few hundred products of up to seven links, each with a relative
rounding of a few units of 2^-48. Small lattices (including extents
that differ in every direction and the smallest legal extent, 4) are compared
in full; the 32^4 benchmark lattice, in the launch configuration the benchmark
times (sqcg_hisq_smear on device buffers), on sampled sites that the oracle
evaluates one by one, plus the free-field closed form and gauge covariance.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import hisq

pytestmark = pytest.mark.gpu

TOL = 1e-12


def maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 8, 10, 12), (8, 8, 8, 8)])
def test_hisq_matches_oracle(sqcg, L):
    thin = synth.thin_links(L, 1100 + L[0], width=0.3)
    want_f, want_l = hisq.hisq_links(L, thin)
    with sqcg.Lattice(L) as lat:
        fat, lng = lat.hisq_load_links(thin, return_links=True)
    assert maxrel(fat, want_f) <= TOL
    assert maxrel(lng, want_l) <= TOL


def test_hisq_free_field(sqcg):
    L = (8, 6, 4, 10)
    thin = np.broadcast_to(np.eye(3, dtype=complex), (synth.volume(L), 4, 3, 3)).copy()
    with sqcg.Lattice(L) as lat:
        fat, lng = lat.hisq_load_links(thin, return_links=True)
    # unit links: the products are exact; what remains is the float-float split of the coefficients
    # (2^-48 relative each) and the rounding of the sums, a few units of 3.6e-15 on entries near 1
    assert np.max(np.abs(fat - 9.0 / 8.0 * np.eye(3))) < 1e-13
    assert np.max(np.abs(lng + np.eye(3) / 24.0)) < 1e-13


@pytest.mark.parametrize("which", ["asqtad_like", "staples_and_lepage_only", "five_only"])
def test_hisq_custom_coefficients(sqcg, which):
    L = (6, 4, 8, 4)
    thin = synth.thin_links(L, 1200, width=0.5)
    if which == "asqtad_like":  # level 1 is the identity smearing, level 2 the asqtad fattening
        l1 = {"one_link": 1.0}
        l2 = {"one_link": 5 / 8, "three_staple": 1 / 16, "five_staple": 1 / 64, "seven_staple": 1 / 384,
              "lepage": -1 / 16}
    elif which == "staples_and_lepage_only":  # no 5/7-staple field: the final kernel wraps S only
        l1 = {"one_link": 0.5, "three_staple": 0.1}
        l2 = {"one_link": 0.7, "three_staple": 0.05, "lepage": 0.03}
    else:
        l1 = {"one_link": 0.3, "five_staple": 0.02}
        l2 = {"one_link": 0.9, "seven_staple": 0.01}
    naik = -0.05
    want_f, want_l = hisq.hisq_links(L, thin, level1=l1, level2=l2, naik_coeff=naik)
    with sqcg.Lattice(L) as lat:
        fat, lng = lat.hisq_load_links(thin, coeffs=sqcg.hisq_coeffs(l1, l2, naik), return_links=True)
    assert maxrel(fat, want_f) <= TOL
    assert maxrel(lng, want_l) <= TOL


def test_hisq_links_drive_the_cg(sqcg):
    """HISQ links installed by the library give the CG the oracle's operator; 12-real long links are refused
    (the long links are U(3), not SU(3) times a real scale)."""
    L, m, tol = (8, 8, 8, 8), 0.05, 1e-9
    thin = synth.thin_links(L, 1300, width=0.3)
    fat, lng = hisq.hisq_links(L, thin)
    b = synth.gaussian_source(L, 1301)
    with sqcg.Lattice(L) as lat:
        with pytest.raises(sqcg.SqcgError) as e:
            lat.hisq_load_links(thin, recon12=True)
        assert e.value.name == "RECON_REJECTED"
        lat.hisq_load_links(thin)
        x = lat.new_spinor()
        info = lat.cg_solve(m, lat.pack(b), x, tol=tol, mode=sqcg.MODE_MIXED)
        got = lat.unpack(x)
        # the Dslash itself on the installed links
        psi = synth.gaussian_source(L, 1302)
        out = lat.new_spinor()
        lat.dslash(1, lat.pack(psi), out)
        assert np.linalg.norm(lat.unpack(out) - oracle.dslash(L, fat, lng, psi, 1)) <= 1e-12 * np.linalg.norm(
            lat.unpack(out))
    assert info.status == 0
    assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, b, got) <= tol


def test_hisq_gauge_covariance_16(sqcg):
    L = (16, 16, 16, 16)
    thin = synth.thin_links(L, 1400, width=0.3)
    G = synth.random_gauge(L, 1401)
    with sqcg.Lattice(L) as lat:
        fat, lng = lat.hisq_load_links(thin, return_links=True)
        fat_g, lng_g = lat.hisq_load_links(synth.gauge_transform_links(L, thin, G, 1), return_links=True)
    assert maxrel(fat_g, synth.gauge_transform_links(L, fat, G, 1)) <= 1e-12
    assert maxrel(lng_g, synth.gauge_transform_links(L, lng, G, 3)) <= 1e-12


def test_hisq_32_device_call_sampled_sites(sqcg):
    """The benchmark lattice through the device entry point, sampled against the site-by-site oracle."""
    import torch

    L = (32, 32, 32, 32)
    thin = synth.thin_links(L, 1002)
    V = synth.volume(L)
    d_thin = torch.from_numpy(thin.view(np.float64).reshape(-1)).cuda()
    d_fat = torch.empty_like(d_thin)
    d_lng = torch.empty_like(d_thin)
    ws = torch.empty(sqcg.hisq_workspace_bytes(L), dtype=torch.uint8, device="cuda")
    sqcg.hisq_smear(L, d_thin, d_fat, d_lng, ws)
    fat = d_fat.cpu().numpy().view(np.complex128).reshape(V, 4, 3, 3)
    lng = d_lng.cpu().numpy().view(np.complex128).reshape(V, 4, 3, 3)
    c = synth.site_coords(L)
    edge = np.nonzero((c == 0).all(axis=1) | (c == 31).all(axis=1))[0]
    rng = np.random.default_rng(3)
    sites = np.unique(np.concatenate([edge, rng.choice(V, 2, replace=False), [V // 2 + 17]]))
    want_f, want_l = hisq.hisq_links_at(L, thin, sites)
    assert maxrel(fat[sites], want_f) <= TOL
    assert maxrel(lng[sites], want_l) <= TOL
    # every fat link of a unitary thin field has the same Frobenius-norm bound: |fat| <= sum |c| sqrt(3)
    bound = (1 + 6 / 16 + 24 / 64 + 48 / 384 + 6 / 8) * np.sqrt(3)
    assert np.all(np.linalg.norm(fat, axis=(-2, -1)) <= bound + 1e-12)


def test_hisq_errors(sqcg):
    import torch

    L = (4, 4, 4, 4)
    V = synth.volume(L)
    with sqcg.Lattice(L) as lat:
        with pytest.raises(sqcg.SqcgError) as e:  # zero links: the U(3) projection is undefined
            lat.hisq_load_links(np.zeros((V, 4, 3, 3), complex))
        assert e.value.name == "BREAKDOWN"
    with sqcg.Lattice(L, phases_folded=True) as lat:
        with pytest.raises(sqcg.SqcgError) as e:
            lat.hisq_load_links(synth.thin_links(L, 1))
        assert e.value.name == "INVALID_ARG"
    d = torch.zeros(V * 72, dtype=torch.float64, device="cuda")
    f, l = torch.empty_like(d), torch.empty_like(d)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(sqcg.SqcgError) as e:
        sqcg.hisq_smear(L, d, f, l, small)
    assert e.value.name == "INVALID_ARG"
    assert sqcg.hisq_workspace_bytes((4, 4, 4, 5)) == 0
