"""Pins of the HISQ link-construction oracle (oracle/hisq.py) against facts that do not come from it.

* Tree-level improvement (HISQ action, hep-lat/0610092): with unit thin links the
  operator's free dispersion c1 sin p + c3 sin 3p must equal p + O(p^5), i.e.
  c1 + 3 c3 = 1 and c1 + 27 c3 = 0: fat = 9/8, long = -1/24.
* The fat7 level equals the symmetrised product over the three other directions
  of (1/2 + (S_+ + S_-)/4), S_+- the forward/backward staple operators (the
  definition of the fat7 smearing), written here independently as operator
  compositions; the Lepage term equals S_+ S_+ + S_- S_- (same sign twice).
* Gauge covariance of fat and long links.
* U(3) projection = unitary polar factor: W^+ W = 1, W^+ V Hermitian positive,
  the same as the SVD polar factor (a library routine), idempotent.
* A constant field g on every link: every path reduces to g.
"""

import itertools

import numpy as np
import pytest

import synth
from oracle import hisq

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

L_SMALL = (6, 4, 4, 8)


def test_free_field_tree_level_improvement():
    L = (4, 4, 4, 4)
    eye = np.broadcast_to(np.eye(3, dtype=complex), (synth.volume(L), 4, 3, 3)).copy()
    fat, lng = hisq.hisq_links(L, eye)
    c1 = fat[..., 0, 0].real
    c3 = lng[..., 0, 0].real
    assert np.allclose(fat, c1[..., None, None] * np.eye(3), atol=1e-14)
    assert np.allclose(lng, c3[..., None, None] * np.eye(3), atol=1e-14)
    # dispersion c1 sin p + c3 sin 3p = (c1 + 3 c3) p - (c1 + 27 c3) p^3 / 6 + O(p^5)
    assert np.allclose(c1 + 3 * c3, 1.0, atol=1e-14)
    assert np.allclose(c1 + 27 * c3, 0.0, atol=1e-14)
    # the fat7 level alone is normalised to one
    fat7 = hisq.smear(L, eye, hisq.FAT7)
    assert np.allclose(fat7, eye, atol=1e-14)


def _wrap(L, U5, X5, rho, sign):
    """Staple operator on a link field X (every direction): forward or backward in rho."""
    Lx, Ly, Lz, Lt = L
    ax = (3, 2, 1, 0)
    out = np.empty_like(X5)
    for mu in range(4):
        if sign > 0:
            a = U5[..., rho, :, :]
            x = np.roll(X5[..., mu, :, :], -1, axis=ax[rho])
            b = np.roll(U5[..., rho, :, :], -1, axis=ax[mu])  # U_rho(n + mu)
            out[..., mu, :, :] = a @ x @ np.conj(np.swapaxes(b, -1, -2))
        else:
            a = np.roll(U5[..., rho, :, :], 1, axis=ax[rho])  # U_rho(n - rho)
            x = np.roll(X5[..., mu, :, :], 1, axis=ax[rho])
            b = np.roll(np.roll(U5[..., rho, :, :], 1, axis=ax[rho]), -1, axis=ax[mu])  # U_rho(n - rho + mu)
            out[..., mu, :, :] = np.conj(np.swapaxes(a, -1, -2)) @ x @ b
    return out


def _fat7_by_operator_products(L, U):
    Lx, Ly, Lz, Lt = L
    U5 = U.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)
    out = np.zeros_like(U5)

    def f(X, rho):
        return 0.5 * X + 0.25 * (_wrap(L, U5, X, rho, 1) + _wrap(L, U5, X, rho, -1))

    for mu in range(4):
        others = [d for d in range(4) if d != mu]
        acc = np.zeros_like(U5[..., mu, :, :])
        for a, b, c in itertools.permutations(others):
            acc += f(f(f(U5, c), b), a)[..., mu, :, :]
        out[..., mu, :, :] = acc / 6.0
    return out.reshape(-1, 4, 3, 3), U5


def test_fat7_is_the_symmetrised_operator_product():
    U = synth.thin_links(L_SMALL, 11, width=0.8)
    want, _ = _fat7_by_operator_products(L_SMALL, U)
    got = hisq.smear(L_SMALL, U, hisq.FAT7)
    assert np.max(np.abs(got - want)) < 1e-13


def test_lepage_term_is_the_same_sign_double_staple():
    U = synth.thin_links(L_SMALL, 12, width=0.8)
    Lx, Ly, Lz, Lt = L_SMALL
    U5 = U.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)
    want = np.zeros_like(U5)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            for s in (1, -1):
                want[..., mu, :, :] += _wrap(L_SMALL, U5, _wrap(L_SMALL, U5, U5, nu, s), nu, s)[..., mu, :, :]
    got = hisq.smear(L_SMALL, U, {"lepage": 1.0})
    for mu in range(4):
        assert np.max(np.abs(got.reshape(U5.shape)[..., mu, :, :] - want[..., mu, :, :])) < 1e-13


def test_gauge_covariance():
    L = L_SMALL
    U = synth.thin_links(L, 13, width=0.5)
    G = synth.random_gauge(L, 14)
    fat, lng = hisq.hisq_links(L, U)
    fat_g, lng_g = hisq.hisq_links(L, synth.gauge_transform_links(L, U, G, 1))
    assert np.max(np.abs(fat_g - synth.gauge_transform_links(L, fat, G, 1))) < 1e-12
    assert np.max(np.abs(lng_g - synth.gauge_transform_links(L, lng, G, 3))) < 1e-12


def test_u3_projection_is_the_polar_factor():
    rng = np.random.default_rng(15)
    # well-conditioned like smeared links (the eigh route loses ~eps * cond(V)^2)
    V = 0.5 * (rng.standard_normal((500, 3, 3)) + 1j * rng.standard_normal((500, 3, 3))) + 2 * np.eye(3)
    W = hisq.u3_project(V)
    eye = np.eye(3)
    assert np.max(np.abs(np.conj(np.swapaxes(W, -1, -2)) @ W - eye)) < 1e-13
    P = np.conj(np.swapaxes(W, -1, -2)) @ V
    assert np.max(np.abs(P - np.conj(np.swapaxes(P, -1, -2)))) < 1e-12
    assert np.all(np.linalg.eigvalsh(0.5 * (P + np.conj(np.swapaxes(P, -1, -2)))) > 0)
    X, _, Yh = np.linalg.svd(V)
    assert np.max(np.abs(W - X @ Yh)) < 1e-12
    assert np.max(np.abs(hisq.u3_project(W) - W)) < 1e-13
    assert np.max(np.abs(hisq.u3_project(3.7 * V) - W)) < 1e-13


def test_constant_field_reduces_every_path():
    L = (4, 4, 4, 6)
    g = synth.random_su3(np.random.default_rng(16), 1, width=1.0)[0]
    U = np.broadcast_to(g, (synth.volume(L), 4, 3, 3)).copy()
    fat, lng = hisq.hisq_links(L, U)
    assert np.max(np.abs(fat - 9.0 / 8.0 * g)) < 1e-13
    assert np.max(np.abs(lng + (g @ g @ g) / 24.0)) < 1e-13


def test_sites_evaluation_matches_the_whole_lattice():
    L = L_SMALL
    U = synth.thin_links(L, 17, width=0.5)
    fat, lng = hisq.hisq_links(L, U)
    sites = [0, 5, 77, synth.volume(L) - 1]
    f, l = hisq.hisq_links_at(L, U, sites)
    assert np.max(np.abs(f - fat[sites])) < 1e-13
    assert np.max(np.abs(l - lng[sites])) < 1e-13


# planted mistakes must fail at least one pin
def _mutated_paths(kind_bad):
    orig = hisq.staple_paths

    def paths(mu):
        k = orig(mu)
        if kind_bad == "five_wrong_order":  # closes nu before rho: still ends at n + mu, but not a nested staple
            k["five_staple"] = [[p[0], p[1], p[2], p[4], p[3]] for p in k["five_staple"]]
        if kind_bad == "seven_missing":
            k["seven_staple"] = k["seven_staple"][:-8]
        return k

    return paths


@pytest.mark.parametrize("mutant", ["five_wrong_order", "seven_missing", "one_link", "lepage_sign"])
def test_planted_mistakes_are_caught(monkeypatch, mutant):
    L = L_SMALL
    U = synth.thin_links(L, 18, width=0.8)
    if mutant in ("five_wrong_order", "seven_missing"):
        monkeypatch.setattr(hisq, "staple_paths", _mutated_paths(mutant))
        want, _ = _fat7_by_operator_products(L, U)
        assert np.max(np.abs(hisq.smear(L, U, hisq.FAT7) - want)) > 1e-6
    else:
        lv2 = dict(hisq.HISQ_LEVEL2)
        if mutant == "one_link":
            lv2["one_link"] = 5.0 / 8.0
        else:
            lv2["lepage"] = 1.0 / 8.0
        eye = np.broadcast_to(np.eye(3, dtype=complex), (synth.volume((4, 4, 4, 4)), 4, 3, 3)).copy()
        fat, lng = hisq.hisq_links((4, 4, 4, 4), eye, level2=lv2)
        c1, c3 = fat[0, 0, 0, 0].real, lng[0, 0, 0, 0].real
        assert abs(c1 + 3 * c3 - 1.0) > 1e-3 or abs(c1 + 27 * c3) > 1e-3
