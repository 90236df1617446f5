"""FP64 numpy oracle for HISQ link construction (thin links -> fat and long links).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it to produce expected values. The CUDA library never
imports or calls it, and it imports nothing from the CUDA library.

The paper's benchmark application evolves the HISQ action (Sec. 4); the CG it
times consumes the HISQ fat and long links. The construction is the HISQ
action's (Follana et al., hep-lat/0610092), written here as a plain sum over
explicit link paths:

1. V = smear(U, level-1 coefficients): one link, 3-, 5- and 7-link staples
   (fat7: 1/8, 1/16, 1/64, 1/384);
2. W = U(3) projection of V: W = V (V^+ V)^(-1/2), through the Hermitian
   eigendecomposition of V^+ V;
3. fat = smear(W, level-2 coefficients): the same staples plus the 5-link
   Lepage staple (-1/8), one-link coefficient 1;
   long = naik * W_mu(n) W_mu(n+mu) W_mu(n+2mu), naik = -1/24.

A path is a list of signed steps (+d or -d, d = 0..3 for x, y, z, t); its
product multiplies U_d(y) for a forward step from y and U_d(y-d)^+ for a
backward step. Every staple path in direction mu starts at n and ends at
n + mu. Links are unphased and periodic in every direction, and every
coefficient is the one for unphased links (all staples positive, the Lepage
term negative). The staggered phases and the time-boundary sign are folded
into the resulting fat and long links when they are loaded; on phased thin
links the 3- and 7-link staple coefficients would change sign instead, since
their paths' phase products are minus the direct link's.

Pins (tests/test_oracle_hisq.py): tree-level improvement of the free field
(fat = 9/8, long = -1/24, i.e. c1 + 3 c3 = 1 and c1 + 27 c3 = 0 for the
dispersion sin-expansion), the fat7 part against the symmetrised product of
(1/2 + (staple_+ + staple_-)/4) operators, gauge covariance, the polar
decomposition properties of the projection, and a constant-field case.
"""

from __future__ import annotations

import itertools

import numpy as np

# coefficients of one smearing level: one link, 3-staple, 5-staple, 7-staple, Lepage
FAT7 = {"one_link": 1.0 / 8.0, "three_staple": 1.0 / 16.0, "five_staple": 1.0 / 64.0,
        "seven_staple": 1.0 / 384.0, "lepage": 0.0}
HISQ_LEVEL2 = {"one_link": 1.0, "three_staple": 1.0 / 16.0, "five_staple": 1.0 / 64.0,
               "seven_staple": 1.0 / 384.0, "lepage": -1.0 / 8.0}
HISQ_NAIK = -1.0 / 24.0


def _dims(L):
    L = tuple(int(v) for v in L)
    if len(L) != 4 or any(v < 4 or v % 2 for v in L):
        raise ValueError("lattice extents must be 4 even integers >= 4")
    return L


def _as5(U, L):
    """[V][4][3][3] lex -> (Lt, Lz, Ly, Lx, 4, 3, 3)."""
    Lx, Ly, Lz, Lt = L
    return np.asarray(U, dtype=np.complex128).reshape(Lt, Lz, Ly, Lx, 4, 3, 3)


_AXIS = (3, 2, 1, 0)  # numpy axis of direction x, y, z, t in the (t, z, y, x) site array


def _shift(field, disp):
    """field at n + disp for every n (periodic)."""
    out = field
    for d in range(4):
        if disp[d]:
            out = np.roll(out, -disp[d], axis=_AXIS[d])
    return out


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def path_product(U5, steps):
    """Product of links along `steps` (signed directions, encoded as (d, +1|-1)) from every site."""
    Lt, Lz, Ly, Lx = U5.shape[:4]
    M = np.broadcast_to(np.eye(3, dtype=np.complex128), (Lt, Lz, Ly, Lx, 3, 3)).copy()
    pos = [0, 0, 0, 0]
    for d, s in steps:
        if s > 0:
            link = _shift(U5[..., d, :, :], pos)
            pos[d] += 1
        else:
            pos[d] -= 1
            link = _dag(_shift(U5[..., d, :, :], pos))
        M = M @ link
    return M, tuple(pos)


def staple_paths(mu):
    """All paths of one smearing level in direction mu, grouped by kind: lists of step lists."""
    others = [d for d in range(4) if d != mu]
    kinds = {"one_link": [[(mu, 1)]], "three_staple": [], "five_staple": [], "seven_staple": [], "lepage": []}
    for nu in others:
        for s in (1, -1):
            kinds["three_staple"].append([(nu, s), (mu, 1), (nu, -s)])
            kinds["lepage"].append([(nu, s), (nu, s), (mu, 1), (nu, -s), (nu, -s)])
    for nu, rho in itertools.permutations(others, 2):
        for s, t in itertools.product((1, -1), repeat=2):
            kinds["five_staple"].append([(nu, s), (rho, t), (mu, 1), (rho, -t), (nu, -s)])
    for nu, rho, sig in itertools.permutations(others, 3):
        for s, t, r in itertools.product((1, -1), repeat=3):
            kinds["seven_staple"].append([(nu, s), (rho, t), (sig, r), (mu, 1), (sig, -r), (rho, -t), (nu, -s)])
    return kinds


def smear(L, U, coeffs):
    """One smearing level: sum over every path kind of coefficient x path product. [V][4][3][3] in and out."""
    L = _dims(L)
    U5 = _as5(U, L)
    out = np.zeros_like(U5)
    for mu in range(4):
        for kind, paths in staple_paths(mu).items():
            c = coeffs.get(kind, 0.0)
            if c == 0.0:
                continue
            for steps in paths:
                M, end = path_product(U5, steps)
                assert end == tuple(1 if d == mu else 0 for d in range(4))
                out[..., mu, :, :] += c * M
    return out.reshape(-1, 4, 3, 3)


def u3_project(V):
    """W = V (V^+ V)^(-1/2) for every matrix of a [..., 3, 3] array, via eigh of the Hermitian V^+ V."""
    V = np.asarray(V, dtype=np.complex128)
    Q = _dag(V) @ V
    lam, E = np.linalg.eigh(Q)
    if np.any(lam <= 0):
        raise ValueError("singular link in the U(3) projection")
    Qinv_half = (E * (1.0 / np.sqrt(lam))[..., None, :]) @ _dag(E)
    return V @ Qinv_half


def naik(L, W, coeff=HISQ_NAIK):
    """long_mu(n) = coeff * W_mu(n) W_mu(n+mu) W_mu(n+2mu)."""
    L = _dims(L)
    W5 = _as5(W, L)
    out = np.empty_like(W5)
    for mu in range(4):
        M, end = path_product(W5, [(mu, 1)] * 3)
        out[..., mu, :, :] = coeff * M
    return out.reshape(-1, 4, 3, 3)


def hisq_links(L, thin, level1=FAT7, level2=HISQ_LEVEL2, naik_coeff=HISQ_NAIK):
    """Thin links -> (fat, long), both [V][4][3][3] complex128, unphased and periodic."""
    V1 = smear(L, thin, level1)
    W = u3_project(V1)
    return smear(L, W, level2), naik(L, W, naik_coeff)


# ---------------------------------------------------------------------------
# the same construction at a few sites of a large lattice (for sampled checks)
# ---------------------------------------------------------------------------
class _SiteEval:
    """Path products on demand with periodic lex indexing; level-1 projected links memoised."""

    def __init__(self, L, thin, level1):
        self.L = _dims(L)
        self.U = np.asarray(thin, dtype=np.complex128).reshape(-1, 4, 3, 3)
        self.level1 = level1
        self.W = {}

    def lex(self, c):
        Lx, Ly, Lz, Lt = self.L
        x, y, z, t = (c[0] % Lx, c[1] % Ly, c[2] % Lz, c[3] % Lt)
        return x + Lx * (y + Ly * (z + Lz * t))

    def walk(self, link, start, steps):
        M = np.eye(3, dtype=np.complex128)
        pos = list(start)
        for d, s in steps:
            if s > 0:
                M = M @ link(pos, d)
                pos[d] += 1
            else:
                pos[d] -= 1
                M = M @ _dag(link(pos, d))
        return M

    def thin_link(self, pos, d):
        return self.U[self.lex(pos), d]

    def fat_at(self, link, start, mu, coeffs):
        acc = np.zeros((3, 3), dtype=np.complex128)
        for kind, paths in staple_paths(mu).items():
            c = coeffs.get(kind, 0.0)
            if c:
                for steps in paths:
                    acc += c * self.walk(link, start, steps)
        return acc

    def w_link(self, pos, d):
        key = (self.lex(pos), d)
        if key not in self.W:
            V = self.fat_at(self.thin_link, pos, d, self.level1)
            self.W[key] = u3_project(V)
        return self.W[key]


def hisq_links_at(L, thin, sites_lex, level1=FAT7, level2=HISQ_LEVEL2, naik_coeff=HISQ_NAIK):
    """(fat, long) at the listed lex sites only: arrays [nsites][4][3][3]."""
    ev = _SiteEval(L, thin, level1)
    Lx, Ly, Lz, _ = ev.L
    fat = np.empty((len(sites_lex), 4, 3, 3), dtype=np.complex128)
    lng = np.empty_like(fat)
    for i, n in enumerate(sites_lex):
        n = int(n)
        c = [n % Lx, (n // Lx) % Ly, (n // (Lx * Ly)) % Lz, n // (Lx * Ly * Lz)]
        for mu in range(4):
            fat[i, mu] = ev.fat_at(ev.w_link, c, mu, level2)
            lng[i, mu] = naik_coeff * ev.walk(ev.w_link, c, [(mu, 1)] * 3)
    return fat, lng
