"""Seeded synthetic inputs for the staggered CG: gauge links, sources, gauge transforms.

This module is input plumbing shared by the oracle tests, the GPU tests and the
benchmark. It contains none of the operator's or the solvers' arithmetic: no
staggered phases, no boundary signs, no Dslash, no CG. It only draws random
numbers and arranges them in the host formats that both sides accept.

Host formats (the same ones the C-ABI takes):

* lattice extents ``L = (Lx, Ly, Lz, Lt)``, all even; sites in lexicographic order
  ``lex = x + Lx*(y + Ly*(z + Lz*t))`` (x fastest), so a numpy array of shape
  ``(Lt, Lz, Ly, Lx, ...)`` flattened in C order is in lex order;
* gauge field: complex128 array ``[V][4][3][3]``, direction order x, y, z, t,
  matrix row-major, forward links only (the standard MILC storage);
* colour vector on one parity: complex128 array ``[Vh][3]`` holding the sites of
  that parity in increasing lex order (the even-odd order ``lex // 2``).

Seeds (fixed by convention for the benchmark workloads): gauge field
``1000 + config``, source ``2000 + 100*config + rhs``.
"""

from __future__ import annotations

import os

import numpy as np

__all__ = [
    "volume",
    "site_coords",
    "parity_sites",
    "random_su3",
    "thin_links",
    "fat_long_links",
    "unit_links",
    "gaussian_source",
    "plane_wave",
    "random_gauge",
    "gauge_transform_links",
    "gauge_transform_parity_field",
    "inverse_sqrt_rational",
]

# Gell-Mann matrices: a basis of the traceless Hermitian 3x3 matrices.
_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1], _GELL_MANN[1][1, 0] = -1j, 1j
_GELL_MANN[2][0, 0], _GELL_MANN[2][1, 1] = 1, -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2], _GELL_MANN[4][2, 0] = -1j, 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2], _GELL_MANN[6][2, 1] = -1j, 1j
_GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def volume(L) -> int:
    L = tuple(int(v) for v in L)
    if len(L) != 4 or any(v <= 0 or v % 2 for v in L):
        raise ValueError(f"lattice extents must be 4 positive even integers, got {L}")
    return L[0] * L[1] * L[2] * L[3]


def site_coords(L) -> np.ndarray:
    """int64 array [V][4] of (x, y, z, t) for every site in lex order."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1).astype(np.int64)


def parity_sites(L, parity: int) -> np.ndarray:
    """lex indices of the sites of one parity, in increasing order ([Vh])."""
    c = site_coords(L)
    return np.nonzero((c.sum(axis=1) & 1) == parity)[0]


def _reunitarise(U: np.ndarray) -> np.ndarray:
    """Project a batch of near-SU(3) matrices onto SU(3): Gram-Schmidt on rows 0, 1;
    row 2 = conj(row0 x row1)."""
    a = U[..., 0, :]
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = U[..., 1, :]
    b = b - np.sum(np.conj(a) * b, axis=-1, keepdims=True) * a
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    c = np.conj(np.cross(a, b))
    return np.stack([a, b, c], axis=-2)


def _su3_from_gaussians(g: np.ndarray, width: float) -> np.ndarray:
    """exp(i*width*H) for H = sum_a g_a lambda_a / 2, one matrix per row of g, re-unitarised."""
    H = np.einsum("na,aij->nij", g, _GELL_MANN) * 0.5
    w, v = np.linalg.eigh(H)
    U = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * width * w), np.conj(v))
    return _reunitarise(U)


# above this many matrices the per-matrix work runs in a process pool (numpy's batched eigh holds
# the GIL); every matrix is computed on its own, so the result is the same bit for bit
_PARALLEL_MIN = 1 << 20


def random_su3(rng: np.random.Generator, n: int, width: float = 0.3, workers: int | None = None) -> np.ndarray:
    """n random SU(3) matrices U = exp(i*width*H), H = sum_a g_a lambda_a / 2, g_a ~ N(0,1).

    The exponential is taken through the Hermitian eigendecomposition of H, then
    the result is re-unitarised so that U is SU(3) to rounding. All random numbers
    are drawn first, in one stream; large batches are then split over `workers`
    spawned processes (default: all host cores)."""
    g = rng.standard_normal((n, 8))
    if workers is None:
        workers = (os.cpu_count() or 1) if n >= _PARALLEL_MIN else 1
    if workers <= 1:
        return _su3_from_gaussians(g, width)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    chunks = np.array_split(g, 4 * workers)
    # spawn, not fork: callers may already hold a CUDA context
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_su3_from_gaussians, chunks, [width] * len(chunks)))
    return np.concatenate(parts)


def thin_links(L, seed: int, width: float = 0.3) -> np.ndarray:
    """Random SU(3) gauge field [V][4][3][3] (complex128), seeded."""
    V = volume(L)
    rng = np.random.default_rng(seed)
    return random_su3(rng, V * 4, width).reshape(V, 4, 3, 3)


def fat_long_links(L, seed: int, width: float = 0.3, fat_scale: float = 0.9,
                   long_scale: float = -1.0 / 24.0):
    """The benchmark's fat and long links, built from one seeded thin field W.

    F_mu(n) = fat_scale * W_mu(n);
    L_mu(n) = long_scale * W_mu(n) W_mu(n+mu) W_mu(n+2mu)  (periodic wrap).
    Returns (fat, long), each complex128 [V][4][3][3]. No phases or boundary
    signs are applied: the operator applies those."""
    Lx, Ly, Lz, Lt = L
    W = thin_links(L, seed, width)
    fat = fat_scale * W
    W5 = W.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)
    lng = np.empty_like(W5)
    for mu, axis in enumerate((3, 2, 1, 0)):
        w0 = W5[..., mu, :, :]
        w1 = np.roll(w0, -1, axis=axis)  # W_mu(n + mu)
        w2 = np.roll(w0, -2, axis=axis)  # W_mu(n + 2mu)
        lng[..., mu, :, :] = long_scale * (w0 @ w1 @ w2)
    return fat, lng.reshape(-1, 4, 3, 3)


def unit_links(L, c1: float = 1.0, c3: float = 1.0):
    """Free field: fat = c1 * identity, long = c3 * identity on every link."""
    V = volume(L)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3))
    return c1 * eye.copy(), c3 * eye.copy()


def gaussian_source(L, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Gaussian complex colour vector on one parity: [Vh][3] (or [nrhs][Vh][3]),
    real and imaginary parts N(0,1), seeded."""
    Vh = volume(L) // 2
    rng = np.random.default_rng(seed)
    shape = (Vh, 3) if nrhs is None else (nrhs, Vh, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def plane_wave(L, k, parity: int, colour=(1.0, 0.0, 0.0), antiperiodic_t: bool = True) -> np.ndarray:
    """Plane wave exp(i p.n) * colour on the sites of one parity ([Vh][3]).

    k = integer wave numbers (kx, ky, kz, kt); p_mu = 2 pi k_mu / L_mu, except
    p_t = (2 kt + 1) pi / Lt when the time direction is antiperiodic."""
    c = site_coords(L)[parity_sites(L, parity)]
    p = [2 * np.pi * k[mu] / L[mu] for mu in range(3)]
    p.append((2 * k[3] + (1 if antiperiodic_t else 0)) * np.pi / L[3])
    phase = np.exp(1j * (c.astype(np.float64) @ np.asarray(p)))
    return phase[:, None] * np.asarray(colour, dtype=np.complex128)[None, :]


def random_gauge(L, seed: int, width: float = 1.0) -> np.ndarray:
    """Random gauge transformation G(n) in SU(3), [V][3][3]."""
    rng = np.random.default_rng(seed)
    return random_su3(rng, volume(L), width)


def gauge_transform_links(L, U: np.ndarray, G: np.ndarray, hop: int) -> np.ndarray:
    """U_mu(n) -> G(n) U_mu(n) G(n + hop*mu)^dagger for a link that spans `hop` sites."""
    Lx, Ly, Lz, Lt = L
    G5 = G.reshape(Lt, Lz, Ly, Lx, 3, 3)
    U5 = U.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)
    out = np.empty_like(U5)
    for mu, axis in enumerate((3, 2, 1, 0)):
        Gf = np.roll(G5, -hop, axis=axis)
        out[..., mu, :, :] = G5 @ U5[..., mu, :, :] @ np.conj(np.swapaxes(Gf, -1, -2))
    return out.reshape(U.shape)


def gauge_transform_parity_field(L, psi: np.ndarray, G: np.ndarray, parity: int) -> np.ndarray:
    """psi(n) -> G(n) psi(n) for a [Vh][3] field on one parity."""
    Gp = G[parity_sites(L, parity)]
    return np.einsum("nij,nj->ni", Gp, psi)


def inverse_sqrt_rational(npoles: int, lo: float, hi: float):
    """Poles and residues of a rational approximation r(x) = a0 + sum_k a_k / (x + beta_k) of x^(-1/2)
    for x in [lo, hi] (an RHMC-style input: apply it to M^+M with shifts 4 m^2 + beta_k).

    From x^(-1/2) = (2/pi) int_0^(pi/2) d(theta) / (sin^2 theta + x cos^2 theta) with c = sqrt(lo hi),
    x -> x / c and Gauss-Legendre nodes theta_k, weights w_k on [0, pi/2]:
    a_k = sqrt(c) (2/pi) w_k / cos^2 theta_k, beta_k = c tan^2 theta_k, a0 = 0. Returns (a0, a, beta)."""
    c = np.sqrt(lo * hi)
    u, w = np.polynomial.legendre.leggauss(npoles)
    theta = (u + 1.0) * np.pi / 4.0
    wt = w * np.pi / 4.0
    a = np.sqrt(c) * (2.0 / np.pi) * wt / np.cos(theta) ** 2
    beta = c * np.tan(theta) ** 2
    return 0.0, a, beta
