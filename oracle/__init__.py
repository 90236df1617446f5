"""FP64 CPU oracle for the improved-staggered Dslash, normal operator and CG.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it to produce expected values. The CUDA library never
imports or calls it, and it imports nothing from the CUDA library.

The arithmetic lives in ``sqcg_oracle.c`` (plain loops, lexicographic layout,
phases and boundary signs applied explicitly at every hop). This wrapper only
marshals numpy arrays and converts between the one-parity host format
(``[Vh][3]``, sites of one parity in increasing lex order) and the oracle's
full-lattice ``[V][3]`` arrays, with its own index code.

Parity pins (tests/test_oracle.py): free-field closed-form spectrum,
anti-Hermiticity D_eo^+ = -D_oe, gauge covariance, Hermiticity and positivity
of the normal operator, brute-force dense solve on 4^4, closed-form free-field
solves. The multi-shift expected values are the plain definition (one CG per
shift), pinned by the same closed form.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sqcg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over sites when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_dslash.argtypes = [P, I, P, P, P, P, I, I]
            lib.oracle_dslash.restype = None
            lib.oracle_dslash_sites.argtypes = [P, I, P, P, P, ctypes.c_long, P, P]
            lib.oracle_dslash_sites.restype = None
            lib.oracle_normal_op.argtypes = [P, I, P, P, ctypes.c_double, P, P, P, I]
            lib.oracle_normal_op.restype = None
            lib.oracle_cg.argtypes = [P, I, P, P, ctypes.c_double, P, P, ctypes.c_double, I, I,
                                      ctypes.POINTER(ctypes.c_double)]
            lib.oracle_cg.restype = I
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = I
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _dims(L):
    L = np.ascontiguousarray(np.asarray(L, dtype=np.int32))
    if L.shape != (4,) or np.any(L <= 0) or np.any(L % 2):
        raise ValueError("lattice extents must be 4 positive even integers")
    return L


def _links(U, V):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    if U.shape != (V, 4, 3, 3):
        raise ValueError(f"links must have shape ({V}, 4, 3, 3)")
    return U


def _ptr(a):
    return a.ctypes.data


def parity_of_sites(L) -> np.ndarray:
    """Parity (x+y+z+t) mod 2 of every lex site, computed from n by division."""
    Lx, Ly, Lz, Lt = (int(v) for v in L)
    n = np.arange(Lx * Ly * Lz * Lt, dtype=np.int64)
    x = n % Lx
    y = (n // Lx) % Ly
    z = (n // (Lx * Ly)) % Lz
    t = n // (Lx * Ly * Lz)
    return (x + y + z + t) % 2


def to_full(L, field_parity: np.ndarray, parity: int) -> np.ndarray:
    """One-parity [Vh][3] field -> full-lattice [V][3] (other parity zero)."""
    par = parity_of_sites(L)
    full = np.zeros((par.size, 3), dtype=np.complex128)
    full[par == parity] = field_parity
    return full


def to_parity(L, full: np.ndarray, parity: int) -> np.ndarray:
    par = parity_of_sites(L)
    return np.ascontiguousarray(full[par == parity])


def dslash(L, fat, lng, psi, out_parity: int, antiperiodic_t: bool = True, nthreads: int = 0):
    """(D psi) on the sites of out_parity; psi is a [Vh][3] field on the other parity."""
    Ld = _dims(L)
    V = int(np.prod(Ld))
    fat, lng = _links(fat, V), _links(lng, V)
    inp = to_full(Ld, np.asarray(psi, dtype=np.complex128), 1 - out_parity)
    out = np.zeros_like(inp)
    nt = nthreads if nthreads > 0 else max_threads()
    _load().oracle_dslash(_ptr(Ld), int(antiperiodic_t), _ptr(fat), _ptr(lng), _ptr(inp), _ptr(out),
                          int(out_parity), int(nt))
    return to_parity(Ld, out, out_parity)


def dslash_sites(L, fat, lng, psi, in_parity: int, sites_lex, antiperiodic_t: bool = True):
    """(D psi) at the listed lex sites (all of parity 1 - in_parity); returns [nsites][3]."""
    Ld = _dims(L)
    V = int(np.prod(Ld))
    fat, lng = _links(fat, V), _links(lng, V)
    inp = to_full(Ld, np.asarray(psi, dtype=np.complex128), in_parity)
    sites = np.ascontiguousarray(np.asarray(sites_lex, dtype=np.int64))
    out = np.zeros((sites.size, 3), dtype=np.complex128)
    _load().oracle_dslash_sites(_ptr(Ld), int(antiperiodic_t), _ptr(fat), _ptr(lng), _ptr(inp),
                                int(sites.size), _ptr(sites), _ptr(out))
    return out


def normal_op(L, fat, lng, sigma: float, x_even, antiperiodic_t: bool = True, nthreads: int = 0):
    """(sigma - D_eo D_oe) x on the even sites ([Vh][3] in, [Vh][3] out)."""
    Ld = _dims(L)
    V = int(np.prod(Ld))
    fat, lng = _links(fat, V), _links(lng, V)
    x = to_full(Ld, np.asarray(x_even, dtype=np.complex128), 0)
    y = np.zeros_like(x)
    tmp = np.zeros_like(x)
    nt = nthreads if nthreads > 0 else max_threads()
    _load().oracle_normal_op(_ptr(Ld), int(antiperiodic_t), _ptr(fat), _ptr(lng), float(sigma),
                             _ptr(x), _ptr(y), _ptr(tmp), int(nt))
    return to_parity(Ld, y, 0)


def cg(L, fat, lng, sigma: float, b_even, tol: float = 1e-12, max_iter: int = 100000,
       x0=None, antiperiodic_t: bool = True, nthreads: int = 0):
    """Solve (sigma - D_eo D_oe) x = b by CG. Returns (x_even, iterations, true_rel_resid).

    iterations is -1 on breakdown (<p, A p> <= 0)."""
    Ld = _dims(L)
    V = int(np.prod(Ld))
    fat, lng = _links(fat, V), _links(lng, V)
    b = to_full(Ld, np.asarray(b_even, dtype=np.complex128), 0)
    x = to_full(Ld, np.zeros_like(b_even) if x0 is None else np.asarray(x0, dtype=np.complex128), 0)
    res = ctypes.c_double(0.0)
    nt = nthreads if nthreads > 0 else max_threads()
    it = _load().oracle_cg(_ptr(Ld), int(antiperiodic_t), _ptr(fat), _ptr(lng), float(sigma), _ptr(b),
                           _ptr(x), float(tol), int(max_iter), int(nt), ctypes.byref(res))
    return to_parity(Ld, x, 0), int(it), float(res.value)


def multishift_solutions(L, fat, lng, shifts, b_even, tol: float = 1e-12, max_iter: int = 100000,
                         antiperiodic_t: bool = True, nthreads: int = 0):
    """Expected multi-shift result by definition: x_s = (sigma_s - D_eo D_oe)^-1 b, one CG per shift."""
    out = []
    for s in shifts:
        x, it, res = cg(L, fat, lng, float(s), b_even, tol, max_iter, None, antiperiodic_t, nthreads)
        out.append((x, it, res))
    return out


def rational_apply(L, fat, lng, shifts, residues, a0, b_even, tol: float = 1e-12, max_iter: int = 100000,
                   antiperiodic_t: bool = True, nthreads: int = 0):
    """Expected rational-function application by definition: a0 b + sum_s a_s (sigma_s - D_eo D_oe)^-1 b."""
    out = float(a0) * np.asarray(b_even, dtype=np.complex128)
    for (x, _, _), a in zip(multishift_solutions(L, fat, lng, shifts, b_even, tol, max_iter, antiperiodic_t,
                                                 nthreads), residues):
        out = out + float(a) * x
    return out


def dense_normal_matrix(L, fat, lng, sigma: float, antiperiodic_t: bool = True):
    """The normal operator as a dense matrix, one column per unit vector (tiny lattices only)."""
    Ld = _dims(L)
    Vh = int(np.prod(Ld)) // 2
    n = Vh * 3
    if n > 8192:
        raise ValueError("dense_normal_matrix is for tiny lattices")
    A = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        A[:, j] = normal_op(Ld, fat, lng, sigma, e.reshape(Vh, 3), antiperiodic_t, nthreads=1).ravel()
    return A


def true_rel_residual(L, fat, lng, sigma: float, b_even, x_even, antiperiodic_t: bool = True,
                      nthreads: int = 0) -> float:
    """|b - (sigma - D_eo D_oe) x| / |b| computed by the oracle in FP64."""
    Ax = normal_op(L, fat, lng, sigma, x_even, antiperiodic_t, nthreads)
    b = np.asarray(b_even, dtype=np.complex128)
    return float(np.linalg.norm(b - Ax) / np.linalg.norm(b))
