"""GB300-native improved-staggered CG (arXiv:1611.00728): Python binding.

A thin ctypes layer over the C ABI in ``include/sqcg.h`` (``libsqcg.so``,
built in-tree by ``paper_1611_00728_gb300.build``). Every step of the Dslash
and the solvers runs in the library's CUDA kernels; this module only marshals
arguments. PyTorch provides device memory (tensors) and the CUDA stream.

Device colour vectors are torch tensors of shape ``(3, Vh, 2)`` (colour,
site, re/im) in float64 (``F64``) or float32 (``F32``): the library's
structure-of-arrays layout. Host colour vectors are numpy complex128
``[Vh][3]`` in parity order (sites of one parity in increasing lex order).
"""

from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

__all__ = [
    "F64", "F32", "FF", "MODE_F64", "MODE_MIXED", "ANTIPERIODIC_T", "PHASES_FOLDED", "RECON12_LONG",
    "SqcgError", "Info", "Lattice", "library", "library_path", "FLOPS_PER_SITE", "cg_solve_batched",
    "batched_tuning", "batched_tuning_ex", "pin_batched_tuning", "Network", "NN_NPARAMS", "NN_LAYERS", "NN_GATES", "HisqCoeffs", "SmearLevel", "hisq_coeffs", "hisq_smear",
    "hisq_workspace_bytes", "HISQ_FLOPS_PER_LINK", "MS_SHIFT_RU", "MS_NO_RU", "NN_MIX_FP32", "NN_MIX_BF16",
]

F64, F32, FF = 0, 1, 2  # FF: float-float (hi, lo floats per real), device vectors (3, Vh, 4) float32
NN_MIX_FP32, NN_MIX_BF16 = 0, 1  # arithmetic of the inference 8 -> 8 channel mixing (sqcg_nn_set_mixing)
MODE_F64, MODE_MIXED = 0, 1
MS_SHIFT_RU = 0x10  # OR-ed into a multi-shift mode: shift-aware reliable updates (sqcg_multishift_ru_record)
MS_NO_RU = 0x20  # OR-ed into a mixed multi-shift mode: no base reliable updates in the shared loop
ANTIPERIODIC_T, PHASES_FOLDED = 1, 2
RECON12_LONG = 1
EIGHT_WAY = 2
#: parameters of the preconditioner network (see include/sqcg.h for the layout)
NN_NPARAMS = 1472
#: host parameter layout of the network, as include/sqcg.h states it: per layer the slice of
#: interleaved (re, im) weights and the complex weight shape (tap, out, in); per gate the slices
#: of its a[8] and b[8]
NN_LAYERS = ((slice(0, 144), (9, 8, 1)), (slice(144, 1296), (9, 8, 8)), (slice(1296, 1440), (9, 1, 8)))
NN_GATES = ((slice(1440, 1448), slice(1448, 1456)), (slice(1456, 1464), slice(1464, 1472)))
assert NN_LAYERS[-1][0].stop == NN_GATES[0][0].start and NN_GATES[-1][1].stop == NN_NPARAMS
#: MILC's flop count of one Dslash output site: 16 x 66 (3x3 complex mat-vec) + 15 x 6 (adds)
FLOPS_PER_SITE = 1146

OK = 0
ERR_NAMES = {
    -1: "INVALID_ARG", -2: "CUDA", -3: "NOT_CONVERGED", -4: "BREAKDOWN", -5: "RECON_REJECTED",
    -6: "NO_LINKS", -7: "NO_MEMORY", -8: "SCRATCH_TOO_SMALL",
}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def library_path() -> str:
    return os.path.join(_HERE, "libsqcg.so")


class SqcgError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        self.name = ERR_NAMES.get(code, str(code))
        msg = library().sqcg_strerror(code).decode()
        super().__init__(f"{what}: {self.name} ({msg})")


#: counted flops of one HISQ link (3x3 complex products only, 198 flops each): 48 products per
#: smearing level (12 in the 3-staples, 24 in the 5/7-staple fields, 12 in the final wraps), two
#: levels, plus 2 for the Naik link; the U(3) projection and the additions are not counted
HISQ_FLOPS_PER_LINK = (2 * 48 + 2) * 198


class SmearLevel(ctypes.Structure):
    _fields_ = [("one_link", ctypes.c_double), ("three_staple", ctypes.c_double), ("five_staple", ctypes.c_double),
                ("seven_staple", ctypes.c_double), ("lepage", ctypes.c_double)]


class HisqCoeffs(ctypes.Structure):
    _fields_ = [("level1", SmearLevel), ("level2", SmearLevel), ("naik", ctypes.c_double)]


def hisq_coeffs(level1: dict, level2: dict, naik: float) -> HisqCoeffs:
    """Coefficient struct from dicts with keys one_link, three_staple, five_staple, seven_staple, lepage."""
    def lv(d):
        return SmearLevel(*[float(d.get(k, 0.0)) for k, _ in SmearLevel._fields_])

    return HisqCoeffs(lv(level1), lv(level2), float(naik))


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("status", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double), ("launches", ctypes.c_int),
                ("fallback", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build_if_needed():
    """Compile libsqcg.so in-tree when it is missing or older than its sources."""
    from . import build as _b

    return _b.build()


def library():
    """Load libsqcg.so. There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_1611_00728_gb300.build` "
                               "(the CUDA library is required; there is no CPU path)")
        lib = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.sqcg_create.argtypes = [P, I, P, ctypes.POINTER(P)]
        lib.sqcg_destroy.argtypes = [P]
        lib.sqcg_set_stream.argtypes = [P, P]
        lib.sqcg_set_reliable_update.argtypes = [P, D, I]
        lib.sqcg_set_update_arithmetic.argtypes = [P, I]
        lib.sqcg_spinor_bytes.argtypes = [P, I, ctypes.POINTER(ctypes.c_size_t)]
        lib.sqcg_load_links.argtypes = [P, P, P, I]
        lib.sqcg_pack_spinor.argtypes = [P, I, P, P]
        lib.sqcg_unpack_spinor.argtypes = [P, I, P, P]
        lib.sqcg_dslash.argtypes = [P, I, I, P, P]
        lib.sqcg_normal_op.argtypes = [P, D, I, P, P]
        lib.sqcg_normal_op_noalloc.argtypes = [P, D, I, P, P]
        lib.sqcg_cg_solve.argtypes = [P, D, P, P, D, I, I, ctypes.POINTER(Info)]
        lib.sqcg_multishift_cg_solve.argtypes = [P, I, P, P, P, P, I, I, P]
        lib.sqcg_multishift_ru_record.argtypes = [P, I, P, P, P, P, P]
        lib.sqcg_rational_apply.argtypes = [P, I, P, P, D, P, P, D, I, I, P]
        lib.sqcg_cg_solve_batched.argtypes = [I, P, P, P, P, P, D, I, P]
        lib.sqcg_batched_tuning.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.sqcg_batched_tuning_ex.argtypes = [P] + [ctypes.POINTER(I)] * 5
        lib.sqcg_batched_pin_tuning.argtypes = [I] * 5
        lib.sqcg_nn_create.argtypes = [P, ctypes.POINTER(P)]
        lib.sqcg_nn_destroy.argtypes = [P]
        lib.sqcg_nn_nparams.argtypes = []
        lib.sqcg_nn_set_params.argtypes = [P, P]
        lib.sqcg_nn_get_params.argtypes = [P, P, I]
        lib.sqcg_nn_apply.argtypes = [P, P, P]
        lib.sqcg_nn_set_loss.argtypes = [P, I]
        lib.sqcg_nn_set_mixing.argtypes = [P, I]
        lib.sqcg_nn_loss_grad.argtypes = [P, D, P, P, ctypes.POINTER(D), P]
        lib.sqcg_nn_train.argtypes = [P, D, I, P, P, I, I, D, ctypes.c_ulonglong, ctypes.POINTER(D),
                                      ctypes.POINTER(D)]
        lib.sqcg_make_training_pair.argtypes = [P, D, P, P, P, P, P]
        lib.sqcg_fcg_solve_nn.argtypes = [P, P, D, P, P, D, I, ctypes.POINTER(Info)]
        lib.sqcg_hisq_workspace_bytes.argtypes = [P]
        lib.sqcg_hisq_workspace_bytes.restype = ctypes.c_size_t
        lib.sqcg_hisq_smear.argtypes = [P, P, P, P, P, P, ctypes.c_size_t, P]
        lib.sqcg_hisq_load_links.argtypes = [P, P, P, I, P, P]
        lib.sqcg_strerror.argtypes = [I]
        lib.sqcg_strerror.restype = ctypes.c_char_p
        for name in ("sqcg_create", "sqcg_destroy", "sqcg_set_stream", "sqcg_set_reliable_update", "sqcg_spinor_bytes",
                     "sqcg_set_update_arithmetic",
                     "sqcg_load_links",
                     "sqcg_pack_spinor", "sqcg_unpack_spinor", "sqcg_dslash", "sqcg_normal_op", "sqcg_cg_solve",
                     "sqcg_normal_op_noalloc", "sqcg_nn_create", "sqcg_nn_destroy", "sqcg_nn_nparams",
                     "sqcg_nn_set_params", "sqcg_nn_get_params", "sqcg_nn_apply", "sqcg_nn_set_loss", "sqcg_nn_set_mixing", "sqcg_nn_loss_grad", "sqcg_nn_train",
                     "sqcg_make_training_pair", "sqcg_fcg_solve_nn",
                     "sqcg_multishift_cg_solve", "sqcg_multishift_ru_record", "sqcg_cg_solve_batched", "sqcg_batched_tuning", "sqcg_rational_apply",
                     "sqcg_batched_tuning_ex", "sqcg_batched_pin_tuning",
                     "sqcg_hisq_smear", "sqcg_hisq_load_links"):
            getattr(lib, name).restype = I
        _lib = lib
    return _lib


def _check(code: int, what: str):
    if code != OK:
        raise SqcgError(code, what)
    return code


def _torch():
    import torch

    return torch


class Lattice:
    """One lattice geometry with its links on the current CUDA device.

    dims = (Lx, Ly, Lz, Lt), all even and >= 4. antiperiodic_t: extra -1 on
    forward hops across the last time slice. phases_folded: the links passed to
    load_links already carry the staggered phases and boundary sign."""

    def __init__(self, dims, antiperiodic_t: bool = True, phases_folded: bool = False):
        torch = _torch()
        self.dims = tuple(int(v) for v in dims)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        flags = (ANTIPERIODIC_T if antiperiodic_t else 0) | (PHASES_FOLDED if phases_folded else 0)
        d = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        _check(library().sqcg_create(d, flags, ctypes.c_void_p(stream), ctypes.byref(h)), "sqcg_create")
        self._h = h
        self.recon12 = False
        self._networks = weakref.WeakSet()  # networks bound to this lattice: closed with it

    # -- lifetime ---------------------------------------------------------
    def close(self):
        for net in list(getattr(self, "_networks", ())):
            net.close()
        if getattr(self, "_h", None) is not None and self._h.value:
            library().sqcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_reliable_update(self, delta: float = 0.001, interval: int = 100):
        """Mixed-precision trigger: FP64 true residual when |r| < delta * max|r| since the last one, or every
        `interval` iterations."""
        _check(library().sqcg_set_reliable_update(self._h, float(delta), int(interval)), "sqcg_set_reliable_update")

    def set_update_arithmetic(self, prec: int):
        """Arithmetic of the mixed solve's true-residual recomputations: FF (default) or F64."""
        _check(library().sqcg_set_update_arithmetic(self._h, int(prec)), "sqcg_set_update_arithmetic")

    def _sync_stream(self):
        library().sqcg_set_stream(self._h, ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream))

    # -- data -------------------------------------------------------------
    def load_links(self, fat: np.ndarray, lng: np.ndarray, recon12: bool = False, eight_way: bool = False):
        """fat, lng: complex128 [V][4][3][3] host arrays (forward links, lex order). recon12: FP32 long links
        as two rows (checked); eight_way: FP32 copy also stores the backward links at the site that uses them."""
        fat = np.ascontiguousarray(fat, dtype=np.complex128)
        lng = np.ascontiguousarray(lng, dtype=np.complex128)
        if fat.shape != (self.V, 4, 3, 3) or lng.shape != (self.V, 4, 3, 3):
            raise ValueError(f"links must have shape ({self.V}, 4, 3, 3)")
        self._sync_stream()
        opts = (RECON12_LONG if recon12 else 0) | (EIGHT_WAY if eight_way else 0)
        _check(library().sqcg_load_links(self._h, fat.ctypes.data, lng.ctypes.data, opts), "sqcg_load_links")
        self.recon12 = recon12

    def hisq_load_links(self, thin: np.ndarray, coeffs: HisqCoeffs | None = None, recon12: bool = False,
                        eight_way: bool = False, return_links: bool = False):
        """HISQ fat and long links built on the GPU from host thin links (complex128 [V][4][3][3], unphased)
        and installed as this lattice's links. return_links: also return the (fat, long) host arrays."""
        thin = np.ascontiguousarray(thin, dtype=np.complex128)
        if thin.shape != (self.V, 4, 3, 3):
            raise ValueError(f"thin links must have shape ({self.V}, 4, 3, 3)")
        fat = np.empty_like(thin) if return_links else None
        lng = np.empty_like(thin) if return_links else None
        self._sync_stream()
        opts = (RECON12_LONG if recon12 else 0) | (EIGHT_WAY if eight_way else 0)
        _check(library().sqcg_hisq_load_links(self._h, thin.ctypes.data, ctypes.byref(coeffs) if coeffs else None,
                                              opts, fat.ctypes.data if return_links else None,
                                              lng.ctypes.data if return_links else None), "sqcg_hisq_load_links")
        self.recon12 = recon12
        return (fat, lng) if return_links else None

    def new_spinor(self, prec: int = F64, count: int | None = None):
        """Zeroed device colour vector(s) in the library layout: (3, Vh, 2), or (3, Vh, 4) for FF."""
        torch = _torch()
        dt = torch.float64 if prec == F64 else torch.float32
        last = 4 if prec == FF else 2
        shape = (3, self.Vh, last) if count is None else (count, 3, self.Vh, last)
        return torch.zeros(shape, dtype=dt, device="cuda")

    @staticmethod
    def _check_spinor(t, prec, Vh):
        torch = _torch()
        dt = torch.float64 if prec == F64 else torch.float32
        last = 4 if prec == FF else 2
        if t.dtype != dt or tuple(t.shape) != (3, Vh, last) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA tensor (3, {Vh}, {last}) of {dt}, got {t.dtype} "
                             f"{tuple(t.shape)}")
        return ctypes.c_void_p(t.data_ptr())

    def pack(self, host: np.ndarray, prec: int = F64, out=None):
        """Host parity-order complex [Vh][3] -> device vector (3, Vh, 2)."""
        host = np.ascontiguousarray(host, dtype=np.complex128)
        if host.shape != (self.Vh, 3):
            raise ValueError(f"host field must have shape ({self.Vh}, 3)")
        out = self.new_spinor(prec) if out is None else out
        self._sync_stream()
        _check(library().sqcg_pack_spinor(self._h, prec, host.ctypes.data, self._check_spinor(out, prec, self.Vh)),
               "sqcg_pack_spinor")
        return out

    def unpack(self, dev, prec: int = F64, out: np.ndarray | None = None) -> np.ndarray:
        """Device vector -> host parity-order complex128 [Vh][3] (synchronises)."""
        out = np.empty((self.Vh, 3), dtype=np.complex128) if out is None else out
        self._sync_stream()
        _check(library().sqcg_unpack_spinor(self._h, prec, self._check_spinor(dev, prec, self.Vh), out.ctypes.data),
               "sqcg_unpack_spinor")
        return out

    # -- operators --------------------------------------------------------
    def dslash(self, out_parity: int, inp, out, prec: int = F64):
        """out = D inp on the sites of out_parity (asynchronous)."""
        self._sync_stream()
        _check(library().sqcg_dslash(self._h, out_parity, prec, self._check_spinor(inp, prec, self.Vh),
                                     self._check_spinor(out, prec, self.Vh)), "sqcg_dslash")
        return out

    def normal_op(self, sigma: float, x, y, prec: int = F64):
        """y = (sigma - D_eo D_oe) x on the even sites (asynchronous)."""
        self._sync_stream()
        _check(library().sqcg_normal_op(self._h, float(sigma), prec, self._check_spinor(x, prec, self.Vh),
                                        self._check_spinor(y, prec, self.Vh)), "sqcg_normal_op")
        return y

    def normal_op_noalloc(self, sigma: float, x, y, prec: int = F64):
        """y = (sigma - D_eo D_oe) x without allocating device memory: the
        intermediate lives in a fixed scratch array of the library (for callers
        that cannot allocate; see sqcg_normal_op_noalloc in include/sqcg.h)."""
        self._sync_stream()
        _check(library().sqcg_normal_op_noalloc(self._h, float(sigma), prec, self._check_spinor(x, prec, self.Vh),
                                                self._check_spinor(y, prec, self.Vh)), "sqcg_normal_op_noalloc")
        return y

    # -- solvers ----------------------------------------------------------
    def cg_solve(self, mass: float, b, x, tol: float = 1e-8, max_iter: int = 10000, mode: int = MODE_MIXED,
                 raise_on_error: bool = True) -> Info:
        """Solve (4 mass^2 - D_eo D_oe) x = b; x holds the initial guess. Returns Info."""
        info = Info()
        self._sync_stream()
        rc = library().sqcg_cg_solve(self._h, float(mass), self._check_spinor(b, F64, self.Vh),
                                     self._check_spinor(x, F64, self.Vh), float(tol), int(max_iter), int(mode),
                                     ctypes.byref(info))
        if raise_on_error:
            _check(rc, "sqcg_cg_solve")
        return info

    def rational_apply(self, shifts, residues, a0: float, b, out, tol: float = 1e-8, max_iter: int = 10000,
                       mode: int = MODE_MIXED, raise_on_error: bool = True):
        """out = a0 b + sum_s residues[s] (shifts[s] - D_eo D_oe)^-1 b (one multi-shift solve). Returns Info per shift."""
        n = len(shifts)
        if len(residues) != n:
            raise ValueError("one residue per shift")
        sh = (ctypes.c_double * n)(*[float(v) for v in shifts])
        rs = (ctypes.c_double * n)(*[float(v) for v in residues])
        infos = (Info * n)()
        self._sync_stream()
        rc = library().sqcg_rational_apply(self._h, n, sh, rs, float(a0), self._check_spinor(b, F64, self.Vh),
                                           self._check_spinor(out, F64, self.Vh), float(tol), int(max_iter), int(mode),
                                           infos)
        if raise_on_error:
            _check(rc, "sqcg_rational_apply")
        return list(infos)

    def multishift_cg_solve(self, shifts, b, xs, tol=1e-8, max_iter: int = 10000, mode: int = MODE_MIXED,
                            raise_on_error: bool = True):
        """Solve (shifts[s] - D_eo D_oe) xs[s] = b for all shifts. Returns a list of Info."""
        n = len(shifts)
        sh = (ctypes.c_double * n)(*[float(s) for s in shifts])
        tols = [float(tol)] * n if np.isscalar(tol) else [float(t) for t in tol]
        tl = (ctypes.c_double * n)(*tols)
        ptrs = (ctypes.c_void_p * n)(*[self._check_spinor(x, F64, self.Vh).value for x in xs])
        infos = (Info * n)()
        self._sync_stream()
        rc = library().sqcg_multishift_cg_solve(self._h, n, sh, self._check_spinor(b, F64, self.Vh), ptrs, tl,
                                                int(max_iter), int(mode), infos)
        if raise_on_error:
            _check(rc, "sqcg_multishift_cg_solve")
        return list(infos)

    def multishift_ru_record(self):
        """Reliable updates of the last multi-shift solve (the mixed mode's base updates, or shift-aware with
        mode | MS_SHIFT_RU): a list of (iteration, |r_0| / |b|, losses |r_s - zeta'_s r_0| / |b| per shift in
        the caller's order; NaN where not measured)."""
        nu, ns = ctypes.c_int(), ctypes.c_int()
        _check(library().sqcg_multishift_ru_record(self._h, 0, ctypes.byref(nu), ctypes.byref(ns), None, None, None),
               "sqcg_multishift_ru_record")
        m = min(nu.value, 16)
        it = (ctypes.c_int * max(m, 1))()
        base = (ctypes.c_double * max(m, 1))()
        loss = (ctypes.c_double * max(m * ns.value, 1))()
        _check(library().sqcg_multishift_ru_record(self._h, m, ctypes.byref(nu), ctypes.byref(ns), it, base, loss),
               "sqcg_multishift_ru_record")
        return [(it[u], base[u], [loss[u * ns.value + j] for j in range(ns.value)]) for u in range(m)]


def cg_solve_batched(lattices, masses, bs, xs, tol: float = 1e-8, max_iter: int = 10000,
                     raise_on_error: bool = True):
    """Batched mixed-precision CG over several lattices and many right-hand sides.

    lattices: list of Lattice (links loaded); masses: one mass per lattice;
    bs[k], xs[k]: contiguous CUDA float64 tensors (nrhs_k, 3, Vh_k, 2) holding
    the sources and the initial guesses / solutions. Returns a list (one per
    lattice) of lists of Info (one per RHS)."""
    n = len(lattices)
    if not (len(masses) == len(bs) == len(xs) == n):
        raise ValueError("one mass, b and x per lattice")
    torch = _torch()
    nrhs = []
    for lat, b, x in zip(lattices, bs, xs):
        for t in (b, x):
            if t.dtype != torch.float64 or t.dim() != 4 or tuple(t.shape[1:]) != (3, lat.Vh, 2) or not t.is_cuda \
                    or not t.is_contiguous():
                raise ValueError(f"expected a contiguous CUDA float64 tensor (nrhs, 3, {lat.Vh}, 2)")
        if b.shape[0] != x.shape[0]:
            raise ValueError("b and x must hold the same number of right-hand sides")
        nrhs.append(int(b.shape[0]))
    lattices[0]._sync_stream()
    ctxs = (ctypes.c_void_p * n)(*[lat._h.value for lat in lattices])
    nr = (ctypes.c_int * n)(*nrhs)
    ms = (ctypes.c_double * n)(*[float(m) for m in masses])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (Info * sum(nrhs))()
    rc = library().sqcg_cg_solve_batched(n, ctxs, nr, ms, bp, xp, float(tol), int(max_iter), infos)
    if raise_on_error:
        _check(rc, "sqcg_cg_solve_batched")
    out, k = [], 0
    for r in nrhs:
        out.append(list(infos[k:k + r]))
        k += r
    return out


def batched_tuning(lattice) -> tuple[int, int]:
    """(RHS block width, site block size) the autotuner chose for the last batched solve led by lattice."""
    W, T = ctypes.c_int(), ctypes.c_int()
    _check(library().sqcg_batched_tuning(lattice._h, ctypes.byref(W), ctypes.byref(T)), "sqcg_batched_tuning")
    return W.value, T.value


def batched_tuning_ex(lattice) -> dict:
    """The full FP32 Dslash configuration of the last batched solve led by lattice: W, WT (RHS per thread),
    T, carve (shared-memory carveout in percent, -1 = default) and warp_sites (32 or 16 sites per warp)."""
    v = [ctypes.c_int() for _ in range(5)]
    _check(library().sqcg_batched_tuning_ex(lattice._h, *[ctypes.byref(c) for c in v]), "sqcg_batched_tuning_ex")
    return dict(zip(("W", "WT", "T", "carve", "warp_sites"), (c.value for c in v)))


def pin_batched_tuning(W: int, WT: int = 1, T: int = 64, carve: int = -1, warp_sites: int = 32):
    """Pin the FP32 Dslash configuration of batched solves planned from now on (W = 0: autotune again)."""
    _check(library().sqcg_batched_pin_tuning(int(W), int(WT), int(T), int(carve), int(warp_sites)),
           "sqcg_batched_pin_tuning")


class Network:
    """The gauge-covariant preconditioner network bound to one Lattice (its links).

    Vectors are FP32 even-site device vectors (3, Vh, 2) float32."""

    def __init__(self, lattice: Lattice):
        self.lattice = lattice
        h = ctypes.c_void_p()
        _check(library().sqcg_nn_create(lattice._h, ctypes.byref(h)), "sqcg_nn_create")
        self._h = h
        lattice._networks.add(self)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            library().sqcg_nn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (NN_NPARAMS,):
            raise ValueError(f"expected {NN_NPARAMS} parameters")
        self.lattice._sync_stream()
        _check(library().sqcg_nn_set_params(self._h, p.ctypes.data), "sqcg_nn_set_params")

    def get_params(self, bf16_rounded: bool = False) -> np.ndarray:
        p = np.empty(NN_NPARAMS, dtype=np.float32)
        self.lattice._sync_stream()
        _check(library().sqcg_nn_get_params(self._h, p.ctypes.data, int(bf16_rounded)), "sqcg_nn_get_params")
        return p

    def set_loss(self, norm: int):
        """Training loss norm: 1 = A-norm of the error (default), 2 = A^2-norm (preconditioned residual)."""
        _check(library().sqcg_nn_set_loss(self._h, int(norm)), "sqcg_nn_set_loss")

    def set_mixing(self, mode: int):
        """Inference 8 -> 8 channel mixing: NN_MIX_FP32 (CUDA cores, default) or NN_MIX_BF16 (tensor cores)."""
        _check(library().sqcg_nn_set_mixing(self._h, int(mode)), "sqcg_nn_set_mixing")

    def apply(self, r, z):
        lat = self.lattice
        lat._sync_stream()
        _check(library().sqcg_nn_apply(self._h, lat._check_spinor(r, F32, lat.Vh), lat._check_spinor(z, F32, lat.Vh)),
               "sqcg_nn_apply")
        return z

    def loss_grad(self, sigma: float, r, e):
        lat = self.lattice
        loss = ctypes.c_double()
        grad = np.empty(NN_NPARAMS, dtype=np.float32)
        lat._sync_stream()
        _check(library().sqcg_nn_loss_grad(self._h, float(sigma), lat._check_spinor(r, F32, lat.Vh),
                                           lat._check_spinor(e, F32, lat.Vh), ctypes.byref(loss), grad.ctypes.data),
               "sqcg_nn_loss_grad")
        return loss.value, grad

    def train(self, sigma: float, r_pairs, e_pairs, steps: int, batch: int = 8, lr: float = 1e-2, seed: int = 1):
        """r_pairs, e_pairs: CUDA float32 tensors (npairs, 3, Vh, 2). Returns (first, last) batch loss."""
        lat = self.lattice
        torch = _torch()
        for t in (r_pairs, e_pairs):
            if t.dtype != torch.float32 or t.dim() != 4 or tuple(t.shape[1:]) != (3, lat.Vh, 2) or not t.is_cuda \
                    or not t.is_contiguous():
                raise ValueError(f"expected a contiguous CUDA float32 tensor (npairs, 3, {lat.Vh}, 2)")
        if r_pairs.shape[0] != e_pairs.shape[0]:
            raise ValueError("as many errors as residuals")
        first, last = ctypes.c_double(), ctypes.c_double()
        lat._sync_stream()
        _check(library().sqcg_nn_train(self._h, float(sigma), int(r_pairs.shape[0]), r_pairs.data_ptr(),
                                       e_pairs.data_ptr(), int(steps), int(batch), float(lr), int(seed),
                                       ctypes.byref(first), ctypes.byref(last)), "sqcg_nn_train")
        return first.value, last.value

    def make_pair(self, sigma: float, b, x_k, x_star, r_out, e_out):
        """r = b - A x_k (FP64, rounded to FP32), e = x_star - x_k (FP32)."""
        lat = self.lattice
        lat._sync_stream()
        _check(library().sqcg_make_training_pair(lat._h, float(sigma), lat._check_spinor(b, F64, lat.Vh),
                                                 lat._check_spinor(x_k, F64, lat.Vh),
                                                 lat._check_spinor(x_star, F64, lat.Vh),
                                                 lat._check_spinor(r_out, F32, lat.Vh),
                                                 lat._check_spinor(e_out, F32, lat.Vh)), "sqcg_make_training_pair")

    def fcg_solve(self, mass: float, b, x, tol: float = 1e-8, max_iter: int = 10000,
                  raise_on_error: bool = True) -> Info:
        """Flexible CG preconditioned by this network on its lattice."""
        lat = self.lattice
        info = Info()
        lat._sync_stream()
        rc = library().sqcg_fcg_solve_nn(lat._h, self._h, float(mass), lat._check_spinor(b, F64, lat.Vh),
                                         lat._check_spinor(x, F64, lat.Vh), float(tol), int(max_iter),
                                         ctypes.byref(info))
        if raise_on_error:
            _check(rc, "sqcg_fcg_solve_nn")
        return info


def hisq_workspace_bytes(dims) -> int:
    return int(library().sqcg_hisq_workspace_bytes((ctypes.c_int * 4)(*[int(v) for v in dims])))


def hisq_smear(dims, thin, fat, lng, workspace, coeffs: HisqCoeffs | None = None):
    """Device HISQ smearing: thin, fat, lng are contiguous CUDA float64 tensors of V*4*9*2 values in the host
    link order [V][4][3][3][re, im]; workspace a CUDA tensor of at least hisq_workspace_bytes(dims) bytes.
    Runs on the current stream and synchronises it."""
    torch = _torch()
    V = int(np.prod(dims))
    for t in (thin, fat, lng):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != V * 72:
            raise ValueError("links must be contiguous CUDA float64 tensors of V*4*9*2 values")
    if not workspace.is_cuda or not workspace.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")
    nbytes = workspace.numel() * workspace.element_size()
    _check(library().sqcg_hisq_smear((ctypes.c_int * 4)(*[int(v) for v in dims]), thin.data_ptr(), fat.data_ptr(),
                                     lng.data_ptr(), ctypes.byref(coeffs) if coeffs else None, workspace.data_ptr(),
                                     nbytes, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
           "sqcg_hisq_smear")
