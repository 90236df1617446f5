"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/sqcg.h declares. No compute call is made here."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sqcg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sqcg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1611_00728_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sqcg_create", "sqcg_destroy", "sqcg_load_links", "sqcg_dslash", "sqcg_cg_solve",
                 "sqcg_multishift_cg_solve", "sqcg_strerror"):
        assert want in names


def test_binding_constants_match_the_header():
    """Every mode, flag and precision the binding passes through the ABI has the header's value."""
    import paper_1611_00728_gb300 as sq

    text = open(HEADER).read()
    defs = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define SQCG_([A-Z0-9_]+)\s+\(?(-?(?:0x)?[0-9a-fA-F]+)\)?", text)}
    pairs = {"F64": "F64", "F32": "F32", "FF": "FF", "MODE_F64": "MODE_F64", "MODE_MIXED": "MODE_MIXED",
             "ANTIPERIODIC_T": "ANTIPERIODIC_T", "PHASES_FOLDED": "PHASES_FOLDED", "RECON12_LONG": "RECON12_LONG",
             "EIGHT_WAY": "EIGHT_WAY", "MS_SHIFT_RU": "MS_SHIFT_RU", "MS_NO_RU": "MS_NO_RU",
             "NN_MIX_FP32": "NN_MIX_FP32", "NN_MIX_BF16": "NN_MIX_BF16", "NN_NPARAMS": "NN_NPARAMS"}
    for py, c in pairs.items():
        assert getattr(sq, py) == defs[c], (py, getattr(sq, py), defs[c])
    errs = {v: k[len("ERR_"):] for k, v in defs.items() if k.startswith("ERR_")}
    assert sq.ERR_NAMES == errs
    # the multi-shift flags sit above every mode value and apart from each other
    assert defs["MS_SHIFT_RU"] & defs["MS_NO_RU"] == 0
    assert max(defs["MODE_F64"], defs["MODE_MIXED"]) < min(defs["MS_SHIFT_RU"], defs["MS_NO_RU"])


def test_library_loads_and_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_exported_symbols_are_c_linkage(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sqcg_[a-z0-9_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_library_built_for_sm_103a():
    """Every translation unit is compiled, and the library linked, for sm_103a only (the build's own
    nvcc command lines; no binary tool inspects the result)."""
    from paper_1611_00728_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    cmds = build.commands()
    assert cmds, "no translation units"
    for cmd in cmds:
        gencodes = [cmd[k + 1] for k, a in enumerate(cmd) if a == "-gencode"]
        assert gencodes == ["arch=compute_103a,code=sm_103a"], cmd
        assert "-arch" not in cmd and not any(a.startswith("--gpu-architecture") for a in cmd), cmd


def test_strerror_needs_no_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.sqcg_strerror.restype = ctypes.c_char_p
    assert lib.sqcg_strerror(0) == b"ok"
    assert b"invalid" in lib.sqcg_strerror(-1)
    assert b"converged" in lib.sqcg_strerror(-3)


def test_create_rejects_bad_extents_without_touching_the_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    for dims in [(7, 8, 8, 8), (8, 8, 8, 2), (0, 8, 8, 8)]:
        d = (ctypes.c_int * 4)(*dims)
        assert lib.sqcg_create(d, 1, None, ctypes.byref(h)) == -1
    d = (ctypes.c_int * 4)(8, 8, 8, 8)
    assert lib.sqcg_create(d, 64, None, ctypes.byref(h)) == -1  # unknown flag


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1611_00728_gb300 as pkg

    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU path"):
        pkg.library()


def test_host_side_argument_checks(libpath):
    """Checks that return before any CUDA call: lattice extents, the 2^28-site index limit, flags,
    null handles, and the HISQ workspace size (host arithmetic only)."""
    lib = ctypes.CDLL(libpath)
    lib.sqcg_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.sqcg_hisq_workspace_bytes.argtypes = [ctypes.c_void_p]
    lib.sqcg_hisq_workspace_bytes.restype = ctypes.c_size_t
    lib.sqcg_destroy.argtypes = [ctypes.c_void_p]
    h = ctypes.c_void_p()

    def create(dims, flags=1):
        return lib.sqcg_create((ctypes.c_int * 4)(*dims), flags, None, ctypes.byref(h))

    for dims in ((8, 8, 8, 5), (2, 8, 8, 8), (8, 8, 0, 8), (8, -8, 8, 8), (128, 128, 128, 130)):
        assert create(dims) == -1, dims
        assert not h.value
    assert create((8, 8, 8, 8), flags=4) == -1  # unknown flag
    assert lib.sqcg_create(None, 1, None, ctypes.byref(h)) == -1
    assert lib.sqcg_destroy(None) == 0
    # 32^4: (4 thin + 36 staple + 12 Z + 4 projected) fields of V 3x3 complex doubles, plus a flag
    V = 32 ** 4
    assert lib.sqcg_hisq_workspace_bytes((ctypes.c_int * 4)(32, 32, 32, 32)) == 56 * 9 * V * 16 + 256
    assert lib.sqcg_hisq_workspace_bytes((ctypes.c_int * 4)(4, 4, 4, 3)) == 0
    assert lib.sqcg_hisq_workspace_bytes(None) == 0


def test_multishift_record_checks_its_arguments(libpath):
    """The shift-aware update record is read on the host; a missing context or output is refused."""
    lib = ctypes.CDLL(libpath)
    f = lib.sqcg_multishift_ru_record
    f.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5
    n, ns = ctypes.c_int(), ctypes.c_int()
    assert f(None, 4, ctypes.byref(n), ctypes.byref(ns), None, None, None) == -1
    assert f(None, 4, None, None, None, None, None) == -1


def test_batched_pin_tuning_checks(libpath):
    """The pinned batched Dslash configuration is validated on the host (no CUDA call)."""
    lib = ctypes.CDLL(libpath)
    pin = lib.sqcg_batched_pin_tuning
    pin.argtypes = [ctypes.c_int] * 5
    bad = [(3, 1, 64, -1, 32), (4, 8, 64, -1, 32), (2, 4, 64, -1, 32), (4, 3, 64, -1, 32),  # W, WT
           (6, 2, 32, -1, 32), (12, 8, 32, -1, 32), (24, 2, 32, -1, 32),
           (4, 1, 48, -1, 32), (4, 1, 256, -1, 32), (16, 1, 64, -1, 32),  # T: multiple of 32, <= 128, T W/WT <= 512
           (4, 1, 64, 101, 32), (4, 1, 64, -2, 32),  # carveout
           (4, 4, 64, -1, 16), (8, 2, 32, -1, 8), (2, 1, 32, -1, 24)]  # warp_sites: 16 needs W / WT even
    for args in bad:
        assert pin(*args) == -1, args
    for args in [(1, 1, 32, -1, 32), (16, 4, 128, 50, 0), (8, 4, 128, -1, 16), (16, 2, 64, 25, 16), (2, 1, 32, -1, 16),
                 (12, 2, 64, -1, 16), (12, 4, 128, -1, 32)]:
        assert pin(*args) == 0, args
    assert pin(0, 0, 0, 0, 0) == 0  # back to autotuning


def test_binding_pin_batched_tuning(libpath):
    """The binding's pin call reaches the host-side checks (no GPU needed) and raises on a bad shape."""
    import paper_1611_00728_gb300 as sq

    sq.pin_batched_tuning(16, WT=2, T=32, carve=-1)
    with pytest.raises(sq.SqcgError) as e:
        sq.pin_batched_tuning(16, WT=1, T=64)  # 64 x 16 threads > 512
    assert e.value.name == "INVALID_ARG"
    sq.pin_batched_tuning(0)


def test_binding_network_layout_matches_the_library(libpath):
    """The binding's parameter layout (used to hand weights to the oracle) covers exactly the
    library's parameter count, with no gap or overlap."""
    import paper_1611_00728_gb300 as sq

    lib = ctypes.CDLL(libpath)
    assert lib.sqcg_nn_nparams() == sq.NN_NPARAMS
    covered = np.zeros(sq.NN_NPARAMS, int)
    for sl, shape in sq.NN_LAYERS:
        assert sl.stop - sl.start == 2 * int(np.prod(shape))
        covered[sl] += 1
    for ga, gb in sq.NN_GATES:
        covered[ga] += 1
        covered[gb] += 1
    assert np.all(covered == 1)
