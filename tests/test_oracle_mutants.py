"""Strength of the oracle pins: plant a plausible mistake in a copy of the oracle
source, build it, and check that at least one pin in test_oracle.py fails.

The mistakes are planted only in a temporary copy compiled on the CPU; the
committed oracle is untouched.
"""

import contextlib
import ctypes
import os
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sqcg_oracle.c")

# (name, original text, planted text)
MUTANTS = [
    ("drop Naik term", "for (int k = 0; k < 2; ++k)", "for (int k = 0; k < 1; ++k)"),
    ("backward hop sign", "add_mdv(out, -hop_sign(", "add_mdv(out, hop_sign("),
    ("missing dagger on backward link", "add_mdv(out, -hop_sign(L, apbc, y, mu, d)", "add_mv(out, -hop_sign(L, apbc, y, mu, d)"),
    ("backward link read at n", "link(U, m, mu), psi + m * 3", "link(U, n, mu), psi + m * 3"),
    ("wrong staggered phase", "for (int nu = 0; nu < mu; ++nu) s += x[nu];", "for (int nu = 0; nu <= mu; ++nu) s += x[nu];"),
    ("boundary sign only on one-hop crossings", "x[3] + d >= L[3]", "x[3] + 1 >= L[3]"),
    ("boundary sign taken at the output site", "-hop_sign(L, apbc, y, mu, d)", "-hop_sign(L, apbc, x, mu, d)"),
    ("long hop of length 2", "(k == 0) ? 1 : 3", "(k == 0) ? 1 : 2"),
    ("transposed link", "s += U[a * 3 + b] * v[b];", "s += U[b * 3 + a] * v[b];"),
    ("normal operator sign", "sigma * x[n * 3 + a] - y[n * 3 + a]", "sigma * x[n * 3 + a] + y[n * 3 + a]"),
    ("CG beta inverted", "const double beta = rr_new / rr;", "const double beta = rr / rr_new;"),
    ("CG residual update sign", "r[i] -= alpha * Ap[i];", "r[i] += alpha * Ap[i];"),
]


def _pin_suite():
    """Run a representative set of pins; return the names of those that fail."""
    checks = {
        "free field D": lambda: pins.test_free_field_single_hop_closed_form((6, 8, 10, 12), True),
        "free field D (periodic)": lambda: pins.test_free_field_single_hop_closed_form((8, 10, 12, 14), False),
        "free field spectrum": lambda: pins.test_free_field_normal_spectrum((6, 8, 10, 12), True),
        "anti-Hermiticity": lambda: pins.test_anti_hermiticity((6, 8, 10, 12)),
        "gauge covariance": lambda: pins.test_gauge_covariance((6, 8, 10, 12), 0),
        "Hermitian positive": lambda: pins.test_normal_op_hermitian_positive((4, 4, 4, 4)),
        "dense LU": pins.test_cg_matches_dense_lu_4444,
        "free field solve": lambda: pins.test_free_field_solve_closed_form(True),
    }
    failed = []
    for name, fn in checks.items():
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


@contextlib.contextmanager
def _oracle_library(path):
    saved = oracle._lib
    oracle._lib = None
    real_build = oracle.build
    try:
        oracle._LIB_PATH_SAVED = oracle._LIB_PATH
        oracle._LIB_PATH = path
        oracle.build = lambda force=False: path
        yield
    finally:
        oracle._LIB_PATH = oracle._LIB_PATH_SAVED
        oracle.build = real_build
        oracle._lib = saved


def test_unmodified_oracle_passes_all_pins():
    assert _pin_suite() == []


@pytest.mark.parametrize("name,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, planted):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation anchor not found: {orig}"
    with tempfile.TemporaryDirectory() as d:
        cpath = os.path.join(d, "mutant.c")
        so = os.path.join(d, "libmutant.so")
        with open(cpath, "w") as f:
            f.write(src.replace(orig, planted, 1))
        subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", so, cpath, "-lm"],
                       check=True)
        with _oracle_library(so):
            failed = _pin_suite()
            ctypes.CDLL(so)  # keep symbol resolution honest
    assert failed, f"planted mistake '{name}' passed every pin"
