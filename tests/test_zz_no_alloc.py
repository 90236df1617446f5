"""sqcg_normal_op_noalloc: the normal operator for callers that cannot allocate
device memory when they apply it (their device memory belongs to their own
allocator or pool, or they cannot accept an allocation's latency). It keeps
its intermediate in a fixed array inside the library instead of the context's
workspace.

Checked, through the C ABI, on a fresh context whose solver workspace does not
exist yet: the call must leave the device's free memory unchanged, and its
result must match both sqcg_normal_op and the FP64 oracle's normal operator,
on two calls in a row, with the tolerances of the other operator tests. This
file is collected last so that a run stopping at the first failure has already
run everything else; it also passes alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
MiB = 1 << 20


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _noalloc(lib, lat, sigma, prec, x, y):
    lat._sync_stream()
    return lib.sqcg_normal_op_noalloc(lat._h, ctypes.c_double(sigma), prec, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L", [(16, 16, 16, 16), (8, 10, 12, 14)])
def test_noalloc_matches_oracle_and_normal_op_two_calls(sqcg, links_cache, L, prec):
    import torch

    fat, lng = links_cache(L, 1001)
    sigma = 4 * 0.05 ** 2
    lib = sqcg.library()
    xs_host = [synth.gaussian_source(L, seed) for seed in (31, 32)]
    # First use in this process of the fixed scratch and of these kernels (module loading may
    # reserve device memory once per process); a throwaway context takes it.
    with sqcg.Lattice(L) as warm:
        warm.load_links(fat, lng)
        wx, wy = warm.pack(xs_host[0], prec), warm.new_spinor(prec)
        assert _noalloc(lib, warm, sigma, prec, wx, wy) == 0
        torch.cuda.synchronize()
    with sqcg.Lattice(L) as lat:  # fresh context: no solver workspace yet
        lat.load_links(fat, lng)
        xs = [lat.pack(h, prec) for h in xs_host]
        got = [lat.new_spinor(prec) for _ in xs]
        want = [lat.new_spinor(prec) for _ in xs]
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for call in range(2):  # two calls in a row, different inputs, before any workspace exists
            assert _noalloc(lib, lat, sigma, prec, xs[call], got[call]) == 0, call
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free0 - free1 < 2 * MiB, (free0, free1)  # nothing allocated (page granularity)
        for call in range(2):
            lat.normal_op(sigma, xs[call], want[call], prec)  # allocates the context's workspace
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        for call in range(2):
            g, w = lat.unpack(got[call], prec), lat.unpack(want[call], prec)
            x_used = lat.unpack(xs[call], prec)  # the FP32 input as rounded on the device
            ref = oracle.normal_op(L, fat, lng, sigma, x_used)
            assert rel(g, ref) <= TOL[prec], (call, rel(g, ref))
            assert rel(g, w) <= TOL[prec], (call, rel(g, w))
    # the check above can see an allocation: the workspace (FP64 and FP32 r, p, Ap, tmp) is larger than 2 MiB
    Vh = int(np.prod(L)) // 2
    if 288 * Vh > 4 * MiB:
        assert free1 - free2 >= 2 * MiB, (free1, free2)


def test_noalloc_rejects_lattices_beyond_the_scratch(sqcg):
    lib = sqcg.library()
    with sqcg.Lattice((32, 32, 32, 32)) as lat:  # 524288 sites per parity
        x, y = lat.new_spinor(1), lat.new_spinor(1)
        rc = _noalloc(lib, lat, 0.1, 1, x, y)
        assert rc == -8
        assert b"too large" in lib.sqcg_strerror(rc)
