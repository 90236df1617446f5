"""Batched multi-RHS CG over lattices of different volumes, through the C ABI.

Every right-hand side must reach a true relative residual <= tol, recomputed
here by the FP64 oracle from the returned x; a batched solve must agree with
the single-RHS solver. The full batched workload (16 sources each on 16^4,
24^4 and 32^3x64, m = 0.02) is checked on the oracle's FP64 true residual for
every one of its 48 solutions.
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def make_batch(sq, lat, srcs):
    b = torch.stack([lat.pack(s) for s in srcs]).contiguous()
    x = torch.zeros_like(b)
    return b, x


@pytest.mark.parametrize("recon", [False, True])
def test_batched_small_uneven(sqcg, links_cache, recon):
    specs = [((8, 8, 8, 8), 3, 0.1), ((6, 8, 10, 12), 5, 0.05), ((4, 4, 4, 8), 2, 0.2)]
    tol = 1e-9
    lats, bs, xs, srcs, links = [], [], [], [], []
    for n, (L, nr, m) in enumerate(specs):
        fat, lng = links_cache(L, 400 + n)
        lat = sqcg.Lattice(L)
        lat.load_links(fat, lng, recon12=recon and n == 1)
        s = [synth.gaussian_source(L, 5000 + 10 * n + j) for j in range(nr)]
        b, x = make_batch(sqcg, lat, s)
        lats.append(lat); bs.append(b); xs.append(x); srcs.append(s); links.append((fat, lng))
    infos = sqcg.cg_solve_batched(lats, [m for _, _, m in specs], bs, xs, tol=tol, max_iter=5000)
    W, T = sqcg.batched_tuning(lats[0])
    assert W in (1, 2, 4, 8, 12, 16) and T in (32, 64, 128, 256)
    for n, (L, nr, m) in enumerate(specs):
        fat, lng = links[n]
        for j in range(nr):
            assert infos[n][j].status == 0 and infos[n][j].true_rel_resid <= tol
            x = lats[n].unpack(xs[n][j])
            assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, srcs[n][j], x) <= tol
    # agrees with the single-RHS solver on the same system
    L, nr, m = specs[0]
    dx = lats[0].new_spinor()
    lats[0].cg_solve(m, bs[0][1], dx, tol=1e-12, max_iter=5000, mode=0)
    ref = lats[0].unpack(dx)
    got = lats[0].unpack(xs[0][1])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 10 * tol
    # a second call with the same arguments reuses the cached plan and graph
    for x in xs:
        x.zero_()
    infos2 = sqcg.cg_solve_batched(lats, [m for _, _, m in specs], bs, xs, tol=tol, max_iter=5000)
    assert [i.iters for i in infos2[1]] == [i.iters for i in infos[1]]
    for lat in lats:
        lat.close()


def test_batched_edge_cases(sqcg, links_cache):
    L = (8, 8, 8, 8)
    fat, lng = links_cache(L, 1001)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        srcs = [synth.gaussian_source(L, 7000 + j) for j in range(3)]
        srcs[1] = np.zeros_like(srcs[1])  # zero source -> x = 0
        b, x = make_batch(sqcg, lat, srcs)
        x.fill_(1.0)  # initial guesses (the zero source must still give x = 0)
        infos = sqcg.cg_solve_batched([lat], [0.1], [b], [x], tol=1e-8)[0]
        assert all(i.status == 0 for i in infos)
        assert not torch.any(x[1])
        for j in (0, 2):
            assert oracle.true_rel_residual(L, fat, lng, 0.04, srcs[j], lat.unpack(x[j])) <= 1e-8
        # max_iter reached
        x.zero_()
        infos = sqcg.cg_solve_batched([lat], [0.1], [b], [x], tol=1e-14, max_iter=4, raise_on_error=False)[0]
        assert infos[0].status == -3 and infos[0].iters <= 4
        # NaN source -> breakdown for that RHS only
        bad = [s.copy() for s in srcs]
        bad[2][5, 0] = np.nan
        b2, x2 = make_batch(sqcg, lat, bad)
        infos = sqcg.cg_solve_batched([lat], [0.1], [b2], [x2], tol=1e-8, raise_on_error=False)[0]
        assert infos[0].status == 0 and infos[2].status == -4
        # invalid arguments
        with pytest.raises(sqcg.SqcgError):
            sqcg.cg_solve_batched([lat, lat], [0.1, 0.1], [b, b], [x, x2])  # same context twice


def test_batched_full_workload(sqcg, links_cache):
    """16 sources each on 16^4, 24^4 and 32^3x64 at m = 0.02, FP32 with FP64 reliable updates, tol 1e-8."""
    specs = [(16, 16, 16, 16), (24, 24, 24, 24), (32, 32, 32, 64)]
    m, tol, nr = 0.02, 1e-8, 16
    lats, bs, xs, srcs, links = [], [], [], [], []
    for n, L in enumerate(specs):
        fat, lng = links_cache(L, 1004 + n)
        lat = sqcg.Lattice(L)
        lat.load_links(fat, lng)
        s = synth.gaussian_source(L, 2400 + 10 * n, nrhs=nr)
        b, x = make_batch(sqcg, lat, list(s))
        lats.append(lat); bs.append(b); xs.append(x); srcs.append(s); links.append((fat, lng))
    infos = sqcg.cg_solve_batched(lats, [m] * 3, bs, xs, tol=tol, max_iter=20000)
    for n in range(3):
        assert all(i.status == 0 and i.true_rel_resid <= tol for i in infos[n])
    # every one of the 48 solutions, recomputed by the FP64 oracle
    for n, L in enumerate(specs):
        fat, lng = links[n]
        for j in range(nr):
            x = lats[n].unpack(xs[n][j])
            res = oracle.true_rel_residual(L, fat, lng, 4 * m * m, srcs[n][j], x)
            assert res <= tol, (L, j, res)
            assert abs(res - infos[n][j].true_rel_resid) <= 1e-3 * tol, (L, j, res, infos[n][j].true_rel_resid)
    for lat in lats:
        lat.close()


def test_batched_from_two_host_threads(sqcg, links_cache):
    """Two host threads, each with its own contexts, tune and solve at the same time (the tuning state is
    process-wide and guarded); both answers are checked against the oracle."""
    import threading

    specs = [((8, 8, 8, 8), 2, 0.1, 300), ((6, 8, 10, 12), 3, 0.08, 301)]
    results, errors = {}, []

    def work(k, L, nr, m, seed):
        try:
            fat, lng = links_cache(L, seed)
            with sqcg.Lattice(L) as lat:
                lat.load_links(fat, lng)
                srcs = [synth.gaussian_source(L, 7100 + 10 * k + j) for j in range(nr)]
                b, x = make_batch(sqcg, lat, srcs)
                infos = sqcg.cg_solve_batched([lat], [m], [b], [x], tol=1e-9)[0]
                results[k] = [(i.status, oracle.true_rel_residual(L, fat, lng, 4 * m * m, s, lat.unpack(x[j])))
                              for j, (i, s) in enumerate(zip(infos, srcs))]
        except Exception as e:  # reported below
            errors.append(repr(e))

    # links first (the fixture caches them), then the threads
    for k, (L, nr, m, seed) in enumerate(specs):
        links_cache(L, seed)
    threads = [threading.Thread(target=work, args=(k, *spec)) for k, spec in enumerate(specs)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for k in range(len(specs)):
        assert all(st == 0 and res <= 1e-9 for st, res in results[k]), results[k]


@pytest.mark.parametrize("cfg", [dict(W=4, WT=1, T=64, carve=-1, warp_sites=32),
                                 dict(W=4, WT=1, T=32, carve=-1, warp_sites=16),
                                 dict(W=8, WT=2, T=128, carve=-1, warp_sites=32),
                                 dict(W=8, WT=2, T=64, carve=-1, warp_sites=16),
                                 dict(W=16, WT=2, T=32, carve=-1, warp_sites=16),
                                 dict(W=16, WT=4, T=64, carve=50, warp_sites=32),
                                 dict(W=16, WT=4, T=128, carve=-1, warp_sites=16),
                                 dict(W=2, WT=2, T=32, carve=25, warp_sites=32),
                                 dict(W=4, WT=4, T=32, carve=-1, warp_sites=32),
                                 dict(W=12, WT=2, T=32, carve=-1, warp_sites=16),
                                 dict(W=12, WT=4, T=64, carve=-1, warp_sites=32)])
def test_batched_pinned_configurations(sqcg, links_cache, cfg):
    """Every FP32 Dslash instantiation (1, 2 or 4 RHS per thread; warps of 32 sites of one RHS group or 16 sites
    of two; block widths W of powers of two and 12), pinned instead of tuned, on an uneven batch with a ragged RHS block and a 12-real long-link
    lattice: each RHS reaches tol on the oracle."""
    specs = [((8, 8, 8, 8), 5, 0.1), ((6, 8, 10, 12), 3, 0.05), ((4, 4, 4, 8), 1, 0.2)]
    tol = 1e-9
    sqcg.pin_batched_tuning(**cfg)
    try:
        lats, bs, xs, srcs, links = [], [], [], [], []
        for n, (L, nr, m) in enumerate(specs):
            fat, lng = links_cache(L, 410 + n)
            lat = sqcg.Lattice(L)
            lat.load_links(fat, lng, recon12=n == 1)
            s = [synth.gaussian_source(L, 5200 + 10 * n + j) for j in range(nr)]
            b, x = make_batch(sqcg, lat, s)
            lats.append(lat); bs.append(b); xs.append(x); srcs.append(s); links.append((fat, lng))
        infos = sqcg.cg_solve_batched(lats, [m for _, _, m in specs], bs, xs, tol=tol, max_iter=5000)
        assert sqcg.batched_tuning_ex(lats[0]) == cfg
    finally:
        sqcg.pin_batched_tuning(0)
    for n, (L, nr, m) in enumerate(specs):
        fat, lng = links[n]
        for j in range(nr):
            assert infos[n][j].status == 0 and infos[n][j].true_rel_resid <= tol
            assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, srcs[n][j], lats[n].unpack(xs[n][j])) <= tol
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("max_iter", [5000, 9])
def test_batched_eager_and_graph_modes_are_bit_identical(sqcg, links_cache, monkeypatch, max_iter):
    """The captured batched loop and the eager profiling mode (one launch per kernel, the host branching where
    the graph's conditional nodes do) give identical iterates; max_iter = 9 ends every RHS on the bound."""
    specs = [((8, 8, 8, 8), 5, 0.1), ((6, 8, 10, 12), 3, 0.05)]
    out = {}
    for mode in ("graph", "eager"):
        if mode == "eager":
            monkeypatch.setenv("SQCG_LAUNCH_MODE", "eager")
        else:
            monkeypatch.delenv("SQCG_LAUNCH_MODE", raising=False)
        lats, bs, xs = [], [], []
        for n, (L, nr, m) in enumerate(specs):
            fat, lng = links_cache(L, 420 + n)
            lat = sqcg.Lattice(L)
            lat.load_links(fat, lng, recon12=n == 1)
            b, x = make_batch(sqcg, lat, [synth.gaussian_source(L, 5300 + 10 * n + j) for j in range(nr)])
            lats.append(lat); bs.append(b); xs.append(x)
        infos = sqcg.cg_solve_batched(lats, [m for _, _, m in specs], bs, xs, tol=1e-9, max_iter=max_iter,
                                      raise_on_error=False)
        out[mode] = ([x.cpu().numpy() for x in xs], [(i.status, i.iters, i.reliable_updates) for r in infos for i in r])
        for lat in lats:
            lat.close()
    g, e = out["graph"], out["eager"]
    assert g[1] == e[1]
    assert all(np.array_equal(a, c) for a, c in zip(g[0], e[0]))
    assert all(st == (0 if max_iter == 5000 else -3) for st, _, _ in g[1])


@pytest.mark.parametrize("arith", ["FF", "F64"])
def test_batched_update_arithmetic_and_initial_guess(sqcg, links_cache, arith):
    """The batched solve's true-residual passes in float-float (default) or FP64 arithmetic, on two uneven
    lattices, once from zero and once from a nonzero initial guess (which takes the all-RHS initial
    residual pass); every solution is checked on the oracle's FP64 true residual."""
    specs = [((8, 8, 8, 8), 3, 0.1, 1001), ((6, 8, 10, 12), 2, 0.05, 55)]
    lats, bs, xs, srcs, links = [], [], [], [], []
    for n, (L, nr, m, seed) in enumerate(specs):
        fat, lng = links_cache(L, seed)
        lat = sqcg.Lattice(L)
        lat.load_links(fat, lng, recon12=True)
        lat.set_update_arithmetic(getattr(sqcg, arith))
        s = [synth.gaussian_source(L, 7300 + 10 * n + j) for j in range(nr)]
        b, x = make_batch(sqcg, lat, s)
        lats.append(lat); bs.append(b); xs.append(x); srcs.append(s); links.append((fat, lng))
    masses = [m for _, _, m, _ in specs]
    for start in ("zero", "guess"):
        if start == "guess":
            for x in xs:
                x.normal_()
        infos = sqcg.cg_solve_batched(lats, masses, bs, xs, tol=1e-9, max_iter=5000)
        for n, (L, nr, m, _) in enumerate(specs):
            fat, lng = links[n]
            for j in range(nr):
                assert infos[n][j].status == 0
                res = oracle.true_rel_residual(L, fat, lng, 4 * m * m, srcs[n][j], lats[n].unpack(xs[n][j]))
                assert res <= 1e-9, (arith, start, L, j, res)
                assert abs(res - infos[n][j].true_rel_resid) <= 1e-12, (res, infos[n][j].true_rel_resid)
    for lat in lats:
        lat.close()
