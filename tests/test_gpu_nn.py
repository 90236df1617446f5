"""Preconditioner network and flexible CG on the GPU vs the FP64 numpy oracle (oracle/nn.py).

Forward pass and training gradient are compared element by element with the
oracle evaluated on the same BF16-rounded weights; the GPU accumulates in FP32,
so the bars are relative errors of 1e-5 (forward) and 1e-4 (loss, gradient).
Flexible-CG solutions must reach the true relative residual tol recomputed by
the FP64 oracle; the fallback to plain CG is exercised with a network that
outputs zero.
"""

import numpy as np
import pytest
import torch

import oracle
import oracle.nn as onn
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def flat_to_params(p):
    """Host parameter layout (include/sqcg.h) -> oracle parameter dict."""
    p = np.asarray(p, dtype=np.float64)
    c = p[:1440].reshape(-1, 2)
    w = c[:, 0] + 1j * c[:, 1]
    return {"W": [w[:72].reshape(9, 8, 1), w[72:648].reshape(9, 8, 8), w[648:720].reshape(9, 1, 8)],
            "gates": [(p[1440:1448], p[1448:1456]), (p[1456:1464], p[1464:1472])]}


def params_to_flat(d):
    out = np.zeros(1472)
    w = np.concatenate([d["W"][0].ravel(), d["W"][1].ravel(), d["W"][2].ravel()])
    out[:1440:2], out[1:1440:2] = w.real, w.imag
    out[1440:1448], out[1448:1456] = d["gates"][0]
    out[1456:1464], out[1464:1472] = d["gates"][1]
    return out.astype(np.float32)


def to_f32(x):
    return np.asarray(x, dtype=np.complex64).astype(np.complex128)


def bf16c(z):
    """Round each real component to bfloat16, to nearest even (the GPU's conversion of the taps)."""
    def r(x):
        b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(np.real(z)) + 1j * r(np.imag(z))


@pytest.mark.parametrize("L", [(4, 4, 4, 6), (8, 8, 8, 8), (6, 8, 10, 12)])
def test_network_bf16_mixing_matches_the_rounded_oracle(sqcg, links_cache, L):
    """The tensor-core 8 -> 8 mixing (NN_MIX_BF16) computes the FP64 network with the second layer's nine
    tap fields rounded to BF16 (the weights are BF16 values already) and FP32 sums. So it matches the oracle
    forward pass with exactly that rounding inserted, to FP32 accuracy, up to the rare component whose FP32
    and FP64 values round to different BF16 neighbours (one in 2^16, each a 2^-8 change of one term); and
    it differs from the unrounded network by about the BF16 unit roundoff 2^-9."""
    fat, lng = links_cache(L, 51)
    r = to_f32(synth.gaussian_source(L, 52))
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(5, scale=0.6)))
        net.set_mixing(sqcg.NN_MIX_BF16)
        got = lat.unpack(net.apply(lat.pack(r, sqcg.F32), lat.new_spinor(sqcg.F32)), sqcg.F32)
        params = flat_to_params(net.get_params(bf16_rounded=True))
        with pytest.raises(sqcg.SqcgError):
            net.set_mixing(2)
        net.close()
    U = onn.folded_fat(L, fat)
    par = oracle.parity_of_sites(L)
    s = np.sqrt(r.size) / np.linalg.norm(r)
    h0 = np.zeros((1, par.size, 3), dtype=np.complex128)
    h0[0, par == 0] = r * s
    W, gates = params["W"], params["gates"]
    h1, _ = onn.gate(onn.conv(L, U, W[0], h0), *gates[0])
    taps = [bf16c(t) for t in onn.transports(L, U, h1)]
    a2 = sum(np.einsum("oi,inc->onc", W[1][k], taps[k]) for k in range(len(taps)))
    h2, _ = onn.gate(a2, *gates[1])
    want = onn.conv(L, U, W[2], h2)[0, par == 0] / s
    assert rel(got, want) <= 1e-4
    exact = onn.apply(L, fat, params, r)
    assert 1e-5 < rel(got, exact) <= 2.0 ** -6


@pytest.mark.parametrize("L", [(4, 4, 4, 6), (8, 8, 8, 8), (6, 8, 10, 12)])
def test_network_forward_matches_oracle(sqcg, links_cache, L):
    fat, lng = links_cache(L, 51)
    r = to_f32(synth.gaussian_source(L, 52))
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(5, scale=0.6)))
        z = net.apply(lat.pack(r, sqcg.F32), lat.new_spinor(sqcg.F32))
        got = lat.unpack(z, sqcg.F32)
        want = onn.apply(L, fat, flat_to_params(net.get_params(bf16_rounded=True)), r)
        net.close()
    assert rel(got, want) <= 1e-5


def test_network_gauge_covariance_on_gpu(sqcg, links_cache):
    L = (8, 8, 8, 8)
    fat, lng = links_cache(L, 53)
    G = synth.random_gauge(L, 54)
    r = synth.gaussian_source(L, 55)
    params = params_to_flat(onn.init_params(6, scale=0.6))
    outs = []
    for f, l, src in [(fat, lng, r), (synth.gauge_transform_links(L, fat, G, 1), synth.gauge_transform_links(L, lng, G, 3),
                                      synth.gauge_transform_parity_field(L, r, G, 0))]:
        with sqcg.Lattice(L) as lat:
            lat.load_links(f, l)
            net = sqcg.Network(lat)
            net.set_params(params)
            outs.append(lat.unpack(net.apply(lat.pack(src, sqcg.F32), lat.new_spinor(sqcg.F32)), sqcg.F32))
            net.close()
    assert rel(outs[1], synth.gauge_transform_parity_field(L, outs[0], G, 0)) <= 1e-5


@pytest.mark.parametrize("norm", [1, 2])
def test_loss_and_gradient_match_oracle(sqcg, links_cache, norm):
    L, sigma = (4, 4, 4, 6), 0.05
    fat, lng = links_cache(L, 56)
    r = to_f32(synth.gaussian_source(L, 57))
    e = to_f32(np.linalg.solve(oracle.dense_normal_matrix(L, fat, lng, sigma), r.ravel()).reshape(r.shape))
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(7, scale=0.7)))
        net.set_loss(norm)
        loss, grad = net.loss_grad(sigma, lat.pack(r, sqcg.F32), lat.pack(e, sqcg.F32))
        p = flat_to_params(net.get_params(bf16_rounded=True))
        net.close()
    want_loss, g = onn.loss_and_grad(L, fat, lng, p, r, e, sigma, norm=norm)
    want = params_to_flat(g).astype(np.float64)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)
    assert rel(grad.astype(np.float64), want) <= 1e-4
    for lo, hi in [(0, 144), (144, 1296), (1296, 1440), (1440, 1472)]:  # every block of parameters
        assert rel(grad[lo:hi].astype(np.float64), want[lo:hi]) <= 1e-3


def test_training_kernels_ignore_the_inference_mixing(sqcg, links_cache):
    """The BF16 tensor-core mixing is an inference option: the loss and gradient (the training forward
    pass keeps its pre-activations and runs in FP32) are the same bits with either setting, while the
    network's inference output changes and comes back bit for bit when FP32 mixing is set again."""
    L, sigma = (4, 4, 4, 6), 0.05
    fat, lng = links_cache(L, 56)
    r = to_f32(synth.gaussian_source(L, 57))
    e = to_f32(synth.gaussian_source(L, 58))
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(7, scale=0.7)))
        dr, de = lat.pack(r, sqcg.F32), lat.pack(e, sqcg.F32)

        def infer():
            return lat.unpack(net.apply(dr, lat.new_spinor(sqcg.F32)), sqcg.F32)

        l32, g32 = net.loss_grad(sigma, dr, de)
        z32 = infer()
        net.set_mixing(sqcg.NN_MIX_BF16)
        l16, g16 = net.loss_grad(sigma, dr, de)
        z16 = infer()
        net.set_mixing(sqcg.NN_MIX_FP32)
        zb = infer()
        net.close()
    assert l16 == l32 and np.array_equal(g16, g32)
    assert not np.array_equal(z16, z32) and np.array_equal(zb, z32)


def make_pairs(sqcg, lat, net, fat, lng, m, seeds, ks):
    """(r_k, e_k) pairs from CG iterates x_k (CG from 0 truncated at k iterations) and a tight x*."""
    sigma = 4 * m * m
    rs, es = [], []
    for sd in seeds:
        b = lat.pack(synth.gaussian_source(lat.dims, sd))
        xs = lat.new_spinor()
        lat.cg_solve(m, b, xs, tol=1e-12, max_iter=20000, mode=0)
        for k in ks:
            xk = lat.new_spinor()
            if k > 0:  # the k-th CG iterate from x0 = 0 (k = 0: x0 itself)
                lat.cg_solve(m, b, xk, tol=1e-30, max_iter=k, mode=0, raise_on_error=False)
            r32, e32 = lat.new_spinor(sqcg.F32), lat.new_spinor(sqcg.F32)
            net.make_pair(sigma, b, xk, xs, r32, e32)
            rs.append(r32)
            es.append(e32)
    return torch.stack(rs).contiguous(), torch.stack(es).contiguous()


def test_training_pair_matches_oracle(sqcg, links_cache):
    L, m = (8, 8, 8, 8), 0.05
    fat, lng = links_cache(L, 58)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        b = synth.gaussian_source(L, 59)
        xk = synth.gaussian_source(L, 60)
        xs = synth.gaussian_source(L, 61)
        r32, e32 = lat.new_spinor(sqcg.F32), lat.new_spinor(sqcg.F32)
        net.make_pair(4 * m * m, lat.pack(b), lat.pack(xk), lat.pack(xs), r32, e32)
        assert rel(lat.unpack(r32, sqcg.F32), b - oracle.normal_op(L, fat, lng, 4 * m * m, xk)) <= 1e-6
        assert rel(lat.unpack(e32, sqcg.F32), xs - xk) <= 1e-6
        net.close()


def test_training_lowers_loss_and_fcg_converges(sqcg, links_cache):
    L, m, tol = (8, 8, 8, 8), 0.02, 1e-8
    fat, lng = links_cache(L, 62)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(8, scale=0.3)))
        net.set_loss(2)
        R, E = make_pairs(sqcg, lat, net, fat, lng, m, seeds=[70, 71, 72], ks=[0, 2, 5, 10, 20])
        first, last = net.train(4 * m * m, R, E, steps=150, batch=4, lr=2e-2, seed=3)
        assert last < first
        # held-out source: flexible CG preconditioned by the trained network
        b = synth.gaussian_source(L, 90)
        x = lat.new_spinor()
        info = net.fcg_solve(m, lat.pack(b), x, tol=tol, max_iter=2000)
        assert info.status == 0 and info.true_rel_resid <= tol
        assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, b, lat.unpack(x)) <= tol
        net.close()


def test_fcg_falls_back_to_plain_cg(sqcg, links_cache):
    L, m, tol = (8, 8, 8, 8), 0.05, 1e-8
    fat, lng = links_cache(L, 63)
    b = synth.gaussian_source(L, 91)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)  # all parameters zero: N(r) = 0, so <z, r> = 0 (breakdown)
        x = lat.new_spinor()
        info = net.fcg_solve(m, lat.pack(b), x, tol=tol, max_iter=2000)
        assert info.fallback == 1 and info.status == 0
        assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, b, lat.unpack(x)) <= tol
        net.close()


def test_fcg_reuses_its_graph_and_follows_new_links(sqcg, links_cache):
    """The captured flexible-CG loop is reused for the same buffers (identical iterates), starts from a
    nonzero guess through the FP64 residual, and is recaptured when the links change."""
    L, m, tol = (8, 8, 8, 8), 0.05, 1e-8
    fat, lng = links_cache(L, 62)
    fat2, lng2 = links_cache(L, 64)
    b = synth.gaussian_source(L, 92)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(8, scale=0.3)))
        db, x = lat.pack(b), lat.new_spinor()
        i1 = net.fcg_solve(m, db, x, tol=tol, max_iter=2000)
        x1 = lat.unpack(x)
        x.zero_()
        i2 = net.fcg_solve(m, db, x, tol=tol, max_iter=2000)
        assert i1.status == i2.status == 0 and i1.iters == i2.iters
        assert np.array_equal(x1, lat.unpack(x))
        # nonzero initial guess: half the solution
        x.copy_(lat.pack(0.5 * x1))
        i3 = net.fcg_solve(m, db, x, tol=tol, max_iter=2000)
        assert i3.status == 0
        assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, b, lat.unpack(x)) <= tol
        # new links on the same context
        lat.load_links(fat2, lng2)
        x.zero_()
        i4 = net.fcg_solve(m, db, x, tol=tol, max_iter=2000)
        assert i4.status == 0
        assert oracle.true_rel_residual(L, fat2, lng2, 4 * m * m, b, lat.unpack(x)) <= tol
        # the tensor-core mixing: the loop is recaptured with it and still ends on the FP64 true residual (this
        # untrained network stalls the flexible loop with either mixing, so plain CG finishes both solves)
        net.set_mixing(sqcg.NN_MIX_BF16)
        x.zero_()
        i5 = net.fcg_solve(m, db, x, tol=tol, max_iter=2000)
        assert i5.status == 0 and i5.fallback == i4.fallback
        assert oracle.true_rel_residual(L, fat2, lng2, 4 * m * m, b, lat.unpack(x)) <= tol
        net.close()


def test_fcg_with_tensor_core_mixing_on_the_trained_network(sqcg):
    """The committed trained network (16^4, m = 0.005, held-out gauge field and source): flexible CG with the
    BF16 tensor-core mixing needs the iterations of the FP32 mixing within 10 %, without falling back to plain
    CG, and reaches the true relative residual recomputed by the FP64 oracle."""
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1611_00728_gb300",
                        "trained", "fcg_network_16x16x16x16.npy")
    if not os.path.exists(path):
        pytest.skip("no trained parameters")
    L, m, tol = (16, 16, 16, 16), 0.005, 1e-8
    fat, lng = synth.fat_long_links(L, 9000)
    b = synth.gaussian_source(L, 9100)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng, recon12=True)
        net = sqcg.Network(lat)
        net.set_params(np.load(path).astype(np.float32))
        db, x = lat.pack(b), lat.new_spinor()
        info = {}
        for mix in (sqcg.NN_MIX_FP32, sqcg.NN_MIX_BF16):
            net.set_mixing(mix)
            x.zero_()
            info[mix] = net.fcg_solve(m, db, x, tol=tol, max_iter=5000)
            assert info[mix].status == 0 and info[mix].fallback == 0
            assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, b, lat.unpack(x)) <= tol
        i32, i16 = info[sqcg.NN_MIX_FP32].iters, info[sqcg.NN_MIX_BF16].iters
        assert abs(i16 - i32) <= max(2, i32 // 10), (i32, i16)
        net.close()


@pytest.mark.parametrize("max_iter", [2000, 7])
def test_fcg_eager_and_graph_modes_are_bit_identical(sqcg, links_cache, monkeypatch, max_iter):
    """The captured flexible-CG loop and the eager profiling mode (one launch per kernel, the host branching
    where the graph's conditional nodes do) give identical iterates; max_iter = 7 ends on the iteration bound
    and hands over to plain CG."""
    L, m, tol = (8, 8, 8, 8), 0.05, 1e-8
    fat, lng = links_cache(L, 62)
    b = synth.gaussian_source(L, 93)
    out = {}
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        # a near-identity network (self taps 1, open gates) with small random taps: a preconditioner that keeps
        # the flexible CG converging, so the loop runs to the FP64 confirmation without falling back
        d = onn.init_params(8, scale=0.02)
        for w in d["W"]:
            w[0, 0, 0] += 1.0
        d["gates"] = [(np.zeros(8), np.full(8, 10.0)), (np.zeros(8), np.full(8, 10.0))]
        net.set_params(params_to_flat(d))
        db = lat.pack(b)
        for mode in ("graph", "eager"):
            if mode == "eager":
                monkeypatch.setenv("SQCG_LAUNCH_MODE", "eager")
            else:
                monkeypatch.delenv("SQCG_LAUNCH_MODE", raising=False)
            x = lat.new_spinor()
            info = net.fcg_solve(m, db, x, tol=tol, max_iter=max_iter, raise_on_error=False)
            out[mode] = (info.status, info.iters, info.reliable_updates, info.fallback, lat.unpack(x))
        net.close()
    g, e = out["graph"], out["eager"]
    assert g[:4] == e[:4] and np.array_equal(g[4], e[4])
    if max_iter == 7:  # the loop ends on the bound, plain CG takes over with what is left and stops too
        assert g[3] == 1 and g[0] == -3
    else:
        assert g[3] == 0 and g[0] == 0
        assert oracle.true_rel_residual(L, fat, lng, 4 * m * m, b, g[4]) <= tol


def test_network_closes_with_its_lattice(sqcg, links_cache):
    """A network left open is closed with its lattice (before the context it uses is destroyed)."""
    L = (4, 4, 4, 6)
    fat, lng = links_cache(L, 65)
    with sqcg.Lattice(L) as lat:
        lat.load_links(fat, lng)
        net = sqcg.Network(lat)
        net.set_params(params_to_flat(onn.init_params(8, scale=0.3)))
    assert net._h is None
    with pytest.raises(sqcg.SqcgError):
        net.set_params(params_to_flat(onn.init_params(8, scale=0.3)))
