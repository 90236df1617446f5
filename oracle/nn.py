"""FP64 numpy oracle of the gauge-covariant preconditioner network and its training gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). The CUDA library never uses it.

The network is not in the paper (arXiv:1611.00728 has no preconditioner); it is
the learned preconditioner of the flexible CG built around the paper's
single-mass CG (Sec. 3). Definition, written out plainly:

* fields live on the full lattice, C channels, each a colour vector per site;
* a parallel-transport convolution layer with complex channel weights
  W[tap][c_out][c_in], taps 0 = self, 1 + 2mu = forward hop, 2 + 2mu = backward hop:

      out_c(n) = sum_c' W[0][c][c'] in_c'(n)
               + sum_mu ( W[1+2mu][c][c'] F~_mu(n)        in_c'(n+mu)
                        + W[2+2mu][c][c'] F~_mu(n-mu)^dag in_c'(n-mu) )

  with F~ the fat links times eta_mu and the boundary sign (the Dslash's links);
* a gauge-invariant gate after layers 1 and 2: h_c(n) <- h_c(n) * sigmoid(a_c |h_c(n)|^2 + b_c);
* network N: even-site input r (odd sites zero) -> layer1 (1->8) -> gate -> layer2 (8->8) -> gate
  -> layer3 (8->1) -> even-site output. The input is scaled to unit RMS per complex
  component first (s = sqrt(3 Vh) / |r|) and the output scaled back by 1/s, so N(c r) = c N(r)
  for real c > 0.

Gauge covariance holds because the weights mix channels only (colour-blind),
links carry colour, and the gate depends on the gauge-invariant |h|.

Training loss for one (residual r, error e) pair with e = A^-1 r, d = N(r) - e,
A = sigma - D_eo D_oe, in one of two norms:
    norm 1:  L = <d, A d> / <e, r>         (A-norm of the error relative to that of e)
    norm 2:  L = <A d, A d> / <r, r>       (A^2-norm: the residual of the preconditioned
                                            step, |A N(r) - r|^2 / |r|^2, since A e = r)
"""

from __future__ import annotations

import numpy as np

import oracle

NTAP = 9
CHANNELS = (1, 8, 8, 1)


def _axes():
    return (3, 2, 1, 0)  # numpy axis of x, y, z, t in a (Lt, Lz, Ly, Lx, ...) array


def folded_fat(L, fat, antiperiodic_t: bool = True) -> np.ndarray:
    """Fat links times eta_mu(n) and the forward-hop boundary sign, [V][4][3][3]."""
    Lx, Ly, Lz, Lt = L
    V = Lx * Ly * Lz * Lt
    n = np.arange(V)
    x, y, z, t = n % Lx, (n // Lx) % Ly, (n // (Lx * Ly)) % Lz, n // (Lx * Ly * Lz)
    out = np.array(fat, dtype=np.complex128, copy=True)
    etas = [np.ones(V), (-1.0) ** x, (-1.0) ** (x + y), (-1.0) ** (x + y + z)]
    for mu in range(4):
        s = etas[mu].copy()
        if mu == 3 and antiperiodic_t:
            s = np.where(t + 1 >= Lt, -s, s)
        out[:, mu] *= s[:, None, None]
    return out


def init_params(seed: int = 0, scale: float = 0.3):
    """Random initial parameters (complex weights per layer, gate a, b per gated layer)."""
    rng = np.random.default_rng(seed)
    Ws = []
    for l in range(3):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        w = (rng.standard_normal((NTAP, cout, cin)) + 1j * rng.standard_normal((NTAP, cout, cin)))
        Ws.append(w * scale / np.sqrt(NTAP * cin))
    gates = [(np.full(CHANNELS[1], -0.5), np.full(CHANNELS[1], 1.0)),
             (np.full(CHANNELS[2], -0.5), np.full(CHANNELS[2], 1.0))]
    return {"W": Ws, "gates": gates}


def _shift(L, f, mu, d):
    """f(n + d mu) for a full-lattice field f[..., V, 3] (periodic)."""
    Lx, Ly, Lz, Lt = L
    g = f.reshape(f.shape[:-2] + (Lt, Lz, Ly, Lx, 3))
    ax = len(f.shape) - 2 + _axes()[mu]
    return np.roll(g, -d, axis=ax).reshape(f.shape)


def transports(L, U, h):
    """The 9 tap fields of h[C][V][3]: self, U_mu(n) h(n+mu), U_mu(n-mu)^dag h(n-mu)."""
    Lx, Ly, Lz, Lt = L
    taps = [h]
    for mu in range(4):
        Umu = U[:, mu]
        fwd = np.einsum("nab,cnb->cna", Umu, _shift(L, h, mu, +1))
        Um = np.roll(Umu.reshape(Lt, Lz, Ly, Lx, 3, 3), 1, axis=_axes()[mu]).reshape(-1, 3, 3)  # U_mu(n - mu)
        bwd = np.einsum("nba,cnb->cna", np.conj(Um), _shift(L, h, mu, -1))
        taps += [fwd, bwd]
    return taps


def conv(L, U, W, h):
    """One parallel-transport conv layer: h[C_in][V][3] -> [C_out][V][3]."""
    taps = transports(L, U, h)
    out = np.zeros((W.shape[1],) + h.shape[1:], dtype=np.complex128)
    for k in range(NTAP):
        out += np.einsum("oi,inc->onc", W[k], taps[k])
    return out


def gate(h, a, b):
    s = np.sum(np.abs(h) ** 2, axis=-1)  # [C][V]
    g = 1.0 / (1.0 + np.exp(-(a[:, None] * s + b[:, None])))
    return h * g[..., None], (s, g)


def forward(L, U, params, r_even):
    """N(r) on the even sites, with the intermediates needed for the gradient."""
    par = oracle.parity_of_sites(L)
    V = par.size
    r_even = np.asarray(r_even, dtype=np.complex128)
    s = np.sqrt(r_even.size) / np.linalg.norm(r_even)
    h0 = np.zeros((1, V, 3), dtype=np.complex128)
    h0[0, par == 0] = r_even * s
    W, gates = params["W"], params["gates"]
    a1 = conv(L, U, W[0], h0)
    h1, g1 = gate(a1, *gates[0])
    a2 = conv(L, U, W[1], h1)
    h2, g2 = gate(a2, *gates[1])
    a3 = conv(L, U, W[2], h2)
    z = a3[0, par == 0] / s
    cache = dict(s=s, h0=h0, a1=a1, h1=h1, g1=g1, a2=a2, h2=h2, g2=g2, par=par)
    return z, cache


def apply(L, fat, params, r_even, antiperiodic_t: bool = True):
    return forward(L, folded_fat(L, fat, antiperiodic_t), params, r_even)[0]


def conv_adjoint_input(L, U, W, g):
    """Adjoint of conv with respect to its input: grad_in = sum_taps W^H (transport^dag) g."""
    Lx, Ly, Lz, Lt = L
    out = np.einsum("oi,onc->inc", np.conj(W[0]), g)
    for mu in range(4):
        Umu = U[:, mu]
        U5 = Umu.reshape(Lt, Lz, Ly, Lx, 3, 3)
        Um = np.roll(U5, 1, axis=_axes()[mu]).reshape(-1, 3, 3)  # U_mu(m - mu)
        # forward tap: out(n) += W U_mu(n) h(n+mu)  ->  grad_h(m) += W^H U_mu(m-mu)^dag g(m-mu)
        gm = _shift(L, g, mu, -1)
        t = np.einsum("nba,onb->ona", np.conj(Um), gm)
        out += np.einsum("oi,onc->inc", np.conj(W[1 + 2 * mu]), t)
        # backward tap: out(n) += W U_mu(n-mu)^dag h(n-mu)  ->  grad_h(m) += W^H U_mu(m) g(m+mu)
        gp = _shift(L, g, mu, +1)
        t = np.einsum("nab,onb->ona", Umu, gp)
        out += np.einsum("oi,onc->inc", np.conj(W[2 + 2 * mu]), t)
    return out


def conv_weight_grad(L, U, h, g):
    """dL/dW[tap][o][i] = sum_n <tap_i(n), g_o(n)> (complex gradient convention dL/dRe + i dL/dIm)."""
    taps = transports(L, U, h)
    return np.stack([np.einsum("inc,onc->oi", np.conj(t), g) for t in taps])


def gate_backward(h, a, b, cache, gout):
    """Gradient through h -> h * sigmoid(a |h|^2 + b); returns (grad_h, grad_a, grad_b)."""
    s, g = cache
    # out = h g(s); dout = g dh + h g' ds, g' = g (1 - g) (a), ds = 2 Re(h^* dh)
    proj = np.real(np.sum(np.conj(h) * gout, axis=-1))  # Re <h, gout> per channel, site
    gp = g * (1 - g)
    grad_h = g[..., None] * gout + (2 * a[:, None] * gp * proj)[..., None] * h
    grad_a = np.sum(gp * s * proj, axis=1)
    grad_b = np.sum(gp * proj, axis=1)
    return grad_h, grad_a, grad_b


def loss_and_grad(L, fat, lng, params, r_even, e_even, sigma, antiperiodic_t: bool = True, norm: int = 1):
    """Training loss of one (r, e) pair (norm 1 or 2, see the module docstring) and its
    gradient w.r.t. every parameter.

    The loss is invariant under (r, e) -> (c r, c e) because N(c r) = c N(r)."""
    U = folded_fat(L, fat, antiperiodic_t)
    z, c = forward(L, U, params, r_even)
    d = z - e_even
    Ad = oracle.normal_op(L, fat, lng, sigma, d, antiperiodic_t)
    if norm == 1:
        er = np.real(np.vdot(e_even, r_even))
        loss = float(np.real(np.vdot(d, Ad)) / er)
        gz = 2.0 * Ad / er  # dL/dz (complex convention: dL/dRe z + i dL/dIm z)
    else:
        rr = np.real(np.vdot(r_even, r_even))
        loss = float(np.real(np.vdot(Ad, Ad)) / rr)
        gz = 2.0 * oracle.normal_op(L, fat, lng, sigma, Ad, antiperiodic_t) / rr
    par = c["par"]
    W, gates = params["W"], params["gates"]
    g3 = np.zeros((1, par.size, 3), dtype=np.complex128)
    g3[0, par == 0] = gz / c["s"]
    dW3 = conv_weight_grad(L, U, c["h2"], g3)
    gh2 = conv_adjoint_input(L, U, W[2], g3)
    ga2, da2, db2 = gate_backward(c["a2"], *gates[1], c["g2"], gh2)
    dW2 = conv_weight_grad(L, U, c["h1"], ga2)
    gh1 = conv_adjoint_input(L, U, W[1], ga2)
    ga1, da1, db1 = gate_backward(c["a1"], *gates[0], c["g1"], gh1)
    dW1 = conv_weight_grad(L, U, c["h0"], ga1)
    grads = {"W": [dW1, dW2, dW3], "gates": [(da1, db1), (da2, db2)]}
    return loss, grads
