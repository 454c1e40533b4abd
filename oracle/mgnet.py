"""Oracle: CoeffNet + MgNet V-cycle, the physics-informed loss and Adam (Sec. 3).

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Float64 NumPy.  The network
is written as a sequence of textbook primitive operations recorded on a small
tape; reverse mode walks the tape backwards with each primitive's own
derivative.  Pinned by finite differences (P16), by scipy's correlate2d for
the convolutions, by the transposed-convolution adjoint identity (P11) and by
the identity-network special case (zero projection: the network returns its
input, so the preconditioner reduces to block Jacobi).

Readings of the paper (Sec. 3.1-3.4, silent or ambiguous there):
* CoeffNet input (Sec. 3.2): log sigma_T, log sigma_a, log eps and log tau per
  cell; level l: conv 3x3 (stride 1 at level 0, stride 2 after) -> batch
  normalisation (batch statistics) -> ReLU; two 1x1 heads give the level's
  operator and solution-operator encodings a = 1 + head, ainv = 1 + head
  (width of the MgNet level), so an untrained net gates by one.
* MgNet (Sec. 3.3): lift 1x1 (2M -> C_0); smoothing
  u <- u + (B_l * act(f - (A_l * u) o a_l)) o ainv_l with 3x3 convs A_l, B_l;
  act is the identity by default (Sec. 3.3 names convolutional smoothers
  and no activation; the operator they approximate is linear) or ReLU;
  restriction f_{l+1} = R_l * (f_l - (A_l * u_l) o a_l), 3x3 stride 2;
  prolongation u_l <- u_l + P_l *^T u_{l+1}, transposed 4x4 stride 2; one
  pre- and one post-smoothing step per level (two on the coarsest); width
  C_l = min(C_0 2^l, C_max); zero padding; no biases in MgNet, so the map is
  positively homogeneous.
* Output: psi_d = x + proj(u_0) (1x1, C_0 -> 2M) in face-flux space, the
  input of the map D of Eq. loss; with proj = 0 the network is the identity.
* Input scaling: x = r / rms(r), output rms(r) psi_d.
* Loss (Eq. loss, unfiltered): mean over the batch of ||x - A D psi_d|| / ||x||.
"""
from __future__ import annotations

import numpy as np

from . import tfps

BN_EPS = 1e-5


# --------------------------------------------------------------------------
# primitive operations (definitions)
# --------------------------------------------------------------------------
def conv2d(x, w, stride, pad):
    """out[b,o,y,x] = sum_{c,ky,kx} w[o,c,ky,kx] xp[b,c,s y + ky, s x + kx], xp zero-padded by pad."""
    B, C, H, Wd = x.shape
    O, _, k, _ = w.shape
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (Wd + 2 * pad - k) // stride + 1
    out = np.zeros((B, O, Ho, Wo))
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], patch)
    return out


def conv2d_T(x, w, stride, pad, out_hw):
    """Transposed convolution, w[c,o,ky,kx]: every input pixel (h, w) adds
    w[c,o,ky,kx] x[b,c,h,w] at output (s h + ky - pad, s w + kx - pad)."""
    B, C, H, Wd = x.shape
    _, O, k, _ = w.shape
    Hf = stride * (H - 1) + k
    Wf = stride * (Wd - 1) + k
    full = np.zeros((B, O, max(Hf, out_hw[0] + pad), max(Wf, out_hw[1] + pad)))
    for ky in range(k):
        for kx in range(k):
            full[:, :, ky:ky + stride * (H - 1) + 1:stride, kx:kx + stride * (Wd - 1) + 1:stride] += \
                np.einsum("co,bchw->bohw", w[:, :, ky, kx], x)
    return full[:, :, pad:pad + out_hw[0], pad:pad + out_hw[1]]


def conv2d_wgrad(x, dy, k, stride, pad):
    """dW[o,c,ky,kx] = sum_{b,y,x} dy[b,o,y,x] xp[b,c,s y + ky, s x + kx] (conv2d's weight gradient)."""
    B, C, H, Wd = x.shape
    _, O, Ho, Wo = dy.shape
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    dw = np.zeros((O, C, k, k))
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            dw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dy, patch)
    return dw


# --------------------------------------------------------------------------
# tape
# --------------------------------------------------------------------------
class Tape:
    """Records values and the backward rule of every primitive applied."""

    def __init__(self):
        self.vals = []
        self.rules = []          # (out_id, fn(grad_out) -> list of (id, grad))

    def leaf(self, value):
        self.vals.append(np.asarray(value, np.float64))
        self.rules.append(None)
        return len(self.vals) - 1

    def _out(self, value, rule):
        self.vals.append(value)
        self.rules.append(rule)
        return len(self.vals) - 1

    def v(self, i):
        return self.vals[i]

    # ---- primitives -------------------------------------------------------
    def conv(self, x, w, stride, pad):
        X, Wt = self.vals[x], self.vals[w]
        H, Wd = X.shape[2:]

        def rule(g):
            return [(x, conv2d_T(g, Wt, stride, pad, (H, Wd))),
                    (w, conv2d_wgrad(X, g, Wt.shape[2], stride, pad))]
        return self._out(conv2d(X, Wt, stride, pad), rule)

    def convT(self, x, w, stride, pad, out_hw):
        X, Wt = self.vals[x], self.vals[w]

        def rule(g):
            # adjoint of a transposed convolution is the plain convolution
            return [(x, conv2d(g, Wt, stride, pad)),
                    (w, conv2d_wgrad(g, X, Wt.shape[2], stride, pad))]
        return self._out(conv2d_T(X, Wt, stride, pad, out_hw), rule)

    def conv1x1(self, x, w):
        X, Wt = self.vals[x], self.vals[w]

        def rule(g):
            return [(x, np.einsum("oc,bohw->bchw", Wt, g)), (w, np.einsum("bohw,bchw->oc", g, X))]
        return self._out(np.einsum("oc,bchw->bohw", Wt, X), rule)

    def head(self, x, w, bias):
        """1 + conv1x1(x, w) + bias (per output channel)."""
        X, Wt, bv = self.vals[x], self.vals[w], self.vals[bias]

        def rule(g):
            return [(x, np.einsum("oc,bohw->bchw", Wt, g)), (w, np.einsum("bohw,bchw->oc", g, X)),
                    (bias, g.sum(axis=(0, 2, 3)))]
        return self._out(1.0 + np.einsum("oc,bchw->bohw", Wt, X) + bv[None, :, None, None], rule)

    def add(self, a, b):
        return self._out(self.vals[a] + self.vals[b], lambda g: [(a, g), (b, g)])

    def sub(self, a, b):
        return self._out(self.vals[a] - self.vals[b], lambda g: [(a, g), (b, -g)])

    def mul(self, a, b):
        A, Bv = self.vals[a], self.vals[b]
        return self._out(A * Bv, lambda g: [(a, g * Bv), (b, g * A)])

    def relu(self, a):
        A = self.vals[a]
        return self._out(np.maximum(A, 0.0), lambda g: [(a, g * (A > 0))])

    def bn(self, x, gamma, beta):
        """Batch normalisation over (batch, H, W) per channel, biased variance."""
        X, G, Bt = self.vals[x], self.vals[gamma], self.vals[beta]
        mu = X.mean(axis=(0, 2, 3), keepdims=True)
        var = X.var(axis=(0, 2, 3), keepdims=True)
        inv = 1.0 / np.sqrt(var + BN_EPS)
        xh = (X - mu) * inv
        cnt = X.shape[0] * X.shape[2] * X.shape[3]

        def rule(g):
            gg = g * G[None, :, None, None]
            dx = inv / cnt * (cnt * gg - gg.sum(axis=(0, 2, 3), keepdims=True)
                              - xh * (gg * xh).sum(axis=(0, 2, 3), keepdims=True))
            return [(x, dx), (gamma, (g * xh).sum(axis=(0, 2, 3))), (beta, g.sum(axis=(0, 2, 3)))]
        return self._out(G[None, :, None, None] * xh + Bt[None, :, None, None], rule)

    def backward(self, out, grad):
        grads = [None] * len(self.vals)
        grads[out] = grad
        for i in range(len(self.vals) - 1, -1, -1):
            if grads[i] is None or self.rules[i] is None:
                continue
            for j, gj in self.rules[i](grads[i]):
                grads[j] = gj if grads[j] is None else grads[j] + gj
        return grads


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def coeff_inputs(md):
    """CoeffNet input channels per cell (Sec. 3.2 reading): log sigma_T,
    log sigma_a, log eps, log tau with tau = sigma_T h / eps."""
    h = 1.0 / md.I
    eps = np.broadcast_to(np.asarray(md.eps, np.float64), md.sigma_T.shape)
    return np.stack([np.log(md.sigma_T), np.log(md.sigma_a), np.log(eps),
                     np.log(md.sigma_T * h / eps)]).reshape(4, md.I, md.I)


def forward(params, shape, coeff_x, x):
    """Network forward on a batch.

    coeff_x: (B, 4, I, I) CoeffNet inputs; x: (B, 2M, I, I) normalised network
    inputs (face-flux space).  Returns (tape, ids) where ids['psi'] is psi_d.
    """
    t = Tape()
    P = {k: t.leaf(v) for k, v in params.items()}
    L = shape.levels
    # CoeffNet
    g = t.leaf(coeff_x)
    a, ai = [], []
    for l in range(L):
        z = t.conv(g, P[f"coef{l}.w"], 1 if l == 0 else 2, 1)
        g = t.relu(t.bn(z, P[f"coef{l}.gamma"], P[f"coef{l}.beta"]))
        a.append(t.head(g, P[f"a{l}.w"], P[f"a{l}.b"]))
        ai.append(t.head(g, P[f"ainv{l}.w"], P[f"ainv{l}.b"]))
    # MgNet V-cycle
    xi = t.leaf(x)
    f = [None] * L
    u = [None] * L
    f[0] = t.conv1x1(xi, P["lift.w"])

    def smooth(l, ul):
        if ul is None:                          # u = 0: A * u vanishes
            tt = f[l]
        else:
            tt = t.sub(f[l], t.mul(t.conv(ul, P[f"A{l}.w"], 1, 1), a[l]))
        inner = t.relu(tt) if shape.act == "relu" else tt
        corr = t.mul(t.conv(inner, P[f"B{l}.w"], 1, 1), ai[l])
        return corr if ul is None else t.add(ul, corr)

    for l in range(L - 1):
        u[l] = smooth(l, None)
        res = t.sub(f[l], t.mul(t.conv(u[l], P[f"A{l}.w"], 1, 1), a[l]))
        f[l + 1] = t.conv(res, P[f"R{l}.w"], 2, 1)
    u[L - 1] = smooth(L - 1, smooth(L - 1, None))
    for l in range(L - 2, -1, -1):
        hw = t.v(f[l]).shape[2:]
        u[l] = t.add(u[l], t.convT(u[l + 1], P[f"P{l}.w"], 2, 1, hw))
        u[l] = smooth(l, u[l])
    psi = t.add(xi, t.conv1x1(u[0], P["proj.w"]))
    return t, {"params": P, "x": xi, "psi": psi, "coeff": g}


def apply_net(params, shape, coeff_x, r):
    """Preconditioner map in face-flux space: z = rms(r) Net(r / rms(r)) for one
    vector r of length 2M*I*I (direction-major = channel-major image)."""
    M, I = shape.M, int(np.sqrt(r.size // (2 * shape.M)))
    s = np.sqrt(np.mean(r * r))
    if s == 0.0:
        return np.zeros_like(r)
    x = (r / s).reshape(1, 2 * M, I, I)
    t, ids = forward(params, shape, coeff_x[None], x)
    return s * t.v(ids["psi"]).ravel()


def B_apply(p, D, v):
    """A D v (block-Jacobi preconditioned operator) through the TFPS oracle."""
    return p.apply(tfps.block_apply(D, v.reshape(2 * p.M, -1))).ravel()


def B_adjoint(p, D, v):
    """(A D)^T v = D^T A^T v."""
    return tfps.block_apply_T(D, p.apply_adjoint(v.reshape(2 * p.M, -1))).ravel()


def loss_and_grad(params, shape, problems, Ds, coeff_xs, rs):
    """Eq. loss (unfiltered), batch mean of ||x - A D psi_d|| / ||x||, x = r/rms(r),
    and its gradient with respect to every parameter."""
    Bn = len(rs)
    M = shape.M
    xs = []
    for r in rs:
        s = np.sqrt(np.mean(r * r))
        xs.append(r / s)
    I = problems[0].I
    X = np.stack([x.reshape(2 * M, I, I) for x in xs])
    t, ids = forward(params, shape, np.stack(coeff_xs), X)
    psi = t.v(ids["psi"])
    total = 0.0
    gpsi = np.zeros_like(psi)
    for b in range(Bn):
        res = xs[b] - B_apply(problems[b], Ds[b], psi[b].ravel())
        nr, nx = np.linalg.norm(res), np.linalg.norm(xs[b])
        total += nr / nx / Bn
        gpsi[b] = (-B_adjoint(problems[b], Ds[b], res) / (nr * nx * Bn)).reshape(2 * M, I, I)
    grads = t.backward(ids["psi"], gpsi)
    P = ids["params"]
    return total, {k: grads[i] if grads[i] is not None else np.zeros_like(params[k])
                   for k, i in P.items()}


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every parameter; state holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    tstep = state["t"]
    for k in params:
        m = state.setdefault("m", {}).setdefault(k, np.zeros_like(params[k]))
        v = state.setdefault("v", {}).setdefault(k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** tstep)
        vh = v / (1 - beta2 ** tstep)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def cosine_lr(lr0, step, total):
    """Cosine annealing of the learning rate (Sec. 4.1)."""
    return 0.5 * lr0 * (1.0 + np.cos(np.pi * min(step, total) / total))
