"""Pins of the MgNet/CoeffNet oracle: convolutions against scipy, the
transposed-convolution adjoint identity (P11), finite-difference gradients
(P16), the identity-network special case and Adam's first step."""
import numpy as np
import pytest
from scipy import signal

from oracle import mgnet, tfps
from paper_2604_23265_gb300 import workloads as W


def test_conv2d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 9, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    for stride in (1, 2):
        out = mgnet.conv2d(x, w, stride, 1)
        for b in range(2):
            for o in range(4):
                ref = sum(signal.correlate2d(np.pad(x[b, c], 1), w[o, c], mode="valid") for c in range(3))
                np.testing.assert_allclose(out[b, o], ref[::stride, ::stride], atol=1e-12)


@pytest.mark.parametrize("k,s,p,H", [(3, 1, 1, 8), (3, 2, 1, 8), (4, 2, 1, 4)])
def test_P11_transposed_conv_is_adjoint(k, s, p, H):
    rng = np.random.default_rng(1)
    if (k, s) == (4, 2):        # prolongation: coarse H -> fine 2H
        x = rng.standard_normal((2, 3, 2 * H, 2 * H))
    else:
        x = rng.standard_normal((2, 3, H, H))
    w = rng.standard_normal((5, 3, k, k))
    y = mgnet.conv2d(x, w, s, p)
    z = rng.standard_normal(y.shape)
    lhs = np.sum(y * z)
    rhs = np.sum(x * mgnet.conv2d_T(z, w, s, p, x.shape[2:]))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _small(levels=2, batch=2, seed=0, proj=0.3, act="linear"):
    shape = W.NetShape(M=4, levels=levels, c0=4, cmax=8, cc=4, ccmax=8, act=act)
    params = W.init_params(shape, seed=seed, proj_scale=proj)
    meds = [W.polynomial_diffusion(s, I=8, M=4) for s in range(batch)]
    probs = [tfps.Problem(m.I, m.M, m.sigma_T, m.sigma_a, m.q, m.eps, m.g, m.inflow) for m in meds]
    Ds = [p.block_inverse() for p in probs]
    cx = [mgnet.coeff_inputs(m) for m in meds]
    rs = [W.random_vector(m.n, 100 + s) for s, m in enumerate(meds)]
    return shape, params, probs, Ds, cx, rs


@pytest.mark.parametrize("levels,act", [(1, "linear"), (2, "linear"), (3, "linear"), (2, "relu"),
                                        (3, "relu")])
def test_P16_gradients_match_finite_differences(levels, act):
    shape, params, probs, Ds, cx, rs = _small(levels=levels, act=act)
    loss, grads = mgnet.loss_and_grad(params, shape, probs, Ds, cx, rs)
    rng = np.random.default_rng(5)
    for trial in range(3):
        d = {k: rng.standard_normal(v.shape) for k, v in params.items()}
        h = 1e-7
        lp = mgnet.loss_and_grad({k: v + h * d[k] for k, v in params.items()}, shape, probs, Ds, cx, rs)[0]
        lm = mgnet.loss_and_grad({k: v - h * d[k] for k, v in params.items()}, shape, probs, Ds, cx, rs)[0]
        fd = (lp - lm) / (2 * h)
        an = sum(np.sum(grads[k] * d[k]) for k in params)
        assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-3), (fd, an)


def test_every_parameter_gets_a_gradient():
    shape, params, probs, Ds, cx, rs = _small(levels=3)
    _, grads = mgnet.loss_and_grad(params, shape, probs, Ds, cx, rs)
    for k, g in grads.items():
        assert g.shape == params[k].shape
        assert np.abs(g).max() > 0, k


def test_identity_network_is_block_jacobi():
    """proj = 0: psi_d = x, so z = r and the loss is ||r - A D r|| / ||r||."""
    shape, params, probs, Ds, cx, rs = _small(proj=0.0)
    z = mgnet.apply_net(params, shape, cx[0], rs[0])
    np.testing.assert_allclose(z, rs[0], rtol=1e-15)
    loss, _ = mgnet.loss_and_grad(params, shape, probs[:1], Ds[:1], cx[:1], rs[:1])
    ref = np.linalg.norm(rs[0] - mgnet.B_apply(probs[0], Ds[0], rs[0])) / np.linalg.norm(rs[0])
    assert abs(loss - ref) <= 1e-13


def test_network_is_positively_homogeneous():
    shape, params, probs, Ds, cx, rs = _small(proj=0.5)
    z1 = mgnet.apply_net(params, shape, cx[0], rs[0])
    z2 = mgnet.apply_net(params, shape, cx[0], 3.5 * rs[0])
    np.testing.assert_allclose(z2, 3.5 * z1, rtol=0, atol=1e-12 * np.abs(z2).max())


def test_batchnorm_normalises():
    t = mgnet.Tape()
    rng = np.random.default_rng(2)
    x = t.leaf(rng.standard_normal((3, 5, 4, 4)) * 7 + 2)
    y = t.v(t.bn(x, t.leaf(np.ones(5)), t.leaf(np.zeros(5))))
    np.testing.assert_allclose(y.mean(axis=(0, 2, 3)), 0, atol=1e-12)
    np.testing.assert_allclose(y.var(axis=(0, 2, 3)), 1, rtol=1e-6)


def test_adam_first_step_moves_by_lr_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    mgnet.adam_step(p, g, {}, lr=0.01)
    np.testing.assert_allclose(p["w"], [0.99, -1.99, 2.99], atol=1e-7)


def test_adam_constant_gradient_moves_by_lr_every_step():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each of
    five steps moves a parameter by lr g / (|g| + eps).  A wrong power of
    either beta in the bias corrections breaks this from step 2 on."""
    g0 = np.array([0.5, -4.0, 2e-3, 7.0])
    p = {"w": np.zeros(4)}
    st = {}
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        mgnet.adam_step(p, {"w": g0.copy()}, st, lr=lr)
        np.testing.assert_allclose(p["w"], -t * lr * g0 / (np.abs(g0) + eps), rtol=1e-12, atol=0)
        np.testing.assert_allclose(st["m"]["w"], (1 - 0.9 ** t) * g0, rtol=1e-13)
        np.testing.assert_allclose(st["v"]["w"], (1 - 0.999 ** t) * g0 ** 2, rtol=1e-13)


def test_adam_alternating_gradient_closed_form():
    """Gradient (-1)^(t+1) g: the geometric sums give
    m_t = (1 - b1) g (-1)^(t+1) (1 - (-b1)^t) / (1 + b1) and v_t = (1 - b2^t) g^2,
    so the step at t is lr (-1)^(t+1) g c_t / (|g| + eps) with
    c_t = (1 - b1)(1 - (-b1)^t) / ((1 + b1)(1 - b1^t)): c_1 = 1, c_2 = 1/19.
    Pins the relative weighting of old and new gradients in m (a swapped b1
    and 1 - b1 gives c_2 = 0.81/0.19 instead) and the bias correction of v."""
    b1 = 0.9
    g0 = np.array([3.0, -0.25])
    p = {"w": np.zeros(2)}
    st = {}
    lr = 0.1
    expect = np.zeros(2)
    for t in range(1, 6):
        sgn = (-1.0) ** (t + 1)
        mgnet.adam_step(p, {"w": sgn * g0}, st, lr=lr)
        c = (1 - b1) * (1 - (-b1) ** t) / ((1 + b1) * (1 - b1 ** t))
        expect = expect - lr * sgn * g0 * c / (np.abs(g0) + 1e-8)
        np.testing.assert_allclose(p["w"], expect, rtol=1e-12, atol=1e-16)
    assert abs((1 - b1) * (1 - b1 ** 2) / ((1 + b1) * (1 - b1 ** 2)) - 1 / 19) < 1e-15


def test_cosine_schedule_endpoints():
    assert mgnet.cosine_lr(1e-3, 0, 100) == 1e-3
    assert abs(mgnet.cosine_lr(1e-3, 100, 100)) < 1e-18
    assert abs(mgnet.cosine_lr(1e-3, 50, 100) - 5e-4) < 1e-15
