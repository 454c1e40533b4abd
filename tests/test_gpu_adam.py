"""GPU parity of the optimizer and of whole training steps against the oracle
(Sec. 4.1: Adam, learning rate 1e-3 with cosine annealing).

* The device Adam kernel, driven for five steps by the device's own
  gradients (read back before each step), against ``oracle.mgnet.adam_step``
  driven by the same gradients: every parameter and both moments, element by
  element.  The bar is FP32 rounding: per step a few roundings of the moments
  and of the update (at most 1e-5 of lr per element) and one rounding of the
  parameter (2^-24 |p|).
* Five training steps on the device against five oracle training steps
  (oracle gradients, oracle Adam) from the same weights: the loss trajectory
  to 1e-4 relative, and each tensor's total update in direction.
* A training run is bit-reproducible: the weight-gradient and loss
  reductions add in a fixed order.
"""
import struct

import numpy as np
import pytest

from oracle import mgnet as OM, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


def _setup(seed=0, I=16, M=8, levels=3):
    from paper_2604_23265_gb300 import rte
    shape = W.NetShape(M=M, levels=levels, c0=8, cmax=16, cc=4, ccmax=8)
    params = W.init_params(shape, seed=seed, proj_scale=0.3, vcycle_scale=0.5)
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    md = W.grf_diffusive(seed + 3, I=I, M=M, eps=1e-2)
    ctx = rte.Context.from_medium(md)
    net = rte.MgNet(shape)
    net.set_params(params)
    rs = [W.random_vector(ctx.n, 50 + b) for b in range(3)]
    return rte, shape, params, md, ctx, net, rs


def _read_checkpoint(path, count):
    """Weights, first and second Adam moments and the step of a MGNET003 file."""
    raw = open(path, "rb").read()
    assert raw[:8] == b"MGNET003"
    off = 8 + 7 * 4
    cnt, step = struct.unpack_from("<qq", raw, off)
    assert cnt == count
    off += 16
    arr = np.frombuffer(raw, dtype=np.float32, count=3 * count, offset=off)
    return arr[:count].astype(np.float64), arr[count:2 * count].astype(np.float64), \
        arr[2 * count:].astype(np.float64), step


def test_adam_kernel_matches_oracle_over_five_steps(lib, tmp_path):
    rte, shape, params, md, ctx, net, rs = _setup()
    rt = [torch.tensor(r, device="cuda") for r in rs]
    p0 = net.get_params().astype(np.float64)
    flat = {"w": p0.copy()}
    state = {}
    lr0, total = 1e-3, 20
    grads = []
    for t in range(5):
        lr = OM.cosine_lr(lr0, t, total)
        _, g = net.loss_grad(ctx, rt)
        grads.append(g.astype(np.float64))
        net.train_step(ctx, rt, lr)
        OM.adam_step(flat, {"w": grads[-1]}, state, lr=lr)
        T = t + 1
        net.save(tmp_path / "ck.bin")
        p, m, v, step = _read_checkpoint(tmp_path / "ck.bin", net.count)
        assert step == T
        gmax = np.max(np.abs(np.stack(grads)), axis=0)
        # moments: a few FP32 roundings per step (the FP32 constants 0.9f, 0.1f,
        # 0.999f, 0.001f are within 4 ulp of 0.9, 0.1, 0.999, 0.001; m is
        # bounded by the largest gradient seen)
        np.testing.assert_array_less(np.abs(m - state["m"]["w"]), 16 * T * U32 * gmax + 1e-30)
        np.testing.assert_array_less(np.abs(v - state["v"]["w"]), 16 * T * U32 * state["v"]["w"] + 1e-30)
        # parameters: one rounding of p and at most 1e-5 lr of the update per step
        bar = T * (2 * U32 * np.abs(flat["w"]) + 1e-5 * lr0)
        np.testing.assert_array_less(np.abs(p - flat["w"]), bar + 1e-30)
    np.testing.assert_array_equal(net.get_params().astype(np.float64), p)
    ctx.close()
    net.close()


def test_training_steps_follow_oracle_training(lib):
    rte, shape, params, md, ctx, net, rs = _setup(seed=1)
    rt = [torch.tensor(r, device="cuda") for r in rs]
    prob = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    D = prob.block_inverse()
    cx = OM.coeff_inputs(md)
    po = {k: v.copy() for k, v in params.items()}
    state = {}
    lr0, total = 1e-3, 10
    for t in range(5):
        lr = OM.cosine_lr(lr0, t, total)
        lg = net.train_step(ctx, rt, lr)
        lo, go = OM.loss_and_grad(po, shape, [prob] * 3, [D] * 3, [cx] * 3, rs)
        OM.adam_step(po, go, state, lr=lr)
        assert abs(lg - lo) <= 1e-4 * lo, (t, lg, lo)
    got = rte.MgNet.unflatten(net.get_params(), shape)
    for k in params:
        dg = got[k] - params[k]
        do = po[k] - params[k]
        if np.linalg.norm(do) == 0:
            continue
        cos = float(np.dot(dg.ravel(), do.ravel()) / (np.linalg.norm(dg) * np.linalg.norm(do)))
        assert cos >= 0.999, (k, cos)
    ctx.close()
    net.close()


def test_training_is_bit_reproducible(lib):
    runs = []
    for _ in range(2):
        rte, shape, params, md, ctx, net, rs = _setup(seed=2, I=32, M=8, levels=4)
        rt = [torch.tensor(r, device="cuda") for r in rs]
        losses = [net.train_step(ctx, rt, 2e-3) for _ in range(4)]
        _, g = net.loss_grad(ctx, rt)
        runs.append((losses, net.get_params(), g))
        ctx.close()
        net.close()
    assert runs[0][0] == runs[1][0]
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])
