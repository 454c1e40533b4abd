"""Parity at the full sizes of the workloads, in the configuration the
benchmark runs them, on properties the FP64 oracle can check at that size:

* network train + apply shape (128 x 128 cells, M = 32, 4 levels, 64 channels
  doubling per level to 512, BF16 tensor cores): the forward against the
  oracle, and the FP32 training loss and every gradient against the oracle;
* benchmark solve (256 x 256, M = 64, eps = 1e-3, MgNet-FGMRES(50)): the true
  relative residual of the returned solution, recomputed by the oracle's FP64
  operator, meets 1e-8;
* grouped mixed-size solves (grids up to 256 x 256, M in {16, 32}, eps down to
  1e-4, per-M networks): every solve equals its lone solve bit for bit, and the
  reported residual is the oracle's;
* the largest serving request (512 x 512, M = 64): served in the mix it equals
  the lone solve bit for bit, and its reported residual is the oracle's.
"""
import numpy as np
import pytest

from oracle import mgnet as OM, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _problem(md):
    return tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)


def _oracle_relres(md, x, ctx):
    """True relative residual ||b - A x|| / ||b|| by the oracle's FP64 operator
    assembled on the context's own exported eigenbasis (the system the device
    solved; the basis itself is checked against the oracle's eigen-solver in
    the full-size apply test), and the rounding bar of its comparison with the
    device's FP64 value: 1e-12 of ||A x|| / ||b||, the apply's parity bar."""
    p = _problem(md)
    xi, L, mat = ctx.export_basis()
    np.testing.assert_array_equal(mat, p.mat_id)
    p.use_basis(xi, L)
    b = p.rhs().ravel()
    ax = p.apply(x.reshape(2 * md.M, -1)).ravel()
    bar = 1e-12 * np.linalg.norm(ax) / np.linalg.norm(b)
    return np.linalg.norm(b - ax) / np.linalg.norm(b), bar


def test_network_shape_at_full_size_matches_oracle(lib):
    from paper_2604_23265_gb300 import rte
    md = W.training_medium(seed=3, I=128, M=32)
    shape = W.NetShape(M=32, levels=4, c0=64, cmax=512, cc=8, ccmax=32)
    params = W.init_params(shape, seed=1, proj_scale=0.1, vcycle_scale=0.5)
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    ctx = rte.Context.from_medium(md)
    net = rte.MgNet(shape)
    net.set_params(params)
    r = W.random_vector(ctx.n, 11)
    z = torch.zeros(ctx.n, dtype=torch.float32, device="cuda")
    net.precond(ctx, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert rte.MgNet.kernel_status() == 0
    ref = OM.apply_net(params, shape, OM.coeff_inputs(md), r)
    zc = z.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(zc))
    assert _rel(zc - r, ref - r) <= 2e-2
    # training arithmetic (FP32) at this size: loss and gradients
    p = _problem(md)
    loss, g = net.loss_grad(ctx, [torch.tensor(r, device="cuda")])
    lref, gref = OM.loss_and_grad(params, shape, [p], [p.block_inverse()], [OM.coeff_inputs(md)], [r])
    assert abs(loss - lref) <= 1e-5 * lref
    G = rte.MgNet.unflatten(g, shape)
    big = max(np.linalg.norm(v) for v in gref.values())
    for k in gref:
        scale = max(np.linalg.norm(gref[k]), 1e-3 * big)
        err = np.linalg.norm(G[k] - gref[k]) / scale
        assert err <= 1e-3, (k, err)
    ctx.close()
    net.close()


def test_benchmark_solve_residual_by_oracle(lib):
    from paper_2604_23265_gb300 import rte, train
    media = [W.grf_diffusive(seed=101 + i, I=256, M=64) for i in range(2)]
    net, tctx, _, _ = train.train_for(media, shape=train.default_shape(64, 256), steps=150, batch=8)
    for c in tctx:
        c.close()
    md = W.grf_diffusive(seed=0, I=256, M=64)
    ctx = rte.Context.from_medium(md)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, pc=net, tol=1e-8, restart=50)
    assert info["converged"], info
    rel, bar = _oracle_relres(md, x.cpu().numpy(), ctx)
    assert abs(rel - info["relres"]) <= bar
    assert rel <= 1e-8
    ctx.close()
    net.close()


def _net(rte, M, seed):
    from paper_2604_23265_gb300 import train
    shape = train.default_shape(M, 256)
    net = rte.MgNet(shape)
    net.set_params(W.init_params(shape, seed=seed, proj_scale=0.02, vcycle_scale=0.5))
    return net


def test_grouped_mixed_sizes_at_full_size(lib):
    from paper_2604_23265_gb300 import rte
    nets = {16: _net(rte, 16, 1), 32: _net(rte, 32, 2)}
    layout = [(256, 32), (128, 16), (64, 32), (128, 32), (64, 16), (256, 16)]
    media = [W.mixed_instance(700 + i, grids=(I,), dirs=(M,), eps_range=(1e-4, 1.0)) for i, (I, M) in
             enumerate(layout)]
    pcs = [nets[md.M] if i % 3 != 2 else None for i, md in enumerate(media)]
    kw = dict(tol=1e-8, restart=50, max_iter=120)
    ctxs = [rte.Context.from_medium(md) for md in media]
    lone = []
    for c, pc in zip(ctxs, pcs):
        x = torch.zeros(c.n, dtype=torch.float64, device="cuda")
        lone.append((x, c.solve(x, pc=pc, raise_on_error=False, **kw)))
    xs = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = rte.solve_group(ctxs, xs, pcs=pcs, **kw)
    for (x1, i1), x2, i2 in zip(lone, xs, infos):
        assert i2["status"] in ("OK", "ENOTCONV"), i2
        assert i2["iterations"] == i1["iterations"] and i2["fell_back"] == i1["fell_back"]
        assert torch.equal(x1, x2)
    k = 4                                   # 64 x 64, M = 16
    rel, bar = _oracle_relres(media[k], xs[k].cpu().numpy(), ctxs[k])
    assert abs(rel - infos[k]["relres"]) <= bar + 1e-12 * rel
    for c in ctxs:
        c.close()


def test_largest_serving_request(lib):
    from paper_2604_23265_gb300 import rte
    big = W.mixed_instance(77, grids=(512,), dirs=(64,), eps_range=(1e-3, 1e-3), g_range=(0.5, 0.5))
    small = [W.mixed_instance(78 + i, grids=(64,), dirs=(16,), eps_range=(1e-2, 1.0)) for i in range(2)]
    kw = dict(tol=1e-8, max_iter=40)
    srv = rte.Server(slots=3, max_device_bytes=200 << 30, grouped=True)
    ids = [srv.submit(md, **kw) for md in [small[0], big, small[1]]]
    got = [srv.wait(i) for i in ids]
    srv.close()
    res, psi = got[1]
    assert res["status"] in ("OK", "ENOTCONV"), res
    ctx = rte.Context.from_medium(big)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, raise_on_error=False, **kw)
    ref = torch.zeros(big.M * big.I * big.I, dtype=torch.float64, device="cuda")
    ctx.reconstruct(x, ref)
    torch.cuda.synchronize()
    assert res["iterations"] == info["iterations"]
    np.testing.assert_array_equal(psi, ref.cpu().numpy())
    rel, bar = _oracle_relres(big, x.cpu().numpy(), ctx)
    ctx.close()
    assert abs(rel - info["relres"]) <= bar + 1e-12 * rel
