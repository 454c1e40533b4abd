"""Grouped solves (rte_solve_group): several solves in lockstep with their
Arnoldi steps in shared launches give, solve by solve, the bits of the lone
solve -- same iterations, same solution -- for mixed grids, direction counts,
eps and g, with and without a network, and when some solves end early."""
import numpy as np
import pytest

from oracle import krylov, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mixed(count, seed=0, grids=(8, 12, 16, 24), dirs=(4, 8, 16)):
    return [W.mixed_instance(seed * 100 + i, grids=grids, dirs=dirs, eps_range=(1e-2, 1.0), g_range=(0.0, 0.8))
            for i in range(count)]


def _lone(rte, md, pc=None, **kw):
    ctx = rte.Context.from_medium(md)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, pc=pc, raise_on_error=False, **kw)
    return ctx, x, info


@pytest.mark.parametrize("count,inner", [(1, "f32"), (6, "f32"), (9, "f64")])
def test_group_is_bit_identical_to_lone_solves(lib, count, inner):
    from paper_2604_23265_gb300 import rte
    prec = rte.RTE_F32 if inner == "f32" else rte.RTE_F64
    media = _mixed(count, seed=count)
    lone = [_lone(rte, md, tol=1e-10, restart=20, inner_precision=prec) for md in media]
    ctxs = [rte.Context.from_medium(md) for md in media]
    xs = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = rte.solve_group(ctxs, xs, tol=1e-10, restart=20, inner_precision=prec)
    for (c1, x1, i1), x2, i2 in zip(lone, xs, infos):
        assert i2["status"] == "OK" and i2["converged"], i2
        assert i2["iterations"] == i1["iterations"] and i2["cycles"] == i1["cycles"]
        assert torch.equal(x1, x2)
    # and the solution is the oracle's (dense LU) on the smallest instance:
    # residual by the oracle's operator, and the angular flux at the cell centres
    # (the coefficients themselves cancel heavily, so psi is compared, to
    # cond(A) times the 1e-10 residual)
    i = int(np.argmin([md.I * md.M for md in media]))
    md = media[i]
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    xl = krylov.dense_solve(p.assemble(), p.rhs().ravel())
    r = p.rhs().ravel() - p.apply(xs[i].cpu().numpy().reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(p.rhs()) <= 1e-10
    psi = p.reconstruct(xs[i].cpu().numpy().reshape(2 * md.M, -1)).ravel()
    psil = p.reconstruct(xl.reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(psi - psil) <= 1e-5 * np.linalg.norm(psil)


def test_group_with_networks_and_early_endings(lib):
    """Three solves with one network and grid size (their V-cycles run as one
    batch of tensor-core layers), one with max_iter reached, one with a zero
    right-hand side, the rest block Jacobi: each equals its lone solve."""
    from paper_2604_23265_gb300 import rte
    media = _mixed(5, seed=7, grids=(16,), dirs=(8,))
    zero = W.mixed_instance(999, grids=(8,), dirs=(8,))
    zero.q = np.zeros_like(zero.q)
    zero.inflow = W.zero_inflow(zero.I, zero.M)
    media.append(zero)
    shape = W.NetShape(M=8, levels=2, c0=8, cmax=16, cc=4, ccmax=8)
    net = rte.MgNet(shape)
    net.set_params(W.init_params(shape, seed=1, proj_scale=0.02, vcycle_scale=0.5))
    pcs = [net, net, net, None, None, None]
    kws = dict(tol=1e-9, restart=15, max_iter=60)
    lone = [_lone(rte, md, pc=pc, **kws) for md, pc in zip(media, pcs)]
    ctxs = [rte.Context.from_medium(md) for md in media]
    xs = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = rte.solve_group(ctxs, xs, pcs=pcs, **kws)
    statuses = set()
    for (c1, x1, i1), x2, i2 in zip(lone, xs, infos):
        assert i2["iterations"] == i1["iterations"] and i2["fell_back"] == i1["fell_back"], (i1, i2)
        assert torch.equal(x1, x2)
        statuses.add(i2["status"])
    assert infos[-1]["converged"] and infos[-1]["iterations"] == 0      # zero right-hand side
    assert "ENOTCONV" in statuses or all(i["converged"] for i in infos)


def test_group_rejects_shared_contexts_and_mixed_streams(lib):
    from paper_2604_23265_gb300 import rte
    md = _mixed(1)[0]
    c = rte.Context.from_medium(md)
    x = torch.zeros(c.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rte.RteError):
        rte.solve_group([c, c], [x, x])
    s = torch.cuda.Stream()
    c2 = rte.Context.from_medium(md, stream=s)
    x2 = torch.zeros(c2.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rte.RteError):
        rte.solve_group([c, c2], [x, x2])
