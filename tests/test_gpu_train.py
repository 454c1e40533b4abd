"""The learned preconditioner trained on the GPU by the library's own kernels
beats the method without it: on an unseen diffusive medium (32x32 cells,
M = 8, eps = 1e-3) MgNet-FGMRES needs far fewer iterations than block-Jacobi
GMRES, and the solution still matches the oracle's dense LU solution."""
import numpy as np
import pytest

from oracle import krylov, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_trained_mgnet_beats_block_jacobi(lib):
    from paper_2604_23265_gb300 import rte, train
    media = [W.grf_diffusive(s, I=32, M=8, eps=1e-3) for s in range(1, 9)]
    net, ctxs, losses, secs = train.train_for(media, steps=600, batch=8, lr0=3e-3, seed=0)
    assert np.mean(losses[-50:]) < 0.6 * np.mean(losses[:20])
    test = W.grf_diffusive(1000, I=32, M=8, eps=1e-3)
    ctx = rte.Context.from_medium(test)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    bj = ctx.solve(x, tol=1e-8, restart=50)
    x.zero_()
    mg = ctx.solve(x, pc=net, tol=1e-8, restart=50)
    assert bj["converged"] and mg["converged"] and not mg["fell_back"], (bj, mg)
    assert mg["iterations"] * 4 <= bj["iterations"], (bj["iterations"], mg["iterations"])
    p = tfps.Problem(test.I, test.M, test.sigma_T, test.sigma_a, test.q, test.eps, test.g, test.inflow)
    b = p.rhs().ravel()
    r = b - p.apply(x.cpu().numpy().reshape(2 * test.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-8



def test_checkpoint_resumes_training(lib, tmp_path):
    """A 40-step run saved with its Adam state after 20 steps and resumed from
    the file at step 20 ends where the uninterrupted run ends (up to the
    rounding of the atomic weight-gradient sums); resuming from the weights
    alone (the Adam state reset) does not."""
    from paper_2604_23265_gb300 import rte, train
    media = [W.grf_diffusive(s, I=16, M=8, eps=1e-2) for s in range(1, 3)]
    shape = W.NetShape(M=8, levels=3, c0=8, cmax=16, cc=4, ccmax=8)
    ctxs = [rte.Context.from_medium(md) for md in media]
    inputs = [train.training_inputs(c, md, 8, 8, 5 + i) for i, (c, md) in enumerate(zip(ctxs, media))]
    kw = dict(steps=40, batch=4, lr0=3e-3, seed=9)

    def fresh():
        n = rte.MgNet(shape)
        n.set_params(W.init_params(shape, seed=4, proj_scale=0.0, vcycle_scale=0.5))
        return n

    a = fresh()
    train.train(a, ctxs, inputs, **kw)
    c = fresh()
    train.train(c, ctxs, inputs, checkpoint=lambda it, n, ls: n.save(tmp_path / "ck.bin") if it == 20 else None,
                every=20, **kw)
    d = fresh()
    d.load(tmp_path / "ck.bin")
    train.train(d, ctxs, inputs, start_step=20, **kw)
    p0, pa, pd = fresh().get_params(), a.get_params(), d.get_params()
    assert np.linalg.norm(pd - pa) <= 1e-3 * np.linalg.norm(pa - p0)
    e = fresh()
    e.load(tmp_path / "ck.bin")
    e.set_params(e.get_params())                  # same weights, Adam state reset
    train.train(e, ctxs, inputs, start_step=20, **kw)
    assert np.linalg.norm(e.get_params() - pa) > 10 * np.linalg.norm(pd - pa)
    for ctx in ctxs:
        ctx.close()
