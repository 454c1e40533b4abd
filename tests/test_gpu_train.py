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
