"""GPU parity of the ATFPS loss filter (Sec. 2.3, Eq. loss_delta) against the
FP64 oracle on the same seeded media: the selection, F y and F^T r element by
element, and the filtered loss with every parameter's gradient.  The media
have two materials with a spread of optical thickness, so part of the basis
is dropped and the interface bases mix kept and dropped functions."""
import numpy as np
import pytest

from oracle import atfps as OA, mgnet as OM, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _medium(I, M, seed, eps=0.05):
    rng = np.random.default_rng(seed)
    N = I * I
    sT = W.checkerboard_sigma_T(I, 3, (0.5, 20.0), seed)
    sa = np.where(sT > 1, 0.3, 0.1)
    return W.Medium(I, M, sT, sa, rng.uniform(0, 1, N), np.full(N, eps), 0.4, W.random_inflow(I, M, seed + 1))


def _pair(md):
    from paper_2604_23265_gb300 import rte
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    return p, rte.Context.from_medium(md)


CASES = [(7, 8, 0, 1e-2), (12, 16, 1, 1e-1), (9, 4, 2, 1e-3), (10, 8, 3, 0.0)]


@pytest.mark.parametrize("I,M,seed,delta", CASES)
def test_selection_and_filter_match_oracle(lib, I, M, seed, delta):
    md = _medium(I, M, seed)
    p, ctx = _pair(md)
    F, mask = OA.filter_operator(p, delta)
    rows = ctx.atfps_setup(delta)
    np.testing.assert_array_equal(ctx.atfps_mask(), mask.astype(np.uint8))
    assert rows == F.shape[0]
    if 0 < delta:
        assert 0 < mask.mean() < 1          # some functions dropped, some kept
    rng = np.random.default_rng(seed + 50)
    y = rng.standard_normal(ctx.n)
    out = torch.zeros(max(rows, 1), dtype=torch.float64, device="cuda")
    ctx.atfps_apply(torch.tensor(y, device="cuda"), out)
    ref = F @ y
    assert _rel(out.cpu().numpy()[:rows], ref) <= 1e-9
    r = rng.standard_normal(rows)
    back = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.atfps_apply_t(torch.tensor(r, device="cuda"), back)
    assert _rel(back.cpu().numpy(), F.T @ r) <= 1e-9


def test_transport_regime_keeps_everything(lib):
    """Pin P12 on the device: with eps = 1 and thin cells nothing is dropped at
    delta = 1e-2, so every interface keeps all its coordinates."""
    md = W.checkerboard_transport(seed=0, I=8, M=8)
    p, ctx = _pair(md)
    rows = ctx.atfps_setup(1e-2)
    assert ctx.atfps_mask().all()
    assert rows == ctx.n


@pytest.mark.parametrize("levels,batch,delta", [(2, 2, 1e-2), (1, 1, 1e-1)])
def test_filtered_loss_and_gradients_match_oracle(lib, levels, batch, delta):
    from paper_2604_23265_gb300 import rte
    I, M = 12, 8
    md = _medium(I, M, 7)
    p, ctx = _pair(md)
    ctx.atfps_setup(delta)
    shape = W.NetShape(M=M, levels=levels, c0=8, cmax=16, cc=4, ccmax=8)
    params = W.init_params(shape, seed=3, proj_scale=0.3)
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    net = rte.MgNet(shape)
    net.set_params(params)
    net.loss = rte.MgNet.FILTERED
    rs = [W.random_vector(ctx.n, 20 + b) for b in range(batch)]
    loss, g = net.loss_grad(ctx, [torch.tensor(r, device="cuda") for r in rs])
    D = p.block_inverse()
    F, mask = OA.filter_operator(p, delta)
    cx = OM.coeff_inputs(md)
    lref, gref = OA.loss_and_grad_filtered(params, shape, [p] * batch, [D] * batch, [F] * batch,
                                           [mask] * batch, [cx] * batch, rs)
    assert abs(loss - lref) <= 1e-5 * lref
    G = rte.MgNet.unflatten(g, shape)
    for k in gref:
        scale = max(np.linalg.norm(gref[k]), 1e-3 * max(np.linalg.norm(v) for v in gref.values()))
        err = np.linalg.norm(G[k] - gref[k]) / scale
        assert err <= 1e-3, (k, err)


def test_filtered_training_reduces_loss_and_needs_a_filter(lib):
    from paper_2604_23265_gb300 import rte
    md = _medium(16, 8, 9)
    p, ctx = _pair(md)
    shape = W.NetShape(M=8, levels=3, c0=8, cmax=16, cc=4, ccmax=8)
    net = rte.MgNet(shape)
    net.set_params(W.init_params(shape, seed=0, proj_scale=0.0, vcycle_scale=0.5))
    net.loss = rte.MgNet.FILTERED
    rs = [torch.tensor(W.random_vector(ctx.n, 40 + b), device="cuda") for b in range(4)]
    with pytest.raises(rte.RteError):
        net.train_step(ctx, rs, 3e-3)             # no filter on the context yet
    ctx.atfps_setup(1e-2)
    first = net.train_step(ctx, rs, 3e-3)
    for _ in range(60):
        last = net.train_step(ctx, rs, 3e-3)
    assert last < 0.9 * first
    with pytest.raises(rte.RteError):
        net.loss = 5
