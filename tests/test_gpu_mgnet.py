"""GPU parity of the MgNet preconditioner against the FP64 oracle (same seeded
weights and inputs): forward, loss, every parameter's gradient, training and
the MgNet-preconditioned solve.  FP32 network arithmetic: relative L2 bars of
1e-4 (outputs) and 1e-3 (gradients: the bar the oracle's own gradients meet
against finite differences; FP32 sums over up to 65k products stay two orders
below it); the tensor-core forward (BF16 operands): 2e-2."""
import numpy as np
import pytest

from oracle import krylov, mgnet as OM, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _setup(I=16, M=8, levels=3, seed=0, proj=0.5, c0=8, cmax=16, cc=4, ccmax=8, act="linear"):
    from paper_2604_23265_gb300 import rte
    shape = W.NetShape(M=M, levels=levels, c0=c0, cmax=cmax, cc=cc, ccmax=ccmax, act=act)
    params = W.init_params(shape, seed=seed, proj_scale=proj)
    # round the weights to float32 so both sides use identical values
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    md = W.grf_diffusive(seed + 3, I=I, M=M, eps=1e-2)
    ctx = rte.Context.from_medium(md)
    net = rte.MgNet(shape)
    net.set_params(params)
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    return rte, shape, params, md, ctx, net, p


@pytest.mark.parametrize("I,M,levels", [(16, 8, 3), (24, 4, 2), (32, 16, 4), (8, 8, 1)])
def test_forward_matches_oracle(lib, I, M, levels):
    rte, shape, params, md, ctx, net, p = _setup(I=I, M=M, levels=levels)
    net.precision = rte.MgNet.FP32
    r = W.random_vector(ctx.n, 7)
    z = torch.zeros(ctx.n, dtype=torch.float32, device="cuda")
    net.precond(ctx, torch.tensor(r, device="cuda"), z)
    ref = OM.apply_net(params, shape, OM.coeff_inputs(md), r)
    assert _rel(z.cpu().numpy(), ref) <= 1e-4
    za = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    net.apply(ctx, torch.tensor(r, device="cuda"), za)
    refa = tfps.block_apply(p.block_inverse(), ref.reshape(2 * M, -1)).ravel()
    assert _rel(za.cpu().numpy(), refa) <= 1e-4 * np.linalg.cond(p.blocks()).max() ** 0.5 + 1e-4


# Tensor-core (BF16 operands, FP32 accumulation) forward against the FP64
# oracle under identical weights: relative L2 <= 2e-2 on the output and on the
# network's own part z - r (psi_d - x).  The shapes cover input channels that
# are not a multiple of 16 (2M = 8), output channels below 16 (c0 = 8), one to
# three pipeline stages, 128-pixel tiles with a ragged tail (24 x 24, 8 x 8
# coarse grids), 64-channel levels (72 KB of weights per CTA), and a 128-wide
# lift / projection (M = 64, 128 TMEM columns), the largest direction count
# (M = 80: 160-wide lift input and projection, 256 TMEM columns), ReLU
# smoothers, and layers whose weights are streamed per (tap, 64-channel block)
# stage: widths 64-256 (one slice), 64-512 (two slices of 256 output channels)
# and 40-320 (two slices of 160, channel blocks padded, ReLU on the gathers).
@pytest.mark.parametrize("I,M,levels,c0,cmax,act", [(16, 8, 3, 8, 16, "linear"), (24, 4, 2, 8, 16, "linear"),
                                                    (32, 16, 4, 16, 64, "linear"), (8, 8, 1, 8, 16, "linear"),
                                                    (64, 64, 4, 16, 64, "linear"), (40, 20, 2, 24, 48, "linear"),
                                                    (32, 8, 3, 16, 32, "relu"), (16, 80, 2, 16, 32, "linear"),
                                                    (16, 8, 3, 64, 256, "linear"), (16, 8, 4, 64, 512, "linear"),
                                                    (24, 8, 4, 40, 320, "relu")])
def test_tensor_core_forward_matches_oracle(lib, I, M, levels, c0, cmax, act):
    rte, shape, params, md, ctx, net, p = _setup(I=I, M=M, levels=levels, c0=c0, cmax=cmax,
                                                 cc=4, ccmax=8, act=act)
    assert net.precision == rte.MgNet.BF16
    r = W.random_vector(ctx.n, 7)
    z = torch.zeros(ctx.n, dtype=torch.float32, device="cuda")
    net.precond(ctx, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert rte.MgNet.kernel_status() == 0
    ref = OM.apply_net(params, shape, OM.coeff_inputs(md), r)
    zc = z.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(zc))
    assert _rel(zc, ref) <= 2e-2
    assert _rel(zc - r, ref - r) <= 2e-2
    # and against the FP32 CUDA-core path of the same network
    net.precision = rte.MgNet.FP32
    z32 = torch.zeros_like(z)
    net.precond(ctx, torch.tensor(r, device="cuda"), z32)
    assert _rel(zc - r, z32.cpu().numpy() - r) <= 2e-2


def test_tensor_core_repeated_applications_are_identical(lib):
    """The first application packs the weights; later ones chain the layers by
    programmatic dependent launch.  Every application gives the same bits."""
    rte, shape, params, md, ctx, net, p = _setup(I=32, M=8, levels=3, c0=16, cmax=32)
    r = torch.tensor(W.random_vector(ctx.n, 5), device="cuda")
    outs = []
    for k in range(4):
        z = torch.full((ctx.n,), float("nan"), dtype=torch.float32, device="cuda")
        net.precond(ctx, r, z)
        outs.append(z.cpu().numpy())
    assert rte.MgNet.kernel_status() == 0
    assert np.all(np.isfinite(outs[0]))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_tensor_core_forward_at_full_size_matches_fp32_path(lib):
    """At the benchmark size (256 x 256 cells, M = 64, 6 levels, widths 16-64)
    the tensor-core network agrees with the FP32 CUDA-core path (itself at
    parity with the oracle at small sizes) to the BF16 bar, on the network's
    own part z - r."""
    from paper_2604_23265_gb300 import rte, train
    md = W.grf_diffusive(seed=0, I=256, M=64)
    ctx = rte.Context.from_medium(md)
    shape = train.default_shape(md.M, md.I)
    net = rte.MgNet(shape)
    net.set_params(W.init_params(shape, seed=2, proj_scale=0.05, vcycle_scale=0.5))
    r = torch.tensor(W.random_vector(ctx.n, 3), device="cuda")
    z16 = torch.zeros(ctx.n, dtype=torch.float32, device="cuda")
    net.precond(ctx, r, z16)
    net.precision = rte.MgNet.FP32
    z32 = torch.zeros_like(z16)
    net.precond(ctx, r, z32)
    torch.cuda.synchronize()
    assert rte.MgNet.kernel_status() == 0
    rf = r.float()
    d16, d32 = (z16 - rf).double(), (z32 - rf).double()
    assert torch.isfinite(d16).all()
    assert (torch.linalg.norm(d16 - d32) / torch.linalg.norm(d32)).item() <= 2e-2
    ctx.close()


def test_precision_switch_rejects_unknown_value(lib):
    rte, shape, params, md, ctx, net, p = _setup(I=8, M=8, levels=1)
    with pytest.raises(rte.RteError):
        net.precision = 2
    assert net.precision == rte.MgNet.BF16


@pytest.mark.parametrize("levels,batch", [(1, 1), (2, 3), (3, 2)])
def test_loss_and_gradients_match_oracle(lib, levels, batch):
    rte, shape, params, md, ctx, net, p = _setup(I=16, M=8, levels=levels, proj=0.3)
    rs = [W.random_vector(ctx.n, 20 + b) for b in range(batch)]
    loss, g = net.loss_grad(ctx, [torch.tensor(r, device="cuda") for r in rs])
    D = p.block_inverse()
    cx = OM.coeff_inputs(md)
    lref, gref = OM.loss_and_grad(params, shape, [p] * batch, [D] * batch, [cx] * batch, rs)
    assert abs(loss - lref) <= 1e-5 * lref
    G = rte.MgNet.unflatten(g, shape)
    for k in gref:
        scale = max(np.linalg.norm(gref[k]), 1e-3 * max(np.linalg.norm(v) for v in gref.values()))
        err = np.linalg.norm(G[k] - gref[k]) / scale
        assert err <= 1e-3, (k, err)


def test_training_reduces_loss(lib):
    rte, shape, params, md, ctx, net, p = _setup(I=16, M=8, levels=3, proj=0.0)
    net.set_params(W.init_params(shape, seed=0, proj_scale=0.0, vcycle_scale=0.5))
    rs = [torch.tensor(W.random_vector(ctx.n, 40 + b), device="cuda") for b in range(4)]
    first = net.train_step(ctx, rs, 3e-3)
    for _ in range(100):
        last = net.train_step(ctx, rs, 3e-3)
    assert last < 0.8 * first


def test_mgnet_preconditioned_solve(lib):
    """With a zero projection the network is the identity, so MgNet-FGMRES takes
    exactly block Jacobi's iterations; the solution matches the oracle's dense
    LU solution."""
    rte, shape, params, md, ctx, net, p = _setup(I=16, M=8, levels=3, proj=0.0)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ref_info = ctx.solve(x, tol=1e-12, restart=40)
    x.zero_()
    info = ctx.solve(x, pc=net, tol=1e-12, restart=40, stall_ratio=10.0)
    assert info["converged"] and not info["fell_back"], info
    assert info["iterations"] == ref_info["iterations"]
    xl = krylov.dense_solve(p.assemble(), p.rhs().ravel())
    psi = torch.zeros(md.M * md.I * md.I, dtype=torch.float64, device="cuda")
    ctx.reconstruct(x, psi)
    ref = p.reconstruct(xl.reshape(2 * md.M, -1)).ravel()
    assert _rel(psi.cpu().numpy(), ref) <= 1e-6          # cond(A) x tol on this medium
    r = p.rhs().ravel() - p.apply(x.cpu().numpy().reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(p.rhs()) <= 2e-12


def test_tensor_core_network_solve_reaches_tolerance(lib):
    """A non-trivial network on the tensor cores preconditions a solve to a
    true FP64 relative residual of 1e-10 (flexible GMRES absorbs the BF16
    rounding of the preconditioner)."""
    rte, shape, params, md, ctx, net, p = _setup(I=32, M=8, levels=3, proj=0.05)
    net.set_params(W.init_params(shape, seed=1, proj_scale=0.05, vcycle_scale=0.5))
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, pc=net, tol=1e-10, restart=40, stall_ratio=10.0)
    assert info["converged"] and not info["fell_back"], info
    assert rte.MgNet.kernel_status() == 0
    r = p.rhs().ravel() - p.apply(x.cpu().numpy().reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(p.rhs()) <= 1e-10


def test_stalled_network_falls_back_to_block_jacobi(lib):
    """A network that does not help (large random projection) is replaced by
    block Jacobi after a cycle that reduces the true residual too little."""
    rte, shape, params, md, ctx, net, p = _setup(I=16, M=8, levels=3, proj=0.5)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, pc=net, tol=1e-10, restart=40, stall_ratio=0.9)
    assert info["converged"] and info["fell_back"], info


def test_save_load_roundtrip(lib, tmp_path):
    rte, shape, params, md, ctx, net, p = _setup()
    net.save(tmp_path / "w.bin")
    net2 = rte.MgNet(shape)
    net2.load(tmp_path / "w.bin")
    np.testing.assert_array_equal(net.get_params(), net2.get_params())
    raw = bytearray((tmp_path / "w.bin").read_bytes())
    raw[100] ^= 0xFF
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(rte.RteError):
        net2.load(tmp_path / "bad.bin")


def test_injected_nan_network_falls_back_alone_and_grouped(lib):
    """Host-side fault injection: a network whose every output is NaN makes the
    first Arnoldi step non-finite; the solver drops it, switches to block
    Jacobi and converges, alone and in a lockstep group, with no device
    fault.  Clearing the fault restores the network's own solve."""
    rte, shape, params, md, ctx, net, p = _setup(I=16, M=8, levels=3, proj=0.05)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    good = ctx.solve(x, pc=net, tol=1e-10, restart=30)
    net.inject_fault(rte.MgNet.FAULT_NAN)
    x.zero_()
    bad = ctx.solve(x, pc=net, tol=1e-10, restart=30)
    assert bad["converged"] and bad["fell_back"], bad
    assert torch.isfinite(x).all()
    r = p.rhs().ravel() - p.apply(x.cpu().numpy().reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(p.rhs()) <= 1e-10
    ctx2 = rte.Context.from_medium(md)
    xs = [torch.zeros(ctx2.n, dtype=torch.float64, device="cuda")]
    grp = rte.solve_group([ctx2], xs, pcs=[net], tol=1e-10, restart=30)
    assert grp[0]["iterations"] == bad["iterations"] and torch.equal(xs[0], x)
    net.inject_fault(rte.MgNet.FAULT_NONE)
    x.zero_()
    again = ctx.solve(x, pc=net, tol=1e-10, restart=30)
    assert again["iterations"] == good["iterations"] and again["fell_back"] == good["fell_back"]
    with pytest.raises(rte.RteError):
        net.inject_fault(7)
    ctx2.close()
