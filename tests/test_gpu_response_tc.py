"""Response apply on the tensor cores from the tabulated node tables.

On a context whose blocks are interpolated in ln tau, R_C = sum_p w_Cp R_p
over the cell's eight stencil nodes, so R z is applied per tile of cells as
sum_q w_Cq (R_q z_C) with BF16 MMAs (three parts per operand, six products,
FP32 accumulation).  Checked through rte_response_apply, w = A D v = v - P R v
(Sec. 4, block-Jacobi right preconditioning in face-flux space):

* against the FP64 oracle, element by element, at the per-cell FP32 path's
  bar: 2M-term FP32 sums of O(1) transfer coefficients, 8 M 2^-24 of the
  largest |v| (the interpolation adds 1e-9 of the blocks' size on these
  well-conditioned media, below FP32 in the diffusive limit);
* against the per-cell FP32 path on the same context;
* ragged tiles (cell counts that are no multiple of 128, bins of a few cells),
  tiles straddling materials, 2M = 32, 64, 128;
* at the benchmark size (256 x 256, M = 64, eps = 1e-3) on sampled cells
  against the oracle, in the launch configuration the benchmark solve uses;
* grouped solves on tabulated contexts stay bit-identical to lone solves.
"""
import numpy as np
import pytest

from oracle import tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _oracle(md):
    return tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)


def _materials(md, k, seed):
    """sigma_a = rho sigma_T with rho from k values by region: k materials."""
    rng = np.random.default_rng(seed)
    rho = np.array([0.05, 0.3, 0.12, 0.6])[:k]
    I = md.I
    iy, ix = np.divmod(np.arange(I * I), I)
    region = ((ix * k) // I + (iy * 2) // I + rng.integers(0, 2, I * I) * (ix % 7 == 0)) % k
    md.sigma_a = rho[region] * md.sigma_T
    return md


def _tab(md):
    from paper_2604_23265_gb300 import rte
    ctx = rte.Context.from_medium(md, block_mode=rte.Context.BLOCKS_TABULATED)
    assert ctx.tabulated_nodes() > 0
    return rte, ctx


def _both_paths(rte, ctx, v):
    w = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    assert ctx.response_on_tensor_cores()
    ctx.response_apply(torch.tensor(v.ravel(), device="cuda"), w)
    w_tc = w.cpu().numpy()
    ctx.set_response_path(rte.Context.RESPONSE_PER_CELL)
    assert not ctx.response_on_tensor_cores()
    ctx.response_apply(torch.tensor(v.ravel(), device="cuda"), w)
    w_pc = w.cpu().numpy()
    ctx.set_response_path(rte.Context.RESPONSE_AUTO)
    return w_tc, w_pc


CASES = [
    # I, M, eps, materials, seed
    (64, 16, 0.3, 1, 1),       # 4096 cells, 2M = 32
    (72, 32, 0.3, 3, 2),       # 5184 cells (ragged last tile), tiles across materials, 2M = 64
    (45, 64, 0.3, 2, 3),       # 2025 cells, 2M = 128
    (64, 16, 1e-3, 1, 4),      # diffusive limit
]


@pytest.mark.parametrize("I,M,eps,nmat,seed", CASES)
def test_response_tc_matches_oracle_and_per_cell(lib, I, M, eps, nmat, seed):
    md = _materials(W.grf_diffusive(seed=seed, I=I, M=M, eps=eps), nmat, seed)
    rte, ctx = _tab(md)
    p = _oracle(md)
    xi, L, _ = ctx.export_basis()
    p.use_basis(xi, L)
    v = W.random_vector(ctx.n, seed + 30).reshape(2 * M, -1)
    w_tc, w_pc = _both_paths(rte, ctx, v)
    ref = p.apply(tfps.block_apply(p.block_inverse(), v)).ravel()
    bar = 8 * M * 2.0 ** -24 * np.abs(v).max()
    assert np.abs(w_tc - ref).max() <= bar
    assert np.abs(w_tc - w_pc).max() <= bar
    # as accurate as the per-cell FP32 path up to a small factor: the node
    # tables are rounded to FP32 (x0 + x1 + x2 exactly) and combined with the
    # Lagrange weights in FP32, whose absolute sum on the central interval of
    # an 8-point stencil is at most 1.49; the per-cell R_C is rounded once
    assert np.linalg.norm(w_tc - ref) <= 4 * np.linalg.norm(w_pc - ref) + 1e-30
    ctx.close()


def test_response_tc_zero_and_single_direction_inputs(lib):
    """Degenerate inputs: v = 0 gives w = 0 exactly; a v supported on one slot
    of one cell changes only that cell's rows and its neighbours' rows."""
    md = W.grf_diffusive(seed=8, I=64, M=32, eps=0.3)
    rte, ctx = _tab(md)
    n, N = ctx.n, md.I * md.I
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    ctx.response_apply(torch.zeros(n, dtype=torch.float64, device="cuda"), w)
    assert torch.count_nonzero(w).item() == 0
    c = 33 * md.I + 17
    v = np.zeros((2 * md.M, N))
    v[5, c] = 1.0
    ctx.response_apply(torch.tensor(v.ravel(), device="cuda"), w)
    wn = w.cpu().numpy().reshape(2 * md.M, N)
    touched = np.nonzero(np.abs(wn).sum(axis=0))[0]
    assert set(touched.tolist()) <= {c, c - 1, c + 1, c - md.I, c + md.I}
    p = _oracle(md)
    xi, L, _ = ctx.export_basis()
    p.use_basis(xi, L)
    ref = p.block_jacobi_rows(v, touched)
    assert np.abs(wn[:, touched] - ref).max() <= 8 * md.M * 2.0 ** -24
    ctx.close()


def test_response_tc_keeps_each_cells_gain(lib):
    """One optical thickness for every cell, between two nodes (ln tau / 0.04 =
    0.515, where the 8-point Lagrange weights rounded to FP32 would sum to
    1 + 5e-8): the tensor-core R z must not rescale R_C.  With every cell on
    the same weights, a rescaling is the component of (tensor-core - per-cell)
    along the response itself; rounding to nearest alone leaves about 1e-10
    there, while a gain of 5e-8 is the size of the absorption 1 - gamma of the
    diffusive benchmark medium.  The tensor cores' FP32 accumulation is not
    rounded to nearest: the products of the main parts are kept in their own
    accumulator (eight additions a node), which bounds the loss it leaves to
    about one FP32 ulp."""
    md = W.grf_diffusive(seed=10, I=64, M=16, eps=0.3)
    N = md.I * md.I
    md.sigma_T = np.full(N, 0.3 * md.I * np.exp(0.04 * 0.515))    # tau = sigma_T h / eps
    md.sigma_a = 0.05 * md.sigma_T
    rte, ctx = _tab(md)
    v = W.random_vector(ctx.n, 41)
    w_tc, w_pc = _both_paths(rte, ctx, v)
    po = v - w_pc                                       # P R v on the per-cell path
    gain = np.dot(w_pc - w_tc, po) / np.dot(po, po)     # (R_tc - R_pc) v along R v
    assert abs(gain) <= 1e-7, gain
    ctx.close()


def test_response_tc_benchmark_size_sampled(lib):
    """256 x 256, M = 64, eps = 1e-3 (the benchmark medium; automatic block mode
    tabulates it and selects the tensor-core path): sampled cells, their rows
    of A D v against the oracle (blocks of those cells and their neighbours
    only), and the whole vector against the per-cell FP32 path."""
    from paper_2604_23265_gb300 import rte
    md = W.grf_diffusive(0)
    ctx = rte.Context.from_medium(md)
    assert ctx.tabulated_nodes() > 0 and ctx.response_on_tensor_cores()
    v = W.random_vector(ctx.n, 77).reshape(2 * md.M, -1)
    w_tc, w_pc = _both_paths(rte, ctx, v)
    bar = 8 * md.M * 2.0 ** -24 * np.abs(v).max()
    assert np.abs(w_tc - w_pc).max() <= bar
    p = _oracle(md)
    xi, L, _ = ctx.export_basis()
    p.use_basis(xi, L)
    N, I = md.I * md.I, md.I
    rng = np.random.default_rng(5)
    cells = np.unique(np.concatenate([[0, I - 1, N - I, N - 1, 128, N // 2 + 7], rng.integers(0, N, 40)]))
    ref = p.block_jacobi_rows(v, cells)
    got = w_tc.reshape(2 * md.M, N)[:, cells]
    assert np.abs(got - ref).max() <= bar
    ctx.close()


def test_group_on_tabulated_contexts_is_bit_identical(lib):
    """Grouped solves whose contexts take the tensor-core response (one
    launch per item before the grouped gather) reproduce the lone solves bit
    for bit, alongside a small context on the per-cell path."""
    from paper_2604_23265_gb300 import rte
    media = [W.grf_diffusive(seed=20 + i, I=64, M=16, eps=e) for i, e in enumerate((0.3, 0.05))]
    media.append(W.mixed_instance(5, grids=(12,), dirs=(8,)))
    modes = [rte.Context.BLOCKS_TABULATED, rte.Context.BLOCKS_TABULATED, rte.Context.BLOCKS_AUTO]

    def ctx_of(md, mode):
        return rte.Context.from_medium(md, block_mode=mode)

    lone = []
    for md, mode in zip(media, modes):
        c = ctx_of(md, mode)
        x = torch.zeros(c.n, dtype=torch.float64, device="cuda")
        info = c.solve(x, tol=1e-9, restart=30)
        lone.append((c, x, info))
    assert [c.response_on_tensor_cores() for c, _, _ in lone] == [True, True, False]
    ctxs = [ctx_of(md, mode) for md, mode in zip(media, modes)]
    xs = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = rte.solve_group(ctxs, xs, tol=1e-9, restart=30)
    for (c1, x1, i1), x2, i2 in zip(lone, xs, infos):
        assert i1["converged"] and i2["converged"], (i1, i2)
        assert i2["iterations"] == i1["iterations"]
        assert torch.equal(x1, x2)
