"""Set-up by interpolation in ln tau (rte_setup_ex, RTE_BLOCKS_TABULATED)
against the per-cell FP64 inversion (RTE_BLOCKS_EXACT) on the same medium.

A cell's blocks depend on it only through (material, tau), so D(tau) and
R(tau) of a material can be tabulated at nodes tau = exp(0.04 i) and each
cell's blocks interpolated (8 points, in ln tau).  The bars: on a
well-conditioned medium the interpolation itself (1e-9 of the block's
largest entry); in the diffusive limit the exact inversion carries its own
rounding, cond(G_C) u64 relative, and the two paths agree to a small multiple
of it; R is stored in FP32 on both paths.  The solve on tabulated blocks meets
its tolerance by the oracle's FP64 residual.
"""
import numpy as np
import pytest

from oracle import tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pair(md):
    from paper_2604_23265_gb300 import rte
    ex = rte.Context.from_medium(md, block_mode=rte.Context.BLOCKS_EXACT)
    tb = rte.Context.from_medium(md, block_mode=rte.Context.BLOCKS_TABULATED)
    assert ex.tabulated_nodes() == 0 and tb.tabulated_nodes() > 0
    return rte, ex, tb


@pytest.mark.parametrize("eps,M", [(0.3, 8), (1e-3, 16)])
def test_tabulated_blocks_match_exact(lib, eps, M):
    md = W.grf_diffusive(seed=5, I=48, M=M, eps=eps)
    rte, ex, tb = _pair(md)
    De, Re = ex.export_blocks()
    Dt, Rt = tb.export_blocks()
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    cond = np.linalg.cond(p.blocks())                       # per cell
    dmax = np.abs(De).max(axis=(1, 2))
    bar_d = (64 * cond * 2.0 ** -52 + 1e-9) * dmax
    assert np.all(np.abs(Dt - De).max(axis=(1, 2)) <= bar_d)
    rmax = np.abs(Re).max(axis=(1, 2))
    bar_r = (4 * 2.0 ** -24 + 64 * cond * 2.0 ** -52 + 1e-9) * rmax
    assert np.all(np.abs(Rt.astype(np.float64) - Re).max(axis=(1, 2)) <= bar_r)
    ex.close()
    tb.close()


def test_tabulated_solve_meets_tolerance_by_oracle(lib):
    md = W.grf_diffusive(seed=6, I=64, M=16, eps=1e-3)
    rte, ex, tb = _pair(md)
    xs = []
    for ctx in (ex, tb):
        x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
        info = ctx.solve(x, tol=1e-8, restart=50)
        assert info["converged"], info
        xs.append((x.cpu().numpy(), info))
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    xi, L, mat = tb.export_basis()
    p.use_basis(xi, L)
    b = p.rhs().ravel()
    r = b - p.apply(xs[1][0].reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    # the same iteration count to within a few steps
    assert abs(xs[1][1]["iterations"] - xs[0][1]["iterations"]) <= max(3, xs[0][1]["iterations"] // 20)
    ex.close()
    tb.close()


def test_auto_mode_tabulates_large_single_material_media_only(lib):
    from paper_2604_23265_gb300 import rte
    big = rte.Context.from_medium(W.grf_diffusive(seed=7, I=128, M=8))          # 16,384 cells, 1 material
    small = rte.Context.from_medium(W.grf_diffusive(seed=7, I=32, M=8))         # 1,024 cells
    many = rte.Context.from_medium(W.polynomial_medium(3, "interface", I=64, M=4, layout=0))
    assert big.tabulated_nodes() > 0
    assert small.tabulated_nodes() == 0
    assert many.tabulated_nodes() == 0
    for c in (big, small, many):
        c.close()
