"""Eigenbases of media with many materials (1 - gamma varying from cell to
cell, the paper's independent sigma_T and sigma_a fields), computed batched on
the device: equal to the host FP64 eigen-solver material by material, and the
operator and the solve built on them at parity with the oracle."""
import numpy as np
import pytest

from oracle import krylov, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _per_cell_gamma(I, M, seed, eps=0.05, g=0.4):
    rng = np.random.default_rng(seed)
    N = I * I
    sT = np.exp(W.gaussian_field(I, 0.2, seed))
    rho = np.exp(np.log(0.01) + (np.log(0.3) - np.log(0.01)) * rng.uniform(0, 1, N))
    return W.Medium(I, M, sT, rho * sT, rng.uniform(0, 1, N), np.full(N, eps), g, W.random_inflow(I, M, seed + 1))


@pytest.mark.parametrize("I,M,seed", [(6, 8, 0), (5, 4, 1), (5, 64, 2), (5, 80, 3)])
def test_device_bases_equal_host_bases(lib, I, M, seed):
    from paper_2604_23265_gb300 import rte
    md = _per_cell_gamma(I, M, seed)
    ctx = rte.Context.from_medium(md)
    xi, L, mat = ctx.export_basis()
    omg = np.unique(md.eps ** 2 * md.sigma_a / md.sigma_T)
    assert len(omg) == xi.shape[0] > 16                    # the device path
    for j in list(range(0, len(omg), max(1, len(omg) // 6))) + [len(omg) - 1]:
        for axis in (0, 1):
            hx, hL = rte.eigenbasis(M, md.g, min(omg[j], 1.0), axis)
            # xi = -1 / mu: the slowest modes (large mu) carry the rounding of
            # mu relative to the spectrum's scale, not to their own size
            np.testing.assert_allclose(xi[j, axis * M:(axis + 1) * M], hx, rtol=0, atol=1e-12 * np.abs(hx).max())
            np.testing.assert_allclose(L[j][:, axis * M:(axis + 1) * M], hL, rtol=0, atol=1e-9)
    ctx.close()


@pytest.mark.parametrize("I,M,seed", [(16, 8, 4), (12, 16, 5)])
def test_many_material_medium_matches_oracle(lib, I, M, seed):
    from paper_2604_23265_gb300 import rte
    md = _per_cell_gamma(I, M, seed)
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    ctx = rte.Context.from_medium(md)
    assert ctx.info()["nmat"] == I * I
    x = W.random_vector(ctx.n, 3)
    y = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.apply(torch.tensor(x, device="cuda"), y)
    ref = p.apply(x.reshape(2 * M, -1)).ravel()
    rel = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert rel <= 1e-12 + 2.0 ** -52 / p.omg.min()
    xs = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(xs, tol=1e-12, restart=40)
    assert info["converged"], info
    xl = krylov.dense_solve(p.assemble(), p.rhs().ravel())
    psi = torch.zeros(M * I * I, dtype=torch.float64, device="cuda")
    ctx.reconstruct(xs, psi)
    ref = p.reconstruct(xl.reshape(2 * M, -1)).ravel()
    assert np.linalg.norm(psi.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
    ctx.close()
