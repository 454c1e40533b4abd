"""GPU parity of the df64 Gram-Schmidt step (the solver's Arnoldi arithmetic,
rte_cgs2_df64) against the FP64 kernels (rte_cgs2) and the definition.

df64 vectors carry 48 significant bits, so inputs are drawn in FP64 and
rounded to the nearest df64 value (hi = (float)x, lo = (float)(x - hi)); both
paths then see exactly the same numbers.  The bar is 1e-14 of ||w||: each df64
product is exact to about 2^-47 relative and the running sums keep 48 bits, so
a projection carries an error of order 2^-48 ||v|| ||w|| = 3.6e-15 ||w||,
against 1e-16 for the FP64 kernels.  The sizes cover one ragged 128-element
chunk tail, many chunks per block, and the pipeline depths of K = 1 (eight
stages) to K = 64 (two stages, one block per SM).
"""
import numpy as np
import pytest

from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _split(x):
    """FP64 array -> (hi, lo) float32 planes and the exact FP64 value hi + lo."""
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo, hi.astype(np.float64) + lo.astype(np.float64)


def _df_tensor(rows):
    """rows: list of (hi, lo) -> float32 device tensor [rows][2][n]."""
    return torch.tensor(np.concatenate([np.concatenate([h, l]) for h, l in rows]), device="cuda")


def _case(n, k, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    Vs = [_split(np.ascontiguousarray(Q[:, j])) for j in range(k)]
    w = rng.standard_normal(n) + Q @ (rng.standard_normal(k) * 5.0)
    return Vs, _split(w)


CASES = [(19, 8, 1), (19, 8, 7), (19, 8, 64), (64, 32, 1), (64, 32, 13), (64, 32, 50), (64, 32, 64)]


@pytest.mark.parametrize("I,M,k", CASES)
def test_cgs2_df64_matches_fp64_kernels_and_definition(lib, I, M, k):
    from paper_2604_23265_gb300 import rte
    ctx = rte.Context.from_medium(W.checkerboard_transport(1, I=I, M=M))
    n = ctx.n
    Vs, (wh, wl, w64) = _case(n, k, 100 * I + k)
    V64 = np.stack([v[2] for v in Vs])
    # FP64 kernels on the same (df64-representable) values
    Vd = torch.tensor(V64.ravel(), device="cuda")
    wd = torch.tensor(w64, device="cuda")
    hd = torch.zeros(k + 1, dtype=torch.float64, device="cuda")
    ctx.cgs2(Vd, k, wd, hd)
    # df64 kernels
    Vf = _df_tensor([(v[0], v[1]) for v in Vs])
    wf = _df_tensor([(wh, wl)])
    hf = torch.zeros(k + 1, dtype=torch.float64, device="cuda")
    ctx.cgs2_df64(Vf, k, wf, hf)
    torch.cuda.synchronize()
    h64, hdf = hd.cpu().numpy(), hf.cpu().numpy()
    wn = np.linalg.norm(w64)
    bar = 1e-14 * wn
    np.testing.assert_array_less(np.abs(hdf - h64), bar)
    # the definition: h = V^T w, w_out = (I - V V^T) w / ||.||
    href = V64 @ w64
    r = w64 - V64.T @ href
    np.testing.assert_array_less(np.abs(hdf[:k] - href), bar)
    assert abs(hdf[k] - np.linalg.norm(r)) <= bar
    wo = wf.cpu().numpy().astype(np.float64)
    wout = wo[:n] + wo[n:]
    amp = wn / np.linalg.norm(r)             # normalisation amplifies by ||w|| / ||r||
    assert np.linalg.norm(wout - wd.cpu().numpy()) <= 1e-14 * amp
    assert np.linalg.norm(wout - r / np.linalg.norm(r)) <= 1e-14 * amp
    # the output is a normalised df64 vector: |lo| <= ulp(hi)
    hi, lo = wo[:n], wo[n:]
    assert np.all(np.abs(lo) <= np.spacing(np.abs(hi).astype(np.float32)).astype(np.float64))
    ctx.close()


@pytest.mark.parametrize("k", [8, 40, 64])
def test_arnoldi_basis_df64_is_orthonormal_and_follows_fp64(lib, k):
    """The df64 Arnoldi process (the solver's) keeps V^T V = I to 1e-12 on the
    diffusive medium where the Krylov vectors are nearly dependent (pin P15),
    and its first vectors follow the FP64 process's."""
    from paper_2604_23265_gb300 import rte
    md = W.grf_diffusive(seed=2, I=24, M=8, eps=1e-3)
    ctx = rte.Context.from_medium(md)
    n = ctx.n
    Vf = torch.zeros(k * 2 * n, dtype=torch.float32, device="cuda")
    ctx.arnoldi_basis_df64(k, Vf)
    v = Vf.view(k, 2, n).double()
    V = (v[:, 0, :] + v[:, 1, :]).cpu().numpy()
    assert np.abs(V @ V.T - np.eye(k)).max() <= 1e-12
    Vd = torch.zeros(k * n, dtype=torch.float64, device="cuda")
    ctx.arnoldi_basis(k, Vd)
    V64 = Vd.cpu().numpy().reshape(k, n)
    for j in range(min(k, 8)):
        assert np.linalg.norm(V[j] - V64[j]) <= 1e-10, j
    ctx.close()


def test_df64_solve_residual_by_oracle(lib):
    """A block-Jacobi solve of the benchmark's diffusive medium (smaller grid)
    with the df64 Arnoldi step converges, and the oracle's FP64 residual of its
    solution (on the device's exported basis) meets 1e-8."""
    from oracle import tfps
    from paper_2604_23265_gb300 import rte
    md = W.grf_diffusive(seed=4, I=32, M=16, eps=1e-3)
    ctx = rte.Context.from_medium(md)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, tol=1e-8, restart=50)
    assert info["converged"], info
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    xi, L, mat = ctx.export_basis()
    p.use_basis(xi, L)
    b = p.rhs().ravel()
    r = b - p.apply(x.cpu().numpy().reshape(2 * md.M, -1)).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    ctx.close()
