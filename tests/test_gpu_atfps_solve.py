"""GPU parity of the compressed ATFPS solve and the layer reconstruction (Sec.
2.3.3-2.3.4) against the FP64 oracle on the same seeded media: the smooth
solution of the compressed system and the full solution with layers, compared
on the face-midpoint values of the solution (the coefficients themselves
cancel heavily in the diffusive regime); delta = 0 against the full TFPS
solve; the closed form q / sigma_a; and at 64 x 64 x M 16 the O(delta) face
accuracy against the library's own full solve."""
import numpy as np
import pytest

from oracle import atfps as OA, tfps
from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _grf(I, M, eps, seed):
    md = W.grf_diffusive(seed, I=I, M=M, eps=eps)
    md.inflow = W.random_inflow(I, M, seed + 5)
    return md


def _prob(md):
    return tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)


def _faces(p, alpha):
    return p.face_values(np.asarray(alpha).reshape(2 * p.M, -1))


def _solve(ctx, delta, layers, **kw):
    ctx.atfps_setup(delta)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.atfps_solve(x, layers=layers, **kw)
    return x.cpu().numpy(), info


CASES = [(8, 8, 1e-2, 0, 1e-2), (12, 8, 3e-2, 1, 1e-3), (16, 4, 1e-2, 2, 1e-2), (10, 16, 1e-2, 3, 1e-1)]


@pytest.mark.parametrize("I,M,eps,seed,delta", CASES)
def test_compressed_solve_and_layers_match_oracle(lib, I, M, eps, seed, delta):
    from paper_2604_23265_gb300 import rte
    md = _grf(I, M, eps, seed)
    p = _prob(md)
    ctx = rte.Context.from_medium(md)
    full_ref, smooth_ref, mask = OA.atfps_solution(p, delta)
    assert 0 < mask.mean() < 1
    # the compressed system inherits the conditioning of the slow modes: the
    # FP64 residual reaches 1e-11 on these media, the face values 1e-8
    xs, info = _solve(ctx, delta, False, tol=1e-11, restart=60, max_iter=3000)
    assert info["converged"], (info["relres"], info["iterations"])
    # dropped slots stay exactly zero without layers
    assert np.all(xs.reshape(2 * M, -1)[~mask] == 0.0)
    scale = np.abs(_faces(p, full_ref)).max()
    assert np.abs(_faces(p, xs) - _faces(p, smooth_ref)).max() <= 1e-8 * scale
    xf, info = _solve(ctx, delta, True, tol=1e-11, restart=60, max_iter=3000)
    assert np.abs(_faces(p, xf) - _faces(p, full_ref)).max() <= 1e-8 * scale
    ctx.close()


def test_delta_zero_equals_the_full_solve(lib):
    from paper_2604_23265_gb300 import rte
    md = _grf(12, 8, 1e-2, 4)
    p = _prob(md)
    ctx = rte.Context.from_medium(md)
    xc, info = _solve(ctx, 0.0, True, tol=1e-11, max_iter=3000)
    assert info["converged"]
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.solve(x, tol=1e-12)
    fv = _faces(p, x.cpu().numpy())
    assert np.abs(_faces(p, xc) - fv).max() <= 1e-9 * np.abs(fv).max()
    ctx.close()


def test_closed_form_q_over_sigma_a(lib):
    from paper_2604_23265_gb300 import rte
    I, M = 16, 8
    N = I * I
    sa = 0.5
    md = W.Medium(I, M, np.full(N, 20.0), np.full(N, sa), np.ones(N), np.full(N, 0.05), 0.3,
                  np.full((4, I, M), 1.0 / sa))
    ctx = rte.Context.from_medium(md)
    rows = ctx.atfps_setup(1e-2)
    assert rows < ctx.n
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.atfps_solve(x, tol=1e-12)
    psi = torch.zeros(M * N, dtype=torch.float64, device="cuda")
    ctx.reconstruct(x, psi)
    np.testing.assert_allclose(psi.cpu().numpy(), 1.0 / sa, rtol=1e-12)
    ctx.close()


def test_face_accuracy_is_order_delta_at_64(lib):
    """64 x 64, M = 16, eps = 1e-2: the face values of the compressed
    solution with layers are within delta (times the solution's size) of the
    full TFPS solution's, and much closer than without layers."""
    from paper_2604_23265_gb300 import rte
    md = _grf(64, 16, 1e-2, 6)
    p = _prob(md)
    ctx = rte.Context.from_medium(md)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.solve(x, tol=1e-12)
    ref = _faces(p, x.cpu().numpy())
    scale = np.abs(ref).max()
    last = None
    for delta in (1e-2, 1e-3):
        xf, info = _solve(ctx, delta, True, tol=1e-10, max_iter=5000)
        assert info["converged"], info
        xs, _ = _solve(ctx, delta, False, tol=1e-10, max_iter=5000)
        ef = np.abs(_faces(p, xf) - ref).max()
        es = np.abs(_faces(p, xs) - ref).max()
        assert ef <= delta * scale
        assert ef <= 5e-2 * es
        if last is not None:
            assert ef < last
        last = ef
    ctx.close()
