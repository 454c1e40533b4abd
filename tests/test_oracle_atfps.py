"""Pins of the ATFPS filter (Sec. 2.3) and the filtered loss (Eq. loss_delta)."""
import numpy as np
import pytest

from oracle import atfps, krylov, mgnet, tfps
from paper_2604_23265_gb300 import workloads as W


def _prob(md):
    return tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)


def test_selection_rule():
    md = W.grf_diffusive(1, I=8, M=8, eps=1e-2)
    p = _prob(md)
    mask = atfps.selection(p, 1e-2)
    a = np.abs(p.xi[p.mat_id]).T
    np.testing.assert_array_equal(mask, np.exp(-0.5 * a * p.tau[None, :]) > 1e-2)
    # the slowest function of every centring group is kept in the diffusive regime
    M2 = p.M // 2
    for grp in range(4):
        sl = slice(grp * M2, (grp + 1) * M2)
        k = np.argmin(np.abs(p.xi[0][sl])) + grp * M2
        assert mask[k].all()
    assert not mask.all()


def test_interface_basis_invariants():
    md = W.grf_diffusive(2, I=6, M=8, eps=1e-2)
    p = _prob(md)
    mask = atfps.selection(p, 1e-2)
    for kind, cm, cp, fm, fp in atfps.interfaces(p)[:40]:
        groups = [(cm, fm)] + ([(cp, fp)] if kind == "in" else [])
        rows = None if kind == "in" else p.dirs[fm]
        E, s = atfps.interface_basis(p, groups, mask, rows)
        np.testing.assert_allclose(np.abs(E).max(axis=0), 1.0, rtol=1e-14)
        if s > 1:
            Qs = E[:, :s] / np.linalg.norm(E[:, :s], axis=0)
            np.testing.assert_allclose(Qs.T @ Qs, np.eye(s), atol=1e-12)
        assert np.linalg.cond(E) < 1e12


def test_P12_transport_regime_keeps_everything():
    """eps = 1: nothing is dropped at delta = 1e-2, and the filtered residual of
    the exact solution vanishes with the unfiltered one (same minimiser)."""
    md = W.checkerboard_transport(0, I=8, M=8)
    p = _prob(md)
    F, mask = atfps.filter_operator(p, 1e-2)
    assert mask.all()
    assert F.shape[0] == 2 * p.M * p.N          # one kept coordinate per row of A
    D = p.block_inverse()
    r = W.random_vector(2 * p.M * p.N, 3)
    # psi solving A D psi = r exactly (dense LU of the assembled operator)
    A = p.assemble().toarray()
    Dfull = np.zeros_like(A)
    N = p.N
    for c in range(N):
        idx = np.arange(2 * p.M) * N + c
        Dfull[np.ix_(idx, idx)] = D[c]
    psi = np.linalg.solve(A @ Dfull, r)
    res = atfps.filtered_residual(p, D, F, mask, psi, r)
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(F @ r)
    # and a non-solution has a non-zero filtered residual
    assert np.linalg.norm(atfps.filtered_residual(p, D, F, mask, r, r)) > 1e-3


def test_P13_delta_zero_is_scaled_orthogonal_projection():
    """delta = 0 keeps every function; per interface the kept coordinates are
    diag(||q_k||_inf) Q^T applied to the jump."""
    md = W.grf_diffusive(3, I=5, M=8, eps=1e-2)
    p = _prob(md)
    F, mask = atfps.filter_operator(p, 0.0)
    assert mask.all()
    y = W.random_vector(2 * p.M * p.N, 4)
    Fy = F @ y
    kind, cm, cp, fm, fp = atfps.interfaces(p)[0]
    E, s = atfps.interface_basis(p, [(cm, fm), (cp, fp)], mask)
    assert s == p.M
    N, M2 = p.N, p.M // 2
    J = np.zeros(p.M)
    for m in range(p.M):
        if m in p.dirs[fm]:
            J[m] = y[(fm * M2 + list(p.dirs[fm]).index(m)) * N + cm]
        else:
            J[m] = -y[(fp * M2 + list(p.dirs[fp]).index(m)) * N + cp]
    Qn = E / np.linalg.norm(E, axis=0)
    scale = 1.0 / np.abs(Qn).max(axis=0)          # E = Qn diag(1/||q||_inf)
    np.testing.assert_allclose(Fy[:p.M], (Qn.T @ J) / scale, atol=1e-10)


def test_filtered_loss_gradient_matches_finite_differences():
    shape = W.NetShape(M=4, levels=2, c0=4, cmax=8, cc=4, ccmax=8)
    params = W.init_params(shape, seed=1, proj_scale=0.3)
    md = W.polynomial_diffusion(0, I=8, M=4)
    p = _prob(md)
    D = p.block_inverse()
    F, mask = atfps.filter_operator(p, 1e-2)
    cx = mgnet.coeff_inputs(md)
    rs = [W.random_vector(2 * p.M * p.N, 10 + b) for b in range(2)]
    args = ([p, p], [D, D], [F, F], [mask, mask], [cx, cx], rs)
    loss, grads = atfps.loss_and_grad_filtered(params, shape, *args)
    d = {k: np.random.default_rng(2).standard_normal(v.shape) for k, v in params.items()}
    h = 1e-7          # small enough not to straddle a ReLU kink
    lp = atfps.loss_and_grad_filtered({k: v + h * d[k] for k, v in params.items()}, shape, *args)[0]
    lm = atfps.loss_and_grad_filtered({k: v - h * d[k] for k, v in params.items()}, shape, *args)[0]
    fd = (lp - lm) / (2 * h)
    an = sum(np.sum(grads[k] * d[k]) for k in params)
    assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-3)
