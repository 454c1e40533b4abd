"""Pins of the FP64 oracle's DOM/TFPS system against facts the paper and the
mathematics fix (closed forms, invariants, exact solutions, brute force)."""
import numpy as np
import pytest

from oracle import krylov, tfps
from paper_2604_23265_gb300 import workloads as W


def _problem(md):
    return tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)


def _uniform(I, M, sT, sa, q, eps, g, inflow=None):
    N = I * I
    return tfps.Problem(I, M, np.full(N, sT), np.full(N, sa), np.full(N, q), eps, g, inflow)


# --------------------------------------------------------------------- Sec 2.1
@pytest.mark.parametrize("M", [4, 8, 16, 32, 64])
def test_quadrature_symmetric_and_nonzero(M):
    theta, c, s, w = tfps.quadrature(M)
    assert np.all(np.abs(c) > 1e-3) and np.all(np.abs(s) > 1e-3)
    assert np.isclose(w.sum(), 1.0)
    assert (c > 0).sum() == M // 2 and (s > 0).sum() == M // 2
    np.testing.assert_allclose(c[::-1], c, atol=1e-15)  # theta -> -theta


def test_quadrature_rejects_bad_M():
    with pytest.raises(ValueError):
        tfps.quadrature(6)


@pytest.mark.parametrize("M", [4, 16, 64])
@pytest.mark.parametrize("g", [0.0, 0.3, 0.5, 0.9])
def test_P1_hg_normalised(M, g):
    """P1: sum_n kappa_mn w_n = 1, K symmetric circulant; HG shape ratio (Eq. hg)."""
    K = tfps.hg_matrix(M, g)
    theta, _, _, w = tfps.quadrature(M)
    np.testing.assert_allclose(K @ w, 1.0, atol=1e-15 * M)
    np.testing.assert_array_equal(K, K.T)
    for m in range(M):
        np.testing.assert_allclose(K[m], np.roll(K[0], m), rtol=1e-12)
    d = theta[1] - theta[0]
    expect = ((1 + g * g - 2 * g) / (1 + g * g - 2 * g * np.cos(d))) ** 1.5
    assert np.isclose(K[0, 1] / K[0, 0], expect, rtol=1e-13)


def test_P1_isotropic_is_all_ones():
    np.testing.assert_allclose(tfps.hg_matrix(16, 0.0), np.ones((16, 16)), rtol=1e-15)


# --------------------------------------------------------------------- Sec 2.2
@pytest.mark.parametrize("M,g", [(8, 0.0), (16, 0.5), (32, 0.8), (64, 0.5)])
@pytest.mark.parametrize("omg", [0.9, 0.1, 1e-3, 5e-8])
@pytest.mark.parametrize("which", ["c", "s"])
def test_P2_eigen_residual(M, g, omg, which):
    """P2: (gamma K W - I) l = xi D l with M/2 negative and M/2 positive xi, ||l||_inf = 1."""
    K = tfps.hg_matrix(M, g)
    _, c, s, _ = tfps.quadrature(M)
    d = c if which == "c" else s
    xi, L = tfps.eigenbasis(omg, K, d)
    gam = 1.0 - omg
    lhs = (gam * K / M - np.eye(M)) @ L
    rhs = d[:, None] * L * xi[None, :]
    scale = max(1.0, np.abs(xi).max())
    assert np.abs(lhs - rhs).max() <= 1e-12 * scale
    assert (xi < 0).sum() == M // 2 and (xi > 0).sum() == M // 2
    assert np.all(np.diff(xi) > 0)
    np.testing.assert_allclose(np.abs(L).max(axis=0), 1.0, rtol=1e-8)
    # normalisation: the first (near-)maximal entry is exactly +1
    for k in range(M):
        a = np.abs(L[:, k])
        p = np.nonzero(a >= (1 - 1e-8) * a.max())[0][0]
        assert L[p, k] == 1.0


@pytest.mark.parametrize("M", [8, 16, 32])
@pytest.mark.parametrize("omg", [0.5, 1e-2, 1e-6])
def test_P3_isotropic_dispersion(M, omg):
    """P3 (g=0, KW = 11^T/M): odd modes have xi = -1/c_m exactly; even modes obey
    1 = (gamma/M) sum_m 1/(1 + xi c_m); the slowest obeys xi^2 ~ 2(1-gamma)."""
    K = tfps.hg_matrix(M, 0.0)
    _, c, _, _ = tfps.quadrature(M)
    xi, L = tfps.eigenbasis(omg, K, c)
    gam = 1.0 - omg
    odd = np.abs(L.sum(axis=0)) < 1e-8
    assert odd.sum() == M // 2
    np.testing.assert_allclose(np.sort(xi[odd]), np.sort(-1.0 / c[: M // 2]), rtol=1e-12)
    for x in xi[~odd]:
        assert abs(gam / M * np.sum(1.0 / (1.0 + x * c)) - 1.0) < 1e-11
    slow = np.min(np.abs(xi))
    if omg < 1e-3:
        assert abs(slow ** 2 / (2 * omg / gam) - 1.0) < 10 * omg + 1e-9


@pytest.mark.parametrize("M", [8, 16])
def test_P4_pure_absorber(M):
    """P4 (gamma=0): xi = -1/c_m with eigenvectors spanning the unit vectors of equal c_m."""
    K = tfps.hg_matrix(M, 0.4)
    _, c, _, _ = tfps.quadrature(M)
    xi, L = tfps.eigenbasis(1.0, K, c)
    np.testing.assert_allclose(np.sort(xi), np.sort(-1.0 / c), rtol=1e-13)
    for k in range(M):
        support = np.abs(L[:, k]) > 1e-12
        assert np.allclose(c[support], -1.0 / xi[k], rtol=1e-12)


def test_P5_constant_particular_solution():
    """P5: piecewise medium with q/sigma_a constant and matching inflow -> b = 0,
    alpha = 0 and psi = q/sigma_a everywhere (closed form of Eq. RTE)."""
    I, M = 8, 8
    rng = np.random.default_rng(3)
    sa = rng.uniform(0.1, 2.0, I * I)
    sT = sa + rng.uniform(0.5, 5.0, I * I)
    q = 0.7 * sa
    p = tfps.Problem(I, M, sT, sa, q, 0.05, 0.5, np.full((4, I, M), 0.7))
    b = p.rhs()
    assert np.abs(b).max() < 1e-15
    psi = p.reconstruct(np.zeros_like(b))
    np.testing.assert_allclose(psi, 0.7, rtol=1e-15)


def _slab_case(axis, I=8, M=8, g=0.5, eps=0.1, sT=2.0, sa=0.3, q=0.6, seed=5):
    """Exact DOM slab solution in a uniform medium (P6)."""
    p0 = _uniform(I, M, sT, sa, q, eps, g)
    sTe = sT / eps
    c, s = p0.c, p0.s
    xi_all, L_all = p0.xi[0], p0.L[0]
    sl = slice(0, M) if axis == 0 else slice(M, 2 * M)
    xi, L = xi_all[sl], L_all[:, sl]
    a = np.random.default_rng(seed).uniform(-1, 1, M)
    z0 = np.where(xi < 0, 0.0, 1.0)

    def u(z):  # (M,) angular flux at coordinate z along the slab axis
        return L @ (a * np.exp(sTe * xi * (z - z0))) + q / sa
    h = 1.0 / I
    inflow = np.zeros((4, I, M))
    for j in range(I):
        mid = (j + 0.5) * h
        if axis == 0:
            inflow[0, j] = u(0.0); inflow[1, j] = u(1.0)
            inflow[2, j] = u(mid); inflow[3, j] = u(mid)
        else:
            inflow[2, j] = u(0.0); inflow[3, j] = u(1.0)
            inflow[0, j] = u(mid); inflow[1, j] = u(mid)
    p = _uniform(I, M, sT, sa, q, eps, g, inflow)
    iy, ix = np.divmod(np.arange(I * I), I)
    pos = ix if axis == 0 else iy
    alpha = np.zeros((2 * M, I * I))
    for k in range(M):
        zref = pos * h if xi[k] < 0 else (pos + 1) * h
        alpha[sl.start + k] = a[k] * np.exp(sTe * xi[k] * (zref - z0[k]))
    centres = np.stack([u((pp + 0.5) * h) for pp in pos], axis=1)
    return p, alpha, centres


@pytest.mark.parametrize("axis", [0, 1])
def test_P6_slab_exact(axis):
    """P6: the TFPS system reproduces the exact slab solution of the DO-RTE."""
    p, alpha, centres = _slab_case(axis)
    b = p.rhs()
    r = b - p.apply(alpha)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)
    x = krylov.dense_solve(p.assemble(), b.ravel()).reshape(alpha.shape)
    np.testing.assert_allclose(x, alpha, atol=1e-11)
    np.testing.assert_allclose(p.reconstruct(x), centres, atol=1e-11)


def test_P7_fgmres_matches_dense_lu():
    """P7: block-Jacobi FGMRES solution equals the dense LU solution (16x16 cells, M=8)."""
    I, M = 16, 8
    rng = np.random.default_rng(11)
    sT = np.exp(rng.standard_normal(I * I))
    p = tfps.Problem(I, M, sT, 0.2 * sT, rng.uniform(0, 1, I * I), 0.3, 0.5,
                     W.random_inflow(I, M, 2))
    b = p.rhs().ravel()
    x_lu = krylov.dense_solve(p.assemble(), b)
    D = p.block_inverse()
    x, info = krylov.fgmres(lambda v: p.apply(v.reshape(2 * M, -1)).ravel(), b,
                            lambda v, j: tfps.block_apply(D, v.reshape(2 * M, -1)).ravel(),
                            tol=1e-13, restart=60)
    assert info["converged"]
    assert np.linalg.norm(x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)


def test_matrix_free_equals_assembled():
    I, M = 6, 8
    md = W.polynomial_diffusion(1, I=I, M=M)
    p = _problem(md)
    A = p.assemble()
    x = W.random_vector(p.M * 2 * p.N, 4)
    np.testing.assert_allclose(p.apply(x.reshape(2 * M, -1)).ravel(), A @ x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(p.apply_adjoint(x.reshape(2 * M, -1)).ravel(), A.T @ x, rtol=0, atol=1e-13)


def test_P8_blocks_are_diagonal_blocks():
    I, M = 5, 8
    rng = np.random.default_rng(0)
    sT = rng.uniform(0.5, 4, I * I)
    p = tfps.Problem(I, M, sT, 0.3 * sT, np.ones(I * I), 0.2, 0.6)
    A = p.assemble().toarray()
    G = p.blocks()
    N = p.N
    for c in range(N):
        idx = np.arange(2 * M) * N + c
        np.testing.assert_array_equal(A[np.ix_(idx, idx)], G[c])


def test_block_jacobi_rows_match_assembled_operator():
    """The restricted A D v of ``block_jacobi_rows`` (blocks of the sampled
    cells and their neighbours only) equals A D v from the assembled sparse A,
    with D the inverses of A's own diagonal blocks, at every sampled cell
    (interior, edge and corner cells; three materials)."""
    I, M = 7, 8
    rng = np.random.default_rng(3)
    sT = rng.uniform(0.5, 4, I * I)
    sa = np.choose(rng.integers(0, 3, I * I), [0.1 * sT, 0.3 * sT, 0.05 * sT])
    p = tfps.Problem(I, M, sT, sa, np.ones(I * I), 0.3, 0.5)
    A = p.assemble().toarray()
    N, n2 = p.N, 2 * M
    v = W.random_vector(n2 * N, 21).reshape(n2, N)
    alpha = np.zeros_like(v)
    for c in range(N):
        idx = np.arange(n2) * N + c
        alpha[:, c] = np.linalg.solve(A[np.ix_(idx, idx)], v[:, c])
    ref = (A @ alpha.ravel()).reshape(n2, N)
    cells = np.array([0, 3, I - 1, I, 24, N - I, N - 1, 17])
    np.testing.assert_allclose(p.block_jacobi_rows(v, cells), ref[:, cells], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(p.blocks_at(cells), p.blocks()[cells])


def test_P9_AD_invariant_to_eigenvector_signs():
    """P9: A D does not depend on the sign of any basis vector."""
    I, M = 6, 8
    md = W.polynomial_diffusion(2, I=I, M=M)
    p = _problem(md)
    r = W.random_vector(2 * M * p.N, 9).reshape(2 * M, -1)
    y1 = p.apply(tfps.block_apply(p.block_inverse(), r))
    flip = np.where(np.random.default_rng(1).uniform(size=2 * M) < 0.5, -1.0, 1.0)
    p.L = p.L * flip[None, None, :]
    y2 = p.apply(tfps.block_apply(p.block_inverse(), r))
    np.testing.assert_allclose(y1, y2, atol=1e-12)


def test_use_basis_takes_the_given_eigenpairs():
    """Problem.use_basis (how a device's exported basis enters the oracle):
    its own basis changes nothing; a basis with flipped column signs gives the
    same traces for the coefficients with the same signs flipped (so the given
    L is used); eigenvalues scaled by 2 give the decays of a cell twice as
    thick (so the given xi is used)."""
    I, M = 5, 8
    md = W.polynomial_diffusion(3, I=I, M=M)
    p = _problem(md)
    x = W.random_vector(2 * M * p.N, 4).reshape(2 * M, -1)
    y0 = p.apply(x)
    q = _problem(md).use_basis(p.xi, p.L)
    np.testing.assert_array_equal(q.apply(x), y0)
    flip = np.where(np.random.default_rng(3).uniform(size=2 * M) < 0.5, -1.0, 1.0)
    q = _problem(md).use_basis(p.xi, p.L * flip[None, None, :])
    np.testing.assert_allclose(q.apply(x * flip[:, None]), y0, rtol=0, atol=1e-14 * np.abs(y0).max())
    q = _problem(md).use_basis(2 * p.xi, p.L)
    np.testing.assert_allclose(q.dec, _problem(md).dec ** 2, rtol=1e-13, atol=0)


def test_P10_adjoint_dot():
    I, M = 7, 16
    md = W.checkerboard_transport(1, I=I, M=M)
    p = _problem(md)
    x = W.random_vector(2 * M * p.N, 1).reshape(2 * M, -1)
    y = W.random_vector(2 * M * p.N, 2).reshape(2 * M, -1)
    lhs = np.sum(p.apply(x) * y)
    rhs = np.sum(x * p.apply_adjoint(y))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) * 10 + 1e-13
    D = p.block_inverse()
    assert abs(np.sum(tfps.block_apply(D, x) * y) - np.sum(x * tfps.block_apply_T(D, y))) < 1e-10


def _solve(p):
    b = p.rhs().ravel()
    x = krylov.dense_solve(p.assemble(), b)
    return p.reconstruct(x.reshape(2 * p.M, -1))


def test_P14_mirror_symmetry():
    """P14: mirroring the medium in x and the directions c -> -c mirrors the solution."""
    I, M = 6, 8
    rng = np.random.default_rng(21)
    sT = rng.uniform(0.5, 3.0, I * I)
    sa = 0.25 * sT
    q = rng.uniform(0, 1, I * I)
    inflow = rng.uniform(0, 1, (4, I, M))
    p = tfps.Problem(I, M, sT, sa, q, 0.4, 0.6, inflow)
    mirror_cell = lambda a: a.reshape(I, I)[:, ::-1].ravel()
    mdir = (M // 2 - 1 - np.arange(M)) % M
    inflow_m = np.zeros_like(inflow)
    inflow_m[0][:, mdir] = inflow[1]
    inflow_m[1][:, mdir] = inflow[0]
    inflow_m[2][:, mdir] = inflow[2][::-1]
    inflow_m[3][:, mdir] = inflow[3][::-1]
    pm = tfps.Problem(I, M, mirror_cell(sT), mirror_cell(sa), mirror_cell(q), 0.4, 0.6, inflow_m)
    psi = _solve(p)
    psim = _solve(pm)
    expect = np.zeros_like(psi)
    for m in range(M):
        expect[mdir[m]] = mirror_cell(psi[m])
    np.testing.assert_allclose(psim, expect, atol=1e-12)


def test_transpose_symmetry():
    """Swapping x and y (and c <-> s) transposes the solution: checks the y-type path."""
    I, M = 5, 8
    rng = np.random.default_rng(8)
    sT = rng.uniform(0.5, 3.0, I * I)
    q = rng.uniform(0, 1, I * I)
    inflow = rng.uniform(0, 1, (4, I, M))
    p = tfps.Problem(I, M, sT, 0.3 * sT, q, 0.3, 0.5, inflow)
    tr = lambda a: a.reshape(I, I).T.ravel()
    tdir = (M // 4 - 1 - np.arange(M)) % M
    inflow_t = np.zeros_like(inflow)
    for side, other in ((0, 2), (1, 3), (2, 0), (3, 1)):
        inflow_t[other][:, tdir] = inflow[side]
    pt = tfps.Problem(I, M, tr(sT), tr(0.3 * sT), tr(q), 0.3, 0.5, inflow_t)
    psi, psit = _solve(p), _solve(pt)
    expect = np.zeros_like(psi)
    for m in range(M):
        expect[tdir[m]] = tr(psi[m])
    np.testing.assert_allclose(psit, expect, atol=1e-12)


def test_P15_arnoldi_orthonormal_and_finite():
    I, M = 3, 4
    md = W.polynomial_diffusion(3, I=I, M=M)
    p = _problem(md)
    n = 2 * M * p.N
    A = lambda v: p.apply(v.reshape(2 * M, -1)).ravel()
    V, H = krylov.arnoldi(A, W.random_vector(n, 0), 30)
    assert np.abs(V @ V.T - np.eye(V.shape[0])).max() < 1e-12
    b = p.rhs().ravel()
    x, info = krylov.fgmres(A, b, lambda v, j: v, tol=1e-12, restart=n)
    assert info["converged"] and info["iters"] <= n


def test_one_cell_incoming_traces_equal_inflow():
    """I=1: every face is a boundary face; the solved incoming traces equal the inflow."""
    M = 8
    inflow = np.random.default_rng(4).uniform(0, 1, (4, 1, M))
    p = tfps.Problem(1, M, [3.0], [0.5], [0.2], 0.5, 0.3, inflow)
    x = np.linalg.solve(p.blocks()[0], p.rhs()[:, 0])
    F = p.face_values(x[:, None])
    for f in range(4):
        np.testing.assert_allclose(F[f][p.dirs[f], 0], inflow[f, 0, p.dirs[f]], atol=1e-13)
