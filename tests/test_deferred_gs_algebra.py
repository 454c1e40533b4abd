"""The deferred form of classical Gram-Schmidt with reorthogonalisation that
the solver's Arnoldi step uses (two passes over the basis a step), restated in
NumPy and checked against the defining relations of flexible GMRES:

  step j: z_j = M_j(u_j) with u_j = beta_{j-1} v_j + V c_j (row j not yet fixed),
          w = A z_j;
  pass 1: v_j = (u_j - V[:j] c_j) / beta_{j-1};  h1 = V[:j+1]^T w
  pass 2: w' = w - V[:j+1] h1 (into row j + 1);  h2 = V[:j+1]^T w';  nu = ||w'||^2
  column: H[:j+1, j] = (h1 + h2) / beta_{j-1},  beta_j = sqrt(nu - ||h2||^2),
          H[j+1, j] = beta_j / beta_{j-1};  c_{j+1} = h2.

With zhat_j = z_j / beta_{j-1} the relation A Zhat = V H holds with V
orthonormal, and zhat_j = v_j + V c_j / beta_{j-1} when M is the identity
(block Jacobi), the correction the solver applies to y at the cycle end.
"""
import numpy as np


def _deferred_arnoldi(A, Ms, v0, k, h1_error=0.0, rng=None):
    """h1_error > 0: the first projection carries an absolute error of that
    size times ||w|| per component, as an FP32 dot would."""
    n = A.shape[0]
    V = np.zeros((k + 1, n))
    V[0] = v0
    betas = [1.0]                  # betas[j] = beta_{j-1}
    c = np.zeros(0)
    H = np.zeros((k + 1, k))
    Z = []
    U = np.zeros((k + 1, k + 1))   # U[j, i] = c_j[i] / beta_{j-1}
    for j in range(k):
        u = V[j].copy()
        z = Ms[j] @ u
        Z.append(z)
        w = A @ z
        V[j] = (u - V[:j].T @ c) / betas[j]                       # pass 1: fix row j
        h1 = V[:j + 1] @ w
        if h1_error:
            h1 = h1 + h1_error * np.linalg.norm(w) * rng.standard_normal(j + 1)
        wp = w - V[:j + 1].T @ h1                                  # pass 2
        h2 = V[:j + 1] @ wp
        nu = wp @ wp
        bj = np.sqrt(nu - h2 @ h2)
        H[:j + 1, j] = (h1 + h2) / betas[j]
        H[j + 1, j] = bj / betas[j]
        V[j + 1] = wp                                              # u_{j+1}, fixed next step
        U[j + 1, :j + 1] = h2 / bj
        c = h2
        betas.append(bj)
    # the last row is fixed as the next step would
    V[k] = (V[k] - V[:k].T @ c) / betas[k]
    Zhat = np.array([Z[j] / betas[j] for j in range(k)])
    return V, H, Zhat, U


def test_deferred_arnoldi_relation_and_orthogonality():
    rng = np.random.default_rng(0)
    n, k = 300, 40
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    Ms = [np.eye(n) + 0.05 * rng.standard_normal((n, n)) / np.sqrt(n) for _ in range(k)]   # flexible
    v0 = rng.standard_normal(n)
    v0 /= np.linalg.norm(v0)
    V, H, Zhat, _ = _deferred_arnoldi(A, Ms, v0, k)
    assert np.abs(V @ V.T - np.eye(k + 1)).max() <= 1e-13
    assert np.abs(A @ Zhat.T - V.T @ H).max() <= 1e-12 * np.abs(A).max() * np.sqrt(n)


def test_identity_preconditioner_correction_matches_stored_vectors():
    """Block Jacobi stores no z: zhat_j = v_j + V U[j], so Zhat y = V (y + U^T y)."""
    rng = np.random.default_rng(1)
    n, k = 200, 30
    A = np.eye(n) + 0.5 * rng.standard_normal((n, n)) / np.sqrt(n)
    v0 = rng.standard_normal(n)
    v0 /= np.linalg.norm(v0)
    V, H, Zhat, U = _deferred_arnoldi(A, [np.eye(n)] * k, v0, k)
    y = rng.standard_normal(k)
    yprime = y + U[:k, :k].T @ y
    np.testing.assert_allclose(Zhat.T @ y, V[:k].T @ yprime, rtol=0, atol=1e-12)


def test_gmres_minimum_from_the_deferred_relation():
    """The least-squares step on H gives the same residual as a dense solve
    restricted to span(Zhat): ||beta e1 - H y|| = ||r0 - A Zhat y||."""
    rng = np.random.default_rng(2)
    n, k = 150, 25
    A = np.eye(n) + 0.4 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    beta = np.linalg.norm(b)
    Ms = [np.eye(n) + 0.1 * rng.standard_normal((n, n)) / np.sqrt(n) for _ in range(k)]
    V, H, Zhat, _ = _deferred_arnoldi(A, Ms, b / beta, k)
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(H, e1, rcond=None)
    r_ls = np.linalg.norm(e1 - H @ y)
    r_true = np.linalg.norm(b - A @ (Zhat.T @ y))
    assert abs(r_ls - r_true) <= 1e-10 * beta
    # and it is the minimum over span(Zhat)
    yd, *_ = np.linalg.lstsq(A @ Zhat.T, b, rcond=None)
    assert r_true <= np.linalg.norm(b - A @ Zhat.T @ yd) * (1 + 1e-8)


def test_inexact_first_projection_keeps_the_relations():
    """The solver forms h1 in FP32 (error about 1e-5 ||w||): the step subtracts
    the h1 it formed and the second projection removes what h1 missed, so
    A Zhat = V H and the orthogonality of V hold as with an exact h1."""
    rng = np.random.default_rng(3)
    n, k = 300, 40
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    Ms = [np.eye(n) + 0.05 * rng.standard_normal((n, n)) / np.sqrt(n) for _ in range(k)]
    v0 = rng.standard_normal(n)
    v0 /= np.linalg.norm(v0)
    V, H, Zhat, _ = _deferred_arnoldi(A, Ms, v0, k, h1_error=3e-5, rng=np.random.default_rng(4))
    assert np.abs(V @ V.T - np.eye(k + 1)).max() <= 1e-13
    assert np.abs(A @ Zhat.T - V.T @ H).max() <= 1e-12 * np.abs(A).max() * np.sqrt(n)
    # with one linear preconditioner the Krylov space is the exact one, so
    # the GMRES residual after k steps is too (the basis of span(Zhat) is
    # not: the preconditioner sees u_j = beta v_j + V c_j, and c_j is larger)
    Mfix = [Ms[0]] * k
    b = v0 * 3.0
    res = []
    for err in (0.0, 3e-5):
        V, H, Zhat, _ = _deferred_arnoldi(A, Mfix, v0, k, h1_error=err, rng=np.random.default_rng(6))
        e1 = np.zeros(k + 1)
        e1[0] = 3.0
        y, *_ = np.linalg.lstsq(H, e1, rcond=None)
        res.append(np.linalg.norm(b - A @ (Zhat.T @ y)))
    assert abs(res[0] - res[1]) <= 1e-9 * 3.0


def test_inexact_first_projection_near_breakdown():
    """With w nearly in the span of V (||w'|| = 1e-7 ||w||) the loss of
    orthogonality grows as (h1 error / ||w'||) times the working precision."""
    rng = np.random.default_rng(5)
    n, k = 200, 10
    Q, _ = np.linalg.qr(rng.standard_normal((n, k + 1)))
    V = Q[:, :k].T
    w = V.T @ rng.standard_normal(k) + 1e-7 * Q[:, k]
    h1 = V @ w + 3e-5 * np.linalg.norm(w) * rng.standard_normal(k)
    wp = w - V.T @ h1
    h2 = V @ wp
    wpp = wp - V.T @ h2
    v = wpp / np.linalg.norm(wpp)
    loss = np.abs(V @ v).max()
    bound = 8 * 2.0 ** -52 * np.linalg.norm(wp) / np.linalg.norm(wpp)
    assert loss <= bound
    assert abs(np.linalg.norm(wpp) - 1e-7 * np.linalg.norm(Q[:, k])) <= 1e-3 * 1e-7


def test_fp32_first_projection_error_is_about_1e5_of_w():
    """The first projection as the kernel forms it: FP32 products of the hi
    planes, summed in FP32 per lane over the lane's share of the vector (a few
    hundred products), then the lane sums in FP64.  Its error against the
    exact V^T w stays near 1e-5 ||w|| or below."""
    rng = np.random.default_rng(7)
    n, k, lanes = 1 << 18, 4, 512
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    V = Q.T
    w = rng.standard_normal(n) + V.T @ (10.0 * rng.standard_normal(k))
    Vh, wh = V.astype(np.float32), w.astype(np.float32)
    exact = V @ w
    for r in range(k):
        prod = (Vh[r] * wh).reshape(-1, lanes)          # row i: one product per lane
        acc = np.zeros(lanes, np.float32)
        for row in prod:                                 # sequential FP32 sums per lane
            acc = (acc + row).astype(np.float32)
        h1 = float(np.sum(acc.astype(np.float64)))
        assert abs(h1 - exact[r]) <= 3e-5 * np.linalg.norm(w)
