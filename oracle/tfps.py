"""Oracle: DOM quadrature, HG kernel, TFPS basis and the linear system A alpha = b.

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Plain float64 NumPy; every
function cites the passage of the paper it restates.

Conventions (the paper is silent or garbled on these; each is a stated reading)
------------------------------------------------------------------------------
* Grid: unit square, I x I cells, h = 1/I; cell index c = iy*I + ix, cell
  (iy, ix) = [ix h, (ix+1) h] x [iy h, (iy+1) h]  (Sec. 2.2).
* Directions: M (total, M % 4 == 0), theta_m = 2 pi (m + 1/2) / M,
  (c_m, s_m) = (cos, sin), w_m = 1/M.  M here is the paper's 4M (Sec. 2.1).
* Scaling (Eq. RTE): sigma_T_eff = sigma_T/eps, sigma_s_eff = sigma_T/eps -
  eps*sigma_a, 1 - gamma = eps^2 sigma_a / sigma_T computed directly,
  particular solution q_eff/(sigma_T_eff - sigma_s_eff) = q/sigma_a.
* Kernel matrix: kappa_mn = HG(u_m . u_n) (Eq. hg), scaled by one scalar so
  that sum_n kappa_mn w_n = 1.
* Slots of the 2M unknowns of a cell: [W-centred M/2 | E-centred M/2 |
  S-centred M/2 | N-centred M/2]; W = x-type with xi < 0, E = x-type xi > 0,
  S = y-type xi < 0, N = y-type xi > 0, each group in ascending xi.
* Rows of a cell: [W-face incoming (c_m>0) | E-face incoming (c_m<0) |
  S-face incoming (s_m>0) | N-face incoming (s_m<0)], directions ascending m.
  Each interior face's equations belong to the cell the direction enters.
* Eigenvector normalisation: l / l_p with p the lowest index such that
  |l_p| >= (1 - 1e-8) max|l|, so ||l||_inf = 1 to 1e-8 and l_p = +1 exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

FACES = ("W", "E", "S", "N")
OPP = {0: 1, 1: 0, 2: 3, 3: 2}


# --------------------------------------------------------------------------
# Sec. 2.1: quadrature and scattering kernel
# --------------------------------------------------------------------------
def quadrature(M: int):
    """Uniform directions on the circle (stated reading of Sec. 2.1 / Fig. DOM).

    Returns (theta, c, s, w).  Pinned by: tests on symmetry and sums.
    """
    if M % 4 != 0 or M <= 0:
        raise ValueError("M must be a positive multiple of 4")
    m = np.arange(M, dtype=np.float64)
    theta = 2.0 * np.pi * (m + 0.5) / M
    return theta, np.cos(theta), np.sin(theta), np.full(M, 1.0 / M)


def hg_matrix(M: int, g: float):
    """Scattering matrix K from the HG kernel (Eq. hg) on the DOM set (Eq. DORTE_2d).

    kappa_mn = (1-g^2)/(1+g^2-2g u_m.u_n)^{3/2}, then one scalar scaling so that
    sum_n kappa_mn w_n = 1 (normalisation reading).  Pinned by P1.
    """
    theta, _, _, w = quadrature(M)
    mu = np.cos(theta[:, None] - theta[None, :])
    k = (1.0 - g * g) / (1.0 + g * g - 2.0 * g * mu) ** 1.5
    rowsum = k @ w
    return k / rowsum.mean()


# --------------------------------------------------------------------------
# Sec. 2.2: local eigenproblem [gamma K W - I] l = xi C l
# --------------------------------------------------------------------------
def _normalise(l: np.ndarray) -> np.ndarray:
    """||l||_inf = 1 (Sec. 2.2): divide by the first entry within 1e-8 of the
    largest magnitude, so near-ties (symmetric directions) pick the same entry
    on any machine; that entry becomes exactly +1, ||l||_inf <= 1 + 1e-8."""
    amax = np.max(np.abs(l))
    p = int(np.nonzero(np.abs(l) >= (1.0 - 1e-8) * amax)[0][0])
    return l / l[p]


def reflection(M: int, axis: int) -> np.ndarray:
    """Direction permutation that fixes c (axis 0: theta -> -theta) or s
    (axis 1: theta -> pi - theta); it pairs the M directions without fixed points."""
    m = np.arange(M)
    return (M - 1 - m) if axis == 0 else (M // 2 - 1 - m) % M


def _pencil(one_minus_gamma, K, d, P):
    """Eigenpairs of diag(d) l = mu S l restricted to the orthonormal columns P."""
    M = K.shape[0]
    gamma = 1.0 - one_minus_gamma
    KW = K / M
    ImKW = -KW.copy()
    # diagonal of I - KW written as the sum of the off-diagonal KW entries of
    # its row (equal to 1 - KW_mm when rows of KW sum to one)
    off = KW.sum(axis=1) - np.diag(KW)
    ImKW[np.diag_indices(M)] = off
    S = P.T @ (one_minus_gamma * np.eye(M) + gamma * ImKW) @ P
    S = 0.5 * (S + S.T)
    Dg = P.T @ np.diag(d) @ P
    R = sla.cholesky(S, lower=False)          # S = R^T R
    Rinv = sla.solve_triangular(R, np.eye(S.shape[0]), lower=False)
    B = Rinv.T @ Dg @ Rinv
    B = 0.5 * (B + B.T)
    mu, Y = np.linalg.eigh(B)
    return -1.0 / mu, P @ (Rinv @ Y)


def eigenbasis(one_minus_gamma: float, K: np.ndarray, d: np.ndarray, axis: int = None):
    """Eigenpairs of (gamma K W - I) l = xi diag(d) l (Eq. discretization_2D_eigenfunc_constraint).

    d = c (x-type, xi_y = 0, axis 0) or s (y-type, xi_x = 0, axis 1).  Solved as
    the symmetric definite pencil diag(d) l = mu S l with S = I - gamma K W (SPD),
    mu = -1/xi.  The pencil commutes with the reflection of the directions that
    leaves d unchanged, so it splits into mirror-symmetric and antisymmetric
    halves (orthonormal bases (e_a +- e_R(a))/sqrt 2); each half is solved by
    Cholesky S = R^T R and the symmetric eigenproblem of R^-T D R^-1 (library
    primitives).  The split makes the basis unique where a symmetric and an
    antisymmetric mode nearly share xi.  Returns xi ascending (ties: symmetric
    first) and L (M, M) with columns the normalised eigenvectors.
    Pinned by P2, P3, P4.
    """
    M = K.shape[0]
    if axis is None:
        axis = 0 if np.allclose(d, d[reflection(M, 0)]) else 1
    Rm = reflection(M, axis)
    if not np.allclose(d, d[Rm], rtol=0, atol=1e-14):
        raise ValueError("d is not invariant under the reflection of its axis")
    a = np.array([m for m in range(M) if m < Rm[m]])
    Ps = np.zeros((M, M // 2))
    Pa = np.zeros((M, M // 2))
    Ps[a, np.arange(M // 2)] = Ps[Rm[a], np.arange(M // 2)] = np.sqrt(0.5)
    Pa[a, np.arange(M // 2)] = np.sqrt(0.5)
    Pa[Rm[a], np.arange(M // 2)] = -np.sqrt(0.5)
    xs, Ls = _pencil(one_minus_gamma, K, d, Ps)
    xa, La = _pencil(one_minus_gamma, K, d, Pa)
    xi = np.concatenate([xs, xa])
    L = np.concatenate([Ls, La], axis=1)
    L = np.stack([_normalise(L[:, k]) for k in range(M)], axis=1)
    parity = np.concatenate([np.zeros(M // 2), np.ones(M // 2)])
    order = np.lexsort((parity, xi))
    return xi[order], L[:, order]


# --------------------------------------------------------------------------
# Problem set-up (Sec. 2.2, Eqs. 2DTFPS_continuity_cond, 2DTFPS_boundary_cond)
# --------------------------------------------------------------------------
class Problem:
    """All data of one TFPS system.  Inputs are cell averages (Sec. 2.2).

    sigma_T, sigma_a, q : (I*I,) arrays, cell c = iy*I + ix
    eps : scalar or (I*I,) array
    g : HG anisotropy
    inflow : (4, I, M) array [side W,E,S,N][face along side][direction] or None
    """

    def __init__(self, I, M, sigma_T, sigma_a, q, eps, g, inflow=None):
        self.I, self.M = int(I), int(M)
        N = self.I * self.I
        self.N = N
        self.h = 1.0 / self.I
        self.sigma_T = np.asarray(sigma_T, np.float64).reshape(N)
        self.sigma_a = np.asarray(sigma_a, np.float64).reshape(N)
        self.q = np.asarray(q, np.float64).reshape(N)
        self.eps = np.broadcast_to(np.asarray(eps, np.float64), (N,)).copy()
        self.g = float(g)
        if np.any(self.sigma_a <= 0) or np.any(self.sigma_T <= 0) or np.any(self.eps <= 0):
            raise ValueError("sigma_T, sigma_a, eps must be positive")
        self.inflow = (np.zeros((4, self.I, self.M)) if inflow is None
                       else np.asarray(inflow, np.float64).reshape(4, self.I, self.M))
        # Eq. RTE scaling
        self.sT = self.sigma_T / self.eps                       # sigma_T_eff
        self.omg = self.eps ** 2 * self.sigma_a / self.sigma_T   # 1 - gamma
        self.tau = self.sT * self.h                              # optical thickness
        self.chis = self.q / self.sigma_a                        # particular solution
        self.theta, self.c, self.s, self.w = quadrature(self.M)
        self.K = hg_matrix(self.M, self.g)
        # one eigenbasis per distinct value of 1 - gamma (materials)
        vals, inv = np.unique(self.omg, return_inverse=True)
        self.mat_id = inv.reshape(N)
        self.nmat = len(vals)
        M2 = self.M // 2
        self.xi = np.zeros((self.nmat, 2 * self.M))
        self.L = np.zeros((self.nmat, self.M, 2 * self.M))
        for j, om in enumerate(vals):
            xx, Lx = eigenbasis(om, self.K, self.c, 0)
            xy, Ly = eigenbasis(om, self.K, self.s, 1)
            # slots: W (xi<0), E (xi>0), S (xi<0), N (xi>0)
            self.xi[j] = np.concatenate([xx, xy])
            self.L[j] = np.concatenate([Lx, Ly], axis=1)
            assert np.all(xx[:M2] < 0) and np.all(xx[M2:] > 0)
            assert np.all(xy[:M2] < 0) and np.all(xy[M2:] > 0)
        # incoming direction sets per face (Sec. 2.2, Eq. boundary_condition_2d)
        m = np.arange(self.M)
        self.dirs = [m[self.c > 0], m[self.c < 0], m[self.s > 0], m[self.s < 0]]
        # decay factor of each slot at each face: d[k, f, cell] (Eq. 2D_eigenfunc)
        self.dec = self._decays()

    def use_basis(self, xi, L):
        """Replace the eigenbases by given ones (same materials, same slot order).

        xi (nmat, 2M), L (nmat, M, 2M).  The operator of Eq. 2DTFPS_linear_sys
        is then assembled on exactly those eigenpairs, so an implementation that
        exports its own basis can be compared on A alone, apart from how its
        eigen-solver rounds the slowly decaying modes (whose conditioning is
        1/(1 - gamma)).  Returns self."""
        xi = np.asarray(xi, np.float64).reshape(self.nmat, 2 * self.M)
        L = np.asarray(L, np.float64).reshape(self.nmat, self.M, 2 * self.M)
        self.xi = xi.copy()
        self.L = L.copy()
        self.dec = self._decays()
        return self

    # slot k -> the face its basis function is centred at (0..3)
    def slot_face(self, k):
        return k // (self.M // 2)

    def _decays(self):
        """Value of chi_C^k at the midpoint of face f, divided by l^k (Eq. 2D_eigenfunc)."""
        M, N = self.M, self.N
        a = np.abs(self.xi[self.mat_id])            # (N, 2M)
        t = self.tau[:, None]
        full = np.exp(-t * a)
        half = np.exp(-0.5 * t * a)
        d = np.zeros((2 * M, 4, N))
        for k in range(2 * M):
            fk = self.slot_face(k)
            for f in range(4):
                if f == fk:
                    d[k, f] = 1.0
                elif f == OPP[fk]:
                    d[k, f] = full[:, k]
                else:
                    d[k, f] = half[:, k]
        return d

    def neighbour(self, f):
        """Index of the neighbour of every cell across face f, -1 at the boundary."""
        I = self.I
        iy, ix = np.divmod(np.arange(self.N), I)
        if f == 0:
            nb = np.where(ix > 0, iy * I + ix - 1, -1)
        elif f == 1:
            nb = np.where(ix < I - 1, iy * I + ix + 1, -1)
        elif f == 2:
            nb = np.where(iy > 0, (iy - 1) * I + ix, -1)
        else:
            nb = np.where(iy < I - 1, (iy + 1) * I + ix, -1)
        return nb

    def boundary_face_index(self, f):
        """Position of each cell's face f along its side of the square (for inflow)."""
        iy, ix = np.divmod(np.arange(self.N), self.I)
        return iy if f in (0, 1) else ix

    # ----------------------------------------------------------------------
    def traces(self, alpha):
        """Homogeneous face-midpoint traces T[f][m, c] = sum_k alpha_ck chi_c^k(f_mid)_m.

        alpha: (2M, N).  Restates Eq. 2DTFPS_continuity_cond's left side per face.
        """
        T = np.zeros((4, self.M, self.N))
        for f in range(4):
            coef = alpha * self.dec[:, f, :]
            for j in range(self.nmat):
                cells = np.nonzero(self.mat_id == j)[0]
                T[f][:, cells] = self.L[j] @ coef[:, cells]
        return T

    def apply(self, alpha):
        """y = A alpha (Eq. 2DTFPS_linear_sys): rows of Eqs. 2DTFPS_continuity_cond / boundary_cond.

        Interior row (C, f, m): T_{C,f,m} - T_{nbr,opp f,m}; boundary row: T_{C,f,m}.
        alpha, y : (2M, N).
        """
        M2 = self.M // 2
        T = self.traces(alpha)
        y = np.zeros((2 * self.M, self.N))
        for f in range(4):
            dirs = self.dirs[f]
            nb = self.neighbour(f)
            own = T[f][dirs, :]
            other = np.zeros_like(own)
            inside = nb >= 0
            other[:, inside] = T[OPP[f]][dirs][:, nb[inside]]
            y[f * M2:(f + 1) * M2] = own - other
        return y

    def apply_adjoint(self, y):
        """alpha = A^T y, the transpose of ``apply``."""
        M2 = self.M // 2
        U = np.zeros((4, self.M, self.N))
        for f in range(4):
            dirs = self.dirs[f]
            nb = self.neighbour(f)
            yf = y[f * M2:(f + 1) * M2]
            U[f][dirs, :] += yf
            inside = np.nonzero(nb >= 0)[0]
            np.subtract.at(U[OPP[f]], (dirs[:, None], nb[inside][None, :]), yf[:, inside])
        alpha = np.zeros((2 * self.M, self.N))
        for f in range(4):
            for j in range(self.nmat):
                cells = np.nonzero(self.mat_id == j)[0]
                alpha[:, cells] += self.dec[:, f, cells] * (self.L[j].T @ U[f][:, cells])
        return alpha

    def rhs(self):
        """b of Eq. 2DTFPS_linear_sys: particular-solution jumps and inflow data."""
        M2 = self.M // 2
        b = np.zeros((2 * self.M, self.N))
        for f in range(4):
            dirs = self.dirs[f]
            nb = self.neighbour(f)
            pos = self.boundary_face_index(f)
            inside = nb >= 0
            blk = np.zeros((M2, self.N))
            blk[:, inside] = (self.chis[nb[inside]] - self.chis[inside])[None, :]
            out = ~inside
            blk[:, out] = self.inflow[f][pos[out]][:, dirs].T - self.chis[out][None, :]
            b[f * M2:(f + 1) * M2] = blk
        return b

    def assemble(self):
        """Sparse A assembled entry by entry from the definitions (n = 2 M N)."""
        M, M2, N = self.M, self.M // 2, self.N
        n = 2 * M * N
        rows, cols, vals = [], [], []
        for f in range(4):
            dirs = self.dirs[f]
            nb = self.neighbour(f)
            for c in range(N):
                Lc = self.L[self.mat_id[c]]
                for r, m in enumerate(dirs):
                    row = (f * M2 + r) * N + c
                    for k in range(2 * M):
                        rows.append(row); cols.append(k * N + c)
                        vals.append(Lc[m, k] * self.dec[k, f, c])
                    if nb[c] >= 0:
                        o = nb[c]
                        Lo = self.L[self.mat_id[o]]
                        for k in range(2 * M):
                            rows.append(row); cols.append(k * N + o)
                            vals.append(-Lo[m, k] * self.dec[k, OPP[f], o])
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    def blocks(self):
        """Per-cell diagonal blocks G_C (N, 2M, 2M): G[c][row, k] = d/d alpha_ck of row."""
        M, M2 = self.M, self.M // 2
        G = np.zeros((self.N, 2 * M, 2 * M))
        for f in range(4):
            dirs = self.dirs[f]
            for c in range(self.N):
                Lc = self.L[self.mat_id[c]]
                G[c, f * M2:(f + 1) * M2, :] = Lc[dirs, :] * self.dec[:, f, c][None, :]
        return G

    def block_inverse(self):
        """D_C = G_C^{-1} for every cell (block Jacobi, Sec. 4; D of Eq. loss)."""
        return np.linalg.inv(self.blocks())

    def blocks_at(self, cells):
        """G_C of the given cells only, (len(cells), 2M, 2M): ``blocks`` restricted,
        for media too large to hold every block."""
        M, M2 = self.M, self.M // 2
        cells = np.asarray(cells, dtype=np.int64)
        G = np.zeros((len(cells), 2 * M, 2 * M))
        for f in range(4):
            dirs = self.dirs[f]
            for i, c in enumerate(cells):
                Lc = self.L[self.mat_id[c]]
                G[i, f * M2:(f + 1) * M2, :] = Lc[dirs, :] * self.dec[:, f, c][None, :]
        return G

    def block_jacobi_rows(self, v, cells):
        """Rows of the given cells of A D v (Sec. 4: block-Jacobi right
        preconditioning; Eq. 2DTFPS_continuity_cond / boundary_cond rows), with
        D_C = G_C^{-1} formed only for those cells and their neighbours.
        v : (2M, N).  Returns (2M, len(cells))."""
        M2 = self.M // 2
        cells = np.asarray(cells, dtype=np.int64)
        nbs = [self.neighbour(f)[cells] for f in range(4)]
        need = np.unique(np.concatenate([cells] + [nb[nb >= 0] for nb in nbs]))
        G = self.blocks_at(need)
        alpha = np.linalg.solve(G, v[:, need].T[:, :, None])[:, :, 0].T      # (2M, |need|)
        where = {int(c): i for i, c in enumerate(need)}

        def trace(f, c):
            a = alpha[:, where[int(c)]] * self.dec[:, f, c]
            return self.L[self.mat_id[c]] @ a

        y = np.zeros((2 * self.M, len(cells)))
        for f in range(4):
            dirs = self.dirs[f]
            for i, c in enumerate(cells):
                row = trace(f, c)[dirs]
                nb = nbs[f][i]
                if nb >= 0:
                    row = row - trace(OPP[f], nb)[dirs]
                y[f * M2:(f + 1) * M2, i] = row
        return y

    def reconstruct(self, alpha):
        """Angular flux at cell centres, psi[m, c] (Eq. 2DTFPS_sol at the cell centre)."""
        a = np.abs(self.xi[self.mat_id])            # (N, 2M)
        e = np.exp(-0.5 * self.tau[:, None] * a).T  # (2M, N)
        coef = alpha * e
        psi = np.zeros((self.M, self.N))
        for j in range(self.nmat):
            cells = np.nonzero(self.mat_id == j)[0]
            psi[:, cells] = self.L[j] @ coef[:, cells]
        return psi + self.chis[None, :]

    def face_values(self, alpha):
        """Full solution at every face midpoint: traces plus the particular solution."""
        return self.traces(alpha) + self.chis[None, None, :]


def block_apply(D, r):
    """z_C = D_C r_C for every cell; D (N, 2M, 2M), r (2M, N)."""
    return np.einsum("cij,jc->ic", D, r)


def block_apply_T(D, r):
    """z_C = D_C^T r_C for every cell."""
    return np.einsum("cji,jc->ic", D, r)
