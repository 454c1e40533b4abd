"""Oracle: ATFPS filtering of the physics-informed loss (Sec. 2.3, Eq. loss_delta).

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Float64 NumPy/SciPy.

Steps, in the paper's order:
* selection (Eq. def_V_delta): basis function k of cell C is kept iff
  exp(-|xi_k| sigma_T,C h / 2) > delta (the garbled lambda of that equation is
  read as xi);
* interface bases (Sec. 2.3.2): for an interior interface the kept functions
  centred there (C- then C+, each in ascending |xi|) are orthonormalised by a
  Householder QR (sign: diag(R) > 0), the dropped ones are appended (C- then
  C+, ascending |xi|), and every column is scaled to max-norm one; on the
  boundary the same is done with the incoming components only;
* projections P^k (Sec. 2.3.2): coordinates of a vector in that basis;
* ATFPS rows (Eqs. 2DAdaptiveTFPS_continuity_cond / boundary_cond): the
  projections, onto the kept coordinates, of the midpoint jump of the solution
  built from the kept functions only;
* filtered loss (Eq. loss_delta): with the network input r as right-hand side
  (the paper's "directly using the network input") and D_delta = mask o D,
  loss_delta = ||F (A (mask o D psi_d) - r)|| / ||r||, F the stacked kept
  projections of every interface.  The jump across an interior interface,
  T_{C-} - T_{C+} over all M directions, is read off the rows of A: the rows
  of C+ entering through the shared face carry -(jump), those of C- carry
  +(jump).
Pinned by P12 (transport regime: nothing is dropped), P13 (delta = 0: the
projection is diag(||q||_inf) Q^T), basis invariants and finite differences.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import mgnet, tfps


def selection(p: "tfps.Problem", delta: float) -> np.ndarray:
    """mask[k, c]: basis function k of cell c is kept (Eq. def_V_delta)."""
    a = np.abs(p.xi[p.mat_id])                       # (N, 2M)
    return (np.exp(-0.5 * a * p.tau[:, None]) > delta).T


def _qr_pos(S):
    """Householder QR (library primitive) with the signs of R's diagonal made positive."""
    Q, R = np.linalg.qr(S, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn[None, :]


def interface_basis(p, cells_groups, mask, rows=None):
    """E (columns: orthonormalised kept functions, then dropped ones, each
    max-norm one) and the number s of kept columns for one interface.

    cells_groups: [(cell, slot group), ...] -- the functions centred at the
    interface (C- first).  rows: direction subset (incoming components on a
    boundary) or None for all M directions.
    """
    M2 = p.M // 2
    kept, dropped = [], []
    for c, grp in cells_groups:
        slots = grp * M2 + np.arange(M2)
        order = slots[np.argsort(np.abs(p.xi[p.mat_id[c]][slots]), kind="stable")]
        Lc = p.L[p.mat_id[c]]
        for k in order:
            col = Lc[:, k] if rows is None else Lc[rows, k]
            (kept if mask[k, c] else dropped).append(col)
    s = len(kept)
    cols = []
    if s:
        cols.append(_qr_pos(np.stack(kept, axis=1)))
    if dropped:
        cols.append(np.stack(dropped, axis=1))
    E = np.concatenate(cols, axis=1)
    E = E / np.abs(E).max(axis=0, keepdims=True)
    return E, s


def interfaces(p):
    """Every interface as (kind, C-, C+, face of C- , face of C+):
    interior vertical (C- left, C+ right), interior horizontal (C- below,
    C+ above), and boundary faces (C+ = -1)."""
    I = p.I
    out = []
    for iy in range(I):
        for ix in range(I - 1):
            out.append(("in", iy * I + ix, iy * I + ix + 1, 1, 0))
    for iy in range(I - 1):
        for ix in range(I):
            out.append(("in", iy * I + ix, (iy + 1) * I + ix, 3, 2))
    for iy in range(I):
        out.append(("bd", iy * I, -1, 0, -1))
        out.append(("bd", iy * I + I - 1, -1, 1, -1))
    for ix in range(I):
        out.append(("bd", ix, -1, 2, -1))
        out.append(("bd", (I - 1) * I + ix, -1, 3, -1))
    return out


def filter_operator(p, delta, cond_max=1e12):
    """Sparse F (kept coordinates x n) mapping a row-space vector y (rows of A)
    to the kept interface projections, and the selection mask."""
    mask = selection(p, delta)
    M, M2, N = p.M, p.M // 2, p.N
    pos = {}
    for f in range(4):
        for j, m in enumerate(p.dirs[f]):
            pos[(f, m)] = j
    rows, cols, vals = [], [], []
    r0 = 0
    for kind, cm, cp, fm, fp in interfaces(p):
        if kind == "in":
            E, s = interface_basis(p, [(cm, fm), (cp, fp)], mask)
            if s == 0:
                continue
            if np.linalg.cond(E) > cond_max:
                raise np.linalg.LinAlgError("interface basis is singular")
            Einv = np.linalg.inv(E)[:s]              # kept coordinates
            # jump J[m] = T_{C-} - T_{C+}: rows of C- (face fm, m entering C-)
            # carry +J[m]; rows of C+ (face fp, m entering C+) carry -J[m]
            for m in range(M):
                if (fm, m) in pos:
                    col = (fm * M2 + pos[(fm, m)]) * N + cm
                    sign = 1.0
                else:
                    col = (fp * M2 + pos[(fp, m)]) * N + cp
                    sign = -1.0
                for k in range(s):
                    rows.append(r0 + k); cols.append(col); vals.append(sign * Einv[k, m])
            r0 += s
        else:
            dirs = p.dirs[fm]
            E, s = interface_basis(p, [(cm, fm)], mask, rows=dirs)
            if s == 0:
                continue
            if np.linalg.cond(E) > cond_max:
                raise np.linalg.LinAlgError("interface basis is singular")
            Einv = np.linalg.inv(E)[:s]
            for jj in range(len(dirs)):
                col = (fm * M2 + jj) * N + cm
                for k in range(s):
                    rows.append(r0 + k); cols.append(col); vals.append(Einv[k, jj])
            r0 += s
    F = sp.csr_matrix((vals, (rows, cols)), shape=(r0, 2 * M * N))
    return F, mask


def filtered_residual(p, D, F, mask, psi, r):
    """F (A (mask o D psi) - r): the ATFPS residual of Eq. loss_delta."""
    alpha = tfps.block_apply(D, psi.reshape(2 * p.M, -1)) * mask
    return F @ (p.apply(alpha).ravel() - r)


def loss_and_grad_filtered(params, shape, problems, Ds, Fs, masks, coeff_xs, rs):
    """Eq. loss_delta averaged over a batch, ||F(A D_delta psi_d - x)|| / ||x||,
    x = r / rms(r), with its gradient for every network parameter."""
    Bn = len(rs)
    M = shape.M
    I = problems[0].I
    xs = [r / np.sqrt(np.mean(r * r)) for r in rs]
    X = np.stack([x.reshape(2 * M, I, I) for x in xs])
    t, ids = mgnet.forward(params, shape, np.stack(coeff_xs), X)
    psi = t.v(ids["psi"])
    total = 0.0
    gpsi = np.zeros_like(psi)
    for b in range(Bn):
        p, D, F, mask = problems[b], Ds[b], Fs[b], masks[b]
        res = filtered_residual(p, D, F, mask, psi[b].ravel(), xs[b])
        nr, nx = np.linalg.norm(res), np.linalg.norm(xs[b])
        total += nr / nx / Bn
        if nr > 0:
            u = (F.T @ res).reshape(2 * M, -1)
            g = tfps.block_apply_T(D, p.apply_adjoint(u) * mask)
            gpsi[b] = (g / (nr * nx * Bn)).reshape(2 * M, I, I)
    grads = t.backward(ids["psi"], gpsi)
    P = ids["params"]
    return total, {k: grads[i] if grads[i] is not None else np.zeros_like(params[k])
                   for k, i in P.items()}


# ------------------------------------------------------------------ compressed solve
# Sec. 2.3.3 (Eq. 2DAdaptiveTFPS_linear_sys) and Sec. 2.3.4 (Eqs.
# 2DAdaptive_TFPS_layer1 / layer2).  Pinned by P17 (delta = 0: the compressed
# solution is the TFPS solution), P18 (closed form q / sigma_a), P19 (the
# reconstructed layers cancel the dropped projections of every interface jump
# up to the neglected cross-face terms; a wrong sign doubles them) and P20
# (accuracy improves as delta decreases; layers recover the face values).


def interface_columns(p, cells_groups, mask, rows=None):
    """The functions behind the columns of ``interface_basis``'s E, in the
    same order (kept, then dropped): (cell, slot, side, scale) with side 0
    for C- (or the boundary cell) and 1 for C+, and scale the max-norm the
    column had before E's scaling to one (the dropped columns are l^k itself,
    restricted to the incoming rows on a boundary)."""
    M2 = p.M // 2
    kept, dropped = [], []
    for side, (c, grp) in enumerate(cells_groups):
        slots = grp * M2 + np.arange(M2)
        order = slots[np.argsort(np.abs(p.xi[p.mat_id[c]][slots]), kind="stable")]
        Lc = p.L[p.mat_id[c]]
        for k in order:
            col = Lc[:, k] if rows is None else Lc[rows, k]
            (kept if mask[k, c] else dropped).append((c, int(k), side, float(np.abs(col).max())))
    return kept + dropped


def compressed_system(p, delta):
    """Eq. 2DAdaptiveTFPS_linear_sys: the rows are the kept projections of
    every interface jump (Eqs. 2DAdaptiveTFPS_continuity_cond / boundary_cond,
    F of ``filter_operator``) of the solution built from the kept functions
    only; the unknowns are the kept coefficients in [2M][N] order.  Returns
    (A_bar, b_bar, keep, mask): A_bar = F A[:, keep], b_bar = F b."""
    F, mask = filter_operator(p, delta)
    keep = np.flatnonzero(mask.ravel())
    A = p.assemble().tocsc()
    return (F @ A[:, keep]).tocsr(), F @ p.rhs().ravel(), keep, mask


def compressed_solve(p, delta):
    """The smooth coefficients: the compressed system solved by dense LU,
    scattered into [2M][N] with zeros at the dropped functions."""
    from . import krylov
    Ab, bb, keep, mask = compressed_system(p, delta)
    alpha = np.zeros(2 * p.M * p.N)
    alpha[keep] = krylov.dense_solve(Ab, bb)
    return alpha.reshape(2 * p.M, p.N), mask


def interface_jumps(p, alpha):
    """Per interface (``interfaces`` order) the midpoint jump of the solution
    built from alpha: psi_{C-} - psi_{C+} over all M directions on an interior
    interface, psi_C - inflow over the incoming directions on a boundary,
    read off the rows of A alpha - b (rows of C- carry +jump, of C+ -jump)."""
    M2 = p.M // 2
    y = p.apply(alpha) - p.rhs()
    pos = {(f, m): j for f in range(4) for j, m in enumerate(p.dirs[f])}
    out = []
    for kind, cm, cp, fm, fp in interfaces(p):
        if kind == "in":
            J = np.empty(p.M)
            for m in range(p.M):
                if (fm, m) in pos:
                    J[m] = y[fm * M2 + pos[(fm, m)], cm]
                else:
                    J[m] = -y[fp * M2 + pos[(fp, m)], cp]
        else:
            J = y[fm * M2:(fm + 1) * M2, cm].copy()
        out.append(J)
    return out


def layer_reconstruction(p, alpha_smooth, mask):
    """Eqs. 2DAdaptive_TFPS_layer1 / layer2: every dropped coefficient from
    the dropped projection of its interface's jump of the smooth solution,
    alpha_{C-}^k = P^k(psi_{C+} - psi_{C-}), alpha_{C+}^k = P^k(psi_{C-} -
    psi_{C+}), on a boundary alpha_C^k = P^k(inflow - psi_C); P^k l^k = 1 is
    read as the coordinate in the basis of unit max-norm columns divided by
    the column's scale."""
    alpha = np.array(alpha_smooth, dtype=np.float64, copy=True)
    for (kind, cm, cp, fm, fp), J in zip(interfaces(p), interface_jumps(p, alpha_smooth)):
        if kind == "in":
            groups, rows = [(cm, fm), (cp, fp)], None
        else:
            groups, rows = [(cm, fm)], p.dirs[fm]
        E, s = interface_basis(p, groups, mask, rows=rows)
        cols = interface_columns(p, groups, mask, rows=rows)
        if s == len(cols):
            continue
        beta = np.linalg.solve(E, J)[s:]
        for b, (c, k, side, scale) in zip(beta, cols[s:]):
            alpha[k, c] = (-b if side == 0 else b) / scale
    return alpha


def atfps_solution(p, delta):
    """(alpha_delta with layers, alpha_smooth, mask): the compressed solve
    followed by the layer reconstruction."""
    smooth, mask = compressed_solve(p, delta)
    return layer_reconstruction(p, smooth, mask), smooth, mask
