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
