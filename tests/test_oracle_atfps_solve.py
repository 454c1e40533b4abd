"""Pins of the compressed ATFPS solve and the layer reconstruction (Sec.
2.3.3-2.3.4, Eqs. 2DAdaptiveTFPS_linear_sys, 2DAdaptive_TFPS_layer1 / layer2)
against what the mathematics fixes: delta = 0 gives the TFPS solution (P17),
a medium whose exact solution is q / sigma_a (P18), the reconstructed layers
cancel the dropped projections of every interface jump (P19: a sign or scale
slip in the layer formulas leaves them at the size of the smooth solution's),
and the O(delta) behaviour of the a-posteriori estimate (Theorem
theo:posteriori): the face values converge as delta decreases and the layers
recover them (P20)."""
import numpy as np
import pytest

from oracle import atfps, krylov, tfps
from paper_2604_23265_gb300 import workloads as W


def _prob(md):
    return tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)


def _grf(I, M, eps, seed):
    md = W.grf_diffusive(seed, I=I, M=M, eps=eps)
    md.inflow = W.random_inflow(I, M, seed + 5)
    return md


def _full(p):
    return krylov.dense_solve(p.assemble(), p.rhs().ravel()).reshape(2 * p.M, -1)


@pytest.mark.parametrize("delta", [0.3, 1e-2])
def test_compressed_system_is_square(delta):
    p = _prob(_grf(8, 8, 1e-2, 0))
    Ab, bb, keep, mask = atfps.compressed_system(p, delta)
    assert Ab.shape == (keep.size, keep.size) == (bb.size, int(mask.sum()))
    assert 0 < mask.mean() < 1


def test_P17_delta_zero_is_the_tfps_solution():
    p = _prob(_grf(8, 8, 1e-2, 1))
    full, smooth, mask = atfps.atfps_solution(p, 0.0)
    assert mask.all()
    np.testing.assert_array_equal(full, smooth)
    ref = _full(p)
    fv = p.face_values(ref)
    assert np.abs(p.face_values(full) - fv).max() <= 1e-10 * np.abs(fv).max()


def test_P18_closed_form_q_over_sigma_a():
    """Homogeneous medium, q = 1, isotropic inflow q / sigma_a: psi = q /
    sigma_a everywhere; with functions dropped (thick cells) the compressed
    solve and the layers reproduce it."""
    I, M = 8, 8
    N = I * I
    sT, sa = 20.0, 0.5
    md = W.Medium(I, M, np.full(N, sT), np.full(N, sa), np.ones(N), np.full(N, 0.05), 0.3,
                  np.full((4, I, M), 1.0 / sa))
    p = _prob(md)
    full, smooth, mask = atfps.atfps_solution(p, 1e-2)
    assert not mask.all()
    np.testing.assert_allclose(p.reconstruct(full), 1.0 / sa, rtol=1e-12)
    np.testing.assert_allclose(p.face_values(full), 1.0 / sa, rtol=1e-12)


@pytest.mark.parametrize("I,M,eps,seed,delta", [(8, 8, 1e-2, 0, 1e-2), (12, 8, 3e-2, 1, 1e-3), (16, 4, 1e-2, 2, 1e-2)])
def test_P19_layers_cancel_the_dropped_projections(I, M, eps, seed, delta):
    p = _prob(_grf(I, M, eps, seed))
    full, smooth, mask = atfps.atfps_solution(p, delta)
    big_s, big_f = 0.0, 0.0
    for (kind, cm, cp, fm, fp), js, jf in zip(atfps.interfaces(p), atfps.interface_jumps(p, smooth),
                                              atfps.interface_jumps(p, full)):
        groups, rows = ([(cm, fm), (cp, fp)], None) if kind == "in" else ([(cm, fm)], p.dirs[fm])
        E, s = atfps.interface_basis(p, groups, mask, rows)
        if s == E.shape[1]:
            continue
        big_s = max(big_s, np.abs(np.linalg.solve(E, js)[s:]).max())
        big_f = max(big_f, np.abs(np.linalg.solve(E, jf)[s:]).max())
    # what remains are the neglected traces of layers centred on other faces,
    # each at most delta times its coefficient
    assert big_f <= 2 * p.M * delta * np.abs(full).max()
    assert big_f <= 1e-2 * big_s


@pytest.mark.parametrize("I,M,eps,seed", [(8, 8, 1e-2, 0), (12, 8, 3e-2, 1)])
def test_P20_face_values_converge_with_delta(I, M, eps, seed):
    p = _prob(_grf(I, M, eps, seed))
    ref = p.face_values(_full(p))
    errs = []
    for delta in (1e-1, 1e-2, 1e-3, 1e-4):
        full, smooth, mask = atfps.atfps_solution(p, delta)
        e_full = np.abs(p.face_values(full) - ref).max()
        e_smooth = np.abs(p.face_values(smooth) - ref).max()
        assert e_full <= delta * np.abs(ref).max()           # O(delta), constant 1 on these media
        if delta <= 1e-2:
            assert e_full <= 1e-2 * e_smooth                 # the layers recover the face values
        errs.append(e_full)
    assert all(b < a for a, b in zip(errs, errs[1:]))
