"""The library's host FP64 eigen-solver (rte_eigenbasis, used by rte_setup)
against the oracle's eigen-decomposition; runs without a GPU."""
import numpy as np
import pytest

from oracle import tfps


@pytest.fixture(scope="module")
def rte():
    from paper_2604_23265_gb300 import _build, rte as mod
    _build.build()
    mod.load()
    return mod


@pytest.mark.parametrize("M,g,omg", [(4, 0.0, 0.5), (8, 0.4, 1.0), (16, 0.0, 0.1), (32, 0.5, 0.0128),
                                     (64, 0.5, 2.25e-4), (64, 0.5, 5e-8), (64, 0.9, 1e-10),
                                     (112, 0.3, 1e-3)])
@pytest.mark.parametrize("axis", [0, 1])
def test_host_eigenbasis_matches_oracle(rte, M, g, omg, axis):
    """xi and L agree up to the conditioning 2^-52/(1-gamma) of the slow modes."""
    K = tfps.hg_matrix(M, g)
    _, c, s, _ = tfps.quadrature(M)
    xo, Lo = tfps.eigenbasis(omg, K, c if axis == 0 else s, axis)
    xg, Lg = rte.eigenbasis(M, g, omg, axis)
    cond = 2.0 ** -52 / omg
    assert np.all(np.abs(xg - xo) <= (1e-12 + 8 * cond) * np.abs(xo))
    assert np.abs(Lg - Lo).max() <= 1e-12 + 8 * cond
    lhs = ((1 - omg) * K / M - np.eye(M)) @ Lg
    rhs = (c if axis == 0 else s)[:, None] * Lg * xg[None, :]
    # backward error of the Cholesky-based pencil grows like 1/(1-gamma)
    assert np.abs(lhs - rhs).max() <= 1e-12 * max(1.0, np.abs(xg).max()) + 1e-3 * cond


def test_host_eigenbasis_rejects_bad_input(rte):
    with pytest.raises(rte.RteError):
        rte.eigenbasis(6, 0.0, 0.5, 0)
    with pytest.raises(rte.RteError):
        rte.eigenbasis(8, 0.0, 0.0, 0)
