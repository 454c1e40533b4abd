"""Golden values (tests/golden/, each file citing its source): the closed-form
spectrum of the 4-direction isotropic eigenproblem of Eq.
discretization_2D_eigenfunc_constraint, checked against the oracle and
against the library's host eigen-solver (rte_eigenbasis, no GPU needed)."""
import os

import numpy as np
import pytest

from oracle import tfps

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows():
    rows = []
    with open(os.path.join(GOLDEN, "isotropic_m4_eigenvalues.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("axis", [0, 1])
def test_isotropic_m4_spectrum_oracle(axis):
    K = tfps.hg_matrix(4, 0.0)
    _, c, s, _ = tfps.quadrature(4)
    for om, *xs in _rows():
        xi, _ = tfps.eigenbasis(om, K, c if axis == 0 else s, axis)
        np.testing.assert_allclose(xi, xs, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("axis", [0, 1])
def test_isotropic_m4_spectrum_library(axis):
    from paper_2604_23265_gb300 import _build, rte
    _build.build()
    for om, *xs in _rows():
        xi, _ = rte.eigenbasis(4, 0.0, om, axis)
        np.testing.assert_allclose(xi, xs, rtol=1e-12, atol=1e-14)
