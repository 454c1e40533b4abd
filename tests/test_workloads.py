"""Host-side checks of the seeded media generators of the paper's regimes
(Sec. 4.1): the diffusion regime is the generator used since the start, the
transport regime has eps = 1, and the six sharp-interface layouts put the
diffusive eps exactly on their region; every medium satisfies the paper's
constraints (sigma_a > 0, sigma_T - sigma_a >= 0.2)."""
import numpy as np
import pytest

from paper_2604_23265_gb300 import workloads as W


def test_diffusion_regime_is_the_paper_generator():
    for s in range(5):
        a, b = W.polynomial_diffusion(s), W.polynomial_medium(s, "diffusion")
        for f in ("sigma_T", "sigma_a", "q", "eps"):
            np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
        assert np.all(a.eps == a.eps[0]) and 0.001 <= a.eps[0] <= 0.011


@pytest.mark.parametrize("layout", range(6))
def test_interface_layouts(layout):
    I = 32
    md = W.polynomial_medium(7, "interface", I=I, layout=layout)
    diff = (md.eps < 1).reshape(I, I)                  # [iy][ix]
    assert np.all(md.eps[md.eps < 1] == md.eps[md.eps < 1][0])
    half = np.zeros((I, I), bool)
    if layout in (0, 1):
        half[:, :I // 2] = True                        # x < 1/2
    elif layout in (2, 3):
        half[:I // 2, :] = True                        # y < 1/2
    else:
        half[I // 4:3 * I // 4, I // 4:3 * I // 4] = True
    expect = half if layout in (0, 2, 4) else ~half
    np.testing.assert_array_equal(diff, expect)


@pytest.mark.parametrize("regime", ["diffusion", "transport", "interface"])
def test_paper_constraints(regime):
    for s in range(8):
        md = W.polynomial_medium(s, regime)
        assert np.all(md.sigma_a > 0) and np.all(md.sigma_T - md.sigma_a >= 0.2 - 1e-12)
        assert np.all(md.eps > 0) and np.all(md.eps <= 1)
        if regime == "transport":
            assert np.all(md.eps == 1.0)
    with pytest.raises(ValueError):
        W.polynomial_medium(0, "sharp")
