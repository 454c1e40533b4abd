"""Seeded synthetic inputs for the radiative-transfer solver.

This module holds no arithmetic of the method itself: it only draws media,
sources, inflow data, right-hand sides and network weights from seeded random
number generators, with the shapes and value distributions of the paper's
workloads (Sec. 4) and of the benchmark configurations below.  Both the CUDA
path and the CPU checker take their inputs from here.

All per-cell arrays are float64 of shape (I*I,), cell c = iy*I + ix, cell
(iy, ix) covering [ix h, (ix+1) h] x [iy h, (iy+1) h], h = 1/I.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Medium:
    """One RTE instance: grid, directions and cell-averaged data."""
    I: int
    M: int
    sigma_T: np.ndarray
    sigma_a: np.ndarray
    q: np.ndarray
    eps: np.ndarray          # per cell
    g: float
    inflow: np.ndarray       # (4, I, M): side W,E,S,N / face along side / direction

    @property
    def n(self) -> int:
        return 2 * self.M * self.I * self.I


def _gauss3():
    x = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    w = np.array([5.0, 8.0, 5.0]) / 18.0
    return 0.5 * (x + 1.0), w          # nodes on [0, 1], weights sum to 1


def cell_average(I: int, fn) -> np.ndarray:
    """Average of fn(x, y) over every cell by 3x3 Gauss-Legendre (exact to degree 5)."""
    t, w = _gauss3()
    h = 1.0 / I
    iy, ix = np.divmod(np.arange(I * I), I)
    out = np.zeros(I * I)
    for a in range(3):
        for b in range(3):
            x = (ix + t[a]) * h
            y = (iy + t[b]) * h
            out += w[a] * w[b] * fn(x, y)
    return out


def checkerboard_sigma_T(I: int, blocks: int = 4, values=(1.0, 10.0), seed: int = 0):
    """sigma_T constant on a blocks x blocks arrangement of equal squares, each drawn from values."""
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(values), size=(blocks, blocks))
    iy, ix = np.divmod(np.arange(I * I), I)
    by = iy * blocks // I
    bx = ix * blocks // I
    return np.asarray(values, np.float64)[pick[by, bx]]


def gaussian_field(I: int, ell: float, seed: int = 0) -> np.ndarray:
    """Stationary Gaussian field at cell centres: mean 0, unit sample std,
    squared-exponential covariance exp(-r^2 / (2 ell^2)), by FFT filtering of
    white noise on a 2x zero-padded periodic grid."""
    rng = np.random.default_rng(seed)
    P = 2 * I
    noise = rng.standard_normal((P, P))
    k = np.fft.fftfreq(P, d=1.0 / I)            # frequencies for spacing h = 1/I
    kx, ky = np.meshgrid(k, k, indexing="xy")
    spec = np.exp(-0.5 * (2.0 * np.pi * ell) ** 2 * (kx ** 2 + ky ** 2))
    field = np.real(np.fft.ifft2(np.fft.fft2(noise) * np.sqrt(spec)))[:I, :I]
    field = field - field.mean()
    field = field / field.std()
    return field.reshape(I * I)


def central_source(I: int, lo: float = 0.4, hi: float = 0.6) -> np.ndarray:
    """Cell average of the indicator of [lo, hi]^2 (partial cells fractional)."""
    h = 1.0 / I
    e = np.arange(I) * h
    frac = np.clip(np.minimum(e + h, hi) - np.maximum(e, lo), 0.0, None) / h
    return np.outer(frac, frac).reshape(I * I)


def polynomial_coefficient(I: int, rng, degree: int) -> np.ndarray:
    """(2 + sum_k cx_k (x-1/2)^k)(2 + sum_k cy_k (y-1/2)^k), c ~ U[-1, 1] (Sec. 4.1)."""
    cx = rng.uniform(-1.0, 1.0, degree + 1)
    cy = rng.uniform(-1.0, 1.0, degree + 1)

    def fn(x, y):
        px = 2.0 + sum(cx[k] * (x - 0.5) ** k for k in range(degree + 1))
        py = 2.0 + sum(cy[k] * (y - 0.5) ** k for k in range(degree + 1))
        return px * py
    return cell_average(I, fn)


def zero_inflow(I: int, M: int) -> np.ndarray:
    return np.zeros((4, I, M))


def random_inflow(I: int, M: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, (4, I, M))


# ---------------------------------------------------------------------------
# Benchmark configurations
# ---------------------------------------------------------------------------
def checkerboard_transport(seed: int = 0, I: int = 32, M: int = 16) -> Medium:
    """32x32 cells, M=16, g=0, eps=1, 4x4 blocks of sigma_T in {1, 10},
    sigma_a=0.1, q=1, zero inflow (FP64, block-Jacobi GMRES to 1e-10)."""
    N = I * I
    return Medium(I, M, checkerboard_sigma_T(I, 4, (1.0, 10.0), seed),
                  np.full(N, 0.1), np.ones(N), np.ones(N), 0.0, zero_inflow(I, M))


def grf_diffusive(seed: int = 0, I: int = 256, M: int = 64, eps: float = 1e-3,
                  g: float = 0.5, ell: float = 0.1) -> Medium:
    """256x256 cells, M=64, g=0.5, eps=1e-3, sigma_T = exp(GRF, ell=0.1),
    sigma_a = 0.05 sigma_T, q = 1 on the central 0.2 x 0.2 square, zero inflow."""
    N = I * I
    sT = np.exp(gaussian_field(I, ell, seed))
    return Medium(I, M, sT, 0.05 * sT, central_source(I), np.full(N, eps), g,
                  zero_inflow(I, M))


def training_medium(seed: int, I: int = 128, M: int = 32) -> Medium:
    """Training media: ell ~ U[0.05, 0.2], sigma_T = exp(GRF), sigma_a = rho sigma_T
    with rho log-uniform in [0.01, 0.2], eps log-uniform in [1e-4, 1e-1],
    g ~ U[0, 0.8], q = 1 on [0.4, 0.6]^2, zero inflow."""
    rng = np.random.default_rng(seed)
    ell = rng.uniform(0.05, 0.2)
    rho = np.exp(rng.uniform(np.log(0.01), np.log(0.2)))
    eps = np.exp(rng.uniform(np.log(1e-4), np.log(1e-1)))
    g = rng.uniform(0.0, 0.8)
    sT = np.exp(gaussian_field(I, ell, seed + 7919))
    N = I * I
    return Medium(I, M, sT, rho * sT, central_source(I), np.full(N, eps), g,
                  zero_inflow(I, M))


def mixed_instance(seed: int, grids=(64, 128, 256), dirs=(16, 32),
                   eps_range=(1e-4, 1.0), g_range=(0.0, 0.8)) -> Medium:
    """One instance of the mixed-size batch: I from grids, M from dirs,
    eps log-uniform in eps_range, medium as the training media."""
    rng = np.random.default_rng(seed)
    I = int(rng.choice(grids))
    M = int(rng.choice(dirs))
    ell = rng.uniform(0.05, 0.2)
    rho = np.exp(rng.uniform(np.log(0.01), np.log(0.2)))
    eps = np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1])))
    g = rng.uniform(*g_range)
    sT = np.exp(gaussian_field(I, ell, seed + 104729))
    N = I * I
    return Medium(I, M, sT, rho * sT, central_source(I), np.full(N, eps), g,
                  zero_inflow(I, M))


INTERFACE_LAYOUTS = ("diffusion left, transport right", "transport left, diffusion right",
                     "diffusion bottom, transport top", "transport bottom, diffusion top",
                     "diffusion in [0.25, 0.75]^2, transport outside", "transport in [0.25, 0.75]^2, diffusion outside")


def polynomial_medium(seed: int, regime: str = "diffusion", I: int = 32, M: int = 4, layout=None) -> Medium:
    """Paper-shaped instance (Sec. 4.1): polynomial sigma_T and sigma_a of
    degree n ~ {1..4}, sigma_T shifted so sigma_T - sigma_a >= 0.2, q = 1,
    zero inflow, and eps by regime: diffusion eps = 0.01 (c + 0.1), c ~ U[0, 1];
    transport eps = 1; interface: the diffusion eps on one part of the square
    and 1 on the rest, in one of the six layouts of INTERFACE_LAYOUTS (by cell
    centre; layout = seed mod 6 unless given)."""
    rng = np.random.default_rng(20260 + seed)
    n = int(rng.integers(1, 5))
    sT = polynomial_coefficient(I, rng, n)
    sa = polynomial_coefficient(I, rng, n)
    gap = np.min(sT - sa)
    if gap < 0.2:
        sT = sT + (0.2 - gap)
    eps_d = 0.01 * (rng.uniform(0.0, 1.0) + 0.1)
    N = I * I
    if regime == "diffusion":
        eps = np.full(N, eps_d)
    elif regime == "transport":
        eps = np.ones(N)
    elif regime == "interface":
        lay = seed % 6 if layout is None else int(layout)
        xc = (np.arange(I) + 0.5) / I
        X, Y = np.meshgrid(xc, xc)                  # X[iy, ix], cell iy * I + ix
        box = (np.abs(X - 0.5) < 0.25) & (np.abs(Y - 0.5) < 0.25)
        diff = [X < 0.5, X >= 0.5, Y < 0.5, Y >= 0.5, box, ~box][lay]
        eps = np.where(diff.ravel(), eps_d, 1.0)
    else:
        raise ValueError("regime is diffusion, transport or interface")
    return Medium(I, M, sT, sa, np.ones(N), eps, 0.0, zero_inflow(I, M))


def polynomial_diffusion(seed: int, I: int = 32, M: int = 4) -> Medium:
    """The diffusion-regime paper-shaped instance (polynomial_medium)."""
    return polynomial_medium(seed, "diffusion", I, M)


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


# ---------------------------------------------------------------------------
# MgNet / CoeffNet weights (seeded initial values, shared by both sides)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class NetShape:
    """Widths of CoeffNet and MgNet.  M: directions (2M input/output channels);
    levels: V-cycle depth; c0/cmax: MgNet width at level 0 and its cap;
    cc/ccmax: CoeffNet width at level 0 and its cap; cin: CoeffNet inputs."""
    M: int
    levels: int = 4
    c0: int = 16
    cmax: int = 128
    cc: int = 8
    ccmax: int = 32
    cin: int = 4
    act: str = "linear"      # smoother activation: "linear" or "relu"

    def width(self, l):
        return min(self.c0 * 2 ** l, self.cmax)

    def cwidth(self, l):
        return min(self.cc * 2 ** l, self.ccmax)


def param_shapes(s: NetShape):
    """Ordered (name, shape) of every parameter; conv weights [out][in][k][k],
    transposed-conv weights [in][out][k][k]."""
    out = []
    for l in range(s.levels):
        cin = s.cin if l == 0 else s.cwidth(l - 1)
        out.append((f"coef{l}.w", (s.cwidth(l), cin, 3, 3)))
        out.append((f"coef{l}.gamma", (s.cwidth(l),)))
        out.append((f"coef{l}.beta", (s.cwidth(l),)))
        out.append((f"a{l}.w", (s.width(l), s.cwidth(l))))
        out.append((f"a{l}.b", (s.width(l),)))
        out.append((f"ainv{l}.w", (s.width(l), s.cwidth(l))))
        out.append((f"ainv{l}.b", (s.width(l),)))
    out.append(("lift.w", (s.width(0), 2 * s.M)))
    for l in range(s.levels):
        out.append((f"A{l}.w", (s.width(l), s.width(l), 3, 3)))
        out.append((f"B{l}.w", (s.width(l), s.width(l), 3, 3)))
    for l in range(s.levels - 1):
        out.append((f"R{l}.w", (s.width(l + 1), s.width(l), 3, 3)))
        out.append((f"P{l}.w", (s.width(l + 1), s.width(l), 4, 4)))
    out.append(("proj.w", (2 * s.M, s.width(0))))
    return out


def init_params(s: NetShape, seed: int = 0, proj_scale: float = 0.0, vcycle_scale: float = 1.0):
    """He-style normal weights, BN gamma = 1, beta = 0, head biases 0; the
    projection starts at proj_scale (0: the network returns its input) and the
    V-cycle convolutions (A, B, R, P) are multiplied by vcycle_scale."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, shape in param_shapes(s):
        if name.endswith(".gamma"):
            v = np.ones(shape)
        elif name.endswith(".beta") or name.endswith(".b"):
            v = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else 1
            if name.startswith("P"):
                fan_in = shape[0] * 4          # transposed conv: inputs per output
            v = rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)
            if name.startswith(("a", "ainv")):
                v = v * 0.1
            if name == "proj.w":
                v = v * proj_scale
            if name[0] in "ABRP":
                v = v * vcycle_scale
        params[name] = v.astype(np.float64)
    return params
