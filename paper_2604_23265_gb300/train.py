"""Training of the MgNet preconditioner on the GPU (Sec. 3.4, Sec. 4.1).

The network is trained with the library's own forward, backward and Adam
kernels (``MgNet.train_step``) on the physics-informed loss of Eq. loss,
||x - A D psi_d|| / ||x||, or on its ATFPS-filtered form (Eq. loss_delta,
Sec. 2.3), with the learning rate annealed by a cosine schedule (Sec. 4.1:
initial rate 1e-3 there).

Training inputs are generated by the plain solver's own operators for each
training medium:
* Arnoldi vectors of the block-Jacobi preconditioned operator B = A D (the
  vectors the classical iteration works with), and
* residuals x = B e of smooth errors e (a smooth random field, the same in
  every face-flux slot of a cell, plus 10% white noise).  These carry the
  low-frequency error components block Jacobi cannot remove; a residual loss
  over Arnoldi vectors alone hardly sees them, since B is small exactly there.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import rte, workloads


def training_inputs(ctx, md, n_krylov=32, n_smooth=32, seed=0, noise=0.1):
    """List of device vectors (float64, length n) for one medium."""
    import torch
    out = []
    if n_krylov > 0:
        V = torch.empty(n_krylov * ctx.n, dtype=torch.float64, device="cuda")
        ctx.arnoldi_basis(n_krylov, V)
        out += [V[j * ctx.n:(j + 1) * ctx.n] for j in range(n_krylov)]
    rng = np.random.default_rng(seed)
    for k in range(n_smooth):
        ell = rng.uniform(0.1, 0.4)
        base = workloads.gaussian_field(md.I, ell, seed * 1000 + k)
        e = np.tile(base, 2 * md.M) + noise * rng.standard_normal(ctx.n)
        et = torch.tensor(e, dtype=torch.float64, device="cuda")
        x = torch.empty_like(et)
        ctx.response_apply(et, x)
        out.append(x)
    return out


def train(net, ctxs, inputs, steps=600, batch=8, lr0=3e-3, seed=0, log=None):
    """Adam + cosine annealing; each step draws one medium and `batch` of its
    inputs.  Returns the list of batch losses."""
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.time()
    for it in range(steps):
        lr = 0.5 * lr0 * (1.0 + math.cos(math.pi * it / steps))
        m = int(rng.integers(len(ctxs)))
        pool = inputs[m]
        idx = rng.choice(len(pool), size=min(batch, len(pool)), replace=False)
        loss = net.train_step(ctxs[m], [pool[i] for i in idx], lr)
        losses.append(loss)
        if log is not None and (it % 100 == 0 or it == steps - 1):
            log(f"step {it} loss {loss:.4f} lr {lr:.2e} {time.time() - t0:.1f}s")
    return losses


def default_shape(M, I, c0=16, cmax=64):
    """Network widths used for a grid of I x I cells with M directions: a
    V-cycle down to an 8 x 8 coarsest grid (at least one level)."""
    levels = max(1, int(round(math.log2(I))) - 2)
    return workloads.NetShape(M=M, levels=levels, c0=c0, cmax=cmax, cc=8, ccmax=32, act="linear")


def train_for(media, shape=None, steps=600, batch=8, lr0=3e-3, n_krylov=32, n_smooth=32, seed=0,
              log=None, loss="plain", delta=1e-2):
    """Create a network for the media's (I, M), generate inputs and train it
    with the plain loss (Eq. loss) or the ATFPS-filtered one (Eq. loss_delta,
    selection threshold delta).  Returns (net, contexts, losses, seconds)."""
    I, M = media[0].I, media[0].M
    shape = shape or default_shape(M, I)
    net = rte.MgNet(shape)
    net.set_params(workloads.init_params(shape, seed=seed, proj_scale=0.0, vcycle_scale=0.5))
    t0 = time.time()
    ctxs = [rte.Context.from_medium(md) for md in media]
    if loss == "filtered":
        for c in ctxs:
            c.atfps_setup(delta)
        net.loss = rte.MgNet.FILTERED
    elif loss != "plain":
        raise ValueError("loss is 'plain' or 'filtered'")
    inputs = [training_inputs(c, md, n_krylov, n_smooth, seed + 17 * i)
              for i, (c, md) in enumerate(zip(ctxs, media))]
    losses = train(net, ctxs, inputs, steps, batch, lr0, seed, log)
    return net, ctxs, losses, time.time() - t0
