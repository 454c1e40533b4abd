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
  over Arnoldi vectors alone hardly sees them, since B is small exactly there;
* or the paper's recipe (Sec. 4.1): random right-hand sides, unit white-noise
  vectors in face-flux space (random_inputs).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import rte, workloads


def random_inputs(ctx, count, seed=0):
    """The paper's recipe (Sec. 4.1): random right-hand sides, here unit
    white-noise vectors in face-flux space (float64 device vectors)."""
    import torch
    g = np.random.default_rng(seed)
    return [torch.tensor(g.standard_normal(ctx.n) / math.sqrt(ctx.n), device="cuda") for _ in range(count)]


def training_inputs(ctx, md, n_krylov=32, n_smooth=32, seed=0, noise=0.1, n_random=0):
    """List of device vectors (float64, length n) for one medium: n_krylov
    Arnoldi vectors, n_smooth residuals of smooth errors and n_random random
    right-hand sides."""
    import torch
    out = random_inputs(ctx, n_random, seed + 104729) if n_random > 0 else []
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


def train(net, ctxs, inputs, steps=600, batch=8, lr0=3e-3, seed=0, log=None, checkpoint=None, every=0,
          start_step=0):
    """Adam + cosine annealing; each step draws one medium and `batch` of its
    inputs.  checkpoint(step, net, losses) is called every `every` steps and
    after the last one.  start_step resumes a run of `steps` steps (from a
    network saved with its Adam state, MgNet.save / load): the draws of the
    earlier steps are replayed and the schedule continues at start_step.
    Returns the list of batch losses of the steps run."""
    rng = np.random.default_rng(seed)
    for _ in range(start_step):
        m = int(rng.integers(len(ctxs)))
        rng.choice(len(inputs[m]), size=min(batch, len(inputs[m])), replace=False)
    losses = []
    t0 = time.time()
    for it in range(start_step, steps):
        if checkpoint is not None and every > 0 and it % every == 0:
            checkpoint(it, net, losses)
        lr = 0.5 * lr0 * (1.0 + math.cos(math.pi * it / steps))
        m = int(rng.integers(len(ctxs)))
        pool = inputs[m]
        idx = rng.choice(len(pool), size=min(batch, len(pool)), replace=False)
        loss = net.train_step(ctxs[m], [pool[i] for i in idx], lr)
        losses.append(loss)
        if log is not None and (it % 100 == 0 or it == steps - 1):
            log(f"step {it} loss {loss:.4f} lr {lr:.2e} {time.time() - t0:.1f}s")
    if checkpoint is not None and every > 0:
        checkpoint(steps, net, losses)
    return losses


def default_shape(M, I, c0=16, cmax=64):
    """Network widths used for a grid of I x I cells with M directions: a
    V-cycle down to an 8 x 8 coarsest grid (at least one level)."""
    levels = max(1, int(round(math.log2(I))) - 2)
    return workloads.NetShape(M=M, levels=levels, c0=c0, cmax=cmax, cc=8, ccmax=32, act="linear")


def validation_loss(net, ctxs, inputs, batch=8):
    """Mean loss of the network (no update) over held-out media, `batch`
    inputs of each."""
    vals = [net.loss_grad(c, inp[:batch])[0] for c, inp in zip(ctxs, inputs)]
    return float(np.mean(vals))


def train_for(media, shape=None, steps=600, batch=8, lr0=3e-3, n_krylov=32, n_smooth=32, seed=0,
              log=None, loss="plain", delta=1e-2, val_media=None, val_every=0, curve=None, n_random=0):
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
    inputs = [training_inputs(c, md, n_krylov, n_smooth, seed + 17 * i, n_random=n_random)
              for i, (c, md) in enumerate(zip(ctxs, media))]
    check = None
    vctx = []
    if val_media:
        # held-out media (the paper's validation split): the same loss, no update
        vctx = [rte.Context.from_medium(md) for md in val_media]
        if loss == "filtered":
            for c in vctx:
                c.atfps_setup(delta)
        vin = [training_inputs(c, md, n_krylov, n_smooth, seed + 7919 + 17 * i, n_random=n_random)
               for i, (c, md) in enumerate(zip(vctx, val_media))]

        def check(it, n, so_far):
            recent = so_far[-val_every:]
            if curve is not None:
                curve.append({"step": it, "train_loss": float(np.mean(recent)) if recent else None,
                              "val_loss": validation_loss(n, vctx, vin, batch)})
    losses = train(net, ctxs, inputs, steps, batch, lr0, seed, log, checkpoint=check, every=val_every)
    for c in vctx:
        c.close()
    return net, ctxs, losses, time.time() - t0
