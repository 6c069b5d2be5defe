"""Learned warm start of the steady RC-LBM solve (library plumbing; the
paper solves every lattice from rest).

A WarmNet (include/lbm_nn.h; forward, backward and Adam as CUDA kernels of
the library) is trained on steady lid-driven cavities that the batched
solver itself produces, and predicts, for a new instance, initial fields
from which the unmodified scheme continues to the same steady residual.  The
rest state stays the fallback and the yardstick: the warm start is measured as
steps and wall time to the residual against the rest start.

Instances: nx x ny = n x n cells, aspect ratio a, lid speed U, Re = U n / nu,
seeded solid rectangles (<= 10 % of the cells, 2-cell fluid margin).
Per-cell network inputs (4 channels): solid flag, a, log10(Re) / 3,
U / 0.05.  Targets (3 channels): (rho - 1) c_s^2 / U^2, u_x / U, u_y / U.
The host assembles the input planes and rescales predictions (argument
marshalling); every network and solver operation runs in the library's
kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W
from .lbm import (Batch, lbm_nn_create, lbm_nn_destroy, lbm_nn_forward, lbm_nn_get_params,
                  lbm_nn_prolong, lbm_nn_set_params, lbm_nn_train_step)


def cavity_set(count, seed, n=64, a_range=(0.5, 1.0), re_range=(20.0, 200.0),
               u_range=(0.03, 0.08), coverage=0.10, tau_range=(0.55, 2.0)):
    """Seeded lid-driven cavity instances (see the module docstring).
    c_s^2 = stable_cs2(a); when tau = 1/2 + nu / c_s^2 would exceed tau_max,
    U is lowered to bring tau to tau_max; when it would fall below tau_min,
    Re is drawn again."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        a = float(rng.uniform(*a_range))
        Re = float(np.exp(rng.uniform(np.log(re_range[0]), np.log(re_range[1]))))
        U = float(rng.uniform(*u_range))
        cs2 = W.stable_cs2(a)
        nu = U * n / Re
        if 0.5 + nu / cs2 < tau_range[0]:
            continue
        if 0.5 + nu / cs2 > tau_range[1]:
            nu = (tau_range[1] - 0.5) * cs2
            U = nu * Re / n
        mask = W.random_obstacles(n, n, seed=int(rng.integers(1 << 31)), coverage=coverage)
        out.append(W.cavity(n, n, a, cs2, U, Re).with_(mask=mask))
    return out


def inputs_of(wls):
    """(count, n, n, 4) float32 input planes."""
    x = np.zeros((len(wls), wls[0].ny, wls[0].nx, 4), np.float32)
    for k, w in enumerate(wls):
        x[k, ..., 0] = 0.0 if w.mask is None else w.mask
        x[k, ..., 1] = w.a
        x[k, ..., 2] = np.log10(w.info["Re"]) / 3.0
        x[k, ..., 3] = w.info["U"] / 0.05
    return x


def targets_of(wl, rho, ux, uy):
    """Scaled steady fields; zero at solid cells (which the loss ignores)."""
    U = wl.info["U"]
    fluid = np.ones((wl.ny, wl.nx)) if wl.mask is None else (wl.mask == 0)
    t = np.stack([(rho - 1.0) * wl.cs2 / (U * U), ux / U, uy / U], axis=-1)
    return (t * fluid[..., None]).astype(np.float32)


def fields_of(wl, y):
    """Predicted (rho, ux, uy) of one instance from its network output."""
    U = wl.info["U"]
    rho = 1.0 + y[..., 0].astype(np.float64) * U * U / wl.cs2
    return rho, y[..., 1].astype(np.float64) * U, y[..., 2].astype(np.float64) * U


def coarsen(x, t, fluid, factor):
    """Inputs, targets and fluid flags of a network working on a grid
    `factor` times coarser than the instances (data preparation; the network
    sees the whole cavity within its receptive field): inputs averaged over
    factor x factor blocks (channel 0 becomes the block's solid fraction, so a
    coarse cell is fluid where less than half of its block is solid), targets
    averaged over the block's fluid cells."""
    if factor == 1:
        return x, t, fluid
    xc = coarsen_inputs(x, factor)
    n, H, W, _ = x.shape
    h, w = H // factor, W // factor
    blk = lambda a: a.reshape(n, h, factor, w, factor, *a.shape[3:])
    fl = blk(fluid.astype(np.float64))
    cnt = fl.sum(axis=(2, 4))
    tc = (blk(t) * fl[..., None]).sum(axis=(2, 4)) / np.maximum(cnt, 1.0)[..., None]
    flc = (xc[..., 0] < 0.5).astype(np.uint8)
    return xc, (tc * flc[..., None]).astype(np.float32), flc


def coarsen_inputs(x, factor):
    """Input planes averaged over factor x factor blocks (see coarsen)."""
    n, H, W, c = x.shape
    if factor < 1 or H % factor or W % factor:
        raise ValueError(f"{H} x {W} instances do not split into {factor} x {factor} blocks")
    if factor == 1:
        return x
    return x.reshape(n, H // factor, factor, W // factor, factor, c).mean(axis=(2, 4)).astype(
        np.float32)


def fluid_of(wls):
    return np.stack([(w.mask == 0) if w.mask is not None else np.ones((w.ny, w.nx), bool)
                     for w in wls]).astype(np.uint8)


def solve(wls, tol=1e-8, check=100, max_steps=400_000, inits=None, stream=None, tune=False):
    """Runs every instance to a steady residual <= tol in one batch (the
    residual of two-step mean velocities, lbm_batch_residuals).  inits: None
    (rest) or one (rho, ux, uy) per instance.  Returns the batch result:
    residuals, steps per instance, wall seconds, final fields, and the mean
    of the final fields and those one step later (which cancels the
    alternating motion of the scheme's staggered invariants)."""
    t0 = time.perf_counter()
    b = Batch(wls, stream=stream)
    try:
        if inits is not None:
            for k, (r, u, v) in enumerate(inits):
                b.init_fields(k, r, u, v)
        if tune:
            b.tune(trial_steps=5)
        st, res = b.run(tol, check_every=check, max_steps=max_steps)
        steps = np.array([b.step_count(k) for k in range(len(wls))])
        secs = time.perf_counter() - t0
        fields = [b.moments(k) for k in range(len(wls))]
        for k in range(len(wls)):
            b.set_active(k, True)
        b.step(1)
        mean = [tuple(0.5 * (a + c) for a, c in zip(fields[k], b.moments(k)))
                for k in range(len(wls))]
    finally:
        b.close()
    return {"status": st, "residual": res, "steps": steps, "seconds": secs, "fields": fields,
            "mean_fields": mean}


class WarmStart:
    """A WarmNet on the GPU with its training loop."""

    def __init__(self, channels=(32, 64, 128, 256), n=64, max_batch=16, seed=0, stream=None):
        self.channels = list(channels)
        self.n = n
        self.max_batch = max_batch
        self.nn = lbm_nn_create(self.channels, max_batch, n, n, seed=seed, stream=stream)

    def close(self):
        if getattr(self, "nn", None):
            lbm_nn_destroy(self.nn)
            self.nn = None

    def __del__(self):
        self.close()

    def params(self):
        return lbm_nn_get_params(self.nn)

    def set_params(self, p):
        lbm_nn_set_params(self.nn, p)

    def predict(self, x):
        out = []
        for i in range(0, len(x), self.max_batch):
            out.append(lbm_nn_forward(self.nn, x[i:i + self.max_batch]))
        return np.concatenate(out)

    def predict_fine(self, x, fluid, factor):
        """Predictions for instances `factor` times finer than the network's
        grid: the network on the block-averaged inputs, then its outputs
        prolonged to the instances' grid and put through the output stage
        there (lbm_nn_prolong, on the GPU).  x: the instances' input planes;
        fluid: their fluid flags."""
        if factor == 1:
            return self.predict(x)
        xc = coarsen_inputs(x, factor)
        out = []
        for i in range(0, len(x), self.max_batch):
            y = lbm_nn_forward(self.nn, xc[i:i + self.max_batch])
            out.append(lbm_nn_prolong(self.nn, y, factor, fluid[i:i + self.max_batch]))
        return np.concatenate(out)

    def train(self, x, t, fluid, epochs, lr=1e-3, seed=0, lr_final=None):
        """Adam over shuffled mini-batches; returns the mean loss per epoch.
        The learning rate decays geometrically to lr_final (default lr / 10)."""
        rng = np.random.default_rng(seed)
        lr_final = lr / 10.0 if lr_final is None else lr_final
        hist = []
        nb = (len(x) + self.max_batch - 1) // self.max_batch
        total = max(1, epochs * nb - 1)
        step = 0
        for _ in range(epochs):
            order = rng.permutation(len(x))
            losses = []
            for i in range(0, len(x), self.max_batch):
                idx = order[i:i + self.max_batch]
                rate = lr * (lr_final / lr) ** (step / total)
                losses.append(lbm_nn_train_step(self.nn, x[idx], t[idx], fluid[idx], rate))
                step += 1
            hist.append(float(np.mean(losses)))
        return hist


def build_dataset(count, seed, n=64, tol=1e-8, max_steps=400_000, stream=None):
    """Steady states of `count` seeded instances from the batched solver,
    keeping those that reached the residual: (instances, inputs, targets,
    fluid, solve result of all instances)."""
    wls = cavity_set(count, seed, n=n)
    res = solve(wls, tol=tol, max_steps=max_steps, stream=stream)
    r = res["residual"]
    keep = [k for k in range(len(wls)) if 0.0 <= r[k] <= tol]
    kw = [wls[k] for k in keep]
    t = np.stack([targets_of(wls[k], *res["mean_fields"][k]) for k in keep])
    return kw, inputs_of(kw), t, fluid_of(kw), res
