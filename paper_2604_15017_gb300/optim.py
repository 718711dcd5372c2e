"""Inverse problem driver: recover continuous scene parameters from a target B-mode image
(Sec. 3.4 parameterisation, Sec. 3.5 micro-batching, Sec. 3.7 optimiser, Alg. 1).

The optimiser keeps unconstrained variables theta_u on the device; every iteration maps them
to physical parameters (clip to [0, 1], scale into the admissible ranges: ``us_param_map``),
runs each micro-batch forward with its path record kept, takes the l1/l2 image loss against
that micro-batch's target and the adjoint back to dL/dtheta, sums the micro-batch gradients
(Eq. microbatch_loss) and makes one Adam step (``us_adam_step``: chain through the scale and
the clip, global-norm clipping, per-parameter learning rates for parameter groups).  Monte
Carlo seeds stay fixed per micro-batch (common random numbers), so successive iterations see
the same ray realisations.

Micro-batches are acquisitions: subsets of the transmit angles (``split_angles``: an exact
partition of the compounded acquisition) or independent realisations with a share of the rays
(``split_rays``: the stochastic split).
"""
from __future__ import annotations

import numpy as np
import torch

from . import usrt


def split_angles(acq, n_batches):
    """Micro-batches over transmit angles: round-robin subsets of acq['angles']."""
    ang = list(acq["angles"])
    out = []
    for b in range(min(n_batches, len(ang))):
        a = dict(acq)
        a["angles"] = ang[b::n_batches]
        out.append(a)
    return out


def split_rays(acq, n_batches):
    """Micro-batches over rays: n_batches acquisitions with n_rays / n_batches rays per element
    each (drawn with distinct seeds by the optimiser)."""
    out = []
    for _ in range(n_batches):
        a = dict(acq)
        a["n_rays"] = max(1, int(acq["n_rays"]) // n_batches)
        out.append(a)
    return out


class InverseProblem:
    """theta: initial physical parameters (3M + 2: c, rho, alpha per medium, A_s, f0); lo / hi:
    admissible ranges (lo == hi keeps a parameter fixed); lr: one learning rate per parameter
    (or a scalar); batches: the micro-batch acquisitions; seed: base seed (micro-batch b uses
    seed + b)."""

    def __init__(self, ctx, scene, theta, lo, hi, lr, batches, img, seed, beta1=0.9, beta2=0.999, eps=1e-8,
                 clip_norm=0.0, mode=usrt.MODE_RECORD):
        dev = ctx.device
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        n = lo.size
        self.ctx, self.scene, self.img, self.seed, self.mode = ctx, scene, img, int(seed), mode
        self.batches = list(batches)
        self.lo = torch.tensor(lo, dtype=torch.float32, device=dev)
        self.hi = torch.tensor(hi, dtype=torch.float32, device=dev)
        self.lr = torch.tensor(np.broadcast_to(np.asarray(lr, np.float64), (n,)).copy(), dtype=torch.float32, device=dev)
        span = hi - lo  # a zero-width range holds its parameter fixed (its gradient is scaled by 0)
        tu = np.divide(np.asarray(theta, dtype=np.float64) - lo, span, out=np.full(n, 0.5), where=span > 0)
        self.theta_u = torch.tensor(tu, dtype=torch.float32, device=dev)
        self.m = torch.zeros(n, dtype=torch.float32, device=dev)
        self.v = torch.zeros(n, dtype=torch.float32, device=dev)
        self.grad = torch.zeros(n, dtype=torch.float32, device=dev)
        self.theta = torch.empty(n, dtype=torch.float32, device=dev)
        self.hyper = dict(beta1=beta1, beta2=beta2, eps=eps, clip_norm=clip_norm)
        self.k = 0
        self.targets = None

    def physical(self):
        """The physical parameters the next iteration uses (host float32 array)."""
        self.ctx.param_map(self.theta_u, self.lo, self.hi, out=self.theta)
        return self.theta.cpu().numpy()

    def set_targets(self, theta_target):
        """Render each micro-batch's target image at theta_target with that micro-batch's seed."""
        self.targets = []
        for b, acq in enumerate(self.batches):
            _, bref = self.ctx.forward(self.scene, theta_target, acq, self.img, seed=self.seed + b)
            self.targets.append(bref.clone())

    def step(self):
        """One iteration of Alg. 1; returns the summed micro-batch loss (host float)."""
        th = self.physical()
        self.grad.zero_()
        loss = 0.0
        for b, acq in enumerate(self.batches):
            rf, bm = self.ctx.forward(self.scene, th, acq, self.img, seed=self.seed + b,
                                      keep_record=self.mode == usrt.MODE_RECORD)
            lb, gb = self.ctx.loss(self.img, bm, self.targets[b])
            g, _ = self.ctx.adjoint(self.scene, th, acq, self.img, self.seed + b, rf, gb, mode=self.mode)
            self.grad += g
            loss += float(lb)
        self.k += 1
        self.ctx.adam_step(self.theta_u, self.grad, self.lo, self.hi, self.lr, self.m, self.v, self.k, **self.hyper)
        return loss

    def run(self, n_iter):
        """n_iter iterations; returns the loss history."""
        return [self.step() for _ in range(n_iter)]
