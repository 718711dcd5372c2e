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
partition of the compounded acquisition), sub-apertures of emitting elements
(``split_elements``: an exact partition too, the rays keeping their indices), or independent
realisations with a share of the rays (``split_rays``: the stochastic split).

Shape parameters (a radius, a wall thickness, ...) join the material ones through a
``ShapeModel``: a mesh generator q -> (triangles, vertex tangents d tris / d q).  Every
iteration rebuilds and re-uploads the mesh at the current q, takes the adjoint with the vertex
gradient (``us_adjoint_shape``) and contracts it with the tangents (``us_shape_param_grad``);
Adam then steps materials and shape together.
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


def split_elements(acq, n_batches):
    """Micro-batches over emitting elements: n_batches contiguous sub-apertures (tx_elem,
    n_tx_elem).  With one seed they partition the full aperture's realisation exactly (a ray
    keeps its index), so the micro-batch losses' RF adds up to the full acquisition's."""
    ne = int(acq["n_elem"])
    n_batches = max(1, min(n_batches, ne))
    bounds = [round(b * ne / n_batches) for b in range(n_batches + 1)]
    out = []
    for b in range(n_batches):
        a = dict(acq)
        a["tx_elem"], a["n_tx_elem"] = bounds[b], bounds[b + 1] - bounds[b]
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


class ShapeModel:
    """make(q) -> (tris [n_tris, 9], dtris_dq [n_shape, n_tris, 9]) for physical shape
    parameters q; the scene's media, scatterers and r_s come from the workload dict w (the
    triangle count and media must not depend on q)."""

    def __init__(self, make, w, q0):
        self.make, self.w = make, w
        self.q0 = np.atleast_1d(np.asarray(q0, dtype=np.float64))

    def upload(self, ctx, q):
        tris, dq = self.make(np.asarray(q, dtype=np.float64))
        w = self.w
        sid = ctx.upload_scene(tris, w["media"], w["M"], w["scat_pos"], w["scat_amp"], w["r_s"],
                               rough=w.get("rough", False))
        return sid, torch.tensor(np.asarray(dq), dtype=torch.float32, device=ctx.device), len(tris)


class InverseProblem:
    """theta: initial physical parameters (3M + 2: c, rho, alpha per medium, A_s, f0); lo / hi:
    admissible ranges (lo == hi keeps a parameter fixed); lr: one learning rate per parameter
    (or a scalar); batches: the micro-batch acquisitions; seed: base seed (micro-batch b uses
    seed + b).  With a ShapeModel the parameter vector continues with its shape parameters
    (theta, lo, hi and lr then cover 3M + 2 + n_shape entries) and ``scene`` is ignored: the
    mesh is rebuilt at every iteration."""

    def __init__(self, ctx, scene, theta, lo, hi, lr, batches, img, seed, beta1=0.9, beta2=0.999, eps=1e-8,
                 clip_norm=0.0, mode=usrt.MODE_RECORD, shape=None):
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
        self.losses = torch.zeros(len(self.batches), dtype=torch.float32, device=dev)  # per micro-batch
        self.theta = torch.empty(n, dtype=torch.float32, device=dev)
        self.hyper = dict(beta1=beta1, beta2=beta2, eps=eps, clip_norm=clip_norm)
        self.k = 0
        self.targets = None
        self.shape = shape
        self.n_shape = 0 if shape is None else len(shape.q0)
        self.n_mat = n - self.n_shape

    def physical(self):
        """The physical parameters the next iteration uses (host float32 array)."""
        self.ctx.param_map(self.theta_u, self.lo, self.hi, out=self.theta)
        return self.theta.cpu().numpy()

    def _scene_at(self, q):
        """(scene id, vertex tangents or None, n_tris, owned) for shape parameters q."""
        if self.shape is None:
            return self.scene, None, 0, False
        sid, dq, nt = self.shape.upload(self.ctx, q)
        return sid, dq, nt, True

    def set_targets(self, theta_target):
        """Render each micro-batch's target image at theta_target (with a ShapeModel: materials
        then shape parameters) with that micro-batch's seed."""
        theta_target = np.asarray(theta_target, dtype=np.float64)
        sid, _, _, owned = self._scene_at(theta_target[self.n_mat:])
        self.targets = []
        for b, acq in enumerate(self.batches):
            _, bref = self.ctx.forward(sid, theta_target[:self.n_mat], acq, self.img, seed=self.seed + b)
            self.targets.append(bref.clone())
        if owned:
            self.ctx.release_scene(sid)

    def step(self):
        """One iteration of Alg. 1; returns the summed micro-batch loss (host float).

        The host waits for the device twice per iteration: for the physical parameters (the
        forward call takes them from host memory) and for the summed loss at the end; the
        micro-batches' losses stay on the device until then."""
        full = self.physical()
        th = full[:self.n_mat]
        sid, dq, nt, owned = self._scene_at(full[self.n_mat:])
        self.grad.zero_()
        for b, acq in enumerate(self.batches):
            rf, bm = self.ctx.forward(sid, th, acq, self.img, seed=self.seed + b,
                                      keep_record=self.mode == usrt.MODE_RECORD)
            _, gb = self.ctx.loss(self.img, bm, self.targets[b], out=self.losses[b:b + 1])
            if dq is None:
                g, _ = self.ctx.adjoint(sid, th, acq, self.img, self.seed + b, rf, gb, mode=self.mode)
                self.grad += g
            else:
                g, gtris = self.ctx.adjoint_shape(sid, th, acq, self.img, self.seed + b, rf, gb, nt, mode=self.mode)
                self.grad[:self.n_mat] += g
                self.grad[self.n_mat:] += self.ctx.shape_param_grad(gtris, dq)
        if owned:
            self.ctx.release_scene(sid)
        self.k += 1
        self.ctx.adam_step(self.theta_u, self.grad, self.lo, self.hi, self.lr, self.m, self.v, self.k, **self.hyper)
        return float(self.losses.sum())

    def run(self, n_iter):
        """n_iter iterations; returns the loss history."""
        return [self.step() for _ in range(n_iter)]
