"""FP64 reference of the optimiser arithmetic of the inverse problem (arXiv 2604.15017).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the benchmark's CPU leg, never by the
product path.  Plain numpy, written from the paper's equations:

  * Sec. 3.4: unconstrained variables clipped to [0, 1] (Eq. clip01) and scaled into admissible
    ranges (Eq. scale_phys); the clip's derivative is 1 inside (0, 1) and 0 outside
    (Eq. clip_grad).
  * Sec. 3.7: Adam with bias corrections (Eq. adam) and per-parameter learning rates
    (parameter groups), after clipping the gradient (the paper does not say which clipping:
    read here as scaling the whole gradient to a maximum global L2 norm).
  * Alg. 1 / Eq. microbatch_loss: per iteration the gradients of the micro-batch losses are
    summed, then one update is made.
"""
from __future__ import annotations

import numpy as np


def clip01(theta_u):
    """Eq. clip01."""
    return np.clip(np.asarray(theta_u, dtype=np.float64), 0.0, 1.0)


def scale_phys(theta_n, lo, hi):
    """Eq. scale_phys: theta = lo + theta_n (hi - lo)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + np.asarray(theta_n, dtype=np.float64) * (hi - lo)


def clip_grad_mask(theta_u):
    """Eq. clip_grad: d theta_n / d theta_u."""
    tu = np.asarray(theta_u, dtype=np.float64)
    return ((tu > 0.0) & (tu < 1.0)).astype(np.float64)


def grad_unconstrained(theta_u, grad_phys, lo, hi):
    """Chain rule from dL/dtheta (physical) to dL/dtheta_u through Eq. scale_phys and Eq. clip01."""
    return np.asarray(grad_phys, dtype=np.float64) * (np.asarray(hi, np.float64) - np.asarray(lo, np.float64)) \
        * clip_grad_mask(theta_u)


def clip_global_norm(g, max_norm):
    """Scale g down to L2 norm max_norm when it is longer (max_norm <= 0: unchanged)."""
    g = np.asarray(g, dtype=np.float64)
    norm = float(np.sqrt(np.sum(g * g)))
    if max_norm > 0.0 and norm > max_norm:
        return g * (max_norm / norm)
    return g


def adam_step(theta_u, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Eq. adam with the standard bias corrections; returns (theta_u, m, v).  lr is a scalar or
    one rate per parameter (parameter groups); step counts from 1."""
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    theta_u = np.asarray(theta_u, dtype=np.float64) - np.asarray(lr, dtype=np.float64) * mh / (np.sqrt(vh) + eps)
    return theta_u, m, v


def optimiser_step(theta_u, grad_phys, lo, hi, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, clip_norm=0.0):
    """One update of Alg. 1 from the summed physical gradient of the iteration's micro-batches."""
    g = clip_global_norm(grad_unconstrained(theta_u, grad_phys, lo, hi), clip_norm)
    return adam_step(theta_u, g, m, v, step, lr, beta1, beta2, eps)


def optimise(theta_u0, lo, hi, grad_fn, n_iter, lr, beta1=0.9, beta2=0.999, eps=1e-8, clip_norm=0.0):
    """Alg. 1 driven by grad_fn(theta_phys) -> (loss, summed physical gradient); returns the
    trajectories of theta_u and of the loss."""
    tu = np.asarray(theta_u0, dtype=np.float64).copy()
    m = np.zeros_like(tu)
    v = np.zeros_like(tu)
    traj, losses = [tu.copy()], []
    for k in range(1, n_iter + 1):
        loss, g = grad_fn(scale_phys(clip01(tu), lo, hi))
        losses.append(float(loss))
        tu, m, v = optimiser_step(tu, g, lo, hi, m, v, k, lr, beta1, beta2, eps, clip_norm)
        traj.append(tu.copy())
    return np.array(traj), np.array(losses)
