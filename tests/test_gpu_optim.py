"""Inverse problem on the GPU (Sec. 3.4, 3.5, 3.7, Alg. 1) against the optimiser oracle.

* the parameter map and the Adam step kernels against ``oracle.optim`` over several steps,
  with saturated parameters, two learning-rate groups and norm clipping (FP32 vs FP64: 1e-5
  relative of the step size);
* a micro-batched inverse run driven by the CUDA path against the same run driven by the FP64
  oracle's forward and gradient (losses within 5 %, the B-mode tolerance carried into a mean
  squared dB error; parameters within a fifth of a learning rate on every component whose
  gradient is not lost in Monte Carlo noise);
* a sim-to-sim recovery of a few parameters: the loss falls and they move toward the target.
"""
import numpy as np
import pytest
import torch

from oracle import optim as OP
from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_15017_gb300 import usrt

    c = usrt.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def test_param_map_and_adam_step_match_the_oracle(ctx):
    rng = np.random.default_rng(5)
    n = 38
    lo = rng.uniform(0.5, 1.0, n)
    hi = lo + rng.uniform(0.5, 2.0, n)
    tu = rng.uniform(-0.2, 1.2, n)  # some saturated at either bound
    lr = np.where(np.arange(n) < 20, 0.05, 0.01)
    tu_d, lo_d, hi_d, lr_d = dev(tu), dev(lo), dev(hi), dev(lr)
    th = ctx.param_map(tu_d, lo_d, hi_d)
    assert np.allclose(th.cpu().numpy(), OP.scale_phys(OP.clip01(tu), lo, hi), rtol=1e-6)
    m, v = np.zeros(n), np.zeros(n)
    m_d, v_d = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    tu_ref = tu.astype(np.float32).astype(np.float64)
    for k in range(1, 6):
        g = rng.normal(size=n).astype(np.float32).astype(np.float64) * 10.0
        clip = 5.0 if k % 2 else 0.0
        ctx.adam_step(tu_d, dev(g), lo_d, hi_d, lr_d, m_d, v_d, k, clip_norm=clip)
        tu_ref, m, v = OP.optimiser_step(tu_ref, g, lo, hi, m, v, k, lr, clip_norm=clip)
        got = tu_d.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - tu_ref) <= 1e-5 * lr + 1e-7), (k, np.abs(got - tu_ref).max())


def _oracle_grad_fn(w, batches, seed, targets):
    def fn(theta):
        loss, grad = 0.0, np.zeros(len(theta))
        for b, acq in enumerate(batches):
            wb = dict(w, acq=acq)
            ref = O.forward(wb, seed=seed + b, theta=theta)
            lb, gb = O.loss(w["img"], ref["b"], targets[b])
            grf = O.bmode_vjp(acq, w["img"], ref["rf"], gb)
            loss += lb
            grad += ref["run"].gradient(grf)
        return loss, grad
    return fn


def test_micro_batched_inverse_run_matches_the_oracle_driven_run(ctx):
    from paper_2604_15017_gb300 import optim

    w = P.slab_scatterers(n_rays=800)
    sid = ctx.upload_workload(w)
    th0 = np.asarray(w["theta"], np.float64)
    lo, hi = 0.8 * th0, 1.2 * th0
    batches = optim.split_rays(w["acq"], 2)
    lr = 0.05
    prob = optim.InverseProblem(ctx, sid, th0, lo, hi, lr, batches, w["img"], seed=w["seed"])
    prob.set_targets(w["theta_target"])
    targets = [O.forward(dict(w, acq=a), seed=w["seed"] + b, theta=w["theta_target"])["b"] for b, a in enumerate(batches)]
    fn = _oracle_grad_fn(w, batches, w["seed"], targets)
    n_iter = 3
    losses = [prob.step() for _ in range(n_iter)]
    traj, ref_losses = OP.optimise((th0 - lo) / (hi - lo), lo, hi, fn, n_iter, lr)
    assert np.allclose(losses, ref_losses, rtol=5e-2), (losses, ref_losses)
    # components whose oracle gradient stands clear of the Monte Carlo noise at every iteration
    grads = []
    for k in range(n_iter):
        grads.append(fn(OP.scale_phys(OP.clip01(traj[k]), lo, hi))[1] * (hi - lo))
    grads = np.abs(np.array(grads))
    clear = np.all(grads >= 1e-2 * grads.max(axis=1, keepdims=True), axis=0)
    assert clear.sum() >= 3
    got = prob.theta_u.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - traj[-1])[clear] <= 0.2 * lr), np.c_[got, traj[-1], clear]
    ctx.release_scene(sid)


def test_sim_to_sim_recovery_of_densities_attenuation_and_scatter_amplitude(ctx):
    """Sound speeds and f0 held fixed (zero-width ranges), the target made with the slab's
    density and attenuation and the scatter amplitude off by 5-10 %: the loss falls and the
    free parameters move toward the target."""
    from paper_2604_15017_gb300 import optim

    w = P.slab_scatterers(n_rays=1500)
    sid = ctx.upload_workload(w)
    th0 = np.asarray(w["theta"], np.float64)
    M = w["M"]
    free = np.array([4, 5, 3 * M])  # rho and alpha of the slab, A_s
    tgt = th0.copy()
    tgt[free] *= np.array([1.05, 0.9, 1.1])
    lo, hi = th0.copy(), th0.copy()
    lo[free], hi[free] = 0.8 * th0[free], 1.2 * th0[free]
    prob = optim.InverseProblem(ctx, sid, th0, lo, hi, 0.02, optim.split_rays(w["acq"], 2), w["img"], seed=w["seed"])
    prob.set_targets(tgt)
    losses = prob.run(25)
    th = prob.physical().astype(np.float64)
    assert losses[-1] < 0.3 * losses[0], losses
    assert np.all(np.abs(th[free] - tgt[free]) < np.abs(th0[free] - tgt[free])), np.c_[th[free], tgt[free], th0[free]]
    fixed = np.setdiff1d(np.arange(len(th0)), free)
    assert np.allclose(th[fixed], th0[fixed], rtol=1e-6)
    ctx.release_scene(sid)


def test_sim_to_sim_recovery_of_the_cylinder_radius_and_wall_density(ctx):
    """Shape and material together (the paper's cylinder experiment over R and Z, without the
    roughness): the tube's radius 5.0 -> 5.15 mm and the wall's density (impedance) +8 %; the
    mesh is rebuilt at every iteration and the radius gradient is the vertex gradient
    contracted with d tris / dR.  The loss is sharp in R (the wall echoes move by 0.2 us per
    0.15 mm), so R circles the target within a few um while the density settles."""
    from paper_2604_15017_gb300 import optim

    w = P.hollow_cylinder(n_rays=1500)
    n_mat = len(w["theta"])
    shape = optim.ShapeModel(lambda q: (lambda m: (m[0], m[2][None]))(P.hollow_cylinder_mesh(radius=q[0])), w,
                             [w["radius"]])
    th0 = np.concatenate([w["theta"], [w["radius"]]])
    free = np.array([4, n_mat])  # rho of the wall, R
    tgt = th0.copy()
    tgt[4] *= 1.08
    tgt[n_mat] = 5.15e-3
    lo, hi = th0.copy(), th0.copy()
    lo[4], hi[4] = 0.85 * th0[4], 1.15 * th0[4]
    lo[n_mat], hi[n_mat] = 4.7e-3, 5.3e-3
    prob = optim.InverseProblem(ctx, None, th0, lo, hi, 0.02, optim.split_rays(w["acq"], 2), w["img"],
                                seed=w["seed"], shape=shape)
    prob.set_targets(tgt)
    hist = []
    for _ in range(45):
        th = prob.physical().astype(np.float64)  # the parameters this iteration's loss belongs to
        hist.append((prob.step(), th))
    best_loss, th = min(hist, key=lambda t: t[0])
    assert best_loss < 0.2 * hist[0][0], [h[0] for h in hist]
    assert np.all(np.abs(th[free] - tgt[free]) < 0.5 * np.abs(th0[free] - tgt[free])), np.c_[th[free], tgt[free]]
    fixed = np.setdiff1d(np.arange(len(th0)), free)
    assert np.allclose(th[fixed], th0[fixed], rtol=1e-6)


def test_sim_to_sim_recovery_on_a_rough_walled_cylinder(ctx):
    """The same recovery with a rough wall (GGX roughness 0.2, held fixed): the radius gradient
    runs through rough events (sampled facet normals follow the moving mesh).  The loss is flat
    in R for the first 0.05 mm here and Adam overshoots the density afterwards, so the check is
    on the best iterate of 45: its loss below a fifth of the first, both parameters more than
    halfway to the target."""
    from paper_2604_15017_gb300 import optim

    w = P.with_roughness(P.hollow_cylinder(n_rays=1500), [0.0, 0.2, 0.0])
    n_mat = len(w["theta"])
    shape = optim.ShapeModel(lambda q: (lambda m: (m[0], m[2][None]))(P.hollow_cylinder_mesh(radius=q[0])), w,
                             [w["radius"]])
    th0 = np.concatenate([w["theta"], [w["radius"]]])
    free = np.array([4, n_mat])
    tgt = th0.copy()
    tgt[4] *= 1.08
    tgt[n_mat] = 5.15e-3
    lo, hi = th0.copy(), th0.copy()
    lo[4], hi[4] = 0.85 * th0[4], 1.15 * th0[4]
    lo[n_mat], hi[n_mat] = 4.7e-3, 5.3e-3
    prob = optim.InverseProblem(ctx, None, th0, lo, hi, 0.02, optim.split_rays(w["acq"], 2), w["img"],
                                seed=w["seed"], shape=shape)
    prob.set_targets(tgt)
    hist = []
    for _ in range(45):
        th = prob.physical().astype(np.float64)  # the parameters this iteration's loss belongs to
        hist.append((prob.step(), th))
    best_loss, th = min(hist, key=lambda t: t[0])
    assert best_loss < 0.2 * hist[0][0], [h[0] for h in hist]
    assert np.all(np.abs(th[free] - tgt[free]) < 0.5 * np.abs(th0[free] - tgt[free])), np.c_[th[free], tgt[free]]
