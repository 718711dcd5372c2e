"""Pins of the optimiser oracle (Sec. 3.4, Sec. 3.7, Alg. 1) against closed forms and an
independent implementation (CPU only)."""
import numpy as np
import pytest

from oracle import optim as OP


def test_clip_and_scale_map_endpoints_and_interior():
    lo = np.array([1400.0, 900.0, 0.1])
    hi = np.array([1700.0, 1200.0, 1.5])
    tu = np.array([-0.3, 0.25, 1.7])
    th = OP.scale_phys(OP.clip01(tu), lo, hi)
    assert th[0] == lo[0] and th[2] == hi[2]
    assert th[1] == pytest.approx(900.0 + 0.25 * 300.0)
    # the clip's derivative: 1 strictly inside, 0 at or beyond the bounds
    assert list(OP.clip_grad_mask([-0.1, 0.0, 0.5, 1.0, 1.2])) == [0.0, 0.0, 1.0, 0.0, 0.0]


def test_gradient_chain_through_scale_matches_finite_differences():
    rng = np.random.default_rng(1)
    lo, hi = rng.uniform(0, 1, 5), rng.uniform(2, 3, 5)
    tu = rng.uniform(0.1, 0.9, 5)
    a = rng.normal(size=5)

    def f(t):  # a smooth function of the physical parameters
        return float(np.sum(a * np.sin(OP.scale_phys(OP.clip01(t), lo, hi))))

    g_phys = a * np.cos(OP.scale_phys(tu, lo, hi))
    g = OP.grad_unconstrained(tu, g_phys, lo, hi)
    h = 1e-6
    fd = np.array([(f(tu + h * e) - f(tu - h * e)) / (2 * h) for e in np.eye(5)])
    assert np.allclose(g, fd, rtol=1e-7, atol=1e-9)


def test_first_adam_step_is_lr_times_sign():
    # bias-corrected first moments are g and g^2, so the first step is lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3])
    tu, m, v = OP.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8)
    assert np.allclose(tu, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_matches_torch_adam_on_a_quadratic():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    A = rng.normal(size=(6, 6))
    Q = A @ A.T + np.eye(6)
    b = rng.normal(size=6)
    x0 = rng.normal(size=6)
    lr = np.array([0.05] * 3 + [0.01] * 3)  # two parameter groups
    xt = [torch.tensor(x0[:3].copy(), dtype=torch.float64, requires_grad=True),
          torch.tensor(x0[3:].copy(), dtype=torch.float64, requires_grad=True)]
    opt = torch.optim.Adam([{"params": [xt[0]], "lr": 0.05}, {"params": [xt[1]], "lr": 0.01}], betas=(0.9, 0.999),
                           eps=1e-8)
    x, m, v = x0.copy(), np.zeros(6), np.zeros(6)
    Qt, bt = torch.tensor(Q), torch.tensor(b)
    for k in range(1, 21):
        g = Q @ x - b
        x, m, v = OP.adam_step(x, g, m, v, k, lr)
        opt.zero_grad()
        xx = torch.cat(xt)
        (0.5 * xx @ Qt @ xx - bt @ xx).backward()
        opt.step()
    assert np.allclose(x, torch.cat(xt).detach().numpy(), rtol=1e-10, atol=1e-12)


def test_global_norm_clipping():
    g = np.array([3.0, 4.0])
    assert np.allclose(OP.clip_global_norm(g, 1.0), [0.6, 0.8])
    assert np.allclose(OP.clip_global_norm(g, 10.0), g)
    assert np.allclose(OP.clip_global_norm(g, 0.0), g)


def test_optimise_recovers_a_quadratic_minimum_inside_the_box():
    lo, hi = np.zeros(3), np.full(3, 2.0)
    target = np.array([0.3, 1.1, 1.7])

    def grad_fn(th):
        return float(np.sum((th - target) ** 2)), 2.0 * (th - target)

    traj, losses = OP.optimise(np.full(3, 0.5), lo, hi, grad_fn, 400, lr=0.02)
    assert losses[-1] < 1e-6 * losses[0]
    assert np.allclose(OP.scale_phys(OP.clip01(traj[-1]), lo, hi), target, atol=1e-3)


def test_saturated_parameter_gets_no_update_until_gradient_points_inward():
    lo, hi = np.zeros(2), np.ones(2)
    tu = np.array([1.3, 0.5])
    out, m, v = OP.optimiser_step(tu, np.array([-5.0, 1.0]), lo, hi, np.zeros(2), np.zeros(2), 1, 0.1)
    assert out[0] == 1.3 and out[1] < 0.5


def test_element_sub_apertures_partition_the_realisation():
    """Micro-batches over emitting elements (Eq. microbatch_loss): disjoint sub-apertures with
    one seed are the full aperture's paths, split; their RF and their gradient for one dL/dRF
    add up to the full acquisition's (the transport is linear in its emitters)."""
    from oracle import oracle as O
    from paper_2604_15017_gb300 import optim, phantoms as P

    w = P.slab_scatterers(n_rays=60)
    full = O.forward(w)
    grf = np.random.default_rng(2).normal(size=full["rf"].shape)
    parts = optim.split_elements(w["acq"], 3)
    assert [a["n_tx_elem"] for a in parts] == [21, 22, 21] and parts[1]["tx_elem"] == 21
    rf = np.zeros_like(full["rf"])
    g = np.zeros(len(w["theta"]))
    for a in parts:
        r = O.forward(dict(w, acq=a))
        rf += r["rf"]
        g += r["run"].gradient(grf)
    assert np.allclose(rf, full["rf"], rtol=1e-12, atol=1e-12 * np.abs(full["rf"]).max())
    g_full = full["run"].gradient(grf)
    assert np.allclose(g, g_full, rtol=1e-10, atol=1e-12 * np.abs(g_full).max())
