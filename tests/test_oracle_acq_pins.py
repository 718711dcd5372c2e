"""Pins of the oracle's acquisition-parameter derivatives (c_bf and the steering angles) against
finite differences (CPU only).  The acquisition parameters move only the emission time stamps
and the beamforming delays, never a path's decisions, so a forward run at a perturbed
acquisition with the same seed is the same realisation: central differences of the linear
functional <grf, RF> and of <gi, DAS(RF)> check the derivatives directly.

Step sizes: DAS interpolates the record linearly, so <gi, DAS(RF)> is piecewise smooth in the
delays with a kink at every sample crossing; a step of 1e-9 (relative for c_bf, radians for an
angle) crosses almost none of them.  The emission time stamp holds |sin theta|, whose kink at
theta = 0 (a steering angle of the transport pin) makes the central difference there converge
only linearly in the step, to the sgn(0) = 0 derivative; a step of 1e-8 puts that error below
1e-5 relative."""
import numpy as np

from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P

MM = 1e-3


def perturbed(acq, which, h):
    """which: 0 = c_bf, 1 = pitch (relative steps), 2 + t = steering angle t (radians)"""
    a = dict(acq)
    if which == 0:
        a["c_bf"] = acq["c_bf"] * (1.0 + h)
    elif which == 1:
        a["pitch"] = acq["pitch"] * (1.0 + h)
    else:
        ang = list(acq["angles"])
        ang[which - 2] = ang[which - 2] + h
        a["angles"] = ang
    return a


def step(acq, which, h):
    return acq["c_bf"] * h if which == 0 else (acq["pitch"] * h if which == 1 else h)


def test_das_acquisition_derivatives_match_finite_differences():
    acq = P.acquisition(32, 0.3 * MM, 1024, [-9.0, 0.0, 11.0], 1, 1, 1540.0)
    img = P.image(24, 128, -4 * MM, 4 * MM, 2 * MM, 18 * MM)
    rng = np.random.default_rng(3)
    n = 3000
    rf = O.splat(acq, 5e6, rng.integers(0, 3, n), rng.integers(0, 32, n), rng.uniform(0, 1024 / 40e6, n),
                 rng.normal(size=n))
    gi = rng.normal(size=(24, 128))
    g = O.das_acq_vjp(acq, img, rf, gi)
    for which in range(5):
        h = 1e-9
        fp = np.sum(gi * O.das(perturbed(acq, which, h), img, rf))
        fm = np.sum(gi * O.das(perturbed(acq, which, -h), img, rf))
        fd = (fp - fm) / (2 * step(acq, which, h))
        assert abs(fd - g[which]) <= 1e-4 * abs(g[which]) + 1e-9 * np.abs(g).max(), (which, fd, g[which])


def test_transport_acquisition_derivatives_match_finite_differences():
    w = P.slab_scatterers(n_rays=300)
    w["acq"] = dict(w["acq"], angles=[-0.1, 0.0, 0.12])
    ref = O.forward(w)
    run = ref["run"]
    rng = np.random.default_rng(4)
    grf = rng.normal(size=ref["rf"].shape)
    g = run.gradient_acq(grf)
    assert g.shape == (5,) and np.abs(g).max() > 0
    rec0 = run.records()
    for which in range(5):
        h = 1e-8
        wp = dict(w, acq=perturbed(w["acq"], which, h))
        wm = dict(w, acq=perturbed(w["acq"], which, -h))
        rp, rm = O.forward(wp), O.forward(wm)
        for k in rec0:  # the same realisation
            assert np.array_equal(rp["run"].records()[k], rec0[k])
        fd = (np.sum(grf * rp["rf"]) - np.sum(grf * rm["rf"])) / (2 * step(w["acq"], which, h))
        assert abs(fd - g[which]) <= 1e-4 * abs(g[which]) + 1e-6 * np.abs(g).max(), (which, fd, g[which])


def test_scene_gradient_unchanged_by_the_acquisition_slots():
    w = P.slab_scatterers(n_rays=200)
    ref = O.forward(w)
    grf = np.random.default_rng(5).normal(size=ref["rf"].shape)
    g_scene = ref["run"].gradient(grf)
    assert np.all(np.isfinite(g_scene))
    # the extended gradient's scene part is the plain gradient (same duals, more slots)
    full = ref["run"].gradient_acq(grf, full=True)
    assert full.shape == (len(g_scene) + 2 + len(w["acq"]["angles"]),)
    assert np.allclose(full[:len(g_scene)], g_scene, rtol=1e-12, atol=1e-12 * np.abs(g_scene).max())
