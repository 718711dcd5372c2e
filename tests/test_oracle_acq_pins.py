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
import pytest

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


@pytest.mark.parametrize("f_number", [0.0, 1.5])
def test_das_acquisition_derivatives_match_finite_differences(f_number):
    """f_number 1.5: the dynamic aperture's weights move with the pitch too (clamped to one
    pitch at the shallowest depths)."""
    acq = P.acquisition(32, 0.3 * MM, 1024, [-9.0, 0.0, 11.0], 1, 1, 1540.0)
    img = P.image(24, 128, -4 * MM, 4 * MM, 0.5 * MM, 18 * MM, f_number=f_number)
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


def test_dynamic_aperture_weights():
    """Receive F-number (dynamic aperture, a Hann window of half-width max(z / 2F, pitch) centred
    on the pixel): at depths where the half-width is clamped to one pitch, a pixel straight
    below element e sees that element alone with weight 1 (its neighbours sit at |xi| = 1), and
    a pixel more than a pitch away from every element with data sees nothing; deeper, the
    aperture widens.  The transposed DAS stays the adjoint."""
    n_e, pitch = 16, 0.3 * MM
    acq = P.acquisition(n_e, pitch, 1024, [0.0, 7.0], 1, 1, 1540.0)
    xe = (np.arange(n_e) - 0.5 * (n_e - 1)) * pitch
    rng = np.random.default_rng(8)
    rf = np.zeros((2, n_e, 1024))
    rf[:, 5, :] = rng.normal(size=(2, 1024))  # data on element 5 only
    # lines through the element centres; depths 0.2 .. 0.8 mm: z / (2 * 2.0) < pitch
    img = P.image(n_e, 16, xe[0], xe[-1], 0.2 * MM, 0.8 * MM, f_number=2.0)
    dyn = O.das(acq, img, rf)
    hann = O.das(acq, dict(img, f_number=0.0), rf)
    w5 = 0.5 * (1.0 - np.cos(2.0 * np.pi * 6 / (n_e + 1)))
    assert np.allclose(dyn[5], hann[5] / w5, rtol=1e-12, atol=1e-12)
    assert np.all(dyn[np.r_[0:4, 7:n_e]] == 0.0) and np.abs(dyn[5]).max() > 0
    # deeper (z / 2F = 2 pitches at 2.4 mm): element 5 reaches lines 4 and 6 with cos^2(pi/4) = 1/2,
    # lines 3 and 7 not at all
    deep = P.image(n_e, 16, xe[0], xe[-1], 2.4 * MM, 2.4 * MM + 15e-6, f_number=2.0)
    dd = O.das(acq, deep, rf)[:, 0]
    hd = O.das(acq, dict(deep, f_number=0.0), rf)[:, 0] / w5  # element 5's samples, unweighted
    assert np.allclose(dd[[4, 5, 6]], [0.5 * hd[4], hd[5], 0.5 * hd[6]], rtol=1e-12, atol=1e-15)
    assert dd[3] == 0.0 and dd[7] == 0.0
    # adjoint identity with the dynamic aperture
    img2 = P.image(12, 64, -2 * MM, 2 * MM, 0.5 * MM, 12 * MM, f_number=1.2)
    x = rng.normal(size=(2, n_e, 1024))
    y = rng.normal(size=(12, 64))
    lhs = np.sum(O.das(acq, img2, x) * y)
    rhs = np.sum(x * O.das_adjoint(acq, img2, y))
    assert abs(lhs - rhs) <= 1e-10 * np.abs(x).sum()


def test_transport_acquisition_derivatives_on_a_rough_scene():
    """The acquisition slots follow the roughness slots (theta of 4M + 2), and rough events move
    with the pitch's emission origins like smooth ones."""
    w = P.with_roughness(P.slab_scatterers(n_rays=200), [0.0, 0.25])
    w["acq"] = dict(w["acq"], angles=[-0.1, 0.12])
    ref = O.forward(w)
    grf = np.random.default_rng(9).normal(size=ref["rf"].shape)
    full = ref["run"].gradient_acq(grf, full=True)
    assert full.shape == (4 * w["M"] + 2 + 2 + 2,)
    g = full[4 * w["M"] + 2:]
    rec0 = ref["run"].records()
    for which in range(4):
        h = 1e-8
        rp = O.forward(dict(w, acq=perturbed(w["acq"], which, h)))
        rm = O.forward(dict(w, acq=perturbed(w["acq"], which, -h)))
        for k in rec0:
            assert np.array_equal(rp["run"].records()[k], rec0[k])
        fd = (np.sum(grf * rp["rf"]) - np.sum(grf * rm["rf"])) / (2 * step(w["acq"], which, h))
        assert abs(fd - g[which]) <= 1e-4 * abs(g[which]) + 1e-6 * np.abs(g).max(), (which, fd, g[which])
