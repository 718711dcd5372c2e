"""Pins of the oracle's emission, receive directivity and secondary-ray selection weight (CPU).

Each test compares the oracle with a value fixed independently of it:

* emission (Sec. 2.3.1, Eq. directivity, Eq. pressure_mc): the sampled directions against the
  cosine-weighted distribution P(theta <= t) = sin^2 t (Kolmogorov-Smirnov), the origins against
  the uniform distribution over the element face, and the expected echo of a planar reflector
  against the closed-form projected solid angle that the estimator integrates (the view factor
  of a parallel rectangle), which fixes the weight pi / N_r and the direction density together;
* receive directivity (Eq. cutoff): arrival amplitudes of rays injected at known angles
  against the trapezoid with main-lobe angle 20 deg and cutoff 45 deg;
* secondary-ray selection weight (Sec. 2.3.3): the mean contribution per element of a
  scatterer event against a * A_s * s_j * attenuation * f_rx, the uniform choice among N_e
  elements cancelled by the weight N_e.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P

MM = 1e-3
KAPPA = math.log(10.0) / 20.0 * 1e-4  # amplitude Np per (dB/cm/MHz) * Hz * m


def ks_statistic(samples, cdf):
    """One-sample Kolmogorov-Smirnov distance sup |F_n - F|."""
    x = np.sort(np.asarray(samples))
    n = len(x)
    f = cdf(x)
    return max(np.max(np.arange(1, n + 1) / n - f), np.max(f - np.arange(0, n) / n))


def ks_bound(n, alpha=1e-4):
    """Asymptotic critical value of the KS distance at level alpha."""
    return math.sqrt(-0.5 * math.log(alpha / 2.0) / n)


def small_acq(**kw):
    args = dict(n_elem=16, pitch=0.3 * MM, n_samples=2048, angles_deg=[0.0], n_rays=1000, k_max=1, c_bf=1500.0)
    args.update(kw)
    return P.acquisition(**args)


# ------------------------------------------------------------------------------------------
# emission
# ------------------------------------------------------------------------------------------
def test_emission_directions_are_cosine_weighted_and_origins_uniform():
    acq = small_acq(n_rays=20000)
    e = 5
    o, w, a0, tau0 = O.emit(acq, seed=3, tx=0, ray_lo=e * acq["n_rays"], n=acq["n_rays"])
    n = len(a0)
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    assert np.all(w[:, 2] > 0)  # into the half space in front of the element
    sin2 = 1.0 - w[:, 2] ** 2
    # cosine-weighted: P(theta <= t) = sin^2 t, so sin^2 theta is uniform on [0, 1]
    assert ks_statistic(sin2, lambda x: x) < ks_bound(n)
    # a uniform hemisphere (P(theta <= t) = 1 - cos t) is rejected by the same test
    assert ks_statistic(w[:, 2], lambda x: x) > 5 * ks_bound(n)
    phi = np.mod(np.arctan2(w[:, 1], w[:, 0]), 2 * math.pi)
    assert ks_statistic(phi, lambda x: x / (2 * math.pi)) < ks_bound(n)
    xe = (e - 0.5 * (acq["n_elem"] - 1)) * acq["pitch"]
    ux = (o[:, 0] - xe) / acq["pitch"] + 0.5
    uy = o[:, 1] / acq["h_el"] + 0.5
    assert np.all((ux >= 0) & (ux < 1) & (uy >= 0) & (uy < 1)) and np.all(o[:, 2] == 0.0)
    assert ks_statistic(ux, lambda x: x) < ks_bound(n)
    assert ks_statistic(uy, lambda x: x) < ks_bound(n)
    # the cosine term over the cosine-weighted density (cos / pi) is pi, averaged over N_r rays
    assert np.allclose(a0, math.pi / acq["n_rays"], rtol=1e-15)
    assert np.all(tau0 == 0.0)  # unsteered


def rect_projected_solid_angle(h, x1, x2, y1, y2):
    """Integral over the rectangle [x1, x2] x [y1, y2] of the plane at height h of
    cos^2(theta) / r^2 = h^2 / (h^2 + x^2 + y^2)^2 (the projected solid angle it subtends seen
    from the origin): the textbook view factor of a parallel rectangle with a corner above the
    point, pi F = (1/2) [a / sqrt(h^2 + a^2) atan(b / sqrt(h^2 + a^2)) + (b <-> a)], combined
    over the four corners with signs."""
    def corner(x, y):
        a, b = abs(x), abs(y)
        if a == 0.0 or b == 0.0:
            return 0.0
        sa, sb = math.sqrt(h * h + a * a), math.sqrt(h * h + b * b)
        v = 0.5 * (a / sa * math.atan(b / sa) + b / sb * math.atan(a / sb))
        return math.copysign(1.0, x) * math.copysign(1.0, y) * v
    return corner(x2, y2) - corner(x1, y2) - corner(x2, y1) + corner(x1, y1)


def test_rect_projected_solid_angle_closed_form():
    """The closed form against direct quadrature (and the half-space limit pi)."""
    h, x1, x2, y1, y2 = 0.02, -0.004, 0.011, -0.0025, 0.0025
    xs, wx = np.polynomial.legendre.leggauss(200)
    ys, wy = np.polynomial.legendre.leggauss(200)
    X = 0.5 * (x2 - x1) * xs + 0.5 * (x2 + x1)
    Y = 0.5 * (y2 - y1) * ys + 0.5 * (y2 + y1)
    f = h * h / (h * h + X[:, None] ** 2 + Y[None, :] ** 2) ** 2
    quad = 0.25 * (x2 - x1) * (y2 - y1) * (wx[:, None] * wy[None, :] * f).sum()
    assert abs(rect_projected_solid_angle(h, x1, x2, y1, y2) - quad) < 1e-12 * max(1.0, quad)
    assert abs(rect_projected_solid_angle(1.0, -1e6, 1e6, -1e6, 1e6) - math.pi) < 1e-5


def test_emission_planar_reflector_echo_matches_projected_solid_angle():
    """Expected echo of a planar reflector (Eq. pressure_mc with f_d of Eq. directivity).

    A reflector at depth d whose medium has the same sound speed (so R = (rho2 - rho1) /
    (rho2 + rho1) at every angle and no refraction), always reflected (fixed split q = 1,
    weight R), no attenuation, receive directivity 1 everywhere.  Emitting from one element,
    the expected amplitude arriving at element j is R times the projected solid angle of
    element j's mirror image (a rectangle at height 2 d) averaged over the emitting face:
    E = R * mean_x0 integral_rect_j (2 d)^2 / ((2 d)^2 + rho^2)^2 dA."""
    d = 4 * MM
    n_elem, pitch, h_el = 16, 0.3 * MM, 5 * MM
    rho1, rho2, c = 1000.0, 2000.0, 1500.0
    R = (rho2 - rho1) / (rho2 + rho1)
    tris = P.box_mesh((-30 * MM, -30 * MM, d), (30 * MM, 30 * MM, d + 10 * MM))
    media = np.tile(np.array([[0, 1]], dtype=np.int32), (len(tris), 1))
    sp, sa = P.empty_scatterers()
    theta = P.theta_vector([(c, rho1, 0.0), (c, rho2, 0.0)])
    e_tx = 6
    n_rays = 400000
    acq = P.acquisition(n_elem, pitch, 2048, [0.0], n_rays, 1, c, h_el=h_el, alpha_m_deg=90.0, alpha_c_deg=90.0,
                        split_mode=1, split_q=1.0, tx_elem=e_tx)
    sc = O.Scene(tris, media, sp, sa, 0.1 * MM)
    run = O.Run(sc, theta, 2, acq, seed=9)
    arr = run.arrivals()
    assert np.all(arr["kind"] == 0)
    got = np.bincount(arr["e"], weights=arr["a"], minlength=n_elem)
    cnt = np.bincount(arr["e"], minlength=n_elem)
    # closed form, averaged over the emitting face by Gauss-Legendre quadrature
    gx, wx = np.polynomial.legendre.leggauss(24)
    gy, wy = np.polynomial.legendre.leggauss(24)
    xe = (e_tx - 0.5 * (n_elem - 1)) * pitch
    want = np.zeros(n_elem)
    for j in range(n_elem):
        xj = (j - 0.5 * (n_elem - 1)) * pitch
        acc = 0.0
        for a, wa in zip(gx, wx):
            x0 = xe + 0.5 * pitch * a
            for b, wb in zip(gy, wy):
                y0 = 0.5 * h_el * b
                acc += 0.25 * wa * wb * rect_projected_solid_angle(
                    2 * d, xj - 0.5 * pitch - x0, xj + 0.5 * pitch - x0, -0.5 * h_el - y0, 0.5 * h_el - y0)
        want[j] = R * acc
    # Monte Carlo error: the count at element j is binomial with p_j = want_j / (pi R)
    p = want / (math.pi * R)
    sigma = math.pi * R / n_rays * np.sqrt(n_rays * p * (1 - p))
    assert np.all(np.abs(got - want) <= 4 * sigma + 1e-15), (got, want, sigma)
    total_sigma = math.pi * R / n_rays * math.sqrt(n_rays * p.sum() * (1 - p.sum()))
    assert abs(got.sum() - want.sum()) <= 4 * total_sigma
    # every arrival carries the same weight pi R / N_r
    assert np.allclose(arr["a"], math.pi * R / n_rays, rtol=1e-12)
    assert cnt.sum() == len(arr["a"])


# ------------------------------------------------------------------------------------------
# receive directivity, Eq. cutoff
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("phi_deg", [0.0, 90.0, 37.0])
def test_receive_directivity_trapezoid(phi_deg):
    """Rays injected toward the array at angle t to its normal arrive with amplitude f(t):
    1 up to the main-lobe angle (20 deg), (45 - t) / 25 up to the cutoff (45 deg), 0 beyond."""
    sp, sa = P.empty_scatterers()
    sc = O.Scene(np.zeros((0, 9)), np.zeros((0, 2), np.int32), sp, sa, 0.1 * MM)
    theta = P.theta_vector([(1540.0, 1000.0, 0.0)])
    acq = P.acquisition(64, 0.3 * MM, 2048, [0.0], 1, 2, 1540.0)
    phi = math.radians(phi_deg)
    z0 = 0.5 * MM  # every ray below lands on the array (|x| <= 9.6 mm, |y| <= 2.5 mm)
    for t_deg, want in [(0.0, 1.0), (10.0, 1.0), (19.9, 1.0), (30.0, 0.6), (40.0, 0.2), (44.0, 0.04),
                        (45.5, 0.0), (50.0, 0.0), (70.0, 0.0)]:
        t = math.radians(t_deg)
        w = np.array([math.sin(t) * math.cos(phi), math.sin(t) * math.sin(phi), -math.cos(t)])
        arr, rec, _ = O.trace_injected(sc, theta, 1, acq, [0.1 * MM, 0.2 * MM, z0], w, a0=1.0)
        if want == 0.0:
            assert arr == [] and rec[0, 0] == O.CLS_XDCR  # reached the array, cut off
        else:
            assert len(arr) == 1 and arr[0][3] == 0
            assert abs(arr[0][2] - want) < 1e-12, (t_deg, arr[0][2], want)
            assert abs(arr[0][1] - z0 / math.cos(t) / 1540.0) < 1e-18


# ------------------------------------------------------------------------------------------
# secondary-ray (receiver-guided) selection weight, Sec. 2.3.3
# ------------------------------------------------------------------------------------------
def test_secondary_ray_mean_per_element_matches_closed_form():
    """One scatterer in a homogeneous attenuating medium, a primary injected through its centre.
    At the scatterer event an element e' is drawn uniformly and the secondary ray carries
    a * A_s * s_j * N_e * exp(-kappa alpha f0 D_e') * f_rx(angle_e'), so the mean over draws of
    what element j receives is a * A_s * s_j * exp(-kappa alpha f0 D_j) * f_rx(angle_j), with the
    arrival time tau + D_j / c.  A weight without the N_e, or with the choice counted twice,
    misses the mean by a factor N_e."""
    n_elem, pitch = 64, 0.3 * MM
    c, alpha, f0, As, s_j = 1540.0, 0.5, 5e6, 1.3, 0.7
    xs, zs, z_in = 1.2 * MM, 8 * MM, 1 * MM
    sc = O.Scene(np.zeros((0, 9)), np.zeros((0, 2), np.int32), np.array([[xs, 0.0, zs]]), np.array([s_j]),
                 0.1 * MM)
    theta = P.theta_vector([(c, 1000.0, alpha)], amp_scale=As, f0=f0)
    acq = P.acquisition(n_elem, pitch, 2048, [0.0], 1, 3, c)
    n_draw = 12000
    got = np.zeros(n_elem)
    chosen = np.zeros(n_elem, np.int64)
    a1 = math.exp(-KAPPA * alpha * f0 * z_in)
    xe = (np.arange(n_elem) - 0.5 * (n_elem - 1)) * pitch
    D = np.hypot(xe - xs, zs)
    ang = np.degrees(np.arctan2(np.abs(xe - xs), zs))
    frx = np.clip((45.0 - ang) / 25.0, 0.0, 1.0)
    want = a1 * As * s_j * np.exp(-KAPPA * alpha * f0 * D) * frx
    for r in range(n_draw):
        arr, rec, _ = O.trace_injected(sc, theta, 1, acq, [xs, 0.0, zs - z_in], [0.0, 0.0, 1.0], a0=1.0, ray=r)
        assert rec[0, 0] == O.CLS_SCAT and rec[1, 0] == O.CLS_NONE  # the primary passes and escapes
        e2 = rec[0, 3]
        chosen[e2] += 1
        if frx[e2] == 0.0:
            assert arr == []
            continue
        assert len(arr) == 1 and arr[0][0] == e2 and arr[0][3] == 1
        assert abs(arr[0][2] - n_elem * want[e2]) < 1e-12 * n_elem * want.max()
        assert abs(arr[0][1] - (z_in + D[e2]) / c) < 1e-17
        got[e2] += arr[0][2]
    got /= n_draw
    chi2 = ((chosen - n_draw / n_elem) ** 2 / (n_draw / n_elem)).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)
    # the element choice is uniform (chi-square, 63 degrees of freedom, over the draws whose
    # secondary ray reached an element and the rest counted through the record)
    # per element: a draw contributes N_e want_j with probability 1 / N_e
    sigma = want * np.sqrt((n_elem - 1) / n_draw)
    inside = want > 0
    assert np.all(np.abs(got[inside] - want[inside]) <= 4.5 * sigma[inside])
    assert np.all(got[~inside] == 0.0)
    # the total over elements: a draw contributes N_e want_e' for a uniform e'
    var = (n_elem * (want ** 2).sum() - want.sum() ** 2) / n_draw
    assert abs(got.sum() - want.sum()) <= 4 * math.sqrt(var)
    assert abs(got.sum() / want.sum() - 1) < 0.05
