"""Pins of the oracle's rough interfaces (Sec. 2.3.2, Eq. GGX_PDF; CPU only).

* The sampled microfacet normals follow D(h) (h.n), D the paper's GGX distribution: their
  polar angles against the cumulative distribution integrated numerically from Eq. GGX_PDF
  (Kolmogorov-Smirnov), uniform azimuths, unit length, and a tilted macro normal.
* alpha -> 0 is the smooth interface (same RF).
* The roughness gradient of the fixed realisation against central differences of the
  oracle's own forward (same seed, records asserted identical).
"""
import numpy as np

from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P


def ggx_pdf_theta_cdf(alpha):
    """Cumulative distribution of the microfacet polar angle for the density D(h) (h.n) over
    the hemisphere, D of Eq. GGX_PDF, by trapezoidal quadrature."""
    t = np.linspace(0.0, np.pi / 2, 40001)
    d = alpha ** 2 / (np.pi * (np.cos(t) ** 2 * (alpha ** 2 - 1.0) + 1.0) ** 2)
    dens = d * np.cos(t) * np.sin(t) * 2.0 * np.pi
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(t))])
    return t, cdf


def test_sampled_microfacet_normals_follow_the_ggx_distribution():
    rng = np.random.default_rng(0)
    n_s = 20000
    for alpha, n in ((0.3, np.array([0.0, 0.0, 1.0])), (0.8, np.array([0.6, -0.48, -0.64]))):
        t, cdf = ggx_pdf_theta_cdf(alpha)
        assert abs(cdf[-1] - 1.0) < 1e-6  # D (h.n) is normalised over the hemisphere
        u = rng.random((n_s, 2))
        hs = np.array([O.ggx_normal(n, alpha, a, b) for a, b in u])
        assert np.abs(np.linalg.norm(hs, axis=1) - 1.0).max() < 1e-12
        th = np.sort(np.arccos(np.clip(hs @ n, -1.0, 1.0)))
        ks = np.max(np.abs(np.interp(th, t, cdf) - np.arange(1, n_s + 1) / n_s))
        assert ks < 1.63 / np.sqrt(n_s), ks  # 1 % level
        # azimuth about n uniform: the tangential parts have no preferred direction
        tang = hs - np.outer(hs @ n, n)
        assert np.linalg.norm(tang.mean(axis=0)) < 4.0 * np.linalg.norm(tang, axis=1).mean() / np.sqrt(n_s)


def test_vanishing_roughness_is_the_smooth_interface():
    w = P.slab_scatterers(n_rays=300)
    smooth = O.forward(w)["rf"]
    rough = O.forward(P.with_roughness(w, [0.0, 1e-7]))["rf"]
    assert np.linalg.norm(rough - smooth) <= 1e-5 * np.linalg.norm(smooth)


def test_roughness_gradient_matches_finite_differences():
    w = P.with_roughness(P.slab_scatterers(n_rays=300), [0.0, 0.2])
    ref = O.forward(w)
    grf = np.random.default_rng(4).normal(size=ref["rf"].shape)
    g = ref["run"].gradient(grf)
    assert g.shape == (4 * w["M"] + 2,) and g[-2] == 0.0 and g[-1] != 0.0
    rec0 = ref["run"].records()
    h = 1e-6
    tp, tm = w["theta"].copy(), w["theta"].copy()
    tp[-1] += h
    tm[-1] -= h
    rp, rm = O.forward(w, theta=tp), O.forward(w, theta=tm)
    for r in (rp, rm):
        for k in rec0:
            assert np.array_equal(r["run"].records()[k], rec0[k])
    fd = (np.sum(grf * rp["rf"]) - np.sum(grf * rm["rf"])) / (2 * h)
    assert abs(fd - g[-1]) <= 1e-5 * abs(g[-1]), (fd, g[-1])
    # the other parameters' gradient through rough events, against one of them
    i = 4  # rho of the slab
    tp, tm = w["theta"].copy(), w["theta"].copy()
    tp[i] *= 1 + 1e-7
    tm[i] *= 1 - 1e-7
    fd = (np.sum(grf * O.forward(w, theta=tp)["rf"]) - np.sum(grf * O.forward(w, theta=tm)["rf"])) / (2e-7 * w["theta"][i])
    assert abs(fd - g[i]) <= 1e-4 * abs(g[i]), (fd, g[i])


# ------------------------------------------------------------------------------------------
# secondary rays at rough interface events (Sec. 2.3.3) combined with the primary by the
# balance heuristic: the same expectation as the primary's own sampling alone
# ------------------------------------------------------------------------------------------
MM = 1e-3


def per_element_sums(e, a, n_elem):
    s = np.bincount(e, weights=a, minlength=n_elem)
    v = np.bincount(e, weights=a * a, minlength=n_elem)  # variance of a sum of rare contributions
    return s, v


def rough_box(depth, alpha, c_in=2000.0):
    tris = P.box_mesh((-60 * MM, -60 * MM, depth), (60 * MM, 60 * MM, depth + 40 * MM))
    media = np.tile(np.array([[0, 1]], dtype=np.int32), (len(tris), 1))
    sp, sa = P.empty_scatterers()
    theta = np.concatenate([P.theta_vector([(1500.0, 1000.0, 0.0), (c_in, 1300.0, 0.0)]), [0.0, alpha]])
    return O.Scene(tris, media, sp, sa, 0.1 * MM, rough=True), theta


def compare_modes(sums):
    """mode 0 (the primary's sampling alone) against mode 2 (the secondary ray alone: every
    factor of the BSDF evaluation) and mode 1 (both, balance heuristic), per element.  The
    secondary ray aims at the element's centre, a midpoint rule over the element's solid angle,
    so the elements here are small next to the angular scale on which the BSDF varies."""
    s0, v0 = sums[0]
    for mode in (1, 2):
        s1, v1 = sums[mode]
        sig = np.sqrt(v0 + v1)
        assert np.all(np.abs(s1 - s0) <= 4.5 * sig + 1e-12), (mode, np.c_[s0, s1, sig])
        assert abs(s1.sum() - s0.sum()) <= 4 * np.sqrt(v0.sum() + v1.sum()), (mode, s0.sum(), s1.sum())
        assert abs(s1.sum() / s0.sum() - 1.0) < 0.03, (mode, s0.sum(), s1.sum())
    # the balance heuristic lowers the variance below the primary's alone
    assert np.sqrt(sums[1][1].sum()) < np.sqrt(v0.sum())


def injected(n_ray, z0, sx, seed=3):
    rng = np.random.default_rng(seed)
    o = np.stack([rng.uniform(-1.5, 1.5, n_ray) * MM, rng.uniform(-0.2, 0.2, n_ray) * MM, np.full(n_ray, z0)], 1)
    w = np.stack([rng.normal(0, sx, n_ray), rng.normal(0, 0.05, n_ray), -np.ones(n_ray)], 1)
    return o, w / np.linalg.norm(w, axis=1)[:, None]


def test_rough_secondary_rays_reflection_keep_the_expectation():
    """Rays injected above a rough interface at 6 mm (alpha 0.6, always reflected, facets that
    reflect totally included): what reaches each element directly after the reflection, out to
    elements seen at 65 deg from the interface normal (Smith masking of the outgoing side)."""
    sc, theta = rough_box(6 * MM, 0.6)
    o, w = injected(2_000_000, 2 * MM, 0.3)
    w[:, 2] *= -1.0  # downward
    sums = {}
    for nee in (0, 1, 2):
        acq = P.acquisition(128, 0.2 * MM, 4096, [0.0], 1, 1, 1500.0, h_el=0.4 * MM, alpha_m_deg=90.0,
                            alpha_c_deg=90.0, split_mode=1, split_q=1.0, rough_nee=nee)
        sums[nee] = O.inject_sums(sc, theta, 2, acq, o, w)
    compare_modes(sums)


def test_rough_secondary_rays_refraction_keep_the_expectation():
    """Rays injected inside a slower medium toward its rough upper face at 10 mm (alpha 0.5,
    always transmitted into the faster medium above, where the probe is): what reaches each
    element directly after the refraction."""
    sc, theta = rough_box(10 * MM, 0.5)
    o, w = injected(1_000_000, 14 * MM, 0.2)
    sums = {}
    for nee in (0, 1, 2):
        acq = P.acquisition(64, 0.2 * MM, 4096, [0.0], 1, 1, 1500.0, h_el=0.4 * MM, alpha_m_deg=90.0,
                            alpha_c_deg=90.0, split_mode=1, split_q=0.0, rough_nee=nee)
        sums[nee] = O.inject_sums(sc, theta, 2, acq, o, w)
    compare_modes(sums)
