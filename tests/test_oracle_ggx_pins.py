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
