"""Pins of the oracle's shape derivatives (directional derivatives along vertex tangent fields)
against finite differences (CPU only).  Moving the triangles by h * tangent with the same seed
gives the same realisation as long as no decision flips (the records are compared), so central
differences of <grf, RF> check the derivative of every geometric term the fixed-sample model
differentiates: hit distances on the moved planes, the normals in reflection, refraction and
the Fresnel coefficients, and the secondary rays' crossing distances and transmission
coefficients.  Steps of 1e-8 m (tangents of unit size) flip no decision on these scenes."""
import numpy as np

from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P


def fd_along(w, vt, grf, h=1e-8):
    run0 = O.forward(w)["run"]
    rec0 = run0.records()
    rp, rm = O.forward(dict(w, tris=w["tris"] + h * vt)), O.forward(dict(w, tris=w["tris"] - h * vt))
    for r in (rp, rm):
        for k in rec0:
            assert np.array_equal(r["run"].records()[k], rec0[k])
    return (np.sum(grf * rp["rf"]) - np.sum(grf * rm["rf"])) / (2 * h)


def check(w, tangents, seed):
    ref = O.forward(w)
    grf = np.random.default_rng(seed).normal(size=ref["rf"].shape)
    g = ref["run"].gradient_shape(grf, np.stack(tangents))
    assert np.all(np.abs(g) > 0)
    for j, vt in enumerate(tangents):
        fd = fd_along(w, vt, grf)
        assert abs(fd - g[j]) <= 1e-5 * abs(g[j]), (j, fd, g[j])
    return ref, grf, g


def test_slab_interface_depth_and_random_vertex_motion():
    """The slab's top interface moved down (every vertex at z = 20 mm, side faces included), and
    a random motion of every triangle vertex (tilted normals, moved planes)."""
    w = P.slab_scatterers(n_rays=300)
    t = w["tris"]
    depth = np.zeros_like(t)
    for k in range(3):
        depth[np.isclose(t[:, 3 * k + 2], 20e-3), 3 * k + 2] = 1.0
    rand = np.random.default_rng(1).normal(size=t.shape)
    check(w, [depth, rand], 4)


def test_hollow_cylinder_radius():
    """d/dR of the tube (both surfaces move outward): the tangent is exact, the mesh's vertices
    being linear in R."""
    w = P.hollow_cylinder(n_rays=100)
    wp = P.hollow_cylinder(n_rays=100, radius=w["radius"] + 1e-6)
    assert np.allclose((wp["tris"] - w["tris"]) / 1e-6, w["dtris_dR"], atol=1e-6)
    check(w, [w["dtris_dR"]], 5)


def test_shape_gradient_is_linear_in_the_tangent_and_keeps_the_scene_gradient():
    w = P.slab_scatterers(n_rays=200)
    ref = O.forward(w)
    grf = np.random.default_rng(6).normal(size=ref["rf"].shape)
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=w["tris"].shape), rng.normal(size=w["tris"].shape)
    full = ref["run"].gradient_shape(grf, np.stack([a, b, 2.0 * a - 3.0 * b]), full=True)
    n_th = len(w["theta"])
    assert np.allclose(full[n_th + 2], 2.0 * full[n_th] - 3.0 * full[n_th + 1], rtol=1e-9,
                       atol=1e-12 * np.abs(full[n_th:]).max())
    assert np.allclose(full[:n_th], ref["run"].gradient(grf), rtol=1e-12, atol=1e-12 * np.abs(full[:n_th]).max())


def test_rough_walled_cylinder_radius():
    """d/dR through rough events: the sampled facet normal follows the moving macro normal (its
    tangent frame and tilt), and so do the microfacet weight's cosines."""
    w = P.with_roughness(P.hollow_cylinder(n_rays=100), [0.0, 0.2, 0.0])
    check(w, [w["dtris_dR"]], 6)
