"""Rough interfaces on the GPU (Sec. 2.3.2, Eq. GGX_PDF; row N1) against the FP64 oracle, whose
sampling, smooth limit and roughness gradient tests/test_oracle_ggx_pins.py pins.

* event sequences (primitive, class, choice; a path ended at a rough event ends on both
  sides) >= 99.9 % of paths identical, RF relative L2 <= 1e-3: a microfacet normal turns a
  ray by up to tens of degrees, so a rough event that ends a path in one precision and not in
  the other (a facet met edge-on, an outgoing direction grazing the macro surface) happens a
  little more often than a smooth split flips;
* the adjoint (roughness entries included) within 1e-3 relative of the oracle's gradient for
  the same dL/dRF, as for smooth scenes (plus 1e-4 of the largest sensitivity);
* roughness 0 reproduces the smooth scene; shape gradients through rough events (the
  cylinder's radius) against the oracle's directional derivatives.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_15017_gb300 import usrt

    c = usrt.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.float32).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def agreement(rec, ora):
    """Share of paths with identical events: primitive, class, choice, and the element of the
    secondary ray of every event that has one (scatterers; rough interfaces with rough_nee)."""
    r = rec.astype(np.int64) & 0xFFFFFFFF
    cls, pid, ch, aux = (r >> 20) & 3, r & 0xFFFFF, (r >> 22) & 3, (r >> 24) & 0xFF
    same = (cls == ora["cls"]) & ((pid == ora["id"]) | (ora["cls"] == 0))
    tri = ora["cls"] == O.CLS_TRI
    same &= ~tri | (ch == ora["choice"]) | (ora["choice"] == O.CH_NONE)
    with_nee = (ora["cls"] >= O.CLS_TRI) & (ora["aux"] >= 0)
    same &= ~with_nee | (aux == ora["aux"])
    return same.all(axis=1).mean()


def rough_inclusions(n_rays=200):
    w = P.inclusions(n_regions=3, n_scat=3000, n_rays=n_rays, k_max=6, n_samples=2048, angles_deg=[-6.0, 6.0],
                     n_lines=64, n_depth=512, n_elem=32, n_lat=24, n_lon=40)
    r = np.zeros(w["M"])
    r[1:] = np.linspace(0.05, 0.3, w["M"] - 1)
    return P.with_roughness(w, r)


def with_rough_nee(w):
    w = dict(w)
    w["acq"] = dict(w["acq"], rough_nee=1)
    return w


def assert_rough_nee_matters(w, grf, g_ref, tol_scale):
    """With secondary rays at rough events the oracle's gradient must differ from the one
    without them by far more than the tolerance, so that an adjoint ignoring them fails."""
    w0 = dict(w)
    w0["acq"] = dict(w["acq"], rough_nee=0)
    g0 = O.forward(w0)["run"].gradient(grf)
    assert np.max(np.abs(g_ref - g0) / tol_scale) > 5.0


def run_pair(ctx, w):
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["status"] == 0 and st["dropped"] == 0
    ref = O.forward(w)
    acq = w["acq"]
    n = len(acq["angles"]) * acq["n_elem"] * acq["n_rays"]
    rec = ctx.record(0, n, acq["k_max"]).cpu().numpy()
    return sid, rf, b, ref, rec


@pytest.mark.parametrize("make", ["slab", "inclusions"])
def test_rough_forward_matches_oracle(ctx, make):
    w = P.with_roughness(P.slab_scatterers(n_rays=800), [0.0, 0.25]) if make == "slab" else rough_inclusions()
    sid, rf, b, ref, rec = run_pair(ctx, w)
    assert agreement(rec, ref["run"].records()) >= 0.999
    assert rel_l2(rf.double().cpu().numpy(), ref["rf"]) <= 1e-3, rel_l2(rf.double().cpu().numpy(), ref["rf"])
    ctx.release_scene(sid)


@pytest.mark.parametrize("make", ["slab", "inclusions", "cylinder"])
def test_rough_secondary_rays_forward_matches_oracle(ctx, make):
    """Secondary rays at rough interface events (Sec. 2.3.3) with the balance weights against
    the primary's direct hits: the same events (secondary-ray elements included) and RF."""
    if make == "slab":
        w = P.with_roughness(P.slab_scatterers(n_rays=800), [0.0, 0.25])
    elif make == "inclusions":
        w = rough_inclusions()
    else:
        w = P.with_roughness(P.hollow_cylinder(n_rays=400), [0.0, 0.2, 0.0])
    w = with_rough_nee(w)
    sid, rf, b, ref, rec = run_pair(ctx, w)
    assert agreement(rec, ref["run"].records()) >= 0.999
    arr = ref["run"].arrivals()
    recs = ref["run"].records()
    rough_ev = (recs["cls"] == O.CLS_TRI) & (recs["aux"] >= 0)
    assert rough_ev.any()  # the scene has rough events with secondary rays
    err = rel_l2(rf.double().cpu().numpy(), ref["rf"])
    assert err <= 1e-3, err
    st = ctx.stats()
    c = ref["run"].counters()
    assert abs(st["nee_queries"] - c["nee"]) <= 2e-3 * c["nee"]
    ctx.release_scene(sid)


@pytest.mark.parametrize("rnee", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_rough_adjoint_matches_oracle(ctx, mode, rnee):
    w = P.with_roughness(P.slab_scatterers(n_rays=1200), [0.0, 0.25])
    w = with_rough_nee(w) if rnee else w
    sid, rf, b, ref, rec = run_pair(ctx, w)
    grf = np.random.default_rng(51).normal(size=ref["rf"].shape).astype(np.float32).astype(np.float64)
    g_ref = ref["run"].gradient(grf)
    assert g_ref.shape == (4 * w["M"] + 2,)
    g = ctx.transport_vjp(sid, w["theta"], w["acq"], w["seed"], dev(grf), mode=mode).double().cpu().numpy()
    scale = np.abs(g_ref * np.maximum(np.abs(w["theta"]), 1e-2))
    err = np.abs(g - g_ref) * np.maximum(np.abs(w["theta"]), 1e-2)
    assert np.all(err <= 1e-3 * scale + 1e-4 * scale.max()), np.c_[g, g_ref]
    if rnee:
        assert_rough_nee_matters(w, grf, g_ref, (1e-3 * scale + 1e-4 * scale.max()) / np.maximum(np.abs(w["theta"]), 1e-2))
    ctx.release_scene(sid)


@pytest.mark.parametrize("rnee", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_rough_cylinder_adjoint(ctx, mode, rnee):
    """The hollow cylinder with a rough wall: curved interfaces, refraction into and out of the
    wall, scatterers behind it whose secondary rays cross it; with rnee, secondary rays from the
    wall's events too."""
    w = P.with_roughness(P.hollow_cylinder(n_rays=400), [0.0, 0.2, 0.0])
    w = with_rough_nee(w) if rnee else w
    sid, rf, b, ref, rec = run_pair(ctx, w)
    assert agreement(rec, ref["run"].records()) >= 0.999
    grf = np.random.default_rng(52).normal(size=ref["rf"].shape).astype(np.float32).astype(np.float64)
    g_ref = ref["run"].gradient(grf)
    assert g_ref[-2] != 0.0
    g = ctx.transport_vjp(sid, w["theta"], w["acq"], w["seed"], dev(grf), mode=mode).double().cpu().numpy()
    scale = np.abs(g_ref * np.maximum(np.abs(w["theta"]), 1e-2))
    err = np.abs(g - g_ref) * np.maximum(np.abs(w["theta"]), 1e-2)
    assert np.all(err <= 1e-3 * scale + 1e-4 * scale.max()), np.c_[g, g_ref]
    if rnee:
        assert_rough_nee_matters(w, grf, g_ref, (1e-3 * scale + 1e-4 * scale.max()) / np.maximum(np.abs(w["theta"]), 1e-2))
    ctx.release_scene(sid)


def test_zero_roughness_is_the_smooth_scene(ctx):
    w = P.slab_scatterers(n_rays=300)
    sid0 = ctx.upload_workload(w)
    rf0, _ = ctx.forward(sid0, w["theta"], w["acq"], w["img"], seed=w["seed"])
    wr = P.with_roughness(w, [0.0, 0.0])
    sid1 = ctx.upload_workload(wr)
    rf1, _ = ctx.forward(sid1, wr["theta"], wr["acq"], wr["img"], seed=w["seed"])
    assert torch.equal(rf0, rf1)
    ctx.release_scene(sid0)
    ctx.release_scene(sid1)


@pytest.mark.parametrize("rnee", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_rough_cylinder_radius_gradient(ctx, mode, rnee):
    """Shape through rough events: the sampled facet normal follows the macro normal (its
    tangent frame and tilt) and the microfacet weight's cosines follow it too; with rnee, the
    secondary rays from rough events (the event point on the moving plane, its normal in the
    BSDF) and the balance weights."""
    w = P.with_roughness(P.hollow_cylinder(n_rays=400), [0.0, 0.2, 0.0])
    w = with_rough_nee(w) if rnee else w
    sid, rf, b, ref, rec = run_pair(ctx, w)
    grf = np.random.default_rng(53).normal(size=ref["rf"].shape).astype(np.float32).astype(np.float64)
    tangents = np.stack([w["dtris_dR"], np.random.default_rng(4).normal(size=w["tris"].shape)])
    g_ref = ref["run"].gradient_shape(grf, tangents)
    _, gtris = ctx.transport_vjp_shape(sid, w["theta"], w["acq"], w["seed"], dev(grf), len(w["tris"]), mode=mode)
    got = ctx.shape_param_grad(gtris, dev(tangents)).double().cpu().numpy()
    scale = np.abs(gtris.double().cpu().numpy()[None] * tangents).reshape(2, -1).sum(axis=1)
    assert np.all(np.abs(got - g_ref) <= 2e-3 * np.abs(g_ref) + 2e-4 * scale), np.c_[got, g_ref, scale]
    ctx.release_scene(sid)


@pytest.mark.parametrize("rnee", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_rough_acquisition_gradient(ctx, mode, rnee):
    """Acquisition gradients on a rough scene (the path adjoint's rough + acquisition variant):
    the acquisition slots follow the roughness slots; with rnee, the secondary rays from rough
    events move with their target elements and the balance weights with the element faces."""
    w = P.with_roughness(P.slab_scatterers(n_rays=800), [0.0, 0.25])
    w = with_rough_nee(w) if rnee else w
    sid, rf, b, ref, rec = run_pair(ctx, w)
    grf = np.random.default_rng(54).normal(size=ref["rf"].shape).astype(np.float32).astype(np.float64)
    full = ref["run"].gradient_acq(grf, full=True)
    n_th = len(w["theta"])
    gth, gacq = ctx.transport_vjp_acq(sid, w["theta"], w["acq"], w["seed"], dev(grf), mode=mode)
    ga, fa = gacq.double().cpu().numpy(), full[n_th:]
    assert np.all(np.abs(ga - fa) <= 2e-3 * np.abs(fa) + 1e-4 * np.abs(fa).max()), np.c_[ga, fa]
    g = gth.double().cpu().numpy()
    scale = np.abs(full[:n_th] * np.maximum(np.abs(w["theta"]), 1e-2))
    err = np.abs(g - full[:n_th]) * np.maximum(np.abs(w["theta"]), 1e-2)
    assert np.all(err <= 1e-3 * scale + 1e-4 * scale.max()), np.c_[g, full[:n_th]]
    ctx.release_scene(sid)


def test_rough_scene_through_a_batch(ctx):
    """A rough scene's 4M + 2 parameters through the batched request path (forward, loss and
    adjoint in one request) equal the single calls."""
    from paper_2604_15017_gb300 import usrt

    w = P.with_roughness(P.slab_scatterers(n_rays=300), [0.0, 0.2])
    sid = ctx.upload_workload(w)
    _, bref = ctx.forward(sid, w["theta_target"], w["acq"], w["img"], seed=w["seed"])
    bref = bref.clone()
    out = usrt.Batch(ctx, [dict(scene=sid, theta=w["theta"], acq=w["acq"], img=w["img"], seed=w["seed"],
                                bref=bref)]).run()[0]
    torch.cuda.synchronize()
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    loss, gb = ctx.loss(w["img"], b, bref)
    g, _ = ctx.adjoint(sid, w["theta"], w["acq"], w["img"], w["seed"], rf, gb)
    assert out["grad"].shape == (4 * w["M"] + 2,)
    assert abs(float(out["loss"]) - float(loss)) <= 1e-4 * abs(float(loss))
    assert torch.allclose(out["grad"], g, rtol=1e-3, atol=1e-4 * float(g.abs().max()))
    ctx.release_scene(sid)
