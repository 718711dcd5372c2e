"""Shape gradients on the GPU (dL/d(triangle vertices), fixed-sample; row N2) against the FP64
oracle's directional derivatives, which tests/test_oracle_shape_pins.py pins to finite
differences.  The GPU returns the whole vertex gradient; it is compared through contractions
with tangent fields (us_shape_param_grad, the chain rule to shape parameters): the slab's
interface depth, random motions of every vertex, single vertex coordinates, and the radius of
the hollow cylinder.  Tolerance: 2e-3 of the derivative plus 2e-4 of sum |dL/dv * dv/dq| (the
contraction cancels; the per-vertex sums carry FP32 rounding and atomics in any order)."""
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


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def slab_tangents(w, seed=1, n_random=2):
    t = w["tris"]
    depth = np.zeros_like(t)
    for k in range(3):
        depth[np.isclose(t[:, 3 * k + 2], 20e-3), 3 * k + 2] = 1.0
    rng = np.random.default_rng(seed)
    return [depth] + [rng.normal(size=t.shape) for _ in range(n_random)]


def compare(ctx, gtris, tangents, ref):
    tan = np.stack(tangents)
    got = ctx.shape_param_grad(gtris, dev(tan)).double().cpu().numpy()
    g = gtris.double().cpu().numpy()
    scale = np.abs(g[None] * tan).reshape(len(tan), -1).sum(axis=1)
    err = np.abs(got - ref)
    assert np.all(err <= 2e-3 * np.abs(ref) + 2e-4 * scale), np.c_[got, ref, scale]
    return got


@pytest.mark.parametrize("mode", [0, 1])
def test_transport_vjp_shape_matches_oracle(ctx, mode):
    w = P.slab_scatterers(n_rays=1500)
    sid = ctx.upload_workload(w)
    ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    ref = O.forward(w)
    grf = f32(np.random.default_rng(31).normal(size=ref["rf"].shape))
    tangents = slab_tangents(w)
    # single coordinates: the z of the two top-face triangles' first vertices, an x
    top = np.nonzero(np.isclose(w["tris"][:, 2], 20e-3) & np.isclose(w["tris"][:, 5], 20e-3))[0]
    for i, a in ((top[0], 2), (top[1], 2), (top[0], 0)):
        e = np.zeros_like(w["tris"])
        e[i, a] = 1.0
        tangents.append(e)
    g_ref = ref["run"].gradient_shape(grf, np.stack(tangents))
    gth, gtris = ctx.transport_vjp_shape(sid, w["theta"], w["acq"], w["seed"], dev(grf), len(w["tris"]), mode=mode)
    compare(ctx, gtris, tangents, g_ref)
    g_plain = ctx.transport_vjp(sid, w["theta"], w["acq"], w["seed"], dev(grf), mode=mode)
    assert torch.allclose(gth, g_plain, rtol=1e-4, atol=1e-5 * float(g_plain.abs().max()))
    ctx.release_scene(sid)


@pytest.mark.parametrize("mode", [0, 1])
def test_hollow_cylinder_radius_gradient(ctx, mode):
    """The tube's radius (both surfaces): secondary rays from the tissue cross the wall twice
    on their way back, so the crossing terms of the secondary-ray adjoint carry much of it."""
    w = P.hollow_cylinder(n_rays=400)
    sid = ctx.upload_workload(w)
    ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    ref = O.forward(w)
    grf = f32(np.random.default_rng(32).normal(size=ref["rf"].shape))
    tangents = [w["dtris_dR"], np.random.default_rng(3).normal(size=w["tris"].shape)]
    g_ref = ref["run"].gradient_shape(grf, np.stack(tangents))
    _, gtris = ctx.transport_vjp_shape(sid, w["theta"], w["acq"], w["seed"], dev(grf), len(w["tris"]), mode=mode)
    compare(ctx, gtris, tangents, g_ref)
    ctx.release_scene(sid)


def test_adjoint_shape_equals_its_parts(ctx):
    w = P.hollow_cylinder(n_rays=300)
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    gb = torch.randn_like(b) * (b > -60)
    gth, gtris = ctx.adjoint_shape(sid, w["theta"], w["acq"], w["img"], w["seed"], rf, gb, len(w["tris"]))
    grf = ctx.bmode_vjp(w["acq"], w["img"], rf, gb)
    gth2, gtris2 = ctx.transport_vjp_shape(sid, w["theta"], w["acq"], w["seed"], grf, len(w["tris"]))
    tan = dev(np.stack([w["dtris_dR"]]))
    a, b2 = ctx.shape_param_grad(gtris, tan), ctx.shape_param_grad(gtris2, tan)
    size = float((gtris.abs() * tan[0].abs()).sum())
    assert abs(float(a[0]) - float(b2[0])) <= 1e-4 * size
    assert torch.allclose(gth, gth2, rtol=1e-4, atol=1e-5 * float(gth2.abs().max()))
    # the oracle on the GPU's dL/dRF
    ref = O.forward(w)
    g_ref = ref["run"].gradient_shape(grf.double().cpu().numpy(), w["dtris_dR"][None])
    assert abs(float(a[0]) - g_ref[0]) <= 2e-3 * abs(g_ref[0]) + 2e-4 * size
    ctx.release_scene(sid)


def test_shape_param_grad_contracts_in_a_fixed_order(ctx):
    rng = np.random.default_rng(7)
    n = 12345
    g = f32(rng.normal(size=(n, 9)))
    tan = f32(rng.normal(size=(3, n, 9)))
    out1 = ctx.shape_param_grad(dev(g), dev(tan))
    out2 = ctx.shape_param_grad(dev(g), dev(tan))
    assert torch.equal(out1, out2)
    ref = np.einsum("ij,kij->k", g, tan)
    assert np.allclose(out1.double().cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(g).sum() / n ** 0.5)
