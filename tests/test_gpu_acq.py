"""Acquisition-parameter gradients on the GPU (the beamforming sound speed c_bf, the element
pitch and the steering angles, through the emission of Sec. 2.3.1, the secondary rays' target
elements of Sec. 2.3.3 and the delays of Eq. das) against the FP64 oracle's derivatives, which
tests/test_oracle_acq_pins.py pins to finite differences.

The DAS part's slope is that of the interpolation interval holding each delay, so GPU and
oracle must place the delays in the same intervals: the geometry is given in float32-exact
values (the library takes pitch, image corners and angles as float32), and the angles are
float32 values whose sine is a float32 to ~1e-13 (the library rounds sin and cos to float32
before the delays).  With ordinary values a delay shifts by ~1e-6 samples and about one tap in
3e5 lands in the neighbouring interval, moving a component by ~0.3 %.  Tolerances:

* DAS part: 1e-3 relative per component (FP32 sums over ~1e5 taps; the delays agree to ~1e-7
  samples, so the interpolation intervals are the oracle's).
* transport part: 2e-3 relative per component, as the scene gradient's 1e-3 with the time
  adjoint's extra FP32 steps; its scene slots equal us_transport_vjp's up to summation order.
* full chain: its parts on the same inputs as the oracle's, within 2e-3 of the two parts'
  magnitudes (they cancel in some components).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15017_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

MM = 1e-3


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_15017_gb300 import usrt

    c = usrt.Context(0)
    yield c
    c.close()


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda()


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def exact_sine_angle(deg):
    """The float32 angle near `deg` degrees whose sine is closest to a float32 value."""
    if deg == 0:
        return 0.0
    t = np.float32(np.deg2rad(deg))
    c = (t + np.arange(-50000, 50000, dtype=np.float64) * float(np.spacing(t))).astype(np.float32).astype(np.float64)
    s = np.sin(c)
    return float(c[np.argmin(np.abs(s - s.astype(np.float32).astype(np.float64)))])


def exact_angles(degs):
    return [exact_sine_angle(d) for d in degs]


def within(got, ref, rel, floor=0.0):
    err = np.abs(np.asarray(got, np.float64) - ref)
    return np.all(err <= rel * np.abs(ref) + floor * np.abs(ref).max())


@pytest.mark.parametrize("n_tx,n_lines,n_depth,f_number", [(3, 24, 128, 0.0), (20, 37, 256, 0.0), (3, 24, 128, 1.5)])
def test_das_acq_vjp_matches_oracle(ctx, n_tx, n_lines, n_depth, f_number):
    """20 transmits with a ragged tail; 37 x 256 pixels: a ragged last block; F-number 1.5: the
    dynamic aperture, whose weights move with the pitch too."""
    degs = [-9.0, 0.0, 11.0] if n_tx == 3 else list(np.linspace(-15, 15, n_tx - 1)) + [0.0]
    acq = dict(P.acquisition(32, float(np.float32(0.3 * MM)), 1024, degs, 1, 1, 1540.0), angles=exact_angles(degs))
    img = P.image(n_lines, n_depth, *(float(np.float32(v)) for v in (-4 * MM, 4 * MM, 2 * MM, 18 * MM)),
                  f_number=f_number)
    rng = np.random.default_rng(n_tx)
    n = 3000 * n_tx
    rf = f32(O.splat(acq, 5e6, rng.integers(0, n_tx, n), rng.integers(0, 32, n), rng.uniform(0, 1024 / 40e6, n),
                     rng.normal(size=n)))
    gi = f32(rng.normal(size=(n_lines, n_depth)))
    ref = O.das_acq_vjp(acq, img, rf, gi)
    got = ctx.das_acq_vjp(acq, img, dev(rf), dev(gi)).double().cpu().numpy()
    assert within(got, ref, 1e-3), np.c_[got, ref]


def test_das_and_transposed_das_with_a_dynamic_aperture(ctx):
    """F-number 1.2 (aperture clamped to one pitch above 0.72 mm): DAS per pixel within the
    interpolation bound of the fixed-window test, and the transposed DAS, on both the direct and
    the TMA-staged kernels."""
    from paper_2604_15017_gb300 import usrt

    degs = [-8.0, 0.0, 8.0]
    acq = dict(P.acquisition(32, float(np.float32(0.3 * MM)), 1024, degs, 1, 1, 1540.0), angles=exact_angles(degs))
    img = P.image(37, 256, *(float(np.float32(v)) for v in (-4 * MM, 4 * MM, 0.3 * MM, 18 * MM)), f_number=1.2)
    rng = np.random.default_rng(41)
    n = 9000
    rf = f32(O.splat(acq, 5e6, rng.integers(0, 3, n), rng.integers(0, 32, n), rng.uniform(0, 1024 / 40e6, n),
                     rng.normal(size=n)))
    ref = O.das(acq, img, rf)
    bound = 2e-3 * O.das(acq, img, np.abs(rf)) + 1e-6 * np.abs(ref).max()
    for tma in (0, 1):
        ctx.set_option(usrt.OPT_DAS_TMA, tma)
        got = ctx.das(acq, img, dev(rf)).cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound), (tma, np.max(np.abs(got - ref) - bound))
    ctx.set_option(usrt.OPT_DAS_TMA, 0)  # the library's default
    gi = f32(rng.normal(size=ref.shape))
    adj = ctx.das_adjoint(acq, img, dev(gi)).double().cpu().numpy()
    aref = O.das_adjoint(acq, img, gi)
    assert np.linalg.norm(adj - aref) <= 1e-3 * np.linalg.norm(aref)


def slab_with_angles(n_rays, degs):
    """The slab phantom with float32-exact pitch and image corners and exact-sine angles."""
    w = P.slab_scatterers(n_rays=n_rays)
    w["acq"] = dict(w["acq"], angles=exact_angles(degs), pitch=float(np.float32(w["acq"]["pitch"])))
    w["img"] = dict(w["img"], **{k: float(np.float32(w["img"][k])) for k in ("x0", "x1", "z0", "z1")})
    return w


@pytest.mark.parametrize("mode", [0, 1])
def test_transport_vjp_acq_matches_oracle(ctx, mode):
    w = slab_with_angles(1500, [-6.0, 0.0, 7.0])
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    ref = O.forward(w)
    grf = f32(np.random.default_rng(21).normal(size=ref["rf"].shape))
    full = ref["run"].gradient_acq(grf, full=True)
    n_th = len(w["theta"])
    gth, gacq = ctx.transport_vjp_acq(sid, w["theta"], w["acq"], w["seed"], dev(grf), mode=mode)
    assert within(gacq.double().cpu().numpy(), full[n_th:], 2e-3), np.c_[gacq.cpu().numpy(), full[n_th:]]
    # the scene slots are those of the plain transport VJP up to FP32 summation order (the
    # active-path list and, in recompute mode, the job order come from atomics): 1e-4, as for
    # the record-mode image reuse in test_gpu_parity.py
    g_plain = ctx.transport_vjp(sid, w["theta"], w["acq"], w["seed"], dev(grf), mode=mode)
    assert torch.allclose(gth, g_plain, rtol=1e-4, atol=1e-5 * float(g_plain.abs().max()))
    ctx.release_scene(sid)


@pytest.mark.parametrize("mode", [0, 1])
def test_adjoint_acq_end_to_end(ctx, mode):
    """The full chain equals its two parts issued by hand (same kernels, FP32 summation order
    aside), and each part matches the oracle's on the same inputs (the GPU's RF, dL/dI_rf and
    dL/dRF; the envelope/log VJP that makes them is parity-tested on its own).  The DAS and
    transport parts cancel to a few per cent in some components (a longer array moves where
    echoes are recorded and where the beamformer looks alike), so the bound is relative to
    |DAS part| + |transport part|."""
    w = slab_with_angles(800, [-5.0, 0.0, 4.0])
    sid = ctx.upload_workload(w)
    acq, img = w["acq"], w["img"]
    rf, b = ctx.forward(sid, w["theta"], acq, img, seed=w["seed"], keep_record=True)
    ref = O.forward(w)
    rng = np.random.default_rng(22)
    gb_d = dev(rng.normal(size=ref["b"].shape) * (ref["b"] > -60))
    gth, gacq = ctx.adjoint_acq(sid, w["theta"], acq, img, w["seed"], rf, gb_d, mode=mode)
    got = gacq.double().cpu().numpy()
    # the two parts by hand
    gi_d = ctx.envlog_vjp(img, ctx.das(acq, img, rf), gb_d)
    grf_d = ctx.das_adjoint(acq, img, gi_d)
    p_das = ctx.das_acq_vjp(acq, img, rf, gi_d).double().cpu().numpy()
    p_tr = ctx.transport_vjp_acq(sid, w["theta"], acq, w["seed"], grf_d, mode=mode)[1].double().cpu().numpy()
    size = np.abs(p_das) + np.abs(p_tr)
    assert np.all(np.abs(got - (p_das + p_tr)) <= 1e-4 * size + 1e-6 * size.max()), np.c_[got, p_das + p_tr]
    # each part against the oracle on the same inputs
    rf_g, gi_g, grf_g = (t.double().cpu().numpy() for t in (rf, gi_d, grf_d))
    g_das = O.das_acq_vjp(acq, img, rf_g, gi_g)
    g_tr = ref["run"].gradient_acq(grf_g)
    size = np.abs(g_das) + np.abs(g_tr)
    assert np.all(np.abs(got - (g_das + g_tr)) <= 2e-3 * size + 1e-4 * size.max()), np.c_[got, g_das + g_tr, g_das]
    # the scene part equals the plain adjoint's
    gth_plain, _ = ctx.adjoint(sid, w["theta"], acq, img, w["seed"], rf, gb_d, mode=mode)
    assert torch.allclose(gth, gth_plain, rtol=1e-4, atol=1e-5 * float(gth_plain.abs().max()))
    ctx.release_scene(sid)


def test_acq_gradient_is_refused_without_an_output(ctx):
    from paper_2604_15017_gb300 import usrt

    w = P.two_layer(n_rays=50)
    sid = ctx.upload_workload(w)
    grf = torch.zeros(ctx.rf_shape(w["acq"]), device="cuda")
    th = usrt._f32(w["theta"])
    ad, ang = usrt.acq_desc(w["acq"])
    gth = torch.empty(len(th), device="cuda")
    import ctypes as C

    rc = usrt.lib().us_transport_vjp_acq(ctx.h, int(sid), th.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ad), 1,
                                         1, usrt._ptr(grf), usrt._ptr(gth), None, None)
    assert rc == usrt.US_ERR_ARG
    ctx.release_scene(sid)
