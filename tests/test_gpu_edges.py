"""Edge cases of the CUDA path against the FP64 oracle: ragged sizes (records, image lines and
element counts that fill no tile), scenes with scatterers but no triangles and with nothing at
all, one ray per element, the smallest and largest interaction budgets, more transmits than
the tiled kernels stage, tiny sample records, and an empty batch.  Tolerances as in
test_gpu_parity.py."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda()


def no_triangles(w):
    w = dict(w)
    w["tris"] = np.zeros((0, 9))
    w["media"] = np.zeros((0, 2), dtype=np.int32)
    return w


def parity(ctx, w, seq_min=0.9999):
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    torch.cuda.synchronize()
    ref = O.forward(w)
    st = ctx.stats()
    assert st["status"] == 0 and st["dropped"] == 0
    acq = w["acq"]
    n_paths = len(acq["angles"]) * acq["n_elem"] * acq["n_rays"]
    rec = ctx.record(0, n_paths, acq["k_max"]).cpu().numpy()
    ora = ref["run"].records()
    r = rec.astype(np.int64) & 0xFFFFFFFF
    same = (((r >> 20) & 3) == ora["cls"]) & (((r & 0xFFFFF) == ora["id"]) | (ora["cls"] == 0))
    assert same.all(axis=1).mean() >= seq_min
    rf_g = rf.double().cpu().numpy()
    if np.abs(ref["rf"]).max() == 0:
        assert np.all(rf_g == 0)
    else:
        assert rel_l2(rf_g, ref["rf"]) <= 1e-4, rel_l2(rf_g, ref["rf"])
        live = ref["b"] > -60.0
        assert np.max(np.abs(b.cpu().numpy() - ref["b"])[live]) <= 0.05
    ctx.release_scene(sid)
    return ref


def test_ragged_record_image_and_element_count(ctx):
    # 2044 samples (not a multiple of the splat's 8 samples per thread), 37 lines (not a multiple
    # of the DAS tiles), 20 elements
    ref = parity(ctx, P.two_layer(n_rays=300, n_samples=2044, n_lines=37, n_depth=256, n_elem=20))
    assert np.abs(ref["rf"]).max() > 0


def test_scatterers_without_triangles(ctx):
    parity(ctx, no_triangles(P.slab_scatterers(n_rays=600)))


def test_empty_scene_records_nothing(ctx):
    w = no_triangles(P.two_layer(n_rays=50))
    ref = parity(ctx, w)
    assert np.abs(ref["rf"]).max() == 0


def test_one_ray_per_element_and_budget_of_one_interaction(ctx):
    ref = parity(ctx, no_triangles(P.slab_scatterers(n_rays=1, n_scat=20000, k_max=1)))
    assert np.abs(ref["rf"]).max() > 0


def test_largest_interaction_budget(ctx):
    w = P.inclusions(n_regions=3, n_scat=2000, n_rays=60, k_max=15, n_samples=2048, angles_deg=[0.0], n_lines=64,
                     n_depth=512, n_elem=32, n_lat=24, n_lon=40)
    parity(ctx, w)


def test_twenty_transmits_das_and_transposed_das(ctx):
    acq = P.acquisition(24, 0.3 * MM, 1024, list(np.linspace(-15, 15, 20)), 1, 1, 1540.0)
    img = P.image(37, 256, -3.5 * MM, 3.5 * MM, 1 * MM, 18 * MM)
    rng = np.random.default_rng(9)
    n = 8000
    rf = O.splat(acq, 5e6, rng.integers(0, 20, n), rng.integers(0, 24, n), rng.uniform(0, 1024 / 40e6, n),
                 rng.normal(size=n)).astype(np.float32).astype(np.float64)
    ref = O.das(acq, img, rf)
    bound = 2e-3 * O.das(acq, img, np.abs(rf)) + 1e-6 * np.abs(ref).max()
    got = ctx.das(acq, img, dev(rf)).cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound)
    gi = rng.normal(size=ref.shape).astype(np.float32).astype(np.float64)
    adj = ctx.das_adjoint(acq, img, dev(gi)).double().cpu().numpy()
    aref = O.das_adjoint(acq, img, gi)
    assert rel_l2(adj, aref) <= 1e-3


@pytest.mark.parametrize("ns", [4, 1020])
def test_splat_tiny_and_ragged_records(ctx, ns):
    acq = P.acquisition(6, 0.3 * MM, ns, [0.0, 4.0], 1, 1, 1540.0)
    rng = np.random.default_rng(ns)
    n = 3000
    tx = rng.integers(0, 2, n).astype(np.int32)
    e = rng.integers(0, 6, n).astype(np.int32)
    tau = rng.uniform(-1e-6, ns / 40e6 + 1e-6, n).astype(np.float32).astype(np.float64)
    a = rng.normal(size=n).astype(np.float32).astype(np.float64)
    ref = O.splat(acq, 5e6, tx, e, tau, a)
    got = ctx.splat(acq, 5e6, dev(tx, torch.int32), dev(e, torch.int32), dev(tau), dev(a)).cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


def test_empty_batch_is_a_no_op(ctx):
    from paper_2604_15017_gb300 import usrt

    assert usrt.Batch(ctx, []).run() == []


def test_second_stream_gives_the_sequential_results(ctx):
    """Secondary rays and their job sort on the lane's second stream (the default) against the
    same call with everything on one stream: RF and gradient equal up to FP32 summation order
    (the arrival and job orders come from atomics either way)."""
    from paper_2604_15017_gb300 import usrt

    w = P.slab_scatterers(n_rays=600)
    sid = ctx.upload_workload(w)
    out = {}
    for opt in (0, 100):
        ctx.set_option(usrt.OPT_NEE_STREAM, opt)
        rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
        gb = torch.ones_like(b) * (b > -60)
        g, _ = ctx.adjoint(sid, w["theta"], w["acq"], w["img"], w["seed"], rf, gb)
        torch.cuda.synchronize()
        out[opt] = (rf.clone(), g.clone(), ctx.stats())
    ctx.set_option(usrt.OPT_NEE_STREAM, 100)
    (rf0, g0, s0), (rf1, g1, s1) = out[0], out[100]
    assert s0["segments"] == s1["segments"] and s0["nee_queries"] == s1["nee_queries"]
    assert s0["arrivals"] == s1["arrivals"]
    assert float((rf0 - rf1).norm()) <= 1e-5 * float(rf0.norm())
    assert torch.allclose(g0, g1, rtol=1e-4, atol=1e-5 * float(g0.abs().max()))
    ctx.release_scene(sid)


def test_element_sub_apertures_partition_the_frame(ctx):
    """Micro-batches over emitting elements (sub-apertures with one seed) add up to the full
    aperture's RF and gradient for one dL/dRF, as the oracle's do; a sub-aperture past the array
    is refused."""
    from paper_2604_15017_gb300 import optim, usrt

    w = P.slab_scatterers(n_rays=300)
    sid = ctx.upload_workload(w)
    rf_full, _ = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    grf = torch.randn_like(rf_full)
    g_full = ctx.transport_vjp(sid, w["theta"], w["acq"], w["seed"], grf)
    rf_sum = torch.zeros_like(rf_full)
    g_sum = torch.zeros_like(g_full)
    for a in optim.split_elements(w["acq"], 3):
        rf, _ = ctx.forward(sid, w["theta"], a, w["img"], seed=w["seed"], keep_record=True)
        rf_sum += rf
        g_sum += ctx.transport_vjp(sid, w["theta"], a, w["seed"], grf)
    torch.cuda.synchronize()
    assert float((rf_sum - rf_full).norm()) <= 1e-5 * float(rf_full.norm())
    assert torch.allclose(g_sum, g_full, rtol=1e-4, atol=1e-5 * float(g_full.abs().max()))
    bad = dict(w["acq"], tx_elem=60, n_tx_elem=8)
    with pytest.raises(usrt.UsrtError):
        ctx.forward(sid, w["theta"], bad, w["img"], seed=w["seed"])
    ctx.release_scene(sid)


def test_adjoint_reads_no_stale_workspace(ctx):
    """The transport VJP on a context whose workspaces hold a deeper pass's data, against the
    oracle.  Paths whose last event (at k_max) is a scatterer started no secondary ray there,
    so no seed may be read for that event from the buffer a previous call left."""
    # dense scatterers (mean free path ~0.4 mm): many paths cross the layer interface, scatter
    # and end at a scatterer at k_max = 2; the deeper pass before it (half the paths, K_max 6)
    # leaves secondary-ray seeds of its events 4 and 5 where the shallow pass keeps its k_max
    # events
    w = P.slab_scatterers(n_rays=300, n_scat=200000, k_max=2)
    big = P.slab_scatterers(n_rays=150, n_scat=200000, k_max=6)
    sid = ctx.upload_workload(big)
    rf, b = ctx.forward(sid, big["theta"], big["acq"], big["img"], seed=big["seed"], keep_record=True)
    ctx.transport_vjp(sid, big["theta"], big["acq"], big["seed"], torch.randn_like(rf) * 1e6)  # large seeds
    ctx.release_scene(sid)
    sid = ctx.upload_workload(w)
    rf, _ = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    acq = w["acq"]
    rec = ctx.record(0, len(acq["angles"]) * acq["n_elem"] * acq["n_rays"], acq["k_max"]).cpu().numpy()
    cls = ((rec.astype(np.int64) & 0xFFFFFFFF) >> 20) & 3
    assert ((cls[:, -1] == 3) & (cls[:, 1] == 3)).mean() > 0.03  # swept paths that end so
    ref = O.forward(w)
    grf = np.random.default_rng(61).normal(size=ref["rf"].shape).astype(np.float32).astype(np.float64)
    g_ref = ref["run"].gradient(grf)
    g = ctx.transport_vjp(sid, w["theta"], acq, w["seed"], dev(grf)).double().cpu().numpy()
    scale = np.abs(g_ref * w["theta"])
    err = np.abs(g - g_ref) * np.abs(w["theta"])
    assert np.all(err <= 1e-3 * scale + 1e-4 * scale.max()), np.c_[g, g_ref]
    ctx.release_scene(sid)
