"""GPU parity at the benchmark configurations themselves (against the FP64 oracle).

* the differentiation configuration: the inclusion scene (12 regions, 199,680 triangles, 1e5
  scatterers), one unsteered plane wave, at most 4 interactions, 1e5 rays, 41 parameters;
  forward parity, the transport VJP in record and recompute mode for the oracle's dL/dRF, and
  the whole adjoint chain from the oracle's dL/dB;
* the full inclusion frame (16 plane waves, 16.0M paths, at most 8 interactions, 4096 samples,
  256 x 1024 pixels): every path's event sequence, the whole RF and the whole B-mode image;
* delay-and-sum, its transpose and the envelope/log stage at that frame's dimensions.

Tolerances are those of the hot path (Philox bit-exact, >= 99.99 % identical event sequences,
RF relative L2 <= 1e-4, B-mode <= 0.05 dB above -60 dB, adjoint within 1e-3 of the oracle's FP64
gradient); the DAS bounds follow from the FP32 interpolation position (a few ulps of ~4000
samples) times the interpolation slope.
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda()


def decode(rec):
    r = rec.astype(np.int64) & 0xFFFFFFFF
    return dict(id=r & 0xFFFFF, cls=(r >> 20) & 3, choice=(r >> 22) & 3, aux=(r >> 24) & 0xFF)


def sequence_agreement(gpu_rec, ora):
    """Per path: identical primitive, class, interface choice and secondary-ray element at every
    event the oracle recorded."""
    g = decode(gpu_rec)
    same = (g["cls"] == ora["cls"]) & ((g["id"] == ora["id"]) | (ora["cls"] == 0))
    tri = ora["cls"] == O.CLS_TRI
    same &= ~tri | (g["choice"] == ora["choice"]) | (ora["choice"] == O.CH_NONE)
    scat = ora["cls"] == O.CLS_SCAT
    same &= ~scat | (g["aux"] == np.maximum(ora["aux"], 0)) | (ora["aux"] < 0)
    return same.all(axis=1)


def f32_inputs(w):
    """The workload with every value the C ABI takes as float32 (triangles, scatterers, theta,
    the acquisition's real fields and angles) rounded to float32: the problem the GPU solves,
    which the oracle then solves in FP64."""
    w = dict(w)
    r = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)
    for k in ("tris", "scat_pos", "scat_amp", "theta", "theta_target"):
        if k in w:
            w[k] = r(w[k])
    w["r_s"] = float(np.float32(w["r_s"]))
    acq = dict(w["acq"])
    for k in ("pitch", "h_el", "fs", "bw", "alpha_m", "alpha_c", "c_bf", "split_q"):
        acq[k] = float(np.float32(acq[k]))
    acq["angles"] = [float(np.float32(a)) for a in acq["angles"]]
    w["acq"] = acq
    return w


def ulp_perturbed(w, seed):
    """The float32 workload with every triangle vertex, scatterer position and parameter moved by
    one float32 ulp up or down (seeded signs)."""
    rng = np.random.default_rng(seed)
    w = dict(w)
    for k in ("tris", "scat_pos", "theta"):
        a = np.asarray(w[k], np.float32)
        up = rng.integers(0, 2, size=a.shape).astype(bool)
        w[k] = np.where(up, np.nextafter(a, np.float32(np.inf)), np.nextafter(a, np.float32(-np.inf))).astype(np.float64)
    return w


def check_bmode(bg, bref, tol=0.05, frac=1.0, cap=None):
    """B-mode within tol dB on pixels above -60 dB: on all of them, or on the fraction frac with
    every pixel within cap."""
    live = bref > -60.0
    assert live.mean() > 0.01
    err = np.abs(bg - bref)[live]
    assert np.mean(err <= tol) >= frac, (np.mean(err <= tol), np.sort(err)[-10:])
    assert err.max() <= (tol if cap is None else cap), (err.max(), np.sort(err)[-10:])
    return float(err.max())


def oracle_arrivals(run):
    a = run.arrivals()
    return dict(tx=a["tx"], e=a["e"], tau=a["tau"], a=a["a"], path=a["path"])


def cat(parts):
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def subset(arr, keep):
    return {k: v[keep] for k, v in arr.items()}


def compare_frame(ctx, w, rf, b, agree, ora_arr, rf_ora):
    """Parity of a forward pass whose per-path agreement mask is `agree` (indexed by path).

    On the paths whose event sequences agree (and whose arrivals match within 1e-3 samples and
    1e-3 relative, else they count as disagreeing; at most 0.01 % of all paths disagree): the
    same arrivals (element, transmit), 99 % of the amplitudes within 1e-4; the RF these arrivals
    make within 1e-4 relative L2, and its B-mode within 0.05 dB above -60 dB on 99.99 % of those
    pixels, every one within 0.1 dB.  Over all paths: the
    RF difference is at most 1e-4 of the RF plus the RF of the disagreeing paths' arrivals, each
    side its own (a path whose decisions flip between FP32 and FP64 makes other echoes).
    Returns diagnostics."""
    acq, img = w["acq"], w["img"]
    fs, ne = acq["fs"], acq["n_elem"]
    ga = {k: v.cpu().numpy() for k, v in ctx.arrivals(acq).items()}
    assert len(ga["path"]) == ctx.stats()["arrivals"]
    assert np.all(ga["path"] < len(agree))
    # the GPU keeps arrivals whose time lies within its fixed-point range
    in_range = (ora_arr["tau"] * fs >= -60.0) & (ora_arr["tau"] * fs < (1 << 14) - 70.0)
    # Arrivals are grouped by (path, channel row) and paired in time order within a group.  A
    # group may hold an arrival on one side only, or pair arrivals of different events, where
    # floating point takes a discrete decision inside a secondary ray (total internal reflection
    # at a crossing, the receive cutoff) that the event sequence does not show: such a path
    # joins the disagreeing ones.
    nrow = len(acq["angles"]) * ne
    agree = agree.copy()
    amax = np.abs(ora_arr["a"]).max()
    n_extra = 0
    for _ in range(4):
        g_ok, o_ok = agree[ga["path"]], agree[ora_arr["path"]] & in_range
        gm, om = subset(ga, g_ok), subset(ora_arr, o_ok)
        kgrp_g = gm["path"].astype(np.int64) * nrow + gm["tx"] * ne + gm["e"]
        kgrp_o = om["path"].astype(np.int64) * nrow + om["tx"] * ne + om["e"]
        ug, cg = np.unique(kgrp_g, return_counts=True)
        uo, co = np.unique(kgrp_o, return_counts=True)
        allk = np.union1d(ug, uo)
        cnt_g = np.zeros(len(allk), np.int64)
        cnt_o = np.zeros(len(allk), np.int64)
        cnt_g[np.searchsorted(allk, ug)] = cg
        cnt_o[np.searchsorted(allk, uo)] = co
        flip = np.unique(allk[cnt_g != cnt_o] // nrow)
        if len(flip) == 0:
            kg = np.lexsort((gm["tau"], kgrp_g))
            ko = np.lexsort((om["tau"], kgrp_o))
            dt = np.abs(gm["tau"][kg] - om["tau"][ko]) * fs
            da = np.abs(gm["a"][kg].astype(np.float64) - om["a"][ko])
            rel = da / (np.abs(om["a"][ko]) + 1e-6 * amax)
            # a time off by more than 1e-3 samples, or an amplitude by more than 1e-3, is another
            # event's arrival, another crossing set (a crossing at a triangle edge), or geometry
            # whose FP32 evaluation is ill-conditioned (a receive angle within a few hundredths
            # of a degree of the cutoff, a crossing at the critical angle): counted with the
            # paths that decide differently
            flip = np.unique(om["path"][ko][(dt > 1e-3) | (rel > 1e-3)])
            if len(flip) == 0:
                break
        agree[flip] = False
        n_extra += len(flip)
    else:
        raise AssertionError("arrival pairing did not settle")
    assert agree.mean() >= 0.9999, agree.mean()
    g_ok, o_ok = agree[ga["path"]], agree[ora_arr["path"]] & in_range
    ga_a, oa_a = gm, om
    for k in ("path", "tx", "e"):
        assert np.array_equal(gm[k][kg], om[k][ko]), k
    # FP32 against FP64 on the agreeing paths: times within 1e-3 samples, amplitudes within 1e-3,
    # 99 % of them within 1e-4 (the rest through geometry near a cutoff or critical angle, where
    # the FP32 angle's ~1e-7 rad error is a large part of f_rx or cos(theta_t))
    assert dt.max() <= 1e-3 and rel.max() <= 1e-3
    assert np.mean(rel <= 1e-4) >= 0.99, np.quantile(rel, [0.99, 0.999])
    f0 = w["theta"][3 * w["M"] + 1]

    def gpu_splat(arr):
        return ctx.splat(acq, f0, dev(arr["tx"], torch.int32), dev(arr["e"], torch.int32), dev(arr["tau"]),
                         dev(arr["a"])).double().cpu().numpy()

    rf_g = rf.double().cpu().numpy()
    # the exported arrivals are those the forward pass splatted (us_splat takes their times as
    # float32 seconds, ~1e-4 samples coarser than the transport's fixed-point times)
    assert rel_l2(gpu_splat(ga), rf_g) <= 1e-4
    # the agreeing paths' RF: the forward pass's own RF less the disagreeing paths' arrivals
    # (re-splatting the agreeing ones instead would add the float32 times' phase error)
    rf_g_d = gpu_splat(subset(ga, ~g_ok)) if (~g_ok).any() else np.zeros_like(rf_g)
    rf_g_a = rf_g - rf_g_d
    rf_o_d = O.splat(acq, f0, *[ora_arr[k][~o_ok] for k in ("tx", "e", "tau", "a")])
    rf_o_a = rf_ora - rf_o_d
    err_a = rel_l2(rf_g_a, rf_o_a)
    assert err_a <= 1e-4, err_a
    # B-mode: 0.05 dB on 99.99 % of the live pixels, every one within 0.1 dB.  An arrival time
    # carries the FP32 coordinates' resolution (~3.7e-9 m at 40 mm, a few ps over a path: up to
    # 2.6e-4 samples measured, 2e-4 rad of pulse phase); at the rare dark pixels where strong
    # echoes nearly cancel, that phase error is amplified some 30 times in the envelope
    _, _, b_o_a = O.bmode(acq, img, rf_o_a)
    db_a = check_bmode(ctx.bmode(acq, img, dev(rf_g_a)).cpu().numpy(), b_o_a, frac=0.9999, cap=0.1)
    err_all = float(np.linalg.norm(rf_g - rf_ora))
    bound = 1e-4 * np.linalg.norm(rf_ora) + np.linalg.norm(rf_g_d) + np.linalg.norm(rf_o_d)
    assert err_all <= bound, (err_all, bound)
    _, _, b_o = O.bmode(acq, img, rf_ora)
    live = b_o > -60.0
    diag = dict(agree=float(agree.mean()), n_disagree=int((~agree).sum()), n_secondary_flips=n_extra,
                dt_max=float(dt.max()), rel_q9999=float(np.quantile(rel, 0.9999)), rf_agree=err_a,
                db_agree=db_a, rf_all=rel_l2(rf_g, rf_ora),
                db_all=float(np.abs(b.cpu().numpy() - b_o)[live].max()))
    print(w["name"], diag)
    return diag


# ------------------------------------------------------------------------------------------
# differentiation configuration: 41 parameters, record and recompute
# ------------------------------------------------------------------------------------------
def clear_of_clip(gb, b, dr=60.0, margin=0.1):
    """dL/dB zeroed on pixels within `margin` dB of the dynamic-range clip: there the clip mask
    (no gradient at or below -DR) could differ between two images that agree within 0.05 dB, so
    both sides are given a loss gradient that does not depend on it."""
    return np.where(np.abs(b + dr) > margin, gb, 0.0)


@pytest.fixture(scope="module")
def c3(ctx):
    w = f32_inputs(P.differentiation())
    assert w["M"] == 13 and len(w["theta"]) == 41
    assert w["acq"]["n_elem"] * w["acq"]["n_rays"] >= 100000 and w["acq"]["k_max"] == 4
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    torch.cuda.synchronize()
    sc = O.Scene.from_workload(w)
    ref = O.forward(w, scene=sc)
    tgt = O.forward(w, theta=w["theta_target"], scene=sc)
    _, gb = O.loss(w["img"], ref["b"], tgt["b"])
    gb = clear_of_clip(gb, ref["b"])
    grf = O.bmode_vjp(w["acq"], w["img"], ref["rf"], gb)
    grf32 = grf.astype(np.float32).astype(np.float64)
    g_ref, cond = ref["run"].gradient_cond(grf32)
    g_chain, cond_chain = ref["run"].gradient_cond(grf)
    # the oracle's own spread under one-ulp moves of its float32 inputs: the transport gradient
    # for the same dL/dRF, and the chain for the same dL/dB
    spread = np.zeros_like(g_ref)
    spread_chain = np.zeros_like(g_ref)
    for k in range(3):
        wp = ulp_perturbed(w, 100 + k)
        rp = O.forward(wp, scene=O.Scene.from_workload(wp))
        spread = np.maximum(spread, np.abs(rp["run"].gradient(grf32) - g_ref))
        gp = rp["run"].gradient(O.bmode_vjp(w["acq"], w["img"], rp["rf"], gb))
        spread_chain = np.maximum(spread_chain, np.abs(gp - g_chain))
    yield dict(w=w, sid=sid, rf=rf, b=b, ref=ref, gb=gb, grf32=grf32, g_ref=g_ref, cond=cond, g_chain=g_chain,
               cond_chain=cond_chain, spread=spread, spread_chain=spread_chain)
    ctx.release_scene(sid)


def test_c3_forward_parity(ctx, c3):
    w, ref = c3["w"], c3["ref"]
    acq = w["acq"]
    n_paths = acq["n_elem"] * acq["n_rays"]
    # arrivals of this forward pass (the fixture's call) before any other call runs
    rf, b = ctx.forward(c3["sid"], w["theta"], acq, w["img"], seed=w["seed"], keep_record=True)
    rec = ctx.record(0, n_paths, acq["k_max"]).cpu().numpy()
    agree = sequence_agreement(rec, ref["run"].records())
    assert agree.mean() >= 0.9999, (agree.mean(), np.flatnonzero(~agree)[:10])
    st = ctx.stats()
    assert st["status"] == 0 and st["dropped"] == 0
    compare_frame(ctx, w, rf, b, agree, oracle_arrivals(ref["run"]), ref["rf"])


def assert_gradient(g, g_ref, cond, spread, rel=1e-3, floor=2e-5):
    """Per component: within rel of the oracle's FP64 gradient, plus floor times the component's
    condition (the sum over arrivals of |contribution|: FP32 sums of terms that cancel cannot
    resolve less), plus twice the spread of the FP64 gradient itself when the float32 inputs move
    by one ulp (paths near a critical angle or an edge flip their decisions and carry
    derivative terms in 1 / cos(theta_t): FP32 arithmetic cannot resolve a component more
    finely than its own input precision does).  Returns (number of components whose spread is
    below rel |g_ref|, largest err / |g_ref| among those)."""
    err = np.abs(g - g_ref)
    bad = err > rel * np.abs(g_ref) + floor * cond + 2.0 * spread
    assert not bad.any(), np.c_[np.flatnonzero(bad), g[bad], g_ref[bad], cond[bad], spread[bad]]
    well = spread <= rel * np.abs(g_ref)
    return int(well.sum()), float((err[well] / np.abs(g_ref[well])).max(initial=0.0))


@pytest.mark.parametrize("mode", [0, 1])
def test_c3_transport_vjp_41_parameters(ctx, c3, mode):
    w = c3["w"]
    if mode == 0:  # a record-mode adjoint needs the forward pass of these inputs, kept
        ctx.forward(c3["sid"], w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    g = ctx.transport_vjp(c3["sid"], w["theta"], w["acq"], w["seed"], dev(c3["grf32"]), mode=mode)
    g = g.double().cpu().numpy()
    assert len(g) == 41
    print("c3 transport vjp mode", mode, "well-conditioned components, worst relative error:",
          assert_gradient(g, c3["g_ref"], c3["cond"], c3["spread"]))


def test_c3_adjoint_chain_from_the_oracle_image_gradient(ctx, c3):
    """The whole backward chain (envelope/log VJP on the GPU's own image, transposed DAS, splat
    and path adjoints) for the oracle's dL/dB, against the oracle's chain."""
    w = c3["w"]
    rf, _ = ctx.forward(c3["sid"], w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
    g, _ = ctx.adjoint(c3["sid"], w["theta"], w["acq"], w["img"], w["seed"], rf, dev(c3["gb"]), mode=0)
    print("c3 chain: well-conditioned components, worst relative error:",
          assert_gradient(g.double().cpu().numpy(), c3["g_chain"], c3["cond_chain"], c3["spread_chain"]))


# ------------------------------------------------------------------------------------------
# the full inclusion frame: every path, the whole RF and B-mode
# ------------------------------------------------------------------------------------------
def test_c2_full_frame(ctx):
    w = f32_inputs(P.inclusions())
    acq, img = w["acq"], w["img"]
    n_paths = len(acq["angles"]) * acq["n_elem"] * acq["n_rays"]
    assert n_paths == 16 * 128 * 7813
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], acq, img, seed=w["seed"], keep_record=True)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["n_paths"] == n_paths and st["status"] == 0 and st["dropped"] == 0
    sc = O.Scene.from_workload(w)
    rf_ref = np.zeros(ctx.rf_shape(acq))
    chunk = 2_000_000
    agree = np.zeros(n_paths, bool)
    parts = []
    for lo in range(0, n_paths, chunk):
        hi = min(n_paths, lo + chunk)
        run = O.Run(sc, w["theta"], w["M"], acq, w["seed"], path_lo=lo, path_hi=hi)
        rec = ctx.record(lo, hi - lo, acq["k_max"]).cpu().numpy()
        agree[lo:hi] = sequence_agreement(rec, run.records())
        rf_ref += run.rf()
        parts.append(oracle_arrivals(run))
        del run
    assert agree.mean() >= 0.9999, agree.mean()
    compare_frame(ctx, w, rf, b, agree, cat(parts), rf_ref)
    ctx.release_scene(sid)


# ------------------------------------------------------------------------------------------
# image stages at the full frame's dimensions
# ------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c2_image_case():
    w = P.inclusions(n_rays=1)
    acq, img = w["acq"], w["img"]
    rng = np.random.default_rng(31)
    n = 200000
    rf = O.splat(acq, 5e6, rng.integers(0, len(acq["angles"]), n), rng.integers(0, acq["n_elem"], n),
                 rng.uniform(0, acq["n_samples"] / acq["fs"], n), rng.normal(size=n))
    rf = rf.astype(np.float32).astype(np.float64)
    irf = O.das(acq, img, rf)
    return acq, img, rf, irf


def test_c2_das(ctx, c2_image_case):
    acq, img, rf, irf = c2_image_case
    got = ctx.das(acq, img, dev(rf)).double().cpu().numpy()
    bound = 2e-3 * O.das(acq, img, np.abs(rf)) + 1e-6 * np.abs(irf).max()
    assert np.all(np.abs(got - irf) <= bound), np.max(np.abs(got - irf) - bound)
    assert rel_l2(got, irf) <= 1e-4


def dilated(a):
    """max over each sample and its two neighbours along the time axis"""
    m = a.copy()
    m[..., 1:] = np.maximum(m[..., 1:], a[..., :-1])
    m[..., :-1] = np.maximum(m[..., :-1], a[..., 1:])
    return m


def das_adjoint_bound(acq, img, gi, ref):
    """A tap whose FP32 interpolation position (error ~1e-3 samples) falls into the neighbouring
    interval moves a share of at most that error times w |g| onto the next sample: every entry is
    bounded by 2e-3 of the transposed |gi| at that sample or a neighbour."""
    return 2e-3 * dilated(O.das_adjoint(acq, img, np.abs(gi))) + 1e-6 * np.abs(ref).max()


def test_c2_das_adjoint(ctx, c2_image_case):
    acq, img, rf, irf = c2_image_case
    rng = np.random.default_rng(32)
    gi = rng.normal(size=(img["n_lines"], img["n_depth"])).astype(np.float32).astype(np.float64)
    ref = O.das_adjoint(acq, img, gi)
    got = ctx.das_adjoint(acq, img, dev(gi)).double().cpu().numpy()
    bound = das_adjoint_bound(acq, img, gi, ref)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)
    assert rel_l2(got, ref) <= 2e-4


def test_c2_envlog(ctx, c2_image_case):
    acq, img, rf, irf = c2_image_case
    irf32 = irf.astype(np.float32).astype(np.float64)
    bref, _ = O.log_compress(img, O.envelope(img, irf32))
    got = ctx.envlog(img, dev(irf32)).cpu().numpy()
    check_bmode(got, bref)
    assert np.max(np.abs(got - bref)) <= 0.05 + 1e-6
