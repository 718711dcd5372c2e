"""Serving loop on the GPU: a request's outputs in a served mix (continuous batching over lanes,
overlapping requests of different scenes and kinds) equal its outputs when run alone, and the
memory admission bound holds."""
import numpy as np
import pytest
import torch

from paper_2604_15017_gb300 import phantoms as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_15017_gb300 import usrt

    c = usrt.Context(0)
    yield c
    c.close()


def _workloads(ctx, n, seed):
    ws = P.batch_workloads(n=n, seed=seed, scale=0.01)
    items, singles = [], []
    for w in ws:
        sid = ctx.upload_workload(w)
        it = dict(scene=sid, theta=w["theta"], acq=w["acq"], img=w["img"], seed=w["seed"])
        if w["adjoint"]:
            _, bref = ctx.forward(sid, w["theta_target"], w["acq"], w["img"], seed=w["seed"])
            it["bref"] = bref.clone()
            rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"], keep_record=True)
            loss, gb = ctx.loss(w["img"], b, it["bref"])
            g, _ = ctx.adjoint(sid, w["theta"], w["acq"], w["img"], w["seed"], rf, gb)
            single = dict(rf=rf.clone(), bmode=b.clone(), loss=loss.clone(), grad=g.clone())
        else:
            rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=w["seed"])
            single = dict(rf=rf.clone(), bmode=b.clone())
        items.append(it)
        singles.append(single)
    torch.cuda.synchronize()
    return ws, items, singles


def _check(w, out, single):
    rf, b, loss, grad = out
    a, r = rf.double().cpu().numpy(), single["rf"].double().cpu().numpy()
    assert np.linalg.norm(a - r) <= 1e-5 * np.linalg.norm(r) + 1e-30
    assert float((b - single["bmode"]).abs().max()) <= 0.05
    if w["adjoint"]:
        assert abs(float(loss) - float(single["loss"])) <= 1e-4 * abs(float(single["loss"])) + 1e-6
        g1, g2 = grad.double().cpu().numpy(), single["grad"].double().cpu().numpy()
        th = np.abs(w["theta"])
        assert np.all(np.abs(g1 - g2) * th <= 1e-3 * np.abs(g2) * th + 1e-4 * np.max(np.abs(g2) * th))


def test_served_mix_matches_requests_alone(ctx):
    from paper_2604_15017_gb300 import serve

    ws, items, singles = _workloads(ctx, 8, seed=21)
    srv = serve.Server(ctx, n_lanes=3, keep_outputs=True)
    srv.warmup(items)
    # a burst of four, then the rest spaced so that they arrive while earlier ones still run
    arrivals = [(0.0, it) for it in items[:4]] + [(0.001 * (k + 1), it) for k, it in enumerate(items[4:])]
    stats = srv.run(arrivals)
    torch.cuda.synchronize()
    assert stats["requests"] == len(items) and srv.max_running >= 2
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    for i, (w, s_) in enumerate(zip(ws, singles)):
        _check(w, srv.outputs[i], s_)
    for it in items:
        ctx.release_scene(it["scene"])


def test_memory_admission_serialises_under_a_small_budget(ctx):
    from paper_2604_15017_gb300 import serve

    ws, items, singles = _workloads(ctx, 4, seed=22)
    probe = serve.Server(ctx, n_lanes=4)
    need = [probe.bytes_needed(it) for it in items]
    assert all(n > 0 for n in need)
    srv = serve.Server(ctx, n_lanes=4, mem_budget_bytes=min(need) + 1, keep_outputs=True)
    stats = srv.run([(0.0, it) for it in items])
    torch.cuda.synchronize()
    assert stats["requests"] == len(items) and srv.max_running == 1
    for i, (w, s_) in enumerate(zip(ws, singles)):
        _check(w, srv.outputs[i], s_)
    for it in items:
        ctx.release_scene(it["scene"])
