"""Continuous-batching request server on one GPU.

Requests (forward B-mode, or forward + loss + adjoint against a target image) arrive over time
for scenes that stay resident on the device (BVHs uploaded once).  The server keeps a queue,
admits a request when a lane (a slot with its own stream and workspaces inside the library) is
free and its memory estimate fits under the budget beside the requests already running, and
issues it on that lane's stream, so requests that arrive while others run overlap on the
device.  Each request writes into output buffers owned by its lane.  Completion is observed
through a CUDA event per request; latency = completion - arrival (host clock).
"""
from __future__ import annotations

import collections
import ctypes as C
import time

import numpy as np
import torch

from . import usrt


class _LaneBuffers:
    """Output buffers of one lane, grown to the largest request it has served."""

    def __init__(self, device):
        self.device = device
        self.rf = torch.empty(0, device=device)
        self.bmode = torch.empty(0, device=device)
        self.loss = torch.zeros(1, device=device)
        self.grad = torch.zeros(128, device=device)

    def views(self, rf_shape, img_shape, n_theta):
        n_rf = int(np.prod(rf_shape))
        n_b = int(np.prod(img_shape))
        if self.rf.numel() < n_rf:
            self.rf = torch.empty(n_rf, device=self.device)
        if self.bmode.numel() < n_b:
            self.bmode = torch.empty(n_b, device=self.device)
        if self.grad.numel() < n_theta:
            self.grad = torch.zeros(n_theta, device=self.device)
        return (self.rf[:n_rf].view(rf_shape), self.bmode[:n_b].view(img_shape), self.loss,
                self.grad[:n_theta])


class Server:
    """requests: dicts with scene, theta, acq, img, seed, and bref (device tensor) for
    forward + adjoint requests."""

    def __init__(self, ctx, n_lanes=4, mem_budget_bytes=120 << 30, keep_outputs=False):
        self.ctx = ctx
        self.n_lanes = n_lanes
        self.budget = mem_budget_bytes
        self.keep_outputs = keep_outputs
        self.streams = [torch.cuda.Stream() for _ in range(n_lanes)]
        self.buffers = [_LaneBuffers(ctx.device) for _ in range(n_lanes)]
        self.busy = [None] * n_lanes
        self.reserved = 0
        self.queue = collections.deque()
        self.records = {}
        self.outputs = {}
        self.max_running = 0

    def _request_struct(self, r, lane):
        th = usrt._f32(r["theta"])
        ad, ang = usrt.acq_desc(r["acq"])
        idesc = usrt.img_desc(r["img"])
        rf, b, loss, grad = self.buffers[lane].views(self.ctx.rf_shape(r["acq"]),
                                                     (r["img"]["n_lines"], r["img"]["n_depth"]), len(th))
        bref = r.get("bref")
        req = usrt.Request(int(r["scene"]), th.ctypes.data_as(C.POINTER(C.c_float)), C.pointer(ad), C.pointer(idesc),
                           int(r.get("seed", 0)) & (2**64 - 1), rf.data_ptr(), b.data_ptr(),
                           bref.data_ptr() if bref is not None else None,
                           loss.data_ptr() if bref is not None else None,
                           grad.data_ptr() if bref is not None else None)
        return req, (th, ad, ang, idesc), (rf, b, loss if bref is not None else None, grad if bref is not None else None)

    def bytes_needed(self, r):
        """The library's estimate of the device bytes request r occupies while it runs."""
        th = usrt._f32(r["theta"])
        ad, ang = usrt.acq_desc(r["acq"])
        idesc = usrt.img_desc(r["img"])
        adj = 1 if r.get("bref") is not None else None  # only whether it is NULL is read
        req = usrt.Request(int(r["scene"]), th.ctypes.data_as(C.POINTER(C.c_float)), C.pointer(ad), C.pointer(idesc),
                           0, None, None, adj, None, None)
        v = C.c_size_t()
        self.ctx._check(usrt.lib().us_request_bytes(self.ctx.h, C.byref(req), C.byref(v)))
        return v.value

    def warmup(self, requests):
        """Run every request once on every lane, so each lane's workspaces reach the size of the
        largest request before serving starts (workspace growth reallocates, which synchronises)."""
        big = max(requests, key=self.bytes_needed)
        for lane in range(self.n_lanes):
            req, keep, outs = self._request_struct(big, lane)
            self.ctx._check(usrt.lib().us_run_request(self.ctx.h, lane + 1, C.byref(req),
                                                      C.c_void_p(self.streams[lane].cuda_stream)))
        torch.cuda.synchronize()

    def submit(self, rid, r, t_arrival):
        self.queue.append((rid, r, t_arrival))
        self.records[rid] = {"arrival": t_arrival}

    def _poll(self):
        now = time.perf_counter()
        for i, b in enumerate(self.busy):
            if b is not None and b["event"].query():
                rec = self.records[b["rid"]]
                rec["done"] = now
                if self.keep_outputs:
                    self.outputs[b["rid"]] = b["out_copy"]
                self.reserved -= b["bytes"]
                self.busy[i] = None

    def _dispatch(self):
        while self.queue:
            free = [i for i, b in enumerate(self.busy) if b is None]
            if not free:
                return
            rid, r, t_arr = self.queue[0]
            need = r.get("_bytes")
            if need is None:
                need = r["_bytes"] = self.bytes_needed(r)
            if self.reserved + need > self.budget and any(b is not None for b in self.busy):
                return  # memory admission: wait until running requests release their share
            self.queue.popleft()
            lane = free[0]
            st = self.streams[lane]
            req, keep, outs = self._request_struct(r, lane)
            self.ctx._check(usrt.lib().us_run_request(self.ctx.h, lane + 1, C.byref(req), C.c_void_p(st.cuda_stream)))
            out_copy = None
            if self.keep_outputs:
                with torch.cuda.stream(st):
                    out_copy = tuple(None if o is None else o.clone() for o in outs)
            ev = torch.cuda.Event()
            ev.record(st)
            self.records[rid]["start"] = time.perf_counter()
            self.busy[lane] = dict(rid=rid, event=ev, bytes=need, keep=keep, out_copy=out_copy)
            self.reserved += need
            self.max_running = max(self.max_running, sum(b is not None for b in self.busy))

    def run(self, arrivals):
        """arrivals: list of (t_offset_seconds, request dict), sorted by time.  Returns stats."""
        t0 = time.perf_counter()
        i = 0
        n = len(arrivals)
        while i < n or self.queue or any(b is not None for b in self.busy):
            now = time.perf_counter() - t0
            while i < n and arrivals[i][0] <= now:
                self.submit(i, arrivals[i][1], t0 + arrivals[i][0])
                i += 1
            self._poll()
            self._dispatch()
            if not self.queue and all(b is None for b in self.busy) and i < n:
                time.sleep(max(0.0, min(0.001, arrivals[i][0] - (time.perf_counter() - t0))))
            else:
                time.sleep(0.0002)
        t1 = time.perf_counter()
        lat = np.array([r["done"] - r["arrival"] for r in self.records.values()])
        return dict(requests=n, seconds=t1 - t0, throughput=n / (t1 - t0), p50_ms=float(np.percentile(lat, 50) * 1e3),
                    p99_ms=float(np.percentile(lat, 99) * 1e3), mean_ms=float(lat.mean() * 1e3))


def run_sequential(ctx, arrivals, stream=None):
    """The plain path to compare against: one request at a time, in arrival order, each issued
    when it has arrived and the previous one has finished, on one stream."""
    srv = Server(ctx, n_lanes=1)
    st = stream or srv.streams[0]
    t0 = time.perf_counter()
    lat = []
    for t_arr, r in arrivals:
        while time.perf_counter() - t0 < t_arr:
            time.sleep(0.0002)
        req, keep, outs = srv._request_struct(r, 0)
        ctx._check(usrt.lib().us_run_request(ctx.h, 1, C.byref(req), C.c_void_p(st.cuda_stream)))
        st.synchronize()
        lat.append(time.perf_counter() - (t0 + t_arr))
    t1 = time.perf_counter()
    lat = np.array(lat)
    n = len(arrivals)
    return dict(requests=n, seconds=t1 - t0, throughput=n / (t1 - t0), p50_ms=float(np.percentile(lat, 50) * 1e3),
                p99_ms=float(np.percentile(lat, 99) * 1e3), mean_ms=float(lat.mean() * 1e3))


def poisson_arrivals(rate_hz, seconds, seed):
    """Arrival times (s) of a Poisson process of rate rate_hz over [0, seconds)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > seconds:
            return out
        out.append(t)
