"""Python binding of the usrt C ABI (``include/usrt.h``).

Argument marshalling only: every arithmetic step runs in the CUDA kernels of
``_build/libusrt.so``.  PyTorch supplies device memory and the current CUDA stream; the
library raises ``UsrtError`` when a call fails and ``RuntimeError`` when it cannot be loaded
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libusrt.so")

US_OK, US_ERR_ARG, US_ERR_OOM, US_ERR_CUDA, US_ERR_TIMEOUT, US_ERR_OVERFLOW, US_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
MODE_RECORD, MODE_RECOMPUTE = 0, 1

# the C ABI's entry points (each declared in include/usrt.h)
EXPORTS = ["us_create", "us_destroy", "us_last_error", "us_scene_upload", "us_scene_release", "us_memory",
           "us_philox_fill", "us_forward", "us_get_stats", "us_get_record", "us_get_arrivals", "us_splat", "us_das", "us_envlog",
           "us_bmode", "us_loss", "us_envlog_vjp", "us_das_adjoint", "us_bmode_vjp", "us_splat_adjoint",
           "us_transport_vjp", "us_adjoint", "us_envlog_noalloc", "us_profile", "us_profile_read",
           "us_launch_count", "us_set_option", "us_forward_batch", "us_autotune_batch",
           "us_run_request", "us_request_bytes", "us_param_map", "us_adam_step", "us_das_acq_vjp",
           "us_transport_vjp_acq", "us_adjoint_acq", "us_transport_vjp_shape", "us_adjoint_shape",
           "us_shape_param_grad", "us_get_status", "us_set_envlog_fused",
           "us_set_das_adj_tiled"]
OPT_DAS_TMA, OPT_LANES, OPT_NEE_STREAM, OPT_FAULT_BARRIER = 0, 1, 2, 3
STAGES = ["generate", "traverse", "interact", "nee", "splat_sort", "splat_rows", "das", "envlog", "loss",
          "envlog_vjp", "das_adj", "nee_adj", "path_adj", "other", "das_acq", "ray_sort", "job_sort"]


class UsrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("usrt error %d: %s" % (code, msg))
        self.code = code


class SceneDesc(C.Structure):
    _fields_ = [("n_tris", C.c_int32), ("tris", C.POINTER(C.c_float)), ("media", C.POINTER(C.c_int32)),
                ("n_media", C.c_int32), ("n_scat", C.c_int32), ("scat_pos", C.POINTER(C.c_float)),
                ("scat_amp", C.POINTER(C.c_float)), ("r_s", C.c_float), ("rough", C.c_int32)]


class AcqDesc(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("pitch", C.c_float), ("h_el", C.c_float), ("n_tx", C.c_int32),
                ("angles", C.POINTER(C.c_float)), ("fs", C.c_float), ("n_samples", C.c_int32),
                ("k_max", C.c_int32), ("n_rays", C.c_int32), ("bw", C.c_float), ("alpha_m", C.c_float),
                ("alpha_c", C.c_float), ("c_bf", C.c_float), ("split_mode", C.c_int32), ("split_q", C.c_float),
                ("stream_id", C.c_uint32), ("tx_elem", C.c_int32), ("n_tx_elem", C.c_int32),
                ("rough_nee", C.c_int32)]


class ImgDesc(C.Structure):
    _fields_ = [("n_lines", C.c_int32), ("n_depth", C.c_int32), ("x0", C.c_float), ("x1", C.c_float),
                ("z0", C.c_float), ("z1", C.c_float), ("dr_db", C.c_float), ("lambda1", C.c_float),
                ("lambda2", C.c_float), ("f_number", C.c_float)]


class Request(C.Structure):
    _fields_ = [("scene", C.c_uint64), ("theta", C.POINTER(C.c_float)), ("acq", C.POINTER(AcqDesc)),
                ("img", C.POINTER(ImgDesc)), ("seed", C.c_uint64), ("rf_dev", C.c_void_p),
                ("bmode_dev", C.c_void_p), ("bref_dev", C.c_void_p), ("loss_dev", C.c_void_p),
                ("dL_dtheta_dev", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("n_paths", C.c_int64), ("segments", C.c_int64), ("nee_queries", C.c_int64),
                ("arrivals", C.c_int64), ("dropped", C.c_int64), ("status", C.c_int32), ("pad", C.c_int32),
                ("live", C.c_int64 * 17)]


_lib = None
_lock = threading.Lock()
VP = C.c_void_p


def lib():
    """Load the in-tree library (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _b
                _b.build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("usrt CUDA library missing: " + LIB_PATH)
            l = C.CDLL(LIB_PATH)
            l.us_create.argtypes = [C.POINTER(VP), C.c_int, C.c_size_t]
            l.us_destroy.argtypes = [VP]
            l.us_destroy.restype = None
            l.us_last_error.argtypes = [VP]
            l.us_last_error.restype = C.c_char_p
            l.us_scene_upload.argtypes = [VP, C.POINTER(SceneDesc), C.POINTER(C.c_uint64)]
            l.us_scene_release.argtypes = [VP, C.c_uint64]
            l.us_memory.argtypes = [VP, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
            l.us_philox_fill.argtypes = [VP] + [C.c_uint32] * 6 + [C.c_int64, VP, VP]
            l.us_forward.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc), C.POINTER(ImgDesc),
                                     C.c_uint64, C.c_int, VP, VP, VP]
            l.us_get_stats.argtypes = [VP, C.POINTER(Stats)]
            l.us_get_record.argtypes = [VP, C.c_int64, C.c_int64, VP, VP]
            l.us_get_arrivals.argtypes = [VP, C.c_int64, C.c_int64, VP, VP]
            l.us_get_status.argtypes = [VP, C.c_int, C.POINTER(C.c_int)]
            l.us_set_envlog_fused.argtypes = [C.c_int]
            l.us_set_envlog_fused.restype = None
            l.us_set_das_adj_tiled.argtypes = [C.c_int]
            l.us_set_das_adj_tiled.restype = None
            l.us_splat.argtypes = [VP, C.POINTER(AcqDesc), C.c_float, C.c_int64, VP, VP, VP, VP, VP, VP]
            l.us_das.argtypes = [VP, C.POINTER(AcqDesc), C.POINTER(ImgDesc), VP, VP, VP]
            l.us_envlog.argtypes = [VP, C.POINTER(ImgDesc), VP, VP, VP]
            l.us_bmode.argtypes = [VP, C.POINTER(AcqDesc), C.POINTER(ImgDesc), VP, VP, VP]
            l.us_loss.argtypes = [VP, C.POINTER(ImgDesc), VP, VP, VP, VP, VP]
            l.us_envlog_vjp.argtypes = [VP, C.POINTER(ImgDesc), VP, VP, VP, VP]
            l.us_das_adjoint.argtypes = [VP, C.POINTER(AcqDesc), C.POINTER(ImgDesc), VP, VP, VP]
            l.us_bmode_vjp.argtypes = [VP, C.POINTER(AcqDesc), C.POINTER(ImgDesc), VP, VP, VP, VP]
            l.us_splat_adjoint.argtypes = [VP, C.POINTER(AcqDesc), C.c_float, C.c_int64, VP, VP, VP, VP, VP, VP, VP,
                                           VP, VP]
            l.us_transport_vjp.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc), C.c_uint64,
                                           C.c_int, VP, VP, VP]
            l.us_adjoint.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc), C.POINTER(ImgDesc),
                                     C.c_uint64, C.c_int, VP, VP, VP, VP, VP]
            l.us_das_acq_vjp.argtypes = [VP, C.POINTER(AcqDesc), C.POINTER(ImgDesc), VP, VP, VP, VP]
            l.us_transport_vjp_acq.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc),
                                               C.c_uint64, C.c_int, VP, VP, VP, VP]
            l.us_adjoint_acq.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc),
                                         C.POINTER(ImgDesc), C.c_uint64, C.c_int, VP, VP, VP, VP, VP, VP]
            l.us_transport_vjp_shape.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc),
                                                 C.c_uint64, C.c_int, VP, VP, VP, VP]
            l.us_adjoint_shape.argtypes = [VP, C.c_uint64, C.POINTER(C.c_float), C.POINTER(AcqDesc),
                                           C.POINTER(ImgDesc), C.c_uint64, C.c_int, VP, VP, VP, VP, VP, VP]
            l.us_shape_param_grad.argtypes = [VP, C.c_int64, VP, C.c_int, VP, VP, VP]
            l.us_profile.argtypes = [VP, C.c_int]
            l.us_profile_read.argtypes = [VP, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]
            l.us_launch_count.argtypes = [VP, C.POINTER(C.c_int64)]
            l.us_set_option.argtypes = [VP, C.c_int, C.c_int]
            l.us_forward_batch.argtypes = [VP, C.c_int, C.POINTER(Request), VP]
            l.us_run_request.argtypes = [VP, C.c_int, C.POINTER(Request), VP]
            l.us_request_bytes.argtypes = [VP, C.POINTER(Request), C.POINTER(C.c_size_t)]
            l.us_autotune_batch.argtypes = [VP, C.c_int, C.POINTER(Request), VP, C.POINTER(C.c_int),
                                            C.POINTER(C.c_int)]
            l.us_param_map.argtypes = [VP, C.c_int, VP, VP, VP, VP, VP]
            l.us_adam_step.argtypes = [VP, C.c_int, VP, VP, VP, VP, VP, C.c_float, C.c_float, C.c_float, C.c_float,
                                       C.c_int, VP, VP, VP]
            _lib = l
    return _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def acq_desc(acq):
    """Acquisition dict (phantoms.acquisition) -> (AcqDesc, keep-alive angle array)."""
    ang = _f32(acq["angles"])
    d = AcqDesc(int(acq["n_elem"]), float(acq["pitch"]), float(acq["h_el"]), len(ang),
                ang.ctypes.data_as(C.POINTER(C.c_float)), float(acq["fs"]), int(acq["n_samples"]),
                int(acq["k_max"]), int(acq["n_rays"]), float(acq["bw"]), float(acq["alpha_m"]),
                float(acq["alpha_c"]), float(acq["c_bf"]), int(acq.get("split_mode", 0)),
                float(acq.get("split_q", 0.5)), int(acq.get("stream_id", 0)) & 0xFFFFFFFF,
                int(acq.get("tx_elem", -1)), int(acq.get("n_tx_elem", 0)), int(acq.get("rough_nee", 1)))
    return d, ang


def img_desc(img):
    return ImgDesc(int(img["n_lines"]), int(img["n_depth"]), float(img["x0"]), float(img["x1"]), float(img["z0"]),
                   float(img["z1"]), float(img.get("dr_db", 60.0)), float(img.get("lambda1", 0.0)),
                   float(img.get("lambda2", 1.0)), float(img.get("f_number", 0.0)))


def set_envlog_fused(enable):
    """Process-wide: the cooperative fused envelope kernel (True, default) or always the
    two-kernel path (False)."""
    lib().us_set_envlog_fused(int(bool(enable)))


def set_das_adj_tiled(enable):
    """Process-wide: the tiled transposed-DAS kernel (True, default; n_tx <= 32) or always the
    untiled one (False).  Same bits either way."""
    lib().us_set_das_adj_tiled(int(bool(enable)))


class Context:
    """One library context on one CUDA device (scenes, records and workspaces stay resident)."""

    def __init__(self, device=0, mem_budget_bytes=0):
        self.device = torch.device("cuda", device)
        h = VP()
        rc = lib().us_create(C.byref(h), int(device), int(mem_budget_bytes))
        if rc != US_OK:
            raise UsrtError(rc, "us_create failed")
        self.h = h
        self.scene_media = {}

    def _check(self, rc):
        if rc != US_OK:
            raise UsrtError(rc, lib().us_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().us_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory(self):
        u, b = C.c_size_t(), C.c_size_t()
        self._check(lib().us_memory(self.h, C.byref(u), C.byref(b)))
        return u.value, b.value

    # ---- tracing --------------------------------------------------------------------------
    def profile(self, enable=True):
        self._check(lib().us_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """{stage: (device ms, kernel launches)} since profile(True) (synchronises)."""
        n = len(STAGES)
        ms = (C.c_double * n)()
        ln = (C.c_int64 * n)()
        self._check(lib().us_profile_read(self.h, ms, ln, n))
        return {STAGES[i]: (ms[i], ln[i]) for i in range(n)}

    def set_option(self, option, value):
        self._check(lib().us_set_option(self.h, int(option), int(value)))

    def device_status(self, clear=True):
        """Status of the kernels outside the transport since the last clear (0, or a negative
        us_status such as US_ERR_TIMEOUT); synchronises the device."""
        st = C.c_int(0)
        self._check(lib().us_get_status(self.h, int(bool(clear)), C.byref(st)))
        return st.value

    def launch_count(self):
        v = C.c_int64()
        self._check(lib().us_launch_count(self.h, C.byref(v)))
        return v.value

    # ---- scenes ---------------------------------------------------------------------------
    def upload_scene(self, tris, media, n_media, scat_pos, scat_amp, r_s, rough=False):
        tris = _f32(np.asarray(tris).reshape(-1, 9))
        media = np.ascontiguousarray(np.asarray(media, dtype=np.int32).reshape(-1, 2))
        sp = _f32(np.asarray(scat_pos).reshape(-1, 3))
        sa = _f32(np.asarray(scat_amp).reshape(-1))
        d = SceneDesc(len(tris), tris.ctypes.data_as(C.POINTER(C.c_float)), media.ctypes.data_as(C.POINTER(C.c_int32)),
                      int(n_media), len(sa), sp.ctypes.data_as(C.POINTER(C.c_float)),
                      sa.ctypes.data_as(C.POINTER(C.c_float)), float(r_s), int(bool(rough)))
        sid = C.c_uint64()
        self._check(lib().us_scene_upload(self.h, C.byref(d), C.byref(sid)))
        self.scene_media[sid.value] = int(n_media)
        return sid.value

    def upload_workload(self, w):
        return self.upload_scene(w["tris"], w["media"], w["M"], w["scat_pos"], w["scat_amp"], w["r_s"],
                                 rough=w.get("rough", False))

    def release_scene(self, sid):
        self._check(lib().us_scene_release(self.h, int(sid)))

    # ---- S1 -----------------------------------------------------------------------------------
    def philox_fill(self, c0, c1, c2, c3, k0, k1, n, out=None, stream=None):
        out = out if out is not None else torch.empty(4 * n, dtype=torch.int32, device=self.device)
        self._check(lib().us_philox_fill(self.h, c0 & 0xFFFFFFFF, c1, c2, c3, k0, k1, n, _ptr(out), _stream(stream)))
        return out

    # ---- forward ----------------------------------------------------------------------------
    def rf_shape(self, acq):
        return (len(acq["angles"]), int(acq["n_elem"]), int(acq["n_samples"]))

    def forward(self, scene, theta, acq, img=None, seed=0, keep_record=False, rf=None, bmode=None, stream=None):
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        idesc = img_desc(img) if img is not None else None
        rf = rf if rf is not None else torch.empty(self.rf_shape(acq), dtype=torch.float32, device=self.device)
        if img is not None and bmode is None:
            bmode = torch.empty((img["n_lines"], img["n_depth"]), dtype=torch.float32, device=self.device)
        self._check(lib().us_forward(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ad),
                                     C.byref(idesc) if idesc is not None else None, int(seed) & (2**64 - 1),
                                     int(bool(keep_record)), _ptr(rf), _ptr(bmode), _stream(stream)))
        return rf, bmode

    def stats(self):
        s = Stats()
        self._check(lib().us_get_stats(self.h, C.byref(s)))
        return dict(n_paths=s.n_paths, segments=s.segments, nee_queries=s.nee_queries, arrivals=s.arrivals,
                    dropped=s.dropped, status=s.status, live=[int(v) for v in s.live])

    def record(self, path_lo, n, k_max, stream=None):
        out = torch.empty((n, k_max + 1), dtype=torch.int32, device=self.device)
        self._check(lib().us_get_record(self.h, int(path_lo), int(n), _ptr(out), _stream(stream)))
        return out

    def arrivals(self, acq, stream=None):
        """The last forward pass's arrival list as (tx, e, tau [s], a, path) tensors on the device,
        in append order."""
        n = int(self.stats()["arrivals"])
        raw = torch.empty((max(n, 1), 4), dtype=torch.int32, device=self.device)
        self._check(lib().us_get_arrivals(self.h, 0, n, _ptr(raw), _stream(stream)))
        raw = raw[:n]
        ne = int(acq["n_elem"])
        row = raw[:, 0].to(torch.int64)
        tq = raw[:, 1].to(torch.int64) & 0xFFFFFFFF
        tau = (tq.double() * 2.0 ** -18 - 64.0) / float(acq["fs"])
        return dict(tx=(row // ne).to(torch.int32), e=(row % ne).to(torch.int32), tau=tau,
                    a=raw[:, 2].contiguous().view(torch.float32), path=raw[:, 3].to(torch.int64) & 0xFFFFFFFF)

    def splat(self, acq, f0, tx, e, tau, a, rf=None, stream=None):
        ad, ang = acq_desc(acq)
        rf = rf if rf is not None else torch.empty(self.rf_shape(acq), dtype=torch.float32, device=self.device)
        self._check(lib().us_splat(self.h, C.byref(ad), float(f0), int(tau.numel()), _ptr(tx), _ptr(e), _ptr(tau),
                                   _ptr(a), _ptr(rf), _stream(stream)))
        return rf

    def das(self, acq, img, rf, out=None, stream=None):
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        out = out if out is not None else torch.empty((img["n_lines"], img["n_depth"]), dtype=torch.float32,
                                                      device=self.device)
        self._check(lib().us_das(self.h, C.byref(ad), C.byref(idesc), _ptr(rf), _ptr(out), _stream(stream)))
        return out

    def envlog(self, img, irf, out=None, stream=None):
        idesc = img_desc(img)
        out = out if out is not None else torch.empty_like(irf)
        self._check(lib().us_envlog(self.h, C.byref(idesc), _ptr(irf), _ptr(out), _stream(stream)))
        return out

    def bmode(self, acq, img, rf, out=None, stream=None):
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        out = out if out is not None else torch.empty((img["n_lines"], img["n_depth"]), dtype=torch.float32,
                                                      device=self.device)
        self._check(lib().us_bmode(self.h, C.byref(ad), C.byref(idesc), _ptr(rf), _ptr(out), _stream(stream)))
        return out

    # ---- loss and adjoint -------------------------------------------------------------------
    def loss(self, img, b, bref, grad=True, stream=None, out=None):
        idesc = img_desc(img)
        loss = out if out is not None else torch.empty(1, dtype=torch.float32, device=self.device)
        gb = torch.empty_like(b) if grad else None
        self._check(lib().us_loss(self.h, C.byref(idesc), _ptr(b), _ptr(bref), _ptr(loss), _ptr(gb), _stream(stream)))
        return loss, gb

    def envlog_vjp(self, img, irf, gb, stream=None):
        idesc = img_desc(img)
        gi = torch.empty_like(irf)
        self._check(lib().us_envlog_vjp(self.h, C.byref(idesc), _ptr(irf), _ptr(gb), _ptr(gi), _stream(stream)))
        return gi

    def das_adjoint(self, acq, img, gi, stream=None):
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        grf = torch.empty(self.rf_shape(acq), dtype=torch.float32, device=self.device)
        self._check(lib().us_das_adjoint(self.h, C.byref(ad), C.byref(idesc), _ptr(gi), _ptr(grf), _stream(stream)))
        return grf

    def bmode_vjp(self, acq, img, rf, gb, stream=None):
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        grf = torch.empty(self.rf_shape(acq), dtype=torch.float32, device=self.device)
        self._check(lib().us_bmode_vjp(self.h, C.byref(ad), C.byref(idesc), _ptr(rf), _ptr(gb), _ptr(grf),
                                       _stream(stream)))
        return grf

    def splat_adjoint(self, acq, f0, tx, e, tau, a, grf, stream=None):
        ad, ang = acq_desc(acq)
        n = int(tau.numel())
        ga, gt, gf = (torch.empty(n, dtype=torch.float32, device=self.device) for _ in range(3))
        self._check(lib().us_splat_adjoint(self.h, C.byref(ad), float(f0), n, _ptr(tx), _ptr(e), _ptr(tau), _ptr(a),
                                           _ptr(grf), _ptr(ga), _ptr(gt), _ptr(gf), _stream(stream)))
        return ga, gt, gf

    def transport_vjp(self, scene, theta, acq, seed, grf, mode=MODE_RECORD, out=None, stream=None):
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        out = out if out is not None else torch.empty(len(th), dtype=torch.float32, device=self.device)
        self._check(lib().us_transport_vjp(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ad),
                                           int(seed) & (2**64 - 1), int(mode), _ptr(grf), _ptr(out), _stream(stream)))
        return out

    def adjoint(self, scene, theta, acq, img, seed, rf, gb, mode=MODE_RECORD, want_grf=False, stream=None):
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        gth = torch.empty(len(th), dtype=torch.float32, device=self.device)
        grf = torch.empty(self.rf_shape(acq), dtype=torch.float32, device=self.device) if want_grf else None
        self._check(lib().us_adjoint(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ad),
                                     C.byref(idesc), int(seed) & (2**64 - 1), int(mode), _ptr(rf), _ptr(gb),
                                     _ptr(gth), _ptr(grf), _stream(stream)))
        return gth, grf

    # ---- acquisition-parameter gradients: [dL/dc_bf, dL/dpitch, dL/dth_0, ..., dL/dth_{ntx-1}] ----
    def das_acq_vjp(self, acq, img, rf, gi, stream=None):
        """DAS part: sum_p gi(p) dI_rf(p)/d(c_bf, pitch, steering angles), the RF held fixed."""
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        out = torch.empty(2 + len(acq["angles"]), dtype=torch.float32, device=self.device)
        self._check(lib().us_das_acq_vjp(self.h, C.byref(ad), C.byref(idesc), _ptr(rf), _ptr(gi), _ptr(out),
                                         _stream(stream)))
        return out

    def transport_vjp_acq(self, scene, theta, acq, seed, grf, mode=MODE_RECORD, stream=None):
        """Transport part: (dL/dtheta, dL/d(c_bf, pitch, steering angles)) from dL/dRF."""
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        gth = torch.empty(len(th), dtype=torch.float32, device=self.device)
        gacq = torch.empty(2 + len(acq["angles"]), dtype=torch.float32, device=self.device)
        self._check(lib().us_transport_vjp_acq(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)),
                                               C.byref(ad), int(seed) & (2**64 - 1), int(mode), _ptr(grf), _ptr(gth),
                                               _ptr(gacq), _stream(stream)))
        return gth, gacq

    def adjoint_acq(self, scene, theta, acq, img, seed, rf, gb, mode=MODE_RECORD, stream=None):
        """Full adjoint with the acquisition gradient: (dL/dtheta, dL/d(c_bf, pitch, steering angles))."""
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        gth = torch.empty(len(th), dtype=torch.float32, device=self.device)
        gacq = torch.empty(2 + len(acq["angles"]), dtype=torch.float32, device=self.device)
        self._check(lib().us_adjoint_acq(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ad),
                                         C.byref(idesc), int(seed) & (2**64 - 1), int(mode), _ptr(rf), _ptr(gb),
                                         _ptr(gth), _ptr(gacq), None, _stream(stream)))
        return gth, gacq

    # ---- shape gradients: dL/d(triangle vertices) [n_tris, 9] ----
    def transport_vjp_shape(self, scene, theta, acq, seed, grf, n_tris, mode=MODE_RECORD, stream=None):
        """Transport part: (dL/dtheta, dL/dtris) from dL/dRF."""
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        gth = torch.empty(len(th), dtype=torch.float32, device=self.device)
        gtris = torch.empty((int(n_tris), 9), dtype=torch.float32, device=self.device)
        self._check(lib().us_transport_vjp_shape(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)),
                                                 C.byref(ad), int(seed) & (2**64 - 1), int(mode), _ptr(grf),
                                                 _ptr(gth), _ptr(gtris), _stream(stream)))
        return gth, gtris

    def adjoint_shape(self, scene, theta, acq, img, seed, rf, gb, n_tris, mode=MODE_RECORD, stream=None):
        """Full adjoint: (dL/dtheta, dL/dtris)."""
        th = _f32(theta)
        ad, ang = acq_desc(acq)
        idesc = img_desc(img)
        gth = torch.empty(len(th), dtype=torch.float32, device=self.device)
        gtris = torch.empty((int(n_tris), 9), dtype=torch.float32, device=self.device)
        self._check(lib().us_adjoint_shape(self.h, int(scene), th.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ad),
                                           C.byref(idesc), int(seed) & (2**64 - 1), int(mode), _ptr(rf), _ptr(gb),
                                           _ptr(gth), _ptr(gtris), None, _stream(stream)))
        return gth, gtris

    def shape_param_grad(self, gtris, dtris_dq, stream=None):
        """dL/dq_j = sum dL/dtris * dtris/dq_j for the tangents dtris_dq [n_param, n_tris, 9]."""
        n_param = int(dtris_dq.shape[0])
        out = torch.empty(n_param, dtype=torch.float32, device=self.device)
        self._check(lib().us_shape_param_grad(self.h, int(gtris.shape[0]), _ptr(gtris), n_param, _ptr(dtris_dq),
                                              _ptr(out), _stream(stream)))
        return out

    # ---- inverse problem: parameterisation and optimiser step (Sec. 3.4, 3.7) ----
    def param_map(self, theta_u, lo, hi, out=None, stream=None):
        """Physical parameters lo + clip(theta_u, 0, 1) (hi - lo) (device tensors)."""
        out = torch.empty_like(theta_u) if out is None else out
        self._check(lib().us_param_map(self.h, theta_u.numel(), _ptr(theta_u), _ptr(lo), _ptr(hi), _ptr(out),
                                       _stream(stream)))
        return out

    def adam_step(self, theta_u, grad_phys, lo, hi, lr, m, v, step, beta1=0.9, beta2=0.999, eps=1e-8, clip_norm=0.0,
                  stream=None):
        """One Adam step on theta_u (in place) from dL/dtheta of the physical parameters."""
        self._check(lib().us_adam_step(self.h, theta_u.numel(), _ptr(theta_u), _ptr(grad_phys), _ptr(lo), _ptr(hi),
                                       _ptr(lr), float(beta1), float(beta2), float(eps), float(clip_norm), int(step),
                                       _ptr(m), _ptr(v), _stream(stream)))
        return theta_u


class Batch:
    """A prepared batch of requests (device outputs allocated once, so the batch can be run
    repeatedly and captured in a CUDA graph).  items: dicts with scene, theta, acq, img, seed and
    optionally bref (a device tensor: forward + loss + adjoint)."""

    def __init__(self, ctx, items):
        self.ctx = ctx
        self.items = items
        self._keep = []
        n = len(items)
        self.reqs = (Request * n)()
        self.outputs = []
        for i, it in enumerate(items):
            th = _f32(it["theta"])
            ad, ang = acq_desc(it["acq"])
            idesc = img_desc(it["img"])
            rf = torch.empty(ctx.rf_shape(it["acq"]), dtype=torch.float32, device=ctx.device)
            b = torch.empty((it["img"]["n_lines"], it["img"]["n_depth"]), dtype=torch.float32, device=ctx.device)
            bref = it.get("bref")
            loss = torch.zeros(1, dtype=torch.float32, device=ctx.device) if bref is not None else None
            g = torch.zeros(len(th), dtype=torch.float32, device=ctx.device) if bref is not None else None
            self._keep += [th, ad, ang, idesc]
            self.reqs[i] = Request(int(it["scene"]), th.ctypes.data_as(C.POINTER(C.c_float)), C.pointer(ad),
                                   C.pointer(idesc), int(it.get("seed", 0)) & (2**64 - 1), rf.data_ptr(),
                                   b.data_ptr(), bref.data_ptr() if bref is not None else None,
                                   loss.data_ptr() if loss is not None else None,
                                   g.data_ptr() if g is not None else None)
            self.outputs.append(dict(rf=rf, bmode=b, loss=loss, grad=g))

    def run(self, stream=None):
        self.ctx._check(lib().us_forward_batch(self.ctx.h, len(self.items), self.reqs, _stream(stream)))
        return self.outputs

    def run_one(self, i, lane, stream=None):
        """Request i alone on `lane` (1..16) and `stream` (serving)."""
        self.ctx._check(lib().us_run_request(self.ctx.h, int(lane), C.byref(self.reqs[i]), _stream(stream)))
        return self.outputs[i]

    def bytes_needed(self, i):
        v = C.c_size_t()
        self.ctx._check(lib().us_request_bytes(self.ctx.h, C.byref(self.reqs[i]), C.byref(v)))
        return v.value

    def autotune(self, stream=None):
        bl, bt = C.c_int(), C.c_int()
        self.ctx._check(lib().us_autotune_batch(self.ctx.h, len(self.items), self.reqs, _stream(stream), C.byref(bl),
                                                C.byref(bt)))
        return bl.value, bt.value


class BModeSimulation(torch.autograd.Function):
    """theta -> B-mode image, differentiable with the fixed-sample adjoint (Sec. 3.2-3.3).

    forward = us_forward (transport, splat, DAS, envelope, log) keeping the path record;
    backward = us_adjoint (envelope/log VJP, transposed DAS, splat adjoint, path adjoint).
    theta is a CPU float tensor; the returned gradient is moved back to the CPU.
    """

    @staticmethod
    def forward(fctx, theta, ctx, scene, acq, img, seed):
        th = theta.detach().cpu().numpy().astype(np.float32)
        rf, b = ctx.forward(scene, th, acq, img, seed, keep_record=True)
        fctx.save_for_backward(theta)
        fctx.usrt = (ctx, scene, acq, img, seed, th, rf)
        return b

    @staticmethod
    def backward(fctx, gb):
        ctx, scene, acq, img, seed, th, rf = fctx.usrt
        gth, _ = ctx.adjoint(scene, th, acq, img, seed, rf, gb.contiguous().float(), mode=MODE_RECORD)
        return gth.to(fctx.saved_tensors[0].device, fctx.saved_tensors[0].dtype), None, None, None, None, None
