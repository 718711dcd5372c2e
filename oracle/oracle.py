"""Python face of the FP64 CPU oracle (``usrt_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, the package smoke check and the benchmark's
CPU-baseline leg, never by the product path.  It shares no code with the CUDA library; it
takes the plain arrays and dictionaries that the seeded input generators return.

What it computes (all in double precision) follows arXiv 2604.15017:
  * Philox4x32-10 sample streams (Salmon et al., SC'11)
  * full-path transport with receiver-guided secondary rays (Sec. 2.3.1-2.3.3)
  * pulse splat (Eq. axial_sig), DAS (Eq. das), Hilbert envelope, log compression and the
    dynamic-range clip (Sec. 2.3.4), the l1+l2 loss (Eq. weighted_l1_l2_loss)
  * the image-chain vector-Jacobian product (Eq. das_adjoint plus the envelope/log derivative)
  * the fixed-sample gradient (Sec. 3.2, Eq. chain_rule) by forward-mode dual numbers through a
    replay of the frozen decisions, and the replay itself for finite differences.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "usrt_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

# flat descriptor layouts (mirrors the enums of usrt_oracle.cpp)
ACQ_KEYS = ["n_elem", "pitch", "h_el", "n_tx", "fs", "n_samples", "k_max", "n_rays", "bw", "alpha_m",
            "alpha_c", "c_bf", "split_mode", "split_q", "stream_id", "tx_elem", "n_tx_elem", "rough_nee"]
IMG_KEYS = ["n_lines", "n_depth", "x0", "x1", "z0", "z1", "dr_db", "lambda1", "lambda2", "f_number"]
IMG_DEFAULTS = {"dr_db": 60.0, "lambda1": 0.0, "lambda2": 1.0, "f_number": 0.0}

CLS_NONE, CLS_XDCR, CLS_TRI, CLS_SCAT = 0, 1, 2, 3
CH_NONE, CH_REFLECT, CH_TRANSMIT, CH_TIR = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None

D = C.POINTER(C.c_double)
I = C.POINTER(C.c_int)
L = C.POINTER(C.c_longlong)
U = C.POINTER(C.c_uint32)


def build(force=False):
    """Compile the oracle with g++ (no GPU, no CUDA)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, SRC, "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            l = C.CDLL(LIB_PATH)
            l.ora_philox.argtypes = [C.c_uint32] * 6 + [U]
            l.ora_philox_fill.argtypes = [C.c_uint32] * 6 + [C.c_longlong, U]
            l.ora_scene_create.restype = C.c_void_p
            l.ora_scene_create.argtypes = [C.c_int, D, I, C.c_int, D, D, C.c_double, C.c_int, C.c_int]
            l.ora_ggx_normal.argtypes = [D, C.c_double, C.c_double, C.c_double, D]
            l.ora_scene_free.argtypes = [C.c_void_p]
            l.ora_closest.argtypes = [C.c_void_p, D, D, C.c_int, C.c_int, D]
            l.ora_interface.argtypes = [D, D, C.c_double, C.c_double, C.c_double, C.c_double, D]
            l.ora_emit.argtypes = [D, D, C.c_uint64, C.c_int, C.c_longlong, C.c_longlong, D]
            l.ora_trace.restype = C.c_void_p
            l.ora_trace.argtypes = [C.c_void_p, D, C.c_int, D, D, C.c_uint64, C.c_int, C.c_longlong, C.c_longlong]
            l.ora_run_free.argtypes = [C.c_void_p]
            l.ora_run_n_arrivals.restype = C.c_longlong
            l.ora_run_n_arrivals.argtypes = [C.c_void_p]
            l.ora_run_counters.argtypes = [C.c_void_p, L]
            l.ora_run_arrivals.argtypes = [C.c_void_p, I, I, D, D, L, I, I]
            l.ora_run_records.argtypes = [C.c_void_p, I, I, I, I]
            l.ora_splat_run.argtypes = [C.c_void_p, D, D]
            l.ora_splat.argtypes = [D, D, C.c_double, C.c_longlong, I, I, D, D, D]
            l.ora_splat_adjoint.argtypes = [D, D, C.c_double, C.c_longlong, I, I, D, D, D, D, D, D]
            l.ora_das.argtypes = [D, D, D, D, D]
            l.ora_das_adjoint.argtypes = [D, D, D, D, D]
            l.ora_das_acq_vjp.argtypes = [D, D, D, D, D, D]
            l.ora_hilbert.argtypes = [D, C.c_int, D]
            l.ora_envelope.argtypes = [D, D, D]
            l.ora_log_compress.restype = C.c_longlong
            l.ora_log_compress.argtypes = [D, D, D]
            l.ora_loss.restype = C.c_double
            l.ora_loss.argtypes = [D, D, D, D]
            l.ora_envlog_vjp.argtypes = [D, D, D, D]
            l.ora_replay_rf.argtypes = [C.c_void_p, C.c_void_p, D, C.c_uint64, C.c_int, D]
            l.ora_gradient.argtypes = [C.c_void_p, C.c_void_p, D, C.c_uint64, C.c_int, D, D]
            l.ora_gradient_cond.argtypes = [C.c_void_p, C.c_void_p, D, C.c_uint64, C.c_int, D, D, D]
            l.ora_gradient_acq.argtypes = [C.c_void_p, C.c_void_p, D, C.c_uint64, C.c_int, D, D]
            l.ora_gradient_shape.argtypes = [C.c_void_p, C.c_void_p, D, C.c_uint64, C.c_int, D, C.c_int, D, D]
            l.ora_inject_sums.argtypes = [C.c_void_p, D, C.c_int, D, D, C.c_uint64, C.c_longlong, D, D, C.c_int, D, D]
            l.ora_trace_injected.restype = C.c_int
            l.ora_trace_injected.argtypes = [C.c_void_p, D, C.c_int, D, D, C.c_uint64, D, D, C.c_double, C.c_double,
                                             C.c_int, C.c_longlong, I, C.c_int, C.c_int, C.c_int, I, D, D, I, I, D]
            _lib = l
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(D)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(I)


def default_threads():
    return max(1, os.cpu_count() or 1)


def acq_array(acq):
    vals = dict(acq)
    vals["n_tx"] = len(acq["angles"])
    vals.setdefault("n_tx_elem", 0)
    vals.setdefault("rough_nee", 1)
    arr = np.array([float(vals[k]) for k in ACQ_KEYS], dtype=np.float64)
    ang = np.asarray(acq["angles"], dtype=np.float64)
    return arr, ang


def img_array(img):
    return np.array([float(img[k] if k in img else IMG_DEFAULTS[k]) for k in IMG_KEYS], dtype=np.float64)


# --------------------------------------------------------------------------------------------
def philox(ctr, key):
    """One Philox4x32-10 block: ctr = 4 uint32, key = 2 uint32 -> 4 uint32."""
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox(*[int(c) & 0xFFFFFFFF for c in ctr], *[int(k) & 0xFFFFFFFF for k in key],
                     out.ctypes.data_as(U))
    return out


def philox_fill(c0_base, c1, c2, c3, k0, k1, n):
    out = np.zeros(4 * n, dtype=np.uint32)
    lib().ora_philox_fill(c0_base & 0xFFFFFFFF, c1, c2, c3, k0, k1, n, out.ctypes.data_as(U))
    return out.reshape(n, 4)


def emit(acq, seed, tx, ray_lo, n):
    """Emission of rays ray_lo .. ray_lo + n - 1 of transmit tx (Sec. 2.3.1): arrays of origins
    (n, 3), directions (n, 3), weights (n,) and transmit time stamps (n,)."""
    a_arr, ang = acq_array(acq)
    out = np.zeros((n, 8))
    lib().ora_emit(a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), C.c_uint64(seed), int(tx), int(ray_lo), int(n),
                   out.ctypes.data_as(D))
    return out[:, 0:3], out[:, 3:6], out[:, 6], out[:, 7]


def interface(w, nin, c1, c2, rho1, rho2):
    """Interface event: dict(tir, cos_i, cos_t, R, T, wr, wt)."""
    out = np.zeros(11)
    lib().ora_interface(_d(w)[1], _d(nin)[1], c1, c2, rho1, rho2, out.ctypes.data_as(D))
    return dict(tir=bool(out[0]), cos_i=out[1], cos_t=out[2], R=out[3], T=out[4], wr=out[5:8].copy(),
                wt=out[8:11].copy())


class Scene:
    """Triangles (nt, 9) with media (nt, 2) = (front, back); scatterers (ns, 3) + amplitudes."""

    def __init__(self, tris, media, scat_pos, scat_amp, r_s, bvh=None, rough=False):
        self.rough = bool(rough)  # theta carries a GGX roughness per medium (4M + 2 entries)
        self.tris, tp = _d(np.asarray(tris).reshape(-1, 9))
        self.media, mp = _i(np.asarray(media).reshape(-1, 2))
        self.sp, spp = _d(np.asarray(scat_pos).reshape(-1, 3))
        self.sa, sap = _d(np.asarray(scat_amp).reshape(-1))
        nt, ns = len(self.tris), len(self.sa)
        if bvh is None:
            bvh = nt + ns > 10000
        self.h = lib().ora_scene_create(nt, tp, mp, ns, spp, sap, float(r_s), int(bool(bvh)), int(self.rough))

    @classmethod
    def from_workload(cls, w, bvh=None):
        return cls(w["tris"], w["media"], w["scat_pos"], w["scat_amp"], w["r_s"], bvh=bvh, rough=w.get("rough", False))

    def closest(self, o, w, xcls=0, xid=-1):
        out = np.zeros(3)
        lib().ora_closest(self.h, _d(o)[1], _d(w)[1], xcls, xid, out.ctypes.data_as(D))
        return out[0], int(out[1]), int(out[2])

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_scene_free(self.h)
            self.h = None


class Run:
    """Forward transport over a range of paths: frozen decisions + arrival list."""

    def __init__(self, scene, theta, M, acq, seed, nthreads=None, path_lo=0, path_hi=-1):
        self.scene = scene
        self.theta = np.asarray(theta, dtype=np.float64)
        self.M = int(M)
        self.acq = acq
        self.seed = int(seed)
        a, ang = acq_array(acq)
        self._a, self._ang = a, ang
        th, thp = _d(self.theta)
        n = nthreads or default_threads()
        self.h = lib().ora_trace(scene.h, thp, self.M, a.ctypes.data_as(D), ang.ctypes.data_as(D),
                                 C.c_uint64(self.seed), n, path_lo, path_hi)
        ntx = len(acq["angles"])
        per_tx = (acq["n_elem"] if acq.get("tx_elem", -1) < 0 else max(1, acq.get("n_tx_elem", 0))) * acq["n_rays"]
        self.path_lo = path_lo
        self.n_paths = (ntx * per_tx if path_hi < 0 else path_hi) - path_lo

    def counters(self):
        out = np.zeros(2, dtype=np.int64)
        lib().ora_run_counters(self.h, out.ctypes.data_as(L))
        return dict(segments=int(out[0]), nee=int(out[1]))

    def arrivals(self):
        n = lib().ora_run_n_arrivals(self.h)
        tx = np.zeros(n, np.int32)
        e = np.zeros(n, np.int32)
        tau = np.zeros(n)
        a = np.zeros(n)
        path = np.zeros(n, np.int64)
        kind = np.zeros(n, np.int32)
        ev = np.zeros(n, np.int32)
        lib().ora_run_arrivals(self.h, tx.ctypes.data_as(I), e.ctypes.data_as(I), tau.ctypes.data_as(D),
                               a.ctypes.data_as(D), path.ctypes.data_as(L), kind.ctypes.data_as(I),
                               ev.ctypes.data_as(I))
        return dict(tx=tx, e=e, tau=tau, a=a, path=path, kind=kind, ev=ev)

    def records(self):
        k1 = self.acq["k_max"] + 1
        n = self.n_paths * k1
        out = [np.zeros(n, np.int32) for _ in range(4)]
        lib().ora_run_records(self.h, *[o.ctypes.data_as(I) for o in out])
        return {k: o.reshape(self.n_paths, k1) for k, o in zip(["cls", "id", "choice", "aux"], out)}

    def rf(self, theta=None):
        acq = self.acq
        out = np.zeros((len(acq["angles"]), acq["n_elem"], acq["n_samples"]))
        th = self.theta if theta is None else np.asarray(theta, np.float64)
        lib().ora_splat_run(self.h, _d(th)[1], out.ctypes.data_as(D))
        return out

    def replay_rf(self, theta, nthreads=None):
        acq = self.acq
        out = np.zeros((len(acq["angles"]), acq["n_elem"], acq["n_samples"]))
        th, thp = _d(theta)
        lib().ora_replay_rf(self.scene.h, self.h, thp, C.c_uint64(self.seed), nthreads or default_threads(),
                            out.ctypes.data_as(D))
        return out

    @property
    def n_theta(self):
        """3M + 2 scene parameters, 4M + 2 with a roughness per medium."""
        return 3 * self.M + 2 + (self.M if self.scene.rough else 0)

    def gradient(self, grf, theta=None, nthreads=None):
        """d/dtheta of sum(grf * RF) on this frozen realisation."""
        th = self.theta if theta is None else np.asarray(theta, np.float64)
        th, thp = _d(th)
        g, gp = _d(grf)
        out = np.zeros(self.n_theta)
        lib().ora_gradient(self.scene.h, self.h, thp, C.c_uint64(self.seed), nthreads or default_threads(), gp,
                           out.ctypes.data_as(D))
        return out

    def gradient_cond(self, grf, theta=None, nthreads=None):
        """(gradient, condition): the gradient of gradient() and, per component, the sum over
        arrivals of the absolute value of each arrival's contribution to it."""
        th = self.theta if theta is None else np.asarray(theta, np.float64)
        th, thp = _d(th)
        g, gp = _d(grf)
        out = np.zeros(self.n_theta)
        cond = np.zeros(self.n_theta)
        lib().ora_gradient_cond(self.scene.h, self.h, thp, C.c_uint64(self.seed), nthreads or default_threads(), gp,
                                out.ctypes.data_as(D), cond.ctypes.data_as(D))
        return out, cond

    def gradient_acq(self, grf, theta=None, nthreads=None, full=False):
        """d/d(c_bf, pitch, steering angles) of sum(grf * RF) on this frozen realisation (Sec.
        2.3.1 emission: time stamps and origins; Sec. 2.3.3 secondary rays: their target element
        centres).  Returns 2 + n_tx values, or with ``full`` the scene gradient followed by them."""
        th = self.theta if theta is None else np.asarray(theta, np.float64)
        th, thp = _d(th)
        g, gp = _d(grf)
        n_th = self.n_theta
        out = np.zeros(n_th + 2 + len(self.acq["angles"]))
        rc = lib().ora_gradient_acq(self.scene.h, self.h, thp, C.c_uint64(self.seed), nthreads or default_threads(), gp,
                                    out.ctypes.data_as(D))
        if rc != 0:
            raise ValueError("too many parameters for the oracle's dual numbers")
        return out if full else out[n_th:]

    def gradient_shape(self, grf, vtan, theta=None, nthreads=None, full=False):
        """Directional derivatives of sum(grf * RF) along vertex tangent fields vtan
        [n_shape, n_tris, 9] (d tris / d q_j) on this frozen realisation: hit distances, normals
        and secondary-ray crossings follow the moved triangles, the decisions stay.  Returns
        n_shape values, or with ``full`` the scene gradient followed by them."""
        th = self.theta if theta is None else np.asarray(theta, np.float64)
        th, thp = _d(th)
        g, gp = _d(grf)
        vt = np.ascontiguousarray(vtan, dtype=np.float64)
        n_shape = vt.shape[0]
        assert vt.shape[1:] == (len(self.scene.tris), 9)
        n_th = self.n_theta
        out = np.zeros(n_th + n_shape)
        rc = lib().ora_gradient_shape(self.scene.h, self.h, thp, C.c_uint64(self.seed), nthreads or default_threads(),
                                      gp, n_shape, vt.ctypes.data_as(D), out.ctypes.data_as(D))
        if rc != 0:
            raise ValueError("too many parameters for the oracle's dual numbers")
        return out if full else out[n_th:]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_run_free(self.h)
            self.h = None


def ggx_normal(n, alpha, u2, u3):
    """GGX microfacet normal around the unit normal n for the uniforms u2, u3."""
    h = np.zeros(3)
    lib().ora_ggx_normal(_d(n)[1], float(alpha), float(u2), float(u3), h.ctypes.data_as(D))
    return h


def splat(acq, f0, tx, e, tau, a):
    a_arr, ang = acq_array(acq)
    out = np.zeros((len(acq["angles"]), acq["n_elem"], acq["n_samples"]))
    n = len(tau)
    lib().ora_splat(a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), float(f0), n, _i(tx)[1], _i(e)[1],
                    _d(tau)[1], _d(a)[1], out.ctypes.data_as(D))
    return out


def splat_adjoint(acq, f0, tx, e, tau, a, grf):
    a_arr, ang = acq_array(acq)
    n = len(tau)
    ga, gt, gf = np.zeros(n), np.zeros(n), np.zeros(n)
    txa, txp = _i(tx)
    ea, ep = _i(e)
    ta, tp = _d(tau)
    aa, ap = _d(a)
    g, gp = _d(grf)
    lib().ora_splat_adjoint(a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), float(f0), n, txp, ep, tp, ap, gp,
                            ga.ctypes.data_as(D), gt.ctypes.data_as(D), gf.ctypes.data_as(D))
    return ga, gt, gf


def das(acq, img, rf):
    a_arr, ang = acq_array(acq)
    out = np.zeros((img["n_lines"], img["n_depth"]))
    r, rp = _d(rf)
    lib().ora_das(a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), img_array(img).ctypes.data_as(D), rp,
                  out.ctypes.data_as(D))
    return out


def das_adjoint(acq, img, gi):
    a_arr, ang = acq_array(acq)
    out = np.zeros((len(acq["angles"]), acq["n_elem"], acq["n_samples"]))
    g, gp = _d(gi)
    lib().ora_das_adjoint(a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), img_array(img).ctypes.data_as(D), gp,
                          out.ctypes.data_as(D))
    return out


def das_acq_vjp(acq, img, rf, gi):
    """sum_p gi(p) dI(p)/d(c_bf, pitch, steering angles), the RF held fixed: 2 + n_tx values."""
    a_arr, ang = acq_array(acq)
    out = np.zeros(2 + len(acq["angles"]))
    r, rp = _d(rf)
    g, gp = _d(gi)
    lib().ora_das_acq_vjp(a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), img_array(img).ctypes.data_as(D), rp, gp,
                          out.ctypes.data_as(D))
    return out


def hilbert(x):
    x, xp = _d(x)
    y = np.zeros(len(x))
    lib().ora_hilbert(xp, len(x), y.ctypes.data_as(D))
    return y


def envelope(img, irf):
    i, ip = _d(irf)
    out = np.zeros_like(i)
    lib().ora_envelope(img_array(img).ctypes.data_as(D), ip, out.ctypes.data_as(D))
    return out


def log_compress(img, env):
    e, ep = _d(env)
    out = np.zeros_like(e)
    am = lib().ora_log_compress(img_array(img).ctypes.data_as(D), ep, out.ctypes.data_as(D))
    return out, int(am)


def loss(img, b, bref):
    bb, bp = _d(b)
    r, rp = _d(bref)
    g = np.zeros_like(bb)
    val = lib().ora_loss(img_array(img).ctypes.data_as(D), bp, rp, g.ctypes.data_as(D))
    return val, g


def envlog_vjp(img, irf, gb):
    i, ip = _d(irf)
    g, gp = _d(gb)
    out = np.zeros_like(i)
    lib().ora_envlog_vjp(img_array(img).ctypes.data_as(D), ip, gp, out.ctypes.data_as(D))
    return out


def bmode(acq, img, rf):
    """RF -> (I_rf, envelope, B-mode in dB)."""
    irf = das(acq, img, rf)
    env = envelope(img, irf)
    b, _ = log_compress(img, env)
    return irf, env, b


def bmode_vjp(acq, img, rf, gb):
    """dL/dRF from dL/dB through log, envelope and DAS."""
    irf = das(acq, img, rf)
    gi = envlog_vjp(img, irf, gb)
    return das_adjoint(acq, img, gi)


def forward(w, seed=None, theta=None, nthreads=None, scene=None, path_lo=0, path_hi=-1):
    """Whole forward hot path for a workload dict (phantoms): RF, I_rf, envelope, B-mode."""
    sc = scene or Scene.from_workload(w)
    th = w["theta"] if theta is None else theta
    run = Run(sc, th, w["M"], w["acq"], w["seed"] if seed is None else seed, nthreads, path_lo, path_hi)
    rf = run.rf()
    irf, env, b = bmode(w["acq"], w["img"], rf)
    return dict(scene=sc, run=run, rf=rf, irf=irf, env=env, b=b)


def trace_injected(scene, theta, M, acq, o, w, a0=1.0, tau0=0.0, tx=0, ray=0, forced=None, physical=False,
                   seed=0):
    """One injected path; returns (arrivals list of (e, tau, a, kind), records (k_max+1, 4), last state).

    The last state is the position and direction (6 values) at the path's final hit."""
    a_arr, ang = acq_array(acq)
    cap = acq["k_max"] + 2
    e = np.zeros(cap, np.int32)
    tau = np.zeros(cap)
    a = np.zeros(cap)
    kind = np.zeros(cap, np.int32)
    rec = np.zeros(4 * (acq["k_max"] + 1), np.int32)
    last = np.full(6, np.nan)
    f = np.asarray(forced if forced is not None else [], np.int32)
    n = lib().ora_trace_injected(scene.h, _d(theta)[1], M, a_arr.ctypes.data_as(D), ang.ctypes.data_as(D),
                                 C.c_uint64(seed), _d(o)[1], _d(w)[1], float(a0), float(tau0), tx, ray,
                                 f.ctypes.data_as(I) if len(f) else None, len(f), int(physical), cap,
                                 e.ctypes.data_as(I), tau.ctypes.data_as(D), a.ctypes.data_as(D),
                                 kind.ctypes.data_as(I), rec.ctypes.data_as(I), last.ctypes.data_as(D))
    arr = [(int(e[i]), float(tau[i]), float(a[i]), int(kind[i])) for i in range(n)]
    return arr, rec.reshape(-1, 4), last


def inject_sums(scene, theta, M, acq, o, w, seed=0, nthreads=None):
    """Injected paths (origins o[n, 3], unit directions w[n, 3], weight 1): per element, the
    sum of what the paths deposit there and the sum of the squares of the per-path amounts."""
    a_arr, ang = acq_array(acq)
    o, op = _d(np.asarray(o).reshape(-1, 3))
    w, wp = _d(np.asarray(w).reshape(-1, 3))
    s = np.zeros(acq["n_elem"])
    s2 = np.zeros(acq["n_elem"])
    lib().ora_inject_sums(scene.h, _d(theta)[1], M, a_arr.ctypes.data_as(D), ang.ctypes.data_as(D), C.c_uint64(seed),
                          len(o), op, wp, nthreads or default_threads(), s.ctypes.data_as(D), s2.ctypes.data_as(D))
    return s, s2
