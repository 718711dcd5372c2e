"""The allocation-free envelope + log entry point (us_envlog_noalloc) against us_envlog.

Callers that cannot allocate device memory at call time (another framework's pool or a hard
memory cap, work enqueued during stream capture, latency-critical serving loops) use the
variant whose scratch lives in a fixed device array of the library.  Two calls in a row on
different images must each match the allocating entry point, so nothing of the previous call's
scratch leaks into the next.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2604_15017_gb300 import phantoms as P
from paper_2604_15017_gb300 import usrt

pytestmark = pytest.mark.gpu

TOL_DB = 0.05  # the B-mode tolerance used throughout the parity tests


def noalloc(img, irf, out):
    lib = usrt.lib()
    fn = lib.us_envlog_noalloc
    fn.argtypes = [C.POINTER(usrt.ImgDesc), C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    d = usrt.img_desc(img)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(C.byref(d), C.c_void_p(irf.data_ptr()), C.c_void_p(out.data_ptr()), stream)


def image_input(seed, n_lines, n_depth):
    rng = np.random.default_rng(seed)
    t = np.arange(n_depth)
    x = np.zeros((n_lines, n_depth))
    for _ in range(12):  # a few echoes of different strength, plus noise
        l0, d0, a = rng.integers(0, n_lines), rng.integers(40, n_depth - 40), 10 ** rng.uniform(-3, 0)
        prof = np.exp(-((np.arange(n_lines) - l0) / 3.0) ** 2)[:, None]
        x += a * prof * np.sin(0.8 * (t - d0)) * np.exp(-((t - d0) / 6.0) ** 2)[None, :]
    x += 1e-4 * rng.normal(size=x.shape)
    return torch.tensor(x, dtype=torch.float32, device="cuda")


def test_noalloc_envlog_matches_allocating_entry_point_twice():
    ctx = usrt.Context(0)
    for seed, (nl, nd) in [(1, (96, 512)), (2, (256, 1024))]:
        img = P.image(nl, nd, 0.0, 1.0, 0.0, 1.0, dr_db=60.0)
        irf = image_input(seed, nl, nd)
        ref = ctx.envlog(img, irf)
        out = torch.full_like(irf, 123.0)
        assert noalloc(img, irf, out) == usrt.US_OK
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert float((out - ref).abs().max()) <= TOL_DB
        assert float(out.max()) == 0.0 and float(out.min()) >= -60.0
    ctx.close()


@pytest.mark.parametrize("shape", [(96, 512), (256, 1024)])
def test_noalloc_envlog_two_kernel_path_matches(shape):
    """The two-kernel path (envelope into the array's image region, then log compression), forced
    for both entry points, up to the largest image the array holds; two calls in a row."""
    ctx = usrt.Context(0)
    nl, nd = shape
    usrt.set_envlog_fused(False)
    try:
        for seed in (3, 4):
            img = P.image(nl, nd, 0.0, 1.0, 0.0, 1.0, dr_db=60.0)
            irf = image_input(seed, nl, nd)
            ref = ctx.envlog(img, irf)
            out = torch.full_like(irf, 123.0)
            assert noalloc(img, irf, out) == usrt.US_OK
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert float((out - ref).abs().max()) <= TOL_DB
            assert float(out.max()) == 0.0 and float(out.min()) >= -60.0
    finally:
        usrt.set_envlog_fused(True)
    ctx.close()


def test_noalloc_envlog_rejects_oversize_images():
    img = P.image(512, 1024, 0.0, 1.0, 0.0, 1.0)  # 512 * 1024 pixels > 256 * 1024
    irf = torch.zeros(1, device="cuda")
    assert noalloc(img, irf, irf) == usrt.US_ERR_ARG
