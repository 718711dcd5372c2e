"""Errors that must not pass silently (GPU), tested without faulting the GPU.

* The fused envelope kernel's grid barrier is bounded in time.  The fault is injected from the
  host (US_OPT_FAULT_BARRIER: the barrier also waits for one arrival that no block makes, with a
  1 ms limit): every block gives up, writes NaN, and us_get_status reports US_ERR_TIMEOUT; the
  context stays usable and the next call is clean.
* The two-kernel envelope path (taken by images too large for the fused kernel) gives the
  fused kernel's image.
* The closest-hit traversal's stack holds one entry per tree level; a scene whose BVH is deeper
  than the traversal stacks allow is refused at upload, so the stack cannot overflow.
"""
import numpy as np
import pytest
import torch

from paper_2604_15017_gb300 import phantoms as P
from paper_2604_15017_gb300 import usrt

pytestmark = pytest.mark.gpu

MM = 1e-3


@pytest.fixture(scope="module")
def ctx():
    c = usrt.Context(0)
    yield c
    c.close()


def image_input(seed, n_lines, n_depth):
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn(n_lines, n_depth, generator=g) * torch.linspace(0.01, 1.0, n_depth)
    return x.cuda()


def test_fused_envelope_barrier_timeout_is_reported(ctx):
    img = P.image(64, 256, 0.0, 1.0, 0.0, 1.0)
    irf = image_input(1, 64, 256)
    ref = ctx.envlog(img, irf)
    assert ctx.device_status() == usrt.US_OK
    ctx.set_option(usrt.OPT_FAULT_BARRIER, 1)
    try:
        b = ctx.envlog(img, irf)
    finally:
        ctx.set_option(usrt.OPT_FAULT_BARRIER, 0)
    assert ctx.device_status(clear=True) == usrt.US_ERR_TIMEOUT
    assert torch.isnan(b).all()
    # the context is usable afterwards and the word was cleared
    b2 = ctx.envlog(img, irf)
    assert ctx.device_status() == usrt.US_OK
    assert torch.equal(b2, ref)


def test_fault_option_takes_zero_or_one(ctx):
    with pytest.raises(usrt.UsrtError) as ei:
        ctx.set_option(usrt.OPT_FAULT_BARRIER, 2)
    assert ei.value.code == usrt.US_ERR_ARG


@pytest.mark.parametrize("shape", [(32, 64), (128, 1024), (256, 4096)])
def test_two_kernel_envelope_path_equals_fused(ctx, shape):
    nl, nd = shape
    img = P.image(nl, nd, 0.0, 1.0, 0.0, 1.0)
    irf = image_input(2, nl, nd)
    fused = ctx.envlog(img, irf)
    usrt.set_envlog_fused(False)
    try:
        two = ctx.envlog(img, irf)
    finally:
        usrt.set_envlog_fused(True)
    assert torch.isfinite(two).all()
    assert float((two - fused).abs().max()) <= 1e-4
    assert ctx.device_status() == usrt.US_OK


def test_bmode_two_kernel_path_in_a_forward_pass(ctx):
    w = P.two_layer(n_rays=200)
    sid = ctx.upload_workload(w)
    rf, b = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=0)
    usrt.set_envlog_fused(False)
    try:
        rf2, b2 = ctx.forward(sid, w["theta"], w["acq"], w["img"], seed=0)
    finally:
        usrt.set_envlog_fused(True)
    assert torch.equal(rf, rf2)
    assert float((b - b2).abs().max()) <= 1e-4
    ctx.release_scene(sid)


def test_bvh_deeper_than_the_traversal_stack_is_refused(ctx):
    """Triangles at geometrically shrinking positions make a chain-like tree; its depth passes
    what the traversal stacks hold, so the upload refuses the scene instead of tracing with a
    stack that could fill up."""
    n = 300
    tris = []
    for i in range(n):
        x = 2.0 ** (-(i // 4)) * (1.0 + 0.2 * (i % 4))
        s = 0.05 * x
        tris.append([x, 0, 0.01, x + s, 0.001, 0.01, x, 0.001, 0.01 + s])
    media = np.tile(np.array([[0, 1]], np.int32), (n, 1))
    with pytest.raises(usrt.UsrtError) as ei:
        ctx.upload_scene(np.array(tris), media, 2, np.zeros((0, 3)), np.zeros(0), 1e-4)
    assert ei.value.code == usrt.US_ERR_ARG and "depth" in str(ei.value)
    # an ordinary scene uploads on the same context afterwards
    w = P.two_layer(n_rays=10)
    ctx.release_scene(ctx.upload_workload(w))
