"""vi_render_host_noalloc: rendering for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: a plug-in whose host application owns the
GPU's memory, a process under a hard device-memory cap, a real-time loop that
cannot take an allocation's latency.  This entry point renders with the
context's resident data into a host buffer, using only a fixed device array
inside the library for the march's work counter and the frame's staging.

These tests call it through the C ABI and check its frames against vi_render's
(the existing entry point): the same kernel with the same parameters on the
same data, so the frames must be equal bit for bit, on two calls in a row (the
shared array keeps the previous call's contents, which must not leak into the
next frame).  They also check that a call allocates nothing: on a fresh
context, before any vi_render, a byte budget that refuses every new buffer
still lets it run, and the device's free memory does not move across a call.
The file is named to be collected last, and passes both alone in a fresh
process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture()
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    ctx = vi.Context(0)
    yield ctx, vi, ph
    ctx.close()


def _load(ctx, sc):
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir, sc.light_color)
    ctx.build_attenuation(sc.n_slices, sc.slice_res, sc.mode,
                          cone_half_angle_deg=sc.cone_half_angle_deg,
                          shell_radius_vox=sc.shell_radius_vox)


def _noalloc(vi, ctx, sc, W, H, ert):
    """One call of vi_render_host_noalloc straight through the C ABI."""
    out = np.full((H, W, 4), np.nan, dtype=np.float32)
    ro = vi.RenderOpts(float(ert), (C.c_float * 4)(*map(float, sc.bg)), 0.0, 0, None, None)
    rc = vi.library().vi_render_host_noalloc(ctx.h, C.byref(vi.camera(sc.camera)), int(W), int(H),
                                             float(sc.step_vox), C.c_void_p(out.ctypes.data),
                                             C.byref(ro))
    return rc, out


def test_noalloc_allocates_nothing(setup):
    """On a fresh context, before any vi_render: with a budget of one byte
    the context can grow no buffer, yet the call succeeds (vi_render, which
    stages host output in a context buffer, is refused); and once the
    library's device code is loaded, the device's free memory is the same
    before and after a call."""
    import torch
    ctx, vi, ph = setup
    sc = ph.blob64_shell(ert=0.95)
    sc.mode = vi.CONE
    _load(ctx, sc)
    ctx.set_memory_budget(1)
    for _ in range(2):                      # the first call may load the module's code
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc, out = _noalloc(vi, ctx, sc, 256, 256, sc.ert)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert rc == vi.OK, vi.error_string(rc)
        assert np.isfinite(out).all()
    assert free1 == free0
    with pytest.raises(vi.ViError) as e:     # host output needs a staging buffer
        ctx.render(sc.camera, 256, 256, sc.step_vox, out=np.empty((256, 256, 4), np.float32),
                   ert=sc.ert)
    assert e.value.code == vi.ENOMEM
    ctx.set_memory_budget(0)
    ref = ctx.render(sc.camera, 256, 256, sc.step_vox, ert=sc.ert, bg=sc.bg).cpu().numpy()
    assert np.array_equal(out, ref)


def test_noalloc_frames_match_vi_render_on_two_calls_in_a_row(setup):
    ctx, vi, ph = setup
    sc = ph.blob64_shell(ert=0.95)
    sc.mode = vi.CONE
    _load(ctx, sc)
    # Two different frames in a row: the second one must not see the first.
    for W, H in ((256, 256), (200, 120)):
        ref = ctx.render(sc.camera, W, H, sc.step_vox, ert=sc.ert, bg=sc.bg).cpu().numpy()
        rc, out = _noalloc(vi, ctx, sc, W, H, sc.ert)
        assert rc == vi.OK, vi.error_string(rc)
        assert np.array_equal(out, ref)
    # Same frame twice more: identical results, call after call.
    rc1, a = _noalloc(vi, ctx, sc, 256, 256, sc.ert)
    rc2, b = _noalloc(vi, ctx, sc, 256, 256, sc.ert)
    assert rc1 == rc2 == vi.OK
    assert np.array_equal(a, b)


def test_noalloc_rejects_frames_above_its_array(setup):
    ctx, vi, ph = setup
    sc = ph.blob64_shell()
    _load(ctx, sc)
    rc, out = _noalloc(vi, ctx, sc, 513, 512, sc.ert)
    assert rc == vi.EINVAL
    assert np.isnan(out).all()          # nothing was written
    rc, out = _noalloc(vi, ctx, sc, 512, 512, sc.ert)
    assert rc == vi.OK and np.isfinite(out).all()
