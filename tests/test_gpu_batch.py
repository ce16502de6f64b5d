"""Batched frames (vi_render_batch): several contexts' frames in persistent
launches, each frame's tiles waiting on the device until its context has
published its stack (vi_post_ready), at most a stated time.  Every frame must
equal the frame vi_render gives from the same context, and the FP64 oracle's
within the image tolerance; a frame whose context never publishes must come
back VI_ETIMEOUT within the limit, with the others rendered and the GPU still
usable.  The wait is made to run out on the host side of the protocol (a
context that never posts), never by faulting or hanging the GPU."""
import time

import numpy as np
import pytest

from gpu_common import FORMAT_HALF_ULP, IMAGE_TOL, check_frame, oracle_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    return torch, ph, vi


def scenes(ph, vi):
    """Four small scenes of four kinds: u8 / u16 volumes, FP32 / FP16 stacks,
    modes none, shadow, shell, cone; ragged image sizes."""
    out = []
    specs = [(vi.NONE, vi.F32, False, (37, 29)), (vi.SHADOW, vi.F16, True, (64, 40)),
             (vi.SHELL, vi.F32, True, (45, 51)), (vi.CONE, vi.F16, False, (80, 64))]
    for k, (mode, fmt, u16, (W, H)) in enumerate(specs):
        sc = ph.blob64_shell(seed=30 + k, ert=0.95 if k % 2 else 2.0)
        if u16:
            sc.volume = ph.ct_phantom(40, 30 + k)
            sc.tf, sc.vmin, sc.vmax = ph.tf_ct(512, 30 + k), 0.0, 4095.0
        else:
            sc.volume = ph.gaussian_blobs(36, 30 + k)
        sc.mode, sc.fmt = mode, fmt
        sc.n_slices, sc.slice_res, sc.width, sc.height = 21 + k, 33, W, H
        sc.camera = ph.orbit_camera(ph.random_direction(np.random.default_rng(k)), k % 2 == 0, 2.4)
        out.append(sc)
    return out


def prepare(vi, sc, stream=None, post=True):
    ctx = vi.Context(0, stream=stream)
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir, sc.light_color)
    ctx.build_attenuation(sc.n_slices, sc.slice_res, sc.mode, format=sc.fmt)
    if post:
        ctx.post_ready()
    return ctx


def test_batched_frames_equal_vi_render_and_the_oracle(env):
    import oracle
    torch, ph, vi = env
    oracle.build()
    scs = scenes(ph, vi)
    ctxs = [prepare(vi, sc) for sc in scs]
    frames = []
    for c, sc in zip(ctxs, scs):
        frames.append(dict(ctx=c, cam=sc.camera, W=sc.width, H=sc.height, step_vox=sc.step_vox,
                           ert=sc.ert, out=torch.full((sc.height, sc.width, 4), float("nan"),
                                                       device="cuda"),
                           sample_counts=torch.full((sc.height, sc.width), -1, dtype=torch.int32,
                                                    device="cuda")))
    rc, st = vi.render_batch(frames, wait_ms=5000.0)
    torch.cuda.synchronize()
    assert rc == vi.OK and st == [vi.OK] * len(scs)
    for c, sc, fr in zip(ctxs, scs, frames):
        ref = c.render(sc.camera, sc.width, sc.height, sc.step_vox, ert=sc.ert)
        torch.cuda.synchronize()
        got = fr["out"].cpu().numpy()
        assert np.array_equal(got, ref.cpu().numpy())
        ora = oracle_frame(oracle, sc)
        check_frame(got, fr["sample_counts"].cpu().numpy(), ora, IMAGE_TOL + FORMAT_HALF_ULP[sc.fmt])
    for c in ctxs:
        c.close()


def test_batch_on_another_stream_follows_the_publication(env):
    """The batch is enqueued on its own stream right after a large sweep was
    enqueued on the context's stream: it runs after the context's
    publication, and the frame equals vi_render's."""
    torch, ph, vi = env
    sc = scenes(ph, vi)[3]
    other = torch.cuda.Stream()
    ctx = prepare(vi, sc, stream=other, post=False)
    ctx.build_attenuation(512, 1024, sc.mode, format=sc.fmt)   # a 512 x 1024^2 stack
    ctx.post_ready()
    out = torch.full((sc.height, sc.width, 4), float("nan"), device="cuda")
    rc, st = vi.render_batch([dict(ctx=ctx, cam=sc.camera, W=sc.width, H=sc.height,
                                   step_vox=sc.step_vox, ert=sc.ert, out=out)],
                             stream=torch.cuda.current_stream(), wait_ms=10000.0)
    assert rc == vi.OK and st == [vi.OK]
    other.synchronize()
    ref = ctx.render(sc.camera, sc.width, sc.height, sc.step_vox, ert=sc.ert)
    other.synchronize()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    ctx.close()


def test_wait_that_runs_out_returns_timeout_and_the_gpu_stays_usable(env):
    """One context never posts: with a 1 ms limit its frame comes back
    VI_ETIMEOUT, the kernel returns, the other frames are rendered, and the
    device keeps working (a plain frame and a second batch afterwards)."""
    torch, ph, vi = env
    scs = scenes(ph, vi)
    ctxs = [prepare(vi, sc, post=(k != 1)) for k, sc in enumerate(scs)]
    frames = [dict(ctx=c, cam=sc.camera, W=sc.width, H=sc.height, step_vox=sc.step_vox,
                   ert=sc.ert, out=torch.zeros((sc.height, sc.width, 4), device="cuda"))
              for c, sc in zip(ctxs, scs)]
    t0 = time.perf_counter()
    rc, st = vi.render_batch(frames, wait_ms=1.0)
    elapsed = time.perf_counter() - t0
    assert rc == vi.ETIMEOUT
    assert st[1] == vi.ETIMEOUT and [s for k, s in enumerate(st) if k != 1] == [vi.OK] * 3
    assert elapsed < 5.0
    for k in (0, 2, 3):
        ref = ctxs[k].render(scs[k].camera, scs[k].width, scs[k].height, scs[k].step_vox,
                             ert=scs[k].ert)
        torch.cuda.synchronize()
        assert np.array_equal(frames[k]["out"].cpu().numpy(), ref.cpu().numpy())
    # The late context publishes: the same batch now renders in full.
    ctxs[1].post_ready()
    rc, st = vi.render_batch(frames, wait_ms=5000.0)
    assert rc == vi.OK and st == [vi.OK] * 4
    for c in ctxs:
        c.sync()
        c.close()


def test_batch_arguments_are_validated(env):
    torch, ph, vi = env
    sc = scenes(ph, vi)[0]
    ctx = prepare(vi, sc)
    out = torch.zeros((sc.height, sc.width, 4), device="cuda")
    fr = dict(ctx=ctx, cam=sc.camera, W=sc.width, H=sc.height, step_vox=sc.step_vox, out=out)
    with pytest.raises(vi.ViError) as e:
        vi.render_batch([fr], wait_ms=-1.0)
    assert e.value.code == vi.EINVAL
    with pytest.raises(vi.ViError) as e:
        vi.render_batch([fr] * (vi.BATCH_MAX_FRAMES + 1))
    assert e.value.code == vi.EINVAL
    ctx.build_attenuation(sc.n_slices, sc.slice_res, vi.SHADOW, format=vi.BF16)
    with pytest.raises(vi.ViError) as e:      # BF16 stacks are not batched
        vi.render_batch([fr])
    assert e.value.code == vi.EINVAL
    ctx.close()
