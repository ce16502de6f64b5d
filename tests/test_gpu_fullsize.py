"""Full-size parity in the benchmark's launch configuration for the two large
workloads, on sampled outputs the oracle computes one by one:

- the precision workload: 512^3 uint16 blobs, 512 slices of 1024^2 in FP32
  (cone) and FP16 (shell), 1920 x 1080 perspective;
- the large-volume workload: 1024^3 uint16 CT phantom (2 GiB), 1024 slices of
  2048^2 in FP16 (8 GiB on the device), cone, 3840 x 2160 perspective, ERT 0.99.

The oracle builds the whole FP64 stack (4 GiB and 32 GiB of host memory) and
checks 20 000 random texels, then renders 3000 random pixels plus a full image
row and compares them, sample counts included.  Tolerances: 1e-5 on the stack
and 1e-4 on the image for FP32, plus half an ulp at 1 for FP16 storage.
"""
import numpy as np
import pytest

from gpu_common import FORMAT_HALF_ULP, IMAGE_TOL, STACK_TOL, check_frame, gpu_frame, oracle_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, vi
    build.build()
    c = vi.Context(0)
    yield c
    c.close()


def check_sampled(ctx, orc, sc, fmt, mode, seed):
    gpu, counts = gpu_frame(ctx, sc, fmt=fmt, mode=mode, counts=True)
    n, R, got_fmt, _ = ctx.attenuation_info()
    assert (n, R, got_fmt) == (sc.n_slices, sc.slice_res, fmt)
    B = ctx.get_attenuation()
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    ref_B = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
    rng = np.random.default_rng(seed)
    kk, jj, ii = (rng.integers(0, d, 20000) for d in ref_B.shape)
    err_B = np.abs(B[kk, jj, ii].astype(np.float64) - ref_B[kk, jj, ii])
    assert err_B.max() <= STACK_TOL + FORMAT_HALF_ULP[fmt], err_B.max()
    assert ref_B[kk, jj, ii].min() < 0.5          # the light is really attenuated
    del B
    W, H = sc.width, sc.height
    xs = np.concatenate([rng.integers(0, W, 3000), np.arange(W)])
    ys = np.concatenate([rng.integers(0, H, 3000), np.full(W, H // 2)])
    ora = oracle_frame(orc, sc, mode=mode, xs=xs, ys=ys, stack=ref_B)
    check_frame(gpu[ys, xs], counts[ys, xs], ora, IMAGE_TOL + FORMAT_HALF_ULP[fmt])
    assert (ora[0][:, 3] > 0.5).mean() > 0.05     # the volume is in view


@pytest.fixture(scope="module")
def blob512():
    from paper_2008_06134_gb300 import phantoms as ph
    return ph.blob512_precision()


def test_blob512_cone_fp32_full_size_sampled(ctx, orc, blob512):
    check_sampled(ctx, orc, blob512, fmt=0, mode=3, seed=1)


def test_blob512_shell_fp16_full_size_sampled(ctx, orc, blob512):
    check_sampled(ctx, orc, blob512, fmt=1, mode=2, seed=2)


def test_ct1024_cone_fp16_full_size_sampled(ctx, orc):
    from paper_2008_06134_gb300 import phantoms as ph
    sc = ph.ct1024_large()
    assert sc.volume.shape == (1024, 1024, 1024) and sc.volume.dtype == np.uint16
    check_sampled(ctx, orc, sc, fmt=1, mode=3, seed=3)
