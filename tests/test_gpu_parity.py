"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Same seeded inputs on both sides.  Floating point: max abs error <= 1e-4 per
RGBA channel for the FP32 path (1e-5 on the attenuation stack).  Integer
decisions (sample counts, slice / texel / voxel cells, the binary32 sample
positions) must match bit for bit.
"""
import numpy as np
import pytest

from gpu_common import (FORMAT_HALF_ULP, IMAGE_TOL, STACK_TOL, check_frame, gpu_frame,
                        oracle_frame)

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


@pytest.fixture(scope="module")
def blob():
    from paper_2008_06134_gb300 import phantoms as ph
    return ph.blob64_shell()


def ragged_scene(mode, persp, seed=11):
    """Non-cubic volume, ragged image / light resolutions, odd slice count."""
    from paper_2008_06134_gb300 import phantoms as ph
    rng = np.random.default_rng(seed)
    vol = ph.gaussian_blobs(48, seed)[:27, :33, :40].copy()
    sc = ph.blob64_shell(seed)
    sc.volume = vol
    sc.n_slices, sc.slice_res = 37, 45
    sc.width, sc.height = 53, 37
    sc.mode = mode
    sc.light_dir = ph.random_direction(rng)
    sc.camera = ph.orbit_camera(ph.random_direction(rng), persp, 2.4 if persp else 2.0)
    sc.step_vox = 0.37
    return sc


def test_sweep_stack_matches_oracle(ctx, orc, blob):
    gpu_frame(ctx, blob)
    B = ctx.get_attenuation().astype(np.float64)
    light = orc.light_setup(blob.light_dir, blob.n_slices, blob.slice_res)
    ref = orc.build_stack(blob.volume, blob.tf, blob.vmin, blob.vmax, light)
    assert B.shape == ref.shape
    assert np.abs(B - ref).max() <= STACK_TOL
    assert B[0].min() == 1.0


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_frame_matches_oracle_blob64(ctx, orc, blob, mode):
    gpu, counts = gpu_frame(ctx, blob, mode=mode, counts=True)
    ora = oracle_frame(orc, blob, mode=mode)
    check_frame(gpu, counts, ora)
    assert ora[3].sum() > 2_000_000  # the whole frame was marched


@pytest.mark.parametrize("mode,persp", [(0, False), (1, True), (2, False), (3, True), (3, False)])
def test_ragged_sizes_match_oracle(ctx, orc, mode, persp):
    sc = ragged_scene(mode, persp)
    gpu, counts = gpu_frame(ctx, sc, counts=True)
    ora = oracle_frame(orc, sc)
    check_frame(gpu, counts, ora)
    assert np.array_equal(counts, ora[3])
    if mode:
        B = ctx.get_attenuation().astype(np.float64)
        light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
        ref_B = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
        assert np.abs(B - ref_B).max() <= STACK_TOL


@pytest.mark.parametrize("mode,persp", [(0, False), (1, False), (2, True), (3, True)])
def test_trace_is_bit_exact(ctx, orc, mode, persp):
    """Every integer decision and every binary32 position of a ray agrees."""
    sc = ragged_scene(mode, persp, seed=5)
    gpu_frame(ctx, sc)
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    stack = None
    if mode:
        stack = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
    ro = orc.render_opts(mode, sc.step_vox, sc.ert, sc.bg, sc.light_color,
                         cone_half_angle_deg=sc.cone_half_angle_deg,
                         shell_radius_vox=sc.shell_radius_vox)
    rng = np.random.default_rng(1)
    traced = 0
    for _ in range(12):
        x, y = int(rng.integers(sc.width)), int(rng.integers(sc.height))
        g = ctx.trace_pixel(sc.camera, sc.width, sc.height, sc.step_vox, x, y, ert=sc.ert)
        o = orc.trace_pixel(sc.volume, sc.tf, sc.vmin, sc.vmax, light, stack, sc.camera,
                            sc.width, sc.height, ro, x, y)
        assert g.shape == o.shape, (x, y, g.shape, o.shape)
        assert np.array_equal(g, o), (x, y, np.argwhere(g != o)[:5])
        traced += len(g)
    assert traced > 100


def test_empty_volume_is_background_bit_exact(ctx):
    from paper_2008_06134_gb300 import phantoms as ph
    sc = ph.blob64_shell()
    sc.volume = np.zeros((20, 21, 22), np.uint8)
    sc.tf = np.zeros((256, 4), np.float32)
    sc.tf[1:] = (1, 1, 1, 0.5)
    sc.width, sc.height = 33, 17
    bg = (0.1, 0.2, 0.3, 0.4)
    for mode in (0, 1, 2, 3):
        gpu, _ = gpu_frame(ctx, sc, mode=mode, bg=bg)
        assert np.all(gpu == np.array(bg, dtype=np.float32).astype(np.float64))
        if mode:
            assert ctx.get_attenuation().min() == 1.0


@pytest.mark.parametrize("fmt", [1, 2, 3])
def test_storage_formats_within_rounding(ctx, orc, blob, fmt):
    """FP16 / BF16 / UNORM16 storage: each stored value is the FP32 one rounded,
    so the stack and the image stay within half an ulp of the format (plus the
    FP32 tolerance) of the FP64 oracle."""
    from paper_2008_06134_gb300 import vi
    for mode in (1, 3):
        gpu, _ = gpu_frame(ctx, blob, mode=mode, fmt=fmt)
        check_frame(gpu, None, oracle_frame(orc, blob, mode=mode), FORMAT_HALF_ULP[fmt] + IMAGE_TOL)
    raw = ctx.get_attenuation()
    B = vi.decode_stack(raw, fmt)
    light = orc.light_setup(blob.light_dir, blob.n_slices, blob.slice_res)
    ref_B = orc.build_stack(blob.volume, blob.tf, blob.vmin, blob.vmax, light)
    assert np.abs(B - ref_B).max() <= FORMAT_HALF_ULP[fmt] * 1.0001 + STACK_TOL


def test_opacity_correction_and_compensation(ctx, orc, blob):
    gpu, _ = gpu_frame(ctx, blob, mode=1, build_oc=1, comp_n=1.5, opacity_correction=1)
    check_frame(gpu, None, oracle_frame(orc, blob, mode=1, build_oc=1, comp_n=1.5,
                                        opacity_correction=1))
    B = ctx.get_attenuation().astype(np.float64)
    light = orc.light_setup(blob.light_dir, blob.n_slices, blob.slice_res)
    ref_B = orc.build_stack(blob.volume, blob.tf, blob.vmin, blob.vmax, light,
                            opacity_correction=1, comp_n=1.5)
    assert np.abs(B - ref_B).max() <= STACK_TOL


def test_early_ray_termination_and_background(ctx, orc, blob):
    bg = (0.2, 0.1, 0.05, 0.3)
    gpu, counts = gpu_frame(ctx, blob, mode=3, ert=0.6, bg=bg, counts=True)
    ora = oracle_frame(orc, blob, mode=3, ert=0.6, bg=bg)
    check_frame(gpu, counts, ora)
    ns = ora[3]
    assert (ns < ns.max()).any()


def test_ct256_cone_full_size_sampled(ctx, orc):
    """The benchmark's workload (256^3 uint16 CT phantom, 256 x 512^2 FP32 stack,
    cone 15 deg, 1024^2 perspective, ERT 0.99) in the benchmark's launch
    configuration; the oracle checks sampled texels of the stack and sampled
    pixels of the frame (plus two full rows)."""
    from paper_2008_06134_gb300 import phantoms as ph
    sc = ph.ct256_cone()
    gpu, counts = gpu_frame(ctx, sc, counts=True)
    B = ctx.get_attenuation()
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    ref_B = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
    rng = np.random.default_rng(0)
    kk, jj, ii = (rng.integers(0, d, 20000) for d in ref_B.shape)
    assert np.abs(B[kk, jj, ii] - ref_B[kk, jj, ii]).max() <= STACK_TOL
    xs = np.concatenate([rng.integers(0, 1024, 3000), np.arange(1024), np.arange(1024)])
    ys = np.concatenate([rng.integers(0, 1024, 3000), np.full(1024, 500), np.full(1024, 700)])
    ora = oracle_frame(orc, sc, xs=xs, ys=ys, stack=ref_B)
    check_frame(gpu[ys, xs], counts[ys, xs], ora)
    assert (ora[0][:, 3] > 0.5).mean() > 0.05  # the phantom is in view
