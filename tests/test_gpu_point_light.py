"""Parity of the point light (rays from a light position, perspective texel
columns) with the FP64 oracle, through the C ABI: stacks, frames in every
mode, bit-exact traces, storage formats and the variant options.  Same
tolerances as the directional light."""
import math

import numpy as np
import pytest

from gpu_common import FORMAT_HALF_ULP, IMAGE_TOL, STACK_TOL, check_frame, gpu_frame, oracle_frame

pytestmark = pytest.mark.gpu

POSITIONS = {"near": (0.5 + 0.62, 0.5 - 0.45, 0.5 + 0.66),     # 1.0 from the centre
             "far": (0.5 - 1.9, 0.5 + 1.4, 0.5 + 2.2)}


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
def vi_mod():
    from paper_2008_06134_gb300 import vi
    return vi


def scene(mode, persp, seed=41):
    """Non-cubic blob volume, ragged image and light resolutions."""
    from paper_2008_06134_gb300 import phantoms as ph
    rng = np.random.default_rng(seed)
    sc = ph.blob64_shell(seed)
    sc.volume = ph.gaussian_blobs(48, seed)[:31, :38, :44].copy()
    sc.tf[:, 3] *= 3.0
    sc.n_slices, sc.slice_res = 43, 53
    sc.width, sc.height = 59, 47
    sc.mode = mode
    sc.camera = ph.orbit_camera(ph.random_direction(rng), persp, 2.4 if persp else 2.0)
    sc.step_vox = 0.43
    sc.ert = 0.97
    return sc


@pytest.mark.parametrize("where", ["near", "far"])
def test_point_light_stack_matches_oracle(ctx, orc, vi_mod, where):
    sc = scene(vi_mod.SHADOW, True)
    pos = POSITIONS[where]
    gpu_frame(ctx, sc, light_pos=pos)
    B = ctx.get_attenuation().astype(np.float64)
    light = orc.point_light_setup(pos, sc.n_slices, sc.slice_res)
    ref = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
    assert B.shape == ref.shape
    assert np.abs(B - ref).max() <= STACK_TOL
    assert ref.min() < 0.5                      # the light is really attenuated


@pytest.mark.parametrize("where", ["near", "far"])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_point_light_frames_match_oracle(ctx, orc, vi_mod, mode, where):
    sc = scene(mode, persp=mode != 2)
    pos = POSITIONS[where]
    gpu, counts = gpu_frame(ctx, sc, counts=True, light_pos=pos)
    check_frame(gpu, counts, oracle_frame(orc, sc, light_pos=pos))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_point_light_traces_are_bit_exact(ctx, orc, vi_mod, mode):
    """Per-sample light coordinates (with the perspective divide), slice and
    texel cells of the sample and of every scattering point agree bit for bit."""
    sc = scene(mode, persp=True, seed=43)
    pos = POSITIONS["near"]
    gpu_frame(ctx, sc, light_pos=pos)
    light = orc.point_light_setup(pos, sc.n_slices, sc.slice_res)
    stack = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light) if mode else None
    ro = orc.render_opts(mode, sc.step_vox, sc.ert, sc.bg, sc.light_color,
                         cone_half_angle_deg=sc.cone_half_angle_deg,
                         shell_radius_vox=sc.shell_radius_vox)
    rng = np.random.default_rng(4)
    traced = 0
    for _ in range(10):
        x, y = int(rng.integers(sc.width)), int(rng.integers(sc.height))
        g = ctx.trace_pixel(sc.camera, sc.width, sc.height, sc.step_vox, x, y, ert=sc.ert)
        o = orc.trace_pixel(sc.volume, sc.tf, sc.vmin, sc.vmax, light, stack, sc.camera,
                            sc.width, sc.height, ro, x, y)
        assert g.shape == o.shape, (x, y, g.shape, o.shape)
        assert np.array_equal(g, o), (x, y, np.argwhere(g != o)[:5])
        traced += len(g)
    assert traced > 100


@pytest.mark.parametrize("fmt", [1, 2, 3])
def test_point_light_storage_formats(ctx, orc, vi_mod, fmt):
    sc = scene(vi_mod.CONE, persp=True, seed=47)
    pos = POSITIONS["far"]
    gpu, _ = gpu_frame(ctx, sc, fmt=fmt, light_pos=pos)
    check_frame(gpu, None, oracle_frame(orc, sc, light_pos=pos), IMAGE_TOL + FORMAT_HALF_ULP[fmt])


def test_point_light_with_every_variant(ctx, orc, vi_mod):
    sc = scene(vi_mod.SHELL, persp=True, seed=53)
    pos = POSITIONS["near"]
    kw = dict(quantity=vi_mod.OPTICAL_DEPTH, shell_count=2, slice_filter=vi_mod.SLICE_LINEAR,
              light_pos=pos)
    gpu, _ = gpu_frame(ctx, sc, fmt=vi_mod.F16, **kw)
    check_frame(gpu, None, oracle_frame(orc, sc, **kw), IMAGE_TOL + FORMAT_HALF_ULP[1] / math.e)


def test_point_light_position_is_validated_and_replaced(ctx, vi_mod):
    sc = scene(vi_mod.CONE, persp=True)
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    for pos in ((0.5, 0.5, 0.5), (0.5, 0.5, 1.45), (float("nan"), 0.0, 3.0)):
        with pytest.raises(vi_mod.ViError) as e:
            ctx.set_point_light(pos)
        assert e.value.code == vi_mod.EINVAL
    # A directional light set after a point light replaces it.
    ctx.set_point_light(POSITIONS["far"])
    ctx.set_light(sc.light_dir)
    ctx.build_attenuation(sc.n_slices, sc.slice_res, vi_mod.CONE)
    a = ctx.render(sc.camera, sc.width, sc.height, sc.step_vox, ert=sc.ert).cpu().numpy()
    with vi_mod.Context(0) as c2:
        c2.load_volume(sc.volume)
        c2.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
        c2.set_light(sc.light_dir)
        c2.build_attenuation(sc.n_slices, sc.slice_res, vi_mod.CONE)
        b = c2.render(sc.camera, sc.width, sc.height, sc.step_vox, ert=sc.ert).cpu().numpy()
    assert np.array_equal(a, b)
