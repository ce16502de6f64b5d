"""Parity of the variant options with the FP64 oracle, through the C ABI:
the optical-depth stack (the extinction form of Eq. 5-6), linear filtering
between slices, several shells (Section 3.2.3), alone and together.

Tolerances follow the same arithmetic as the base path: 1e-4 per RGBA channel
for FP32; a 16-bit optical depth D adds at most exp(-D) D half-ulp(1) <=
half-ulp(1) / e to a light factor, which bounds the image error too (the
coefficient is a convex combination of light factors, the compositing weights
sum to at most 1)."""
import math

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


@pytest.fixture(scope="module")
def vi_mod():
    from paper_2008_06134_gb300 import vi
    return vi


def blob_scene(mode):
    from paper_2008_06134_gb300 import phantoms as ph
    sc = ph.blob64_shell(ert=0.98)
    sc.mode = mode
    return sc


def ragged_scene(mode, persp, seed=17):
    """Non-cubic volume, ragged image and light resolutions, odd slice count."""
    from paper_2008_06134_gb300 import phantoms as ph
    rng = np.random.default_rng(seed)
    sc = ph.blob64_shell(seed)
    sc.volume = ph.gaussian_blobs(48, seed)[:29, :35, :42].copy()
    sc.tf[:, 3] *= 3.0                     # denser: deep shadows, optical depths up to ~10
    sc.n_slices, sc.slice_res = 41, 37
    sc.width, sc.height = 61, 43
    sc.mode = mode
    sc.light_dir = ph.random_direction(rng)
    sc.camera = ph.orbit_camera(ph.random_direction(rng), persp, 2.4 if persp else 2.0)
    sc.step_vox = 0.41
    return sc


@pytest.mark.parametrize("which", ["blob64", "ragged"])
def test_depth_stack_matches_oracle(ctx, orc, vi_mod, which):
    sc = blob_scene(vi_mod.SHADOW) if which == "blob64" else ragged_scene(vi_mod.SHADOW, True)
    gpu_frame(ctx, sc, quantity=vi_mod.OPTICAL_DEPTH)
    D = ctx.get_attenuation().astype(np.float64)
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    ref = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light, quantity=orc.OPTICAL_DEPTH)
    assert D.shape == ref.shape
    assert D[0].max() == 0.0 and D.min() >= 0.0
    # The light it stands for, and the depth itself where the light is not negligible.
    assert np.abs(np.exp(-D) - np.exp(-ref)).max() <= STACK_TOL
    live = ref < 30.0
    rel = np.abs(D - ref)[live] / np.maximum(1.0, ref[live])
    assert rel.max() <= 2e-5
    assert ref.max() > 1.0                     # the scene really attenuates


@pytest.mark.parametrize("fmt", [0, 1, 2])
@pytest.mark.parametrize("mode", [1, 2, 3])
def test_depth_frames_match_oracle(ctx, orc, vi_mod, mode, fmt):
    sc = ragged_scene(mode, persp=mode != 2)
    gpu, counts = gpu_frame(ctx, sc, fmt=fmt, counts=True, quantity=vi_mod.OPTICAL_DEPTH)
    check_frame(gpu, counts, oracle_frame(orc, sc, quantity=orc.OPTICAL_DEPTH),
                IMAGE_TOL + FORMAT_HALF_ULP[fmt] / math.e)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_linear_slice_filter_matches_oracle(ctx, orc, vi_mod, mode):
    sc = ragged_scene(mode, persp=True, seed=23)
    gpu, counts = gpu_frame(ctx, sc, counts=True, slice_filter=vi_mod.SLICE_LINEAR)
    ora = oracle_frame(orc, sc, slice_filter=orc.SLICE_LINEAR)
    check_frame(gpu, counts, ora)
    ref = ora[0]
    # It is a different image from the nearest-slice one.
    near, *_ = oracle_frame(orc, sc)
    assert np.abs(near - ref).max() > 10 * IMAGE_TOL


@pytest.mark.parametrize("shells", [2, 4])
def test_several_shells_match_oracle(ctx, orc, vi_mod, shells):
    sc = blob_scene(vi_mod.SHELL)
    sc.shell_radius_vox = 1.5
    gpu, counts = gpu_frame(ctx, sc, counts=True, shell_count=shells)
    check_frame(gpu, counts, oracle_frame(orc, sc, shell_count=shells))


def test_all_variants_together(ctx, orc, vi_mod):
    sc = ragged_scene(vi_mod.SHELL, persp=True, seed=29)
    gpu, _ = gpu_frame(ctx, sc, fmt=vi_mod.F16, quantity=vi_mod.OPTICAL_DEPTH, shell_count=3,
                       slice_filter=vi_mod.SLICE_LINEAR)
    check_frame(gpu, None, oracle_frame(orc, sc, quantity=orc.OPTICAL_DEPTH, shell_count=3,
                                        slice_filter=orc.SLICE_LINEAR),
                IMAGE_TOL + FORMAT_HALF_ULP[1] / math.e)


@pytest.mark.parametrize("mode,shells", [(1, 1), (2, 3), (3, 1)])
def test_variant_traces_are_bit_exact(ctx, orc, vi_mod, mode, shells):
    """Linear slice filtering and several shells: every integer decision (the
    lower slice of each lookup, texel cells) and binary32 position agrees."""
    sc = ragged_scene(mode, persp=True, seed=31)
    gpu_frame(ctx, sc, shell_count=shells, slice_filter=vi_mod.SLICE_LINEAR,
              quantity=vi_mod.OPTICAL_DEPTH)
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    stack = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light, quantity=orc.OPTICAL_DEPTH)
    ro = orc.render_opts(mode, sc.step_vox, sc.ert, sc.bg, sc.light_color,
                         cone_half_angle_deg=sc.cone_half_angle_deg,
                         shell_radius_vox=sc.shell_radius_vox, quantity=orc.OPTICAL_DEPTH,
                         slice_filter=orc.SLICE_LINEAR, shell_count=shells)
    rng = np.random.default_rng(3)
    traced = 0
    for _ in range(10):
        x, y = int(rng.integers(sc.width)), int(rng.integers(sc.height))
        g = ctx.trace_pixel(sc.camera, sc.width, sc.height, sc.step_vox, x, y, ert=sc.ert,
                            slice_filter=vi_mod.SLICE_LINEAR)
        o = orc.trace_pixel(sc.volume, sc.tf, sc.vmin, sc.vmax, light, stack, sc.camera,
                            sc.width, sc.height, ro, x, y)
        assert g.shape == o.shape, (x, y, g.shape, o.shape)
        assert np.array_equal(g, o), (x, y, np.argwhere(g != o)[:5])
        traced += len(g)
    assert traced > 100


def test_variant_options_are_validated(ctx, vi_mod):
    sc = blob_scene(vi_mod.SHELL)
    gpu_frame(ctx, sc)
    for kw in (dict(quantity=2), dict(quantity=vi_mod.OPTICAL_DEPTH, format=vi_mod.UNORM16),
               dict(shell_count=5), dict(shell_count=-1)):
        with pytest.raises(vi_mod.ViError) as e:
            ctx.build_attenuation(sc.n_slices, sc.slice_res, vi_mod.SHELL, **kw)
        assert e.value.code == vi_mod.EINVAL
    ctx.build_attenuation(sc.n_slices, sc.slice_res, vi_mod.SHELL)
    with pytest.raises(vi_mod.ViError) as e:
        ctx.render(sc.camera, 8, 8, 0.5, slice_filter=2)
    assert e.value.code == vi_mod.EINVAL


def test_server_serves_variants_like_a_context(ctx, vi_mod):
    import torch
    sc = ragged_scene(vi_mod.CONE, persp=True, seed=37)
    opts = dict(quantity=vi_mod.OPTICAL_DEPTH, format=vi_mod.F16)
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir)
    ctx.build_attenuation(sc.n_slices, sc.slice_res, vi_mod.CONE, **opts)
    want = ctx.render(sc.camera, sc.width, sc.height, sc.step_vox, ert=sc.ert,
                      slice_filter=vi_mod.SLICE_LINEAR).cpu().numpy()
    with vi_mod.Server(0, slots=2) as s:
        vid = s.add_volume(sc.volume)
        out = torch.empty((sc.height, sc.width, 4), device="cuda")
        t = s.submit(vid, sc.tf, sc.vmin, sc.vmax, sc.light_dir, sc.n_slices, sc.slice_res,
                     vi_mod.CONE, sc.camera, sc.width, sc.height, sc.step_vox, out, ert=sc.ert,
                     slice_filter=vi_mod.SLICE_LINEAR, **opts)
        assert s.wait(t) == (vi_mod.REQ_DONE, vi_mod.OK)
        bad = torch.empty((8, 8, 4), device="cuda")
        with pytest.raises(vi_mod.ViError):
            s.submit(vid, sc.tf, sc.vmin, sc.vmax, sc.light_dir, 8, 8, vi_mod.CONE, sc.camera,
                     8, 8, 0.5, bad, quantity=vi_mod.OPTICAL_DEPTH, format=vi_mod.UNORM16)
    assert np.array_equal(out.cpu().numpy(), want)
