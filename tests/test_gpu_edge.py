"""Edge cases and error paths of the C ABI on the GPU, each checked against the
oracle where there is a result to check."""
import numpy as np
import pytest

from gpu_common import IMAGE_TOL, check_frame, gpu_frame, oracle_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, vi
    build.build()
    return vi


@pytest.fixture()
def ctx(vi):
    c = vi.Context(0)
    yield c
    c.close()


def small_scene(**kw):
    from paper_2008_06134_gb300 import phantoms as ph
    sc = ph.blob64_shell()
    sc.volume = ph.gaussian_blobs(24, 3)
    sc.n_slices, sc.slice_res, sc.width, sc.height = 19, 21, 29, 23
    for k, v in kw.items():
        setattr(sc, k, v)
    return sc


def check_against_oracle(ctx, orc, sc, **kw):
    gpu, counts = gpu_frame(ctx, sc, counts=True, **kw)
    ora = oracle_frame(orc, sc, **kw)
    check_frame(gpu, counts, ora)
    return gpu, ora[0]


def test_render_needs_inputs_and_fresh_stack(ctx, vi):
    sc = small_scene()
    cam = sc.camera
    with pytest.raises(vi.ViError) as e:
        ctx.render(cam, 8, 8, 0.5)
    assert e.value.code == vi.ESTATE
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    with pytest.raises(vi.ViError) as e:
        ctx.build_attenuation(8, 8, vi.SHADOW)   # no light yet
    assert e.value.code == vi.ESTATE
    ctx.build_attenuation(8, 8, vi.NONE)        # NONE needs no light
    ctx.render(cam, 8, 8, 0.5)
    ctx.set_light((0, 0, 1))
    ctx.build_attenuation(8, 8, vi.SHADOW)
    ctx.render(cam, 8, 8, 0.5)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)   # stack goes stale
    with pytest.raises(vi.ViError) as e:
        ctx.render(cam, 8, 8, 0.5)
    assert e.value.code == vi.ESTATE
    ctx.build_attenuation(8, 8, vi.SHADOW)
    ctx.set_light((1, 0, 0))
    with pytest.raises(vi.ViError) as e:
        ctx.render(cam, 8, 8, 0.5)
    assert e.value.code == vi.ESTATE
    ctx.build_attenuation(8, 8, vi.SHADOW)
    ctx.load_volume(sc.volume)
    with pytest.raises(vi.ViError) as e:
        ctx.render(cam, 8, 8, 0.5)
    assert e.value.code == vi.ESTATE
    ctx.sync()


def test_invalid_arguments(ctx, vi):
    sc = small_scene()
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light((0.2, 0.3, 0.9))
    bad = [
        lambda: ctx.set_light((0, 0, 0)),
        lambda: ctx.set_light((np.nan, 0, 1)),
        lambda: ctx.set_transfer_function(sc.tf[:1], 0, 1),
        lambda: ctx.set_transfer_function(sc.tf, 5, 5),
        lambda: ctx.set_transfer_function(np.full((4, 4), 2.0, np.float32), 0, 1),
        lambda: ctx.build_attenuation(0, 8, vi.SHADOW),
        lambda: ctx.build_attenuation(8, 0, vi.SHADOW),
        lambda: ctx.build_attenuation(8, 8, 7),
        lambda: ctx.build_attenuation(8, 8, vi.SHADOW, format=9),
        lambda: ctx.build_attenuation(8, 8, vi.CONE, cone_half_angle_deg=90),
        lambda: ctx.build_attenuation(8, 8, vi.SHELL, shell_radius_vox=0),
        lambda: ctx.build_attenuation(1 << 20, 1 << 14, vi.SHADOW),
    ]
    for f in bad:
        with pytest.raises(vi.ViError) as e:
            f()
        assert e.value.code == vi.EINVAL
    ctx.build_attenuation(8, 8, vi.SHADOW)
    good = ((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), 1, 40.0, 0.5)
    for cam, W, H, step in [
        (((0.5, 0.5, 0.5), (0.5, 0.5, 0.5), (0, 1, 0), 1, 40.0, 0.5), 4, 4, 0.5),  # eye == target
        (((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 0, 1), 1, 40.0, 0.5), 4, 4, 0.5),  # up || view
        (((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), 1, 0.0, 0.5), 4, 4, 0.5),   # fovy 0
        (((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), 0, 40.0, -1.0), 4, 4, 0.5), # ortho < 0
        (good, -1, 4, 0.5), (good, 4, 4, 0.0), (good, 4, 4, float("nan")),
    ]:
        buf = np.empty((4, 4, 4), np.float32)   # host buffer: the C ABI checks W, H itself
        with pytest.raises(vi.ViError) as e:
            ctx.render(cam, W, H, step, out=buf)
        assert e.value.code == vi.EINVAL
    import torch
    empty = torch.empty((0, 5, 4), device="cuda")
    ctx.render(good, 5, 0, 0.5, out=empty)   # W or H == 0: nothing to do
    ctx.sync()


def test_memory_budget_refusal_keeps_previous_state(ctx, vi):
    sc = small_scene()
    ctx.load_volume(sc.volume)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir)
    ctx.build_attenuation(8, 16, vi.SHADOW)
    a = ctx.render(sc.camera, 16, 16, 0.5).cpu().numpy()
    ctx.set_memory_budget(sc.volume.nbytes + 256 * 16 + 8 * 16 * 16 * 4 + 16 * 16 * 16 + 4096)
    with pytest.raises(vi.ViError) as e:
        ctx.build_attenuation(512, 512, vi.SHADOW)
    assert e.value.code == vi.ENOMEM
    b = ctx.render(sc.camera, 16, 16, 0.5).cpu().numpy()
    assert np.array_equal(a, b)
    ctx.set_memory_budget(0)
    ctx.build_attenuation(64, 64, vi.SHADOW)
    ctx.sync()


def test_host_and_device_buffers_agree(ctx, vi, orc):
    import torch
    sc = small_scene(mode=3)
    dev, _ = gpu_frame(ctx, sc)
    host = np.empty((sc.height, sc.width, 4), np.float32)
    ctx.render(sc.camera, sc.width, sc.height, sc.step_vox, out=host)
    assert np.array_equal(host.astype(np.float64), dev)
    ctx.load_volume(torch.from_numpy(sc.volume).cuda())   # device-pointer volume
    ctx.build_attenuation(sc.n_slices, sc.slice_res, 3)
    again = ctx.render(sc.camera, sc.width, sc.height, sc.step_vox).cpu().numpy()
    assert np.array_equal(again.astype(np.float64), dev)
    before = ctx.launch_count()
    ctx.build_attenuation(sc.n_slices, sc.slice_res, 3)
    ctx.render(sc.camera, sc.width, sc.height, sc.step_vox)
    assert ctx.launch_count() == before + 2
    # VI_OUT_HOST_ASYNC: the copy is enqueued on the context's stream and the
    # frame is complete at vi_sync, into page-locked and pageable memory alike.
    for pinned in (True, False):
        buf = torch.full((sc.height, sc.width, 4), float("nan"), pin_memory=pinned)
        ctx.render(sc.camera, sc.width, sc.height, sc.step_vox, out=buf, host_async=True)
        ctx.sync()
        assert np.array_equal(buf.numpy().astype(np.float64), dev)
    assert vi.library().vi_render(ctx.h, None, 1, 1, 0.5, None, 3, None) == vi.EINVAL


@pytest.mark.parametrize("case", ["one-slice", "one-texel", "one-voxel", "two-entry-tf",
                                  "axis-light", "view-parallel-light", "eye-inside",
                                  "grazing-ortho", "wide-shell", "edge-shell", "edge-cone"])
def test_degenerate_cases_match_oracle(ctx, orc, case):
    from paper_2008_06134_gb300 import phantoms as ph
    sc = small_scene(mode=3)
    if case == "one-slice":
        sc.n_slices = 1
    elif case == "one-texel":
        sc.slice_res = 1
    elif case == "one-voxel":
        sc.volume = np.full((1, 1, 1), 180, np.uint8)
    elif case == "two-entry-tf":
        sc.tf = np.array([[0.1, 0.2, 0.3, 0.0], [0.9, 0.8, 0.7, 0.2]], np.float32)
    elif case == "axis-light":
        sc.light_dir = np.array([0, -1, 0], np.float32)
    elif case == "view-parallel-light":
        sc.light_dir = np.array([0, 0, -1], np.float32)
        sc.camera = ph.Camera((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), True, 35.0)
    elif case == "eye-inside":
        sc.camera = ph.Camera((0.45, 0.5, 0.55), (0.9, 0.7, 0.5), (0, 0, 1), True, 70.0)
    elif case == "grazing-ortho":
        sc.camera = ph.Camera((0.5, -1.0, 0.5), (0.5, 0.5, 0.5), (0, 0, 1), False, 40.0, 0.5)
        sc.width, sc.height = 32, 32   # pixel centres land on cube faces
    elif case == "wide-shell":
        sc.mode = 2
        sc.shell_radius_vox = 3.5
    elif case in ("edge-shell", "edge-cone"):
        # Lookup points that reach past the slice's texels for samples near the
        # volume's silhouette (their coordinates must be clamped) and stay
        # inside for samples near its centre (the clamps are skipped): both
        # lookup paths of the shell and cone kernels in one frame.
        if case == "edge-shell":
            sc.mode = 2
            sc.shell_radius_vox = 8.0
        else:
            sc.n_slices = 6
            sc.cone_half_angle_deg = 30.0
        sc.volume = np.full((24, 24, 24), 120, np.uint8)
    check_against_oracle(ctx, orc, sc)


def test_skip_flags_follow_tf_changes_and_clamped_values(ctx, orc):
    """Empty-space skipping must never drop a sample that has alpha > 0: the TF
    here is zero except at its two end entries, which only values clamped
    below vmin / above vmax reach; then the TF changes without reloading the
    volume."""
    sc = small_scene(mode=1)
    M = 64
    tf = np.zeros((M, 4), np.float32)
    tf[:, :3] = (0.9, 0.5, 0.2)
    tf[0, 3] = 0.3
    tf[-1, 3] = 0.05
    sc.tf, sc.vmin, sc.vmax = tf, 60.0, 140.0   # blob values run 0..~220
    check_against_oracle(ctx, orc, sc)
    tf2 = np.zeros((M, 4), np.float32)
    tf2[:, :3] = 1.0
    tf2[30:34, 3] = 0.4                          # a narrow band in the middle
    sc.tf = tf2
    check_against_oracle(ctx, orc, sc)
    sc.mode = 3
    check_against_oracle(ctx, orc, sc)
