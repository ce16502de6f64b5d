"""The checked build (libvi_checked.so, compiled with VI_DEBUG_BOUNDS=1): every
sweep, march and grid kernel tests each voxel, brick, TF, stack, output and
raw-voxel index before the access and counts a bad one instead of making it.

The parity scenes, the degenerate cases, the method variants, the point light,
ragged and one-pixel images, the full-size benchmark frame, a stack large
enough for the lockstep sweep, traces and the render server all run through it
with no violation, and give the release library's frames (the checks change
no arithmetic: integer results equal, images within 1e-6)."""
import numpy as np
import pytest

from gpu_common import gpu_frame

pytestmark = pytest.mark.gpu

SAME_TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    vi.debug_bounds(0)  # start from a clear record
    checked = vi.Context(0, checked=True)
    release = vi.Context(0)
    yield torch, ph, vi, checked, release
    checked.close()
    release.close()


def small_scene(ph, **kw):
    sc = ph.blob64_shell()
    sc.volume = ph.gaussian_blobs(24, 3)
    sc.n_slices, sc.slice_res, sc.width, sc.height = 19, 21, 29, 23
    for k, v in kw.items():
        setattr(sc, k, v)
    return sc


def assert_clean_and_same(env, sc, **kw):
    torch, ph, vi, checked, release = env
    got, got_n = gpu_frame(checked, sc, counts=True, **kw)
    n, site, idx = vi.debug_bounds(0)
    assert n == 0, f"{n} bounds violations, first at site {site}, index {idx}"
    ref, ref_n = gpu_frame(release, sc, counts=True, **kw)
    assert np.array_equal(got_n, ref_n)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= SAME_TOL


CASES = ["shell", "cone-f16", "shadow-bf16", "cone-unorm16", "ct-perspective", "non-cubic",
         "one-slice", "one-texel", "one-voxel", "two-entry-tf", "axis-light",
         "view-parallel-light", "eye-inside", "grazing-ortho", "wide-shell", "one-pixel",
         "ragged-image", "optical-depth", "linear-slices", "four-shells",
         "opacity-correction", "compensation", "point-light-cone", "point-light-shell"]


@pytest.mark.parametrize("case", CASES)
def test_checked_kernels_make_no_bad_access(env, case):
    torch, ph, vi, checked, release = env
    sc = small_scene(ph, mode=vi.CONE)
    kw = {}
    if case == "shell":
        sc.mode = vi.SHELL
    elif case == "cone-f16":
        kw["fmt"] = vi.F16
    elif case == "shadow-bf16":
        sc.mode, kw["fmt"] = vi.SHADOW, vi.BF16
    elif case == "cone-unorm16":
        kw["fmt"] = vi.UNORM16
    elif case == "ct-perspective":
        ct = ph.ct256_cone(n=48)
        ct.n_slices, ct.slice_res, ct.width, ct.height = 40, 48, 64, 48
        sc = ct
    elif case == "non-cubic":
        sc.volume = ph.gaussian_blobs(40, 13)[:28, :36, :40].copy()
    elif case == "one-slice":
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
        sc.width, sc.height = 32, 32
    elif case == "wide-shell":
        sc.mode, sc.shell_radius_vox = vi.SHELL, 3.5
    elif case == "one-pixel":
        sc.width = sc.height = 1
    elif case == "ragged-image":
        sc.width, sc.height = 57, 31
    elif case == "optical-depth":
        kw.update(quantity=vi.OPTICAL_DEPTH, fmt=vi.F16)
    elif case == "linear-slices":
        kw["slice_filter"] = vi.SLICE_LINEAR
    elif case == "four-shells":
        sc.mode, kw["shell_count"] = vi.SHELL, 4
    elif case == "opacity-correction":
        kw.update(opacity_correction=1, build_oc=1)
    elif case == "compensation":
        kw["comp_n"] = 2.0
    elif case == "point-light-cone":
        kw["light_pos"] = (0.5, 0.5, 1.7)
    elif case == "point-light-shell":
        sc.mode, kw["light_pos"] = vi.SHELL, (1.4, -0.3, 0.6)
    assert_clean_and_same(env, sc, **kw)


def test_checked_full_size_frame(env):
    """The benchmark frame (256^3 u16, 256 x 512^2 FP32 stack over several
    stack textures, cone, 1024^2 perspective, ERT 0.99)."""
    torch, ph, vi, checked, release = env
    assert_clean_and_same(env, ph.ct256_cone())


def test_checked_lockstep_sweep(env):
    """1024 slices of 1024^2 (2^30 texel-slices, FP16): the sweep's lockstep
    mode and a stack over many textures."""
    torch, ph, vi, checked, release = env
    sc = small_scene(ph, mode=vi.SHADOW)
    sc.volume = ph.gaussian_blobs(64, 5)
    sc.n_slices, sc.slice_res, sc.width, sc.height = 1024, 1024, 64, 48
    assert_clean_and_same(env, sc, fmt=vi.F16)


def test_checked_traces(env):
    """Per-sample traces of a few pixels are the same through both libraries."""
    torch, ph, vi, checked, release = env
    sc = small_scene(ph, mode=vi.CONE)
    recs = []
    for ctx in (checked, release):
        gpu_frame(ctx, sc)
        recs.append([ctx.trace_pixel(sc.camera, sc.width, sc.height, sc.step_vox, x, y)
                     for x, y in ((14, 11), (0, 0), (28, 22), (7, 19))])
    assert vi.debug_bounds(0)[0] == 0
    for a, b in zip(*recs):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_checked_server_with_graphs(env):
    """Served frames through the checked library, launched as CUDA graphs."""
    torch, ph, vi, checked, release = env
    vol = ph.ct_phantom(48, 12)
    tf = ph.tf_ct(512, 12)
    outs = {}
    for lib_checked in (True, False):
        frames = []
        with vi.Server(0, slots=3, graphs=True, checked=lib_checked) as s:
            vid = s.add_volume(vol)
            tickets = []
            for q in range(8):
                cam = ph.orbit_camera(ph.random_direction(np.random.default_rng(q)), True, 2.4)
                out = torch.full((40, 48, 4), float("nan"), device="cuda")
                tickets.append(s.submit(vid, tf, 0.0, 4095.0, (0.3, -0.2, 0.9), 24, 40,
                                        [vi.SHADOW, vi.SHELL, vi.CONE][q % 3], cam, 48, 40,
                                        0.5, out, format=[vi.F32, vi.F16][q % 2], ert=0.95))
                frames.append(out)
            for t in tickets:
                assert s.wait(t) == (vi.REQ_DONE, vi.OK)
        torch.cuda.synchronize()
        outs[lib_checked] = [f.cpu().numpy() for f in frames]
        if lib_checked:
            assert vi.debug_bounds(0)[0] == 0
    for a, b in zip(outs[True], outs[False]):
        assert np.abs(a - b).max() <= SAME_TOL
