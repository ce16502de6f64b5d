"""The lockstep sweep against the FP64 oracle, texel by texel.

The sweep takes its lockstep kernel (a warp's 32 columns step through the
slices together, with warp-wide transparent runs over the skip-distance boxes)
for stacks of 2^29 texel-slices and more; at such sizes the full-size tests
can compare only sampled texels.  Here the library's threshold is lowered
through its environment variable, so the same kernel sweeps stacks small
enough for the oracle to check every texel, with ragged sizes, empty space
around the volume, both voxel types, every storage format and both stored
quantities, and the frames rendered from them.
"""
import numpy as np
import pytest

from gpu_common import FORMAT_HALF_ULP, STACK_TOL, check_frame, gpu_frame, oracle_frame

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx(monkeypatch):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, vi
    build.build()
    monkeypatch.setenv("VI_SWEEP_LOCKSTEP_MIN", "1")   # every stack in lockstep
    c = vi.Context(0)
    yield c
    c.close()


def scene(case):
    from paper_2008_06134_gb300 import phantoms as ph
    rng = np.random.default_rng(31)
    if case == "ct-cone":
        sc = ph.ct256_cone()
        sc.volume = ph.ct_phantom(72, 31)          # empty space around an ellipsoid
        sc.tf = ph.tf_ct(4096, 31)
        sc.n_slices, sc.slice_res, sc.width, sc.height = 61, 83, 57, 45
    else:
        sc = ph.blob64_shell(31)
        sc.volume = ph.gaussian_blobs(56, 31)[:41, :50, :56].copy()
        sc.n_slices, sc.slice_res, sc.width, sc.height = 53, 70, 49, 38
        sc.mode = 2
    sc.light_dir = ph.random_direction(rng)
    sc.camera = ph.orbit_camera(ph.random_direction(rng), True, 2.4)
    return sc


@pytest.mark.parametrize("case,fmt", [("ct-cone", 0), ("ct-cone", 1), ("blob-shell", 0),
                                      ("blob-shell", 3)])
def test_lockstep_stack_and_frame_match_oracle(ctx, orc, case, fmt):
    from paper_2008_06134_gb300 import vi
    sc = scene(case)
    gpu, counts = gpu_frame(ctx, sc, fmt=fmt, counts=True)
    B = vi.decode_stack(ctx.get_attenuation(), fmt)
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    ref = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
    assert B.shape == ref.shape
    assert np.abs(B - ref).max() <= STACK_TOL + FORMAT_HALF_ULP[fmt]
    assert ref.min() < 0.5                     # the light is really attenuated
    ora = oracle_frame(orc, sc, stack=ref)
    check_frame(gpu, counts, ora, 1e-4 + FORMAT_HALF_ULP[fmt])


def test_lockstep_optical_depth_matches_oracle(ctx, orc):
    """The extinction form (Eq. 5-6) through the same kernel: the stored optical
    depth D_k against the oracle's, as the light it stands for and, where that
    light is not negligible, as a depth."""
    from paper_2008_06134_gb300 import vi
    sc = scene("ct-cone")
    gpu_frame(ctx, sc, quantity=vi.OPTICAL_DEPTH)
    D = ctx.get_attenuation().astype(np.float64)
    light = orc.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    ref = orc.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light, quantity=orc.OPTICAL_DEPTH)
    assert D.shape == ref.shape
    assert np.abs(np.exp(-D) - np.exp(-ref)).max() <= STACK_TOL
    live = ref < 30.0
    assert (np.abs(D - ref)[live] / np.maximum(1.0, ref[live])).max() <= 2e-5
    assert ref.max() > 1.0


def test_lockstep_and_per_lane_stacks_agree(orc, monkeypatch):
    """The two sweep kernels give the same stack bit for bit (the same per
    slice arithmetic in the same order; only the schedule differs)."""
    import torch
    from paper_2008_06134_gb300 import build, vi
    build.build()
    sc = scene("ct-cone")
    stacks = []
    for threshold in ("1", str(1 << 40)):
        monkeypatch.setenv("VI_SWEEP_LOCKSTEP_MIN", threshold)
        with vi.Context(0) as c:
            gpu_frame(c, sc)
            stacks.append(c.get_attenuation())
    torch.cuda.synchronize()
    assert np.array_equal(stacks[0], stacks[1])
