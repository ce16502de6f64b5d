"""The empty-space skipping grid against its definition, by brute force.

Skipping is exact only if no brick or cell that a visible sample can start in
is left unflagged.  The image tests catch a wrong flag only where some tested
ray happens to cross it, and a wrong skip distance that is too small only
costs time, so here the grid the library builds (`vi_get_skip_grid`) is
checked directly on small volumes with ragged sizes:

- a flag must be set when some value in the block's range reaches a TF
  entry with alpha > 0 with positive lerp weight (the block's voxels plus its
  one-voxel apron on the high sides, clamped to the volume; entry j has
  positive weight at TF coordinate x exactly when |x - j| < 1, Section 3.1.1
  classification), and may be set only when such an entry lies within one
  more entry of the range (the margin for the binary32 TF coordinate);
- a cell's skip distance is exactly the L-infinity distance in cells to the
  nearest flagged cell in the grid, capped at 32;
- a flagged cell lies in a flagged brick.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BRICK, CELL, CAP = 16, 8, 32


@pytest.fixture()
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06134_gb300 import build, vi
    build.build()
    c = vi.Context(0)
    yield c
    c.close()


def block_ranges(vol, size, shape):
    """Min and max over each block's voxels and its high-side apron, clamped."""
    nz, ny, nx = vol.shape
    lo = np.empty(shape, np.float64)
    hi = np.empty(shape, np.float64)
    for bz in range(shape[0]):
        zi = np.clip(np.arange(bz * size, bz * size + size + 1), 0, nz - 1)
        for by in range(shape[1]):
            yi = np.clip(np.arange(by * size, by * size + size + 1), 0, ny - 1)
            for bx in range(shape[2]):
                xi = np.clip(np.arange(bx * size, bx * size + size + 1), 0, nx - 1)
                blk = vol[np.ix_(zi, yi, xi)]
                lo[bz, by, bx] = blk.min()
                hi[bz, by, bx] = blk.max()
    return lo, hi


def reach(lo, hi, tf, vmin, vmax):
    """(must, may): whether a lit entry is reachable from [lo, hi] with positive
    weight, and whether one lies within one more entry of it."""
    M = tf.shape[0]
    vmin, vmax = float(np.float32(vmin)), float(np.float32(vmax))
    scale = (M - 1) / (vmax - vmin)
    xl = np.clip((lo - vmin) * scale, 0.0, M - 1.0)
    xh = np.clip((hi - vmin) * scale, 0.0, M - 1.0)
    lit = np.flatnonzero(tf[:, 3] > 0).astype(np.float64)

    def any_in(a, b, closed):
        if closed:
            return np.searchsorted(lit, b, "right") - np.searchsorted(lit, a, "left") > 0
        return np.searchsorted(lit, b, "left") - np.searchsorted(lit, a, "right") > 0

    eps = 1e-3   # keep the binary32 TF coordinate's rounding out of the decision
    must = any_in(xl - 1.0 + eps, xh + 1.0 - eps, closed=False)
    may = any_in(xl - 2.0 - eps, xh + 2.0 + eps, closed=True)
    return must, may


def linf_distance(lit_mask):
    shape = lit_mask.shape
    pts = np.argwhere(lit_mask)
    if len(pts) == 0:
        return np.full(shape, CAP, np.int64)
    allc = np.indices(shape).reshape(3, -1).T
    d = np.abs(allc[:, None, :] - pts[None, :, :]).max(-1).min(1)
    return np.minimum(d, CAP).reshape(shape)


def check_grid(ctx, vol, tf, vmin, vmax, want_both=True):
    flags, skip = ctx.get_skip_grid()
    nz, ny, nx = vol.shape
    nb = tuple(-(-n // BRICK) for n in (nz, ny, nx))
    assert flags.shape == nb
    assert skip.shape == tuple(2 * n for n in nb)
    assert set(np.unique(flags)) <= {0, 1}
    assert skip.max() <= CAP
    for grid, size, lit in ((flags, BRICK, flags == 1), (skip, CELL, skip == 0)):
        lo, hi = block_ranges(vol.astype(np.float64), size, grid.shape)
        must, may = reach(lo, hi, tf, vmin, vmax)
        assert np.all(lit[must]), f"{size}^3 blocks that can be visible are unflagged"
        assert not np.any(lit[~may]), f"{size}^3 blocks flagged beyond the one-entry margin"
        if want_both:   # the case separates the two outcomes
            assert must.any() and (~may).any()
    assert np.array_equal(skip.astype(np.int64), linf_distance(skip == 0))
    cell_lit = (skip == 0).reshape(nb[0], 2, nb[1], 2, nb[2], 2).any(axis=(1, 3, 5))
    assert np.all(flags[cell_lit] == 1)
    return flags, skip


def test_ct_phantom_grid_matches_definition(ctx):
    from paper_2008_06134_gb300 import phantoms as ph
    vol = ph.ct_phantom(72, 31)[:, :61, :53].copy()      # ragged: partial bricks and cells
    tf = ph.tf_ct(4096, 31)
    ctx.load_volume(vol)
    ctx.set_transfer_function(tf, 0.0, 4095.0)
    check_grid(ctx, vol, tf, 0.0, 4095.0)
    # A TF window that is not [0, max]: values below vmin map to entry 0.
    ctx.set_transfer_function(tf, 300.0, 3500.0)
    check_grid(ctx, vol, tf, 300.0, 3500.0)


def test_blob_grid_follows_transfer_function(ctx):
    from paper_2008_06134_gb300 import phantoms as ph
    vol = ph.gaussian_blobs(56, 31)[:41, :50, :56].copy()
    ctx.load_volume(vol)
    for seed in (3, 4, 5):
        tf = ph.tf_random_pl(256, seed)
        ctx.set_transfer_function(tf, 0.0, 255.0)
        check_grid(ctx, vol, tf, 0.0, 255.0, want_both=False)
    # A narrow lit band: both outcomes occur.
    tf = np.zeros((256, 4), np.float32)
    tf[150:160, 3] = 0.05
    ctx.set_transfer_function(tf, 0.0, 255.0)
    check_grid(ctx, vol, tf, 0.0, 255.0)


def test_long_volume_reaches_the_distance_cap(ctx):
    """One small bright block at one end of a 300-voxel-long volume: the far
    cells are more than 32 cells away and read the cap."""
    vol = np.zeros((20, 24, 300), np.uint8)
    vol[5:12, 8:16, 4:12] = 200
    tf = np.zeros((256, 4), np.float32)
    tf[100:, 3] = 0.2
    ctx.load_volume(vol)
    ctx.set_transfer_function(tf, 0.0, 255.0)
    flags, skip = check_grid(ctx, vol, tf, 0.0, 255.0)
    assert skip.max() == CAP and (skip == CAP).sum() > 0
    assert 1 <= (skip == 0).sum() <= 8


def test_all_clear_and_all_lit_transfer_functions(ctx):
    from paper_2008_06134_gb300 import phantoms as ph
    vol = ph.gaussian_blobs(40, 7)[:, :33, :].copy()
    ctx.load_volume(vol)
    clear = np.zeros((64, 4), np.float32)
    ctx.set_transfer_function(clear, 0.0, 255.0)
    flags, skip = check_grid(ctx, vol, clear, 0.0, 255.0, want_both=False)
    assert not flags.any() and np.all(skip == CAP)
    lit = np.full((64, 4), 0.1, np.float32)
    ctx.set_transfer_function(lit, 0.0, 255.0)
    flags, skip = check_grid(ctx, vol, lit, 0.0, 255.0, want_both=False)
    assert flags.all() and not skip.any()


def test_skip_grid_needs_volume_and_transfer_function(ctx):
    from paper_2008_06134_gb300 import vi
    with pytest.raises(vi.ViError) as e:
        ctx.get_skip_grid()
    assert e.value.code == vi.ESTATE
    ctx.load_volume(np.zeros((8, 8, 8), np.uint8))
    with pytest.raises(vi.ViError) as e:
        ctx.get_skip_grid()
    assert e.value.code == vi.ESTATE
