"""The skipping-grid checks of test_gpu_skip_grid.py, run on the CPU against a
numpy stand-in for the library's grid.

The stand-in builds the grid from its documented definition: per 16^3 brick
and 8^3 cell, the value range over its voxels and the one-voxel apron on the
high sides (clamped to the volume); a flag when the TF entries within one
entry of the range's FP64 TF coordinates hold an alpha > 0; the cells' skip
distances as the capped L-infinity distance transform of the cell flags, in
three separable passes.  The GPU test's checks must accept it, and must
reject it once a plausible mistake is planted: the apron left out of the
cells, the x and z axes of the cell grid swapped, the z pass of the distance
transform left out.  So each of those mistakes in the CUDA grid would fail
the GPU test.
"""
import numpy as np
import pytest

import test_gpu_skip_grid as checks

GPU_CASES = ("test_ct_phantom_grid_matches_definition", "test_blob_grid_follows_transfer_function",
             "test_long_volume_reaches_the_distance_cap",
             "test_all_clear_and_all_lit_transfer_functions")


def ranges(vol, size, shape, apron=1):
    nz, ny, nx = vol.shape
    lo = np.empty(shape)
    hi = np.empty(shape)
    for bz in range(shape[0]):
        zi = np.clip(np.arange(bz * size, bz * size + size + apron), 0, nz - 1)
        for by in range(shape[1]):
            yi = np.clip(np.arange(by * size, by * size + size + apron), 0, ny - 1)
            for bx in range(shape[2]):
                xi = np.clip(np.arange(bx * size, bx * size + size + apron), 0, nx - 1)
                blk = vol[np.ix_(zi, yi, xi)]
                lo[bz, by, bx], hi[bz, by, bx] = blk.min(), blk.max()
    return lo, hi


def flags_of(lo, hi, tf, vmin, vmax):
    """Lit entries within one entry of the range's TF coordinates [x_lo, x_hi]:
    entries floor(x_lo) - 1 .. floor(x_hi) + 2, clamped to the table."""
    M = tf.shape[0]
    vmin, vmax = float(np.float32(vmin)), float(np.float32(vmax))
    scale = (M - 1) / (vmax - vmin)
    lit = np.concatenate([[0], np.cumsum(tf[:, 3] > 0)])
    e_lo = np.clip(np.floor((lo - vmin) * scale).astype(np.int64) - 1, 0, M - 2)
    e_hi = np.clip(np.floor((hi - vmin) * scale).astype(np.int64) + 2, 1, M - 1)
    return (lit[e_hi + 1] - lit[e_lo] > 0).astype(np.uint8)


def distance_passes(lit, axes=(2, 1, 0)):
    cur = np.where(lit, 0, checks.CAP).astype(np.int64)
    for ax in axes:
        n = cur.shape[ax]
        out = np.full_like(cur, checks.CAP)
        for d in range(-(checks.CAP - 1), checks.CAP):
            if abs(d) >= n:
                continue
            shifted = np.full_like(cur, 1 << 20)
            src, dst = [slice(None)] * 3, [slice(None)] * 3
            src[ax], dst[ax] = (slice(d, n), slice(0, n - d)) if d >= 0 else \
                (slice(0, n + d), slice(-d, n))
            shifted[tuple(dst)] = cur[tuple(src)]
            out = np.minimum(out, np.maximum(abs(d), shifted))
        cur = out
    return cur.astype(np.uint8)


class GridStandIn:
    """The three context calls the GPU test makes, on the host."""
    mistake = None

    def load_volume(self, vol):
        self.vol = vol

    def set_transfer_function(self, tf, vmin, vmax):
        self.tf, self.vmin, self.vmax = tf, vmin, vmax

    def get_skip_grid(self):
        vol = self.vol.astype(np.float64)
        nb = tuple(-(-n // checks.BRICK) for n in vol.shape)
        nc = tuple(2 * n for n in nb)
        flags = flags_of(*ranges(vol, checks.BRICK, nb), self.tf, self.vmin, self.vmax)
        apron = 0 if self.mistake == "cells-without-apron" else 1
        cell = flags_of(*ranges(vol, checks.CELL, nc, apron), self.tf, self.vmin, self.vmax)
        axes = (2, 1) if self.mistake == "no-z-pass" else (2, 1, 0)
        skip = distance_passes(cell == 1, axes)
        if self.mistake == "cell-axes-swapped":
            skip = np.ascontiguousarray(skip.transpose(2, 1, 0)).reshape(skip.shape)
        return flags, skip


def run_cases(mistake):
    failed = []
    for name in GPU_CASES:
        ctx = GridStandIn()
        ctx.mistake = mistake
        try:
            getattr(checks, name)(ctx)
        except AssertionError:
            failed.append(name)
    return failed


def test_checks_accept_the_grid_of_the_definition():
    assert run_cases(None) == []


@pytest.mark.parametrize("mistake", ["cells-without-apron", "cell-axes-swapped", "no-z-pass"])
def test_checks_reject_a_planted_mistake(mistake):
    assert run_cases(mistake), f"no GPU skip-grid check fails with {mistake}"
