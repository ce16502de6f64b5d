"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: a
closed form, an invariant, a library routine (numpy.interp), the paper's own
formula written in a different form (Eq. 2's product form, Eq. 11's Rodrigues
rotation), or an exact brute-force integral (Eq. 1).  They are chosen so that a
dropped term, a wrong sign, a wrong index or a transposed operand in any stage
of the oracle fails at least one of them.  No GPU is needed.
"""
import math

import numpy as np
import pytest

H_SQRT3 = math.sqrt(3.0) / 2.0


def step_tf(M=256, ranges=()):
    """TF with constant RGBA over entry ranges [lo, hi) and zero elsewhere."""
    tf = np.zeros((M, 4), dtype=np.float32)
    for lo, hi, rgba in ranges:
        tf[lo:hi] = rgba
    return tf


def f32(x):
    """The binary32 value a TF entry actually stores."""
    return float(np.float32(x))


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def cam(eye, target, up, persp=False, fovy=40.0, hh=0.5):
    return (tuple(eye), tuple(target), tuple(up), int(persp), float(fovy), float(hh))


# --------------------------------------------------------------------------
# Eq. 8 and the light frame (Eq. 10's light view).

@pytest.mark.parametrize("d", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0, -1, 0), (1, 1, 1),
                               (-1, 2, -3), (0.3, -0.5, 0.81), (-1e-3, 1, 0)])
def test_eq8_min_max_closed_form(orc, d):
    lt = orc.light_setup(d, 16, 8)
    L = unit(d)
    verts = np.array([[(c >> a) & 1 for a in range(3)] for c in range(8)], dtype=np.float64)
    dots = verts @ L
    # Eq. 8 as printed (vertex extremes) and its closed form sum(min(0, L_a)).
    assert lt.min == pytest.approx(dots.min(), abs=1e-6)
    assert lt.max == pytest.approx(dots.max(), abs=1e-6)
    assert lt.min == pytest.approx(np.minimum(L, 0).sum(), abs=1e-6)
    assert lt.max == pytest.approx(np.maximum(L, 0).sum(), abs=1e-6)
    assert lt.dL * 16 == pytest.approx(lt.max - lt.min, rel=1e-6)
    assert lt.kappa * lt.dL == pytest.approx(1.0, rel=1e-6)
    assert lt.Lc == pytest.approx(0.5 * L.sum(), abs=1e-6)


@pytest.mark.parametrize("seed", range(6))
def test_light_frame_is_right_handed_orthonormal(orc, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    lt = orc.light_setup(d, 8, 8)
    L, U, V = (np.array(x[:], dtype=np.float64) for x in (lt.L, lt.U, lt.V))
    assert np.allclose(L, unit(d), atol=1e-6)
    for a, b in ((U, L), (V, L), (U, V)):
        assert abs(a @ b) < 1e-6
    assert np.linalg.norm(U) == pytest.approx(1.0, abs=1e-6)
    assert np.linalg.norm(V) == pytest.approx(1.0, abs=1e-6)
    assert np.linalg.det(np.stack([U, V, L])) == pytest.approx(1.0, abs=1e-5)
    # U comes from the world axis least aligned with L.
    ax = int(np.argmin(np.abs(L)))
    assert lt.axis == ax
    assert U[ax] > 0 and abs(U[ax]) == pytest.approx(np.sqrt(1 - L[ax] ** 2), abs=1e-6)
    assert lt.sigma == pytest.approx(8 / (2 * H_SQRT3), rel=1e-6)


@pytest.mark.parametrize("seed", range(4))
def test_texel_world_and_light_coords_are_inverse(orc, seed):
    """Texel (i, j) of slice k lies at c + (min + k dL - L.c) L + u_i U + v_j V with
    u_i = (2(i + 1/2)/R - 1) h, and maps back to (lambda, tu, tv) = (k, i, j)."""
    rng = np.random.default_rng(100 + seed)
    d = rng.normal(size=3)
    n, R = int(rng.integers(3, 40)), int(rng.integers(2, 70))
    lt = orc.light_setup(d, n, R)
    L, U, V = (np.array(x[:], dtype=np.float64) for x in (lt.L, lt.U, lt.V))
    c = np.full(3, 0.5)
    for _ in range(20):
        i, j, k = int(rng.integers(R)), int(rng.integers(R)), int(rng.integers(n))
        X = orc.texel_world(lt, i, j, k).astype(np.float64)
        u_i = (2 * (i + 0.5) / R - 1) * H_SQRT3
        v_j = (2 * (j + 0.5) / R - 1) * H_SQRT3
        assert (X - c) @ U == pytest.approx(u_i, abs=2e-6)
        assert (X - c) @ V == pytest.approx(v_j, abs=2e-6)
        assert X @ L == pytest.approx(lt.min + k * (lt.max - lt.min) / n, abs=2e-6)
        lam, tu, tv = orc.light_coords(lt, X)
        assert lam == pytest.approx(k, abs=1e-3 * max(1, n / 64))
        assert tu == pytest.approx(i, abs=1e-3 * max(1, R / 64))
        assert tv == pytest.approx(j, abs=1e-3 * max(1, R / 64))
        # Eq. 9 with nearest-slice selection: a point on plane k reads slice k.
        _, rec = orc.stack_lookup(np.zeros((n, R, R)), lt, lam, tu, tv)
        assert rec[0] == k


# --------------------------------------------------------------------------
# Reconstruction and classification.

def test_trilinear_reproduces_linear_field_and_clamps(orc):
    nx, ny, nz = 5, 7, 9
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = lambda X, Y, Z: 1000 + 37 * X + 101 * Y + 307 * Z
    vol = f(x, y, z).astype(np.uint16)
    rng = np.random.default_rng(7)
    N = np.array([nx, ny, nz], dtype=np.float64)
    for _ in range(200):
        P = rng.uniform(0.5 / N, 1 - 0.5 / N).astype(np.float32)
        v, cell = orc.sample_volume(vol, P)
        X = P.astype(np.float64) * N - 0.5
        assert v == pytest.approx(f(*X), abs=1e-3)
        assert cell == tuple(np.floor(X).astype(int))
    # Outer half voxel: clamp to edge along that axis only.
    P = np.array([0.2 / nx, 0.5, 1 - 0.1 / nz], dtype=np.float32)
    v, _ = orc.sample_volume(vol, P)
    assert v == pytest.approx(f(0.0, 0.5 * ny - 0.5, nz - 1.0), abs=1e-3)


def test_tf_lookup_matches_numpy_interp(orc):
    rng = np.random.default_rng(3)
    M, vmin, vmax = 37, -50.0, 913.0
    tf = rng.uniform(0, 1, size=(M, 4)).astype(np.float32)
    for v in rng.uniform(vmin - 100, vmax + 100, size=300):
        x = (v - vmin) / (vmax - vmin) * (M - 1)
        want = [np.interp(x, np.arange(M), tf[:, ch].astype(np.float64)) for ch in range(4)]
        assert np.allclose(orc.tf_lookup(tf, vmin, vmax, v), want, atol=1e-12)


def test_stack_lookup_bilinear_reproduces_linear_and_clamps(orc):
    n, R = 5, 10
    k, j, i = np.meshgrid(np.arange(n), np.arange(R), np.arange(R), indexing="ij")
    B = 0.1 + 0.01 * i + 0.001 * j + 0.0001 * k
    lt = orc.light_setup((0.2, 0.3, 0.9), n, R)
    rng = np.random.default_rng(5)
    for _ in range(200):
        lam, tu, tv = rng.uniform(-1, n), rng.uniform(-2, R + 1), rng.uniform(-2, R + 1)
        lam32, tu32, tv32 = np.float32(lam), np.float32(tu), np.float32(tv)
        kk = int(min(max(np.floor(np.float32(lam32 + np.float32(0.5))), 0), n - 1))
        want = (0.1 + 0.01 * np.clip(float(tu32), 0, R - 1) + 0.001 * np.clip(float(tv32), 0, R - 1)
                + 0.0001 * kk)
        got, rec = orc.stack_lookup(B, lt, lam32, tu32, tv32)
        assert got == pytest.approx(want, abs=1e-12)
        assert rec[0] == kk


# --------------------------------------------------------------------------
# Algorithm 1: the attenuation buffer.

def slab_scene(a=f32(0.3)):
    N, z_lo, z_hi = 16, 5, 9
    vol = np.zeros((N, N, N), np.uint8)
    vol[z_lo:z_hi + 1] = 200
    tf = step_tf(256, [(100, 256, (1, 1, 1, a))])
    return vol, tf, N, z_lo, z_hi


def test_T1_homogeneous_slab_is_geometric_series(orc):
    """Light +z through a slab of opacity a: B_k = (1 - a)^(planes j < k in the slab)."""
    a = f32(0.3)
    vol, tf, N, z_lo, z_hi = slab_scene(a)
    n, R = 50, 24
    lt = orc.light_setup((0, 0, 1), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    d = np.arange(n) / n
    in_slab = (d >= z_lo / N) & (d <= (z_hi + 1) / N)
    m = np.concatenate([[0], np.cumsum(in_slab)[:-1]])
    u = (2 * (np.arange(R) + 0.5) / R - 1) * H_SQRT3
    inside = np.abs(u) <= 0.5
    want = np.ones((n, R, R))
    cols = inside[:, None] & inside[None, :]          # [j, i]
    want[:, cols] = ((1 - a) ** m)[:, None]
    assert np.abs(B - want).max() < 1e-12
    assert B[0].min() == 1.0  # exclusive convention: slice 0 sees full light


def test_T1_comp_n_darkening_compensation(orc):
    """(1 + alpha)^c compensation scales every stored slice, clamped at 1."""
    a, c = f32(0.3), 2.0
    vol, tf, N, z_lo, z_hi = slab_scene(a)
    n, R = 50, 8
    lt = orc.light_setup((0, 0, 1), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt, comp_n=c)
    d = np.arange(n) / n
    in_slab = (d >= z_lo / N) & (d <= (z_hi + 1) / N)
    m = np.concatenate([[0], np.cumsum(in_slab)[:-1]])
    want = np.minimum(1.0, (1 - a) ** m * (1 + a * in_slab) ** c)
    col = B[:, R // 2, R // 2]
    assert np.abs(col - want).max() < 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_T1_homogeneous_cube_oblique_light(orc, seed):
    """Full homogeneous cube, oblique light: B_k = (1 - a)^(#{j < k : P_j in cube})."""
    a = f32(0.2)
    N = 8
    vol = np.full((N, N, N), 200, np.uint8)
    tf = step_tf(256, [(100, 256, (1, 1, 1, a))])
    rng = np.random.default_rng(20 + seed)
    d = rng.normal(size=3)
    n, R = 37, 16
    lt = orc.light_setup(d, n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    L = unit(d)
    U, V = np.array(lt.U[:], float), np.array(lt.V[:], float)
    mn, mx = np.minimum(L, 0).sum(), np.maximum(L, 0).sum()
    s = mn + np.arange(n) * (mx - mn) / n - 0.5 * L.sum()
    checked = 0
    for j in range(R):
        for i in range(R):
            u = (2 * (i + 0.5) / R - 1) * H_SQRT3
            v = (2 * (j + 0.5) / R - 1) * H_SQRT3
            P = 0.5 + s[:, None] * L[None, :] + u * U[None, :] + v * V[None, :]
            margin = np.minimum(P, 1 - P).min(axis=1)
            if np.any(np.abs(margin) < 1e-5):
                continue
            inside = margin >= 0
            m = np.concatenate([[0], np.cumsum(inside)[:-1]])
            assert np.abs(B[:, j, i] - (1 - a) ** m).max() < 1e-12
            checked += 1
    assert checked > R * R // 2


def blob_scene(N=24, sigma=5.0, peak=20000):
    idx = np.arange(N) + 0.5 - N / 2
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    vol = np.rint(peak * np.exp(-(x * x + y * y + z * z) / (2 * sigma * sigma))).astype(np.uint16)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = 1.0
    tf[:, 3] = np.linspace(0.0, 0.08, 256)
    return vol, tf, 0.0, float(peak)


def test_T4_corrected_sweep_converges_to_exact_light_march(orc):
    """With opacity correction, B at a fixed point approaches Eq. 1's exact
    transmittance exp(-int kappa) at first order as the slice count grows."""
    vol, tf, vmin, vmax = blob_scene()
    d = (0.3, -0.5, 0.81)
    R, i, j = 8, 3, 4
    errs = []
    for n in (16, 32, 64, 128, 256, 512, 1024):
        lt = orc.light_setup(d, n, R)
        B = orc.build_stack(vol, tf, vmin, vmax, lt, opacity_correction=1)
        k = n // 2
        P = orc.texel_world(lt, i, j, k).astype(np.float64)
        exact = orc.transmittance_bruteforce(vol, tf, vmin, vmax, np.array(lt.L[:], float), P,
                                             m=40000)
        assert 0.05 < exact < 0.95  # the column crosses the blob
        errs.append(abs(B[k, j, i] - exact))
    errs = np.array(errs)
    assert np.all(np.diff(errs) < 0), errs
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios[2:] > 1.6) and np.all(ratios[2:] < 2.5), ratios  # O(1/n)


def test_T4_uncorrected_sweep_darkens_with_slice_count(orc):
    """Without correction every slice applies the full TF opacity, so the same
    point gets darker as slices are added (the effect compensated in 4.)."""
    vol, tf, vmin, vmax = blob_scene()
    d = (0.3, -0.5, 0.81)
    vals = []
    for n in (16, 32, 64, 128):
        lt = orc.light_setup(d, n, 8)
        B = orc.build_stack(vol, tf, vmin, vmax, lt)
        vals.append(B[n // 2, 4, 3])
    assert np.all(np.diff(vals) < 0), vals


# --------------------------------------------------------------------------
# The eye pass: compositing, sample counts, orientation.

def homog_cube(a=f32(0.25), rgb=(0.2, 0.5, 0.9), N=16):
    vol = np.full((N, N, N), 200, np.uint8)
    tf = step_tf(256, [(100, 256, (*rgb, a))])
    return vol, tf


@pytest.mark.parametrize("persp", [False, True])
def test_T9_no_illumination_homogeneous_cube(orc, persp):
    """Mode NONE: A = 1 - (1 - a)^m and C = rgb (1 - (1 - a)^m), m the exact
    sample count (Eq. 2 / Eq. 3 with constant samples)."""
    a, rgb = f32(0.25), np.array([0.2, 0.5, 0.9], dtype=np.float32).astype(np.float64)
    vol, tf = homog_cube(a, rgb)
    lt = orc.light_setup((0, 0, 1), 4, 4)
    W = H = 1 if persp else 8
    c = cam((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), persp, 30.0, 0.5)
    ro = orc.render_opts(orc.NONE, 0.5)
    img, alt, amb, ns = orc.render_image(vol, tf, 0, 255, lt, None, c, W, H, ro)
    m = 32  # t in [2, 3), dt = 0.5 / 16
    assert np.all(ns == m)
    assert np.allclose(img[..., 3], 1 - (1 - a) ** m, atol=1e-12)
    assert np.allclose(img[..., :3], rgb * (1 - (1 - a) ** m), atol=1e-12)


def test_T9_sample_count_on_oblique_rays(orc):
    a = f32(0.1)
    vol, tf = homog_cube(a, (1, 1, 1))
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((2.3, -1.1, 1.7), (0.45, 0.55, 0.5), (0, 0, 1), False, 40, 0.7)
    ro = orc.render_opts(orc.NONE, 0.7)
    W = H = 16
    img, alt, amb, ns = orc.render_image(vol, tf, 0, 255, lt, None, c, W, H, ro)
    fr = orc.frame_setup(c, W, H, 0.7, 16)
    checked = 0
    for y in range(H):
        for x in range(W):
            ray = orc.ray_setup(lt, fr, ro, x, y)
            if not ray.hit:
                assert ns[y, x] == 0 and img[y, x, 3] == 0.0
                continue
            span = (float(ray.t1) - float(ray.t0)) / float(fr.dt)
            if abs(span - round(span)) < 1e-3:
                continue
            m = int(math.ceil(span))
            assert ns[y, x] == m
            assert img[y, x, 3] == pytest.approx(1 - (1 - a) ** m, abs=1e-12)
            checked += 1
    assert checked > 50


def test_T5_front_to_back_matches_eq2_product_form(orc):
    """Two layers (red over blue) seen from above: Eq. 3's iteration must equal
    Eq. 2's sum C = sum_i C_i prod_{j<i} (1 - A_j) over the known samples."""
    N, a1, a2 = 16, f32(0.15), f32(0.4)
    vol = np.zeros((N, N, N), np.uint8)
    vol[8:] = 100   # z in [0.5, 1]: red
    vol[:8] = 200   # z in [0, 0.5]: blue
    tf = step_tf(256, [(50, 150, (1, 0, 0, a1)), (150, 256, (0, 0, 1, a2))])
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    ro = orc.render_opts(orc.NONE, 0.5)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, None, c, 4, 4, ro)
    Ci = [np.array([a1, 0, 0])] * 16 + [np.array([0, 0, a2])] * 16   # opacity-weighted
    Ai = [a1] * 16 + [a2] * 16
    C = sum(Ci[i] * np.prod([1 - Ai[j] for j in range(i)]) for i in range(32))
    A = 1 - np.prod([1 - x for x in Ai])
    assert np.allclose(img[..., :3], C, atol=1e-12)
    assert np.allclose(img[..., 3], A, atol=1e-12)
    assert img[0, 0, 0] > img[0, 0, 2]  # the front (red) layer dominates


def test_image_orientation(orc):
    """Row 0 is the top of the image; +x of the camera frame is to the right."""
    N = 16
    vol = np.zeros((N, N, N), np.uint8)
    vol[:, :4, :4] = 200   # x, y in [0, 1/4)
    tf = step_tf(256, [(100, 256, (1, 1, 1, 0.3))])
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, None, c, 16, 16, orc.render_opts(orc.NONE, 0.5))
    A = img[..., 3]
    assert A[13:, :3].min() > 0.5       # bottom-left
    assert A[:10, :].max() == 0.0 and A[:, 6:].max() == 0.0


def test_T3_empty_volume_returns_background_exactly(orc):
    N = 12
    vol = np.zeros((N, N, N), np.uint16)
    tf = step_tf(64, [(1, 64, (1, 1, 1, 0.5))])
    bg = (0.1, 0.2, 0.3, 0.4)
    for mode in (orc.NONE, orc.SHADOW, orc.SHELL, orc.CONE):
        lt = orc.light_setup((0.3, 0.2, -0.9), 9, 11)
        B = orc.build_stack(vol, tf, 0, 1000, lt)
        assert B.min() == 1.0
        c = cam((1.9, 1.7, 1.3), (0.5, 0.5, 0.5), (0, 0, 1), True, 40, 0.5)
        ro = orc.render_opts(mode, 0.5, bg=bg)
        img, *_ = orc.render_image(vol, tf, 0, 1000, lt, B, c, 9, 7, ro)
        assert np.all(img == np.array(bg, dtype=np.float32).astype(np.float64))


def test_T2_opaque_plate_casts_exact_shadow(orc):
    """An opaque (alpha = 1, black) plate under a receiver slab, light +z, camera
    looking down: inside the plate's footprint the receiver gets no light
    (C = 0, A = 1); outside it receives (1 - a)^(receiver planes before it)."""
    N, a = 32, f32(0.25)
    vol = np.zeros((N, N, N), np.uint8)
    vol[12:14, 8:24, 8:24] = 255      # plate: z in [0.375, 0.4375], x, y in [0.25, 0.75]
    vol[24:28] = 100                   # receiver: z in [0.75, 0.875]
    tf = step_tf(256, [(50, 151, (1, 1, 1, a)), (200, 256, (0, 0, 0, 1.0))])
    ramp = np.linspace(0, 1, 51)[1:-1]
    tf[151:200, :3] = (1 - ramp)[:, None]
    tf[151:200, 3] = a + (1 - a) * ramp
    n, R = 50, 64
    lt = orc.light_setup((0, 0, 1), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, B, c, 64, 64,
                               orc.render_opts(orc.SHADOW, 0.5))
    # Receiver samples: z_i = 1 - i/64, i = 8..16; light planes j/50 in [0.75, 0.875].
    planes = [j for j in range(n) if 0.75 <= j / n <= 0.875]
    z = 1 - np.arange(8, 17) / 64
    k = np.clip(np.floor(n * z + 0.5), 0, n - 1)
    e = np.array([sum(1 for j in planes if j < kk) for kk in k])
    lit = a * np.sum((1 - a) ** np.arange(9) * (1 - a) ** e)
    xs = (np.arange(64) + 0.5) / 64
    inner = np.abs(xs - 0.5) < 0.25 - 0.09
    outer = np.abs(xs - 0.5) > 0.25 + 0.09
    # Within a texel of the cube's side faces the lookup blends in light
    # columns that pass outside the cube (no medium there), so stay clear.
    in_cube = np.abs(xs - 0.5) < 0.5 - 2 * H_SQRT3 / R
    shadow = img[np.ix_(inner, inner)]
    assert np.all(shadow[..., :3] == 0.0) and np.allclose(shadow[..., 3], 1.0, atol=1e-15)
    out_mask = (outer[:, None] | outer[None, :]) & in_cube[:, None] & in_cube[None, :]
    assert out_mask.sum() > 500
    assert np.allclose(img[out_mask][:, :3], lit, atol=1e-12)
    assert np.allclose(img[out_mask][:, 3], 1 - (1 - a) ** 9, atol=1e-12)


@pytest.mark.parametrize("mode", ["shell", "cone"])
def test_T7_scattering_on_homogeneous_medium(orc, mode):
    """Homogeneous cube, light +z so B_k = (1 - a)^k; a vertical eye ray.  The
    coefficient is the mean of (1 - a)^k over the neighbours' slices: shell
    S +- r e_a (four at the sample's own slice), cone rings n = 1, 2 slices
    towards the light (four points each)."""
    N, a = 32, f32(0.1)
    vol = np.full((N, N, N), 200, np.uint8)
    tf = step_tf(256, [(100, 256, (1, 1, 1, a))])
    n, R = 50, 64
    lt = orc.light_setup((0, 0, 1), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    assert np.allclose(B[:, R // 2, R // 2], (1 - a) ** np.arange(n), atol=1e-14)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.25)
    md = orc.SHELL if mode == "shell" else orc.CONE
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, B, c, 4, 4, orc.render_opts(md, 0.5))
    z = 1 - np.arange(64) / 64
    ks = lambda lam: np.clip(np.floor(lam + 0.5), 0, n - 1)
    lam = n * z
    if mode == "shell":
        r = n / N  # one voxel in slice units
        coef = (4 * (1 - a) ** ks(lam) + (1 - a) ** ks(lam + r) + (1 - a) ** ks(lam - r)) / 6
    else:
        coef = 4 * ((1 - a) ** ks(lam - 1) + (1 - a) ** ks(lam - 2)) / 8
    C = np.sum(a * (1 - a) ** np.arange(64) * coef)
    assert np.allclose(img[..., :3], C, atol=1e-12)


def test_single_slice_shadow_equals_no_illumination(orc):
    """n = 1: the only slice is the one nearest the light, which (exclusive
    buffer) holds full light, so every coefficient is 1."""
    sys_vol = np.random.default_rng(0).integers(0, 255, size=(10, 11, 12)).astype(np.uint8)
    tf = np.random.default_rng(1).uniform(0, 0.2, size=(256, 4)).astype(np.float32)
    lt = orc.light_setup((0.4, -0.2, 0.7), 1, 5)
    B = orc.build_stack(sys_vol, tf, 0, 255, lt)
    assert B.min() == 1.0
    c = cam((1.9, 1.7, 1.3), (0.5, 0.5, 0.5), (0, 0, 1), True, 40, 0.5)
    ref, *_ = orc.render_image(sys_vol, tf, 0, 255, lt, None, c, 12, 9, orc.render_opts(orc.NONE, 0.5))
    for mode in (orc.SHADOW, orc.SHELL, orc.CONE):
        img, *_ = orc.render_image(sys_vol, tf, 0, 255, lt, B, c, 12, 9, orc.render_opts(mode, 0.5))
        assert np.allclose(img, ref, atol=1e-14)


def test_early_ray_termination_threshold(orc):
    a = f32(0.25)
    vol, tf = homog_cube(a, (1, 1, 1))
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    ro = orc.render_opts(orc.NONE, 0.5, ert=0.9)
    img, alt, amb, ns = orc.render_image(vol, tf, 0, 255, lt, None, c, 4, 4, ro)
    m = next(q for q in range(1, 100) if 1 - (1 - a) ** q > 0.9)
    assert np.all(ns == m) and not amb.any()
    assert np.allclose(img[..., 3], 1 - (1 - a) ** m, atol=1e-12)
    assert np.all(img == alt)


# Early ray termination window (Eq. 3 with the test A > ert after each
# sample, reading R12).  Homogeneous cube, alpha a = 0.25, vertical orthographic
# rays with 32 samples: after q samples A_q = 1 - 0.75^q (A_7 = 0.86652,
# A_8 = 0.89989, A_9 = 0.92492, A_11 = 0.95776, A_12 = 0.96832, A_30 = 0.99982,
# A_31 = 0.99987, A_32 = 0.99990) and C = rgb A_q.  The window runs from the
# first sample with A > ert - band to the first with A > ert + band (or the
# ray's last sample); each case below is worked out by hand from those values:
# (ert, band, window kind, samples of the binary64 decision, of alt, of the
# window's end).
def _a_after(q, a=f32(0.25)):
    return 1 - (1 - a) ** q


ERT_WINDOW_CASES = [
    # A_8 just above ert, inside the band: stop at 8 (binary64) or 9 (A_9 > ert + band).
    (lambda: _a_after(8) - 4e-6, 1e-5, 1, 8, 9, 9),
    # A_8 just below ert, inside the band: stop at 9 (binary64) or already at 8.
    (lambda: _a_after(8) + 4e-6, 1e-5, 1, 9, 8, 9),
    # ert between A_8 + band and A_9 - band: one outcome.
    (lambda: 0.91, 1e-5, 0, 9, 9, 9),
    # The ray ends (32 samples) with A_32 in the band below ert: one outcome, all samples.
    (lambda: _a_after(32) + 4e-6, 1e-5, 0, 32, 32, 32),
    # A_32 in the band above ert, A_31 below it: the window is the last sample alone.
    (lambda: _a_after(32) - 4e-6, 1e-5, 0, 32, 32, 32),
    # A_31 in the band below ert, A_32 past ert + band: stop at 32 or at 31.
    (lambda: _a_after(31) + 4e-6, 1e-5, 1, 32, 31, 32),
    # A wide band: samples 7..12 are in the window, the binary64 decision is 9.
    (lambda: 0.9, 0.06, 2, 9, 7, 12),
    # A_30..A_32 in the window and the ray ends inside it: decision 31, window start 30.
    (lambda: _a_after(31) - 1e-6, 5e-5, 2, 31, 30, 32),
    # A wide band whose binary64 decision is its first sample (A_8 > 0.8998;
    # A_10 = 0.94369 is the first past 0.9298): alt is the window's end.
    (lambda: 0.8998, 0.03, 2, 8, 10, 10),
]


@pytest.mark.parametrize("case", range(len(ERT_WINDOW_CASES)))
def test_early_ray_termination_window(orc, case):
    ert_of, band, want_win, want_ns, want_alt, want_end = ERT_WINDOW_CASES[case]
    a = f32(0.25)
    rgb = np.array([0.2, 0.5, 0.9], dtype=np.float32).astype(np.float64)
    vol, tf = homog_cube(a, rgb)
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    ro = orc.render_opts(orc.NONE, 0.5, ert=ert_of(), ert_band=band)
    xs, ys = np.array([0, 1, 0, 1]), np.array([0, 0, 1, 1])
    out, alt, win, ns, ns_alt, end, ns_end = orc.render_window(vol, tf, 0, 255, lt, None, c,
                                                               2, 2, ro, xs, ys)
    assert np.all(win == want_win)
    assert np.all(ns == want_ns) and np.all(ns_alt == want_alt)
    assert np.all(ns_end == want_end)
    for img, q in ((out, want_ns), (alt, want_alt), (end, want_end)):
        assert np.allclose(img[:, 3], _a_after(q), atol=1e-14)
        assert np.allclose(img[:, :3], rgb * _a_after(q), atol=1e-14)
    # render_pixels reports the same decision with a boolean flag.
    out2, alt2, amb2, ns2 = orc.render_pixels(vol, tf, 0, 255, lt, None, c, 2, 2, ro, xs, ys)
    assert np.array_equal(out2, out) and np.array_equal(alt2, alt)
    assert np.array_equal(amb2, win > 0) and np.array_equal(ns2, ns)


def test_opacity_correction_in_eye_pass(orc):
    a, s = f32(0.25), 0.5
    vol, tf = homog_cube(a, (1, 1, 1))
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    ro = orc.render_opts(orc.NONE, s, opacity_correction=1)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, None, c, 2, 2, ro)
    assert np.allclose(img[..., 3], 1 - (1 - a) ** (32 * s), atol=1e-12)


def test_background_and_light_colour(orc):
    a = f32(0.3)
    vol, tf = homog_cube(a, (0.5, 0.5, 0.5))
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    bg, col = (0.9, 0.1, 0.3, 0.5), (1.0, 0.5, 0.25)
    ro = orc.render_opts(orc.NONE, 0.5, bg=bg, color=col)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, None, c, 2, 2, ro)
    A = 1 - (1 - a) ** 32
    want_rgb = 0.5 * np.array(col) * A + (1 - A) * np.array(bg[:3], dtype=np.float32)
    assert np.allclose(img[..., :3], want_rgb, atol=1e-7)
    assert np.allclose(img[..., 3], A + (1 - A) * np.float32(0.5), atol=1e-7)


def test_eye_inside_volume(orc):
    a = f32(0.2)
    vol, tf = homog_cube(a, (1, 1, 1))
    lt = orc.light_setup((0, 0, 1), 4, 4)
    c = cam((0.5, 0.5, 0.5), (1.5, 0.5, 0.5), (0, 0, 1), True, 10, 0.5)
    img, alt, amb, ns = orc.render_image(vol, tf, 0, 255, lt, None, c, 1, 1,
                                         orc.render_opts(orc.NONE, 0.5))
    assert ns[0, 0] == 16  # t in [0, 0.5), dt = 1/32
    assert img[0, 0, 3] == pytest.approx(1 - (1 - a) ** 16, abs=1e-12)


# --------------------------------------------------------------------------
# Scattering geometry against the paper's own formulas.

def rodrigues(B, L, theta):
    """Eq. 11: rotation of B by theta about the unit axis L."""
    return (B * math.cos(theta) + np.cross(L, B) * math.sin(theta)
            + (L @ B) * L * (1 - math.cos(theta)))


def test_rodrigues_invariants():
    rng = np.random.default_rng(9)
    for _ in range(20):
        L = unit(rng.normal(size=3))
        B = rng.normal(size=3)
        B -= (B @ L) * L
        for th in rng.uniform(0, 2 * np.pi, size=4):
            A = rodrigues(B, L, th)
            assert np.linalg.norm(A) == pytest.approx(np.linalg.norm(B))
            assert abs(A @ L) < 1e-12
        assert np.allclose(rodrigues(B, L, 0.0), B)
        assert np.allclose(rodrigues(B, L, np.pi), -B)


@pytest.mark.parametrize("seed", range(5))
def test_cone_points_match_rodrigues_construction(orc, seed):
    """The cone's eight lookup points, expressed as light-space offsets from the
    sample, equal c_n + rho_n A_m with c_n = S - n dL L, rho_n = n dL tan(phi)
    and A_m = Eq. 11 rotation by m pi/2 of B_proj, the unit part of E - S
    orthogonal to L."""
    rng = np.random.default_rng(40 + seed)
    d = rng.normal(size=3)
    n, R = int(rng.integers(16, 300)), int(rng.integers(16, 600))
    lt = orc.light_setup(d, n, R)
    L, U, V = (np.array(x[:], dtype=np.float64) for x in (lt.L, lt.U, lt.V))
    view = unit(rng.normal(size=3))
    eye = 0.5 - 2.5 * view
    c = cam(eye, (0.5, 0.5, 0.5), (0, 0, 1) if abs(view[2]) < 0.9 else (0, 1, 0), True, 40, 0.5)
    phi = float(rng.uniform(5, 40))
    ro = orc.render_opts(orc.CONE, 0.5, cone_half_angle_deg=phi)
    fr = orc.frame_setup(c, 32, 24, 0.5, 64)
    tanphi = math.tan(math.radians(phi))
    for _ in range(5):
        ray = orc.ray_setup(lt, fr, ro, int(rng.integers(32)), int(rng.integers(24)))
        dvec = np.array(ray.d[:], dtype=np.float64)
        E_S = -dvec
        Bp = unit(E_S - (E_S @ L) * L)
        for ring in (1, 2):
            for m in range(4):
                A = rodrigues(Bp, L, m * np.pi / 2)
                w = -ring * lt.dL * L + ring * lt.dL * tanphi * A
                want = np.array([lt.kappa * (L @ w), lt.sigma * (U @ w), lt.sigma * (V @ w)])
                got = np.array(ray.nb[(ring - 1) * 4 + m][:], dtype=np.float64)
                assert np.allclose(got, want, atol=2e-5 * max(1.0, np.abs(want).max()))
    assert ray.nnb == 8


def test_cone_falls_back_to_U_when_view_is_parallel_to_light(orc):
    lt = orc.light_setup((0, 0, 1), 32, 32)
    c = cam((0.5, 0.5, -2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    ro = orc.render_opts(orc.CONE, 0.5)
    fr = orc.frame_setup(c, 1, 1, 0.5, 16)
    ray = orc.ray_setup(lt, fr, ro, 0, 0)
    nb = np.array([ray.nb[q][:] for q in range(8)])
    assert np.all(nb[:4, 0] == -1) and np.all(nb[4:, 0] == -2)
    assert nb[0, 1] > 0 and nb[0, 2] == 0  # B_proj = U
    assert nb[1, 1] == 0 and nb[1, 2] > 0  # quarter turn about L: V


@pytest.mark.parametrize("seed", range(3))
def test_shell_points_are_axis_neighbours(orc, seed):
    rng = np.random.default_rng(60 + seed)
    d = rng.normal(size=3)
    n, R, Nmax = 64, 128, 48
    lt = orc.light_setup(d, n, R)
    L, U, V = (np.array(x[:], dtype=np.float64) for x in (lt.L, lt.U, lt.V))
    ro = orc.render_opts(orc.SHELL, 0.5, shell_radius_vox=1.5)
    c = cam((2, 2, 2), (0.5, 0.5, 0.5), (0, 0, 1), True, 40, 0.5)
    fr = orc.frame_setup(c, 4, 4, 0.5, Nmax)
    ray = orc.ray_setup(lt, fr, ro, 1, 2)
    assert ray.nnb == 6
    r = 1.5 / Nmax
    for a in range(3):
        for s, sign in enumerate((1.0, -1.0)):
            w = np.zeros(3)
            w[a] = sign * r
            want = np.array([lt.kappa * (L @ w), lt.sigma * (U @ w), lt.sigma * (V @ w)])
            assert np.allclose(np.array(ray.nb[2 * a + s][:], float), want, atol=1e-5)


def test_oracle_rejects_invalid_input(orc):
    with pytest.raises(ValueError):
        orc.light_setup((0, 0, 0), 4, 4)
    with pytest.raises(ValueError):
        orc.light_setup((np.nan, 0, 1), 4, 4)
    with pytest.raises(ValueError):
        orc.light_setup((0, 0, 1), 0, 4)


# --------------------------------------------------------------------------
# Variants: the extinction form of the buffer (Eq. 5-6), linear filtering
# between slices, several shells (Section 3.2.3).

def test_depth_buffer_is_summed_extinction_on_slab(orc):
    """Eq. 5-6: the buffer holds D_k = m_k (-ln(1 - a)), m_k the slab planes
    before plane k; exp(-D_k) is T1's geometric series."""
    a = f32(0.3)
    vol, tf, N, z_lo, z_hi = slab_scene(a)
    n, R = 50, 24
    lt = orc.light_setup((0, 0, 1), n, R)
    D = orc.build_stack(vol, tf, 0, 255, lt, quantity=orc.OPTICAL_DEPTH)
    d = np.arange(n) / n
    in_slab = (d >= z_lo / N) & (d <= (z_hi + 1) / N)
    m = np.concatenate([[0], np.cumsum(in_slab)[:-1]])
    tau = -math.log(1.0 - a)
    col = D[:, R // 2, R // 2]
    assert np.abs(col - m * tau).max() < 1e-12
    assert np.abs(np.exp(-col) - (1 - a) ** m).max() < 1e-12
    assert D[0].max() == 0.0                     # slice 0: no medium before it
    corner = D[:, 0, 0]                          # a column that misses the cube
    assert np.all(corner == 0.0)


def test_depth_buffer_caps_opaque_layers(orc):
    """An opaque layer (alpha = 1, tau infinite) leaves exactly the cap 64
    behind it; depth never decreases, and exp(-D) is the transmittance 0 to
    within exp(-64)."""
    N = 16
    vol = np.zeros((N, N, N), np.uint8)
    vol[4:12] = 255
    tf = step_tf(256, [(128, 256, (1, 1, 1, 1.0))])
    n, R = 32, 8
    lt = orc.light_setup((0, 0, 1), n, R)
    D = orc.build_stack(vol, tf, 0, 255, lt, quantity=orc.OPTICAL_DEPTH)
    T = orc.build_stack(vol, tf, 0, 255, lt)
    col = D[:, R // 2, R // 2]
    assert col[0] == 0.0 and np.all(col[: int(0.2 * n)] == 0.0)   # before the layer
    assert np.all(col[int(0.8 * n):] == orc.DEPTH_MAX)               # behind it: capped
    assert np.all(np.diff(col) >= 0.0) and col.max() == orc.DEPTH_MAX
    assert np.isfinite(D).all()
    assert np.abs(np.exp(-D) - T).max() < 1e-27


def test_depth_comp_n_subtracts_log_compensation(orc):
    """(1 + alpha)^c compensation in depth form: D' = max(0, D - c ln(1 + alpha))."""
    a, c = f32(0.3), 2.0
    vol, tf, N, z_lo, z_hi = slab_scene(a)
    n, R = 50, 8
    lt = orc.light_setup((0, 0, 1), n, R)
    D = orc.build_stack(vol, tf, 0, 255, lt, comp_n=c, quantity=orc.OPTICAL_DEPTH)
    d = np.arange(n) / n
    in_slab = (d >= z_lo / N) & (d <= (z_hi + 1) / N)
    m = np.concatenate([[0], np.cumsum(in_slab)[:-1]])
    want = np.maximum(0.0, m * -math.log(1 - a) - c * np.log1p(a * in_slab))
    assert np.abs(D[:, R // 2, R // 2] - want).max() < 1e-12


def test_depth_and_transmittance_buffers_agree_at_texel_centres(orc):
    """exp(-sum of -ln(1 - alpha)) = prod(1 - alpha) on an arbitrary volume and light."""
    vol, tf, vmin, vmax = blob_scene()
    tf[:, 3] *= 6.0                              # up to alpha 0.48 per sample
    lt = orc.light_setup((0.3, -0.5, 0.81), 40, 20)
    T = orc.build_stack(vol, tf, vmin, vmax, lt)
    D = orc.build_stack(vol, tf, vmin, vmax, lt, quantity=orc.OPTICAL_DEPTH)
    assert T.min() < 0.5                         # the light is really attenuated
    assert np.abs(np.exp(-D) - T).max() < 1e-12


def linear_field(n, R):
    k, j, i = np.meshgrid(np.arange(n), np.arange(R), np.arange(R), indexing="ij")
    return 0.1 + 0.01 * i + 0.001 * j + 0.0001 * k


@pytest.mark.parametrize("quantity", ["transmittance", "depth"])
@pytest.mark.parametrize("slices", ["nearest", "linear"])
def test_light_lookup_reproduces_linear_field(orc, quantity, slices):
    """Bilinear in (tu, tv), nearest or linear in lambda, clamped at every edge;
    an optical-depth buffer returns exp(-value)."""
    n, R = 5, 10
    B = linear_field(n, R)
    lt = orc.light_setup((0.2, 0.3, 0.9), n, R)
    q = orc.OPTICAL_DEPTH if quantity == "depth" else orc.TRANSMITTANCE
    sf = orc.SLICE_LINEAR if slices == "linear" else orc.SLICE_NEAREST
    ro = orc.render_opts(orc.SHADOW, 0.5, quantity=q, slice_filter=sf)
    rng = np.random.default_rng(7)
    for _ in range(300):
        lam, tu, tv = (np.float32(x) for x in (rng.uniform(-1.5, n + 0.5), rng.uniform(-2, R + 1),
                                               rng.uniform(-2, R + 1)))
        if slices == "linear":
            kk = int(min(max(np.floor(lam), 0), n - 1))
            lam_eff = min(max(float(lam), 0.0), n - 1.0)
        else:
            kk = int(min(max(np.floor(np.float32(lam + np.float32(0.5))), 0), n - 1))
            lam_eff = kk
        v = (0.1 + 0.01 * np.clip(float(tu), 0, R - 1) + 0.001 * np.clip(float(tv), 0, R - 1)
             + 0.0001 * lam_eff)
        want = math.exp(-v) if quantity == "depth" else v
        got, rec = orc.light_lookup(B, lt, ro, lam, tu, tv)
        assert got == pytest.approx(want, abs=1e-12)
        assert rec[0] == kk


@pytest.mark.parametrize("quantity", ["transmittance", "depth"])
def test_T7_multi_shell_on_homogeneous_medium(orc, quantity):
    """Two shells of radius 1 and 2 voxels (12 points, equal weights) on a
    homogeneous cube under light +z, in either buffer form: the coefficient is
    the mean of (1 - a)^k over the points' nearest slices."""
    N, a = 32, f32(0.1)
    vol = np.full((N, N, N), 200, np.uint8)
    tf = step_tf(256, [(100, 256, (1, 1, 1, a))])
    n, R = 50, 64
    q = orc.OPTICAL_DEPTH if quantity == "depth" else orc.TRANSMITTANCE
    lt = orc.light_setup((0, 0, 1), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt, quantity=q)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.25)
    ro = orc.render_opts(orc.SHELL, 0.5, quantity=q, shell_count=2)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, B, c, 4, 4, ro)
    z = 1 - np.arange(64) / 64
    ks = lambda lam: np.clip(np.floor(lam + 0.5), 0, n - 1)
    lam = n * z
    r = n / N
    coef = (8 * (1 - a) ** ks(lam) + (1 - a) ** ks(lam + r) + (1 - a) ** ks(lam - r)
            + (1 - a) ** ks(lam + 2 * r) + (1 - a) ** ks(lam - 2 * r)) / 12
    C = np.sum(a * (1 - a) ** np.arange(64) * coef)
    assert np.allclose(img[..., :3], C, atol=1e-12)


def test_linear_slice_filter_shadow_on_homogeneous_medium(orc):
    """Light +z through a homogeneous cube (B_k = (1 - a)^k), a vertical eye ray,
    shadow mode with linear slice filtering: the coefficient at lambda is
    (1 - w)(1 - a)^k0 + w (1 - a)^(k0 + 1), k0 = floor(lambda), w = lambda - k0."""
    N, a = 32, f32(0.1)
    vol = np.full((N, N, N), 200, np.uint8)
    tf = step_tf(256, [(100, 256, (1, 1, 1, a))])
    n, R = 50, 64
    lt = orc.light_setup((0, 0, 1), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.25)
    ro = orc.render_opts(orc.SHADOW, 0.5, slice_filter=orc.SLICE_LINEAR)
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, B, c, 4, 4, ro)
    lam = np.clip(n * (1 - np.arange(64) / 64), 0, n - 1)
    k0 = np.floor(lam)
    k1 = np.minimum(k0 + 1, n - 1)
    w = lam - k0
    coef = (1 - w) * (1 - a) ** k0 + w * (1 - a) ** k1
    C = np.sum(a * (1 - a) ** np.arange(64) * coef)
    assert np.allclose(img[..., :3], C, atol=1e-12)
    # Linear filtering differs from the nearest slice here (lambda is not on a plane).
    ref, *_ = orc.render_image(vol, tf, 0, 255, lt, B, c, 4, 4, orc.render_opts(orc.SHADOW, 0.5))
    assert np.abs(img - ref).max() > 1e-5


def test_shell_points_of_several_shells(orc):
    """Shell q of Q holds the axis neighbours at q r."""
    rng = np.random.default_rng(71)
    d = rng.normal(size=3)
    n, R, Nmax = 64, 128, 48
    lt = orc.light_setup(d, n, R)
    L, U, V = (np.array(x[:], dtype=np.float64) for x in (lt.L, lt.U, lt.V))
    ro = orc.render_opts(orc.SHELL, 0.5, shell_radius_vox=1.25, shell_count=3)
    c = cam((2, 2, 2), (0.5, 0.5, 0.5), (0, 0, 1), True, 40, 0.5)
    fr = orc.frame_setup(c, 4, 4, 0.5, Nmax)
    ray = orc.ray_setup(lt, fr, ro, 1, 2)
    assert ray.nnb == 18
    for q in (1, 2, 3):
        r = q * 1.25 / Nmax
        for a in range(3):
            for s, sign in enumerate((1.0, -1.0)):
                w = np.zeros(3)
                w[a] = sign * r
                want = np.array([lt.kappa * (L @ w), lt.sigma * (U @ w), lt.sigma * (V @ w)])
                got = np.array(ray.nb[6 * (q - 1) + 2 * a + s][:], float)
                assert np.allclose(got, want, atol=1e-5)


def test_variant_options_are_validated(orc):
    vol = np.zeros((4, 4, 4), np.uint8)
    tf = step_tf(16, [(1, 16, (1, 1, 1, 0.1))])
    lt = orc.light_setup((0, 0, 1), 4, 4)
    with pytest.raises(ValueError):
        orc.build_stack(vol, tf, 0, 255, lt, quantity=2)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    c = cam((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5)
    for kw in (dict(quantity=2), dict(slice_filter=2), dict(shell_count=5), dict(shell_count=-1)):
        with pytest.raises(ValueError):
            orc.render_image(vol, tf, 0, 255, lt, B, c, 2, 2, orc.render_opts(orc.SHELL, 0.5, **kw))


# --------------------------------------------------------------------------
# Point light (f4): rays from a light position, perspective texel grid.

def random_light_pos(rng, lo=1.2, hi=4.0):
    d = unit(rng.normal(size=3))
    return 0.5 + rng.uniform(lo, hi) * d


@pytest.mark.parametrize("seed", range(5))
def test_point_light_frame(orc, seed):
    rng = np.random.default_rng(80 + seed)
    P = random_light_pos(rng)
    n, R = 33, 48
    lt = orc.point_light_setup(P, n, R)
    P32 = np.array(lt.P[:], float)
    a = unit(0.5 - P32)
    L, U, V = (np.array(x[:], float) for x in (lt.L, lt.U, lt.V))
    assert np.allclose(L, a, atol=1e-6)
    assert abs(U @ L) < 1e-6 and abs(V @ L) < 1e-6 and abs(U @ V) < 1e-6
    assert np.allclose(np.cross(L, U), V, atol=1e-6)
    verts = np.array([[(c >> b) & 1 for b in range(3)] for c in range(8)], float)
    depth = (verts - P32) @ a
    assert lt.min == pytest.approx(depth.min(), abs=1e-5)
    assert lt.max == pytest.approx(depth.max(), abs=1e-5)
    assert lt.min > 0.0
    dc = np.linalg.norm(0.5 - P32)
    g = (math.sqrt(3) / 2) / math.sqrt(dc * dc - 0.75)
    assert lt.h == pytest.approx(g, rel=1e-5)
    assert lt.sigma == pytest.approx(R / (2 * g), rel=1e-5)
    assert lt.point == 1


@pytest.mark.parametrize("seed", range(3))
def test_point_light_frustum_holds_the_cube(orc, seed):
    """Every point of the cube falls inside the texel grid and the slice range."""
    rng = np.random.default_rng(90 + seed)
    lt = orc.point_light_setup(random_light_pos(rng, 1.0, 1.5), 20, 32)
    pts = np.vstack([np.array([[(c >> b) & 1 for b in range(3)] for c in range(8)], float),
                     rng.uniform(0, 1, size=(500, 3))])
    for X in pts:
        lam, tu, tv = orc.light_coords(lt, X)
        assert -1e-3 <= lam <= 20 + 1e-3
        assert -0.5 - 1e-3 <= tu <= 31.5 + 1e-3 and -0.5 - 1e-3 <= tv <= 31.5 + 1e-3


@pytest.mark.parametrize("seed", range(3))
def test_point_light_texel_round_trip(orc, seed):
    """The point of texel (i, j) on slice k maps back to (k, i, j)."""
    rng = np.random.default_rng(100 + seed)
    n, R = 25, 40
    lt = orc.point_light_setup(random_light_pos(rng), n, R)
    for _ in range(200):
        i, j, k = (int(x) for x in (rng.integers(R), rng.integers(R), rng.integers(n)))
        X = orc.texel_world(lt, i, j, k)
        lam, tu, tv = orc.light_coords(lt, X)
        assert abs(lam - k) < 1e-3 and abs(tu - i) < 1e-3 and abs(tv - j) < 1e-3


@pytest.mark.parametrize("seed", range(3))
def test_point_light_homogeneous_cube_counts_planes_on_each_ray(orc, seed):
    """Homogeneous cube: B_k of a column is (1 - a)^m, m the planes j < k whose
    depth lies between where the column's ray enters and leaves the cube
    (ray-box intersection in FP64)."""
    a = f32(0.2)
    N = 8
    vol = np.full((N, N, N), 200, np.uint8)
    tf = step_tf(256, [(100, 256, (1, 1, 1, a))])
    rng = np.random.default_rng(110 + seed)
    n, R = 37, 16
    lt = orc.point_light_setup(random_light_pos(rng, 1.1, 2.0), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    P = np.array(lt.P[:], float)
    L, U, V = (np.array(x[:], float) for x in (lt.L, lt.U, lt.V))
    g = lt.h
    d = lt.min + np.arange(n) * (lt.max - lt.min) / n
    checked = 0
    for j in range(R):
        for i in range(R):
            u = (2 * (i + 0.5) / R - 1) * g
            v = (2 * (j + 0.5) / R - 1) * g
            w = L + u * U + v * V
            with np.errstate(divide="ignore"):
                t0 = (0.0 - P) / w
                t1 = (1.0 - P) / w
            lo, hi = np.minimum(t0, t1).max(), np.maximum(t0, t1).min()
            if lo > hi:
                inside = np.zeros(n, bool)
            else:
                if np.any(np.abs(d - lo) < 1e-5) or np.any(np.abs(d - hi) < 1e-5):
                    continue
                inside = (d >= lo) & (d <= hi)
            m = np.concatenate([[0], np.cumsum(inside)[:-1]])
            assert np.abs(B[:, j, i] - (1 - a) ** m).max() < 1e-12
            checked += 1
    assert checked > R * R // 2


def test_point_light_plate_shadow_grows_by_similar_triangles(orc):
    """Light at height 2.5 above an opaque plate (half width 0.1, z in
    [0.5625, 0.625]) over a receiver slab (z in [0.125, 0.25]); camera below.
    The plate's umbra on the receiver's top face is the plate scaled by
    (2.5 - 0.25) / (2.5 - 0.5625) (from its lower face): receiver pixels well
    inside get no light, pixels well outside get the unshadowed closed form.
    A directional light would give half width 0.1 instead of 0.116."""
    N, a = 64, f32(0.25)
    vol = np.zeros((N, N, N), np.uint8)
    vol[36:40, 26:38, 26:38] = 255            # plate: x, y in [0.40625, 0.59375]
    vol[8:16] = 100                            # receiver: z in [0.125, 0.25]
    tf = step_tf(256, [(50, 151, (1, 1, 1, a)), (200, 256, (0, 0, 0, 1.0))])
    ramp = np.linspace(0, 1, 51)[1:-1]
    tf[151:200, :3] = (1 - ramp)[:, None]
    tf[151:200, 3] = a + (1 - a) * ramp
    n, R = 128, 256
    lt = orc.point_light_setup((0.5, 0.5, 2.5), n, R)
    B = orc.build_stack(vol, tf, 0, 255, lt)
    W = 128
    c = cam((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), False, 40, 0.5 / W)  # 1 x 1 frame
    img, *_ = orc.render_image(vol, tf, 0, 255, lt, B, c, W, 1,
                               orc.render_opts(orc.SHADOW, 0.5))
    xs = (np.arange(W) + 0.5) / W
    # The camera looks along +z with up +y: image x runs along -x of the world.
    half_plate = (38 - 26) / 2 / N              # 0.09375
    umbra = half_plate * (2.5 - 0.25) / (2.5 - 40 / N)
    penumbra = half_plate * (2.5 - 0.125) / (2.5 - 36 / N)
    dist = np.abs(xs - 0.5)
    dark = dist < umbra - 0.02
    lit = (dist > penumbra + 0.02) & (dist < 0.45)
    assert dark.sum() > 10 and lit.sum() > 10
    assert np.all(img[0, dark, :3] < 1e-3 * img[0, lit, :3].max())
    # Lit receiver: 17 samples z = i/128, i = 16..32 (first seen: i = 16); the
    # planes are z = 1 - j/128, so sample i sits on plane 128 - i and receives
    # the light through the 32 - i receiver planes above it:
    # C = sum_s a (1 - a)^s (1 - a)^(16 - s) = 17 a (1 - a)^16.
    assert np.allclose(img[0, lit, :3], 17 * a * (1 - a) ** 16, atol=1e-12)
    # Between 0.1 and the umbra edge a directional light would already be lit.
    between = (dist > half_plate + 0.005) & (dist < umbra - 0.005)
    assert between.sum() >= 2 and np.all(img[0, between, :3] < 1e-3 * img[0, lit, :3].max())


@pytest.mark.parametrize("mode", ["shadow", "shell", "cone"])
def test_point_light_far_away_approaches_directional(orc, mode):
    """A light 2000 units away along -L gives nearly the directional frame."""
    vol, tf, vmin, vmax = blob_scene(N=24)
    tf[:, 3] *= 4.0
    L = unit((0.3, -0.4, 0.87))
    n, R = 24, 48
    md = {"shadow": orc.SHADOW, "shell": orc.SHELL, "cone": orc.CONE}[mode]
    ro = orc.render_opts(md, 0.5)
    c = cam((2.2, 1.9, 1.4), (0.5, 0.5, 0.5), (0, 0, 1), True, 40, 0.5)
    ltd = orc.light_setup(L, n, R)
    ltp = orc.point_light_setup(0.5 - 2000.0 * L, n, R)
    Bd = orc.build_stack(vol, tf, vmin, vmax, ltd)
    Bp = orc.build_stack(vol, tf, vmin, vmax, ltp)
    imd, *_ = orc.render_image(vol, tf, vmin, vmax, ltd, Bd, c, 24, 20, ro)
    imp, *_ = orc.render_image(vol, tf, vmin, vmax, ltp, Bp, c, 24, 20, ro)
    # The columns of the far light still tilt by up to g = 4e-4: about 0.02
    # voxel of drift across the cube, so steep edges differ by up to ~0.015.
    assert np.abs(Bd - Bp).mean() < 2e-4 and np.abs(Bd - Bp).max() < 0.03
    assert np.abs(imd - imp).mean() < 2e-4 and np.abs(imd - imp).max() < 0.01
    assert imd[..., 3].max() > 0.2


@pytest.mark.parametrize("seed", range(4))
def test_point_light_scattering_points(orc, seed):
    """Shell points are S +- q r e_a; cone ring n is centred n dL from S
    towards the light, its four points lie at radius n dL tan(phi) in the plane
    orthogonal to the light direction at S, a quarter turn apart, the first
    one towards the eye."""
    rng = np.random.default_rng(120 + seed)
    lt = orc.point_light_setup(random_light_pos(rng), 40, 64)
    S = rng.uniform(0.1, 0.9, size=3)
    d = unit(rng.normal(size=3))
    Nmax = 48
    sh = orc.point_neighbours(lt, orc.render_opts(orc.SHELL, 0.5, shell_radius_vox=1.5,
                                                  shell_count=2), Nmax, S, d)
    assert sh.shape == (12, 3)
    for q in (1, 2):
        for a in range(3):
            for sgn, s in enumerate((1.0, -1.0)):
                want = np.array(S, np.float32).astype(float)
                want[a] += s * q * 1.5 / Nmax
                assert np.allclose(sh[6 * (q - 1) + 2 * a + sgn], want, atol=1e-6)
    phi = 20.0
    co = orc.point_neighbours(lt, orc.render_opts(orc.CONE, 0.5, cone_half_angle_deg=phi),
                              Nmax, S, d)
    assert co.shape == (8, 3)
    P = np.array(lt.P[:], float)
    w = unit(S - P)
    toward_eye = -d - (-d @ w) * w
    for ring in (1, 2):
        dist = ring * lt.dL
        centre = S - dist * w
        pts = co[4 * (ring - 1):4 * ring].astype(float) - centre
        assert np.allclose(np.linalg.norm(pts, axis=1), dist * math.tan(math.radians(phi)),
                           rtol=1e-4)
        assert np.allclose(pts @ w, 0.0, atol=1e-6)
        assert abs(pts[0] @ pts[1]) < 1e-8 and np.allclose(pts[2], -pts[0], atol=1e-6)
        assert np.allclose(np.cross(w, pts[0]), pts[1], atol=1e-6)   # quarter turn about w
        assert pts[0] @ toward_eye > 0


def test_point_light_rejects_positions_inside_its_sphere(orc):
    for P in ((0.5, 0.5, 0.5), (0.5, 0.5, 1.4), (1.2, 0.9, 0.5), (np.nan, 0, 2)):
        with pytest.raises(ValueError):
            orc.point_light_setup(P, 8, 8)
    orc.point_light_setup((0.5, 0.5, 1.5), 8, 8)
