"""Seeded synthetic inputs: volumes, transfer functions, lights and cameras.

This module only draws and shapes input data. It holds none of the rendering
method's arithmetic (no slicing, no attenuation, no compositing), so both the
CUDA path and the FP64 oracle can take their inputs from it.

The volumes stand in for the paper's CT datasets (*Engine*, *Foot*, 256^3, 8 bit;
Section 4), which are not available here:

* ``gaussian_blobs`` -- a sum of isotropic Gaussian blobs plus uniform noise.
* ``ct_phantom``     -- nested ellipsoids (soft tissue ~1000, bone ~3000) with
  Gaussian noise, rotated by a random quaternion; a CT-like 16-bit phantom.

All draws use ``numpy.random.default_rng`` (PCG64) with a fixed draw order, so
a seed fixes every value.  Volumes are stored z-major: ``vol[z, y, x]`` with x
fastest, the layout the library and the oracle both read.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Scattering modes and storage formats, by the names the library uses.
MODE_NONE, MODE_SHADOW, MODE_SHELL, MODE_CONE = 0, 1, 2, 3
FMT_F32, FMT_F16, FMT_BF16, FMT_UNORM16 = 0, 1, 2, 3


def _child(seed: int, stream: int) -> np.random.Generator:
    """Independent generator for one part of a scene (volume, TF, directions)."""
    return np.random.default_rng([int(seed), int(stream)])


def gaussian_blobs(n: int = 64, seed: int = 1, nblobs: int = 8,
                   sigma=(3.0, 10.0), peak: float = 200.0, noise=(0.0, 20.0),
                   dtype=np.uint8, sigma_scale: float = 1.0,
                   value_scale: float = 1.0) -> np.ndarray:
    """Sum of ``nblobs`` isotropic Gaussian blobs plus uniform noise.

    Draw order: centres ~ U[0, n)^3, sigmas ~ U[sigma] * sigma_scale, then one
    noise value per voxel ~ U[noise] (z, y, x order).  Blobs are evaluated at
    integer voxel coordinates.  Values are ``value_scale * (blobs + noise)``,
    rounded to nearest and clamped to the dtype's range.
    """
    rng = _child(seed, 0)
    centres = rng.uniform(0.0, float(n), size=(nblobs, 3))
    sig = rng.uniform(sigma[0], sigma[1], size=nblobs) * sigma_scale
    hi = float(np.iinfo(dtype).max)
    out = np.empty((n, n, n), dtype=dtype)
    idx = np.arange(n, dtype=np.float64)
    # One z-slab at a time keeps the working set small for 512^3 and up.
    slab = max(1, min(n, (1 << 24) // (n * n)))
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        acc = np.zeros((z1 - z0, n, n), dtype=np.float64)
        for b in range(nblobs):
            cx, cy, cz = centres[b]
            s2 = 2.0 * sig[b] * sig[b]
            gx = np.exp(-(idx - cx) ** 2 / s2)
            gy = np.exp(-(idx - cy) ** 2 / s2)
            gz = np.exp(-(idx[z0:z1] - cz) ** 2 / s2)
            acc += peak * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        acc += rng.uniform(noise[0], noise[1], size=acc.shape)
        acc *= value_scale
        out[z0:z1] = np.clip(np.rint(acc), 0.0, hi).astype(dtype)
    return out


def _quaternion_matrix(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def ct_phantom(n: int = 256, seed: int = 2, noise_sigma: float = 30.0,
               dtype=np.uint16) -> np.ndarray:
    """CT-like phantom of nested ellipsoids.

    An outer ellipsoid (semi-axes 0.45, 0.38, 0.30 of n) of soft tissue with a
    mean drawn from U[950, 1050] holds three bone ellipsoids (semi-axes 0.15-0.3
    of the outer ones, means U[2900, 3100]).  Background 0.  Gaussian noise of
    sigma ``noise_sigma`` is added to every voxel, then values are clamped at 0
    and rounded.  The whole phantom is rotated by a uniform random quaternion.

    Draw order: quaternion (4 normals), soft mean, then per bone: centre offset
    (3), semi-axis scales (3), mean; then the noise field (z, y, x order).
    """
    rng = _child(seed, 0)
    rot = _quaternion_matrix(rng.normal(size=4))
    soft = rng.uniform(950.0, 1050.0)
    outer = np.array([0.45, 0.38, 0.30]) * n
    bones = []
    for _ in range(3):
        off = rng.uniform(-0.4, 0.4, size=3) * outer
        ax = outer * rng.uniform(0.15, 0.30, size=3)
        bones.append((off, ax, rng.uniform(2900.0, 3100.0)))
    hi = float(np.iinfo(dtype).max)
    out = np.empty((n, n, n), dtype=dtype)
    c = np.arange(n, dtype=np.float64) + 0.5 - 0.5 * n
    slab = max(1, min(n, (1 << 22) // (n * n)))
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        Z, Y, X = np.meshgrid(c[z0:z1], c, c, indexing="ij")
        # Coordinates in the phantom's own frame: q = rot^T p.
        qx = rot[0, 0] * X + rot[1, 0] * Y + rot[2, 0] * Z
        qy = rot[0, 1] * X + rot[1, 1] * Y + rot[2, 1] * Z
        qz = rot[0, 2] * X + rot[1, 2] * Y + rot[2, 2] * Z
        val = np.zeros(X.shape, dtype=np.float64)
        inside = (qx / outer[0]) ** 2 + (qy / outer[1]) ** 2 + (qz / outer[2]) ** 2 <= 1.0
        val[inside] = soft
        for off, ax, bone in bones:
            m = (((qx - off[0]) / ax[0]) ** 2 + ((qy - off[1]) / ax[1]) ** 2
                 + ((qz - off[2]) / ax[2]) ** 2) <= 1.0
            val[m] = bone
        val += rng.normal(0.0, noise_sigma, size=val.shape)
        out[z0:z1] = np.clip(np.rint(val), 0.0, hi).astype(dtype)
    return out


def ct_phantom_device(n: int = 1024, seed: int = 5, noise_sigma: float = 30.0,
                      device: str = "cuda"):
    """The CT ellipsoid phantom of ``ct_phantom`` for large n, built on a CUDA
    device with torch (2 GiB at n = 1024 is minutes of numpy).

    Geometry (rotation, soft-tissue mean, bones) is drawn exactly as in
    ``ct_phantom``; the ellipsoid tests run in float32, and the noise of z-slab
    s (64 slices) comes from a torch CUDA generator seeded with
    1000 * seed + s.  Values are rounded and clamped to [0, 65535].  Returns an
    int16 torch tensor on ``device`` holding the uint16 bits (the values
    therefore differ from ``ct_phantom(n, seed)``; the distribution does not).
    """
    import torch
    rng = _child(seed, 0)
    rot = _quaternion_matrix(rng.normal(size=4))
    soft = rng.uniform(950.0, 1050.0)
    outer = np.array([0.45, 0.38, 0.30]) * n
    bones = []
    for _ in range(3):
        off = rng.uniform(-0.4, 0.4, size=3) * outer
        ax = outer * rng.uniform(0.15, 0.30, size=3)
        bones.append((off, ax, rng.uniform(2900.0, 3100.0)))
    out = torch.empty((n, n, n), dtype=torch.int16, device=device)
    c = torch.arange(n, dtype=torch.float32, device=device) + (0.5 - 0.5 * n)
    X = c.view(1, 1, n)
    Y = c.view(1, n, 1)
    R = [[float(rot[i, j]) for j in range(3)] for i in range(3)]
    slab = 64
    for s in range((n + slab - 1) // slab):
        z0, z1 = s * slab, min(n, (s + 1) * slab)
        Z = c[z0:z1].view(-1, 1, 1)
        # Coordinates in the phantom's own frame: q = rot^T p.
        qx = R[0][0] * X + R[1][0] * Y + R[2][0] * Z
        qy = R[0][1] * X + R[1][1] * Y + R[2][1] * Z
        qz = R[0][2] * X + R[1][2] * Y + R[2][2] * Z
        val = torch.zeros_like(qx)
        inside = (qx / outer[0]) ** 2 + (qy / outer[1]) ** 2 + (qz / outer[2]) ** 2 <= 1.0
        val[inside] = soft
        for off, ax, bone in bones:
            m = (((qx - off[0]) / ax[0]) ** 2 + ((qy - off[1]) / ax[1]) ** 2
                 + ((qz - off[2]) / ax[2]) ** 2) <= 1.0
            val[m] = bone
        gen = torch.Generator(device=device)
        gen.manual_seed(1000 * seed + s)
        val += noise_sigma * torch.randn(val.shape, generator=gen, device=device)
        u = torch.clamp(torch.round(val), 0.0, 65535.0).to(torch.int32)
        out[z0:z1] = (u - 65536 * (u >= 32768).to(torch.int32)).to(torch.int16)
    return out


def tf_random_pl(M: int = 256, seed: int = 1, npoints: int = 4,
                 alpha_max: float = 0.1) -> np.ndarray:
    """Random piecewise-linear RGBA transfer function with ``M`` entries.

    ``npoints`` control points at sorted U[0, M-1] positions, RGB ~ U[0, 1],
    alpha ~ U[0, alpha_max].  Alpha is 0 left of the first point; every channel
    is constant right of the last.  Straight (not premultiplied) colour.
    """
    rng = _child(seed, 1)
    pos = np.sort(rng.uniform(0.0, M - 1.0, size=npoints))
    rgb = rng.uniform(0.0, 1.0, size=(npoints, 3))
    a = rng.uniform(0.0, alpha_max, size=npoints)
    e = np.arange(M, dtype=np.float64)
    tf = np.empty((M, 4), dtype=np.float64)
    for ch in range(3):
        tf[:, ch] = np.interp(e, pos, rgb[:, ch])
    tf[:, 3] = np.interp(e, pos, a, left=0.0)
    return tf.astype(np.float32)


def tf_ct(M: int = 4096, seed: int = 2, vmax: float = 4095.0) -> np.ndarray:
    """CT-style transfer function over [0, vmax] with ``M`` entries.

    Alpha is 0 below ~500, ~0.02 over soft tissue (900-1100, warm colour), 0
    again around 1400, and ramps to ~0.3 for bone (2700-3300, white).  The
    control-point positions are jittered by U[-20, 20] from the seed.
    """
    rng = _child(seed, 1)
    base = np.array([0.0, 500.0, 900.0, 1100.0, 1400.0, 2700.0, 3300.0, vmax])
    jit = rng.uniform(-20.0, 20.0, size=base.size)
    jit[0] = 0.0
    jit[-1] = 0.0
    pos = np.sort(base + jit)
    alpha = np.array([0.0, 0.0, 0.02, 0.02, 0.0, 0.3, 0.3, 0.3])
    r = np.array([0.0, 0.8, 0.9, 0.9, 0.9, 1.0, 1.0, 1.0])
    g = np.array([0.0, 0.4, 0.6, 0.6, 0.7, 1.0, 1.0, 1.0])
    b = np.array([0.0, 0.3, 0.5, 0.5, 0.6, 1.0, 1.0, 1.0])
    v = np.arange(M, dtype=np.float64) * (vmax / (M - 1))
    tf = np.stack([np.interp(v, pos, ch) for ch in (r, g, b, alpha)], axis=1)
    return tf.astype(np.float32)


def random_direction(rng: np.random.Generator) -> np.ndarray:
    """Uniform direction on the unit sphere (normalised Gaussian triple)."""
    while True:
        d = rng.normal(size=3)
        nrm = np.linalg.norm(d)
        if nrm > 1e-6:
            return (d / nrm).astype(np.float32)


@dataclasses.dataclass
class Camera:
    """Pinhole (perspective) or orthographic camera in unit-cube coordinates."""
    eye: tuple
    target: tuple
    up: tuple
    perspective: bool
    fovy_deg: float = 40.0
    ortho_half_height: float = 0.8660254

    def as_tuple(self):
        return (tuple(map(float, self.eye)), tuple(map(float, self.target)),
                tuple(map(float, self.up)), int(self.perspective),
                float(self.fovy_deg), float(self.ortho_half_height))


def orbit_camera(view_dir: np.ndarray, perspective: bool, distance: float,
                 fovy_deg: float = 40.0, ortho_half_height: float = 0.8660254) -> Camera:
    """Camera looking along ``view_dir`` at the cube centre from ``distance``."""
    f = np.asarray(view_dir, dtype=np.float64)
    f = f / np.linalg.norm(f)
    c = np.array([0.5, 0.5, 0.5])
    eye = c - distance * f
    up = np.array([0.0, 0.0, 1.0]) if abs(f[2]) < 0.9 else np.array([0.0, 1.0, 0.0])
    return Camera(tuple(eye.astype(np.float32)), (0.5, 0.5, 0.5), tuple(up),
                  perspective, fovy_deg, ortho_half_height)


@dataclasses.dataclass
class Scene:
    """Everything one frame needs: volume, TF, light, stack shape, camera."""
    name: str
    volume: np.ndarray
    tf: np.ndarray
    vmin: float
    vmax: float
    light_dir: np.ndarray
    light_color: tuple
    n_slices: int
    slice_res: int
    mode: int
    camera: Camera
    width: int
    height: int
    step_vox: float
    ert: float
    bg: tuple = (0.0, 0.0, 0.0, 0.0)
    fmt: int = FMT_F32
    cone_half_angle_deg: float = 15.0
    shell_radius_vox: float = 1.0

    @property
    def dtype_code(self) -> int:
        return 0 if self.volume.dtype == np.uint8 else 1


def blob64_shell(seed: int = 1, ert: float = 2.0) -> Scene:
    """64^3 uint8 Gaussian blobs, 256-entry random TF, 64 light slices of
    128x128, 256x256 orthographic view, step 0.5 voxel, shell scattering."""
    vol = gaussian_blobs(64, seed)
    tf = tf_random_pl(256, seed)
    drng = _child(seed, 2)
    light = random_direction(drng)
    view = random_direction(drng)
    cam = orbit_camera(view, perspective=False, distance=2.0)
    return Scene("blob64-u8 shell 64x128^2 256^2-ortho", vol, tf, 0.0, 255.0, light,
                 (1.0, 1.0, 1.0), 64, 128, MODE_SHELL, cam, 256, 256, 0.5, ert)


def ct256_cone(seed: int = 2, n: int = 256, ert: float = 0.99) -> Scene:
    """256^3 uint16 CT-like ellipsoid phantom, 4096-entry TF, 256 light slices of
    512x512, cone scattering (15 deg), 1024x1024 perspective (eye 2.6 from the
    centre, fovy 40 deg), step 0.5 voxel, early ray termination at 0.99."""
    vol = ct_phantom(n, seed)
    tf = tf_ct(4096, seed)
    drng = _child(seed, 2)
    light = random_direction(drng)
    view = random_direction(drng)
    cam = orbit_camera(view, perspective=True, distance=2.6, fovy_deg=40.0)
    return Scene(f"ct{n}-u16 cone15 256x512^2 1024^2-persp", vol, tf, 0.0, 4095.0, light,
                 (1.0, 1.0, 1.0), 256, 512, MODE_CONE, cam, 1024, 1024, 0.5, ert)


def blob512_precision(seed: int = 3, n: int = 512, mode: int = MODE_CONE) -> Scene:
    """512^3 uint16 Gaussian-blob phantom (the 64^3 generator scaled: sigma x 8,
    centres in [0, 512), values x 256), the 256-entry random TF over [0, 65535],
    512 light slices of 1024x1024, 1920x1080 perspective, step 0.5 voxel."""
    vol = gaussian_blobs(n, seed, sigma_scale=n / 64.0, dtype=np.uint16, value_scale=256.0)
    tf = tf_random_pl(256, seed)
    drng = _child(seed, 2)
    light = random_direction(drng)
    view = random_direction(drng)
    cam = orbit_camera(view, perspective=True, distance=2.6, fovy_deg=40.0)
    return Scene(f"blob{n}-u16 512x1024^2 1920x1080-persp", vol, tf, 0.0, 65535.0, light,
                 (1.0, 1.0, 1.0), 512, 1024, mode, cam, 1920, 1080, 0.5, 2.0)


def ct1024_large(seed: int = 5, n: int = 1024) -> Scene:
    """1024^3 uint16 CT ellipsoid phantom (2 GiB, built on the CUDA device),
    the 4096-entry CT TF, 1024 light slices of 2048 x 2048 stored FP16 (8 GiB),
    cone scattering (15 deg), 3840 x 2160 perspective (eye 2.6 from the centre,
    fovy 40 deg), step 0.5 voxel, early ray termination at 0.99."""
    vol = ct_phantom_device(n, seed).cpu().numpy().view(np.uint16)
    tf = tf_ct(4096, seed)
    drng = _child(seed, 2)
    light = random_direction(drng)
    view = random_direction(drng)
    cam = orbit_camera(view, perspective=True, distance=2.6, fovy_deg=40.0)
    return Scene(f"ct{n}-u16 cone15 1024x2048^2-f16 3840x2160-persp", vol, tf, 0.0, 4095.0,
                 light, (1.0, 1.0, 1.0), 1024, 2048, MODE_CONE, cam, 3840, 2160, 0.5, 0.99,
                 fmt=FMT_F16)


def unit(v) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    return v / math.sqrt(float(v @ v))


# ---- Serving mix: many volumes, a stream of requests -------------------------

SERVING_SIZES = ((256, 256), (512, 512), (1024, 768), (1280, 720), (1920, 1080))


@dataclasses.dataclass
class ServedVolume:
    """One registered volume of the serving mix with its transfer function."""
    name: str
    n: int
    kind: str          # "blob-u8" or "ellipsoid-u16"
    seed: int
    tf: np.ndarray
    vmin: float
    vmax: float

    def generate(self) -> np.ndarray:
        if self.kind == "blob-u8":
            return gaussian_blobs(self.n, self.seed, sigma_scale=self.n / 64.0)
        return ct_phantom(self.n, self.seed)


def serving_volumes(seed: int = 4) -> list:
    """The volumes of the serving mix: {128, 256, 512}^3 x {uint8 Gaussian
    blobs with a 256-entry random TF, uint16 CT ellipsoids with the 4096-entry
    CT TF}, plus a second 128^3 blob and 256^3 ellipsoid (8 volumes, so that a
    residency limit of 6 forces evictions).  Volumes are generated on demand
    (``generate``); each has its own seed derived from ``seed``."""
    out = []
    specs = [(128, "blob-u8"), (128, "ellipsoid-u16"), (256, "blob-u8"), (256, "ellipsoid-u16"),
             (512, "blob-u8"), (512, "ellipsoid-u16"), (128, "blob-u8"), (256, "ellipsoid-u16")]
    for i, (n, kind) in enumerate(specs):
        s = 100 * seed + i
        if kind == "blob-u8":
            out.append(ServedVolume(f"blob{n}-u8#{i}", n, kind, s, tf_random_pl(256, s), 0.0,
                                    255.0))
        else:
            out.append(ServedVolume(f"ct{n}-u16#{i}", n, kind, s, tf_ct(4096, s), 0.0, 4095.0))
    return out


def serving_requests(n_volumes: int, count: int = 512, rate_per_s: float = 300.0,
                     seed: int = 4) -> list:
    """``count`` render requests with Poisson arrivals at ``rate_per_s``.

    Each request draws, in this order: the inter-arrival gap ~ Exp(rate), the
    volume uniformly, the image size from SERVING_SIZES, the slice count from
    {64, 128, 256, 512}, the slice resolution from {256, 512}, the mode from
    {shadow, shell, cone}, and the light and view directions uniformly on the
    sphere (perspective camera 2.6 from the centre, fovy 40 deg).  Step 0.5
    voxel, early ray termination at 0.99."""
    rng = _child(seed, 3)
    t = 0.0
    reqs = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        vol = int(rng.integers(n_volumes))
        W, H = SERVING_SIZES[int(rng.integers(len(SERVING_SIZES)))]
        n = int((64, 128, 256, 512)[rng.integers(4)])
        R = int((256, 512)[rng.integers(2)])
        mode = int((MODE_SHADOW, MODE_SHELL, MODE_CONE)[rng.integers(3)])
        light = random_direction(rng)
        cam = orbit_camera(random_direction(rng), perspective=True, distance=2.6, fovy_deg=40.0)
        reqs.append(dict(arrival_s=t, volume=vol, width=W, height=H, n_slices=n, slice_res=R,
                         mode=mode, light_dir=light, camera=cam, step_vox=0.5, ert=0.99))
    return reqs
