"""FP64 CPU oracle of slice-based illuminated ray casting (ctypes wrapper).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The
library (``paper_2008_06134_gb300``) never imports it and has no CPU path.

The arithmetic lives in ``vi_oracle.c``; this module compiles it with the host
C compiler (``build()``) and marshals numpy arrays.  Functions whose result
no closed form, invariant or brute-force check pins are listed as "parity
unpinned" here and in the design notes; at present there are none.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vi_oracle.c")
_LIB = os.path.join(_HERE, "libvi_oracle.so")
_lock = threading.Lock()
_lib = None

TRACE_WORDS = 40
TRACE_NONE = 0x7FFFFFFF
NONE, SHADOW, SHELL, CONE = 0, 1, 2, 3
TRANSMITTANCE, OPTICAL_DEPTH = 0, 1      # what the attenuation buffer holds
SLICE_NEAREST, SLICE_LINEAR = 0, 1      # slice filtering of a lookup
DEPTH_MAX = 64.0                         # cap of a stored optical depth
MAX_SHELLS = 4
MAX_NB = 6 * MAX_SHELLS


def build(force: bool = False) -> str:
    """Compile ``vi_oracle.c`` into ``libvi_oracle.so`` (in place)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cc = os.environ.get("CC", "cc")
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("nx", C.c_int),
                ("ny", C.c_int), ("nz", C.c_int)]


class TF(C.Structure):
    _fields_ = [("rgba", C.c_void_p), ("M", C.c_int), ("vmin", C.c_float),
                ("vmax", C.c_float)]


class Light(C.Structure):
    _fields_ = [("L", C.c_float * 3), ("min", C.c_float), ("max", C.c_float),
                ("dL", C.c_float), ("kappa", C.c_float), ("Lc", C.c_float),
                ("U", C.c_float * 3), ("V", C.c_float * 3), ("h", C.c_float),
                ("sigma", C.c_float), ("rho0", C.c_float), ("n", C.c_int),
                ("R", C.c_int), ("axis", C.c_int), ("point", C.c_int),
                ("P", C.c_float * 3)]


class BuildOpts(C.Structure):
    _fields_ = [("opacity_correction", C.c_int), ("comp_n", C.c_float), ("quantity", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("perspective", C.c_int), ("fovy_deg", C.c_float),
                ("ortho_half_height", C.c_float)]


class RenderOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("ert", C.c_float), ("bg", C.c_float * 4),
                ("color", C.c_float * 3), ("ambient", C.c_float), ("step_vox", C.c_float),
                ("opacity_correction", C.c_int), ("cone_half_angle_deg", C.c_float),
                ("shell_radius_vox", C.c_float), ("ert_band", C.c_double),
                ("quantity", C.c_int), ("slice_filter", C.c_int), ("shell_count", C.c_int)]


class Frame(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("f", C.c_float * 3), ("r", C.c_float * 3),
                ("u", C.c_float * 3), ("sx", C.c_float), ("sy", C.c_float), ("dt", C.c_float),
                ("perspective", C.c_int), ("W", C.c_int), ("H", C.c_int), ("Nmax", C.c_int)]


class Ray(C.Structure):
    _fields_ = [("hit", C.c_int), ("o", C.c_float * 3), ("d", C.c_float * 3),
                ("t0", C.c_float), ("t1", C.c_float), ("lo", C.c_float * 3),
                ("ld", C.c_float * 3), ("nnb", C.c_int), ("nb", (C.c_float * 3) * MAX_NB)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # VI_ORACLE_LIB points at another build of vi_oracle.c; the mutation
            # tests use it to load copies with a planted mistake.
            path = os.environ.get("VI_ORACLE_LIB") or build()
            L = C.CDLL(path)
            P = C.POINTER
            L.orc_light_setup.argtypes = [P(C.c_float), C.c_int, C.c_int, P(Light)]
            L.orc_build_stack.argtypes = [P(Volume), P(TF), P(Light), P(BuildOpts), C.c_void_p]
            L.orc_build_stack_rows.argtypes = [P(Volume), P(TF), P(Light), P(BuildOpts), C.c_int,
                                               C.c_int, C.c_void_p]
            L.orc_frame_setup.argtypes = [P(Camera), C.c_int, C.c_int, C.c_float, C.c_int, P(Frame)]
            L.orc_ray_setup.argtypes = [P(Light), P(Frame), P(RenderOpts), C.c_int, C.c_int, P(Ray)]
            L.orc_light_coords.argtypes = [P(Light), P(C.c_float), P(C.c_float)]
            L.orc_point_light_setup.argtypes = [P(C.c_float), C.c_int, C.c_int, P(Light)]
            L.orc_point_neighbours.argtypes = [P(Light), P(RenderOpts), C.c_int, P(C.c_float),
                                               P(C.c_float), P(C.c_float)]
            L.orc_render_pixels.argtypes = [P(Volume), P(TF), P(Light), C.c_void_p, P(Camera),
                                            C.c_int, C.c_int, P(RenderOpts), C.c_void_p,
                                            C.c_void_p, C.c_long, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p]
            L.orc_trace_pixel.argtypes = [P(Volume), P(TF), P(Light), C.c_void_p, P(Camera),
                                          C.c_int, C.c_int, P(RenderOpts), C.c_int, C.c_int,
                                          C.c_void_p, C.c_int, P(C.c_int)]
            L.orc_transmittance_bruteforce.argtypes = [P(Volume), P(TF), P(C.c_double),
                                                       P(C.c_double), C.c_long]
            L.orc_transmittance_bruteforce.restype = C.c_double
            L.orc_sample_volume.argtypes = [P(Volume), P(C.c_float), P(C.c_int)]
            L.orc_sample_volume.restype = C.c_double
            L.orc_tf_lookup.argtypes = [P(TF), C.c_double, P(C.c_double)]
            L.orc_tf_lookup.restype = None
            L.orc_texel_world.argtypes = [P(Light), C.c_int, C.c_int, C.c_int, P(C.c_float)]
            L.orc_stack_lookup.argtypes = [C.c_void_p, P(Light), C.c_float, C.c_float, C.c_float,
                                           P(C.c_int)]
            L.orc_stack_lookup.restype = C.c_double
            L.orc_light_lookup.argtypes = [C.c_void_p, P(Light), P(RenderOpts), C.c_float,
                                           C.c_float, C.c_float, P(C.c_int)]
            L.orc_light_lookup.restype = C.c_double
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_get_threads())


def _f3(v):
    return (C.c_float * 3)(*[float(x) for x in v])


# Keep-alive references for the buffers a Volume / TF points into.
class _Held:
    def __init__(self, struct, *bufs):
        self.struct = struct
        self.bufs = bufs


def volume(vol: np.ndarray) -> _Held:
    vol = np.ascontiguousarray(vol)
    if vol.dtype == np.uint8:
        code = 0
    elif vol.dtype == np.uint16:
        code = 1
    else:
        raise TypeError("volume must be uint8 or uint16")
    nz, ny, nx = vol.shape
    return _Held(Volume(vol.ctypes.data, code, nx, ny, nz), vol)


def transfer_function(rgba: np.ndarray, vmin: float, vmax: float) -> _Held:
    rgba = np.ascontiguousarray(rgba, dtype=np.float32)
    return _Held(TF(rgba.ctypes.data, rgba.shape[0], float(vmin), float(vmax)), rgba)


def light_setup(direction, n: int, R: int) -> Light:
    out = Light()
    rc = lib().orc_light_setup(_f3(direction), int(n), int(R), C.byref(out))
    if rc:
        raise ValueError(f"orc_light_setup rejected the input ({rc})")
    return out


def build_stack(vol: np.ndarray, tf: np.ndarray, vmin: float, vmax: float, light: Light,
                opacity_correction: int = 0, comp_n: float = 0.0,
                quantity: int = TRANSMITTANCE) -> np.ndarray:
    """Algorithm 1: the (n, R, R) attenuation buffer, binary64 (transmittances,
    or optical depths with ``quantity=OPTICAL_DEPTH``)."""
    V = volume(vol)
    T = transfer_function(tf, vmin, vmax)
    B = np.empty((light.n, light.R, light.R), dtype=np.float64)
    opts = BuildOpts(int(opacity_correction), float(comp_n), int(quantity))
    rc = lib().orc_build_stack(C.byref(V.struct), C.byref(T.struct), C.byref(light),
                               C.byref(opts), B.ctypes.data)
    if rc:
        raise ValueError(f"orc_build_stack failed ({rc})")
    return B


def build_stack_rows(vol, tf, vmin, vmax, light: Light, j0: int, j1: int, out: np.ndarray,
                     opacity_correction: int = 0, comp_n: float = 0.0,
                     quantity: int = TRANSMITTANCE) -> np.ndarray:
    """Algorithm 1 on texel rows [j0, j1) only, written into ``out`` (n, R, R)."""
    V = volume(vol)
    T = transfer_function(tf, vmin, vmax)
    assert out.dtype == np.float64 and out.flags.c_contiguous
    assert out.shape == (light.n, light.R, light.R)
    opts = BuildOpts(int(opacity_correction), float(comp_n), int(quantity))
    rc = lib().orc_build_stack_rows(C.byref(V.struct), C.byref(T.struct), C.byref(light),
                                    C.byref(opts), int(j0), int(j1), out.ctypes.data)
    if rc:
        raise ValueError(f"orc_build_stack_rows failed ({rc})")
    return out


def camera(cam) -> Camera:
    """Accepts a ``phantoms.Camera`` or an (eye, target, up, persp, fovy, hh) tuple."""
    t = cam.as_tuple() if hasattr(cam, "as_tuple") else cam
    eye, target, up, persp, fovy, hh = t
    return Camera(_f3(eye), _f3(target), _f3(up), int(persp), float(fovy), float(hh))


def render_opts(mode: int, step_vox: float, ert: float = 2.0, bg=(0, 0, 0, 0),
                color=(1, 1, 1), ambient: float = 0.0, opacity_correction: int = 0,
                cone_half_angle_deg: float = 15.0, shell_radius_vox: float = 1.0,
                ert_band: float = 1e-5, quantity: int = 0, slice_filter: int = 0,
                shell_count: int = 1) -> RenderOpts:
    return RenderOpts(int(mode), float(ert), (C.c_float * 4)(*map(float, bg)),
                      _f3(color), float(ambient), float(step_vox), int(opacity_correction),
                      float(cone_half_angle_deg), float(shell_radius_vox), float(ert_band),
                      int(quantity), int(slice_filter), int(shell_count))


def render_window(vol, tf, vmin, vmax, light: Light, stack, cam, W: int, H: int,
                  ro: RenderOpts, xs, ys):
    """Render the pixels (xs[i], ys[i]) of a W x H frame, with the early ray
    termination window of each (reading R12 of Eq. 3).

    Returns (rgba, alt, window, nsamples, nsamples_alt, end, nsamples_end):
    rgba, alt and end are (count, 4) float64, window (count,) uint8, the sample
    counts (count,) int64.  Where the accumulated opacity passes within
    ``ro.ert_band`` of the threshold a binary32 renderer may stop anywhere
    from the first sample with A > ert - band to the first with A > ert + band
    (or the ray's end).  window = 0: one outcome (alt = end = rgba); 1: two,
    rgba (the binary64 decision) and alt; 2: three or more, every stop from
    the window's start to ``end``, with rgba the binary64 decision and alt the
    window's start (or its end, if the decision is at the start).
    """
    V = volume(vol)
    T = transfer_function(tf, vmin, vmax)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    n = xs.size
    out = np.empty((n, 4), dtype=np.float64)
    alt = np.empty((n, 4), dtype=np.float64)
    amb = np.zeros(n, dtype=np.uint8)
    ns = np.zeros(n, dtype=np.int64)
    ns_alt = np.zeros(n, dtype=np.int64)
    end = np.empty((n, 4), dtype=np.float64)
    ns_end = np.zeros(n, dtype=np.int64)
    Bp = None
    if stack is not None:
        stack = np.ascontiguousarray(stack, dtype=np.float64)
        Bp = stack.ctypes.data
    cam_s = camera(cam)
    rc = lib().orc_render_pixels(C.byref(V.struct), C.byref(T.struct), C.byref(light), Bp,
                                 C.byref(cam_s), int(W), int(H), C.byref(ro), xs.ctypes.data,
                                 ys.ctypes.data, n, out.ctypes.data, alt.ctypes.data,
                                 amb.ctypes.data, ns.ctypes.data, ns_alt.ctypes.data,
                                 end.ctypes.data, ns_end.ctypes.data)
    if rc:
        raise ValueError(f"orc_render_pixels failed ({rc})")
    return out, alt, amb, ns, ns_alt, end, ns_end


def render_pixels(vol, tf, vmin, vmax, light: Light, stack, cam, W: int, H: int,
                  ro: RenderOpts, xs, ys):
    """Render the pixels (xs[i], ys[i]) of a W x H frame.

    Returns (rgba, alt, ambiguous, nsamples): rgba and alt are (count, 4)
    float64, ambiguous (count,) bool, nsamples (count,) int64.  ``ambiguous``
    marks pixels where early ray termination has more than one valid outcome
    (see ``render_window``); there ``alt`` holds the other end of the window.
    """
    out, alt, win, ns, *_ = render_window(vol, tf, vmin, vmax, light, stack, cam, W, H, ro,
                                          xs, ys)
    return out, alt, win.astype(bool), ns


def render_image(vol, tf, vmin, vmax, light, stack, cam, W, H, ro):
    """Whole W x H frame; returns (H, W, 4) rgba, (H, W, 4) alt, (H, W)
    ambiguous and (H, W) sample counts."""
    ys, xs = np.mgrid[0:H, 0:W]
    out, alt, amb, ns = render_pixels(vol, tf, vmin, vmax, light, stack, cam, W, H, ro,
                                      xs.ravel(), ys.ravel())
    return (out.reshape(H, W, 4), alt.reshape(H, W, 4), amb.reshape(H, W),
            ns.reshape(H, W))


def trace_pixel(vol, tf, vmin, vmax, light, stack, cam, W, H, ro, x, y, max_rec=8192):
    V = volume(vol)
    T = transfer_function(tf, vmin, vmax)
    rec = np.zeros((max_rec, TRACE_WORDS), dtype=np.int32)
    nrec = C.c_int(0)
    Bp = None
    if stack is not None:
        stack = np.ascontiguousarray(stack, dtype=np.float64)
        Bp = stack.ctypes.data
    cam_s = camera(cam)
    rc = lib().orc_trace_pixel(C.byref(V.struct), C.byref(T.struct), C.byref(light), Bp,
                               C.byref(cam_s), int(W), int(H), C.byref(ro), int(x), int(y),
                               rec.ctypes.data, max_rec, C.byref(nrec))
    if rc:
        raise ValueError(f"orc_trace_pixel failed ({rc})")
    return rec[: nrec.value].copy()


def frame_setup(cam, W, H, step_vox, nmax) -> Frame:
    fr = Frame()
    rc = lib().orc_frame_setup(C.byref(camera(cam)), int(W), int(H), float(step_vox),
                               int(nmax), C.byref(fr))
    if rc:
        raise ValueError("orc_frame_setup rejected the camera")
    return fr


def ray_setup(light: Light, frame: Frame, ro: RenderOpts, x: int, y: int) -> Ray:
    ray = Ray()
    lib().orc_ray_setup(C.byref(light), C.byref(frame), C.byref(ro), int(x), int(y),
                        C.byref(ray))
    return ray


def light_coords(light: Light, X) -> np.ndarray:
    """(lambda, tu, tv) of the world point X (binary32 index path)."""
    out = (C.c_float * 3)()
    lib().orc_light_coords(C.byref(light), _f3(X), out)
    return np.array(out[:], dtype=np.float32)


def point_light_setup(position, n: int, R: int) -> Light:
    """Frame of a point light at ``position`` (at least 1 from the cube centre)."""
    out = Light()
    rc = lib().orc_point_light_setup(_f3(position), int(n), int(R), C.byref(out))
    if rc:
        raise ValueError(f"orc_point_light_setup rejected the input ({rc})")
    return out


def point_neighbours(light: Light, ro: RenderOpts, nmax: int, S, d) -> np.ndarray:
    """World positions of a sample's shell / cone points under a point light."""
    out = (C.c_float * (3 * MAX_NB))()
    k = lib().orc_point_neighbours(C.byref(light), C.byref(ro), int(nmax), _f3(S), _f3(d), out)
    if k < 0:
        raise ValueError("orc_point_neighbours rejected the input")
    return np.array(out[: 3 * k], dtype=np.float32).reshape(k, 3)


def texel_world(light: Light, i: int, j: int, k: int) -> np.ndarray:
    out = (C.c_float * 3)()
    lib().orc_texel_world(C.byref(light), int(i), int(j), int(k), out)
    return np.array(out[:], dtype=np.float32)


def sample_volume(vol: np.ndarray, P):
    V = volume(vol)
    cell = (C.c_int * 3)()
    v = lib().orc_sample_volume(C.byref(V.struct), _f3(P), cell)
    return v, tuple(cell[:])


def tf_lookup(tf: np.ndarray, vmin: float, vmax: float, v: float) -> np.ndarray:
    T = transfer_function(tf, vmin, vmax)
    out = (C.c_double * 4)()
    lib().orc_tf_lookup(C.byref(T.struct), float(v), out)
    return np.array(out[:])


def light_lookup(stack, light: Light, ro: RenderOpts, lam, tu, tv):
    """One lookup's light factor under ``ro``'s slice filter and buffer quantity."""
    stack = np.ascontiguousarray(stack, dtype=np.float64)
    rec = (C.c_int * 3)()
    v = lib().orc_light_lookup(stack.ctypes.data, C.byref(light), C.byref(ro), float(lam),
                               float(tu), float(tv), rec)
    return v, tuple(rec[:])


def stack_lookup(stack, light: Light, lam, tu, tv):
    stack = np.ascontiguousarray(stack, dtype=np.float64)
    rec = (C.c_int * 3)()
    v = lib().orc_stack_lookup(stack.ctypes.data, C.byref(light), float(lam), float(tu),
                               float(tv), rec)
    return v, tuple(rec[:])


def transmittance_bruteforce(vol, tf, vmin, vmax, L, P, m: int = 20000) -> float:
    V = volume(vol)
    T = transfer_function(tf, vmin, vmax)
    Ld = (C.c_double * 3)(*map(float, L))
    Pd = (C.c_double * 3)(*map(float, P))
    return float(lib().orc_transmittance_bruteforce(C.byref(V.struct), C.byref(T.struct), Ld,
                                                     Pd, int(m)))


def render_scene(scene, xs=None, ys=None, ert_band: float = 1e-5, stack=None):
    """Convenience: sweep + eye pass for a ``phantoms.Scene`` on the oracle."""
    light = light_setup(scene.light_dir, scene.n_slices, scene.slice_res)
    if stack is None and scene.mode != NONE:
        stack = build_stack(scene.volume, scene.tf, scene.vmin, scene.vmax, light)
    ro = render_opts(scene.mode, scene.step_vox, scene.ert, scene.bg, scene.light_color,
                     cone_half_angle_deg=scene.cone_half_angle_deg,
                     shell_radius_vox=scene.shell_radius_vox, ert_band=ert_band)
    if xs is None:
        img, alt, amb, ns = render_image(scene.volume, scene.tf, scene.vmin, scene.vmax, light,
                                         stack, scene.camera, scene.width, scene.height, ro)
        return img, alt, amb, ns, stack, light
    out, alt, amb, ns = render_pixels(scene.volume, scene.tf, scene.vmin, scene.vmax, light,
                                      stack, scene.camera, scene.width, scene.height, ro, xs, ys)
    return out, alt, amb, ns, stack, light
