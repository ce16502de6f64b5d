"""Thin ctypes binding of the C ABI in ``include/vi.h``.

Argument marshalling only: every step of the method runs in ``libvi.so``'s
CUDA kernels.  Methods of :class:`Context` carry the C names without the
``vi_`` prefix (``load_volume`` is ``vi_load_volume`` and so on).  Device
buffers are passed as torch CUDA tensors (their ``data_ptr()``), host buffers
as numpy arrays.  There is no CPU path: if ``libvi.so`` is missing, loading
fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvi.so")
# The same library built with every kernel's memory indices checked
# (VI_DEBUG_BOUNDS=1; violations read with debug_bounds()).
LIB_CHECKED_PATH = os.path.join(HERE, "libvi_checked.so")

OK, EINVAL, ENOMEM, ESTATE, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4, -5
OUT_HOST, OUT_DEVICE, OUT_HOST_ASYNC = 0, 1, 2   # where vi_render's output lives
U8, U16 = 0, 1
NONE, SHADOW, SHELL, CONE = 0, 1, 2, 3
F32, F16, BF16, UNORM16 = 0, 1, 2, 3
TRANSMITTANCE, OPTICAL_DEPTH = 0, 1   # what the stack holds
SLICE_NEAREST, SLICE_LINEAR = 0, 1    # slice filtering of a lookup
DEPTH_MAX = 64.0
MAX_SHELLS = 4
TRACE_WORDS = 40
NOALLOC_MAX_PIXELS = 512 * 512
TRACE_NONE = 0x7FFFFFFF

# Every symbol include/vi.h declares, in order.
EXPORTS = ("vi_create", "vi_destroy", "vi_set_memory_budget", "vi_load_volume",
           "vi_set_transfer_function", "vi_set_light", "vi_set_point_light",
           "vi_build_attenuation", "vi_render", "vi_sync", "vi_error_string",
           "vi_attenuation_info", "vi_get_attenuation", "vi_trace_pixel", "vi_launch_count",
           "vi_measure_peaks", "vi_post_ready", "vi_render_batch", "vi_render_host_noalloc", "vi_debug_bounds", "vi_server_create", "vi_server_destroy",
           "vi_server_add_volume", "vi_server_submit", "vi_server_wait", "vi_server_cancel",
           "vi_server_timing", "vi_server_release", "vi_server_get_stats",
           "vi_server_set_graphs", "vi_server_set_batching", "vi_server_set_eviction",
           "vi_get_skip_grid")
EVICT_LRU, EVICT_COST = 0, 1
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4


class ViError(RuntimeError):
    def __init__(self, code: int, call: str):
        self.code = code
        super().__init__(f"{call}: {error_string(code)} ({code})")


class BuildOpts(C.Structure):
    _fields_ = [("format", C.c_int), ("cone_half_angle_deg", C.c_float),
                ("shell_radius_vox", C.c_float), ("opacity_correction", C.c_int),
                ("comp_n", C.c_float), ("quantity", C.c_int), ("shell_count", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("perspective", C.c_int), ("eye", C.c_float * 3), ("target", C.c_float * 3),
                ("up", C.c_float * 3), ("fovy_deg", C.c_float), ("ortho_half_height", C.c_float)]


class RenderOpts(C.Structure):
    _fields_ = [("ert", C.c_float), ("bg", C.c_float * 4), ("ambient", C.c_float),
                ("opacity_correction", C.c_int), ("sample_counts", C.c_void_p),
                ("lit_counts", C.c_void_p), ("slice_filter", C.c_int)]


class BatchFrame(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("camera", Camera), ("width", C.c_int),
                ("height", C.c_int), ("step_vox", C.c_float), ("out_rgba", C.c_void_p),
                ("opts", RenderOpts), ("status", C.c_int)]


class Request(C.Structure):
    _fields_ = [("volume_id", C.c_int), ("tf_rgba", C.c_void_p), ("tf_entries", C.c_int),
                ("tf_vmin", C.c_float), ("tf_vmax", C.c_float), ("light_dir", C.c_float * 3),
                ("light_color", C.c_float * 3), ("n_slices", C.c_int), ("slice_res", C.c_int),
                ("mode", C.c_int), ("build", BuildOpts), ("camera", Camera), ("width", C.c_int),
                ("height", C.c_int), ("step_vox", C.c_float), ("render", RenderOpts),
                ("out_rgba", C.c_void_p), ("out_on_device", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("cancelled", C.c_uint64), ("volume_loads", C.c_uint64),
                ("volume_evictions", C.c_uint64), ("queued", C.c_int), ("running", C.c_int),
                ("resident_volumes", C.c_int), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("stack_reuses", C.c_uint64),
                ("graph_launches", C.c_uint64), ("graph_instantiations", C.c_uint64),
                ("batches", C.c_uint64), ("batched_frames", C.c_uint64),
                ("volume_load_bytes", C.c_uint64)]


_libs = {}


def library(checked: bool = False) -> C.CDLL:
    """Load ``libvi.so``, or with ``checked`` ``libvi_checked.so`` (both built
    by ``python -m paper_2008_06134_gb300.build``)."""
    path = LIB_CHECKED_PATH if checked else LIB_PATH
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is not built; run `python -m paper_2008_06134_gb300.build` "
            "(needs nvcc) -- there is no CPU fallback")
    L = C.CDLL(path)
    P, vp, i, f, sz = C.POINTER, C.c_void_p, C.c_int, C.c_float, C.c_size_t
    L.vi_create.argtypes = [P(vp), i, vp]
    L.vi_destroy.argtypes = [vp]
    L.vi_set_memory_budget.argtypes = [vp, sz]
    L.vi_load_volume.argtypes = [vp, vp, i, i, i, i, i]
    L.vi_set_transfer_function.argtypes = [vp, vp, i, f, f]
    L.vi_set_light.argtypes = [vp, vp, vp]
    L.vi_set_point_light.argtypes = [vp, vp, vp]
    L.vi_build_attenuation.argtypes = [vp, i, i, i, P(BuildOpts)]
    L.vi_render.argtypes = [vp, P(Camera), i, i, f, vp, i, P(RenderOpts)]
    L.vi_sync.argtypes = [vp]
    L.vi_error_string.argtypes = [i]
    L.vi_error_string.restype = C.c_char_p
    L.vi_attenuation_info.argtypes = [vp, P(i), P(i), P(i), P(sz)]
    L.vi_get_attenuation.argtypes = [vp, vp, sz, i]
    L.vi_trace_pixel.argtypes = [vp, P(Camera), i, i, f, P(RenderOpts), i, i, vp, i, P(i)]
    L.vi_launch_count.argtypes = [vp, P(C.c_uint64)]
    L.vi_get_skip_grid.argtypes = [vp, P(i), vp, sz, vp, sz]
    L.vi_render_host_noalloc.argtypes = [vp, P(Camera), i, i, f, vp, P(RenderOpts)]
    L.vi_post_ready.argtypes = [vp]
    L.vi_measure_peaks.argtypes = [i, P(C.c_double), P(C.c_double)]
    L.vi_render_batch.argtypes = [P(BatchFrame), i, vp, C.c_double]
    d, u64 = C.c_double, C.c_uint64
    L.vi_server_create.argtypes = [P(vp), i, i, sz, i]
    L.vi_server_destroy.argtypes = [vp]
    L.vi_server_add_volume.argtypes = [vp, vp, i, i, i, i, P(i)]
    L.vi_server_submit.argtypes = [vp, P(Request), P(u64)]
    L.vi_server_wait.argtypes = [vp, u64, d, P(i), P(i)]
    L.vi_server_cancel.argtypes = [vp, u64]
    L.vi_server_timing.argtypes = [vp, u64, P(d), P(d), P(d)]
    L.vi_server_release.argtypes = [vp, u64]
    L.vi_server_get_stats.argtypes = [vp, P(ServerStats)]
    L.vi_server_set_graphs.argtypes = [vp, i]
    L.vi_server_set_batching.argtypes = [vp, i, C.c_double]
    L.vi_server_set_eviction.argtypes = [vp, i]
    L.vi_debug_bounds.argtypes = [i, P(C.c_uint64), P(i), P(C.c_int64)]
    _libs[path] = L
    return L


def debug_bounds(device: int = 0):
    """(violations, first site, first index) of the checked library's kernels
    on ``device`` since the last call (vi_debug_bounds), which clears them."""
    L = library(checked=True)
    n, site, idx = C.c_uint64(), C.c_int(), C.c_int64()
    _check(L.vi_debug_bounds(int(device), C.byref(n), C.byref(site), C.byref(idx)),
           "vi_debug_bounds")
    return n.value, site.value, idx.value


def error_string(code: int) -> str:
    return library().vi_error_string(int(code)).decode()


def _check(code: int, call: str) -> None:
    if code != OK:
        raise ViError(code, call)


def _f3(v):
    return (C.c_float * 3)(*[float(x) for x in v])


def camera(cam) -> Camera:
    """From a ``phantoms.Camera`` or an (eye, target, up, persp, fovy, half_height) tuple."""
    t = cam.as_tuple() if hasattr(cam, "as_tuple") else cam
    eye, target, up, persp, fovy, hh = t
    return Camera(int(persp), _f3(eye), _f3(target), _f3(up), float(fovy), float(hh))


def _ptr(buf):
    """(pointer, on_device) of a torch tensor or numpy array."""
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr(), int(buf.is_cuda)
    return buf.ctypes.data, 0


class Context:
    """One ``vi_ctx``: a device, a stream and the resident volume / TF / stack."""

    def __init__(self, device: int = 0, stream=None, checked: bool = False):
        L = library(checked)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        h = C.c_void_p()
        _check(L.vi_create(C.byref(h), int(device), C.c_void_p(self.stream)), "vi_create")
        self.h = h
        self.L = L

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.vi_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_memory_budget(self, nbytes: int) -> None:
        _check(self.L.vi_set_memory_budget(self.h, int(nbytes)), "vi_set_memory_budget")

    def load_volume(self, vol, dtype: int | None = None) -> None:
        """``vol``: [nz, ny, nx] uint8 / uint16, numpy (host) or torch (host or
        device).  ``dtype`` (U8 / U16) overrides the element type, e.g. for a
        torch int16 tensor holding uint16 bits."""
        dt = str(vol.dtype)
        if dtype is not None:
            code = int(dtype)
            size = vol.element_size() if hasattr(vol, "element_size") else vol.itemsize
            if size != (1 if code == U8 else 2):
                raise TypeError("element size does not match dtype")
        elif dt.endswith("uint8"):
            code = U8
        elif dt.endswith("uint16"):
            code = U16
        else:
            raise TypeError("volume must be uint8 or uint16")
        if hasattr(vol, "is_contiguous") and not vol.is_contiguous():
            raise ValueError("volume tensor must be contiguous")
        if isinstance(vol, np.ndarray):
            vol = np.ascontiguousarray(vol)
        nz, ny, nx = vol.shape
        p, dev = _ptr(vol)
        _check(self.L.vi_load_volume(self.h, C.c_void_p(p), code, nx, ny, nz, dev),
               "vi_load_volume")

    def set_transfer_function(self, rgba, vmin: float, vmax: float) -> None:
        rgba = np.ascontiguousarray(rgba, dtype=np.float32)
        if rgba.ndim != 2 or rgba.shape[1] != 4:
            raise ValueError("transfer function must be (M, 4)")
        _check(self.L.vi_set_transfer_function(self.h, C.c_void_p(rgba.ctypes.data),
                                               rgba.shape[0], float(vmin), float(vmax)),
               "vi_set_transfer_function")

    def set_light(self, direction, color=(1.0, 1.0, 1.0)) -> None:
        _check(self.L.vi_set_light(self.h, _f3(direction), _f3(color)), "vi_set_light")

    def set_point_light(self, position, color=(1.0, 1.0, 1.0)) -> None:
        """A point light at ``position`` (at least 1 from the cube centre)."""
        _check(self.L.vi_set_point_light(self.h, _f3(position), _f3(color)),
               "vi_set_point_light")

    def build_attenuation(self, n_slices: int, slice_res: int, mode: int, format: int = F32,
                          cone_half_angle_deg: float = 15.0, shell_radius_vox: float = 1.0,
                          opacity_correction: int = 0, comp_n: float = 0.0,
                          quantity: int = TRANSMITTANCE, shell_count: int = 1) -> None:
        o = BuildOpts(int(format), float(cone_half_angle_deg), float(shell_radius_vox),
                      int(opacity_correction), float(comp_n), int(quantity), int(shell_count))
        _check(self.L.vi_build_attenuation(self.h, int(n_slices), int(slice_res), int(mode),
                                           C.byref(o)), "vi_build_attenuation")

    @staticmethod
    def _render_opts(ert, bg, ambient, opacity_correction, sample_counts=None,
                     lit_counts=None, slice_filter=SLICE_NEAREST) -> RenderOpts:
        ptrs = []
        for buf in (sample_counts, lit_counts):
            cp = None
            if buf is not None:
                cp, dev = _ptr(buf)
                if not dev:
                    raise ValueError("per-pixel counters must be device tensors")
            ptrs.append(cp)
        return RenderOpts(float(ert), (C.c_float * 4)(*map(float, bg)), float(ambient),
                          int(opacity_correction), *ptrs, int(slice_filter))

    def render(self, cam, W: int, H: int, step_vox: float, out=None, ert: float = 2.0,
               bg=(0.0, 0.0, 0.0, 0.0), ambient: float = 0.0, opacity_correction: int = 0,
               sample_counts=None, lit_counts=None, slice_filter: int = SLICE_NEAREST,
               host_async: bool = False):
        """Render into ``out`` ((H, W, 4) float32; torch CUDA tensor or numpy /
        pinned torch host tensor).  With ``out=None`` a torch CUDA tensor is
        allocated and returned.  ``host_async`` (host ``out`` only): enqueue
        the frame's copy on the context's stream and return; it is complete
        after ``sync()`` (VI_OUT_HOST_ASYNC)."""
        if out is None:
            import torch
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        p, dev = _ptr(out)
        if host_async:
            if dev:
                raise ValueError("host_async needs a host output")
            dev = OUT_HOST_ASYNC
        ro = self._render_opts(ert, bg, ambient, opacity_correction, sample_counts, lit_counts,
                               slice_filter)
        _check(self.L.vi_render(self.h, C.byref(camera(cam)), int(W), int(H), float(step_vox),
                                C.c_void_p(p), dev, C.byref(ro)), "vi_render")
        return out

    def sync(self) -> None:
        _check(self.L.vi_sync(self.h), "vi_sync")

    def attenuation_info(self):
        n, R, fmt, nb = C.c_int(), C.c_int(), C.c_int(), C.c_size_t()
        _check(self.L.vi_attenuation_info(self.h, C.byref(n), C.byref(R), C.byref(fmt),
                                          C.byref(nb)), "vi_attenuation_info")
        return n.value, R.value, fmt.value, nb.value

    def get_attenuation(self) -> np.ndarray:
        """The stack as stored: (n, R, R) float32 / float16 / uint16 (bf16 as uint16 bits)."""
        n, R, fmt, nb = self.attenuation_info()
        dt = {F32: np.float32, F16: np.float16, BF16: np.uint16, UNORM16: np.uint16}[fmt]
        out = np.empty((n, R, R), dtype=dt)
        _check(self.L.vi_get_attenuation(self.h, C.c_void_p(out.ctypes.data), out.nbytes, 0),
               "vi_get_attenuation")
        return out

    def get_skip_grid(self):
        """vi_get_skip_grid: (brick_flags, cell_skip) as uint8 arrays
        (nbz, nby, nbx) and (cnz, cny, cnx)."""
        dims = (C.c_int * 6)()
        _check(self.L.vi_get_skip_grid(self.h, dims, None, 0, None, 0), "vi_get_skip_grid")
        nbx, nby, nbz, cnx, cny, cnz = list(dims)
        flags = np.empty((nbz, nby, nbx), dtype=np.uint8)
        skip = np.empty((cnz, cny, cnx), dtype=np.uint8)
        _check(self.L.vi_get_skip_grid(self.h, dims, C.c_void_p(flags.ctypes.data), flags.nbytes,
                                       C.c_void_p(skip.ctypes.data), skip.nbytes),
               "vi_get_skip_grid")
        return flags, skip

    def trace_pixel(self, cam, W, H, step_vox, x, y, ert=2.0, bg=(0, 0, 0, 0), ambient=0.0,
                    opacity_correction=0, max_rec=8192, slice_filter=SLICE_NEAREST) -> np.ndarray:
        rec = np.zeros((max_rec, TRACE_WORDS), dtype=np.int32)
        n = C.c_int(0)
        ro = self._render_opts(ert, bg, ambient, opacity_correction, slice_filter=slice_filter)
        _check(self.L.vi_trace_pixel(self.h, C.byref(camera(cam)), int(W), int(H),
                                     float(step_vox), C.byref(ro), int(x), int(y),
                                     C.c_void_p(rec.ctypes.data), int(max_rec), C.byref(n)),
               "vi_trace_pixel")
        return rec[: n.value].copy()

    def render_host_noalloc(self, cam, W: int, H: int, step_vox: float, out=None,
                            ert: float = 2.0, bg=(0.0, 0.0, 0.0, 0.0), ambient: float = 0.0,
                            opacity_correction: int = 0) -> np.ndarray:
        """vi_render_host_noalloc: the frame into a host (H, W, 4) float32 array,
        with no device allocation (W * H <= NOALLOC_MAX_PIXELS)."""
        if out is None:
            out = np.empty((H, W, 4), dtype=np.float32)
        ro = self._render_opts(ert, bg, ambient, opacity_correction)
        _check(self.L.vi_render_host_noalloc(self.h, C.byref(camera(cam)), int(W), int(H),
                                             float(step_vox), C.c_void_p(out.ctypes.data),
                                             C.byref(ro)), "vi_render_host_noalloc")
        return out

    def post_ready(self) -> None:
        """vi_post_ready: publish this context's stack to batched frames."""
        _check(self.L.vi_post_ready(self.h), "vi_post_ready")

    def launch_count(self) -> int:
        v = C.c_uint64(0)
        _check(self.L.vi_launch_count(self.h, C.byref(v)), "vi_launch_count")
        return int(v.value)


def measure_peaks(device: int = 0) -> dict:
    """vi_measure_peaks: the FP32 FMA rate and L2 read bandwidth of the device."""
    L = library()
    f, l2 = C.c_double(), C.c_double()
    _check(L.vi_measure_peaks(int(device), C.byref(f), C.byref(l2)), "vi_measure_peaks")
    return {"fp32_tflops": f.value, "l2_read_gbs": l2.value}


BATCH_MAX_FRAMES = 64


def render_batch(frames, stream=None, wait_ms: float = 1000.0):
    """vi_render_batch: render several contexts' frames in persistent launches.

    ``frames`` is a list of dicts with keys ctx, cam, W, H, step_vox, out (an
    (H, W, 4) float32 CUDA tensor) and optionally ert, bg, sample_counts.
    Returns (rc, statuses): the call's status and each frame's (VI_OK or
    VI_ETIMEOUT); argument errors raise ViError."""
    n = len(frames)
    arr = (BatchFrame * n)()
    keep = []
    for k, fr in enumerate(frames):
        p, dev = _ptr(fr["out"])
        if not dev:
            raise ValueError("batched frames render into device tensors")
        arr[k].ctx = fr["ctx"].h
        arr[k].camera = camera(fr["cam"])
        arr[k].width, arr[k].height = int(fr["W"]), int(fr["H"])
        arr[k].step_vox = float(fr["step_vox"])
        arr[k].out_rgba = p
        arr[k].opts = Context._render_opts(fr.get("ert", 2.0), fr.get("bg", (0, 0, 0, 0)), 0.0, 0,
                                           sample_counts=fr.get("sample_counts"))
        keep.append(fr["out"])
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    L = frames[0]["ctx"].L
    rc = L.vi_render_batch(arr, n, C.c_void_p(int(stream)), float(wait_ms))
    if rc not in (OK, ETIMEOUT):
        raise ViError(rc, "vi_render_batch")
    return rc, [arr[k].status for k in range(n)]


def decode_stack(raw: np.ndarray, fmt: int) -> np.ndarray:
    """Stored stack values as float64."""
    if fmt == F32 or fmt == F16:
        return raw.astype(np.float64)
    if fmt == BF16:
        return (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return raw.astype(np.float64) / 65535.0


class Server:
    """A vi_server: continuous batching of render requests over resident volumes."""

    def __init__(self, device: int = 0, slots: int = 4, memory_budget: int = 0,
                 max_resident_volumes: int = 0, graphs: bool = False, checked: bool = False,
                 batching: bool = False, batch_wait_ms: float = 10000.0,
                 eviction: int | None = None):
        L = library(checked)
        h = C.c_void_p()
        _check(L.vi_server_create(C.byref(h), int(device), int(slots), int(memory_budget),
                                  int(max_resident_volumes)), "vi_server_create")
        self.h, self.L = h, L
        self._keep = {}   # host volumes and outputs the server reads or writes later
        if graphs:
            self.set_graphs(True)
        if batching:
            self.set_batching(True, batch_wait_ms)
        if eviction is not None:
            self.set_eviction(eviction)

    def set_eviction(self, policy: int) -> None:
        """Choose which idle volume is evicted when room is needed:
        EVICT_COST (GreedyDual on the reload cost, the default) or EVICT_LRU
        (vi_server_set_eviction)."""
        _check(self.L.vi_server_set_eviction(self.h, int(policy)), "vi_server_set_eviction")

    def set_batching(self, enabled: bool, wait_ms: float = 10000.0) -> None:
        """March the requests admitted in one scheduling pass as one batch of
        persistent launches (vi_server_set_batching)."""
        _check(self.L.vi_server_set_batching(self.h, int(bool(enabled)), float(wait_ms)),
               "vi_server_set_batching")

    def set_graphs(self, enabled: bool) -> None:
        """Launch each later request's sweep, march and output copy as one
        CUDA graph (vi_server_set_graphs)."""
        _check(self.L.vi_server_set_graphs(self.h, int(bool(enabled))), "vi_server_set_graphs")

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.vi_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_volume(self, vol, dtype: int | None = None) -> int:
        """Register a (nz, ny, nx) volume: a uint8 / uint16 numpy array, or a
        contiguous host torch tensor (page-locked, so reloads after eviction
        copy at full speed) whose 16-bit data is taken as VI_U16 unless
        ``dtype`` says otherwise.  The server keeps a reference to it."""
        if hasattr(vol, "data_ptr"):
            if vol.is_cuda or not vol.is_contiguous() or vol.dim() != 3:
                raise ValueError("volume must be a contiguous 3-D host tensor")
            code = dtype if dtype is not None else (U8 if vol.element_size() == 1 else U16)
            ptr = vol.data_ptr()
        else:
            vol = np.ascontiguousarray(vol)
            code = dtype if dtype is not None else (U8 if vol.dtype == np.uint8 else U16)
            ptr = vol.ctypes.data
        nz, ny, nx = vol.shape
        vid = C.c_int(-1)
        _check(self.L.vi_server_add_volume(self.h, C.c_void_p(ptr), int(code), nx, ny, nz,
                                           C.byref(vid)), "vi_server_add_volume")
        self._keep[("vol", vid.value)] = vol
        return vid.value

    def submit(self, volume_id, tf, vmin, vmax, light_dir, n_slices, slice_res, mode, cam, W, H,
               step_vox, out, light_color=(1.0, 1.0, 1.0), format=F32,
               cone_half_angle_deg=15.0, shell_radius_vox=1.0, ert=2.0,
               bg=(0.0, 0.0, 0.0, 0.0), quantity=TRANSMITTANCE, shell_count=1,
               slice_filter=SLICE_NEAREST, sample_counts=None) -> int:
        """Queue a render request; ``sample_counts`` (optional (H, W) int32 CUDA
        tensor) receives the samples composited per pixel."""
        tf = np.ascontiguousarray(tf, dtype=np.float32)
        p, dev = _ptr(out)
        q = Request(int(volume_id), C.c_void_p(tf.ctypes.data), tf.shape[0], float(vmin),
                    float(vmax), _f3(light_dir), _f3(light_color), int(n_slices),
                    int(slice_res), int(mode),
                    BuildOpts(int(format), float(cone_half_angle_deg), float(shell_radius_vox),
                              0, 0.0, int(quantity), int(shell_count)),
                    camera(cam), int(W), int(H), float(step_vox),
                    Context._render_opts(ert, bg, 0.0, 0, sample_counts=sample_counts,
                                         slice_filter=slice_filter),
                    C.c_void_p(p), dev)
        t = C.c_uint64(0)
        _check(self.L.vi_server_submit(self.h, C.byref(q), C.byref(t)), "vi_server_submit")
        self._keep[("out", t.value)] = (out, sample_counts)
        return t.value

    def wait(self, ticket: int, timeout_ms: float = 60000.0):
        """(status, result) of a request; raises ViError(ETIMEOUT) on timeout."""
        st, res = C.c_int(0), C.c_int(0)
        rc = self.L.vi_server_wait(self.h, C.c_uint64(ticket), float(timeout_ms), C.byref(st),
                                   C.byref(res))
        if rc != OK:
            raise ViError(rc, "vi_server_wait")
        return st.value, res.value

    def cancel(self, ticket: int) -> int:
        return int(self.L.vi_server_cancel(self.h, C.c_uint64(ticket)))

    def timing(self, ticket: int):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        _check(self.L.vi_server_timing(self.h, C.c_uint64(ticket), C.byref(a), C.byref(b),
                                       C.byref(c)), "vi_server_timing")
        return a.value, b.value, c.value

    def release(self, ticket: int) -> None:
        _check(self.L.vi_server_release(self.h, C.c_uint64(ticket)), "vi_server_release")
        self._keep.pop(("out", ticket), None)

    def stats(self) -> dict:
        st = ServerStats()
        _check(self.L.vi_server_get_stats(self.h, C.byref(st)), "vi_server_get_stats")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}
