"""Shared helpers of the GPU parity tests: run a scene through the C ABI and
through the oracle on the same seeded inputs, and compare."""
import numpy as np

# FP32 path vs the FP64 oracle, per RGBA channel on [0, 1].
IMAGE_TOL = 1e-4
# FP32 attenuation stack vs the FP64 oracle: an FP32 product of up to n
# factors plus the FP32 reconstruction error stays well inside this.
STACK_TOL = 1e-5
# Half an ulp at 1 of each storage format, the rounding each stored value may add.
FORMAT_HALF_ULP = {0: 0.0, 1: 2.0 ** -12, 2: 2.0 ** -9, 3: 0.5 / 65535.0}


def gpu_frame(ctx, scene, mode=None, fmt=0, counts=False, ert=None, bg=None,
              opacity_correction=0, comp_n=0.0, build_oc=0, quantity=0, shell_count=1,
              slice_filter=0, light_pos=None):
    import torch
    mode = scene.mode if mode is None else mode
    ctx.load_volume(scene.volume)
    ctx.set_transfer_function(scene.tf, scene.vmin, scene.vmax)
    if light_pos is None:
        ctx.set_light(scene.light_dir, scene.light_color)
    else:
        ctx.set_point_light(light_pos, scene.light_color)
    ctx.build_attenuation(scene.n_slices, scene.slice_res, mode, format=fmt,
                          cone_half_angle_deg=scene.cone_half_angle_deg,
                          shell_radius_vox=scene.shell_radius_vox,
                          opacity_correction=build_oc, comp_n=comp_n, quantity=quantity,
                          shell_count=shell_count)
    cnt = None
    if counts:
        cnt = torch.zeros((scene.height, scene.width), dtype=torch.int32, device="cuda")
    out = ctx.render(scene.camera, scene.width, scene.height, scene.step_vox,
                     ert=scene.ert if ert is None else ert,
                     bg=scene.bg if bg is None else bg,
                     opacity_correction=opacity_correction, sample_counts=cnt,
                     slice_filter=slice_filter)
    torch.cuda.synchronize()
    ctx.sync()
    img = out.cpu().numpy().astype(np.float64)
    return img, (cnt.cpu().numpy() if counts else None)


def oracle_frame(orc, scene, mode=None, xs=None, ys=None, stack=None, ert=None, bg=None,
                 opacity_correction=0, comp_n=0.0, build_oc=0, ert_band=1e-5, quantity=0,
                 shell_count=1, slice_filter=0, light_pos=None):
    mode = scene.mode if mode is None else mode
    if light_pos is None:
        light = orc.light_setup(scene.light_dir, scene.n_slices, scene.slice_res)
    else:
        light = orc.point_light_setup(light_pos, scene.n_slices, scene.slice_res)
    if stack is None and mode != orc.NONE:
        stack = orc.build_stack(scene.volume, scene.tf, scene.vmin, scene.vmax, light,
                                opacity_correction=build_oc, comp_n=comp_n, quantity=quantity)
    ro = orc.render_opts(mode, scene.step_vox, scene.ert if ert is None else ert,
                         scene.bg if bg is None else bg, scene.light_color,
                         opacity_correction=opacity_correction,
                         cone_half_angle_deg=scene.cone_half_angle_deg,
                         shell_radius_vox=scene.shell_radius_vox, ert_band=ert_band,
                         quantity=quantity, slice_filter=slice_filter, shell_count=shell_count)
    if xs is None:
        ys_, xs_ = np.mgrid[0:scene.height, 0:scene.width]
        xs_, ys_ = xs_.ravel(), ys_.ravel()
    else:
        xs_, ys_ = xs, ys
    img, alt, win, ns, ns_alt, end, ns_end = orc.render_window(
        scene.volume, scene.tf, scene.vmin, scene.vmax, light, stack, scene.camera,
        scene.width, scene.height, ro, xs_, ys_)
    if xs is None:
        shape = (scene.height, scene.width)
        img, alt, end = (a.reshape(*shape, 4) for a in (img, alt, end))
        win, ns, ns_alt, ns_end = (a.reshape(shape) for a in (win, ns, ns_alt, ns_end))
    window = {"win": win, "ns_alt": ns_alt, "end": end, "ns_end": ns_end}
    return img, alt, win > 0, ns, stack, light, ro, window


def image_errors(gpu, ref, alt, amb):
    """Per-pixel max-channel error; ERT-ambiguous pixels may match either outcome."""
    e_main = np.abs(gpu - ref).max(axis=-1)
    e_alt = np.abs(gpu - alt).max(axis=-1)
    return np.where(amb, np.minimum(e_main, e_alt), e_main)


# Early ray termination (Eq. 3, reading R12): where the binary64 opacity passes
# within the oracle's band (1e-5) of the threshold, a binary32 renderer may stop
# at any sample of a short window.  A ray that reaches the threshold has one
# with a chance of about 2 band / (alpha (1 - ert)), the band against the
# opacity step there: near 10 % for soft tissue (alpha 0.02) at ert = 0.99,
# under 1 % for bone.  Whole frames that terminate at 0.99 have 0.2-0.5 % of
# their pixels in a window, the sampled rows through the 1024^3 volume 1.6 %.
# A larger share means the band or the window logic has widened.
MAX_AMBIGUOUS_FRACTION = 0.05


def check_frame(gpu, counts, ora, tol=IMAGE_TOL):
    """Compare a GPU frame (and its per-pixel sample counts, if given) with the
    oracle's (the tuple oracle_frame returns).  Every pixel must match a valid
    early-termination outcome within tol: without an ERT window the binary64
    one, with its exact sample count; with a window of two samples the outcome
    whose sample count the GPU reports; with a longer window any stop inside
    it (the composited colour and opacity grow monotonically along it, so they
    lie between the window's two ends).  Returns the per-pixel errors."""
    ref, alt, amb, ns, *_, w = ora
    win, ns_alt, end, ns_end = w["win"], w["ns_alt"], w["end"], w["ns_end"]
    gpu = np.asarray(gpu, dtype=np.float64).reshape(ref.shape)
    assert amb.mean() <= MAX_AMBIGUOUS_FRACTION, amb.mean()
    e_main = np.abs(gpu - ref).max(axis=-1)
    e_alt = np.abs(gpu - alt).max(axis=-1)
    # The window's two ends: its start is alt unless the decision is there.
    first = np.where((ns_alt < ns)[..., None], alt, ref)
    lo, hi = np.minimum(first, end), np.maximum(first, end)
    e_hull = np.maximum(np.maximum(lo - gpu, gpu - hi), 0.0).max(axis=-1)
    if counts is None:
        err = np.where(win == 0, e_main, np.where(win == 1, np.minimum(e_main, e_alt), e_hull))
    else:
        counts = np.asarray(counts).reshape(ns.shape)
        n_first = np.minimum(ns, ns_alt)
        err = np.full(ns.shape, np.inf)
        err = np.where(counts == ns, e_main, err)
        err = np.where((win > 0) & (counts == ns_alt), np.minimum(err, e_alt), err)
        inside = (win == 2) & (counts >= n_first) & (counts <= ns_end)
        err = np.where(inside, np.minimum(err, e_hull), err)
    worst = np.unravel_index(int(np.argmax(err)), err.shape)
    assert err.max() <= tol, (float(err.max()), worst, int(win[worst]))
    return err
