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
        img, alt, amb, ns = orc.render_image(scene.volume, scene.tf, scene.vmin, scene.vmax,
                                             light, stack, scene.camera, scene.width,
                                             scene.height, ro)
    else:
        img, alt, amb, ns = orc.render_pixels(scene.volume, scene.tf, scene.vmin, scene.vmax,
                                              light, stack, scene.camera, scene.width,
                                              scene.height, ro, xs, ys)
    return img, alt, amb, ns, stack, light, ro


def image_errors(gpu, ref, alt, amb):
    """Per-pixel max-channel error; ERT-ambiguous pixels may match either outcome."""
    e_main = np.abs(gpu - ref).max(axis=-1)
    e_alt = np.abs(gpu - alt).max(axis=-1)
    return np.where(amb, np.minimum(e_main, e_alt), e_main)
