"""Fixtures under tests/golden: hand-derived worked examples of the paper's
equations (checked against the oracle here, on the CPU) and the oracle's
frozen outputs on small scenes (the oracle must keep reproducing them; the GPU
test compares the CUDA path with them)."""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def example(name):
    for e in load("hand_worked.json")["examples"]:
        if e["name"] == name:
            return e["inputs"], e["expected"]
    raise KeyError(name)


@pytest.mark.parametrize("name", ["eq8-extreme-vertices-axis-light",
                                  "eq8-extreme-vertices-oblique-light"])
def test_worked_eq8(orc, name):
    inp, exp = example(name)
    lt = orc.light_setup(inp["L"], 4, 4)
    assert lt.min == pytest.approx(exp["min"], abs=1e-6)
    assert lt.max == pytest.approx(exp["max"], abs=1e-6)


def test_worked_eq9(orc):
    inp, exp = example("eq9-slice-of-a-point")
    lt = orc.light_setup(inp["L"], inp["n"], inp["R"])
    lam, tu, tv = orc.light_coords(lt, inp["X"])
    assert lam == pytest.approx(exp["lambda"], abs=1e-5)
    B = np.arange(inp["n"], dtype=np.float64)[:, None, None] * np.ones((1, inp["R"], inp["R"]))
    v, rec = orc.stack_lookup(B, lt, lam, tu, tv)
    assert rec[0] == exp["slice"] and v == exp["slice"]


def test_worked_eq3(orc):
    """Two one-voxel layers, no illumination: an orthographic ray starting at
    the first voxel's centre (x = 0.25, inside the cube) steps one voxel to the
    second (x = 0.75), so its two samples are exactly the fixture's layers
    (voxel values 0 and 255 select TF entries 0 and 1); the frame is the
    fixture's Eq. 3 result."""
    inp, exp = example("eq3-two-layers-front-to-back")
    vol = np.array([[[0, 255]]], dtype=np.uint8)           # nz = ny = 1, nx = 2
    tf = np.array([inp["front"], inp["back"]], dtype=np.float32)
    cam = ((0.25, 0.5, 0.5), (1.0, 0.5, 0.5), (0, 0, 1), 0, 40.0, 0.1)
    lt = orc.light_setup((0, 0, 1), 1, 1)
    out, _, _, ns = orc.render_pixels(vol, tf, 0, 255, lt, None, cam, 1, 1,
                                      orc.render_opts(orc.NONE, 1.0), np.array([0]),
                                      np.array([0]))
    assert ns[0] == 2
    assert np.allclose(out[0, :3], exp["C"], atol=1e-15)
    assert out[0, 3] == pytest.approx(exp["A"], abs=1e-15)


def test_worked_attenuation_through_a_slab(orc):
    """Algorithm 1 and Eq. 5-6 on a slab of constant opacity, light +z."""
    inp, exp_t = example("algorithm1-attenuation-through-a-slab")
    _, exp_d = example("eq5-6-optical-depth-through-a-slab")
    a, m = inp["alpha"], inp["planes_before"]
    N = 16
    vol = np.zeros((N, N, N), np.uint8)
    vol[4:12] = 200
    tf = np.zeros((256, 4), np.float32)
    tf[100:] = (1, 1, 1, a)
    n, R = 16, 8
    lt = orc.light_setup((0, 0, 1), n, R)
    T = orc.build_stack(vol, tf, 0, 255, lt)
    D = orc.build_stack(vol, tf, 0, 255, lt, quantity=orc.OPTICAL_DEPTH)
    # Planes k / 16 in the slab [0.25, 0.75]: k = 4 .. 12; plane 4 + m has m before it.
    a32 = float(np.float32(a))
    k = 4 + m
    assert T[k, R // 2, R // 2] == pytest.approx((1 - a32) ** m, abs=1e-12)
    assert (1 - a) ** m == pytest.approx(exp_t["B"], abs=1e-12)
    assert D[k, R // 2, R // 2] == pytest.approx(-m * math.log(1 - a32), abs=1e-12)
    assert -math.log(1 - a) == pytest.approx(exp_d["tau"], abs=1e-15)
    assert m * exp_d["tau"] == pytest.approx(exp_d["D"], abs=1e-15)


def test_worked_cone_ring_radii(orc):
    inp, exp = example("eq11-12-cone-ring-radii")
    t = math.tan(math.radians(inp["phi_deg"]))
    assert inp["dL"] * t == pytest.approx(exp["radius_ring1"], rel=1e-12)
    assert 2 * inp["dL"] * t == pytest.approx(exp["radius_ring2"], rel=1e-12)
    # The oracle's cone points: ring offsets in texels are n dL tan(phi) sigma.
    lt = orc.light_setup((0, 0, 1), 100, 64)
    ro = orc.render_opts(orc.CONE, 0.5, cone_half_angle_deg=inp["phi_deg"])
    fr = orc.frame_setup(((0.3, 0.4, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 1, 40.0, 0.5), 4, 4, 0.5, 16)
    ray = orc.ray_setup(lt, fr, ro, 1, 1)
    for ring in (1, 2):
        off = np.array(ray.nb[4 * (ring - 1)][1:3], float)
        assert np.linalg.norm(off) == pytest.approx(ring * lt.dL * t * lt.sigma, rel=1e-5)


def test_oracle_reproduces_its_frozen_outputs(orc):
    """The oracle's outputs on the small scenes of make_oracle_golden.py are
    unchanged (to the last few ulps)."""
    import sys
    sys.path.insert(0, HERE)
    import make_oracle_golden as mg
    g = load("oracle_small.json")
    vol, tf, cam = mg.scene()
    W, H, n, R = 12, 9, 11, 13
    for name, mode, pos, opts in mg.CASES:
        light = (orc.light_setup((0.3, -0.2, 0.9), n, R) if pos is None
                 else orc.point_light_setup(pos, n, R))
        B = None if mode == orc.NONE else orc.build_stack(vol, tf, 0, 255, light,
                                                          quantity=opts.get("quantity", 0))
        ro = orc.render_opts(mode, 0.5, 0.95, (0.1, 0.2, 0.3, 0.0), ert_band=0.0, **opts)
        img, _, _, ns = orc.render_image(vol, tf, 0, 255, light, B, cam, W, H, ro)
        case = g["cases"][name]
        assert np.allclose(img.reshape(-1), case["image_rgba"], rtol=0, atol=1e-13), name
        assert ns.reshape(-1).tolist() == case["samples"], name
        if B is not None:
            assert np.allclose(B.reshape(-1)[::7], case["stack_every_7th"], rtol=0, atol=1e-13)


@pytest.mark.gpu
def test_gpu_reproduces_the_frozen_oracle_outputs():
    """The CUDA path, through the C ABI, against the stored oracle frames."""
    import sys
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from gpu_common import IMAGE_TOL
    from paper_2008_06134_gb300 import build, vi
    build.build()
    sys.path.insert(0, HERE)
    import make_oracle_golden as mg
    g = load("oracle_small.json")
    vol, tf, cam = mg.scene()
    W, H, n, R = 12, 9, 11, 13
    with vi.Context(0) as c:
        c.load_volume(vol)
        c.set_transfer_function(tf, 0, 255)
        for name, mode, pos, opts in mg.CASES:
            if pos is None:
                c.set_light((0.3, -0.2, 0.9))
            else:
                c.set_point_light(pos)
            c.build_attenuation(n, R, mode, quantity=opts.get("quantity", 0),
                                shell_count=opts.get("shell_count", 1))
            cnt = torch.zeros((H, W), dtype=torch.int32, device="cuda")
            img = c.render(cam, W, H, 0.5, ert=0.95, bg=(0.1, 0.2, 0.3, 0.0),
                           slice_filter=opts.get("slice_filter", 0), sample_counts=cnt)
            got = img.cpu().numpy().astype(np.float64).reshape(-1)
            want = np.array(g["cases"][name]["image_rgba"])
            assert np.abs(got - want).max() <= IMAGE_TOL, (name, np.abs(got - want).max())
            assert cnt.cpu().numpy().reshape(-1).tolist() == g["cases"][name]["samples"], name
