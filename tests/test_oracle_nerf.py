"""Pins of the oracle's radiance-field colour (Step 2 with a NeRF colour network, Eq. 8 with the
sample window): the network's output activation and its inputs, through the whole shading path,
against closed forms of networks built to expose them.

Colour network: sigmoid(MLP([gamma_10(x), gamma_4(d)])) with x the sample's object-local position
and d the ray's local direction (63 + 27 inputs); the shaded colour is sum_j w_j c_j over the
window's samples with opacity A = sum_j w_j.
"""
import math

import numpy as np

from paper_2308_04669_gb300 import scenegen as sg

HID, WID = 2, 8


def _scene(nerf_w, R=None):
    t = sg.make_type(sg.SDF_SPHERE, 0, 0, 2, 8, HID, WID, nedf_seed=3)
    t.nerf_w = sg.f32(nerf_w)
    Rm = np.eye(3) if R is None else R
    return sg.Scene("n", 33, 33, sg.f32([0.3, 0.2, 3.0]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]), [t],
                    np.zeros(1, np.uint32), sg.f32(Rm.reshape(1, 9)), sg.f32([[0, 0, 0]]), sg.f32([1.0]))


def _layers(w):
    dims = sg.mlp_dims(sg.NERF_IN, HID, WID, 3)
    out, off = [], 0
    for fi, fo in zip(dims[:-1], dims[1:]):
        out.append((w[off:off + fi * fo].reshape(fo, fi), w[off + fi * fo:off + fi * fo + fo]))
        off += fi * fo + fo
    return out


def _zeros():
    return np.zeros(sg.mlp_param_count(sg.mlp_dims(sg.NERF_IN, HID, WID, 3)), np.float64)


def test_constant_colour_network_gives_opacity_times_sigmoid(orc):
    """All weights zero, output biases b: every sample's colour is sigmoid(b), so the shaded
    colour is A sigmoid(b) with A the window's opacity."""
    w = _zeros()
    b = np.array([0.7, -1.2, 2.5])
    _layers(w)[-1][1][:] = b
    sc = _scene(w)
    r = orc.render(orc.OracleScene(sc), depth_mode=orc.DEPTH_EXACT)
    hit = r["id"] != 0xFFFFFFFF
    assert hit.sum() > 50
    A = r["rgba"][hit, 3]
    assert A.min() > 0.5
    sig = 1.0 / (1.0 + np.exp(-np.float32(b).astype(np.float64)))     # the scene stores float32 weights
    assert np.allclose(r["rgba"][hit, :3], A[:, None] * sig[None, :], rtol=0, atol=1e-12)


def test_colour_network_inputs_are_position_and_direction_encodings(orc):
    """A network that passes one input feature through (first layer picks it with a large positive
    offset so the ReLUs stay linear, the output subtracts the offset): red = sigmoid(d_x) (the
    local direction's x, input 63), green = sigmoid(sin(2 x_z)) (input 3 + 3 * 1 + 2 of the
    position encoding), blue = sigmoid(cos(2 d_y)) (input 63 + 3 + 12 + 3 * 1 + 1).  Samples of
    one pixel share d but not x, so green is checked against the sample-weighted mean."""
    C = 4.0
    picks = [63, 3 + 3 * 1 + 2, 63 + 3 + 12 + 3 * 1 + 1]
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])   # local = R^T world
    w = _zeros()
    L = _layers(w)
    for o, k in enumerate(picks):
        L[0][0][o, k] = 1.0
        L[0][1][o] = C
        L[1][0][o, o] = 1.0
        L[2][0][o, o] = 1.0
        L[2][1][o] = -C
    sc = _scene(w, R)
    osc = orc.OracleScene(sc)
    r = orc.render(osc, depth_mode=orc.DEPTH_EXACT)
    hit = np.nonzero(r["id"] != 0xFFFFFFFF)[0]
    assert len(hit) > 50
    for p in hit[::7]:
        o_, d_ = np.zeros(3), np.zeros(3)
        orc.lib().orc_camera_ray(osc.ptr, int(p % 33), int(p // 33), orc._dp(o_), orc._dp(d_))
        dl = R.T @ d_
        A = r["rgba"][p, 3]
        assert abs(r["rgba"][p, 0] - A / (1.0 + math.exp(-dl[0]))) < 1e-12
        assert abs(r["rgba"][p, 2] - A / (1.0 + math.exp(-math.cos(2.0 * dl[1])))) < 1e-12
        # green: sin(2 z) over the window's samples, each within [D - h, D + h] of the surface
        D = r["depth"][p]
        zs = [(o_ + (D + s) * d_) @ R[:, 2] for s in (-sc.shade_half, sc.shade_half)]
        lo, hi = sorted(1.0 / (1.0 + np.exp(-np.sin(2.0 * np.array(zs)))))
        g = r["rgba"][p, 1] / A
        assert lo - 1e-9 <= g <= hi + 1e-9 or abs(hi - lo) < 1e-3
