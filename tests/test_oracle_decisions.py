"""Pins of the oracle's remaining decision logic against closed forms.

* The MLP-mode decisions of a depth query (Algorithm 1's NeDF generation with the confidence
  fallback and the depth check of Section "Deferred Shading"): constant-output networks on the
  analytic sphere, whose surface depth is a quadratic root, so each branch's result is known.
* The signed distance functions of the five extra object kinds of the 4096-instance workload,
  against their zero sets and distances in closed form, and the plain volume rendering of several
  instances on one ray (front to back by entry distance, Algorithm 1's plain counterpart).

Each test is chosen so that breaking its branch (a reversed comparison, a wrong bracket, a wrong
order or axis) fails it.
"""
import math

import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .test_oracle_pins import constant_nedf, one_instance_scene

LN9 = math.log(9.0)              # logit whose confidence max(p, 1 - p) is exactly 0.9
EYE, DIR = np.array([0.0, 0.0, 3.0]), np.array([0.0, 0.0, -1.0])
SURF = 2.5                       # ray from (0,0,3) along -z meets the r = 0.5 sphere at t = 2.5
H = float(np.float32(0.05))       # the depth check's half window (shade_half, a float32 input)


def _query(orc, m, a, **kw):
    """Query of the one-sphere scene with a network whose output is the constant (m, a)."""
    sc = one_instance_scene(sg.SDF_SPHERE, nedf_w=constant_nedf(m, a))
    osc = orc.OracleScene(sc)
    assert osc.c.shade_half == H
    kw.setdefault("march_n", 4096)
    kw.setdefault("march_b", 60)
    hit, out, _ = orc.query(osc, 0, EYE, DIR, **kw)
    return hit, out[0]


def _m_for_depth(D):
    """m such that the NeDF's depth on the test ray is D (Eq. 2: D = t_perp - rb m, t_perp = 3),
    rounded to float32 as the weights are; _depth_of(m) is the depth the network then gives."""
    return float(np.float32(3.0 - D))


def _depth_of(m):
    return 3.0 - m


# ------------------------------------------------------------------------------------------------
# confidence fallback
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_confidence_below_threshold_goes_to_the_plain_method(orc, sign):
    """conf = max(p, 1-p) with p = sigmoid(a): just under 0.9 the pair is re-answered by the plain
    method (exact surface 2.5), just over it keeps the network's answer."""
    m = _m_for_depth(2.8)                                        # the network says 2.8, 0.3 off
    D_net = _depth_of(m)
    hit, D = _query(orc, m, sign * (LN9 - 1e-3), fallback_conf=0.9)
    assert hit and abs(D - SURF) < 1e-9                          # marched: the true surface
    hit, D = _query(orc, m, sign * (LN9 + 1e-3), fallback_conf=0.9)
    if sign > 0:
        assert hit and abs(D - D_net) < 1e-12                    # confident hit: the network's depth
    else:
        assert not hit                                           # confident miss stays a miss
    # without the fallback the network's answer stands at any confidence
    hit, D = _query(orc, m, sign * (LN9 - 1e-3), fallback_conf=0.0)
    assert hit == (sign > 0) and (not hit or abs(D - D_net) < 1e-12)


def test_confidence_threshold_is_a_probability_not_a_logit(orc):
    """A logit of 0.95 (p = 0.72) is below the 0.9 confidence although above 0.9 as a number."""
    hit, D = _query(orc, _m_for_depth(2.8), 0.95, fallback_conf=0.9)
    assert hit and abs(D - SURF) < 1e-9


# ------------------------------------------------------------------------------------------------
# depth check and refinement in [D - h, D + h]
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("delta", [-0.049, -0.031, -0.004, 0.0007, 0.017, 0.0449])
@pytest.mark.parametrize("steps", [1, 2, 4, 8])
def test_refinement_halves_the_window_towards_the_surface(orc, delta, steps):
    """A NeDF hit within h of the surface is bisected `steps` times on the half-density level:
    the result is the midpoint of a bracket of width 2h / 2^steps that holds the surface, i.e. a
    point D - h + (k + 1/2) 2h / 2^steps within h / 2^steps of the closed-form root."""
    m = _m_for_depth(SURF + delta)
    D0 = _depth_of(m)
    hit, D = _query(orc, m, 5.0, refine_steps=steps)
    assert hit
    w = 2 * H / 2 ** steps
    assert abs(D - SURF) <= 0.5 * w + 1e-12
    k = (D - (D0 - H)) / w - 0.5
    assert abs(k - round(k)) < 1e-6 and 0 <= round(k) < 2 ** steps


def test_refinement_error_shrinks_with_each_step(orc):
    errs = [abs(_query(orc, _m_for_depth(SURF + 0.0371), 5.0, refine_steps=s)[1] - SURF) for s in range(1, 13)]
    assert errs[-1] <= 2 * H / 2 ** 13 + 1e-15 and errs[-1] < errs[0] / 100


@pytest.mark.parametrize("delta", [0.2, -0.2, 0.07, -0.06])
def test_hit_outside_the_window_is_an_outlier(orc, delta):
    """No half-density crossing inside [D - h, D + h]: with outlier re-answering the plain method
    gives the surface; without it the network's depth is kept unrefined."""
    m = _m_for_depth(SURF + delta)
    D0 = _depth_of(m)
    hit, D = _query(orc, m, 5.0, refine_steps=4, outlier_resample=1)
    assert hit and abs(D - SURF) < 1e-9
    hit, D = _query(orc, m, 5.0, refine_steps=4, outlier_resample=0)
    assert hit and abs(D - D0) < 1e-12


def test_low_confidence_pairs_are_not_refined(orc):
    """A pair sent to the plain method by the confidence test keeps the plain method's finer depth
    (it is not bisected again in the window)."""
    hit, D = _query(orc, _m_for_depth(SURF + 0.03), LN9 - 0.5, fallback_conf=0.9, refine_steps=1)
    assert hit and abs(D - SURF) < 1e-9                          # 1 refinement step would leave ~0.025


def test_refinement_does_not_touch_misses(orc):
    hit, D = _query(orc, _m_for_depth(SURF + 0.01), -5.0, refine_steps=4, outlier_resample=1)
    assert not hit


# ------------------------------------------------------------------------------------------------
# signed distance functions of the extra object kinds
# ------------------------------------------------------------------------------------------------
def _sdf(orc, kind, x):
    return orc.sdf(kind, sg.DEFAULT_PARAMS[kind], np.asarray(x, np.float64))


def test_capsule_cylinder_caps_and_distances(orc):
    a, r = sg.DEFAULT_PARAMS[sg.SDF_CAPSULE]
    a, r = float(np.float32(a)), float(np.float32(r))
    for phi in np.linspace(0, 2 * np.pi, 7):
        for y in (-a, -0.1, 0.0, 0.2, a):                        # side of the cylinder
            assert abs(_sdf(orc, sg.SDF_CAPSULE, [r * math.cos(phi), y, r * math.sin(phi)])) < 1e-7
        for th in (0.0, 0.4, 1.2):                               # the two hemispherical caps
            p = [r * math.sin(th) * math.cos(phi), a + r * math.cos(th), r * math.sin(th) * math.sin(phi)]
            assert abs(_sdf(orc, sg.SDF_CAPSULE, p)) < 1e-7
            p[1] = -p[1]
            assert abs(_sdf(orc, sg.SDF_CAPSULE, p)) < 1e-7
    assert abs(_sdf(orc, sg.SDF_CAPSULE, [0.5, 0.1, 0.0]) - (0.5 - r)) < 1e-7
    assert abs(_sdf(orc, sg.SDF_CAPSULE, [0.0, 0.8, 0.0]) - (0.8 - a - r)) < 1e-7
    assert abs(_sdf(orc, sg.SDF_CAPSULE, [0.0, 0.0, 0.0]) + r) < 1e-7


def test_rounded_cone_is_the_hull_of_its_two_spheres(orc):
    """The convex hull of two balls is the union of the balls interpolated between them (centre
    and radius linear in t); outside it the distance is min_t |x - c(t)| - r(t), found here by
    brute force over t.  Its poles are the closed-form zero set."""
    r1, y1, r2, y2 = [float(np.float32(v)) for v in sg.DEFAULT_PARAMS[sg.SDF_ROUNDCONE]]
    assert abs(_sdf(orc, sg.SDF_ROUNDCONE, [0, y1 - r1, 0])) < 1e-7
    assert abs(_sdf(orc, sg.SDF_ROUNDCONE, [0, y2 + r2, 0])) < 1e-7
    t = np.linspace(0.0, 1.0, 200001)
    c_y, rad = y1 + t * (y2 - y1), r1 + t * (r2 - r1)
    rng = np.random.default_rng(5)
    n_out = 0
    for _ in range(300):
        x = rng.uniform(-0.7, 0.7, size=3)
        q = math.hypot(x[0], x[2])
        brute = np.min(np.hypot(q, x[1] - c_y) - rad)
        got = _sdf(orc, sg.SDF_ROUNDCONE, x)
        if brute > 0:
            assert abs(got - brute) < 1e-6, (x, got, brute)
            n_out += 1
        else:
            assert got <= 1e-9                                   # inside the hull: non-positive
    assert n_out > 100


def test_two_sphere_union(orc):
    c, r = [float(np.float32(v)) for v in sg.DEFAULT_PARAMS[sg.SDF_TWOSPHERE]]
    for sx in (-1, 1):
        for th in np.linspace(0, 2 * np.pi, 9):
            p = [sx * c + r * math.cos(th), r * math.sin(th) * 0.6, r * math.sin(th) * 0.8]
            if math.dist(p, [-sx * c, 0, 0]) >= r:                # not inside the other sphere
                assert abs(_sdf(orc, sg.SDF_TWOSPHERE, p)) < 1e-7
    assert abs(_sdf(orc, sg.SDF_TWOSPHERE, [0, 0, 0]) + (r - c)) < 1e-7       # between the centres
    assert abs(_sdf(orc, sg.SDF_TWOSPHERE, [0, 0.9, 0]) - (math.hypot(c, 0.9) - r)) < 1e-7
    assert abs(_sdf(orc, sg.SDF_TWOSPHERE, [1.0, 0, 0]) - (1.0 - c - r)) < 1e-7


def test_octahedron_vertices_faces_and_face_normal_distance(orc):
    a = float(np.float32(sg.DEFAULT_PARAMS[sg.SDF_OCTA][0]))
    for ax in range(3):
        for sgn in (-1, 1):
            v = [0.0, 0.0, 0.0]
            v[ax] = sgn * a
            assert abs(_sdf(orc, sg.SDF_OCTA, v)) < 1e-7
    rng = np.random.default_rng(3)
    for _ in range(50):                                          # points on the faces
        b = rng.dirichlet([1, 1, 1]) * a * rng.choice([-1, 1], size=3)
        assert abs(_sdf(orc, sg.SDF_OCTA, b)) < 1e-7
    # along a face normal through the face centre the closest point is that centre: exact distance
    n = np.array([1.0, -1.0, 1.0]) / math.sqrt(3)
    for t in (0.5, 0.8, 1.3):
        assert abs(_sdf(orc, sg.SDF_OCTA, t * n) - (t - a / math.sqrt(3))) < 1e-7
    assert _sdf(orc, sg.SDF_OCTA, [0, 0, 0]) < 0


def _plain_torus_z(p, R, r):
    """Ring of radius R in the xy plane (axis z), tube radius r: exact distance."""
    return math.hypot(math.hypot(p[0], p[1]) - R, p[2]) - r


def test_twisted_torus_untwists_to_the_plain_torus(orc):
    """Rotating a point about y by the twist angle k y (the rotation that takes (x, z) to
    (x cos - z sin, x sin + z cos)) turns the twisted torus back into the plain ring in the xy
    plane: the twist is about y, proportional to y, and the ring's axis is z."""
    R, r, k = [float(np.float32(v)) for v in sg.DEFAULT_PARAMS[sg.SDF_TWISTTORUS]]
    rng = np.random.default_rng(9)
    for _ in range(200):
        x = rng.uniform(-0.8, 0.8, size=3)
        th = k * x[1]
        u = [x[0] * math.cos(th) - x[2] * math.sin(th), x[1], x[0] * math.sin(th) + x[2] * math.cos(th)]
        assert abs(_sdf(orc, sg.SDF_TWISTTORUS, x) - _plain_torus_z(u, R, r)) < 1e-7
    # in the plane y = 0 there is no twist: the tube centres (+-R, 0, 0) of the plain ring
    for c in ([R, 0.0, 0.0], [-R, 0.0, 0.0]):
        assert abs(_sdf(orc, sg.SDF_TWISTTORUS, c) + r) < 1e-7
    # a tube centre off the plane y = 0 is found by twisting the plain ring's point back
    for phi in (0.5, 1.1, 2.0, -0.8):
        c = np.array([R * math.cos(phi), R * math.sin(phi), 0.0])
        th = -k * c[1]
        x = [c[0] * math.cos(th) - c[2] * math.sin(th), c[1], c[0] * math.sin(th) + c[2] * math.cos(th)]
        assert abs(_sdf(orc, sg.SDF_TWISTTORUS, x) + r) < 1e-7
        assert abs(_sdf(orc, sg.SDF_TWISTTORUS, c) + r) > 1e-3   # the untwisted point is not the centre


# ------------------------------------------------------------------------------------------------
# plain volume rendering of several instances on one ray
# ------------------------------------------------------------------------------------------------
def _two_sphere_colour_scene(order):
    """Two opaque spheres (r 0.5) on the camera's axis at z = +1 (front, red) and z = -1.5 (back,
    blue); `order` lists which of the two is instance 0."""
    red = sg.make_type(sg.SDF_SPHERE, 0, 0, 2, 8, albedo=(1.0, 0.0, 0.0), nedf_seed=1)
    blue = sg.make_type(sg.SDF_SPHERE, 0, 1, 2, 8, albedo=(0.0, 0.0, 1.0), nedf_seed=2)
    T = {"front": [0.0, 0.0, 1.0], "back": [0.0, 0.0, -1.5]}
    ty = {"front": 0, "back": 1}
    return sg.Scene("two-colours", 33, 33, sg.f32([0, 0, 4]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]),
                    [red, blue], np.array([ty[k] for k in order], np.uint32),
                    sg.f32(np.tile(np.eye(3).reshape(1, 9), (2, 1))), sg.f32([T[k] for k in order]),
                    sg.f32([1, 1]))


@pytest.mark.parametrize("order", [("front", "back"), ("back", "front")])
def test_volume_render_composites_front_to_back_in_both_index_orders(orc, order):
    osc = orc.OracleScene(_two_sphere_colour_scene(order))
    centre = 16 * 33 + 16
    rgba = orc.volume_render(osc, 128, px=np.array([centre]))[0]
    assert np.allclose(rgba, [1.0, 0.0, 0.0, 1.0], atol=1e-12)   # the front sphere's colour only


def test_volume_render_semi_transparent_front_lets_the_back_through(orc):
    """A front sphere thinner than one optical depth: the back sphere's colour is attenuated by the
    front's transmittance, whatever the index order (closed form for two constant media)."""
    res = []
    for order in (("front", "back"), ("back", "front")):
        sc = _two_sphere_colour_scene(order)
        sc.types[0].params[0] = np.float32(0.0)                 # front type: a point sphere ...
        sc.sigma_max = 50.0
        osc = orc.OracleScene(sc)
        res.append(orc.volume_render(osc, 512, px=np.array([16 * 33 + 16]))[0])
    assert np.allclose(res[0], res[1], atol=1e-12)
    # ... whose density on the axis is 50 sigmoid(-|x|/0.01): integral over the line is
    # 2 * 50 * 0.01 * ln 2, so the red opacity is 1 - exp(-0.693...) = 0.5 and blue gets the rest
    a_red = 1 - math.exp(-2 * 50 * 0.01 * math.log(2.0))
    assert abs(res[0][0] - a_red) < 2e-3
    assert abs(res[0][2] - (1 - a_red)) < 2e-3 and abs(res[0][3] - 1) < 1e-9


# ------------------------------------------------------------------------------------------------
# rounding knife edges (how far a value may move before a BF16 / E4M3 cast changes)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", [0, 1])
def test_round_margin_is_the_distance_to_the_next_rounding_change(orc, fmt):
    """Against torch's own casts: moving x by 0.98 of its margin keeps the rounded value, moving it
    by 1.02 of the margin in one of the two directions changes it."""
    torch = pytest.importorskip("torch")
    cast = torch.bfloat16 if fmt == 0 else torch.float8_e4m3fn
    rng = np.random.default_rng(21 + fmt)
    lo, hi = (-6, 6) if fmt == 0 else (-3.2, 2.6)
    xs = rng.normal(size=3000) * 10.0 ** rng.uniform(lo, hi, 3000)
    xs = np.concatenate([xs, [1.0, 1.5, 2.0 ** -7 * 3, 100.3]])
    if fmt == 1:                            # torch's cast does not saturate: compare below 432
        xs = np.concatenate([xs[np.abs(xs) < 420], [2.0 ** -9, 0.001, 300.0]])
        # saturating convention: everything above the 416 / 448 midpoint rounds to 448
        assert orc.round_margin(470.0, 1) == 38.0 and orc.round_margin(-448.0, 1) == 16.0
    rnd = lambda v: torch.tensor(np.asarray(v, np.float64)).to(cast).to(torch.float64).numpy()
    m = np.array([orc.round_margin(v, fmt) for v in xs])
    assert np.all(m > 0)
    assert orc.round_margin(100.0, 1) == 0.0 and orc.round_margin(1.0 + 2.0 ** -8, 0) == 0.0   # ties
    keep = m > 1e-5 * np.abs(xs)            # torch casts doubles through float32: 2% of m must exceed its ulp
    xs, m = xs[keep], m[keep]
    base = rnd(xs)
    assert np.array_equal(rnd(xs + 0.98 * m), base) and np.array_equal(rnd(xs - 0.98 * m), base)
    moved = (rnd(xs + 1.02 * m) != base) | (rnd(xs - 1.02 * m) != base)
    assert moved.all(), xs[~moved][:5]


def test_mlp_qmargin_reports_the_tightest_rounded_value(orc):
    """A one-hidden-unit network whose activation is placed at a chosen distance from a BF16
    boundary: the row's margin is that distance over the sum's magnitude."""
    dims = [78, 1, 2]
    w = np.zeros(sg.mlp_param_count(dims))
    x = np.zeros(78)
    x[0] = 1.0                                                   # an exactly representable input
    w[0] = 1.0                                                   # W0[0][0]
    # midpoint of 1 and 1 + 2^-7 is 1 + 2^-8; the bias 2^-8 - 2^-15 (exact in BF16, so its two-part
    # BF16 form is itself) puts the pre-activation 2^-15 below it
    w[78] = 2.0 ** -8 - 2.0 ** -15
    y, m = orc.mlp_qmargin(w, dims, x, orc.QUANT_BF16)
    assert abs(m - 2.0 ** -15 / (1.0 + abs(w[78]))) < 1e-15
    _, m_none = orc.mlp_qmargin(w, dims, x, orc.QUANT_NONE)
    assert m_none == math.inf


# ------------------------------------------------------------------------------------------------
# knife-edge diagnostics of queries and frames
# ------------------------------------------------------------------------------------------------
def _flip_net(pre, w_out, b_m=0.0, a=5.0, width=8):
    """One-hidden-layer NeDF weights whose first hidden unit has pre-activation `pre` for every
    input (its bias), every other unit 0; m = b_m + w_out * (that unit, as rounded), a = `a`."""
    dims = sg.mlp_dims(sg.NEDF_IN, 1, width, 2)
    w = np.zeros(sg.mlp_param_count(dims))
    off = sg.NEDF_IN * width
    w[off] = pre                                                 # bias of unit 0, layer 0
    off += width
    w[off] = w_out                                               # W_out[0][0]
    w[off + 2 * width] = b_m
    w[off + 2 * width + 1] = a
    return w.astype(np.float32).astype(np.float64), dims


def test_mlp_flip_rounds_one_value_the_other_way(orc):
    pre = 1.0 + 2.0 ** -8 - 2.0 ** -16                                 # just below the 1 | 1+2^-7 midpoint
    w, dims = _flip_net(pre, 0.5)
    x = np.zeros(sg.NEDF_IN)
    y, ci, cm = orc.mlp_flip(w, dims, x, orc.QUANT_BF16, -1, 3)
    assert abs(y[0] - 0.5 * 1.0) < 1e-15                         # rounds down to 1
    assert ci[0] == sg.NEDF_IN and abs(cm[0] - 2.0 ** -16 / pre) < 1e-12   # unit 0 of layer 0: the knife edge
    yf, _, _ = orc.mlp_flip(w, dims, x, orc.QUANT_BF16, int(ci[0]), 0)
    assert abs(yf[0] - 0.5 * (1.0 + 2.0 ** -7)) < 1e-15          # ... and up when flipped
    assert np.all(np.diff(cm[np.isfinite(cm)]) >= 0)
    # E4M3 (FP8 mode: every hidden activation is E4M3): the grid at 1 is 1/8
    w2, dims2 = _flip_net(1.0 + 2.0 ** -4 + 1e-7, 0.5)
    y2, ci2, _ = orc.mlp_flip(w2, dims2, x, orc.QUANT_FP8, -1, 1)
    yf2, _, _ = orc.mlp_flip(w2, dims2, x, orc.QUANT_FP8, int(ci2[0]), 0)
    assert {round(y2[0] / 0.5, 12), round(yf2[0] / 0.5, 12)} == {1.0, 1.125}


def test_query_spread_is_the_depth_change_of_one_flip(orc):
    """A row with one activation 2^-16 below a BF16 boundary: its depth may move by rb * w_out *
    2^-7; the FP32 mode has no spread."""
    for rb in (1.0, 2.0):
        w, dims = _flip_net(1.0 + 2.0 ** -8 - 2.0 ** -16, 0.25, b_m=0.1)
        sc = one_instance_scene(sg.SDF_SPHERE, nedf_w=w, hidden=1, width=8, rb=rb)
        osc = orc.OracleScene(sc)
        _, _, (mg, dm, dsp) = orc.query_diag(osc, 0, EYE, DIR, quant=orc.QUANT_BF16)
        assert abs(dsp - rb * 0.25 * 2.0 ** -7) < 1e-12 and dm == math.inf
        _, _, (mg, dm, dsp) = orc.query_diag(osc, 0, EYE, DIR)
        assert dsp == 0.0
        # far from any boundary there is nothing to flip
        w, dims = _flip_net(1.0 + 2.0 ** -9, 0.25, b_m=0.1)
        sc = one_instance_scene(sg.SDF_SPHERE, nedf_w=w, hidden=1, width=8, rb=rb)
        assert orc.query_diag(orc.OracleScene(sc), 0, EYE, DIR, quant=orc.QUANT_BF16)[2][2] == 0.0


def _inside_sphere(t, r=0.5):
    """The one-sphere test ray's point at t is inside the r-sphere (closed form: |3 - t| <= r)."""
    return abs(3.0 - t) <= r


CAP = 1e-4      # tests with a larger relative margin are never knife edges and are not recorded


def _capped_min(items, need=0.0):
    return min((r for r, c in items if r < CAP and c >= need), default=math.inf)


@pytest.mark.parametrize("delta", [-3e-4, 2e-4, 0.0251, -0.0124, 0.04])
def test_query_dmargin_of_the_refinement_is_the_closest_tested_point(orc, delta):
    """The refinement tests the window ends and its midpoints; a test's margin is
    | |3 - t| - r | over |o_local| + |t| + rb, and its consequence half its bracket (H, H/2, ...;
    unbounded for the window's ends)."""
    m = _m_for_depth(SURF + delta)
    D0 = _depth_of(m)
    sc = one_instance_scene(sg.SDF_SPHERE, nedf_w=constant_nedf(m, 5.0))
    osc = orc.OracleScene(sc)
    _, out, (mg, dm, dsp) = orc.query_diag(osc, 0, EYE, DIR, refine_steps=4)
    lo, hi = D0 - H, D0 + H
    rel = lambda t: abs(abs(3.0 - t) - 0.5) / (3.0 + abs(t) + 1.0)
    items = [(rel(lo), math.inf), (rel(hi), math.inf)]
    for _ in range(4):
        mid = 0.5 * (lo + hi)
        items.append((rel(mid), 0.5 * (hi - lo)))
        if _inside_sphere(mid):
            hi = mid
        else:
            lo = mid
    assert abs(out[0] - 0.5 * (lo + hi)) < 1e-12 and dsp == 0.0
    assert dm == _capped_min(items) or abs(dm - _capped_min(items)) < 1e-12
    if abs(delta) < 1e-3:
        assert dm < CAP                                          # the first midpoint is D0 itself
    for k in range(5):
        need = H / 2 ** k + 1e-12
        got = orc.query_diag(osc, 0, EYE, DIR, need=need, refine_steps=4)[2][1]
        want = _capped_min(items, need)
        assert got == want or abs(got - want) < 1e-12, k


@pytest.mark.parametrize("n", [16, 13, 29])
def test_query_dmargin_of_the_plain_method(orc, n):
    """MARCH mode: the samples t_k = te + k (tx - te) / N up to the crossing (unbounded
    consequence), then the bisection steps (half their bracket)."""
    sc = one_instance_scene(sg.SDF_SPHERE)
    osc = orc.OracleScene(sc)
    _, out, (mg, dm, _) = orc.query_diag(osc, 0, EYE, DIR, depth_mode=orc.DEPTH_MARCH, march_n=n, march_b=3)
    te, tx = 2.0, 4.0                                            # the unit bound along the axis
    rel = lambda t: abs(abs(3.0 - t) - 0.5) / (3.0 + abs(t) + 1.0)
    items, ts, lo, hi = [], [], None, None
    for k in range(n + 1):
        t = te + (tx - te) * k / n
        ts.append(t)
        items.append((rel(t), math.inf))
        if k > 0 and _inside_sphere(t) and not _inside_sphere(ts[-2]):
            lo, hi = ts[-2], t
            break
    for _ in range(3):
        mid = 0.5 * (lo + hi)
        items.append((rel(mid), 0.5 * (hi - lo)))
        if _inside_sphere(mid):
            hi = mid
        else:
            lo = mid
    assert abs(out[0] - 0.5 * (lo + hi)) < 1e-12
    assert dm == _capped_min(items) or abs(dm - _capped_min(items)) < 1e-12
    big = orc.query_diag(osc, 0, EYE, DIR, need=1.0, depth_mode=orc.DEPTH_MARCH, march_n=n, march_b=3)[2][1]
    assert big == _capped_min(items, 1.0)


def test_frame_gap_is_reduced_by_both_depth_spreads(orc):
    """Two instances with the same knife-edge network one behind the other: the reported gap is
    the depth difference less both instances' flip shifts (BF16), the plain difference in FP32."""
    w, dims = _flip_net(1.0 + 2.0 ** -8 - 2.0 ** -16, 0.25, b_m=0.1)
    t = sg.make_type(sg.SDF_SPHERE, 0, 0, 1, 8, nedf_seed=1)
    t.nedf_w = w.astype(np.float32)
    sc = sg.Scene("two", 33, 33, sg.f32([0, 0, 4]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]), [t],
                  np.zeros(2, np.uint32), sg.f32(np.tile(np.eye(3).reshape(1, 9), (2, 1))),
                  sg.f32([[0, 0, 0.5], [0, 0, -0.25]]), sg.f32([1, 1]))
    px = np.array([16 * 33 + 16])
    o32 = orc.render(orc.OracleScene(sc), px=px)
    ob = orc.render(orc.OracleScene(sc), px=px, quant=orc.QUANT_BF16)
    assert abs(o32["gap"][0] - 0.75) < 1e-6 and o32["dmargin"][0] == math.inf
    assert abs(ob["gap"][0] - (o32["gap"][0] - 2 * 0.25 * 2.0 ** -7)) < 1e-6


def test_frame_alternative_outcome_takes_the_critical_test_the_other_way(orc):
    """Centre pixel of the one-sphere frame, plain-method depths with 16 samples over the bound
    chord [2, 4]: sample 4 lies exactly on the surface (t = 2.5, margin 0).  Taken as inside it ends
    the march there and 3 bisections of [2.375, 2.5] give 2.4921875; taken the other way the
    crossing moves to 2.625 and the bisections of [2.5, 2.625] give 2.5078125."""
    sc = one_instance_scene(sg.SDF_SPHERE)
    px = np.array([32 * 65 + 32])
    o = orc.render(orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=16, march_b=3)
    assert o["depth"][0] == 2.4921875 and o["has_alt"][0] and o["alt_depth"][0] == 2.5078125
    assert o["alt_id"][0] == 0 and o["dmargin"][0] > 1e-6               # no second knife edge
    # the alternative shading is the primary's window moved by the depth difference
    assert not np.allclose(o["alt_rgba"][0], o["rgba"][0], atol=1e-6)
    # a sphere of radius 0.45 puts the surface at 0.275 of the chord, which no sample or
    # bisection midpoint of 17 samples comes within 1e-6 (relative) of: no alternative
    sc45 = one_instance_scene(sg.SDF_SPHERE, params=[0.45])
    o = orc.render(orc.OracleScene(sc45), px=px, depth_mode=orc.DEPTH_MARCH, march_n=17, march_b=3)
    assert not o["has_alt"][0] and np.isnan(o["alt_depth"][0]) and abs(o["depth"][0] - 2.55) < 0.01
    o = orc.render(orc.OracleScene(sc), px=px, alt=False, depth_mode=orc.DEPTH_MARCH, march_n=16, march_b=3)
    assert "has_alt" not in o


# ------------------------------------------------------------------------------------------------
# BF16 training: the gradient with BF16 operands, against torch autograd
# ------------------------------------------------------------------------------------------------
def test_bf16_training_gradient_matches_torch_autograd(orc):
    """The oracle's BF16-mode loss and gradient (reading 29) against torch's autograd in float64 on
    the same rounded operands: weights and layer inputs rounded to BF16 in the forward pass (the
    saved activations are those BF16 values), the error signal of each hidden layer rounded to BF16
    on its way back (a rounding applied to the gradient alone), the loss derivative unrounded."""
    torch = pytest.importorskip("torch")
    hidden, width = 3, 16
    sc = one_instance_scene(sg.SDF_TORUS, params=[0.4, 0.15], hidden=hidden, width=width)
    rng = np.random.default_rng(31)
    t = sc.types[0]
    t.nedf_w = (rng.normal(size=t.nedf_w.shape[0]) * 0.4).astype(np.float32)
    osc = orc.OracleScene(sc)
    o, d = orc.train_rays(1.0, 3, 0, 48)
    m_star, h_star = orc.train_labels(osc, 0, o, d)
    loss_o, g_o = orc.nedf_loss_grad(osc, 0, o, d, m_star, h_star, quant=orc.QUANT_BF16)

    # a rounded operand: the value rounded to BF16, the derivative passed through unchanged
    rnd = lambda x: x.detach().to(torch.float32).to(torch.bfloat16).to(torch.float64)
    bf = lambda x: x + (rnd(x) - x).detach()

    class GradBF16(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            return x.clone()

        @staticmethod
        def backward(ctx, g):
            return rnd(g)

    dims = sg.mlp_dims(sg.NEDF_IN, hidden, width, 2)
    w = torch.tensor(t.nedf_w.astype(np.float64), requires_grad=True)
    feats, keep = [], []
    for k in range(o.shape[0]):
        dd = d[k] / np.linalg.norm(d[k])
        kept, f, _ = orc.nedf_features(o[k], dd, 1.0)
        keep.append(kept)
        feats.append(f if kept else np.zeros(sg.NEDF_IN))
    X = torch.tensor(np.array(feats))
    keep = torch.tensor(keep)
    off, h = 0, bf(X)
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        W = w[off: off + fi * fo].reshape(fo, fi); off += fi * fo
        b = w[off: off + fo]; off += fo
        z = h @ bf(W).T + b
        if l + 1 < len(dims) - 1:
            z = GradBF16.apply(z)                   # the hidden layer's error signal in BF16
            h = bf(torch.relu(z))
        else:
            h = z
    mm, aa = h[:, 0], h[:, 1]
    hs = torch.tensor(h_star.astype(np.float64))
    ms = torch.tensor(m_star)
    bce = torch.clamp(aa, min=0) - hs * aa + torch.log1p(torch.exp(-aa.abs()))
    n_hit = hs.sum()
    loss = (0.1 * bce * keep).sum() / o.shape[0] + ((mm - ms) ** 2 * hs * keep).sum() / n_hit
    loss.backward()
    assert abs(loss.item() - loss_o) < 1e-12
    assert np.allclose(w.grad.numpy(), g_o, rtol=1e-10, atol=1e-13)
    # the unrounded oracle differs from it: the rounding points are real
    _, g_n = orc.nedf_loss_grad(osc, 0, o, d, m_star, h_star)
    assert np.abs(g_n - g_o).max() > 1e-6


def test_mlp_flip2_rounds_two_values_the_other_way(orc):
    """Two hidden units placed just off BF16 rounding boundaries (1 + 2^-8 - 2^-16 rounds to 1, else
    1 + 2^-7; 2 + 2^-7 + 2^-15 rounds to 2 + 2^-6, else 2; both biases exact as two BF16 parts)
    feeding m = h0 / 2 + h1 / 4: each flip and both together give the closed-form outputs."""
    dims = sg.mlp_dims(sg.NEDF_IN, 1, 8, 2)
    w = np.zeros(sg.mlp_param_count(dims))
    off = sg.NEDF_IN * 8
    w[off] = 1.0 + 2.0 ** -8 - 2.0 ** -16
    w[off + 1] = 2.0 + 2.0 ** -7 + 2.0 ** -15
    w[off + 8] = 0.5                                             # W_out[0][0]
    w[off + 8 + 1] = 0.25                                        # W_out[0][1]
    x = np.zeros(sg.NEDF_IN)
    y0, ci, _ = orc.mlp_flip(w, dims, x, orc.QUANT_BF16, -1, 2)
    h0, h1 = sg.NEDF_IN, sg.NEDF_IN + 1                          # value indices of the two units
    assert set(ci.tolist()) == {h0, h1}
    assert y0[0] == 0.5 * 1.0 + 0.25 * (2.0 + 2.0 ** -6)
    assert orc.mlp_flip(w, dims, x, orc.QUANT_BF16, h0, 0)[0][0] == 0.5 * (1.0 + 2.0 ** -7) + 0.25 * (2.0 + 2.0 ** -6)
    assert orc.mlp_flip(w, dims, x, orc.QUANT_BF16, h1, 0)[0][0] == 0.5 * 1.0 + 0.25 * 2.0
    assert orc.mlp_flip2(w, dims, x, orc.QUANT_BF16, h0, h1)[0] == 0.5 * (1.0 + 2.0 ** -7) + 0.25 * 2.0
    assert orc.mlp_flip2(w, dims, x, orc.QUANT_BF16, h0, h0)[0] == orc.mlp_flip(w, dims, x, orc.QUANT_BF16, h0, 0)[0][0]


def test_mlp_flipset_rounds_any_set_of_values_the_other_way(orc):
    """Three hidden units just off BF16 rounding boundaries (the two of the two-flip pin plus
    4 + 2^-6 - 2^-14, which rounds to 4, else 4 + 2^-5) feeding m = h0 / 2 + h1 / 4 + h2 / 8: every
    subset of flips gives its closed-form output, the empty set the plain rounding."""
    import itertools
    dims = sg.mlp_dims(sg.NEDF_IN, 1, 8, 2)
    w = np.zeros(sg.mlp_param_count(dims))
    off = sg.NEDF_IN * 8
    w[off] = 1.0 + 2.0 ** -8 - 2.0 ** -16
    w[off + 1] = 2.0 + 2.0 ** -7 + 2.0 ** -15
    w[off + 2] = 4.0 + 2.0 ** -6 - 2.0 ** -14
    w[off + 8], w[off + 9], w[off + 10] = 0.5, 0.25, 0.125       # W_out[0][0 .. 2]
    x = np.zeros(sg.NEDF_IN)
    units = [sg.NEDF_IN, sg.NEDF_IN + 1, sg.NEDF_IN + 2]
    plain = [1.0, 2.0 + 2.0 ** -6, 4.0]
    other = [1.0 + 2.0 ** -7, 2.0, 4.0 + 2.0 ** -5]
    _, ci, _ = orc.mlp_flip(w, dims, x, orc.QUANT_BF16, -1, 3)
    assert set(ci.tolist()) == set(units)
    for k in range(4):
        for sub in itertools.combinations(range(3), k):
            h = [other[j] if j in sub else plain[j] for j in range(3)]
            y = orc.mlp_flipset(w, dims, x, orc.QUANT_BF16, [units[j] for j in sub])
            assert y[0] == 0.5 * h[0] + 0.25 * h[1] + 0.125 * h[2], sub


# ------------------------------------------------------------------------------------------------
# miss check (reading 30): a confident miss verified by density samples along the bound chord
# ------------------------------------------------------------------------------------------------
def test_confident_miss_through_the_object_is_re_answered(orc):
    """The network says 'miss' with confidence 0.993 (a = -5) on a ray through the sphere: with the
    miss check the plain method answers (the surface at 2.5); without it the miss stands."""
    hit, D = _query(orc, _m_for_depth(2.8), -5.0, fallback_conf=0.9, miss_check=16)
    assert hit and abs(D - SURF) < 1e-9
    hit, _ = _query(orc, _m_for_depth(2.8), -5.0, fallback_conf=0.9, miss_check=0)
    assert not hit


def test_miss_check_keeps_true_misses_and_ignores_hits(orc):
    """A ray through the bound that passes the sphere (offset 0.7 > r = 0.5) stays a miss with no
    plain-method work; a confident hit is not sampled (the check is for misses only)."""
    sc = one_instance_scene(sg.SDF_SPHERE, nedf_w=constant_nedf(_m_for_depth(2.8), -5.0))
    osc = orc.OracleScene(sc)
    eye = np.array([0.0, 0.7, 3.0])
    hit, out, (mg, dm, _) = orc.query_diag(osc, 0, eye, DIR, need=np.inf, fallback_conf=0.9, miss_check=16,
                                           march_n=4096, march_b=60)
    assert not hit and out[3] < out[4]                   # inside the bound, no crossing
    # the 16 midpoints' margins: | |p| - 0.5 | over |o| + |t| + 1, the smallest at the closest approach
    te, tx = out[3], out[4]
    ts = te + (np.arange(16) + 0.5) * (tx - te) / 16
    rel = np.abs(np.linalg.norm(eye[None, :] + ts[:, None] * DIR[None, :], axis=1) - 0.5) / (np.linalg.norm(eye) + ts + 1)
    assert dm == math.inf or abs(dm - rel.min()) < 1e-12     # margins above 1e-4 are not recorded
    hit, D = _query(orc, _m_for_depth(2.8), 5.0, miss_check=16)
    assert hit and abs(D - _depth_of(_m_for_depth(2.8))) < 1e-12
