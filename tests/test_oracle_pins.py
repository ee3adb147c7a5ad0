"""Pins of the FP64 oracle against things other than itself.

Each test checks an oracle function against a closed form, an invariant, an independent library
routine, brute force, or a number the paper prints (tests/golden/paper_constants.json), chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails at least one of them.
"""
import copy
import json
import math
import os

import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_instance_scene(kind, params=None, W=65, H=65, eye=(0, 0, 3), s=1.0, T=(0, 0, 0), R=None,
                       rb=1.0, lights=((2, 3, 2),), hidden=2, width=8, nedf_w=None):
    t = sg.make_type(kind, 0, 0, hidden, width, rb=rb, params=params, nedf_seed=11)
    if nedf_w is not None:
        t.nedf_w = nedf_w
    return sg.Scene("t", W, H, sg.f32(eye), sg.f32([0, 0, 0]), 40.0, sg.f32(lights), [t],
                    np.zeros(1, np.uint32), sg.f32((np.eye(3) if R is None else R).reshape(1, 9)),
                    sg.f32([T]), sg.f32([s]))


def constant_nedf(m, a, hidden=2, width=8):
    """Packed NeDF weights whose output is the constant (m, a): all weights zero, output bias."""
    dims = sg.mlp_dims(sg.NEDF_IN, hidden, width, 2)
    w = np.zeros(sg.mlp_param_count(dims), np.float32)
    w[-2:] = [m, a]
    return w


# ------------------------------------------------------------------------------------------------
# Random streams
# ------------------------------------------------------------------------------------------------
def test_splitmix64_published_vectors(orc):
    # First outputs of SplitMix64 from state 0 and from state 1234567 (Steele et al. 2014;
    # the values quoted with the reference implementation used to seed xoshiro generators).
    assert [int(x) for x in sg.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert int(sg.splitmix64(1234567, 1)[0]) == 6457827717110365317
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF and orc.splitmix64(0, 2) == 0x06C45D188009454F


# ------------------------------------------------------------------------------------------------
# Camera, transform, bound
# ------------------------------------------------------------------------------------------------
def test_camera_pinhole_closed_form(orc):
    sc = one_instance_scene(sg.SDF_SPHERE, W=65, H=33)
    osc = orc.OracleScene(sc)
    th = math.tan(math.radians(20.0))
    o, d = orc.camera_ray(osc, 32, 16)            # centre pixel (odd sizes) looks at the target
    assert np.allclose(o, [0, 0, 3]) and np.allclose(d, [0, 0, -1], atol=1e-15)
    _, d = orc.camera_ray(osc, 32, 0)             # top row, centre column: elevation angle
    assert math.isclose(math.atan2(d[1], -d[2]), math.atan((1 - 1 / 33) * th), rel_tol=1e-13)
    assert d[0] == pytest.approx(0.0, abs=1e-15)
    _, d = orc.camera_ray(osc, 64, 16)            # right edge (+x when looking down -z)
    assert math.isclose(math.atan2(d[0], -d[2]), math.atan((1 - 1 / 65) * th * 65 / 33), rel_tol=1e-13)
    for (i, j) in [(0, 0), (5, 7), (64, 32)]:
        _, d = orc.camera_ray(osc, i, j)
        assert abs(np.linalg.norm(d) - 1) < 1e-15


def test_transform_round_trip_and_scale(orc):
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.linalg.det(q))
    sc = one_instance_scene(sg.SDF_SPHERE, s=2.5, T=(0.3, -1.2, 0.7))
    osc = orc.OracleScene(sc)
    osc.R[:] = q.reshape(-1)                       # exact float64 rotation (no f32 rounding)
    T, s = osc.T.copy(), osc.s[0]
    for _ in range(5):
        x = rng.normal(size=3) * 4
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        ol, dl = orc.to_local(osc, 0, x, d)
        assert np.allclose(s * q @ ol + T, x, atol=1e-13)        # G(G^-1(x)) = x
        assert np.allclose(q @ dl, d, atol=1e-14)                # direction rotates back
        assert abs(np.linalg.norm(dl) - 1) < 1e-15


def test_bound_closed_forms(orc):
    kept, b = orc.bound([0, 0, 3], [0, 0, -1], 1.0)
    assert kept and np.allclose(b, [2, 4, 3, 1])                 # te, tx, t_perp, disc
    kept, b = orc.bound([0, 1.5, 3], [0, 0, -1], 1.0)
    assert not kept and b[3] == pytest.approx(-1.25)             # misses: disc < 0
    kept, _ = orc.bound([0, 0, -3], [0, 0, -1], 1.0)
    assert not kept                                              # sphere behind the origin
    kept, b = orc.bound([0, 0, 0.5], [0, 0, -1], 1.0)
    assert kept and np.allclose(b[:3], [0, 1.5, 0.5])            # origin inside: te clamps to 0
    kept, b = orc.bound([0, 0, 3], [0, 0, -1], 2.0)
    assert kept and np.allclose(b[:2], [1, 5])


# ------------------------------------------------------------------------------------------------
# Encoding and networks
# ------------------------------------------------------------------------------------------------
def test_posenc_layout_and_paper_input_dim(orc):
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    x = np.array([0.3, -1.1, 2.0])
    f = orc.posenc(x, 10)
    # Appendix A: 16 points x 10-level encoding = 1008 inputs, so the identity is included.
    assert f.shape[0] * g["points_per_ray"]["value"] == g["nedf_input_dim"]["value"]
    assert np.array_equal(f[:3], x)
    for k in range(10):
        assert np.allclose(f[3 + 3 * k: 6 + 3 * k], np.sin(x * 2.0 ** k), atol=0, rtol=1e-15)
        assert np.allclose(f[33 + 3 * k: 36 + 3 * k], np.cos(x * 2.0 ** k), atol=0, rtol=1e-15)
    assert orc.posenc(np.zeros(6), 6).shape[0] == sg.NEDF_IN == 78
    assert sg.NERF_IN == 90


def test_paper_network_parameter_count():
    """Appendix A architecture -> about 2.41 M parameters = 9.2 MiB FP32, consistent with the
    printed 13 MB for NeDF + NeRF of which 3 MB is the NeRF (Section 'Storage and Speed')."""
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    Di, Df, nb = g["nedf_input_dim"]["value"], g["feature_dim"]["value"], g["residual_blocks"]["value"]
    Nc, Nf = g["coarse_bins"]["value"], g["fine_bins"]["value"]
    params = (Di * Df + Df) + nb * 2 * (Df * Df + Df) + (Df * (Nc + 1) + Nc + 1) + (Df * Nf + Nf)
    mb = params * 4 / 1e6
    total, nerf = g["storage_nedf_plus_nerf_mb"]["value"], g["storage_nerf_mb"]["value"]
    assert abs(mb - (total - nerf)) < 0.7


def test_mlp_matches_torch_float64(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    dims = [78, 32, 32, 32, 2]
    w = rng.normal(size=sg.mlp_param_count(dims)) * 0.3
    x = rng.normal(size=78)
    y = orc.mlp(w, dims, x)
    h = torch.tensor(x, dtype=torch.float64)
    off = 0
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        W = torch.tensor(w[off: off + fi * fo].reshape(fo, fi)); off += fi * fo
        b = torch.tensor(w[off: off + fo]); off += fo
        h = torch.nn.functional.linear(h, W, b)
        if l + 1 < len(dims) - 1:
            h = torch.relu(h)
    assert np.allclose(y, h.numpy(), rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    xs = np.concatenate([(rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000)).astype(np.float32),
                         np.float32([1.00390625, 1.01171875, -3.0078125, 0.0])])   # ties to even
    ref = torch.tensor(xs).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.round_bf16(float(v)) for v in xs])
    assert np.array_equal(got, ref)


def test_e4m3_rounding_matches_torch_and_closed_forms(orc):
    """OCP E4M3: 3 fraction bits, normals from 2^-6, subnormal spacing 2^-9, largest finite 448."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    xs = rng.normal(size=4000) * 10.0 ** rng.uniform(-3.5, 2.3, 4000)
    xs = xs[np.abs(xs) < 440.0]
    ref = torch.tensor(xs).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([orc.round_e4m3(float(v)) for v in xs])
    assert np.array_equal(got, ref)
    # representable values are fixed points; the grid around 1 is 1/8
    for v in (1.0, 1.125, 1.875, 448.0, 2.0 ** -6, 2.0 ** -9, 7 * 2.0 ** -9, -240.0):
        assert orc.round_e4m3(v) == v
    assert orc.round_e4m3(1.0625) == 1.0 and orc.round_e4m3(1.1875) == 1.25        # ties to even
    assert orc.round_e4m3(2.0 ** -10) == 0.0 and orc.round_e4m3(3 * 2.0 ** -11) == 2.0 ** -9
    assert orc.round_e4m3(500.0) == 448.0 and orc.round_e4m3(-1e6) == -448.0      # saturation
    assert orc.round_e4m3(0.0) == 0.0


def test_fp8_scale_is_the_power_of_two_filling_the_e4m3_range(orc):
    for m in (448.0, 449.0, 0.1, 224.0, 224.0001, 3.0e-5, 1.0):
        s = orc.fp8_scale(m)
        assert s == 2.0 ** np.round(np.log2(s))
        assert 224.0 < m / s <= 448.0
    assert orc.fp8_scale(0.0) == 1.0


def test_mlp_fp8_mode_matches_torch_float8(orc):
    """FP8 mode: layer 0 in BF16, hidden layers' weights s * E4M3(W / s), activations E4M3, output
    layer weights BF16; checked against torch's own float8 / bfloat16 casts and float64 matmuls."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    dims = [78, 64, 64, 64, 2]
    w = (rng.normal(size=sg.mlp_param_count(dims)) * 0.2).astype(np.float32).astype(np.float64)
    x = rng.normal(size=78).astype(np.float32).astype(np.float64)
    y = orc.mlp(w, dims, x, quant=orc.QUANT_FP8)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))
    bf = lambda a: t(a).to(torch.float32).to(torch.bfloat16).to(torch.float64)
    f8 = lambda a: t(a).to(torch.float8_e4m3fn).to(torch.float64)
    h = bf(x)
    off = 0
    n = len(dims) - 1
    for l in range(n):
        fi, fo = dims[l], dims[l + 1]
        W = w[off: off + fi * fo].reshape(fo, fi); off += fi * fo
        b = t(w[off: off + fo]); off += fo
        if l == 0:                               # the BF16 first layer: the bias as two BF16 parts
            b = bf(b.numpy()) + bf((b - bf(b.numpy())).numpy())
        if 0 < l < n - 1:
            s = 2.0 ** np.ceil(np.log2(np.abs(W).max() / 448.0))
            Wq = s * f8(W / s)
        else:
            Wq = bf(W)
        h = h @ Wq.T + b
        if l + 1 < n:
            h = f8(torch.relu(h).numpy())
    assert np.allclose(y, h.numpy(), rtol=1e-12, atol=1e-12)


def test_mlp_bf16_mode_matches_torch_rounded_operands(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    dims = [78, 64, 64, 2]
    w = (rng.normal(size=sg.mlp_param_count(dims)) * 0.2).astype(np.float32).astype(np.float64)
    x = rng.normal(size=78).astype(np.float32).astype(np.float64)
    y = orc.mlp(w, dims, x, quant=orc.QUANT_BF16)
    bf = lambda a: torch.tensor(a).to(torch.float32).to(torch.bfloat16).to(torch.float64)
    h = torch.tensor(x)
    off = 0
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        W = bf(w[off: off + fi * fo].reshape(fo, fi)); off += fi * fo
        b = torch.tensor(w[off: off + fo]); off += fo
        if l + 1 < len(dims) - 1:                # hidden layers: the bias as two BF16 parts
            b = bf(b.numpy()) + bf((b - bf(b.numpy())).numpy())
        hq = bf(h.numpy()) if l else bf(x)
        h = hq @ W.T + b
        if l + 1 < len(dims) - 1:
            h = torch.relu(h)
    assert np.allclose(y, h.numpy(), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------------
# Depth: closed forms, the plain method's convergence, Eq. 2 worked example
# ------------------------------------------------------------------------------------------------
def torus_first_root(o, d, R, r, te, tx):
    """Smallest real root in [te, tx] of (|p|^2 + R^2 - r^2)^2 = 4 R^2 (px^2 + pz^2), p = o + t d."""
    o, d = np.asarray(o, float), np.asarray(d, float)
    dd, od, oo = d @ d, o @ d, o @ o
    k = oo + R * R - r * r
    # (dd t^2 + 2 od t + k)^2 - 4R^2((dx^2+dz^2) t^2 + 2(ox dx + oz dz) t + ox^2 + oz^2)
    a2 = d[0] ** 2 + d[2] ** 2
    a1 = 2 * (o[0] * d[0] + o[2] * d[2])
    a0 = o[0] ** 2 + o[2] ** 2
    poly = np.polymul([dd, 2 * od, k], [dd, 2 * od, k])
    poly = np.polysub(poly, 4 * R * R * np.array([a2, a1, a0]))
    roots = np.roots(poly)
    real = sorted(x.real for x in roots if abs(x.imag) < 1e-7 and te <= x.real <= tx)
    return real[0] if real else None


def test_exact_depth_closed_forms(orc):
    rng = np.random.default_rng(9)
    n_torus = 0
    for _ in range(400):
        o = rng.normal(size=3); o = 3 * o / np.linalg.norm(o)
        tgt = rng.uniform(-0.6, 0.6, size=3)
        d = tgt - o; d /= np.linalg.norm(d)
        kept, b = orc.bound(o, d, 1.0)
        assert kept
        # sphere r = 0.5: |o + t d| = r
        hit, D = orc.exact_depth(sg.SDF_SPHERE, [0.5], o, d, b[0], b[1])
        bb, cc = o @ d, o @ o - 0.25
        if bb * bb - cc >= 0:
            assert hit and abs(D - (-bb - math.sqrt(bb * bb - cc))) < 1e-12
        else:
            assert not hit
        # torus: quartic roots from numpy (independent of the oracle's scan)
        hit, D = orc.exact_depth(sg.SDF_TORUS, [0.4, 0.15], o, d, b[0], b[1])
        ref = torus_first_root(o, d, 0.4, 0.15, b[0], b[1])
        assert hit == (ref is not None)
        if ref is not None:
            n_torus += 1
            assert abs(D - ref) < 1e-7
        # box: brute-force scan of |x|_inf style containment on a very fine grid
        hit, D = orc.exact_depth(sg.SDF_BOX, [0.35, 0.35, 0.35], o, d, b[0], b[1])
        ts = np.linspace(b[0], b[1], 200001)
        inside = np.all(np.abs(o[None] + ts[:, None] * d[None]) <= 0.35, axis=1)
        if inside.any():
            assert hit and abs(D - ts[np.argmax(inside)]) <= (b[1] - b[0]) / 200000 + 1e-12
        else:
            assert not hit
    assert n_torus > 50


def test_march_converges_to_exact(orc):
    sc = one_instance_scene(sg.SDF_SPHERE)
    osc = orc.OracleScene(sc)
    rng = np.random.default_rng(10)
    for _ in range(50):
        o = rng.normal(size=3); o = 3 * o / np.linalg.norm(o)
        d = rng.uniform(-0.4, 0.4, size=3) - o; d /= np.linalg.norm(d)
        _, b = orc.bound(o, d, 1.0)
        h1, Dm = orc.march_depth(osc, 0, o, d, b[0], b[1], 4096, 60)
        h2, De = orc.exact_depth(sg.SDF_SPHERE, [0.5], o, d, b[0], b[1])
        assert h1 == h2
        if h1:
            assert abs(Dm - De) < 1e-9   # sigmoid(0) = 1/2: the half-density level is sdf = 0


def test_eq2_worked_example(orc):
    """Ray along -z from (0,0,3), sphere r = 0.5 inside the unit bound: t_perp = 3, D = 2.5, so
    mu* = 0.5 (Eq. 2).  A network that outputs m = mu / l reproduces D; scale s multiplies it."""
    sc = one_instance_scene(sg.SDF_SPHERE)
    osc = orc.OracleScene(sc)
    m, h = orc.train_labels(osc, 0, np.array([[0, 0, 1.0]]), np.array([[0, 0, -1.0]]), 256, 8)
    # the label ray starts on the bound at z = 1: t_perp = 1, D = 0.5, mu = 0.5, m = mu / rb
    assert h[0] == 1 and abs(m[0] - 0.5) < 2.0 / 256 / 2 ** 8
    for s, rb in [(1.0, 1.0), (2.0, 1.0), (1.0, 2.0)]:
        scn = one_instance_scene(sg.SDF_SPHERE, s=s, rb=rb, nedf_w=constant_nedf(0.5 / rb, 1.0))
        o2 = orc.OracleScene(scn)
        hit, q, _ = orc.query(o2, 0, np.array([0, 0, 3.0]), np.array([0, 0, -1.0]))
        assert hit
        assert abs(q[5] - 3.0 / s) < 1e-14                       # local t_perp
        assert abs(s * q[0] - (3.0 - s * 0.5)) < 1e-14           # Eq. 7: D = |o-p| - s mu
    # negative logit or depth behind the origin -> no hit
    o3 = orc.OracleScene(one_instance_scene(sg.SDF_SPHERE, nedf_w=constant_nedf(0.5, -1.0)))
    assert not orc.query(o3, 0, np.array([0, 0, 3.0]), np.array([0, 0, -1.0]))[0]
    o4 = orc.OracleScene(one_instance_scene(sg.SDF_SPHERE, nedf_w=constant_nedf(3.5, 1.0)))
    assert not orc.query(o4, 0, np.array([0, 0, 3.0]), np.array([0, 0, -1.0]))[0]


def test_scaled_instance_world_depth(orc):
    for s in [0.5, 1.0, 2.0]:
        sc = one_instance_scene(sg.SDF_SPHERE, s=s, T=(0.2, -0.1, 0.0), W=65, H=65)
        r = orc.render(orc.OracleScene(sc), px=np.array([32 * 65 + 32]), depth_mode=orc.DEPTH_EXACT)
        c = sg.f32([0.2, -0.1, 0.0]).astype(float); o = np.array([0, 0, 3.0]); d = np.array([0, 0, -1.0])
        bb = (o - c) @ d; cc = (o - c) @ (o - c) - (0.5 * s) ** 2
        assert abs(r["depth"][0] - (-bb - math.sqrt(bb * bb - cc))) < 1e-12


# ------------------------------------------------------------------------------------------------
# Step 1: z-min (Algorithm 1) -- brute force, ties, permutation invariance
# ------------------------------------------------------------------------------------------------
def two_sphere_scene(T0, T1, W=33, H=33):
    t = sg.make_type(sg.SDF_SPHERE, 0, 0, 2, 8, nedf_seed=1)
    return sg.Scene("two", W, H, sg.f32([0, 0, 4]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]), [t],
                    np.zeros(2, np.uint32), sg.f32(np.tile(np.eye(3).reshape(1, 9), (2, 1))),
                    sg.f32([T0, T1]), sg.f32([1, 1]))


def test_zmin_nearest_and_lowest_id_on_ties(orc):
    r = orc.render(orc.OracleScene(two_sphere_scene((0, 0, -1.0), (0, 0, 1.0))), px=np.array([16 * 33 + 16]),
                   depth_mode=orc.DEPTH_EXACT)
    assert r["id"][0] == 1 and abs(r["depth"][0] - 2.5) < 1e-12 and abs(r["gap"][0] - 2.0) < 1e-12
    r = orc.render(orc.OracleScene(two_sphere_scene((0, 0, 0.5), (0, 0, 0.5))), depth_mode=orc.DEPTH_EXACT)
    hit = r["id"] != 0xFFFFFFFF
    assert hit.sum() > 20 and np.all(r["id"][hit] == 0) and np.all(r["gap"][hit] == 0)


def test_zmin_permutation_invariance(orc):
    sc = sg.three_types_scene(48, 48, nerf=False)
    perm = np.random.default_rng(2).permutation(sc.n_inst)
    for mode in (orc.DEPTH_MLP, orc.DEPTH_EXACT):
        a = orc.render(orc.OracleScene(sc), depth_mode=mode)
        b = orc.render(orc.OracleScene(sc.permuted(perm)), depth_mode=mode)
        assert np.array_equal(a["depth"], b["depth"])
        hit = a["id"] != 0xFFFFFFFF
        assert hit.sum() > 100
        ok = hit & (a["gap"] > 1e-4)
        assert np.array_equal(a["id"][ok], perm[b["id"][ok]])
        assert np.array_equal(b["id"] == 0xFFFFFFFF, ~hit)


def test_zmin_brute_force_exact(orc):
    """Depth buffer = min over instances of the closed-form sphere depth (spheres only)."""
    rng = np.random.default_rng(12)
    t = sg.make_type(sg.SDF_SPHERE, 0, 0, 2, 8, nedf_seed=1)
    n = 12
    T = sg.f32(rng.uniform(-1.5, 1.5, size=(n, 3)))
    sc = sg.Scene("b", 24, 24, sg.f32([0, 0, 6]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]), [t],
                  np.zeros(n, np.uint32), sg.f32(np.tile(np.eye(3).reshape(1, 9), (n, 1))), T,
                  sg.f32(np.ones(n)))
    osc = orc.OracleScene(sc)
    r = orc.render(osc, depth_mode=orc.DEPTH_EXACT)
    for p in range(24 * 24):
        o, d = orc.camera_ray(osc, p % 24, p // 24)
        best, bid = np.inf, 0xFFFFFFFF
        for m in range(n):
            c = T[m].astype(float)
            bb = (o - c) @ d; cc = (o - c) @ (o - c) - 0.25
            if bb * bb - cc >= 0 and -bb - math.sqrt(bb * bb - cc) > 0:
                D = -bb - math.sqrt(bb * bb - cc)
                if D < best:
                    best, bid = D, m
        assert r["id"][p] == bid
        if bid != 0xFFFFFFFF:
            assert abs(r["depth"][p] - best) < 1e-12


# ------------------------------------------------------------------------------------------------
# Step 2: shading quadrature (Eq. 8 over the sample window)
# ------------------------------------------------------------------------------------------------
def test_composite_constant_slab_and_empty(orc):
    for sig, n, dl in [(3.0, 8, 0.0125), (50.0, 8, 0.0125), (0.7, 16, 0.1)]:
        c = np.array([0.2, 0.5, 0.9])
        out = orc.composite_samples(np.full(n, sig), np.tile(c, n), dl)
        A = 1 - math.exp(-sig * n * dl)                        # 1 - exp(-sigma L)
        assert abs(out[3] - A) < 1e-14 and np.allclose(out[:3], c * A, rtol=1e-13)
    out = orc.composite_samples(np.zeros(8), np.ones(24), 0.0125)
    assert np.all(out == 0)
    out = orc.composite_samples(np.array([1e9, 5.0]), np.array([1, 0, 0, 0, 1, 0.0]), 0.1)
    assert abs(out[3] - 1) < 1e-15 and abs(out[0] - 1) < 1e-15 and abs(out[1]) < 1e-15


def test_shading_window_centred_on_surface(orc):
    """Head-on ray at a sphere: sdf along the ray is D - t, antisymmetric about the surface, so the
    window's densities pair up to sigma_max and sum to (n/2) sigma_max; A = 1 - exp(-s dt n sigma_max / 2)."""
    for s in [1.0, 2.0]:
        sc = one_instance_scene(sg.SDF_SPHERE, s=s, W=65, H=65)
        r = orc.render(orc.OracleScene(sc), px=np.array([32 * 65 + 32]), depth_mode=orc.DEPTH_EXACT)
        dt = 2 * float(np.float32(0.05)) / 8
        A = 1 - math.exp(-s * dt * 4 * 50.0)
        assert abs(r["rgba"][0, 3] - A) < 1e-9
        assert np.allclose(r["rgba"][0, :3], np.float32(0.7) * r["rgba"][0, 3], rtol=1e-12)


# ------------------------------------------------------------------------------------------------
# Step 3: shadows (Algorithm 2)
# ------------------------------------------------------------------------------------------------
def point_segment_distance(c, a, b):
    ab = b - a
    t = np.clip((c - a) @ ab / (ab @ ab), 0, 1)
    return np.linalg.norm(a + t * ab - c)


def test_sphere_on_plane_shadow(orc):
    floor = sg.make_type(sg.SDF_BOX, 0, 0, 2, 8, params=[4.0, 0.05, 4.0], rb=5.7, nedf_seed=2)
    ball = sg.make_type(sg.SDF_SPHERE, 0, 1, 2, 8, nedf_seed=3)
    L = np.array([0.7, 5.0, 0.3])
    sc = sg.Scene("plane", 48, 48, sg.f32([0, 4, 5]), sg.f32([0, 0, 0]), 40.0, sg.f32([L]), [floor, ball],
                  np.array([0, 1], np.uint32), sg.f32(np.tile(np.eye(3).reshape(1, 9), (2, 1))),
                  sg.f32([[0, -0.05, 0], [0, 0.6, 0]]), sg.f32([1, 1]))
    osc = orc.OracleScene(sc)
    r = orc.render(osc, depth_mode=orc.DEPTH_EXACT)
    c = np.array([0, 0.6, 0])
    floor_px = np.nonzero(r["id"] == 0)[0]
    n_shadow = n_checked = 0
    for k in floor_px:
        o, d = orc.camera_ray(osc, k % 48, k // 48)
        x = o + r["depth"][k] * d
        dist = point_segment_distance(c, L, x)
        if abs(dist - 0.5) < 1e-3:
            continue
        n_checked += 1
        expect = 0.5 if dist < 0.5 else 1.0
        n_shadow += expect == 0.5
        assert r["shadow"][k] == expect
    assert n_checked > 500 and n_shadow > 20


def test_single_sphere_self_shadow_terminator(orc):
    sc = sg.tiny_sphere_scene()
    osc = orc.OracleScene(sc)
    r = orc.render(osc, depth_mode=orc.DEPTH_EXACT)
    L = np.array([2.0, 3.0, 2.0])
    checked = 0
    for k in np.nonzero(r["id"] == 0)[0]:
        o, d = orc.camera_ray(osc, k % 64, k // 64)
        x = o + r["depth"][k] * d
        n = x / np.linalg.norm(x)
        cosl = n @ (L - x) / np.linalg.norm(L - x)
        if abs(cosl) < 0.1:
            continue
        checked += 1
        assert r["shadow"][k] == (1.0 if cosl > 0 else 0.5)
        assert np.allclose(r["out"][k, :3], r["rgba"][k, :3] * r["shadow"][k])
    assert checked > 300
    miss = r["id"] == 0xFFFFFFFF
    assert np.all(r["shadow"][miss] == 1) and np.all(r["rgba"][miss] == 0) and np.all(np.isinf(r["depth"][miss]))


# ------------------------------------------------------------------------------------------------
# Plain method colour (front-to-back volume rendering)
# ------------------------------------------------------------------------------------------------
def test_volume_render_opaque_centre_and_empty_corner(orc):
    sc = one_instance_scene(sg.SDF_SPHERE, W=65, H=65)
    osc = orc.OracleScene(sc)
    rgba = orc.volume_render(osc, 128, px=np.array([32 * 65 + 32, 0]))
    assert abs(rgba[0, 3] - 1) < 1e-12 and np.allclose(rgba[0, :3], np.float32(0.7), rtol=1e-12)
    assert np.all(rgba[1] == 0)                                  # corner ray misses the bound


# ------------------------------------------------------------------------------------------------
# Learned part: sampler statistics, loss of a constant network, finite differences, Adam
# ------------------------------------------------------------------------------------------------
def test_train_rays_distribution(orc):
    o, d = orc.train_rays(1.0, 2, 0, 100000)
    assert np.allclose(np.linalg.norm(o, axis=1), 1, atol=1e-12)
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-12)
    cos = -(o * d).sum(1)
    assert np.all(cos >= -1e-12)
    assert abs(cos.mean() - 2.0 / 3.0) < 5e-3                   # cosine-weighted: E[cos] = 2/3
    assert np.all(np.abs(o.mean(0)) < 1e-2)                     # uniform on the sphere
    o2, d2 = orc.train_rays(1.0, 2, 500, 10)                    # counter based: ray r is ray r
    assert np.array_equal(o2, o[500:510]) and np.array_equal(d2, d[500:510])


def test_loss_of_constant_network(orc):
    sc = one_instance_scene(sg.SDF_SPHERE, nedf_w=constant_nedf(0.3, -0.4))
    osc = orc.OracleScene(sc)
    o, d = orc.train_rays(1.0, 7, 0, 64)
    m, h = orc.train_labels(osc, 0, o, d)
    loss, _ = orc.nedf_loss_grad(osc, 0, o, d, m, h)
    hit = h == 1
    assert 5 < hit.sum() < 60
    m0, a0 = float(np.float32(0.3)), float(np.float32(-0.4))   # the network's stored outputs
    bce_hit = math.log1p(math.exp(-a0))     # BCE(a, 1) = softplus(-a)
    bce_miss = math.log1p(math.exp(a0))     # BCE(a, 0) = softplus(a)
    ref = ((m0 - m[hit]) ** 2).mean() + 0.1 * (hit.sum() * bce_hit + (~hit).sum() * bce_miss) / 64
    assert abs(loss - ref) < 1e-13


@pytest.mark.parametrize("hidden,width", [(2, 8), (3, 16)])
def test_gradient_central_differences(orc, hidden, width):
    sc = one_instance_scene(sg.SDF_TORUS, params=[0.4, 0.15], hidden=hidden, width=width)
    rng = np.random.default_rng(hidden)
    t = sc.types[0]
    t.nedf_w = (rng.normal(size=t.nedf_w.shape[0]) * 0.4).astype(np.float32)
    osc = orc.OracleScene(sc)
    o, d = orc.train_rays(1.0, 3, 0, 24)
    m, h = orc.train_labels(osc, 0, o, d)
    assert 0 < h.sum() < 24
    w0 = t.nedf_w.astype(np.float64)
    _, g = orc.nedf_loss_grad(osc, 0, o, d, m, h)
    idx = rng.choice(w0.shape[0], 40, replace=False)
    for i in idx:
        vals = []
        for sgn in (+1, -1):
            w = w0.copy(); w[i] += sgn * 1e-6
            o2 = orc.OracleScene(sc, nedf_override={0: w})
            vals.append(orc.nedf_loss_grad(o2, 0, o, d, m, h)[0])
        fd = (vals[0] - vals[1]) / 2e-6
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9


def test_adam_first_step_is_signed_lr(orc):
    theta = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, -1e-2])
    m, v = np.zeros(4), np.zeros(4)
    orc.adam(theta, g, m, v, 1, 1e-3)
    assert np.allclose(theta, np.array([1.0, -2.0, 0.5, 3.0]) - 1e-3 * np.sign(g), rtol=0, atol=1e-3 * 1e-5)


def _sphere_sample_smax(o, d, depth, n=8):
    """Largest density over the n midpoint samples of [D - h, D + h] on the world ray (identity
    instance): the analytic sphere density 50 sigmoid(-(|x| - 0.5) / w), in closed form, with the
    scene's FP32 constants h = 0.05 and w = 0.01 as the oracle and the GPU receive them."""
    h, w = float(np.float32(0.05)), float(np.float32(0.01))
    ts = depth - h + (np.arange(n) + 0.5) * (2 * h / n)
    x = o[None, :] + ts[:, None] * d[None, :]
    sdf = np.linalg.norm(x, axis=1) - 0.5
    return float(np.max(50.0 / (1.0 + np.exp(sdf / w))))


def test_shade_outlier_resampling(orc):
    """Step-2 outlier resampling ("rs", Section "Deferred Shading"; threshold 1 = 2 % of the peak
    density, the reading of "extremely small"): on the tiny sphere with the untrained 4x64 NeDF,
    whose depths mostly miss the surface, a pixel is re-rendered exactly when the largest of its 8
    sample densities (closed form) is below the threshold; a re-rendered pixel whose ray passes deep
    through the sphere gets the volume-rendered colour of an opaque albedo-0.7 object, (0.7, 0.7,
    0.7, 1) (the quadrature telescopes to c (1 - T) and T vanishes); every other pixel keeps its
    deferred-shading colour; with exact depths nothing is re-rendered."""
    sc = sg.tiny_sphere_scene()
    osc = orc.OracleScene(sc)
    base = orc.render(osc, depth_mode=orc.DEPTH_MLP, n_threads=4)
    rs = orc.render(osc, depth_mode=orc.DEPTH_MLP, n_threads=4, shade_resample=128, shade_sigma_min=1.0)
    hit = base["id"] != 0xFFFFFFFF
    assert hit.sum() > 500
    n_rs = deep = 0
    for k in np.nonzero(hit)[0]:
        p = int(base["px"][k])
        o, d = orc.camera_ray(osc, p % sc.W, p // sc.W)
        smax = _sphere_sample_smax(np.asarray(o), np.asarray(d), base["depth"][k])
        assert abs(rs["shade_smax"][k] - smax) <= 1e-9 * max(1.0, smax)
        if abs(smax - 1.0) < 1e-6:
            continue                                   # knife edge of the threshold
        if smax < 1.0:
            n_rs += 1
            b = np.linalg.norm(np.cross(o, d))           # the ray's distance from the centre
            if b < 0.45:
                deep += 1
                assert np.allclose(rs["rgba"][k], [0.7, 0.7, 0.7, 1.0], atol=1e-8), (k, rs["rgba"][k])
        else:
            assert np.array_equal(rs["rgba"][k], base["rgba"][k])
    assert n_rs > 100 and deep >= 10, (n_rs, deep)
    assert np.array_equal(rs["rgba"][~hit], base["rgba"][~hit])
    ex = orc.render(osc, depth_mode=orc.DEPTH_EXACT, n_threads=4)
    ex_rs = orc.render(osc, depth_mode=orc.DEPTH_EXACT, n_threads=4, shade_resample=128, shade_sigma_min=1.0)
    assert np.nanmin(ex_rs["shade_smax"]) > 20.0
    assert np.array_equal(ex["rgba"], ex_rs["rgba"])


def test_parallel_light_shadow_is_an_orthographic_projection(orc):
    """A parallel light (direction w) shadows a floor point x exactly when the half-line from x
    towards the light, x - t w (t > 0), passes within the ball's radius of its centre: the ball's
    orthographic projection along w.  The ball itself is lit on the side facing the light."""
    floor = sg.make_type(sg.SDF_BOX, 0, 0, 2, 8, params=[4.0, 0.05, 4.0], rb=5.7, nedf_seed=2)
    ball = sg.make_type(sg.SDF_SPHERE, 0, 1, 2, 8, nedf_seed=3)
    w = np.array([0.35, -1.0, 0.2])
    sc = sg.Scene("plane-parallel", 48, 48, sg.f32([0, 4, 5]), sg.f32([0, 0, 0]), 40.0, sg.f32([w]), [floor, ball],
                  np.array([0, 1], np.uint32), sg.f32(np.tile(np.eye(3).reshape(1, 9), (2, 1))),
                  sg.f32([[0, -0.05, 0], [0, 0.6, 0]]), sg.f32([1, 1]), light_parallel=np.array([1]))
    osc = orc.OracleScene(sc)
    r = orc.render(osc, depth_mode=orc.DEPTH_EXACT)
    c = np.array([0, 0.6, 0])
    wn = np.asarray(sg.f32(w), np.float64)
    wn = wn / np.linalg.norm(wn)
    n_shadow = n_checked = n_ball = 0
    for k in np.nonzero(r["id"] != 0xFFFFFFFF)[0]:
        o, d = orc.camera_ray(osc, k % 48, k // 48)
        x = o + r["depth"][k] * d
        if r["id"][k] == 0:
            t = max(0.0, float((c - x) @ (-wn)))                 # closest point of the half-line
            dist = np.linalg.norm(c - (x - t * wn))
            if abs(dist - 0.5) < 1e-3:
                continue
            n_checked += 1
            expect = 0.5 if dist < 0.5 else 1.0
            n_shadow += expect == 0.5
            assert r["shadow"][k] == expect
        else:
            nrm = (x - c) / np.linalg.norm(x - c)
            cosl = float(nrm @ (-wn))
            if abs(cosl) < 0.1:
                continue
            n_ball += 1
            assert r["shadow"][k] == (1.0 if cosl > 0 else 0.5)
    assert n_checked > 500 and n_shadow > 20 and n_ball > 50, (n_checked, n_shadow, n_ball)
