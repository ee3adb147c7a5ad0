"""Pins of the oracle's classifier intersection network (Section "Intersection network", Eq. 3-4
and 6, Appendix A) against the paper's printed numbers, closed forms, invariants and independent
library routines: its input layout, the segment operator and the argmax decode, the residual
structure, the BCE loss and its gradient, and the BF16 rounding points.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        return json.load(f)


def _layers(w):
    """The packed classifier as a list of (W, b) float64 pairs (layout of scenegen.cls_layers)."""
    out, off = [], 0
    for fi, fo in sg.cls_layers():
        out.append((w[off:off + fi * fo].reshape(fo, fi), w[off + fi * fo:off + fi * fo + fo]))
        off += fi * fo + fo
    assert off == w.size
    return out


def _pack(layers):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers]).astype(np.float64)


def test_architecture_matches_the_papers_numbers(orc):
    g = _golden()
    assert sg.CLS_IN == g["nedf_input_dim"]["value"] == g["points_per_ray"]["value"] * 3 * (1 + 2 * g["pe_levels"]["value"])
    assert (sg.CLS_W, sg.CLS_BLOCKS, sg.CLS_NC, sg.CLS_NF) == tuple(
        g[k]["value"] for k in ("feature_dim", "residual_blocks", "coarse_bins", "fine_bins"))
    # storage: NeDF + NeRF 13 MB of which 3 MB NeRF (both rounded to whole MB), so the NeDF holds
    # 10 +- 1 MB of float32 weights (a 512-wide body, or 8 or 32 blocks, would not)
    n = orc.cls_param_count()
    assert n == sg.cls_param_count()
    mb = n * 4 / 1e6
    nedf_mb = g["storage_nedf_plus_nerf_mb"]["value"] - g["storage_nerf_mb"]["value"]
    assert abs(mb - nedf_mb) <= 1.0, mb


def test_input_is_sixteen_encoded_points_on_the_chord(orc):
    rng = np.random.default_rng(4)
    for _ in range(20):
        o = rng.uniform(-3, 3, 3)
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        o = o - (o @ d + 2.5) * d                        # 2.5 before the tangency point
        feat, bd = orc.cls_features(o, d, 1.0)
        if feat is None:
            continue
        pts = feat.reshape(16, 63)[:, :3]
        # the ends are the chord's entry and exit on the bound sphere, spacing uniform along d
        assert np.allclose(np.linalg.norm(pts[[0, -1]], axis=1), 1.0, atol=1e-12)
        steps = np.diff(pts, axis=0)
        assert np.allclose(steps, steps[0], atol=1e-12)
        assert np.allclose(steps[0] / np.linalg.norm(steps[0]), d, atol=1e-12)
        assert np.linalg.norm(pts[0] - o) < np.linalg.norm(pts[-1] - o)
        # each point's block: identity, sin(2^k p) for k = 0..9, cos(2^k p), coordinate fastest
        for j in (0, 7, 15):
            blk = feat.reshape(16, 63)[j]
            k = np.arange(10)[:, None]
            assert np.allclose(blk[3:33].reshape(10, 3), np.sin(2.0 ** k * pts[j]), atol=1e-14)
            assert np.allclose(blk[33:63].reshape(10, 3), np.cos(2.0 ** k * pts[j]), atol=1e-14)


def test_segment_operator_and_argmax_decode_are_inverse(orc):
    """Decoding the one-hot bins of S(m) gives back m to within one fine bin, from below."""
    rng = np.random.default_rng(5)
    fine = 2.0 / (sg.CLS_NC * sg.CLS_NF)
    for m in np.concatenate([rng.uniform(-1, 1, 300), [-1.0, 0.0, 0.5, 1.0 - 1e-12]]):
        c, f = orc.cls_segment(m)
        logits = np.full(sg.CLS_OUT, -1.0)
        logits[0] = 0.3
        logits[1 + c] = 2.0
        logits[1 + sg.CLS_NC + f] = 2.0
        md, a, c2, f2, gap = orc.cls_decode(logits)
        assert (c2, f2) == (c, f) and a == 0.3 and gap == 3.0
        assert md <= m + 1e-15 and m - md < fine + 1e-15
    assert orc.cls_segment(-1.0) == (0, 0) and orc.cls_segment(0.0) == (32, 0)
    assert orc.cls_segment(1.0) == (63, 127) and orc.cls_segment(-1.0 + fine * 1.5) == (0, 1)
    # ties: the first maximum wins
    logits = np.zeros(sg.CLS_OUT)
    assert orc.cls_decode(logits)[2:4] == (0, 0)


def _input(rng):
    """The encoded input of a random ray through the unit bound."""
    import oracle
    d = rng.normal(size=3); d /= np.linalg.norm(d)
    feat, _ = oracle.cls_features(0.3 * rng.normal(size=3) - 2.0 * d, d, 1.0)
    return feat


def test_zero_body_reduces_to_a_two_layer_network(orc):
    """W1 = b1 = W2 = b2 = 0 makes every residual block ReLU(h): the network is then
    tail(ReLU(head(x))), checked with numpy matrix products."""
    L = _layers(sg.cls_weights(21).astype(np.float64))
    for k in range(1, 1 + 2 * sg.CLS_BLOCKS):
        L[k] = (np.zeros_like(L[k][0]), np.zeros_like(L[k][1]))
    w = _pack(L)
    x = _input(np.random.default_rng(6))
    h = np.maximum(L[0][0] @ x + L[0][1], 0.0)
    ref = np.concatenate([L[-2][0] @ h + L[-2][1], L[-1][0] @ h + L[-1][1]])
    assert np.allclose(orc.cls_forward(w, x), ref, rtol=1e-12, atol=1e-12)


def test_linear_regime_is_the_composed_affine_map(orc):
    """Non-negative weights, biases and inputs keep every ReLU inactive, so the network is one
    affine map: each block h -> (I + W2 W1) h + W2 b1 + b2.  Composed with numpy and compared."""
    rng = np.random.default_rng(7)
    L = [(rng.uniform(0, 2e-3, W.shape), rng.uniform(0, 1e-2, b.shape)) for W, b in _layers(sg.cls_weights(1))]
    w = _pack(L)
    x = rng.uniform(0, 1, sg.CLS_IN)
    A, c = L[0]
    M, v = A.copy(), c.copy()                          # h0 = M x + v
    for k in range(sg.CLS_BLOCKS):
        (W1, b1), (W2, b2) = L[1 + 2 * k], L[2 + 2 * k]
        B = np.eye(sg.CLS_W) + W2 @ W1
        M, v = B @ M, B @ v + W2 @ b1 + b2
    TA, TB = L[-2], L[-1]
    ref = np.concatenate([TA[0] @ (M @ x + v) + TA[1], TB[0] @ (M @ x + v) + TB[1]])
    assert np.allclose(orc.cls_forward(w, x), ref, rtol=1e-11, atol=0)


def test_loss_closed_forms(orc):
    """All-zero network: every logit 0, each logistic cross-entropy log 2, so L = 2.1 log 2 when
    some rays hit.  Logit +Z on the labelled bins and the hit, -Z elsewhere: every term is
    log(1 + e^-Z)."""
    n = orc.cls_param_count()
    x = np.stack([_input(np.random.default_rng(s)) for s in (8, 9)])
    L0, g0 = orc.cls_loss_grad(np.zeros(n), x, np.array([0.2, 0.0]), np.array([1, 0]))
    assert abs(L0 - 2.1 * math.log(2.0)) < 1e-12
    Z, m_star = 3.0, -0.37
    c, f = orc.cls_segment(m_star)
    w = np.zeros(n)
    lay = _layers(w)                                   # views into w
    bA, bB = lay[-2][1], lay[-1][1]
    bA[:] = -Z
    bA[0] = Z
    bA[1 + c] = Z
    bB[:] = -Z
    bB[f] = Z
    L1, _ = orc.cls_loss_grad(w, x[:1], np.array([m_star]), np.array([1]))
    assert abs(L1 - 2.1 * math.log1p(math.exp(-Z))) < 1e-12
    # the coefficient on the hit term is the paper's 0.1 (a ray without a hit has no bin terms)
    L2, _ = orc.cls_loss_grad(w, x[:1], np.array([m_star]), np.array([0]))
    assert abs(L2 - _golden()["bce_alpha_weight"]["value"] * math.log1p(math.exp(Z))) < 1e-12


def test_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(10)
    w = sg.cls_weights(31).astype(np.float64)
    x = np.stack([_input(np.random.default_rng(s)) for s in (11, 12, 13)])
    m_star, hit = np.array([0.31, -0.62, 0.0]), np.array([1, 1, 0])
    L, g = orc.cls_loss_grad(w, x, m_star, hit)
    offs = np.cumsum([0] + [fi * fo + fo for fi, fo in sg.cls_layers()])
    picks = []
    for li in (0, 1, 2, 31, 32, 33, 34):             # head, first block, last block, both tails
        fi, fo = sg.cls_layers()[li]
        picks += list(offs[li] + rng.integers(0, fi * fo, 3)) + list(offs[li] + fi * fo + rng.integers(0, fo, 2))
    h = 1e-4          # the loss sums thousands of terms: smaller steps drown in its rounding
    for i in picks:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        num = (orc.cls_loss_grad(wp, x, m_star, hit)[0] - orc.cls_loss_grad(wm, x, m_star, hit)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * abs(g[i]) + 1e-10, (i, num, g[i])


def test_bf16_mode_rounds_the_layer_inputs(orc):
    """BF16 mode against torch: weights, the network input and every layer input rounded to
    bfloat16, products and sums in float64."""
    torch = pytest.importorskip("torch")

    def q(a):
        return torch.as_tensor(a, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()

    w = sg.cls_weights(41).astype(np.float64)
    L = [(q(W), b) for W, b in _layers(w)]
    x = _input(np.random.default_rng(14))
    h = q(L[0][0] @ q(x) + L[0][1])
    for k in range(sg.CLS_BLOCKS):
        (W1, b1), (W2, b2) = L[1 + 2 * k], L[2 + 2 * k]
        t = q(np.maximum(W1 @ h + b1, 0.0))
        h = q(np.maximum(h + W2 @ t + b2, 0.0))
    ref = np.concatenate([L[-2][0] @ h + L[-2][1], L[-1][0] @ h + L[-1][1]])
    got = orc.cls_forward(w, x, orc.QUANT_BF16)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    assert np.abs(got - orc.cls_forward(w, x)).max() > 1e-4      # the rounding is really there


def test_query_uses_the_classifier(orc):
    """orc_query on a classifier type: m and the hit logit are the decode of the forward pass on
    the 16 encoded chord points; D = t_perp - l m (Eq. 2)."""
    t = sg.make_type(sg.SDF_SPHERE, 0, 0, 0, 0, nedf_seed=17, nedf_arch=sg.ARCH_CLASSIFIER)
    sc = sg.Scene("c", 33, 33, sg.f32([0, 0, 3]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]), [t],
                  np.zeros(1, np.uint32), sg.f32(np.eye(3).reshape(1, 9)), sg.f32([[0, 0, 0]]), sg.f32([1.0]))
    osc = orc.OracleScene(sc)
    out = orc.render(osc, px=np.array([16 * 33 + 16, 5 * 33 + 20], np.int64), depth_mode=orc.DEPTH_MLP)
    o = np.array([0.0, 0.0, 3.0])
    for k, p in enumerate([16 * 33 + 16, 5 * 33 + 20]):
        i, j = p % 33, p // 33
        oo, dd = np.zeros(3), np.zeros(3)
        orc.lib().orc_camera_ray(osc.ptr, i, j, orc._dp(oo), orc._dp(dd))
        feat, bd = orc.cls_features(oo, dd, 1.0)
        m, a, _, _, _ = orc.cls_decode(orc.cls_forward(t.nedf_w, feat))
        D = bd[2] - m
        hit = a > 0 and D > 0
        assert (out["id"][k] == 0) == hit
        if hit:
            assert abs(out["depth"][k] - D) < 1e-12
    assert np.allclose(oo, o)
