"""Learned part on the GPU vs the FP64 oracle: training set, loss and gradient, Adam, state."""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2308_04669_gb300 import build
    build.build()
    import torch
    from paper_2308_04669_gb300 import native
    assert torch.cuda.is_available()
    return native


def labels_on_gpu(native, sc, t, n, seed):
    import torch
    r = native.renderer_for(sc)
    o = torch.empty(n, 3, device="cuda"); d = torch.empty(n, 3, device="cuda")
    m = torch.empty(n, device="cuda"); h = torch.empty(n, device="cuda")
    r.make_labels(t, n, seed, 256, 8, o, d, m, h)
    torch.cuda.synchronize()
    return r, o, d, m, h


def test_training_rays_and_labels(lib, orc):
    """The training rays are the oracle's (same counter draws); their plain-method labels match the
    oracle's element by element (hit bit-exact, m* within 1e-4) except on rays with a march test
    at a knife edge (DMARGIN, relative to the coordinates; for m* only tests whose consequence
    reaches 1e-4 r_b count), which are counted."""
    from .gpu_helpers import DMARGIN
    sc = sg.three_types_scene(8, 8, nerf=False)
    n = 4000
    for t in range(3):
        r, o, d, m, h = labels_on_gpu(lib, sc, t, n, 2)
        go, gd = o.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)
        oo, od = orc.train_rays(1.0, 2, 0, n)
        assert np.abs(go - oo).max() < 1e-5 and np.abs(gd - od).max() < 1e-5   # same counter draws
        # the type alone at the origin: world rays are its local rays
        one = sg.Scene("one", 8, 8, sg.f32([0, 0, 3]), sg.f32([0, 0, 0]), 40.0, sg.f32([[2, 3, 2]]), [sc.types[t]],
                       np.zeros(1, np.uint32), sg.f32(np.eye(3).reshape(1, 9)), sg.f32([[0, 0, 0]]), sg.f32([1.0]))
        osc = orc.OracleScene(one)
        om, oh = orc.train_labels(orc.OracleScene(sc), t, go, gd, 256, 8)
        knife_hit = np.zeros(n, bool)
        knife_m = np.zeros(n, bool)
        for i in range(n):
            hit_q, q, dg = orc.query_diag(osc, 0, go[i], gd[i], need=np.inf, depth_mode=orc.DEPTH_MARCH,
                                          march_n=256, march_b=8)
            assert hit_q == (oh[i] == 1)
            knife_hit[i] = dg[1] <= DMARGIN or abs(q[3] - q[4]) < 1e-6   # grazing the bound
            knife_m[i] = knife_hit[i] or orc.query_diag(osc, 0, go[i], gd[i], need=1e-4, depth_mode=orc.DEPTH_MARCH,
                                                        march_n=256, march_b=8)[2][1] <= DMARGIN
        gh = h.cpu().numpy() > 0.5
        assert np.array_equal(gh[~knife_hit], oh[~knife_hit] == 1)
        both = gh & (oh == 1) & ~knife_m
        assert close(m.cpu().numpy()[both], om[both], 1e-4, 1e-4).all()
        assert 0.05 < gh.mean() < 0.95 and knife_m.mean() < 0.05
        print(f"type {t}: knife edges {knife_hit.sum()} (hit) / {knife_m.sum()} (m*) of {n}")
        r.close()


def test_loss_and_gradient_match_oracle(lib, orc):
    import torch
    sc = sg.three_types_scene(8, 8, nerf=False)
    osc = orc.OracleScene(sc)
    n = 300
    r, o, d, m, h = labels_on_gpu(lib, sc, 1, n, 9)
    g = torch.zeros(sc.types[1].nedf_w.shape[0], device="cuda")
    loss = r.loss_grad(1, o, d, m, h, g)
    ol, og = orc.nedf_loss_grad(osc, 1, o.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64),
                                m.cpu().numpy().astype(np.float64), (h.cpu().numpy() > 0.5).astype(np.int32))
    assert abs(loss - ol) <= 1e-4 * abs(ol)
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.abs(og).max()
    assert np.all(np.abs(gg - og) <= 1e-4 * scale + 1e-3 * np.abs(og))
    r.close()


@pytest.mark.parametrize("scene_fn,t,n", [(lambda: sg.three_types_scene(8, 8, nerf=False), 1, 300),
                                           (lambda: sg.three_types_scene(8, 8, nerf=False), 2, 3000),
                                           (sg.tiny_sphere_scene, 0, 777)])
def test_bf16_loss_and_gradient_match_oracle(lib, orc, scene_fn, t, n):
    """The tensor-core training path (BF16 operands, FP32 accumulation; BF16 handles) against the
    oracle's BF16-training gradient (reading 29).  The loss agrees to 1e-5 relative.  The gradient
    of each layer agrees in norm to half the layer's own BF16 rounding effect (the gap between the
    oracle's BF16 and FP64 gradients) and to 5e-4 of the largest element: the remaining differences
    are values an FP32 sum rounds to the other BF16 neighbour (a missing term or mask, a transposed
    operand, would be tens of per cent of the layer).  Widths 128 and 64;
    ragged row counts (300: two 128-row tiles and a tail; 3000: three batch splits of 1024)."""
    import torch
    sc = scene_fn()
    osc = orc.OracleScene(sc)
    r0, o, d, m, h = labels_on_gpu(lib, sc, t, n, 9)
    r0.close()
    r = lib.renderer_for(sc, precision=lib.PREC_BF16)
    g = torch.zeros(sc.types[t].nedf_w.shape[0], device="cuda")
    loss = r.loss_grad(t, o, d, m, h, g)
    args = (o.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64),
            m.cpu().numpy().astype(np.float64), (h.cpu().numpy() > 0.5).astype(np.int32))
    ol, og = orc.nedf_loss_grad(osc, t, *args, quant=orc.QUANT_BF16)
    _, og64 = orc.nedf_loss_grad(osc, t, *args)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss - ol) <= 1e-5 * abs(ol)
    scale = np.abs(og).max()
    dims = sc.types[t].nedf_dims
    off, bad = 0, []
    for l in range(len(dims) - 1):
        k = dims[l] * dims[l + 1] + dims[l + 1]
        e = np.linalg.norm(gg[off:off + k] - og[off:off + k])
        gap = np.linalg.norm(og[off:off + k] - og64[off:off + k])
        e64 = np.linalg.norm(gg[off:off + k] - og64[off:off + k])
        print(f"layer {l}: |g - g_bf16| {e:.3e}  |g_bf16 - g_fp64| {gap:.3e}  |g - g_fp64| {e64:.3e}  "
              f"|g_bf16| {np.linalg.norm(og[off:off + k]):.3e}")
        if not e <= 0.5 * gap + 5e-4 * scale:
            bad.append((l, e, gap))
        off += k
    assert not bad, bad
    print(f"loss gpu {loss:.6f} oracle {ol:.6f}; max |g - g_bf16| / max |g_bf16| = {np.abs(gg - og).max() / scale:.2e}")
    r.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_training_reduces_loss_and_state_round_trip(lib, prec):
    sc = sg.three_types_scene(8, 8, nerf=False)
    r = lib.renderer_for(sc, precision=lib.PREC_FP32 if prec == "fp32" else lib.PREC_BF16)
    r.make_labels(0, 1 << 16, 2)
    first = r.train_step(0, 4096, 1e-3, want_loss=True)
    for _ in range(150):
        r.train_step(0, 4096, 1e-3)
    last = r.train_step(0, 4096, 1e-3, want_loss=True)
    assert last < 0.5 * first, (first, last)
    blob = r.save_state()
    w0 = r.get_nedf_weights(0, sc.types[0].nedf_w.shape[0])
    for _ in range(5):
        r.train_step(0, 4096, 1e-3)
    assert not np.array_equal(w0, r.get_nedf_weights(0, w0.shape[0]))
    r.load_state(blob)
    assert np.array_equal(w0, r.get_nedf_weights(0, w0.shape[0]))
    r.close()


def _depth_frame(r, sc, **opts):
    import torch
    o = r.get_options()
    for k, v in opts.items():
        setattr(o, k, v)
    r.set_options(o)
    n = sc.W * sc.H
    depth = torch.empty(n, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    st = r.render(r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights), depth, ids, None, None, None,
                  stats=True)
    torch.cuda.synchronize()
    return depth.cpu().numpy().astype(np.float64), ids.cpu().numpy(), st


def _against_judge(frame, judge):
    """Hit agreement, id agreement and depth error (in bound radii; every instance has s r_b = 1)."""
    d, i, _ = frame
    jd, ji, _ = judge
    hit, jhit = i != -1, ji != -1
    same = hit & jhit & (i == ji)
    err = np.abs(d - jd)[same]
    return dict(hit_agree=float((hit == jhit).mean()), id_agree=float((i == ji).mean()),
                mean_err=float(err.mean()), median_err=float(np.median(err)), p99_err=float(np.quantile(err, 0.99)))


def test_training_gain_over_untrained_network(lib):
    """What the learned part buys: the bare NeDF against a fine ray-march judge, before and after
    training each type on ray-march labels, and how many queries the confidence test hands to the
    plain method (sections "Neural Depth Fields (NeDF)" and "Fast NeRF Composition with NeDF")."""
    sc = sg.three_types_scene(256, 256, nerf=False)
    r = lib.renderer_for(sc)
    judge = _depth_frame(r, sc, depth_source=1, march_steps=1024, march_bisect=24, fallback_conf=0.0,
                         refine_steps=0, outlier_resample=0)
    bare = dict(depth_source=0, fallback_conf=0.0, refine_steps=0, outlier_resample=0)
    full = dict(depth_source=0, fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    before = _against_judge(_depth_frame(r, sc, **bare), judge)
    fb_before = _depth_frame(r, sc, **full)[2].fallback_pairs
    for t in range(len(sc.types)):
        r.make_labels(t, 1 << 18, 2 + t, 256, 8)
        for _ in range(600):
            r.train_step(t, 8192, 1e-3)
    after = _against_judge(_depth_frame(r, sc, **bare), judge)
    fr = _depth_frame(r, sc, **full)
    with_checks = _against_judge(fr, judge)
    fb_after = fr[2].fallback_pairs
    primary = fr[2].primary_pairs
    print(f"\nbefore {before}\nafter {after}\nwith fallback+refine {with_checks}\n"
          f"fallback pairs {fb_before} -> {fb_after} of {primary}")
    assert after["hit_agree"] > 0.97 and after["hit_agree"] > before["hit_agree"] + 0.1
    assert after["median_err"] < 0.2 * before["median_err"]
    assert after["median_err"] < 0.05
    assert fb_after < 0.5 * fb_before
    assert with_checks["id_agree"] > 0.99 and with_checks["median_err"] < 0.01
    r.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_resumed_training_repeats_the_uninterrupted_run_bitwise(lib, prec):
    """Training steps are deterministic, and the saved state holds everything a step depends on
    (weights, Adam moments, step count, batch cursor): save after 20 steps, run 15 more, reload and
    run the same 15 again; both runs end with identical weights, bit for bit."""
    sc = sg.three_types_scene(8, 8, nerf=False)
    r = lib.renderer_for(sc, precision=lib.PREC_FP32 if prec == "fp32" else lib.PREC_BF16)
    r.make_labels(1, 1 << 15, 3)
    for _ in range(20):
        r.train_step(1, 3000, 1e-3)           # 3000 rows: two gradient splits, one ragged
    blob = r.save_state()
    for _ in range(15):
        r.train_step(1, 3000, 1e-3)
    w_a = r.get_nedf_weights(1, sc.types[1].nedf_w.shape[0])
    r.load_state(blob)
    for _ in range(15):
        r.train_step(1, 3000, 1e-3)
    w_b = r.get_nedf_weights(1, sc.types[1].nedf_w.shape[0])
    assert np.array_equal(w_a, w_b)
    r.close()
