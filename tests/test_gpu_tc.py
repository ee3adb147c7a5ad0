"""BF16 tensor-core path (tcgen05 MMAs, TMEM accumulators) vs the oracle in BF16-operand mode.

The oracle's QUANT_BF16 mode rounds every layer's inputs and weights to BF16 and accumulates in
FP64; the kernels accumulate in FP32 in TMEM.  Network rows agree to the FP32 summation order
(within 1e-7, bounded at 1e-6) unless an FP32 sum lands on the other side of a BF16 rounding
boundary than the FP64 sum; such a row is accepted only when rounding one of the oracle's six
values nearest to a boundary the other way reproduces it within the same bound, and those rows are
counted.  Frames then compare element by element at the FP32 tolerance, the oracle's knife edges
(flip spreads included) counted and left out.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, check_network_rows, compare_volume, frame_vs_oracle, gpu_frame

pytestmark = pytest.mark.gpu

# rows explained by one rounding flip: measured 2.2-2.7 % of rows (6 x 128 network)
BF16_FLIP_ROWS = 0.05


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2308_04669_gb300 import build
    build.build()


def run_query(sc, t, o32, d32, precision):
    import torch
    from paper_2308_04669_gb300 import native
    r = native.renderer_for(sc, precision=precision)
    out = torch.empty(o32.shape[0], 4, device="cuda")
    r.nedf_query(t, torch.tensor(o32, device="cuda"), torch.tensor(d32, device="cuda"), out)
    torch.cuda.synchronize()
    r.close()
    return out.cpu().numpy().astype(np.float64)


def query_rays(seed, n):
    rng = np.random.default_rng(seed)
    o32 = rng.normal(size=(n, 3))
    o32 = (2.5 * o32 / np.linalg.norm(o32, axis=1, keepdims=True)).astype(np.float32)
    d32 = (-o32 + rng.normal(size=(n, 3)) * 0.8).astype(np.float32)   # mostly towards the bound
    return o32, d32


def query_features(orc, o32, d32, rb):
    """The oracle's encoded inputs of each ray (None where the bound culls it), and the culled rows
    that are no knife edge of the cull."""
    feats, culled = [], []
    for i in range(o32.shape[0]):
        dd = d32[i].astype(np.float64); dd /= np.linalg.norm(dd)
        kept, f, b = orc.nedf_features(o32[i].astype(np.float64), dd, float(rb))
        feats.append(f if kept else None)
        if not kept and abs(b[3]) > 1e-4:
            culled.append(i)
    return feats, np.array(culled, np.int64)


@pytest.mark.parametrize("scene_fn", [sg.tiny_sphere_scene, lambda: sg.three_types_scene(8, 8, nerf=False)])
def test_bf16_nedf_query_matches_bf16_oracle(orc, scene_fn):
    from paper_2308_04669_gb300 import native
    sc = scene_fn()
    n = 1500                      # 5 full tiles of 256 rows and a ragged tail
    o32, d32 = query_rays(4, n)
    for t in range(len(sc.types)):
        g = run_query(sc, t, o32, d32, native.PREC_BF16)
        feats, culled = query_features(orc, o32, d32, sc.types[t].rb)
        assert np.all(g[culled, 3] == 0) and np.all(np.isinf(g[culled, 2]))
        w = sc.types[t].nedf_w.astype(np.float64)
        rep = check_network_rows(orc, g[:, :2], w, sc.types[t].nedf_dims, feats, orc.QUANT_BF16, BF16_FLIP_ROWS)
        assert rep["rows"] > 600
        errs_fp = [np.abs(g[i, :2] - orc.mlp(w, sc.types[t].nedf_dims, f)).max() for i, f in enumerate(feats)
                   if f is not None]
        print(f"type {t}: {rep}; median |bf16 gpu - fp64 network| {np.median(errs_fp):.2e}")


def test_bf16_shading_matches_bf16_oracle(orc):
    """Step 2 on the tensor cores (NeRF 8x256 streamed layer by layer), surface depths from the
    plain method so that every shaded pixel has non-trivial opacity and colour: element-wise at the
    FP32 tolerance (a BF16 rounding flip in the colour network moves a colour by ~1e-4)."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 800, 8)
    g = gpu_frame(sc, precision=native.PREC_BF16, depth_source=1)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4,
                             quant=orc.QUANT_BF16, n_threads=8)
    assert rep["hit"] > 200 and rep["colour_max_err"] < 5e-4
    hit = o["id"] != NOID
    assert (o["rgba"][hit][:, 3] > 0.3).mean() > 0.5


def test_bf16_full_frame_nedf(orc):
    """Steps 1-3 with the NeDF on the tensor cores against the BF16-operand oracle; the two agree
    to FP32-accumulation error, so the FP32 path's knife-edge margins and tolerances apply."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 500, 9)
    g = gpu_frame(sc, precision=native.PREC_BF16)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, quant=orc.QUANT_BF16, n_threads=8)
    assert rep["hit"] > 100


def test_bf16_refine_and_outlier_resample(orc):
    """Confidence fallback, window refinement and outlier re-answering on the tensor-core path
    (fallback pairs run in their own pass) against the oracle with the same options."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128, nerf=False)
    px = sg.pixel_subset(128, 128, 600, 10)
    kw = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    g = gpu_frame(sc, precision=native.PREC_BF16, **kw)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, quant=orc.QUANT_BF16, march_n=128, march_b=4, n_threads=8, **kw, max_excluded=0.08)
    assert g["stats"].fallback_pairs > 0 and rep["hit"] > 100


def test_bf16_plain_method_frame(orc):
    """The plain method's colour frame with its NeRF on the tensor cores (sample rows of every
    (ray, instance) pair, weights T * alpha, per-pair sums) against the BF16-operand oracle."""
    from paper_2308_04669_gb300 import native
    from .test_gpu_render import _march_gpu
    sc = sg.three_types_scene(96, 96)
    g = _march_gpu(sc, 64, 0, precision=native.PREC_BF16)
    px = sg.pixel_subset(96, 96, 400, 3)
    o, vm = orc.volume_render(orc.OracleScene(sc), 64, px=px, n_threads=8, quant=orc.QUANT_BF16, margins=True)
    compare_volume(g[px], o, vm)
    assert (o[:, 3] > 0.5).sum() > 30
    es = _march_gpu(sc, 64, 1, precision=native.PREC_BF16)
    assert np.abs(es - g).max() < 2e-3


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_every_stage_size_on_a_large_frame(prec):
    """The weight ring's handshake at every stage size the autotuner tries (and the smallest and
    largest the API accepts) on the 1024-instance scene, where each CTA walks many tiles of both
    slots and every type: a clean status word (no bounded wait ran out) and bitwise the same
    depth, id and colour buffers as the default schedule."""
    import torch
    from paper_2308_04669_gb300 import native
    sc = sg.thousand_scene(512, 512)
    r = native.renderer_for(sc, precision=native.PREC_BF16 if prec == "bf16" else native.PREC_FP8)
    o = r.get_options()
    o.fallback_conf, o.refine_steps, o.outlier_resample = 0.9, 4, 1
    r.set_options(o)
    cam, li = r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights)
    n = sc.W * sc.H

    def frame():
        d = torch.empty(n, device="cuda"); i = torch.empty(n, dtype=torch.int32, device="cuda")
        c = torch.empty(n, 4, device="cuda")
        st = r.render(cam, li, d, i, c, None, None, stats=True)
        torch.cuda.synchronize()
        assert st.status == 0 and st.primary_pairs > 100000 and st.shadow_pairs > 100000
        return d.cpu().numpy(), i.cpu().numpy(), c.cpu().numpy()

    ref = frame()
    for b in (1024, 4096, 8192, 12288, 16384, 20480, 24576, 28672, 32768, 36864, 40960, 49152, 65536, 131072):
        r.set_schedule([b] * native.N_SCHEDULE)
        for _ in range(2):
            got = frame()
            assert all(np.array_equal(x, y) for x, y in zip(ref, got)), b
    # the NeDF engines' operand order (BF16 width 128: swapped or unswapped; ignored in E4M3)
    for order in (1, 2):
        for b in (8192, 36864):
            r.set_schedule([b] * native.N_SCHEDULE, [0, 0, order, order, order])
            got = frame()
            assert all(np.array_equal(x, y) for x, y in zip(ref, got)), (order, b)
    r.close()


def test_schedule_changes_timing_not_results():
    """The stage size of the weight stream (set by hand or by the autotuner) never changes a
    frame: every schedule gives bitwise the same depth, id and colour buffers."""
    import torch
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    for prec in (native.PREC_BF16, native.PREC_FP8):
        r = native.renderer_for(sc, precision=prec)
        o = r.get_options()
        o.fallback_conf, o.refine_steps, o.outlier_resample = 0.9, 4, 1
        r.set_options(o)
        cam, li = r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights)
        n = sc.W * sc.H

        def frame():
            d = torch.empty(n, device="cuda"); i = torch.empty(n, dtype=torch.int32, device="cuda")
            c = torch.empty(n, 4, device="cuda")
            r.render(cam, li, d, i, c, None, None)
            torch.cuda.synchronize()
            return d.cpu().numpy(), i.cpu().numpy(), c.cpu().numpy()

        ref = frame()
        for b in (8192, 32768, 65536, 1024):
            r.set_schedule([b] * native.N_SCHEDULE)
            got = frame()
            assert all(np.array_equal(x, y) for x, y in zip(ref, got)), b
        tuned = r.autotune(cam, li, reps=1)
        assert all(v["stage_bytes"] in (8192, 12288, 16384, 24576, 32768, 36864, 49152, 65536) for v in tuned.values())
        want = ("swapped", "unswapped") if prec == native.PREC_BF16 else ("fixed",)
        assert tuned["step1_nedf"]["operand_order"] in want and tuned["step3_nedf"]["operand_order"] in want
        assert tuned["step2_shade"]["ms"] > 0 and tuned["step1_nedf"]["ms"] > 0
        assert r.get_schedule()["step3_nedf"] == tuned["step3_nedf"]["stage_bytes"]
        got = frame()
        assert all(np.array_equal(x, y) for x, y in zip(ref, got))
        with pytest.raises(native.NedfError):
            r.set_schedule([1000] * native.N_SCHEDULE)
        r.close()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_sm_pair_engine_matches_one_sm_engine(prec):
    """The NeRF at width 256 runs on SM pairs (tcgen05 MMAs of cta_group::2, M = 256 across two
    SMs) with operand order 1 of the shading and plain-method kernels, on one SM by default (0)
    and with order 2.  On the 1024-instance scene (every SM pair walks many tiles of both slots and every
    type) at every stage size: depth and id bitwise equal, colours element-wise within 2e-6 (the
    two engines fold the last layer's two column halves in a different FP32 order), the
    plain-method colour frame likewise, and clean status words."""
    import torch
    from paper_2308_04669_gb300 import native
    sc = sg.thousand_scene(512, 512)
    r = native.renderer_for(sc, precision=native.PREC_BF16 if prec == "bf16" else native.PREC_FP8)
    cam, li = r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights)
    n = sc.W * sc.H

    def frame():
        d = torch.empty(n, device="cuda"); i = torch.empty(n, dtype=torch.int32, device="cuda")
        c = torch.empty(n, 4, device="cuda")
        st = r.render(cam, li, d, i, c, None, None, stats=True)
        torch.cuda.synchronize()
        assert st.status == 0 and st.hit_pixels > 10000
        return d.cpu().numpy(), i.cpu().numpy(), c.cpu().numpy().astype(np.float64)

    def march():
        c = torch.empty(n, 4, device="cuda")
        r.render_march(cam, 64, 0, c)
        torch.cuda.synchronize()
        return c.cpu().numpy().astype(np.float64)

    r.set_schedule([0] * native.N_SCHEDULE, [2, 2, 0, 0, 0])
    one_sm, one_sm_march = frame(), march()
    for b in (4096, 8192, 12288, 24576, 36864, 65536):
        r.set_schedule([b] * native.N_SCHEDULE, [1, 1, 0, 0, 0])
        got = frame()
        assert np.array_equal(got[0], one_sm[0]) and np.array_equal(got[1], one_sm[1]), b
        err = np.abs(got[2] - one_sm[2]).max()
        print(f"{prec} stage {b}: max |pair - one SM| colour {err:.2e}")
        assert err <= 2e-6, (b, err)
    got_march = march()
    err = np.abs(got_march - one_sm_march).max()
    print(f"{prec} plain-method colour: max |pair - one SM| {err:.2e}")
    assert (one_sm_march[:, 3] > 0.1).sum() > 10000 and err <= 2e-6
    r.close()
