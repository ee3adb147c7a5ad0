"""BF16 tensor-core path (tcgen05 MMAs, TMEM accumulators) vs the oracle in BF16-operand mode.

The oracle's QUANT_BF16 mode rounds every layer's inputs and weights to BF16 and accumulates in
FP64; the kernels accumulate in FP32 in TMEM.  Differences come from accumulation order and from
the rare activation that lands on the other side of a BF16 rounding boundary (one BF16 ulp,
2^-8 relative, on one of 128-256 inputs of the next layer), so the network outputs are compared
with a 1e-2 absolute + 1e-2 relative bound and a median error bound of 1e-3.  The error of the
BF16 path against the unrounded FP64 network is reported alongside.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, close, compare_frame, gpu_frame

pytestmark = pytest.mark.gpu

BF16_ABS, BF16_REL = 1e-2, 1e-2


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


@pytest.mark.parametrize("scene_fn", [sg.tiny_sphere_scene, lambda: sg.three_types_scene(8, 8, nerf=False)])
def test_bf16_nedf_query_matches_bf16_oracle(orc, scene_fn):
    from paper_2308_04669_gb300 import native
    sc = scene_fn()
    rng = np.random.default_rng(4)
    n = 1500                      # 11 full tiles of 128 rows and a ragged tail
    o32 = rng.normal(size=(n, 3))
    o32 = (2.5 * o32 / np.linalg.norm(o32, axis=1, keepdims=True)).astype(np.float32)
    d32 = (-o32 + rng.normal(size=(n, 3)) * 0.8).astype(np.float32)   # mostly towards the bound
    for t in range(len(sc.types)):
        g = run_query(sc, t, o32, d32, native.PREC_BF16)
        w = sc.types[t].nedf_w.astype(np.float64)
        errs, errs_fp = [], []
        for i in range(n):
            dd = d32[i].astype(np.float64); dd /= np.linalg.norm(dd)
            kept, f, b = orc.nedf_features(o32[i].astype(np.float64), dd, float(sc.types[t].rb))
            if not kept:
                if abs(b[3]) > 1e-4:
                    assert g[i, 3] == 0 and np.isinf(g[i, 2])
                continue
            yq = orc.mlp(w, sc.types[t].nedf_dims, f, quant=orc.QUANT_BF16)
            yf = orc.mlp(w, sc.types[t].nedf_dims, f)
            assert close(g[i, :2], yq, BF16_ABS, BF16_REL).all(), (i, g[i, :2], yq)
            errs.append(np.abs(g[i, :2] - yq).max())
            errs_fp.append(np.abs(g[i, :2] - yf).max())
        assert len(errs) > 600
        assert np.median(errs) < 1e-3
        print(f"type {t}: median |bf16 gpu - bf16 oracle| {np.median(errs):.2e}, "
              f"median |bf16 gpu - fp64 network| {np.median(errs_fp):.2e}")


def test_bf16_shading_matches_bf16_oracle(orc):
    """Step 2 on the tensor cores (NeRF 8x256 streamed layer by layer), surface depths from the
    plain method so that every shaded pixel has non-trivial opacity and colour."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 500, 8)
    g = gpu_frame(sc, precision=native.PREC_BF16, depth_source=1)
    o = orc.render(orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4,
                   quant=orc.QUANT_BF16, n_threads=8)
    same = (g["id"][px] == o["id"]) & (o["id"] != NOID) & (o["pmargin"] > 1e-3) & (o["gap"] > 1e-4)
    assert same.sum() > 40
    ok = close(g["rgba"][px][same], o["rgba"][same], 2e-3, 2e-3)
    assert ok.mean() > 0.995, np.abs(g["rgba"][px][same] - o["rgba"][same]).max()
    assert (o["rgba"][same][:, 3] > 0.3).mean() > 0.5


def test_bf16_full_frame_nedf(orc):
    """Steps 1-3 with the NeDF on the tensor cores against the BF16-operand oracle; the two agree
    to FP32-accumulation error, so the FP32 path's knife-edge margins and tolerances apply."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 500, 9)
    g = gpu_frame(sc, precision=native.PREC_BF16)
    o = orc.render(orc.OracleScene(sc), px=px, quant=orc.QUANT_BF16, n_threads=8)
    rep = compare_frame(g, o, px)
    assert rep["hit"] > 100


def test_bf16_refine_and_outlier_resample(orc):
    """Confidence fallback, window refinement and outlier re-answering on the tensor-core path
    (fallback pairs run in their own pass) against the oracle with the same options."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128, nerf=False)
    px = sg.pixel_subset(128, 128, 600, 10)
    kw = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    g = gpu_frame(sc, precision=native.PREC_BF16, **kw)
    o = orc.render(orc.OracleScene(sc), px=px, quant=orc.QUANT_BF16, march_n=128, march_b=4, n_threads=8, **kw)
    rep = compare_frame(g, o, px, max_excluded=0.08)
    assert g["stats"].fallback_pairs > 0 and rep["hit"] > 100


def test_bf16_thousand_instances_stats(orc):
    """The 1024-instance workload runs clean on the tensor-core path and agrees with FP32 on the
    pair counts (binning does not depend on precision)."""
    from paper_2308_04669_gb300 import native
    sc = sg.thousand_scene()
    a = gpu_frame(sc, precision=native.PREC_FP32)
    b = gpu_frame(sc, precision=native.PREC_BF16)
    assert a["stats"].primary_pairs == b["stats"].primary_pairs
    assert b["stats"].status == 0
    both = (a["id"] != NOID) & (b["id"] != NOID)
    assert (a["id"][both] == b["id"][both]).mean() > 0.97


def test_bf16_plain_method_frame(orc):
    """The plain method's colour frame with its NeRF on the tensor cores (sample rows of every
    (ray, instance) pair, weights T * alpha, per-pair sums) against the BF16-operand oracle."""
    from paper_2308_04669_gb300 import native
    from .test_gpu_render import _march_gpu
    sc = sg.three_types_scene(96, 96)
    g = _march_gpu(sc, 64, 0, precision=native.PREC_BF16)
    px = sg.pixel_subset(96, 96, 160, 3)
    o = orc.volume_render(orc.OracleScene(sc), 64, px=px, n_threads=8, quant=orc.QUANT_BF16)
    ok = close(g[px], o)
    assert ok.mean() > 0.995 and (o[:, 3] > 0.5).sum() > 10
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
        assert tuned["step2_shade"]["ms"] > 0 and tuned["step1_nedf"]["ms"] > 0
        assert r.get_schedule()["step3_nedf"] == tuned["step3_nedf"]["stage_bytes"]
        got = frame()
        assert all(np.array_equal(x, y) for x, y in zip(ref, got))
        with pytest.raises(native.NedfError):
            r.set_schedule([1000] * native.N_SCHEDULE)
        r.close()
