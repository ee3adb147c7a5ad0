"""E4M3 tensor-core path (first layer BF16, later hidden layers E4M3 with per-layer power-of-two
weight scales, E4M3 activations, FP32 accumulation) vs the oracle's FP8 mode.

The oracle's QUANT_FP8 mode rounds the same operands with the same scales (both sides derive the
scale from max|W| alone, exactly) and sums in FP64.  An E4M3 step is 1/8 of a binade, so an
activation lands on the other side of a rounding boundary only when the FP32 sums (or the
16-significant-bit bias of the first layer) move it across one; such a flip changes one input of
the next layer by one E4M3 step.  Rows are therefore compared with a median bound, a bound that
almost all rows meet, and a loose bound for every row.  The FP8 path's error against the
unrounded FP64 network is reported alongside.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, close, gpu_frame

pytestmark = pytest.mark.gpu


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
def test_fp8_nedf_query_matches_fp8_oracle(orc, scene_fn):
    from paper_2308_04669_gb300 import native
    sc = scene_fn()
    rng = np.random.default_rng(5)
    n = 1500                      # 5 full tiles of 256 rows and a ragged tail
    o32 = rng.normal(size=(n, 3))
    o32 = (2.5 * o32 / np.linalg.norm(o32, axis=1, keepdims=True)).astype(np.float32)
    d32 = (-o32 + rng.normal(size=(n, 3)) * 0.8).astype(np.float32)
    for t in range(len(sc.types)):
        g = run_query(sc, t, o32, d32, native.PREC_FP8)
        w = sc.types[t].nedf_w.astype(np.float64)
        errs, errs_fp, errs_q = [], [], []
        for i in range(n):
            dd = d32[i].astype(np.float64); dd /= np.linalg.norm(dd)
            kept, f, b = orc.nedf_features(o32[i].astype(np.float64), dd, float(sc.types[t].rb))
            if not kept:
                if abs(b[3]) > 1e-4:
                    assert g[i, 3] == 0 and np.isinf(g[i, 2])
                continue
            yq = orc.mlp(w, sc.types[t].nedf_dims, f, quant=orc.QUANT_FP8)
            yf = orc.mlp(w, sc.types[t].nedf_dims, f)
            assert close(g[i, :2], yq, 5e-2, 5e-2).all(), (i, g[i, :2], yq)
            errs.append(np.abs(g[i, :2] - yq).max())
            errs_fp.append(np.abs(g[i, :2] - yf).max())
            errs_q.append(np.abs(yq - yf).max())
        errs = np.array(errs)
        assert len(errs) > 600
        assert np.median(errs) < 1e-6
        assert (errs < 1e-4).mean() > 0.99
        print(f"type {t}: |fp8 gpu - fp8 oracle| median {np.median(errs):.2e} p99 {np.quantile(errs, 0.99):.2e}; "
              f"|fp8 gpu - fp64 network| median {np.median(errs_fp):.2e}; "
              f"|fp8 oracle - fp64 network| median {np.median(errs_q):.2e}")


def test_fp8_shading_matches_fp8_oracle(orc):
    """Step 2 with the NeRF's hidden layers in E4M3, surface depths from the plain method."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 500, 8)
    g = gpu_frame(sc, precision=native.PREC_FP8, depth_source=1)
    o = orc.render(orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4,
                   quant=orc.QUANT_FP8, n_threads=8)
    same = (g["id"][px] == o["id"]) & (o["id"] != NOID) & (o["pmargin"] > 1e-3) & (o["gap"] > 1e-4)
    assert same.sum() > 40
    err = np.abs(g["rgba"][px][same] - o["rgba"][same])
    assert (err.max(axis=1) < 5e-3).mean() > 0.97, np.quantile(err, 0.99)
    assert err.max() < 5e-2
    assert (o["rgba"][same][:, 3] > 0.3).mean() > 0.5


def test_fp8_frame_with_refinement_matches_fp8_oracle(orc):
    """Steps 1-3 with the E4M3 NeDF, confidence fallback, 4-step refinement and outlier
    re-answering.  Refinement puts every kept hit on the density's half level, so depths agree to
    the FP32 tolerance wherever the ids agree; ids may differ only where an E4M3 step moved the
    hit logit or confidence across its threshold."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128, nerf=False)
    px = sg.pixel_subset(128, 128, 600, 10)
    kw = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    g = gpu_frame(sc, precision=native.PREC_FP8, **kw)
    o = orc.render(orc.OracleScene(sc), px=px, quant=orc.QUANT_FP8, march_n=128, march_b=4, n_threads=8, **kw)
    gid = g["id"][px]
    decided = (o["pmargin"] > 1e-2) & ((o["gap"] > 1e-4) | (o["id"] == NOID))
    assert (gid[decided] == o["id"][decided]).mean() > 0.995
    same = decided & (gid == o["id"]) & (o["id"] != NOID)
    assert same.sum() > 100
    assert close(g["depth"][px][same], o["depth"][same]).mean() > 0.99
    assert g["stats"].fallback_pairs > 0 and g["stats"].status == 0


def test_fp8_plain_method_frame(orc):
    """The plain method's colour frame with the NeRF's hidden layers in E4M3."""
    from paper_2308_04669_gb300 import native
    from .test_gpu_render import _march_gpu
    sc = sg.three_types_scene(96, 96)
    g = _march_gpu(sc, 64, 0, precision=native.PREC_FP8)
    px = sg.pixel_subset(96, 96, 160, 3)
    o = orc.volume_render(orc.OracleScene(sc), 64, px=px, n_threads=8, quant=orc.QUANT_FP8)
    err = np.abs(g[px] - o).max(axis=1)
    assert (err < 5e-3).mean() > 0.97 and err.max() < 5e-2 and (o[:, 3] > 0.5).sum() > 10


def test_fp8_thousand_instances_frame_agrees_with_bf16(orc):
    """The 1024-instance workload on the E4M3 path: clean status, the same pair counts as BF16, and
    ids that agree with BF16 almost everywhere once both refine and re-answer outliers."""
    from paper_2308_04669_gb300 import native
    sc = sg.thousand_scene()
    kw = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    a = gpu_frame(sc, precision=native.PREC_BF16, **kw)
    b = gpu_frame(sc, precision=native.PREC_FP8, **kw)
    assert a["stats"].primary_pairs == b["stats"].primary_pairs
    assert b["stats"].status == 0
    both = (a["id"] != NOID) & (b["id"] != NOID)
    assert (a["id"][both] == b["id"][both]).mean() > 0.97
