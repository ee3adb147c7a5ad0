"""E4M3 tensor-core path (first layer BF16, later hidden layers E4M3 with per-layer power-of-two
weight scales, E4M3 activations, FP32 accumulation) vs the oracle's FP8 mode.

The oracle's QUANT_FP8 mode rounds the same operands with the same scales (both sides derive the
scale from max|W| alone, exactly) and sums in FP64.  A network row agrees to the FP32 summation
order, or is accepted when rounding one of the oracle's six values nearest to a rounding boundary
the other way reproduces it (an FP32 sum fell on the other side of that boundary); such rows are
counted.  An E4M3 step is 1/8 of a binade, so one flip moves a colour by up to ~2e-3: colours are
compared at 4e-3 absolute / 1e-3 relative, element by element.  The FP8 path's error against the
unrounded FP64 network is reported alongside.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, check_network_rows, compare_volume, frame_vs_oracle, gpu_frame
from .test_gpu_tc import query_features, query_rays, run_query

pytestmark = pytest.mark.gpu

# rows explained by one rounding flip: measured 0.6-1.0 % of rows (6 x 128 network)
FP8_FLIP_ROWS = 0.03
FP8_COLOUR_TOL = (4e-3, 1e-3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2308_04669_gb300 import build
    build.build()


@pytest.mark.parametrize("scene_fn", [sg.tiny_sphere_scene, lambda: sg.three_types_scene(8, 8, nerf=False)])
def test_fp8_nedf_query_matches_fp8_oracle(orc, scene_fn):
    from paper_2308_04669_gb300 import native
    sc = scene_fn()
    n = 1500                      # 5 full tiles of 256 rows and a ragged tail
    o32, d32 = query_rays(5, n)
    for t in range(len(sc.types)):
        g = run_query(sc, t, o32, d32, native.PREC_FP8)
        feats, culled = query_features(orc, o32, d32, sc.types[t].rb)
        assert np.all(g[culled, 3] == 0) and np.all(np.isinf(g[culled, 2]))
        w = sc.types[t].nedf_w.astype(np.float64)
        rep = check_network_rows(orc, g[:, :2], w, sc.types[t].nedf_dims, feats, orc.QUANT_FP8, FP8_FLIP_ROWS)
        assert rep["rows"] > 600
        errs_fp = [np.abs(g[i, :2] - orc.mlp(w, sc.types[t].nedf_dims, f)).max() for i, f in enumerate(feats)
                   if f is not None]
        print(f"type {t}: {rep}; median |fp8 gpu - fp64 network| {np.median(errs_fp):.2e}")


def test_fp8_shading_matches_fp8_oracle(orc):
    """Step 2 with the NeRF's hidden layers in E4M3, surface depths from the plain method."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 800, 8)
    g = gpu_frame(sc, precision=native.PREC_FP8, depth_source=1)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4,
                             quant=orc.QUANT_FP8, n_threads=8, colour_tol=FP8_COLOUR_TOL)
    assert rep["hit"] > 200
    hit = o["id"] != NOID
    assert (o["rgba"][hit][:, 3] > 0.3).mean() > 0.5


def test_fp8_frame_with_refinement_matches_fp8_oracle(orc):
    """Steps 1-3 with the E4M3 NeDF, confidence fallback, 4-step refinement and outlier
    re-answering, element by element; the oracle's decision margins include the change one E4M3
    rounding flip of the network could make."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128, nerf=False)
    px = sg.pixel_subset(128, 128, 600, 10)
    kw = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    g = gpu_frame(sc, precision=native.PREC_FP8, **kw)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, quant=orc.QUANT_FP8, march_n=128, march_b=4, n_threads=8, **kw, max_excluded=0.1, colour_tol=FP8_COLOUR_TOL)
    assert rep["hit"] > 100
    assert g["stats"].fallback_pairs > 0 and g["stats"].status == 0


def test_fp8_plain_method_frame(orc):
    """The plain method's colour frame with the NeRF's hidden layers in E4M3."""
    from paper_2308_04669_gb300 import native
    from .test_gpu_render import _march_gpu
    sc = sg.three_types_scene(96, 96)
    g = _march_gpu(sc, 64, 0, precision=native.PREC_FP8)
    px = sg.pixel_subset(96, 96, 400, 3)
    o, vm = orc.volume_render(orc.OracleScene(sc), 64, px=px, n_threads=8, quant=orc.QUANT_FP8, margins=True)
    compare_volume(g[px], o, vm, tol=FP8_COLOUR_TOL)
    assert (o[:, 3] > 0.5).sum() > 30
