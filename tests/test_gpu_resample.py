"""Step-2 outlier resampling ("rs", Section "Deferred Shading") on the GPU against the oracle.

A shaded pixel whose largest density over its n_shade samples is below the threshold (1, 2 % of the
peak density: the reading of "extremely small") is re-rendered by the plain method's volume
rendering of every object on its ray.  The untrained NeDF's depths mostly miss the surface, so
without refinement most hit pixels are outliers.  Pixels whose oracle sample maximum lies within 1 %
of the threshold are knife edges (FP32 vs FP64 densities) and are not compared.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, close, decided_pixels, gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2308_04669_gb300 import build
    build.build()


def _compare(sc, g, o, px, abs_tol, rel_tol):
    """Element-wise colour of decided pixels (decided_pixels: the Step-1 margins include every
    bound's cull discriminant on the ray, the plain method's only other decisions), with the
    knife edges of the re-render test itself (sample maximum within 1 % of the threshold) counted
    and left out."""
    gid = g["id"][px]
    decided = decided_pixels(o)
    same = decided & (gid == o["id"]) & (o["id"] != NOID)
    assert not (decided & (gid != o["id"])).any()
    edge = np.abs(o["shade_smax"] - 1.0) < 0.01
    rs = same & ~edge & (o["shade_smax"] < 1.0)
    kept = same & ~edge & (o["shade_smax"] >= 1.0)
    assert rs.sum() > 50 and kept.sum() > 10, (rs.sum(), kept.sum())
    for m in (rs, kept):
        ok = close(g["rgba"][px][m], o["rgba"][m], abs_tol, rel_tol).all(axis=1)
        assert ok.all(), ((~ok).sum(), np.abs(g["rgba"][px][m] - o["rgba"][m]).max())
    # the count of re-rendered pixels: the oracle's decisions, give or take the knife edges
    n_or = int((o["shade_smax"] < 1.0).sum())
    n_edge = int((np.abs(o["shade_smax"] - 1.0) < 0.01).sum())
    print(f"re-rendered {rs.sum()}, kept {kept.sum()}, knife edges {int((same & edge).sum())}, "
          f"undecided {int((~decided).sum())} of {len(px)}")
    return n_or, n_edge, rs.sum()


def test_resampling_fp32_matches_oracle(orc):
    """FP32 path, tiny sphere (albedo colour), every pixel: deferred-shading colour where the density
    test passes, the plain method's volume-rendered colour where it does not."""
    from paper_2308_04669_gb300 import native
    sc = sg.tiny_sphere_scene()
    g = gpu_frame(sc, precision=native.PREC_FP32, shade_resample=128, shade_sigma_min=1.0)
    o = orc.render(orc.OracleScene(sc), n_threads=8, shade_resample=128, shade_sigma_min=1.0)
    px = o["px"]
    n_or, n_edge, n_cmp = _compare(sc, g, o, px, 2e-3, 1e-3)
    assert abs(int(g["stats"].resampled_pixels) - n_or) <= n_edge + 2, (g["stats"].resampled_pixels, n_or, n_edge)
    assert g["stats"].status == 0
    # off: nothing re-rendered
    g0 = gpu_frame(sc, precision=native.PREC_FP32)
    assert g0["stats"].resampled_pixels == 0


def test_resampling_bf16_nerf_matches_oracle(orc):
    """BF16 tensor-core path with the colour networks (three types): the re-rendered pixels carry the
    plain method's BF16 colour (its rows run through the tensor-core colour engine), the others the
    deferred-shading colour; both against the oracle's BF16 mode on a seeded pixel subset."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(96, 96)
    g = gpu_frame(sc, precision=native.PREC_BF16, shade_resample=64, shade_sigma_min=1.0)
    px = sg.pixel_subset(96, 96, 700, 21)
    o = orc.render(orc.OracleScene(sc), px=px, n_threads=8, quant=orc.QUANT_BF16, shade_resample=64,
                   shade_sigma_min=1.0)
    _compare(sc, g, o, px, 2e-3, 1e-3)
    assert g["stats"].resampled_pixels > 0 and g["stats"].status == 0
