"""Oracle parity at the configurations the bench times.

* The 1024-instance workload (sphere / torus / box, 1024 x 1024, 4 point lights) with NeDF
  networks trained on the GPU by the library's own training step, in BF16 and in E4M3, with the
  confidence fallback at 0.9, 4 refinement steps and outlier re-answering: 2,500 seeded pixels
  against the oracle in the matching rounding mode (ids bit-exact on decided pixels; depth, colour,
  shadow and composite element by element; knife edges counted).
* A smaller scene of the stress workload's kind (all 8 object types, the same instance density, 8
  lights) in FP32 with plain-method depths and in BF16 with the NeDF path.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, frame_vs_oracle

pytestmark = pytest.mark.gpu

# the bench frame's options (bench.py), on the device and in the oracle's names
FRAME_OPTS = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1, miss_check=64)
GPU_MARCH = dict(march_steps=256, march_bisect=8)
ORC_MARCH = dict(march_n=256, march_b=8)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2308_04669_gb300 import build
    build.build()


def trained_frame(sc, precision, steps, batch=16384, **opts):
    """Trains every type's NeDF on plain-method labels (2^20 rays, seed 2 + type), renders the
    frame with `opts`, and returns it with the trained FP32 weights."""
    import torch
    from paper_2308_04669_gb300 import native
    r = native.renderer_for(sc, precision=precision)
    for t in range(len(sc.types)):
        r.make_labels(t, 1 << 20, 2 + t, 256, 8)
        for _ in range(steps):
            r.train_step(t, batch, 1e-3)
    w = {t: r.get_nedf_weights(t, sc.types[t].nedf_w.shape[0]).astype(np.float64) for t in range(len(sc.types))}
    o = r.get_options()
    for k, v in opts.items():
        setattr(o, k, v)
    r.set_options(o)
    n = sc.W * sc.H
    bufs = [torch.empty(n, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n, 4, device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, 4, device="cuda")]
    st = r.render(r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights), *bufs, stats=True)
    torch.cuda.synchronize()
    r.close()
    g = dict(depth=bufs[0].cpu().numpy().astype(np.float64), id=bufs[1].cpu().numpy().view(np.uint32),
             rgba=bufs[2].cpu().numpy().astype(np.float64), shadow=bufs[3].cpu().numpy().astype(np.float64),
             out=bufs[4].cpu().numpy().astype(np.float64), stats=st)
    return g, w


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_thousand_instance_frame_matches_oracle(orc, prec):
    from paper_2308_04669_gb300 import native
    from .test_gpu_fp8 import FP8_COLOUR_TOL
    sc = sg.thousand_scene()
    precision = native.PREC_BF16 if prec == "bf16" else native.PREC_FP8
    quant = orc.QUANT_BF16 if prec == "bf16" else orc.QUANT_FP8
    g, w = trained_frame(sc, precision, 600, **FRAME_OPTS, **GPU_MARCH)
    assert g["stats"].status == 0 and g["stats"].primary_pairs > 1_500_000 and g["stats"].fallback_pairs > 0
    # E4M3: one flipped activation moves m by up to ~5e-2, as much as the depth check's half window
    # h, so the window decisions of many refined pairs are knife edges (about a third of the
    # pixels), and most shadow tests sit inside their decision margin; four times the pixels keep
    # enough of both decided
    px = sg.pixel_subset(sc.W, sc.H, 2500 if prec == "bf16" else 10000, 7)
    kw = {} if prec == "bf16" else dict(colour_tol=FP8_COLOUR_TOL)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc, nedf_override=w), px=px, quant=quant, n_threads=16,
                             max_excluded=0.1 if prec == "bf16" else 0.45, **FRAME_OPTS, **ORC_MARCH, **kw)
    # E4M3's spread leaves most shadow tests of this frame within the decision margin (their
    # pixels' shadows undetermined and not compared); BF16 must decide many more
    assert rep["hit"] > 600 and rep["pixels"] * (1 - rep["excluded"]) > 2000
    assert rep["shadowed"] > (50 if prec == "bf16" else 10), rep


def test_stress_kind_frame_fp32_plain_method_matches_oracle(orc):
    """All 8 object kinds (capsule, rounded cone, two-sphere union, twisted torus and octahedron
    besides the bench's three) at the stress workload's instance density, depths from the plain
    method: the device SDFs, 8-light shadow binning and shading against the oracle."""
    from paper_2308_04669_gb300 import native
    from .gpu_helpers import gpu_frame
    sc = sg.stress_scene(256, 256, n_inst=512)
    g = gpu_frame(sc, precision=native.PREC_FP32, depth_source=1, march_steps=128, march_bisect=4)
    px = sg.pixel_subset(sc.W, sc.H, 2000, 9)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4, n_threads=16)
    hit_types = {int(sc.inst_type[i]) for i in o["id"][o["id"] != NOID]}
    assert rep["hit"] > 200 and rep["shadowed"] > 50 and hit_types == set(range(8)), hit_types
    assert g["stats"].status == 0


def test_stress_kind_frame_bf16_nedf_matches_oracle(orc):
    from paper_2308_04669_gb300 import native
    sc = sg.stress_scene(256, 256, n_inst=512)
    g, w = trained_frame(sc, native.PREC_BF16, 300, **FRAME_OPTS, **GPU_MARCH)
    px = sg.pixel_subset(sc.W, sc.H, 2000, 10)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc, nedf_override=w), px=px, quant=orc.QUANT_BF16, n_threads=16,
                             max_excluded=0.1, **FRAME_OPTS, **ORC_MARCH)
    assert rep["hit"] > 200 and g["stats"].status == 0
