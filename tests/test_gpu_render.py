"""CUDA render path vs the FP64 oracle (Steps 1-3 of Algorithm 1 / Algorithm 2), through the C ABI."""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

from .gpu_helpers import NOID, close, compare_volume, frame_vs_oracle, gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2308_04669_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def test_tiny_sphere_full_frame_nedf(orc):
    """64x64, one sphere, NeDF 4x64 (random init): every pixel, every buffer."""
    sc = sg.tiny_sphere_scene()
    g = gpu_frame(sc)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc))
    assert rep["hit"] > 1000
    assert g["stats"].status == 0


def test_tiny_sphere_full_frame_march(orc):
    """Same scene answered by the plain method (surface depths, real shading and shadows)."""
    sc = sg.tiny_sphere_scene()
    g = gpu_frame(sc, depth_source=1, march_steps=128, march_bisect=4)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4)
    assert rep["hit"] > 500 and rep["shadowed"] > 50
    assert (o["rgba"][:, 3] > 0.5).sum() > 500


@pytest.mark.parametrize("W,H", [(67, 45), (1, 1), (3, 130)])
def test_ragged_sizes(orc, W, H):
    sc = sg.three_types_scene(W, H, nerf=False)
    g = gpu_frame(sc)
    o = frame_vs_oracle(g, orc.OracleScene(sc), max_excluded=0.2 if W * H < 10 else 0.05)[1]


def test_three_types_nerf_subset(orc):
    """3 types x 16 instances, NeDF 6x128, NeRF 8x256, 2 lights at 128x128; oracle on a subset."""
    sc = sg.three_types_scene(128, 128)
    px = sg.pixel_subset(128, 128, 600, 5)
    for mode, kw in [(0, {}), (1, dict(depth_source=1))]:
        g = gpu_frame(sc, **kw)
        rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, march_n=128, march_b=4, n_threads=8,
                                 depth_mode=orc.DEPTH_MLP if mode == 0 else orc.DEPTH_MARCH)
        assert rep["hit"] > 30


def test_three_types_full_size_sampled(orc):
    """The 512x512 workload itself, sampled pixels."""
    sc = sg.three_types_scene()
    px = sg.pixel_subset(512, 512, 300, 6)
    g = gpu_frame(sc, depth_source=1)
    o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4, n_threads=8)[1]


def test_thousand_instances_sampled(orc):
    """1024 instances at 1024x1024 with 4 lights: sampled pixels against the oracle."""
    sc = sg.thousand_scene()
    px = sg.pixel_subset(1024, 1024, 200, 7)
    g = gpu_frame(sc)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), px=px, n_threads=8)
    assert g["stats"].status == 0 and g["stats"].primary_pairs > 500000


def test_refine_and_outlier_resample_fp32(orc):
    """FP32 path with the confidence fallback, window refinement and outlier re-answering."""
    sc = sg.three_types_scene(96, 96, nerf=False)
    kw = dict(fallback_conf=0.9, refine_steps=4, outlier_resample=1)
    g = gpu_frame(sc, **kw)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), march_n=128, march_b=4, n_threads=8, **kw, max_excluded=0.08)
    assert g["stats"].fallback_pairs > 0 and rep["hit"] > 500


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_miss_check_frame_matches_oracle(orc, prec):
    """NeDF misses checked by 16 density samples along the bound chord, with refinement and outlier
    re-answering: Steps 1-3 against the oracle with the same options.  The untrained networks'
    hit logits sit near zero, so the 0.9 confidence test would send nearly every pair to the plain
    method; with the confidence test off every miss is a confident one and the untrained networks
    answer many wrong misses for the check to catch."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(96, 96, nerf=False)
    kw = dict(fallback_conf=0.0, refine_steps=4, outlier_resample=1, miss_check=16)
    precision = native.PREC_FP32 if prec == "fp32" else native.PREC_BF16
    g = gpu_frame(sc, precision=precision, **kw)
    g0 = gpu_frame(sc, precision=precision, **dict(kw, miss_check=0))
    okw = dict(quant=orc.QUANT_NONE if prec == "fp32" else orc.QUANT_BF16)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), march_n=128, march_b=4, n_threads=8, max_excluded=0.1, **kw, **okw)
    assert rep["hit"] > 1000 and g["stats"].status == 0
    # the check re-answers pairs the network called confident misses: more plain-method pairs and
    # more hit pixels than without it
    assert g["stats"].fallback_pairs > g0["stats"].fallback_pairs
    assert (g["id"] != NOID).sum() > (g0["id"] != NOID).sum()


def test_light_inside_scene_bound(orc):
    """A light inside the scene's bound cannot use a shadow-map camera: every instance is tested."""
    sc = sg.three_types_scene(96, 96, nerf=False)
    sc.lights = sg.f32([[0.3, 0.2, -0.1], [1.0, 9.0, 2.0]])
    g = gpu_frame(sc, depth_source=1)
    rep, o = frame_vs_oracle(g, orc.OracleScene(sc), depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4, n_threads=8)
    assert rep["shadowed"] > 50


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_parallel_lights(orc, precision):
    """A parallel light (rays from infinity along its direction; the shadow-map grid is then
    orthographic) beside a point light: Steps 1-3 against the oracle, whose parallel-light rays start
    far beyond every object's bound."""
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(96, 96, nerf=False)
    sc.lights = sg.f32([[-0.4, -1.0, -0.3], [1.0, 9.0, 2.0]])
    sc.light_parallel = np.array([1, 0])
    if precision == "fp32":
        g = gpu_frame(sc, depth_source=1)
        rep, o = frame_vs_oracle(g, orc.OracleScene(sc), depth_mode=orc.DEPTH_MARCH, march_n=128, march_b=4, n_threads=8)
    else:
        g = gpu_frame(sc, precision=native.PREC_BF16)
        rep, o = frame_vs_oracle(g, orc.OracleScene(sc), quant=orc.QUANT_BF16, n_threads=8, max_excluded=0.1)
    assert rep["shadowed"] > 50 and g["stats"].status == 0


def test_empty_and_out_of_view(orc):
    sc = sg.tiny_sphere_scene()
    sc.inst_T = sg.f32([[0, 50, 0]])          # far outside the frustum
    g = gpu_frame(sc)
    assert np.all(g["id"] == NOID) and np.all(np.isinf(g["depth"]))
    assert np.all(g["rgba"] == 0) and np.all(g["shadow"] == 1)
    assert g["stats"].primary_pairs == 0 and g["stats"].hit_pixels == 0


def test_permutation_invariance_gpu(orc):
    sc = sg.three_types_scene(96, 96, nerf=False)
    perm = np.random.default_rng(1).permutation(sc.n_inst)
    a = gpu_frame(sc)
    b = gpu_frame(sc.permuted(perm))
    assert np.array_equal(a["depth"], b["depth"])
    hit = a["id"] != NOID
    o = orc.render(orc.OracleScene(sc))
    ok = hit & (o["gap"] > 1e-4)
    assert np.array_equal(a["id"][ok], perm[b["id"][ok]])


def test_nedf_query_isolated(orc):
    """The network alone on arbitrary local rays, including culled ones."""
    import torch
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(8, 8, nerf=False)
    r = native.renderer_for(sc)
    rng = np.random.default_rng(0)
    n = 1000
    o = rng.normal(size=(n, 3)) * 1.5
    d = rng.normal(size=(n, 3))
    o32, d32 = o.astype(np.float32), d.astype(np.float32)
    out = torch.empty(n, 4, device="cuda")
    osc = orc.OracleScene(sc)
    for t in range(3):
        r.nedf_query(t, torch.tensor(o32, device="cuda"), torch.tensor(d32, device="cuda"), out)
        g = out.cpu().numpy().astype(np.float64)
        for i in range(n):
            dd = d32[i].astype(np.float64); dd /= np.linalg.norm(dd)
            kept, f, b = orc.nedf_features(o32[i].astype(np.float64), dd, 1.0)
            if abs(b[3]) < 1e-4:
                continue
            if not kept:
                assert g[i, 3] == 0 and np.isinf(g[i, 2])
                continue
            y = orc.mlp(sc.types[t].nedf_w.astype(np.float64), sc.types[t].nedf_dims, f)
            assert close([g[i, 0], g[i, 1]], y, 1e-5, 1e-5).all(), (i, g[i], y)   # FP32 sums, FP32 sin/cos
            assert g[i, 3] == float(y[1] > 0 and b[2] - y[0] > 0) or abs(y[1]) < 1e-4
    r.close()


def test_render_host_matches_device(orc):
    import torch
    from paper_2308_04669_gb300 import native
    sc = sg.tiny_sphere_scene()
    r = native.renderer_for(sc)
    cam, li = r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights)
    n = sc.W * sc.H
    dd = torch.empty(n, device="cuda")
    r.render(cam, li, depth=dd)
    hd = np.empty(n, np.float32)
    hid = np.empty(n, np.uint32)
    r.render_host(cam, li, depth=hd, id=hid)
    assert np.array_equal(dd.cpu().numpy(), hd)
    r.close()


def test_invalid_arguments_rejected():
    from paper_2308_04669_gb300 import native
    sc = sg.tiny_sphere_scene()
    r = native.renderer_for(sc)
    with pytest.raises(native.NedfError) as e:
        r.set_instances([5], sc.inst_R, sc.inst_T, sc.inst_s)      # type out of range
    assert e.value.code == native.NEDF_ERR_ARG
    with pytest.raises(native.NedfError):
        r.set_instances([0], sc.inst_R, sc.inst_T, [0.0])            # s <= 0
    with pytest.raises(native.NedfError):
        r.set_instances([0], sc.inst_R, sc.inst_T, [float("nan")])
    with pytest.raises(native.NedfError):
        r.render(r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(np.zeros((33, 3))))
    with pytest.raises(native.NedfError):
        r.render(r.camera(sc.eye, sc.target, 0.0), r.lights(sc.lights))
    o = r.get_options()
    o.n_shade = 0
    with pytest.raises(native.NedfError):
        r.set_options(o)
    r.close()
    with pytest.raises(native.NedfError):
        native.Renderer(0, 10, 1, 1, 4, 64)
    with pytest.raises(native.NedfError) as e:
        native.Renderer(10, 10, 1, 1, 4, 96)
    assert e.value.code == native.NEDF_ERR_UNSUPPORTED


def test_pair_capacity_overflow_is_reported(orc):
    from paper_2308_04669_gb300 import native
    sc = sg.tiny_sphere_scene()
    r = native.Renderer(sc.W, sc.H, 1, 1, 4, 64, primary_pair_capacity=100)
    r.load_scene(sc)
    with pytest.raises(native.NedfError) as e:
        r.render(r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights), stats=True)
    assert e.value.code == native.NEDF_ERR_CAPACITY
    r.close()


def _march_gpu(sc, n_samples, early_stop, precision=0):
    import torch
    from paper_2308_04669_gb300 import native
    r = native.renderer_for(sc, precision=precision)
    rgba = torch.empty(sc.W * sc.H, 4, device="cuda")
    r.render_march(r.camera(sc.eye, sc.target, sc.fov_deg), n_samples, early_stop, rgba)
    torch.cuda.synchronize()
    r.sync()
    out = rgba.cpu().numpy().astype(np.float64)
    r.close()
    return out


def test_plain_method_frame_dense_matches_oracle(orc):
    """Plain method (every NeRF volume rendered front to back), albedo sphere, full frame."""
    sc = sg.tiny_sphere_scene()
    g = _march_gpu(sc, 128, 0)
    o, vm = orc.volume_render(orc.OracleScene(sc), 128, margins=True)
    compare_volume(g, o, vm)
    assert (o[:, 3] > 0.5).sum() > 500


def test_plain_method_frame_nerf_subset(orc):
    """Three types with 8x256 colour networks, overlapping bounds; subset of pixels."""
    sc = sg.three_types_scene(96, 96)
    g = _march_gpu(sc, 64, 0)
    px = sg.pixel_subset(96, 96, 400, 3)
    o, vm = orc.volume_render(orc.OracleScene(sc), 64, px=px, n_threads=8, margins=True)
    compare_volume(g[px], o, vm)
    assert (o[:, 3] > 0.5).sum() > 30


def test_plain_method_early_stop_bound(orc):
    """Early stop (T < 1e-4, weights < 1e-6 skipped) changes colour by at most ~1e-3."""
    sc = sg.three_types_scene(96, 96)
    dense = _march_gpu(sc, 128, 0)
    es = _march_gpu(sc, 128, 1)
    assert np.abs(dense - es).max() < 2e-3
