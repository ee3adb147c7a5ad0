"""Helpers for the GPU tests: run the CUDA path through the C ABI and compare with the oracle."""
import numpy as np

NOID = 0xFFFFFFFF

# FP32 tolerance of the render path against the FP64 oracle: 2e-3 absolute or 1e-3 relative.
ABS_TOL, REL_TOL = 2e-3, 1e-3
# Decisions closer than this to their threshold in the oracle are not compared (cull
# discriminant / rb^2, hit logit, D > 0, fallback confidence, shadow tests); depth ties within
# GAP leave more than one correct id.
MARGIN, GAP = 1e-3, 1e-4


def gpu_frame(scene, precision=0, **opts):
    import torch
    from paper_2308_04669_gb300 import native
    r = native.renderer_for(scene, precision=precision)
    if opts:
        o = r.get_options()
        for k, v in opts.items():
            setattr(o, k, v)
        r.set_options(o)
    n = scene.W * scene.H
    dev = "cuda"
    depth = torch.empty(n, dtype=torch.float32, device=dev)
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    rgba = torch.empty(n, 4, dtype=torch.float32, device=dev)
    shadow = torch.empty(n, dtype=torch.float32, device=dev)
    out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    st = r.render(r.camera(scene.eye, scene.target, scene.fov_deg), r.lights(scene.lights, scene.light_parallel), depth, ids, rgba,
                  shadow, out, stats=True)
    torch.cuda.synchronize()
    res = dict(depth=depth.cpu().numpy().astype(np.float64), id=ids.cpu().numpy().view(np.uint32),
               rgba=rgba.cpu().numpy().astype(np.float64), shadow=shadow.cpu().numpy().astype(np.float64),
               out=out.cpu().numpy().astype(np.float64), stats=st)
    r.close()
    return res


def close(a, b, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    """Element-wise |a - b| <= max(abs_tol, rel_tol |b|); infinities must match exactly."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    inf = np.isinf(b)
    ok = np.where(inf, a == b, np.abs(a - b) <= np.maximum(abs_tol, rel_tol * np.abs(np.where(inf, 0, b))))
    return ok


def compare_frame(g, o, px, check_colour=True, check_shadow=True, max_excluded=0.05):
    """Compares the GPU frame g (full image) with the oracle result o on pixels px."""
    gid = g["id"][px]
    oid = o["id"]
    decided = (o["pmargin"] > MARGIN) & ((o["gap"] > GAP) | (oid == NOID))
    excluded = 1.0 - decided.mean()
    assert excluded <= max_excluded, f"{excluded:.3f} of pixels at knife edges"
    bad = decided & (gid != oid)
    assert not bad.any(), f"{bad.sum()} id mismatches, e.g. px {px[bad][:5]} gpu {gid[bad][:5]} orc {oid[bad][:5]}"
    same = decided & (gid == oid)
    ok = close(g["depth"][px][same], o["depth"][same])
    assert ok.all(), f"depth mismatch: {np.nonzero(~ok)[0][:5]}"
    report = dict(pixels=len(px), hit=int((oid != NOID).sum()), excluded=float(excluded))
    if check_colour:
        okc = close(g["rgba"][px][same], o["rgba"][same])
        assert okc.mean() >= 0.999, f"colour mismatch {1 - okc.mean():.4f}"
        report["colour_max_err"] = float(np.abs(g["rgba"][px][same] - o["rgba"][same]).max(initial=0))
    if check_shadow:
        sd = same & (o["smargin"] > MARGIN)
        assert np.array_equal(g["shadow"][px][sd], o["shadow"][sd]), "shadow mismatch"
        oko = close(g["out"][px][sd], o["out"][sd])
        assert oko.mean() >= 0.999
        report["shadowed"] = int((o["shadow"][sd] < 1).sum())
    return report
