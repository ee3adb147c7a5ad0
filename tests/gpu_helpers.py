"""Helpers for the GPU tests: run the CUDA path through the C ABI and compare with the oracle.

Every comparison is element-wise.  Pixels the oracle marks as knife edges are left out and
counted:
* a discrete decision within MARGIN of its threshold (cull discriminant / rb^2, hit logit, D > 0,
  fallback confidence, depth-check window, shadow test), each already reduced by the change one
  BF16 / E4M3 rounding flip of the network could cause;
* a depth tie (gap <= GAP, the gap already reduced by both depths' flip spreads);
* two depth tests (the plain method's or the refinement's inside tests) whose points lie within
  DMARGIN, relative to the coordinate magnitude, of the surface.
A single such depth test is no exclusion: FP32 and FP64 may take different branches there, moving
the depth by part of a bracket and with it the shading window, so the oracle also renders the
pixel with that test taken the other way, and the GPU must match one of the two outcomes exactly
as it would match one.  The pixels that match the alternative are counted.
"""
import numpy as np

NOID = 0xFFFFFFFF

# FP32 tolerance of the render path against the FP64 oracle: 2e-3 absolute or 1e-3 relative.
ABS_TOL, REL_TOL = 2e-3, 1e-3
# Decision margins (see the module docstring).  DMARGIN: FP32 coordinates carry a relative error of
# about 2^-23 of their magnitude (about 1e-7: the device evaluates ol + t dl with |ol|, t up to ~100);
# 3e-7 leaves a factor of 3.
MARGIN, GAP, DMARGIN = 1e-3, 1e-4, 3e-7
# Network rows: agreement with the oracle's rounding mode where no value rounds differently (FP32
# summation order only; measured within 1e-7).
ROW_ABS, ROW_REL = 1e-6, 1e-6


def gpu_frame(scene, precision=0, nedf_weights=None, **opts):
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
    with np.errstate(invalid="ignore"):
        ok = np.where(inf, a == b, np.abs(a - b) <= np.maximum(abs_tol, rel_tol * np.abs(np.where(inf, 0, b))))
    return ok


def decided_pixels(o):
    """The oracle's pixels that are no knife edge of any kind (see the module docstring); a pixel
    with an alternative outcome is decided when its second most critical depth test is clear."""
    return (o["pmargin"] > MARGIN) & ((o["gap"] > GAP) | (o["id"] == NOID)) & (o["dmargin"] > DMARGIN)


def _matches(g, px, ref, prefix, shadow_ok, colour_tol, depth_tol, check_colour, check_shadow):
    """Per pixel: does the GPU frame match the oracle outcome ref[prefix + ...] element by element?"""
    ids, depth = ref[prefix + "id"], ref[prefix + "depth"]
    hit = ids != NOID
    gd = g["depth"][px]
    ok = g["id"][px] == ids
    ok &= np.where(hit, close(gd, np.where(hit, depth, 0.0), *depth_tol), np.isinf(gd))
    if check_colour:
        ok &= ~hit | close(g["rgba"][px], ref[prefix + "rgba"], *colour_tol).all(axis=1)
    if check_shadow:
        sh = (g["shadow"][px] == ref[prefix + "shadow"]) & close(g["out"][px], ref[prefix + "out"], *colour_tol).all(axis=1)
        ok &= ~(hit & shadow_ok) | sh
    return ok


def compare_frame(g, o, px, check_colour=True, check_shadow=True, max_excluded=0.05, colour_tol=(ABS_TOL, REL_TOL),
                  depth_tol=(ABS_TOL, REL_TOL)):
    """Compares the GPU frame g (full image) with the oracle result o on pixels px, element by
    element on every pixel that is not a counted knife edge: ids bit-exact, depth and colour within
    their tolerances, shadows exactly where the shadow tests are decided, the composite."""
    oid = o["id"]
    decided = decided_pixels(o)
    excluded = 1.0 - decided.mean()
    shadow_ok = o["smargin"] > MARGIN
    report = dict(pixels=len(px), hit=int((oid != NOID).sum()), excluded=float(excluded),
                  excluded_pmargin=int((o["pmargin"] <= MARGIN).sum()),
                  excluded_gap=int(((o["gap"] <= GAP) & (oid != NOID)).sum()),
                  excluded_dmargin=int((o["dmargin"] <= DMARGIN).sum()),
                  shadow_undecided=int((decided & (oid != NOID) & ~shadow_ok).sum()))
    assert excluded <= max_excluded, f"{excluded:.3f} of pixels at knife edges: {report}"
    args = (shadow_ok, colour_tol, depth_tol, check_colour, check_shadow)
    prim = _matches(g, px, o, "", *args)
    alt = o["has_alt"] & _matches(g, px, o, "alt_", *args) if "has_alt" in o else np.zeros_like(prim)
    bad = decided & ~prim & ~alt
    if bad.any():
        k = np.nonzero(bad)[0][:4]
        detail = [dict(px=int(px[i]), gpu=(int(g["id"][px[i]]), float(g["depth"][px[i]]), g["rgba"][px[i]].round(5).tolist(),
                                            float(g["shadow"][px[i]])),
                       orc=(int(oid[i]), float(o["depth"][i]), o["rgba"][i].round(5).tolist(), float(o["shadow"][i])),
                       has_alt=bool(o.get("has_alt", np.zeros(1, bool))[i] if "has_alt" in o else False),
                       dmargin=float(o["dmargin"][i])) for i in k]
        raise AssertionError(f"{bad.sum()} of {decided.sum()} decided pixels differ: {detail}")
    same = decided & prim & (oid != NOID)
    report["alternative_matches"] = int((decided & ~prim & alt).sum())
    report["with_alternative"] = int((decided & o["has_alt"]).sum()) if "has_alt" in o else 0
    if check_colour and same.any():
        report["colour_max_err"] = float(np.abs(g["rgba"][px][same] - o["rgba"][same]).max())
    else:
        report["colour_max_err"] = 0.0
    report["depth_max_rel_err"] = float((np.abs(g["depth"][px][same] - o["depth"][same]) / o["depth"][same]).max(initial=0))
    if check_shadow:
        report["shadowed"] = int((o["shadow"][decided & (oid != NOID) & shadow_ok] < 1).sum())
    print("compare_frame", report)
    return report


def compare_volume(g_rgba, o_rgba, vmargin, tol=(ABS_TOL, REL_TOL), max_excluded=0.05):
    """The plain method's colour frame against the oracle's volume rendering, element by element
    on every pixel whose cull and front-to-back order decisions are clear of their thresholds by
    MARGIN (the rest are counted)."""
    keep = vmargin > MARGIN
    excluded = 1.0 - keep.mean()
    assert excluded <= max_excluded, excluded
    ok = close(g_rgba[keep], o_rgba[keep], *tol).all(axis=1)
    err = np.abs(g_rgba[keep] - o_rgba[keep])
    assert ok.all(), f"{(~ok).sum()} pixels differ, max err {err.max():.2e}"
    rep = dict(pixels=len(keep), excluded=int((~keep).sum()), max_err=float(err.max(initial=0)))
    print("compare_volume", rep)
    return rep


def check_network_rows(orc, g, w, dims, feats, quant, max_flip_rows):
    """GPU network outputs g[i] = (m, a) against the oracle's rounding mode, row by row.  A row
    either agrees within ROW_ABS / ROW_REL, or a single value of it that lies near a rounding
    boundary (one of the oracle's 6 nearest), rounded the other way, makes the oracle agree with it
    within the same bound: an FP32 sum on the GPU fell on the other side of that boundary.  Rows of
    the second kind are counted and bounded by max_flip_rows (a fraction)."""
    n_tight = n_flip = 0
    flips_needed = []
    for i, f in enumerate(feats):
        if f is None:
            continue
        y, ci, cm = orc.mlp_flip(w, dims, f, quant, -1, 6)
        if close(g[i], y, ROW_ABS, ROW_REL).all():
            n_tight += 1
            continue
        explained = False
        for c in ci:
            if c < 0:
                break
            yf, _, _ = orc.mlp_flip(w, dims, f, quant, int(c), 0)
            if close(g[i], yf, ROW_ABS, ROW_REL).all():
                explained = True
                break
        assert explained, f"row {i}: gpu {g[i]} oracle {y}, not explained by one rounding flip (margins {cm})"
        n_flip += 1
        flips_needed.append(float(np.abs(g[i] - y).max()))
    rows = n_tight + n_flip
    assert rows > 0 and n_flip <= max_flip_rows * rows, (n_flip, rows)
    return dict(rows=rows, flip_rows=n_flip, flip_err_max=max(flips_needed, default=0.0))
