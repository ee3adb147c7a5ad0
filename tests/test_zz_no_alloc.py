"""The allocation-free Step-1 entry point against the handle-based renderer and the oracle.

nedf_compose_depth_noalloc serves callers that cannot allocate device memory (a host that owns
all device memory through its own pool, a real-time loop that must not allocate): every buffer is
the caller's, and the library's only scratch is a fixed array inside it.  This file is collected
last so that, if it fails, a run stopped at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


def instance_records(scene) -> np.ndarray:
    rec = np.zeros(scene.n_inst, dtype=np.dtype([("type", "<u4"), ("R", "<f4", 9), ("T", "<f4", 3), ("s", "<f4")]))
    rec["type"], rec["R"], rec["T"], rec["s"] = scene.inst_type, scene.inst_R, scene.inst_T, scene.inst_s
    assert rec.dtype.itemsize == 56
    return rec


def _noalloc(native, sc, inst, w, cam):
    import torch
    n = sc.W * sc.H
    rb = (C.c_float * len(sc.types))(*[t.rb for t in sc.types])
    t0 = sc.types[0]
    depth = torch.full((n,), float("nan"), device="cuda")
    ids = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    rc = native._lib.nedf_compose_depth_noalloc(sc.W, sc.H, C.byref(cam), inst.shape[0] // 56, inst.data_ptr(),
                                                 len(sc.types), rb, t0.nedf_hidden, t0.nedf_width,
                                                 w.data_ptr(), depth.data_ptr(), ids.data_ptr(), None)
    assert rc == native.NEDF_OK, native._lib.nedf_compose_last_error(None)
    torch.cuda.synchronize()
    return depth.cpu().numpy(), ids.cpu().numpy().view(np.uint32)


def test_depth_noalloc_matches_render_and_oracle_on_two_calls(orc):
    import torch
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native

    from .gpu_helpers import GAP, MARGIN, NOID, close

    sc = sg.three_types_scene(160, 120, nerf=False)
    n = sc.W * sc.H
    cam = native.Renderer.camera(sc.eye, sc.target, sc.fov_deg)
    # the existing entry point (handle, default options: no fallback, no refinement)
    r = native.renderer_for(sc)
    d_ref = torch.empty(n, device="cuda")
    i_ref = torch.empty(n, dtype=torch.int32, device="cuda")
    r.render(cam, r.lights(sc.lights), d_ref, i_ref)
    torch.cuda.synchronize()
    r.close()
    d_ref, i_ref = d_ref.cpu().numpy(), i_ref.cpu().numpy().view(np.uint32)
    assert (i_ref != NOID).sum() > 1000

    # the FP64 oracle's Step 1 on a seeded pixel sample (ids and depths; its shading is not used)
    px = sg.pixel_subset(sc.W, sc.H, 1500, 11)
    o = orc.render(orc.OracleScene(sc), px=px, n_threads=8)
    decided = (o["pmargin"] > MARGIN) & ((o["gap"] > GAP) | (o["id"] == NOID))
    assert decided.mean() > 0.95 and (o["id"][decided] != NOID).sum() > 100
    # sampled pixels at the oracle's knife edges (hit logit near 0, or a depth tie)
    tied = np.zeros(n, bool)
    tied[px[~decided]] = True

    # caller-owned inputs and outputs
    inst = torch.from_numpy(instance_records(sc).view(np.uint8).copy()).cuda()
    w = torch.from_numpy(np.concatenate([t.nedf_w for t in sc.types]).astype(np.float32)).cuda()
    for call in range(2):
        d, i = _noalloc(native, sc, inst, w, cam)
        # against the oracle: ids bit-exact on decided pixels, depth element-wise
        assert np.array_equal(i[px][decided], o["id"][decided]), f"call {call}: id differs from the oracle"
        hit = decided & (o["id"] != NOID)
        assert close(d[px][hit], o["depth"][hit]).all(), f"call {call}: depth differs from the oracle"
        # against the existing entry point, every pixel: where the ids differ, either both hit at
        # the same depth within the tolerance (a tie the two summation orders break differently)
        # or the pixel is one of the oracle's knife edges; depths agree wherever the ids do
        diff = i != i_ref
        both = diff & (i != NOID) & (i_ref != NOID)
        assert close(d[both], d_ref[both]).all(), f"call {call}: ids differ away from a depth tie"
        assert not (diff & ~both & ~tied)[px].any(), f"call {call}: hit/miss differs on a decided pixel"
        assert (diff & ~both).sum() <= 3, f"call {call}: {(diff & ~both).sum()} hit/miss differences"
        same = ~diff & (i_ref != NOID)
        assert close(d[same], d_ref[same]).all()
        assert (np.isinf(d) == (i == NOID)).all()


def test_depth_noalloc_skips_instances_of_unknown_type():
    """A record whose type is not below n_types writes no pixel (the call cannot check device
    records on the host); the other instances' result is unchanged bit for bit."""
    import torch
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native

    sc = sg.three_types_scene(96, 72, nerf=False)
    cam = native.Renderer.camera(sc.eye, sc.target, sc.fov_deg)
    w = torch.from_numpy(np.concatenate([t.nedf_w for t in sc.types]).astype(np.float32)).cuda()
    rec = instance_records(sc)
    d0, i0 = _noalloc(native, sc, torch.from_numpy(rec.view(np.uint8).copy()).cuda(), w, cam)
    assert (i0 != 0xFFFFFFFF).sum() > 200
    bad = rec.copy()
    bad["type"][::3] = [len(sc.types), 64, 0xFFFFFFFF] * (len(bad[::3]) // 3) + [64] * (len(bad[::3]) % 3)
    d1, i1 = _noalloc(native, sc, torch.from_numpy(bad.view(np.uint8).copy()).cuda(), w, cam)
    skipped = set(np.nonzero(bad["type"] >= len(sc.types))[0].tolist())
    assert not np.isin(i1, list(skipped)).any()
    # removing the skipped instances from the valid list gives the same pixels
    keep = np.array([k not in skipped for k in range(sc.n_inst)])
    only = rec.copy()
    only["s"][~keep] = 0.0          # a non-positive scale is skipped as well
    d2, i2 = _noalloc(native, sc, torch.from_numpy(only.view(np.uint8).copy()).cuda(), w, cam)
    assert np.array_equal(i1, i2) and np.array_equal(d1.view(np.uint32), d2.view(np.uint32))
    assert (i1 != i0).any()


def test_depth_noalloc_rejects_oversized_frames():
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native
    cam = native.Renderer.camera([0, 0, 3], [0, 0, 0], 40)
    rb = (C.c_float * 1)(1.0)
    rc = native._lib.nedf_compose_depth_noalloc(1024, 1024, C.byref(cam), 1, 16, 1, rb, 4, 64, 16, 16, 16, None)
    assert rc == native.NEDF_ERR_ARG
    assert b"512" in native._lib.nedf_compose_last_error(None)
