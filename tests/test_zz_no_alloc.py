"""The allocation-free Step-1 entry point against the handle-based renderer.

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


def test_depth_noalloc_matches_render_on_two_calls():
    import torch
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native

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
    d_ref, i_ref = d_ref.cpu().numpy(), i_ref.cpu().numpy()
    assert (i_ref != -1).sum() > 1000

    # caller-owned inputs and outputs
    inst = torch.from_numpy(instance_records(sc).view(np.uint8).copy()).cuda()
    w = torch.from_numpy(np.concatenate([t.nedf_w for t in sc.types]).astype(np.float32)).cuda()
    rb = (C.c_float * len(sc.types))(*[t.rb for t in sc.types])
    t0 = sc.types[0]
    for call in range(2):
        depth = torch.full((n,), float("nan"), device="cuda")
        ids = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        rc = native._lib.nedf_compose_depth_noalloc(sc.W, sc.H, C.byref(cam), sc.n_inst, inst.data_ptr(),
                                                     len(sc.types), rb, t0.nedf_hidden, t0.nedf_width,
                                                     w.data_ptr(), depth.data_ptr(), ids.data_ptr(), None)
        assert rc == native.NEDF_OK, native._lib.nedf_compose_last_error(None)
        torch.cuda.synchronize()
        d, i = depth.cpu().numpy(), ids.cpu().numpy()
        assert (i == i_ref).mean() > 0.999, f"call {call}: id agreement {(i == i_ref).mean()}"
        same = (i == i_ref) & (i_ref != -1)
        assert np.all(np.abs(d[same] - d_ref[same]) <= np.maximum(2e-3, 1e-3 * np.abs(d_ref[same])))
        assert (np.isinf(d) == (i == -1)).all()


def test_depth_noalloc_rejects_oversized_frames():
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native
    cam = native.Renderer.camera([0, 0, 3], [0, 0, 0], 40)
    rb = (C.c_float * 1)(1.0)
    rc = native._lib.nedf_compose_depth_noalloc(1024, 1024, C.byref(cam), 1, 16, 1, rb, 4, 64, 16, 16, 16, None)
    assert rc == native.NEDF_ERR_ARG
    assert b"512" in native._lib.nedf_compose_last_error(None)
