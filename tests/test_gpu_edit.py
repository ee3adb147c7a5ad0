"""Buffer reuse while one object is manipulated (Section "CUDA implementation": the other objects'
rendering is frozen and their buffers reused).

The edit frame is built from the frozen part's packed depth/id keys, colours and occlusion bits
plus the moved instance alone: the per-pixel minimum over all instances is the minimum of the
frozen keys and the moved instance's keys; a pixel's colour depends only on its winner; a pixel's
occlusion is the OR over occluders.  Every per-pair and per-pixel computation is a pure function
of its inputs, so an edit frame must equal the whole frame bit for bit.
"""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2308_04669_gb300 import build
    build.build()


def _buffers(r, n, fn):
    import torch
    d = torch.empty(n, device="cuda"); i = torch.empty(n, dtype=torch.int32, device="cuda")
    c = torch.empty(n, 4, device="cuda"); s = torch.empty(n, device="cuda"); o = torch.empty(n, 4, device="cuda")
    st = fn(d, i, c, s, o)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (d, i, c, s, o)], st


def _run(sc, precision, moves):
    from paper_2308_04669_gb300 import native
    r = native.renderer_for(sc, precision=precision)
    o = r.get_options()
    o.fallback_conf, o.refine_steps, o.outlier_resample = 0.9, 4, 1
    r.set_options(o)
    cam, li = r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights, sc.light_parallel)
    n = sc.W * sc.H
    full, st0 = _buffers(r, n, lambda d, i, c, s, o_: r.render(cam, li, d, i, c, s, o_, stats=True))
    ids = full[1].view(np.uint32)
    won = np.bincount(ids[ids != 0xFFFFFFFF], minlength=len(sc.inst_type))
    e = int(np.argmax(won))                       # the instance that covers the most pixels
    r.begin_edit(cam, li, e)
    T = sc.inst_T.copy()
    checked = 0
    for dT in moves:
        T[e] = sc.inst_T[e] + np.asarray(dT, np.float32)
        r.set_instances(sc.inst_type, sc.inst_R, T, sc.inst_s)
        got, st = _buffers(r, n, lambda d, i, c, s, o_: r.render_edit(d, i, c, s, o_, stats=True))
        ref, st_full = _buffers(r, n, lambda d, i, c, s, o_: r.render(cam, li, d, i, c, s, o_, stats=True))
        assert st.status == 0 and st_full.status == 0
        assert st.primary_pairs < st_full.primary_pairs          # only the moved instance's pairs
        for k, (a, b) in enumerate(zip(got, ref)):
            same = np.array_equal(a.view(np.uint32), b.view(np.uint32))
            assert same, (dT, k, int((a.view(np.uint32) != b.view(np.uint32)).sum()))
        checked += int((got[1].view(np.uint32) == e).sum())
    assert checked > 0                                           # the moved instance was on screen
    # another instance changes: the frozen buffers are stale, so the edit frame is refused
    T2 = T.copy()
    T2[(e + 1) % len(T2)] += 0.1
    r.set_instances(sc.inst_type, sc.inst_R, T2, sc.inst_s)
    with pytest.raises(native.NedfError):
        r.render_edit()
    r.end_edit()
    with pytest.raises(native.NedfError):
        r.render_edit()
    r.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_edit_frames_equal_whole_frames(prec):
    from paper_2308_04669_gb300 import native
    p = {"fp32": native.PREC_FP32, "bf16": native.PREC_BF16, "fp8": native.PREC_FP8}[prec]
    _run(sg.three_types_scene(128, 128), p, [(0.3, -0.2, 0.1), (-0.6, 0.4, 0.5), (1.5, 0.0, -1.0)])


def test_edit_frames_with_a_parallel_light():
    from paper_2308_04669_gb300 import native
    sc = sg.three_types_scene(128, 128, nerf=False)
    sc.lights = sg.f32([[-0.4, -1.0, -0.3], [1.0, 9.0, 2.0]])
    sc.light_parallel = np.array([1, 0])
    _run(sc, native.PREC_BF16, [(0.3, -0.2, 0.1), (-0.6, 0.4, 0.5)])


def test_edit_frames_equal_whole_frames_thousand_instances():
    from paper_2308_04669_gb300 import native
    _run(sg.thousand_scene(384, 384), native.PREC_BF16, [(0.5, 0.5, 0.0), (-2.0, 1.0, 3.0)])
