"""Debug checks and host-side fault injection: guard bytes and work-list invariants after real
frames, a forced status word, and a device wait that runs out (a bounded mbarrier wait on a phase
that nothing completes).  None of these faults, traps or hangs the GPU."""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native as n
    return n


def _frame(r, sc):
    import torch
    n = sc.W * sc.H
    d = torch.empty(n, device="cuda")
    i = torch.empty(n, dtype=torch.int32, device="cuda")
    st = r.render(r.camera(sc.eye, sc.target, sc.fov_deg), r.lights(sc.lights), d, i, None, None, None, stats=True)
    return st, d, i


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_guards_and_work_list_invariants_after_frames(native, prec):
    sc = sg.three_types_scene(192, 160)
    r = native.renderer_for(sc, precision=prec)
    o = r.get_options()
    o.fallback_conf, o.refine_steps, o.outlier_resample = 0.9, 4, 1
    r.set_options(o)
    for _ in range(2):
        st, _, _ = _frame(r, sc)
        assert st.status == 0 and st.primary_pairs > 0 and st.shadow_pairs > 0
        r.validate()
    o.depth_source = native.DEPTH_MARCH
    r.set_options(o)
    _frame(r, sc)
    r.validate()
    r.close()


def test_forced_status_word_is_reported_and_cleared(native):
    sc = sg.tiny_sphere_scene()
    r = native.renderer_for(sc)
    for bits, code in ((4, native.NEDF_ERR_TIMEOUT), (1, native.NEDF_ERR_CAPACITY), (2, native.NEDF_ERR_CAPACITY)):
        r.inject_status(bits)
        with pytest.raises(native.NedfError) as e:
            r.sync()
        assert e.value.code == code
        r.sync()                                  # the word was cleared with the report
    st, d, _ = _frame(r, sc)                      # and the handle still renders
    assert st.status == 0 and np.isfinite(d.cpu().numpy()).any()
    r.close()


def test_device_wait_runs_out_and_reports_timeout(native):
    """An mbarrier wait that nothing completes gives up after its limit; the kernel returns, the
    host reads the timeout, and the same context renders a correct frame afterwards."""
    sc = sg.tiny_sphere_scene()
    r = native.renderer_for(sc, precision=native.PREC_BF16)
    st0, d0, i0 = _frame(r, sc)
    r.check_wait_limit()
    st1, d1, i1 = _frame(r, sc)
    assert st1.status == 0
    assert np.array_equal(d0.cpu().numpy(), d1.cpu().numpy()) and np.array_equal(i0.cpu().numpy(), i1.cpu().numpy())
    r.close()
