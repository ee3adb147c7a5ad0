"""Supervision by a generic radiance field's density network on the GPU (plugin mode: labels
from Eq. 5 on an MLP density, Section "Intersection network"): the labels against the oracle, and
the NeDF trained on them against the same kind of labels on held-out rays."""
import numpy as np
import pytest

from paper_2308_04669_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu

HIDDEN, WIDTH, SAMPLES = 2, 64, 128


@pytest.fixture(scope="module")
def lib():
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native
    return native


def _labels(r, w, n, seed):
    import torch
    o = torch.empty(n, 3, device="cuda"); d = torch.empty(n, 3, device="cuda")
    m = torch.empty(n, device="cuda"); h = torch.empty(n, device="cuda")
    r.make_labels_density(0, n, seed, SAMPLES, HIDDEN, WIDTH, w, o, d, m, h)
    torch.cuda.synchronize()
    return o, d, m, h


def test_density_labels_match_oracle(lib, orc):
    sc = sg.tiny_sphere_scene()
    r = lib.renderer_for(sc)
    w = sg.density_weights(9, HIDDEN, WIDTH)
    n = 1500
    o, d, m, h = _labels(r, w, n, 5)
    go, gd = o.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)
    oo, od = orc.train_rays(1.0, 5, 0, n)
    assert np.abs(go - oo).max() < 1e-5 and np.abs(gd - od).max() < 1e-5     # the same rays as make_labels
    om, oh, oa = orc.density_labels(w.astype(np.float64), HIDDEN, WIDTH, 1.0, SAMPLES, go, gd)
    gh = h.cpu().numpy() > 0.5
    decided = np.abs(oa - 0.5) > 1e-3
    assert decided.mean() > 0.98
    assert np.array_equal(gh[decided], oh[decided] == 1)
    both = decided & gh
    gm = m.cpu().numpy().astype(np.float64)
    err = np.abs(gm[both] - om[both])
    assert 0.2 < gh.mean() < 0.8 and err.max() < 2e-3, (gh.mean(), err.max())
    print(f"hits {gh.mean():.3f}; |m* gpu - oracle| median {np.median(err):.2e} max {err.max():.2e}")
    r.close()


def test_nedf_learns_a_density_networks_depth(lib):
    """The regression NeDF trained on density-network labels, judged on held-out rays labelled
    the same way: hit agreement and depth error before and after training."""
    import torch
    sc = sg.tiny_sphere_scene()
    r = lib.renderer_for(sc)
    w = sg.density_weights(9, HIDDEN, WIDTH)
    ho, hd, hm, hh = _labels(r, w, 1 << 14, 77)                  # held out

    def judge():
        out = torch.empty(ho.shape[0], 4, device="cuda")
        r.nedf_query(0, ho, hd, out)
        torch.cuda.synchronize()
        q = out.cpu().numpy()
        lab = hh.cpu().numpy() > 0.5
        both = lab & (q[:, 3] > 0.5)
        return dict(hit_agree=float(((q[:, 3] > 0.5) == lab).mean()),
                    median_err=float(np.median(np.abs(q[both, 0] - hm.cpu().numpy()[both]))) if both.any() else 1.0)

    before = judge()
    r.make_labels_density(0, 1 << 17, 3, SAMPLES, HIDDEN, WIDTH, w)
    losses = [r.train_step(0, 8192, 1e-3, want_loss=True) for _ in range(600)]
    after = judge()
    print(f"before {before} after {after}; loss {losses[0]:.4f} -> {np.mean(losses[-20:]):.4f}")
    assert np.mean(losses[-20:]) < 0.3 * losses[0]
    # the small NeDF of this scene (4 x 64) against blobs with sharp edges: a clear gain, not a fit
    assert after["hit_agree"] > 0.8 and after["hit_agree"] > before["hit_agree"] + 0.15
    assert after["median_err"] < 0.5 * before["median_err"]
    r.close()
