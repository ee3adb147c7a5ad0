"""Pins of the oracle's supervision by a density network (plugin mode: the NeDF's labels from
Eq. 5 on a generic radiance field's density) against closed forms: a constant density (a
geometric series), an empty field, and a density ramp behind a plane, whose termination depth
tends to the plane crossing plus the mean of a Gaussian-tailed stopping distance.
"""
import math

import numpy as np

from paper_2308_04669_gb300 import scenegen as sg


def _net(hidden=1, width=64):
    return np.zeros(sg.mlp_param_count(sg.mlp_dims(sg.DENS_IN, hidden, width, 1)), np.float64)


def _layers(w, hidden, width):
    dims = sg.mlp_dims(sg.DENS_IN, hidden, width, 1)
    out, off = [], 0
    for fi, fo in zip(dims[:-1], dims[1:]):
        out.append((w[off:off + fi * fo].reshape(fo, fi), w[off + fi * fo:off + fi * fo + fo]))
        off += fi * fo + fo
    return out


def test_constant_density_is_a_geometric_series(orc):
    """sigma = b everywhere (output bias only): with q = exp(-b delta) the weights are
    (1 - q) q^i, so A = 1 - q^N and A D = (1 - q) sum_i q^i t_i in closed form."""
    rng = np.random.default_rng(3)
    for b, N in ((0.7, 64), (3.0, 128), (40.0, 96)):
        w = _net()
        w[-1] = b
        o = rng.normal(size=(5, 3)); o /= np.linalg.norm(o, axis=1, keepdims=True)
        d = -o + 0.5 * rng.normal(size=(5, 3))
        m, h, a = orc.density_labels(w, 1, 64, 1.0, N, o, d)
        for k in range(5):
            dd = d[k] / np.linalg.norm(d[k])
            tp = -o[k] @ dd
            disc = tp * tp - (o[k] @ o[k] - 1.0)
            te, tx = tp - math.sqrt(disc), tp + math.sqrt(disc)
            delta = (tx - te) / N
            q = math.exp(-b * delta)
            A = 1.0 - q ** N
            S0 = (1 - q ** N) / (1 - q)
            S1 = q * (1 - N * q ** (N - 1) + (N - 1) * q ** N) / (1 - q) ** 2
            D = (1 - q) * (te * S0 + delta * (S1 + 0.5 * S0)) / A
            assert abs(a[k] - A) < 1e-12
            assert h[k] == (A > 0.5)
            if h[k]:
                assert abs(m[k] - (tp - D)) < 1e-12


def test_empty_field_has_no_hits(orc):
    w = sg.density_weights(2)
    w[-1] = -1e3                                   # ReLU(output) = 0 everywhere
    rng = np.random.default_rng(4)
    o = rng.normal(size=(20, 3)); o /= np.linalg.norm(o, axis=1, keepdims=True)
    m, h, a = orc.density_labels(w, 2, 64, 1.0, 64, o, -o)
    assert not h.any() and not a.any() and not m.any()


def test_density_ramp_behind_a_plane(orc):
    """sigma = ReLU(K (c - z)) (a hidden unit passes z + 2, the output is K (c + 2 - h)): a ray
    down the z axis from z = 1 crosses the plane at t_c = 1 - c and then stops at an extra
    distance s with P(s > u) = exp(-K u^2 / 2), mean sqrt(pi / (2 K))."""
    for K, c in ((2e4, 0.3), (5e3, -0.4)):
        w = _net()
        (W0, b0), (W1, b1) = _layers(w, 1, 64)        # views into w
        W0[0, 2] = 1.0
        b0[0] = 2.0
        W1[0, 0] = -K
        b1[0] = K * (c + 2.0)
        assert abs(orc.density_net(w, 1, 64, np.array([0.1, 0.2, c - 0.01])) - K * 0.01) < 1e-9
        N = 2048
        m, h, a = orc.density_labels(w, 1, 64, 1.0, N, np.array([[0.0, 0.0, 1.0]]), np.array([[0.0, 0.0, -1.0]]))
        D = 1.0 - m[0]                                 # t_perp = 1 on this ray
        delta = 2.0 / N
        assert h[0] == 1 and a[0] > 0.999
        assert abs(D - (1.0 - c + math.sqrt(math.pi / (2 * K)))) < 1.5 * delta, D
