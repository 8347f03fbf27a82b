"""Input generators: seeded, shaped like the paper's workloads."""
from pathlib import Path

import numpy as np

from paper_2104_04653_gb300 import workloads as W

GOLDEN = Path(__file__).resolve().parent / "golden"


def test_bl_front_closed_form():
    """Welge tangent of the Section 5 fractional flow: s_f = 1/sqrt(M+1)."""
    rows = [l.split() for l in (GOLDEN / "bl_front.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    for M, sf in rows:
        M, sf = float(M), float(sf)
        assert abs(W.bl_front_saturation(M) - sf) < 1e-15
        # tangency checked numerically: f'(s_f) = f(s_f)/s_f
        f = lambda s: M * s * s / (M * s * s + (1 - s) ** 2)
        d = (f(sf + 1e-7) - f(sf - 1e-7)) / 2e-7
        assert abs(d - f(sf) / sf) < 1e-6


def test_bl_profile_monotone_and_bounded():
    rng = np.random.default_rng(0)
    s = W.bl_saturation(64, 64, 1 / 64, 5, 5.0, rng)
    assert s.min() == 0.0 and s.max() <= 1.0
    behind = s[s > 0]
    assert behind.min() >= W.bl_front_saturation(5.0) - 1e-12
    # saturation decreases along x behind the front
    row = s[10]
    nz = row[row > 0]
    assert np.all(np.diff(nz) <= 1e-12)
    lam = W.total_mobility(s, 1.0, 5.0)
    assert lam.min() > 0


def test_grf_statistics():
    rng = np.random.default_rng(1)
    n = 128
    f = np.stack([W.grf_exponential(n, n, 1 / n, 2.0, 0.1, rng) for _ in range(8)])
    assert abs(f.var() - 2.0) < 0.4
    # correlation at lag 0.1 ~ exp(-1)
    lag = int(0.1 * n)
    c = np.mean(f[:, :, :-lag] * f[:, :, lag:]) / f.var()
    assert abs(c - np.exp(-1)) < 0.12


def test_channels_binary_and_seeded():
    a = W.config2()
    b = W.config2()
    assert np.array_equal(a.K, b.K)
    vals = np.unique(a.K)
    assert set(vals) == {1e-3, 1e3}
    assert (a.K == 1e3).mean() > 0.05


def test_config_shapes():
    c1 = W.config1()
    assert c1.K.shape == (1, 64, 64) and c1.pure_neumann
    assert abs(c1.q.sum()) < 1e-9
    c2 = W.config2()
    assert c2.K.shape == (1, 64, 256) and c2.n_iface(0) == 108
    assert int(c2.iface_nU[0][0] + c2.iface_nP[0][0]) == 8
