"""Pins of the sampled full-size checks (oracle/sampled.py) against the whole
oracle on small grids: given the oracle's own interface solution the
re-solved subdomains reproduce its pressures and the continuity defects of
Eq. "mrc2" vanish to rounding; a perturbed interface unknown shows up in its
interface's defect; the global balance holds for the oracle's fluxes and
fails for a perturbed boundary flux."""
import numpy as np

from oracle import mrcm_oracle as O
from oracle import sampled as S
from paper_2104_04653_gb300 import workloads as W


def _full(prob):
    ref = O.mrcm_solve(prob, return_system=True)
    x = np.concatenate([sy["x"] for sy in ref["systems"]])
    return ref, x


def _probs():
    grav = W.config3(n_real=2, n=64)
    rng = np.random.default_rng(3)
    grav.grav = [K * rng.uniform(0.5, 2.0, K.shape) for K in grav.K]
    return [W.config3(n_real=2, n=64), W.config2(nx=64, ny=32), grav]


def test_oracle_solution_passes_the_sampled_checks():
    for prob in _probs():
        ref, x = _full(prob)
        wp, wd = S.sampled_checks(prob, ref["p"], x, np.random.default_rng(0), n_sub=8, n_if=8)
        assert wp <= 1e-12 and wd <= 1e-12, (prob.name, wp, wd)


def test_perturbed_interface_unknown_is_caught():
    prob = W.config3(n_real=2, n=64)
    ref, x = _full(prob)
    lay = O.Layout(prob, 0)
    g = 3
    f = lay.ifaces[g]
    xb = x.copy()
    xb[f["off"]] *= 1.0 + 1e-6                      # U_0 of interface 3, realisation 0
    worst = 0.0
    for seed in range(40):                          # until interface 3 is sampled
        rng = np.random.default_rng(seed)
        if g not in rng.choice(len(lay.ifaces), size=6, replace=False):
            continue
        _, wd = S.sampled_checks(prob, ref["p"], xb, np.random.default_rng(seed), n_sub=0,
                                 n_if=6, reals=[0])
        worst = max(worst, wd)
    assert worst > 1e-9, worst


def test_global_balance():
    prob = W.config3(n_real=2, n=64)
    ref, _ = _full(prob)
    assert S.global_balance(prob, ref["ux"], ref["uy"]) <= 1e-12
    ux = ref["ux"].copy()
    ux[1][5, -1] += 1e-6
    assert S.global_balance(prob, ux, ref["uy"]) > 1e-8
