"""Pins of the transport oracle (oracle/transport.py; Section 4, Eqs.
"BL2D_Newton" to "up_fluxes_impli", the inflection-point trust region of
Section 4.1).

What fixes it, independently of its own formulas:
* the flux function's derivatives against central differences of f, and the
  inflection point of the symmetric case M = 1 (f(1 - s) = 1 - f(s), so
  f''(1/2) = 0);
* the Jacobian against central differences of the residual, on a grid with
  velocities of both signs;
* on one row of cells with a uniform velocity the upwind step couples each
  cell to its left neighbour only, so it can be solved by marching cell by
  cell with a scalar bisection: the trust-region Newton iterate must equal
  it, at CFL numbers from 0.5 to 1000;
* a converged step conserves water exactly: the change of the water volume
  equals dt times the net boundary inflow (a divergence-free velocity from
  the oracle's fine-grid Darcy solve);
* no flow leaves the saturation unchanged;
* under refinement the 1-D solution approaches the closed-form
  Buckley-Leverett profile (rarefaction, then the shock at the Welge
  saturation 1/sqrt(M + 1) of tests/golden/bl_front.txt) in L1;
* two planted mistakes are caught: downwind instead of upwind fluxes break
  the 1-D agreement, and a Jacobian without its couplings costs iterations.
"""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from oracle import transport as T
from paper_2104_04653_gb300 import workloads as W


def test_flux_derivatives_against_differences():
    for M in (1.0, 5.0, 10.0):
        s = np.linspace(0.02, 0.98, 25)
        e = 1e-6
        d1 = (T.frac_flow(s + e, M) - T.frac_flow(s - e, M)) / (2 * e)
        d2 = (T.frac_flow_d1(s + e, M) - T.frac_flow_d1(s - e, M)) / (2 * e)
        assert np.allclose(T.frac_flow_d1(s, M), d1, rtol=1e-7, atol=1e-9)
        assert np.allclose(T.frac_flow_d2(s, M), d2, rtol=1e-6, atol=1e-7)
    assert abs(T.inflection_point(1.0) - 0.5) < 1e-12
    for M in (5.0, 10.0):
        st = T.inflection_point(M)
        assert T.frac_flow_d2(st - 1e-6, M) > 0 > T.frac_flow_d2(st + 1e-6, M)


def _rand_case(seed, nx=7, ny=5):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.0, 1.0, (ny, nx))
    ux = rng.normal(size=(ny, nx + 1))
    uy = rng.normal(size=(ny + 1, nx))
    return s, ux, uy


def test_jacobian_against_differences():
    M, h, dt = 10.0, 0.1, 0.37
    for seed in range(3):
        s, ux, uy = _rand_case(seed)
        s_old = np.zeros_like(s)
        J = T.jacobian(s, ux, uy, h, dt, M).toarray()
        e = 1e-7
        Jd = np.zeros_like(J)
        for k in range(s.size):
            sp_, sm_ = s.copy().ravel(), s.copy().ravel()
            sp_[k] += e
            sm_[k] -= e
            Jd[:, k] = (T.residual(sp_.reshape(s.shape), s_old, ux, uy, h, dt, M).ravel() -
                        T.residual(sm_.reshape(s.shape), s_old, ux, uy, h, dt, M).ravel()) / (2 * e)
        assert np.allclose(J, Jd, rtol=1e-6, atol=1e-7)


def _row(n, u=1.0):
    return np.zeros((1, n)), np.full((1, n + 1), u), np.zeros((2, n))


@pytest.mark.parametrize("cfl", [0.5, 3.0, 10.0, 100.0, 1000.0])
def test_newton_equals_marching_on_one_row(cfl):
    M, n = 10.0, 64
    h = 1.0 / n
    dt = cfl * h
    s0, ux, uy = _row(n)
    # from the dry state, then from the state one step later
    for _ in range(2):
        got, it, _ = T.newton_step(s0, ux, uy, h, dt, M, eta=1e-14, max_iter=2000)
        ref = T.march_1d(s0[0], 1.0, h, dt, M)
        assert np.abs(got[0] - ref).max() <= 1e-12, (cfl, it)
        s0 = got


def test_converged_step_conserves_water():
    M = 10.0
    prob = W.config1()                       # 64x64 GRF, quarter five-spot
    prob = W.make_problem(64, 64, 16, prob.K[0], bc=W.bc_left_right(64, 64), n_u=2, n_p=2)
    ref = O.fine_solve(prob)
    ux, uy = ref["ux"][0], ref["uy"][0]
    h = prob.h
    s0 = np.zeros((64, 64))
    for dt in (2e-3, 2e-2):
        s, it, _ = T.newton_step(s0, ux, uy, h, dt, M, eta=1e-14, max_iter=3000)
        dv = float(np.sum(s - s0)) * h * h
        out = T.boundary_outflow(s, ux, uy, h, M)
        assert abs(dv + dt * out) <= 1e-11 * dt * abs(out) + 1e-15, (dt, dv, out, it)
        assert s.min() >= 0.0 and s.max() <= 1.0


def test_no_flow_leaves_saturation_unchanged():
    rng = np.random.default_rng(1)
    s0 = rng.uniform(0, 1, (6, 9))
    s, it, _ = T.newton_step(s0, np.zeros((6, 10)), np.zeros((7, 9)), 0.1, 5.0, 10.0, eta=1e-14)
    assert it == 1 and np.array_equal(s, s0)


def _bl_exact(x, t, M):
    """The Buckley-Leverett solution from s = 0 with s = 1 injected at x = 0:
    the rarefaction f'(s) = x / t on [s_f, 1] up to the shock x_f = t f'(s_f),
    s_f = 1/sqrt(M + 1) (Welge), then 0."""
    sf = 1.0 / np.sqrt(M + 1.0)
    xf = t * float(T.frac_flow_d1(sf, M))
    out = np.zeros_like(x)
    for i, xx in enumerate(x):
        if xx >= xf:
            continue
        lo, hi = sf, 1.0                      # f' decreases on [s_f, 1]
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if T.frac_flow_d1(mid, M) > xx / t:
                lo = mid
            else:
                hi = mid
        out[i] = 0.5 * (lo + hi)
    return out


def test_converges_to_the_buckley_leverett_solution():
    """After 0.3 pore volumes at CFL 0.5 the implicit upwind solution
    approaches the closed-form Buckley-Leverett profile in L1 as the grid is
    refined (first-order upwind smears the shock: about O(h^0.75))."""
    M, t = 10.0, 0.3
    errs = []
    for n in (50, 100, 200):
        h = 1.0 / n
        dt = 0.5 * h
        s = np.zeros(n)
        for _ in range(int(round(t / dt))):
            s = T.march_1d(s, 1.0, h, dt, M)
        x = (np.arange(n) + 0.5) * h
        errs.append(float(np.sum(np.abs(s - _bl_exact(x, t, M))) * h))
    assert errs[2] < 0.02 and errs[0] / errs[1] > 1.3 and errs[1] / errs[2] > 1.3, errs


def _mistake_breaks_agreement(monkeypatch, name, fn):
    M, n = 10.0, 32
    h = 1.0 / n
    dt = 5.0 * h
    s0, ux, uy = _row(n)
    monkeypatch.setattr(T, name, fn)
    got, _, _ = T.newton_step(s0, ux, uy, h, dt, M, eta=1e-14, max_iter=500)
    ref = T.march_1d(s0[0], 1.0, h, dt, M)
    return np.abs(got[0] - ref).max()


def test_planted_downwind_flux_is_caught(monkeypatch):
    orig = T.residual

    def downwind(s, s_old, ux, uy, h, dt, M, s_in=1.0):
        return orig(s, s_old, -np.asarray(ux), -np.asarray(uy), h, dt, M, s_in)

    assert _mistake_breaks_agreement(monkeypatch, "residual", downwind) > 1e-3


def test_planted_dropped_coupling_is_caught(monkeypatch):
    """A Jacobian without its upwind couplings still has the right root, but
    Newton loses its fast convergence: it needs more iterations."""
    M, n = 10.0, 32
    h = 1.0 / n
    dt = 5.0 * h
    s0, ux, uy = _row(n)
    _, it_ok, _ = T.newton_step(s0, ux, uy, h, dt, M, eta=1e-14, max_iter=500)
    orig = T.jacobian

    def diag_only(s, ux, uy, h, dt, M):
        import scipy.sparse as sp
        return sp.diags(orig(s, ux, uy, h, dt, M).diagonal()).tocsr()

    monkeypatch.setattr(T, "jacobian", diag_only)
    _, it_bad, _ = T.newton_step(s0, ux, uy, h, dt, M, eta=1e-14, max_iter=500)
    assert it_bad > it_ok + 5, (it_ok, it_bad)
