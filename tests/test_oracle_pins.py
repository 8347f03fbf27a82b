"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test would fail under a plausible mistake in the oracle: a wrong
transmissibility or Robin constant (linear pressure, fine-grid equality,
brute force), a wrong sign of sigma or of a test row (symmetry, balance),
a transposed interface index (fine-grid equality, brute force), a dropped
source or boundary term (mass balance).
"""
from pathlib import Path

import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2104_04653_gb300 import workloads as W

GOLDEN = Path(__file__).resolve().parent / "golden"


def _load(name):
    rows = [l.split() for l in (GOLDEN / name).read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=np.float64)


def _random_problem(nx, ny, s, n_u, n_p, seed, pure_neumann=False, var=2.0, alpha=True):
    rng = np.random.default_rng(seed)
    K = np.exp(np.sqrt(var) * rng.standard_normal((ny, nx)))
    h = 1.0 / ny
    if pure_neumann:
        p = W.make_problem(nx, ny, s, K, q=W.five_spot_sources(nx, ny, h),
                           bc=W.bc_no_flow(nx, ny), n_u=n_u, n_p=n_p, pure_neumann=True)
    else:
        p = W.make_problem(nx, ny, s, K, bc=W.bc_left_right(nx, ny), n_u=n_u, n_p=n_p)
    if alpha:
        p.alpha = [rng.uniform(0.3, 3.0, (p.n_iface(0), s))]
    return p


# ------------------------------------------------------------------ (i) closed form
def test_linear_pressure_exact():
    """Homogeneous K, p = 1 - x: exact for the fine grid and for MRCM with
    linear interface spaces (Section 3.1 default spaces)."""
    nx, ny, s = 32, 16, 8
    h = 1.0 / ny
    prob = W.make_problem(nx, ny, s, np.full((ny, nx), 3.0),
                          bc=W.bc_linear_pressure(nx, ny, h), n_u=2, n_p=2)
    gold = _load("linear_pressure.txt")
    for sol in (O.mrcm_solve(prob), O.fine_solve(prob)):
        p = sol["p"][0]
        for i, val in gold:
            np.testing.assert_allclose(p[:, int(i)], val, atol=1e-12)
        np.testing.assert_allclose(sol["ux"][0], 3.0, rtol=1e-12)
        np.testing.assert_allclose(sol["uy"][0], 0.0, atol=1e-11)


def test_linear_pressure_exact_mixed_subdomain_sizes():
    """The same closed form with 16 x 16 and 32 x 32 subdomains in one batch
    (one realisation each)."""
    nx, ny = 64, 64
    h = 1.0 / ny
    prob = W.make_problem(nx, ny, [16, 32], np.full((2, ny, nx), 0.7),
                          bc=W.bc_linear_pressure(nx, ny, h), n_u=2, n_p=2)
    sol = O.mrcm_solve(prob)
    xc = (np.arange(nx) + 0.5) * h
    for r in range(2):
        np.testing.assert_allclose(sol["p"][r], np.broadcast_to(1.0 - xc, (ny, nx)), atol=1e-12)
        np.testing.assert_allclose(sol["ux"][r], 0.7, rtol=1e-12)
        np.testing.assert_allclose(sol["uy"][r], 0.0, atol=1e-11)


# ------------------------------------------------------------------ (ii) special case
@pytest.mark.parametrize("pure_neumann", [False, True])
@pytest.mark.parametrize("alpha", [0.05, 1.0, 20.0])
def test_full_spaces_equal_fine_grid(pure_neumann, alpha):
    """With every fine-face indicator in both interface spaces, MRCM imposes
    exact continuity of face pressure and flux, i.e. it is the fine-grid
    two-point solve, for any alpha > 0 (Eq. "mrc1", "mrc2")."""
    nx, ny, s = 16, 16, 8
    prob = _random_problem(nx, ny, s, s, s, seed=7, pure_neumann=pure_neumann, alpha=False)
    prob.alpha = [np.full((prob.n_iface(0), s), alpha)]
    ep, eu = O.errors(O.mrcm_solve(prob), O.fine_solve(prob))
    assert ep < 1e-11 and eu < 1e-11


# ------------------------------------------------------------------ (iii) invariants
def test_local_operators_spd_and_symmetric():
    prob = W.config2(nx=64, ny=32)
    lay = O.Layout(prob, 0)
    kap = prob.lam[0] * prob.K[0]
    for J in range(lay.Sy):
        for I in range(lay.Sx):
            A = O.Local(prob, 0, lay, I, J, kap).A
            assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
            np.linalg.cholesky(A)          # raises if not SPD


def test_interface_matrix_symmetric_quasidefinite():
    """Negating the flux-continuity rows makes the interface matrix
    symmetric, with a negative definite U-block and a positive definite
    P-block (quasi-definite): what lets the GPU eliminate without pivoting."""
    prob = _random_problem(64, 32, 16, 3, 2, seed=11)
    sysm = O.mrcm_solve(prob, return_system=True)["systems"][0]
    M, lay = sysm["M"], sysm["layout"]
    isP = np.zeros(M.shape[0], bool)
    for f in lay.ifaces:
        isP[f["off"] + f["nU"]:f["off"] + f["nU"] + f["nP"]] = True
    S = np.where(isP[:, None], -M, M)
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    S = 0.5 * (S + S.T)
    assert np.linalg.eigvalsh(S[np.ix_(~isP, ~isP)]).max() < 0
    assert np.linalg.eigvalsh(S[np.ix_(isP, isP)]).min() > 0


def _cell_outflow(prob, r, sol, lay):
    """Sum of outward fluxes of every cell from p and the one-sided
    interface velocities."""
    ny, nx, h, s = prob.ny, prob.nx, prob.h, lay.s
    kap = prob.lam[r] * prob.K[r]
    p = sol["p"][r]
    gam = sol["gamma_u"][r]
    out = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            for side, di, dj in (("W", -1, 0), ("E", 1, 0), ("S", 0, -1), ("N", 0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    if (i // s, j // s) == (ii // s, jj // s):
                        out[j, i] += O.harmonic_T(kap[j, i], kap[jj, ii]) * (p[j, i] - p[jj, ii])
                    else:
                        if side in ("E", "W"):
                            g = (j // s) * (lay.Sx - 1) + min(i, ii) // s
                            e = j % s
                        else:
                            g = (lay.Sx - 1) * lay.Sy + (min(j, jj) // s) * lay.Sx + i // s
                            e = i % s
                        sd = 0 if side in ("E", "N") else 1
                        out[j, i] += h * gam[g, sd, e]
                else:
                    k = O.boundary_face(prob, side, i, j)
                    if prob.bc_type[k] == O.DIRICHLET:
                        out[j, i] += 2 * kap[j, i] * (p[j, i] - prob.bc_val[k])
                    else:
                        out[j, i] += prob.bc_val[k] * h
    return out


@pytest.mark.parametrize("pure_neumann,n,s", [(False, 32, 8), (True, 32, 8), (False, 64, 32)])
def test_mass_balance_and_interface_balance(pure_neumann, n, s):
    prob = _random_problem(n, n, s, 2, 3, seed=5, pure_neumann=pure_neumann)
    sol = O.mrcm_solve(prob)
    lay = O.Layout(prob, 0)
    h = prob.h
    out = _cell_outflow(prob, 0, sol, lay)
    src = prob.q[0] * h * h
    assert np.abs(out - src).max() <= 1e-11 * max(1.0, np.abs(out).max())
    gam = sol["gamma_u"][0]
    for g, f in enumerate(lay.ifaces):
        # flux continuity tested by every pressure function (Eq. "mrc2")
        jump = f["psi"] @ (h * (gam[g, 0] + gam[g, 1]))
        assert np.abs(jump).max() <= 1e-11 * max(1.0, np.abs(gam[g]).max())
    # global balance: sources = boundary outflow
    total_src = src.sum()
    bnd = out.sum()
    assert abs(total_src - bnd) <= 1e-10 * max(1.0, np.abs(out).sum())


def test_basis_family_invariance():
    """Legendre and monomial functions span the same spaces: (p, u) agree."""
    prob = _random_problem(32, 32, 8, 3, 3, seed=9)
    a = O.mrcm_solve(prob)
    prob.basis = "monomial"
    b = O.mrcm_solve(prob)
    ep, eu = O.errors(a, b)
    assert ep < 1e-11 and eu < 1e-11


def test_legendre_values():
    """Interface functions: Legendre polynomials at face midpoints."""
    v = O.interface_functions(4, 4)
    t = np.array([-0.75, -0.25, 0.25, 0.75])
    np.testing.assert_allclose(v[0], 1.0)
    np.testing.assert_allclose(v[1], t)
    np.testing.assert_allclose(v[2], 0.5 * (3 * t ** 2 - 1))
    np.testing.assert_allclose(v[3], 0.5 * (5 * t ** 3 - 3 * t))


# ------------------------------------------------------------------ (iv) brute force
@pytest.mark.parametrize("case", [(4, 4, 2, 1, 1, False), (8, 8, 4, 2, 2, False),
                                  (8, 8, 4, 2, 1, True), (8, 4, 4, 1, 2, False),
                                  (12, 8, 4, 3, 2, True), (12, 12, 4, 0, 2, False),
                                  (12, 12, 4, 2, 0, False)])
def test_monolithic_brute_force(case):
    """The basis + interface path equals one dense solve of all cell, face
    and interface unknowns with the Robin condition written literally."""
    nx, ny, s, nu, npp, pn = case
    prob = _random_problem(nx, ny, s, nu, npp, seed=nx * 100 + ny, pure_neumann=pn)
    sol = O.mrcm_solve(prob)
    mono = O.monolithic_solve(prob)
    assert O.rel_l2(mono["p"], sol["p"][0]) < 1e-11
    assert O.rel_l2(mono["gamma_u"], sol["gamma_u"][0]) < 1e-11


def test_refinement_self_difference():
    """The oracle's own rounding: plain FP64 vs extended-precision refined
    local solves on the high-contrast channel workload (1e6 contrast)."""
    prob = W.config2(nx=128, ny=64)
    ep, eu = O.errors(O.mrcm_solve(prob), O.mrcm_solve(prob, refine=True))
    assert ep < 1e-10 and eu < 1e-9


def test_planted_robin_constant_mistake_is_caught(monkeypatch):
    """A wrong Robin transmissibility (alpha H/h + 1 instead of + 1/2) must
    break the fine-grid equality pin."""
    prob = _random_problem(16, 16, 8, 8, 8, seed=1, alpha=False)
    good = O.errors(O.mrcm_solve(prob), O.fine_solve(prob))
    monkeypatch.setattr(O, "robin_T", lambda kc, a, H, h: kc / (a * H / h + 1.0))
    bad = O.errors(O.mrcm_solve(prob), O.fine_solve(prob))
    assert max(good) < 1e-11 and max(bad) > 1e-4


def test_planted_sigma_mistake_is_caught(monkeypatch):
    """Dropping sigma (the n_check . n_i sign) in the Robin data must break
    the brute-force pin."""
    prob = _random_problem(8, 8, 4, 2, 2, seed=3)
    mono = O.monolithic_solve(prob)
    real = O.robin_data
    monkeypatch.setattr(O, "robin_data", lambda f, sigma, beta, x: real(f, 1.0, beta, x))
    sol = O.mrcm_solve(prob)
    # reconstruction uses robin_data for the one-sided interface velocities
    assert O.rel_l2(mono["gamma_u"], sol["gamma_u"][0]) > 1e-3
