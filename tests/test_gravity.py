"""Pins of the gravity term of the Darcy solve in the oracle (Eq.
"Darcy_wg": u = -K (lambda grad p - lambda_g g grad h), the height h along
+y).  The gravity velocity w = K lambda_g g enters the two-point fluxes as
(kappa_l w_r + kappa_r w_l)/(kappa_l + kappa_r) on faces normal to y (the
face pressure eliminated between the two half-cell fluxes), as w_c on
Dirichlet faces and as w_c T_R / (2 kappa_c) on Robin faces."""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from paper_2104_04653_gb300 import workloads as W


def _with_gravity(prob, w):
    prob.grav = [np.asarray(w, np.float64)]
    return prob


def test_hydrostatic_closed_form():
    """Homogeneous kappa = 2 and w = 3, no flow through any boundary, no
    sources: u = 0 everywhere and p = (w / kappa) y + c, for the fine grid
    and for MRCM with linear spaces."""
    n, s = 64, 16
    prob = W.make_problem(n, n, s, np.full((n, n), 2.0), bc=W.bc_no_flow(n, n), n_u=2, n_p=2,
                          pure_neumann=True)
    _with_gravity(prob, np.full((n, n), 3.0))
    y = (np.arange(n) + 0.5) * prob.h
    exact = np.repeat((1.5 * (y - y.mean()))[:, None], n, axis=1)
    for sol in (O.fine_solve(prob), O.mrcm_solve(prob)):
        np.testing.assert_allclose(sol["p"][0], exact, atol=1e-12)
        # velocities are differences of O(1) pressures over h = 1/64: roundoff
        assert np.abs(sol["ux"][0]).max() < 1e-10 and np.abs(sol["uy"][0]).max() < 1e-10


def _heterogeneous(nx, ny, s, n_u, n_p, seed, pure_neumann=False):
    rng = np.random.default_rng(seed)
    K = np.exp(1.5 * rng.standard_normal((ny, nx)))
    h = 1.0 / ny
    if pure_neumann:
        prob = W.make_problem(nx, ny, s, K, q=W.five_spot_sources(nx, ny, h),
                              bc=W.bc_no_flow(nx, ny), n_u=n_u, n_p=n_p, pure_neumann=True)
    else:
        prob = W.make_problem(nx, ny, s, K, bc=W.bc_left_right(nx, ny), n_u=n_u, n_p=n_p)
    prob.lam = rng.uniform(0.5, 2.0, (1, ny, nx))
    return _with_gravity(prob, K * rng.uniform(0.5, 3.0, (ny, nx)))


@pytest.mark.parametrize("pure_neumann", [False, True])
def test_full_spaces_equal_fine_grid_with_gravity(pure_neumann):
    """Full interface spaces make MRCM the fine-grid two-point solve, with
    the gravity term too."""
    nx, ny, s = 16, 16, 8
    prob = _heterogeneous(nx, ny, s, s, s, seed=3, pure_neumann=pure_neumann)
    ep, eu = O.errors(O.mrcm_solve(prob), O.fine_solve(prob))
    assert ep < 1e-11 and eu < 1e-11, (ep, eu)


@pytest.mark.parametrize("case", [(8, 8, 4, 2, 2, False), (8, 8, 4, 2, 1, True),
                                  (12, 8, 4, 3, 2, False)])
def test_monolithic_brute_force_with_gravity(case):
    """The basis and interface path with gravity equals one dense solve of
    all cell, face and interface unknowns with the half-cell flux law
    u = 2 kappa (p_c - p_f)/h + n_y w_c and the Robin condition written
    literally."""
    nx, ny, s, nu, npp, pn = case
    prob = _heterogeneous(nx, ny, s, nu, npp, seed=nx * 10 + ny, pure_neumann=pn)
    sol = O.mrcm_solve(prob)
    mono = O.monolithic_solve(prob)
    assert O.rel_l2(mono["p"], sol["p"][0]) < 1e-11
    assert O.rel_l2(mono["gamma_u"], sol["gamma_u"][0]) < 1e-11


def test_zero_gravity_changes_nothing():
    prob = _heterogeneous(32, 32, 16, 2, 2, seed=9)
    prob.grav = None
    plain = O.mrcm_solve(prob)
    _with_gravity(prob, np.zeros((32, 32)))
    zero = O.mrcm_solve(prob)
    for k in ("p", "ux", "uy"):
        assert np.array_equal(plain[k], zero[k])


def test_gravity_changes_the_solution_and_keeps_the_mass_balance():
    """A real gravity field moves the solution; every cell still balances
    its sources (outward face velocities, interface faces one-sided)."""
    prob = _heterogeneous(32, 32, 16, 2, 2, seed=11)
    sol = O.mrcm_solve(prob)
    w = prob.grav[0]
    prob.grav = None
    assert O.rel_l2(O.mrcm_solve(prob)["p"], sol["p"]) > 1e-3
    prob.grav = [w]
    ux, uy, h = sol["ux"][0], sol["uy"][0], prob.h
    lay = O.Layout(prob, 0)
    s = lay.s
    gam = sol["gamma_u"][0]
    ny, nx = prob.ny, prob.nx
    for j in range(ny):
        for i in range(nx):
            out = 0.0
            for side in ("W", "E", "S", "N"):
                on_if = ((side == "E" and i % s == s - 1 and i < nx - 1) or
                         (side == "W" and i % s == 0 and i > 0) or
                         (side == "N" and j % s == s - 1 and j < ny - 1) or
                         (side == "S" and j % s == 0 and j > 0))
                if on_if:        # the cell's own one-sided velocity
                    if side in ("E", "W"):
                        g = (j // s) * (lay.Sx - 1) + (i // s - (1 if side == "W" else 0))
                        out += gam[g, 0 if side == "E" else 1, j % s]
                    else:
                        g = (lay.Sx - 1) * lay.Sy + (j // s - (1 if side == "S" else 0)) * lay.Sx + i // s
                        out += gam[g, 0 if side == "N" else 1, i % s]
                else:
                    out += {"W": -ux[j, i], "E": ux[j, i + 1], "S": -uy[j, i], "N": uy[j + 1, i]}[side]
            assert abs(out * h - prob.q[0, j, i] * h * h) < 1e-11 * max(1.0, np.abs(gam).max())


def test_set_gravity_needs_a_context():
    from paper_2104_04653_gb300 import build, mrcm
    build.build()
    assert mrcm.lib().mrcm_set_gravity(None, None) == mrcm.MRCM_EINVAL
