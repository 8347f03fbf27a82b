"""Pins of the oracle GMRES (oracle/gmres.py) against facts fixed by the
mathematics, and against an independent library implementation."""
import numpy as np
import pytest

from oracle import gmres as G


def _rng(seed):
    return np.random.default_rng(seed)


def _nonsym(n, seed, shift=4.0):
    r = _rng(seed)
    return shift * np.eye(n) + r.standard_normal((n, n)) / np.sqrt(n)


def test_distinct_eigenvalues_bound_the_steps():
    # the Krylov space of a diagonalisable A with d distinct eigenvalues has
    # dimension <= d, so full GMRES is exact after d steps
    r = _rng(1)
    n, lam = 30, np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    S = np.eye(n) + 0.1 * r.standard_normal((n, n))
    A = S @ np.diag(np.resize(lam, n)) @ np.linalg.inv(S)
    b = r.standard_normal(n)
    x, info = G.gmres(A, b, restart=n, tol=1e-10)
    assert info["converged"] and info["iters"] <= 5, info
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)


def test_first_step_closed_form():
    # one step from x0 = 0 minimises ||b - a A b|| over a: a = (b.Ab)/(Ab.Ab)
    A = _nonsym(20, 2)
    b = _rng(3).standard_normal(20)
    x, info = G.gmres(A, b, restart=1, tol=1e-30, maxiter=1)
    Ab = A @ b
    a = np.dot(b, Ab) / np.dot(Ab, Ab)
    assert info["iters"] == 1
    assert np.linalg.norm(x - a * b) <= 1e-14 * np.linalg.norm(a * b)


@pytest.mark.parametrize("restart", [5, 50])
def test_matches_direct_solve(restart):
    A = _nonsym(50, 4)
    b = _rng(5).standard_normal(50)
    x, info = G.gmres(A, b, restart=restart, tol=1e-13)
    ref = np.linalg.solve(A, b)
    assert info["converged"]
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_right_preconditioned_solution_and_monotone_history():
    A = _nonsym(60, 6, shift=1.5)
    blocks = [(k, 4) for k in range(0, 60, 4)]
    P = G.block_jacobi(A, blocks)
    b = _rng(7).standard_normal(60)
    x, info = G.gmres(A, b, P=P, restart=8, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(x)
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-15)       # restarted GMRES never increases the residual


def test_exact_block_preconditioner_converges_in_one_step():
    r = _rng(8)
    A = np.zeros((24, 24))
    blocks = [(k, 6) for k in range(0, 24, 6)]
    for off, m in blocks:
        A[off:off + m, off:off + m] = 3 * np.eye(m) + r.standard_normal((m, m))
    P = G.block_jacobi(A, blocks)
    b = r.standard_normal(24)
    x, info = G.gmres(A, b, P=P, tol=1e-12)
    assert info["iters"] == 1
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_iteration_count_matches_library_gmres():
    # an MRCM interface system with block-Jacobi, against scipy's GMRES on
    # the same explicitly preconditioned operator
    spla = pytest.importorskip("scipy.sparse.linalg")
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config5(3, n=64)
    out = O.mrcm_solve(prob, return_system=True)
    S = out["systems"][0]
    M, f = S["M"], S["rhs"]
    P = G.block_jacobi(M, G.diagonal_blocks(S["layout"].ifaces))
    _, info = G.gmres(M @ P, f, restart=20, tol=1e-8)
    cnt = [0]
    spla.gmres(M @ P, f, rtol=1e-8, atol=0.0, restart=20, maxiter=200,
               callback=lambda _: cnt.__setitem__(0, cnt[0] + 1), callback_type="pr_norm")
    assert info["converged"]
    assert abs(info["iters"] - cnt[0]) <= 2, (info["iters"], cnt[0])


def test_stall_rule():
    # a Jordan-like shift operator makes GMRES stagnate for n - 1 steps
    n = 40
    A = np.roll(np.eye(n), 1, axis=0)
    b = np.zeros(n)
    b[0] = 1.0
    _, info = G.gmres(A, b, restart=n, tol=1e-12, stall_window=10)
    assert info["stalled"] and not info["converged"]
    assert info["iters"] == 11


def test_planted_rotation_sign_is_caught(monkeypatch):
    good = G.givens
    monkeypatch.setattr(G, "givens", lambda a, b: (good(a, b)[0], -good(a, b)[1]))
    A = _nonsym(50, 4)
    b = _rng(5).standard_normal(50)
    x, info = G.gmres(A, b, restart=50, tol=1e-13, maxiter=200)
    ref = np.linalg.solve(A, b)
    assert not (info["converged"] and np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref))
