"""Plain FP64 restarted GMRES with right preconditioning, and the block
preconditioners of the MRCM interface system.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  It shares no code with
the CUDA library.

The paper does not say how the interface system (Section 3, Eq. "mrc2") is
solved.  For systems too large for a direct solve this module is the
textbook method, written out step by step:

* GMRES (Saad and Schultz, SIAM J. Sci. Stat. Comput. 7, 1986) with right
  preconditioning (Saad, "Iterative Methods for Sparse Linear Systems",
  2nd ed., Section 9.3.2): solve A P y = b, return x = P y;
* the Arnoldi basis by modified Gram-Schmidt, the small least-squares
  problem by Givens rotations, restart after ``restart`` steps;
* stopping when the TRUE relative residual ||b - A x|| / ||b|| is at most
  ``tol`` (the rotated right-hand side only decides when to look);
* block-Jacobi: P = blockdiag(A_gg^-1) over the interfaces g (each block is
  the m x m coupling of one interface's unknowns with themselves).

An optional stall rule stops the solve when the residual estimate fell by
less than ``stall_factor`` over the last ``stall_window`` iterations; the
GPU path uses the same rule to leave a learned preconditioner for
block-Jacobi.

Pinned by ``tests/test_oracle_gmres.py``: convergence in at most d steps for
a matrix with d distinct eigenvalues, the closed-form first step, agreement
with a direct solve, monotone residuals, one-step convergence with an exact
block-diagonal preconditioner, iteration counts of an independent library
GMRES on the same operator, and a planted mistake.
"""
from __future__ import annotations

import numpy as np


def _apply(A, v):
    return A(v) if callable(A) else A @ v


def givens(a, b):
    """Rotation (c, s) with [c s; -s c] [a; b] = [r; 0], r = hypot(a, b)."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(A, b, P=None, restart=40, tol=1e-10, maxiter=5000, stall_window=0,
          stall_factor=0.9):
    """Restarted right-preconditioned GMRES.

    A, P: matrices or callables (P = None: identity).  Returns (x, info) with
    info = dict(iters, resid (true relative residual), converged, stalled,
    history (residual estimate relative to ||b|| after every iteration)).
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    info = dict(iters=0, resid=0.0, converged=True, stalled=False, history=[])
    if bnorm == 0.0:
        return np.zeros(n), info
    Pm = (lambda v: v) if P is None else (lambda v: _apply(P, v))
    y = np.zeros(n)                      # iterate of the preconditioned system
    it = 0
    hist = info["history"]
    while True:
        r = b - _apply(A, Pm(y))
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        info["resid"] = rel
        if rel <= tol or it >= maxiter or info["stalled"]:
            break
        k = restart
        V = np.zeros((k + 1, n))
        H = np.zeros((k + 1, k))
        cs, sn = np.zeros(k), np.zeros(k)
        g = np.zeros(k + 1)
        g[0] = beta
        V[0] = r / beta
        j = 0
        while j < k:
            w = _apply(A, Pm(V[j]))
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                          # earlier rotations
                hi, hk = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hk
                H[i + 1, j] = -sn[i] * hi + cs[i] * hk
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            hnext = H[j + 1, j]
            H[j + 1, j] = 0.0
            j += 1
            it += 1
            est = abs(g[j]) / bnorm
            hist.append(est)
            if stall_window and it > stall_window and est > stall_factor * hist[-1 - stall_window]:
                info["stalled"] = True
            if est <= tol or it >= maxiter or info["stalled"] or hnext == 0.0:
                break
            V[j] = w / hnext
        # least squares: R z = g on the first j rows
        z = np.zeros(j)
        for i in range(j - 1, -1, -1):
            z[i] = (g[i] - np.dot(H[i, i + 1:j], z[i + 1:j])) / H[i, i]
        y = y + V[:j].T @ z
    info["iters"] = it
    info["converged"] = info["resid"] <= tol
    return Pm(y), info


def diagonal_blocks(blocks):
    """(offset, size) of every interface's unknowns from an oracle layout's
    interface list (``Layout.ifaces``)."""
    return [(f["off"], f["nU"] + f["nP"]) for f in blocks]


def block_jacobi(A, blocks):
    """Dense block-diagonal P with P_gg = A_gg^{-1} on every (offset, size)."""
    P = np.zeros_like(A)
    for off, m in blocks:
        sl = slice(off, off + m)
        P[sl, sl] = np.linalg.inv(A[sl, sl])
    return P
