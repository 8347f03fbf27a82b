"""Plain FP64 CPU oracle of the implicit saturation transport (Section 4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s accuracy and CPU-baseline legs may import this module.  It
shares no code with the CUDA library.

One implicit Euler step of the transport equation (Eq. "BL2D") with the
velocity frozen at u^n (Eq. "BL2D_Newton"), discretised by finite volumes
with first-order upwind fluxes (Eqs. "fluxes_impli", "up_fluxes_impli"):

    H_I(s) = s_I - s_I^n + (dt / V_I) F_I(s) = 0              (Eq. "BL2D_Newton7")

F_I is the net outflow of cell I: over each face, the face length times the
outward normal velocity times f at the upwind side -- the cell itself when
the flow leaves it, the neighbour when it enters, and the injection
saturation s_in at an inlet boundary face.  The fractional flow with
quadratic relative permeabilities (Section 5) is f(s) = M s^2 / (M s^2 +
(1 - s)^2), M = mu_o / mu_w.

Newton's method (Eq. "BL2D_Newton8") solves H' d = -H with the exact
Jacobian of the upwind scheme (a sparse linear solve, scipy's LU as the
library primitive), and the inflection-point trust region of Section 4.1
guards each update: the new value is kept in [0, 1], and a cell whose new
value lies on the other side of the inflection point of f than its old
value (f''(new) f''(old) < 0) takes the average of the two.  The loop stops
when the update is small: ||s^{nu+1} - s^nu|| <= eta.

Readings of points the paper leaves open (the CUDA path follows the same):
* the norm of the stopping test is the discrete L2 norm of the update over
  the cells, sqrt(sum_I d_I^2 |V_I|) (area-weighted; |V_I| = h^2), and the
  update tested is the one actually taken (after halving and clipping);
* the paper states the [0, 1] constraint and the halving without an order:
  the new value is clipped first and the crossing test is made on the
  clipped value (the test on an unclipped value far outside [0, 1], where
  the formula of f'' has no meaning, lets a cell at 0 jump to 1 and back
  for ever); the halving is applied once per cell and iteration;
* inlet boundary faces (normal velocity into the domain) carry f(s_in) with
  s_in = 1 (water injection, "the domain is initially filled with oil, with
  water being injected"); faces with zero normal velocity carry nothing;
* the velocities on the subdomain interfaces are the single-valued face
  velocities the Darcy solve reports (the mean of the two one-sided values).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------- flux function
def frac_flow(s, M):
    """f(s) = M s^2 / (M s^2 + (1 - s)^2) (Section 5)."""
    s = np.asarray(s, np.float64)
    a, b = M * s * s, (1.0 - s) ** 2
    return a / (a + b)


def frac_flow_d1(s, M):
    """f'(s) = 2 M s (1 - s) / (M s^2 + (1 - s)^2)^2 (quotient rule)."""
    s = np.asarray(s, np.float64)
    den = M * s * s + (1.0 - s) ** 2
    return 2.0 * M * s * (1.0 - s) / (den * den)


def frac_flow_d2(s, M):
    """f''(s): with g = 2 M s (1 - s) and q = (M s^2 + (1 - s)^2)^2,
    f'' = (g' q - g q') / q^2, g' = 2 M (1 - 2 s),
    q' = 2 (M s^2 + (1 - s)^2) (2 M s - 2 (1 - s))."""
    s = np.asarray(s, np.float64)
    den = M * s * s + (1.0 - s) ** 2
    g = 2.0 * M * s * (1.0 - s)
    gp = 2.0 * M * (1.0 - 2.0 * s)
    denp = 2.0 * M * s - 2.0 * (1.0 - s)
    return (gp * den - 2.0 * g * denp) / den ** 3


def inflection_point(M):
    """The s in (0, 1) with f''(s) = 0, by bisection (f'' > 0 at 0, < 0 at 1)."""
    lo, hi = 1e-12, 1.0 - 1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if frac_flow_d2(mid, M) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# --------------------------------------------------------------- residual, Jacobian
def _face_velocities(ux, uy):
    """Outward normal velocity of each cell through its W, E, S, N faces."""
    ux = np.asarray(ux, np.float64)
    uy = np.asarray(uy, np.float64)
    return (-ux[:, :-1], ux[:, 1:], -uy[:-1, :], uy[1:, :])


def residual(s, s_old, ux, uy, h, dt, M, s_in=1.0):
    """H(s) of Eq. "BL2D_Newton7" on the [ny, nx] grid (V = h^2, faces h)."""
    ny, nx = s.shape
    f = frac_flow(s, M)
    f_in = float(frac_flow(s_in, M))
    out = np.zeros((ny, nx))
    uW, uE, uS, uN = _face_velocities(ux, uy)
    # neighbour f through each face; the inlet value outside the domain
    fW = np.empty_like(f)
    fW[:, 1:] = f[:, :-1]
    fW[:, 0] = f_in
    fE = np.empty_like(f)
    fE[:, :-1] = f[:, 1:]
    fE[:, -1] = f_in
    fS = np.empty_like(f)
    fS[1:, :] = f[:-1, :]
    fS[0, :] = f_in
    fN = np.empty_like(f)
    fN[:-1, :] = f[1:, :]
    fN[-1, :] = f_in
    for un, fn in ((uW, fW), (uE, fE), (uS, fS), (uN, fN)):
        out += np.where(un > 0.0, un * f, un * fn) * h
    return s - s_old + dt / (h * h) * out


def jacobian(s, ux, uy, h, dt, M):
    """dH/ds of the upwind scheme, sparse [n, n] (cells row-major)."""
    ny, nx = s.shape
    n = nx * ny
    d1 = frac_flow_d1(s, M)
    c = dt / h
    uW, uE, uS, uN = _face_velocities(ux, uy)
    diag = np.ones((ny, nx))
    rows, cols, vals = [], [], []
    idx = np.arange(n).reshape(ny, nx)
    for un, di, dj in ((uW, -1, 0), (uE, 1, 0), (uS, 0, -1), (uN, 0, 1)):
        diag += c * np.where(un > 0.0, un, 0.0) * d1
        # inflow from an interior neighbour: dH_I / ds_J = c u_out f'(s_J)
        jj, ii = np.nonzero(un <= 0.0)
        nj, ni = jj + dj, ii + di
        ok = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny)
        jj, ii, nj, ni = jj[ok], ii[ok], nj[ok], ni[ok]
        v = c * un[jj, ii] * d1[nj, ni]
        nz = v != 0.0
        rows.append(idx[jj, ii][nz])
        cols.append(idx[nj, ni][nz])
        vals.append(v[nz])
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


# --------------------------------------------------------------- Newton
def newton_step(s_old, ux, uy, h, dt, M, eta=1e-6, max_iter=100, s_in=1.0,
                trust_region=True, s0=None):
    """One implicit transport step from s_old: returns (s_new, iterations,
    list of update norms).  ``trust_region=False`` gives plain Newton with
    the clip only (for comparison)."""
    s = np.array(s_old if s0 is None else s0, np.float64, copy=True)
    norms = []
    for it in range(1, max_iter + 1):
        H = residual(s, s_old, ux, uy, h, dt, M, s_in)
        J = jacobian(s, ux, uy, h, dt, M)
        d = spla.spsolve(J.tocsc(), -H.ravel()).reshape(s.shape)
        new = np.clip(s + d, 0.0, 1.0)
        if trust_region:
            cross = (frac_flow_d2(new, M) * frac_flow_d2(s, M)) < 0.0
            new = np.where(cross, 0.5 * (new + s), new)
        nrm = float(np.sqrt(np.sum((new - s) ** 2) * h * h))
        norms.append(nrm)
        s = new
        if nrm <= eta:
            return s, it, norms
    return s, max_iter, norms


def boundary_outflow(s, ux, uy, h, M, s_in=1.0):
    """Net water outflow through the domain boundary per unit time:
    sum over boundary faces of h u_out f(upwind)."""
    f = frac_flow(s, M)
    f_in = float(frac_flow(s_in, M))
    ux = np.asarray(ux)
    uy = np.asarray(uy)
    tot = 0.0
    for un, fc in ((-ux[:, 0], f[:, 0]), (ux[:, -1], f[:, -1]), (-uy[0, :], f[0, :]),
                   (uy[-1, :], f[-1, :])):
        tot += float(np.sum(np.where(un > 0.0, un * fc, un * f_in))) * h
    return tot


# --------------------------------------------------------------- 1-D brute force
def march_1d(s_old, u, h, dt, M, s_in=1.0):
    """The implicit upwind step on one row of cells with a uniform velocity
    u > 0 (left to right): cell i depends only on itself and cell i-1, so
    the step is solved cell by cell, each a scalar equation
    s - s_old + (dt/h) u (f(s) - f_up) = 0, increasing in s, by bisection to
    the last bit.  An algorithm independent of Newton's."""
    c = dt / h * u

    def fs(x):                      # f of one value, in plain floats
        a = M * x * x
        return a / (a + (1.0 - x) * (1.0 - x))

    out = np.empty_like(np.asarray(s_old, np.float64))
    f_up = fs(float(s_in))
    for i, so in enumerate(np.asarray(s_old, np.float64).tolist()):
        lo, hi = 0.0, 1.0
        g = lambda x: x - so + c * (fs(x) - f_up)
        if g(lo) >= 0.0:
            x = lo
        elif g(hi) <= 0.0:
            x = hi
        else:
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if g(mid) > 0.0:
                    hi = mid
                else:
                    lo = mid
                if hi - lo <= 1e-17:
                    break
            x = 0.5 * (lo + hi)
        out[i] = x
        f_up = fs(x)
    return out


# --------------------------------------------------------------- SI / SFI
def si_step(prob, s_old, dt, M, darcy, eta=1e-6, max_iter=100, s_in=1.0):
    """One sequential implicit step (Section 4): the Darcy solve with the
    mobility of s_old (``darcy(prob, s)`` returns p, ux, uy for one
    realisation), then the implicit transport with those velocities."""
    p, ux, uy = darcy(prob, s_old)
    s_new, it, _ = newton_step(s_old, ux, uy, prob.h, dt, M, eta, max_iter, s_in)
    return s_new, it, (p, ux, uy)


def sfi_step(prob, s_old, dt, M, darcy, tol=1e-4, max_outer=20, eta=1e-6, max_iter=100,
             s_in=1.0):
    """One sequential fully implicit step (Section 5.4): repeat the Darcy
    solve with the mobility of the latest saturation iterate and the
    transport step from s_old with its velocities, until the largest change
    of the saturation between outer iterations is below tol."""
    s_k = np.array(s_old, np.float64, copy=True)
    newton_its = []
    for k in range(1, max_outer + 1):
        p, ux, uy = darcy(prob, s_k)
        s_new, it, _ = newton_step(s_old, ux, uy, prob.h, dt, M, eta, max_iter, s_in)
        newton_its.append(it)
        change = float(np.max(np.abs(s_new - s_k)))
        s_k = s_new
        if change < tol:
            return s_k, k, newton_its, (p, ux, uy)
    return s_k, max_outer, newton_its, (p, ux, uy)
