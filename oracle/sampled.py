"""Sampled checks of an MRCM solution at sizes the whole oracle cannot solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s accuracy and CPU-baseline legs may import this module.  It
uses the oracle's own building blocks (``mrcm_oracle``) and nothing of the
CUDA library.

Given an interface solution x (the unknowns of Eq. "mrc2" in the canonical
order), two things can be recomputed one at a time, in FP64:

* the local Robin problem (Eq. "mrc1") of one subdomain with the Robin data
  g = -beta sigma U_H + P_H that x defines: its pressures are what the
  reconstruction must return on that subdomain;
* on one interface, the two weak continuity conditions of Eq. "mrc2" --
  pressure continuity tested with each flux function phi_k, flux continuity
  tested with each pressure function psi_k -- from the two local solutions
  on either side.  Their defects are the interface system's residual rows,
  computed without the solver's own residual.

``global_balance`` is the discrete divergence theorem over the whole grid:
the sources equal the boundary outflow.
"""
from __future__ import annotations

import numpy as np

from . import mrcm_oracle as O


def local_solution(prob, r, lay, kappa, x, I, J):
    """Pressures [s, s] of subdomain (I, J) from the Robin data of x, and,
    per interface edge, the outward velocity and face pressure traces."""
    lo = O.Local(prob, r, lay, I, J, kappa)
    rhs = lo.b0.copy()
    data = {}
    for side, (g, sigma) in lo.edges.items():
        f = lay.ifaces[g]
        gd = O.robin_data(f, sigma, lo.beta[side], x)
        data[side] = gd
        rhs += lo.robin_rhs(side, gd)
    p = O.solve_local(lo.A, rhs[:, None], refine=True)[:, 0]
    s, h = lay.s, lay.h
    tr = {}
    for side, gd in data.items():
        pc = np.array([p[O.edge_face_cell(side, e, s)[1] * s + O.edge_face_cell(side, e, s)[0]]
                       for e in range(s)])
        u = lo.TR[side] * (pc - gd) / h + lo.wR[side]
        tr[side] = (u, gd + lo.beta[side] * u)       # Robin: -beta u + p_f = g
    return p.reshape(s, s), tr


def sampled_checks(prob, p, x, rng, n_sub=6, n_if=6, reals=None):
    """Largest relative pressure mismatch over sampled subdomains and largest
    relative continuity defect over sampled interfaces, for the realisations
    ``reals`` (all by default).  ``p`` is [R, ny, nx]; ``x`` the interface
    unknowns of every realisation, concatenated in canonical order."""
    reals = range(prob.n_real) if reals is None else reals
    starts, off = [], 0
    for r in range(prob.n_real):
        starts.append(off)
        off += int(np.sum(np.asarray(prob.iface_nU[r]) + np.asarray(prob.iface_nP[r])))
    worst_p = worst_d = 0.0
    for r in reals:
        lay = O.Layout(prob, r)
        s = lay.s
        kappa = prob.lam[r] * prob.K[r]
        xr = x[starts[r]:starts[r] + lay.n_unknowns]
        corners = [(0, 0), (lay.Sx - 1, 0), (0, lay.Sy - 1), (lay.Sx - 1, lay.Sy - 1),
                   (lay.Sx // 2, lay.Sy // 2)]
        subs = corners + [(int(rng.integers(lay.Sx)), int(rng.integers(lay.Sy)))
                          for _ in range(max(0, n_sub - len(corners)))]
        for I, J in subs:
            pl, _ = local_solution(prob, r, lay, kappa, xr, I, J)
            pg = p[r, J * s:(J + 1) * s, I * s:(I + 1) * s]
            e = np.linalg.norm(pg - pl) / max(np.linalg.norm(pl), 1e-300)
            worst_p = max(worst_p, e)
        if not lay.ifaces:
            continue
        for g in rng.choice(len(lay.ifaces), size=min(n_if, len(lay.ifaces)), replace=False):
            f = lay.ifaces[int(g)]
            Ls, Rs = ("E", "W") if f["kind"] == "V" else ("N", "S")
            _, trL = local_solution(prob, r, lay, kappa, xr, *f["L"])
            _, trR = local_solution(prob, r, lay, kappa, xr, *f["R"])
            (uL, pfL), (uR, pfR) = trL[Ls], trR[Rs]
            h = lay.h
            for k in range(f["nU"]):          # pressure continuity, tested by phi_k
                d = h * np.dot(f["phi"][k], pfL - pfR)
                sc = h * np.dot(np.abs(f["phi"][k]), np.abs(pfL) + np.abs(pfR))
                worst_d = max(worst_d, abs(d) / max(sc, 1e-300))
            for k in range(f["nP"]):          # flux continuity, tested by psi_k
                d = h * np.dot(f["psi"][k], uL + uR)
                sc = h * np.dot(np.abs(f["psi"][k]), np.abs(uL) + np.abs(uR))
                worst_d = max(worst_d, abs(d) / max(sc, 1e-300))
    return worst_p, worst_d


def global_balance(prob, ux, uy):
    """max over realisations |sum q h^2 - boundary outflow| relative to the
    sources, or to the boundary inflow when there are none."""
    h = prob.h
    worst = 0.0
    for r in range(prob.n_real):
        src = float(prob.q[r].sum()) * h * h
        out = (ux[r][:, -1].sum() - ux[r][:, 0].sum() + uy[r][-1, :].sum() - uy[r][0, :].sum()) * h
        scale = max(abs(src), float(np.abs(ux[r][:, 0]).sum() * h), 1e-300)
        worst = max(worst, abs(src - out) / scale)
    return worst
