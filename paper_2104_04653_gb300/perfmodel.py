"""Algorithmic work of each hot-path call, for roofline reporting.

Counts are the method's own work on the layout the kernels use (block
tridiagonal local operators with explicit s x s Schur-block inverses, the
interface matrix by slabs), not the instructions a kernel happens to issue.
"""
from __future__ import annotations

import numpy as np


def _ncols(prob, r=0):
    s = prob.sub_size[r]
    sx, sy = prob.nx // s, prob.ny // s
    nV = (sx - 1) * sy
    m = np.asarray(prob.iface_nU[r]) + np.asarray(prob.iface_nP[r])
    cols = []
    for J in range(sy):
        for I in range(sx):
            c = 1
            if I > 0:
                c += m[J * (sx - 1) + I - 1]
            if I < sx - 1:
                c += m[J * (sx - 1) + I]
            if J > 0:
                c += m[nV + (J - 1) * sx + I]
            if J < sy - 1:
                c += m[nV + J * sx + I]
            cols.append(int(c))
    return cols


def call_work(call: str, prob, solver=None) -> dict:
    s = prob.sub_size[0]
    n = s * s
    R = prob.n_real
    cols = [c for r in range(R) for c in _ncols(prob, r)]
    nsub = len(cols)
    info = solver.mrcm_get_info(check=False) if solver is not None else {}
    sweeps = 1 + int(info.get("local_sweeps_max", 0) or 0)
    if call == "factor_local":
        flops = 2.0 * nsub * s ** 4            # s Gauss-Jordan inverses of s x s blocks
        byts = nsub * n * (16 + 48) + nsub * s ** 3 * 4
        return {"kernel": "k_factor", "bound": "alu", "flops": flops, "bytes": byts,
                "per_unit": "2 s^4 flop per subdomain (s block inverses of s^3 FMA)"}
    if call == "build_basis":
        solve = 2.0 * (2 * s - 1) * s * s      # 2s-1 block steps of an s x s matvec
        flops = sweeps * solve * sum(cols)
        byts = sum(c * n * 8 for c in cols) + nsub * (s ** 3 * 4 + 6 * n * 8)
        return {"kernel": "k_basis", "bound": "alu", "flops": flops, "bytes": byts,
                "sweeps": sweeps,
                "per_unit": "(1 + refinement sweeps) x 2 (2s-1) s^2 flop per basis column"}
    if call == "solve_interface":
        m = sum(int(np.sum(np.asarray(prob.iface_nU[r]) + np.asarray(prob.iface_nP[r])))
                for r in range(R))
        return {"kernel": "k_bcr_update/k_iface_solve", "bound": "alu",
                "flops": 0.0, "bytes": float(m * 8), "per_unit": "see DESIGN.md"}
    if call == "reconstruct":
        byts = sum(c * n * 8 for c in cols) + prob.cells() * 8 * 3
        return {"kernel": "k_recon_cells", "bound": "hbm", "flops": 0.0, "bytes": float(byts),
                "per_unit": "basis columns read once (8 B per column per cell) + p, ux, uy"}
    raise ValueError(call)
