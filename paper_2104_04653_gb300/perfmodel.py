"""Algorithmic work of each hot-path call, for roofline reporting.

Counts are the method's own work on the layout the kernels use (block
tridiagonal local operators with explicit s x s Schur-block inverses, the
interface matrix by slabs), not the instructions a kernel happens to issue.
"""
from __future__ import annotations

import os

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


def _sizes_and_cols(prob):
    """(subdomain edge s, basis columns) of every subdomain of the batch."""
    out = []
    for r in range(prob.n_real):
        s = prob.sub_size[r]
        out += [(s, c) for c in _ncols(prob, r)]
    return out


def call_work(call: str, prob, solver=None) -> dict:
    subs = _sizes_and_cols(prob)
    R = prob.n_real
    info = solver.mrcm_get_info(check=False) if solver is not None else {}
    sweeps = 1 + int(info.get("local_sweeps_max", 0) or 0)
    if call == "factor_local":
        flops = sum(2.0 * s ** 4 for s, _ in subs)    # s Gauss-Jordan inverses of s x s blocks
        byts = sum(s * s * (16 + 48) + s ** 3 * 4 for s, _ in subs)
        sizes = sorted({sz for sz, _ in subs})
        kern = " + ".join({16: "k_factor", 32: "k_factor_warp"}[sz] for sz in sizes)
        return {"kernel": kern, "bound": "alu", "flops": flops, "bytes": float(byts),
                "per_unit": "2 s^4 flop per subdomain (s block inverses of s^3 FMA)"}
    if call == "build_basis":
        # 2s-1 block steps of an s x s matvec per column and sweep
        flops = sum(sweeps * 2.0 * (2 * s - 1) * s * s * c for s, c in subs)
        byts = sum(c * s * s * 8 + s ** 3 * 4 + 6 * s * s * 8 for s, c in subs)
        sizes = sorted({sz for sz, _ in subs})
        kern = " + ".join({16: "k_basis", 32: "k_basis32"}[sz] for sz in sizes)
        return {"kernel": kern, "bound": "alu", "flops": flops, "bytes": float(byts),
                "sweeps": sweeps,
                "per_unit": "(1 + refinement sweeps) x 2 (2s-1) s^2 flop per basis column"}
    if call == "solve_interface":
        # block cyclic reduction over slabs (one column of subdomains each)
        # plus the refinement sweeps, counted on the method's own layout
        tot_f32 = tot_f64 = 0.0
        inv_f32 = gemm_f32 = solve_f32 = 0.0
        sweeps = 1 + int(info.get("iface_sweeps", 0) or 0)
        for r in range(R):
            s_ = prob.sub_size[r]
            sx, sy = prob.nx // s_, prob.ny // s_
            m = np.asarray(prob.iface_nU[r]) + np.asarray(prob.iface_nP[r])
            nV = (sx - 1) * sy
            xdir = sx >= sy
            K = sx if xdir else sy
            sizes = []
            for k in range(K):
                if xdir:
                    ids = [nV + J * sx + k for J in range(sy - 1)]
                    ids += [J * (sx - 1) + k for J in range(sy)] if k < sx - 1 else []
                else:
                    ids = [k * (sx - 1) + I for I in range(sx - 1)]
                    ids += [nV + k * sx + I for I in range(sx)] if k < sy - 1 else []
                sizes.append(int(sum(m[i] for i in ids)))
            b = max(sizes) if sizes else 0
            lev, st = 0, 1
            while st < K:
                surv = list(range(0, K, 2 * st))
                odd = list(range(st, K, 2 * st))
                inv_f32 += len(odd) * 2.0 * b ** 3                   # Gauss-Jordan inverses
                for k in surv:
                    if k - st >= 0:
                        gemm_f32 += 3 * 2.0 * b ** 3                  # X, X C_l, X A_l
                    if k + st < K:
                        gemm_f32 += 3 * 2.0 * b ** 3                  # Y, Y A_r, Y C_r
                st *= 2
                lev += 1
            inv_f32 += 2.0 * b ** 3                                   # root inverse
            # refinement: FP64 residual rows (2 flops per term) and the solve
            cols = _ncols(prob, r)
            terms = 0                     # FP64 terms of all interface rows
            for g in range(len(m)):
                if g < nV:
                    J, I = divmod(g, sx - 1)
                    L, Rr = J * sx + I, J * sx + I + 1
                else:
                    J, I = divmod(g - nV, sx)
                    L, Rr = J * sx + I, (J + 1) * sx + I
                terms += int(m[g]) * (cols[L] - 1 + cols[Rr] - 1)
            solve = 2.0 * b * b * (4 * (K - 1) + 1)
            tot_f64 += sweeps * 2.0 * terms
            solve_f32 += max(sweeps - 1, 0) * solve
        tot_f32 = inv_f32 + gemm_f32 + solve_f32
        path = solver.interface_path() if solver is not None else "cluster"
        kern = {"cluster": "k_iface_cluster", "slab": "k_bcr_level + k_iface_solve",
                "wide-slab": "k_gj_* + k_tc_gemm_split + k_big_solve", "gmres": "k_gmres",
                "none": "-"}[path]
        # the wide-slab path's block products run on the tensor cores (FP32
        # path, 3 x TF32); its inverses, solves and residuals on SIMT pipes
        prec = getattr(getattr(solver, "desc", None), "prec", 1) if solver is not None else 1
        tc = path == "wide-slab" and prec == 1 and not os.environ.get("MRCM_NO_TENSOR_CORES")
        return {"kernel": kern, "bound": "tensor" if tc else "alu", "flops": tot_f32 + tot_f64,
                "flops_fp32": tot_f32, "flops_fp64": tot_f64,
                "flops_inverse": inv_f32, "flops_products": gemm_f32, "flops_solve": solve_f32,
                "bytes": float(sum(int(np.sum(np.asarray(prob.iface_nU[r]) +
                                              np.asarray(prob.iface_nP[r]))) for r in range(R)) * 8),
                "per_unit": "per level: 2 b^3 per eliminated slab (inverse) + 6 b^3 x2 per "
                            "surviving slab (three GEMMs per side); per sweep 2 flop per FP64 "
                            "residual term and 2 b^2 per slab matvec"}
    if call == "reconstruct":
        byts = sum(c * s * s * 8 for s, c in subs) + prob.cells() * 8 * 3
        return {"kernel": "k_recon_cells", "bound": "hbm", "flops": 0.0, "bytes": float(byts),
                "per_unit": "basis columns read once (8 B per column per cell) + p, ux, uy"}
    raise ValueError(call)


def survey_work(prob, solver=None) -> dict:
    """The method's work per solve counted as the scope table of the build
    counts it (banded work, not the dense blocks the kernels use): factor
    n s^2 = s^4 flop per subdomain; solve 4 n s flop per right-hand side and
    sweep (a forward and a backward banded substitution); 40 B per cell of
    HBM traffic for the whole path (K and lambda in, p, ux and uy out);
    7 m^2 x 12 B per interface for one interface SpMV (block-sparse, at most
    seven m x m blocks per block row: 8 B value + 4 B index)."""
    info = solver.mrcm_get_info(check=False) if solver is not None else {}
    sweeps = 1 + int(info.get("local_sweeps_max", 0) or 0)
    subs = _sizes_and_cols(prob)
    factor = sum(float(s) ** 4 for s, _ in subs)
    solve = sum(sweeps * 4.0 * s * s * s * c for s, c in subs)
    spmv = 0.0
    for r in range(prob.n_real):
        m = np.asarray(prob.iface_nU[r]) + np.asarray(prob.iface_nP[r])
        spmv += float(np.sum(7.0 * m.astype(np.float64) ** 2 * 12.0))
    return {"factor_flops": factor, "solve_flops": solve, "flops": factor + solve,
            "path_bytes": 40.0 * prob.cells(), "iface_spmv_bytes": spmv, "sweeps": sweeps,
            "per_unit": "factor s^4 per subdomain; solve 4 n s per RHS per sweep; 40 B per cell; "
                        "7 m^2 x 12 B per interface per SpMV"}
