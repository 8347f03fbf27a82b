"""Plain FP64 CPU oracle of MRCM on a quadtree decomposition: subdomains of
two sizes inside one realisation, with interfaces that cover half of a large
subdomain's edge (non-conforming in the subdomain sense).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s accuracy and CPU-baseline legs may import this module.  It
uses the coefficient helpers of ``mrcm_oracle`` and shares no code with the
CUDA library.

Layout (the paper's Section 3 allows any non-overlapping decomposition; the
quadtree is the workload's reading).  Realisation r is covered by blocks of
B x B cells (B = prob.sub_size[r]); a block whose entry of prob.refine[r]
([ny/B][nx/B]) is nonzero is split into four (B/2) x (B/2) subdomains.
Subdomains are numbered by (y0, x0).  An interface is a maximal run of grid
faces shared by the same two subdomains: B or B/2 faces long.  Vertical
interfaces (normal +x) come first, ordered by (y0, x), then horizontal ones
(normal +y) by (y, x0); "L" is the subdomain on the -x / -y side.  On a
layout without refinement this is the order, numbering and normal of the
uniform oracle.

Readings (the same in the CUDA path):
* the fixed normal of every interface is +x or +y (the left or lower
  subdomain is "L"), as on uniform layouts; with two sizes the lower-index
  subdomain may lie on either side, and any fixed orientation gives the same
  solution (U_H changes sign);
* H of beta = alpha H / kappa (Eq. "beta") is the length of the interface the
  face belongs to (B h or B h / 2), so beta is the same on both sides of an
  interface and equals the uniform reading H = s h without refinement;
* interface functions are sampled at the midpoints of the interface's own
  faces (t in [-1, 1] along it).

Everything else follows ``mrcm_oracle``: the local Robin problems
(Eq. "mrc1"), one local solve per interface function plus the particular
one, the interface system (Eq. "mrc2") solved densely, the combination.
Pure-Neumann problems and gravity are not covered here.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mrcm_oracle as O


class QLayout:
    """Subdomains and interface segments of one realisation."""

    def __init__(self, prob, r):
        nx, ny = prob.nx, prob.ny
        B = prob.sub_size[r]
        ref = np.zeros((ny // B, nx // B), bool) if getattr(prob, "refine", None) is None \
            else np.asarray(prob.refine[r], bool).reshape(ny // B, nx // B)
        if B % 2 or nx % B or ny % B:
            raise ValueError("grid not divisible into blocks")
        subs = []
        for BJ in range(ny // B):
            for BI in range(nx // B):
                if ref[BJ, BI]:
                    h2 = B // 2
                    for j in range(2):
                        for i in range(2):
                            subs.append((BI * B + i * h2, BJ * B + j * h2, h2))
                else:
                    subs.append((BI * B, BJ * B, B))
        subs.sort(key=lambda t: (t[1], t[0]))
        self.subs = subs
        self.h = prob.h
        owner = np.full((ny, nx), -1)
        for k, (x0, y0, s) in enumerate(subs):
            owner[y0:y0 + s, x0:x0 + s] = k
        self.owner = owner
        vert, horiz = [], []
        for x in range(1, nx):
            y = 0
            while y < ny:
                L, R = owner[y, x - 1], owner[y, x]
                if L == R:
                    y += 1
                    continue
                y1 = y
                while y1 < ny and owner[y1, x - 1] == L and owner[y1, x] == R:
                    y1 += 1
                vert.append(dict(kind="V", x=x, y0=y, len=y1 - y, L=int(L), R=int(R)))
                y = y1
        for y in range(1, ny):
            x = 0
            while x < nx:
                L, R = owner[y - 1, x], owner[y, x]
                if L == R:
                    x += 1
                    continue
                x1 = x
                while x1 < nx and owner[y - 1, x1] == L and owner[y, x1] == R:
                    x1 += 1
                horiz.append(dict(kind="H", y=y, x0=x, len=x1 - x, L=int(L), R=int(R)))
                x = x1
        vert.sort(key=lambda f: (f["y0"], f["x"]))
        horiz.sort(key=lambda f: (f["y"], f["x0"]))
        self.ifaces = vert + horiz
        nU, nP = prob.iface_nU[r], prob.iface_nP[r]
        if len(nU) != len(self.ifaces):
            raise ValueError(f"{len(self.ifaces)} interfaces, {len(nU)} sizes given")
        off = 0
        for g, f in enumerate(self.ifaces):
            Lg = f["len"]
            f["nU"], f["nP"] = int(nU[g]), int(nP[g])
            f["off"] = off
            off += f["nU"] + f["nP"]
            if getattr(prob, "iface_fn", None) is None:
                f["phi"] = O.interface_functions(f["nU"], Lg, prob.basis)
                f["psi"] = O.interface_functions(f["nP"], Lg, prob.basis)
            else:
                phi, psi = prob.iface_fn[r][g]
                f["phi"] = np.asarray(phi, np.float64).reshape(f["nU"], Lg)
                f["psi"] = np.asarray(psi, np.float64).reshape(f["nP"], Lg)
            f["alpha"] = (np.ones(Lg) if prob.alpha is None
                          else np.asarray(prob.alpha[r][g], np.float64).reshape(Lg))
        self.n_unknowns = off
        # face -> (interface, face index along it, side of the interface)
        self.face_if = {}
        for g, f in enumerate(self.ifaces):
            for e in range(f["len"]):
                if f["kind"] == "V":
                    self.face_if[("V", f["x"], f["y0"] + e)] = (g, e)
                else:
                    self.face_if[("H", f["y"], f["x0"] + e)] = (g, e)


class QLocal:
    """The local Robin problem (Eq. "mrc1") of subdomain k."""

    def __init__(self, prob, r, lay, k, kappa):
        x0, y0, s = lay.subs[k]
        h = lay.h
        self.s, self.x0, self.y0, self.n = s, x0, y0, s * s
        n = s * s
        A = np.zeros((n, n))
        b0 = np.zeros(n)
        kap = kappa[y0:y0 + s, x0:x0 + s]
        self.kap = kap
        # per side: per face (interface g, index along it, sigma) or None
        self.faces = {}
        for side in ("W", "E", "S", "N"):
            lst = []
            for e in range(s):
                if side == "W":
                    key = ("V", x0, y0 + e)
                elif side == "E":
                    key = ("V", x0 + s, y0 + e)
                elif side == "S":
                    key = ("H", y0, x0 + e)
                else:
                    key = ("H", y0 + s, x0 + e)
                ge = lay.face_if.get(key)
                if ge is None:
                    lst.append(None)
                else:
                    sigma = 1.0 if side in ("E", "N") else -1.0
                    lst.append((ge[0], ge[1], sigma))
            self.faces[side] = lst
        self.TR, self.beta = {}, {}
        for side, lst in self.faces.items():
            TR = np.zeros(s)
            be = np.zeros(s)
            for e, fe in enumerate(lst):
                if fe is None:
                    continue
                a, b = O.edge_face_cell(side, e, s)
                kc = kap[b, a]
                f = lay.ifaces[fe[0]]
                H = f["len"] * h
                al = f["alpha"][fe[1]]
                TR[e] = O.robin_T(kc, al, H, h)
                be[e] = al * H / kc
            self.TR[side], self.beta[side] = TR, be
        for b in range(s):
            for a in range(s):
                c = b * s + a
                kc = kap[b, a]
                gi, gj = x0 + a, y0 + b
                b0[c] += prob.q[r, gj, gi] * h * h
                for side, da, db in (("W", -1, 0), ("E", 1, 0), ("S", 0, -1), ("N", 0, 1)):
                    aa, bb = a + da, b + db
                    if 0 <= aa < s and 0 <= bb < s:
                        T = O.harmonic_T(kc, kap[bb, aa])
                        A[c, c] += T
                        A[c, bb * s + aa] -= T
                        continue
                    e = b if side in ("W", "E") else a
                    if self.faces[side][e] is not None:      # Robin face on Gamma
                        A[c, c] += self.TR[side][e]
                    else:                                     # physical boundary
                        kk = O.boundary_face(prob, side, gi, gj)
                        if prob.bc_type[kk] == O.DIRICHLET:
                            A[c, c] += 2.0 * kc
                            b0[c] += 2.0 * kc * prob.bc_val[kk]
                        else:
                            b0[c] -= prob.bc_val[kk] * h
        self.A, self.b0 = A, b0

    def robin_rhs(self, gdata):
        """RHS of Robin data gdata[side][e] (zero where not given)."""
        s = self.s
        b = np.zeros(self.n)
        for side, gd in gdata.items():
            for e in range(s):
                if gd[e] != 0.0:
                    a, bb = O.edge_face_cell(side, e, s)
                    b[bb * s + a] += self.TR[side][e] * gd[e]
        return b

    def data_of(self, lay, g, col_fn):
        """Robin data on this subdomain's faces of interface g for one
        function: col_fn = ("U", k) -> -beta sigma phi_k, ("P", k) -> psi_k."""
        s = self.s
        out = {}
        f = lay.ifaces[g]
        for side, lst in self.faces.items():
            gd = np.zeros(s)
            hit = False
            for e, fe in enumerate(lst):
                if fe is None or fe[0] != g:
                    continue
                hit = True
                kind, k = col_fn
                if kind == "U":
                    gd[e] = -self.beta[side][e] * fe[2] * f["phi"][k][fe[1]]
                else:
                    gd[e] = f["psi"][k][fe[1]]
            if hit:
                out[side] = gd
        return out

    def ifaces_touching(self):
        return sorted({fe[0] for lst in self.faces.values() for fe in lst if fe is not None})


def mrcm_solve(prob, return_system=False):
    """Discrete MRCM solution on the quadtree layout of every realisation:
    p [R, ny, nx], ux [R, ny, nx+1], uy [R, ny+1, nx] and the one-sided
    interface velocities gamma_u (per realisation, per interface [2, len])."""
    if prob.pure_neumann:
        raise ValueError("the quadtree oracle covers problems with boundary pressure data")
    if getattr(prob, "grav", None) is not None:
        raise ValueError("the quadtree oracle has no gravity term")
    R, ny, nx, h = prob.n_real, prob.ny, prob.nx, prob.h
    P = np.zeros((R, ny, nx))
    UX = np.zeros((R, ny, nx + 1))
    UY = np.zeros((R, ny + 1, nx))
    gam, systems = [], []
    for r in range(R):
        lay = QLayout(prob, r)
        kappa = prob.lam[r] * prob.K[r]
        locs, basis = [], []
        # steps 1-2: local operators and the multiscale basis
        for k in range(len(lay.subs)):
            lo = QLocal(prob, r, lay, k, kappa)
            locs.append(lo)
            cols, rhs = [(None, None)], [lo.b0]
            for g in lo.ifaces_touching():
                f = lay.ifaces[g]
                for kk in range(f["nU"]):
                    cols.append((g, f["off"] + kk))
                    rhs.append(lo.robin_rhs(lo.data_of(lay, g, ("U", kk))))
                for kk in range(f["nP"]):
                    cols.append((g, f["off"] + f["nU"] + kk))
                    rhs.append(lo.robin_rhs(lo.data_of(lay, g, ("P", kk))))
            X = O.solve_local(lo.A, np.stack(rhs, axis=1))
            basis.append((cols, X))
        # step 3: the interface system
        n = lay.n_unknowns
        M = np.zeros((n, n))
        rhs = np.zeros(n)

        def traces(k, g, ci):
            """Outward velocity and face pressure of column ci of subdomain k
            on the faces of interface g (ordered along g)."""
            lo = locs[k]
            cols, X = basis[k]
            cg, cu = cols[ci]
            f = lay.ifaces[g]
            u = np.zeros(f["len"])
            pf = np.zeros(f["len"])
            own = None
            if cg == g:
                kk = cu - f["off"]
                own = lo.data_of(lay, g, ("U", kk) if kk < f["nU"] else ("P", kk - f["nU"]))
            for side, lst in lo.faces.items():
                for e, fe in enumerate(lst):
                    if fe is None or fe[0] != g:
                        continue
                    a, b = O.edge_face_cell(side, e, lo.s)
                    gd = own[side][e] if own is not None and side in own else 0.0
                    ue = lo.TR[side][e] * (X[b * lo.s + a, ci] - gd) / h
                    u[fe[1]] = ue
                    pf[fe[1]] = gd + lo.beta[side][e] * ue
            return u, pf

        for g, f in enumerate(lay.ifaces):
            for k, sgn in ((f["L"], +1.0), (f["R"], -1.0)):
                cols, X = basis[k]
                for ci, (cg, cu) in enumerate(cols):
                    u, pf = traces(k, g, ci)
                    for kk in range(f["nU"]):             # pressure continuity, tested by phi_k
                        v = sgn * h * np.dot(f["phi"][kk], pf)
                        if ci == 0:
                            rhs[f["off"] + kk] -= v
                        else:
                            M[f["off"] + kk, cu] += v
                    for kk in range(f["nP"]):             # flux continuity, tested by psi_k
                        v = h * np.dot(f["psi"][kk], u)
                        row = f["off"] + f["nU"] + kk
                        if ci == 0:
                            rhs[row] -= v
                        else:
                            M[row, cu] += v
        if n == 0:
            x = np.zeros(0)
        elif n <= 4096:
            x = np.linalg.solve(M, rhs)
        else:
            x = spla.spsolve(sp.csr_matrix(M), rhs)
        if return_system:
            systems.append(dict(M=M, rhs=rhs, x=x, layout=lay))
        # step 4: combination, one-sided interface velocities, face velocities
        p = np.zeros((ny, nx))
        gamma = [np.zeros((2, f["len"])) for f in lay.ifaces]
        for k, lo in enumerate(locs):
            cols, X = basis[k]
            coef = np.array([1.0] + [x[cu] for (_, cu) in cols[1:]])
            pl = X @ coef
            s = lo.s
            p[lo.y0:lo.y0 + s, lo.x0:lo.x0 + s] = pl.reshape(s, s)
            for side, lst in lo.faces.items():
                for e, fe in enumerate(lst):
                    if fe is None:
                        continue
                    g, ei, sigma = fe
                    f = lay.ifaces[g]
                    U = x[f["off"]:f["off"] + f["nU"]]
                    Pv = x[f["off"] + f["nU"]:f["off"] + f["nU"] + f["nP"]]
                    UH = U @ f["phi"][:, ei] if f["nU"] else 0.0
                    PH = Pv @ f["psi"][:, ei] if f["nP"] else 0.0
                    gd = -lo.beta[side][e] * sigma * UH + PH
                    a, b = O.edge_face_cell(side, e, s)
                    gamma[g][0 if sigma > 0 else 1, ei] = lo.TR[side][e] * (pl[b * s + a] - gd) / h
        ux, uy = _fluxes(prob, r, p, lay, gamma)
        P[r], UX[r], UY[r] = p, ux, uy
        gam.append(gamma)
    out = dict(p=P, ux=UX, uy=UY, gamma_u=gam)
    if return_system:
        out["systems"] = systems
    return out


def _fluxes(prob, r, p, lay, gamma):
    """Two-point fluxes inside subdomains, the mean of the one-sided
    velocities on interface faces, boundary data on physical faces."""
    ny, nx, h = prob.ny, prob.nx, prob.h
    kap = prob.lam[r] * prob.K[r]
    ux = np.zeros((ny, nx + 1))
    uy = np.zeros((ny + 1, nx))
    for j in range(ny):
        for i in range(1, nx):
            fe = lay.face_if.get(("V", i, j))
            if fe is not None:
                g, e = fe
                ux[j, i] = 0.5 * (gamma[g][0, e] - gamma[g][1, e])
            else:
                ux[j, i] = O.harmonic_T(kap[j, i - 1], kap[j, i]) * (p[j, i - 1] - p[j, i]) / h
    for j in range(1, ny):
        for i in range(nx):
            fe = lay.face_if.get(("H", j, i))
            if fe is not None:
                g, e = fe
                uy[j, i] = 0.5 * (gamma[g][0, e] - gamma[g][1, e])
            else:
                uy[j, i] = O.harmonic_T(kap[j - 1, i], kap[j, i]) * (p[j - 1, i] - p[j, i]) / h
    for j in range(ny):
        for side, i, sign in (("W", 0, -1.0), ("E", nx - 1, 1.0)):
            k = O.boundary_face(prob, side, i, j)
            un = (2.0 * kap[j, i] * (p[j, i] - prob.bc_val[k]) / h
                  if prob.bc_type[k] == O.DIRICHLET else prob.bc_val[k])
            ux[j, 0 if side == "W" else nx] = sign * un
    for i in range(nx):
        for side, j, sign in (("S", 0, -1.0), ("N", ny - 1, 1.0)):
            k = O.boundary_face(prob, side, i, j)
            un = (2.0 * kap[j, i] * (p[j, i] - prob.bc_val[k]) / h
                  if prob.bc_type[k] == O.DIRICHLET else prob.bc_val[k])
            uy[0 if side == "S" else ny, i] = sign * un
    return ux, uy
