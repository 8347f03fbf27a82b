"""Plain FP64 CPU oracle of the MRCM Darcy solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library: it reads the inputs produced by
``paper_2104_04653_gb300.workloads`` and nothing else of the package.

It computes, slowly and in the order the paper states it, the discrete MRCM
solution of the Darcy problem (Section 2, Eq. "Darcy"):

1. for every subdomain, the local Robin problem (Section 3, Eq. "mrc1") is
   discretised by lowest-order Raviart-Thomas with trapezoidal quadrature on
   square cells, i.e. the two-point flux F = T (p_c - p_c') with the harmonic
   transmissibility 2 k_L k_R / (k_L + k_R) between cells, 2 k_c towards a
   prescribed boundary pressure, and a Robin transmissibility
   T_R = k_c / (alpha H / h + 1/2) towards the interface data
   g = -beta sigma U_H + P_H, beta = alpha H / k_c (Eq. "beta");
2. one local solve per interface function on each interface edge of the
   subdomain plus one for sources and boundary data gives the multiscale
   basis (text after Eq. "beta");
3. the traces of the basis enter the interface system (Eq. "mrc2", which by
   the Robin condition is the weak continuity of Eq. "compatibility"), solved
   densely by LU with partial pivoting;
4. the solution is the linear combination of the basis with the interface
   coefficients.

Readings of points the paper leaves open (the same readings hold for the
CUDA path):
interface functions are Legendre polynomials sampled at face midpoints of
t in [-1, 1]; unknowns per interface are ordered [U_0..U_{nU-1},
P_0..P_{nP-1}]; on an interface face the reported velocity is the mean of
the two one-sided normal velocities; a pure-Neumann problem is solved with
the interface system bordered by its constant-pressure null vector, and the
pressure is shifted to zero cell mean.

Pinned by ``tests/test_oracle_pins.py``: exact linear pressure, equality with
the fine-grid solve for full interface spaces, symmetry/definiteness of the
local operators, the symmetric structure of the interface matrix, local mass
balance, interface flux balance, basis-family invariance and a monolithic
brute-force solve on tiny grids.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

NEUMANN, DIRICHLET = 0, 1


# --------------------------------------------------------------- coefficients
def harmonic_T(kl, kr):
    """Cell-to-cell transmissibility on square cells (RT0 + trapezoid)."""
    return 2.0 * kl * kr / (kl + kr)


def robin_T(kc, alpha, H, h):
    """Transmissibility from a cell centre to Robin data g across a Robin
    face with beta = alpha H / k_c (Eq. "mrc1" last row, Eq. "beta")."""
    return kc / (alpha * H / h + 0.5)


def interface_functions(n_fn, s, family="legendre"):
    """[n_fn, s] values of the interface functions at face midpoints."""
    t = -1.0 + (2.0 * np.arange(s) + 1.0) / s
    out = np.zeros((n_fn, s))
    for k in range(n_fn):
        if family == "legendre":
            c = np.zeros(k + 1)
            c[k] = 1.0
            out[k] = np.polynomial.legendre.legval(t, c)
        elif family == "monomial":
            out[k] = t ** k
        else:
            raise ValueError(family)
    return out


# --------------------------------------------------------------- topology
class Layout:
    """Subdomains and interfaces of one realisation (canonical ordering)."""

    def __init__(self, prob, r):
        self.nx, self.ny = prob.nx, prob.ny
        self.s = s = prob.sub_size[r]
        self.h = prob.h
        self.H = s * self.h
        self.Sx, self.Sy = self.nx // s, self.ny // s
        if self.Sx * s != self.nx or self.Sy * s != self.ny:
            raise ValueError("grid not divisible into subdomains")
        self.ifaces = []
        nU, nP = prob.iface_nU[r], prob.iface_nP[r]
        for J in range(self.Sy):                      # vertical interfaces
            for I in range(self.Sx - 1):
                self.ifaces.append(dict(kind="V", L=(I, J), R=(I + 1, J)))
        for J in range(self.Sy - 1):                  # horizontal interfaces
            for I in range(self.Sx):
                self.ifaces.append(dict(kind="H", L=(I, J), R=(I, J + 1)))
        off = 0
        for g, f in enumerate(self.ifaces):
            f["nU"], f["nP"] = int(nU[g]), int(nP[g])
            f["off"] = off
            off += f["nU"] + f["nP"]
            if getattr(prob, "iface_fn", None) is None:
                f["phi"] = interface_functions(f["nU"], s, prob.basis)
                f["psi"] = interface_functions(f["nP"], s, prob.basis)
            else:                                     # per-interface tables
                phi, psi = prob.iface_fn[r][g]
                f["phi"] = np.asarray(phi, np.float64).reshape(f["nU"], s)
                f["psi"] = np.asarray(psi, np.float64).reshape(f["nP"], s)
            if prob.alpha is None:
                f["alpha"] = np.ones(s)
            else:
                f["alpha"] = np.asarray(prob.alpha[r][g], np.float64)
        self.n_unknowns = off
        # edge table: (I,J) -> {side: (iface index, sigma)}
        self.edges = {}
        for g, f in enumerate(self.ifaces):
            I, J = f["L"]
            self.edges.setdefault((I, J), {})["E" if f["kind"] == "V" else "N"] = (g, +1)
            I, J = f["R"]
            self.edges.setdefault((I, J), {})["W" if f["kind"] == "V" else "S"] = (g, -1)


def edge_face_cell(side, e, s):
    """Local cell (a, b) adjacent to face e of the subdomain edge ``side``."""
    return {"W": (0, e), "E": (s - 1, e), "S": (e, 0), "N": (e, s - 1)}[side]


def boundary_face(prob, side, i, j):
    """Index into bc arrays of the physical face ``side`` of global cell."""
    nx, ny = prob.nx, prob.ny
    return {"W": j, "E": ny + j, "S": 2 * ny + i, "N": 2 * ny + nx + i}[side]


# --------------------------------------------------------------- local problem
class Local:
    """The discrete local Robin problem of one subdomain (Eq. "mrc1")."""

    def __init__(self, prob, r, lay, I, J, kappa):
        s, h = lay.s, lay.h
        self.I, self.J, self.s = I, J, s
        self.n = n = s * s
        self.kap = kappa[J * s:(J + 1) * s, I * s:(I + 1) * s]
        self.edges = lay.edges.get((I, J), {})
        A = np.zeros((n, n))
        b0 = np.zeros(n)
        # Robin transmissibility and beta on each interface edge face
        self.TR, self.beta = {}, {}
        for side, (g, sigma) in self.edges.items():
            f = lay.ifaces[g]
            kc = np.array([self.kap[edge_face_cell(side, e, s)[::-1]] for e in range(s)])
            self.TR[side] = robin_T(kc, f["alpha"], lay.H, h)
            self.beta[side] = f["alpha"] * lay.H / kc
        for b in range(s):
            for a in range(s):
                c = b * s + a
                kc = self.kap[b, a]
                gi, gj = I * s + a, J * s + b
                b0[c] += prob.q[r, gj, gi] * h * h
                for side, da, db in (("W", -1, 0), ("E", 1, 0), ("S", 0, -1), ("N", 0, 1)):
                    aa, bb = a + da, b + db
                    if 0 <= aa < s and 0 <= bb < s:          # interior face
                        T = harmonic_T(kc, self.kap[bb, aa])
                        A[c, c] += T
                        A[c, bb * s + aa] -= T
                    elif side in self.edges:                  # Robin face on Gamma
                        e = b if side in ("W", "E") else a
                        A[c, c] += self.TR[side][e]
                    else:                                     # physical boundary
                        k = boundary_face(prob, side, gi, gj)
                        if prob.bc_type[k] == DIRICHLET:
                            T = 2.0 * kc
                            A[c, c] += T
                            b0[c] += T * prob.bc_val[k]
                        else:
                            b0[c] -= prob.bc_val[k] * h
        self.A, self.b0 = A, b0

    def robin_rhs(self, side, g):
        """RHS of Robin data g (length s) on edge ``side``: T_R g at the
        adjacent cells."""
        s = self.s
        b = np.zeros(self.n)
        for e in range(s):
            a, bb = edge_face_cell(side, e, s)
            b[bb * s + a] += self.TR[side][e] * g[e]
        return b


def robin_data(f, sigma, beta, x):
    """g = -beta sigma U_H + P_H on one side of interface f, for the
    interface unknown vector x (Eq. "mrc1")."""
    U = x[f["off"]:f["off"] + f["nU"]]
    P = x[f["off"] + f["nU"]:f["off"] + f["nU"] + f["nP"]]
    UH = U @ f["phi"] if f["nU"] else np.zeros(len(beta))
    PH = P @ f["psi"] if f["nP"] else np.zeros(len(beta))
    return -beta * sigma * UH + PH


# --------------------------------------------------------------- the solve
def solve_local(A, B, refine=False):
    """Cholesky solve A X = B (library routine); with ``refine``, one step of
    residual refinement with the residual in extended precision."""
    cf = sla.cho_factor(A, lower=True)
    X = sla.cho_solve(cf, B)
    if refine:
        Al = A.astype(np.longdouble)
        R = (B.astype(np.longdouble) - Al @ X.astype(np.longdouble)).astype(np.float64)
        X = X + sla.cho_solve(cf, R)
    return X


def mrcm_solve(prob, refine=False, return_system=False):
    """Discrete MRCM solution for every realisation of ``prob``.

    Returns dict with p [R,ny,nx], ux [R,ny,nx+1], uy [R,ny+1,nx] (normal
    velocities, + along +x / +y), ``gamma_u`` (per realisation, per interface
    [2, s] one-sided outward velocities L then R) and, if requested, the
    interface matrices, right-hand sides and solutions.
    """
    R = prob.n_real
    ny, nx, h = prob.ny, prob.nx, prob.h
    P = np.zeros((R, ny, nx))
    UX = np.zeros((R, ny, nx + 1))
    UY = np.zeros((R, ny + 1, nx))
    gam, systems = [], []
    for r in range(R):
        lay = Layout(prob, r)
        s = lay.s
        kappa = prob.lam[r] * prob.K[r]
        locs = {}
        basis = {}
        # --- steps 1-2: local operators and multiscale basis (text after Eq. "beta")
        for J in range(lay.Sy):
            for I in range(lay.Sx):
                lo = Local(prob, r, lay, I, J, kappa)
                locs[(I, J)] = lo
                cols, rhs = [("part", None, None)], [lo.b0]
                for side, (g, sigma) in sorted(lo.edges.items()):
                    f = lay.ifaces[g]
                    for k in range(f["nU"]):
                        gk = -lo.beta[side] * sigma * f["phi"][k]
                        cols.append((side, g, f["off"] + k))
                        rhs.append(lo.robin_rhs(side, gk))
                    for k in range(f["nP"]):
                        gk = f["psi"][k].copy()
                        cols.append((side, g, f["off"] + f["nU"] + k))
                        rhs.append(lo.robin_rhs(side, gk))
                X = solve_local(lo.A, np.stack(rhs, axis=1), refine)
                basis[(I, J)] = (cols, X)
        # --- step 3: interface system (Eq. "mrc2")
        n = lay.n_unknowns
        M = np.zeros((n, n))
        rhs = np.zeros(n)

        def edge_traces(IJ, side, col_index):
            """Flux and pressure traces on edge ``side`` of subdomain IJ for
            basis column ``col_index`` (0 = particular solution)."""
            lo = locs[IJ]
            cols, X = basis[IJ]
            g_if, sigma = lo.edges[side]
            f = lay.ifaces[g_if]
            cside, cg, cu = cols[col_index]
            gdata = np.zeros(s)
            if cside == side:           # this column's Robin data lives here
                k = cu - f["off"]
                if k < f["nU"]:
                    gdata = -lo.beta[side] * sigma * f["phi"][k]
                else:
                    gdata = f["psi"][k - f["nU"]].copy()
            pc = np.array([X[edge_face_cell(side, e, s)[1] * s + edge_face_cell(side, e, s)[0],
                             col_index] for e in range(s)])
            u = lo.TR[side] * (pc - gdata) / h           # outward normal velocity
            pf = gdata + lo.beta[side] * u               # face pressure
            return u, pf

        for gi, f in enumerate(lay.ifaces):
            Lside = "E" if f["kind"] == "V" else "N"
            Rside = "W" if f["kind"] == "V" else "S"
            for IJ, side, sgn in ((f["L"], Lside, +1.0), (f["R"], Rside, -1.0)):
                cols, X = basis[IJ]
                for ci, (cside, cg, cu) in enumerate(cols):
                    u, pf = edge_traces(IJ, side, ci)
                    for k in range(f["nU"]):              # pressure continuity, tested by phi_k
                        v = sgn * h * np.dot(f["phi"][k], pf)
                        if ci == 0:
                            rhs[f["off"] + k] -= v
                        else:
                            M[f["off"] + k, cu] += v
                    for k in range(f["nP"]):              # flux continuity, tested by psi_k
                        v = h * np.dot(f["psi"][k], u)
                        row = f["off"] + f["nU"] + k
                        if ci == 0:
                            rhs[row] -= v
                        else:
                            M[row, cu] += v
        if prob.pure_neumann:
            z = null_vector(lay)
            Mb = np.zeros((n + 1, n + 1))
            Mb[:n, :n] = M
            Mb[:n, n] = z
            Mb[n, :n] = z
            xb = np.linalg.solve(Mb, np.append(rhs, 0.0))
            x = xb[:n]
        elif n == 0:
            x = np.zeros(0)
        elif n <= 4096:
            x = np.linalg.solve(M, rhs)
        else:
            x = spla.spsolve(sp.csr_matrix(M), rhs)
        if return_system:
            systems.append(dict(M=M, rhs=rhs, x=x, layout=lay))
        # --- step 4: linear combination and fluxes (text after Eq. "beta")
        p = np.zeros((ny, nx))
        gamma_u = np.zeros((len(lay.ifaces), 2, s))
        for (I, J), (cols, X) in basis.items():
            coef = np.array([1.0] + [x[cu] for (_, _, cu) in cols[1:]])
            p[J * s:(J + 1) * s, I * s:(I + 1) * s] = (X @ coef).reshape(s, s)
        for (I, J), lo in locs.items():
            pl = p[J * s:(J + 1) * s, I * s:(I + 1) * s].reshape(-1)
            for side, (g_if, sigma) in lo.edges.items():
                f = lay.ifaces[g_if]
                g = robin_data(f, sigma, lo.beta[side], x)
                pc = np.array([pl[edge_face_cell(side, e, s)[1] * s + edge_face_cell(side, e, s)[0]]
                               for e in range(s)])
                gamma_u[g_if, 0 if sigma > 0 else 1] = lo.TR[side] * (pc - g) / h
        ux, uy = fluxes_from_pressure(prob, r, p, lay, gamma_u)
        if prob.pure_neumann:
            p = p - p.mean()
        P[r], UX[r], UY[r] = p, ux, uy
        gam.append(gamma_u)
    out = dict(p=P, ux=UX, uy=UY, gamma_u=gam)
    if return_system:
        out["systems"] = systems
    return out


def null_vector(lay):
    """P_H = 1 on every interface, U_H = 0: the constant-pressure mode of the
    pure-Neumann interface system (needs the constant in every P space)."""
    z = np.zeros(lay.n_unknowns)
    for f in lay.ifaces:
        # coefficients c with c @ psi == 1 (least squares; exact when 1 is in the span)
        c, *_ = np.linalg.lstsq(f["psi"].T, np.ones(lay.s), rcond=None)
        z[f["off"] + f["nU"]:f["off"] + f["nU"] + f["nP"]] = c
    return z


def fluxes_from_pressure(prob, r, p, lay, gamma_u):
    """Face normal velocities from cell pressures: two-point fluxes on faces
    inside a subdomain, the mean of the one-sided velocities on interface
    faces, and boundary data / Dirichlet fluxes on physical faces."""
    ny, nx, h, s = prob.ny, prob.nx, prob.h, lay.s
    kap = prob.lam[r] * prob.K[r]
    ux = np.zeros((ny, nx + 1))
    uy = np.zeros((ny + 1, nx))
    for j in range(ny):
        for i in range(1, nx):
            if i % s == 0:
                I, J = i // s - 1, j // s
                g = J * (lay.Sx - 1) + I
                e = j % s
                ux[j, i] = 0.5 * (gamma_u[g, 0, e] - gamma_u[g, 1, e])
            else:
                T = harmonic_T(kap[j, i - 1], kap[j, i])
                ux[j, i] = T * (p[j, i - 1] - p[j, i]) / h
    nV = (lay.Sx - 1) * lay.Sy
    for j in range(1, ny):
        for i in range(nx):
            if j % s == 0:
                I, J = i // s, j // s - 1
                g = nV + J * lay.Sx + I
                e = i % s
                uy[j, i] = 0.5 * (gamma_u[g, 0, e] - gamma_u[g, 1, e])
            else:
                T = harmonic_T(kap[j - 1, i], kap[j, i])
                uy[j, i] = T * (p[j - 1, i] - p[j, i]) / h
    for j in range(ny):
        for side, i, sign in (("W", 0, -1.0), ("E", nx - 1, 1.0)):
            k = boundary_face(prob, side, i, j)
            un = (2.0 * kap[j, i] * (p[j, i] - prob.bc_val[k]) / h
                  if prob.bc_type[k] == DIRICHLET else prob.bc_val[k])
            ux[j, 0 if side == "W" else nx] = sign * un
    for i in range(nx):
        for side, j, sign in (("S", 0, -1.0), ("N", ny - 1, 1.0)):
            k = boundary_face(prob, side, i, j)
            un = (2.0 * kap[j, i] * (p[j, i] - prob.bc_val[k]) / h
                  if prob.bc_type[k] == DIRICHLET else prob.bc_val[k])
            uy[0 if side == "S" else ny, i] = sign * un
    return ux, uy


# --------------------------------------------------------------- fine grid
def fine_solve(prob):
    """Global two-point-flux solve on the fine grid (no decomposition): the
    discretisation of Eq. "Darcy" that MRCM approximates."""
    R, ny, nx, h = prob.n_real, prob.ny, prob.nx, prob.h
    P = np.zeros((R, ny, nx))
    UX = np.zeros((R, ny, nx + 1))
    UY = np.zeros((R, ny + 1, nx))
    N = nx * ny
    for r in range(R):
        kap = prob.lam[r] * prob.K[r]
        rows, cols, vals = [], [], []
        b = (prob.q[r] * h * h).reshape(-1).copy()
        for j in range(ny):
            for i in range(nx):
                c = j * nx + i
                for side, di, dj in (("W", -1, 0), ("E", 1, 0), ("S", 0, -1), ("N", 0, 1)):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < nx and 0 <= jj < ny:
                        T = harmonic_T(kap[j, i], kap[jj, ii])
                        rows += [c, c]
                        cols += [c, jj * nx + ii]
                        vals += [T, -T]
                    else:
                        k = boundary_face(prob, side, i, j)
                        if prob.bc_type[k] == DIRICHLET:
                            rows.append(c)
                            cols.append(c)
                            vals.append(2.0 * kap[j, i])
                            b[c] += 2.0 * kap[j, i] * prob.bc_val[k]
                        else:
                            b[c] -= prob.bc_val[k] * h
        A = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
        if prob.pure_neumann:
            one = sp.csr_matrix(np.ones((N, 1)))
            Ab = sp.bmat([[A, one], [one.T, None]]).tocsc()
            p = spla.spsolve(Ab, np.append(b, 0.0))[:N]
        else:
            p = spla.spsolve(A.tocsc(), b)
        p = p.reshape(ny, nx)
        ux = np.zeros((ny, nx + 1))
        uy = np.zeros((ny + 1, nx))
        ux[:, 1:nx] = harmonic_T(kap[:, :-1], kap[:, 1:]) * (p[:, :-1] - p[:, 1:]) / h
        uy[1:ny, :] = harmonic_T(kap[:-1, :], kap[1:, :]) * (p[:-1, :] - p[1:, :]) / h
        for j in range(ny):
            for side, i, sign in (("W", 0, -1.0), ("E", nx - 1, 1.0)):
                k = boundary_face(prob, side, i, j)
                un = (2.0 * kap[j, i] * (p[j, i] - prob.bc_val[k]) / h
                      if prob.bc_type[k] == DIRICHLET else prob.bc_val[k])
                ux[j, 0 if side == "W" else nx] = sign * un
        for i in range(nx):
            for side, j, sign in (("S", 0, -1.0), ("N", ny - 1, 1.0)):
                k = boundary_face(prob, side, i, j)
                un = (2.0 * kap[j, i] * (p[j, i] - prob.bc_val[k]) / h
                      if prob.bc_type[k] == DIRICHLET else prob.bc_val[k])
                uy[0 if side == "S" else ny, i] = sign * un
        if prob.pure_neumann:
            p = p - p.mean()
        P[r], UX[r], UY[r] = p, ux, uy
    return dict(p=P, ux=UX, uy=UY)


# --------------------------------------------------------------- brute force
def monolithic_solve(prob, r=0):
    """Brute force for tiny grids, written from Eq. "mrc1"/"mrc2" directly.

    ONE dense system whose unknowns are every cell pressure, and on every
    interface face and side the face pressure p_f and the outward normal
    velocity u, plus the interface coefficients (U_H, P_H).  Equations:
    cell balances (two-point fluxes inside a subdomain, the half-cell flux
    2 kappa (p_c - p_f) on an interface face), the half-cell flux law
    u = 2 kappa (p_c - p_f)/h, the Robin condition -beta u + p_f =
    -beta sigma U_H + P_H with beta = alpha H / kappa written as given, and
    the interface conditions of Eq. "mrc2".  No Robin transmissibility, no
    basis and no linear combination: it checks those derivations."""
    lay = Layout(prob, r)
    s, h = lay.s, prob.h
    kap = prob.lam[r] * prob.K[r]
    ny, nx = prob.ny, prob.nx
    nc = nx * ny
    faces = []                                # (iface, side index, e, cell (i, j))
    for g, f in enumerate(lay.ifaces):
        for side, IJ in ((0, f["L"]), (1, f["R"])):
            I, J = IJ
            for e in range(s):
                if f["kind"] == "V":
                    i = I * s + (s - 1 if side == 0 else 0)
                    j = J * s + e
                else:
                    i = I * s + e
                    j = J * s + (s - 1 if side == 0 else 0)
                faces.append((g, side, e, i, j))
    nf = len(faces)
    fidx = {(g, sd, e): k for k, (g, sd, e, _, _) in enumerate(faces)}
    o_pf, o_u, o_x = nc, nc + nf, nc + 2 * nf
    N = o_x + lay.n_unknowns
    A = np.zeros((N, N))
    b = np.zeros(N)
    sub_of = lambda i, j: (i // s, j // s)
    row = 0
    # cell balances: sum of outward fluxes = q h^2
    for j in range(ny):
        for i in range(nx):
            c = j * nx + i
            b[row] = prob.q[r, j, i] * h * h
            for side, di, dj in (("W", -1, 0), ("E", 1, 0), ("S", 0, -1), ("N", 0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    if sub_of(i, j) == sub_of(ii, jj):
                        T = 2.0 * kap[j, i] * kap[jj, ii] / (kap[j, i] + kap[jj, ii])
                        A[row, c] += T
                        A[row, jj * nx + ii] -= T
                    else:                    # interface face: flux h*u of this side
                        if side in ("E", "W"):
                            g = (j // s) * (lay.Sx - 1) + min(i, ii) // s
                            e = j % s
                        else:
                            g = (lay.Sx - 1) * lay.Sy + (min(j, jj) // s) * lay.Sx + i // s
                            e = i % s
                        sd = 0 if side in ("E", "N") else 1
                        A[row, o_u + fidx[(g, sd, e)]] += h
                else:
                    k = boundary_face(prob, side, i, j)
                    if prob.bc_type[k] == DIRICHLET:
                        A[row, c] += 2.0 * kap[j, i]
                        b[row] += 2.0 * kap[j, i] * prob.bc_val[k]
                    else:
                        b[row] -= prob.bc_val[k] * h
            row += 1
    # half-cell flux law and Robin condition on every interface face and side
    for k, (g, sd, e, i, j) in enumerate(faces):
        f = lay.ifaces[g]
        kc = kap[j, i]
        A[row, o_u + k] = 1.0
        A[row, j * nx + i] -= 2.0 * kc / h
        A[row, o_pf + k] += 2.0 * kc / h
        row += 1
        beta = f["alpha"][e] * lay.H / kc
        sigma = 1.0 if sd == 0 else -1.0
        A[row, o_u + k] = -beta
        A[row, o_pf + k] = 1.0
        for q_ in range(f["nU"]):
            A[row, o_x + f["off"] + q_] += beta * sigma * f["phi"][q_, e]
        for q_ in range(f["nP"]):
            A[row, o_x + f["off"] + f["nU"] + q_] -= f["psi"][q_, e]
        row += 1
    # interface conditions (Eq. "mrc2")
    for g, f in enumerate(lay.ifaces):
        for q_ in range(f["nU"]):
            for e in range(s):
                A[row, o_pf + fidx[(g, 0, e)]] += h * f["phi"][q_, e]
                A[row, o_pf + fidx[(g, 1, e)]] -= h * f["phi"][q_, e]
            row += 1
        for q_ in range(f["nP"]):
            for e in range(s):
                A[row, o_u + fidx[(g, 0, e)]] += h * f["psi"][q_, e]
                A[row, o_u + fidx[(g, 1, e)]] += h * f["psi"][q_, e]
            row += 1
    assert row == N
    if prob.pure_neumann:
        # constant mode: every pressure (cell, face, P_0) shifts together;
        # border with the zero cell-sum condition and the left null vector
        Ab = np.zeros((N + 1, N + 1))
        Ab[:N, :N] = A
        Ab[N, :nc] = 1.0
        Ab[:N, N] = _left_null(A)
        sol = np.linalg.solve(Ab, np.append(b, 0.0))[:N]
    else:
        sol = np.linalg.solve(A, b)
    p = sol[:nc].reshape(ny, nx)
    if prob.pure_neumann:
        p = p - p.mean()
    gam = np.zeros((len(lay.ifaces), 2, s))
    for k, (g, sd, e, i, j) in enumerate(faces):
        gam[g, sd, e] = sol[o_u + k]
    return dict(p=p, x=sol[o_x:], gamma_u=gam)


def _left_null(A):
    """Unit left null vector of a matrix with a one-dimensional left kernel."""
    u, sv, vt = np.linalg.svd(A.T)
    return vt[-1]


# --------------------------------------------------------------- norms
def rel_l2(a, b):
    """Relative L2 difference ||a - b|| / ||b|| (0 when both vanish)."""
    nb = np.linalg.norm(b)
    d = np.linalg.norm(a - b)
    return d / nb if nb > 0 else d


def errors(sol, ref):
    """Max over realisations of the relative L2 error of p (cells) and of u
    (all faces of ux and uy together)."""
    ep, eu = 0.0, 0.0
    for r in range(ref["p"].shape[0]):
        ep = max(ep, rel_l2(sol["p"][r], ref["p"][r]))
        ua = np.concatenate([sol["ux"][r].ravel(), sol["uy"][r].ravel()])
        ub = np.concatenate([ref["ux"][r].ravel(), ref["uy"][r].ravel()])
        eu = max(eu, rel_l2(ua, ub))
    return ep, eu
