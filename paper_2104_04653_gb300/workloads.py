"""Seeded synthetic inputs for the MRCM Darcy solve.

This module only *generates inputs*: permeability fields, total-mobility
fields, sources, boundary data and the per-interface space sizes.  It holds
none of the method's arithmetic (no transmissibility, no local solve, no
interface system), so both the CUDA path and the CPU oracle can consume what
it produces without sharing any of the method's code.

Grid conventions (Section 2, Eq. "Darcy"; Section 3, Eq. "mrc1"):

* one realisation is an ``nx x ny`` grid of square cells of side
  ``h = ly / ny`` on ``[0, nx*h] x [0, ly]``; arrays are ``[n_real][ny][nx]``,
  x fastest;
* subdomains are ``s x s`` cells (``s`` per realisation), numbered row-major
  ``S = J*Sx + I``;
* interfaces are listed in a canonical order: first the vertical ones
  (between ``(I,J)`` and ``(I+1,J)``) row-major by ``(J, I)``, then the
  horizontal ones (between ``(I,J)`` and ``(I,J+1)``) row-major by ``(J, I)``;
  the fixed normal points out of the smaller-index subdomain (Section 3,
  below Eq. "compatibility"), i.e. +x or +y;
* boundary faces are listed left (``ny``), right (``ny``), bottom (``nx``),
  top (``nx``); ``bc_type`` 0 = prescribed outward normal velocity ``u_b``,
  1 = prescribed pressure ``p_b`` (Eq. "Darcy").

Recipes (one per workload; seeds ``1000*config + realisation``):

1. 64x64 unit square, log K a Gaussian random field (exponential covariance,
   variance 2, correlation length 0.1) by circulant embedding, quarter
   five-spot with no-flow boundaries, 4x4 subdomains of 16x16, linear spaces.
2. 256x64 on [0,4]x[0,1], binary channelised K (1e3 in four seeded sinusoidal
   channels of width 4 cells, 1e-3 elsewhere), left inflow / right p=0,
   16x16 subdomains, cubic spaces (4 functions per space).
3. ``n_real`` lognormal realisations (variance 3), half with 16x16 and half
   with 32x32 subdomains, per-interface total size m in {2,4,6,8}.
4. 2048x2048 binary channels (64 channels, contrast 1e6), 32x32 subdomains.
5. 512x512 lognormal K with two-phase total mobility from seeded analytic
   Buckley-Leverett fronts (quadratic relative permeabilities, M = 5).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

BC_NEUMANN = 0
BC_DIRICHLET = 1


@dataclass
class Problem:
    """One batch of Darcy problems sharing a grid (all arrays FP64 / int)."""

    nx: int
    ny: int
    ly: float
    sub_size: List[int]               # [n_real] subdomain edge in cells
    K: np.ndarray                     # [n_real, ny, nx]
    lam: np.ndarray                   # [n_real, ny, nx] total mobility
    q: np.ndarray                     # [n_real, ny, nx] source density
    bc_type: np.ndarray               # [2*ny + 2*nx] int8
    bc_val: np.ndarray                # [2*ny + 2*nx] float64
    iface_nU: List[np.ndarray]        # per realisation, canonical order
    iface_nP: List[np.ndarray]
    alpha: Optional[List[np.ndarray]] = None   # per realisation, [n_iface, s]
    # per realisation, per interface: (flux functions [nU, s], pressure
    # functions [nP, s]) at face midpoints; None: the family given by ``basis``
    iface_fn: Optional[list] = None
    # per realisation [ny, nx]: the gravity velocity K lambda_g g of Eq.
    # "Darcy_wg" (along +y, the direction of the height h); None: no gravity
    grav: Optional[list] = None
    # per realisation [ny/B][nx/B] int8 (B = sub_size[r]): a nonzero block is
    # split into four (B/2) x (B/2) subdomains (quadtree); None: uniform
    refine: Optional[list] = None
    pure_neumann: bool = False
    basis: str = "legendre"           # interface function family
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_real(self) -> int:
        return int(self.K.shape[0])

    @property
    def h(self) -> float:
        return self.ly / self.ny

    @property
    def lx(self) -> float:
        return self.nx * self.h

    def n_iface(self, r: int) -> int:
        return n_interfaces(self.nx, self.ny, self.sub_size[r])

    def cells(self) -> int:
        return self.n_real * self.nx * self.ny


def n_interfaces(nx: int, ny: int, s: int) -> int:
    sx, sy = nx // s, ny // s
    return (sx - 1) * sy + sx * (sy - 1)


# ---------------------------------------------------------------- fields
def grf_exponential(nx: int, ny: int, h: float, variance: float,
                    corr_len: float, rng: np.random.Generator) -> np.ndarray:
    """Stationary Gaussian field on cell centres, C(r) = var*exp(-r/corr_len).

    Circulant embedding (Dietrich & Newsam 1997): embed the grid in a periodic
    grid padded at least 2x, take the FFT of the first row of the block
    circulant covariance as its eigenvalues, check they are non-negative
    (else pad more), and colour complex white noise with their square roots.
    """
    pad = 2
    while True:
        mx, my = pad * nx, pad * ny
        dx = h * np.minimum(np.arange(mx), mx - np.arange(mx))
        dy = h * np.minimum(np.arange(my), my - np.arange(my))
        r = np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2)
        c = variance * np.exp(-r / corr_len)
        lam = np.fft.fft2(c).real
        if lam.min() >= -1e-8 * lam.max():
            break
        pad *= 2
    lam = np.clip(lam, 0.0, None)
    w = rng.standard_normal((my, mx)) + 1j * rng.standard_normal((my, mx))
    y = np.fft.fft2(np.sqrt(lam / (mx * my)) * w)
    return np.ascontiguousarray(y.real[:ny, :nx])


def sinusoidal_channels(nx: int, ny: int, n_ch: int, rng: np.random.Generator,
                        k_hi: float = 1e3, k_lo: float = 1e-3,
                        half_width: float = 2.0, scale: float = 1.0) -> np.ndarray:
    """Binary K: k_hi inside seeded sinusoidal channels, k_lo elsewhere.

    Centreline y = y0 + A sin(2 pi x / L + phi) in cell units with
    y0 ~ U(ny/8, 7 ny/8), A ~ U(2,8)*scale, L ~ U(64,256)*scale,
    phi ~ U(0, 2 pi); a cell is in the channel when its centre lies within
    ``half_width`` cells of the centreline.
    """
    xc = np.arange(nx) + 0.5
    yc = np.arange(ny) + 0.5
    K = np.full((ny, nx), k_lo)
    for _ in range(n_ch):
        y0 = rng.uniform(ny / 8.0, 7.0 * ny / 8.0)
        A = rng.uniform(2.0, 8.0) * scale
        L = rng.uniform(64.0, 256.0) * scale
        phi = rng.uniform(0.0, 2.0 * np.pi)
        centre = y0 + A * np.sin(2.0 * np.pi * xc / L + phi)
        inside = np.abs(yc[:, None] - centre[None, :]) < half_width
        K[inside] = k_hi
    return K


def total_mobility(s: np.ndarray, mu_w: float = 1.0, mu_o: float = 5.0) -> np.ndarray:
    """lambda(s) = k_rw/mu_w + k_ro/mu_o with k_rw = s^2, k_ro = (1-s)^2
    (Eq. "fluxos1" with the relative permeabilities of Section 5)."""
    return s * s / mu_w + (1.0 - s) ** 2 / mu_o


def _frac_flow_slope(s: np.ndarray, M: float) -> np.ndarray:
    """d/ds of f(s) = M s^2 / (M s^2 + (1-s)^2) (Section 5)."""
    d = M * s * s + (1.0 - s) ** 2
    return 2.0 * M * s * (1.0 - s) / (d * d)


def bl_front_saturation(M: float) -> float:
    """Welge tangent point of the quadratic-k_r fractional flow from s=0."""
    return 1.0 / np.sqrt(M + 1.0)


def bl_saturation(nx: int, ny: int, h: float, step: int, M: float,
                  rng: np.random.Generator, nbisect: int = 60) -> np.ndarray:
    """Analytic Buckley-Leverett-shaped saturation behind a perturbed front.

    Front x_f(y) = 0.09*step*(1 + 0.05 sin(2 pi y n_y + phi)), n_y in {1,2,3}
    and phi seeded.  Behind the front s solves f'(s)/f'(s_f) = x/x_f on
    [s_f, 1] (bisection; f' decreases there); ahead of it s = 0.
    """
    n_y = int(rng.integers(1, 4))
    phi = rng.uniform(0.0, 2.0 * np.pi)
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    xf = 0.09 * step * (1.0 + 0.05 * np.sin(2.0 * np.pi * yc * n_y + phi))
    sf = bl_front_saturation(M)
    dsf = _frac_flow_slope(np.array(sf), M)
    ratio = xc[None, :] / xf[:, None]
    behind = ratio < 1.0
    lo = np.full(ratio.shape, sf)
    hi = np.ones(ratio.shape)
    for _ in range(nbisect):
        mid = 0.5 * (lo + hi)
        g = _frac_flow_slope(mid, M) / dsf - ratio
        # g decreases in s: g > 0 means the root lies above mid
        up = g > 0.0
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    s = np.where(behind, 0.5 * (lo + hi), 0.0)
    return s


# ---------------------------------------------------------------- boundary data
def bc_left_right(nx: int, ny: int, u_in: float = 1.0, p_out: float = 0.0):
    """Inflow u.n = -u_in on the left, p = p_out on the right, no flow
    top and bottom (the paper's default set-up, Section 5)."""
    t = np.zeros(2 * ny + 2 * nx, dtype=np.int8)
    v = np.zeros(2 * ny + 2 * nx)
    v[:ny] = -u_in
    t[ny:2 * ny] = BC_DIRICHLET
    v[ny:2 * ny] = p_out
    return t, v


def bc_no_flow(nx: int, ny: int):
    return np.zeros(2 * ny + 2 * nx, dtype=np.int8), np.zeros(2 * ny + 2 * nx)


def bc_linear_pressure(nx: int, ny: int, h: float):
    """p = 1 - x on the left and right boundaries, no flow top and bottom."""
    t = np.zeros(2 * ny + 2 * nx, dtype=np.int8)
    v = np.zeros(2 * ny + 2 * nx)
    t[:2 * ny] = BC_DIRICHLET
    v[:ny] = 1.0
    v[ny:2 * ny] = 1.0 - nx * h
    return t, v


# ---------------------------------------------------------------- problems
def uniform_spaces(nx: int, ny: int, s: int, n_u: int, n_p: int):
    n = n_interfaces(nx, ny, s)
    return np.full(n, n_u, np.int32), np.full(n, n_p, np.int32)


def make_problem(nx, ny, s, K, lam=None, q=None, bc=None, n_u=2, n_p=2,
                 pure_neumann=False, ly=1.0, alpha=None, basis="legendre",
                 name="custom") -> Problem:
    """Single-realisation (or stacked) problem with uniform spaces; s is one
    subdomain size for every realisation or a list with one per realisation."""
    K = np.asarray(K, dtype=np.float64)
    if K.ndim == 2:
        K = K[None]
    R = K.shape[0]
    lam = np.ones_like(K) if lam is None else np.asarray(lam, np.float64).reshape(K.shape)
    q = np.zeros_like(K) if q is None else np.asarray(q, np.float64).reshape(K.shape)
    if bc is None:
        bc = bc_no_flow(nx, ny)
    sizes = [int(s)] * R if np.ndim(s) == 0 else [int(v) for v in s]
    spaces = [uniform_spaces(nx, ny, sz, n_u, n_p) for sz in sizes]
    return Problem(nx=nx, ny=ny, ly=ly, sub_size=sizes, K=K, lam=lam, q=q,
                   bc_type=np.asarray(bc[0], np.int8), bc_val=np.asarray(bc[1], np.float64),
                   iface_nU=[sp[0] for sp in spaces], iface_nP=[sp[1] for sp in spaces],
                   alpha=alpha, pure_neumann=pure_neumann, basis=basis, name=name)


def five_spot_sources(nx: int, ny: int, h: float) -> np.ndarray:
    """Unit-rate injector in cell (0,0) and producer in cell (nx-1, ny-1)."""
    q = np.zeros((ny, nx))
    q[0, 0] = 1.0 / (h * h)
    q[ny - 1, nx - 1] = -1.0 / (h * h)
    return q


def config1(seed_offset: int = 0) -> Problem:
    """64x64 GRF quarter five-spot, 4x4 subdomains of 16x16, linear spaces."""
    nx = ny = 64
    h = 1.0 / ny
    rng = np.random.default_rng(1000 * 1 + seed_offset)
    logk = grf_exponential(nx, ny, h, 2.0, 0.1, rng)
    p = make_problem(nx, ny, 16, np.exp(logk), q=five_spot_sources(nx, ny, h),
                     bc=bc_no_flow(nx, ny), n_u=2, n_p=2, pure_neumann=True,
                     name="gaussian-64x64-s16-m4-fivespot")
    return p


def config2(nx: int = 256, ny: int = 64, s: int = 16, n_fn: int = 4,
            n_ch: int = 4) -> Problem:
    """256x64 binary channels (contrast 1e6), 16x16 subdomains, cubic spaces."""
    rng = np.random.default_rng(1000 * 2)
    K = sinusoidal_channels(nx, ny, n_ch, rng)
    h = 1.0 / ny
    return make_problem(nx, ny, s, K, bc=bc_left_right(nx, ny), n_u=n_fn, n_p=n_fn,
                        name=f"channels-{nx}x{ny}-s{s}-m{2 * n_fn}")


def config3_realisation(r: int, n_real: int, n: int, variance: float):
    """Field, subdomain size and interface sizes of realisation r of
    config3 (its own seed, so realisations can be drawn in any order)."""
    h = 1.0 / n
    rng = np.random.default_rng(1000 * 3 + r)
    K = np.exp(grf_exponential(n, n, h, variance, 0.1, rng))
    s = 16 if r < n_real // 2 else 32
    m = rng.choice(np.array([2, 4, 6, 8], np.int32), size=n_interfaces(n, n, s))
    return K, s, m


def config3(n_real: int = 32, n: int = 1024, variance: float = 3.0,
            workers: int = 1) -> Problem:
    """Lognormal realisations; r < n_real/2 use 16x16 subdomains, the rest
    32x32; each interface draws its total size m from {2,4,6,8}.  With
    workers > 1 the realisations are drawn by that many spawned processes
    (same values: every realisation has its own seed)."""
    if workers > 1 and n_real > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=min(workers, n_real),
                                 mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(config3_realisation, range(n_real), [n_real] * n_real,
                                [n] * n_real, [variance] * n_real))
    else:
        parts = [config3_realisation(r, n_real, n, variance) for r in range(n_real)]
    K = np.stack([p[0] for p in parts])
    subs = [p[1] for p in parts]
    nus = [(p[2] // 2).astype(np.int32) for p in parts]
    nps = [(p[2] // 2).astype(np.int32) for p in parts]
    t, v = bc_left_right(n, n)
    return Problem(nx=n, ny=n, ly=1.0, sub_size=subs, K=K, lam=np.ones_like(K),
                   q=np.zeros_like(K), bc_type=t, bc_val=v, iface_nU=nus, iface_nP=nps,
                   name=f"lognormal-{n_real}x{n}x{n}-s16/32-m2..8")


def window(prob: Problem, r: int, n: int) -> Problem:
    """Realisation r of prob cut to its lower-left n x n cells (n a multiple
    of its subdomain size), with the same subdomain size, the interface
    sizes of the interfaces it keeps, and left-to-right boundary data: a
    sample of the workload at a size the CPU oracle solves in seconds."""
    s = prob.sub_size[r]
    if n % s or n > prob.nx or n > prob.ny:
        raise ValueError("window must be a multiple of the subdomain size")
    sx, sy = prob.nx // s, prob.ny // s
    wx = wy = n // s
    nV = (sx - 1) * sy
    ids = [J * (sx - 1) + I for J in range(wy) for I in range(wx - 1)]
    ids += [nV + J * sx + I for J in range(wy - 1) for I in range(wx)]
    ids = np.asarray(ids, np.int64)
    t, v = bc_left_right(n, n)
    ly = n * prob.h
    return Problem(nx=n, ny=n, ly=ly, sub_size=[s], K=prob.K[r:r + 1, :n, :n].copy(),
                   lam=prob.lam[r:r + 1, :n, :n].copy(), q=prob.q[r:r + 1, :n, :n].copy(),
                   bc_type=t, bc_val=v, iface_nU=[prob.iface_nU[r][ids]],
                   iface_nP=[prob.iface_nP[r][ids]], basis=prob.basis,
                   name=f"{prob.name}[r={r}, {n}x{n} window]")


def config4(n: int = 2048, s: int = 32, n_ch: int = 64, seed: int = 4000) -> Problem:
    """Binary channels with contrast 1e6 on an n x n grid, s x s subdomains."""
    rng = np.random.default_rng(seed)
    K = sinusoidal_channels(n, n, n_ch, rng, scale=n / 256.0)
    return make_problem(n, n, s, K, bc=bc_left_right(n, n), n_u=2, n_p=2,
                        name=f"channels-{n}x{n}-s{s}-m4")


def config5(step: int, n: int = 512, s: int = 16, M: float = 5.0) -> Problem:
    """Lognormal K (variance 2) with total mobility from an analytic front
    after ``step`` steps (1..10)."""
    h = 1.0 / n
    rngk = np.random.default_rng(1000 * 5)
    K = np.exp(grf_exponential(n, n, h, 2.0, 0.1, rngk))
    rngs = np.random.default_rng(1000 * 5 + step)
    sat = bl_saturation(n, n, h, step, M, rngs)
    lam = total_mobility(sat, 1.0, M)
    p = make_problem(n, n, s, K, lam=lam, bc=bc_left_right(n, n), n_u=2, n_p=2,
                     name=f"bl-front-{n}x{n}-s{s}-step{step}")
    p.meta["saturation"] = sat
    return p


def quadtree_interface_lengths(nx: int, ny: int, B: int, refine) -> List[int]:
    """Face counts of the interfaces of a quadtree layout in canonical
    order (vertical by (y0, x), then horizontal by (y, x0)): B between two
    unsplit blocks, B/2 wherever a split block takes part.  Layout only."""
    ref = np.asarray(refine, bool).reshape(ny // B, nx // B)
    h2 = B // 2
    # owner block at (B/2)-resolution: (block, quadrant) or (block, -1)
    own = np.empty((ny // h2, nx // h2), dtype=object)
    for j in range(ny // h2):
        for i in range(nx // h2):
            bj, bi = j // 2, i // 2
            own[j, i] = (bj, bi, (j % 2) * 2 + (i % 2)) if ref[bj, bi] else (bj, bi, -1)
    vert, horiz = [], []
    for i in range(1, nx // h2):
        j = 0
        while j < ny // h2:
            L, R = own[j, i - 1], own[j, i]
            if L == R:
                j += 1
                continue
            j1 = j
            while j1 < ny // h2 and own[j1, i - 1] == L and own[j1, i] == R:
                j1 += 1
            vert.append((j * h2, i * h2, (j1 - j) * h2))
            j = j1
    for j in range(1, ny // h2):
        i = 0
        while i < nx // h2:
            L, R = own[j - 1, i], own[j, i]
            if L == R:
                i += 1
                continue
            i1 = i
            while i1 < nx // h2 and own[j - 1, i1] == L and own[j, i1] == R:
                i1 += 1
            horiz.append((j * h2, i * h2, (i1 - i) * h2))
            i = i1
    vert.sort()
    horiz.sort()
    return [v[2] for v in vert] + [hz[2] for hz in horiz]


def quadtree_problem(nx, ny, B, K, refine, lam=None, q=None, bc=None, n_u=2, n_p=2,
                     m_choices=None, seed=0, name="quadtree") -> Problem:
    """Realisations of nx x ny cells in B x B blocks, each block split into
    four (B/2)-subdomains where refine[r] is nonzero.  Interface sizes: n_u
    and n_p, or (m_choices) a seeded total m per interface, nU = nP = m/2."""
    K = np.asarray(K, np.float64)
    if K.ndim == 2:
        K = K[None]
    R = K.shape[0]
    lam = np.ones_like(K) if lam is None else np.asarray(lam, np.float64).reshape(K.shape)
    q = np.zeros_like(K) if q is None else np.asarray(q, np.float64).reshape(K.shape)
    if bc is None:
        bc = bc_left_right(nx, ny)
    rng = np.random.default_rng(seed)
    nus, nps, refs = [], [], []
    for r in range(R):
        ref = np.asarray(refine[r], np.int8).reshape(ny // B, nx // B)
        refs.append(ref)
        L = quadtree_interface_lengths(nx, ny, B, ref)
        if m_choices is None:
            nus.append(np.full(len(L), n_u, np.int32))
            nps.append(np.full(len(L), n_p, np.int32))
        else:
            m = rng.choice(np.asarray(m_choices, np.int32), size=len(L))
            nus.append((m // 2).astype(np.int32))
            nps.append((m // 2).astype(np.int32))
    return Problem(nx=nx, ny=ny, ly=1.0, sub_size=[B] * R, K=K, lam=lam, q=q,
                   bc_type=np.asarray(bc[0], np.int8), bc_val=np.asarray(bc[1], np.float64),
                   iface_nU=nus, iface_nP=nps, refine=refs, name=name)


def random_refinement(nx, ny, B, frac, rng) -> np.ndarray:
    """A seeded refinement mask with about frac of the blocks split."""
    return (rng.random((ny // B, nx // B)) < frac).astype(np.int8)


def gpu_arrays(p: Problem):
    """Flattened, contiguous host arrays in the library's input layout."""
    return (np.ascontiguousarray(p.K.reshape(-1)),
            np.ascontiguousarray(p.lam.reshape(-1)),
            np.ascontiguousarray(p.q.reshape(-1)))
