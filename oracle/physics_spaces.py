"""Physics-based interface spaces and adaptive Robin parameter (Section 3,
"Interface spaces", Eqs. "new_basis1" to "new_basis6"; the alpha values of
Section 5's channelised experiments).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  It shares no code with
the CUDA library (which does not take per-interface function tables yet:
its binding refuses a problem that carries them).

What it computes, per realisation and interface [a, b] (length H, s faces of
width h, face e = [e h, (e+1) h], functions sampled at face midpoints):

* structures: a face is *high* when both cells next to it have
  log10(K / K_ref) > +threshold and *low* when both have < -threshold,
  K_ref the geometric mean of K over the realisation; each maximal run of
  high (low) faces e0..e1 is one channel (barrier) with support
  [a_k, b_k] = [e0 h, (e1 + 1) h].  The paper gives no detector; this
  threshold rule (default 1.5, a factor of about 30) is the reading used.
* pressure space with N_high >= 1 channels (Eqs. "new_basis1" to
  "new_basis3"): psi_0 falls linearly from 1 at a to 0 at a_1; psi_k
  (k = 1..N_high) rises linearly on (b_{k-1}, a_k), is 1 on the channel
  (a_k, b_k) and falls linearly on (b_k, a_{k+1}), with b_0 = a and
  a_{N_high+1} = b; psi_{N_high+1} rises linearly from 0 at b_{N_high} to 1
  at b.  2 + N_high functions.
* flux space with N_low >= 1 barriers (Eqs. "new_basis4" to "new_basis6"):
  the indicators of (a, a_1), of each barrier (a_k, b_k) and of each gap
  (b_k, a_{k+1}), with a_{N_low+1} = b.  1 + 2 N_low functions.
* a function that vanishes at every face midpoint (a structure that
  touches an end of the interface empties psi_0 / phi_0 or
  psi_{N+1} / phi_{2N}) is dropped: it would make the interface system
  singular.
* interfaces without structures of a kind get the linear polynomials (the
  Legendre P0 and P1 at the midpoints) for that space.
* alpha = 1e-2 on every face of an interface that a channel crosses and
  1e2 on every other interface (Section 5).

Pinned by ``tests/test_physics_spaces.py``: partition of unity of both
spaces, the function counts, values against the closed forms of the
equations on a hand-made interface, the detector on planted channels and
barriers, and solves of the oracle with these spaces.
"""
from __future__ import annotations

import copy

import numpy as np

from oracle import mrcm_oracle as O

THRESHOLD = 1.5
ALPHA_CHANNEL = 1e-2
ALPHA_OTHER = 1e2


def runs(mask):
    """Maximal runs of True in a boolean vector, as (e0, e1) inclusive."""
    out, e0 = [], None
    for e, v in enumerate(list(mask) + [False]):
        if v and e0 is None:
            e0 = e
        elif not v and e0 is not None:
            out.append((e0, e - 1))
            e0 = None
    return out


def pressure_functions(channels, s, h):
    """Midpoint values [n, s] of the pressure functions for channel
    supports [(a_k, b_k)] on [0, s h] (empty list: none)."""
    a, b = 0.0, s * h
    x = (np.arange(s) + 0.5) * h
    N = len(channels)
    A = [ck[0] for ck in channels] + [b]          # a_1 .. a_N, a_{N+1} = b
    B = [a] + [ck[1] for ck in channels]          # b_0 = a, b_1 .. b_N
    f = []
    # psi_0: (a_1 - x) / (a_1 - a) on (a, a_1)
    v = np.zeros(s)
    m = (x > a) & (x < A[0])
    v[m] = (A[0] - x[m]) / (A[0] - a)
    f.append(v)
    for k in range(1, N + 1):
        v = np.zeros(s)
        lo, mid0, mid1, hi = B[k - 1], A[k - 1], B[k], A[k]
        up = (x > lo) & (x < mid0)
        v[up] = (x[up] - lo) / (mid0 - lo)
        v[(x >= mid0) & (x <= mid1)] = 1.0
        dn = (x > mid1) & (x < hi)
        v[dn] = (hi - x[dn]) / (hi - mid1)
        f.append(v)
    # psi_{N+1}: (x - b_N) / (b - b_N) on (b_N, b)
    v = np.zeros(s)
    m = (x > B[N]) & (x < b)
    v[m] = (x[m] - B[N]) / (b - B[N])
    f.append(v)
    return np.array([v for v in f if np.any(v != 0.0)])


def flux_functions(barriers, s, h):
    """Midpoint values [n, s] of the flux functions for barrier supports
    [(a_k, b_k)] on [0, s h]."""
    a, b = 0.0, s * h
    x = (np.arange(s) + 0.5) * h
    N = len(barriers)
    A = [bk[0] for bk in barriers] + [b]
    f = [((x > a) & (x < A[0])).astype(float)]
    for k in range(1, N + 1):
        ak, bk = barriers[k - 1]
        f.append(((x > ak) & (x < bk)).astype(float))
        f.append(((x > bk) & (x < A[k])).astype(float))
    return np.array([v for v in f if np.any(v != 0.0)])


def interface_cells(lay, f):
    """K-grid (row, col) index arrays of the two cells next to each face of
    interface f, along the interface (left/bottom side first)."""
    s = lay.s
    I, J = f["L"]
    e = np.arange(s)
    if f["kind"] == "V":                          # faces along y at x = (I+1) s
        rows = J * s + e
        return (rows, np.full(s, (I + 1) * s - 1)), (rows, np.full(s, (I + 1) * s))
    cols = I * s + e                              # faces along x at y = (J+1) s
    return (np.full(s, (J + 1) * s - 1), cols), (np.full(s, (J + 1) * s), cols)


def structures(K, lay, f, threshold=THRESHOLD, kref=None):
    """Channel and barrier supports [(a_k, b_k)] of interface f."""
    kref = np.exp(np.log(K).mean()) if kref is None else kref
    (r0, c0), (r1, c1) = interface_cells(lay, f)
    l0 = np.log10(K[r0, c0] / kref)
    l1 = np.log10(K[r1, c1] / kref)
    h = lay.h
    hi = [(e0 * h, (e1 + 1) * h) for e0, e1 in runs((l0 > threshold) & (l1 > threshold))]
    lo = [(e0 * h, (e1 + 1) * h) for e0, e1 in runs((l0 < -threshold) & (l1 < -threshold))]
    return hi, lo


def physics_problem(prob, threshold=THRESHOLD, alpha_channel=ALPHA_CHANNEL,
                    alpha_other=ALPHA_OTHER, adaptive_alpha=True):
    """A copy of prob with physics-based spaces on every interface that
    structures cross (linear polynomials elsewhere) and, if adaptive_alpha,
    the adaptive alpha; the per-interface tables go to ``iface_fn``."""
    out = copy.deepcopy(prob)
    out.iface_nU, out.iface_nP, out.iface_fn = [], [], []
    out.alpha = [] if adaptive_alpha else prob.alpha
    for r in range(prob.n_real):
        lay = O.Layout(prob, r)
        s, h = lay.s, lay.h
        K = prob.K[r]
        kref = np.exp(np.log(K).mean())
        nU, nP, tabs, al = [], [], [], []
        for f in lay.ifaces:
            hi, lo = structures(K, lay, f, threshold, kref)
            psi = pressure_functions(hi, s, h) if hi else O.interface_functions(2, s, "legendre")
            phi = flux_functions(lo, s, h) if lo else O.interface_functions(2, s, "legendre")
            nU.append(phi.shape[0])
            nP.append(psi.shape[0])
            tabs.append((phi, psi))
            al.append(np.full(s, alpha_channel if hi else alpha_other))
        out.iface_nU.append(np.array(nU, np.int32))
        out.iface_nP.append(np.array(nP, np.int32))
        out.iface_fn.append(tabs)
        if adaptive_alpha:
            out.alpha.append(np.array(al))
    out.name = prob.name + "-physics"
    return out
