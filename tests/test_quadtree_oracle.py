"""Pins of the quadtree MRCM oracle (oracle/quadtree.py): subdomains of two
sizes inside one realisation (Section 3's non-overlapping decomposition,
read as a one-level quadtree), with interfaces covering half of a large
subdomain's edge.

What fixes it, independently of its own code:
* without refinement it is the uniform oracle (mrcm_oracle), which has its
  own pins: same p, u and one-sided interface velocities;
* with full interface spaces (as many functions as faces on every
  interface) MRCM equals the fine-grid two-point solve for any alpha (the
  same special case that pins the uniform oracle);
* homogeneous K with p = 1 - x on the left and right boundaries and no flow
  above and below: every layout reproduces the linear pressure exactly with
  linear spaces;
* per-cell mass balance inside every subdomain with the one-sided interface
  velocities, and zero net flux through every interface (1 is in every
  pressure space);
* the layout enumeration agrees with the input generator's count and
  lengths (two independent codes).
"""
import numpy as np
import pytest

from oracle import mrcm_oracle as O
from oracle import quadtree as Q
from paper_2104_04653_gb300 import workloads as W


def _mixed(nx=32, ny=16, B=8, seed=0, full=False, alpha=None, family="legendre"):
    rng = np.random.default_rng(seed)
    K = np.exp(1.2 * rng.standard_normal((ny, nx)))
    ref = np.zeros((ny // B, nx // B), np.int8)
    ref[0, 1] = ref[1, 2] = 1
    prob = W.quadtree_problem(nx, ny, B, K, [ref], q=rng.standard_normal((ny, nx)))
    if full:
        L = W.quadtree_interface_lengths(nx, ny, B, ref)
        prob.iface_nU = [np.array(L, np.int32)]
        prob.iface_nP = [np.array(L, np.int32)]
    if alpha is not None:
        L = W.quadtree_interface_lengths(nx, ny, B, ref)
        prob.alpha = [[np.full(l, alpha) for l in L]]
    prob.basis = family
    return prob


def test_layout_matches_the_input_generator():
    rng = np.random.default_rng(1)
    for B, nx, ny in ((8, 32, 16), (16, 64, 64), (32, 128, 96)):
        ref = W.random_refinement(nx, ny, B, 0.4, rng)
        prob = W.quadtree_problem(nx, ny, B, np.ones((ny, nx)), [ref])
        lay = Q.QLayout(prob, 0)
        assert [f["len"] for f in lay.ifaces] == W.quadtree_interface_lengths(nx, ny, B, ref)
        # every face between two different subdomains belongs to exactly one interface
        n_faces = sum(f["len"] for f in lay.ifaces)
        own = lay.owner
        cut = int(np.sum(own[:, 1:] != own[:, :-1]) + np.sum(own[1:, :] != own[:-1, :]))
        assert n_faces == cut


def test_uniform_layout_is_the_uniform_oracle():
    from paper_2104_04653_gb300 import workloads as W2
    rng = np.random.default_rng(2)
    for B in (8, 16):
        K = np.exp(rng.standard_normal((32, 48)))
        uni = W2.make_problem(48, 32, B, K, q=rng.standard_normal((32, 48)),
                              bc=W2.bc_left_right(48, 32), n_u=2, n_p=3)
        qt = W2.quadtree_problem(48, 32, B, K, [np.zeros((32 // B, 48 // B))], q=uni.q,
                                 n_u=2, n_p=3)
        a, b = O.mrcm_solve(uni), Q.mrcm_solve(qt)
        for k in ("p", "ux", "uy"):
            assert np.abs(a[k] - b[k]).max() <= 1e-12 * np.abs(a[k]).max(), k
        for ga, gb in zip(a["gamma_u"][0], b["gamma_u"][0]):
            assert np.abs(ga - gb).max() <= 1e-11 * max(np.abs(ga).max(), 1.0)


@pytest.mark.parametrize("alpha", [0.05, 1.0, 20.0])
def test_full_spaces_equal_the_fine_grid(alpha):
    prob = _mixed(full=True, alpha=alpha)
    fine = O.fine_solve(prob)
    got = Q.mrcm_solve(prob)
    ep, eu = O.errors(got, fine)
    assert ep <= 1e-10 and eu <= 1e-10, (ep, eu)


def test_linear_pressure_is_exact():
    nx, ny, B = 32, 32, 8
    ref = np.zeros((ny // B, nx // B), np.int8)
    ref[1, 1] = ref[2, 3] = ref[0, 0] = 1
    t, v = W.bc_linear_pressure(nx, ny, 1.0 / ny)
    prob = W.quadtree_problem(nx, ny, B, np.full((ny, nx), 3.0), [ref], bc=(t, v))
    got = Q.mrcm_solve(prob)
    x = (np.arange(nx) + 0.5) / ny
    assert np.abs(got["p"][0] - (1.0 - x)[None, :]).max() <= 1e-12
    assert np.abs(got["ux"][0] - 3.0).max() <= 1e-11 and np.abs(got["uy"][0]).max() <= 1e-11


def test_mass_balance_and_interface_flux_balance():
    prob = _mixed(seed=4)
    prob.iface_nU = [np.full_like(prob.iface_nU[0], 2)]
    prob.iface_nP = [np.full_like(prob.iface_nP[0], 3)]
    got = Q.mrcm_solve(prob)
    lay = Q.QLayout(prob, 0)
    h = prob.h
    ux, uy, gam = got["ux"][0], got["uy"][0], got["gamma_u"][0]
    # one-sided velocities on interface faces, the rest as reported
    for k, (x0, y0, s) in enumerate(lay.subs):
        for b in range(s):
            for a in range(s):
                i, j = x0 + a, y0 + b
                out = 0.0
                for key, sign, uval in ((("V", i, j), -1.0, ux[j, i]), (("V", i + 1, j), 1.0, ux[j, i + 1]),
                                        (("H", j, i), -1.0, uy[j, i]), (("H", j + 1, i), 1.0, uy[j + 1, i])):
                    fe = lay.face_if.get(key)
                    if fe is not None and (a in (0, s - 1) or b in (0, s - 1)):
                        g, e = fe
                        f = lay.ifaces[g]
                        mine = 0 if f["L"] == k else 1
                        if f["L"] == k or f["R"] == k:
                            out += gam[g][mine, e] * h
                            continue
                    out += sign * uval * h
                assert abs(out - prob.q[0, j, i] * h * h) <= 1e-11 * (1 + abs(prob.q[0, j, i]) * h * h)
    for g, f in enumerate(lay.ifaces):
        assert abs(np.sum(gam[g][0]) + np.sum(gam[g][1])) <= 1e-10 * (1 + np.abs(gam[g]).sum())


def test_basis_family_invariance():
    a = Q.mrcm_solve(_mixed(seed=5, family="legendre"))
    b = Q.mrcm_solve(_mixed(seed=5, family="monomial"))
    ep, eu = O.errors(a, b)
    assert ep <= 1e-10 and eu <= 1e-10
