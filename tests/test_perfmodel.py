"""The algorithmic work behind the bench's roofline numbers
(paper_2104_04653_gb300/perfmodel.py), recounted by hand on a 32 x 32 grid
of four 16 x 16-cell subdomains with m = 4 unknowns on each of its four
interfaces."""
import numpy as np


def _prob():
    from paper_2104_04653_gb300 import workloads as W
    n = 32
    return W.make_problem(n, n, 16, np.ones((n, n)), bc=W.bc_left_right(n, n), n_u=2, n_p=2)


def test_counts_by_hand():
    from paper_2104_04653_gb300 import perfmodel as PM
    prob = _prob()
    s, nsub, cols = 16, 4, 9            # every subdomain: 1 particular + 2 interfaces x 4
    f = PM.call_work("factor_local", prob)
    assert f["flops"] == 2.0 * nsub * s ** 4
    b = PM.call_work("build_basis", prob)
    assert b["flops"] == 1 * 2.0 * (2 * s - 1) * s * s * (nsub * cols)
    # two slabs of 12 and 4 unknowns (b = 12): one eliminated slab (inverse),
    # one survivor with a right neighbour (three products), the root
    # inverse; one FP64 residual sweep over 4 interfaces x 4 rows x 16 terms
    i = PM.call_work("solve_interface", prob)
    bb = 12
    assert i["flops_fp32"] == 2.0 * bb ** 3 + 3 * 2.0 * bb ** 3 + 2.0 * bb ** 3
    assert i["flops_fp64"] == 2.0 * 4 * 4 * 16
    r = PM.call_work("reconstruct", prob)
    assert r["bytes"] == nsub * cols * s * s * 8 + 32 * 32 * 8 * 3


def test_survey_counts_by_hand():
    """The scope table's own counts: factor s^4 per subdomain, solve 4 n s
    per RHS per sweep, 40 B per cell, 7 m^2 x 12 B per interface."""
    from paper_2104_04653_gb300 import perfmodel as PM
    prob = _prob()
    s, nsub, cols = 16, 4, 9
    w = PM.survey_work(prob)
    assert w["factor_flops"] == nsub * s ** 4
    assert w["solve_flops"] == 4.0 * s * s * s * nsub * cols
    assert w["path_bytes"] == 40.0 * 32 * 32
    assert w["iface_spmv_bytes"] == 4 * 7 * 16 * 12


def test_mixed_sizes_count_each_realisation_with_its_own_size():
    """A batch of one 16 x 16-cell and one 32 x 32-cell realisation on a
    64 x 64 grid, m = 4 everywhere: 16 subdomains of s = 16 and 4 of
    s = 32, each counted with its own size."""
    from paper_2104_04653_gb300 import perfmodel as PM, workloads as W
    n = 64
    p16 = W.make_problem(n, n, 16, np.ones((n, n)), bc=W.bc_left_right(n, n), n_u=2, n_p=2)
    p32 = W.make_problem(n, n, 32, np.ones((n, n)), bc=W.bc_left_right(n, n), n_u=2, n_p=2)
    both = W.Problem(nx=n, ny=n, ly=1.0, sub_size=[16, 32], K=np.ones((2, n, n)),
                     lam=np.ones((2, n, n)), q=np.zeros((2, n, n)), bc_type=p16.bc_type,
                     bc_val=p16.bc_val, iface_nU=p16.iface_nU + p32.iface_nU,
                     iface_nP=p16.iface_nP + p32.iface_nP)
    f = PM.call_work("factor_local", both)
    assert f["flops"] == 16 * 2.0 * 16 ** 4 + 4 * 2.0 * 32 ** 4
    assert f["kernel"] == "k_factor + k_factor_warp"
    # basis columns: 4x4 grid: corners 2 edges, sides 3, inside 4 (x 4 + 1);
    # 2x2 grid: every subdomain 2 edges
    c16 = 4 * 9 + 8 * 13 + 4 * 17
    c32 = 4 * 9
    b = PM.call_work("build_basis", both)
    assert b["flops"] == 2.0 * 31 * 256 * c16 + 2.0 * 63 * 1024 * c32
    w = PM.survey_work(both)
    assert w["factor_flops"] == 16 * 16 ** 4 + 4 * 32 ** 4
    assert w["solve_flops"] == 4.0 * 16 ** 3 * c16 + 4.0 * 32 ** 3 * c32
