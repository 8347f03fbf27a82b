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
