"""The allocation-free local solve, against the five-call path.

mrcm_local_solve_noalloc serves callers that cannot call cudaMalloc (code
inside another runtime's memory pool, or a process whose device footprint is
fixed after start-up); its scratch is a fixed array inside the library.  A
problem made of a single 16 x 16 subdomain has no interface, so the MRCM
solution returned by the five-call path (mrcm_setup ... mrcm_reconstruct) is
exactly the local solve: the two entry points must agree.  Two calls in a row
check that nothing stale survives in the shared scratch.  This file sorts
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-8     # the relative L2 tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04653_gb300 import build
    build.build()


def _problem(n, seed):
    from paper_2104_04653_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    s = 16
    K = np.exp(1.5 * rng.standard_normal((n, s, s)))
    lam = rng.uniform(0.3, 1.2, (n, s, s))
    q = rng.standard_normal((n, s, s))
    t = np.zeros(4 * s, np.int8)
    v = np.zeros(4 * s)
    t[:2 * s] = W.BC_DIRICHLET                  # left and right: pressure
    v[:s] = rng.uniform(0.5, 1.5, s)
    v[s:2 * s] = rng.uniform(-0.5, 0.5, s)
    v[2 * s:] = rng.uniform(-0.3, 0.3, 2 * s)   # bottom and top: normal velocity
    prob = W.make_problem(s, s, s, K, lam=lam, q=q, bc=(t, v), name="single-subdomain")
    return prob


def _noalloc_inputs(prob):
    """Cell kappa, boundary-face transmissibilities and right-hand sides of
    the local two-point operator (harmonic faces inside; 2 kappa at a
    prescribed pressure; 0 at a prescribed velocity)."""
    n, s, h = prob.n_real, prob.nx, prob.h
    kap = prob.lam * prob.K
    tface = np.zeros((n, 4, s))
    rhs = prob.q * h * h
    bt, bv = prob.bc_type, prob.bc_val
    edges = {0: (lambda e: (e, 0), 0), 1: (lambda e: (e, s - 1), s),
             2: (lambda e: (0, e), 2 * s), 3: (lambda e: (s - 1, e), 3 * s)}
    for side, (cell, off) in edges.items():
        for e in range(s):
            j, i = cell(e)
            k = off + e
            if bt[k] == 1:
                tface[:, side, e] = 2.0 * kap[:, j, i]
                rhs[:, j, i] += 2.0 * kap[:, j, i] * bv[k]
            else:
                rhs[:, j, i] -= bv[k] * h
    return kap, tface, rhs


def test_noalloc_matches_five_call_path():
    import torch
    from paper_2104_04653_gb300 import mrcm
    for call, (n, seed) in enumerate([(5, 11), (3, 12)]):     # two calls in a row
        prob = _problem(n, seed)
        solver = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
        Kd, Ld, Qd = mrcm.device_inputs(prob)
        p_ref, _, _ = solver.solve(Kd, Ld, Qd)
        solver.mrcm_get_info()
        kap, tface, rhs = _noalloc_inputs(prob)
        kw = dict(dtype=torch.float64, device="cuda")
        x = torch.full((n, 16, 16), float("nan"), **kw)
        mrcm.local_solve_noalloc(torch.as_tensor(kap, **kw), torch.as_tensor(tface, **kw),
                                 torch.as_tensor(rhs, **kw), x)
        torch.cuda.synchronize()
        a, b = x.cpu().numpy(), p_ref.cpu().numpy()
        for r in range(n):
            err = np.linalg.norm(a[r] - b[r]) / np.linalg.norm(b[r])
            assert err <= TOL, (call, r, err)
        solver.close()


def test_noalloc_rejects_oversized_batch():
    import torch
    from paper_2104_04653_gb300 import mrcm
    kw = dict(dtype=torch.float64, device="cuda")
    t = torch.zeros((65, 16, 16), **kw)
    with pytest.raises(mrcm.MrcmError) as e:
        mrcm.local_solve_noalloc(t, torch.zeros((65, 4, 16), **kw), t, t.clone())
    assert e.value.status == mrcm.MRCM_EINVAL
    assert "1..64" in str(e.value)
