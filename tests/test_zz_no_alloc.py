"""The allocation-free local solve, against the five-call path.

mrcm_local_solve_noalloc serves callers that cannot call cudaMalloc (code
inside another runtime's memory pool, or a process whose device footprint is
fixed after start-up); its scratch is a fixed array inside the library.  A
problem made of a single 16 x 16 subdomain has no interface, so the MRCM
solution returned by the five-call path (mrcm_setup ... mrcm_reconstruct) is
exactly the local solve: the entry point must agree with it and with the
oracle's local solve.  Calls in a row of 3, 64 (the array's limit) and 1
subdomains check that nothing stale survives in the shared scratch, and the
device's free memory is unchanged across them.  This file sorts
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


def _oracle_local(prob):
    """The oracle's local solve of every 16 x 16 subdomain (one per
    realisation): the Robin-free local operator of Eq. "mrc1" with the
    physical boundary data, by Cholesky."""
    from oracle import mrcm_oracle as O
    out = []
    for r in range(prob.n_real):
        lay = O.Layout(prob, r)
        lo = O.Local(prob, r, lay, 0, 0, prob.lam[r] * prob.K[r])
        out.append(O.solve_local(lo.A, lo.b0[:, None])[:, 0].reshape(16, 16))
    return np.stack(out)


def test_noalloc_matches_oracle_and_five_call_path_without_allocating():
    """Three calls in a row (3, then 64 -- the size of the shared array --
    then 1 subdomain) against the oracle's local solve and the five-call
    path.  The second call is larger than the first, so stale scratch from
    the first would reach its output if the kernel read before writing.
    The device's free memory is the same before and after the three calls
    (measured after one set-up call, which looks up the array's address)."""
    import torch
    from paper_2104_04653_gb300 import mrcm
    kw = dict(dtype=torch.float64, device="cuda")
    cases = [(3, 12), (64, 13), (1, 14)]
    probs = [_problem(n, seed) for n, seed in cases]
    ins = []
    for prob in probs:
        kap, tface, rhs = _noalloc_inputs(prob)
        ins.append((torch.as_tensor(kap, **kw), torch.as_tensor(tface, **kw),
                    torch.as_tensor(rhs, **kw),
                    torch.full((prob.n_real, 16, 16), float("nan"), **kw)))
    # set-up call (first call on the device), then the measured calls
    warm = torch.empty_like(ins[0][3])
    mrcm.local_solve_noalloc(ins[0][0], ins[0][1], ins[0][2], warm)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for kap, tface, rhs, x in ins:
        mrcm.local_solve_noalloc(kap, tface, rhs, x)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    for call, (prob, (_, _, _, x)) in enumerate(zip(probs, ins)):
        got = x.cpu().numpy()
        ora = _oracle_local(prob)
        solver = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
        p_ref, _, _ = solver.solve(*mrcm.device_inputs(prob))
        solver.mrcm_get_info()
        five = p_ref.cpu().numpy()
        solver.close()
        for r in range(prob.n_real):
            e_o = np.linalg.norm(got[r] - ora[r]) / np.linalg.norm(ora[r])
            e_f = np.linalg.norm(got[r] - five[r]) / np.linalg.norm(five[r])
            assert e_o <= TOL and e_f <= TOL, (call, r, e_o, e_f)


def test_noalloc_rejects_oversized_batch():
    import torch
    from paper_2104_04653_gb300 import mrcm
    kw = dict(dtype=torch.float64, device="cuda")
    t = torch.zeros((65, 16, 16), **kw)
    with pytest.raises(mrcm.MrcmError) as e:
        mrcm.local_solve_noalloc(t, torch.zeros((65, 4, 16), **kw), t, t.clone())
    assert e.value.status == mrcm.MRCM_EINVAL
    assert "1..64" in str(e.value)
