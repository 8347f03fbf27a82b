"""Failure handling on the GPU, with every fault injected on the host.

- Refinement-stall recovery: a subdomain's stored FP32 inverse Schur blocks are
  rounded to 2 explicit mantissa bits (mrcm_test_degrade_factor), so that its
  mixed-precision refinement stalls on a contrast-1e6 field as a factor of too
  low a precision does.  The same mrcm_build_basis re-factors that subdomain
  in FP64 and solves its columns again; the result meets the FP64 oracle.  With
  the recovery off, or with more stalled subdomains than it has room for, the
  call reports MRCM_EIRSTALL.  A factor rounded to bfloat16 precision (7 bits)
  does not stall there: the refinement converges, in more sweeps.
- Pure-Neumann compatibility: sources that do not balance the boundary outflow
  give MRCM_EINCOMPAT; balanced ones solve.
No case faults, traps or hangs a kernel."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04653_gb300 import build
    build.build()


def _mods():
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm, workloads as W
    return O, mrcm, W


BITS = 2          # mantissa bits of the degraded factor: the refinement stalls


def _degrade(s, sub, bits=BITS):
    L = s.L
    L.mrcm_test_degrade_factor.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
    L.mrcm_test_degrade_factor.restype = ctypes.c_int32
    return L.mrcm_test_degrade_factor(s.ctx, sub, bits)


def _run(s, dev, degrade=(), bits=BITS):
    """The five calls one by one, with the factor of the subdomains in
    `degrade` rounded between factor_local and build_basis."""
    _, mrcm, _ = _mods()
    K, L, Q = dev
    s.mrcm_factor_local(K, L)
    for g in degrade:
        assert _degrade(s, g, bits) == mrcm.MRCM_OK
    s.mrcm_build_basis(Q)
    out = s.alloc_outputs()
    try:
        s.mrcm_solve_interface()
        s.mrcm_reconstruct(*out)
    except mrcm.MrcmError:
        pass
    return out, s.mrcm_get_info(check=False)


def _err(O, out, ref):
    p, ux, uy = out
    ep, eu = O.errors(dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy()), ref)
    return max(ep, eu)


def _channels32():
    _, _, W = _mods()
    return W.config4(n=128, s=32, n_ch=4)      # contrast 1e6, 4 x 4 subdomains of 32 x 32


def test_degraded_factor_is_recovered_in_fp64():
    O, mrcm, W = _mods()
    prob = _channels32()
    ref = O.mrcm_solve(prob)
    dev = mrcm.device_inputs(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    out, info = _run(s, dev, degrade=(5,))
    assert info["status"] == "MRCM_OK", info
    assert info["flags"] & mrcm.FLAG_LOCAL_REFACTOR and info["local_refactored"] == 1, info
    assert not info["flags"] & mrcm.FLAG_LOCAL_STALL
    assert _err(O, out, ref) <= TOL
    # the next factorisation starts a new list: a clean solve recovers nothing
    out, info = _run(s, dev)
    assert info["status"] == "MRCM_OK" and info["local_refactored"] == 0, info
    assert not info["flags"] & mrcm.FLAG_LOCAL_REFACTOR
    assert _err(O, out, ref) <= TOL
    # build_basis again on the same factorisation (a degraded one): the listed
    # subdomain is solved again in FP64 each time
    K, L, Q = dev
    s.mrcm_factor_local(K, L)
    assert _degrade(s, 9) == mrcm.MRCM_OK
    for _ in range(2):
        s.mrcm_build_basis(Q)
        s.mrcm_solve_interface()
        out = s.alloc_outputs()
        s.mrcm_reconstruct(*out)
        info = s.mrcm_get_info()
        assert info["local_refactored"] == 1
        assert _err(O, out, ref) <= TOL
    s.close()


def test_bfloat16_factor_converges_without_recovery():
    """The refinement takes a factor accurate to bfloat16 precision as a
    preconditioner: more sweeps (3 with the FP32 factor), no stall."""
    O, mrcm, W = _mods()
    prob = _channels32()
    dev = mrcm.device_inputs(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    out, info = _run(s, dev, degrade=(5,), bits=7)
    assert info["status"] == "MRCM_OK" and info["local_refactored"] == 0, info
    assert info["local_sweeps_max"] > 5, info
    assert _err(O, out, O.mrcm_solve(prob)) <= TOL
    _, info0 = _run(s, dev)
    assert info0["local_sweeps_max"] <= 4, info0
    s.close()


def test_stall_without_recovery_is_reported():
    O, mrcm, W = _mods()
    prob = _channels32()
    dev = mrcm.device_inputs(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, ir_recover=-1))
    _, info = _run(s, dev, degrade=(5,))
    assert info["status"] == "MRCM_EIRSTALL", info
    assert info["flags"] & mrcm.FLAG_LOCAL_STALL and info["local_refactored"] == 0
    assert info["local_resid_max"] > 1e3 * 1e-13
    # the context is still usable: a clean factorisation solves
    out, info = _run(s, dev)
    assert info["status"] == "MRCM_OK", info
    assert _err(O, out, O.mrcm_solve(prob)) <= TOL
    s.close()


def test_more_stalls_than_recovery_slots():
    O, mrcm, W = _mods()
    prob = _channels32()
    dev = mrcm.device_inputs(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, ir_recover=1))
    _, info = _run(s, dev, degrade=(5, 10))
    assert info["status"] == "MRCM_EIRSTALL", info
    assert info["local_refactored"] == 1 and info["flags"] & mrcm.FLAG_LOCAL_STALL
    s.close()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, ir_recover=2))
    out, info = _run(s, dev, degrade=(5, 10))
    assert info["status"] == "MRCM_OK" and info["local_refactored"] == 2, info
    assert _err(O, out, O.mrcm_solve(prob)) <= TOL
    s.close()


def test_recovery_of_16x16_subdomains():
    """More 16 x 16 subdomains than two per SM: their FP32 factor is stored
    (not formed inside the basis kernel), so it can be degraded; the recovery
    then runs the s = 16 FP64 basis kernel."""
    O, mrcm, W = _mods()
    prob = W.config4(n=320, s=16, n_ch=10)     # 400 subdomains
    ref = O.mrcm_solve(prob)
    dev = mrcm.device_inputs(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    out, info = _run(s, dev, degrade=(37, 211))
    assert info["status"] == "MRCM_OK", info
    assert info["local_refactored"] == 2, info
    assert _err(O, out, ref) <= TOL
    s.close()


def test_mixed_sizes_recovery():
    """A batch with 16 x 16 and 32 x 32 realisations: a 32 x 32 subdomain is
    degraded; both FP64 basis kernels run (the s = 16 one finds only empty
    items)."""
    O, mrcm, W = _mods()
    prob = W.config3(n_real=2, n=64)
    ref = O.mrcm_solve(prob)
    dev = mrcm.device_inputs(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    sizes = [16] * 16 + [32] * 4                    # realisation 0: s = 16, 1: s = 32
    assert prob.sub_size[0] == 16 and prob.sub_size[1] == 32
    g32 = sizes.index(32) + 1
    out, info = _run(s, dev, degrade=(g32,))
    assert info["status"] == "MRCM_OK", info
    assert info["local_refactored"] == 1, info
    assert _err(O, out, ref) <= TOL
    s.close()


def test_degrade_hook_refusals():
    O, mrcm, W = _mods()
    prob = W.config2()                               # 64 subdomains of 16 x 16: fused factor
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    K, L, Q = mrcm.device_inputs(prob)
    s.mrcm_factor_local(K, L)
    assert _degrade(s, 3) == mrcm.MRCM_EINVAL      # the basis kernel forms it
    assert _degrade(s, -1) == mrcm.MRCM_EINVAL
    assert _degrade(s, 64) == mrcm.MRCM_EINVAL
    s.close()
    prob = _channels32()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    assert _degrade(s, 0, 0) == mrcm.MRCM_EINVAL
    assert _degrade(s, 0, 23) == mrcm.MRCM_EINVAL
    s.close()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP64))
    assert _degrade(s, 0) == mrcm.MRCM_EINVAL
    s.close()


def test_recovery_changes_nothing_when_nothing_stalls():
    """The recovery launches are always in the call; with no stall they leave
    every output bit for bit as a context without recovery gives."""
    O, mrcm, W = _mods()
    for prob in (W.config2(), _channels32(), W.config3(n_real=2, n=64)):
        dev = mrcm.device_inputs(prob)
        outs = []
        for rec in (0, -1):
            s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, ir_recover=rec))
            p, ux, uy = s.solve(*dev)
            info = s.mrcm_get_info()
            assert info["local_refactored"] == 0
            outs.append([t.cpu().numpy() for t in (p, ux, uy)])
            s.close()
        for a, b in zip(*outs):
            assert np.array_equal(a, b)


def test_pure_neumann_incompatible_sources():
    O, mrcm, W = _mods()
    rng = np.random.default_rng(23)
    n = 64
    K = np.exp(rng.standard_normal((n, n)))
    q = W.five_spot_sources(n, n, 1.0 / n)
    bal = W.make_problem(n, n, 16, K, q=q, bc=W.bc_no_flow(n, n), n_u=2, n_p=2,
                         pure_neumann=True, name="fivespot-balanced")
    q_bad = q.copy()
    q_bad[n // 2, n // 2] += 0.5 / (1.0 / n) ** 2   # an extra half-unit source
    bad = W.make_problem(n, n, 16, K, q=q_bad, bc=W.bc_no_flow(n, n), n_u=2, n_p=2,
                         pure_neumann=True, name="fivespot-unbalanced")
    # a boundary outflow that the sources do not feed
    bt, bv = W.bc_no_flow(n, n)
    bv = bv.copy()
    bv[:n] = 1e-3
    bad_bc = W.make_problem(n, n, 16, K, q=q, bc=(bt, bv), n_u=2, n_p=2,
                            pure_neumann=True, name="fivespot-outflow")
    for prec in (mrcm.PREC_FP64, mrcm.PREC_FP32_IR):
        s = mrcm.Mrcm(bal, mrcm.SolverOptions(prec=prec))
        s.solve(*mrcm.device_inputs(bal))
        assert s.mrcm_get_info()["status"] == "MRCM_OK"
        s.close()
        for prob in (bad, bad_bc):
            s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=prec))
            dev = mrcm.device_inputs(prob)
            try:
                s.solve(*dev)
            except mrcm.MrcmError as e:      # a call may already report it
                assert e.status == mrcm.MRCM_EINCOMPAT
            with pytest.raises(mrcm.MrcmError) as ei:
                s.mrcm_get_info()
            assert ei.value.status == mrcm.MRCM_EINCOMPAT
            info = s.mrcm_get_info(check=False)
            assert info["status"] == "MRCM_EINCOMPAT" and info["flags"] & mrcm.FLAG_INCOMPATIBLE
            s.close()
