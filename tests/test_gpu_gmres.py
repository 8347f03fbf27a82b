"""GPU parity of the GMRES interface path (through the C ABI) against the
FP64 oracle, and its iteration counts against the oracle GMRES.

Tolerance: relative L2 error <= 1e-8 in pressure and face velocities, as for
the direct path; the GMRES stopping test is on the true relative residual
of the interface system.
"""
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
    from oracle import gmres as OG
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm, workloads as W
    return O, OG, mrcm, W


def _opts(prec=1, **kw):
    _, _, mrcm, _ = _mods()
    kw.setdefault("iface_solver", mrcm.IFACE_GMRES)
    return mrcm.SolverOptions(prec=prec, **kw)


def _run(prob, opts, blocks=None):
    import torch
    _, _, mrcm, _ = _mods()
    s = mrcm.Mrcm(prob, opts)
    if blocks is not None:
        s.mrcm_set_precond_blocks(torch.as_tensor(blocks, dtype=torch.float64, device="cuda"))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    p, ux, uy = s.solve(Kd, Ld, Qd)
    info = s.mrcm_get_info()
    out = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy(), info=info,
               gmres=s.uses_gmres(), nprec=s.num_precond_values())
    s.close()
    return out


def _check(prob, opts, ref=None, blocks=None):
    O, _, _, _ = _mods()
    ref = ref if ref is not None else O.mrcm_solve(prob)
    got = _run(prob, opts, blocks)
    ep, eu = O.errors(got, ref)
    assert got["gmres"]
    assert ep <= TOL and eu <= TOL, (prob.name, ep, eu, got["info"])
    assert got["info"]["gmres_iters"] > 0
    assert got["info"]["iface_resid"] <= (opts.gmres_tol or opts.iface_tol)
    return got


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_channels_contrast_1e6(prec):
    """256x64 binary channels, contrast 1e6, m = 8 (the direct path's bench
    workload), solved by block-Jacobi GMRES instead."""
    _, _, _, W = _mods()
    _check(W.config2(), _opts(prec))


def test_gmres_pure_neumann_fivespot():
    """64x64 GRF quarter five-spot: the pinned pressure unknown inside GMRES."""
    _, _, _, W = _mods()
    _check(W.config1(), _opts(1))


def test_gmres_multi_realisation_ragged():
    """Three realisations with ragged per-interface spaces and random alpha:
    each realisation converges on its own CTAs inside one launch."""
    _, _, _, W = _mods()
    nx, ny, R = 80, 48, 3
    rng = np.random.default_rng(12)
    Ks = np.exp(np.sqrt(3.0) * rng.standard_normal((R, ny, nx)))
    prob = W.make_problem(nx, ny, 16, Ks, bc=W.bc_left_right(nx, ny), n_u=2, n_p=2,
                          name="ragged-3x80x48")
    n = prob.n_iface(0)
    prob.iface_nU = [rng.integers(0, 5, n).astype(np.int32) for _ in range(R)]
    prob.iface_nP = [np.maximum(rng.integers(0, 5, n), 1 - u).astype(np.int32)
                     for u in prob.iface_nU]
    prob.alpha = [rng.uniform(0.1, 10.0, (n, 16)) for _ in range(R)]
    prob.q = rng.standard_normal((R, ny, nx))
    _check(prob, _opts(1, gmres_restart=16))


def test_gmres_for_wide_slabs():
    """256x256 lognormal K with Buckley-Leverett mobility, 16x16 subdomains,
    m = 4 (slabs of 124 unknowns) on the GMRES path."""
    _, _, mrcm, W = _mods()
    _check(W.config5(4, n=256), _opts(1))


def _oracle_system(prob):
    O, OG, _, _ = _mods()
    ref = O.mrcm_solve(prob, return_system=True)
    S = ref["systems"][0]
    return ref, S["M"], S["rhs"], OG.diagonal_blocks(S["layout"].ifaces)


@pytest.mark.parametrize("restart", [10, 40])
def test_iteration_count_matches_oracle_gmres(restart):
    """Same operator (up to the basis rounding), preconditioner, restart and
    tolerance: CGS2 on the GPU and MGS in the oracle take the same number
    of steps up to rounding."""
    _, OG, mrcm, W = _mods()
    prob = W.config5(3, n=128)
    ref, M, f, blocks = _oracle_system(prob)
    tol = 1e-10
    _, oi = OG.gmres(M, f, P=OG.block_jacobi(M, blocks), restart=restart, tol=tol)
    got = _check(prob, _opts(1, gmres_restart=restart, gmres_tol=tol), ref=ref)
    n_gpu, n_cpu = got["info"]["gmres_iters"], oi["iters"]
    assert abs(n_gpu - n_cpu) <= max(3, 0.05 * n_cpu), (n_gpu, n_cpu)


def test_unpreconditioned_takes_more_steps():
    _, OG, mrcm, W = _mods()
    prob = W.config5(3, n=64)
    ref, M, f, blocks = _oracle_system(prob)
    bj = _check(prob, _opts(1, gmres_restart=40), ref=ref)
    none = _check(prob, _opts(1, gmres_restart=40, precond=mrcm.PRECOND_NONE), ref=ref)
    _, oi = OG.gmres(M, f, restart=40, tol=1e-13)
    assert none["info"]["gmres_iters"] > bj["info"]["gmres_iters"]
    assert abs(none["info"]["gmres_iters"] - oi["iters"]) <= max(3, 0.05 * oi["iters"])


def _blocks_flat(M, blocks, fn):
    return np.concatenate([fn(M[o:o + m, o:o + m]).reshape(-1) for o, m in blocks])


def test_user_blocks_equal_to_block_jacobi():
    """Caller-supplied blocks that are the exact diagonal-block inverses
    behave as block-Jacobi and never fall back."""
    _, OG, mrcm, W = _mods()
    prob = W.config5(3, n=128)
    ref, M, f, blocks = _oracle_system(prob)
    flat = _blocks_flat(M, blocks, np.linalg.inv)
    bj = _check(prob, _opts(1), ref=ref)
    us = _check(prob, _opts(1, precond=mrcm.PRECOND_USER), ref=ref, blocks=flat)
    assert us["nprec"] == flat.size
    assert not (us["info"]["flags"] & mrcm.FLAG_PRECOND_FALLBACK)
    assert abs(us["info"]["gmres_iters"] - bj["info"]["gmres_iters"]) <= 2


def test_stalled_user_blocks_fall_back_to_block_jacobi():
    """Identity blocks on the contrast-1e6 channels stall (less than 10%
    residual reduction over 10 steps); the solve is rerun with block-Jacobi
    and still meets the tolerance."""
    _, OG, mrcm, W = _mods()
    prob = W.config2()
    ref, M, f, blocks = _oracle_system(prob)
    flat = _blocks_flat(M, blocks, lambda b: np.eye(b.shape[0]))
    got = _check(prob, _opts(1, precond=mrcm.PRECOND_USER), ref=ref, blocks=flat)
    assert got["info"]["flags"] & mrcm.FLAG_PRECOND_FALLBACK
    # the rerun is a fresh block-Jacobi solve: same fields, bit for bit, and
    # the reported count adds the stalled steps to block-Jacobi's
    bj = _run(prob, _opts(1))
    for k in ("p", "ux", "uy"):
        assert np.array_equal(got[k], bj[k]), k
    assert bj["info"]["gmres_iters"] + 10 < got["info"]["gmres_iters"]


def test_user_precond_requires_blocks():
    import torch
    _, _, mrcm, W = _mods()
    prob = W.config5(3, n=64)
    s = mrcm.Mrcm(prob, _opts(1, precond=mrcm.PRECOND_USER))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    s.mrcm_factor_local(Kd, Ld)
    s.mrcm_build_basis(Qd)
    with pytest.raises(mrcm.MrcmError) as e:
        s.mrcm_solve_interface()
    assert e.value.status == mrcm.MRCM_EINVAL
    s.close()
    d = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))      # direct path: no user blocks
    with pytest.raises(mrcm.MrcmError):
        d.mrcm_set_precond_blocks(torch.zeros(d.num_precond_values() or 1,
                                              dtype=torch.float64, device="cuda"))
    d.close()


def test_gmres_graph_replay_matches_eager():
    import torch
    _, _, mrcm, W = _mods()
    prob = W.config5(2, n=128)
    s = mrcm.Mrcm(prob, _opts(1))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    eager = [t.clone() for t in s.solve(Kd, Ld, Qd)]
    out = s.alloc_outputs()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        s.solve(Kd, Ld, Qd, out=out)      # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        s.L.mrcm_set_stream(s.ctx, torch.cuda.current_stream().cuda_stream)
        s.solve(Kd, Ld, Qd, out=out)
    for t in out:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for x, y in zip(eager, out):
        assert torch.equal(x, y)
    s.close()


def test_gmres_is_deterministic_on_a_long_solve():
    """Block-Jacobi GMRES on a 512 x 512 channel system (contrast 1e6,
    32 x 32-cell subdomains, several hundred steps to 1e-8) run in two
    contexts: the same step count and bit-identical fields (every sum is
    taken in a fixed order; no floating-point atomics)."""
    _, _, mrcm, W = _mods()
    prob = W.config4(n=512, s=32, n_ch=16, seed=4001)
    opts = _opts(1, gmres_tol=1e-8, gmres_max=8000)
    a, b = _run(prob, opts), _run(prob, opts)
    assert a["info"]["gmres_iters"] > 100
    assert a["info"]["gmres_iters"] == b["info"]["gmres_iters"]
    for k in ("p", "ux", "uy"):
        assert np.array_equal(a[k], b[k]), k
