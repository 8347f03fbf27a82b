"""GPU parity with 32 x 32-cell subdomains, alone and mixed with 16 x 16
ones in one batch, against the FP64 oracle (relative L2 <= 1e-8)."""
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


def _check(prob, opts):
    O, mrcm, W = _mods()
    ref = O.mrcm_solve(prob)
    s = mrcm.Mrcm(prob, opts)
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    p, ux, uy = s.solve(Kd, Ld, Qd)
    info = s.mrcm_get_info()
    got = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy())
    s.close()
    worst = 0.0
    for r in range(prob.n_real):
        one = {k: v[r:r + 1] for k, v in got.items()}
        rr = {k: ref[k][r:r + 1] for k in ("p", "ux", "uy")}
        ep, eu = O.errors(one, rr)
        worst = max(worst, ep, eu)
    assert worst <= TOL, (prob.name, worst, info)
    return info


@pytest.mark.parametrize("prec", [0, 1])
def test_s32_lognormal(prec):
    O, mrcm, W = _mods()
    rng = np.random.default_rng(21)
    K = np.exp(np.sqrt(2.0) * rng.standard_normal((64, 96)))
    prob = W.make_problem(96, 64, 32, K, bc=W.bc_left_right(96, 64), n_u=2, n_p=2,
                          name="lognormal-96x64-s32")
    _check(prob, mrcm.SolverOptions(prec=prec))


def test_s32_pure_neumann_fivespot():
    O, mrcm, W = _mods()
    rng = np.random.default_rng(22)
    n = 64
    K = np.exp(rng.standard_normal((n, n)))
    prob = W.make_problem(n, n, 32, K, q=W.five_spot_sources(n, n, 1.0 / n),
                          bc=W.bc_no_flow(n, n), n_u=2, n_p=2, pure_neumann=True)
    _check(prob, mrcm.SolverOptions(prec=1))


@pytest.mark.parametrize("prec", [0, 1])
def test_channels_s32_contrast_1e6(prec):
    """The 2048^2 channel workload's generator at 256^2 (8 x 8 subdomains of
    32 x 32 cells, m = 4, contrast 1e6)."""
    O, mrcm, W = _mods()
    _check(W.config4(n=256, s=32, n_ch=8), mrcm.SolverOptions(prec=prec))


def test_channels_s32_gmres():
    O, mrcm, W = _mods()
    info = _check(W.config4(n=256, s=32, n_ch=8),
                  mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES))
    assert info["gmres_iters"] > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_sizes_ragged_spaces_one_batch(prec):
    """The 32-realisation 1024^2 batch's generator at 2 x 128^2: one
    realisation with 16 x 16 and one with 32 x 32 subdomains, interface
    sizes drawn from {2, 4, 6, 8}, lognormal variance 3, in one launch."""
    O, mrcm, W = _mods()
    _check(W.config3(n_real=2, n=128), mrcm.SolverOptions(prec=prec))


def test_mixed_sizes_gmres():
    O, mrcm, W = _mods()
    info = _check(W.config3(n_real=4, n=128),
                  mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES, gmres_restart=30))
    assert info["gmres_iters"] > 0


def test_linear_pressure_mixed_sizes_exact():
    O, mrcm, W = _mods()
    import torch
    nx = ny = 64
    h = 1.0 / ny
    prob = W.make_problem(nx, ny, [16, 32], np.full((2, ny, nx), 0.7),
                          bc=W.bc_linear_pressure(nx, ny, h), n_u=2, n_p=2)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
    p, ux, uy = s.solve(*mrcm.device_inputs(prob))
    xc = (np.arange(nx) + 0.5) * h
    np.testing.assert_allclose(p.cpu().numpy(), np.broadcast_to(1.0 - xc, (2, ny, nx)), atol=1e-11)
    np.testing.assert_allclose(ux.cpu().numpy(), 0.7, rtol=1e-10)
    np.testing.assert_allclose(uy.cpu().numpy(), 0.0, atol=1e-10)
    s.close()


@pytest.mark.parametrize("path", ["cluster", "multi-kernel"])
def test_mixed_sizes_direct_paths(path, monkeypatch):
    """16 x 16 and 32 x 32 subdomains in one batch on the direct interface
    path: the realisation with fewer slabs is padded with empty slabs."""
    O, mrcm, W = _mods()
    if path == "multi-kernel":
        monkeypatch.setenv("MRCM_NO_CLUSTER", "1")
    prob = W.config3(n_real=2, n=64)
    opts = mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_DIRECT)
    info = _check(prob, opts)
    assert info["gmres_iters"] == 0


@pytest.mark.parametrize("case", ["s16", "s32", "mixed"])
def test_every_basis_width_and_autotune(case):
    """The basis kernels' tile widths (RHS columns per CTA) change the time,
    not the result: every width meets the oracle, and the autotuner returns
    one of them and leaves a context that still does."""
    O, mrcm, W = _mods()
    prob = {"s16": lambda: W.config2(), "s32": lambda: W.config4(n=256, s=32, n_ch=8),
            "mixed": lambda: W.config3(n_real=2, n=64)}[case]()
    ref = O.mrcm_solve(prob)
    K, L, Q = mrcm.device_inputs(prob)
    widths = [(w, 8) for w in (4, 8, 12, 16)] + [(12, 4), (12, 16)]
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
    for w16, w32 in widths:
        s.mrcm_set_basis_width(w16, w32)
        p, ux, uy = s.solve(K, L, Q)
        ep, eu = O.errors(dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy()), ref)
        assert ep <= TOL and eu <= TOL, (case, w16, w32, ep, eu)
    c16, c32 = s.mrcm_autotune(K, L, Q, reps=2)
    assert c16 in (4, 8, 12, 16) and c32 in (4, 8, 16)
    p, ux, uy = s.solve(K, L, Q)
    ep, eu = O.errors(dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy()), ref)
    assert ep <= TOL and eu <= TOL
    s.close()
    # the FP64 path has widths 4 and 8 for s = 32 only
    s64 = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP64))
    with pytest.raises(RuntimeError):
        s64.mrcm_set_basis_width(12, 16)
    s64.mrcm_set_basis_width(12, 8)
    s64.close()
