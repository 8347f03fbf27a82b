"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 error <= 1e-8 in pressure (all cells) and in face
velocities (all faces of ux and uy), per realisation, for both the plain
FP64 path and the FP32 path with FP64 refinement.
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
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm, workloads as W
    return O, mrcm, W


def _run(prob, prec, gamma=False, opts=None):
    import torch
    O, mrcm, W = _mods()
    o = opts or mrcm.SolverOptions(prec=prec)
    s = mrcm.Mrcm(prob, o)
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    g = torch.empty(s.num_gamma_values(), dtype=torch.float64, device="cuda") if gamma else None
    p, ux, uy = s.solve(Kd, Ld, Qd, gamma_u=g)
    info = s.mrcm_get_info()
    out = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy(), info=info,
               x=s.interface_solution().cpu().numpy(), path=s.interface_path())
    if gamma:
        out["gamma"] = g.cpu().numpy()
    s.close()
    return out


def _check(prob, prec, tol=TOL, gamma=True, path=None):
    O, mrcm, W = _mods()
    ref = O.mrcm_solve(prob)
    got = _run(prob, prec, gamma=gamma)
    if path is not None:
        assert got["path"] == path, (got["path"], path)
    ep, eu = O.errors(got, ref)
    assert ep <= tol and eu <= tol, (prob.name, prec, ep, eu, got["info"])
    if gamma:
        ref_g = np.concatenate([g.reshape(-1) for g in ref["gamma_u"]])
        assert O.rel_l2(got["gamma"], ref_g) <= 10 * tol
    return ep, eu, got


PRECS = [0, 1]   # FP64, FP32 + FP64 refinement


@pytest.mark.parametrize("prec", PRECS)
def test_gaussian_fivespot_64(prec):
    """64x64 GRF quarter five-spot (pure Neumann), 4x4 subdomains, m = 4."""
    _, _, W = _mods()
    _check(W.config1(), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_channels_256x64_contrast_1e6(prec):
    """The bench workload: 256x64 binary channels, contrast 1e6, m = 8."""
    _, _, W = _mods()
    ep, eu, got = _check(W.config2(), prec)
    if prec == 1:
        assert got["info"]["local_sweeps_max"] >= 1


@pytest.mark.parametrize("prec", PRECS)
def test_multi_realisation_ragged_spaces(prec):
    """Three realisations, per-interface n_U, n_P in 0..4 (ragged RHS counts
    per subdomain), random alpha per face, non-square grid."""
    O, mrcm, W = _mods()
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
    _check(prob, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(32, 16), (16, 48)])
def test_full_spaces_reproduce_fine_grid(prec, shape):
    """n_U = n_P = s: the CUDA path equals the fine-grid two-point solve
    (slabs of one interface: 32 unknowns)."""
    O, mrcm, W = _mods()
    nx, ny = shape
    rng = np.random.default_rng(3)
    K = np.exp(rng.standard_normal((ny, nx)))
    prob = W.make_problem(nx, ny, 16, K, bc=W.bc_left_right(nx, ny), n_u=16, n_p=16)
    got = _run(prob, prec)
    fine = O.fine_solve(prob)
    ep, eu = O.errors(got, fine)
    assert ep <= TOL and eu <= TOL, (ep, eu, got["info"])


@pytest.mark.parametrize("prec", PRECS)
def test_linear_pressure_exact(prec):
    O, mrcm, W = _mods()
    nx, ny = 64, 32
    h = 1.0 / ny
    prob = W.make_problem(nx, ny, 16, np.full((ny, nx), 3.0),
                          bc=W.bc_linear_pressure(nx, ny, h), n_u=2, n_p=2)
    got = _run(prob, prec)
    xc = (np.arange(nx) + 0.5) * h
    assert np.abs(got["p"][0] - (1 - xc)[None, :]).max() < 1e-10
    assert np.abs(got["ux"][0] - 3.0).max() < 1e-9
    assert np.abs(got["uy"][0]).max() < 1e-9


@pytest.mark.parametrize("shape", [(16, 16), (128, 16), (16, 96), (48, 80)])
def test_edge_shapes(shape):
    """One subdomain (no interface), one subdomain row, one column (slabs
    along y), and more subdomain rows than columns."""
    O, mrcm, W = _mods()
    nx, ny = shape
    rng = np.random.default_rng(nx + ny)
    K = np.exp(rng.standard_normal((ny, nx)))
    prob = W.make_problem(nx, ny, 16, K, bc=W.bc_left_right(nx, ny), n_u=2, n_p=3,
                          name=f"edge-{nx}x{ny}")
    for prec in PRECS:
        _check(prob, prec, gamma=prob.n_iface(0) > 0)


def test_monomial_family_matches_legendre():
    O, mrcm, W = _mods()
    rng = np.random.default_rng(8)
    K = np.exp(rng.standard_normal((32, 64)))
    prob = W.make_problem(64, 32, 16, K, bc=W.bc_left_right(64, 32), n_u=3, n_p=3)
    a = _run(prob, 1)
    prob.basis = "monomial"
    b = _run(prob, 1)
    ep, eu = O.errors(a, dict(p=b["p"], ux=b["ux"], uy=b["uy"]))
    assert ep <= TOL and eu <= TOL


def test_time_stepping_mobility_downsized():
    """Two-phase total mobility from an analytic Buckley-Leverett front on a
    lognormal K (the re-factor workload, downsized to 128x128)."""
    O, mrcm, W = _mods()
    for step in (3, 8):
        prob = W.config5(step, n=128)
        for prec in PRECS:
            _check(prob, prec)


def test_ten_refactor_steps_on_one_context():
    """The re-factor workload as a time-stepping loop: steps 1..10 of the
    Buckley-Leverett mobility (downsized to 128x128) solved on ONE context,
    lambda_k copied into the same device buffer before each step; every
    step meets the oracle of its own lambda."""
    import torch
    O, mrcm, W = _mods()
    probs = [W.config5(k, n=128) for k in range(1, 11)]
    s = mrcm.Mrcm(probs[0], mrcm.SolverOptions(prec=1))
    Kd, Ld, Qd = mrcm.device_inputs(probs[0])
    out = s.alloc_outputs()
    for prob in probs:
        assert np.array_equal(prob.K, probs[0].K)         # only the mobility moves
        Ld.copy_(torch.from_numpy(np.ascontiguousarray(prob.lam)).to("cuda"))
        s.solve(Kd, Ld, Qd, out=out)
        got = dict(p=out[0].cpu().numpy(), ux=out[1].cpu().numpy(), uy=out[2].cpu().numpy())
        ep, eu = O.errors(got, O.mrcm_solve(prob))
        assert ep <= TOL and eu <= TOL, (prob.name, ep, eu)
    s.close()


def test_deterministic_and_refactor():
    """Two solves give bitwise-identical results; re-factoring with a new
    lambda on the same context gives the new solution."""
    import torch
    O, mrcm, W = _mods()
    prob = W.config2()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    a = [t.clone() for t in s.solve(Kd, Ld, Qd)]
    b = [t.clone() for t in s.solve(Kd, Ld, Qd)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    lam2 = torch.full_like(Ld, 0.5)
    c = s.solve(Kd, lam2, Qd)
    prob.lam = np.full_like(prob.lam, 0.5)
    ref = O.mrcm_solve(prob)
    ep, eu = O.errors(dict(p=c[0].cpu().numpy(), ux=c[1].cpu().numpy(), uy=c[2].cpu().numpy()), ref)
    assert ep <= TOL and eu <= TOL
    s.close()


def test_graph_capture_replay_matches_eager():
    import torch
    O, mrcm, W = _mods()
    prob = W.config2()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
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


def test_nan_input_reported():
    import torch
    O, mrcm, W = _mods()
    prob = W.config1()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    Kd[0, 5, 5] = float("nan")
    s.solve(Kd, Ld, Qd)
    with pytest.raises(mrcm.MrcmError) as e:
        s.mrcm_get_info()
    assert e.value.status == mrcm.MRCM_ENAN
    s.close()


def test_calling_order_enforced():
    import torch
    O, mrcm, W = _mods()
    prob = W.config1()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
    p, ux, uy = s.alloc_outputs()
    with pytest.raises(mrcm.MrcmError) as e:
        s.mrcm_reconstruct(p, ux, uy)
    assert e.value.status == mrcm.MRCM_EINVAL
    with pytest.raises(mrcm.MrcmError):
        s.mrcm_build_basis(torch.zeros_like(p))
    s.close()


def test_refinement_limit_reports_stall():
    """With no interface refinement sweep the FP32 path cannot reach 1e-13
    on the 1e6-contrast workload: the status says so (no hang)."""
    O, mrcm, W = _mods()
    prob = W.config2()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1, iface_ir_max=0))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    s.solve(Kd, Ld, Qd)
    info = s.mrcm_get_info(check=False)
    assert info["status"] == "MRCM_ENOCONV"
    s.close()


@pytest.mark.parametrize("path", ["cluster", "multi-kernel"])
def test_interface_paths_agree(path, monkeypatch):
    """The one-launch cluster interface solve and the multi-kernel global
    memory one both meet the tolerance on the bench workload, and the
    context reports the one that ran."""
    O, mrcm, W = _mods()
    if path == "multi-kernel":
        monkeypatch.setenv("MRCM_NO_CLUSTER", "1")
    else:
        monkeypatch.delenv("MRCM_NO_CLUSTER", raising=False)
    _check(W.config2(), 1, path="slab" if path == "multi-kernel" else "cluster")


@pytest.mark.parametrize("case,prec,path", [("channels", 0, "slab"), ("channels", 1, "cluster"),
                                             ("resolve-256", 1, "wide-slab"),
                                             ("single", 1, "none")])
def test_interface_path_query(case, prec, path, monkeypatch):
    """mrcm_interface_path names the step-(d) kernels chosen at setup: FP64
    runs the multi-kernel slab reduction (its tiles do not fit one cluster),
    FP32 the cluster kernel, slabs above 64 unknowns the wide-slab path, and
    a single subdomain has no interface system."""
    import torch
    O, mrcm, W = _mods()
    monkeypatch.delenv("MRCM_NO_CLUSTER", raising=False)
    prob = {"channels": W.config2, "resolve-256": lambda: W.config5(2, n=256),
            "single": lambda: W.make_problem(16, 16, 16, np.ones((16, 16)),
                                             bc=W.bc_left_right(16, 16), n_u=2, n_p=2)}[case]()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=prec))
    assert s.interface_path() == path
    s.close()


@pytest.mark.parametrize("case", ["direct-fp64", "direct-mixed", "mixed-sizes", "wide-slabs",
                                  "gmres"])
def test_workspace_poisoned_with_nan_gives_identical_results(case, monkeypatch):
    """With the floating-point workspace filled with NaN bytes at setup
    (MRCM_DEBUG_POISON=1) every path returns the same fields, bit for bit,
    as with an untouched workspace: no step reads a value that no earlier
    step wrote."""
    import torch
    O, mrcm, W = _mods()
    prob, opts = {
        "direct-fp64": (W.config2(), mrcm.SolverOptions(prec=0)),
        "direct-mixed": (W.config2(), mrcm.SolverOptions(prec=1)),
        "mixed-sizes": (W.config3(n_real=2, n=128), mrcm.SolverOptions(prec=1)),
        "wide-slabs": (W.config5(2, n=256), mrcm.SolverOptions(prec=1)),
        "gmres": (W.config4(n=256, s=32, n_ch=8),
                  mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES, gmres_tol=1e-8)),
    }[case]
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    out = []
    for poison in ("0", "1"):
        monkeypatch.setenv("MRCM_DEBUG_POISON", poison)
        s = mrcm.Mrcm(prob, opts)
        out.append(([t.clone() for t in s.solve(Kd, Ld, Qd)], s.mrcm_get_info()))
        s.close()
    (a, ia), (b, ib) = out
    assert ia == ib
    for x, y in zip(a, b):
        assert torch.equal(x, y)
