"""GPU parity of the implicit saturation transport and the SI / SFI steps
(include/mrcm_transport.h; Section 4, Eqs. "BL2D_Newton" to
"up_fluxes_impli", the inflection-point trust region of Section 4.1, the SFI
loop of Section 5.4) against the FP64 oracle (oracle/transport.py), through
the C ABI.

Both sides run the same Newton iteration; the linear solves differ (the
oracle's sparse LU, the library's tile-exact block iterations), by rounding
only.  So the Newton counts must be equal and the saturations agree to
1e-10 (absolute, on values in [0, 1]); the SI / SFI steps add the Darcy
solve, compared at the target's 1e-8."""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

S_TOL = 1e-10
TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04653_gb300 import build
    build.build()


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def _gpu_step(s_old, ux, uy, ly, dt, M, eta=1e-6, plain=False, max_newton=100):
    """s_old [R, ny, nx], ux [R, ny, nx+1], uy [R, ny+1, nx] -> s_new, info."""
    import torch
    from paper_2104_04653_gb300 import transport as TP
    R, ny, nx = s_old.shape
    tp = TP.Transport(nx, ny, R, ly, TP.TransportOptions(M=M, eta=eta, plain_newton=plain,
                                                         max_newton=max_newton))
    so = _dev(s_old)
    sn = torch.empty_like(so)
    lam = torch.empty_like(so)
    tp.mrcm_transport_step(dt, _dev(ux), _dev(uy), so, sn, lam)
    info = tp.mrcm_transport_get_info()
    tp.close()
    return sn.cpu().numpy(), lam.cpu().numpy(), info


def _oracle(s_old, ux, uy, h, dt, M, eta=1e-6, plain=False, max_iter=100):
    from oracle import transport as T
    outs, its = [], []
    for r in range(s_old.shape[0]):
        s, it, _ = T.newton_step(s_old[r], ux[r], uy[r], h, dt, M, eta=eta, max_iter=max_iter,
                                 trust_region=not plain)
        outs.append(s)
        its.append(it)
    return np.stack(outs), its


@pytest.mark.parametrize("cfl", [0.5, 5.0, 50.0, 500.0])
def test_one_row_against_oracle(cfl):
    """64 cells in a row, uniform velocity; from the dry state and from the
    state one step later (two realisations)."""
    from oracle import transport as T
    n, M = 64, 10.0
    h = 1.0 / n
    dt = cfl * h
    s0 = np.zeros((1, n))
    s1 = T.newton_step(s0, np.ones((1, n + 1)), np.zeros((2, n)), h, dt, M, max_iter=500)[0]
    s_old = np.stack([s0, s1])
    ux = np.ones((2, 1, n + 1))
    uy = np.zeros((2, 2, n))
    got, lam, info = _gpu_step(s_old, ux, uy, h, dt, M, max_newton=500)
    ref, its = _oracle(s_old, ux, uy, h, dt, M, max_iter=500)
    assert info["newton_iters"] == its, (info, its)
    assert np.abs(got - ref).max() <= S_TOL
    assert np.allclose(lam, got ** 2 + (1 - got) ** 2 / M, rtol=1e-14, atol=0)


def _fine_velocity(K, seed_bc=None):
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    ny, nx = K.shape
    prob = W.make_problem(nx, ny, 16, K, bc=W.bc_left_right(nx, ny), n_u=2, n_p=2)
    ref = O.fine_solve(prob)
    return ref["ux"][0], ref["uy"][0], prob.h


@pytest.mark.parametrize("dt", [2e-3, 2e-2])
def test_lognormal_fine_velocities_two_realisations(dt):
    """64 x 64 lognormal fields, fine-grid Darcy velocities (a potential
    flow), two realisations stepping together, CFL about 10 and 100."""
    from paper_2104_04653_gb300 import workloads as W
    M = 10.0
    vel = []
    for seed in (0, 1):
        K = np.exp(W.grf_exponential(64, 64, 1 / 64, 2.0, 0.1, np.random.default_rng(seed)))
        vel.append(_fine_velocity(K))
    ux = np.stack([v[0] for v in vel])
    uy = np.stack([v[1] for v in vel])
    h = vel[0][2]
    s_old = np.zeros((2, 64, 64))
    got, _, info = _gpu_step(s_old, ux, uy, 1.0, dt, M, max_newton=400)
    ref, its = _oracle(s_old, ux, uy, h, dt, M, max_iter=400)
    assert info["newton_iters"] == its, (info, its)
    assert np.abs(got - ref).max() <= S_TOL
    # second step from there
    got2, _, info2 = _gpu_step(ref, ux, uy, 1.0, dt, M, max_newton=400)
    ref2, its2 = _oracle(ref, ux, uy, h, dt, M, max_iter=400)
    assert info2["newton_iters"] == its2 and np.abs(got2 - ref2).max() <= S_TOL


def _vortex_velocity(nx, ny, h, seed):
    """A discretely divergence-free field with recirculation: uniform flow
    from the left plus the curl of a seeded stream function (face fluxes
    from differences of psi at the cell corners)."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx + 1) * h, np.arange(ny + 1) * h)
    psi = Y.copy()                                       # uniform flow along +x
    for _ in range(3):
        cx, cy = rng.uniform(0.2, 0.8) * nx * h, rng.uniform(0.2, 0.8) * ny * h
        psi += rng.uniform(-0.4, 0.4) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / 0.02)
    psi[0, :] = psi[0, 0]                                # no flow through bottom and top
    psi[-1, :] = psi[-1, 0]
    ux = (psi[1:, :] - psi[:-1, :]) / h                  # [ny, nx+1]
    uy = -(psi[:, 1:] - psi[:, :-1]) / h                 # [ny+1, nx]
    return ux, uy


@pytest.mark.parametrize("shape", [(50, 37), (16, 16), (33, 80)])
def test_ragged_grids_with_recirculation(shape):
    """Grids that are not multiples of the 16-cell tile, and velocities
    with closed streamlines (the upwind graph has cycles)."""
    nx, ny = shape
    M, h = 10.0, 1.0 / ny
    ux, uy = _vortex_velocity(nx, ny, h, seed=nx)
    rng = np.random.default_rng(ny)
    s_old = rng.uniform(0.0, 0.3, (1, ny, nx))
    dt = 3.0 * h / np.abs(ux).max()
    got, _, info = _gpu_step(s_old, ux[None], uy[None], 1.0, dt, M, eta=1e-10, max_newton=300)
    ref, its = _oracle(s_old, ux[None], uy[None], h, dt, M, eta=1e-10, max_iter=300)
    assert info["newton_iters"] == its, (info, its)
    assert np.abs(got - ref).max() <= S_TOL


def test_no_flow_and_plain_newton():
    from paper_2104_04653_gb300 import workloads as W
    rng = np.random.default_rng(5)
    s_old = rng.uniform(0, 1, (1, 20, 24))
    got, _, info = _gpu_step(s_old, np.zeros((1, 20, 25)), np.zeros((1, 21, 24)), 1.0, 3.0, 10.0)
    assert info["newton_iters"] == [1] and np.array_equal(got, s_old)
    # plain Newton (clip only) at a small time step, where it converges
    K = np.exp(W.grf_exponential(32, 32, 1 / 32, 1.0, 0.1, np.random.default_rng(9)))
    ux, uy, h = _fine_velocity(K)
    s0 = np.zeros((1, 32, 32))
    got, _, info = _gpu_step(s0, ux[None], uy[None], 1.0, 0.2 * h, 10.0, plain=True)
    ref, its = _oracle(s0, ux[None], uy[None], h, 0.2 * h, 10.0, plain=True)
    assert info["newton_iters"] == its and np.abs(got - ref).max() <= S_TOL


def test_water_balance_at_full_size():
    """512 x 512 lognormal field (the re-solve workload) with its fine-grid
    Darcy velocities (divergence-free cell by cell), one large step (about
    20 cells of front travel) to a tight Newton tolerance: the change of
    the water volume equals dt times the net boundary inflow (interior
    fluxes cancel) and the saturation stays in [0, 1] without clipping."""
    from oracle import mrcm_oracle as O, transport as T
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config5(1, n=512)
    ref = O.fine_solve(prob)
    ux, uy = ref["ux"], ref["uy"]
    h, M = prob.h, 5.0
    dt = 20 * h / float(np.abs(ux).max())
    s_old = np.asarray(prob.meta["saturation"])[None]
    got, _, info = _gpu_step(s_old, ux, uy, 1.0, dt, M, eta=1e-12, max_newton=500)
    assert info["flags"] == 0
    dv = float(np.sum(got[0] - s_old[0])) * h * h
    out = T.boundary_outflow(got[0], ux[0], uy[0], h, M)
    assert abs(dv + dt * out) <= 1e-9 * dt * abs(out), (dv, dt * out, info)
    H = T.residual(got[0], s_old[0], ux[0], uy[0], h, dt, M)
    assert np.abs(H).max() <= 1e-10


def test_mrcm_velocities_residual_vanishes_where_not_clipped():
    """The same step with the library's own MRCM velocities.  Their
    interface values (the mean of the two one-sided Robin velocities) are
    not divergence-free cell by cell, so the root of H can leave [0, 1] next
    to the inlet and the clip holds it there; every other cell must solve
    its equation, H_I = 0."""
    from oracle import transport as T
    from paper_2104_04653_gb300 import mrcm, workloads as W
    prob = W.config5(1, n=512)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    p, ux, uy = s.solve(*mrcm.device_inputs(prob))
    s.close()
    ux, uy = ux.cpu().numpy(), uy.cpu().numpy()
    h, M = prob.h, 5.0
    dt = 20 * h / float(np.abs(ux).max())
    s_old = np.asarray(prob.meta["saturation"])[None]
    got, _, info = _gpu_step(s_old, ux, uy, 1.0, dt, M, eta=1e-12, max_newton=500)
    assert info["flags"] == 0
    H = T.residual(got[0], s_old[0], ux[0], uy[0], h, dt, M)
    free = (got[0] > 0.0) & (got[0] < 1.0)
    assert np.abs(H[free]).max() <= 1e-10
    assert got.min() >= 0.0 and got.max() <= 1.0


def _lam(s, M, mu_w=1.0):
    return s * s / mu_w + (1 - s) ** 2 / (M * mu_w)


def _oracle_darcy(M):
    from oracle import mrcm_oracle as O

    def darcy(prob, s):
        q = dataclasses.replace(prob, lam=_lam(s, M)[None])
        ref = O.mrcm_solve(q)
        return ref["p"][0], ref["ux"][0], ref["uy"][0]
    return darcy


def _si_problem():
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config5(2, n=128)
    return prob, np.asarray(prob.meta["saturation"])


def test_si_step_against_oracle():
    """mrcm_si_step on the 128 x 128 front workload (lognormal K, M = 5):
    Darcy with lambda(s^n), then the transport; against the oracle's SI step
    on its own MRCM solve."""
    import torch
    from oracle import transport as T
    from paper_2104_04653_gb300 import mrcm, transport as TP
    prob, s0 = _si_problem()
    M = 5.0
    dt = 0.01
    ref_s, ref_it, (rp, rux, ruy) = T.si_step(prob, s0, dt, M, _oracle_darcy(M))
    ctx = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    tp = TP.Transport(prob.nx, prob.ny, 1, prob.ly, TP.TransportOptions(M=M))
    K, _, Q = mrcm.device_inputs(prob)
    lam = _dev(_lam(s0, M)[None])
    so = _dev(s0[None])
    sn = torch.empty_like(so)
    p, ux, uy = ctx.alloc_outputs()
    TP.mrcm_si_step(ctx, tp, dt, K, lam, Q, so, sn, p, ux, uy)
    info = tp.mrcm_transport_get_info()
    ctx.mrcm_get_info()
    from oracle import mrcm_oracle as O
    ep, eu = O.errors(dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy()),
                      dict(p=rp[None], ux=rux[None], uy=ruy[None]))
    assert ep <= TOL and eu <= TOL
    assert info["newton_iters"] == [ref_it]
    assert np.abs(sn.cpu().numpy()[0] - ref_s).max() <= 1e-8
    assert np.allclose(lam.cpu().numpy()[0], _lam(sn.cpu().numpy()[0], M), rtol=1e-14, atol=0)
    tp.close()
    ctx.close()


def test_sfi_step_against_oracle():
    """mrcm_sfi_step: outer Darcy + transport iterations until the largest
    saturation change is below 1e-4 (Section 5.4), against the oracle's SFI
    step; same outer count, same saturation."""
    import torch
    from oracle import transport as T
    from paper_2104_04653_gb300 import mrcm, transport as TP
    prob, s0 = _si_problem()
    M = 5.0
    dt = 0.02
    ref_s, ref_k, ref_its, _ = T.sfi_step(prob, s0, dt, M, _oracle_darcy(M), tol=1e-4)
    ctx = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR))
    tp = TP.Transport(prob.nx, prob.ny, 1, prob.ly, TP.TransportOptions(M=M))
    K, _, Q = mrcm.device_inputs(prob)
    lam = _dev(_lam(s0, M)[None])
    so = _dev(s0[None])
    sn, sw = torch.empty_like(so), torch.empty_like(so)
    p, ux, uy = ctx.alloc_outputs()
    k = TP.mrcm_sfi_step(ctx, tp, dt, 1e-4, 20, K, lam, Q, so, sn, sw, p, ux, uy)
    assert k == ref_k, (k, ref_k, ref_its)
    assert np.abs(sn.cpu().numpy()[0] - ref_s).max() <= 1e-8
    assert k >= 2
    tp.close()
    ctx.close()


def test_bad_arguments_are_refused():
    import torch
    from paper_2104_04653_gb300 import mrcm, transport as TP
    tp = TP.Transport(8, 8, 1)
    x = torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(mrcm.MrcmError) as e:
        tp.mrcm_transport_step(0.1, torch.zeros((1, 8, 9), dtype=torch.float64, device="cuda"),
                               torch.zeros((1, 9, 8), dtype=torch.float64, device="cuda"), x, x)
    assert e.value.status == mrcm.MRCM_EINVAL
    with pytest.raises(mrcm.MrcmError):
        tp.mrcm_transport_step(-1.0, x, x, x, x.clone())
    tp.close()
