"""GPU tests of the neighbourhood preconditioner of the interface GMRES
(MRCM_PRECOND_NEIGHBOURHOOD): column block g of P holds the columns of the
inverse of the interface matrix restricted to g's neighbourhood that belong
to g (restricted additive Schwarz, one subdomain of overlap, Cai and Sarkis
1999), applied on the right.

The solution must match the FP64 oracle to relative L2 <= 1e-8, and the
step count must match the oracle GMRES with the same preconditioner
(oracle/cnn.py neighbourhood_columns) up to rounding."""
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
    from oracle import cnn as C
    from oracle import gmres as OG
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm, workloads as W
    return O, OG, C, mrcm, W


def _run(prob, precond, **kw):
    _, _, _, mrcm, _ = _mods()
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES, precond=precond,
                                           **kw))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    p, ux, uy = s.solve(Kd, Ld, Qd)
    info = s.mrcm_get_info()
    out = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy(), info=info)
    s.close()
    return out


@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("case", ["channels-256-s32", "fronts-128", "fivespot-pure-neumann"])
def test_solution_matches_oracle(case, shared):
    O, OG, C, mrcm, W = _mods()
    prob = {"channels-256-s32": lambda: W.config4(n=256, s=32, n_ch=8),
            "fronts-128": lambda: W.config5(3, n=128),
            "fivespot-pure-neumann": W.config1}[case]()
    ref = O.mrcm_solve(prob)
    got = _run(prob, mrcm.PRECOND_NEIGHBOURHOOD_SHARED if shared else mrcm.PRECOND_NEIGHBOURHOOD)
    ep, eu = O.errors(got, ref)
    assert ep <= TOL and eu <= TOL, (ep, eu, got["info"])
    assert got["info"]["gmres_iters"] > 0


@pytest.mark.parametrize("shared", [False, True])
def test_step_count_matches_oracle_gmres(shared):
    O, OG, C, mrcm, W = _mods()
    prob = W.config4(n=256, s=32, n_ch=8)
    ref = O.mrcm_solve(prob, return_system=True)
    S = ref["systems"][0]
    tol = 1e-10
    _, oi = OG.gmres(S["M"], S["rhs"], P=C.neighbourhood_columns(S["M"], S["layout"], shared),
                     restart=40, tol=tol)
    got = _run(prob, mrcm.PRECOND_NEIGHBOURHOOD_SHARED if shared else mrcm.PRECOND_NEIGHBOURHOOD,
               gmres_restart=40, gmres_tol=tol)
    n_gpu, n_cpu = got["info"]["gmres_iters"], oi["iters"]
    assert abs(n_gpu - n_cpu) <= max(3, 0.05 * n_cpu), (n_gpu, n_cpu)


def test_fewer_steps_than_block_jacobi():
    """512 x 512 channels (contrast 1e6, 32 x 32 subdomains), GMRES to 1e-8."""
    _, _, _, mrcm, W = _mods()
    prob = W.config4(n=512, s=32, n_ch=16, seed=4001)
    bj = _run(prob, mrcm.PRECOND_BLOCK_JACOBI, gmres_tol=1e-8, gmres_max=8000)
    nb = _run(prob, mrcm.PRECOND_NEIGHBOURHOOD, gmres_tol=1e-8, gmres_max=8000)
    assert nb["info"]["gmres_iters"] * 3 < bj["info"]["gmres_iters"], (nb["info"], bj["info"])
    for k in ("p", "ux", "uy"):
        assert np.linalg.norm(nb[k] - bj[k]) <= 1e-6 * np.linalg.norm(bj[k])


def test_setup_refuses_neighbourhoods_above_160_unknowns():
    """The 256 x 64 channels with m = 8 have neighbourhoods of 216 unknowns:
    more than the shared-memory elimination holds."""
    _, _, _, mrcm, W = _mods()
    with pytest.raises(mrcm.MrcmError) as e:
        mrcm.Mrcm(W.config2(), mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES,
                                                  precond=mrcm.PRECOND_NEIGHBOURHOOD))
    assert e.value.status == mrcm.MRCM_EINVAL


def test_shared_form_serves_eight_unknowns_per_interface():
    """The 256 x 64 channels with m = 8 (neighbourhoods of 216 unknowns,
    refused by the full form): the shared form (at most 56 unknowns) solves
    them, and in fewer steps than block-Jacobi."""
    O, _, _, mrcm, W = _mods()
    prob = W.config2()
    ref = O.mrcm_solve(prob)
    got = _run(prob, mrcm.PRECOND_NEIGHBOURHOOD_SHARED)
    bj = _run(prob, mrcm.PRECOND_BLOCK_JACOBI)
    ep, eu = O.errors(got, ref)
    assert ep <= TOL and eu <= TOL, (ep, eu, got["info"])
    assert 2 * got["info"]["gmres_iters"] < bj["info"]["gmres_iters"], (got["info"], bj["info"])
