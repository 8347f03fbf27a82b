"""GPU parity of the gravity term (mrcm_set_gravity; Eq. "Darcy_wg", the
height along +y) against the FP64 oracle, at relative L2 <= 1e-8 in p and u:
the hydrostatic closed form, heterogeneous fields with both precisions and
both subdomain sizes, the GMRES path and a mixed 16/32 batch."""
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


def _check(prob, prec, **kw):
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm
    ref = O.mrcm_solve(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=prec, **kw))
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    p, ux, uy = s.solve(Kd, Ld, Qd)
    got = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy())
    info = s.mrcm_get_info()
    s.close()
    ep, eu = O.errors(got, ref)
    assert ep <= TOL and eu <= TOL, (prob.name, prec, ep, eu, info)
    return got


def _field(prob, seed):
    rng = np.random.default_rng(seed)
    prob.grav = [K * rng.uniform(0.5, 3.0, K.shape) for K in prob.K]
    return prob


def test_hydrostatic():
    from paper_2104_04653_gb300 import workloads as W
    n = 64
    prob = W.make_problem(n, n, 16, np.full((n, n), 2.0), bc=W.bc_no_flow(n, n), n_u=2, n_p=2,
                          pure_neumann=True)
    prob.grav = [np.full((n, n), 3.0)]
    # the exact flux is zero, so a relative error of u would divide by
    # rounding: p is compared relatively, u absolutely against the size of
    # the gravity velocity K w = 6
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm
    ref = O.mrcm_solve(prob)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=1))
    p, ux, uy = s.solve(*mrcm.device_inputs(prob))
    got = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy())
    s.mrcm_get_info()
    s.close()
    assert O.rel_l2(got["p"], ref["p"]) <= TOL
    scale = 6.0
    assert np.abs(got["ux"]).max() <= TOL * scale and np.abs(got["uy"]).max() <= TOL * scale
    # the closed form: p linear in y with slope w / K = 1.5 (zero mean)
    y = (np.arange(n) + 0.5) / n
    exact = np.broadcast_to((1.5 * (y - y.mean()))[:, None], (n, n))
    assert np.abs(got["p"][0] - exact).max() <= 1e-10 * 1.5


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["fivespot-pure-neumann", "channels-s32", "fronts"])
def test_heterogeneous(case, prec):
    from paper_2104_04653_gb300 import workloads as W
    prob = {"fivespot-pure-neumann": W.config1,
            "channels-s32": lambda: W.config4(n=256, s=32, n_ch=8),
            "fronts": lambda: W.config5(3, n=128)}[case]()
    _check(_field(prob, 5), prec)


def test_gmres_path():
    from paper_2104_04653_gb300 import mrcm, workloads as W
    _check(_field(W.config5(3, n=128), 6), 1, iface_solver=mrcm.IFACE_GMRES)


def test_mixed_sizes():
    from paper_2104_04653_gb300 import workloads as W
    _check(_field(W.config3(n_real=2, n=128), 7), 1)
