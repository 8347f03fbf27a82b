"""GPU parity of MRCM on a one-level quadtree (mrcm_desc.refine: 32 x 32
blocks, some split into four 16 x 16 subdomains, interfaces covering half of
a large subdomain's edge) against the quadtree oracle (oracle/quadtree.py),
through the C ABI, at relative L2 <= 1e-8 in p and u; the step-(d) solve is
GMRES (the direct solvers need uniform subdomains)."""
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


def _run(prob, prec, **kw):
    from paper_2104_04653_gb300 import mrcm
    kw.setdefault("gmres_tol", 1e-12)
    kw.setdefault("gmres_max", 20000)
    s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=prec, **kw))
    assert s.interface_path() == "gmres"
    p, ux, uy = s.solve(*mrcm.device_inputs(prob))
    info = s.mrcm_get_info()
    out = dict(p=p.cpu().numpy(), ux=ux.cpu().numpy(), uy=uy.cpu().numpy(), info=info,
               x=s.interface_solution().cpu().numpy())
    s.close()
    return out


def _layout(n, seed, frac=0.4):
    from paper_2104_04653_gb300 import workloads as W
    return W.random_refinement(n, n, 32, frac, np.random.default_rng(seed))


def _prob(n=128, R=2, seed=0, m_choices=None, frac=0.4):
    from paper_2104_04653_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    K = np.stack([np.exp(W.grf_exponential(n, n, 1.0 / n, 2.0, 0.1, rng)) for _ in range(R)])
    refs = [_layout(n, seed + 10 * r, frac) for r in range(R)]
    return W.quadtree_problem(n, n, 32, K, refs, n_u=2, n_p=2, m_choices=m_choices, seed=seed)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["lognormal-2x128", "ragged-m", "channels-256"])
def test_quadtree_matches_oracle(case, prec):
    from oracle import quadtree as Q, mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    if case == "lognormal-2x128":
        prob = _prob()
    elif case == "ragged-m":
        prob = _prob(seed=3, m_choices=[2, 4, 6, 8])
    else:
        K = W.sinusoidal_channels(256, 256, 8, np.random.default_rng(4000), scale=1.0)
        prob = W.quadtree_problem(256, 256, 32, K, [_layout(256, 7, 0.3)])
    ref = Q.mrcm_solve(prob, return_system=True)
    got = _run(prob, prec)
    ep, eu = O.errors(got, ref)
    assert ep <= TOL and eu <= TOL, (case, prec, ep, eu, got["info"])
    xr = np.concatenate([sy["x"] for sy in ref["systems"]])
    assert np.linalg.norm(got["x"] - xr) <= 1e-8 * np.linalg.norm(xr)   # same unknown order


def test_full_spaces_equal_the_fine_grid():
    """As many functions as faces on every interface: MRCM is the fine-grid
    two-point solve, on the GPU too (the oracle: 8e-13).  A checkerboard of split and unsplit
    32 x 32 blocks makes every interface 16 faces long (full spaces of 32
    unknowns, within the GMRES path's limit) with both sizes present."""
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    n = 128
    ref = ((np.arange(4)[:, None] + np.arange(4)[None, :]) % 2).astype(np.int8)
    K = np.exp(W.grf_exponential(n, n, 1.0 / n, 2.0, 0.1, np.random.default_rng(5)))
    prob = W.quadtree_problem(n, n, 32, K, [ref])
    L = W.quadtree_interface_lengths(n, n, 32, ref)
    assert set(L) == {16}
    prob.iface_nU = [np.full(len(L), 16, np.int32)]
    prob.iface_nP = [np.full(len(L), 16, np.int32)]
    # the full space spanned by one unit function per face (caller tables):
    # (p, u) depend on the span only, and this basis keeps the interface
    # system's condition near 4e5 where the sampled Legendre polynomials of
    # degree 15 give 2e12
    prob.iface_fn = [[(np.eye(16), np.eye(16)) for _ in L]]
    got = _run(prob, 0)
    ep, eu = O.errors(got, O.fine_solve(prob))
    assert ep <= 1e-9 and eu <= 1e-9, (ep, eu)


def test_caller_function_tables_and_alpha():
    """Per-interface function tables (mrcm_desc.iface_fn) and per-face
    alpha on a quadtree layout: random smooth functions of each interface's
    own length."""
    from oracle import quadtree as Q, mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = _prob(n=128, R=1, seed=8)
    rng = np.random.default_rng(9)
    L = W.quadtree_interface_lengths(128, 128, 32, prob.refine[0])
    tabs, al = [], []
    for g, l in enumerate(L):
        t = -1.0 + (2.0 * np.arange(l) + 1.0) / l
        nu, npp = int(prob.iface_nU[0][g]), int(prob.iface_nP[0][g])
        phi = np.stack([np.cos((k + rng.uniform(0, 0.5)) * t) for k in range(nu)])
        psi = np.stack([np.ones(l)] + [np.sin((k + 1) * t + rng.uniform()) for k in range(npp - 1)])
        tabs.append((phi, psi))
        al.append(rng.uniform(0.3, 3.0, l))
    prob.iface_fn = [tabs]
    prob.alpha = [al]
    ref = Q.mrcm_solve(prob)
    got = _run(prob, 1)
    ep, eu = O.errors(got, ref)
    assert ep <= TOL and eu <= TOL, (ep, eu)


def test_zero_mask_is_the_uniform_solve_bit_for_bit():
    """A refine mask with no split block is the uniform 32 x 32 layout: the
    same fields, bit for bit, as without a mask (GMRES both)."""
    from paper_2104_04653_gb300 import mrcm, workloads as W
    prob = _prob(n=128, R=1, seed=11)
    uni = W.make_problem(128, 128, 32, prob.K[0], bc=W.bc_left_right(128, 128), n_u=2, n_p=2)
    zero = W.quadtree_problem(128, 128, 32, prob.K[0], [np.zeros((4, 4), np.int8)])
    a = _run(uni, 1, iface_solver=mrcm.IFACE_GMRES)
    b = _run(zero, 1, iface_solver=mrcm.IFACE_GMRES)
    for k in ("p", "ux", "uy"):
        assert np.array_equal(a[k], b[k]), k


def test_shared_neighbourhood_preconditioner():
    """The neighbourhood preconditioner's shared form (interfaces sharing a
    subdomain with g, both halves of a split edge included) on a quadtree
    layout: the oracle's solution, in fewer GMRES steps than block-Jacobi
    (oracle GMRES on a 256^2 quadtree system: 58 against 246 steps)."""
    from oracle import quadtree as Q, mrcm_oracle as O
    from paper_2104_04653_gb300 import mrcm
    prob = _prob(n=256, R=1, seed=12, frac=0.3)
    ref = Q.mrcm_solve(prob)
    bj = _run(prob, 1, gmres_tol=1e-10)
    nb = _run(prob, 1, gmres_tol=1e-10, precond=mrcm.PRECOND_NEIGHBOURHOOD_SHARED)
    ep, eu = O.errors(nb, ref)
    assert ep <= TOL and eu <= TOL, (ep, eu)
    print(f"\n[quadtree 256^2] GMRES steps to 1e-10: block-Jacobi {bj['info']['gmres_iters']}, "
          f"shared neighbourhood {nb['info']['gmres_iters']}")
    assert nb["info"]["gmres_iters"] * 2 <= bj["info"]["gmres_iters"]
