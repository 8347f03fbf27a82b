"""Pins of the oracle network (oracle/cnn.py): its gradient against central
finite differences, its convolution against a direct sum, its inputs and
training target against their definitions, and the target's sign and use
through the right-preconditioned GMRES it is meant for."""
import numpy as np
import pytest

from oracle import cnn as C


def _tiny(seed=0, B=3, s=4, m=2):
    rng = np.random.default_rng(seed)
    p = C.init_params(m, seed, s)
    p["wh"] = 0.3 * rng.standard_normal(p["wh"].shape)
    p["bh"] = 0.1 * rng.standard_normal(p["bh"].shape)
    for l in (1, 2, 3):
        p[f"b{l}"] = 0.05 * rng.standard_normal(C.CH)
    x = rng.standard_normal((B, 2, 2 * s, 3 * s))
    t = rng.standard_normal((B, m * m))
    return p, x, t


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 6, 8))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = C.conv_s2(x, w, b)
    ref = np.zeros((2, 4, 3, 4))
    for n in range(2):
        for o in range(4):
            for i in range(3):
                for j in range(4):
                    acc = b[o]
                    for c in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                y, xx = 2 * i + ky - 1, 2 * j + kx - 1
                                if 0 <= y < 6 and 0 <= xx < 8:
                                    acc += w[o, c, ky, kx] * x[n, c, y, xx]
                    ref[n, o, i, j] = acc
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def _fd_check(p, x, t, n_probe=6, h=1e-6, wk=None):
    loss, g = C.loss_and_grad(p, x, t, wk)
    rng = np.random.default_rng(5)
    for k in p:
        flat = p[k].reshape(-1)
        gk = g[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(n_probe, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = C.loss_and_grad(p, x, t, wk)
            flat[idx] = old - h
            lm, _ = C.loss_and_grad(p, x, t, wk)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gk[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, gk[idx])
    return loss


def test_gradient_matches_finite_differences():
    p, x, t = _tiny()
    _fd_check(p, x, t)


def test_weighted_gradient_matches_finite_differences():
    p, x, t = _tiny()
    _fd_check(p, x, t, wk=np.array([0.5, 3.0, 0.01, 10.0]))


def test_planted_bias_gradient_mistake_is_caught(monkeypatch):
    good = C.conv_s2_backward

    def bad(x, w, dout):
        dx, dw, db = good(x, w, dout)
        return dx, dw, 0.5 * db
    monkeypatch.setattr(C, "conv_s2_backward", bad)
    p, x, t = _tiny()
    with pytest.raises(AssertionError):
        _fd_check(p, x, t, n_probe=32)


def test_zero_head_is_block_jacobi():
    p = C.init_params(4, 3, 4)
    x = np.random.default_rng(2).standard_normal((5, 2, 8, 12))
    delta, _ = C.forward(p, x)
    assert np.all(delta == 0.0)


def test_adam_first_step_is_lr_times_sign():
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -4.0, 1e-3])}
    st = {}
    C.adam_step(p, g, st, lr=0.01)
    np.testing.assert_allclose(p["a"], [0.99, -1.99, 2.99], rtol=0, atol=1e-7)


def _system(n=64, s=16, seed=3):
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    K = np.exp(1.5 * rng.standard_normal((n, n)))
    prob = W.make_problem(n, n, s, K, bc=W.bc_left_right(n, n), n_u=2, n_p=2)
    out = O.mrcm_solve(prob, return_system=True)
    S = out["systems"][0]
    return prob, S["M"], S["layout"]


def test_window_is_centred_and_canonical():
    prob, M, lay = _system()
    s = lay.s
    kap = np.log10(prob.lam[0] * prob.K[0]) / 3.0
    for g, f in enumerate(lay.ifaces):
        w = C.window(prob, 0, lay, g)
        IL, JL = f["L"]
        # first cell of L sits at (s/2, s/2); the first cell of R at (s/2, 3s/2)
        y0, x0 = JL * s, IL * s
        assert w[0, s // 2, s // 2] == kap[y0, x0]
        if f["kind"] == "V":
            assert w[0, s // 2, s // 2 + s] == kap[y0, x0 + s]
        else:
            assert w[0, s // 2, s // 2 + s] == kap[y0 + s, x0]
        assert w[1].sum() > 0 and set(np.unique(w[1])) <= {0.0, 1.0}


def test_target_with_whole_domain_neighbourhood():
    # 2 x 2 subdomains: every neighbourhood is the whole interface set, so
    # the restricted inverse is the inverse of M itself
    prob, M, lay = _system(n=32, s=16)
    T = C.targets(M, lay, theta=1.0, clip=np.inf)
    Minv = np.linalg.inv(M)
    for g, f in enumerate(lay.ifaces):
        off, m = f["off"], f["nU"] + f["nP"]
        ref = M[off:off + m, off:off + m] @ Minv[off:off + m, off:off + m] - np.eye(m)
        np.testing.assert_allclose(T[g], ref, atol=1e-10)
    assert np.allclose(C.targets(M, lay), np.clip(0.5 * T, -2.0, 2.0))


@pytest.mark.parametrize("seed", [4000, 4002])
def test_targets_reduce_gmres_steps_and_their_negation_does_not(seed):
    """The training target is useful, and its sign is fixed: on 128 x 128
    channel systems (16 x 16-cell subdomains, m = 4, contrast 1e6) the
    blocks M_gg^{-1} (I + Delta_g) with Delta_g = target need fewer
    right-preconditioned GMRES steps to 1e-8 than block-Jacobi (Delta = 0),
    while Delta_g = -target does not converge within 3,000 steps.  Measured:
    163 / 143 (seed 4000) and 143 / 116 (seed 4002) steps."""
    from oracle import gmres as G, mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config4(n=128, s=16, n_ch=4, seed=seed)
    S = O.mrcm_solve(prob, return_system=True)["systems"][0]
    M, rhs, lay = S["M"], S["rhs"], S["layout"]
    T = C.targets(M, lay)
    blocks = G.diagonal_blocks(lay.ifaces)

    def steps(D):
        P = np.zeros_like(M)
        for (off, m), d in zip(blocks, D):
            sl = slice(off, off + m)
            P[sl, sl] = np.linalg.solve(M[sl, sl], np.eye(m) + d)
        _, info = G.gmres(M, rhs, P=P, tol=1e-8, maxiter=3000)
        return info["iters"] if info["converged"] else None

    bj, learned_exact, negated = steps(0 * T), steps(T), steps(-T)
    assert bj is not None and learned_exact is not None
    assert learned_exact < 0.92 * bj, (learned_exact, bj)
    assert negated is None


def test_neighbourhood_rows_are_the_inverse_on_a_whole_domain_neighbourhood():
    # 2 x 2 subdomains: every neighbourhood is the whole interface set, so
    # the rows are those of M^{-1} (M is not symmetric: a transposed block
    # would fail) and GMRES converges in one step
    from oracle import gmres as G
    prob, M, lay = _system(n=32, s=16)
    assert not np.allclose(M, M.T)
    P = C.neighbourhood_rows(M, lay)
    np.testing.assert_allclose(P, np.linalg.inv(M), atol=1e-9 * np.abs(np.linalg.inv(M)).max())
    b = np.random.default_rng(0).standard_normal(M.shape[0])
    _, info = G.gmres(M, b, P=P, tol=1e-10, maxiter=50)
    assert info["converged"] and info["iters"] == 1


def test_neighbourhood_rows_diagonal_block_is_the_target():
    # the (g, g) block of the rows is the B_g of the training target:
    # M_gg B_g - I = target with theta = 1 and no clip
    prob, M, lay = _system(n=64, s=16)
    P = C.neighbourhood_rows(M, lay)
    T = C.targets(M, lay, theta=1.0, clip=np.inf)
    for g, f in enumerate(lay.ifaces):
        off, m = f["off"], f["nU"] + f["nP"]
        sl = slice(off, off + m)
        np.testing.assert_allclose(M[sl, sl] @ P[sl, sl] - np.eye(m), T[g], atol=1e-9)
    # and every row block reaches no further than the neighbourhood
    for g, f in enumerate(lay.ifaces):
        off, m = f["off"], f["nU"] + f["nP"]
        cols = np.flatnonzero(np.abs(P[off:off + m]).sum(axis=0))
        allowed = np.concatenate([np.arange(lay.ifaces[h]["off"], lay.ifaces[h]["off"] +
                                            lay.ifaces[h]["nU"] + lay.ifaces[h]["nP"])
                                  for h in C.neighbourhood(lay, g)])
        assert set(cols) <= set(allowed)


def test_neighbourhood_rows_cut_gmres_steps_on_channels():
    """On the 128 x 128 channel system (contrast 1e6, seed 4000) the
    neighbourhood rows need under a third of block-Jacobi's GMRES steps to
    1e-8 (measured: 25 against 163); the diagonal block alone saves little
    (136)."""
    from oracle import gmres as G, mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config4(n=128, s=16, n_ch=4, seed=4000)
    S = O.mrcm_solve(prob, return_system=True)["systems"][0]
    M, rhs, lay = S["M"], S["rhs"], S["layout"]
    _, bj = G.gmres(M, rhs, P=G.block_jacobi(M, G.diagonal_blocks(lay.ifaces)), tol=1e-8,
                    maxiter=3000)
    _, ras = G.gmres(M, rhs, P=C.neighbourhood_rows(M, lay), tol=1e-8, maxiter=3000)
    assert bj["converged"] and ras["converged"]
    assert ras["iters"] < bj["iters"] / 3, (ras["iters"], bj["iters"])


def test_neighbourhood_columns_are_the_inverse_on_a_whole_domain_neighbourhood():
    from oracle import gmres as G
    prob, M, lay = _system(n=32, s=16)
    P = C.neighbourhood_columns(M, lay)
    Mi = np.linalg.inv(M)
    np.testing.assert_allclose(P, Mi, atol=1e-9 * np.abs(Mi).max())
    b = np.random.default_rng(1).standard_normal(M.shape[0])
    _, info = G.gmres(M, b, P=P, tol=1e-10, maxiter=50)
    assert info["converged"] and info["iters"] == 1


def test_neighbourhood_columns_diagonal_block_is_the_target():
    prob, M, lay = _system(n=64, s=16)
    P = C.neighbourhood_columns(M, lay)
    T = C.targets(M, lay, theta=1.0, clip=np.inf)
    for g, f in enumerate(lay.ifaces):
        off, m = f["off"], f["nU"] + f["nP"]
        sl = slice(off, off + m)
        np.testing.assert_allclose(M[sl, sl] @ P[sl, sl] - np.eye(m), T[g], atol=1e-9)


def test_shared_neighbourhood_columns_cut_gmres_steps():
    """Only the interfaces sharing a subdomain with g (at most 7): still
    about a quarter of block-Jacobi's steps on the 128^2 channels (measured
    42 against 163; the full neighbourhood 24)."""
    from oracle import gmres as G, mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config4(n=128, s=16, n_ch=4, seed=4000)
    S = O.mrcm_solve(prob, return_system=True)["systems"][0]
    M, rhs, lay = S["M"], S["rhs"], S["layout"]
    assert max(len(C.shared_neighbourhood(lay, g)) for g in range(len(lay.ifaces))) == 7
    _, bj = G.gmres(M, rhs, P=G.block_jacobi(M, G.diagonal_blocks(lay.ifaces)), tol=1e-8,
                    maxiter=3000)
    _, sh = G.gmres(M, rhs, P=C.neighbourhood_columns(M, lay, shared=True), tol=1e-8, maxiter=3000)
    assert sh["converged"] and sh["iters"] * 3 < bj["iters"], (sh["iters"], bj["iters"])
