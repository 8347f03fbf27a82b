"""The learned interface preconditioner on the GPU: inputs, forward pass,
gradient and training targets against the oracle (oracle/cnn.py), and the
zero network against block-Jacobi."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04653_gb300 import build
    build.build()


def _mods():
    from oracle import cnn as C
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import learned as LP, mrcm, workloads as W
    return C, O, LP, mrcm, W


def _bf16(a):
    import torch
    return torch.as_tensor(a, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()


def _flat(p):
    return np.concatenate([p[k].reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3", "wh",
                                                      "bh")])


def _unflat(v, like):
    out, o = {}, 0
    for k in ("w1", "b1", "w2", "b2", "w3", "b3", "wh", "bh"):
        n = like[k].size
        out[k] = v[o:o + n].reshape(like[k].shape)
        o += n
    return out


def _rounded(p):
    """Parameters as the kernels use them: convolution and head weights
    rounded to BF16, biases FP32."""
    q = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    for k in ("w1", "w2", "w3", "wh"):
        q[k] = _bf16(q[k])
    return q


def _problem():
    _, _, _, _, W = _mods()
    prob = W.config4(n=128, s=32, n_ch=4)
    rng = np.random.default_rng(7)
    prob.lam = rng.uniform(0.3, 1.0, prob.K.shape)
    return prob


def _ctx(prob, precond=None):
    _, _, _, mrcm, _ = _mods()
    opts = mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES,
                              precond=mrcm.PRECOND_USER if precond is None else precond)
    return mrcm.Mrcm(prob, opts)


def test_windows_match_oracle():
    C, O, LP, mrcm, W = _mods()
    prob = _problem()
    s = _ctx(prob)
    K, lam, q = mrcm.device_inputs(prob)
    x = LP.windows(s, K, lam).float().cpu().numpy()
    lay = O.Layout(prob, 0)
    for g in range(len(lay.ifaces)):
        ref = C.window(prob, 0, lay, g)
        np.testing.assert_array_equal(x[g, 1], ref[1])
        np.testing.assert_allclose(x[g, 0], _bf16(ref[0]), rtol=8e-3, atol=1e-6)
    s.close()


def _random_case(m=4, s=16, B=6, seed=3):
    C, _, _, _, _ = _mods()
    rng = np.random.default_rng(seed)
    p = C.init_params(m, seed, s)
    p["wh"] = 0.05 * rng.standard_normal(p["wh"].shape)
    p["bh"] = 0.05 * rng.standard_normal(p["bh"].shape)
    for l in (1, 2, 3):
        p[f"b{l}"] = 0.05 * rng.standard_normal(C.CH)
    x = _bf16(rng.standard_normal((B, 2, 2 * s, 3 * s)))
    x[:, 1] = (x[:, 1] > 0).astype(np.float64)
    t = rng.standard_normal((B, m * m)).astype(np.float32).astype(np.float64)
    return p, x, t


def _net_with(p, m, s):
    import torch
    _, _, LP, _, _ = _mods()
    net = LP.LearnedPrecond(s, m, max_batch=16, seed=1)
    net.set_params(torch.as_tensor(_flat(p), dtype=torch.float32, device="cuda"))
    return net


def test_forward_matches_oracle():
    import torch
    C, _, _, _, _ = _mods()
    p, x, _ = _random_case()
    net = _net_with(p, 4, 16)
    d = net.forward(torch.as_tensor(x, device="cuda").to(torch.bfloat16)).cpu().numpy()
    ref, _ = C.forward(_rounded(p), x)
    err = np.linalg.norm(d - ref) / np.linalg.norm(ref)
    assert err <= 2e-2, err                 # BF16 activations against FP64 ones
    ref16, _ = C.forward(_rounded(p), x, act_round=_bf16)
    err16 = np.linalg.norm(d - ref16) / np.linalg.norm(ref16)
    assert err16 <= 2e-3, err16             # same roundings: accumulation order only
    net.close()


def test_gradient_matches_oracle():
    import torch
    C, _, _, _, _ = _mods()
    p, x, t = _random_case()
    net = _net_with(p, 4, 16)
    loss, g = net.gradient(torch.as_tensor(x, device="cuda").to(torch.bfloat16),
                           torch.as_tensor(t, dtype=torch.float32, device="cuda"))
    # the oracle with the device's BF16 activation storage: what remains is
    # the FP32 accumulation order and the near-ties of BF16 rounding
    rl, rg = C.loss_and_grad(_rounded(p), x, t, act_round=_bf16)
    assert abs(loss - rl) <= 2e-3 * abs(rl)
    gg = _unflat(g.cpu().numpy().astype(np.float64), p)
    for k in rg:
        err = np.linalg.norm(gg[k] - rg[k]) / max(np.linalg.norm(rg[k]), 1e-30)
        assert err <= 1e-2, (k, err)
    # and against the FP64 oracle, within what BF16 activations allow
    _, rg64 = C.loss_and_grad(_rounded(p), x, t)
    for k in rg64:
        err = np.linalg.norm(gg[k] - rg64[k]) / max(np.linalg.norm(rg64[k]), 1e-30)
        assert err <= 1e-1, (k, err)
    net.close()


def test_training_step_matches_oracle_adam():
    import torch
    C, _, _, _, _ = _mods()
    p, x, t = _random_case(seed=4)
    net = _net_with(p, 4, 16)
    xt = torch.as_tensor(x, device="cuda").to(torch.bfloat16)
    net.train_step(xt, torch.as_tensor(t, dtype=torch.float32, device="cuda"), 1e-3)
    after = _unflat(net.get_params().cpu().numpy().astype(np.float64), p)
    _, g = C.loss_and_grad(_rounded(p), x, t, act_round=_bf16)
    for k in g:
        moved = after[k] - p[k].astype(np.float32).astype(np.float64)
        # the first Adam step moves each entry by lr against its gradient's sign
        assert np.abs(moved).max() <= 1.01e-3 + 1e-6, k
        big = np.abs(g[k]) > 0.05 * np.abs(g[k]).max()
        assert np.all(np.sign(moved[big]) == -np.sign(g[k][big])), k
        assert np.all(np.abs(np.abs(moved[big]) - 1e-3) <= 2e-5), k
    net.close()


def test_targets_match_oracle():
    import torch
    C, O, LP, mrcm, W = _mods()
    prob = _problem()
    s = _ctx(prob)
    K, lam, q = mrcm.device_inputs(prob)
    s.mrcm_factor_local(K, lam)
    s.mrcm_build_basis(q)
    t = LP.targets(s, 4).cpu().numpy()
    s.close()
    out = O.mrcm_solve(prob, return_system=True)
    S = out["systems"][0]
    ref = C.targets(S["M"], S["layout"]).reshape(len(S["layout"].ifaces), -1)
    err = np.linalg.norm(t - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


def test_zero_network_is_block_jacobi():
    C, O, LP, mrcm, W = _mods()
    prob = _problem()
    K, lam, q = mrcm.device_inputs(prob)
    bj = _ctx(prob, precond=mrcm.PRECOND_BLOCK_JACOBI)
    bj.solve(K, lam, q)
    it_bj = bj.mrcm_get_info()["gmres_iters"]
    bj.close()
    net = LP.LearnedPrecond(32, 4, max_batch=64, seed=2)
    s = _ctx(prob)
    s.mrcm_factor_local(K, lam)
    s.mrcm_build_basis(q)
    LP.apply(s, net, K, lam)
    s.mrcm_solve_interface()
    out = s.alloc_outputs()
    s.mrcm_reconstruct(*out)
    info = s.mrcm_get_info()
    assert info["gmres_iters"] == it_bj
    assert not (info["flags"] & mrcm.FLAG_PRECOND_FALLBACK)
    ref = O.mrcm_solve(prob)
    got = dict(p=out[0].cpu().numpy(), ux=out[1].cpu().numpy(), uy=out[2].cpu().numpy())
    ep, eu = O.errors(got, ref)
    assert ep <= 1e-8 and eu <= 1e-8
    s.close()
    net.close()


def test_trained_network_gain(capsys):
    """Train on 32 seeded 256^2 channel systems (contrast 1e6, 32 x 32-cell
    subdomains, m = 4), then on a held-out system: the network predicts the
    held-out targets far better than zero (block-Jacobi), the solve with its
    blocks meets the oracle, GMRES needs a small fraction of the steps it
    takes without a preconditioner, and -- the measured relation, which the
    network does not improve on -- no more than 1.3 times block-Jacobi's."""
    import torch
    C, O, LP, mrcm, W = _mods()
    train_p = [W.config4(n=256, s=32, n_ch=8, seed=5000 + k) for k in range(32)]
    x, t = LP.make_dataset(train_p, 4)
    net = LP.LearnedPrecond(32, 4, max_batch=512, seed=0)
    rep = LP.train(net, x, t, steps=800, batch=256, lr=1e-3)
    held = W.config4(n=256, s=32, n_ch=8, seed=4000)
    xv, tv = LP.make_dataset([held], 4)
    w = 1.0 / t.double().var(dim=0).clamp_min(1e-8)
    val, _ = net.gradient(xv, tv)
    zero = float(((tv.double() ** 2) * w).mean())
    assert val < 0.8 * zero, (val, zero)
    K, lam, q = mrcm.device_inputs(held)
    iters = {}
    for name, pc in (("none", mrcm.PRECOND_NONE), ("block_jacobi", mrcm.PRECOND_BLOCK_JACOBI),
                     ("learned", mrcm.PRECOND_USER)):
        s = mrcm.Mrcm(held, mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES,
                                               precond=pc, gmres_tol=1e-12, gmres_max=20000))
        s.mrcm_factor_local(K, lam)
        s.mrcm_build_basis(q)
        if pc == mrcm.PRECOND_USER:
            LP.apply(s, net, K, lam)
        s.mrcm_solve_interface()
        out = s.alloc_outputs()
        s.mrcm_reconstruct(*out)
        info = s.mrcm_get_info(check=False)
        iters[name] = info["gmres_iters"]
        if name == "learned":
            ref = O.mrcm_solve(held)
            got = dict(p=out[0].cpu().numpy(), ux=out[1].cpu().numpy(), uy=out[2].cpu().numpy())
            ep, eu = O.errors(got, ref)
            assert ep <= 1e-8 and eu <= 1e-8, (ep, eu, info)
        s.close()
    with capsys.disabled():
        print(f"\n[learned preconditioner] held-out loss {val:.3f} (zero {zero:.3f}); "
              f"GMRES steps to 1e-12: {iters}")
    # What the trained network does today, asserted as measured: it does
    # NOT beat block-Jacobi (256 against 210 steps on this held-out system;
    # a block-diagonal correction has little to gain here and the network's
    # error spoils it), but its blocks keep GMRES within 1.3 times
    # block-Jacobi's steps and an order of magnitude under no preconditioner.
    # The neighbourhood preconditioner (tests/test_gpu_nbprecond.py) is the
    # form that beats block-Jacobi.
    assert iters["learned"] * 10 <= iters["none"], iters
    assert iters["learned"] <= 1.3 * iters["block_jacobi"], iters
    net.close()


def test_gmres_after_a_training_run_reads_no_stale_memory(monkeypatch):
    """Block-Jacobi GMRES on a 512^2 channel system (32 x 32 subdomains,
    several hundred steps) in a context created before, and in contexts
    created after, a training run that built and destroyed many contexts
    and network buffers: the same step count and the same fields, bit for
    bit, also with the new context's floating-point workspace filled with
    NaN at setup (MRCM_DEBUG_POISON=1).  A read of memory that no step of
    the solve wrote would show up as a different count, a difference in the
    fields, or NaN."""
    import torch
    C, O, LP, mrcm, W = _mods()
    prob = W.config4(n=512, s=32, n_ch=16, seed=4001)
    Kd, Ld, Qd = mrcm.device_inputs(prob)
    opts = mrcm.SolverOptions(prec=1, iface_solver=mrcm.IFACE_GMRES, gmres_tol=1e-8,
                              gmres_max=8000)

    def solve():
        s = mrcm.Mrcm(prob, opts)
        f = [t.clone() for t in s.solve(Kd, Ld, Qd)]
        info = s.mrcm_get_info()
        s.close()
        return f, info

    monkeypatch.setenv("MRCM_DEBUG_POISON", "0")
    before, ib = solve()
    train_p = [W.config4(n=256, s=32, n_ch=8, seed=5100 + k) for k in range(16)]
    x, t = LP.make_dataset(train_p, 4)
    net = LP.LearnedPrecond(32, 4, max_batch=256, seed=1)
    LP.train(net, x, t, steps=50, batch=128, lr=1e-3)
    net.close()
    del x, t
    torch.cuda.synchronize()
    for poison in ("0", "1"):
        monkeypatch.setenv("MRCM_DEBUG_POISON", poison)
        after, ia = solve()
        assert ia == ib, (poison, ib, ia)
        for a, b in zip(before, after):
            assert torch.equal(a, b), poison
    assert ib["gmres_iters"] > 100
