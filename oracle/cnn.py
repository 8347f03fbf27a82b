"""Plain FP64 forward and backward pass of the learned interface
preconditioner's network, and its training target.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  It shares no code with
the CUDA library.

The paper has no learned component; this network exists only to propose the
block preconditioner of the interface GMRES.  What it computes:

* input: per interface, a 2-channel window of 2s x 3s cells centred on the
  interface in canonical orientation (rows along the interface, columns
  across it, the smaller-index subdomain on the left): channel 0 is
  log10(lambda K) / 3 inside the domain and 0 outside, channel 1 is 1
  inside the domain and 0 outside;
* three 3 x 3 convolutions with stride 2 and zero padding 1, 32 output
  channels each, bias, ReLU;
* a linear map from the whole last feature map (32 x s/4 x 3s/8 values, so
  that positions along the interface stay visible) to m*m outputs, the
  correction Delta_g of the interface's block-Jacobi block:
  P_g = (M_gg)^{-1} (I + Delta_g);
* loss: mean over samples and entries of w_k (Delta_k - target_k)^2, with
  per-entry weights w_k (1 by default; the training driver uses the inverse
  variance of each entry over the training targets, so that every entry is
  fitted relative to its own scale).

The training target of interface g is theta * (M_gg B_g - I), clipped
entrywise to [-2, 2], where B_g is the (g, g) block of the inverse of the
interface matrix restricted to the interfaces whose subdomains lie within
one subdomain of g's two subdomains (Chebyshev distance), and theta = 1/2.
The clip keeps the rare near-singular blocks of high-contrast media (2% of
the targets above 5 in size, some above 100) from dominating the loss.

``neighbourhood_rows`` gives the whole row block of that restricted inverse
instead of its diagonal block: P[g, N(g)] = ((M_N(g))^{-1})[g, :], the rows of
a restricted additive Schwarz preconditioner (Cai and Sarkis, SIAM J. Sci.
Comput. 21, 1999) with one subdomain of overlap.  It is the candidate target
of a network that also proposes the couplings to neighbouring interfaces.

Pinned by ``tests/test_oracle_cnn.py``: central finite differences of the
loss against the analytic gradient, the convolution against a direct
sum, zero head = block-Jacobi, the target against a brute-force
restriction of the dense interface matrix, and the neighbourhood rows
against the full inverse and against the target.
"""
from __future__ import annotations

import numpy as np

CH = 32          # channels of every convolution
THETA = 0.5      # damping of the correction target
CLIP = 2.0       # entrywise bound of the correction target


def n_features(s):
    """Length of the flattened last feature map for subdomain size s."""
    return CH * (2 * s // 8) * (3 * s // 8)


def init_params(m, seed, s=16):
    """He-normal convolution weights, zero biases, zero head (Delta = 0)."""
    rng = np.random.default_rng(seed)
    p = {}
    cin = 2
    for l in (1, 2, 3):
        p[f"w{l}"] = rng.standard_normal((CH, cin, 3, 3)) * np.sqrt(2.0 / (cin * 9))
        p[f"b{l}"] = np.zeros(CH)
        cin = CH
    p["wh"] = np.zeros((m * m, n_features(s)))
    p["bh"] = np.zeros(m * m)
    return p


def conv_s2(x, w, b):
    """3 x 3 convolution, stride 2, zero padding 1: x [B, Cin, H, W] ->
    [B, Cout, H/2, W/2] (H, W even)."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    Ho, Wo = H // 2, W // 2
    out = np.zeros((B, w.shape[0], Ho, Wo))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2]        # [B, C, Ho, Wo]
            out += np.einsum("bchw,oc->bohw", patch, w[:, :, ky, kx])
    return out + b[None, :, None, None]


def conv_s2_backward(x, w, dout):
    """Gradients of conv_s2 w.r.t. x, w and b for upstream dout."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    Ho, Wo = H // 2, W // 2
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2]
            dw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dout, patch)
            dxp[:, :, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2] += np.einsum("bohw,oc->bchw", dout,
                                                                       w[:, :, ky, kx])
    return dxp[:, :, 1:-1, 1:-1], dw, dout.sum(axis=(0, 2, 3))


def forward(p, x, act_round=None):
    """Returns Delta [B, m*m] and the cache of activations.  act_round, if
    given, is applied to every stored activation (to compare with a device
    that keeps activations in a narrower format)."""
    cache = {"a0": x}
    a = x
    for l in (1, 2, 3):
        z = conv_s2(a, p[f"w{l}"], p[f"b{l}"])
        a = np.maximum(z, 0.0)
        if act_round is not None:
            a = act_round(a)
        cache[f"a{l}"] = a
    f = a.reshape(a.shape[0], -1)
    cache["f"] = f
    return f @ p["wh"].T + p["bh"], cache


def loss_and_grad(p, x, target, weights=None, act_round=None):
    """Weighted mean-squared loss and its gradient for every parameter."""
    delta, c = forward(p, x, act_round)
    n = delta.size
    wk = np.ones(delta.shape[1]) if weights is None else np.asarray(weights, np.float64)
    diff = delta - target
    loss = float(np.sum(wk * diff * diff) / n)
    dd = 2.0 * wk * diff / n
    g = {"wh": dd.T @ c["f"], "bh": dd.sum(axis=0)}
    df = dd @ p["wh"]
    da = df.reshape(c["a3"].shape)
    for l in (3, 2, 1):
        dz = da * (c[f"a{l}"] > 0.0)
        dx, g[f"w{l}"], g[f"b{l}"] = conv_s2_backward(c[f"a{l - 1}"], p[f"w{l}"], dz)
        da = dx
    return loss, g


def adam_step(p, g, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) in place; state holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)


# ----------------------------------------------------------------- inputs
def window(prob, r, lay, g):
    """Canonical 2-channel input window of interface g of realisation r."""
    s = lay.s
    f = lay.ifaces[g]
    (IL, JL) = f["L"]
    kap = np.log10(prob.lam[r] * prob.K[r]) / 3.0
    ny, nx = kap.shape
    out = np.zeros((2, 2 * s, 3 * s))
    for a in range(2 * s):            # along the interface
        for c in range(3 * s):        # across it, smaller-index side first
            if f["kind"] == "V":
                y, x = JL * s - s // 2 + a, IL * s - s // 2 + c
            else:
                x, y = IL * s - s // 2 + a, JL * s - s // 2 + c
            if 0 <= x < nx and 0 <= y < ny:
                out[0, a, c] = kap[y, x]
                out[1, a, c] = 1.0
    return out


def neighbourhood(lay, g):
    """Interfaces whose two subdomains include one within Chebyshev
    distance 1 of one of g's two subdomains."""
    cs = [np.array(lay.ifaces[g]["L"]), np.array(lay.ifaces[g]["R"])]
    nb = []
    for h, f in enumerate(lay.ifaces):
        if min(np.abs(a - np.array(b)).max() for a in cs for b in (f["L"], f["R"])) <= 1:
            nb.append(h)
    return nb


def targets(M, lay, theta=THETA, clip=CLIP):
    """theta (M_gg B_g - I), clipped to [-clip, clip], for every interface g
    (see the module text)."""
    out = []
    for g, f in enumerate(lay.ifaces):
        idx = np.concatenate([np.arange(lay.ifaces[h]["off"],
                                        lay.ifaces[h]["off"] + lay.ifaces[h]["nU"] +
                                        lay.ifaces[h]["nP"]) for h in neighbourhood(lay, g)])
        off, m = f["off"], f["nU"] + f["nP"]
        pos = int(np.searchsorted(idx, off))
        Bg = np.linalg.inv(M[np.ix_(idx, idx)])[pos:pos + m, pos:pos + m]
        out.append(np.clip(theta * (M[off:off + m, off:off + m] @ Bg - np.eye(m)), -clip, clip))
    return np.array(out)


def neighbourhood_rows(M, lay):
    """Dense P with P[g, N(g)] = ((M_N(g))^{-1})[g, :] for every interface g,
    N(g) the unknowns of g's neighbourhood (``neighbourhood``), zero
    elsewhere (see the module text)."""
    P = np.zeros_like(M)
    for g, f in enumerate(lay.ifaces):
        idx = np.concatenate([np.arange(lay.ifaces[h]["off"],
                                        lay.ifaces[h]["off"] + lay.ifaces[h]["nU"] +
                                        lay.ifaces[h]["nP"]) for h in neighbourhood(lay, g)])
        off, m = f["off"], f["nU"] + f["nP"]
        pos = int(np.searchsorted(idx, off))
        P[off:off + m, idx] = np.linalg.inv(M[np.ix_(idx, idx)])[pos:pos + m, :]
    return P


def shared_neighbourhood(lay, g):
    """Interfaces that share a subdomain with g (g included), ascending."""
    f = lay.ifaces[g]
    subs = {tuple(f["L"]), tuple(f["R"])}
    return [h for h, fh in enumerate(lay.ifaces) if tuple(fh["L"]) in subs or tuple(fh["R"]) in subs]


def neighbourhood_columns(M, lay, shared=False):
    """Dense P with P[N(g), g] = ((M_N(g))^{-1})[:, g] for every interface g
    (the columns of the restricted inverse that belong to g, placed on the
    rows of g's neighbourhood): the right-preconditioning counterpart of
    ``neighbourhood_rows``, and what the library's neighbourhood
    preconditioner builds.  shared: N(g) = the interfaces that share a
    subdomain with g instead."""
    P = np.zeros_like(M)
    for g, f in enumerate(lay.ifaces):
        nb = shared_neighbourhood(lay, g) if shared else neighbourhood(lay, g)
        idx = np.concatenate([np.arange(lay.ifaces[h]["off"],
                                        lay.ifaces[h]["off"] + lay.ifaces[h]["nU"] +
                                        lay.ifaces[h]["nP"]) for h in nb])
        off, m = f["off"], f["nU"] + f["nP"]
        pos = int(np.searchsorted(idx, off))
        P[idx, off:off + m] = np.linalg.inv(M[np.ix_(idx, idx)])[:, pos:pos + m]
    return P
