"""Why the local factors are FP32 with FP64 refinement and not BF16.

Refinement x += F^{-1} (b - A x) with an approximate factor F contracts the
error by a factor that grows with kappa * u (kappa: condition number of the
Jacobi-scaled local operator, u: the factor's unit roundoff).  On a 32 x 32
subdomain of the contrast-1e6 channels (kappa about 5e3) a Cholesky factor
rounded to FP32 reaches 1e-14 in 3 sweeps; rounded to BF16 it needs 13.  The
factor is rounded after an FP64 factorisation (representation error only),
which favours the low precision: a BF16 factorisation would do worse.  Each
sweep is a full block solve plus an FP64 residual, so BF16's cheaper loads
do not pay for four times the sweeps.
"""
import numpy as np


def _bf16(x):
    """Round FP64 values to BF16 (8 significant bits, nearest even) via FP32."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32)
    lsb = (f >> 16) & 1
    f = ((f + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return f.view(np.float32).astype(np.float64)


def _sweeps(A, b, L, tol=1e-14, cap=30):
    x = np.zeros_like(b)
    for k in range(1, cap + 1):
        r = b - A @ x
        x = x + np.linalg.solve(L.T, np.linalg.solve(L, r))
        if np.linalg.norm(b - A @ x) <= tol * np.linalg.norm(b):
            return k
    return None


def test_bf16_rounding_helper():
    assert _bf16(1.0) == 1.0
    assert _bf16(1.0 + 2.0 ** -8) == 1.0                 # tie: to even
    assert _bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie: to even (up)
    assert _bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7


def test_fp32_factor_refines_and_bf16_does_not():
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config4(n=256, s=32, n_ch=8)
    lay = O.Layout(prob, 0)
    lo = O.Local(prob, 0, lay, 0, 0, prob.lam[0] * prob.K[0])
    A = np.asarray(lo.A.toarray() if hasattr(lo.A, "toarray") else lo.A, dtype=np.float64)
    d = 1.0 / np.sqrt(np.diag(A))
    As = A * d[:, None] * d[None, :]
    kappa = np.linalg.cond(As)
    assert 1e3 < kappa < 1e4
    L = np.linalg.cholesky(As)
    b = np.random.default_rng(0).standard_normal(As.shape[0])
    n32 = _sweeps(As, b, L.astype(np.float32).astype(np.float64))
    n16 = _sweeps(As, b, _bf16(L))
    assert n32 is not None and n32 <= 4, n32
    assert n16 is not None and n16 >= 3 * n32, (n16, n32)
