"""ctypes binding of the learned interface preconditioner
(include/mrcm_learned.h) and its training driver.

Argument marshalling and the training loop only: windows, targets, the
network's forward and backward passes, Adam and the installation of the
blocks all run in the CUDA kernels of ``libmrcm.so``.  Interface systems
for training come from the library's own MRCM path (factor, basis) on
seeded synthetic permeability fields.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import mrcm as _m

EXPORTED = ["mrcm_lp_create", "mrcm_lp_destroy", "mrcm_lp_last_error", "mrcm_lp_set_stream",
            "mrcm_lp_num_params", "mrcm_lp_input_size", "mrcm_lp_set_params",
            "mrcm_lp_get_params", "mrcm_lp_set_loss_weights", "mrcm_lp_forward",
            "mrcm_lp_gradient", "mrcm_lp_train_step", "mrcm_lp_num_samples", "mrcm_lp_windows", "mrcm_lp_targets", "mrcm_lp_apply"]

_bound = False


def lib():
    global _bound
    L = _m.lib()
    if not _bound:
        vp, i32, i64, u64, f32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint64, ctypes.c_float)
        L.mrcm_lp_create.argtypes = [i32, i32, i32, u64, vp, ctypes.POINTER(vp)]
        L.mrcm_lp_create.restype = i32
        L.mrcm_lp_destroy.argtypes = [vp]
        L.mrcm_lp_destroy.restype = None
        L.mrcm_lp_last_error.argtypes = [vp]
        L.mrcm_lp_last_error.restype = ctypes.c_char_p
        L.mrcm_lp_set_stream.argtypes = [vp, vp]
        L.mrcm_lp_set_stream.restype = i32
        L.mrcm_lp_num_params.argtypes = [vp]
        L.mrcm_lp_num_params.restype = i64
        L.mrcm_lp_input_size.argtypes = [vp]
        L.mrcm_lp_input_size.restype = i64
        for f in (L.mrcm_lp_set_params, L.mrcm_lp_get_params, L.mrcm_lp_set_loss_weights):
            f.argtypes = [vp, vp]
            f.restype = i32
        L.mrcm_lp_forward.argtypes = [vp, vp, i32, vp]
        L.mrcm_lp_forward.restype = i32
        L.mrcm_lp_gradient.argtypes = [vp, vp, vp, i32, vp, vp]
        L.mrcm_lp_gradient.restype = i32
        L.mrcm_lp_train_step.argtypes = [vp, vp, vp, i32, f32, vp]
        L.mrcm_lp_train_step.restype = i32
        L.mrcm_lp_num_samples.argtypes = [vp]
        L.mrcm_lp_num_samples.restype = i64
        L.mrcm_lp_windows.argtypes = [vp, vp, vp, i64, i32, vp]
        L.mrcm_lp_windows.restype = i32
        L.mrcm_lp_targets.argtypes = [vp, vp]
        L.mrcm_lp_targets.restype = i32
        L.mrcm_lp_apply.argtypes = [vp, vp, vp, vp]
        L.mrcm_lp_apply.restype = i32
        _bound = True
    return L


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class LearnedPrecond:
    """The network object: weights, Adam state and activation buffers."""

    def __init__(self, s: int, m: int, max_batch: int = 1024, seed: int = 0, stream=None):
        import torch
        self.L = lib()
        self.s, self.m, self.max_batch = s, m, max_batch
        if stream is None:
            stream = torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.L.mrcm_lp_create(s, m, max_batch, seed, ctypes.c_void_p(stream.cuda_stream),
                                   ctypes.byref(h))
        if st != _m.MRCM_OK:
            raise _m.MrcmError(st, self.L.mrcm_lp_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != _m.MRCM_OK:
            raise _m.MrcmError(st, self.L.mrcm_lp_last_error(self.h).decode())

    def set_stream(self, stream):
        self._check(self.L.mrcm_lp_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    @property
    def num_params(self) -> int:
        return int(self.L.mrcm_lp_num_params(self.h))

    @property
    def input_size(self) -> int:
        return int(self.L.mrcm_lp_input_size(self.h))

    def get_params(self):
        import torch
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        self._check(self.L.mrcm_lp_get_params(self.h, _p(out)))
        return out

    def set_params(self, params):
        self._check(self.L.mrcm_lp_set_params(self.h, _p(params.contiguous())))

    def set_loss_weights(self, w):
        """Per-entry loss weights (FP32 CUDA tensor of m*m values)."""
        self._check(self.L.mrcm_lp_set_loss_weights(self.h, _p(w.contiguous())))

    def forward(self, x, B: Optional[int] = None):
        """x: BF16 CUDA tensor [B, 2, 2s, 3s] -> Delta [B, m*m] FP32."""
        import torch
        B = int(x.shape[0]) if B is None else B
        d = torch.empty((B, self.m * self.m), dtype=torch.float32, device="cuda")
        self._check(self.L.mrcm_lp_forward(self.h, _p(x), B, _p(d)))
        return d

    def gradient(self, x, target):
        import torch
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._check(self.L.mrcm_lp_gradient(self.h, _p(x), _p(target), int(x.shape[0]), _p(g),
                                            _p(loss)))
        return float(loss.item()), g

    def train_step(self, x, target, lr: float, loss_out=None):
        self._check(self.L.mrcm_lp_train_step(self.h, _p(x), _p(target), int(x.shape[0]),
                                              float(lr), _p(loss_out)))

    def close(self):
        if getattr(self, "h", None):
            self.L.mrcm_lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- with a context
def num_samples(solver: "_m.Mrcm") -> int:
    return int(lib().mrcm_lp_num_samples(solver.ctx))


def windows(solver: "_m.Mrcm", K, lam, first: int = 0, count: Optional[int] = None, s=None):
    """Network inputs (BF16 [count, 2, 2s, 3s]) of a context's interfaces."""
    import torch
    L = lib()
    n = num_samples(solver)
    count = n - first if count is None else count
    s = solver.prob.sub_size[0] if s is None else s
    x = torch.empty((count, 2, 2 * s, 3 * s), dtype=torch.bfloat16, device="cuda")
    solver._check(L.mrcm_lp_windows(solver.ctx, _p(K), _p(lam), first, count, _p(x)))
    return x


def targets(solver: "_m.Mrcm", m: int):
    """Training targets (FP32 [num_samples, m*m]) after build_basis."""
    import torch
    t = torch.empty((num_samples(solver), m * m), dtype=torch.float32, device="cuda")
    solver._check(lib().mrcm_lp_targets(solver.ctx, _p(t)))
    return t


def apply(solver: "_m.Mrcm", net: LearnedPrecond, K, lam):
    """Install the network's blocks as the context's GMRES preconditioner."""
    solver._check(lib().mrcm_lp_apply(solver.ctx, net.h, _p(K), _p(lam)))


# ------------------------------------------------------------- training
@dataclass
class TrainReport:
    samples: int = 0
    steps: int = 0
    loss_first: float = 0.0
    loss_last: float = 0.0
    losses: List[float] = field(default_factory=list)


def make_dataset(problems, m: int, opts: Optional["_m.SolverOptions"] = None):
    """Windows and targets of every interface of every problem, from the
    library's own factor and basis kernels (GMRES path, caller blocks)."""
    import torch
    opts = opts or _m.SolverOptions(prec=_m.PREC_FP32_IR, iface_solver=_m.IFACE_GMRES,
                                    precond=_m.PRECOND_USER)
    xs, ts = [], []
    for prob in problems:
        solver = _m.Mrcm(prob, opts)
        K, lam, q = _m.device_inputs(prob)
        solver.mrcm_factor_local(K, lam)
        solver.mrcm_build_basis(q)
        xs.append(windows(solver, K, lam))
        ts.append(targets(solver, m))
        solver.close()
    return torch.cat(xs), torch.cat(ts)


def train(net: LearnedPrecond, x, t, steps: int = 400, batch: int = 256, lr: float = 2e-3,
          seed: int = 0, weighted: bool = True) -> TrainReport:
    """Adam on random mini-batches (seeded, drawn on the device); with
    ``weighted`` every entry of Delta is weighted by the inverse variance of
    that entry over the training targets."""
    import torch
    rep = TrainReport(samples=int(x.shape[0]))
    if weighted:
        var = t.double().var(dim=0).clamp_min(1e-8)
        net.set_loss_weights((1.0 / var).float())
    batch = min(batch, net.max_batch, int(x.shape[0]))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = torch.zeros(steps, dtype=torch.float32, device="cuda")
    for k in range(steps):
        idx = torch.randint(0, int(x.shape[0]), (batch,), device="cuda", generator=g)
        net.train_step(x[idx].contiguous(), t[idx].contiguous(), lr, loss)
        hist[k] = loss[0]
    h = hist.cpu().numpy()
    rep.steps, rep.losses = steps, h.tolist()
    rep.loss_first, rep.loss_last = float(h[0]), float(h[-10:].mean())
    return rep
