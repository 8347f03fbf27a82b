"""ctypes binding of the MRCM C ABI (include/mrcm.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels
of ``libmrcm.so``.  Device buffers are torch CUDA tensors (FP64, contiguous)
whose ``data_ptr()`` is passed through; the stream is torch's current CUDA
stream unless one is given.  If the library is missing the import fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from pathlib import Path
from typing import Optional

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libmrcm.so"

MRCM_OK, MRCM_EINVAL, MRCM_ENOMEM, MRCM_ECUDA, MRCM_ENOTSPD = 0, 1, 2, 3, 4
MRCM_EIRSTALL, MRCM_ENOCONV, MRCM_ENAN, MRCM_ETIMEOUT, MRCM_EINCOMPAT = 5, 6, 7, 8, 9
PREC_FP64, PREC_FP32_IR = 0, 1
BASIS_LEGENDRE, BASIS_MONOMIAL = 0, 1
IFACE_AUTO, IFACE_DIRECT, IFACE_GMRES = 0, 1, 2
PRECOND_BLOCK_JACOBI, PRECOND_USER, PRECOND_NONE = 0, 1, 2
PRECOND_NEIGHBOURHOOD, PRECOND_NEIGHBOURHOOD_SHARED = 3, 4
PATH_NONE, PATH_CLUSTER, PATH_SLAB, PATH_WIDE_SLAB, PATH_GMRES = 0, 1, 2, 3, 4
PATH_NAMES = {0: "none", 1: "cluster", 2: "slab", 3: "wide-slab", 4: "gmres"}
FLAG_PRECOND_FALLBACK = 0x40
FLAG_TIMEOUT = 0x80          # a bounded device wait ran out (MRCM_ETIMEOUT)
FLAG_LOCAL_STALL = 0x2
FLAG_INCOMPATIBLE = 0x200    # pure Neumann: sources and boundary outflow do not balance
FLAG_LOCAL_REFACTOR = 0x100  # stalled subdomains re-factored and re-solved in FP64
STATUS_NAMES = {0: "MRCM_OK", 1: "MRCM_EINVAL", 2: "MRCM_ENOMEM", 3: "MRCM_ECUDA",
                4: "MRCM_ENOTSPD", 5: "MRCM_EIRSTALL", 6: "MRCM_ENOCONV", 7: "MRCM_ENAN",
                8: "MRCM_ETIMEOUT", 9: "MRCM_EINCOMPAT"}

EXPORTED = ["mrcm_setup", "mrcm_factor_local", "mrcm_build_basis", "mrcm_solve_interface",
            "mrcm_reconstruct", "mrcm_get_info", "mrcm_set_stream", "mrcm_launch_count",
            "mrcm_num_interface_unknowns", "mrcm_num_gamma_values",
            "mrcm_copy_interface_solution", "mrcm_destroy", "mrcm_last_error", "mrcm_version",
            "mrcm_local_solve_noalloc", "mrcm_uses_gmres", "mrcm_num_precond_values",
            "mrcm_set_precond_blocks", "mrcm_set_basis_width", "mrcm_autotune",
            "mrcm_set_gravity", "mrcm_interface_path"]


class MrcmDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("n_real", ctypes.c_int32),
        ("ly", ctypes.c_double),
        ("sub_size", ctypes.POINTER(ctypes.c_int32)),
        ("iface_nU", ctypes.POINTER(ctypes.c_int32)),
        ("iface_nP", ctypes.POINTER(ctypes.c_int32)),
        ("alpha", ctypes.POINTER(ctypes.c_double)),
        ("bc_type", ctypes.POINTER(ctypes.c_int8)),
        ("bc_val", ctypes.POINTER(ctypes.c_double)),
        ("pure_neumann", ctypes.c_int32),
        ("basis_family", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("ir_tol", ctypes.c_double), ("ir_max", ctypes.c_int32),
        ("iface_tol", ctypes.c_double), ("iface_ir_max", ctypes.c_int32),
        ("iface_solver", ctypes.c_int32), ("precond", ctypes.c_int32),
        ("gmres_restart", ctypes.c_int32), ("gmres_max", ctypes.c_int32),
        ("gmres_tol", ctypes.c_double),
        ("iface_fn", ctypes.POINTER(ctypes.c_double)),
        ("refine", ctypes.POINTER(ctypes.c_int8)),
        ("ir_recover", ctypes.c_int32),
    ]


class MrcmInfo(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_int32), ("local_sweeps_max", ctypes.c_int32),
                ("iface_sweeps", ctypes.c_int32), ("gmres_iters", ctypes.c_int32),
                ("local_resid_max", ctypes.c_double), ("iface_resid", ctypes.c_double),
                ("local_refactored", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib(path: Optional[Path] = None):
    """Load libmrcm.so (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else _LIB_PATH
    if not p.exists():
        raise RuntimeError(f"MRCM CUDA library not built ({p}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(str(p))
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.mrcm_setup.argtypes = [ctypes.POINTER(MrcmDesc), vp, ctypes.POINTER(vp)]
    L.mrcm_setup.restype = i32
    L.mrcm_factor_local.argtypes = [vp, dp, dp]
    L.mrcm_factor_local.restype = i32
    L.mrcm_build_basis.argtypes = [vp, dp]
    L.mrcm_build_basis.restype = i32
    L.mrcm_solve_interface.argtypes = [vp, ctypes.POINTER(MrcmInfo)]
    L.mrcm_solve_interface.restype = i32
    L.mrcm_reconstruct.argtypes = [vp, dp, dp, dp, dp]
    L.mrcm_reconstruct.restype = i32
    L.mrcm_get_info.argtypes = [vp, ctypes.POINTER(MrcmInfo)]
    L.mrcm_get_info.restype = i32
    L.mrcm_set_stream.argtypes = [vp, vp]
    L.mrcm_set_stream.restype = i32
    L.mrcm_launch_count.argtypes = [vp]
    L.mrcm_launch_count.restype = i32
    L.mrcm_num_interface_unknowns.argtypes = [vp]
    L.mrcm_num_interface_unknowns.restype = i64
    L.mrcm_num_gamma_values.argtypes = [vp]
    L.mrcm_num_gamma_values.restype = i64
    L.mrcm_copy_interface_solution.argtypes = [vp, dp]
    L.mrcm_copy_interface_solution.restype = i32
    L.mrcm_destroy.argtypes = [vp]
    L.mrcm_destroy.restype = None
    L.mrcm_last_error.argtypes = [vp]
    L.mrcm_last_error.restype = ctypes.c_char_p
    L.mrcm_version.argtypes = []
    L.mrcm_version.restype = i32
    L.mrcm_local_solve_noalloc.argtypes = [i32, dp, dp, dp, dp, vp]
    L.mrcm_local_solve_noalloc.restype = i32
    L.mrcm_uses_gmres.argtypes = [vp]
    L.mrcm_uses_gmres.restype = i32
    L.mrcm_interface_path.argtypes = [vp]
    L.mrcm_interface_path.restype = i32
    L.mrcm_num_precond_values.argtypes = [vp]
    L.mrcm_num_precond_values.restype = i64
    L.mrcm_set_precond_blocks.argtypes = [vp, dp]
    L.mrcm_set_precond_blocks.restype = i32
    L.mrcm_set_basis_width.argtypes = [vp, i32, i32]
    L.mrcm_set_basis_width.restype = i32
    L.mrcm_autotune.argtypes = [vp, dp, dp, dp, i32, ctypes.POINTER(ctypes.c_int32)]
    L.mrcm_autotune.restype = i32
    L.mrcm_set_gravity.argtypes = [vp, vp]
    L.mrcm_set_gravity.restype = i32
    if path is None:
        _lib = L
    return L


class MrcmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    """Device pointer of a contiguous FP64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("device buffers must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class SolverOptions:
    prec: int = PREC_FP32_IR
    ir_tol: float = 1e-13
    ir_max: int = 30
    iface_tol: float = 1e-13
    iface_ir_max: int = 40
    iface_solver: int = IFACE_AUTO
    precond: int = PRECOND_BLOCK_JACOBI
    gmres_restart: int = 40
    gmres_max: int = 5000
    gmres_tol: float = 0.0          # 0: iface_tol
    ir_recover: int = 0             # FP64 re-factor of stalled subdomains: 0 = 16, < 0 = off


class Mrcm:
    """One MRCM context: the five hot-path calls on a fixed problem layout."""

    def __init__(self, prob, opts: SolverOptions = SolverOptions(), stream=None):
        import torch
        self.L = lib()
        self.prob = prob
        self._keep = []
        nu = np.ascontiguousarray(np.concatenate(prob.iface_nU).astype(np.int32))
        npp = np.ascontiguousarray(np.concatenate(prob.iface_nP).astype(np.int32))
        sub = np.ascontiguousarray(np.asarray(prob.sub_size, np.int32))
        bct = np.ascontiguousarray(prob.bc_type.astype(np.int8))
        bcv = np.ascontiguousarray(prob.bc_val.astype(np.float64))
        alpha = None
        if prob.alpha is not None:
            # per realisation: an [n_iface, s] array, or a list of per-interface
            # arrays (interfaces of different lengths)
            alpha = np.ascontiguousarray(np.concatenate(
                [np.asarray(x, np.float64).reshape(-1) for a in prob.alpha
                 for x in (a if isinstance(a, (list, tuple)) else [a])]))
        self._keep += [nu, npp, sub, bct, bcv, alpha]
        d = MrcmDesc()
        d.nx, d.ny, d.n_real, d.ly = prob.nx, prob.ny, prob.n_real, prob.ly
        d.sub_size = sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.iface_nU = nu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.iface_nP = npp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.alpha = (alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if alpha is not None
                   else ctypes.POINTER(ctypes.c_double)())
        d.bc_type = bct.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
        d.bc_val = bcv.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.pure_neumann = 1 if prob.pure_neumann else 0
        d.basis_family = BASIS_LEGENDRE if prob.basis == "legendre" else BASIS_MONOMIAL
        fn = None
        if getattr(prob, "iface_fn", None) is not None:
            # per interface: nU flux rows then nP pressure rows of s values
            fn = np.ascontiguousarray(np.concatenate(
                [np.concatenate([np.asarray(phi, np.float64).reshape(-1),
                                 np.asarray(psi, np.float64).reshape(-1)])
                 for tabs in prob.iface_fn for phi, psi in tabs]))
            self._keep.append(fn)
        d.iface_fn = (fn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if fn is not None
                      else ctypes.POINTER(ctypes.c_double)())
        ref = None
        if getattr(prob, "refine", None) is not None:
            # per realisation (ny/s) x (nx/s) int8, concatenated
            ref = np.ascontiguousarray(np.concatenate(
                [np.asarray(m, np.int8).reshape(-1) for m in prob.refine]))
            self._keep.append(ref)
        d.refine = (ref.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if ref is not None
                    else ctypes.POINTER(ctypes.c_int8)())
        d.prec = opts.prec
        d.ir_tol, d.ir_max = opts.ir_tol, opts.ir_max
        d.iface_tol, d.iface_ir_max = opts.iface_tol, opts.iface_ir_max
        d.iface_solver, d.precond = opts.iface_solver, opts.precond
        d.gmres_restart, d.gmres_max = opts.gmres_restart, opts.gmres_max
        d.gmres_tol = opts.gmres_tol
        d.ir_recover = opts.ir_recover
        self.desc = d
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ctx = ctypes.c_void_p()
        st = self.L.mrcm_setup(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                               ctypes.byref(ctx))
        if st != MRCM_OK:
            raise MrcmError(st, self.L.mrcm_last_error(None).decode())
        self.ctx = ctx
        self._grav = None
        if getattr(prob, "grav", None) is not None:
            # the gravity velocity K lambda_g g per cell, kept alive with the context
            self._grav = torch.as_tensor(np.stack([np.asarray(w, np.float64) for w in prob.grav]),
                                         device="cuda").contiguous()
            self._check(self.L.mrcm_set_gravity(self.ctx, _ptr(self._grav)))

    # -- the five calls (same names as the C ABI) --------------------------
    def _check(self, st):
        if st != MRCM_OK:
            raise MrcmError(st, self.L.mrcm_last_error(self.ctx).decode())

    def mrcm_factor_local(self, K, lam):
        self._check(self.L.mrcm_factor_local(self.ctx, _ptr(K), _ptr(lam)))

    def mrcm_build_basis(self, q):
        self._check(self.L.mrcm_build_basis(self.ctx, _ptr(q)))

    def mrcm_solve_interface(self, info: bool = False):
        if info:
            inf = MrcmInfo()
            self._check(self.L.mrcm_solve_interface(self.ctx, ctypes.byref(inf)))
            return inf.as_dict()
        self._check(self.L.mrcm_solve_interface(self.ctx, None))
        return None

    def mrcm_reconstruct(self, p, ux, uy, gamma_u=None):
        self._check(self.L.mrcm_reconstruct(self.ctx, _ptr(p), _ptr(ux), _ptr(uy), _ptr(gamma_u)))

    def mrcm_get_info(self, check: bool = True):
        inf = MrcmInfo()
        st = self.L.mrcm_get_info(self.ctx, ctypes.byref(inf))
        if check:
            self._check(st)
        d = inf.as_dict()
        d["status"] = STATUS_NAMES.get(st, st)
        return d

    # -- helpers --------------------------------------------------------
    def launch_count(self) -> int:
        return int(self.L.mrcm_launch_count(self.ctx))

    def num_interface_unknowns(self) -> int:
        return int(self.L.mrcm_num_interface_unknowns(self.ctx))

    def num_gamma_values(self) -> int:
        return int(self.L.mrcm_num_gamma_values(self.ctx))

    def mrcm_set_basis_width(self, nc16: int, nc32: int):
        self._check(self.L.mrcm_set_basis_width(self.ctx, nc16, nc32))

    def mrcm_autotune(self, K, lam, q, reps: int = 3):
        """Time every basis tile width on these inputs and keep the fastest;
        returns (width for 16x16, width for 32x32 subdomains)."""
        ch = (ctypes.c_int32 * 2)()
        self._check(self.L.mrcm_autotune(self.ctx, _ptr(K), _ptr(lam), _ptr(q), reps, ch))
        return int(ch[0]), int(ch[1])

    def uses_gmres(self) -> bool:
        return bool(self.L.mrcm_uses_gmres(self.ctx))

    def interface_path(self) -> str:
        """The step-(d) kernels of this context: "none", "cluster", "slab",
        "wide-slab" or "gmres" (mrcm_interface_path)."""
        return PATH_NAMES[int(self.L.mrcm_interface_path(self.ctx))]

    def num_precond_values(self) -> int:
        return int(self.L.mrcm_num_precond_values(self.ctx))

    def mrcm_set_precond_blocks(self, blocks):
        """Caller-supplied (learned) preconditioner blocks: contiguous FP64
        CUDA tensor of num_precond_values() entries."""
        self._check(self.L.mrcm_set_precond_blocks(self.ctx, _ptr(blocks)))

    def interface_solution(self):
        import torch
        x = torch.empty(self.num_interface_unknowns(), dtype=torch.float64, device="cuda")
        self._check(self.L.mrcm_copy_interface_solution(self.ctx, _ptr(x)))
        return x

    def alloc_outputs(self):
        import torch
        p = self.prob
        R, ny, nx = p.n_real, p.ny, p.nx
        kw = dict(dtype=torch.float64, device="cuda")
        return (torch.empty((R, ny, nx), **kw), torch.empty((R, ny, nx + 1), **kw),
                torch.empty((R, ny + 1, nx), **kw))

    def solve(self, K, lam, q, out=None, gamma_u=None):
        """The whole hot path: factor, basis, interface, reconstruct."""
        if out is None:
            out = self.alloc_outputs()
        self.mrcm_factor_local(K, lam)
        self.mrcm_build_basis(q)
        self.mrcm_solve_interface()
        self.mrcm_reconstruct(*out, gamma_u=gamma_u)
        return out

    def close(self):
        if getattr(self, "ctx", None):
            self.L.mrcm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def local_solve_noalloc(kappa, tface, rhs, x, stream=None):
    """Local subdomain solve with no device allocation (see
    mrcm_local_solve_noalloc in include/mrcm.h).  kappa [n,16,16], tface
    [n,4,16], rhs and x [n,16,16]: contiguous FP64 CUDA tensors."""
    import torch
    L = lib()
    if stream is None:
        stream = torch.cuda.current_stream()
    n = int(kappa.shape[0])
    st = L.mrcm_local_solve_noalloc(n, _ptr(kappa), _ptr(tface), _ptr(rhs), _ptr(x),
                                    ctypes.c_void_p(stream.cuda_stream))
    if st != MRCM_OK:
        raise MrcmError(st, L.mrcm_last_error(None).decode())


def device_inputs(prob):
    """K, lambda, q of a problem as FP64 CUDA tensors."""
    import torch
    kw = dict(dtype=torch.float64, device="cuda")
    return (torch.as_tensor(np.ascontiguousarray(prob.K), **kw),
            torch.as_tensor(np.ascontiguousarray(prob.lam), **kw),
            torch.as_tensor(np.ascontiguousarray(prob.q), **kw))
