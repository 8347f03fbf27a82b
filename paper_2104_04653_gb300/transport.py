"""ctypes binding of the implicit saturation transport and the SI / SFI time
steps (include/mrcm_transport.h).

Argument marshalling only: the Newton loop, its linear solves, the trust
region, the mobility update and the Darcy calls of a step all run in
``libmrcm.so``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import mrcm as _m

EXPORTED = ["mrcm_transport_create", "mrcm_transport_step", "mrcm_transport_get_info",
            "mrcm_transport_set_stream", "mrcm_transport_destroy", "mrcm_transport_last_error",
            "mrcm_si_step", "mrcm_sfi_step"]

FLAG_NEWTON, FLAG_LINEAR, FLAG_NAN = 0x1, 0x2, 0x4


class TransportDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("n_real", ctypes.c_int32),
        ("ly", ctypes.c_double), ("M", ctypes.c_double), ("mu_w", ctypes.c_double),
        ("s_in", ctypes.c_double), ("eta", ctypes.c_double),
        ("max_newton", ctypes.c_int32), ("max_linear", ctypes.c_int32),
        ("plain_newton", ctypes.c_int32),
    ]


class TransportInfo(ctypes.Structure):
    _fields_ = [
        ("newton_iters_max", ctypes.c_int32), ("linear_iters_max", ctypes.c_int32),
        ("update_norm_max", ctypes.c_double), ("change_max", ctypes.c_double),
        ("flags", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_bound = False


def lib():
    global _bound
    L = _m.lib()
    if not _bound:
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.mrcm_transport_create.argtypes = [vp, vp, ctypes.POINTER(vp)]
        L.mrcm_transport_create.restype = i32
        L.mrcm_transport_step.argtypes = [vp, dbl, vp, vp, vp, vp, vp, vp]
        L.mrcm_transport_step.restype = i32
        L.mrcm_transport_get_info.argtypes = [vp, vp, vp]
        L.mrcm_transport_get_info.restype = i32
        L.mrcm_transport_set_stream.argtypes = [vp, vp]
        L.mrcm_transport_set_stream.restype = i32
        L.mrcm_transport_destroy.argtypes = [vp]
        L.mrcm_transport_destroy.restype = None
        L.mrcm_transport_last_error.argtypes = []
        L.mrcm_transport_last_error.restype = ctypes.c_char_p
        L.mrcm_si_step.argtypes = [vp, vp, dbl, vp, vp, vp, vp, vp, vp, vp, vp]
        L.mrcm_si_step.restype = i32
        L.mrcm_sfi_step.argtypes = [vp, vp, dbl, dbl, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                    ctypes.POINTER(i32)]
        L.mrcm_sfi_step.restype = i32
        _bound = True
    return L


@dataclass
class TransportOptions:
    M: float = 10.0
    mu_w: float = 1.0
    s_in: float = 1.0
    eta: float = 1e-6
    max_newton: int = 100
    max_linear: int = 0
    plain_newton: bool = False


class Transport:
    """One transport context for n_real grids of nx x ny cells."""

    def __init__(self, nx: int, ny: int, n_real: int, ly: float = 1.0,
                 opts: TransportOptions = TransportOptions(), stream=None):
        import torch
        self.L = lib()
        d = TransportDesc()
        d.nx, d.ny, d.n_real, d.ly = nx, ny, n_real, ly
        d.M, d.mu_w, d.s_in, d.eta = opts.M, opts.mu_w, opts.s_in, opts.eta
        d.max_newton, d.max_linear = opts.max_newton, opts.max_linear
        d.plain_newton = 1 if opts.plain_newton else 0
        self.desc, self.n_real = d, n_real
        if stream is None:
            stream = torch.cuda.current_stream()
        h = ctypes.c_void_p()
        self._check(self.L.mrcm_transport_create(ctypes.byref(d),
                                                 ctypes.c_void_p(stream.cuda_stream),
                                                 ctypes.byref(h)))
        self.h = h

    def _check(self, st):
        if st != _m.MRCM_OK:
            raise _m.MrcmError(st, self.L.mrcm_transport_last_error().decode())

    def mrcm_transport_step(self, dt, ux, uy, s_old, s_new, lam=None, s_ref=None):
        P = _m._ptr
        self._check(self.L.mrcm_transport_step(self.h, float(dt), P(ux), P(uy), P(s_old),
                                               P(s_new), P(lam), P(s_ref)))

    def mrcm_transport_get_info(self, check: bool = True):
        inf = TransportInfo()
        its = (ctypes.c_int32 * self.n_real)()
        st = self.L.mrcm_transport_get_info(self.h, ctypes.byref(inf), its)
        if check:
            self._check(st)
        d = inf.as_dict()
        d["newton_iters"] = list(its)
        d["status"] = _m.STATUS_NAMES.get(st, st)
        return d

    def set_stream(self, stream):
        self._check(self.L.mrcm_transport_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    def close(self):
        if self.h:
            self.L.mrcm_transport_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mrcm_si_step(darcy: "_m.Mrcm", tp: Transport, dt, K, lam, q, s_old, s_new, p, ux, uy):
    """One sequential implicit step (mrcm_si_step): Darcy with lam, then
    transport; lam receives the mobility of s_new."""
    P = _m._ptr
    st = tp.L.mrcm_si_step(darcy.ctx, tp.h, float(dt), P(K), P(lam), P(q), P(s_old), P(s_new),
                           P(p), P(ux), P(uy))
    tp._check(st)


def mrcm_sfi_step(darcy: "_m.Mrcm", tp: Transport, dt, tol, max_outer, K, lam, q, s_old, s_new,
                  s_work, p, ux, uy) -> int:
    """One sequential fully implicit step (mrcm_sfi_step); returns the outer
    iteration count."""
    P = _m._ptr
    k = ctypes.c_int32()
    st = tp.L.mrcm_sfi_step(darcy.ctx, tp.h, float(dt), float(tol), int(max_outer), P(K), P(lam),
                            P(q), P(s_old), P(s_new), P(s_work), P(p), P(ux), P(uy),
                            ctypes.byref(k))
    tp._check(st)
    return int(k.value)
