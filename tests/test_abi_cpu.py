"""The C-ABI library loads and exports every symbol include/mrcm.h declares
(no compute calls: no GPU needed).  Descriptor validation runs on the host
before any CUDA call, so its errors are checked here too."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def L():
    from paper_2104_04653_gb300 import build, mrcm
    build.build()
    return mrcm.lib()


def test_exports_every_declared_symbol(L):
    hdr = "\n".join(p.read_text() for p in sorted((ROOT / "include").glob("*.h")))
    declared = set(re.findall(r"\b(mrcm_[a-z_]+)\s*\(", hdr))
    assert {"mrcm_setup", "mrcm_factor_local", "mrcm_build_basis", "mrcm_solve_interface",
            "mrcm_reconstruct"} <= declared
    for name in declared:
        assert hasattr(L, name), name
    assert L.mrcm_version() == 1


def _desc(mrcm, nx=64, ny=32, sub=16, prec=1, nU=2, nP=2, pure=0, bct=None):
    sx, sy = nx // max(sub, 1), ny // max(sub, 1)
    nif = max((sx - 1) * sy + sx * (sy - 1), 1)
    keep = dict(sub=np.array([sub], np.int32), nu=np.full(nif, nU, np.int32),
                np_=np.full(nif, nP, np.int32),
                bt=np.zeros(2 * nx + 2 * ny, np.int8) if bct is None else bct,
                bv=np.zeros(2 * nx + 2 * ny))
    d = mrcm.MrcmDesc()
    d.nx, d.ny, d.n_real, d.ly = nx, ny, 1, 1.0
    d.sub_size = keep["sub"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.iface_nU = keep["nu"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.iface_nP = keep["np_"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.bc_type = keep["bt"].ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    d.bc_val = keep["bv"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.pure_neumann = pure
    d.prec = prec
    d.ir_tol, d.ir_max, d.iface_tol, d.iface_ir_max = 1e-13, 30, 1e-13, 40
    return d, keep


@pytest.mark.parametrize("bad", ["nx", "sub", "prec", "nU", "pure_dirichlet", "null", "solver",
                                 "precond", "precond_high", "restart"])
def test_setup_rejects_bad_descriptors(L, bad):
    from paper_2104_04653_gb300 import mrcm
    kw = {}
    if bad == "nx":
        kw = dict(nx=-4)
    elif bad == "sub":
        kw = dict(sub=12)
    elif bad == "prec":
        kw = dict(prec=7)
    elif bad == "nU":
        kw = dict(nU=17)
    elif bad == "pure_dirichlet":
        bt = np.zeros(2 * 64 + 2 * 32, np.int8)
        bt[0] = 1
        kw = dict(pure=1, bct=bt)
    ctx = ctypes.c_void_p()
    field = {"solver": ("iface_solver", 3), "precond": ("precond", -1),
             "precond_high": ("precond", 5), "restart": ("gmres_restart", 65)}.get(bad)
    if bad == "null":
        st = L.mrcm_setup(None, None, ctypes.byref(ctx))
    else:
        d, keep = _desc(mrcm, **kw)
        if field:
            setattr(d, *field)
        st = L.mrcm_setup(ctypes.byref(d), None, ctypes.byref(ctx))
    assert st == mrcm.MRCM_EINVAL
    assert not ctx.value
    assert len(L.mrcm_last_error(None)) > 0


def test_calls_on_null_context_fail_cleanly(L):
    from paper_2104_04653_gb300 import mrcm
    assert L.mrcm_factor_local(None, None, None) == mrcm.MRCM_EINVAL
    assert L.mrcm_build_basis(None, None) == mrcm.MRCM_EINVAL
    assert L.mrcm_solve_interface(None, None) == mrcm.MRCM_EINVAL
    assert L.mrcm_reconstruct(None, None, None, None, None) == mrcm.MRCM_EINVAL
    L.mrcm_destroy(None)
