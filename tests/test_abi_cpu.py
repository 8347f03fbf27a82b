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
    assert L.mrcm_interface_path(None) == -1
    assert L.mrcm_test_degrade_factor(None, 0, 7) == mrcm.MRCM_EINVAL
    L.mrcm_test_fp_convert.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    assert L.mrcm_test_fp_convert(0, 16, None, None) == mrcm.MRCM_EINVAL
    L.mrcm_destroy(None)


def test_seeded_random_descriptors_fail_cleanly(L):
    """500 seeded descriptors, mostly valid, some with one corrupted field:
    setup either refuses them (EINVAL, no context) or gets as far as the
    device (ECUDA here, where there is none); the host code never crashes."""
    from paper_2104_04653_gb300 import mrcm
    rng = np.random.default_rng(2024)
    P = ctypes.POINTER
    seen = set()
    for _ in range(500):
        R = int(rng.integers(1, 4))
        subs = rng.choice([16, 32], size=R).astype(np.int32)
        nx, ny = int(rng.choice([32, 64, 96, 128])), int(rng.choice([32, 64, 128]))
        tot = sum(max(0, (nx // s - 1) * (ny // s) + (nx // s) * (ny // s - 1)) for s in subs)
        nu = rng.integers(1, 5, size=tot + 1).astype(np.int32)
        npp = rng.integers(1, 5, size=tot + 1).astype(np.int32)
        nb = 2 * nx + 2 * ny
        bt = rng.integers(0, 2, size=nb).astype(np.int8)
        bv = rng.standard_normal(nb)
        alpha = rng.uniform(0.1, 2.0, size=max(tot * 32, 1))
        corrupt = int(rng.integers(0, 8))
        if corrupt == 0:
            nu[rng.integers(0, tot + 1)] = int(rng.choice([-1, 40]))
        elif corrupt == 1:
            bt[rng.integers(0, nb)] = 3
        elif corrupt == 2:
            bv[rng.integers(0, nb)] = np.nan
        elif corrupt == 3:
            alpha[rng.integers(0, max(tot * 32, 1))] = -1.0
        d = mrcm.MrcmDesc()
        d.nx, d.ny, d.n_real, d.ly = nx, ny, R, 1.0
        d.sub_size = subs.ctypes.data_as(P(ctypes.c_int32))
        d.iface_nU = nu.ctypes.data_as(P(ctypes.c_int32))
        d.iface_nP = npp.ctypes.data_as(P(ctypes.c_int32))
        d.bc_type = bt.ctypes.data_as(P(ctypes.c_int8))
        d.bc_val = bv.ctypes.data_as(P(ctypes.c_double))
        d.alpha = alpha.ctypes.data_as(P(ctypes.c_double)) if rng.random() < 0.5 \
            else P(ctypes.c_double)()
        d.pure_neumann = int(rng.random() < 0.2)
        d.basis_family, d.prec = int(rng.integers(0, 2)), int(rng.integers(0, 2))
        d.ir_tol, d.ir_max, d.iface_tol, d.iface_ir_max = 1e-13, 30, 1e-13, 40
        d.iface_solver, d.precond = int(rng.integers(0, 3)), int(rng.integers(0, 3))
        d.gmres_restart, d.gmres_max = int(rng.integers(0, 65)), int(rng.integers(0, 100))
        ctx = ctypes.c_void_p()
        st = L.mrcm_setup(ctypes.byref(d), None, ctypes.byref(ctx))
        seen.add(st)
        if st != mrcm.MRCM_OK:
            assert not ctx.value
            assert len(L.mrcm_last_error(None)) > 0
        else:
            L.mrcm_destroy(ctx)
    assert mrcm.MRCM_EINVAL in seen


@pytest.mark.parametrize("bad", ["grid", "M", "mu_w", "s_in", "eta", "newton", "real"])
def test_transport_rejects_bad_descriptors(L, bad):
    """mrcm_transport_create validates its descriptor on the host."""
    from paper_2104_04653_gb300 import mrcm, transport as TP
    TP.lib()
    d = TP.TransportDesc()
    d.nx, d.ny, d.n_real, d.ly, d.M, d.mu_w, d.s_in = 16, 16, 1, 1.0, 10.0, 1.0, 1.0
    setattr(d, *{"grid": ("nx", 0), "M": ("M", -1.0), "mu_w": ("mu_w", 0.0),
                 "s_in": ("s_in", 1.5), "eta": ("eta", -1.0), "newton": ("max_newton", -2),
                 "real": ("n_real", 0)}[bad])
    h = ctypes.c_void_p()
    assert L.mrcm_transport_create(ctypes.byref(d), None, ctypes.byref(h)) == mrcm.MRCM_EINVAL
    assert not h.value
    assert L.mrcm_transport_last_error()


def test_transport_calls_on_null_context_fail_cleanly(L):
    from paper_2104_04653_gb300 import mrcm, transport as TP
    TP.lib()
    assert L.mrcm_transport_step(None, 0.1, None, None, None, None, None, None) == mrcm.MRCM_EINVAL
    assert L.mrcm_transport_get_info(None, None, None) == mrcm.MRCM_EINVAL
    assert L.mrcm_si_step(None, None, 0.1, *([None] * 8)) == mrcm.MRCM_EINVAL
    assert L.mrcm_sfi_step(None, None, 0.1, 1e-4, 5, *([None] * 9), None) == mrcm.MRCM_EINVAL
    L.mrcm_transport_destroy(None)


def test_quadtree_refusals(L):
    """A refine mask is checked on the host: only 32 x 32 blocks split, no
    direct interface solver, no neighbourhood or learned preconditioner."""
    from paper_2104_04653_gb300 import mrcm
    nx = ny = 64
    for case in ("split16", "direct", "nb"):
        sub = 16 if case == "split16" else 32
        nb = nx // sub
        nif = 2 * nb * (nb - 1) + 8          # room for the quadtree's extra interfaces
        keep = dict(sub=np.array([sub], np.int32), nu=np.full(nif, 2, np.int32),
                    np_=np.full(nif, 2, np.int32), bt=np.zeros(2 * nx + 2 * ny, np.int8),
                    bv=np.zeros(2 * nx + 2 * ny), ref=np.zeros(nb * nb, np.int8))
        keep["bt"][:ny] = 1
        keep["ref"][0] = 1
        d = mrcm.MrcmDesc()
        d.nx, d.ny, d.n_real, d.ly = nx, ny, 1, 1.0
        P = ctypes.POINTER
        d.sub_size = keep["sub"].ctypes.data_as(P(ctypes.c_int32))
        d.iface_nU = keep["nu"].ctypes.data_as(P(ctypes.c_int32))
        d.iface_nP = keep["np_"].ctypes.data_as(P(ctypes.c_int32))
        d.bc_type = keep["bt"].ctypes.data_as(P(ctypes.c_int8))
        d.bc_val = keep["bv"].ctypes.data_as(P(ctypes.c_double))
        d.refine = keep["ref"].ctypes.data_as(P(ctypes.c_int8))
        d.prec = 1
        d.ir_tol, d.ir_max, d.iface_tol, d.iface_ir_max = 1e-13, 30, 1e-13, 40
        if case == "direct":
            d.iface_solver = mrcm.IFACE_DIRECT
        if case == "nb":
            d.precond = mrcm.PRECOND_NEIGHBOURHOOD
        ctx = ctypes.c_void_p()
        assert L.mrcm_setup(ctypes.byref(d), None, ctypes.byref(ctx)) == mrcm.MRCM_EINVAL, case
        assert b"refine" in L.mrcm_last_error(None), case
