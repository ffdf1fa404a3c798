"""The C-ABI library loads on a CPU-only machine, exports every entry point
declared in include/mgrit.h, and rejects invalid parameters before touching a
GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2209_06916_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mgrit_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        pytest.skip("libmgrit.so not built (run __graft_entry__.build())")
    return pkg.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mgrit_setup", "mgrit_relax", "mgrit_residual", "mgrit_coarse_apply",
                     "mgrit_solve", "mgrit_destroy", "mgrit_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_texts(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.mgrit_strerror(code)
    assert lib.mgrit_strerror(-7) == b"singular or unstable coarse correction"


@pytest.mark.parametrize("kw", [
    dict(nx=30, nt=128, cfl=0.85, p=1),            # nx too small / not a multiple of 8
    dict(nx=64, nt=128, cfl=0.85, p=6),            # p outside 1..5
    dict(nx=64, nt=128, cfl=0.85, p=0),
    dict(nx=64, nt=130, cfl=0.85, p=1, m=4),       # nt % m
    dict(nx=64, nt=128, cfl=0.85, p=1, m=4, levels=5),  # nt % m^(L-1)
    dict(nx=64, nt=128, cfl=-1.0, p=1),            # c <= 0
    dict(nx=64, nt=128, cfl=0.85, p=3, q=1),       # ERK needs q = p
    dict(nx=64, nt=128, cfl=0.85, p=1, nu=7),      # nu range
    dict(nx=64, nt=128, cfl=0.85, p=1, precision=3),  # precision mode
    dict(nx=8 * 20000, nt=128, cfl=0.85, p=1),     # no chunk geometry (n > 16 CTAs x 256 x 32)
])
def test_invalid_parameters_rejected_on_host(lib, kw):
    prm = pkg.make_params(**kw)
    h = ctypes.c_void_p()
    assert lib.mgrit_setup(ctypes.byref(prm), None, ctypes.byref(h)) == -1
    assert not h.value


@pytest.mark.parametrize("p,q", [(3, 2), (3, 4), (3, 5), (2, 1), (4, 3), (4, 2)])
def test_sdirk_q_outside_the_correction_band_unsupported(lib, p, q):
    """SDIRKq with q != p needs an odd q <= p (the phi_q D^{(q+1)} term);
    even p pairs q = p only."""
    prm = pkg.make_params(64, 128, 2.0, p, kind=pkg.SDIRK, q=q)
    h = ctypes.c_void_p()
    assert lib.mgrit_setup(ctypes.byref(prm), None, ctypes.byref(h)) == -8


def test_binding_refuses_wrong_dtypes():
    import numpy as np
    with pytest.raises(ValueError):
        pkg._ptr(np.zeros(4, dtype=np.float32))


def test_coarse_operator_choice_validated_on_host(lib):
    bad = pkg.make_params(64, 128, 0.85, 1, coarse_op=7)
    h = ctypes.c_void_p()
    assert lib.mgrit_setup(ctypes.byref(bad), None, ctypes.byref(h)) == -1
    # rediscretising ERK at m dt is unstable for practical m c (Sec. 5)
    erk = pkg.make_params(64, 128, 0.85, 1, coarse_op=pkg.REDISC)
    assert lib.mgrit_setup(ctypes.byref(erk), None, ctypes.byref(h)) == -8
    assert not h.value


@pytest.mark.parametrize("kw", [
    dict(coarse_solve=2),                                  # unknown correction solve
    dict(coarse_solve=pkg.GMRES, coarse_op=pkg.SL),        # the direct SL operator has no correction system
    dict(coarse_solve=pkg.GMRES, gmres_maxit=33),          # above the kernel's cap of 32
    dict(coarse_solve=pkg.GMRES, gmres_maxit=-1),
    dict(coarse_solve=pkg.GMRES, gmres_rtol=1.5),          # relative tolerance outside (0, 1)
    dict(coarse_solve=pkg.GMRES, gmres_rtol=-1e-2),
])
def test_gmres_parameters_validated_on_host(lib, kw):
    prm = pkg.make_params(64, 128, 0.85, 3, **kw)
    h = ctypes.c_void_p()
    assert lib.mgrit_setup(ctypes.byref(prm), None, ctypes.byref(h)) == -1
    assert not h.value


def test_estimate_counts_the_gmres_basis(lib):
    """The admission estimate grows by the Krylov basis: max(K_l, 1) x
    (cap + 1) rows of n_x doubles per coarse level."""
    lib.mgrit_estimate_bytes.restype = ctypes.c_int64
    d = pkg.make_params(256, 1024, 0.85, 3, m=4, levels=3)
    g = pkg.make_params(256, 1024, 0.85, 3, m=4, levels=3, coarse_solve=pkg.GMRES, gmres_maxit=20)
    extra = lib.mgrit_estimate_bytes(ctypes.byref(g)) - lib.mgrit_estimate_bytes(ctypes.byref(d))
    assert extra == (64 + 1) * 21 * 256 * 8  # level 1: 64 intervals; level 2 (coarsest): one vector


def test_level_factor_validated_and_estimated(lib):
    """m_coarse: 0 means m; below 2 is rejected; n_t must divide by
    m m_coarse^(levels-2); the admission estimate follows the level sizes."""
    h = ctypes.c_void_p()
    bad = pkg.make_params(64, 128, 0.85, 3, m=4, levels=3, m_coarse=1)
    assert lib.mgrit_setup(ctypes.byref(bad), None, ctypes.byref(h)) == -1
    bad = pkg.make_params(64, 96, 0.85, 3, m=4, levels=3, m_coarse=16)   # 96 = 4 * 24, 24 % 16 != 0
    assert lib.mgrit_setup(ctypes.byref(bad), None, ctypes.byref(h)) == -1
    lib.mgrit_estimate_bytes.restype = ctypes.c_int64
    a = pkg.make_params(256, 1024, 0.85, 3, m=16, levels=3, m_coarse=4)
    # levels: 1024 steps (K 64), 64 steps (K 16), 16 steps (coarsest)
    rows = 2 * 65 + (65 + 2 * 17) + 17
    assert lib.mgrit_estimate_bytes(ctypes.byref(a)) == rows * 256 * 8 + (4 << 20)
