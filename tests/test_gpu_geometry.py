"""Every launch geometry of the step kernels against the CPU oracle.

At setup the library measures the candidate geometries of the coarse-level
and SDIRK step kernels (CTAs per vector C, chunk length P) and keeps the
fastest, so ordinary runs exercise whichever won.  MGRIT_GEOM="C:P" forces
one; each geometry here is checked by one operator application (SL gather +
correction solve, or an SDIRK step: stage solves and L_p mat-vecs with halos
crossing threads and CTAs), to 1e-12 relative as in test_gpu_parity.py, and
a short solve that must match the oracle's MGRIT iteration for iteration."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import mgrit as omg
from oracle import operators as oops
from workloads import ic_fourier, ic_sin4

pytestmark = pytest.mark.gpu

GEOMS = [(c, p) for c in (1, 2, 4, 8, 16) for p in (4, 8, 16, 32)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture
def forced(monkeypatch):
    def set_geom(c, p):
        monkeypatch.setenv("MGRIT_GEOM", "%d:%d" % (c, p))
    yield set_geom
    monkeypatch.delenv("MGRIT_GEOM", raising=False)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def _solver(nx, nt, c, p, m, levels, kind=pkg.ERK, q=0, nu=1, seed=0, precision=pkg.FP64, tol=1e-10):
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, levels=levels, nu=nu, tol=tol, max_iter=40,
                          seed=seed, precision=precision)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("C,P", GEOMS)
def test_coarse_operator_every_geometry(forced, C, P):
    forced(C, P)
    nx, p, c, m, L = 1024, 3, 0.85, 8, 3
    s = _solver(nx, m ** (L - 1) * 2, c, p, m, L)
    x = np.random.default_rng(3).standard_normal((9, nx))
    for lev in range(1, L):
        info = s.level_info(lev)
        assert (int(info[7]), int(info[6])) == (C, P)
        y = torch.empty((9, nx), dtype=torch.float64, device="cuda")
        s.coarse_apply(lev, dev(x), y, 9)
        want = oops.coarse_operator(p, "erk", p, c, m, lev, L).apply(x)
        assert _rel(host(y), want) < 1e-12, (lev, C, P)
    s.close()


@pytest.mark.parametrize("C,P", GEOMS)
def test_sdirk_step_every_geometry(forced, C, P):
    forced(C, P)
    nx = 512
    for (p, q, c) in ((5, 3, 4.0), (5, 5, 6.0), (1, 1, 1.0)):
        s = _solver(nx, 64, c, p, 4, 2, kind=pkg.SDIRK, q=q)
        info = s.level_info(0)
        assert (int(info[7]), int(info[6])) == (C, P)
        x = np.random.default_rng(4).standard_normal((5, nx))
        y = torch.empty((5, nx), dtype=torch.float64, device="cuda")
        s.coarse_apply(0, dev(x), y, 5)
        want = oops.FineOperator(p, "sdirk", q, c).apply(x)
        assert _rel(host(y), want) < 1e-12, (p, q, C, P)
        s.close()


@pytest.mark.parametrize("C,P", [(1, 8), (2, 32), (4, 16), (16, 8)])
def test_solve_matches_oracle_forced_geometry(forced, C, P):
    forced(C, P)
    nx, nt, p, c, m, L = 512, 4 * 4 * 8, 3, 0.85, 4, 3
    u0 = ic_sin4(nx)
    s = _solver(nx, nt, c, p, m, L, seed=3)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    h = omg.Hierarchy(p, "erk", p, c, m, L)
    ref = omg.solve(h, u0, nt, nu=1, tol=1e-10, max_iter=40, seed=3)
    assert st["iterations"] == ref["iterations"]
    assert np.max(np.abs(host(out) - ref["u"][::m])) < 1e-10
    s.close()
    # SDIRK level 0 in the same geometry
    u1 = ic_fourier(nx, seed=4)
    s = _solver(nx, nt, 4.0, 5, m, L, kind=pkg.SDIRK, q=3, seed=3)
    st = s.solve(dev(u1), out, allow_unconverged=True)
    h = omg.Hierarchy(5, "sdirk", 3, 4.0, m, st["levels"])
    ref = omg.solve(h, u1, nt, nu=1, tol=1e-10, max_iter=40, seed=3)
    assert st["iterations"] == ref["iterations"]
    assert np.max(np.abs(host(out) - ref["u"][::m])) < 1e-10 * max(1.0, np.max(np.abs(u1)))
    s.close()


@pytest.mark.parametrize("C,P", [(1, 16), (4, 8), (8, 32)])
def test_mixed_solve_forced_geometry(forced, C, P):
    """FP32 kernels (FP32 SL + FP32 or FP64 correction solves, FP32 SDIRK
    stages) in forced geometries: the refined result matches sequential
    stepping (oracle) to the FP64 solve tolerance."""
    forced(C, P)
    nx, nt, m, L = 512, 4 * 4 * 8, 4, 3
    for kind, p, q, c, u0 in ((pkg.ERK, 3, 3, 0.85, ic_sin4(512)), (pkg.SDIRK, 5, 3, 4.0, ic_fourier(512, seed=2))):
        s = _solver(nx, nt, c, p, m, L, kind=kind, q=q, seed=1, precision=pkg.MIXED, tol=1e-11)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(dev(u0), out, allow_unconverged=True)
        assert st["converged"]
        fine = oops.FineOperator(p, "erk" if kind == pkg.ERK else "sdirk", q, c)
        u = u0.copy()
        ref = [u.copy()]
        for n in range(1, nt + 1):
            u = fine.apply(u)
            if n % m == 0:
                ref.append(u.copy())
        assert _rel(host(out), np.array(ref)) < 1e-10, (kind, C, P)
        s.close()


@pytest.mark.parametrize("code", [1, 2, 4, 8, 17, 18, 20, 24])
def test_level0_stencil_every_tile(monkeypatch, code):
    """Each tile of the level-0 composite-stencil kernel, classic and
    persistent (MGRIT_STENCIL = R, R + 16): a full solve matches the oracle's
    MGRIT iteration for iteration, in FP64 and MIXED (FP32 stencil)."""
    monkeypatch.setenv("MGRIT_STENCIL", str(code))
    nx, nt, p, c, m, L = 2048, 8 * 8 * 4, 3, 0.85, 8, 3
    u0 = ic_sin4(nx)
    s = _solver(nx, nt, c, p, m, L, seed=5)
    info = s.level_info(0)
    assert (int(info[6]), int(info[4])) == (code & 15, code >> 4)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    h = omg.Hierarchy(p, "erk", p, c, m, L)
    ref = omg.solve(h, u0, nt, nu=1, tol=1e-10, max_iter=40, seed=5)
    assert st["iterations"] == ref["iterations"]
    assert np.max(np.abs(host(out) - ref["u"][::m])) < 1e-10
    s.close()
    sm = _solver(nx, nt, c, p, m, L, seed=5, precision=pkg.MIXED, tol=1e-11)
    stm = sm.solve(dev(u0), out)
    assert stm["converged"]
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(h.fine, g)[::m]
    assert np.max(np.abs(host(out) - seq)) < 1e-10 * np.max(np.abs(seq))
    sm.close()
