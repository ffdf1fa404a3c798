"""Dispersive discretisations (even p, Sec. 6.4) on the GPU against the
oracle: U2 / U4 with ERK2 / ERK4 and SDIRK2 / SDIRK4, the coarse SL step on
the eps-dependent node set and the first-order, left-biased D^{(p+1)}_1 in
the correction.  Applications agree with the oracle's to 1e-12 on both node
sets; two-level solves follow the oracle's MGRIT iteration for iteration,
including the jump of the ERK4+U4 factor across c / c_max = 0.24 (m = 2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import coefficients as oco
from oracle import lfa
from oracle import mgrit as omg
from oracle import operators as oops
from workloads import ic_fourier, ic_sin4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def _solver(nx, nt, c, p, m, levels, kind, nu=1, seed=0, precision=pkg.FP64, max_iter=40, tol=1e-10):
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=p, m=m, levels=levels, nu=nu, tol=tol, max_iter=max_iter,
                          seed=seed, precision=precision)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


def _cmax(p):
    return oco.cfl_limit(p)


@pytest.mark.parametrize("kind,p,c,m,levels,nx", [
    (pkg.ERK, 2, 0.35, 4, 3, 512),
    (pkg.ERK, 4, 0.240, 2, 3, 256),    # m c = 0.48: eps < 1/2, nodes centred on x_{i-k}
    (pkg.ERK, 4, 0.261, 2, 3, 256),    # m c = 0.52: eps > 1/2, nodes centred on x_{i-k-1}
    (pkg.ERK, 4, 0.7, 4, 3, 1024),
    (pkg.SDIRK, 2, 1.0, 4, 3, 512),
    (pkg.SDIRK, 4, 1.0, 2, 4, 1024),
])
def test_even_p_operators_match_oracle(kind, p, c, m, levels, nx):
    """Phi (level 0) and Psi_l (every coarse level) on 6 random vectors."""
    kname = "erk" if kind == pkg.ERK else "sdirk"
    s = _solver(nx, m ** (levels - 1) * 2, c, p, m, levels, kind)
    x = np.random.default_rng(p * 7 + m).standard_normal((6, nx))
    y = torch.empty((6, nx), dtype=torch.float64, device="cuda")
    s.coarse_apply(0, dev(x), y, 6)
    assert _rel(host(y), oops.FineOperator(p, kname, p, c).apply(x)) < 1e-12
    for lev in range(1, levels):
        s.coarse_apply(lev, dev(x), y, 6)
        want = oops.coarse_operator(p, kname, p, c, m, lev, levels).apply(x)
        assert _rel(host(y), want) < 1e-12, (lev, _rel(host(y), want))
    s.close()


@pytest.mark.parametrize("kind,p,c,m,nx,nt", [
    (pkg.ERK, 2, 0.35, 4, 128, 512),
    (pkg.ERK, 4, 0.240, 2, 128, 256),
    (pkg.ERK, 4, 0.261, 2, 128, 256),
    (pkg.SDIRK, 2, 1.0, 4, 128, 256),
    (pkg.SDIRK, 4, 1.0, 2, 128, 256),
])
def test_even_p_two_level_solve_matches_oracle(kind, p, c, m, nx, nt):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    u0 = ic_sin4(nx)
    s = _solver(nx, nt, c, p, m, 2, kind, seed=5, max_iter=100)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    ref = omg.solve(omg.Hierarchy(p, kname, p, c, m, 2), u0, nt, nu=1, tol=1e-10, max_iter=100, seed=5)
    assert st["iterations"] == ref["iterations"]
    hist, href = np.array(st["history"]), np.array(ref["history"])
    big = href > 1e-8 * href[0]
    assert np.max(np.abs(hist[big] - href[big]) / href[big]) < 1e-6
    if ref["converged"]:
        assert np.max(np.abs(host(out) - ref["u"][::m])) < 1e-10 * max(1.0, np.max(np.abs(u0)))
    s.close()


def test_erk4_u4_factor_jump_measured_on_the_gpu():
    """Sec. 6.4: ERK4+U4, m = 2, two-level, 2^10 x 2^12: the measured factor
    jumps across c / c_max = 0.24 as the LFA predicts (0.15 -> 0.84)."""
    nx, nt, m = 1 << 10, 1 << 12, 2
    fac = {}
    for frac in (0.23, 0.25):
        c = frac * _cmax(4)
        s = _solver(nx, nt, c, 4, m, 2, pkg.ERK, max_iter=100)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(dev(ic_sin4(nx)), out, allow_unconverged=True)
        pred = lfa.two_level_factor(4, "erk", c, m, omit=10)
        assert st["converged"] and st["conv_factor"] < 1.05 * pred, (frac, st["conv_factor"], pred)
        fac[frac] = st["conv_factor"]
        s.close()
    assert fac[0.25] > 3 * fac[0.23]


@pytest.mark.parametrize("C,P", [(1, 4), (2, 8), (4, 4), (8, 16), (16, 4), (4, 32)])
def test_even_p_every_geometry(monkeypatch, C, P):
    monkeypatch.setenv("MGRIT_GEOM", "%d:%d" % (C, P))
    for kind, p, c, m in ((pkg.ERK, 4, 0.7, 4), (pkg.SDIRK, 2, 1.0, 4)):
        kname = "erk" if kind == pkg.ERK else "sdirk"
        nx, levels = 2048, 3
        s = _solver(nx, m ** (levels - 1) * 2, c, p, m, levels, kind)
        x = np.random.default_rng(C + P).standard_normal((3, nx))
        y = torch.empty((3, nx), dtype=torch.float64, device="cuda")
        for lev in (1, 2):
            s.coarse_apply(lev, dev(x), y, 3)
            want = oops.coarse_operator(p, kname, p, c, m, lev, levels).apply(x)
            assert _rel(host(y), want) < 1e-12, (kind, lev)
        if kind == pkg.SDIRK:
            s.coarse_apply(0, dev(x), y, 3)
            assert _rel(host(y), oops.FineOperator(p, kname, p, c).apply(x)) < 1e-12
        s.close()


@pytest.mark.parametrize("precision", [pkg.MIXED, pkg.MIXED_FAST])
def test_even_p_mixed_precision(precision):
    nx, nt, m = 256, 512, 4
    u0 = ic_fourier(nx, seed=2)
    s = _solver(nx, nt, 0.35, 2, m, 2, pkg.ERK, precision=precision, seed=1, tol=1e-11)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out)
    assert st["converged"]
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(oops.FineOperator(2, "erk", 2, 0.35), g)[::m]
    assert _rel(host(out), seq) < 1e-10
    s.close()
