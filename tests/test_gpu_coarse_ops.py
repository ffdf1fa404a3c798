"""Direct coarse-grid operators on the GPU against the oracle (Sec. 5): the
uncorrected semi-Lagrangian operator S_p^{(m^l dt)} and, for SDIRK, the
rediscretised fine method R_q(-m^l c L_p).  One application agrees to
1e-12 relative; solves agree with the oracle's MGRIT iteration for iteration
(same algorithm, same random iterate); the measured two-level factor sits
near the LFA prediction, as in the Sec. 5.3 figure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
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


def _solver(nx, nt, c, p, m, levels, kind, q, coarse_op, nu=1, seed=0, precision=pkg.FP64, max_iter=40, tol=1e-10):
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, levels=levels, nu=nu, tol=tol, max_iter=max_iter,
                          seed=seed, precision=precision, coarse_op=coarse_op)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


NAME = {pkg.SL: "sl", pkg.REDISC: "redisc"}


@pytest.mark.parametrize("kind,p,q,c,m,levels,nx,coarse_op", [
    (pkg.ERK, 3, 3, 0.85, 8, 3, 1024, pkg.SL),
    (pkg.ERK, 1, 1, 0.85, 4, 3, 256, pkg.SL),
    (pkg.SDIRK, 5, 3, 4.0, 16, 3, 2048, pkg.SL),
    (pkg.SDIRK, 1, 1, 1.0, 2, 4, 256, pkg.REDISC),
    (pkg.SDIRK, 3, 3, 2.0, 4, 3, 512, pkg.REDISC),
    (pkg.SDIRK, 5, 5, 3.0, 4, 3, 1024, pkg.REDISC),
    (pkg.SDIRK, 5, 3, 4.0, 16, 3, 4096, pkg.REDISC),
])
def test_direct_coarse_operator_matches_oracle(kind, p, q, c, m, levels, nx, coarse_op):
    s = _solver(nx, m ** (levels - 1) * 2, c, p, m, levels, kind, q, coarse_op)
    x = np.random.default_rng(11).standard_normal((6, nx))
    kname = "erk" if kind == pkg.ERK else "sdirk"
    for lev in range(1, levels):
        y = torch.empty((6, nx), dtype=torch.float64, device="cuda")
        s.coarse_apply(lev, dev(x), y, 6)
        want = oops.direct_operator(p, kname, q, c, m, lev, NAME[coarse_op]).apply(x)
        assert _rel(host(y), want) < 1e-12, (lev, _rel(host(y), want))
    s.close()


def test_redisc_is_sdirk_only():
    prm = pkg.make_params(64, 64, 0.5, 1, kind=pkg.ERK, m=4, levels=2, coarse_op=pkg.REDISC)
    with pytest.raises(pkg.MgritError) as e:
        pkg.Solver(prm)
    assert e.value.code == -8


@pytest.mark.parametrize("kind,p,q,c,m,levels,nx,nt,coarse_op,nu", [
    (pkg.SDIRK, 1, 1, 1.0, 2, 2, 128, 256, pkg.REDISC, 1),   # the Sec. 5.3 figure setting, two-level
    (pkg.SDIRK, 1, 1, 4.0, 4, 3, 128, 4 * 4 * 8, pkg.REDISC, 1),
    (pkg.SDIRK, 3, 3, 0.5, 2, 3, 128, 2 * 2 * 16, pkg.REDISC, 0),
    (pkg.ERK, 3, 3, 0.85, 4, 3, 256, 4 * 4 * 8, pkg.SL, 1),
    (pkg.ERK, 1, 1, 0.85, 4, 2, 128, 512, pkg.SL, 0),
])
def test_direct_operator_solve_matches_oracle(kind, p, q, c, m, levels, nx, nt, coarse_op, nu):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    u0 = ic_sin4(nx) if p < 5 else ic_fourier(nx, seed=1)
    s = _solver(nx, nt, c, p, m, levels, kind, q, coarse_op, nu=nu, seed=7)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    h = omg.Hierarchy(p, kname, q, c, m, levels, coarse_op=NAME[coarse_op])
    ref = omg.solve(h, u0, nt, nu=nu, tol=1e-10, max_iter=40, seed=7)
    assert st["iterations"] == ref["iterations"]
    hist, href = np.array(st["history"]), np.array(ref["history"])
    big = href > 1e-8 * href[0]
    assert np.max(np.abs(hist[big] - href[big]) / href[big]) < 1e-6
    if ref["converged"]:
        assert np.max(np.abs(host(out) - ref["u"][::m])) < 1e-10 * max(1.0, np.max(np.abs(u0)))
    s.close()


@pytest.mark.parametrize("p,c,m", [(1, 1.0, 2), (1, 4.0, 2), (1, 1.0, 4), (3, 0.5, 2)])
def test_redisc_measured_factor_near_lfa(p, c, m):
    """Two-level MGRIT with rediscretisation at 2^10 x 2^12 (the size of the
    Sec. 5.3 experiments): the final-iteration factor is within [0.5, 1.15]
    of the two-level LFA prediction."""
    nx, nt = 1 << 10, 1 << 12
    s = _solver(nx, nt, c, p, m, 2, pkg.SDIRK, p, pkg.REDISC, max_iter=60)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(ic_sin4(nx)), out, allow_unconverged=True)
    pred = lfa.two_level_factor(p, "sdirk", c, m, coarse_op="redisc")
    assert st["converged"]
    assert 0.5 * pred < st["conv_factor"] < 1.15 * pred, (st["conv_factor"], pred)
    s.close()


def test_mixed_precision_with_rediscretised_levels():
    nx, nt, m, L = 256, 4 * 4 * 8, 4, 3
    u0 = ic_fourier(nx, seed=3)
    s = _solver(nx, nt, 1.0, 1, m, L, pkg.SDIRK, 1, pkg.REDISC, seed=2, precision=pkg.MIXED, tol=1e-11)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out)
    assert st["converged"]
    fine = oops.FineOperator(1, "sdirk", 1, 1.0)
    u, ref = u0.copy(), [u0.copy()]
    for n in range(1, nt + 1):
        u = fine.apply(u)
        if n % m == 0:
            ref.append(u.copy())
    assert _rel(host(out), np.array(ref)) < 1e-10
    s.close()
