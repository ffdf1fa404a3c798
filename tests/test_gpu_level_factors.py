"""A coarsening factor per level on the GPU (the paper's parallel runs
coarsen by m = 16 and then by 4, Sec. 6.3.2): the coarse operators of
every level against the oracle's (step m_1 .. m_l dt, the Sec. 6.2
recursion with the level's factor), and solves iteration for iteration."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _solver(nx, nt, c, p, m, mc, levels, kind=pkg.ERK, q=0, precision=pkg.FP64, coarse_op=pkg.SL_CORRECTED,
            seed=0, tol=1e-10):
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, m_coarse=mc, levels=levels, nu=1, tol=tol,
                          max_iter=40, seed=seed, precision=precision, coarse_op=coarse_op)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("kind,p,q,c,m,mc,levels,nx", [
    (pkg.ERK, 3, 3, 1.38, 16, 4, 4, 1024),
    (pkg.ERK, 1, 1, 0.85, 4, 2, 4, 256),
    (pkg.SDIRK, 3, 3, 5.0, 16, 4, 3, 512),
    (pkg.SDIRK, 5, 3, 4.0, 4, 8, 3, 2048),
])
def test_level_operators_match_oracle(kind, p, q, c, m, mc, levels, nx):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    ms = [m] + [mc] * (levels - 2)
    nt = m * mc ** (levels - 2) * 2
    s = _solver(nx, nt, c, p, m, mc, levels, kind, q)
    x = np.random.default_rng(4).standard_normal((5, nx))
    y = torch.empty((5, nx), dtype=torch.float64, device="cuda")
    step = 1
    for lev in range(1, levels):
        step *= ms[lev - 1]
        assert s.level_info(lev)[5] == step
        s.coarse_apply(lev, dev(x), y, 5)
        want = oops.coarse_operator(p, kname, q, c, ms, lev, levels).apply(x)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), want) < 1e-12, lev
    s.close()


@pytest.mark.parametrize("kind,p,q,c,m,mc,levels,nx,nt,coarse_op", [
    (pkg.ERK, 3, 3, 1.38, 16, 4, 3, 64, 512, pkg.SL_CORRECTED),
    (pkg.ERK, 3, 3, 1.38, 4, 8, 3, 128, 256, pkg.SL_CORRECTED),
    (pkg.SDIRK, 3, 3, 5.0, 16, 4, 3, 64, 512, pkg.SL_CORRECTED),
    (pkg.SDIRK, 1, 1, 1.0, 8, 2, 4, 64, 256, pkg.REDISC),
])
def test_solve_matches_oracle(kind, p, q, c, m, mc, levels, nx, nt, coarse_op):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    ms = [m] + [mc] * (levels - 2)
    u0 = ic_sin4(nx)
    s = _solver(nx, nt, c, p, m, mc, levels, kind, q, coarse_op=coarse_op, seed=3)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    name = {pkg.SL_CORRECTED: "sl_corrected", pkg.REDISC: "redisc"}[coarse_op]
    ref = omg.solve(omg.Hierarchy(p, kname, q, c, ms, levels, coarse_op=name), u0, nt, tol=1e-10, max_iter=40,
                    seed=3)
    assert st["iterations"] == ref["iterations"]
    hist, href = np.array(st["history"]), np.array(ref["history"])
    big = href > 1e-8 * href[0]
    assert np.max(np.abs(hist[big] - href[big]) / href[big]) < 1e-6
    if ref["converged"]:
        torch.cuda.synchronize()
        assert np.max(np.abs(out.cpu().numpy() - ref["u"][::m])) < 1e-10 * max(1.0, np.max(np.abs(u0)))
    s.close()


def test_paper_parallel_configuration_small():
    """m = 16, m_coarse = 4, coarsening until fewer than two time points
    (levels = 0): 4096 steps give levels of 4096, 256, 64, 16, 4 steps;
    MIXED converges to sequential stepping."""
    nx, nt = 256, 4096
    s = _solver(nx, nt, 1.38, 3, 16, 4, 0, precision=pkg.MIXED, seed=1, tol=1e-11)
    u0 = ic_fourier(nx, seed=5)
    out = torch.empty((nt // 16 + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out)
    assert st["converged"] and st["levels"] == 5
    assert [s.level_info(l)[0] for l in range(5)] == [4096, 256, 64, 16, 4]
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(oops.FineOperator(3, "erk", 3, 1.38), g)[::16]
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), seq) < 1e-10
    s.close()


def test_level_factors_with_gmres_correction_solves():
    """GMRES correction solves on levels of steps 16 dt and 64 dt: the same
    iterate and iteration counts as the oracle's GMRES on those levels."""
    from oracle import gmres as ogm
    nx, m, mc, levels = 512, 16, 4, 3
    prm = pkg.make_params(nx, m * mc * 2, 1.38, 3, m=m, m_coarse=mc, levels=levels,
                          coarse_solve=pkg.GMRES)
    s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
    x = np.random.default_rng(8).standard_normal((4, nx))
    y = torch.empty((4, nx), dtype=torch.float64, device="cuda")
    for lev in (1, 2):
        s.coarse_apply(lev, dev(x), y, 4)
        op = oops.coarse_operator(3, "erk", 3, 1.38, [m, mc], lev, levels, gmres=(1e-2, ogm.default_maxit(3)))
        want = op.apply(x)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), want) < 1e-12
        assert s.gmres_stats(lev)[0] == sum(op.gmres_its)
    s.close()


@pytest.mark.parametrize("kind,p,c", [(pkg.ERK, 4, 0.3), (pkg.SDIRK, 2, 1.0)])
def test_level_factors_with_even_p(kind, p, c):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    nx, m, mc, levels = 1024, 8, 2, 4
    s = _solver(nx, m * mc * mc * 2, c, p, m, mc, levels, kind, p)
    x = np.random.default_rng(p).standard_normal((3, nx))
    y = torch.empty((3, nx), dtype=torch.float64, device="cuda")
    for lev in range(1, levels):
        s.coarse_apply(lev, dev(x), y, 3)
        want = oops.coarse_operator(p, kname, p, c, [m, mc, mc], lev, levels).apply(x)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), want) < 1e-12, lev
    s.close()


def test_batch_with_level_factors_equals_standalone():
    """A batch whose solves coarsen differently (uniform and 16 then 4,
    different depths) gives every solve's standalone result bit for bit."""
    from workloads import ic_sin4_noise
    cases = [(256, 1024, 16, 4, pkg.FP64), (512, 2048, 8, 2, pkg.MIXED), (256, 512, 4, 4, pkg.FP64),
             (1024, 4096, 16, 4, pkg.MIXED)]
    prms = [pkg.make_params(nx, nt, 1.2, 3, m=m, m_coarse=mc, levels=0, tol=1e-10, max_iter=60, seed=i,
                            precision=prec) for i, (nx, nt, m, mc, prec) in enumerate(cases)]
    u0s = [ic_sin4_noise(nx, seed=i) for i, (nx, *_rest) in enumerate(cases)]
    b = pkg.Batch(prms, nstreams=2)
    stats = b.solve(u0s, allow_unconverged=True)
    for i, (prm, u0) in enumerate(zip(prms, u0s)):
        s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
        want = np.zeros((prm.nt // prm.m + 1, prm.nx))
        st = s.solve(u0, want, allow_unconverged=True)
        s.close()
        assert st["converged"] and stats[i]["iterations"] == st["iterations"]
        assert np.array_equal(b.get(i), want), i
    b.close()
