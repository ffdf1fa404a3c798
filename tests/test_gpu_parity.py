"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64 everywhere):
  * one operator application (fine step, composite Phi^m, coarse Psi_l): both
    sides round each of at most a few hundred products, so the difference is
    bounded by ~1e-15 * sum|coef| * max|x|; the tests use 1e-12 * max|x|.
  * MGRIT iterates: identical algorithm and random initial iterate (the same
    SplitMix64 stream on both sides), so per-iteration C-point values agree
    to rounding (1e-10 absolute on O(1) data) and iteration counts are equal.
  * converged solution vs sequential stepping: a relative residual does not
    bound the error by itself (the error is at most ||A^{-1}|| ||r||), so the
    solves stop at a 1e-11 relative residual and every C-point must be within
    1e-10 relative (max over all C-points and grid points, over the largest
    value of sequential stepping) of the oracle's sequential stepping.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import coefficients as co
from oracle import lfa
from oracle import mgrit as omg
from oracle import operators as oops
from oracle import rng as orng
from workloads import ic_sin4, ic_sin4_noise

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


def solver(nx, nt, c, p, m, levels, nu=1, tol=1e-10, max_iter=30, seed=0, kind=pkg.ERK, q=0):
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, levels=levels, nu=nu, tol=tol,
                          max_iter=max_iter, seed=seed)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


# ---------------------------------------------------------------------------
# single operators
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p,c,nx", [(1, 0.85, 64), (1, 0.3, 1536), (3, 0.85, 96), (3, 1.38, 4096),
                                    (5, 1.2, 256), (5, 0.6, 40)])
def test_fine_step_matches_oracle(p, c, nx):
    s = solver(nx, 64, c, p, 4, 2)
    x = np.random.default_rng(1).standard_normal((37, nx))
    y = torch.empty((37, nx), dtype=torch.float64, device="cuda")
    s.coarse_apply(0, dev(x), y, 37)
    want = oops.FineOperator(p, "erk", p, c).apply(x)
    assert _rel(host(y), want) < 1e-12


CASES = [  # p, c, m, levels, nx
    (1, 0.85, 4, 2, 256),
    (3, 0.85, 8, 4, 4096),
    (3, 0.85, 8, 4, 96),
    (5, 0.9, 4, 4, 512),
    (3, 1.2, 2, 6, 64),
    (1, 0.5, 16, 3, 1536),
    (5, 1.5, 8, 3, 40),
    (5, 0.9, 16, 4, 4096),   # deep level: |phi| ~ 1e3, slow decay, 16-CTA clusters
    (1, 0.85, 4, 5, 2048),
]


@pytest.mark.parametrize("p,c,m,levels,nx", CASES)
def test_coarse_operators_match_oracle(p, c, m, levels, nx):
    nt = m ** (levels - 1) * 2
    s = solver(nx, nt, c, p, m, levels)
    x = np.random.default_rng(2).standard_normal((19, nx))
    for lev in range(1, levels):
        y = torch.empty((19, nx), dtype=torch.float64, device="cuda")
        s.coarse_apply(lev, dev(x), y, 19)
        op = oops.coarse_operator(p, "erk", p, c, m, lev, levels)
        assert _rel(host(y), op.apply(x)) < 1e-12, lev
        info = s.level_info(lev)
        k, eps = co.sl_shift(c * m ** lev)
        assert int(info[1]) == k and abs(info[2] - eps) < 1e-12
        assert abs(info[3] - co.phi_levels(p, "erk", c, m, levels)[lev - 1]) < 1e-9 * max(1, abs(info[3]))
        assert info[7] >= 1


# ---------------------------------------------------------------------------
# relaxation and residual, level by level
# ---------------------------------------------------------------------------

def _full_from_cpoints(op, uC, m, g=None):
    """All time points of a level from its C-points by F-relaxation."""
    K = uC.shape[0] - 1
    u = np.zeros((K * m + 1, uC.shape[1]))
    u[::m] = uC
    gg = np.zeros_like(u) if g is None else g
    omg.f_relax(op, u, gg, m)
    return u, gg


@pytest.mark.parametrize("p,c,m,nx,nt", [(1, 0.85, 4, 256, 1024), (3, 0.85, 8, 96, 8 * 37),
                                         (5, 1.1, 16, 512, 16 * 9)])
def test_level0_relax_and_residual(p, c, m, nx, nt):
    s = solver(nx, nt, c, p, m, 2)
    K = nt // m
    uC = np.random.default_rng(3).standard_normal((K + 1, nx))
    s.level_set(0, 0, uC)
    s.relax(0, 1)
    got = s.level_get(0, 0)
    fine = oops.FineOperator(p, "erk", p, c)
    u, g = _full_from_cpoints(fine, uC, m)
    omg.c_relax(fine, u, g, m)
    assert _rel(got, u[::m]) < 1e-12
    nrm = s.residual(0)
    omg.f_relax(fine, u, g, m)
    r = omg.c_residual(fine, u, g, m)
    got_r = s.level_get(1, 1)
    assert np.max(np.abs(got_r - r)) < 1e-12 * np.max(np.abs(u))
    assert abs(nrm - np.sqrt(np.sum(r * r))) < 1e-10 * max(1.0, nrm)


def test_coarse_level_relax_and_residual():
    p, c, m, nx, L = 3, 0.85, 4, 128, 3
    nt = m ** 2 * 5
    s = solver(nx, nt, c, p, m, L)
    N1 = nt // m
    rs = np.random.default_rng(4)
    g1 = rs.standard_normal((N1 + 1, nx))
    g1[0] = 0.0
    u1 = rs.standard_normal((N1 // m + 1, nx))
    u1[0] = 0.0
    s.level_set(1, 1, g1)
    s.level_set(1, 0, u1)
    s.relax(1, 1)
    op = oops.coarse_operator(p, "erk", p, c, m, 1, L)
    u, g = _full_from_cpoints(op, u1, m, g1)
    omg.c_relax(op, u, g, m)
    assert _rel(s.level_get(1, 0), u[::m]) < 1e-12
    s.residual(1)
    omg.f_relax(op, u, g, m)
    r = omg.c_residual(op, u, g, m)
    assert np.max(np.abs(s.level_get(2, 1) - r)) < 1e-12 * np.max(np.abs(u))


# ---------------------------------------------------------------------------
# whole solves
# ---------------------------------------------------------------------------

SOLVES = [  # p, c, m, levels, nu, nx, nt
    (1, 0.85, 4, 2, 1, 256, 1024),     # two-level, ERK1+U1 (C1 shape)
    (3, 0.85, 8, 4, 1, 128, 8 ** 3 * 2),  # V-cycle ERK3+U3
    (3, 1.382, 2, 0, 1, 64, 256),      # Table-3 shape, automatic levels
    (5, 0.9, 4, 3, 1, 96, 4 ** 2 * 7),  # ERK5+U5, ragged nx
    (3, 0.85, 4, 3, 2, 64, 16 * 6),    # nu = 2
    (1, 0.85, 4, 3, 0, 64, 16 * 4),    # F-relaxation only
]


@pytest.mark.parametrize("p,c,m,levels,nu,nx,nt", SOLVES)
def test_solve_matches_oracle_mgrit(p, c, m, levels, nu, nx, nt):
    u0 = ic_sin4(nx)
    s = solver(nx, nt, c, p, m, levels, nu=nu, tol=1e-11, max_iter=40, seed=7)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    L = st["levels"]
    h = omg.Hierarchy(p, "erk", p, c, m, L)
    ref = omg.solve(h, u0, nt, nu=nu, tol=1e-11, max_iter=40, seed=7)
    assert st["iterations"] == ref["iterations"]
    assert st["converged"] == ref["converged"]
    hist = np.array(st["history"])
    href = np.array(ref["history"])
    assert len(hist) == len(href)
    big = href > 1e-8 * href[0]
    assert np.max(np.abs(hist[big] - href[big]) / href[big]) < 1e-6
    got = host(out)
    assert np.max(np.abs(got - ref["u"][::m])) < 1e-10
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(h.fine, g)[::m]
    assert _rel(got, seq) < 1e-10, _rel(got, seq)


def test_two_level_f_relaxation_exactness_on_gpu():
    nx, nt, m, c = 64, 48, 4, 1.2
    u0 = ic_sin4(nx)
    s = solver(nx, nt, c, 3, m, 2, nu=0, tol=0.0, max_iter=nt // m)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    s.solve(dev(u0), out, allow_unconverged=True)
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(oops.FineOperator(3, "erk", 3, c), g)[::m]
    assert np.max(np.abs(host(out) - seq)) < 1e-12


def test_random_initial_iterate_matches_splitmix64():
    nx, nt, m = 64, 64, 4
    s = solver(nx, nt, 0.85, 1, m, 2, seed=12345)
    u0 = ic_sin4(nx)
    s.set_initial(dev(u0))
    got = s.level_get(0, 0)
    want = orng.uniform_grid(12345, np.arange(0, nt + 1, m), nx)
    want[0] = u0
    assert np.array_equal(got, want)


def test_solve_is_deterministic():
    nx, nt = 256, 1024
    outs = []
    for _ in range(2):
        s = solver(nx, nt, 0.85, 1, 4, 2, seed=3)
        out = torch.empty((nt // 4 + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(dev(ic_sin4(nx)), out)
        outs.append((host(out), st["history"]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_divergence_reported_above_cfl_limit():
    nx, nt = 64, 256
    s = solver(nx, nt, 2.5, 3, 4, 2, max_iter=30)  # ERK3+U3 is unstable for c > 1.626
    st = s.solve(dev(ic_sin4(nx)), None, allow_unconverged=True)
    assert st["status"] in (-3, -4)


# ---------------------------------------------------------------------------
# full-size workload of the benchmark (4096 x 16384, ERK3+U3, 4-level V-cycle)
# ---------------------------------------------------------------------------

def test_full_size_vcycle_against_sequential_stepping():
    nx, nt, m, c, L = 4096, 16384, 8, 0.85, 4
    u0 = ic_sin4_noise(nx, seed=0)
    s = solver(nx, nt, c, 3, m, L, tol=1e-11, max_iter=30, seed=0)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out)
    assert st["converged"]
    got = host(out)
    fine = oops.FineOperator(3, "erk", 3, c)
    u = u0.copy()
    err = float(np.max(np.abs(got[0] - u0)))
    scale = np.max(np.abs(u0))
    for n in range(1, nt + 1):
        u = fine.apply(u)
        if n % m == 0:
            err = max(err, float(np.max(np.abs(got[n // m] - u))))
            scale = max(scale, float(np.max(np.abs(u))))
    print("full-size: iterations=%d rel err vs sequential=%.3e" % (st["iterations"], err / scale))
    assert err / scale < 1e-10
    # the V-cycle converges as fast as the two-level LFA predicts (Sec. 6.3:
    # little deterioration from two levels to V-cycles)
    assert st["conv_factor"] < 1.2 * lfa.two_level_factor(3, "erk", c, m), st["conv_factor"]


# ---------------------------------------------------------------------------
# GPU sequential time-stepping (the baseline MGRIT is measured against)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p,c,nx,nsteps,every", [(1, 0.85, 256, 1000, 0), (3, 0.85, 4096, 1000, 0),
                                                  (3, 1.2, 96, 77, 7), (5, 0.9, 512, 130, 13),
                                                  (3, 0.85, 4096, 512, 64)])
def test_sequential_stepping_matches_oracle(p, c, nx, nsteps, every):
    s = solver(nx, 64, c, p, 4, 2)
    u0 = ic_sin4_noise(nx, seed=5)
    out = torch.empty(nx, dtype=torch.float64, device="cuda")
    traj = None
    if every:
        traj = torch.zeros((nsteps // every, nx), dtype=torch.float64, device="cuda")
    s.fine_propagate(dev(u0), out, nsteps, every, traj)
    fine = oops.FineOperator(p, "erk", p, c)
    u = u0.copy()
    rows = []
    for n in range(1, nsteps + 1):
        u = fine.apply(u)
        if every and n % every == 0:
            rows.append(u.copy())
    # FP64 rounding accumulates linearly in the number of steps
    assert _rel(host(out), u) < 1e-13 * nsteps
    if every:
        assert _rel(host(traj), np.array(rows)) < 1e-13 * nsteps
    host_out = np.zeros(nx)
    s.fine_propagate(u0, host_out, nsteps)  # host pointers
    assert _rel(host_out, u) < 1e-13 * nsteps


# ---------------------------------------------------------------------------
# graph-resident solve (conditional while node, stop test on the device)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,p,c,m,levels,nu,prec,nx,nt", [
    (pkg.ERK, 3, 0.85, 8, 4, 1, pkg.FP64, 128, 8 ** 3 * 2),
    (pkg.ERK, 1, 0.85, 4, 2, 1, pkg.FP64, 256, 1024),
    (pkg.ERK, 3, 0.85, 4, 3, 2, pkg.FP64, 64, 16 * 6),
    (pkg.SDIRK, 3, 5.0, 4, 3, 1, pkg.FP64, 64, 16 * 8),
    (pkg.ERK, 3, 0.85, 8, 4, 1, pkg.MIXED, 256, 8 ** 3 * 2),   # adaptive inner cycles, odd nu
    (pkg.ERK, 3, 0.85, 4, 3, 2, pkg.MIXED, 64, 16 * 6),        # adaptive, even nu
    (pkg.SDIRK, 5, 4.0, 16, 3, 1, pkg.MIXED, 256, 16 * 16 * 2),
])
def test_graph_solve_equals_eager_solve(kind, p, c, m, levels, nu, prec, nx, nt):
    u0 = ic_sin4(nx)
    res = []
    for graph in (False, True):
        prm = pkg.make_params(nx, nt, c, p, kind=kind, m=m, levels=levels, nu=nu, tol=1e-10, max_iter=40,
                              precision=prec, seed=4)
        s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        if graph:
            for _ in range(2):  # the second launch replays the built graph
                s.solve_async(dev(u0))
                st = s.wait(out)
        else:
            st = s.solve(dev(u0), out)
        res.append((host(out), st))
        s.close()
    (a, sa), (b, sb) = res
    assert sa["iterations"] == sb["iterations"] and sb["converged"]
    assert sa["inner_cycles"] == sb["inner_cycles"]
    assert np.array_equal(a, b)
    assert np.allclose(sa["history"], sb["history"], rtol=0, atol=0)


# ---------------------------------------------------------------------------
# all time points (final F-relaxation, Sec. 2.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,p,q,c,m,levels,nx,nt", [
    (pkg.ERK, 3, 3, 0.85, 8, 3, 256, 8 * 8 * 4),
    (pkg.ERK, 1, 1, 0.85, 4, 2, 128, 256),
    (pkg.SDIRK, 5, 3, 4.0, 16, 3, 512, 16 * 16 * 2),
])
def test_output_all_time_points(kind, p, q, c, m, levels, nx, nt):
    """mgrit_output_all after a solve: rows k m are the returned C-points,
    the rows between are the F-relaxation from them (the oracle's f_relax on
    those C-points), and the whole trajectory matches sequential stepping to
    the solve's accuracy."""
    u0 = ic_sin4(nx)
    s = solver(nx, nt, c, p, m, levels, kind=kind, q=q, tol=1e-11, max_iter=40)
    cpts = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    s.solve(dev(u0), cpts)
    allp = torch.empty((nt + 1, nx), dtype=torch.float64, device="cuda")
    s.output_all(allp)
    got, C = host(allp), host(cpts)
    assert np.array_equal(got[::m], C)
    kname = "erk" if kind == pkg.ERK else "sdirk"
    fine = oops.FineOperator(p, kname, q, c)
    want = np.zeros((nt + 1, nx))
    want[::m] = C
    omg.f_relax(fine, want, np.zeros_like(want), m)
    assert np.max(np.abs(got - want)) < 1e-12 * max(1.0, np.max(np.abs(C)))
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(fine, g)
    assert np.max(np.abs(got - seq)) < 1e-10 * np.max(np.abs(seq))
    s.close()


def test_bounded_wait_times_out_then_completes():
    """mgrit_solve_wait_for: a zero timeout right after launching a solve of
    tens of milliseconds reports MGRIT_ERR_TIMEOUT and leaves the solve in
    flight; a generous one then returns its result unchanged."""
    nx, nt = 4096, 8192
    s = solver(nx, nt, 0.85, 3, 8, 4, tol=1e-10, max_iter=30)
    u0 = dev(ic_sin4_noise(nx, seed=0))
    out = torch.empty((nt // 8 + 1, nx), dtype=torch.float64, device="cuda")
    s.solve_async(u0)
    assert s.wait(out, timeout=0.0) is None
    st = s.wait(out, timeout=60.0)
    assert st is not None and st["converged"]
    ref = torch.empty_like(out)
    st2 = s.solve(u0, ref)
    assert st2["iterations"] == st["iterations"] and torch.equal(out, ref)
    s.close()
