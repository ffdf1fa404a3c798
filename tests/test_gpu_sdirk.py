"""GPU parity of the SDIRK path (stage solves with (I + gamma c L_p) inside
the level-0 kernels) against the CPU oracle.  Tolerances as in
test_gpu_parity.py: one step agrees to ~1e-12 relative (every stage is a
banded solve plus a mat-vec, both well conditioned for these c), solves agree
iteration for iteration."""
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def solver(nx, nt, c, p, q, m, levels, nu=1, tol=1e-10, max_iter=40, seed=0):
    prm = pkg.make_params(nx, nt, c, p, kind=pkg.SDIRK, q=q, m=m, levels=levels, nu=nu, tol=tol,
                          max_iter=max_iter, seed=seed)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("p,q,c,nx", [(1, 1, 1.0, 64), (5, 1, 3.0, 96), (3, 3, 5.0, 256), (3, 1, 2.0, 128),
                                      (5, 5, 6.0, 512), (5, 3, 4.0, 1024), (3, 3, 5.0, 4096),
                                      (5, 3, 4.0, 16384)])
def test_sdirk_step_matches_oracle(p, q, c, nx):
    s = solver(nx, 64, c, p, q, 4, 2)
    x = np.random.default_rng(8).standard_normal((5, nx))
    y = torch.empty((5, nx), dtype=torch.float64, device="cuda")
    s.coarse_apply(0, dev(x), y, 5)
    want = oops.FineOperator(p, "sdirk", q, c).apply(x)
    assert _rel(host(y), want) < 1e-12


@pytest.mark.parametrize("p,q,c,m,levels,nx", [(3, 3, 5.0, 4, 3, 256), (5, 3, 4.0, 16, 3, 512),
                                               (1, 1, 1.0, 4, 4, 128)])
def test_sdirk_coarse_operators_match_oracle(p, q, c, m, levels, nx):
    s = solver(nx, m ** (levels - 1) * 2, c, p, q, m, levels)
    x = np.random.default_rng(9).standard_normal((7, nx))
    for lev in range(1, levels):
        y = torch.empty((7, nx), dtype=torch.float64, device="cuda")
        s.coarse_apply(lev, dev(x), y, 7)
        op = oops.coarse_operator(p, "sdirk", q, c, m, lev, levels)
        # rounding in the correction solve grows with the condition number of
        # I - sum phi D (its symbol ranges over [min, max] on the unit circle)
        w = 2 * np.pi * np.arange(nx) / nx
        sym = np.abs(1.0 + sum(a * np.exp(1j * j * w) for j, a in op.corr.items()))
        kappa = sym.max() / sym.min()
        assert _rel(host(y), op.apply(x)) < max(1e-12, 50 * kappa * 2.0 ** -52), (lev, kappa)


@pytest.mark.parametrize("p,q,c,m,levels,nu,nx,nt", [
    (3, 3, 5.0, 4, 2, 1, 64, 256),      # Table 3 shape (SDIRK3+U3, c = 5)
    (1, 1, 1.0, 4, 3, 1, 64, 16 * 8),   # SDIRK1+U1
    (5, 3, 4.0, 16, 3, 1, 128, 16 * 16 * 2),  # U5 + SDIRK3 (q != p correction)
    (3, 3, 5.0, 4, 3, 0, 64, 16 * 4),   # F-relaxation
])
def test_sdirk_solve_matches_oracle_mgrit(p, q, c, m, levels, nu, nx, nt):
    u0 = ic_sin4(nx) if p < 5 else ic_fourier(nx, seed=1)
    s = solver(nx, nt, c, p, q, m, levels, nu=nu, seed=5, tol=1e-11)
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out, allow_unconverged=True)
    h = omg.Hierarchy(p, "sdirk", q, c, m, st["levels"])
    ref = omg.solve(h, u0, nt, nu=nu, tol=1e-11, max_iter=40, seed=5)
    assert st["iterations"] == ref["iterations"]
    hist, href = np.array(st["history"]), np.array(ref["history"])
    big = href > 1e-8 * href[0]
    assert np.max(np.abs(hist[big] - href[big]) / href[big]) < 1e-6
    got = host(out)
    assert np.max(np.abs(got - ref["u"][::m])) < 1e-10 * max(1.0, np.max(np.abs(u0)))
    # converged solution against the oracle's sequential stepping, every C-point
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(h.fine, g)[::m]
    assert _rel(got, seq) < 1e-10, _rel(got, seq)


@pytest.mark.parametrize("p,q,c,nx,nsteps,every", [(3, 3, 5.0, 256, 100, 10), (5, 3, 4.0, 4096, 40, 0),
                                                    (1, 1, 1.0, 64, 33, 11)])
def test_sdirk_sequential_stepping(p, q, c, nx, nsteps, every):
    s = solver(nx, 64, c, p, q, 4, 2)
    u0 = ic_fourier(nx, seed=2)
    out = torch.empty(nx, dtype=torch.float64, device="cuda")
    traj = torch.zeros((max(1, nsteps // max(1, every)), nx), dtype=torch.float64, device="cuda")
    s.fine_propagate(dev(u0), out, nsteps, every, traj if every else None)
    fine = oops.FineOperator(p, "sdirk", q, c)
    u = u0.copy()
    rows = []
    for n in range(1, nsteps + 1):
        u = fine.apply(u)
        if every and n % every == 0:
            rows.append(u.copy())
    assert _rel(host(out), u) < 1e-13 * nsteps
    if every:
        assert _rel(host(traj), np.array(rows)) < 1e-13 * nsteps
