"""MIXED precision (FP32 inner cycles inside FP64 iterative refinement): the
converged solution must match the FP64 oracle's sequential time-stepping as
closely as the FP64 solver does (the outer residual is FP64, so the FP32
sweeps limit only the rate, not the accuracy)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import mgrit as omg
from oracle import operators as oops
from workloads import ic_fourier, ic_sin4, ic_sin4_noise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _seq(p, kind, q, c, u0, nt, m):
    g = np.zeros((nt + 1, u0.shape[0]))
    g[0] = u0
    return omg.sequential(oops.FineOperator(p, kind, q, c), g)[::m]


CASES = [  # kind, p, q, c, m, levels, nx, nt, inner
    ("erk", 3, 3, 0.85, 8, 4, 512, 8 ** 3 * 2, 2),
    ("erk", 1, 1, 0.85, 4, 2, 256, 1024, 1),
    ("erk", 5, 5, 0.9, 4, 3, 256, 16 * 6, 3),
    ("sdirk", 5, 3, 4.0, 16, 3, 512, 16 * 16 * 2, 2),
    ("sdirk", 3, 3, 5.0, 4, 3, 256, 16 * 8, 2),
    ("erk", 3, 3, 0.85, 8, 4, 512, 8 ** 3 * 2, 0),      # adaptive inner cycles
    ("erk", 3, 3, 0.85, 8, 4, 2048, 8 ** 3 * 8, 0),     # long enough for FP32 noise to show in the error
    ("sdirk", 5, 3, 4.0, 16, 3, 512, 16 * 16 * 2, 0),
    ("sdirk", 5, 5, 6.0, 4, 4, 256, 4 ** 3 * 4, 0),
]


@pytest.mark.parametrize("kind,p,q,c,m,levels,nx,nt,inner", CASES)
def test_mixed_solve_reaches_fp64_accuracy(kind, p, q, c, m, levels, nx, nt, inner):
    u0 = ic_sin4_noise(nx, seed=1) if p < 5 else ic_fourier(nx, seed=1)
    k = pkg.ERK if kind == "erk" else pkg.SDIRK
    stream = torch.cuda.current_stream().cuda_stream
    res = {}
    for prec in (pkg.FP64, pkg.MIXED, pkg.MIXED_FAST):
        prm = pkg.make_params(nx, nt, c, p, kind=k, q=q, m=m, levels=levels, tol=1e-11, max_iter=40,
                              precision=prec, seed=3, inner_cycles=inner)
        s = pkg.Solver(prm, stream=stream)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(u0, device="cuda"), out)
        torch.cuda.synchronize()
        res[prec] = (out.cpu().numpy(), st)
        s.close()
    seq = _seq(p, kind, q, c, u0, nt, m)
    scale = np.max(np.abs(seq))
    e64 = np.max(np.abs(res[pkg.FP64][0] - seq)) / scale
    assert e64 < 1e-10, e64
    for prec in (pkg.MIXED, pkg.MIXED_FAST):
        emx = np.max(np.abs(res[prec][0] - seq)) / scale
        st = res[prec][1]
        assert st["converged"] and st["inner_cycles"] >= st["outer_iterations"] * inner
        # FP32 relaxation inside FP64 refinement reaches the FP64 bound at
        # the same stop tolerance: every C-point within 1e-10 relative
        print("%s: FP64 error %.2e, mixed error %.2e" % (prec, e64, emx))
        assert emx < 1e-10, (prec, e64, emx)


@pytest.mark.parametrize("kind,p,q,c,m,levels,nx,nt", [("erk", 3, 3, 0.85, 8, 4, 512, 8 ** 3 * 2),
                                                      ("sdirk", 5, 3, 4.0, 16, 3, 512, 16 * 16 * 2)])
def test_adaptive_inner_cycles_cut_fp64_residuals(kind, p, q, c, m, levels, nx, nt):
    """Adaptive inner solves (inner_cycles = 0) need fewer FP64 residual
    evaluations than one FP32 cycle per residual, for no more V-cycles than
    a fixed count would spend, at the same accuracy."""
    u0 = ic_sin4_noise(nx, seed=2) if p < 5 else ic_fourier(nx, seed=2)
    k = pkg.ERK if kind == "erk" else pkg.SDIRK
    stream = torch.cuda.current_stream().cuda_stream
    st = {}
    for inner in (1, 0):
        prm = pkg.make_params(nx, nt, c, p, kind=k, q=q, m=m, levels=levels, tol=1e-10, max_iter=40,
                              precision=pkg.MIXED, seed=3, inner_cycles=inner)
        s = pkg.Solver(prm, stream=stream)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st[inner] = s.solve(torch.tensor(u0, device="cuda"), out)
        s.close()
    assert st[0]["converged"] and st[1]["converged"]
    assert st[0]["outer_iterations"] * 2 <= st[1]["outer_iterations"], (st[0], st[1])
    assert st[0]["inner_cycles"] <= st[1]["inner_cycles"] + 16
