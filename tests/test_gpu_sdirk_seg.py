"""GPU parity of the segmented FP64 level-0 SDIRK kernel (one CTA per
CF-interval, 128 points per thread, the stage solves' recurrences entered
through a warm-up over the neighbouring segment) against the CPU oracle, and
against the chunked kernel it replaces.  MGRIT_SDIRK_SEG=1 forces it where it
applies (level_info(0)[4] == 2 shows that it runs), =0 keeps the chunked
kernel.  Tolerances as in test_gpu_sdirk.py: one step to 1e-12 relative,
solves iteration for iteration with the oracle, converged solutions within
1e-10 of sequential stepping."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2209_06916_gb300 as pkg
from oracle import mgrit as omg
from oracle import operators as oops
from workloads import ic_fourier

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


def solver(nx, nt, c, p, q, m, levels, nu=1, tol=1e-11, max_iter=40, seed=0, precision=pkg.FP64):
    prm = pkg.make_params(nx, nt, c, p, kind=pkg.SDIRK, q=q, m=m, levels=levels, nu=nu, tol=tol,
                          max_iter=max_iter, seed=seed, precision=precision)
    return pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)


@pytest.fixture
def seg(monkeypatch):
    def set_policy(v):
        monkeypatch.setenv("MGRIT_SDIRK_SEG", str(v))
    return set_policy


# (p, q, c, nx): every recurrence order of the kernel (U1, U3, U5), one and
# three stages, 32 / 64 / 128 threads per interval
STEPS = [(1, 1, 1.0, 4096), (3, 1, 2.0, 4096), (3, 3, 5.0, 8192), (5, 1, 3.0, 4096), (5, 3, 4.0, 16384),
         (3, 3, 1.0, 16384)]


@pytest.mark.parametrize("p,q,c,nx", STEPS)
def test_seg_step_matches_oracle(seg, p, q, c, nx):
    seg(1)
    s = solver(nx, 64, c, p, q, 4, 2)
    assert s.level_info(0)[4] == 2.0, "the segmented kernel does not run"
    x = np.random.default_rng(8).standard_normal((5, nx))
    y = torch.empty((5, nx), dtype=torch.float64, device="cuda")
    s.coarse_apply(0, dev(x), y, 5)
    want = oops.FineOperator(p, "sdirk", q, c).apply(x)
    assert _rel(host(y), want) < 1e-12
    s.close()


def test_seg_step_unaligned_rows(seg):
    """Caller rows that start 8 bytes past a 16-byte boundary (views one
    element into a buffer): the segmented kernel keeps a stage vector in the
    output rows in 16-byte pairs, so the host sends such rows to the chunked
    kernel instead, with the same result."""
    seg(1)
    p, q, c, nx, nv = 5, 3, 4.0, 4096, 5
    s = solver(nx, 64, c, p, q, 4, 2)
    assert s.level_info(0)[4] == 2.0
    x = np.random.default_rng(9).standard_normal((nv, nx))
    xb = torch.zeros(nv * nx + 1, dtype=torch.float64, device="cuda")
    xb[1:] = dev(x).reshape(-1)
    yb = torch.full((nv * nx + 1,), np.nan, dtype=torch.float64, device="cuda")
    xv, yv = xb[1:], yb[1:]
    assert xv.data_ptr() % 16 == 8 and yv.data_ptr() % 16 == 8
    s.coarse_apply(0, xv, yv, nv)
    want = oops.FineOperator(p, "sdirk", q, c).apply(x)
    assert _rel(host(yv).reshape(nv, nx), want) < 1e-12
    s.close()


@pytest.mark.parametrize("p,q,c,nx", [(5, 3, 8.0, 4096), (1, 1, 4.0, 4096), (5, 3, 4.0, 1024), (5, 5, 4.0, 4096),
                                      (5, 3, 4.0, 32768)])
def test_seg_not_used_where_it_does_not_fit(seg, p, q, c, nx):
    """Warm-up longer than a segment (slow decay at large c), fewer than 32
    or more than 128 segments, five stages: the chunked kernel runs."""
    seg(1)
    s = solver(nx, 64, c, p, q, 4, 2)
    assert s.level_info(0)[4] != 2.0
    s.close()


@pytest.mark.parametrize("p,q,c,m,levels,nx,nt,precision", [
    (5, 3, 4.0, 16, 3, 4096, 16 * 16 * 2, pkg.FP64),   # the 16384 x 65536 scheme at a smaller size
    (3, 3, 5.0, 4, 3, 4096, 4 * 4 * 8, pkg.FP64),      # Table-3 scheme
    (1, 1, 1.0, 4, 3, 4096, 4 * 4 * 4, pkg.FP64),
    (5, 3, 4.0, 16, 3, 4096, 16 * 16 * 2, pkg.MIXED),  # FP64 residuals in refinement
])
def test_seg_solve_matches_oracle(seg, p, q, c, m, levels, nx, nt, precision):
    seg(1)
    u0 = ic_fourier(nx, seed=1)
    s = solver(nx, nt, c, p, q, m, levels, seed=5, precision=precision)
    assert s.level_info(0)[4] == 2.0
    out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
    st = s.solve(dev(u0), out)
    h = omg.Hierarchy(p, "sdirk", q, c, m, levels)
    got = host(out)
    if precision == pkg.FP64:
        ref = omg.solve(h, u0, nt, nu=1, tol=1e-11, max_iter=40, seed=5)
        assert st["iterations"] == ref["iterations"]
        hist, href = np.array(st["history"]), np.array(ref["history"])
        big = href > 1e-8 * href[0]
        assert np.max(np.abs(hist[big] - href[big]) / href[big]) < 1e-6
        assert np.max(np.abs(got - ref["u"][::m])) < 1e-10 * np.max(np.abs(u0))
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(h.fine, g)[::m]
    assert _rel(got, seq) < 1e-10, _rel(got, seq)
    s.close()


def test_seg_equals_chunked_kernel(seg):
    """The same C-relaxation by both kernels (several steps, 64 intervals):
    equal to rounding."""
    nx, m, K = 16384, 16, 64
    res = []
    for pol in (1, 0):
        seg(pol)
        s = solver(nx, m * K, 4.0, 5, 3, m, 2)
        assert (s.level_info(0)[4] == 2.0) == (pol == 1)
        x = np.random.default_rng(3).standard_normal((K + 1, nx))
        s.level_set(0, 0, x)
        s.relax(0, 1)
        res.append(s.level_get(0, 0))
        s.close()
    assert _rel(res[0], res[1]) < 1e-12


def test_seg_full_size_solve(seg):
    """16384 x 65536, U5 + SDIRK3 at c = 4, m = 16, 5 levels, FP64 with the
    segmented kernel: every C-point within 1e-10 of sequential stepping (the
    Fourier closed form), with the chunked kernel's iteration count."""
    nx, nt, m = 16384, 65536, 16
    u0 = ic_fourier(nx, seed=0)
    its = {}
    for pol in (1, 0):
        seg(pol)
        s = solver(nx, nt, 4.0, 5, 3, m, 5, seed=0)
        assert (s.level_info(0)[4] == 2.0) == (pol == 1)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(dev(u0), out)
        its[pol] = st["iterations"]
        if pol == 1:
            lam_m = oops.FineOperator(5, "sdirk", 3, 4.0).symbol(2 * np.pi * np.fft.fftfreq(nx)) ** m
            f = np.fft.fft(u0)
            got = host(out)
            want = np.empty_like(got)
            for k in range(nt // m + 1):
                want[k] = np.real(np.fft.ifft(f))
                f = f * lam_m
            err = _rel(got, want)
            print("segmented kernel, C3 FP64: %d iterations, error %.3e" % (st["iterations"], err))
            assert err < 1e-10
        s.close()
    assert its[0] == its[1]


@pytest.mark.parametrize("p,q,c,nx,m,levels,nt", [
    (5, 3, 4.0, 16384, 16, 3, 16 * 16 * 2),   # 256 segments of 64 points
    (3, 3, 5.0, 4096, 4, 3, 4 * 4 * 8),       # 64 segments
    (1, 1, 1.0, 2048, 4, 3, 4 * 4 * 4),       # 32 segments, one stage
    (5, 1, 3.0, 8192, 8, 3, 8 * 8 * 2),
])
def test_seg32_mixed_solve(seg, p, q, c, nx, m, levels, nt):
    """MIXED inner cycles with the FP32 segmented stage kernel: the refined
    solution within 1e-10 of sequential stepping, in as many refinement
    steps (+-1) as with the chunked FP32 kernel."""
    u0 = ic_fourier(nx, seed=4)
    g = np.zeros((nt + 1, nx))
    g[0] = u0
    seq = omg.sequential(oops.FineOperator(p, "sdirk", q, c), g)[::m]
    outer = {}
    for pol in (1, 0):
        seg(pol)
        s = solver(nx, nt, c, p, q, m, levels, seed=2, precision=pkg.MIXED)
        assert (s.level_info(0)[5] == 1.0) == (pol == 1)
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(dev(u0), out)
        assert st["converged"]
        err = _rel(host(out), seq)
        print("FP32 segmented %d: %d refinement steps, error %.3e" % (pol, st["outer_iterations"], err))
        assert err < 1e-10, err
        outer[pol] = st["outer_iterations"]
        s.close()
    assert abs(outer[1] - outer[0]) <= 1


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.MIXED])
def test_seg_solve_is_deterministic(seg, precision):
    """The same solve in two handles through the segmented kernels: bitwise
    equal C-points and residual histories (fixed-order sums, no atomics on
    the data path)."""
    seg(1)
    p, q, c, m, levels, nx, nt = 5, 3, 4.0, 16, 3, 4096, 16 * 16 * 2
    u0 = ic_fourier(nx, seed=6)
    runs = []
    for _ in range(2):
        s = solver(nx, nt, c, p, q, m, levels, seed=4, precision=precision)
        assert s.level_info(0)[4] == 2.0
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        st = s.solve(dev(u0), out)
        runs.append((host(out), st["history"]))
        s.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]
