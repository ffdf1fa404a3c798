"""Edge cases of the CUDA path against the oracle: the full-size C3
configuration (every C-point against the Fourier closed form
u_n = F^{-1}[lambda(omega)^n F u_0], whose symbol the oracle pins against the
operator's application), the longest vectors the kernels take, and the
degenerate hierarchies the method has (one CF-interval, a one-step coarsest
level, F-relaxation, nu = 2)."""
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


def _closed_form(op, u0, ns):
    """Rows u_n, n in ns, of sequential stepping by the Fourier symbol."""
    nx = u0.shape[0]
    lam = op.symbol(2 * np.pi * np.fft.fftfreq(nx))
    f0 = np.fft.fft(u0)
    return {n: np.real(np.fft.ifft(lam ** n * f0)) for n in ns}


def _solve(prm, u0):
    s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
    out = torch.empty((prm.nt // prm.m + 1, prm.nx), dtype=torch.float64, device="cuda")
    st = s.solve(torch.tensor(u0, dtype=torch.float64, device="cuda"), out, allow_unconverged=True)
    torch.cuda.synchronize()
    s.close()
    return out, st


def _closed_form_rows(op, u0, m, rows):
    """C-point rows u_{k m}, k = 0..rows-1, of sequential stepping by the
    Fourier symbol (one inverse FFT per row)."""
    nx = u0.shape[0]
    lam_m = op.symbol(2 * np.pi * np.fft.fftfreq(nx)) ** m
    f = np.fft.fft(u0)
    out = np.empty((rows, nx))
    for k in range(rows):
        out[k] = np.real(np.fft.ifft(f))
        f = f * lam_m
    return out


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.MIXED, pkg.MIXED_FAST])
def test_full_size_c3_all_cpoints(precision):
    """16384 x 65536, U5 + SDIRK3 at c = 4, m = 16, 5 levels (the bench
    configuration), FP64, MIXED and MIXED_FAST (FP32 correction solves on
    levels with condition numbers up to 4.5e5): all 4097 C-point rows within 1e-10
    relative of sequential stepping by the closed form.  A 1e-10 relative
    residual leaves an error of ~1.7e-10 here (the error is bounded only by
    ||A^{-1}|| ||r||), so the solves stop at 1e-11."""
    nx, nt, m = 16384, 65536, 16
    u0 = ic_fourier(nx, seed=0)
    prm = pkg.make_params(nx, nt, 4.0, 5, kind=pkg.SDIRK, q=3, m=m, levels=5, tol=1e-11, max_iter=40,
                          precision=precision, seed=0)
    out, st = _solve(prm, u0)
    assert st["converged"]
    want = _closed_form_rows(oops.FineOperator(5, "sdirk", 3, 4.0), u0, m, nt // m + 1)
    got = out.cpu().numpy()
    err = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    print("C3 precision %d: %d iterations, max relative error over all C-points %.3e"
          % (precision, st["iterations"], err))
    assert err < 1e-10, err


@pytest.mark.parametrize("kind,p,q,c,nx,m,levels", [
    (pkg.ERK, 3, 3, 0.85, 131072, 4, 3),     # the longest vector the kernels take (16 CTAs x 256 x 32)
    (pkg.SDIRK, 5, 5, 6.0, 65536, 4, 3),     # the longest SDIRK5 vector of the serving mix
])
def test_longest_vectors(kind, p, q, c, nx, m, levels):
    nt = m ** (levels - 1) * 2
    u0 = ic_fourier(nx, seed=3)
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, levels=levels, tol=1e-11, max_iter=30, seed=1)
    out, st = _solve(prm, u0)
    assert st["converged"]
    kname = "erk" if kind == pkg.ERK else "sdirk"
    ks = list(range(nt // m + 1))
    want = _closed_form(oops.FineOperator(p, kname, q, c), u0, [k * m for k in ks])
    got = out.cpu().numpy()
    scale = np.max(np.abs(u0))
    assert max(np.max(np.abs(got[k] - want[k * m])) for k in ks) < 1e-10 * scale


@pytest.mark.parametrize("kind,p,q,c,nx,nt,m,levels,nu", [
    (pkg.ERK, 3, 3, 0.85, 96, 4, 4, 2, 1),       # one CF-interval, a one-step coarsest level
    (pkg.ERK, 1, 1, 0.85, 64, 8, 4, 2, 0),       # two intervals, F-relaxation
    (pkg.ERK, 3, 3, 0.85, 128, 16, 4, 3, 1),     # coarsest level of one step
    (pkg.ERK, 5, 5, 0.9, 128, 32, 2, 5, 2),      # m = 2, five levels, nu = 2
    (pkg.SDIRK, 3, 3, 5.0, 64, 16, 16, 2, 1),    # one interval of sixteen SDIRK steps
    (pkg.SDIRK, 1, 1, 1.0, 64, 64, 4, 4, 0),     # one-step coarsest level, F-relaxation
])
def test_degenerate_hierarchies(kind, p, q, c, nx, nt, m, levels, nu):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    u0 = ic_sin4_noise(nx, seed=2)
    for prec in (pkg.FP64, pkg.MIXED):
        prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, levels=levels, nu=nu, tol=1e-11,
                              max_iter=40, seed=4, precision=prec)
        out, st = _solve(prm, u0)
        g = np.zeros((nt + 1, nx))
        g[0] = u0
        seq = omg.sequential(oops.FineOperator(p, kname, q, c), g)[::m]
        assert st["converged"], (prec, st["iterations"])
        assert np.max(np.abs(out.cpu().numpy() - seq)) < 1e-10 * np.max(np.abs(seq)), prec
        if prec == pkg.FP64:
            ref = omg.solve(omg.Hierarchy(p, kname, q, c, m, levels), u0, nt, nu=nu, tol=1e-11, max_iter=40,
                            seed=4)
            assert st["iterations"] == ref["iterations"]


def test_gmres_at_the_largest_vector():
    """GMRES correction solves (P <= 8 chunks, clusters of up to 16 CTAs x
    256 threads) at n_x = 32768, the largest vector they take; Psi_1 on 3
    random vectors against the oracle's GMRES, same iteration counts."""
    nx, m, levels = 32768, 4, 3
    prm = pkg.make_params(nx, m ** (levels - 1) * 2, 1.38, 3, m=m, levels=levels, coarse_solve=pkg.GMRES)
    s = pkg.Solver(prm, stream=torch.cuda.current_stream().cuda_stream)
    x = np.random.default_rng(3).standard_normal((3, nx))
    y = torch.empty((3, nx), dtype=torch.float64, device="cuda")
    s.coarse_apply(1, torch.tensor(x, device="cuda"), y, 3)
    torch.cuda.synchronize()
    op = oops.coarse_operator(3, "erk", 3, 1.38, m, 1, levels, gmres=(1e-2, 20))
    want = op.apply(x)
    assert np.max(np.abs(y.cpu().numpy() - want)) < 1e-12 * np.max(np.abs(want))
    assert s.gmres_stats(1)[0] == sum(op.gmres_its)
    s.close()
    # one past it is refused on the host
    with pytest.raises(pkg.MgritError):
        pkg.Solver(pkg.make_params(65536, 32, 1.38, 3, m=4, levels=3, coarse_solve=pkg.GMRES))


@pytest.mark.parametrize("kind,p,c,nx,m,levels", [
    (pkg.ERK, 4, 0.3, 131072, 4, 3),    # the longest vector, dispersive U4
    (pkg.SDIRK, 2, 1.0, 65536, 4, 3),
])
def test_even_p_longest_vectors(kind, p, c, nx, m, levels):
    nt = m ** (levels - 1) * 2
    u0 = ic_fourier(nx, seed=8)
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=p, m=m, levels=levels, tol=1e-11, max_iter=40, seed=2)
    out, st = _solve(prm, u0)
    assert st["converged"]
    kname = "erk" if kind == pkg.ERK else "sdirk"
    ks = list(range(nt // m + 1))
    want = _closed_form(oops.FineOperator(p, kname, p, c), u0, [k * m for k in ks])
    got = out.cpu().numpy()
    assert max(np.max(np.abs(got[k] - want[k * m])) for k in ks) < 1e-10 * np.max(np.abs(u0))


@pytest.mark.parametrize("kind,p,c,nx,nt,m,levels,nu", [
    (pkg.ERK, 2, 0.3, 64, 4, 4, 2, 1),        # one CF-interval
    (pkg.ERK, 4, 0.25, 64, 16, 4, 3, 0),      # one-step coarsest level, F-relaxation
    (pkg.SDIRK, 4, 1.0, 64, 8, 2, 3, 1),
])
def test_even_p_degenerate_hierarchies(kind, p, c, nx, nt, m, levels, nu):
    kname = "erk" if kind == pkg.ERK else "sdirk"
    u0 = ic_sin4_noise(nx, seed=6)
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=p, m=m, levels=levels, nu=nu, tol=1e-10, max_iter=60, seed=4)
    out, st = _solve(prm, u0)
    ref = omg.solve(omg.Hierarchy(p, kname, p, c, m, levels), u0, nt, nu=nu, tol=1e-10, max_iter=60, seed=4)
    assert st["converged"] and st["iterations"] == ref["iterations"]
    assert np.max(np.abs(out.cpu().numpy() - ref["u"][::m])) < 1e-10 * np.max(np.abs(u0))


@pytest.mark.parametrize("kind,p,q,c,nx,nt,m,levels,precision", [
    (pkg.ERK, 3, 3, 1.38, 4096, 16384, 8, 4, pkg.FP64),
    (pkg.SDIRK, 5, 3, 4.0, 16384, 65536, 16, 5, pkg.MIXED),
])
def test_full_size_mass_conservation(kind, p, q, c, nx, nt, m, levels, precision):
    """Every step and coarse operator here preserves sum_i u_i (upwind
    stencil, SL weights and correction rows sum to the identity's), so every
    C-point row of the converged full-size solution carries the initial mass
    to rounding and to the stop tolerance."""
    u0 = ic_fourier(nx, seed=4) + 0.5
    prm = pkg.make_params(nx, nt, c, p, kind=kind, q=q, m=m, levels=levels, tol=1e-11, max_iter=40,
                          seed=0, precision=precision)
    out, st = _solve(prm, u0)
    assert st["converged"]
    mass = out.sum(dim=1).cpu().numpy()
    assert np.max(np.abs(mass - u0.sum())) < 1e-10 * np.abs(u0).sum()
