"""Pins of the oracle's GMRES correction solves (Sec. 6.1, Sec. 6.3) against
the definition of the GMRES iterate and against the paper (no GPU)."""
import numpy as np
import pytest

from oracle import coefficients as co
from oracle import gmres as gm
from oracle import mgrit
from oracle import operators as ops
from workloads import ic_sin4


def _random_system(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) + 0.4 * rng.standard_normal((n, n)) / np.sqrt(n)
    return A, rng.standard_normal(n)


def _krylov_minimiser(A, b, k):
    """argmin ||b - A x|| over span{b, A b, .., A^{k-1} b}, from an explicit
    Krylov matrix orthonormalised by QR (no Arnoldi)."""
    K = np.empty((b.shape[0], k))
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = A @ v
    Q, _ = np.linalg.qr(K)
    y, _, _, _ = np.linalg.lstsq(A @ Q, b, rcond=None)
    return Q @ y


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_iterate_is_the_krylov_minimiser(k):
    A, b = _random_system(40, k)
    x, kk, _ = gm.gmres(lambda v: A @ v, b, rtol=0.0, maxit=k)
    assert kk == k
    xd = _krylov_minimiser(A, b, k)
    assert np.max(np.abs(x - xd)) < 1e-10 * np.max(np.abs(xd))


@pytest.mark.parametrize("k", [1, 3, 5])
def test_iterate_is_the_krylov_minimiser_for_the_correction_matrix(k):
    """The same on the correction matrix I - phi D of a level-2 operator."""
    op = ops.coarse_operator(3, "erk", 3, 1.38, 4, 2, 3)
    n = 48
    A = np.eye(n) + ops.dense_circulant(op.corr, n)
    b = op.sl.apply(np.sin(np.pi * np.linspace(-1, 1, n, endpoint=False)) ** 4)
    x, kk, _ = gm.gmres(lambda v: A @ v, b, rtol=0.0, maxit=k)
    xd = _krylov_minimiser(A, b, k)
    assert kk == k
    assert np.max(np.abs(x - xd)) < 1e-10 * np.max(np.abs(xd))


def test_exact_on_the_full_space():
    A, b = _random_system(8, 11)
    x, k, res = gm.gmres(lambda v: A @ v, b, rtol=1e-14, maxit=8)
    assert k <= 8
    assert np.max(np.abs(x - np.linalg.solve(A, b))) < 1e-12
    # the circulant correction solve of a coarse operator: GMRES run to
    # convergence equals the direct circulant solve
    op = ops.coarse_operator(5, "erk", 5, 1.0, 4, 1, 2)
    n = 16
    b = np.cos(np.arange(n) * 0.7) + 0.3
    x, k, _ = gm.gmres(op.correction_matvec, b, rtol=1e-15, maxit=n)
    assert np.max(np.abs(x - ops.circulant_solve(op.corr, b, diag=1.0))) < 1e-11


def test_residual_estimates_and_stop_rule():
    A, b = _random_system(60, 5)
    rtol = 1e-2
    x, k, res = gm.gmres(lambda v: A @ v, b, rtol=rtol, maxit=30)
    nb = np.linalg.norm(b)
    assert 1 < k < 30
    assert abs(res[-1] - np.linalg.norm(b - A @ x)) < 1e-12 * nb
    assert res[-1] <= rtol * nb
    # the first k that meets the rule: k - 1 iterations do not
    xp, kp, _ = gm.gmres(lambda v: A @ v, b, rtol=0.0, maxit=k - 1)
    assert np.linalg.norm(b - A @ xp) > rtol * nb
    # residuals never increase (minimisation over nested spaces)
    assert all(res[i + 1] <= res[i] * (1 + 1e-14) for i in range(len(res) - 1))
    # the cap: maxit iterations at most
    _, kc, _ = gm.gmres(lambda v: A @ v, b, rtol=1e-12, maxit=3)
    assert kc == 3


def test_zero_rhs():
    x, k, res = gm.gmres(lambda v: 2 * v, np.zeros(5))
    assert k == 0 and not x.any()


def test_default_caps():
    """Sec. 6.3: 10 iterations for ERK1+U1, 20 for third and fifth order."""
    assert gm.default_maxit(1) == 10 and gm.default_maxit(3) == 20 and gm.default_maxit(5) == 20


def _levels_until_two(nt, m):
    L, N = 1, nt
    while N // m >= 2:
        N //= m
        L += 1
    return L


def test_mgrit_with_gmres_keeps_the_direct_iteration_counts(golden):
    """Sec. 6.3: the GMRES halting rule (1e-2, at most 20) leaves MGRIT's
    convergence as with direct solves; the V-cycle counts stay within 2 of
    Table 3 (the paper's multilevel ERK runs used GMRES on every level, its
    SDIRK runs direct solves)."""
    cmax = co.cfl_limit(3)
    for kind, nx, nt, m, two, vc in golden("table3_iterations.txt"):
        nx, nt, m, vc = int(nx), int(nt), int(m), int(vc)
        if nx != 64 or (kind == "sdirk" and m < 8):
            continue
        c = 0.85 * cmax if kind == "erk" else 5.0
        L = _levels_until_two(nt, m)
        u0 = ic_sin4(nx)
        hg = mgrit.Hierarchy(3, kind, 3, c, m, L, gmres=(1e-2, gm.default_maxit(3)))
        rg = mgrit.solve(hg, u0, nt, tol=1e-10, max_iter=40)
        rd = mgrit.solve(mgrit.Hierarchy(3, kind, 3, c, m, L), u0, nt, tol=1e-10, max_iter=40)
        assert rg["converged"]
        assert abs(rg["iterations"] - rd["iterations"]) <= 1, (kind, m, rg["iterations"], rd["iterations"])
        assert abs(rg["iterations"] - vc) <= 2, (kind, m, rg["iterations"], vc)
        # GMRES did work on the first coarse level and stopped inside its cap
        its = hg.ops[1].gmres_its
        assert max(its) <= 20 and np.mean(its) >= 1
