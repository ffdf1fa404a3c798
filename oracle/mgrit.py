"""Sequential time-stepping and linear MGRIT, written out literally (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64; every level
stores ALL of its time points (no C-point-only storage, no fusion): F- and
C-relaxation, the C-point residual, the coarse solve and the correction are
separate steps in the order of Sec. 2.2.

Function          paper passage                                          parity pin
----------------  -----------------------------------------------------  ------------------------------
sequential        Eq. (one-step-general): u_{n+1} = Phi u_n + g_{n+1}    FFT closed form; dense space-
                                                                          time solve (tiny grids)
f_relax/c_relax   Sec. 2.2: F- / C-relaxation zero the residual at F- /  -
                  C-points
c_residual        Sec. 2.2: residual at the C-points (the coarse RHS of  -
                  Eq. one-step-coarse-general, injection)
vcycle            Sec. 2.2 / Sec. 6.2: F(CF)^nu pre-relaxation, coarse  two-level F-relaxation exact
                  correction (recursive, the coarsest level by           after nt/m iterations; ideal
                  sequential stepping), F post-relaxation                 Psi = Phi^m exact in one
                                                                          iteration; Table 3 counts
solve             Sec. 5.3 / 6.3 setup: random initial iterate except    converged solution == sequential
                  at t = 0, stop when the l2 norm of the residual has     stepping; final factor near LFA
                  dropped by ``tol`` (10 orders) or after max_iter
"""
import numpy as np

from . import coefficients as co
from . import operators as ops
from . import rng


def sequential(op, g):
    """u_0 = g_0, u_n = Phi u_{n-1} + g_n for n = 1..N  (g has N+1 rows)."""
    g = np.asarray(g, dtype=np.float64)
    u = np.empty_like(g)
    u[0] = g[0]
    for n in range(1, g.shape[0]):
        u[n] = op.apply(u[n - 1]) + g[n]
    return u


def f_relax(op, u, g, m):
    """F-relaxation: u_{km+j} = Phi u_{km+j-1} + g_{km+j}, j = 1..m-1, for
    every CF-interval k at once."""
    K = (u.shape[0] - 1) // m
    base = np.arange(K) * m
    for j in range(1, m):
        idx = base + j
        u[idx] = op.apply(u[idx - 1]) + g[idx]


def c_relax(op, u, g, m):
    """C-relaxation: u_{km} = Phi u_{km-1} + g_{km}, k = 1..N/m."""
    K = (u.shape[0] - 1) // m
    idx = np.arange(1, K + 1) * m
    u[idx] = op.apply(u[idx - 1]) + g[idx]


def c_residual(op, u, g, m):
    """r_k = g_{km} + Phi u_{km-1} - u_{km} at the C-points k = 1..N/m
    (r_0 = 0: the t = 0 row is exact).  Returns N/m + 1 rows."""
    K = (u.shape[0] - 1) // m
    r = np.zeros((K + 1, u.shape[1]), dtype=np.float64)
    idx = np.arange(1, K + 1) * m
    r[1:] = g[idx] + op.apply(u[idx - 1]) - u[idx]
    return r


class Hierarchy:
    """Level operators of a uniform-m hierarchy: level 0 is the fine MOL step
    Phi, level l >= 1 the corrected SL operator Phi^{(m^l dt)} (Eq. MOL-SL-corrected-multilevel),
    or with ``coarse_op`` = "sl" / "redisc" the direct SL operator or the
    rediscretised fine method (operators.direct_operator).  ``coarse`` may
    replace the level-1 operator (e.g. the ideal Phi^m) for a two-level
    hierarchy.  ``gmres`` = (rtol, maxit) solves the correction systems of
    the corrected operators approximately by GMRES (Sec. 6.3)."""

    def __init__(self, p, kind, q, c, m, levels, coarse=None, coarse_op="sl_corrected", gmres=None):
        # ms[l]: fine steps of level l per step of level l+1 (one factor, or
        # one per coarse level)
        self.ms = co.level_factors(m, levels) if levels > 1 else []
        self.m, self.levels = (self.ms[0] if self.ms else m), levels
        self.fine = ops.FineOperator(p, kind, q, c)
        self.ops = [self.fine]
        for l in range(1, levels):
            if l == 1 and coarse is not None:
                self.ops.append(coarse)
            elif coarse_op == "sl_corrected":
                self.ops.append(ops.coarse_operator(p, kind, q, c, m, l, levels, gmres))
            else:
                self.ops.append(ops.direct_operator(p, kind, q, c, m, l, coarse_op))


def vcycle(h, level, u, g, nu):
    """One MGRIT cycle on ``level`` for u_n = Phi_l u_{n-1} + g_n (in place).

    Coarsest level: sequential stepping.  Otherwise F(CF)^nu, C-point
    residual, recursive coarse solve for the error (zero initial guess),
    correction at the C-points and a final F-relaxation.
    """
    op = h.ops[level]
    if level == h.levels - 1:
        u[:] = sequential(op, g)
        return
    m = h.ms[level]
    f_relax(op, u, g, m)
    for _ in range(nu):
        c_relax(op, u, g, m)
        f_relax(op, u, g, m)
    r = c_residual(op, u, g, m)
    e = np.zeros_like(r)
    vcycle(h, level + 1, e, r, nu)
    u[::m] += e
    f_relax(op, u, g, m)


def initial_iterate(u0, nt, seed):
    """Uniform random iterate on all time points except u_0 = u0."""
    nx = u0.shape[0]
    u = np.empty((nt + 1, nx), dtype=np.float64)
    u[0] = u0
    u[1:] = rng.uniform_grid(seed, np.arange(1, nt + 1), nx)
    return u


def solve(h, u0, nt, nu=1, tol=1e-10, max_iter=30, seed=0, u_init=None,
          keep_iterates=False):
    """Linear MGRIT (two-level if h.levels == 2, else V-cycles).

    Each iteration: level-0 pre-relaxation F(CF)^nu, residual norm
    ||r||_2 over all C-points and grid points, stop test
    ||r_it|| <= tol ||r_0||, then the coarse correction and F-relaxation.
    Returns a dict with the final iterate u (all time points, the state whose
    residual was last measured, i.e. after its pre-relaxation), the residual
    norm history, the number of iterations (coarse corrections applied before
    the stop test passed) and, optionally, the C-point iterates after each
    pre-relaxation.
    """
    u0 = np.asarray(u0, dtype=np.float64)
    m = h.m
    u = initial_iterate(u0, nt, seed) if u_init is None else np.array(u_init, dtype=np.float64)
    g = np.zeros_like(u)
    g[0] = u0
    op = h.ops[0]
    history, iterates = [], []
    it = 0
    while True:
        f_relax(op, u, g, m)
        for _ in range(nu):
            c_relax(op, u, g, m)
            f_relax(op, u, g, m)
        r = c_residual(op, u, g, m)
        history.append(float(np.sqrt(np.sum(r * r))))
        if keep_iterates:
            iterates.append(u[::m].copy())
        if history[-1] <= tol * history[0] or it >= max_iter or not np.isfinite(history[-1]):
            break
        e = np.zeros_like(r)
        vcycle(h, 1, e, r, nu)
        u[::m] += e
        f_relax(op, u, g, m)
        it += 1
    converged = bool(history[-1] <= tol * history[0])
    factor = history[-1] / history[-2] if len(history) > 1 and history[-2] > 0 else 0.0
    return {"u": u, "history": history, "iterations": it, "converged": converged,
            "factor": factor, "iterates": iterates}
