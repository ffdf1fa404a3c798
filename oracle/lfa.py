"""Two-level LFA convergence factor (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

rho(E) = max_omega |lambda(omega)|^{m nu} |lambda^m(omega) - mu(omega)|
                    / (1 - |mu(omega)|)                      (Eq. rho-asym)
with lambda, mu the Fourier symbols of Phi and Psi, omega sampled at 2^11
equispaced points of [-pi, pi); omega = 0 and the ``omit`` samples nearest to
it on each side are dropped (footnote to Eq. rho-asym).

Parity pins: Sec. 6.3.4 (FCF factors of the third-order schemes bounded by 0.6)
and Sec. 6.4 (ERK4+U4, m = 2: about 0.15 just below c/c_max = 0.24 and about
0.84 just above).  With direct coarse operators (Sec. 5): the factor with
rediscretisation is bounded below by rho_check (Theorem thm:MOL-rho-lwr-bnd,
Eq. rho-check-MOL) and equals it where smooth characteristic components set
the maximum; rho_check tends to |1 - m^-p| (Eq. rho-check-MOL-asym).
"""
import numpy as np

from . import coefficients as co
from . import operators as ops


def omega_samples(n=1 << 11, omit=0):
    w = -np.pi + 2.0 * np.pi * np.arange(n) / n
    k0 = n // 2  # index of omega = 0
    keep = np.ones(n, dtype=bool)
    keep[k0 - omit:k0 + omit + 1] = False
    return w[keep]


def rho(lam, mu, m, nu):
    """Eq. (rho-asym) evaluated on arrays of symbols; returns the max."""
    num = np.abs(lam) ** (m * nu) * np.abs(lam ** m - mu)
    den = 1.0 - np.abs(mu)
    return float(np.max(num / den))


def corrected_sl_symbol(p, kind, c, m, omega, q=None, d_order=None):
    """Symbol of (I - phi D)^{-1} S_p^{(m dt)} (two-level, Eq. MOL-SL-corrected).

    For even p the SL node set depends on eps (coefficients.sl_nodes), f_{p+1}
    is evaluated on that node set and D is the one-point-left-biased
    first-order stencil (Sec. 6.4).
    """
    q = p if q is None else q
    s = c * m
    k, eps = co.sl_shift(s)
    nodes = co.sl_nodes(p, eps)
    w = co.sl_weights(p, eps)
    f = co.f_poly(p, eps, nodes)
    phi = m * (c * float(co.e_fd(p)) + (-c) ** (p + 1) * co.e_rk(kind, q)) + (-1) ** (p + 1) * f
    d = co.diff_taps(p + 1 if d_order is None else d_order)
    S = sum(wj * np.exp(1j * (j - k) * omega) for j, wj in w.items())
    Dsym = sum(float(dj) * np.exp(1j * j * omega) for j, dj in d.items())
    return S / (1.0 - phi * Dsym)


def two_level_factor(p, kind, c, m, nu=1, omit=0, n=1 << 11, coarse_op="sl_corrected"):
    """LFA factor of two-level MGRIT with the corrected SL coarse operator,
    or with a direct one: ``sl`` (S_p^{(m dt)}) or ``redisc`` (the fine
    method with step m dt, Sec. 5)."""
    omega = omega_samples(n, omit)
    lam = ops.FineOperator(p, kind, p, c).symbol(omega)
    if coarse_op == "sl_corrected":
        mu = corrected_sl_symbol(p, kind, c, m, omega)
    else:
        mu = ops.direct_operator(p, kind, p, c, m, 1, coarse_op).symbol(omega)
    return rho(lam, mu, m, nu)


def rho_check(p, c, m, e_rk_fine, e_rk_coarse):
    """Lower bound of the two-level factor with a direct MOL coarse operator
    on asymptotically smooth characteristic components (Theorem
    thm:MOL-rho-lwr-bnd, Eq. rho-check-MOL), odd p:
        c^p |e_F - m^p e_C| / |e_FD + (m c)^p e_C|."""
    efd = float(co.e_fd(p))
    return c ** p * abs(e_rk_fine - m ** p * e_rk_coarse) / abs(efd + (m * c) ** p * e_rk_coarse)
