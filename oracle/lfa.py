"""Two-level LFA convergence factor (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

rho(E) = max_omega |lambda(omega)|^{m nu} |lambda^m(omega) - mu(omega)|
                    / (1 - |mu(omega)|)                      (Eq. rho-asym)
with lambda, mu the Fourier symbols of Phi and Psi, omega sampled at 2^11
equispaced points of [-pi, pi); omega = 0 and the ``omit`` samples nearest to
it on each side are dropped (footnote to Eq. rho-asym).

Parity pins: Sec. 6.3.4 (FCF factors of the third-order schemes bounded by 0.6)
and Sec. 6.4 (ERK4+U4, m = 2: about 0.15 just below c/c_max = 0.24 and about
0.84 just above).
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


def two_level_factor(p, kind, c, m, nu=1, omit=0, n=1 << 11):
    """LFA factor of two-level MGRIT with the corrected SL coarse operator."""
    omega = omega_samples(n, omit)
    lam = ops.FineOperator(p, kind, p, c).symbol(omega)
    mu = corrected_sl_symbol(p, kind, c, m, omega)
    return rho(lam, mu, m, nu)
