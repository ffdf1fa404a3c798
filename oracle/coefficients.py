"""Discretisation coefficients, derived from the paper's definitions (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written in exact rational
arithmetic where the paper's definitions are rational, FP64 elsewhere.

Function                     paper passage                          parity pin
---------------------------  -------------------------------------  ---------------------------------
upwind_bias(p)               Sec. 4.1 (stencil bias l(p), r(p))     Table 1 via e_fd_from_taps
upwind_taps(p)               Sec. 4.1 (derivative of the degree-p   polynomial exactness, Table 1
                             interpolant on x_i + jh, j=-l..r)
e_fd(p)                      Lemma 4.1, Eq. (e_FD_def)              Table 1 (left), tap moments
rk_stability_poly(q)         Sec. 4.2, Eq. (RK_stab_def)            Table 1 (right), Table 2
erk_tableau(q), q<=4         Sec. 4.2 (classical ERKq)              stage form == polynomial form
sdirk_tableau(q), q<=4       Sec. 4.2 (SDIRK1 = implicit Euler,     Table 1 (right) e_RK values
                             SDIRK2-4 L-stable tableaux)
sdirk5_gamma, sdirk5_*       Sec. 4.2, footnote on SDIRK5           Table 1 e_RK(SDIRK5), L-stability
e_rk(kind, q)                Eq. (e_RK_def)                         Table 1 (right)
cfl_limit(p)                 Sec. 4.3, Table 2                      Table 2 for ERK1-4; ERK5: see below
sl_shift(s)                  Sec. 3 (departure point x_i - alpha    exact shift when s is an integer
                             Delta = x_i^{(Delta)} - h eps)
sl_nodes(p, eps)             Sec. 3 (p+1 nodes nearest departure)   -
sl_weights(p, eps)           Sec. 3 (Lagrange interpolation)        polynomial exactness, sum = 1
f_poly(p, eps)               Lemma 3.1, Eq. (fpoly_def)             SL truncation-error order test
diff_taps(p)                 Eq. (Dp+1_def); s = 2 symmetric for    moments: (p+1)! on x^{p+1}
                             odd p (Sec. 6.3), s = 1 one-point
                             left bias for even p (Sec. 6.4)
phi_levels(...)              Lemma 6.1 Eq. (varphi-constant-MOL-SL) Lemma 6.1 O(h^{p+2}) order test
                             and the Sec. 6.2 multilevel recursion
phi_levels_general(...)      builder reading for q != p: Lemma 4.2   order tests: the dominant term's
                             carries both D^{(p+1)} and D^{(q+1)}     constant gains an order in h on
                             terms; App. B steps applied to each      level 1; level 2 vs (level 1)^m

ERK5: the tableau is not printed.  The stability polynomial is taken as the
degree-5 Taylor polynomial plus beta_6 z^6 with beta_6 = 1/1280, which is what
Table 1's e_RK(ERK5) fixes.  Table 2's ERK5 CFL limit (1.96583) is NOT
reproduced by this polynomial (it gives 1.9403...), so ERK5 is "parity
unpinned" against the paper's exact ERK5 method.
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np

# ----------------------------------------------------------------------------
# Sec. 4.1  Upwind finite differences U_p
# ----------------------------------------------------------------------------


def upwind_bias(p):
    """(l(p), r(p)) of the upwind stencil {x_i + j h}, j = -l..r (Sec. 4.1).

    Odd p: one-point bias, l = (p+1)/2, r = l - 1.
    Even p: two-point bias, l = p/2 + 1, r = l - 2.
    """
    if p < 1:
        raise ValueError("p >= 1")
    if p % 2 == 1:
        l = (p + 1) // 2
        return l, l - 1
    l = p // 2 + 1
    return l, l - 2


def _lagrange_derivative_at(nodes, j, x0):
    """d/ds of the Lagrange basis polynomial of node j, evaluated at s = x0."""
    total = Fraction(0)
    for m in nodes:
        if m == j:
            continue
        term = Fraction(1, j - m)
        for k in nodes:
            if k in (j, m):
                continue
            term *= Fraction(x0 - k, j - k)
        total += term
    return total


def upwind_taps(p):
    """Taps {j: l_j} of L_p with (L_p u)_i = sum_j l_j u_{i+j} (periodic).

    L_p / h differentiates the degree-p interpolant through x_i + j h,
    j = -l(p)..r(p), at x_i (Sec. 4.1).  Exact rationals.
    """
    l, r = upwind_bias(p)
    nodes = list(range(-l, r + 1))
    return {j: _lagrange_derivative_at(nodes, j, 0) for j in nodes}


def e_fd(p):
    """e_FD = (-1)^{r(p)} l(p)! r(p)! / (p+1)!  (Lemma 4.1, Eq. e_FD_def)."""
    l, r = upwind_bias(p)
    return Fraction((-1) ** r * factorial(l) * factorial(r), factorial(p + 1))


def e_fd_from_taps(p):
    """Leading error constant of L_p/h read off its taps.

    Taylor expanding sum_j l_j u(x + jh)/h gives u' + h^p u^{(p+1)} *
    sum_j l_j j^{p+1}/(p+1)! + ..., so d/dx - L_p/h = h^p e_FD u^{(p+1)} with
    e_FD = -sum_j l_j j^{p+1} / (p+1)!.
    """
    taps = upwind_taps(p)
    return -sum(c * Fraction(j) ** (p + 1) for j, c in taps.items()) / factorial(p + 1)


# ----------------------------------------------------------------------------
# Sec. 4.2  Runge-Kutta methods
# ----------------------------------------------------------------------------


def rk_stability_poly(q):
    """Coefficients beta_0..beta_s of the ERKq stability polynomial R_q(z).

    ERK1-4: the order-q Taylor polynomial of exp(z) (q-stage methods of
    order q exist for q <= 4, so R_q has degree q).  ERK5: Taylor degree 5
    plus beta_6 = 1/1280 (from Table 1's e_RK = beta_6 - 1/720).
    """
    if q < 1 or q > 5:
        raise ValueError("ERK order 1..5")
    beta = [Fraction(1, factorial(j)) for j in range(q + 1)]
    if q == 5:
        beta.append(Fraction(1, 1280))
    return beta


def erk_tableau(q):
    """Classical explicit tableaux (A, b) for q = 1..4 (textbook methods).

    Used only to cross-check that the stage form reproduces R_q(z).
    """
    if q == 1:
        return [[0.0]], [1.0]
    if q == 2:  # Heun
        return [[0.0, 0.0], [1.0, 0.0]], [0.5, 0.5]
    if q == 3:  # Kutta's third-order method
        return ([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [-1.0, 2.0, 0.0]],
                [1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0])
    if q == 4:  # classical RK4
        return ([[0.0] * 4, [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1.0, 0]],
                [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0])
    raise ValueError("no ERK5 tableau is printed in the paper")


def _sdirk3_gamma():
    """Root in (0.4, 0.5) of gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6 (L-stable
    3-stage third-order SDIRK)."""
    lo, hi = 0.4, 0.5
    f = lambda g: g ** 3 - 3 * g ** 2 + 1.5 * g - 1.0 / 6.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def sdirk_tableau(q):
    """Stiffly accurate, L-stable SDIRK tableaux (A, b) for q = 1..4.

    SDIRK1: implicit Euler.  SDIRK2: 2 stages, gamma = 1 - 1/sqrt(2).
    SDIRK3: 3 stages, gamma the root above.  SDIRK4: 5 stages, gamma = 1/4.
    The paper defers these tableaux to its earlier work; they are pinned here
    by Table 1's e_RK values.
    """
    if q == 1:
        return [[1.0]], [1.0]
    if q == 2:
        g = 1.0 - 1.0 / np.sqrt(2.0)
        return [[g, 0.0], [1.0 - g, g]], [1.0 - g, g]
    if q == 3:
        g = _sdirk3_gamma()
        b1 = -(6 * g * g - 16 * g + 1) / 4.0
        b2 = (6 * g * g - 20 * g + 5) / 4.0
        return ([[g, 0.0, 0.0], [(1 - g) / 2.0, g, 0.0], [b1, b2, g]], [b1, b2, g])
    if q == 4:
        A = [[0.25, 0, 0, 0, 0],
             [0.5, 0.25, 0, 0, 0],
             [17.0 / 50, -1.0 / 25, 0.25, 0, 0],
             [371.0 / 1360, -137.0 / 2720, 15.0 / 544, 0.25, 0],
             [25.0 / 24, -49.0 / 48, 125.0 / 16, -85.0 / 12, 0.25]]
        return A, list(A[-1])
    raise ValueError("SDIRK5 is handled through its factored stability function")


def _sdirk5_p5(g):
    """z^5 coefficient of trunc_5[(1 - g z)^5 e^z]."""
    return sum(comb(5, j) * (-g) ** j / factorial(5 - j) for j in range(6))


def sdirk5_gamma():
    """gamma of the 5-stage, order-5, L-stable SDIRK stability function.

    For an s-stage SDIRK of order s, R(z) = P(z)/(1 - gamma z)^s with
    P = trunc_s[(1 - gamma z)^s e^z]; L-stability needs deg P < s, i.e. the
    z^5 coefficient vanishes.  We take the root near 0.278 (Table 1 then
    gives e_RK = 5.3005e-4, checked in the tests).
    """
    lo, hi = 0.25, 0.30
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _sdirk5_p5(lo) * _sdirk5_p5(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def sdirk5_numerator(g=None):
    """Coefficients p_0..p_4 of P(z) = trunc_4[(1 - g z)^5 e^z]."""
    if g is None:
        g = sdirk5_gamma()
    return [sum(comb(5, j) * (-g) ** j / factorial(k - j) for j in range(k + 1))
            for k in range(5)]


def e_rk(kind, q):
    """e_RK = beta_{q+1} - 1/(q+1)!  (Eq. e_RK_def), beta from the method."""
    if kind == "erk":
        beta = rk_stability_poly(q)
        bq1 = float(beta[q + 1]) if len(beta) > q + 1 else 0.0
        return bq1 - 1.0 / factorial(q + 1)
    if kind == "sdirk":
        if q == 5:
            g = sdirk5_gamma()
            # R - e^z = -(t_6 z^6 + ...)/(1 - g z)^5, t_6 the z^6 coefficient
            # of (1 - g z)^5 e^z.
            t6 = sum(comb(5, j) * (-g) ** j / factorial(6 - j) for j in range(6))
            return -t6
        A, b = sdirk_tableau(q)
        A = np.array(A, dtype=np.float64)
        b = np.array(b, dtype=np.float64)
        one = np.ones(len(b))
        # Taylor coefficients of R(z) = 1 + z b^T (I - zA)^{-1} 1:
        # beta_j = b^T A^{j-1} 1.
        beta_q1 = b @ np.linalg.matrix_power(A, q) @ one
        return float(beta_q1) - 1.0 / factorial(q + 1)
    raise ValueError(kind)


def rk_stability_value(kind, q, z):
    """R_q(z) for complex z (used by the CFL limit and the LFA)."""
    z = np.asarray(z, dtype=np.complex128)
    if kind == "erk":
        beta = [float(b) for b in rk_stability_poly(q)]
        return sum(bj * z ** j for j, bj in enumerate(beta))
    if q == 5:
        g = sdirk5_gamma()
        P = sdirk5_numerator(g)
        return sum(pk * z ** k for k, pk in enumerate(P)) / (1.0 - g * z) ** 5
    A, b = sdirk_tableau(q)
    A = np.array(A, dtype=np.complex128)
    b = np.array(b, dtype=np.complex128)
    s = len(b)
    out = np.empty(z.shape, dtype=np.complex128)
    for idx, zz in np.ndenumerate(z):
        Y = np.linalg.solve(np.eye(s) - zz * A, np.ones(s))
        out[idx] = 1.0 + zz * (b @ Y)
    return out


def upwind_symbol(p, omega):
    """lambda_L(omega) = sum_j l_j e^{i j omega} of L_p."""
    omega = np.asarray(omega, dtype=np.float64)
    return sum(float(c) * np.exp(1j * j * omega) for j, c in upwind_taps(p).items())


def cfl_limit(p, samples=1 << 14, c_hi=4.0):
    """Largest c with max_omega |R_p(-c lambda_L(omega))| <= 1 for all c' <= c.

    ERKp+Up pairing (q = p), Sec. 4.3 / Table 2.  A coarse scan over c finds
    the first unstable c, then bisection sharpens it.
    """
    omega = np.linspace(-np.pi, np.pi, samples, endpoint=False)
    lam = upwind_symbol(p, omega)

    def stable(c):
        return np.max(np.abs(rk_stability_value("erk", p, -c * lam))) <= 1.0 + 1e-13

    c = 1e-3
    step = 1e-3
    while c < c_hi and stable(c + step):
        c += step
    lo, hi = c, c + step
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo


# ----------------------------------------------------------------------------
# Sec. 3  Semi-Lagrangian step S_p^{(Delta)} and Lemma 3.1
# ----------------------------------------------------------------------------


def sl_shift(s):
    """Split the departure offset s = alpha Delta / h into (k, eps).

    x_i - alpha Delta = x_{i-k} - h eps with x_{i-k} the mesh point just east
    of the departure point and eps in [0, 1) (Sec. 3): k = floor(s),
    eps = s - k.
    """
    k = int(np.floor(s))
    eps = float(s - k)
    if eps >= 1.0:  # guard against floor rounding
        k += 1
        eps -= 1.0
    return k, eps


def sl_nodes(p, eps):
    """Offsets j (relative to x_{i-k}) of the p+1 mesh points nearest to the
    departure point at relative position -eps (Sec. 3).

    Odd p: j = -(p+1)/2 .. (p-1)/2 for every eps in [0, 1).
    Even p: the odd count of nodes is centred on the nearer of x_{i-k} and
    x_{i-k-1}: j = -p/2 .. p/2 if eps < 1/2, else j = -p/2-1 .. p/2-1
    (eps = 1/2 is a tie; this reading takes the left set).
    """
    if p % 2 == 1:
        return list(range(-(p + 1) // 2, (p - 1) // 2 + 1))
    h = p // 2
    if eps < 0.5:
        return list(range(-h, h + 1))
    return list(range(-h - 1, h))


def sl_weights(p, eps):
    """Lagrange weights w_j with (S u)_i = sum_j w_j u_{i-k+j}: the degree-p
    interpolant through x_{i-k} + j h evaluated at x_{i-k} - eps h."""
    nodes = sl_nodes(p, eps)
    x = -eps
    w = {}
    for j in nodes:
        v = 1.0
        for q in nodes:
            if q != j:
                v *= (x - q) / (j - q)
        w[j] = v
    return w


def f_poly(p, z, nodes=None):
    """f_{p+1}(z) = (1/(p+1)!) prod_{j=-l(p)}^{r(p)} (j + z)  (Eq. fpoly_def).

    l(p), r(p) are those of the SL interpolation stencil (Sec. 3), so for
    even p the node set depends on eps (pass ``nodes`` from sl_nodes).
    """
    if nodes is None:
        nodes = sl_nodes(p, z)
    v = 1.0
    for j in nodes:
        v *= (j + z)
    return v / factorial(p + 1)


# ----------------------------------------------------------------------------
# Eq. (Dp+1_def)  difference matrices D^{(p+1)}_s
# ----------------------------------------------------------------------------


def diff_taps(order, p_for_bias=None):
    """Taps {j: d_j} of D^{(order)}_s (unscaled by h), periodic.

    The stencil is the order-th derivative of the degree-``order``
    interpolant through ``order``+1 consecutive nodes, times h^{order}:
    d_j = order! / prod_{k != j} (j - k).  Node sets: for even ``order``
    (odd p, Sec. 6.3: symmetric, s = 2) j = -order/2 .. order/2; for odd
    ``order`` (even p, Sec. 6.4: first order, one-point bias to the left)
    j = -(order+1)/2 .. (order-1)/2.
    """
    if order % 2 == 0:
        nodes = list(range(-order // 2, order // 2 + 1))
    else:
        nodes = list(range(-(order + 1) // 2, (order - 1) // 2 + 1))
    taps = {}
    for j in nodes:
        den = 1
        for k in nodes:
            if k != j:
                den *= (j - k)
        taps[j] = Fraction(factorial(order), den)
    return taps


# ----------------------------------------------------------------------------
# Lemma 6.1 and Sec. 6.2: the truncation-error correction constants
# ----------------------------------------------------------------------------


def level_factors(m, levels):
    """Coarsening factors m_1 .. m_{levels-1} (m_l: fine steps of level l-1
    per step of level l).  ``m`` is one factor for every level, or the list
    of them (the paper's parallel runs coarsen by 16 once and by 4 below,
    Sec. 6.3.2)."""
    if np.isscalar(m):
        return [int(m)] * (levels - 1)
    ms = [int(x) for x in m]
    if len(ms) != levels - 1:
        raise ValueError("need one coarsening factor per coarse level")
    return ms


def level_steps(m, levels):
    """Time step of level l in units of dt: m_1 m_2 .. m_l (l = 1..levels-1)."""
    out, t = [], 1
    for f in level_factors(m, levels):
        t *= f
        out.append(t)
    return out


def level_step(m, level):
    """Time step of level ``level`` in units of dt: m^level for one factor,
    else the product of the first ``level`` factors."""
    if np.isscalar(m):
        return int(m) ** level
    t = 1
    for f in list(m)[:level]:
        t *= int(f)
    return t


def level_shifts(c, m, levels):
    """(k_l, eps_l) of the SL step on level l = 1..levels-1 (step
    m_1 .. m_l dt, so the departure offset is m_1 .. m_l c grid cells)."""
    return [sl_shift(c * t) for t in level_steps(m, levels)]


def phi_levels(p, kind, c, m, levels):
    """phi_{p+1} of level l = 1..levels-1 (index 0 of the result is l=1).

    l = 1:  m_1 [c e_FD + (-c)^{p+1} e_RK] + (-1)^{p+1} f_{p+1}(eps_1)
            (Lemma 6.1, Eq. varphi-constant-MOL-SL)
    l > 1:  (-1)^{p+1} [ -m_l f_{p+1}(eps_{l-1}) + f_{p+1}(eps_l) ] + m_l phi_{l-1}
            (Sec. 6.2, the phi recursion below Eq. MOL-SL-corrected-multilevel,
            written there for one factor m; with level factors m_l the same
            argument -- level l matches m_l steps of level l-1 -- gives m_l in
            place of m).
    q = p is assumed, as in the paper.
    """
    q = p
    efd = float(e_fd(p))
    erk = e_rk(kind, q)
    sgn = (-1) ** (p + 1)
    ms = level_factors(m, levels)
    shifts = level_shifts(c, m, levels)
    out = []
    for idx, (_, eps) in enumerate(shifts):
        f_l = f_poly(p, eps)
        if idx == 0:
            phi = ms[0] * (c * efd + (-c) ** (p + 1) * erk) + sgn * f_l
        else:
            f_prev = f_poly(p, shifts[idx - 1][1])
            phi = sgn * (-ms[idx] * f_prev + f_l) + ms[idx] * out[-1]
        out.append(phi)
    return out


def phi_levels_general(p, kind, q, c, m, levels):
    """Builder reading for q != p (the paper derives the correction for q = p
    only; this extends it).

    Lemma 4.2 gives the one-step error -[c e_FD D^{(p+1)} + (-c)^{q+1} e_RK
    D^{(q+1)}] u.  Repeating the App. B argument keeps the two terms apart:
    Psi = (I - phi_p D^{(p+1)} - phi_q D^{(q+1)})^{-1} S_p with
      phi_p(l=1) = m c e_FD + (-1)^{p+1} f_{p+1}(eps_1),
      phi_p(l>1) = (-1)^{p+1}[-m f(eps_{l-1}) + f(eps_l)] + m phi_p(l-1),
      phi_q(l=1) = m (-c)^{q+1} e_RK,   phi_q(l>1) = m phi_q(l-1).
    For q = p the two constants add up to phi_levels(...).
    Returns a list of (phi_p, phi_q) pairs.

    Pinned by truncation order (tests/test_oracle_coefficients.py): on level
    1 the constant of the dominant error term gains one order in h over a
    zero or sign-flipped constant (phi_q for q < p, phi_p for q > p); on
    level 2 the U5 + SDIRK3 operator matches (level 1)^m to O(h^7), while a
    phi_q recursion without its factor m leaves O(h^4) and a phi_p one
    without m leaves O(h^6).
    """
    efd = float(e_fd(p))
    erk = e_rk(kind, q)
    sgn = (-1) ** (p + 1)
    ms = level_factors(m, levels)
    shifts = level_shifts(c, m, levels)
    out = []
    for idx, (_, eps) in enumerate(shifts):
        f_l = f_poly(p, eps)
        if idx == 0:
            fp = ms[0] * c * efd + sgn * f_l
            fq = ms[0] * (-c) ** (q + 1) * erk
        else:
            f_prev = f_poly(p, shifts[idx - 1][1])
            fp = sgn * (-ms[idx] * f_prev + f_l) + ms[idx] * out[-1][0]
            fq = ms[idx] * out[-1][1]
        out.append((fp, fq))
    return out
