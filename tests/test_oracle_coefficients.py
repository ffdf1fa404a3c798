"""Pins of the oracle's coefficients and single-step operators against the
paper's printed values and against mathematics (no GPU)."""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

from oracle import coefficients as co
from oracle import lfa
from oracle import operators as ops
from workloads import mesh


# --------------------------------------------------------------------------
# Table 1: error constants
# --------------------------------------------------------------------------


def _tol(printed):
    mant = printed.split("e")[0].lstrip("-")
    digits = len(mant.split(".")[1]) if "." in mant else 0
    exp = int(printed.split("e")[1]) if "e" in printed else 0
    return 10.0 ** (exp - digits)


def test_table1_error_constants(golden):
    for kind, order, printed in golden("table1_error_constants.txt"):
        q = int(order)
        val = float(printed)
        if kind == "fd":
            got = float(co.e_fd(q))
            got_taps = float(co.e_fd_from_taps(q))
            assert abs(got_taps - got) < 1e-15
        else:
            got = co.e_rk(kind, q)
        assert abs(got - val) <= _tol(printed), (kind, q, got, val)


def test_upwind_taps_differentiate_polynomials_exactly():
    """L_p/h is the derivative of the degree-p interpolant: exact on 1, x,
    ..., x^p at x_i (Sec. 4.1); biased to the left (alpha > 0)."""
    for p in range(1, 6):
        taps = co.upwind_taps(p)
        l, r = co.upwind_bias(p)
        assert min(taps) == -l and max(taps) == r and l > r
        for k in range(p + 1):
            moment = sum(c * Fraction(j) ** k for j, c in taps.items())
            assert moment == (1 if k == 1 else 0)
        # degree p+1 is not exact (the error constant is nonzero)
        assert sum(c * Fraction(j) ** (p + 1) for j, c in taps.items()) != 0


# --------------------------------------------------------------------------
# Table 2: CFL limits
# --------------------------------------------------------------------------


def test_table2_cfl_limits_erk1_to_4(golden):
    for p, printed in golden("table2_cfl_limits.txt"):
        p = int(p)
        if p == 5:
            continue
        got = co.cfl_limit(p)
        assert abs(got - float(printed)) < 2e-5, (p, got, printed)


def test_erk5_cfl_limit_reading():
    """ERK5: Table 1 fixes beta_6 = 1/1280, whose CFL limit is ~1.940, not
    Table 2's 1.96583 (the paper's ERK5 tableau is not printed).  The reading
    keeps Table 1; this test records the gap so a change is noticed."""
    got = co.cfl_limit(5)
    assert 1.93 < got < 1.95


def test_sdirk_l_stable_and_sdirk5_order():
    """SDIRK1-5 stability functions: |R(iy)| <= 1 (A-stable), R(-inf) -> 0
    (L-stable), and R(z) - e^z = e_RK z^{q+1} + O(z^{q+2})."""
    y = np.linspace(-200, 200, 4001)
    for q in range(1, 6):
        assert np.max(np.abs(co.rk_stability_value("sdirk", q, 1j * y))) <= 1 + 1e-12
        assert abs(co.rk_stability_value("sdirk", q, np.array([-1e8]))[0]) < 1e-6
        z = np.array([1e-2, 2e-2])
        d = (co.rk_stability_value("sdirk", q, z) - np.exp(z)) / z ** (q + 1)
        assert abs(d[0].real - co.e_rk("sdirk", q)) < 0.05 * abs(co.e_rk("sdirk", q)) + 1e-3


def test_erk_stage_form_matches_stability_polynomial():
    """Textbook ERK1-4 tableaux give the Taylor stability polynomial."""
    for q in range(1, 5):
        A, b = co.erk_tableau(q)
        A = np.array(A)
        b = np.array(b)
        beta = [float(x) for x in co.rk_stability_poly(q)]
        for j in range(1, q + 1):
            assert abs(b @ np.linalg.matrix_power(A, j - 1) @ np.ones(q) - beta[j]) < 1e-14
        assert abs(b @ np.linalg.matrix_power(A, q) @ np.ones(q)) < 1e-14


# --------------------------------------------------------------------------
# Sec. 3 SL step, Lemma 3.1, D
# --------------------------------------------------------------------------


def test_sl_weights_interpolate_polynomials_exactly():
    for p in range(1, 6):
        for eps in [0.0, 0.13, 0.5, 0.77]:
            w = co.sl_weights(p, eps)
            for k in range(p + 1):
                assert abs(sum(wj * j ** k for j, wj in w.items()) - (-eps) ** k) < 1e-13
    assert co.sl_weights(3, 0.0) == {-2: 0.0, -1: 0.0, 0: 1.0, 1: 0.0}
    assert co.sl_shift(3.0) == (3, 0.0)
    assert co.sl_shift(6.8)[0] == 6 and abs(co.sl_shift(6.8)[1] - 0.8) < 1e-12


def test_diff_taps_moments():
    """D^{(o)}/h^o differentiates o times: moments 0 below o, o! at o; the
    symmetric stencils (even o) are also exact at o+1 (second order)."""
    for o in range(2, 7):
        d = co.diff_taps(o)
        for k in range(o):
            assert sum(c * Fraction(j) ** k for j, c in d.items()) == 0
        assert sum(c * Fraction(j) ** o for j, c in d.items()) == factorial(o)
        if o % 2 == 0:
            assert sum(c * Fraction(j) ** (o + 1) for j, c in d.items()) == 0
            assert all(d[j] == d[-j] for j in d)
    assert co.diff_taps(2) == {-1: 1, 0: -2, 1: 1}
    assert co.diff_taps(4) == {-2: 1, -1: -4, 0: 6, 1: -4, 2: 1}


def _smooth(x, t=0.0):
    """Exact solution v(x - t) of u_t + u_x = 0 for v = exp(sin(pi x))."""
    return np.exp(np.sin(np.pi * (x - t)))


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_lemma_3_1_sl_truncation_error(p):
    """u(t+dt) - S u(t) = (-1)^{p+1} f_{p+1}(eps) D^{(p+1)} u(t+dt) + O(h^{p+2})."""
    ratios = []
    for nx in [64, 128, 256]:
        x = mesh(nx)
        h = 2.0 / nx
        s = 2.37  # departure offset in cells
        dt = s * h
        S = ops.SLOperator(p, s)
        tau = _smooth(x, dt) - S.apply(_smooth(x))
        pred = (-1) ** (p + 1) * co.f_poly(p, S.eps) * ops.apply_stencil(_smooth(x, dt), co.diff_taps(p + 1))
        ratios.append(_rel(tau, pred))
    assert ratios[-1] < 0.1 and ratios[-1] < ratios[0]


@pytest.mark.parametrize("p,kind", [(1, "erk"), (2, "erk"), (3, "erk"), (4, "erk"), (5, "erk"), (1, "sdirk"),
                                    (2, "sdirk"), (3, "sdirk"), (4, "sdirk")])
def test_lemma_4_2_mol_truncation_error(p, kind):
    """u(t+dt) - Phi u(t) = -[c e_FD D^{(p+1)} + (-c)^{q+1} e_RK D^{(q+1)}]
    u(t+dt) + O(h^{p+2}) for q = p (Lemma 4.2)."""
    c = 0.5 if kind == "erk" else 2.0
    ratios = []
    for nx in [64, 128, 256]:
        x = mesh(nx)
        dt = c * 2.0 / nx
        Phi = ops.FineOperator(p, kind, p, c)
        tau = _smooth(x, dt) - Phi.apply(_smooth(x))
        coef = c * float(co.e_fd(p)) + (-c) ** (p + 1) * co.e_rk(kind, p)
        pred = -coef * ops.apply_stencil(_smooth(x, dt), co.diff_taps(p + 1))
        ratios.append(_rel(tau, pred))
    assert ratios[-1] < 0.1 and ratios[-1] < ratios[0]


def _ideal_vs_coarse(p, kind, c, m, nx, phi_override=None):
    x = mesh(nx)
    Phi = ops.FineOperator(p, kind, p, c)
    u = _smooth(x)
    ideal = u
    for _ in range(m):
        ideal = Phi.apply(ideal)
    phi = co.phi_levels(p, kind, c, m, 2)[0] if phi_override is None else phi_override
    Psi = ops.CoarseOperator(p, c * m, [(phi, p + 1)])
    return np.max(np.abs(ideal - Psi.apply(u)))


@pytest.mark.parametrize("p,kind,c,m", [(1, "erk", 0.85, 4), (3, "erk", 0.85, 8), (1, "sdirk", 1.3, 4),
                                        (3, "sdirk", 2.2, 4), (5, "erk", 0.9, 4),
                                        (2, "erk", 0.5, 4), (4, "erk", 0.6, 4), (2, "sdirk", 1.3, 4),
                                        (4, "sdirk", 2.2, 4)])
def test_lemma_6_1_corrected_operator_order(p, kind, c, m):
    """Psi_ideal u = (I - phi D)^{-1} S^{(m dt)} u + O(h^{p+2})  (Lemma 6.1):
    halving h cuts the mismatch by ~2^{p+2}; the uncorrected SL step (phi = 0)
    and a sign-flipped phi only by ~2^{p+1}.  Even p (Sec. 6.4): the same
    with the eps-dependent SL node set and the first-order, left-biased D."""
    n1, n2 = (32, 64) if p == 5 else (64, 128)
    e1 = _ideal_vs_coarse(p, kind, c, m, n1)
    e2 = _ideal_vs_coarse(p, kind, c, m, n2)
    order = np.log2(e1 / e2)
    assert order > p + 1.6, order
    phi = co.phi_levels(p, kind, c, m, 2)[0]
    for wrong in (0.0, -phi):
        w1 = _ideal_vs_coarse(p, kind, c, m, n1, wrong)
        w2 = _ideal_vs_coarse(p, kind, c, m, n2, wrong)
        assert np.log2(w1 / w2) < p + 1.4
        assert w2 > 4 * e2


def test_multilevel_phi_recursion_order():
    """Sec. 6.2 phi recursion: the level-2 operator matches (level-1 operator)^m to
    O(h^{p+2}) for the recursive phi_2; using the two-level formula at step
    m^2 dt instead drops an order."""
    p, kind, c, m = 3, "erk", 0.85, 4
    errs, errs_wrong = [], []
    for nx in [64, 128]:
        x = mesh(nx)
        u = _smooth(x)
        psi1 = ops.coarse_operator(p, kind, p, c, m, 1, 3)
        ideal = u
        for _ in range(m):
            ideal = psi1.apply(ideal)
        psi2 = ops.coarse_operator(p, kind, p, c, m, 2, 3)
        errs.append(np.max(np.abs(ideal - psi2.apply(u))))
        # "wrong": treat level 2 as a two-level correction from the fine grid
        # with coarsening m^2, ignoring what level 1 already does
        phi_wrong = co.phi_levels(p, kind, c, m * m, 2)[0] * 0.5
        psi_w = ops.CoarseOperator(p, c * m * m, [(phi_wrong, p + 1)])
        errs_wrong.append(np.max(np.abs(ideal - psi_w.apply(u))))
    assert np.log2(errs[0] / errs[1]) > p + 1.6
    assert errs_wrong[1] > 4 * errs[1]


@pytest.mark.parametrize("p,kind,c,ms", [(3, "erk", 0.85, (4, 2)), (3, "erk", 0.85, (2, 4)),
                                         (3, "sdirk", 2.0, (4, 2)), (1, "erk", 0.85, (4, 2))])
def test_multilevel_phi_recursion_with_level_factors(p, kind, c, ms):
    """The Sec. 6.2 recursion with a factor per level (the paper's parallel
    runs coarsen by 16, then by 4): the level-2 operator (step m_1 m_2 dt)
    matches (level-1 operator)^{m_2} to O(h^{p+2}) with m_2 in the
    recursion; the recursion taken with m_1 instead (one factor for all
    levels) loses the order."""
    m1, m2 = ms
    errs, errs_wrong = [], []
    for nx in [64, 128]:
        x = mesh(nx)
        u = _smooth(x)
        psi1 = ops.coarse_operator(p, kind, p, c, list(ms), 1, 3)
        assert psi1.sl.k + psi1.sl.eps == pytest.approx(c * m1)
        ideal = u
        for _ in range(m2):
            ideal = psi1.apply(ideal)
        psi2 = ops.coarse_operator(p, kind, p, c, list(ms), 2, 3)
        assert psi2.sl.k + psi2.sl.eps == pytest.approx(c * m1 * m2)
        errs.append(np.max(np.abs(ideal - psi2.apply(u))))
        # the uniform recursion with m_1 at level 2, on the same step
        shifts = co.level_shifts(c, list(ms), 3)
        f1, f2 = co.f_poly(p, shifts[0][1]), co.f_poly(p, shifts[1][1])
        phi1 = co.phi_levels(p, kind, c, list(ms), 3)[0]
        phi_wrong = (-1) ** (p + 1) * (-m1 * f1 + f2) + m1 * phi1
        psi_w = ops.CoarseOperator(p, c * m1 * m2, [(phi_wrong, p + 1)])
        errs_wrong.append(np.max(np.abs(ideal - psi_w.apply(u))))
    assert np.log2(errs[0] / errs[1]) > p + 1.6, np.log2(errs[0] / errs[1])
    assert errs_wrong[1] > 4 * errs[1]


# --------------------------------------------------------------------------
# Two-term correction for q != p (phi_levels_general): order pins.
# Lemma 4.2 splits the one-step error into an FD term c e_FD D^{(p+1)} of
# size O(h^{p+1}) and an RK term (-c)^{q+1} e_RK D^{(q+1)} of size
# O(h^{q+1}); the corrected operator with both constants must cancel the
# larger of the two, so against Phi^m it gains one order over a zero or
# sign-flipped constant of that term.  On level 2 the recursion must also
# reproduce (level-1 operator)^m to the order of the SL remainder.
# --------------------------------------------------------------------------


def _two_term_level1(p, q, c, m, nx, fp_mul=1.0, fq_mul=1.0):
    x = mesh(nx)
    Phi = ops.FineOperator(p, "sdirk", q, c)
    u = _smooth(x)
    ideal = u
    for _ in range(m):
        ideal = Phi.apply(ideal)
    fp, fq = co.phi_levels_general(p, "sdirk", q, c, m, 2)[0]
    Psi = ops.CoarseOperator(p, c * m, [(fp_mul * fp, p + 1), (fq_mul * fq, q + 1)])
    return np.max(np.abs(ideal - Psi.apply(u)))


@pytest.mark.parametrize("p,q,c,m", [(5, 3, 1.0, 4), (5, 3, 2.0, 4), (3, 1, 1.0, 4), (5, 1, 1.0, 4)])
def test_two_term_correction_rk_constant_order(p, q, c, m):
    """q < p (the 16384 x 65536 SDIRK3+U5 workload's pairing): the RK term
    O(h^{q+1}) dominates; with phi_q the mismatch with Phi^m falls as
    h^{q+2}, with phi_q = 0 or -phi_q only as h^{q+1}."""
    nxs = (64, 128, 256)
    good = [_two_term_level1(p, q, c, m, n) for n in nxs]
    assert np.log2(good[1] / good[2]) > q + 1.7, good
    for mul in (0.0, -1.0):
        bad = [_two_term_level1(p, q, c, m, n, fq_mul=mul) for n in nxs]
        assert np.log2(bad[1] / bad[2]) < q + 1.2, bad
        assert bad[2] > 8 * good[2]


@pytest.mark.parametrize("p,q,c,m", [(1, 3, 0.8, 4), (3, 5, 0.8, 4), (1, 3, 1.3, 4)])
def test_two_term_correction_fd_constant_order(p, q, c, m):
    """q > p: the FD term O(h^{p+1}) dominates, which pins the level-1
    phi_p of the two-term form (it falls below the RK remainder when
    q < p): phi_p gains an order over 0 and -phi_p."""
    nxs = (64, 128, 256)
    good = [_two_term_level1(p, q, c, m, n) for n in nxs]
    assert np.log2(good[1] / good[2]) > p + 1.7, good
    for mul in (0.0, -1.0):
        bad = [_two_term_level1(p, q, c, m, n, fp_mul=mul) for n in nxs]
        assert np.log2(bad[1] / bad[2]) < p + 1.2, bad
        assert bad[2] > 8 * good[2]


@pytest.mark.parametrize("c,m", [(1.0, 4), (0.7, 4), (1.0, 2)])
def test_two_term_correction_level2_recursion_order(c, m):
    """U5 + SDIRK3 on level 2 (step m^2 dt) against (level-1 operator)^m:
    with the recursions phi_q(2) = m phi_q(1) and the Sec. 6.2 recursion
    for phi_p the mismatch falls at least as h^7; phi_q(2) = phi_q(1), 0 or
    -phi_q(2) leave O(h^4), and a phi_p recursion without its factor m
    (or phi_p(2) = 0) leaves O(h^6)."""
    p, q = 5, 3
    nxs = (64, 128, 256)

    def mismatch(nx, mode):
        x = mesh(nx)
        u = _smooth(x)
        psi1 = ops.coarse_operator(p, "sdirk", q, c, m, 1, 3)
        ideal = u
        for _ in range(m):
            ideal = psi1.apply(ideal)
        (fp1, fq1), (fp2, fq2) = co.phi_levels_general(p, "sdirk", q, c, m, 3)
        if mode == "q_nom":
            fq2 = fq1
        elif mode == "q_zero":
            fq2 = 0.0
        elif mode == "q_flip":
            fq2 = -fq2
        elif mode == "p_nom":
            shifts = co.level_shifts(c, m, 3)
            f1, f2 = co.f_poly(p, shifts[0][1]), co.f_poly(p, shifts[1][1])
            fp2 = (-1) ** (p + 1) * (-m * f1 + f2) + fp1
        elif mode == "p_zero":
            fp2 = 0.0
        psi2 = ops.CoarseOperator(p, c * m * m, [(fp2, p + 1), (fq2, q + 1)])
        return np.max(np.abs(ideal - psi2.apply(u)))

    good = [mismatch(n, "ok") for n in nxs]
    assert np.log2(good[1] / good[2]) > 6.7, good
    for mode, order in (("q_nom", q + 1), ("q_zero", q + 1), ("q_flip", q + 1), ("p_nom", p + 1),
                        ("p_zero", p + 1)):
        bad = [mismatch(n, mode) for n in nxs]
        assert np.log2(bad[1] / bad[2]) < order + 0.3, (mode, bad)
        assert bad[2] > 100 * good[2], mode


def test_level_factors_reduce_to_uniform_coarsening():
    """One factor for every level and the list of equal factors give the
    same operators (the recursion is the paper's for uniform m)."""
    a = co.phi_levels(3, "erk", 0.85, 4, 4)
    b = co.phi_levels(3, "erk", 0.85, [4, 4, 4], 4)
    assert a == b
    assert co.level_shifts(1.3, 8, 3) == co.level_shifts(1.3, [8, 8], 3)


# --------------------------------------------------------------------------
# Operators: Fourier symbols, equivalences, conservation, solve convention
# --------------------------------------------------------------------------


@pytest.mark.parametrize("p,kind,q,c", [(1, "erk", 1, 0.85), (3, "erk", 3, 1.2), (5, "erk", 5, 1.1),
                                        (1, "sdirk", 1, 3.0), (3, "sdirk", 3, 5.0), (5, "sdirk", 5, 6.0),
                                        (5, "sdirk", 3, 4.0), (2, "erk", 2, 0.4), (4, "sdirk", 4, 2.0)])
def test_fine_operator_matches_fourier_symbol(p, kind, q, c):
    """Phi is circulant with symbol R_q(-c lambda_L(omega)): applying it
    equals multiplying the DFT by the closed-form symbol."""
    nx = 64
    u = np.random.default_rng(3).standard_normal(nx)
    Phi = ops.FineOperator(p, kind, q, c)
    omega = 2 * np.pi * np.fft.fftfreq(nx)
    want = np.real(np.fft.ifft(Phi.symbol(omega) * np.fft.fft(u)))
    assert np.max(np.abs(Phi.apply(u) - want)) < 1e-12 * max(1.0, np.max(np.abs(want)))


def test_coarse_operator_matches_symbol():
    nx = 64
    u = np.random.default_rng(4).standard_normal(nx)
    for p, kind, c, m, lev, L in [(1, "erk", 0.85, 4, 1, 2), (3, "erk", 0.85, 8, 3, 4), (5, "sdirk", 4.0, 16, 2, 3)]:
        Psi = ops.coarse_operator(p, kind, p, c, m, lev, L)
        omega = 2 * np.pi * np.fft.fftfreq(nx)
        want = np.real(np.fft.ifft(Psi.symbol(omega) * np.fft.fft(u)))
        assert np.max(np.abs(Psi.apply(u) - want)) < 1e-12


def test_circulant_solve_convention_against_dense():
    rng = np.random.default_rng(5)
    taps = {-2: 0.3, -1: -0.7, 0: 0.1, 1: 0.25}
    n = 17
    b = rng.standard_normal((3, n))
    x = ops.circulant_solve(taps, b, diag=2.0)
    A = ops.dense_circulant(taps, n, diag=2.0)
    for i in range(3):
        assert np.max(np.abs(A @ x[i] - b[i])) < 1e-13
    assert np.max(np.abs(ops.apply_stencil(x, taps) + 2.0 * x - b)) < 1e-13


def test_erk1_u1_equals_first_order_sl():
    """ERK1+U1 and S_1^{(dt)} coincide for c < 1 (footnote in Sec. 1, Sec. 6.1)."""
    u = np.random.default_rng(6).standard_normal(50)
    for c in [0.1, 0.5, 0.85, 0.999]:
        a = ops.FineOperator(1, "erk", 1, c).apply(u)
        b = ops.SLOperator(1, c).apply(u)
        assert np.max(np.abs(a - b)) < 1e-14


def test_operators_conserve_mass():
    u = np.random.default_rng(7).standard_normal(96)
    for p in (1, 3, 5):
        for kind, c in (("erk", 0.8), ("sdirk", 4.0)):
            assert abs(np.sum(ops.FineOperator(p, kind, p, c).apply(u)) - np.sum(u)) < 1e-11
        assert abs(np.sum(ops.coarse_operator(p, "erk", p, 0.8, 8, 2, 3).apply(u)) - np.sum(u)) < 1e-11


# --------------------------------------------------------------------------
# LFA values printed in the text
# --------------------------------------------------------------------------


def test_lfa_erk4_u4_discontinuity(golden):
    cmax = co.cfl_limit(4)
    for name, kind, p, m, nu, frac, value, tol in golden("lfa_values.txt"):
        got = lfa.two_level_factor(int(p), kind, float(frac) * cmax, int(m), nu=int(nu), omit=10)
        assert abs(got - float(value)) < float(tol), (name, got)


def test_lfa_fcf_third_order_bounded():
    """Sec. 6.3.4: where F-relaxation exceeds one, FCF stays below 0.6
    (ERK3+U3 over c/c_max <= 0.9 and SDIRK3+U3 over c <= 8, m = 2..16)."""
    cmax = co.cfl_limit(3)
    worst_f = 0.0
    for m in (2, 4, 8, 16):
        for f in np.linspace(0.02, 0.9, 23):
            worst_f = max(worst_f, lfa.two_level_factor(3, "erk", f * cmax, m, nu=0, omit=10))
            assert lfa.two_level_factor(3, "erk", f * cmax, m, nu=1, omit=10) < 0.6
        for c in np.linspace(0.2, 8.0, 14):
            assert lfa.two_level_factor(3, "sdirk", c, m, nu=1, omit=10) < 0.6
    assert worst_f > 1.0
