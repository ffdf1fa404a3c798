"""Time-stepping operators Phi and Psi (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy; every
operator acts on the last axis of an array (one spatial vector per row), with
periodic wrap.  Circulant solves use scipy.linalg.solve_circulant (a library
routine for the plain definition x = C^{-1} b); tests pin its column
convention against a dense LAPACK solve.

Function / class         paper passage                                   parity pin
-----------------------  ----------------------------------------------  -----------------------------
apply_stencil            circulant (A u)_i = sum_j a_j u_{i+j}           dense matrix product
circulant_solve          x = A^{-1} b for circulant A                    dense LAPACK solve
FineOperator.apply       Eq. (MOL_M_def): one RK step of du/dt =         Fourier symbol R_q(-c lambda_L);
                         -alpha L_p/h u; ERK as the polynomial R_q(-cL)   ERK stage form == polynomial;
                         (a sequence of L mat-vecs), SDIRK through its    Lemma 4.2 truncation order;
                         stages with solves by (I + a c L_p) (footnote    mass conservation
                         on the practical form of a step)
SLOperator.apply         Sec. 3: S_p^{(Delta)} interpolation at the       exact shift for integer offset;
                         departure point                                 Lemma 3.1 order
CoarseOperator.apply     Eq. (MOL-SL-corrected[-multilevel])                Lemma 6.1 O(h^{p+2}) match with
                         (I - phi D)^{-1} S_p^{(m^l dt)}; the correction  Phi^m; LFA values (Sec. 6.3.4, 6.4);
                         solve exact or by GMRES (Sec. 6.1, 6.3)           GMRES pins in oracle/gmres.py
direct_operator          Sec. 1 footnote, Sec. 2.2, Sec. 5: direct        symbols == application; LFA with
                         coarse operators -- S_p^{(m^l dt)} ("sl") and    rediscretisation >= the bound of
                         the rediscretised R_q(-m^l c L_p) ("redisc")     Theorem thm:MOL-rho-lwr-bnd
"""
import numpy as np
import scipy.linalg

from . import coefficients as co
from . import gmres as _gm


def apply_stencil(u, taps):
    """(A u)_i = sum_j a_j u_{(i+j) mod n} along the last axis."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    for j, a in taps.items():
        out += float(a) * np.roll(u, -j, axis=-1)
    return out


def circulant_first_column(taps, n, diag=0.0):
    """First column of the circulant matrix A with A_{i,(i+j) mod n} = a_j
    (plus ``diag`` on the diagonal).  Column 0 holds A_{i,0}, i.e. the tap
    a_j lands in row (-j) mod n."""
    col = np.zeros(n, dtype=np.float64)
    col[0] += diag
    for j, a in taps.items():
        col[(-j) % n] += float(a)
    return col


def dense_circulant(taps, n, diag=0.0):
    """Dense n x n matrix with A[i, (i+j) mod n] = a_j (+ diag on i = i)."""
    A = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        A[i, i] += diag
        for j, a in taps.items():
            A[i, (i + j) % n] += float(a)
    return A


def circulant_solve(taps, b, diag=0.0):
    """Solve A x = b (last axis) for the circulant A of ``taps`` + diag I."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[-1]
    col = circulant_first_column(taps, n, diag)
    x = scipy.linalg.solve_circulant(col, b, baxis=b.ndim - 1, outaxis=b.ndim - 1)
    return np.real(x)


def scaled_taps(taps, s):
    return {j: float(a) * s for j, a in taps.items()}


class FineOperator:
    """Phi = M^{(dt)}_{p,q} = R_q(-c L_p)  (Eq. MOL_M_def), c = alpha dt / h.

    kind = "erk": Phi u = sum_j beta_j (-c)^j L_p^j u  (R_q is a polynomial).
    kind = "sdirk", q <= 4: stage equations of the tableau,
        (I + a_ii c L_p) Y_i = u - c sum_{j<i} a_ij L_p Y_j,
        Phi u = u - c sum_i b_i L_p Y_i.
    kind = "sdirk", q = 5: R = P(z)/(1 - gamma z)^5 applied factor by factor,
        the real linear/quadratic factors of P interleaved with the solves by
        (I + gamma c L_p) (the paper's SDIRK5 tableau is not printed).
    """

    def __init__(self, p, kind, q, c):
        self.p, self.kind, self.q, self.c = p, kind, q, float(c)
        self.L = co.upwind_taps(p)
        if kind == "erk":
            self.beta = [float(b) for b in co.rk_stability_poly(q)]
        elif kind == "sdirk":
            if q <= 4:
                self.A, self.b = co.sdirk_tableau(q)
            else:
                self.gamma = co.sdirk5_gamma()
                P = co.sdirk5_numerator(self.gamma)
                roots = np.roots(P[::-1])
                self.factors = []  # polynomials in z, coefficient lists
                used = [False] * len(roots)
                for i, r in enumerate(roots):
                    if used[i]:
                        continue
                    used[i] = True
                    if abs(r.imag) < 1e-12:
                        self.factors.append([1.0, -1.0 / r.real])
                    else:
                        for j in range(i + 1, len(roots)):
                            if not used[j] and abs(roots[j] - np.conj(r)) < 1e-9:
                                used[j] = True
                                break
                        inv = 1.0 / r
                        self.factors.append([1.0, -2.0 * inv.real, abs(inv) ** 2])
        else:
            raise ValueError(kind)

    def Lu(self, u):
        return apply_stencil(u, self.L)

    def apply(self, u):
        u = np.asarray(u, dtype=np.float64)
        c = self.c
        if self.kind == "erk":
            acc = self.beta[0] * u
            v = u
            for j in range(1, len(self.beta)):
                v = self.Lu(v)
                acc = acc + self.beta[j] * (-c) ** j * v
            return acc
        if self.q <= 4:
            s = len(self.b)
            LY = []
            for i in range(s):
                rhs = u.copy()
                for j in range(i):
                    rhs = rhs - c * self.A[i][j] * LY[j]
                Y = circulant_solve(scaled_taps(self.L, self.A[i][i] * c), rhs, diag=1.0)
                LY.append(self.Lu(Y))
            out = u.copy()
            for i in range(s):
                out = out - c * self.b[i] * LY[i]
            return out
        # SDIRK5: z = -c L
        v = u
        solves = 5
        for f in self.factors:
            w = f[0] * v
            zv = v
            for k in range(1, len(f)):
                zv = -c * self.Lu(zv)
                w = w + f[k] * zv
            v = circulant_solve(scaled_taps(self.L, self.gamma * c), w, diag=1.0)
            solves -= 1
        for _ in range(solves):
            v = circulant_solve(scaled_taps(self.L, self.gamma * c), v, diag=1.0)
        return v

    def symbol(self, omega):
        """Fourier symbol R_q(-c lambda_L(omega)) (closed form)."""
        return co.rk_stability_value(self.kind, self.q, -self.c * co.upwind_symbol(self.p, omega))


class SLOperator:
    """S_p^{(Delta)}: (S u)_i = sum_j w_j(eps) u_{i-k+j}, departure offset
    s = alpha Delta / h = k + eps (Sec. 3)."""

    def __init__(self, p, s):
        self.p = p
        self.k, self.eps = co.sl_shift(s)
        self.w = co.sl_weights(p, self.eps)

    def taps(self):
        return {j - self.k: w for j, w in self.w.items()}

    def apply(self, u):
        return apply_stencil(u, self.taps())

    def symbol(self, omega):
        return sum(w * np.exp(1j * (j - self.k) * omega) for j, w in self.w.items())


class CoarseOperator:
    """Phi^{(m^l dt)} = (I - sum_t phi_t D^{(o_t)})^{-1} S_p^{(m^l dt)}.

    With one term (phi, p+1) this is Eq. (MOL-SL-corrected) / (MOL-SL-corrected-multilevel); the
    two-term form is the q != p reading (see coefficients.phi_levels_general).
    ``terms`` is a list of (phi, derivative order).  ``gmres`` = (rtol, maxit)
    replaces the exact correction solve by GMRES from a zero guess, one
    system per row (Sec. 6.1, Sec. 6.3; oracle/gmres.py); the iteration count
    of every solve is appended to ``gmres_its``.
    """

    def __init__(self, p, s, terms, gmres=None):
        self.p = p
        self.sl = SLOperator(p, s)
        self.terms = list(terms)
        corr = {}
        for phi, order in self.terms:
            for j, d in co.diff_taps(order).items():
                corr[j] = corr.get(j, 0.0) - phi * float(d)
        self.corr = corr  # taps of -(sum phi D), the matrix is I + corr
        self.gmres = gmres
        self.gmres_its = []

    def correction_matvec(self, v):
        """(I - sum phi D) v."""
        return v + apply_stencil(v, self.corr)

    def apply(self, u):
        b = self.sl.apply(u)
        if self.gmres is None:
            return circulant_solve(self.corr, b, diag=1.0)
        rtol, maxit = self.gmres
        X, its = _gm.gmres_rows(self.correction_matvec, b.reshape(-1, b.shape[-1]), rtol, maxit)
        self.gmres_its.extend(its)
        return X.reshape(b.shape)

    def symbol(self, omega):
        den = 1.0 + sum(a * np.exp(1j * j * omega) for j, a in self.corr.items())
        return self.sl.symbol(omega) / den


def coarse_operator(p, kind, q, c, m, level, levels, gmres=None):
    """Level-``level`` (>= 1) corrected SL operator of a ``levels``-level
    hierarchy with uniform coarsening m (Eq. MOL-SL-corrected-multilevel and the Sec. 6.2 phi recursion);
    ``gmres`` = (rtol, maxit) solves its correction systems by GMRES."""
    s = c * co.level_step(m, level)
    if q == p:
        phi = co.phi_levels(p, kind, c, m, levels)[level - 1]
        return CoarseOperator(p, s, [(phi, p + 1)], gmres)
    fp, fq = co.phi_levels_general(p, kind, q, c, m, levels)[level - 1]
    return CoarseOperator(p, s, [(fp, p + 1), (fq, q + 1)], gmres)


def direct_operator(p, kind, q, c, m, level, coarse_op):
    """Coarse-grid operator of level ``level`` (>= 1) for the coarse-operator
    choices compared in the paper:

    ``sl_corrected``  the modified operator (I - phi D)^{-1} S_p^{(m^l dt)}
                      (Eq. MOL-SL-corrected-multilevel), ``levels`` unused;
    ``sl``            the direct semi-Lagrangian operator S_p^{(m^l dt)}
                      (Sec. 3, a direct discretization in the sense of the
                      footnote to Sec. 1);
    ``redisc``        rediscretisation: the fine method with the coarse step,
                      R_q(-m^l c L_p) (Sec. 2.2 and the Sec. 1 footnote;
                      analysed in Sec. 5).
    """
    s = c * co.level_step(m, level)
    if coarse_op == "sl":
        return SLOperator(p, s)
    if coarse_op == "redisc":
        return FineOperator(p, kind, q, s)
    raise ValueError(coarse_op)


class PowerOperator:
    """Phi^m as an operator (the ideal coarse-grid operator, Sec. 2.2)."""

    def __init__(self, op, m):
        self.op, self.m = op, m

    def apply(self, u):
        for _ in range(self.m):
            u = self.op.apply(u)
        return u
