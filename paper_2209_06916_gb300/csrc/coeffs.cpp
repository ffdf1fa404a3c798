// Host-side discretisation data for the MGRIT kernels.
//
// Everything here is derived from the paper's definitions in FP64 (with long
// double where a product of many terms is accumulated):
//   upwind taps        Sec. 4.1 (moment conditions of the degree-p derivative)
//   e_FD               Lemma 4.1, Eq. e_FD_def
//   RK data            Sec. 4.2, Eq. RK_stab_def / e_RK_def
//   SL shift, weights  Sec. 3 (departure point, Lagrange interpolation)
//   f_{p+1}            Lemma 3.1, Eq. fpoly_def
//   D^{(p+1)}_2        Eq. Dp+1_def with the symmetric s = 2 choice of Sec. 6.3
//   banded solves      the corrections (I - phi D)^{-1} of Eq. MOL-SL-corrected
//                      and the SDIRK stage matrices (I + a c L_p) (Sec. 4.3)
#include "coeffs.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace mg {

typedef long double ld;

Stencil stencil_identity() {
  Stencil s;
  s.lo = s.hi = 0;
  s.a = {1.0};
  return s;
}

Stencil stencil_mul(const Stencil& x, const Stencil& y) {
  Stencil z;
  z.lo = x.lo + y.lo;
  z.hi = x.hi + y.hi;
  std::vector<ld> acc(z.width(), 0.0L);
  for (int i = 0; i < x.width(); ++i)
    for (int j = 0; j < y.width(); ++j) acc[i + j] += (ld)x.a[i] * (ld)y.a[j];
  z.a.resize(acc.size());
  for (size_t i = 0; i < acc.size(); ++i) z.a[i] = (double)acc[i];
  return z;
}

Stencil stencil_add(const Stencil& x, const Stencil& y, double sy) {
  Stencil z;
  z.lo = std::min(x.lo, y.lo);
  z.hi = std::max(x.hi, y.hi);
  z.a.assign(z.width(), 0.0);
  for (int t = z.lo; t <= z.hi; ++t) z.a[t - z.lo] = x.at(t) + sy * y.at(t);
  return z;
}

void upwind_bias(int p, int* l, int* r) {
  if (p % 2 == 1) {
    *l = (p + 1) / 2;
    *r = *l - 1;
  } else {
    *l = p / 2 + 1;
    *r = *l - 2;
  }
}

// Solve the (p+1)x(p+1) moment system V l = e_1 with V[k][j] = node_j^k by
// Gaussian elimination with partial pivoting in long double.
Stencil upwind_taps(int p) {
  int l, r;
  upwind_bias(p, &l, &r);
  int n = p + 1;
  std::vector<std::vector<ld>> M(n, std::vector<ld>(n + 1, 0.0L));
  for (int k = 0; k < n; ++k) {
    for (int c = 0; c < n; ++c) {
      ld node = (ld)(c - l), v = 1.0L;
      for (int e = 0; e < k; ++e) v *= node;
      M[k][c] = v;
    }
    M[k][n] = (k == 1) ? 1.0L : 0.0L;
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int rr = c + 1; rr < n; ++rr)
      if (fabsl(M[rr][c]) > fabsl(M[piv][c])) piv = rr;
    std::swap(M[c], M[piv]);
    for (int rr = 0; rr < n; ++rr) {
      if (rr == c) continue;
      ld f = M[rr][c] / M[c][c];
      for (int cc = c; cc <= n; ++cc) M[rr][cc] -= f * M[c][cc];
    }
  }
  Stencil s;
  s.lo = -l;
  s.hi = r;
  s.a.resize(n);
  for (int c = 0; c < n; ++c) s.a[c] = (double)(M[c][n] / M[c][c]);
  return s;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

double e_fd(int p) {
  int l, r;
  upwind_bias(p, &l, &r);
  return ((r % 2) ? -1.0 : 1.0) * factorial(l) * factorial(r) / factorial(p + 1);
}

std::vector<double> erk_poly(int q) {
  std::vector<double> b;
  for (int j = 0; j <= q; ++j) b.push_back(1.0 / factorial(j));
  if (q == 5) b.push_back(1.0 / 1280.0);  // Table 1: e_RK(ERK5) = beta_6 - 1/720
  return b;
}

static double newton_root(double (*f)(double), double (*df)(double), double x0) {
  double x = x0;
  for (int it = 0; it < 100; ++it) {
    double dx = f(x) / df(x);
    x -= dx;
    if (std::fabs(dx) < 1e-17) break;
  }
  return x;
}

static double sd3_f(double g) { return g * g * g - 3 * g * g + 1.5 * g - 1.0 / 6.0; }
static double sd3_df(double g) { return 3 * g * g - 6 * g + 1.5; }

bool sdirk_tableau(int q, SdirkTableau* t) {
  *t = SdirkTableau();
  if (q == 1) {
    t->s = 1;
    t->A[0][0] = 1.0;
    t->b[0] = 1.0;
    return true;
  }
  if (q == 2) {
    double g = 1.0 - std::sqrt(0.5);
    t->s = 2;
    t->A[0][0] = g;
    t->A[1][0] = 1.0 - g;
    t->A[1][1] = g;
    t->b[0] = 1.0 - g;
    t->b[1] = g;
    return true;
  }
  if (q == 3) {
    // L-stable 3-stage third-order SDIRK: gamma solves g^3-3g^2+3g/2-1/6 = 0.
    double g = newton_root(sd3_f, sd3_df, 0.4358);
    double b1 = -(6 * g * g - 16 * g + 1) / 4.0, b2 = (6 * g * g - 20 * g + 5) / 4.0;
    t->s = 3;
    t->A[0][0] = g;
    t->A[1][0] = (1 - g) / 2.0;
    t->A[1][1] = g;
    t->A[2][0] = b1;
    t->A[2][1] = b2;
    t->A[2][2] = g;
    t->b[0] = b1;
    t->b[1] = b2;
    t->b[2] = g;
    return true;
  }
  if (q == 4) {
    // L-stable 5-stage fourth-order SDIRK with gamma = 1/4 (stiffly accurate).
    const double A[5][5] = {{0.25, 0, 0, 0, 0},
                            {0.5, 0.25, 0, 0, 0},
                            {17.0 / 50, -1.0 / 25, 0.25, 0, 0},
                            {371.0 / 1360, -137.0 / 2720, 15.0 / 544, 0.25, 0},
                            {25.0 / 24, -49.0 / 48, 125.0 / 16, -85.0 / 12, 0.25}};
    t->s = 5;
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) t->A[i][j] = A[i][j];
    for (int j = 0; j < 5; ++j) t->b[j] = A[4][j];
    return true;
  }
  return false;
}

// z^k coefficient of (1 - g z)^5 e^z.
static double sd5_coef(double g, int k) {
  double s = 0.0;
  for (int j = 0; j <= std::min(k, 5); ++j) {
    double binom = factorial(5) / (factorial(j) * factorial(5 - j));
    s += binom * std::pow(-g, j) / factorial(k - j);
  }
  return s;
}
static double sd5_f(double g) { return sd5_coef(g, 5); }
static double sd5_df(double g) { return (sd5_coef(g + 1e-7, 5) - sd5_coef(g - 1e-7, 5)) / 2e-7; }

double sdirk5_gamma() { return newton_root(sd5_f, sd5_df, 0.278); }

// Roots of a real polynomial sum c[k] z^k (degree d <= 8) by Durand-Kerner
// iteration in complex long double, then Newton polishing.
static std::vector<std::complex<ld>> poly_roots(const std::vector<double>& c) {
  int d = (int)c.size() - 1;
  std::vector<std::complex<ld>> z(d);
  std::vector<ld> a(c.begin(), c.end());
  ld lead = a[d];
  std::complex<ld> seed(0.4L, 0.9L);
  // scale the initial guesses to the root magnitude bound
  ld bound = 0.0L;
  for (int k = 0; k < d; ++k) bound = std::max(bound, fabsl(a[k] / lead));
  bound = 1.0L + bound;
  for (int k = 0; k < d; ++k) z[k] = std::pow(seed, (ld)k) * (bound * 0.5L);
  auto eval = [&](std::complex<ld> x) {
    std::complex<ld> v = a[d];
    for (int k = d - 1; k >= 0; --k) v = v * x + a[k];
    return v;
  };
  for (int it = 0; it < 2000; ++it) {
    ld delta = 0.0L;
    for (int k = 0; k < d; ++k) {
      std::complex<ld> den = lead;
      for (int j = 0; j < d; ++j)
        if (j != k) den *= (z[k] - z[j]);
      std::complex<ld> step = eval(z[k]) / den;
      z[k] -= step;
      delta = std::max(delta, std::abs(step) / std::max((ld)1.0L, std::abs(z[k])));
    }
    if (delta < 1e-30L) break;
  }
  for (int k = 0; k < d; ++k) {  // Newton polish
    for (int it = 0; it < 5; ++it) {
      std::complex<ld> v = a[d], dv = 0.0L;
      for (int j = d - 1; j >= 0; --j) {
        dv = dv * z[k] + v;
        v = v * z[k] + a[j];
      }
      if (std::abs(dv) == 0.0L) break;
      z[k] -= v / dv;
    }
  }
  return z;
}

std::vector<std::vector<double>> sdirk5_factors(double* gamma) {
  double g = sdirk5_gamma();
  if (gamma) *gamma = g;
  std::vector<double> P(5);
  for (int k = 0; k < 5; ++k) P[k] = sd5_coef(g, k);
  auto roots = poly_roots(P);
  std::vector<std::vector<double>> out;
  std::vector<bool> used(roots.size(), false);
  for (size_t i = 0; i < roots.size(); ++i) {
    if (used[i]) continue;
    used[i] = true;
    std::complex<ld> r = roots[i];
    if (fabsl(r.imag()) < 1e-12L * std::abs(r)) {
      out.push_back({1.0, (double)(-1.0L / r.real())});
    } else {
      for (size_t j = i + 1; j < roots.size(); ++j)
        if (!used[j] && std::abs(roots[j] - std::conj(r)) < 1e-9L * std::abs(r)) {
          used[j] = true;
          break;
        }
      std::complex<ld> inv = 1.0L / r;
      out.push_back({1.0, (double)(-2.0L * inv.real()), (double)std::norm(inv)});
    }
  }
  return out;
}

double e_rk(int kind, int q) {
  if (kind == 0) {
    std::vector<double> b = erk_poly(q);
    double bq1 = (int)b.size() > q + 1 ? b[q + 1] : 0.0;
    return bq1 - 1.0 / factorial(q + 1);
  }
  if (q == 5) return -sd5_coef(sdirk5_gamma(), 6);
  SdirkTableau t;
  if (!sdirk_tableau(q, &t)) return 0.0;
  // beta_{q+1} = b^T A^q 1
  std::vector<double> v(t.s, 1.0);
  for (int pw = 0; pw < q; ++pw) {
    std::vector<double> w(t.s, 0.0);
    for (int i = 0; i < t.s; ++i)
      for (int j = 0; j < t.s; ++j) w[i] += t.A[i][j] * v[j];
    v = w;
  }
  double beta = 0.0;
  for (int i = 0; i < t.s; ++i) beta += t.b[i] * v[i];
  return beta - 1.0 / factorial(q + 1);
}

void sl_shift(double s, long long* k, double* eps) {
  double f = std::floor(s);
  double e = s - f;
  if (e >= 1.0) {
    f += 1.0;
    e -= 1.0;
  }
  *k = (long long)f;
  *eps = e;
}

int sl_lo(int p, double eps) {
  if (p % 2) return -(p + 1) / 2;
  return eps < 0.5 ? -p / 2 : -p / 2 - 1;
}

std::vector<double> sl_weights(int p, double eps) {
  int lo = sl_lo(p, eps), n = p + 1;
  std::vector<double> w(n);
  for (int a = 0; a < n; ++a) {
    ld v = 1.0L;
    for (int b = 0; b < n; ++b)
      if (b != a) v *= ((ld)(-eps) - (ld)(lo + b)) / (ld)(a - b);
    w[a] = (double)v;
  }
  return w;
}

double f_poly(int p, double eps) {
  int lo = sl_lo(p, eps), hi = lo + p;
  ld v = 1.0L;
  for (int j = lo; j <= hi; ++j) v *= ((ld)j + (ld)eps);
  return (double)(v / (ld)factorial(p + 1));
}

Stencil central_diff(int order) {
  // h^{order} d^{order}/dx^{order} by the centred difference delta^{order}:
  // taps (-1)^{n+j} C(2n, n+j), j = -n..n, order = 2n.
  int n = order / 2;
  Stencil s;
  s.lo = -n;
  s.hi = n;
  s.a.resize(2 * n + 1);
  for (int j = -n; j <= n; ++j) {
    double binom = factorial(2 * n) / (factorial(n + j) * factorial(n - j));
    s.a[j + n] = (((n + j) % 2) ? -1.0 : 1.0) * binom;
  }
  return s;
}

Stencil diff_stencil(int order) {
  if (order % 2 == 0) return central_diff(order);
  // h^{order} times the order-th derivative of the interpolant through the
  // order + 1 nodes -(order+1)/2 .. (order-1)/2: d_j = order! / prod (j - k)
  Stencil s;
  s.lo = -(order + 1) / 2;
  s.hi = (order - 1) / 2;
  s.a.resize(order + 1);
  for (int j = s.lo; j <= s.hi; ++j) {
    double den = 1.0;
    for (int k = s.lo; k <= s.hi; ++k)
      if (k != j) den *= (double)(j - k);
    s.a[j - s.lo] = factorial(order) / den;
  }
  return s;
}

Stencil erk_step_stencil(int p, int q, double c) {
  Stencil L = upwind_taps(p);
  Stencil Z = L;
  for (double& v : Z.a) v *= -c;  // z = -c L
  std::vector<double> beta = erk_poly(q);
  Stencil acc = stencil_identity();
  acc.a[0] = beta[0];
  Stencil pw = stencil_identity();
  for (size_t j = 1; j < beta.size(); ++j) {
    pw = stencil_mul(pw, Z);
    acc = stencil_add(acc, pw, beta[j]);
  }
  return acc;
}

Stencil stencil_power(const Stencil& s, int m) {
  Stencil r = stencil_identity();
  Stencil b = s;
  int e = m;
  while (e > 0) {
    if (e & 1) r = stencil_mul(r, b);
    e >>= 1;
    if (e) b = stencil_mul(b, b);
  }
  return r;
}

bool band_factor(const Stencil& A, BandFactor* f, std::string* why) {
  *f = BandFactor();
  // trim negligible outer taps
  double amax = 0.0;
  for (double v : A.a) amax = std::max(amax, std::fabs(v));
  int lo = A.lo, hi = A.hi;
  while (lo < 0 && std::fabs(A.at(lo)) <= 1e-15 * amax) ++lo;
  while (hi > 0 && std::fabs(A.at(hi)) <= 1e-15 * amax) --hi;
  int l = -lo, d = hi - lo;
  if (d == 0) {
    f->inv_kappa = 1.0 / A.at(0);
    return true;
  }
  std::vector<double> poly(d + 1);
  for (int k = 0; k <= d; ++k) poly[k] = A.at(k - l);  // z^l a(z) = sum poly[k] z^k
  auto roots = poly_roots(poly);
  std::vector<std::complex<ld>> in, out;
  for (auto& z : roots) {
    ld r = std::abs(z);
    if (fabsl(r - 1.0L) < 1e-9L) {
      if (why) *why = "banded matrix symbol has a root on the unit circle";
      return false;
    }
    (r < 1.0L ? in : out).push_back(z);
  }
  if (in.size() > 3 || out.size() > 3) {
    if (why) *why = "banded factorisation order above 3";
    return false;
  }
  // C(x) = prod_in (1 - zeta x),  F(y) = prod_out (1 - y / zeta)
  std::vector<std::complex<ld>> C(1, 1.0L), F(1, 1.0L);
  for (auto& z : in) {
    std::vector<std::complex<ld>> nc(C.size() + 1, 0.0L);
    for (size_t k = 0; k < C.size(); ++k) {
      nc[k] += C[k];
      nc[k + 1] -= z * C[k];
    }
    C = nc;
  }
  for (auto& z : out) {
    std::vector<std::complex<ld>> nf(F.size() + 1, 0.0L);
    for (size_t k = 0; k < F.size(); ++k) {
      nf[k] += F[k];
      nf[k + 1] -= F[k] / z;
    }
    F = nf;
  }
  std::complex<ld> kappa = (ld)A.at(hi);
  for (auto& z : out) kappa *= -z;
  f->hc = (int)in.size();
  f->ha = (int)out.size();
  for (int q = 1; q <= f->hc; ++q) f->cc[q - 1] = (double)C[q].real();
  for (int q = 1; q <= f->ha; ++q) f->ca[q - 1] = (double)F[q].real();
  f->inv_kappa = (double)(1.0L / kappa.real());
  f->shift = l - f->hc;
  // Check: kappa * E^{hc - l} C(E^{-1}) F(E) must reproduce the taps.
  Stencil Cs, Fs;
  Cs.lo = -f->hc;
  Cs.hi = 0;
  Cs.a.assign(f->hc + 1, 0.0);
  Cs.a[f->hc] = 1.0;
  for (int q = 1; q <= f->hc; ++q) Cs.a[f->hc - q] = f->cc[q - 1];
  Fs.lo = 0;
  Fs.hi = f->ha;
  Fs.a.assign(f->ha + 1, 0.0);
  Fs.a[0] = 1.0;
  for (int q = 1; q <= f->ha; ++q) Fs.a[q] = f->ca[q - 1];
  Stencil P = stencil_mul(Cs, Fs);
  double res = 0.0;
  for (int t = std::min(lo, P.lo + f->hc - l) - 1; t <= std::max(hi, P.hi + f->hc - l) + 1; ++t) {
    double want = A.at(t);
    double got = P.at(t - (f->hc - l)) / f->inv_kappa;
    res = std::max(res, std::fabs(got - want));
  }
  f->max_residual = res / amax;
  if (f->max_residual > 1e-12) {
    if (why) *why = "banded factorisation inaccurate";
    return false;
  }
  return true;
}

static void mat3_mul(const double* a, const double* b, double* c) {
  double t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ld s = 0.0L;
      for (int k = 0; k < 3; ++k) s += (ld)a[i * 3 + k] * (ld)b[k * 3 + j];
      t[i * 3 + j] = (double)s;
    }
  for (int i = 0; i < 9; ++i) c[i] = t[i];
}

static bool mat3_inv(const double* a, int h, double* out) {
  // Gauss-Jordan on the leading h x h block; the rest stays identity.
  ld M[3][6] = {};
  for (int i = 0; i < h; ++i) {
    for (int j = 0; j < h; ++j) M[i][j] = a[i * 3 + j];
    M[i][3 + i] = 1.0L;
  }
  for (int c = 0; c < h; ++c) {
    int piv = c;
    for (int r = c + 1; r < h; ++r)
      if (fabsl(M[r][c]) > fabsl(M[piv][c])) piv = r;
    if (fabsl(M[piv][c]) < 1e-300L) return false;
    for (int k = 0; k < 6; ++k) std::swap(M[c][k], M[piv][k]);
    for (int r = 0; r < h; ++r) {
      if (r == c) continue;
      ld fct = M[r][c] / M[c][c];
      for (int k = 0; k < 6; ++k) M[r][k] -= fct * M[c][k];
    }
  }
  for (int i = 0; i < 9; ++i) out[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < h; ++j) out[i * 3 + j] = (double)(M[i][3 + j] / M[i][i]);
  return true;
}

ScanTables scan_tables(const double* coef, int h, int P, int T) {
  // Recurrence x_j = b_j - sum_{q=1}^h coef[q-1] x_{j-q} along the chunk.
  // state_in[q] = x_{-1-q}; G[j][q] = d x_j / d state_in[q] (b = 0).
  ScanTables t;
  t.h = h;
  t.G.assign((size_t)P * 3, 0.0);
  if (h == 0) return t;
  for (int q = 0; q < h; ++q) {
    std::vector<ld> x(P + h, 0.0L);  // x[h + j] = x_j, x[h-1-q'] = state q'
    x[h - 1 - q] = 1.0L;
    for (int j = 0; j < P; ++j) {
      ld v = 0.0L;
      for (int r = 1; r <= h; ++r) v -= (ld)coef[r - 1] * x[h + j - r];
      x[h + j] = v;
      t.G[(size_t)j * 3 + q] = (double)v;
    }
  }
  // End state component a = x_{P-1-a}: M[a][q] = G[P-1-a][q].
  double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int a = 0; a < h; ++a)
    for (int q = 0; q < h; ++q) M[a * 3 + q] = t.G[(size_t)(P - 1 - a) * 3 + q];
  int full = 0;
  while ((1 << full) < T) ++full;
  double pw[9];
  for (int i = 0; i < 9; ++i) pw[i] = M[i];
  int rounds = 0;
  for (; rounds < full; ++rounds) {
    double nrm = 0.0;
    for (int i = 0; i < 9; ++i) nrm = std::max(nrm, std::fabs(pw[i]));
    if (nrm < 1e-18) break;  // contributions from 2^rounds chunks back vanish
    t.Mpow.insert(t.Mpow.end(), pw, pw + 9);
    mat3_mul(pw, pw, pw);
  }
  t.rounds = rounds;
  if (rounds == full) {
    // pw = M^{2^full} = M^T: periodic closure S = (I - M^T)^{-1} Q.
    double IM[9];
    for (int i = 0; i < 9; ++i) IM[i] = ((i % 4 == 0) ? 1.0 : 0.0) - pw[i];
    if (!mat3_inv(IM, h, t.Cl)) {
      for (int i = 0; i < 9; ++i) t.Cl[i] = (i % 4 == 0) ? 1.0 : 0.0;
    }
  }
  return t;
}

static double mat3_norm(const double* a) {
  double n = 0.0;
  for (int i = 0; i < 9; ++i) n = std::max(n, std::fabs(a[i]));
  return n;
}

DistScanTables dist_scan_tables(const double* coef, int h, int P, int T, int C, double tol) {
  DistScanTables d;
  d.h = h;
  ScanTables base = scan_tables(coef, h, P, 1);  // G only
  d.G = base.G;
  const double I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int a = 0; a < h; ++a)
    for (int q = 0; q < h; ++q) M[a * 3 + q] = d.G[(size_t)(P - 1 - a) * 3 + q];
  // intra-CTA rounds: 2^r < T and M^{2^r} not yet negligible
  double pw[9];
  for (int i = 0; i < 9; ++i) pw[i] = M[i];
  for (int r = 0; (1 << r) < T; ++r) {
    if (mat3_norm(pw) < tol) break;
    d.Mpow.insert(d.Mpow.end(), pw, pw + 9);
    ++d.rounds;
    mat3_mul(pw, pw, pw);
  }
  // per-chunk carry table M^t, t < T, until negligible
  double mt[9];
  for (int i = 0; i < 9; ++i) mt[i] = I3[i];
  for (int t = 0; t < T; ++t) {
    if (t > 0 && mat3_norm(mt) < tol) break;
    d.Mt.insert(d.Mt.end(), mt, mt + 9);
    ++d.tcut;
    mat3_mul(mt, M, mt);
  }
  // Mc = M^T (transfer across a whole CTA)
  double Mc[9];
  for (int i = 0; i < 9; ++i) Mc[i] = I3[i];
  for (int t = 0; t < T; ++t) mat3_mul(Mc, M, Mc);
  double mcj[9];
  for (int i = 0; i < 9; ++i) mcj[i] = I3[i];
  for (int j = 0; j < C; ++j) {
    if (j > 0 && mat3_norm(mcj) < tol) break;
    d.McPow.insert(d.McPow.end(), mcj, mcj + 9);
    ++d.jterms;
    mat3_mul(mcj, Mc, mcj);
  }
  // warp-level tables: M^d (d <= 32) and powers of M^32 for the warp totals
  {
    double md[9];
    for (int i = 0; i < 9; ++i) md[i] = M[i];
    for (int dd = 1; dd <= 32; ++dd) {
      d.Mlane.insert(d.Mlane.end(), md, md + 9);
      if (mat3_norm(md) >= tol) d.dcut = dd;
      mat3_mul(md, M, md);
    }
    double m32[9];
    for (int i = 0; i < 9; ++i) m32[i] = d.Mlane[31 * 9 + i];
    double pj[9];
    for (int i = 0; i < 9; ++i) pj[i] = I3[i];
    const int nw = (T + 31) / 32;
    for (int j = 0; j < std::min(nw, 8); ++j) {
      if (j > 0 && mat3_norm(pj) < tol) break;
      d.M32pow.insert(d.M32pow.end(), pj, pj + 9);
      ++d.wterms;
      mat3_mul(pj, m32, pj);
    }
  }
  if (d.jterms == C && mat3_norm(mcj) >= tol) {
    // the sum wraps the ring: closure (I - Mc^C)^{-1}; mcj = Mc^C here
    double IM[9];
    for (int i = 0; i < 9; ++i) IM[i] = I3[i] - mcj[i];
    if (mat3_inv(IM, h, d.Clc)) d.closure = 1;
  }
  return d;
}

}  // namespace mg
