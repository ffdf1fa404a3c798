// Host-side discretisation data for the MGRIT kernels (FP64 setup, Sec. 3-6).
#pragma once
#include <complex>
#include <string>
#include <vector>

namespace mg {

// A periodic stencil: (A u)_i = sum_{t=lo}^{hi} a[t-lo] u_{i+t}.
struct Stencil {
  int lo = 0, hi = 0;
  std::vector<double> a;
  int width() const { return hi - lo + 1; }
  double at(int t) const { return (t < lo || t > hi) ? 0.0 : a[t - lo]; }
};

Stencil stencil_mul(const Stencil& x, const Stencil& y);  // composition x*y
Stencil stencil_add(const Stencil& x, const Stencil& y, double sy);
Stencil stencil_identity();

// Sec. 4.1: upwind taps of L_p from the moment conditions
// sum_j l_j j^k = delta_{k,1}, k = 0..p, on j = -l(p)..r(p).
Stencil upwind_taps(int p);
void upwind_bias(int p, int* l, int* r);
double e_fd(int p);  // Lemma 4.1

// Sec. 4.2: RK data.
std::vector<double> erk_poly(int q);  // beta_0..beta_s of R_q
struct SdirkTableau {
  int s = 0;
  double A[5][5] = {};
  double b[5] = {};
};
bool sdirk_tableau(int q, SdirkTableau* t);  // q = 1..4
double sdirk5_gamma();
// SDIRK5 through R = prod(real factors of P)/(1 - g z)^5: each factor is a
// polynomial in z of degree 1 or 2 (coefficients c0 + c1 z + c2 z^2).
std::vector<std::vector<double>> sdirk5_factors(double* gamma);
double e_rk(int kind, int q);

// Sec. 3: semi-Lagrangian shift and weights for odd p.
void sl_shift(double s, long long* k, double* eps);
// SL interpolation nodes x_{i-k} + j h, j = sl_lo(p, eps) .. sl_lo + p: odd
// p the (p+1)/2 points west and (p-1)/2 east of x_{i-k}; even p the p + 1
// points centred on the mesh point nearer to the departure point (x_{i-k}
// for eps < 1/2, x_{i-k-1} otherwise, Sec. 3)
int sl_lo(int p, double eps);
std::vector<double> sl_weights(int p, double eps);  // index j - sl_lo(p, eps)
double f_poly(int p, double eps);                    // Eq. fpoly_def on the same node set
Stencil central_diff(int order);                     // D^{(order)}_2, even order
// D^{(order)}_s of the corrected coarse operator (Eq. Dp+1_def): even order
// (odd p, Sec. 6.3) the centred second-order stencil, odd order (even p,
// Sec. 6.4) the first-order stencil with a one-point bias to the left
Stencil diff_stencil(int order);

// ERK one-step stencil R(-c L) and its m-th power (Eq. MOL_M_def).
Stencil erk_step_stencil(int p, int q, double c);
Stencil stencil_power(const Stencil& s, int m);

// Periodic banded solve A y = b factored as
//   A = kappa E^{n_in - l} C(E^{-1}) F(E)
// (Wiener-Hopf split of the symbol's roots inside / outside the unit circle).
struct BandFactor {
  int hc = 0, ha = 0;         // causal / anticausal recurrence orders (<= 3)
  double cc[3] = {0, 0, 0};   // w_i = b_i - sum cc[q-1] w_{i-q}
  double ca[3] = {0, 0, 0};   // v_i = w_i - sum ca[q-1] v_{i+q}
  double inv_kappa = 1.0;
  int shift = 0;              // y_i = v_{i + shift} / kappa
  double max_residual = 0.0;  // check of the refactored taps
};
// taps of A (must have lo <= 0 <= hi); returns false when a root lies on the
// unit circle (singular for some n) or the factorisation is not accurate.
bool band_factor(const Stencil& A, BandFactor* f, std::string* why);

// Chunked-scan tables for one recurrence direction of order h over chunks
// of length P, T chunks per vector (T a power of two).
struct ScanTables {
  int h = 0;
  int rounds = 0;                 // Hillis-Steele rounds actually needed
  std::vector<double> G;          // P * 3: impulse responses G[j*3 + q]
  std::vector<double> Mpow;       // rounds * 9: M^{2^k}, row-major 3x3
  double Cl[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};  // closure (I - M^T)^{-1}
};
ScanTables scan_tables(const double* coef, int h, int P, int T);

// Tables of the cluster-distributed chunk scan: T chunks of P points per CTA,
// C CTAs per vector (see the SolveDir description in kernels.h).
struct DistScanTables {
  int h = 0;
  int rounds = 0;            // intra-CTA (non-circular) Hillis-Steele rounds
  std::vector<double> G;     // P * 3 impulse responses
  std::vector<double> Mpow;  // rounds * 9: M^{2^r}
  std::vector<double> Mt;    // tcut * 9: M^t, t = 0..tcut-1
  int tcut = 0;
  int jterms = 0;            // cluster-level terms
  std::vector<double> McPow; // jterms * 9: (M^T)^j
  double Clc[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  int closure = 0;
  std::vector<double> Mlane;   // 32 * 9: M^d, d = 1..32
  std::vector<double> M32pow;  // wterms * 9: (M^32)^j
  int wterms = 0;
  int dcut = 0;                // largest d <= 32 with M^d not negligible
};
// Terms whose transfer-matrix norm falls below `tol` are dropped (1e-18 for
// FP64 kernels, 1e-10 for FP32 ones).
DistScanTables dist_scan_tables(const double* coef, int h, int P, int T, int C, double tol = 1e-18);

}  // namespace mg
