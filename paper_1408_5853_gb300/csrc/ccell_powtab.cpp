// Host construction of the power-law tables used for lambda(T) = lam0 (T/t_ref)^b.
//
// FP64 pow costs about a hundred FP64-pipe operations on GB300, which has
// little FP64 throughput, and the time step evaluates three conductivities per
// node.  Write x = m 2^e with m in [1, 2): x^b = 2^(e b) m^b.  The factor
// 2^(e b), times the material constant, comes from a table indexed by e; m^b
// comes from a degree-4 polynomial on one of 256 equal mantissa intervals,
// evaluated in the offset u = m - c_q from the interval centre c_q.  Each
// polynomial interpolates m^b at the 5 Chebyshev points of its interval
// (computed in long double); on an interval of half-width 2^-9 the
// interpolation error is at most |d^5 m^b / dm^5| h^5 / (2^4 5!), below 1e-16
// relative for exponents b in [0, 3], so the table value is as accurate as a
// correctly rounded pow up to the rounding of the evaluation itself.  Every table is checked against powl
// at 16 points per interval; a table that misses 4e-16 relative is rejected and
// the kernel falls back to pow.
#include <cmath>

#include "ccell_internal.h"

namespace ccell {

namespace {

// Monomial coefficients a[0..n-1] of the polynomial through (s[k], f[k]).
void interpolate(const long double* s, const long double* f, int n, long double* a) {
  long double V[kPowDeg + 1][kPowDeg + 2];
  for (int r = 0; r < n; ++r) {
    long double p = 1.0L;
    for (int c = 0; c < n; ++c, p *= s[r]) V[r][c] = p;
    V[r][n] = f[r];
  }
  for (int c = 0; c < n; ++c) {  // Gaussian elimination, partial pivoting
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(V[r][c]) > fabsl(V[piv][c])) piv = r;
    for (int k = 0; k <= n; ++k) {
      long double t = V[c][k];
      V[c][k] = V[piv][k];
      V[piv][k] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      const long double f2 = V[r][c] / V[c][c];
      for (int k = c; k <= n; ++k) V[r][k] -= f2 * V[c][k];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    long double acc = V[r][n];
    for (int k = r + 1; k < n; ++k) acc -= V[r][k] * a[k];
    a[r] = acc / V[r][r];
  }
}

}  // namespace

bool build_pow_table(double b, double face_scale, double node_scale, double* tab) {
  const int D = kPowDeg + 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int e = 0; e < kPowNE; ++e) {
    const long double two_eb = powl(2.0L, (long double)(e + kPowEmin) * (long double)b);
    tab[e] = (double)(face_scale * two_eb);
    tab[kPowNE + e] = (double)(node_scale * two_eb);
  }
  double* P = tab + 2 * kPowNE;
  bool ok = true;
  for (int q = 0; q < kPowQ; ++q) {
    const long double c = 1.0L + ((long double)q + 0.5L) / kPowQ;
    const long double h = 0.5L / kPowQ;
    long double s[kPowDeg + 1], f[kPowDeg + 1], a[kPowDeg + 1];
    for (int k = 0; k < D; ++k) {
      s[k] = cosl((2.0L * k + 1.0L) * pi / (2.0L * D));
      f[k] = powl(c + h * s[k], (long double)b);
    }
    interpolate(s, f, D, a);  // polynomial in s = u / h
    long double hn = 1.0L;
    for (int k = 0; k < D; ++k, hn *= h) P[q * D + k] = (double)(a[k] / hn);
    // check the double-precision polynomial as the device evaluates it (FMA Horner)
    const double cd = (double)c;
    for (int t = 0; t <= 16; ++t) {
      const double u = (double)(h * (-1.0L + t / 8.0L));
      double r = P[q * D + kPowDeg];
      for (int k = kPowDeg - 1; k >= 0; --k) r = std::fma(r, u, P[q * D + k]);
      const long double ref = powl((long double)cd + (long double)u, (long double)b);
      if (fabsl(((long double)r - ref) / ref) > 4e-16L) ok = false;
    }
  }
  return ok;
}

}  // namespace ccell
