// Gauss quadrature rules computed on the host for the device kernels.
//
// The nodes of an n-point Gauss rule for a weight w are the eigenvalues of the
// symmetric tridiagonal Jacobi matrix J (diagonal a_k, off-diagonal sqrt(b_k))
// of the monic three-term recurrence of the orthogonal polynomials of w.
// They are found here by bisection on Sturm sequence counts (each eigenvalue is
// bracketed to the last bit), and the weights by the Christoffel formula
// w_i = 1 / sum_{k<n} q_k(x_i)^2 with q_k the orthonormal polynomials.
#include "hfsem_internal.h"

#include <cmath>
#include <stdexcept>

namespace hf {

namespace {

// number of eigenvalues of the tridiagonal (d, off2 = off^2) below x
int sturm_count(int n, const double* d, const double* off2, double x) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    double den = (q == 0.0) ? 1e-300 : q;
    q = d[i] - x - off2[i - 1] / den;
    if (q < 0) ++cnt;
  }
  return cnt;
}

void gauss_from_recurrence(int n, const std::vector<double>& a,
                           const std::vector<double>& b, double mu0,
                           std::vector<double>& x, std::vector<double>& w) {
  // a[0..n-1]: diagonal; b[1..n-1]: squared off-diagonal (b[k] couples k-1,k)
  std::vector<double> off2(n > 1 ? n - 1 : 1, 0.0);
  for (int k = 1; k < n; ++k) off2[k - 1] = b[k];
  // Gershgorin bounds
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    if (i > 0) r += std::sqrt(off2[i - 1]);
    if (i + 1 < n) r += std::sqrt(off2[i]);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    // k-th smallest eigenvalue: count(x) <= k below, count(x) >= k+1 above
    double l = lo, h = hi;
    for (int it = 0; it < 200; ++it) {
      double m = 0.5 * (l + h);
      if (m <= l || m >= h) break;
      if (sturm_count(n, a.data(), off2.data(), m) > k) h = m; else l = m;
    }
    x[k] = 0.5 * (l + h);
  }
  for (int i = 0; i < n; ++i) {
    // orthonormal q_k at x_i: q_{k+1} sqrt(b_{k+1}) = (x - a_k) q_k - sqrt(b_k) q_{k-1}
    double qm1 = 0.0, q = 1.0 / std::sqrt(mu0), s = q * q;
    for (int k = 0; k + 1 < n; ++k) {
      double sb1 = std::sqrt(b[k + 1]);
      double sb0 = (k > 0) ? std::sqrt(b[k]) : 0.0;
      double qn = ((x[i] - a[k]) * q - sb0 * qm1) / sb1;
      qm1 = q;
      q = qn;
      s += q * q;
    }
    w[i] = 1.0 / s;
  }
}

}  // namespace

void gauss_jacobi_rule(int n, double al, double be, std::vector<double>& x,
                       std::vector<double>& w) {
  // weight (1-x)^al (1+x)^be on [-1, 1]
  if (n < 1 || al <= -1.0 || be <= -1.0)
    throw Error(HFSEM_ERR_INVALID_ARG, "gauss_jacobi_rule: bad arguments");
  std::vector<double> a(n), b(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double s = 2.0 * k + al + be;
    a[k] = (k == 0) ? (be - al) / (al + be + 2.0)
                    : (be * be - al * al) / (s * (s + 2.0));
  }
  for (int k = 1; k < n; ++k) {
    double s = 2.0 * k + al + be;
    // at k = 1 the factors k + al + be and s - 1 are equal and cancel (and
    // vanish together when al + be = -1, e.g. the Chebyshev weight)
    b[k] = (k == 1) ? 4.0 * (1.0 + al) * (1.0 + be) / (s * s * (s + 1.0))
                    : 4.0 * k * (k + al) * (k + be) * (k + al + be) /
                          (s * s * (s + 1.0) * (s - 1.0));
  }
  double mu0 = std::exp((al + be + 1.0) * std::log(2.0) + std::lgamma(al + 1.0) +
                        std::lgamma(be + 1.0) - std::lgamma(al + be + 2.0));
  gauss_from_recurrence(n, a, b, mu0, x, w);
}

void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  gauss_jacobi_rule(n, 0.0, 0.0, x, w);
}

}  // namespace hf
