// Host-side data of the time discretisation shared by the structured and the
// mesh solvers: Legendre polynomials, Gauss-Legendre nodes, the time matrices
// and time restriction blocks in the Legendre basis (Section 1,
// eq. chap4_restrictionTime), and the critical parameter mu* (Remark on the
// critical parameter).
#pragma once
#include <cmath>
#include <vector>

#include "stmg.h"

namespace stmg_host {

constexpr int kQmax = ST_MAX_PT + 1;

// ---------------------------------------------------------------------------
// Host-side time data in the Legendre basis (Section 1 definitions evaluated
// in closed form for P_k on the reference slab):
//   K_tau[k][l] = 1 - 2 [l < k and k - l odd]    (from int P_l P_k' = 2 there)
//   M_tau[k][k] = tau / (2k + 1),  psi_k(start) = (-1)^k,  psi_k(end) = 1.
// R1^T, R2^T (eq. chap4_restrictionTime) are the Legendre coefficients of the
// coarse P_l restricted to each fine half, by Gauss-Legendre quadrature.
// ---------------------------------------------------------------------------
inline double legendre_P(int k, double s) {
  double p0 = 1.0, p1 = s;
  if (k == 0) return p0;
  for (int m = 1; m < k; ++m) {
    double p2 = ((2.0 * m + 1.0) * s * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

inline void gauss_legendre(int npts, std::vector<double>& x, std::vector<double>& w) {
  x.assign(npts, 0.0);
  w.assign(npts, 0.0);
  for (int i = 0; i < npts; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (npts + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p = legendre_P(npts, z), pm = legendre_P(npts - 1, z);
      double dp = npts * (z * p - pm) / (z * z - 1.0);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p = legendre_P(npts, z), pm = legendre_P(npts - 1, z);
    double dp = npts * (z * p - pm) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct HostTime {
  int q;
  double K[kQmax * kQmax], Mh[kQmax], st[kQmax], en[kQmax], R1[kQmax * kQmax], R2[kQmax * kQmax];
};

inline HostTime make_time(int p_t) {
  HostTime t{};
  const int q = p_t + 1;
  t.q = q;
  for (int k = 0; k < q; ++k) {
    for (int l = 0; l < q; ++l) t.K[k * q + l] = (l < k && ((k - l) & 1)) ? -1.0 : 1.0;
    t.Mh[k] = 1.0 / (2.0 * k + 1.0);
    t.st[k] = (k & 1) ? -1.0 : 1.0;
    t.en[k] = 1.0;
  }
  std::vector<double> gx, gw;
  gauss_legendre(q + 2, gx, gw);
  // RsT[k][l] = (2k+1)/2 int_{-1}^{1} P_l(c(s)) P_k(s) ds, c(s) = (s -+ 1)/2;
  // R_s[k][l] = RsT[l][k] (coarse k <- fine l).
  for (int k = 0; k < q; ++k) {
    for (int l = 0; l < q; ++l) {
      double a1 = 0.0, a2 = 0.0;
      for (size_t g = 0; g < gx.size(); ++g) {
        a1 += gw[g] * legendre_P(l, 0.5 * (gx[g] - 1.0)) * legendre_P(k, gx[g]);
        a2 += gw[g] * legendre_P(l, 0.5 * (gx[g] + 1.0)) * legendre_P(k, gx[g]);
      }
      const double c = 0.5 * (2.0 * k + 1.0);
      t.R1[l * q + k] = c * a1;   // transpose: row = coarse l, column = fine k
      t.R2[l * q + k] = c * a2;
    }
  }
  return t;
}


// (p, p+1) subdiagonal Pade approximation of exp(z) (textbook closed form);
// mu* solves R(-3 mu) = sqrt(2) - 1 (Remark on the critical parameter).
inline double pade(int p, double z) {
  const int m = p, k = p + 1;
  auto fact = [](int a) { double r = 1.0; for (int i = 2; i <= a; ++i) r *= i; return r; };
  double num = 0.0, den = 0.0;
  for (int j = 0; j <= m; ++j)
    num += fact(m + k - j) * fact(m) / (fact(m + k) * fact(j) * fact(m - j)) * std::pow(z, j);
  for (int j = 0; j <= k; ++j)
    den += fact(m + k - j) * fact(k) / (fact(m + k) * fact(j) * fact(k - j)) * std::pow(-z, j);
  return num / den;
}

inline double mu_star(int p) {
  const double target = std::sqrt(2.0) - 1.0;
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
    double mid = 0.5 * (lo + hi);
    if (pade(p, -3.0 * mid) > target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace stmg_host
