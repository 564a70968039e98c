// Host-side constants of the Bessel order nu used by the K_nu kernels.
//
// Temme's series needs Gamma_1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu)
// and Gamma_2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2 for |mu| <= 1/2.  The
// difference cancels as mu -> 0, so both come from the Taylor series
//   log Gamma(1+mu) = -gamma mu + sum_{k>=2} (-1)^k zeta(k) mu^k / k
// split into its even part E(mu) and odd part O(mu):
//   1/Gamma(1 -+ mu) = exp(-E +- O),  Gamma_1 = e^-E sinh(O)/mu,  Gamma_2 = e^-E cosh(O).
// zeta(k) is summed directly with the Euler-Maclaurin tail.
#pragma once

#include <math.h>

#include "bessel.cuh"

namespace tk {

inline double zeta_em(int s) {
  // sum_{j < N} j^-s + N^(1-s)/(s-1) + N^-s / 2 + sum_p B_2p/(2p)! (s)_(2p-1) N^(-s-2p+1)
  const int N = 16;
  double sum = 0.0;
  for (int j = N - 1; j >= 1; --j) sum += pow((double)j, -(double)s);
  const double Nn = (double)N;
  sum += pow(Nn, 1.0 - s) / (s - 1.0) + 0.5 * pow(Nn, -(double)s);
  // Bernoulli numbers B_2 .. B_12 over (2p)!
  const double b[6] = {1.0 / 6.0 / 2.0,          -1.0 / 30.0 / 24.0,       1.0 / 42.0 / 720.0,
                       -1.0 / 30.0 / 40320.0,    5.0 / 66.0 / 3628800.0,   -691.0 / 2730.0 / 479001600.0};
  double rising = (double)s;  // (s)_(2p-1) for p = 1
  for (int p = 1; p <= 6; ++p) {
    sum += b[p - 1] * rising * pow(Nn, -(double)s - 2.0 * p + 1.0);
    rising *= (s + 2.0 * p - 1.0) * (s + 2.0 * p);
  }
  return sum;
}

// zeta(k) / k for k = 2 .. 64, computed once (they do not depend on nu).
struct ZetaTable {
  double zk[65];
  ZetaTable() {
    zk[0] = zk[1] = 0.0;
    for (int k = 2; k <= 64; ++k) zk[k] = zeta_em(k) / (double)k;
  }
};

inline const ZetaTable& zeta_table() {
  static const ZetaTable t;  // thread-safe one-time initialisation
  return t;
}

inline tk_nu_consts make_nu_consts(double nu) {
  tk_nu_consts c;
  c.nu = nu;
  c.nord = (int)floor(nu + 0.5);
  c.mu = nu - (double)c.nord;
  const double mu = c.mu;
  const double euler_gamma = 0.57721566490153286061;
  double E = 0.0, Oq = -euler_gamma;  // Oq = O(mu) / mu
  const double m2 = mu * mu;
  double pw = 1.0;  // (mu^2)^floor(k/2)
  for (int k = 2; k <= 64; ++k) {
    if (k % 2 == 0) pw *= m2;
    const double z = zeta_table().zk[k];
    if (k % 2 == 0)
      E += z * pw;   // zeta(k) mu^k / k
    else
      Oq -= z * pw;  // zeta(k) mu^(k-1) / k
  }
  const double O = Oq * mu;
  const double sh = (fabs(O) < 1e-6) ? (1.0 + O * O / 6.0) : sinh(O) / O;
  const double eE = exp(-E);
  c.gam1 = eE * Oq * sh;
  c.gam2 = eE * cosh(O);
  c.gpmu = 1.0 / (c.gam2 - mu * c.gam1);
  c.gmmu = 1.0 / (c.gam2 + mu * c.gam1);
  const double pi = 3.141592653589793238;
  c.mupi_sin = (fabs(mu) < 1e-12) ? 1.0 : (mu * pi) / sin(mu * pi);
  c.pref_log = (1.0 - nu) * log(2.0) - lgamma(nu);
  for (int k = 0; k < kTemmeTerms; ++k) {
    const double dk = (double)k;
    c.inv_k2mu2[k] = (k == 0) ? 0.0 : 1.0 / (dk * dk - mu * mu);
    c.inv_kmmu[k] = (k == 0) ? 0.0 : 1.0 / (dk - mu);
    c.inv_kpmu[k] = (k == 0) ? 0.0 : 1.0 / (dk + mu);
    c.inv_k[k] = (k == 0) ? 0.0 : 1.0 / dk;
  }
  // C_k = prod_{j <= k} ((j - 1/2)^2 - mu^2) / j; zero from k = 1 when mu = +-1/2
  c.Ck[0] = 1.0;
  for (int k = 1; k < kMillerTerms; ++k) {
    const double dk = (double)k;
    c.Ck[k] = c.Ck[k - 1] * (((dk - 0.5) * (dk - 0.5) - mu * mu) / dk);
  }
  for (int k = 0; k < kMillerTerms; ++k) {
    const double dk = (double)k;
    c.Mk[k] = (dk + 0.5) * (dk + 0.5) - mu * mu;
  }
  return c;
}

}  // namespace tk
