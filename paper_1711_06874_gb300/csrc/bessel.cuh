// Modified Bessel function of the second kind K_nu(x), real order nu >= 0,
// x > 0, in FP64, and the Matern covariance of Sec. 2.2, Eq. (Matern):
//   C(r) = sigma2 2^(1-nu) / Gamma(nu) z^nu K_nu(z),  z = sqrt(2 nu) r / ell.
//
// The paper names K_nu but gives no method.  This file uses, by name:
//  * Temme's series (N. M. Temme, J. Comput. Phys. 19 (1975) 324) for
//    K_mu, K_{mu+1} with |mu| <= 1/2 and x <= 1.5;
//  * for x > 1.5, Temme's representation K_mu(x) = sqrt(pi) (2x)^mu e^-x
//    U(mu+1/2, 2mu+1, 2x) through the Tricomi function U.  With
//    U_k = U(mu+1/2+k, 2mu+1, 2x) the contiguous relation of U in its first
//    parameter gives ((k+1/2)^2 - mu^2) U_{k+1} = 2(k+x) U_k - U_{k-1}; U_k is
//    its minimal solution, so the ratios U_k/U_{k-1} come from the backward
//    recurrence (Miller's algorithm), and the sum
//      sum_k (1/2-mu)_k (1/2+mu)_k / k! U_k = (2x)^(-mu-1/2)
//    (the Laplace integral of U summed under the integral sign) normalises
//    them, as in the Thompson-Barnett (Comput. Phys. Commun. 47 (1987) 245)
//    treatment.  Differentiating the U representation gives
//      K_{mu+1} / K_mu = (x + mu + 1/2 - (1/4 - mu^2) U_1/U_0) / x;
//  * forward recurrence K_{m+1} = K_{m-1} + (2m/x) K_m up to nu = N + mu.
//
// Gamma_1(mu), Gamma_2(mu), Gamma(1 +- mu) and log Gamma(nu) depend on nu
// only; the host computes them once per kernel (tk_nu_consts) from the
// Taylor series log Gamma(1+mu) = -gamma mu + sum_{k>=2} (-1)^k zeta(k) mu^k / k,
// which has no cancellation as mu -> 0.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define TK_HD __host__ __device__ __forceinline__
#else
#define TK_HD inline
#endif

#ifndef __CUDA_ARCH__
// host builds (the constants' tests): 1 / sqrt(x)
inline double tk_rsqrt_host(double x) { return 1.0 / sqrt(x); }
#define TK_RSQRT(x) tk_rsqrt_host(x)
#else
#define TK_RSQRT(x) rsqrt(x)
#endif

// Terms of Temme's series and of the backward recurrence that are
// precomputed per order, so the device loops need no division.
constexpr int kTemmeTerms = 48;   // x <= 1.5 converges in about 25 terms
constexpr int kMillerTerms = 133;  // N = 12 + ceil(180 / x) <= 132 for x > 1.5

struct tk_nu_consts {
  double nu;        // order
  double mu;        // nu - nord, in [-1/2, 1/2)
  int nord;         // nu = nord + mu
  double gam1;      // (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu)
  double gam2;      // (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2
  double gpmu;      // Gamma(1 + mu)
  double gmmu;      // Gamma(1 - mu)
  double mupi_sin;  // mu pi / sin(mu pi)
  double pref_log;  // (1 - nu) ln 2 - log Gamma(nu)
  double inv_k2mu2[kTemmeTerms];  // 1 / (k^2 - mu^2)
  double inv_kmmu[kTemmeTerms];   // 1 / (k - mu)
  double inv_kpmu[kTemmeTerms];   // 1 / (k + mu)
  double inv_k[kTemmeTerms];      // 1 / k
  double Ck[kMillerTerms];        // (1/2 - mu)_k (1/2 + mu)_k / k!
  double Mk[kMillerTerms];        // (k + 1/2)^2 - mu^2, the recurrence's second coefficient
};

// K_mu(x) and K_{mu+1}(x), both multiplied by e^x, for |mu| <= 1/2, x > 0.
TK_HD void tk_bessel_k_pair_scaled(const tk_nu_consts& c, double x, double* kmu, double* kmu1) {
  const double mu = c.mu;
  if (x <= 1.5) {
    // Temme's series (the terms grow like I_mu(x) while K_mu falls like e^-x,
    // so the series is kept to x <= 1.5 where that cancellation stays small).
    const double lx = log(2.0 / x);
    const double sig = mu * lx;
    const double shs = (fabs(sig) < 1e-8) ? 1.0 + sig * sig / 6.0 : sinh(sig) / sig;
    double f = c.mupi_sin * (cosh(sig) * c.gam1 + shs * lx * c.gam2);
    const double e = exp(sig);  // (2/x)^mu
    double p = 0.5 * e * c.gpmu;
    double q = 0.5 / e * c.gmmu;
    double ck = 1.0;
    const double x2 = 0.25 * x * x;
    double s0 = f, s1 = p;
    for (int k = 1; k < kTemmeTerms; ++k) {
      const double dk = (double)k;
      f = (dk * f + p + q) * c.inv_k2mu2[k];
      p *= c.inv_kmmu[k];
      q *= c.inv_kpmu[k];
      ck *= x2 * c.inv_k[k];
      const double d0 = ck * f;
      const double d1 = ck * (p - dk * f);
      s0 += d0;
      s1 += d1;
      if (fabs(d0) < 1e-17 * fabs(s0) && fabs(d1) < 1e-17 * fabs(s1)) break;
    }
    const double ex = exp(x);
    *kmu = s0 * ex;
    *kmu1 = s1 * (2.0 / x) * ex;
    return;
  }
  // Tricomi-U representation, Miller's backward recurrence on the
  // unnormalised minimal solution u_k (u_{N+1} = 0, u_N = 1), accumulating
  // sum_k C_k u_k on the way; S = sum / u_0 and U_1/U_0 = u_1 / u_0.
  // The recurrence reaches 1e-17 with N of about 12 + 180/x terms; values are
  // rescaled by 2^-600 whenever they pass 2^600.
  // N = 12 + ceil(180 / x) (at most 132 for x > 1.5) from an FP32 quotient,
  // one step longer so that it is never below the FP64 value
  const int N = 13 + (int)(180.0f / (float)x) < kMillerTerms - 1 ? 13 + (int)(180.0f / (float)x) : kMillerTerms - 1;
  const double mu2 = mu * mu;
  const double x2 = 2.0 * x;
  double u_next = 0.0, u = 1.0;  // u_{k+1}, u_k at k = N
  double acc = c.Ck[N];
  double dk2 = 2.0 * (double)N;  // 2 k
  for (int k = N; k >= 1; --k) {
    // u_{k-1} = 2 (k + x) u_k - ((k + 1/2)^2 - mu^2) u_{k+1}
    const double u_prev = fma(dk2 + x2, u, -c.Mk[k] * u_next);
    u_next = u;
    u = u_prev;
    acc = fma(c.Ck[k - 1], u, acc);
    dk2 -= 2.0;
    // |u| grows by at most 2 (k + x) per step (far below 2^100 for any x the
    // grids produce): a check every 4 steps keeps it below 2^1000
    if ((k & 3) == 0 && fabs(u) > 0x1p600) {
      u *= 0x1p-600;
      u_next *= 0x1p-600;
      acc *= 0x1p-600;
    }
  }
  // K_mu e^x = sqrt(pi / (2 x)) u_0 / acc and
  // K_{mu+1} e^x = K_mu e^x (x + mu + 1/2 - (1/4 - mu^2) u_1 / u_0) / x
  //              = sqrt(pi / 2) x^(-1/2) ((x + mu + 1/2) u_0 - (1/4 - mu^2) u_1) / (x acc),
  // with sqrt(pi / 2) = 1.2533...: one division for both
  const double w = 1.2533141373155003 * TK_RSQRT(x) / (x * acc);
  *kmu = w * x * u;
  *kmu1 = w * fma(x + mu + 0.5, u, -(0.25 - mu2) * u_next);
}

// K_nu(x) e^x for the order in c (nu = nord + mu), x > 0.
TK_HD double tk_bessel_k_scaled(const tk_nu_consts& c, double x) {
  double km, kp;
  tk_bessel_k_pair_scaled(c, x, &km, &kp);
  if (c.nord == 0) return km;
  if (c.nord == 1) return kp;
  const double two_over_x = 2.0 / x;
  for (int k = 1; k < c.nord; ++k) {
    const double kn = km + ((c.mu + (double)k) * two_over_x) * kp;
    km = kp;
    kp = kn;
  }
  return kp;
}

// Matern covariance at z = sqrt(2 nu) r / ell; C(0) = sigma2 is the limit.
TK_HD double tk_matern_z(const tk_nu_consts& c, double sigma2, double z) {
  if (z <= 0.0) return sigma2;
  const double lp = c.pref_log + c.nu * log(z) - z;
  return sigma2 * exp(lp) * tk_bessel_k_scaled(c, z);
}
