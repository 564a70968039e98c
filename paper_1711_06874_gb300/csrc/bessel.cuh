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
constexpr int kTemmeTerms = 48;   // x <= 1.5 needs at most 14 terms
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

// Cost model.  An FP64 instruction occupies an SM sub-partition's FP64 unit
// for about as long as 32 lanes take at two lanes per cycle per SM, whatever
// the number of active lanes, so the routines below count FP64 instructions:
// no convergence tests inside the loops (term counts come from FP32
// estimates), no range checks inside the recurrence, one logarithm shared by
// the series and the prefactor, and the e^x of the scaled functions folded
// into the prefactor's exponential.

// Temme's series for x <= 1.5, given lx = log(x):
//   t0 = K_mu(x),  t1 = K_{mu+1}(x) x / 2  (both unscaled).
// The terms needed for 1e-17 grow from 3 (x = 1e-3) to 12 (x = 1.5); the
// count 1 + floor(6 + 6.5 sqrt(x)) keeps at least two in hand over
// |mu| <= 1/2.
TK_HD void tk_bessel_k_temme(const tk_nu_consts& c, double x, double lx, double* t0, double* t1) {
  const double mu = c.mu;
  const double l2x = 0.69314718055994530942 - lx;  // log(2 / x)
  const double sig = mu * l2x;
  const double e = exp(sig);  // (2/x)^mu
  const double ie = 1.0 / e;
  // sinh(sig) / sig: its Taylor series where e - 1/e would cancel
  double shs;
  if (fabs(sig) < 0.5) {
    const double t2 = sig * sig;
    shs = 1.0 / 6402373705728000.0;  // 1 / 18!
    // sum_{j <= 8} t2^j / (2j + 1)!, Horner from the top term
    shs = fma(shs, t2, 1.0 / 355687428096000.0);
    shs = fma(shs, t2, 1.0 / 1307674368000.0);
    shs = fma(shs, t2, 1.0 / 6227020800.0);
    shs = fma(shs, t2, 1.0 / 39916800.0);
    shs = fma(shs, t2, 1.0 / 362880.0);
    shs = fma(shs, t2, 1.0 / 5040.0);
    shs = fma(shs, t2, 1.0 / 120.0);
    shs = fma(shs, t2, 1.0 / 6.0);
    shs = fma(shs, t2, 1.0);
  } else {
    shs = 0.5 * (e - ie) / sig;
  }
  const double ch = 0.5 * (e + ie);  // cosh(sig)
  double f = c.mupi_sin * (ch * c.gam1 + shs * l2x * c.gam2);
  double p = 0.5 * e * c.gpmu;
  double q = 0.5 * ie * c.gmmu;
  double ck = 1.0;
  const double x2 = 0.25 * x * x;
  double s0 = f, s1 = p;
  const int K = 1 + (int)(6.0f + 6.5f * sqrtf((float)x));
  double dk = 0.0;
  for (int k = 1; k <= K; ++k) {
    dk += 1.0;
    f = fma(dk, f, p + q) * c.inv_k2mu2[k];
    p *= c.inv_kmmu[k];
    q *= c.inv_kpmu[k];
    ck *= x2 * c.inv_k[k];
    s0 = fma(ck, f, s0);
    s1 = fma(ck, fma(-dk, f, p), s1);
  }
  *t0 = s0;
  *t1 = s1;
}

// K_mu(x) e^x and K_{mu+1}(x) e^x for |mu| <= 1/2, x > 1.5, through the
// Tricomi-U representation: Miller's backward recurrence on the unnormalised
// minimal solution u_k (u_{N+1} = 0, u_N = 1), accumulating sum_k C_k u_k on
// the way; S = sum / u_0 and U_1/U_0 = u_1 / u_0.  The recurrence reaches
// 1e-17 with N of about 12 + 180/x terms.  |u_k| stays below 1e241 for every
// N <= 132 (its largest growth is at the smallest x), so no rescaling is needed.
TK_HD void tk_bessel_k_miller(const tk_nu_consts& c, double x, double* kmu, double* kmu1) {
  const double mu = c.mu;
  // N = 12 + ceil(180 / x) (at most 132 for x > 1.5) from an FP32 quotient,
  // one step longer so that it is never below the FP64 value
  const int N = 13 + (int)(180.0f / (float)x) < kMillerTerms - 1 ? 13 + (int)(180.0f / (float)x) : kMillerTerms - 1;
  const double mu2 = mu * mu;
  double u_next = 0.0, u = 1.0;  // u_{k+1}, u_k at k = N
  double acc = c.Ck[N];
  // a = 2 (k + x): rounded once at k = N, then lowered by 2 per step, which
  // is exact (a < 2^53), so the loop costs four FP64 instructions a step
  double a = 2.0 * ((double)N + x);
  // unrolled so that the next steps' coefficient loads are issued ahead of
  // the recurrence's dependent FMA (the operations and their order are as
  // written)
#pragma unroll 4
  for (int k = N; k >= 1; --k) {
    // u_{k-1} = 2 (k + x) u_k - ((k + 1/2)^2 - mu^2) u_{k+1}
    const double u_prev = fma(a, u, -c.Mk[k] * u_next);
    u_next = u;
    u = u_prev;
    acc = fma(c.Ck[k - 1], u, acc);
    a -= 2.0;
  }
  // K_mu e^x = sqrt(pi / (2 x)) u_0 / acc and
  // K_{mu+1} e^x = K_mu e^x (x + mu + 1/2 - (1/4 - mu^2) u_1 / u_0) / x
  //              = sqrt(pi / 2) x^(-1/2) ((x + mu + 1/2) u_0 - (1/4 - mu^2) u_1) / (x acc),
  // with sqrt(pi / 2) = 1.2533...: one division for both
  const double w = 1.2533141373155003 * TK_RSQRT(x) / (x * acc);
  *kmu = w * x * u;
  *kmu1 = w * fma(x + mu + 0.5, u, -(0.25 - mu2) * u_next);
}

// Forward recurrence K_{m+1} = K_{m-1} + (2m/x) K_m from K_mu, K_{mu+1} up to
// the order nu = nord + mu (nord >= 2).
TK_HD double tk_bessel_k_forward(const tk_nu_consts& c, double x, double km, double kp) {
  const double two_over_x = 2.0 / x;
  for (int k = 1; k < c.nord; ++k) {
    const double kn = km + ((c.mu + (double)k) * two_over_x) * kp;
    km = kp;
    kp = kn;
  }
  return kp;
}

// Matern covariance at z = sqrt(2 nu) r / ell; C(0) = sigma2 is the limit.
//   C = sigma2 exp(pref_log + nu log z) K_nu(z),  pref_log = (1 - nu) ln 2 - log Gamma(nu).
TK_HD double tk_matern_z(const tk_nu_consts& c, double sigma2, double z) {
  if (z <= 0.0) return sigma2;
  const double lz = log(z);
  double lp = c.pref_log + c.nu * lz;
  if (z <= 1.5) {
    double t0, t1;
    tk_bessel_k_temme(c, z, lz, &t0, &t1);
    if (c.nord == 0) return sigma2 * exp(lp) * t0;
    // K_{mu+1} = t1 (2 / z): the factor goes into the exponent
    if (c.nord == 1) return sigma2 * exp(lp + 0.69314718055994530942 - lz) * t1;
    return sigma2 * exp(lp) * tk_bessel_k_forward(c, z, t0, t1 * (2.0 / z));
  }
  lp -= z;  // the e^z of the scaled functions
  // exp(lp) is zero below -745: the value is 0 (and the recurrence is never
  // run on arguments that large)
  if (lp < -800.0) return 0.0;
  double km, kp;
  tk_bessel_k_miller(c, z, &km, &kp);
  if (c.nord == 0) return sigma2 * exp(lp) * km;
  if (c.nord == 1) return sigma2 * exp(lp) * kp;
  return sigma2 * exp(lp) * tk_bessel_k_forward(c, z, km, kp);
}
