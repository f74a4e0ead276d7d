// lj_consts.h -- constants of the pair potential derived once, on the host,
// from its parameters, and handed to the kernels by value: no kernel forms
// them itself (each form would cost FP64 divisions per thread).  Eq. (1)
// (Lennard-Jones, eps and sigma) is the method's potential; the Morse
// potential V(r) = eps e (e - 2), e = exp(rho (1 - r / re)), with re in the
// sigma slot, is its pair-potential extension.
#pragma once

namespace ljh {

struct LjConsts {
  double eps, sigma;
  double sig2;     // sigma^2
  double gscale;   // 24 eps / sigma^2: gradient factor on unscaled coordinates
  double gs;       // 24 eps / sigma: gradient factor on coordinates divided by sigma
  double e2, e4;   // 2 eps, 4 eps: energy factors of a one-sided / half-pair sum
  float sig2_f;    // sigma^2, FP32
  float gscale_f;  // 24 eps / sigma^2, FP32
  float gs_f;      // 24 eps / sigma, FP32
  float e2_f, e4_f;
  float is_hi, is_lo;   // 1 / sigma as a double-float (hi + lo)
  // Morse (pot == LJ_POT_MORSE; re = sigma)
  int pot;              // LJ_POT_LJ or LJ_POT_MORSE
  double rho;           // range parameter
  double rho_re;        // rho / re: exponent slope
  double m_g;           // 2 eps rho / re: gradient factor
  double m_half;        // eps / 2: energy factor of a one-sided sum
  float rho_f, rho_re_f, m_g_f, m_half_f;
  float rho_lo;         // rho - rho_f: rho as a double-float (rho_f, rho_lo)
  float eps_f;          // eps: energy factor of a half-pair sum
};

inline LjConsts make_consts(double eps, double sigma, int pot = 0, double rho = 0.0) {
  LjConsts k;
  k.eps = eps;
  k.sigma = sigma;
  k.sig2 = sigma * sigma;
  k.gscale = 24.0 * eps / k.sig2;
  k.gs = 24.0 * eps / sigma;
  k.e2 = 2.0 * eps;
  k.e4 = 4.0 * eps;
  const double is = 1.0 / sigma;
  k.sig2_f = (float)k.sig2;
  k.gscale_f = (float)k.gscale;
  k.gs_f = (float)k.gs;
  k.e2_f = (float)k.e2;
  k.e4_f = (float)k.e4;
  k.is_hi = (float)is;
  k.is_lo = (float)(is - (double)k.is_hi);
  k.pot = pot;
  k.rho = rho;
  k.rho_re = rho / sigma;
  k.m_g = 2.0 * eps * rho / sigma;
  k.m_half = 0.5 * eps;
  k.rho_f = (float)k.rho;
  k.rho_re_f = (float)k.rho_re;
  k.m_g_f = (float)k.m_g;
  k.m_half_f = (float)k.m_half;
  k.rho_lo = (float)(rho - (double)k.rho_f);
  k.eps_f = (float)eps;
  return k;
}

}  // namespace ljh
