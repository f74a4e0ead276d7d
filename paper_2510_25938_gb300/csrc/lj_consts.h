// lj_consts.h -- constants of Eq. (1) derived once, on the host, from the
// parameters eps and sigma, and handed to the kernels by value: no kernel
// forms them itself (each form would cost FP64 divisions per thread).
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
};

inline LjConsts make_consts(double eps, double sigma) {
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
  return k;
}

}  // namespace ljh
