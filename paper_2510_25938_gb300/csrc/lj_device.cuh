// lj_device.cuh -- sm_103a device building blocks: teams, team reductions,
// Philox4x32-10, float-float energies and the Eq. (1) pair loops.
//
// A "team" is the group of T threads that owns one candidate cluster:
// one warp (T = 32) or a multiple of 32 threads synchronised by a named
// barrier.  Thread `rank` of a team owns atoms rank, rank + T, ... (A slots)
// and exactly the 3 coordinates / gradient components of those atoms, so
// every vector operation of L-BFGS is thread-local and only the pair loop
// reads other threads' atoms (from shared memory).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ljd {

constexpr unsigned kFull = 0xffffffffu;

enum : int32_t {
  ST_CONVERGED = 0, ST_MAXITER = 1, ST_LS_FAIL = 2, ST_NONFINITE = 3, ST_TIMEOUT = 4,
  ST_BAD_INPUT = 5
};

// ---------------------------------------------------------------------------
// Team
// ---------------------------------------------------------------------------
template <int T>
struct Team {
  static_assert(T % 32 == 0 && T >= 32 && T <= 1024, "team size");
  int rank;       // 0 .. T-1
  int bar;        // named barrier id (T > 32); 1..15
  double* red;    // shared scratch for cross-warp reductions: 2 x 8 x (T/32) doubles
  mutable int flip = 0;   // which half of `red` the next reduction uses
  __device__ __forceinline__ void sync() const {
    if constexpr (T == 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(T) : "memory");
    }
  }
  // Scratch half for the next cross-warp reduction.  Alternating halves
  // makes a barrier before the write unnecessary: a thread can only reach
  // the reduction after next (same half) once every thread has passed the
  // next reduction's barrier, i.e. has finished reading this one.
  __device__ __forceinline__ double* scratch() const {
    double* b = red + (flip ? 8 * (T / 32) : 0);
    flip ^= 1;
    return b;
  }
};

template <typename V>
__device__ __forceinline__ V shfl_xor(V v, int o) { return __shfl_xor_sync(kFull, v, o); }

// Sum of NV values over the team; every thread receives the same bits
// (xor butterfly: partners add the same operands; the cross-warp stage sums
// the per-warp results in the same order on every thread).
template <int T, int NV, typename V>
__device__ __forceinline__ void team_sum(const Team<T>& tm, V (&v)[NV]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += shfl_xor(v[k], o);
  }
  if constexpr (T > 32) {
    static_assert(NV * sizeof(V) <= 8 * sizeof(double), "reduction scratch");
    constexpr int NW = T / 32;
    V* buf = reinterpret_cast<V*>(tm.scratch());
    if ((tm.rank & 31) == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) buf[(tm.rank >> 5) * NV + k] = v[k];
    }
    tm.sync();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      V s = buf[k];
#pragma unroll
      for (int w = 1; w < NW; ++w) s += buf[w * NV + k];
      v[k] = s;
    }
  }
}

template <int T, typename V>
__device__ __forceinline__ V team_sum1(const Team<T>& tm, V x) {
  V v[1] = {x};
  team_sum<T, 1, V>(tm, v);
  return v[0];
}

// Max over the team (inputs are >= 0; a non-finite entry must be passed as +inf).
template <int T, int NV, typename V>
__device__ __forceinline__ void team_max(const Team<T>& tm, V (&v)[NV]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = fmax(v[k], shfl_xor(v[k], o));
  }
  if constexpr (T > 32) {
    constexpr int NW = T / 32;
    V* buf = reinterpret_cast<V*>(tm.scratch());
    if ((tm.rank & 31) == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) buf[(tm.rank >> 5) * NV + k] = v[k];
    }
    tm.sync();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      V s = buf[k];
#pragma unroll
      for (int w = 1; w < NW; ++w) s = fmax(s, buf[w * NV + k]);
      v[k] = s;
    }
  }
}

// |x| with NaN mapped to +inf, so that fmax-based norms flag non-finite input
__device__ __forceinline__ float abs_nan_inf(float x) {
  return (x != x) ? __int_as_float(0x7f800000) : fabsf(x);
}
__device__ __forceinline__ double abs_nan_inf(double x) {
  return (x != x) ? __longlong_as_double(0x7ff0000000000000LL) : fabs(x);
}

// ---------------------------------------------------------------------------
// Float-float energy values (FP32 phase): hi + lo, |lo| <= ulp(hi)/2.
// The FP32 phase keeps its energies in this form so that the line search can
// form energy differences without any FP64 instruction.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = ff_two_sum(a.hi, b);
  return ff_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
// a c for a float-float a and an FP32 constant c: the high product exact by
// TwoProd (FMA), the low word's product and that error added, renormalised;
// ~2^-47 relative for any c (for a power of two it is the exact product)
__device__ __forceinline__ ff ff_scale(ff a, float c) {
  const float p = __fmul_rn(a.hi, c);
  const float lo = fmaf(a.lo, c, fmaf(a.hi, c, -p));
  const float s = __fadd_rn(p, lo);
  return ff{s, __fsub_rn(lo, __fsub_rn(s, p))};
}

// energy-value traits: difference, finiteness, conversion
__device__ __forceinline__ float fdiff(ff a, ff b) {
  return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}
__device__ __forceinline__ double fdiff(double a, double b) { return a - b; }
__device__ __forceinline__ bool fisfinite(ff a) { return isfinite(a.hi); }
__device__ __forceinline__ bool fisfinite(double a) { return isfinite(a); }
__device__ __forceinline__ double fto_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double fto_double(double a) { return a; }

template <int T>
__device__ __forceinline__ ff team_sum_ff(const Team<T>& tm, ff v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff w{shfl_xor(v.hi, o), shfl_xor(v.lo, o)};
    v = ff_add(v, w);
  }
  if constexpr (T > 32) {
    constexpr int NW = T / 32;
    float* buf = reinterpret_cast<float*>(tm.scratch());
    if ((tm.rank & 31) == 0) {
      buf[2 * (tm.rank >> 5)] = v.hi;
      buf[2 * (tm.rank >> 5) + 1] = v.lo;
    }
    tm.sync();
    ff s{buf[0], buf[1]};
#pragma unroll
    for (int w = 1; w < NW; ++w) s = ff_add(s, ff{buf[2 * w], buf[2 * w + 1]});
    v = s;
  }
  return v;
}

// team_sum of s[0..NS-1] and team_max of m[0..1] (inputs >= 0, non-finite
// as +inf) in one pass, one cross-warp exchange; each value gets the
// operations of its own reduction in the same order
template <int T, typename V, typename M, int NS>
__device__ __forceinline__ void team_sums_max2(const Team<T>& tm, V (&s)[NS], M (&m)[2]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] += shfl_xor(s[k], o);
#pragma unroll
    for (int k = 0; k < 2; ++k) m[k] = fmax(m[k], shfl_xor(m[k], o));
  }
  if constexpr (T > 32) {
    constexpr int NW = T / 32;
    static_assert(NS * sizeof(V) + 2 * sizeof(M) <= 8 * sizeof(double), "reduction scratch");
    unsigned char* raw = reinterpret_cast<unsigned char*>(tm.scratch());
    V* bs = reinterpret_cast<V*>(raw);
    M* bm = reinterpret_cast<M*>(raw + ((NS * NW * sizeof(V) + sizeof(M) - 1) / sizeof(M)) * sizeof(M));
    if ((tm.rank & 31) == 0) {
#pragma unroll
      for (int k = 0; k < NS; ++k) bs[(tm.rank >> 5) * NS + k] = s[k];
#pragma unroll
      for (int k = 0; k < 2; ++k) bm[(tm.rank >> 5) * 2 + k] = m[k];
    }
    tm.sync();
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      V a = bs[k];
#pragma unroll
      for (int w = 1; w < NW; ++w) a += bs[w * NS + k];
      s[k] = a;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      M b = bm[k];
#pragma unroll
      for (int w = 1; w < NW; ++w) b = fmax(b, bm[w * 2 + k]);
      m[k] = b;
    }
  }
}

// team_sum_ff of e and team_sum of x in one pass (one cross-warp exchange):
// each value gets exactly the operations, in the order, of its own reduction
template <int T>
__device__ __forceinline__ void team_sum_ff_f(const Team<T>& tm, ff& e, float& x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff w{shfl_xor(e.hi, o), shfl_xor(e.lo, o)};
    e = ff_add(e, w);
    x += shfl_xor(x, o);
  }
  if constexpr (T > 32) {
    constexpr int NW = T / 32;
    float* buf = reinterpret_cast<float*>(tm.scratch());
    if ((tm.rank & 31) == 0) {
      buf[3 * (tm.rank >> 5)] = e.hi;
      buf[3 * (tm.rank >> 5) + 1] = e.lo;
      buf[3 * (tm.rank >> 5) + 2] = x;
    }
    tm.sync();
    ff s{buf[0], buf[1]};
    float t = buf[2];
#pragma unroll
    for (int w = 1; w < NW; ++w) {
      s = ff_add(s, ff{buf[3 * w], buf[3 * w + 1]});
      t += buf[3 * w + 2];
    }
    e = s;
    x = t;
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from the published round
// function and key schedule, and the 53-bit uniform built from two words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double u01_53(uint32_t a, uint32_t b) {
  const double hi = (double)(a >> 5);
  const double lo = (double)(b >> 6);
  return __dmul_rn(__dadd_rn(__dmul_rn(hi, 67108864.0), lo), 1.0 / 9007199254740992.0);
}

// uniform number `draw` of stream `tag` at counter (k, s, w)
__device__ __forceinline__ double stream_u01(uint64_t seed, uint32_t tag, uint32_t draw,
                                             uint32_t k, uint32_t s, uint32_t w) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ tag);
  const uint4 r = philox4x32_10(make_uint4(draw >> 1, k, s, w), key);
  return (draw & 1u) ? u01_53(r.z, r.w) : u01_53(r.x, r.y);
}

// ---------------------------------------------------------------------------
// Pair loops of Eq. (1).  One-sided form: the thread owning atom i sums over
// every j != i, so no two threads write the same gradient entry and the
// result is deterministic.  Per owned atom it returns
//   acc_i = sum_j s2 s6 (2 s6 - 1) (x_i - x_j),  e_i = sum_j s6 (s6 - 1)
// with s2 = sigma^2 / r^2, s6 = s2^3; then grad_i = -(24 eps / sigma^2) acc_i
// and E = 2 eps sum_i e_i (every unordered pair is visited twice).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct alignas(16) PosF { float x, y, z, w; };
struct alignas(16) PosD { double x, y, z, w; };

template <typename X> struct PosOf;
template <> struct PosOf<float> { using type = PosF; };
template <> struct PosOf<double> { using type = PosD; };

// ---------------------------------------------------------------------------
// FP32 pair rows on packed float pairs (sm_100+ FADD2 / FMUL2 / FFMA2: two
// IEEE single operations per instruction, each rounded exactly like its
// scalar form).  Positions are staged two atoms per 32-byte record, atoms
// 2m and 2m+1 in record m (unscaled: differences of the given coordinates
// are the exact-as-possible inputs of r2, and sigma enters as one product
// sigma^2 / r2 where sigma != 1); an odd cluster
// pads its last record with kFarAtom, whose terms underflow to exactly zero
// (r2 ~ 4e36 keeps 1/r2 normal, (1/r2)^2 rounds to 0), so every record holds
// two live lanes and no lane needs a bounds test.  One instruction then
// serves two pair terms, which halves the issue slots of the FP32 row: the
// row is bound by the FMA pipe instead of by instruction issue.
// ---------------------------------------------------------------------------
struct alignas(16) PosF2 {
  float x[2], y[2], z[2], w[2];
};
constexpr float kFarAtom = 0x1p60f;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// stage atom i into its record; the owner of the last atom of an odd
// cluster also writes the padding lane
__device__ __forceinline__ void stage_f32x2(PosF2* pos, int n, int i, float x, float y, float z) {
  PosF2& r = pos[i >> 1];
  const int l = i & 1;
  r.x[l] = x; r.y[l] = y; r.z[l] = z;
  if (i == n - 1 && l == 0) {
    r.x[1] = kFarAtom; r.y[1] = kFarAtom; r.z[1] = kFarAtom;
  }
}

// One-sided row of atom i (position px, py, pz) against the n atoms of
// `pos`: b = sum_j c_ij (x_j - x_i) with c = s2 s6 (2 s6 - 1), s2 = sigma^2
// / r^2 (SIG: sigma != 1, sig2 = sigma^2), and e += sum_j s6 (s6 - 1), the
// self term excluded.  Energy: per lane, blocks of 4 terms summed in FP32,
// the two lanes' block sums added and folded into the float-float `e`
// (FF), or summed in plain FP32 into e.hi (!FF: ~8 ulps of the row, below the
// pair terms' own error; used where the energy is only reported).
template <bool SIG, bool FF = true>
__device__ __forceinline__ void pair_row_f32x2(int n, int i, float px, float py, float pz,
                                               const PosF2* __restrict__ pos, float sig2,
                                               float& bx, float& by, float& bz, ff& e) {
  const int M = (n + 1) >> 1;
  const float2 npx = f2(-px), npy = f2(-py), npz = f2(-pz), m1 = f2(-1.f);
  const int sx = (i & 1) ? -1 : (i >> 1);     // record whose lane 0 is atom i
  const int sy = (i & 1) ? (i >> 1) : -1;     // record whose lane 1 is atom i
  float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f);
  auto term = [&](int m, float2& eb) {
    const float4 xy = *reinterpret_cast<const float4*>(&pos[m].x[0]);
    const float2 zz = *reinterpret_cast<const float2*>(&pos[m].z[0]);
    const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), npx);
    const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), npy);
    const float2 dz = __fadd2_rn(zz, npz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 s2;
    s2.x = (m == sx) ? 0.f : rcp_approx(r2.x);
    s2.y = (m == sy) ? 0.f : rcp_approx(r2.y);
    if constexpr (SIG) s2 = __fmul2_rn(s2, f2(sig2));
    const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
    const float2 t = __fadd2_rn(s6, m1);
    eb = __ffma2_rn(s6, t, eb);
    const float2 c = __fmul2_rn(__fmul2_rn(s2, s6), __fadd2_rn(s6, t));
    ax = __ffma2_rn(c, dx, ax);
    ay = __ffma2_rn(c, dy, ay);
    az = __ffma2_rn(c, dz, az);
  };
  int m = 0;
  for (; m + 4 <= M; m += 4) {
    float2 eb = f2(0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) term(m + u, eb);
    if constexpr (FF) e = ff_add_f(e, __fadd_rn(eb.x, eb.y));
    else e.hi = __fadd_rn(e.hi, __fadd_rn(eb.x, eb.y));
  }
  if (m < M) {
    float2 eb = f2(0.f);
    for (; m < M; ++m) term(m, eb);
    if constexpr (FF) e = ff_add_f(e, __fadd_rn(eb.x, eb.y));
    else e.hi = __fadd_rn(e.hi, __fadd_rn(eb.x, eb.y));
  }
  bx = __fadd_rn(ax.x, ax.y);
  by = __fadd_rn(ay.x, ay.y);
  bz = __fadd_rn(az.x, az.y);
}

// One-sided Morse row of atom i on the same packed records (unscaled
// coordinates): with r from r^2 and a reciprocal square root, e = exp(rho -
// rr r) (rr = rho / re; FP32 __expf), b = sum_j e (e - 1) (x_j - x_i) / r and
// e_row += sum_j e (e - 2), the self term excluded; the padding atom's terms
// vanish (its exponential underflows to 0).  Energy blocks as in
// pair_row_f32x2 (float-float).
__device__ __forceinline__ void morse_row_f32x2(int n, int i, float px, float py, float pz,
                                                const PosF2* __restrict__ pos, float rho,
                                                float rr, float& bx, float& by, float& bz,
                                                ff& e) {
  const int M = (n + 1) >> 1;
  const float2 npx = f2(-px), npy = f2(-py), npz = f2(-pz);
  const float2 nrr = f2(-rr), rho2 = f2(rho), m1 = f2(-1.f), m2 = f2(-2.f);
  const int sx = (i & 1) ? -1 : (i >> 1);     // record whose lane 0 is atom i
  const int sy = (i & 1) ? (i >> 1) : -1;     // record whose lane 1 is atom i
  float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f);
  auto term = [&](int m, float2& eb) {
    const float4 xy = *reinterpret_cast<const float4*>(&pos[m].x[0]);
    const float2 zz = *reinterpret_cast<const float2*>(&pos[m].z[0]);
    const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), npx);
    const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), npy);
    const float2 dz = __fadd2_rn(zz, npz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    if (m == sx) ir.x = 0.f;                   // the self term: r = 0 instead of 0 * inf
    if (m == sy) ir.y = 0.f;
    const float2 x = __ffma2_rn(nrr, __fmul2_rn(r2, ir), rho2);      // rho (1 - r / re)
    float2 ex = make_float2(__expf(x.x), __expf(x.y));
    if (m == sx) ex.x = 0.f;
    if (m == sy) ex.y = 0.f;
    eb = __ffma2_rn(ex, __fadd2_rn(ex, m2), eb);
    const float2 c = __fmul2_rn(__fmul2_rn(ex, __fadd2_rn(ex, m1)), ir);
    ax = __ffma2_rn(c, dx, ax);
    ay = __ffma2_rn(c, dy, ay);
    az = __ffma2_rn(c, dz, az);
  };
  int m = 0;
  for (; m + 4 <= M; m += 4) {
    float2 eb = f2(0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) term(m + u, eb);
    e = ff_add_f(e, __fadd_rn(eb.x, eb.y));
  }
  if (m < M) {
    float2 eb = f2(0.f);
    for (; m < M; ++m) term(m, eb);
    e = ff_add_f(e, __fadd_rn(eb.x, eb.y));
  }
  bx = __fadd_rn(ax.x, ax.y);
  by = __fadd_rn(ay.x, ay.y);
  bz = __fadd_rn(az.x, az.y);
}

// Double-double helpers: exact sum a + b = s + e (Knuth TwoSum).
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return dd{s, e};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  return dd_two_sum(s.hi, __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo)));
}

template <int T>
__device__ __forceinline__ double team_sum_dd(const Team<T>& tm, dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd w{shfl_xor(v.hi, o), shfl_xor(v.lo, o)};
    v = dd_add(v, w);
  }
  if constexpr (T > 32) {
    constexpr int NW = T / 32;
    double* buf = tm.scratch();
    if ((tm.rank & 31) == 0) {
      buf[2 * (tm.rank >> 5)] = v.hi;
      buf[2 * (tm.rank >> 5) + 1] = v.lo;
    }
    tm.sync();
    dd s{buf[0], buf[1]};
#pragma unroll
    for (int w = 1; w < NW; ++w) s = dd_add(s, dd{buf[2 * w], buf[2 * w + 1]});
    v = s;
  }
  return __dadd_rn(v.hi, v.lo);
}

// FP64: the reciprocal is the correctly rounded one; the energy is summed in
// 4-term blocks folded into a compensated (double-double) accumulator, so
// that near a minimum its rounding noise stays below the decreases the
// line search must resolve (|E| ~ 170 for LJ38, decreases ~1e-12).
__device__ __forceinline__ void pair_row_f64(int n, int i, double px, double py, double pz,
                                             const PosD* __restrict__ pos, double sig2,
                                             double& ax, double& ay, double& az, dd& e) {
  ax = 0.0; ay = 0.0; az = 0.0;
  int j = 0;
  for (; j + 4 <= n; j += 4) {
    double eb = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const PosD q = pos[j + u];
      const double dx = px - q.x, dy = py - q.y, dz = pz - q.z;
      const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const double ir2 = (j + u == i) ? 0.0 : __drcp_rn(r2);
      const double s2 = sig2 * ir2;
      const double s6 = s2 * s2 * s2;
      const double t = s6 - 1.0;
      eb = fma(s6, t, eb);
      const double c = (s2 * s6) * (s6 + t);
      ax = fma(c, dx, ax);
      ay = fma(c, dy, ay);
      az = fma(c, dz, az);
    }
    dd s = dd_two_sum(e.hi, eb);
    e.hi = s.hi;
    e.lo = __dadd_rn(e.lo, s.lo);
  }
  double eb = 0.0;
  for (; j < n; ++j) {
    const PosD q = pos[j];
    const double dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double ir2 = (j == i) ? 0.0 : __drcp_rn(r2);
    const double s2 = sig2 * ir2;
    const double s6 = s2 * s2 * s2;
    const double t = s6 - 1.0;
    eb = fma(s6, t, eb);
    const double c = (s2 * s6) * (s6 + t);
    ax = fma(c, dx, ax);
    ay = fma(c, dy, ay);
    az = fma(c, dz, az);
  }
  dd s = dd_two_sum(e.hi, eb);
  e.hi = s.hi;
  e.lo = __dadd_rn(e.lo, s.lo);
}

// ---------------------------------------------------------------------------
// Double-float ("df") arithmetic: a value is hi + lo with two FP32 words
// (~48-bit significand), built from error-free transformations on the FP32
// pipes (TwoSum, and TwoProd via FMA; Dekker 1971, Knuth TAOCP 4.2.2).  The
// mixed path evaluates its polish phase with these: on GB300 one FP64
// instruction issues at ~1/62 the FP32 rate, so ~200 FP32 operations per pair
// cost several times less than ~27 FP64 ones while giving ~1e-14 relative
// accuracy.  Products whose rounded value enters an error term use the _rn
// intrinsics so that no multiply is contracted into a later add.
// ---------------------------------------------------------------------------
struct alignas(16) PosDF { float xh, yh, zh, wh, xl, yl, zl, wl; };

__device__ __forceinline__ ff df_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff df_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff df_sub(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, -b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff df_add_f(ff a, float b) {
  const ff s = ff_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff df_mul(ff a, ff b) {
  const ff p = df_two_prod(a.hi, b.hi);
  const float e = fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, p.lo));
  return df_fast_two_sum(p.hi, e);
}
__device__ __forceinline__ ff df_sqr(ff a) {
  const ff p = df_two_prod(a.hi, a.hi);
  return df_fast_two_sum(p.hi, fmaf(__fmul_rn(2.f, a.hi), a.lo, p.lo));
}
// 1 / a: FP32 reciprocal estimate refined by one Newton step in df,
// w = r + r (1 - a r); relative error ~ (rel. error of r)^2 + 2^-47
__device__ __forceinline__ ff df_rcp(ff a) {
  const float r = rcp_approx(a.hi);
  const ff p = df_two_prod(a.hi, r);
  float t = __fsub_rn(__fsub_rn(1.f, p.hi), p.lo);
  t = fmaf(-a.lo, r, t);
  return df_fast_two_sum(r, __fmul_rn(r, t));
}
__device__ __forceinline__ ff df_from_double(double x) {
  const float h = (float)x;
  return ff{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// |d|^2 of a double-float vector with one renormalisation: the high squares
// exactly (TwoProd by FMA), summed by two TwoSums, and every low-order part
// (their rounding errors, 2 hi lo, the TwoProd errors) gathered in one FP32
// word.  Dropped: lo^2 and the roundings of the low word, ~2^-47 relative.
__device__ __forceinline__ ff df_norm2(ff x, ff y, ff z) {
  const float px = __fmul_rn(x.hi, x.hi), py = __fmul_rn(y.hi, y.hi), pz = __fmul_rn(z.hi, z.hi);
  const float ex = fmaf(x.hi, x.hi, -px), ey = fmaf(y.hi, y.hi, -py), ez = fmaf(z.hi, z.hi, -pz);
  const ff s1 = ff_two_sum(px, py);
  const ff s2 = ff_two_sum(s1.hi, pz);
  float lo = __fadd_rn(__fadd_rn(s1.lo, s2.lo), __fadd_rn(__fadd_rn(ex, ey), ez));
  lo = fmaf(__fadd_rn(x.hi, x.hi), x.lo, lo);
  lo = fmaf(__fadd_rn(y.hi, y.hi), y.lo, lo);
  lo = fmaf(__fadd_rn(z.hi, z.hi), z.lo, lo);
  return df_fast_two_sum(s2.hi, lo);
}

// s += v for a running double-float sum: TwoSum of the high words, every
// rounding error and low word gathered in s.lo (Ogita, Rump and Oishi 2005,
// Sum2); s.lo is renormalised where the sum is stored
__device__ __forceinline__ void df_acc(ff& s, ff v) {
  const ff t = ff_two_sum(s.hi, v.hi);
  s.hi = t.hi;
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, v.lo));
}

// sqrt(a) in double-float (Karp and Markstein, ACM TOMS 1997): y ~ 1/sqrt(a)
// in FP32, s = a y, and one correction s + y (a - s^2) / 2 with a - s^2
// formed exactly (TwoProd); ~2^-46 relative.  a = 0 gives 0.
__device__ __forceinline__ ff df_sqrt(ff a) {
  if (!(a.hi > 0.f)) return ff{0.f, 0.f};
  const float y = rsqrtf(a.hi);
  const float s = __fmul_rn(a.hi, y);
  const ff p = df_two_prod(s, s);
  const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
  return df_fast_two_sum(s, __fmul_rn(__fmul_rn(res, y), 0.5f));
}

// e^x in double-float.  Argument reduction x = k ln 2 + r, k = rint(x / ln 2),
// with ln 2 split into three FP32 words of which the first has 16 bits (so
// k ln2_1 is exact for |k| < 256); then e^r = (e^(r/32))^32, e^(r/32) by its
// Taylor series to degree 7 in double-float Horner form (|r/32| <= 0.0109:
// the first dropped term is below 2^-58), five squarings (which multiply the
// relative error by 32: ~2^-42 in all), and the exact scaling of both words by
// 2^k.  For x < -87.3 (e^x below FP32's normal range) the result is 0.
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kLn2_1 = (float)((double)(long long)(kLn2 * 65536.0) / 65536.0);
constexpr float kLn2_2 = (float)(kLn2 - (double)kLn2_1);
constexpr float kLn2_3 = (float)(kLn2 - (double)kLn2_1 - (double)kLn2_2);
// 1/k! as double-float words (high: the FP32 rounding, low: the FP32
// rounding of the rest), formed at compile time
constexpr float df_hi(double c) { return (float)c; }
constexpr float df_lo(double c) { return (float)(c - (double)(float)c); }
constexpr float kF3h = df_hi(1.0 / 6), kF3l = df_lo(1.0 / 6);
constexpr float kF4h = df_hi(1.0 / 24), kF4l = df_lo(1.0 / 24);
constexpr float kF5h = df_hi(1.0 / 120), kF5l = df_lo(1.0 / 120);
constexpr float kF6h = df_hi(1.0 / 720), kF6l = df_lo(1.0 / 720);
constexpr float kF7h = df_hi(1.0 / 5040), kF7l = df_lo(1.0 / 5040);
__device__ __forceinline__ ff df_exp(ff x) {
  if (x.hi < -87.3f) return ff{0.f, 0.f};
  const float k = rintf(__fmul_rn(x.hi, 1.44269504f));
  ff r = df_add_f(x, -__fmul_rn(k, kLn2_1));            // k ln2_1 exact
  r = df_sub(r, df_two_prod(k, kLn2_2));
  r = df_add_f(r, -__fmul_rn(k, kLn2_3));
  r.hi *= 0.03125f;                                      // r / 32, exact
  r.lo *= 0.03125f;
  ff p{kF7h, kF7l};
  p = df_add(df_mul(p, r), ff{kF6h, kF6l});
  p = df_add(df_mul(p, r), ff{kF5h, kF5l});
  p = df_add(df_mul(p, r), ff{kF4h, kF4l});
  p = df_add(df_mul(p, r), ff{kF3h, kF3l});
  p = df_add(df_mul(p, r), ff{0.5f, 0.f});
  p = df_add_f(df_mul(p, r), 1.f);
  p = df_add_f(df_mul(p, r), 1.f);
#pragma unroll
  for (int i = 0; i < 5; ++i) p = df_sqr(p);
  const float sc = __int_as_float(((int)k + 127) << 23);   // 2^k, k in [-126, 127]
  return ff{p.hi * sc, p.lo * sc};
}

// Morse pair term in double-float on coordinates scaled by 1/re: with
// e = exp(rho (1 - r)), v = e (e - 1) (x_i - x_j) / r and e_pair = e (e - 2)
// (+inf for coincident atoms).  rho is the double-float range parameter.
__device__ __forceinline__ void pair_term_morse_df(const PosDF& a, const PosDF& b, ff rho,
                                                   ff& vx, ff& vy, ff& vz, ff& e) {
  const ff dx = df_sub(ff{a.xh, a.xl}, ff{b.xh, b.xl});
  const ff dy = df_sub(ff{a.yh, a.yl}, ff{b.yh, b.yl});
  const ff dz = df_sub(ff{a.zh, a.zl}, ff{b.zh, b.zl});
  const ff r2 = df_norm2(dx, dy, dz);
  const ff r = df_sqrt(r2);
  const ff ex = df_exp(df_sub(rho, df_mul(rho, r)));
  e = r2.hi > 0.f ? df_mul(ex, df_add_f(ex, -2.f)) : ff{__int_as_float(0x7f800000), 0.f};
  const ff c = df_mul(df_mul(ex, df_add_f(ex, -1.f)), df_rcp(r));
  vx = df_mul(c, dx); vy = df_mul(c, dy); vz = df_mul(c, dz);
}

// One row of the pair sum in df arithmetic, coordinates pre-scaled by
// 1/sigma (so s2 = 1/r^2).  Accumulates acc_i = sum_j s2 s6 (2 s6 - 1) d_ij
// and e_i = sum_j s6 (s6 - 1), both as df.
__device__ __forceinline__ void pair_row_df(int n, int i, ff px, ff py, ff pz,
                                            const PosDF* __restrict__ pos,
                                            ff& ax, ff& ay, ff& az, ff& e) {
  ax = ff{0.f, 0.f}; ay = ff{0.f, 0.f}; az = ff{0.f, 0.f};
#pragma unroll 2
  for (int j = 0; j < n; ++j) {
    const PosDF q = pos[j];
    const ff dx = df_sub(px, ff{q.xh, q.xl});
    const ff dy = df_sub(py, ff{q.yh, q.yl});
    const ff dz = df_sub(pz, ff{q.zh, q.zl});
    const ff r2 = df_norm2(dx, dy, dz);
    ff s2 = df_rcp(r2);
    if (j == i) s2 = ff{0.f, 0.f};
    const ff s6 = df_mul(df_sqr(s2), s2);
    const ff t = df_add_f(s6, -1.f);
    df_acc(e, df_mul(s6, t));
    const ff c = df_mul(df_mul(s2, s6), df_add(s6, t));
    df_acc(ax, df_mul(c, dx));
    df_acc(ay, df_mul(c, dy));
    df_acc(az, df_mul(c, dz));
  }
}

// ---------------------------------------------------------------------------
// Half-pair evaluation (FP64 and double-float): each unordered pair i < j is
// computed once, by thread (p mod T) of the team, p the pair's index in
// row-major order of the upper triangle; its vector v_p = c_ij (x_i - x_j)
// goes to a shared buffer, and after a barrier the thread owning atom i sums
// +v over j > i and -v over j < i.  Every pair costs one evaluation instead
// of two (the one-sided loop visits it from both atoms) and the work splits
// evenly over the team whatever N is -- for N = 38 on a warp, 22 pairs per
// thread instead of 74.  Deterministic: fixed pair order, fixed sum order.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int n_pairs(int n) { return n * (n - 1) / 2; }

// index of pair (i, j), i < j, in the row-major upper triangle
__device__ __forceinline__ int pair_index(int n, int i, int j) {
  return i * (2 * n - i - 1) / 2 + (j - i - 1);
}

// pair_index(n, a, b) = row_base(n, a) + b, so that pair (j, i), j < i, sits at
// row_base(n, j) + i and pair (i, j), j > i, at row_base(n, i) + j;
// row_base(n, j + 1) = row_base(n, j) + n - j - 2, row_base(n, 0) = -1
__device__ __forceinline__ int row_base(int n, int i) {
  return i * (2 * n - i - 1) / 2 - i - 1;
}

// first pair (i, j) of thread `rank` (p = rank); -1 if none
__device__ __forceinline__ void pair_start(int n, int p, int& i, int& j) {
  i = 0;
  int row = n - 1;
  while (row > 0 && p >= row) { p -= row; ++i; --row; }
  j = row > 0 ? i + 1 + p : -1;
}
// advance (i, j) by `step` pairs
__device__ __forceinline__ void pair_advance(int n, int step, int& i, int& j) {
  j += step;
  while (i < n - 1 && j >= n) {
    j -= n;         // j - n = offset past the row end
    ++i;
    j += i + 1;     // first column of the next row is i+1
  }
}

// pair term in FP64: v = c (x_i - x_j) with c = s2 s6 (2 s6 - 1), e = s6 (s6 - 1)
__device__ __forceinline__ void pair_term_f64(const PosD& a, const PosD& b, double sig2,
                                              double& vx, double& vy, double& vz, double& e) {
  const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double s2 = sig2 * __drcp_rn(r2);
  const double s6 = s2 * s2 * s2;
  const double t = s6 - 1.0;
  e = s6 * t;
  const double c = (s2 * s6) * (s6 + t);
  vx = c * dx; vy = c * dy; vz = c * dz;
}

// pair term in double-float on coordinates scaled by 1/sigma
__device__ __forceinline__ void pair_term_df(const PosDF& a, const PosDF& b, ff& vx, ff& vy,
                                             ff& vz, ff& e) {
  const ff dx = df_sub(ff{a.xh, a.xl}, ff{b.xh, b.xl});
  const ff dy = df_sub(ff{a.yh, a.yl}, ff{b.yh, b.yl});
  const ff dz = df_sub(ff{a.zh, a.zl}, ff{b.zh, b.zl});
  const ff r2 = df_norm2(dx, dy, dz);
  const ff s2 = df_rcp(r2);
  const ff s6 = df_mul(df_sqr(s2), s2);
  const ff t = df_add_f(s6, -1.f);
  e = df_mul(s6, t);
  const ff c = df_mul(df_mul(s2, s6), df_add(s6, t));
  vx = df_mul(c, dx); vy = df_mul(c, dy); vz = df_mul(c, dz);
}

// ---------------------------------------------------------------------------
// Double-float evaluation of clusters above the half-pair size: each
// unordered pair once, in tiles of 32 x 32 atom blocks (block b = atoms
// 32b .. 32b+31).  Blocks are paired by the circle method -- round r pairs
// block NB-1 with r and (r+t) mod (NB-1) with (r-t) mod (NB-1), NB even
// (a missing block when the count is odd) -- so that within a round every
// block is in exactly one tile.  A warp takes a tile (I, J): lane l keeps
// atom 32I+l, and atom 32J+l's position and reaction rotate one lane per
// step, so after 32 steps every lane has met every atom of J and holds its
// own J atom's reaction again.  Both sides are then added into per-atom
// double-float accumulators acc[c * n + atom] in shared memory: within a
// round no atom is in two tiles and rounds are separated by a barrier, so
// there are no conflicts and the order is fixed.  A last round takes the
// diagonal tiles (pairs inside a block, each once).  Positions are scaled by
// 1/sigma; v = c (x_i - x_j) as in pair_term_df; e accumulates this lane's
// pair energies s6 (s6 - 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ PosDF shfl_pos(const PosDF& q, int src) {
  PosDF r;
  r.xh = __shfl_sync(kFull, q.xh, src); r.yh = __shfl_sync(kFull, q.yh, src);
  r.zh = __shfl_sync(kFull, q.zh, src); r.wh = 0.f;
  r.xl = __shfl_sync(kFull, q.xl, src); r.yl = __shfl_sync(kFull, q.yl, src);
  r.zl = __shfl_sync(kFull, q.zl, src); r.wl = 0.f;
  return r;
}
__device__ __forceinline__ ff shfl_ff(ff v, int src) {
  return ff{__shfl_sync(kFull, v.hi, src), __shfl_sync(kFull, v.lo, src)};
}

template <int T>
__device__ void df_tile_eval(const Team<T>& tm, int n, const PosDF* __restrict__ pos, ff* acc,
                             ff& e) {
  constexpr int W = T / 32;
  const int lane = tm.rank & 31, warp = tm.rank >> 5;
  for (int i = tm.rank; i < 3 * n; i += T) acc[i] = ff{0.f, 0.f};
  tm.sync();
  const int nb = (n + 31) >> 5;
  const int nbe = nb + (nb & 1);
  const PosDF far{0x1p60f, 0x1p60f, 0x1p60f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto tile = [&](int I, int J) {
    const bool diag = I == J;
    const int i = 32 * I + lane;
    const bool vi = i < n;
    const PosDF pi = vi ? pos[i] : far;
    int jl = 32 * J + lane;
    PosDF pj = jl < n ? pos[jl] : far;
    ff fx{0.f, 0.f}, fy{0.f, 0.f}, fz{0.f, 0.f};
    ff hx{0.f, 0.f}, hy{0.f, 0.f}, hz{0.f, 0.f};   // reaction of the rotating J atom
    const int src = (lane + 1) & 31;
    for (int k = 0; k < 32; ++k) {
      const int jk = 32 * J + ((lane + k) & 31);
      bool act = vi && jk < n;
      if (diag) act = act && k >= 1 && (k < 16 || (k == 16 && lane < 16));
      if (__any_sync(kFull, act)) {
        ff vx, vy, vz, ep;
        pair_term_df(pi, pj, vx, vy, vz, ep);
        if (act) {   // cascaded TwoSum (Sum2): one add on each high word's chain
          df_acc(fx, vx); df_acc(fy, vy); df_acc(fz, vz);
          df_acc(hx, ff{-vx.hi, -vx.lo}); df_acc(hy, ff{-vy.hi, -vy.lo});
          df_acc(hz, ff{-vz.hi, -vz.lo});
          df_acc(e, ep);
        }
      }
      pj = shfl_pos(pj, src);
      hx = shfl_ff(hx, src); hy = shfl_ff(hy, src); hz = shfl_ff(hz, src);
    }
    if (diag) {
      fx = df_add(fx, hx); fy = df_add(fy, hy); fz = df_add(fz, hz);
    } else if (jl < n) {
      acc[jl] = df_add(acc[jl], hx);
      acc[n + jl] = df_add(acc[n + jl], hy);
      acc[2 * n + jl] = df_add(acc[2 * n + jl], hz);
    }
    if (vi) {
      acc[i] = df_add(acc[i], fx);
      acc[n + i] = df_add(acc[n + i], fy);
      acc[2 * n + i] = df_add(acc[2 * n + i], fz);
    }
  };
  for (int r = 0; r < nbe - 1; ++r) {
    for (int t = warp; t < nbe / 2; t += W) {
      const int I = t == 0 ? nbe - 1 : (r + t) % (nbe - 1);
      const int J = t == 0 ? r : (r - t + nbe - 1) % (nbe - 1);
      if (I < nb && J < nb) tile(I, J);
    }
    tm.sync();
  }
  for (int b = warp; b < nb; b += W) tile(b, b);
  tm.sync();
}

// FP64 twin of df_tile_eval (clusters above 256 atoms, same circle-method
// rounds of 32 x 32 tiles): pair terms by pair_term_f64 on unscaled
// coordinates, per-atom FP64 accumulators acc[c * n + atom] in the same
// 24-byte-per-atom slot; a lane's pair energies are summed over its tile,
// then added into e with TwoSum.  Each pair once: the FP64 pipe, which bounds
// these evaluations, does ~40% fewer operations than for two one-sided terms.
__device__ __forceinline__ void shfl_posd(PosD& q, int src) {
  q.x = __shfl_sync(kFull, q.x, src);
  q.y = __shfl_sync(kFull, q.y, src);
  q.z = __shfl_sync(kFull, q.z, src);
}

template <int T>
__device__ void d_tile_eval(const Team<T>& tm, int n, const PosD* __restrict__ pos, double sig2,
                            double* acc, dd& e) {
  constexpr int W = T / 32;
  const int lane = tm.rank & 31, warp = tm.rank >> 5;
  for (int i = tm.rank; i < 3 * n; i += T) acc[i] = 0.0;
  tm.sync();
  const int nb = (n + 31) >> 5;
  const int nbe = nb + (nb & 1);
  const PosD far{0x1p300, 0x1p300, 0x1p300, 0.0};
  auto tile = [&](int I, int J) {
    const bool diag = I == J;
    const int i = 32 * I + lane;
    const bool vi = i < n;
    const PosD pi = vi ? pos[i] : far;
    const int jl = 32 * J + lane;
    PosD pj = jl < n ? pos[jl] : far;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    double hx = 0.0, hy = 0.0, hz = 0.0;   // reaction of the rotating J atom
    double eb = 0.0;
    const int src = (lane + 1) & 31;
    for (int k = 0; k < 32; ++k) {
      const int jk = 32 * J + ((lane + k) & 31);
      bool act = vi && jk < n;
      if (diag) act = act && k >= 1 && (k < 16 || (k == 16 && lane < 16));
      if (__any_sync(kFull, act)) {
        double vx, vy, vz, ep;
        pair_term_f64(pi, pj, sig2, vx, vy, vz, ep);
        if (act) {
          fx += vx; fy += vy; fz += vz;
          hx -= vx; hy -= vy; hz -= vz;
          eb += ep;
        }
      }
      shfl_posd(pj, src);
      hx = __shfl_sync(kFull, hx, src);
      hy = __shfl_sync(kFull, hy, src);
      hz = __shfl_sync(kFull, hz, src);
    }
    const dd t = dd_two_sum(e.hi, eb);
    e.hi = t.hi;
    e.lo = __dadd_rn(e.lo, t.lo);
    if (diag) {
      fx += hx; fy += hy; fz += hz;
    } else if (jl < n) {
      acc[jl] += hx;
      acc[n + jl] += hy;
      acc[2 * n + jl] += hz;
    }
    if (vi) {
      acc[i] += fx;
      acc[n + i] += fy;
      acc[2 * n + i] += fz;
    }
  };
  for (int r = 0; r < nbe - 1; ++r) {
    for (int t = warp; t < nbe / 2; t += W) {
      const int I = t == 0 ? nbe - 1 : (r + t) % (nbe - 1);
      const int J = t == 0 ? r : (r - t + nbe - 1) % (nbe - 1);
      if (I < nb && J < nb) tile(I, J);
    }
    tm.sync();
  }
  for (int b = warp; b < nb; b += W) tile(b, b);
  tm.sync();
}

}  // namespace ljd
