// lj_eval.cu -- lj_energy_grad_batched: batched Eq. (1) energy + gradient
// (and the Morse pair potential through the team kernel).
//
// Uniform batches (2..512 atoms): flat layout, one thread per atom, several
// whole candidates per 512-thread CTA.  Uneven batches: one team per
// candidate (a warp for N <= 64), teams stride over the batch.  Either way
// a candidate's coordinates are read from HBM once, staged in shared memory,
// and every thread sums the pair terms of its own atom(s) (one-sided form:
// deterministic, no atomics).
#include "lj_internal.h"
#include "lj_minimize.cuh"
#include "lj_teams.cuh"

namespace {

using namespace ljd;

template <int T, int A, typename X, typename IO, int POT = LJ_POT_LJ>
__global__ void __launch_bounds__(cta_threads_for(T)) eval_kernel(ljh::EvalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int TPC = cta_threads_for(T) / T;
  const int team = threadIdx.x / T;
  Team<T> tm;
  tm.rank = threadIdx.x % T;
  tm.bar = team + 1;
  void* pos;
  long long* word;
  void* hbuf;
  void* hist;
  carve_team<T>(smem + team * team_smem_bytes<T>(a.max_n, false), a.max_n, false, 0, pos, hbuf,
                hist, tm.red, word);
  MinParams p{};
  p.k = a.k;
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  for (long long c = (long long)blockIdx.x * TPC + team; c < a.n_cand;
       c += (long long)gridDim.x * TPC) {
    long long a0;
    int n;
    if (a.uniform_n > 0) {
      a0 = c * a.uniform_n;
      n = a.uniform_n;
    } else {
      a0 = a.off[c];
      n = (int)(a.off[c + 1] - a0);
    }
    if (n > a.max_n || n < 0) {
      if (tm.rank == 0) a.energy[c] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    X x[A][3], g[A][3];
#pragma unroll
    for (int s = 0; s < A; ++s) {
      const int i = tm.rank + s * T;
#pragma unroll
      for (int k = 0; k < 3; ++k) x[s][k] = i < n ? (X)xin[3 * (a0 + i) + k] : (X)0;
    }
    typename Tr<X>::F E;
    typename Tr<X>::S dummy;
    evaluate<T, A, Prec<X, X, X, 0, POT>>(tm, n, x, g, pos, nullptr, p, nullptr, E, dummy);
    if (gout) {
#pragma unroll
      for (int s = 0; s < A; ++s) {
        const int i = tm.rank + s * T;
        if (i < n) {
#pragma unroll
          for (int k = 0; k < 3; ++k) gout[3 * (a0 + i) + k] = (IO)g[s][k];
        }
      }
    }
    if (tm.rank == 0) a.energy[c] = fto_double(E);
  }
}

// Flat layout for uniform batches: one thread per atom, C = floor(512 / N)
// whole candidates per 512-thread CTA, persistent CTAs striding over tiles of
// C candidates.
constexpr int kFlatThreads = 512;

// ---- FP32, one-sided (clusters of more than kRingMaxN atoms) ---------------
// Per tile: the candidates' positions are staged in
// pair-packed records (double-buffered, so one barrier orders both the
// staging and the reuse of the other buffer), the next tile's coordinates are
// already loading while this tile computes, each thread sums the packed FP32
// row of its own atom (one-sided, no atomics, float-float row energies), and
// the per-atom energies are combined in a fixed order: summed in float-float
// by a segmented shuffle tree within each warp, then the (at most S) warp
// segments of a candidate are added in FP64.  That FP64 step is done by the first C
// threads together (one warp for N >= 16), because an FP64 instruction costs
// a warp the same whatever its active lanes.
__host__ __device__ constexpr int flat_segments(int n) { return (n - 1) / 32 + 2; }

__host__ __device__ constexpr size_t flat_f32_buf_bytes(int n, int C) {
  return align16((size_t)C * ((n + 1) / 2) * sizeof(PosF2)) +
         align16((size_t)C * flat_segments(n) * 2 * sizeof(float));
}

template <typename IO>
__global__ void __launch_bounds__(kFlatThreads) eval_flat_f32_kernel(ljh::EvalArgs a, int C) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.uniform_n;
  const int M = (n + 1) >> 1;
  const int S = flat_segments(n);
  const size_t buf = flat_f32_buf_bytes(n, C);
  const size_t pos_bytes = align16((size_t)C * M * sizeof(PosF2));
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int lc = tid / n;              // candidate within the tile
  const int i = tid - lc * n;          // atom within the candidate
  const bool active = lc < C;
  const int seg = (tid >> 5) - ((lc * n) >> 5);   // this warp's segment of the candidate
  const float gs = a.k.gscale_f;
  const bool unit = a.k.sigma == 1.0;
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  const long long stride = (long long)gridDim.x * C;

  long long c0 = (long long)blockIdx.x * C;
  float nx = 0.f, ny = 0.f, nz = 0.f;   // coordinates of this thread's atom in tile c0
  if (active && c0 + lc < a.n_cand) {
    const long long q = 3 * ((c0 + lc) * n + i);
    nx = (float)xin[q]; ny = (float)xin[q + 1]; nz = (float)xin[q + 2];
  }
  for (int t = 0; c0 < a.n_cand; c0 += stride, ++t) {
    unsigned char* base = smem + (t & 1) * buf;
    PosF2* pos2 = reinterpret_cast<PosF2*>(base) + lc * M;
    float* part = reinterpret_cast<float*>(base + pos_bytes);
    const long long c = c0 + lc;
    const bool live = active && c < a.n_cand;
    const float px = nx, py = ny, pz = nz;
    if (live) stage_f32x2(pos2, n, i, px, py, pz);
    // prefetch the next tile's coordinates (consumed one iteration later)
    {
      const long long cn = c + stride;
      if (active && cn < a.n_cand) {
        const long long q = 3 * (cn * n + i);
        nx = (float)xin[q]; ny = (float)xin[q + 1]; nz = (float)xin[q + 2];
      }
    }
    __syncthreads();
    ff e{0.f, 0.f};
    if (live) {
      float bx, by, bz;
      if (unit)
        pair_row_f32x2<false, true>(n, i, px, py, pz, pos2, 1.f, bx, by, bz, e);
      else
        pair_row_f32x2<true, true>(n, i, px, py, pz, pos2, a.k.sig2_f, bx, by, bz, e);
      if (gout) {
        const long long q = 3 * (c * n + i);
        gout[q] = (IO)(gs * bx);
        gout[q + 1] = (IO)(gs * by);
        gout[q + 2] = (IO)(gs * bz);
      }
    }
    // segmented shuffle tree in float-float: lane l adds lane l + o when both
    // hold atoms of the same candidate; segment heads end with their
    // segment's sum
    ff ev = e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const ff v{__shfl_down_sync(kFull, ev.hi, o), __shfl_down_sync(kFull, ev.lo, o)};
      if (lane + o < 32 && i + o < n) ev = ff_add(ev, v);
    }
    if (live && (lane == 0 || i == 0)) {
      part[2 * (lc * S + seg)] = ev.hi;
      part[2 * (lc * S + seg) + 1] = ev.lo;
    }
    __syncthreads();
    if (tid < C && c0 + tid < a.n_cand) {
      const int w0 = (tid * n) >> 5, w1 = (tid * n + n - 1) >> 5;
      double et = 0.0;
      for (int w = 0; w <= w1 - w0; ++w)
        et += (double)part[2 * (tid * S + w)] + (double)part[2 * (tid * S + w) + 1];
      a.energy[c0 + tid] = et * a.k.e2;
    }
  }
}

template <typename IO>
cudaError_t launch_flat_f32(const ljh::EvalArgs& a, cudaStream_t s) {
  const int n = a.uniform_n;
  const int C = kFlatThreads / n;
  const size_t smem = 2 * flat_f32_buf_bytes(n, C);
  auto k = eval_flat_f32_kernel<IO>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFlatThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + C - 1) / C;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, kFlatThreads, smem, s>>>(a, C);
  return cudaGetLastError();
}


// ---- FP32, small clusters: every unordered pair once ("ring" layout) --------
// Atoms are grouped four to a thread: group g holds atoms 4g .. 4g+3 of its
// candidate, NG = ceil(N / 4) groups, and the missing atoms of the last group
// sit at distinct far positions (2^60, 2^61, 3 * 2^60 in every coordinate)
// whose pair terms underflow to exactly zero (r^2 stays finite in FP32).
// Pairs inside a group are taken by its thread (six, in three packed
// operations).  Pairs between groups follow a ring: at shift k = 1 .. H,
// H = floor(NG / 2), the thread of group g meets group (g + k) mod NG -- 16
// pairs in eight packed operations, each of its own atoms (duplicated in both
// lanes) against the partner's (b0, b1) and (b2, b3).  For even NG the groups
// g and g + H meet twice at shift H, so that shift is split: the lower
// thread takes its atoms a0, a1 against all four of the partner, the upper
// thread all four of its own against the partner's a2, a3 -- eight pairs
// each.  Every unordered pair is evaluated exactly once.
//
// A thread keeps its own atoms' forces in registers (one packed accumulator
// per atom, its two lanes added at the end) and hands each shift's reaction
// on the partner group to shared memory (react[k][partner]: one writer per
// slot); after one barrier every thread subtracts the H reactions addressed
// to its group in the fixed order k = 1 .. H.  The pair energies are summed
// in FP32 per shift (16 terms) and folded into a float-float accumulator;
// per candidate they are combined by a segmented float-float shuffle tree and
// a final FP64 sum of the (at most two) warp segments.  Deterministic: fixed
// pair assignment and summation order.
//
// Cost per unordered pair: 19 FP32 lane operations (packed FADD2 / FMUL2 /
// FFMA2) and one MUFU reciprocal, against 32 lane operations for the two
// one-sided terms of the flat kernel above.  Measured on 65,536 jittered LJ38
// minima: CTAs of 64 threads (and 32) beat 128, 256 and 512; capping the
// registers for more resident warps and eight atoms a thread (255 registers,
// half the warps) were both slower.
constexpr int kRingThreads = 64;   // measured: 64 and 32 beat 128 / 256 / 512
constexpr int kRingMaxN = 48;

struct alignas(16) PosF4 { float x[4], y[4], z[4]; };

__host__ __device__ constexpr int ring_groups(int n) { return (n + 3) >> 2; }
__host__ __device__ constexpr size_t ring_pos_bytes(int n, int C) {
  return align16((size_t)C * ring_groups(n) * sizeof(PosF4));
}
__host__ __device__ constexpr size_t ring_react_bytes(int n, int C) {
  return align16((size_t)(ring_groups(n) / 2) * C * ring_groups(n) * sizeof(PosF4));
}
__host__ __device__ constexpr size_t ring_part_bytes(int C) {
  return align16((size_t)C * 2 * 2 * sizeof(float));
}
__host__ __device__ constexpr size_t ring_smem_bytes(int n, int C) {
  return 2 * ring_pos_bytes(n, C) + ring_react_bytes(n, C) + ring_part_bytes(C);
}

struct V2 {
  float2 x, y, z;
};
__device__ __forceinline__ V2 v2_zero() { return V2{f2(0.f), f2(0.f), f2(0.f)}; }
__device__ __forceinline__ V2 v2_dup(float x, float y, float z) { return V2{f2(x), f2(y), f2(z)}; }
__device__ __forceinline__ void v2_add(V2& a, const V2& b) {
  a.x = __fadd2_rn(a.x, b.x); a.y = __fadd2_rn(a.y, b.y); a.z = __fadd2_rn(a.z, b.z);
}

// One packed operation: the two pairs (X.lane0, Y.lane0) and (X.lane1,
// Y.lane1), given NX = -X (negation is exact, so y + (-x) rounds like
// y - x).  With d = y - x, c = s2 s6 (2 s6 - 1), s2 = sigma^2 / r^2:
// fx += c d (force term on x, in units of the gradient scale 24 eps / sigma^2,
// sign of sum_j c (x_j - x_i)), py += c d (the same vector, to be subtracted
// on y), eb += s6 (s6 - 1).
template <bool SIG>
__device__ __forceinline__ void ring_op(const V2& NX, const V2& Y, float sig2, V2& fx, V2& py,
                                        float2& eb) {
  const float2 dx = __fadd2_rn(Y.x, NX.x);
  const float2 dy = __fadd2_rn(Y.y, NX.y);
  const float2 dz = __fadd2_rn(Y.z, NX.z);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float2 s2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
  if constexpr (SIG) s2 = __fmul2_rn(s2, f2(sig2));
  const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
  const float2 t = __fadd2_rn(s6, f2(-1.f));
  eb = __ffma2_rn(s6, t, eb);
  const float2 c = __fmul2_rn(__fmul2_rn(s2, s6), __fadd2_rn(s6, t));
  fx.x = __ffma2_rn(c, dx, fx.x);
  fx.y = __ffma2_rn(c, dy, fx.y);
  fx.z = __ffma2_rn(c, dz, fx.z);
  py.x = __ffma2_rn(c, dx, py.x);
  py.y = __ffma2_rn(c, dy, py.y);
  py.z = __ffma2_rn(c, dz, py.z);
}

template <typename IO>
__device__ __forceinline__ void ring_load(const IO* __restrict__ xin, long long c, int n, int g,
                                          float (&q)[12]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = 4 * g + a;
    if (i < n) {
      const long long o = 3 * (c * n + i);
      q[3 * a] = (float)xin[o];
      q[3 * a + 1] = (float)xin[o + 1];
      q[3 * a + 2] = (float)xin[o + 2];
    } else {
      const float f = kFarAtom * (float)(1 + (i - n));   // 2^60, 2^61, 3 * 2^60
      q[3 * a] = f; q[3 * a + 1] = f; q[3 * a + 2] = f;
    }
  }
}

template <typename IO, bool SIG>
__global__ void __launch_bounds__(kRingThreads) eval_ring_f32_kernel(ljh::EvalArgs a, int C) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.uniform_n;
  const int NG = ring_groups(n);
  const int H = NG >> 1;
  const bool even = (NG & 1) == 0;
  const size_t pb = ring_pos_bytes(n, C);
  PosF4* react = reinterpret_cast<PosF4*>(smem + 2 * pb);
  float* part = reinterpret_cast<float*>(smem + 2 * pb + ring_react_bytes(n, C));
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int lc = tid / NG;             // candidate within the tile
  const int g = tid - lc * NG;         // group within the candidate
  const bool active = lc < C;
  const int seg = (tid >> 5) - ((lc * NG) >> 5);
  const float gs = a.k.gscale_f;
  const float sig2 = a.k.sig2_f;
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  const long long stride = (long long)gridDim.x * C;
  const int slot = lc * NG;            // first slot of this candidate in a tile buffer

  long long c0 = (long long)blockIdx.x * C;
  float q[12];
  if (active && c0 + lc < a.n_cand) ring_load(xin, c0 + lc, n, g, q);
  for (int t = 0; c0 < a.n_cand; c0 += stride, ++t) {
    PosF4* pos = reinterpret_cast<PosF4*>(smem + (t & 1) * pb);
    const long long c = c0 + lc;
    const bool live = active && c < a.n_cand;
    // own atoms, negated and duplicated in both lanes
    const V2 N0 = v2_dup(-q[0], -q[1], -q[2]), N1 = v2_dup(-q[3], -q[4], -q[5]);
    const V2 N2 = v2_dup(-q[6], -q[7], -q[8]), N3 = v2_dup(-q[9], -q[10], -q[11]);
    if (live) {
      PosF4& r = pos[slot + g];
      *reinterpret_cast<float4*>(r.x) = make_float4(q[0], q[3], q[6], q[9]);
      *reinterpret_cast<float4*>(r.y) = make_float4(q[1], q[4], q[7], q[10]);
      *reinterpret_cast<float4*>(r.z) = make_float4(q[2], q[5], q[8], q[11]);
    }
    // pairs inside the group, packed as (a0,a1)(a0,a2), (a0,a3)(a1,a2),
    // (a1,a3)(a2,a3): their operands, formed before q is overwritten
    const V2 Y12{make_float2(q[3], q[6]), make_float2(q[4], q[7]), make_float2(q[5], q[8])};
    const V2 Y32{make_float2(q[9], q[6]), make_float2(q[10], q[7]), make_float2(q[11], q[8])};
    const V2 Y33 = v2_dup(q[9], q[10], q[11]);
    const V2 NX01{make_float2(-q[0], -q[3]), make_float2(-q[1], -q[4]),
                  make_float2(-q[2], -q[5])};
    const V2 NX12{make_float2(-q[3], -q[6]), make_float2(-q[4], -q[7]),
                  make_float2(-q[5], -q[8])};
    {   // prefetch the next tile's coordinates (consumed one iteration later)
      const long long cn = c + stride;
      if (active && cn < a.n_cand) ring_load(xin, cn, n, g, q);
    }
    __syncthreads();
    ff e{0.f, 0.f};
    // own forces: one packed accumulator per atom, its lanes added at the end
    V2 F0 = v2_zero(), F1 = v2_zero(), F2 = v2_zero(), F3 = v2_zero();
    if (live) {
      {
        float2 eb = f2(0.f);
        V2 G12 = v2_zero(), G32 = v2_zero(), G33 = v2_zero(), F01 = v2_zero(), F12 = v2_zero();
        ring_op<SIG>(N0, Y12, sig2, F0, G12, eb);       // (a0,a1) (a0,a2)
        ring_op<SIG>(NX01, Y32, sig2, F01, G32, eb);    // (a0,a3) (a1,a2)
        ring_op<SIG>(NX12, Y33, sig2, F12, G33, eb);    // (a1,a3) (a2,a3)
        // place each lane's force on its atom's accumulator
        F0.x.y += F01.x.x; F0.y.y += F01.y.x; F0.z.y += F01.z.x;
        F1.x.y += F01.x.y; F1.y.y += F01.y.y; F1.z.y += F01.z.y;
        F1.x.x += F12.x.x; F1.y.x += F12.y.x; F1.z.x += F12.z.x;
        F2.x.x += F12.x.y; F2.y.x += F12.y.y; F2.z.x += F12.z.y;
        F1.x.x -= G12.x.x; F1.y.x -= G12.y.x; F1.z.x -= G12.z.x;
        F2.x.y -= G12.x.y; F2.y.y -= G12.y.y; F2.z.y -= G12.z.y;
        F3.x.x -= G32.x.x; F3.y.x -= G32.y.x; F3.z.x -= G32.z.x;
        F2.x.x -= G32.x.y; F2.y.x -= G32.y.y; F2.z.x -= G32.z.y;
        F3.x.y -= G33.x.x + G33.x.y; F3.y.y -= G33.y.x + G33.y.y; F3.z.y -= G33.z.x + G33.z.y;
        e = ff_add_f(e, __fadd_rn(eb.x, eb.y));
      }
      // the ring shifts
      for (int k = 1; k <= H; ++k) {
        int p = g + k;
        if (p >= NG) p -= NG;
        const PosF4& rb = pos[slot + p];
        const float4 bx = *reinterpret_cast<const float4*>(rb.x);
        const float4 by = *reinterpret_cast<const float4*>(rb.y);
        const float4 bz = *reinterpret_cast<const float4*>(rb.z);
        const V2 B01{make_float2(bx.x, bx.y), make_float2(by.x, by.y), make_float2(bz.x, bz.y)};
        const V2 B23{make_float2(bx.z, bx.w), make_float2(by.z, by.w), make_float2(bz.z, bz.w)};
        float2 eb = f2(0.f);
        V2 P01 = v2_zero(), P23 = v2_zero();     // reactions on (b0, b1), (b2, b3)
        if (!(even && k == H)) {
          ring_op<SIG>(N0, B01, sig2, F0, P01, eb);
          ring_op<SIG>(N0, B23, sig2, F0, P23, eb);
          ring_op<SIG>(N1, B01, sig2, F1, P01, eb);
          ring_op<SIG>(N1, B23, sig2, F1, P23, eb);
          ring_op<SIG>(N2, B01, sig2, F2, P01, eb);
          ring_op<SIG>(N2, B23, sig2, F2, P23, eb);
          ring_op<SIG>(N3, B01, sig2, F3, P01, eb);
          ring_op<SIG>(N3, B23, sig2, F3, P23, eb);
        } else {
          // split shift: the lower thread takes a0, a1 x b0..b3, the upper
          // thread a0..a3 x b2, b3 (its partner's upper half)
          const bool lower = g < H;
          const V2 X2 = lower ? N0 : N1, X3 = lower ? N1 : N2, X4 = lower ? N1 : N3;
          const V2 Y13 = lower ? B01 : B23;
          V2 R1 = v2_zero(), R2 = v2_zero(), R3 = v2_zero(), R4 = v2_zero();
          V2 Q1 = v2_zero(), Q2 = v2_zero(), Q3 = v2_zero(), Q4 = v2_zero();
          ring_op<SIG>(N0, Y13, sig2, R1, Q1, eb);
          ring_op<SIG>(X2, B23, sig2, R2, Q2, eb);
          ring_op<SIG>(X3, Y13, sig2, R3, Q3, eb);
          ring_op<SIG>(X4, B23, sig2, R4, Q4, eb);
          v2_add(F0, R1);
          v2_add(P23, Q2);
          v2_add(P23, Q4);
          if (lower) {
            v2_add(F0, R2);
            v2_add(F1, R3);
            v2_add(F1, R4);
            v2_add(P01, Q1);
            v2_add(P01, Q3);
          } else {
            v2_add(F1, R2);
            v2_add(F2, R3);
            v2_add(F3, R4);
            v2_add(P23, Q1);
            v2_add(P23, Q3);
          }
        }
        e = ff_add_f(e, __fadd_rn(eb.x, eb.y));
        PosF4& w = react[(size_t)(k - 1) * C * NG + slot + p];
        *reinterpret_cast<float4*>(w.x) = make_float4(P01.x.x, P01.x.y, P23.x.x, P23.x.y);
        *reinterpret_cast<float4*>(w.y) = make_float4(P01.y.x, P01.y.y, P23.y.x, P23.y.y);
        *reinterpret_cast<float4*>(w.z) = make_float4(P01.z.x, P01.z.y, P23.z.x, P23.z.y);
      }
    }
    // segmented float-float shuffle tree over the candidate's NG threads
    ff ev = e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const ff v{__shfl_down_sync(kFull, ev.hi, o), __shfl_down_sync(kFull, ev.lo, o)};
      if (lane + o < 32 && g + o < NG) ev = ff_add(ev, v);
    }
    if (live && (lane == 0 || g == 0)) {
      part[4 * lc + 2 * seg] = ev.hi;
      part[4 * lc + 2 * seg + 1] = ev.lo;
    }
    __syncthreads();
    if (live && gout) {
      // own forces (lanes added) minus the reactions handed to this group,
      // k = 1 .. H
      float fx[4] = {F0.x.x + F0.x.y, F1.x.x + F1.x.y, F2.x.x + F2.x.y, F3.x.x + F3.x.y};
      float fy[4] = {F0.y.x + F0.y.y, F1.y.x + F1.y.y, F2.y.x + F2.y.y, F3.y.x + F3.y.y};
      float fz[4] = {F0.z.x + F0.z.y, F1.z.x + F1.z.y, F2.z.x + F2.z.y, F3.z.x + F3.z.y};
      for (int k = 1; k <= H; ++k) {
        const PosF4& r = react[(size_t)(k - 1) * C * NG + slot + g];
        const float4 rx = *reinterpret_cast<const float4*>(r.x);
        const float4 ry = *reinterpret_cast<const float4*>(r.y);
        const float4 rz = *reinterpret_cast<const float4*>(r.z);
        fx[0] -= rx.x; fx[1] -= rx.y; fx[2] -= rx.z; fx[3] -= rx.w;
        fy[0] -= ry.x; fy[1] -= ry.y; fy[2] -= ry.z; fy[3] -= ry.w;
        fz[0] -= rz.x; fz[1] -= rz.y; fz[2] -= rz.z; fz[3] -= rz.w;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = 4 * g + j;
        if (i < n) {
          const long long o = 3 * (c * n + i);
          gout[o] = (IO)(gs * fx[j]);
          gout[o + 1] = (IO)(gs * fy[j]);
          gout[o + 2] = (IO)(gs * fz[j]);
        }
      }
    }
    if (tid < C && c0 + tid < a.n_cand) {
      const int w0 = (tid * NG) >> 5, w1 = (tid * NG + NG - 1) >> 5;
      double et = 0.0;
      for (int w = 0; w <= w1 - w0; ++w)
        et += (double)part[4 * tid + 2 * w] + (double)part[4 * tid + 2 * w + 1];
      a.energy[c0 + tid] = et * a.k.e4;
    }
  }
}

template <typename IO>
cudaError_t launch_ring_f32(const ljh::EvalArgs& a, cudaStream_t s) {
  const int n = a.uniform_n;
  const int C = kRingThreads / ring_groups(n);
  const size_t smem = ring_smem_bytes(n, C);
  const bool unit = a.k.sigma == 1.0;
  auto k = unit ? eval_ring_f32_kernel<IO, false> : eval_ring_f32_kernel<IO, true>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRingThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + C - 1) / C;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, kRingThreads, smem, s>>>(a, C);
  return cudaGetLastError();
}

// ---- FP64, small clusters: every unordered pair once --------------------------
// The ring layout of the FP32 kernel above with scalar FP64 arithmetic: four
// atoms a thread, the six pairs inside a group, then H ring shifts of 16
// pairs (the last one split for an even number of groups), each shift's
// reaction on the partner group handed over in shared memory and subtracted
// by its owner in the order k = 1 .. H.  The reciprocal is the correctly
// rounded one; each shift's 16 pair energies are summed in FP64 and folded
// into a double-double accumulator, and a candidate's groups are combined in
// a fixed-order shared-memory sum.  One FP64 evaluation per unordered pair
// instead of two: on GB300 the FP64 pipe, not the issue rate, bounds this
// kernel, so halving its FP64 operations nearly halves its time.
struct alignas(16) PosD4 { double x[4], y[4], z[4]; };

__host__ __device__ constexpr size_t ringd_pos_bytes(int n, int C) {
  return align16((size_t)C * ring_groups(n) * sizeof(PosD4));
}
__host__ __device__ constexpr size_t ringd_react_bytes(int n, int C) {
  return align16((size_t)(ring_groups(n) / 2) * C * ring_groups(n) * sizeof(PosD4));
}
__host__ __device__ constexpr size_t ringd_smem_bytes(int n, int C) {
  return ringd_pos_bytes(n, C) + ringd_react_bytes(n, C) +
         align16((size_t)C * ring_groups(n) * 2 * sizeof(double));
}

// pair (x, y): f += c (y - x) on x, p += c (y - x) to be subtracted on y,
// e += s6 (s6 - 1), c = s2 s6 (2 s6 - 1), s2 = sigma^2 / r^2
__device__ __forceinline__ void ringd_op(double ax, double ay, double az, double bx, double by,
                                         double bz, double sig2, double& fx, double& fy,
                                         double& fz, double& px, double& py, double& pz,
                                         double& e) {
  const double dx = bx - ax, dy = by - ay, dz = bz - az;
  const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double s2 = sig2 * __drcp_rn(r2);
  const double s6 = s2 * s2 * s2;
  const double t = s6 - 1.0;
  e = fma(s6, t, e);
  const double c = (s2 * s6) * (s6 + t);
  fx = fma(c, dx, fx); fy = fma(c, dy, fy); fz = fma(c, dz, fz);
  px = fma(c, dx, px); py = fma(c, dy, py); pz = fma(c, dz, pz);
}

template <typename IO>
__global__ void __launch_bounds__(kRingThreads) eval_ring_f64_kernel(ljh::EvalArgs a, int C) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.uniform_n;
  const int NG = ring_groups(n);
  const int H = NG >> 1;
  const bool even = (NG & 1) == 0;
  PosD4* pos = reinterpret_cast<PosD4*>(smem);
  PosD4* react = reinterpret_cast<PosD4*>(smem + ringd_pos_bytes(n, C));
  double* esum = reinterpret_cast<double*>(smem + ringd_pos_bytes(n, C) +
                                           ringd_react_bytes(n, C));
  const int tid = threadIdx.x;
  const int lc = tid / NG;
  const int g = tid - lc * NG;
  const bool active = lc < C;
  const double sig2 = a.k.sig2;
  const double gs = a.k.gscale;
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  const int slot = lc * NG;
  for (long long c0 = (long long)blockIdx.x * C; c0 < a.n_cand; c0 += (long long)gridDim.x * C) {
    const long long c = c0 + lc;
    const bool live = active && c < a.n_cand;
    double ax[4], ay[4], az[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = 4 * g + j;
      if (live && i < n) {
        const long long o = 3 * (c * n + i);
        ax[j] = (double)xin[o]; ay[j] = (double)xin[o + 1]; az[j] = (double)xin[o + 2];
      } else {
        const double f = 0x1p300 * (double)(1 + (i - n));   // far padding: terms underflow to 0
        ax[j] = f; ay[j] = f; az[j] = f;
      }
    }
    __syncthreads();       // previous tile's readers of pos / react / esum are done
    if (live) {
      PosD4& r = pos[slot + g];
#pragma unroll
      for (int j = 0; j < 4; ++j) { r.x[j] = ax[j]; r.y[j] = ay[j]; r.z[j] = az[j]; }
    }
    __syncthreads();
    double fx[4] = {0, 0, 0, 0}, fy[4] = {0, 0, 0, 0}, fz[4] = {0, 0, 0, 0};
    dd e{0.0, 0.0};
    if (live) {
      double eb = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) {
          double px = 0, py = 0, pz = 0;
          ringd_op(ax[i], ay[i], az[i], ax[j], ay[j], az[j], sig2, fx[i], fy[i], fz[i], px, py,
                   pz, eb);
          fx[j] -= px; fy[j] -= py; fz[j] -= pz;
        }
      {
        const dd t = dd_two_sum(e.hi, eb);
        e.hi = t.hi;
        e.lo = __dadd_rn(e.lo, t.lo);
      }
      for (int k = 1; k <= H; ++k) {
        int p = g + k;
        if (p >= NG) p -= NG;
        const PosD4& rb = pos[slot + p];
        double bx[4], by[4], bz[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) { bx[j] = rb.x[j]; by[j] = rb.y[j]; bz[j] = rb.z[j]; }
        double px[4] = {0, 0, 0, 0}, py[4] = {0, 0, 0, 0}, pz[4] = {0, 0, 0, 0};
        eb = 0.0;
        // split last shift for even NG: lower thread a0, a1 x b0..b3, upper
        // thread a0..a3 x b2, b3
        const bool split = even && k == H;
        const bool lower = g < H;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (split && (lower ? i >= 2 : j < 2)) continue;
            ringd_op(ax[i], ay[i], az[i], bx[j], by[j], bz[j], sig2, fx[i], fy[i], fz[i], px[j],
                     py[j], pz[j], eb);
          }
        const dd t = dd_two_sum(e.hi, eb);
        e.hi = t.hi;
        e.lo = __dadd_rn(e.lo, t.lo);
        PosD4& w = react[(size_t)(k - 1) * C * NG + slot + p];
#pragma unroll
        for (int j = 0; j < 4; ++j) { w.x[j] = px[j]; w.y[j] = py[j]; w.z[j] = pz[j]; }
      }
      esum[2 * (slot + g)] = e.hi;
      esum[2 * (slot + g) + 1] = e.lo;
    }
    __syncthreads();
    if (live && gout) {
      for (int k = 1; k <= H; ++k) {
        const PosD4& r = react[(size_t)(k - 1) * C * NG + slot + g];
#pragma unroll
        for (int j = 0; j < 4; ++j) { fx[j] -= r.x[j]; fy[j] -= r.y[j]; fz[j] -= r.z[j]; }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = 4 * g + j;
        if (i < n) {
          const long long o = 3 * (c * n + i);
          gout[o] = (IO)(gs * fx[j]);
          gout[o + 1] = (IO)(gs * fy[j]);
          gout[o + 2] = (IO)(gs * fz[j]);
        }
      }
    }
    if (live && g == 0) {
      dd s{esum[2 * slot], esum[2 * slot + 1]};
      for (int q = 1; q < NG; ++q) s = dd_add(s, dd{esum[2 * (slot + q)], esum[2 * (slot + q) + 1]});
      a.energy[c] = __dadd_rn(s.hi, s.lo) * a.k.e4;
    }
  }
}

template <typename IO>
cudaError_t launch_ring_f64(const ljh::EvalArgs& a, cudaStream_t s) {
  const int n = a.uniform_n;
  const int C = kRingThreads / ring_groups(n);
  const size_t smem = ringd_smem_bytes(n, C);
  auto k = eval_ring_f64_kernel<IO>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRingThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + C - 1) / C;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, kRingThreads, smem, s>>>(a, C);
  return cudaGetLastError();
}

// ---- FP64 ------------------------------------------------------------------
// Positions staged as 32-byte records, one-sided FP64 rows with a
// double-double energy, per-candidate energies summed by a fixed-order
// shared-memory tree (log2 N steps).
__host__ __device__ constexpr int pow2_ceil(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

template <typename IO>
__global__ void __launch_bounds__(kFlatThreads) eval_flat_f64_kernel(ljh::EvalArgs a, int C) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.uniform_n;
  PosD* pos = reinterpret_cast<PosD*>(smem);
  double* esum = reinterpret_cast<double*>(smem + align16((size_t)C * n * sizeof(PosD)));
  const int tid = threadIdx.x;
  const int lc = tid / n;              // candidate within the CTA
  const int i = tid - lc * n;          // atom within the candidate
  const bool active = lc < C;
  const double sig2 = a.k.sig2;
  const double gscale = a.k.gscale;
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  const int top = pow2_ceil(n) >> 1;
  for (long long c0 = (long long)blockIdx.x * C; c0 < a.n_cand; c0 += (long long)gridDim.x * C) {
    const long long c = c0 + lc;
    const bool live = active && c < a.n_cand;
    const long long a0 = c * n;
    double px = 0, py = 0, pz = 0;
    if (live) {
      px = (double)xin[3 * (a0 + i)];
      py = (double)xin[3 * (a0 + i) + 1];
      pz = (double)xin[3 * (a0 + i) + 2];
      pos[lc * n + i] = PosD{px, py, pz, 0.0};
    }
    __syncthreads();
    if (live) {
      double ax, ay, az;
      dd ed{0.0, 0.0};
      pair_row_f64(n, i, px, py, pz, pos + lc * n, sig2, ax, ay, az, ed);
      if (gout) {
        gout[3 * (a0 + i)] = (IO)(-gscale * ax);
        gout[3 * (a0 + i) + 1] = (IO)(-gscale * ay);
        gout[3 * (a0 + i) + 2] = (IO)(-gscale * az);
      }
      esum[lc * n + i] = ed.hi + ed.lo;
    }
    // fixed-order tree over each candidate's n per-atom energies
    for (int stride = top; stride > 0; stride >>= 1) {
      __syncthreads();
      if (live && i < stride && i + stride < n) esum[lc * n + i] += esum[lc * n + i + stride];
    }
    __syncthreads();
    if (live && i == 0) a.energy[c] = esum[lc * n] * a.k.e2;
  }
}

template <typename IO>
cudaError_t launch_flat_f64(const ljh::EvalArgs& a, cudaStream_t s) {
  const int n = a.uniform_n;
  const int C = kFlatThreads / n;
  const size_t smem = align16((size_t)C * n * sizeof(PosD)) + (size_t)C * n * sizeof(double);
  auto k = eval_flat_f64_kernel<IO>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFlatThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + C - 1) / C;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, kFlatThreads, smem, s>>>(a, C);
  return cudaGetLastError();
}

template <int T, int A, typename X, typename IO, int POT = LJ_POT_LJ>
cudaError_t launch_one(const ljh::EvalArgs& a, cudaStream_t s) {
  constexpr int threads = cta_threads_for(T);
  constexpr int TPC = threads / T;
  const size_t smem = TPC * team_smem_bytes<T>(a.max_n, false);
  auto k = eval_kernel<T, A, X, IO, POT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + TPC - 1) / TPC;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

namespace ljh {

cudaError_t eval_launch(const EvalArgs& a, cudaStream_t s) {
  if (a.k.pot == LJ_POT_MORSE) {
    // Morse: one team per candidate, one-sided rows, any batch layout
    return dispatch_team(a.max_n, [&](auto TT, auto AA) -> cudaError_t {
      constexpr int T = decltype(TT)::value;
      constexpr int A = decltype(AA)::value;
      constexpr int M = LJ_POT_MORSE;
      const bool fp64 = a.prec == LJ_PREC_FP64;
      if (a.xtype == LJ_F32)
        return fp64 ? launch_one<T, A, double, float, M>(a, s) : launch_one<T, A, float, float, M>(a, s);
      return fp64 ? launch_one<T, A, double, double, M>(a, s) : launch_one<T, A, float, double, M>(a, s);
    });
  }
  // uniform batches of 2..512 atoms: flat thread-per-atom layout
  if (a.uniform_n >= 2 && a.uniform_n <= kFlatThreads) {
    const bool fp64 = a.prec == LJ_PREC_FP64;
    if (a.uniform_n <= kRingMaxN) {
      if (fp64)
        return a.xtype == LJ_F32 ? launch_ring_f64<float>(a, s) : launch_ring_f64<double>(a, s);
      return a.xtype == LJ_F32 ? launch_ring_f32<float>(a, s) : launch_ring_f32<double>(a, s);
    }
    if (a.xtype == LJ_F32) return fp64 ? launch_flat_f64<float>(a, s) : launch_flat_f32<float>(a, s);
    return fp64 ? launch_flat_f64<double>(a, s) : launch_flat_f32<double>(a, s);
  }
  return dispatch_team(a.max_n, [&](auto TT, auto AA) -> cudaError_t {
    constexpr int T = decltype(TT)::value;
    constexpr int A = decltype(AA)::value;
    const bool fp64 = a.prec == LJ_PREC_FP64;
    if (a.xtype == LJ_F32) {
      return fp64 ? launch_one<T, A, double, float>(a, s) : launch_one<T, A, float, float>(a, s);
    }
    return fp64 ? launch_one<T, A, double, double>(a, s) : launch_one<T, A, float, double>(a, s);
  });
}

}  // namespace ljh
