// lj_eval.cu -- lj_energy_grad_batched: batched Eq. (1) energy + gradient.
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

template <int T, int A, typename X, typename IO>
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
    evaluate<T, A, Prec<X, X, X, 0>>(tm, n, x, g, pos, nullptr, p, nullptr, E, dummy);
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

// ---- FP32 ------------------------------------------------------------------
// Per tile: the candidates' positions are staged in
// pair-packed records (double-buffered, so one barrier orders both the
// staging and the reuse of the other buffer), the next tile's coordinates are
// already loading while this tile computes, each thread sums the packed FP32
// row of its own atom (one-sided, no atomics, FP32 block sums), and the
// per-atom energies are combined in a fixed order: summed by a segmented
// shuffle tree within each warp, then the (at most S) warp segments of a
// candidate are added in FP64.  That FP64 step is done by the first C
// threads together (one warp for N >= 16), because an FP64 instruction costs
// a warp the same whatever its active lanes.
__host__ __device__ constexpr int flat_segments(int n) { return (n - 1) / 32 + 2; }

__host__ __device__ constexpr size_t flat_f32_buf_bytes(int n, int C) {
  return align16((size_t)C * ((n + 1) / 2) * sizeof(PosF2)) +
         align16((size_t)C * flat_segments(n) * sizeof(float));
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
        pair_row_f32x2<false, false>(n, i, px, py, pz, pos2, 1.f, bx, by, bz, e);
      else
        pair_row_f32x2<true, false>(n, i, px, py, pz, pos2, a.k.sig2_f, bx, by, bz, e);
      if (gout) {
        const long long q = 3 * (c * n + i);
        gout[q] = (IO)(gs * bx);
        gout[q + 1] = (IO)(gs * by);
        gout[q + 2] = (IO)(gs * bz);
      }
    }
    // segmented shuffle tree: lane l adds lane l + o when both hold atoms of
    // the same candidate; segment heads end with their segment's sum
    float ev = __fadd_rn(e.hi, e.lo);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float v = __shfl_down_sync(kFull, ev, o);
      if (lane + o < 32 && i + o < n) ev = __fadd_rn(ev, v);
    }
    if (live && (lane == 0 || i == 0)) part[lc * S + seg] = ev;
    __syncthreads();
    if (tid < C && c0 + tid < a.n_cand) {
      const int w0 = (tid * n) >> 5, w1 = (tid * n + n - 1) >> 5;
      double et = (double)part[tid * S];
      for (int w = 1; w <= w1 - w0; ++w) et += (double)part[tid * S + w];
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

template <int T, int A, typename X, typename IO>
cudaError_t launch_one(const ljh::EvalArgs& a, cudaStream_t s) {
  constexpr int threads = cta_threads_for(T);
  constexpr int TPC = threads / T;
  const size_t smem = TPC * team_smem_bytes<T>(a.max_n, false);
  auto k = eval_kernel<T, A, X, IO>;
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
  // uniform batches of 2..512 atoms: flat thread-per-atom layout
  if (a.uniform_n >= 2 && a.uniform_n <= kFlatThreads) {
    const bool fp64 = a.prec == LJ_PREC_FP64;
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
