// lj_teams.cuh -- team-size variants and per-team shared-memory carving,
// shared by the kernel translation units.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include "lj_device.cuh"

namespace ljd {

// Team size T and atom slots per thread A for clusters of up to max_n atoms.
// Thread `rank` owns atoms rank + a*T, a < A.
template <class F>
__host__ cudaError_t dispatch_team(int max_n, F&& f) {
  using std::integral_constant;
  if (max_n <= 32) return f(integral_constant<int, 32>{}, integral_constant<int, 1>{});
  if (max_n <= 64) return f(integral_constant<int, 32>{}, integral_constant<int, 2>{});
  if (max_n <= 128) return f(integral_constant<int, 64>{}, integral_constant<int, 2>{});
  if (max_n <= 256) return f(integral_constant<int, 128>{}, integral_constant<int, 2>{});
  if (max_n <= 512) return f(integral_constant<int, 256>{}, integral_constant<int, 2>{});
  if (max_n <= 1024) return f(integral_constant<int, 512>{}, integral_constant<int, 2>{});
  return cudaErrorInvalidValue;
}

__host__ __device__ constexpr int cta_threads_for(int T) { return T < 128 ? 128 : T; }

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Half-pair buffers (24 bytes per pair) are used for clusters of up to
// kHalfMaxN atoms; teams for more than kTileMinN atoms hold the
// double-float tile accumulators (24 bytes per atom) in the same slot; in
// between, double-float evaluations are one-sided (measured: with 3 to 8
// atom blocks a tile round leaves warps idle).
constexpr int kHalfMaxN = 64;
constexpr int kTileMinN = 256;

__host__ __device__ constexpr size_t half_bytes(int max_n, bool half) {
  return !half ? 0
         : max_n <= kHalfMaxN ? align16((size_t)24 * (max_n * (max_n - 1) / 2))
         : max_n > kTileMinN  ? align16((size_t)24 * max_n)
                              : 0;
}

// per-team shared bytes: positions (32-byte records; the FP32 phase uses the
// first half of the same buffer), the optional half-pair buffer, the optional
// L-BFGS history (hist_bytes > 0: kept on chip instead of in the workspace),
// cross-warp reduction scratch (double-buffered), one word
template <int T>
__host__ __device__ constexpr size_t team_smem_bytes(int max_n, bool half, size_t hist_bytes = 0) {
  return align16((size_t)max_n * sizeof(PosD)) + half_bytes(max_n, half) + align16(hist_bytes) +
         (T > 32 ? 2 * 8 * (T / 32) * sizeof(double) : 0) + 16;
}

template <int T>
__device__ __forceinline__ void carve_team(unsigned char* base, int max_n, bool half,
                                           size_t hist_bytes, void*& pos, void*& hbuf,
                                           void*& hist, double*& red, long long*& word) {
  pos = base;
  unsigned char* p = base + align16((size_t)max_n * sizeof(PosD));
  const size_t hb = half_bytes(max_n, half);
  hbuf = hb ? static_cast<void*>(p) : nullptr;
  p += hb;
  hist = hist_bytes ? static_cast<void*>(p) : nullptr;
  p += align16(hist_bytes);
  red = reinterpret_cast<double*>(p);
  p += (T > 32 ? 2 * 8 * (T / 32) * sizeof(double) : 0);
  word = reinterpret_cast<long long*>(p);
}

// History goes on chip when a CTA's shared memory stays within this budget.
constexpr size_t kSmemBudget = 100 * 1024;

}  // namespace ljd
