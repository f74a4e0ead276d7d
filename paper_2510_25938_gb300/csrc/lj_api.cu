// lj_api.cu -- the C ABI of include/lj_bh.h: context, workspace, argument
// validation and kernel dispatch.  Host code only.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <cuda_runtime.h>

#include "../../include/lj_bh.h"
#include "lj_internal.h"

struct lj_ctx {
  int device = 0;
  int sms = 0;
  void* ws = nullptr;                  // L-BFGS history workspace
  size_t ws_bytes = 0;
  void* aux = nullptr;                 // bucket lists / counters of uneven batches
  size_t aux_bytes = 0;
  bool reserved = false;
  unsigned long long* queue = nullptr; // persistent-kernel work counter
  // size buckets of an uneven batch run side by side: one stream each, forked
  // from and joined back into the caller's stream with events (capturable)
  cudaStream_t bucket_stream[ljh::kMaxBuckets] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[ljh::kMaxBuckets] = {};
  int bh_team = 0;                     // LJ_OPT_BH_TEAM (0 = automatic)
  int lbfgs_team = 0;                  // LJ_OPT_LBFGS_TEAM (0 = automatic)
  int tune_team[ljh::kMaxBuckets] = {};  // lj_ctx_autotune: team per size bucket (0 = none)
  double tune_sg[ljh::kMaxBuckets] = {}; // ... and MIXED switch_gtol per bucket (0 = none)
  int tune_hist[ljh::kMaxBuckets] = {};  // ... history in global memory (1) per bucket
  int tune_df[ljh::kMaxBuckets] = {};    // ... one-sided double-float rows (1) per bucket
  bool tuned[ljh::kMaxBuckets] = {};
  int hist_opt = 0;                    // LJ_OPT_HISTORY
  int df_opt = 0;                      // LJ_OPT_DF_EVAL
  int bh_tune_team = 0;                // lj_ctx_autotune_bh choices
  double bh_tune_sg = 0.0;
  int bh_tune_hist = 0;
  bool bh_tuned = false;
  int f32_handover = 4;                // LJ_OPT_F32_HANDOVER (FP32 ulps of |E|)
  int df_handover = 32;                // LJ_OPT_DF_HANDOVER (2^-48 |E| units)
  std::string last_error;
};

namespace {

// Makes ctx->device current for the scope of one call, then restores.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

lj_status fail(lj_ctx* ctx, lj_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

lj_status cuda_fail(lj_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, LJ_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// history bytes per team slot for a given atom bound (largest team variant
// of that bound, FP64 history) -- used only to size reservations
size_t slot_bytes_bound(int max_n, int m) {
  int T = 32, A = 1;
  if (max_n <= 64) {               // any team choice: T * A <= 128
    return (2 * (size_t)m * 128 * 3 * sizeof(double) + 15) & ~size_t(15);
  }
  if (max_n > 32) A = 2;
  if (max_n > 64) T = 64;
  if (max_n > 128) T = 128;
  if (max_n > 256) T = 256;
  if (max_n > 512) T = 512;
  return (2 * (size_t)m * A * 3 * T * sizeof(double) + 15) & ~size_t(15);
}

lj_status ensure_ws(lj_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return LJ_OK;
  if (ctx->reserved) {
    return fail(ctx, LJ_ERR_NO_WORKSPACE,
                "call needs " + std::to_string(bytes) + " workspace bytes, reserved " +
                    std::to_string(ctx->ws_bytes));
  }
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "workspace cudaMalloc");
  ctx->ws_bytes = bytes;
  return LJ_OK;
}

lj_status ensure_aux(lj_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->aux_bytes) return LJ_OK;
  if (ctx->reserved) {
    return fail(ctx, LJ_ERR_NO_WORKSPACE,
                "call needs " + std::to_string(bytes) + " bucket-list bytes, reserved " +
                    std::to_string(ctx->aux_bytes));
  }
  if (ctx->aux) {
    cudaFree(ctx->aux);
    ctx->aux = nullptr;
    ctx->aux_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->aux, bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bucket-list cudaMalloc");
  ctx->aux_bytes = bytes;
  return LJ_OK;
}

// bytes of the bucket lists for n_cand candidates: counters, queues, lists
size_t aux_bytes_for(int64_t n_cand) {
  return 256 + (size_t)ljh::kMaxBuckets * (size_t)n_cand * sizeof(int);
}

lj_status check_batch(lj_ctx* ctx, const lj_batch* b, int* max_n) {
  if (!b) return fail(ctx, LJ_ERR_INVALID_ARG, "batch is NULL");
  if (b->n_cand < 0) return fail(ctx, LJ_ERR_INVALID_ARG, "n_cand < 0");
  if (b->uniform_n < 0) return fail(ctx, LJ_ERR_INVALID_ARG, "uniform_n < 0");
  if (b->uniform_n > 0) {
    *max_n = b->uniform_n;
  } else {
    if (b->n_cand > 0 && !b->d_atom_offset)
      return fail(ctx, LJ_ERR_INVALID_ARG, "uniform_n == 0 needs d_atom_offset");
    if (b->max_n < 0) return fail(ctx, LJ_ERR_INVALID_ARG, "max_n < 0");
    if (b->d_atom_offset && !aligned(b->d_atom_offset, 8))
      return fail(ctx, LJ_ERR_INVALID_ARG, "d_atom_offset misaligned");
    *max_n = b->max_n;
  }
  if (*max_n > LJ_MAX_ATOMS)
    return fail(ctx, LJ_ERR_UNSUPPORTED,
                "clusters of " + std::to_string(*max_n) + " atoms exceed LJ_MAX_ATOMS");
  if (*max_n < 1) *max_n = 1;
  return LJ_OK;
}

lj_status check_pot(lj_ctx* ctx, int32_t potential, double rho) {
  if (potential != LJ_POT_LJ && potential != LJ_POT_MORSE)
    return fail(ctx, LJ_ERR_INVALID_ARG, "unknown pair potential");
  if (potential == LJ_POT_MORSE && !(rho > 0.0 && rho <= 64.0))
    return fail(ctx, LJ_ERR_INVALID_ARG, "Morse rho must be in (0, 64]");
  return LJ_OK;
}

lj_status check_min(lj_ctx* ctx, const lj_lbfgs_params* p) {
  if (!p) return fail(ctx, LJ_ERR_INVALID_ARG, "params is NULL");
  if (p->m < 1 || p->m > LJ_MAX_M) return fail(ctx, LJ_ERR_INVALID_ARG, "m outside 1..LJ_MAX_M");
  if (!(p->gtol > 0.0)) return fail(ctx, LJ_ERR_INVALID_ARG, "gtol must be > 0");
  if (p->max_iter < 0) return fail(ctx, LJ_ERR_INVALID_ARG, "max_iter < 0");
  if (p->max_ls < 1) return fail(ctx, LJ_ERR_INVALID_ARG, "max_ls < 1");
  if (!(p->c1 > 0.0 && p->c1 < p->c2 && p->c2 < 1.0))
    return fail(ctx, LJ_ERR_INVALID_ARG, "need 0 < c1 < c2 < 1");
  if (!(p->alpha_max > 0.0)) return fail(ctx, LJ_ERR_INVALID_ARG, "alpha_max must be > 0");
  if (p->prec != LJ_PREC_FP64 && p->prec != LJ_PREC_MIXED)
    return fail(ctx, LJ_ERR_INVALID_ARG, "minimisation precision must be FP64 or MIXED");
  if (p->prec == LJ_PREC_MIXED && !(p->switch_gtol >= 0.0))
    return fail(ctx, LJ_ERR_INVALID_ARG, "switch_gtol must be >= 0 (0: automatic)");
  if (!(p->eps > 0.0 && std::isfinite(p->eps) && p->sigma > 0.0 && std::isfinite(p->sigma)))
    return fail(ctx, LJ_ERR_INVALID_ARG, "eps and sigma must be finite and > 0");
  return check_pot(ctx, p->potential, p->rho);
}

// size buckets of uneven batches (upper bounds, atoms); the autotuner keeps one
// team size per bucket
constexpr int kBound[ljh::kMaxBuckets] = {32, 64, 128, 256, 512, 1024};
int bucket_of(int n) {
  int b = 0;
  while (b < ljh::kMaxBuckets - 1 && n > kBound[b]) ++b;
  return b;
}

// switch_gtol = 0 asks for the automatic value: the autotuned one of the
// size bucket holding `bucket_n` atoms, else kDefaultSwitchGtol
constexpr double kDefaultSwitchGtol = 1e-3;

// history placement and double-float evaluation form of a size bucket: the
// option when set, else the autotuned choice (LJ_OPT_HISTORY / LJ_OPT_DF_EVAL)
bool hist_global_for(const lj_ctx* ctx, int bucket) {
  if (ctx->hist_opt == 1) return true;
  if (ctx->hist_opt == 2 || bucket < 0) return false;
  return ctx->tune_hist[bucket] != 0;
}
int df_one_sided_for(const lj_ctx* ctx, int bucket) {
  if (ctx->df_opt == 1) return 1;
  if (ctx->df_opt == 2 || bucket < 0) return 0;
  return ctx->tune_df[bucket];
}

ljh::MinParamsH to_host(const lj_ctx* ctx, const lj_lbfgs_params* p, int bucket_n = 0) {
  ljh::MinParamsH h;
  h.f32_resolution = ctx->f32_handover * 5.9604644775390625e-8;    // ulps of 2^-24
  h.df_resolution = ctx->df_handover * 3.552713678800501e-15;      // units of 2^-48
  h.m = p->m; h.max_iter = p->max_iter; h.max_ls = p->max_ls;
  h.gtol = p->gtol; h.c1 = p->c1; h.c2 = p->c2; h.alpha_max = p->alpha_max;
  h.switch_gtol = p->switch_gtol; h.deadline = p->deadline_cycles;
  if (!(h.switch_gtol > 0.0)) {
    const double t = bucket_n > 0 ? ctx->tune_sg[bucket_of(bucket_n)] : 0.0;
    h.switch_gtol = t > 0.0 ? t : kDefaultSwitchGtol;
  }
  h.k = ljh::make_consts(p->eps, p->sigma, p->potential, p->rho);
  h.df_one_sided = df_one_sided_for(ctx, bucket_n > 0 ? bucket_of(bucket_n) : -1);
  return h;
}

// ---- scratch of lbfgs_minimize_batched_noalloc ----------------------------
// The array lives in device-global memory of every GPU that loads this
// library.  Host code must not use its name as an address: the address is
// looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LJ_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
constexpr size_t kNoallocQueueBytes = 256;   // work-queue counter, padded
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// device address of the scratch array on `dev` (current device), set up once
lj_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return LJ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LJ_ERR_CUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return LJ_OK;
}

}  // namespace

extern "C" {

const char* lj_status_string(lj_status s) {
  switch (s) {
    case LJ_OK: return "LJ_OK";
    case LJ_ERR_INVALID_ARG: return "LJ_ERR_INVALID_ARG";
    case LJ_ERR_CUDA: return "LJ_ERR_CUDA";
    case LJ_ERR_NO_WORKSPACE: return "LJ_ERR_NO_WORKSPACE";
    case LJ_ERR_UNSUPPORTED: return "LJ_ERR_UNSUPPORTED";
  }
  return "LJ_STATUS_UNKNOWN";
}

lj_status lj_ctx_create(lj_ctx** out, int device) {
  if (!out) return LJ_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return LJ_ERR_INVALID_ARG;
  lj_ctx* c = new (std::nothrow) lj_ctx();
  if (!c) return LJ_ERR_CUDA;
  c->device = device;
  DeviceGuard g(device);
  if (!g.ok) { delete c; return LJ_ERR_CUDA; }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->queue, 64) != cudaSuccess) { delete c; return LJ_ERR_CUDA; }
  bool ok = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int b = 0; b < ljh::kMaxBuckets && ok; ++b)
    ok = cudaStreamCreateWithFlags(&c->bucket_stream[b], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->join_ev[b], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) { lj_ctx_destroy(c); return LJ_ERR_CUDA; }
  *out = c;
  return LJ_OK;
}

lj_status lj_ctx_destroy(lj_ctx* ctx) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->queue) cudaFree(ctx->queue);
    for (int b = 0; b < ljh::kMaxBuckets; ++b) {
      if (ctx->bucket_stream[b]) cudaStreamDestroy(ctx->bucket_stream[b]);
      if (ctx->join_ev[b]) cudaEventDestroy(ctx->join_ev[b]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  }
  delete ctx;
  return LJ_OK;
}

lj_status lj_ctx_reserve(lj_ctx* ctx, int64_t max_cand, int32_t max_n, int32_t max_m) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  if (max_cand < 0 || max_n < 0 || max_m < 1 || max_m > LJ_MAX_M)
    return fail(ctx, LJ_ERR_INVALID_ARG, "bad reservation sizes");
  if (max_n > LJ_MAX_ATOMS) return fail(ctx, LJ_ERR_UNSUPPORTED, "max_n > LJ_MAX_ATOMS");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  // persistent launches give whole CTAs of up to 4 teams one history slot each
  const int64_t slots = max_cand < 4 ? 4 : (max_cand + 3) / 4 * 4;
  const size_t bytes = (size_t)slots * slot_bytes_bound(max_n < 1 ? 1 : max_n, max_m);
  ctx->reserved = false;
  lj_status st = ensure_ws(ctx, bytes);
  if (st != LJ_OK) return st;
  st = ensure_aux(ctx, aux_bytes_for(max_cand));
  if (st != LJ_OK) return st;
  ctx->reserved = true;
  return LJ_OK;
}

lj_status lj_ctx_set_option(lj_ctx* ctx, lj_option opt, int64_t value) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  switch (opt) {
    case LJ_OPT_BH_TEAM:
    case LJ_OPT_LBFGS_TEAM:
      if (opt == LJ_OPT_BH_TEAM && value != 0 && value != 32 && value != 64 && value != 128)
        return fail(ctx, LJ_ERR_INVALID_ARG, "BH team size must be 0 (automatic), 32, 64 or 128");
      if (opt == LJ_OPT_LBFGS_TEAM && value != 0 && value != 32 && value != 64 && value != 128 &&
          value != 256 && value != 512)
        return fail(ctx, LJ_ERR_INVALID_ARG, "L-BFGS team size must be 0, 32, 64, 128, 256 or 512");
      (opt == LJ_OPT_BH_TEAM ? ctx->bh_team : ctx->lbfgs_team) = (int)value;
      return LJ_OK;
    case LJ_OPT_F32_HANDOVER:
      if (value < 0 || value > 4096) return fail(ctx, LJ_ERR_INVALID_ARG, "F32 handover 0..4096");
      ctx->f32_handover = value ? (int)value : 4;
      return LJ_OK;
    case LJ_OPT_DF_HANDOVER:
      if (value < 0 || value > 65536) return fail(ctx, LJ_ERR_INVALID_ARG, "DF handover 0..65536");
      ctx->df_handover = value ? (int)value : 32;
      return LJ_OK;
    case LJ_OPT_HISTORY:
      if (value < 0 || value > 2) return fail(ctx, LJ_ERR_INVALID_ARG, "history option 0, 1 or 2");
      ctx->hist_opt = (int)value;
      return LJ_OK;
    case LJ_OPT_DF_EVAL:
      if (value < 0 || value > 2) return fail(ctx, LJ_ERR_INVALID_ARG, "DF evaluation option 0, 1 or 2");
      ctx->df_opt = (int)value;
      return LJ_OK;
  }
  return fail(ctx, LJ_ERR_INVALID_ARG, "unknown option");
}

const char* lj_ctx_last_error(const lj_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "NULL ctx";
}

lj_status lj_energy_grad_batched(lj_ctx* ctx, const lj_batch* batch, lj_precision prec,
                                 lj_dtype xtype, const void* d_x, double* d_energy, void* d_grad,
                                 double eps, double sigma, void* stream) {
  return lj_energy_grad_batched_pot(ctx, batch, prec, xtype, d_x, d_energy, d_grad, LJ_POT_LJ,
                                    eps, sigma, 0.0, stream);
}

lj_status lj_energy_grad_batched_pot(lj_ctx* ctx, const lj_batch* batch, lj_precision prec,
                                     lj_dtype xtype, const void* d_x, double* d_energy,
                                     void* d_grad, int32_t potential, double eps, double sigma,
                                     double rho, void* stream) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  int max_n = 0;
  lj_status st = check_batch(ctx, batch, &max_n);
  if (st != LJ_OK) return st;
  if (prec != LJ_PREC_FP64 && prec != LJ_PREC_FP32 && prec != LJ_PREC_MIXED)
    return fail(ctx, LJ_ERR_INVALID_ARG, "bad precision");
  if (xtype != LJ_F32 && xtype != LJ_F64) return fail(ctx, LJ_ERR_INVALID_ARG, "bad dtype");
  if (!(eps > 0.0 && std::isfinite(eps) && sigma > 0.0 && std::isfinite(sigma)))
    return fail(ctx, LJ_ERR_INVALID_ARG, "eps and sigma must be finite and > 0");
  st = check_pot(ctx, potential, rho);
  if (st != LJ_OK) return st;
  if (batch->n_cand == 0) return LJ_OK;
  if (!d_x || !d_energy) return fail(ctx, LJ_ERR_INVALID_ARG, "d_x and d_energy are required");
  const size_t el = xtype == LJ_F32 ? 4 : 8;
  if (!aligned(d_x, el) || !aligned(d_energy, 8) || (d_grad && !aligned(d_grad, el)))
    return fail(ctx, LJ_ERR_INVALID_ARG, "misaligned pointer");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  ljh::EvalArgs a;
  a.n_cand = batch->n_cand;
  a.uniform_n = batch->uniform_n;
  a.off = batch->d_atom_offset;
  a.max_n = max_n;
  a.xtype = xtype;
  a.prec = prec;
  a.x = d_x;
  a.energy = d_energy;
  a.grad = d_grad;
  a.k = ljh::make_consts(eps, sigma, potential, rho);
  cudaError_t e = ljh::eval_launch(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lj_energy_grad_batched launch");
  return LJ_OK;
}

lj_status lbfgs_minimize_batched(lj_ctx* ctx, const lj_batch* batch, const lj_lbfgs_params* p,
                                 double* d_x, double* d_energy, int32_t* d_status,
                                 int32_t* d_iters, int32_t* d_nevals, lj_stats* d_stats,
                                 void* stream) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  int max_n = 0;
  lj_status st = check_batch(ctx, batch, &max_n);
  if (st != LJ_OK) return st;
  st = check_min(ctx, p);
  if (st != LJ_OK) return st;
  if (batch->n_cand == 0) return LJ_OK;
  if (!d_x || !d_energy) return fail(ctx, LJ_ERR_INVALID_ARG, "d_x and d_energy are required");
  if (!aligned(d_x, 8) || !aligned(d_energy, 8) || (d_status && !aligned(d_status, 4)) ||
      (d_iters && !aligned(d_iters, 4)) || (d_nevals && !aligned(d_nevals, 4)) ||
      (d_stats && !aligned(d_stats, 8)))
    return fail(ctx, LJ_ERR_INVALID_ARG, "misaligned pointer");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  const int mixed = p->prec == LJ_PREC_MIXED;
  auto plan_for = [&](int bound, ljh::Plan* pl) {
    const int team = ctx->lbfgs_team ? ctx->lbfgs_team : ctx->tune_team[bucket_of(bound)];
    const bool hg = hist_global_for(ctx, bucket_of(bound));
    return ljh::lbfgs_plan(mixed, p->potential, bound, p->m, batch->n_cand, ctx->device, team,
                           pl, hg);
  };
  if (batch->uniform_n == 0 && max_n > 32 && batch->n_cand > 1) {
    // Uneven batch spanning several size classes: sort candidates into size
    // buckets on the device and drain each bucket with the team shape made
    // for it (one persistent launch per bucket, counts never leave the GPU).
    int nb = 1;
    while (nb < ljh::kMaxBuckets && kBound[nb - 1] < max_n) ++nb;
    ljh::Buckets bk;
    for (int b = 0; b < ljh::kMaxBuckets; ++b) bk.bound[b] = b < nb - 1 ? kBound[b] : max_n;
    ljh::Plan plans[ljh::kMaxBuckets];
    size_t hist_need = 0, hist_sum = 0;
    size_t hist_off[ljh::kMaxBuckets] = {};
    for (int b = 0; b < nb; ++b) {
      cudaError_t e = plan_for(bk.bound[b], &plans[b]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched plan");
      const size_t hb = ((size_t)plans[b].slots * plans[b].slot_bytes + 255) & ~size_t(255);
      hist_off[b] = hist_sum;
      hist_sum += hb;
      hist_need = std::max(hist_need, hb);
    }
    // Buckets run side by side (their persistent launches share the GPU and
    // overlap each other's tails) when every bucket can have its own history
    // region: always without a reservation, within one otherwise; else one
    // after another in the caller's stream, sharing one region.
    const bool side_by_side = !ctx->reserved || hist_sum <= ctx->ws_bytes;
    st = ensure_ws(ctx, side_by_side ? hist_sum : hist_need);
    if (st != LJ_OK) return st;
    st = ensure_aux(ctx, aux_bytes_for(batch->n_cand));
    if (st != LJ_OK) return st;
    unsigned* counts = static_cast<unsigned*>(ctx->aux);
    unsigned long long* queues = reinterpret_cast<unsigned long long*>(
        static_cast<unsigned char*>(ctx->aux) + 128);
    int* lists = reinterpret_cast<int*>(static_cast<unsigned char*>(ctx->aux) + 256);
    cudaError_t e = ljh::bucketize_launch(batch->d_atom_offset, batch->n_cand, nb, bk, counts,
                                          lists, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched bucketize");
    if (side_by_side) {
      e = cudaEventRecord(ctx->fork_ev, (cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched fork");
    }
    for (int b = 0; b < nb; ++b) {
      ljh::LbfgsArgs a;
      a.n_cand = batch->n_cand;
      a.uniform_n = 0;
      a.off = batch->d_atom_offset;
      a.max_n = bk.bound[b];
      a.p = to_host(ctx, p, bk.bound[b]);
      a.mixed = mixed;
      a.x = d_x;
      a.energy = d_energy;
      a.status = d_status;
      a.iters = d_iters;
      a.nevals = d_nevals;
      a.stats = d_stats;
      a.queue = queues + b;
      a.hist = side_by_side ? static_cast<unsigned char*>(ctx->ws) + hist_off[b] : ctx->ws;
      a.hist_slot_bytes = plans[b].slot_bytes;
      a.hist_on_chip = plans[b].hist_on_chip;
      a.list = lists + (size_t)b * batch->n_cand;
      a.list_count = counts + b;
      if (!side_by_side) {
        e = ljh::lbfgs_launch(a, plans[b], (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched launch");
        continue;
      }
      cudaStream_t sb = ctx->bucket_stream[b];
      e = cudaStreamWaitEvent(sb, ctx->fork_ev, 0);
      if (e == cudaSuccess) e = ljh::lbfgs_launch(a, plans[b], sb);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->join_ev[b], sb);
      if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, ctx->join_ev[b], 0);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched launch");
    }
    return LJ_OK;
  }
  ljh::Plan plan;
  cudaError_t e = plan_for(max_n, &plan);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched plan");
  st = ensure_ws(ctx, (size_t)plan.slots * plan.slot_bytes);
  if (st != LJ_OK) return st;
  ljh::LbfgsArgs a;
  a.n_cand = batch->n_cand;
  a.uniform_n = batch->uniform_n;
  a.off = batch->d_atom_offset;
  a.max_n = max_n;
  a.p = to_host(ctx, p, max_n);
  a.mixed = mixed;
  a.x = d_x;
  a.energy = d_energy;
  a.status = d_status;
  a.iters = d_iters;
  a.nevals = d_nevals;
  a.stats = d_stats;
  a.queue = ctx->queue;
  a.hist = ctx->ws;
  a.hist_slot_bytes = plan.slot_bytes;
  a.hist_on_chip = plan.hist_on_chip;
  e = ljh::lbfgs_launch(a, plan, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbfgs_minimize_batched launch");
  return LJ_OK;
}

lj_status bh_step_batched(lj_ctx* ctx, const lj_bh_state* s, const lj_bh_params* p,
                          const lj_bh_trace* trace, lj_stats* d_stats, void* stream) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  if (!s || !p) return fail(ctx, LJ_ERR_INVALID_ARG, "state and params are required");
  lj_status st = check_min(ctx, &p->min);
  if (st != LJ_OK) return st;
  if (s->n_walkers < 0 || s->n_atoms < 0) return fail(ctx, LJ_ERR_INVALID_ARG, "negative sizes");
  if (p->K < 1 || p->K > LJ_MAX_K) return fail(ctx, LJ_ERR_INVALID_ARG, "K outside 1..LJ_MAX_K");
  if (!(p->kT > 0.0)) return fail(ctx, LJ_ERR_INVALID_ARG, "kT must be > 0");
  if (p->interval < 1) return fail(ctx, LJ_ERR_INVALID_ARG, "interval < 1");
  if (!(p->factor > 0.0 && std::isfinite(p->factor)))
    return fail(ctx, LJ_ERR_INVALID_ARG, "factor must be finite and > 0");
  if (p->n_steps < 0) return fail(ctx, LJ_ERR_INVALID_ARG, "n_steps < 0");
  if (s->n_walkers == 0 || p->n_steps == 0) return LJ_OK;
  if (!s->x_cur || !s->e_cur || !s->x_best || !s->e_best || !s->stepsize || !s->win_accept ||
      !s->n_accept)
    return fail(ctx, LJ_ERR_INVALID_ARG, "every state array is required");
  if (!aligned(s->x_cur, 8) || !aligned(s->x_best, 8) || !aligned(s->e_cur, 8) ||
      !aligned(s->e_best, 8) || !aligned(s->stepsize, 8) || !aligned(s->win_accept, 4) ||
      !aligned(s->n_accept, 4) || (d_stats && !aligned(d_stats, 8)))
    return fail(ctx, LJ_ERR_INVALID_ARG, "misaligned pointer");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  const int mixed = p->min.prec == LJ_PREC_MIXED;
  // team, history placement and switch_gtol: the options when set, else
  // the choices of lj_ctx_autotune_bh
  const int team = ctx->bh_team ? ctx->bh_team : (ctx->bh_tuned ? ctx->bh_tune_team : 0);
  const bool hg = ctx->hist_opt == 1 || (ctx->hist_opt == 0 && ctx->bh_tuned && ctx->bh_tune_hist);
  lj_lbfgs_params minp = p->min;
  if (!(minp.switch_gtol > 0.0) && ctx->bh_tuned && ctx->bh_tune_sg > 0.0)
    minp.switch_gtol = ctx->bh_tune_sg;
  ljh::Plan plan;
  cudaError_t e = ljh::bh_plan(mixed, p->min.potential, s->n_atoms, p->min.m, s->n_walkers, p->K,
                                team, &plan, hg);
  if (e == cudaErrorNotSupported)
    return fail(ctx, LJ_ERR_UNSUPPORTED,
                "bh_step_batched supports clusters of up to 256 atoms in this build");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bh_step_batched plan");
  st = ensure_ws(ctx, (size_t)plan.slots * plan.slot_bytes);
  if (st != LJ_OK) return st;
  ljh::BhArgs a;
  a.n_walkers = s->n_walkers;
  a.n_atoms = s->n_atoms;
  a.x_cur = s->x_cur; a.e_cur = s->e_cur; a.x_best = s->x_best; a.e_best = s->e_best;
  a.stepsize = s->stepsize; a.win_accept = s->win_accept; a.n_accept = s->n_accept;
  a.K = p->K; a.kT = p->kT; a.target_rate = p->target_rate; a.factor = p->factor;
  a.interval = p->interval; a.seed = p->seed; a.step0 = p->step0; a.n_steps = p->n_steps;
  a.walker0 = p->walker0;
  a.p = to_host(ctx, &minp);
  a.mixed = mixed;
  if (trace) {
    a.tr = *trace;
  } else {
    std::memset(&a.tr, 0, sizeof(a.tr));
  }
  a.stats = d_stats;
  a.hist = ctx->ws;
  a.hist_slot_bytes = plan.slot_bytes;
  a.hist_on_chip = plan.hist_on_chip;
  e = ljh::bh_launch(a, plan, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bh_step_batched launch");
  return LJ_OK;
}

}  // extern "C"

namespace {

// team sizes a bucket can take (A = ceil(N / T) <= 2), the synthetic tuning
// batch per bucket, and the MIXED hand-over gradients tried
constexpr int kTuneChoices[ljh::kMaxBuckets][3] = {
    {32, 0, 0}, {32, 64, 128}, {64, 128, 0}, {128, 256, 0}, {256, 512, 0}, {512, 0, 0}};
constexpr int kTuneCand[ljh::kMaxBuckets] = {4096, 4096, 2048, 1024, 512, 304};
constexpr double kSgChoices[3] = {1e-3, 3e-4, 1e-4};

// Device buffers and timing of one autotuning call; restores the ctx's team
// option and reservation on destruction.
struct Tuner {
  lj_ctx* ctx;
  cudaStream_t s;
  void* stream;
  double* x = nullptr;     // working copy minimised by each tuning run
  double* x0 = nullptr;    // the tuning starts
  double* e = nullptr;
  lj_stats* st = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int saved_team, saved_bh_team, saved_hist, saved_df;
  bool saved_reserved, saved_bh_tuned;
  Tuner(lj_ctx* c, void* strm)
      : ctx(c), s((cudaStream_t)strm), stream(strm), saved_team(c->lbfgs_team),
        saved_bh_team(c->bh_team), saved_hist(c->hist_opt), saved_df(c->df_opt),
        saved_reserved(c->reserved), saved_bh_tuned(c->bh_tuned) {
    ctx->reserved = false;                // tuning batches may grow the workspace
    ctx->hist_opt = 2;                    // tuning runs ignore earlier tuned choices
    ctx->df_opt = 2;
  }
  ~Tuner() {
    cudaFree(x); cudaFree(x0); cudaFree(e); cudaFree(st);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ctx->lbfgs_team = saved_team;
    ctx->bh_team = saved_bh_team;
    ctx->hist_opt = saved_hist;
    ctx->df_opt = saved_df;
    ctx->reserved = saved_reserved;
    ctx->bh_tuned = saved_bh_tuned;
  }
  lj_status alloc(size_t coords, int64_t n_cand) {
    if (cudaMalloc(&x, coords * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&x0, coords * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&e, (size_t)n_cand * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&st, sizeof(lj_stats)) != cudaSuccess ||
        cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess)
      return fail(ctx, LJ_ERR_CUDA, "autotune: allocation failed");
    return LJ_OK;
  }
  // converged minimisations per ms of the second of two runs on x0
  lj_status rate(const lj_lbfgs_params& p, int64_t nc, int nt, int team, double* out) {
    ctx->lbfgs_team = team;
    lj_batch bt;
    bt.n_cand = nc; bt.uniform_n = nt; bt.d_atom_offset = nullptr; bt.max_n = nt;
    float ms = 0.f;
    unsigned long long conv = 0;
    for (int rep = 0; rep < 2; ++rep) {       // the first run is a warm-up
      cudaMemcpyAsync(x, x0, (size_t)nc * 3 * nt * sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemsetAsync(st, 0, sizeof(lj_stats), s);
      cudaEventRecord(ev0, s);
      lj_status rc = lbfgs_minimize_batched(ctx, &bt, &p, x, e, nullptr, nullptr, nullptr, st,
                                            stream);
      cudaEventRecord(ev1, s);
      if (rc != LJ_OK) return rc;
      if (cudaEventSynchronize(ev1) != cudaSuccess)
        return fail(ctx, LJ_ERR_CUDA, "autotune: tuning run failed");
      cudaEventElapsedTime(&ms, ev0, ev1);
      lj_stats hs;
      if (cudaMemcpy(&hs, st, sizeof(lj_stats), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, LJ_ERR_CUDA, "autotune: reading statistics failed");
      conv = hs.converged;
    }
    *out = ms > 0.f ? (double)conv / ms : 0.0;
    return LJ_OK;
  }
  // the team size, then (MIXED) the switch_gtol of bucket b on the starts in
  // x0, then the history placement (where shared memory holds it, global
  // memory is tried) and, for MIXED buckets above 256 atoms, one-sided
  // double-float rows against tiles
  lj_status bucket(int b, int64_t nc, int nt, int m, lj_precision prec, int* team, double* sg,
                   int* hist, int* df) {
    lj_lbfgs_params p;
    p.m = m; p.gtol = 1e-6; p.max_iter = 15000; p.max_ls = 20; p.c1 = 1e-3; p.c2 = 0.9;
    p.alpha_max = 1e10; p.prec = prec; p.switch_gtol = kDefaultSwitchGtol;
    p.deadline_cycles = 0; p.eps = 1.0; p.sigma = 1.0; p.potential = LJ_POT_LJ; p.rho = 0.0;
    *team = kTuneChoices[b][0];
    if (kTuneChoices[b][1] != 0) {
      double best = -1.0;
      for (int k = 0; k < 3 && kTuneChoices[b][k]; ++k) {
        double r = 0.0;
        lj_status rc = rate(p, nc, nt, kTuneChoices[b][k], &r);
        if (rc != LJ_OK) return rc;
        if (r > best) { best = r; *team = kTuneChoices[b][k]; }
      }
    }
    *sg = 0.0;
    double best = -1.0;
    if (prec == LJ_PREC_MIXED) {
      for (double v : kSgChoices) {
        p.switch_gtol = v;
        double r = 0.0;
        lj_status rc = rate(p, nc, nt, *team, &r);
        if (rc != LJ_OK) return rc;
        if (r > best) { best = r; *sg = v; }
      }
      p.switch_gtol = *sg;
    } else {
      lj_status rc = rate(p, nc, nt, *team, &best);
      if (rc != LJ_OK) return rc;
    }
    *hist = 0;
    *df = 0;
    ljh::Plan pl;
    cudaError_t e = ljh::lbfgs_plan(prec == LJ_PREC_MIXED, LJ_POT_LJ, nt, m, nc, ctx->device,
                                    *team, &pl, false);
    if (e != cudaSuccess) return fail(ctx, LJ_ERR_CUDA, "autotune: plan failed");
    if (pl.hist_on_chip) {                 // the alternative: history in global memory
      ctx->hist_opt = 1;
      double r = 0.0;
      lj_status rc = rate(p, nc, nt, *team, &r);
      ctx->hist_opt = 2;
      if (rc != LJ_OK) return rc;
      if (r > best) { best = r; *hist = 1; }
    }
    if (prec == LJ_PREC_MIXED && nt > 256) {   // tiles (default) against one-sided rows
      ctx->hist_opt = *hist ? 1 : 2;
      ctx->df_opt = 1;
      double r = 0.0;
      lj_status rc = rate(p, nc, nt, *team, &r);
      ctx->df_opt = 2;
      if (rc != LJ_OK) return rc;
      if (r > best) { best = r; *df = 1; }
    }
    return LJ_OK;
  }
};

lj_status check_tune_args(lj_ctx* ctx, int32_t max_n, int32_t m, lj_precision prec) {
  if (max_n < 2 || m < 1 || m > LJ_MAX_M || (prec != LJ_PREC_FP64 && prec != LJ_PREC_MIXED))
    return fail(ctx, LJ_ERR_INVALID_ARG, "autotune: N >= 2, 1 <= m <= LJ_MAX_M, FP64 or MIXED");
  if (max_n > LJ_MAX_ATOMS) return fail(ctx, LJ_ERR_UNSUPPORTED, "N > LJ_MAX_ATOMS");
  return LJ_OK;
}

}  // namespace

extern "C" {

lj_status lj_ctx_autotune(lj_ctx* ctx, int32_t max_n, int32_t m, lj_precision prec,
                          int32_t* out_team, double* out_switch_gtol, void* stream) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  lj_status rc = check_tune_args(ctx, max_n, m, prec);
  if (rc != LJ_OK) return rc;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  const int nb = bucket_of(max_n) + 1;
  int team[ljh::kMaxBuckets] = {};
  double sg[ljh::kMaxBuckets] = {};
  int hist[ljh::kMaxBuckets] = {}, df[ljh::kMaxBuckets] = {};
  {
    Tuner tu(ctx, stream);
    size_t max_x = 0;
    for (int b = 0; b < nb; ++b) {
      const int nt = std::min(kBound[b], max_n) * 3 / 4 + 1;
      max_x = std::max(max_x, (size_t)kTuneCand[b] * 3 * nt);
    }
    rc = tu.alloc(max_x, 4096);
    for (int b = 0; b < nb && rc == LJ_OK; ++b) {
      // a representative size of the bucket: three quarters of its upper end,
      // cube starts at reduced density 0.3
      const int nt = std::min(kBound[b], max_n) * 3 / 4 + 1;
      if (ljh::tune_starts_launch(tu.x0, kTuneCand[b], nt, std::cbrt(nt / 0.3), 0x5eedULL + b,
                                  tu.s) != cudaSuccess) {
        rc = fail(ctx, LJ_ERR_CUDA, "autotune: start generation failed");
        break;
      }
      rc = tu.bucket(b, kTuneCand[b], nt, m, prec, &team[b], &sg[b], &hist[b], &df[b]);
    }
  }
  if (rc != LJ_OK) return rc;
  for (int b = 0; b < ljh::kMaxBuckets; ++b) {
    ctx->tune_team[b] = b < nb ? team[b] : 0;
    ctx->tune_sg[b] = b < nb ? sg[b] : 0.0;
    ctx->tune_hist[b] = b < nb ? hist[b] : 0;
    ctx->tune_df[b] = b < nb ? df[b] : 0;
    ctx->tuned[b] = b < nb;
    if (out_team) out_team[b] = ctx->tune_team[b];
    if (out_switch_gtol) out_switch_gtol[b] = ctx->tune_sg[b];
  }
  return LJ_OK;
}

lj_status lj_ctx_autotune_batch(lj_ctx* ctx, const lj_batch* batch, const double* d_x, int32_t m,
                                lj_precision prec, int64_t max_sample, int32_t* out_team,
                                double* out_switch_gtol, void* stream) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  if (!batch || !d_x || batch->uniform_n < 1 || batch->n_cand < 1 || max_sample < 1)
    return fail(ctx, LJ_ERR_INVALID_ARG,
                "autotune_batch: a uniform batch (uniform_n >= 1), d_x and max_sample >= 1");
  lj_status rc = check_tune_args(ctx, batch->uniform_n, m, prec);
  if (rc != LJ_OK) return rc;
  if (!aligned(d_x, 8)) return fail(ctx, LJ_ERR_INVALID_ARG, "misaligned pointer");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  const int nt = batch->uniform_n;
  const int b = bucket_of(nt);
  const int64_t nc = std::min<int64_t>(batch->n_cand, max_sample);
  int team = 0, hist = 0, df = 0;
  double sg = 0.0;
  {
    Tuner tu(ctx, stream);
    rc = tu.alloc((size_t)nc * 3 * nt, nc);
    if (rc == LJ_OK &&
        cudaMemcpyAsync(tu.x0, d_x, (size_t)nc * 3 * nt * sizeof(double),
                        cudaMemcpyDeviceToDevice, tu.s) != cudaSuccess)
      rc = fail(ctx, LJ_ERR_CUDA, "autotune_batch: copying the sample failed");
    if (rc == LJ_OK) rc = tu.bucket(b, nc, nt, m, prec, &team, &sg, &hist, &df);
  }
  if (rc != LJ_OK) return rc;
  ctx->tune_team[b] = team;
  ctx->tune_sg[b] = sg;
  ctx->tune_hist[b] = hist;
  ctx->tune_df[b] = df;
  ctx->tuned[b] = true;
  if (out_team) *out_team = team;
  if (out_switch_gtol) *out_switch_gtol = sg;
  return LJ_OK;
}

lj_status lj_ctx_get_tuning(const lj_ctx* ctx, int32_t bucket, lj_tuning* out) {
  if (!ctx || !out || bucket < 0 || bucket > LJ_TUNE_BH) return LJ_ERR_INVALID_ARG;
  if (bucket == LJ_TUNE_BH) {
    out->team = ctx->bh_tune_team;
    out->switch_gtol = ctx->bh_tune_sg;
    out->history_global = ctx->bh_tune_hist;
    out->df_one_sided = 0;
    out->tuned = ctx->bh_tuned ? 1 : 0;
  } else {
    out->team = ctx->tune_team[bucket];
    out->switch_gtol = ctx->tune_sg[bucket];
    out->history_global = ctx->tune_hist[bucket];
    out->df_one_sided = ctx->tune_df[bucket];
    out->tuned = ctx->tuned[bucket] ? 1 : 0;
  }
  return LJ_OK;
}

lj_status lj_ctx_autotune_bh(lj_ctx* ctx, const lj_bh_state* state, const lj_bh_params* p,
                             lj_tuning* out, void* stream) {
  if (!ctx) return LJ_ERR_INVALID_ARG;
  if (!state || !p) return fail(ctx, LJ_ERR_INVALID_ARG, "autotune_bh: state and params");
  if (p->n_steps < 1 || state->n_walkers < 1 || state->n_atoms < 2)
    return fail(ctx, LJ_ERR_INVALID_ARG, "autotune_bh: n_steps >= 1, walkers >= 1, atoms >= 2");
  if (p->min.prec != LJ_PREC_FP64 && p->min.prec != LJ_PREC_MIXED)
    return fail(ctx, LJ_ERR_INVALID_ARG, "autotune_bh: FP64 or MIXED");
  if (!state->x_cur || !state->e_cur || !state->x_best || !state->e_best || !state->stepsize ||
      !state->win_accept || !state->n_accept)
    return fail(ctx, LJ_ERR_INVALID_ARG, "autotune_bh: every state array is required");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, LJ_ERR_CUDA, "cudaSetDevice failed");
  const int W = state->n_walkers, n = state->n_atoms;
  const size_t xb = (size_t)W * 3 * n * sizeof(double), sb = (size_t)W * sizeof(double),
               ib = (size_t)W * sizeof(int32_t);
  const bool mixed = p->min.prec == LJ_PREC_MIXED;
  int best_team = 0, best_hist = 0;
  double best_sg = 0.0;
  lj_status rc = LJ_OK;
  {
    Tuner tu(ctx, stream);
    ctx->bh_tuned = false;                       // tuning runs use explicit choices
    // working copies of the walkers (restored before every run)
    lj_bh_state ws = *state;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 2 * xb + 3 * sb + 2 * ib) != cudaSuccess ||
        cudaMalloc(&tu.st, sizeof(lj_stats)) != cudaSuccess ||
        cudaEventCreate(&tu.ev0) != cudaSuccess || cudaEventCreate(&tu.ev1) != cudaSuccess) {
      cudaFree(buf);
      return fail(ctx, LJ_ERR_CUDA, "autotune_bh: allocation failed");
    }
    tu.x = static_cast<double*>(buf);            // freed with the tuner
    unsigned char* q = static_cast<unsigned char*>(buf);
    ws.x_cur = reinterpret_cast<double*>(q); q += xb;
    ws.x_best = reinterpret_cast<double*>(q); q += xb;
    ws.e_cur = reinterpret_cast<double*>(q); q += sb;
    ws.e_best = reinterpret_cast<double*>(q); q += sb;
    ws.stepsize = reinterpret_cast<double*>(q); q += sb;
    ws.win_accept = reinterpret_cast<int32_t*>(q); q += ib;
    ws.n_accept = reinterpret_cast<int32_t*>(q);
    auto rate = [&](int team, double sg, int hist, double* r) -> lj_status {
      ctx->bh_team = team;
      ctx->hist_opt = hist ? 1 : 2;
      lj_bh_params pp = *p;
      if (mixed) pp.min.switch_gtol = sg;
      float ms = 0.f;
      unsigned long long conv = 0;
      for (int rep = 0; rep < 2; ++rep) {        // the first run is a warm-up
        cudaMemcpyAsync(ws.x_cur, state->x_cur, xb, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemcpyAsync(ws.x_best, state->x_best, xb, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemcpyAsync(ws.e_cur, state->e_cur, sb, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemcpyAsync(ws.e_best, state->e_best, sb, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemcpyAsync(ws.stepsize, state->stepsize, sb, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemcpyAsync(ws.win_accept, state->win_accept, ib, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemcpyAsync(ws.n_accept, state->n_accept, ib, cudaMemcpyDeviceToDevice, tu.s);
        cudaMemsetAsync(tu.st, 0, sizeof(lj_stats), tu.s);
        cudaEventRecord(tu.ev0, tu.s);
        lj_status st = bh_step_batched(ctx, &ws, &pp, nullptr, tu.st, stream);
        cudaEventRecord(tu.ev1, tu.s);
        if (st != LJ_OK) return st;
        if (cudaEventSynchronize(tu.ev1) != cudaSuccess)
          return fail(ctx, LJ_ERR_CUDA, "autotune_bh: tuning run failed");
        cudaEventElapsedTime(&ms, tu.ev0, tu.ev1);
        lj_stats hs;
        if (cudaMemcpy(&hs, tu.st, sizeof(lj_stats), cudaMemcpyDeviceToHost) != cudaSuccess)
          return fail(ctx, LJ_ERR_CUDA, "autotune_bh: reading statistics failed");
        conv = hs.converged;
      }
      *r = ms > 0.f ? (double)conv / ms : 0.0;
      return LJ_OK;
    };
    const double sg0 = p->min.switch_gtol > 0.0 ? p->min.switch_gtol : kDefaultSwitchGtol;
    double best = -1.0;
    // threads per candidate (the kernel's choices for up to 64 atoms)
    const int teams[3] = {32, 64, 128};
    const int nteam = n <= 64 ? 3 : 1;
    for (int t = 0; t < nteam && rc == LJ_OK; ++t) {
      const int team = n <= 64 ? teams[t] : 0;
      double r = 0.0;
      rc = rate(team, sg0, 0, &r);
      if (rc == LJ_OK && r > best) { best = r; best_team = team; }
    }
    best_sg = mixed ? sg0 : 0.0;
    if (mixed) {
      for (int v = 0; v < 3 && rc == LJ_OK; ++v) {
        if (kSgChoices[v] == sg0) continue;
        double r = 0.0;
        rc = rate(best_team, kSgChoices[v], 0, &r);
        if (rc == LJ_OK && r > best) { best = r; best_sg = kSgChoices[v]; }
      }
    }
    if (rc == LJ_OK) {                            // history in global memory
      ljh::Plan pl;
      cudaError_t e = ljh::bh_plan(mixed, p->min.potential, n, p->min.m, W, p->K, best_team, &pl,
                                   false);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "autotune_bh plan");
      if (rc == LJ_OK && pl.hist_on_chip) {
        double r = 0.0;
        rc = rate(best_team, best_sg, 1, &r);
        if (rc == LJ_OK && r > best) { best = r; best_hist = 1; }
      }
    }
  }
  if (rc != LJ_OK) return rc;
  ctx->bh_tune_team = best_team;
  ctx->bh_tune_sg = best_sg;
  ctx->bh_tune_hist = best_hist;
  ctx->bh_tuned = true;
  if (out) lj_ctx_get_tuning(ctx, LJ_TUNE_BH, out);
  return LJ_OK;
}

lj_status lbfgs_minimize_batched_noalloc(const lj_batch* batch, const lj_lbfgs_params* p,
                                         double* d_x, double* d_energy, int32_t* d_status,
                                         int32_t* d_iters, int32_t* d_nevals, lj_stats* d_stats,
                                         void* stream) {
  int max_n = 0;
  lj_status st = check_batch(nullptr, batch, &max_n);
  if (st != LJ_OK) return st;
  st = check_min(nullptr, p);
  if (st != LJ_OK) return st;
  if (batch->n_cand == 0) return LJ_OK;
  if (!d_x || !d_energy) return LJ_ERR_INVALID_ARG;
  if (!aligned(d_x, 8) || !aligned(d_energy, 8) || (d_status && !aligned(d_status, 4)) ||
      (d_iters && !aligned(d_iters, 4)) || (d_nevals && !aligned(d_nevals, 4)) ||
      (d_stats && !aligned(d_stats, 8)))
    return LJ_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LJ_ERR_CUDA;
  void* scratch = nullptr;
  st = noalloc_scratch(dev, &scratch);
  if (st != LJ_OK) return st;
  const int mixed = p->prec == LJ_PREC_MIXED;
  static const lj_ctx kDefaults;       // default tuning options
  // scratch layout: [0, 128) work-queue counters, [128, 256) bucket counts,
  // then the bucket lists (uneven batches), then off-chip history slots
  unsigned char* base = static_cast<unsigned char*>(scratch);
  unsigned long long* queues = reinterpret_cast<unsigned long long*>(base);
  unsigned* counts = reinterpret_cast<unsigned*>(base + 128);
  const bool bucketed = batch->uniform_n == 0 && max_n > 32 && batch->n_cand > 1;
  const size_t list_bytes =
      bucketed ? (((size_t)ljh::kMaxBuckets * (size_t)batch->n_cand * sizeof(int) + 255) & ~size_t(255))
               : 0;
  if (kNoallocQueueBytes + list_bytes > LJ_NOALLOC_SCRATCH_BYTES) return LJ_ERR_NO_WORKSPACE;
  int* lists = reinterpret_cast<int*>(base + kNoallocQueueBytes);
  unsigned char* hist = base + kNoallocQueueBytes + list_bytes;
  const size_t avail = LJ_NOALLOC_SCRATCH_BYTES - kNoallocQueueBytes - list_bytes;
  // same bucketing as lbfgs_minimize_batched, so both give the same results
  int nb = 1;
  ljh::Buckets bk;
  if (bucketed) {
    while (nb < ljh::kMaxBuckets && kBound[nb - 1] < max_n) ++nb;
    for (int b = 0; b < ljh::kMaxBuckets; ++b) bk.bound[b] = b < nb - 1 ? kBound[b] : max_n;
  } else {
    bk.bound[0] = max_n;
  }
  ljh::Plan plans[ljh::kMaxBuckets];
  for (int b = 0; b < nb; ++b) {
    cudaError_t e = ljh::lbfgs_plan(mixed, p->potential, bk.bound[b], p->m, batch->n_cand, dev, 0,
                                    &plans[b]);
    if (e != cudaSuccess) return LJ_ERR_CUDA;
    if (!plans[b].hist_on_chip) {
      // launch only as many teams as the scratch holds history slots for
      const int64_t cap = (int64_t)(avail / plans[b].slot_bytes) / plans[b].teams_per_cta;
      if (cap < 1) return LJ_ERR_NO_WORKSPACE;
      if (plans[b].grid > cap) plans[b].grid = (int)cap;
      plans[b].slots = (int64_t)plans[b].grid * plans[b].teams_per_cta;
    }
  }
  if (bucketed) {
    cudaError_t e = ljh::bucketize_launch(batch->d_atom_offset, batch->n_cand, nb, bk, counts,
                                          lists, (cudaStream_t)stream);
    if (e != cudaSuccess) return LJ_ERR_CUDA;
  }
  for (int b = 0; b < nb; ++b) {
    ljh::LbfgsArgs a;
    a.n_cand = batch->n_cand;
    a.uniform_n = batch->uniform_n;
    a.off = batch->d_atom_offset;
    a.max_n = bk.bound[b];
    a.p = to_host(&kDefaults, p, bk.bound[b]);
    a.mixed = mixed;
    a.x = d_x;
    a.energy = d_energy;
    a.status = d_status;
    a.iters = d_iters;
    a.nevals = d_nevals;
    a.stats = d_stats;
    a.queue = queues + b;
    a.hist = hist;
    a.hist_slot_bytes = plans[b].slot_bytes;
    a.hist_on_chip = plans[b].hist_on_chip;
    if (bucketed) {
      a.list = lists + (size_t)b * batch->n_cand;
      a.list_count = counts + b;
    }
    cudaError_t e = ljh::lbfgs_launch(a, plans[b], (cudaStream_t)stream);
    if (e != cudaSuccess) return LJ_ERR_CUDA;
  }
  return LJ_OK;
}

}  // extern "C"
