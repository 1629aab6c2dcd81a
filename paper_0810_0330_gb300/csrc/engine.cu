// engine.cu -- host side of the seed solver: the context, argument checks,
// device memory, the schedule of kernels for each Lanczos / CG step, CUDA
// graphs over runs of steps, status polling, and the C ABI (include/seed.h).
//
// Schedule.  The host knows the step index i of every Lanczos step it issues
// (i advances by one per step while the device recurrence is active), so it
// knows where the Sec. 3 reorthogonalization (when i is a multiple of the
// frequency) falls and issues those kernels only there.  Runs of steps are
// captured once into a CUDA graph per pattern and replayed; all scalars stay
// on the device.  After each run the host copies a small status block to
// pinned memory; it checks the previous run's status while the next run
// executes, so the GPU does not idle on the host.  A run issued after the
// device stopped costs only the launches of kernels that return at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "seed.h"
#include "seed_internal.h"

using namespace seedk;

namespace {

thread_local std::string g_last_error;

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

struct HostStatus {   // pinned, written by cudaMemcpyAsync from SeedState
  int32_t i, active, stop_reason, converged_at;
};

constexpr int kCgBranches = 3;   // concurrent branches of a lockstep CG graph (cg_branches)

}  // namespace

struct seed_ctx {
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t cs = nullptr;           // internal stream (capturable)
  cudaStream_t csb[kCgBranches - 1] = {};   // further branches of the lockstep CG graphs
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kCgBranches - 1] = {};
  cudaEvent_t ev_in = nullptr;
  cudaEvent_t ev_run[2] = {nullptr, nullptr};   // end of a graph run of Lanczos steps, two slots reused
  cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr, t3 = nullptr;
  int kind = 0;                        // 0 = CSR, 1 = Wilson
  seed_dtype dtype = SEED_F64;
  int64_t n = 0;
  size_t esz = 8;                      // element size
  seed_params prm{};
  CsrOp csr{};
  WilsonOp wil{};
  int32_t *nbr = nullptr;

  // seed recurrence
  void *V = nullptr;
  int64_t ldv = 0;
  void *u = nullptr, *f = nullptr, *w = nullptr;
  SeedState *st = nullptr;
  double *alpha_hist = nullptr, *beta_hist = nullptr, *delta_hist = nullptr;
  double2 *eta = nullptr;
  double *partials = nullptr;
  unsigned *tickets = nullptr;
  double2 *Hpart = nullptr, *H = nullptr;
  int rows_per_item = 0, nrb = 0;
  CallArgs *call = nullptr;            // device copy of the caller's X / ldx
  double *colnorm = nullptr;           // scratch norms [kMaxRhs]

  // multi-column work space (grown on demand): R0 / R, P, Q, Wilson temp
  int cap_cols = 0;
  void *R = nullptr, *P = nullptr, *Q = nullptr, *T = nullptr;

  // lockstep CG
  double *cg_d = nullptr;     // 5 * kMaxRhs doubles
  int32_t *cg_i = nullptr;    // 7 * kMaxRhs ints
  int32_t *h_flags = nullptr; // pinned [2][kMaxRhs]
  HostStatus *h_status = nullptr;   // pinned [2]

  // persistent kernels
  int sm_count = 0;
  int pgrid = 0;                       // blocks of a persistent seed launch (0: not available)
  int pgrid_cg = 0;                    // blocks of a persistent CG launch
  unsigned *gsync = nullptr;           // GridSync: count, release, error
  int32_t *h_gerr = nullptr;           // pinned copy of the error flag
  void *f2 = nullptr;                  // second Lanczos-vector buffer (CSR persistent run)
  double *tpart = nullptr;             // per-tile partial sums (persistent Wilson seed run)
  int rgrid_cap[2] = {0, 0};           // most blocks of a reorthogonalizing CSR run, 16 / 32 rows per block
  int scg_cap[2] = {0, 0};             // most blocks of the small-problem CSR CG, 16 / 32 rows per block
  bool allow_small_cg = true;          // the small-problem CSR CG (not on kernel_path 1)
  double *rhpart = nullptr;            // its partial products, 2 x (m_max + 1) x grid doubles
  double2 *Hrows = nullptr;            // FP32 reorthogonalization partials by 4096-row chunks (long vectors)
  int64_t rhpart_grid = 0;             // the grid rhpart was sized for
  bool allow_persistent = true;        // persistent seed runs
  bool allow_persistent_cg = false;    // persistent CG

  // mixed precision: V, u, f, w hold FP32 vectors (vsz bytes per element)
  int precision = 0;
  size_t vsz = 8;
  int64_t nv = 0;                      // length of the Krylov vectors (n, or the tiled FP32 length)
  Layout32 lay{0};                     // FP32 vector layout of the mixed path (tiled for Wilson)
  WilsonOp32 wil32{};
  CsrOp32 csr32{};
  void *op32 = nullptr;                // FP32 copy of the links / matrix values
  void *R32 = nullptr, *P32 = nullptr, *Q32 = nullptr, *T32 = nullptr;
  void *E32 = nullptr;                 // FP32 corrections, cap_cols + 1 columns (column 0 spare)
  CallArgs *call32 = nullptr;          // [0]: seed run (X = E), [1]: mixed CG

  // Sec. 2.3 related right-hand sides: tracked residuals, x_bcg / x_cg, r_bcg, dots and deltas
  void *Rrel = nullptr, *xrel = nullptr, *rrel = nullptr;
  int rel_cap = 0;
  double2 *reldots = nullptr;          // [2 * kMaxRhs]
  void *msX = nullptr, *msR = nullptr; // multiple seeding: solutions and tracked residuals
  int ms_cap = 0;

  // blocked seeding of systems 2..p (seedblock.cu): w_i of the current block,
  // gamma_{i-1} per step, and the flush workspace
  void *Wb = nullptr;
  double *gamma_hist = nullptr;
  BlockBufs blk{};
  TcFlush tcf{};                       // tensor-core flush products (mixed-precision Wilson)
  int *tc_err = nullptr;               // its device error flag

  std::map<std::string, GraphEntry> graphs;
  std::string err;
  seed_stats stats{};
  int last_m = 0;
  bool basis_valid = false;
  bool seeded = false;
  bool timing_project = false;
  bool in_batch = false;               // inside seed_batch_solve (stream ordering done by the batch)
};

namespace {

seed_status fail(seed_ctx *c, seed_status st, const std::string &msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return st;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(ctx, SEED_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

bool is_device_ptr(const void *p, int device) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  if (a.type == cudaMemoryTypeManaged) return true;
  return false;
}

seed_status check_params(seed_ctx *ctx, const seed_params *p) {
  if (!p) return fail(ctx, SEED_EINVAL, "params is NULL");
  if (p->m_max < 1) return fail(ctx, SEED_EINVAL, "m_max must be >= 1");
  if (p->m_max > 1000000) return fail(ctx, SEED_EINVAL, "m_max too large");
  if (p->reorth_freq < 0) return fail(ctx, SEED_EINVAL, "reorth_freq must be >= 0");
  if (p->reorth_passes < 1 || p->reorth_passes > 2) return fail(ctx, SEED_EINVAL, "reorth_passes must be 1 or 2");
  if (p->extra_iters < 0) return fail(ctx, SEED_EINVAL, "extra_iters must be >= 0");
  if (p->maxit_rest < 0 || p->max_restarts < 0) return fail(ctx, SEED_EINVAL, "maxit_rest / max_restarts < 0");
  if (!(p->tol_seed >= 0.0) || !(p->tol_rest >= 0.0) || !(p->breakdown_rel >= 0.0))
    return fail(ctx, SEED_EINVAL, "tolerances must be >= 0");
  if (p->kernel_path < 0 || p->kernel_path > 2) return fail(ctx, SEED_EINVAL, "kernel_path must be 0, 1 or 2");
  if (p->precision < 0 || p->precision > 1) return fail(ctx, SEED_EINVAL, "precision must be 0 or 1");
  if (p->autotune < 0 || p->autotune > 1) return fail(ctx, SEED_EINVAL, "autotune must be 0 or 1");
  if (!(p->reliable_delta >= 0.0 && p->reliable_delta < 1.0))
    return fail(ctx, SEED_EINVAL, "reliable_delta must be in [0, 1)");
  return SEED_OK;
}

// Host-side fault injection (seed_inject_alloc_failure): countdown to the
// device allocation that fails; 0 = disarmed.
std::atomic<int> g_alloc_countdown{0};

bool injected_alloc_failure() {
  int v = g_alloc_countdown.load();
  while (v > 0 && !g_alloc_countdown.compare_exchange_weak(v, v - 1)) {
  }
  return v == 1;
}

template <class Tp>
seed_status dalloc(seed_ctx *ctx, Tp **p, size_t bytes) {
  if (injected_alloc_failure())
    return fail(ctx, SEED_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SEED_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  *p = reinterpret_cast<Tp *>(q);
  return SEED_OK;
}

#define TRY(x)                        \
  do {                                \
    seed_status s_ = (x);             \
    if (s_ != SEED_OK) return s_;     \
  } while (0)

seed_status alloc_common(seed_ctx *ctx) {
  // Krylov vectors: FP64 of length n, or FP32 of length nv (tiled by 32 sites for Wilson)
  const int64_t n = ctx->nv;
  const size_t es = ctx->vsz;
  const int m = ctx->prm.m_max;
  ctx->ldv = (n + 31) / 32 * 32;   // 256-byte aligned columns for complex, 256 B for real
  TRY(dalloc(ctx, &ctx->V, (size_t)ctx->ldv * (m + 1) * es));
  TRY(dalloc(ctx, &ctx->u, n * es));
  TRY(dalloc(ctx, &ctx->f, n * es));
  TRY(dalloc(ctx, &ctx->w, n * es));
  TRY(dalloc(ctx, &ctx->st, sizeof(SeedState)));
  TRY(dalloc(ctx, &ctx->alpha_hist, sizeof(double) * (m + 2)));
  TRY(dalloc(ctx, &ctx->beta_hist, sizeof(double) * (m + 2)));
  TRY(dalloc(ctx, &ctx->delta_hist, sizeof(double) * (m + 2)));
  TRY(dalloc(ctx, &ctx->gamma_hist, sizeof(double) * (m + 2)));
  TRY(dalloc(ctx, &ctx->eta, sizeof(double2) * kMaxRhs));
  TRY(dalloc(ctx, &ctx->call, sizeof(CallArgs) * kCgBranches));   // [b]: branch b of the CG graphs
  TRY(dalloc(ctx, &ctx->colnorm, sizeof(double) * kMaxRhs));
  // block partials: seed dots use up to 5 chunks x vec_blocks(n) x 32; lockstep kernels nc x blocks x 2
  TRY(dalloc(ctx, &ctx->partials, sizeof(double) * kPartials));
  TRY(dalloc(ctx, &ctx->tickets, sizeof(unsigned) * 256));
  // reorthogonalization tiles: ~32 row blocks of >= 256 rows
  int64_t rows = (n + 31) / 32;
  rows = (rows + 255) / 256 * 256;
  if (rows < 256) rows = 256;
  ctx->rows_per_item = (int)rows;
  ctx->nrb = (int)((n + rows - 1) / rows);
  TRY(dalloc(ctx, &ctx->Hpart, sizeof(double2) * (size_t)ctx->nrb * (m + 1) * 2 + 64));
  TRY(dalloc(ctx, &ctx->H, sizeof(double2) * (size_t)(m + 1) * 2));
  // long FP32 vectors: reorthogonalization partials by 4096-row chunks (krylov.cu)
  if (ctx->precision == 1 && n >= 65536)
    TRY(dalloc(ctx, &ctx->Hrows, sizeof(double2) * (size_t)((n + 4095) / 4096) * (m + 1) * 2));
  TRY(dalloc(ctx, &ctx->cg_d, sizeof(double) * kCgDoubles * kMaxRhs));
  TRY(dalloc(ctx, &ctx->cg_i, sizeof(int32_t) * kCgInts * kMaxRhs));
  // call32: [0] seed run (X = E), [1 + b] branch b of the mixed CG graphs
  if (ctx->precision == 1) TRY(dalloc(ctx, &ctx->call32, sizeof(CallArgs) * (1 + kCgBranches)));
  CU(cudaMemsetAsync(ctx->tickets, 0, sizeof(unsigned) * 256, ctx->cs));
  CU(cudaMemsetAsync(ctx->w, 0, n * es, ctx->cs));
  CU(cudaMallocHost(&ctx->h_flags, sizeof(int32_t) * 2 * kMaxRhs));
  CU(cudaMallocHost(&ctx->h_status, sizeof(HostStatus) * 2));
  TRY(dalloc(ctx, &ctx->gsync, sizeof(unsigned) * kGridSyncWords));
  // zeroed here too: the error flag is read after every persistent run, and
  // cudaMalloc memory may hold an earlier allocation's bytes
  CU(cudaMemsetAsync(ctx->gsync, 0, sizeof(unsigned) * kGridSyncWords, ctx->cs));
  TRY(dalloc(ctx, &ctx->f2, n * es));
  TRY(dalloc(ctx, &ctx->tpart, sizeof(double) * (size_t)(12 * ((n / 12 + 31) / 32) + 3)));
  CU(cudaMallocHost(&ctx->h_gerr, sizeof(int32_t) * 2));
  CU(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device));
  int coop = 0;
  CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  ctx->pgrid = coop ? persistent_grid(ctx->kind, ctx->sm_count, false, ctx->precision == 1) : 0;
  ctx->pgrid_cg = coop ? persistent_grid(ctx->kind, ctx->sm_count, true) : 0;
  if (coop && ctx->kind == 0 && ctx->precision == 0)
    for (int q = 0; q < 2; ++q) {
      ctx->rgrid_cap[q] = reorth_run_grid_cap(ctx->sm_count, 16 << q);
      ctx->scg_cap[q] = small_cg_grid_cap(ctx->sm_count, 16 << q);
    }
  return SEED_OK;
}

GridSync grid_sync_bufs(seed_ctx *ctx) {
  GridSync g;
  g.count = ctx->gsync;
  g.release = ctx->gsync + 1;
  g.error = reinterpret_cast<int *>(ctx->gsync + 2);
  g.owners = ctx->gsync + 3;
  g.sm_slots = ctx->gsync + 4;
  return g;
}

seed_status ensure_cols(seed_ctx *ctx, int cols) {
  if (cols <= ctx->cap_cols) return SEED_OK;
  cudaStreamSynchronize(ctx->cs);
  cudaFree(ctx->R); cudaFree(ctx->P); cudaFree(ctx->Q); cudaFree(ctx->T);
  ctx->R = ctx->P = ctx->Q = ctx->T = nullptr;
  cudaFree(ctx->R32); cudaFree(ctx->P32); cudaFree(ctx->Q32); cudaFree(ctx->T32); cudaFree(ctx->E32);
  ctx->R32 = ctx->P32 = ctx->Q32 = ctx->T32 = ctx->E32 = nullptr;
  ctx->cap_cols = 0;
  // graphs captured with the old buffers are stale
  for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
  ctx->graphs.clear();
  const size_t bytes = (size_t)ctx->ldv * cols * ctx->esz;
  TRY(dalloc(ctx, &ctx->R, bytes));
  TRY(dalloc(ctx, &ctx->P, bytes));
  TRY(dalloc(ctx, &ctx->Q, bytes));
  TRY(dalloc(ctx, &ctx->T, bytes));
  if (ctx->precision == 1) {
    const size_t b32 = (size_t)ctx->ldv * cols * ctx->vsz;
    TRY(dalloc(ctx, &ctx->R32, b32));
    TRY(dalloc(ctx, &ctx->P32, b32));
    TRY(dalloc(ctx, &ctx->Q32, b32));
    TRY(dalloc(ctx, &ctx->T32, b32));
    TRY(dalloc(ctx, &ctx->E32, b32 + (size_t)ctx->ldv * ctx->vsz));
  }
  ctx->cap_cols = cols;
  return SEED_OK;
}

// Y = A X on ncols columns (mask: skip columns whose flag is 0).  Returns the kernel count.
int apply_A(seed_ctx *ctx, const void *X, int64_t ldx, void *Y, int64_t ldy, int ncols, const int32_t *mask) {
  if (ctx->kind == 0) {
    launch_csr_spmv(ctx->csr, (const double *)X, ldx, (double *)Y, ldy, ncols, mask, ctx->cs);
    return 1;
  }
  launch_wilson_dslash(ctx->wil, +1, (const double2 *)X, ldx, (double2 *)ctx->T, ctx->ldv, ncols, mask, ctx->cs);
  launch_wilson_dslash(ctx->wil, -1, (const double2 *)ctx->T, ctx->ldv, (double2 *)Y, ldy, ncols, mask, ctx->cs);
  return 2;
}

// Y = A X with the FP32 copy of the operator (mixed precision).  Returns the kernel count.
// tiled: X and Y in the solver's tiled FP32 layout (else the caller's site-major one).
int apply_A32(seed_ctx *ctx, const void *X, int64_t ldx, void *Y, int64_t ldy, int ncols, const int32_t *mask,
              bool tiled = true) {
  if (ctx->kind == 0) {
    launch_csr_spmv32(ctx->csr32, (const float *)X, ldx, (float *)Y, ldy, ncols, mask, ctx->cs);
    return 1;
  }
  launch_wilson_dslash32(ctx->wil32, +1, (const float2 *)X, ldx, (float2 *)ctx->T32, ctx->ldv, ncols, mask, tiled,
                         ctx->cs);
  launch_wilson_dslash32(ctx->wil32, -1, (const float2 *)ctx->T32, ctx->ldv, (float2 *)Y, ldy, ncols, mask, tiled,
                         ctx->cs);
  return 2;
}

template <class T> constexpr bool kLow = std::is_same_v<T, float> || std::is_same_v<T, float2>;

// Blocked seeding (the Sec. 3 seeding of systems 2..p folded into x^2..x^p once per block of
// steps, seedblock.cu) when there are seeded systems and blocks can be long:
// without reorthogonalization or with reorthogonalization every 8 or more steps
// (a block ends at every reorthogonalizing step).
bool blocked_seeding(const seed_ctx *ctx, int nrhs) {
  const int f = ctx->prm.reorth_freq;
  return nrhs >= 2 && (f == 0 || f >= 8);
}

// (each buffer is allocated once; after a failed allocation the next call
// allocates only what is still missing)
// The tensor-core flush serves FP32 complex vectors whose length is a multiple of its 128-element chunk.
bool tc_flush_eligible(const seed_ctx *ctx) {
  return ctx->precision == 1 && ctx->kind == 1 && ctx->nv >= 128 && ctx->nv % 128 == 0;
}

seed_status ensure_block(seed_ctx *ctx) {
  if (ctx->Wb && ctx->blk.Hpart && ctx->blk.G && ctx->blk.Z && (!tc_flush_eligible(ctx) || ctx->tc_err))
    return SEED_OK;
  const BlockBufs lay = block_layout(ctx->nv);
  ctx->blk.nchunk = lay.nchunk;
  ctx->blk.rows = lay.rows;
  ctx->blk.tc = nullptr;
  int chunks = lay.nchunk;
  if (tc_flush_eligible(ctx)) chunks = std::max(chunks, tc_grid(ctx->nv));
  if (!ctx->Wb) TRY(dalloc(ctx, &ctx->Wb, (size_t)ctx->ldv * kSeedBlock * ctx->vsz));
  if (!ctx->blk.Hpart)
    TRY(dalloc(ctx, &ctx->blk.Hpart, sizeof(double2) * (size_t)chunks * kSeedBlock * (kMaxRhs - 1)));
  if (tc_flush_eligible(ctx) && !ctx->tc_err) {
    TRY(dalloc(ctx, (void **)&ctx->tc_err, sizeof(int)));
    CU(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->cs));
  }
  if (!ctx->blk.G) TRY(dalloc(ctx, &ctx->blk.G, sizeof(double2) * (size_t)kSeedBlock * (kMaxRhs - 1)));
  if (!ctx->blk.Z) TRY(dalloc(ctx, &ctx->blk.Z, sizeof(double2) * (size_t)kSeedBlock * (kMaxRhs - 1)));
  return SEED_OK;
}

// E: column 0 of the corrections (system 1); its spare column sits before it
template <class T> T *E_cols(seed_ctx *ctx) { return (T *)ctx->E32 + ctx->ldv; }

template <class T>
SeedBufs<T> seed_bufs(seed_ctx *ctx, int nrhs) {
  SeedBufs<T> b;
  b.n = kLow<T> ? ctx->nv : ctx->n;
  b.nrhs = nrhs;
  b.nblocks = vec_blocks(ctx->n);
  b.V = (T *)ctx->V;
  b.ldv = ctx->ldv;
  b.u = (T *)ctx->u;
  b.f = (T *)ctx->f;
  b.w = (T *)ctx->w;
  b.R0 = (const T *)ctx->R;
  b.ldr = ctx->ldv;
  b.call = ctx->call;
  if constexpr (kLow<T>) {
    b.R0 = (const T *)ctx->R32 + ctx->ldv;   // r_0^2.. (FP32), column 0 holds r_0^1
    b.call = ctx->call32;                    // x^j := FP32 corrections e^j
  }
  b.st = ctx->st;
  b.Wb = (blocked_seeding(ctx, nrhs) && ctx->Wb) ? (T *)ctx->Wb : nullptr;
  b.gamma_hist = ctx->gamma_hist;
  b.alpha_hist = ctx->alpha_hist;
  b.beta_hist = ctx->beta_hist;
  b.delta_hist = ctx->delta_hist;
  b.eta = ctx->eta;
  b.partials = ctx->partials;
  b.tickets = ctx->tickets;
  return b;
}

template <class T>
ReorthBufs<T> reorth_bufs(seed_ctx *ctx) {
  ReorthBufs<T> r;
  r.n = kLow<T> ? ctx->nv : ctx->n;
  r.rows_per_item = ctx->rows_per_item;
  r.nrb = ctx->nrb;
  r.nitems_grid = 152 * 4;
  r.kcap = ctx->prm.m_max + 1;
  r.V = (const T *)ctx->V;
  r.ldv = ctx->ldv;
  r.Hpart = ctx->Hpart;
  r.H = ctx->H;
  r.Hrows = kLow<T> ? ctx->Hrows : nullptr;
  // about two chunks per SM (one wave), within what one SM's L1 holds of v_i and f
  int64_t rc = (r.n + 2 * ctx->sm_count - 1) / (2 * ctx->sm_count);
  rc = (rc + 255) / 256 * 256;
  r.row_chunk = (int32_t)std::min<int64_t>(8192, std::max<int64_t>(4096, rc));
  return r;
}

bool reorth_at(const seed_params &p, int i) { return p.reorth_freq > 0 && i >= 2 && i % p.reorth_freq == 0; }

// Issue one Lanczos step of Sec. 3 (the first step when i == 1).
template <class T>
int issue_seed_step(seed_ctx *ctx, int nrhs, bool reorth) {
  SeedBufs<T> b = seed_bufs<T>(ctx, nrhs);
  // u = A f with f = beta_{i-1} v_i not yet normalized: the dots kernel forms v_i and scales u
  int k = kLow<T> ? apply_A32(ctx, ctx->f, ctx->ldv, ctx->u, ctx->ldv, 1, nullptr)
                  : apply_A(ctx, ctx->f, ctx->ldv, ctx->u, ctx->ldv, 1, nullptr);
  launch_seed_dots<T>(b, ctx->cs);
  launch_seed_update<T>(b, !reorth, ctx->cs);
  k += 2;
  if (reorth) {
    k += launch_seed_flush<T>(b, ctx->blk, ctx->cs);   // reorthogonalization rewrites v_i: fold the block first
    launch_reorth<T>(b, reorth_bufs<T>(ctx), ctx->prm.reorth_passes, ctx->cs);
    k += reorth_kernel_count<T>(ctx->prm.reorth_passes);
  }
  return k;
}

// Capture (once) and launch a graph for the given pattern of steps.
template <class T>
seed_status launch_seed_run(seed_ctx *ctx, int nrhs, const std::vector<char> &pattern) {
  std::string key = (kLow<T> ? "s" : "S") + std::to_string(nrhs) + ":" + std::string(pattern.begin(), pattern.end());
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    GraphEntry g;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(ctx->cs, cudaStreamCaptureModeThreadLocal));
    for (char c : pattern) g.kernels += issue_seed_step<T>(ctx, nrhs, c == 'R');
    g.kernels += launch_seed_flush<T>(seed_bufs<T>(ctx, nrhs), ctx->blk, ctx->cs);   // runs end with a fold
    CU(cudaStreamEndCapture(ctx->cs, &graph));
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, SEED_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    it = ctx->graphs.emplace(key, g).first;
  }
  CU(cudaGraphLaunch(it->second.exec, ctx->cs));
  ctx->stats.graph_launches++;
  ctx->stats.kernel_launches += it->second.kernels;
  return SEED_OK;
}

int run_length(const seed_params &p) {
  if (p.reorth_freq <= 0) return 16;
  if (p.reorth_freq == 1) return 8;
  int best = 1;
  for (int d = 1; d <= 32; ++d)
    if (p.reorth_freq % d == 0) best = d;
  return best >= 8 ? best : 16;
}

// Blocks of a persistent CSR seed run: about 8 rows per thread, at least 16
// blocks, at most the occupancy-derived grid.  Small problems get small grids
// (cheaper barriers, and in a batch several problems' runs fit side by side).
int csr_seed_grid(const seed_ctx *ctx) {
  int64_t b = (ctx->n + 128 * 8 - 1) / (128 * 8);
  if (b < 16) b = 16;
  if (b > ctx->pgrid) b = ctx->pgrid;
  return (int)b;
}

// Runs of steps between reorthogonalizations as one cooperative launch each.
// The Wilson runs take their resident form when the lattice has no more
// 32-site tiles than blocks, else the general one (FP32: the site form, one
// thread per site; 16^3 x 32 mixed seed phase 40.1 ms from graphs of step
// kernels, 37.1 ms in the site form).
bool use_persistent_seed(seed_ctx *ctx) {
  const int f = ctx->prm.reorth_freq;
  return ctx->allow_persistent && ctx->pgrid > 0 && (f == 0 || f >= 8);
}

// Blocks of the persistent CSR CG: one per work item (1024 rows of one column)
// up to the resident limit -- small problems get small grids, whose barriers
// cost less than those of a full grid with idle blocks.
int cg_csr_grid(const seed_ctx *ctx, int nc) {
  const int64_t items = (ctx->n + 1023) / 1024 * nc;
  return (int)std::min<int64_t>(ctx->pgrid_cg, std::max<int64_t>(1, items));
}

// The one-launch seed run of small real CSR problems that reorthogonalize every
// 1 to 7 steps (the streaming form of the seeding): rows per block (16, or 32
// when 16 would need more blocks than can be resident) and the grid; grid 0
// when the problem does not qualify.
struct ReorthRun {
  int rb = 0, grid = 0;
};
ReorthRun reorth_run_shape(const seed_ctx *ctx, int nrhs) {
  const int f = ctx->prm.reorth_freq;
  ReorthRun r;
  if (!ctx->allow_persistent || ctx->kind != 0 || ctx->precision != 0 || f < 1 || f >= 8) return r;
  if (nrhs > kReorthRunMaxRhs || ctx->n > kReorthRunMaxN || ctx->n < 1) return r;
  for (int q = 0; q < 2; ++q) {
    const int rb = 16 << q;
    const int64_t grid = (ctx->n + rb - 1) / rb;
    if (grid <= ctx->rgrid_cap[q]) {
      r.rb = rb;
      r.grid = (int)grid;
      return r;
    }
  }
  return r;
}

// The one-launch lockstep CG of small real CSR problems: rows per block and
// grid, as for the reorthogonalizing seed run; grid 0 when it does not apply.
ReorthRun small_cg_shape(const seed_ctx *ctx, int nc) {
  ReorthRun r;
  if (!ctx->allow_small_cg || ctx->kind != 0 || ctx->precision != 0 || nc > 16 || nc < 1) return r;
  if (ctx->n > kReorthRunMaxN || ctx->n < 1) return r;
  for (int q = 0; q < 2; ++q) {
    const int rb = 16 << q;
    const int64_t grid = (ctx->n + rb - 1) / rb;
    if (grid <= ctx->scg_cap[q]) {
      r.rb = rb;
      r.grid = (int)grid;
      return r;
    }
  }
  return r;
}

seed_status seed_reorth_run(seed_ctx *ctx, int nrhs, ReorthRun shape) {
  const seed_params &p = ctx->prm;
  if (!ctx->rhpart) {
    TRY(dalloc(ctx, &ctx->rhpart, sizeof(double) * 2 * (size_t)(p.m_max + 1) * shape.grid));
    ctx->rhpart_grid = shape.grid;
  }
  if (shape.grid > ctx->rhpart_grid) return fail(ctx, SEED_ECUDA, "internal: reorthogonalizing run grid grew");
  const GridSync g = grid_sync_bufs(ctx);
  SeedBufs<double> b = seed_bufs<double>(ctx, nrhs);
  CU(cudaMemsetAsync(ctx->gsync, 0, sizeof(unsigned) * kGridSyncWords, ctx->cs));
  cudaError_t e = launch_seed_run_csr_reorth(b, ctx->csr, (double *)ctx->f2, g, ctx->partials, ctx->rhpart,
                                             reinterpret_cast<double *>(ctx->H), p.reorth_freq, p.reorth_passes,
                                             p.m_max + 1, shape.rb, shape.grid, ctx->cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SEED_ECUDA, std::string("persistent seed launch: ") + cudaGetErrorString(e));
  }
  ctx->stats.kernel_launches += 1;
  CU(cudaMemcpyAsync(ctx->h_gerr, g.error, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaStreamSynchronize(ctx->cs));
  if (*ctx->h_gerr) return fail(ctx, SEED_ETIMEOUT, "a grid barrier of the persistent seed kernel timed out");
  return SEED_OK;
}

// Runs of Lanczos steps from CUDA graphs, status polled one run behind.
template <class T>
seed_status seed_graph_runs(seed_ctx *ctx, int nrhs) {
  const seed_params &p = ctx->prm;
  // Steps i = 1, 2, ... in runs of L steps aligned so that a run ends at a
  // multiple of the reorthogonalization frequency whenever L divides it.
  const int L = run_length(p);
  int i_next = 1;            // first step of the next run
  int slot = 0, pending = -1;
  bool stopped = false;
  while (!stopped) {
    if (i_next <= p.m_max) {
      int len = L - ((i_next - 1) % L);
      if (i_next + len - 1 > p.m_max) len = p.m_max - i_next + 1;
      std::vector<char> pattern(len);
      for (int q = 0; q < len; ++q) pattern[q] = reorth_at(p, i_next + q) ? 'R' : '.';
      TRY(launch_seed_run<T>(ctx, nrhs, pattern));
      i_next += len;
      CU(cudaMemcpyAsync(&ctx->h_status[slot], &ctx->st->i, sizeof(HostStatus), cudaMemcpyDeviceToHost, ctx->cs));
      CU(cudaEventRecord(ctx->ev_run[slot], ctx->cs));
      if (pending >= 0) {
        // previous run's status (its slot is not recorded again before this wait)
        CU(cudaEventSynchronize(ctx->ev_run[pending]));
        if (!ctx->h_status[pending].active) stopped = true;
      }
      pending = slot;
      slot ^= 1;
    } else {
      stopped = true;
    }
  }
  return SEED_OK;
}

// Segments of steps in one persistent launch each, up to the next step that
// reorthogonalizes (Sec. 3), which runs from a one-step graph.
template <class T>
seed_status seed_persistent_segments(seed_ctx *ctx, int nrhs) {
  const seed_params &p = ctx->prm;
  const GridSync g = grid_sync_bufs(ctx);
  bool launched = false;   // the error flag is this call's only after one of its persistent runs
  for (;;) {
    CU(cudaMemcpyAsync(&ctx->h_status[0], &ctx->st->i, sizeof(HostStatus), cudaMemcpyDeviceToHost, ctx->cs));
    CU(cudaMemcpyAsync(ctx->h_gerr, g.error, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->cs));
    CU(cudaStreamSynchronize(ctx->cs));
    if (launched && *ctx->h_gerr)
      return fail(ctx, SEED_ETIMEOUT, "a grid barrier of the persistent seed kernel timed out");
    const HostStatus hs = ctx->h_status[0];
    if (!hs.active) break;
    const int i = hs.i;
    if (reorth_at(p, i)) {
      TRY(launch_seed_run<T>(ctx, nrhs, std::vector<char>{'R'}));
      continue;
    }
    int i_stop = p.m_max + 1;
    if (p.reorth_freq > 0) i_stop = std::min(i_stop, (i / p.reorth_freq + 1) * p.reorth_freq);
    SeedBufs<T> b = seed_bufs<T>(ctx, nrhs);
    if (b.Wb) i_stop = std::min(i_stop, i + kSeedBlock);   // every run starts a block (blk0 = i)
    CU(cudaMemsetAsync(ctx->gsync, 0, sizeof(unsigned) * kGridSyncWords, ctx->cs));
    cudaError_t e;
    if constexpr (std::is_same_v<T, double2>)
      e = launch_seed_run_wilson(b, ctx->wil, (double2 *)ctx->T, g, ctx->partials, ctx->tpart, i_stop, ctx->pgrid,
                                 ctx->cs);
    else if constexpr (std::is_same_v<T, double>)
      e = launch_seed_run_csr(b, ctx->csr, (double *)ctx->f2, g, ctx->partials, i_stop, csr_seed_grid(ctx), ctx->cs);
    else if constexpr (std::is_same_v<T, float2>)
      e = launch_seed_run_wilson32(b, ctx->wil32, (float2 *)ctx->T32, g, ctx->tpart, i_stop, ctx->pgrid, ctx->cs);
    else
      e = launch_seed_run_csr32(b, ctx->csr32, (float *)ctx->f2, g, ctx->partials, i_stop, csr_seed_grid(ctx),
                                ctx->cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SEED_ECUDA, std::string("persistent seed launch: ") + cudaGetErrorString(e));
    }
    launched = true;
    ctx->stats.kernel_launches += 1 + launch_seed_flush<T>(b, ctx->blk, ctx->cs);
  }
  return SEED_OK;
}

template <class T>
seed_status solve_first_impl(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int nrhs,
                             seed_info *info) {
  const int64_t n = ctx->n;
  const seed_params &p = ctx->prm;
  TRY(ensure_cols(ctx, std::max(nrhs, 1)));
  if (blocked_seeding(ctx, nrhs)) TRY(ensure_block(ctx));
  ctx->basis_valid = false;
  ctx->seeded = false;
  CU(cudaEventRecord(ctx->t0, ctx->cs));

  CallArgs ca{X, ldx, 0};
  CU(cudaMemcpyAsync(ctx->call, &ca, sizeof(ca), cudaMemcpyHostToDevice, ctx->cs));
  SeedState s0{};
  s0.tol_rel = p.tol_seed;
  s0.breakdown_rel = p.breakdown_rel;
  s0.m_max = p.m_max;
  s0.extra_iters = p.extra_iters;
  s0.converged_at = -1;
  s0.stop_at = -1;
  s0.blk0 = 1;
  s0.w_last = 0;
  CU(cudaMemcpyAsync(ctx->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, ctx->cs));
  CU(cudaMemsetAsync(ctx->eta, 0, sizeof(double2) * kMaxRhs, ctx->cs));

  // start: x^j = x_0^j, r_0^j = b^j - A x_0^j (R holds r_0^2.. in columns 0..; r_0^1 in f via seed_start)
  const T *r01 = (const T *)B;
  int kern = 0;
  if (p.x0_zero) {
    launch_zero_cols<T>((T *)X, ldx, n, nrhs, ctx->cs);
    if (nrhs > 1) launch_copy_cols<T>((const T *)B + ldb, ldb, (T *)ctx->R, ctx->ldv, n, nrhs - 1, ctx->cs);
    kern += 1 + (nrhs > 1);
  } else {
    kern += apply_A(ctx, X, ldx, ctx->Q, ctx->ldv, nrhs, nullptr);
    ctx->stats.mvps += nrhs;
    launch_sub_from<T>((const T *)B, ldb, (const T *)ctx->Q, ctx->ldv, (T *)ctx->P, ctx->ldv, n, nrhs, ctx->cs);
    if (nrhs > 1) launch_copy_cols<T>((const T *)ctx->P + ctx->ldv, ctx->ldv, (T *)ctx->R, ctx->ldv, n, nrhs - 1, ctx->cs);
    r01 = (const T *)ctx->P;
    kern += 1 + (nrhs > 1);
  }
  launch_colnorms<T>(n, (const T *)B, ldb, 1, &ctx->st->bnorm1, ctx->partials, ctx->tickets, ctx->cs);
  SeedBufs<T> b = seed_bufs<T>(ctx, nrhs);
  launch_seed_start<T>(b, r01, ctx->cs);
  kern += 2;
  ctx->stats.kernel_launches += kern;

  ReorthRun rr;
  if constexpr (std::is_same_v<T, double>) rr = reorth_run_shape(ctx, nrhs);
  if (rr.grid > 0) {
    TRY(seed_reorth_run(ctx, nrhs, rr));
  } else if (use_persistent_seed(ctx)) {
    TRY(seed_persistent_segments<T>(ctx, nrhs));
  } else {
    TRY(seed_graph_runs<T>(ctx, nrhs));
  }
  CU(cudaStreamSynchronize(ctx->cs));
  CU(cudaGetLastError());

  SeedState st;
  CU(cudaMemcpy(&st, ctx->st, sizeof(st), cudaMemcpyDeviceToHost));
  if (st.stop_reason == STOP_BLOCK) return fail(ctx, SEED_ECUDA, "internal: a seeding block overflowed");
  if (st.stop_reason == STOP_NONFINITE)
    return fail(ctx, SEED_EINVAL, "||b^1 - A x_0^1|| is not finite (NaN or Inf in B, X or the operator)");
  const int steps = st.i >= 1 ? st.i : 0;
  ctx->stats.mvps += (st.beta0 > 0.0) ? steps : 0;
  ctx->last_m = (st.beta0 > 0.0) ? steps : 0;

  // true residual of x^1 (one mvp)
  kern = apply_A(ctx, X, ldx, ctx->Q, ctx->ldv, 1, nullptr);
  launch_sub_from<T>((const T *)B, ldb, (const T *)ctx->Q, ctx->ldv, (T *)ctx->Q, ctx->ldv, n, 1, ctx->cs);
  launch_colnorms<T>(n, (const T *)ctx->Q, ctx->ldv, 1, ctx->colnorm, ctx->partials, ctx->tickets, ctx->cs);
  ctx->stats.kernel_launches += kern + 2;
  ctx->stats.mvps += 1;
  CU(cudaEventRecord(ctx->t1, ctx->cs));
  double rn = 0.0;
  CU(cudaMemcpyAsync(&rn, ctx->colnorm, sizeof(double), cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaStreamSynchronize(ctx->cs));
  CU(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->t0, ctx->t1);
  ctx->stats.ms_seed = ms;

  if (info) {
    std::memset(info, 0, sizeof(seed_info) * nrhs);
    info[0].iters = ctx->last_m;
    info[0].mvps = ctx->last_m + 1 + (p.x0_zero ? 0 : 1);
    info[0].converged = (st.stop_reason == STOP_BREAKDOWN || st.converged_at > 0 || st.beta0 == 0.0) ? 1 : 0;
    info[0].est_relres = st.bnorm1 > 0.0 ? st.rho / st.bnorm1 : 0.0;
    info[0].true_relres = st.bnorm1 > 0.0 ? rn / st.bnorm1 : 0.0;
  }
  ctx->seeded = true;
  ctx->basis_valid = ctx->last_m > 0;
  if (st.stop_reason == STOP_NOTSPD)
    return fail(ctx, SEED_ENOTSPD, "delta_i <= 0 at Lanczos step " + std::to_string(st.i) +
                                       ": operator not positive definite in floating point");
  return SEED_OK;
}

// One lockstep CG iteration on the CG columns c0 .. c0 + c.nc - 1 (c: the view
// of those columns), on stream s, with its own CallArgs slot, partials and
// tickets (two branches of a graph run at the same time on disjoint columns).
template <class T>
int issue_cg_iter(seed_ctx *ctx, const CgCols &c, int c0, cudaStream_t s, const CallArgs *call, double *partials,
                  unsigned *tickets) {
  const int64_t n = ctx->n, ld = ctx->ldv;
  T *P = (T *)ctx->P + (int64_t)c0 * ld, *Q = (T *)ctx->Q + (int64_t)c0 * ld, *R = (T *)ctx->R + (int64_t)c0 * ld;
  int k;
  if (ctx->kind == 0) {
    launch_csr_spmv(ctx->csr, (const double *)P, ld, (double *)Q, ld, c.nc, c.active, s);
    k = 1;
  } else {
    double2 *Tb = (double2 *)ctx->T + (int64_t)c0 * ld;
    launch_wilson_dslash(ctx->wil, +1, (const double2 *)P, ld, Tb, ld, c.nc, c.active, s);
    launch_wilson_dslash(ctx->wil, -1, Tb, ld, (double2 *)Q, ld, c.nc, c.active, s);
    k = 2;
  }
  launch_cg_alpha<T>(n, P, Q, ld, c, partials, tickets, s);
  launch_cg_update<T>(n, call, R, P, Q, ld, c, partials, tickets, s);
  launch_cg_p<T>(n, R, P, ld, c, s);
  return k + 3;
}

// The columns c0 .. c0 + nc - 1 of the per-column CG state.
CgCols cg_sub(const CgCols &c, int c0, int nc) {
  CgCols v = c;
  v.nc = nc;
  for (double **p : {&v.rho, &v.alpha, &v.beta, &v.bnorm, &v.relres, &v.rupd}) *p += c0;
  for (int32_t **p : {&v.active, &v.iters, &v.reached, &v.restarts, &v.converged, &v.needs_check, &v.mvps, &v.upd})
    *p += c0;
  return v;
}

// Lockstep CG graphs split the columns into up to kCgBranches independent
// branches (two columns or more each), one stream each: the branches drift
// against each other, so one branch's vector kernels and kernel tails overlap
// the others' operator applies.  Branch b owns columns start[b] .. start[b+1]-1,
// CallArgs slot b, the b-th part of the partials and the tickets shifted by
// start[b].
int cg_branches(int nc, int start[kCgBranches + 1]) {
  int nb = nc / 2;
  if (nb > kCgBranches) nb = kCgBranches;
  if (nb < 1) nb = 1;
  for (int b = 0; b <= nb; ++b) start[b] = b * nc / nb;
  return nb;
}

// Captures `len` iterations of issue(view, first column, stream, branch) on
// every branch: a fork from cs, the branches, a join back into cs.
template <class F>
int issue_cg_branches(seed_ctx *ctx, const CgCols &c, int len, F &&issue) {
  int start[kCgBranches + 1];
  const int nb = cg_branches(c.nc, start);
  int k = 0;
  if (nb > 1) {
    cudaEventRecord(ctx->ev_fork, ctx->cs);   // a failed call invalidates the capture (reported at its end)
    for (int b = 1; b < nb; ++b) {
      cudaStream_t s = ctx->csb[b - 1];
      cudaStreamWaitEvent(s, ctx->ev_fork, 0);
      const CgCols v = cg_sub(c, start[b], start[b + 1] - start[b]);
      for (int q = 0; q < len; ++q) k += issue(v, start[b], s, b);
      cudaEventRecord(ctx->ev_join[b - 1], s);
    }
  }
  const CgCols v0 = cg_sub(c, 0, start[1]);
  for (int q = 0; q < len; ++q) k += issue(v0, 0, ctx->cs, 0);
  for (int b = 1; b < nb; ++b) cudaStreamWaitEvent(ctx->cs, ctx->ev_join[b - 1], 0);
  return k;
}
double *branch_partials(seed_ctx *ctx, int b) { return ctx->partials + (int64_t)b * (kPartials / kCgBranches); }

CgCols cg_cols(seed_ctx *ctx, int nc) {
  CgCols c;
  c.nc = nc;
  double *d = ctx->cg_d;
  int32_t *q = ctx->cg_i;
  c.rho = d;
  c.alpha = d + kMaxRhs;
  c.beta = d + 2 * kMaxRhs;
  c.bnorm = d + 3 * kMaxRhs;
  c.relres = d + 4 * kMaxRhs;
  c.rupd = d + 5 * kMaxRhs;
  c.active = q;
  c.iters = q + kMaxRhs;
  c.reached = q + 2 * kMaxRhs;
  c.restarts = q + 3 * kMaxRhs;
  c.converged = q + 4 * kMaxRhs;
  c.needs_check = q + 5 * kMaxRhs;
  c.mvps = q + 6 * kMaxRhs;
  c.upd = q + 7 * kMaxRhs;
  c.tol = ctx->prm.tol_rest;
  c.tol_check = 1.5 * ctx->prm.tol_rest;
  c.maxit = ctx->prm.maxit_rest;
  c.max_restarts = ctx->prm.max_restarts;
  // default: a reliable update every two decades of the FP32 recursive residual
  // (16^3 x 32 mixed workload: 171 CG iterations per system at 0.1, 0.03 and
  // 0.01 alike, and 164 -> 155 ms as the FP64 operator runs less often)
  c.delta = ctx->prm.reliable_delta > 0.0 ? ctx->prm.reliable_delta : 0.001;
  return c;
}

struct CgHost {
  std::vector<int32_t> i;
  std::vector<double> d;
  int32_t iters(int j) const { return i[kMaxRhs + j]; }
  int32_t restarts(int j) const { return i[3 * kMaxRhs + j]; }
  int32_t converged(int j) const { return i[4 * kMaxRhs + j]; }
  int32_t mvps(int j) const { return i[6 * kMaxRhs + j]; }
  double relres(int j) const { return d[4 * kMaxRhs + j]; }
};

seed_status read_cg(seed_ctx *ctx, CgHost *h) {
  h->i.resize(kCgInts * kMaxRhs);
  h->d.resize(kCgDoubles * kMaxRhs);
  CU(cudaMemcpyAsync(h->i.data(), ctx->cg_i, sizeof(int32_t) * kCgInts * kMaxRhs, cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaMemcpyAsync(h->d.data(), ctx->cg_d, sizeof(double) * kCgDoubles * kMaxRhs, cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaStreamSynchronize(ctx->cs));
  return SEED_OK;
}

template <class T>
seed_status launch_cg_run(seed_ctx *ctx, const CgCols &c, int len) {
  std::string key = "C" + std::to_string(c.nc) + ":" + std::to_string(len);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    GraphEntry g;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(ctx->cs, cudaStreamCaptureModeThreadLocal));
    g.kernels += issue_cg_branches(ctx, c, len, [&](const CgCols &v, int c0, cudaStream_t s, int b) {
      return issue_cg_iter<T>(ctx, v, c0, s, ctx->call + b, branch_partials(ctx, b), ctx->tickets + c0);
    });
    CU(cudaStreamEndCapture(ctx->cs, &graph));
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, SEED_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    it = ctx->graphs.emplace(key, g).first;
  }
  CU(cudaGraphLaunch(it->second.exec, ctx->cs));
  ctx->stats.graph_launches++;
  ctx->stats.kernel_launches += it->second.kernels;
  return SEED_OK;
}

// Lockstep CG (Sec. 1, Sec. 2.2) on the nc columns of Bc / Xc from the guesses
// in Xc; info: NULL or nc entries.
template <class T>
seed_status cg_impl(seed_ctx *ctx, const T *Bc, int64_t ldb, T *Xc, int64_t ldx, int nc, seed_info *info) {
  const int64_t n = ctx->n, ld = ctx->ldv;
  if (info) std::memset(info, 0, sizeof(seed_info) * nc);
  if (nc <= 0) return SEED_OK;
  TRY(ensure_cols(ctx, nc));
  CU(cudaEventRecord(ctx->t2, ctx->cs));
  // slot b: branch b of the CG graphs (its first column)
  int start[kCgBranches + 1];
  const int nb = cg_branches(nc, start);
  CallArgs ca[kCgBranches];
  for (int b = 0; b < nb; ++b) ca[b] = CallArgs{Xc, ldx, start[b]};
  CU(cudaMemcpyAsync(ctx->call, ca, sizeof(CallArgs) * nb, cudaMemcpyHostToDevice, ctx->cs));
  const CgCols c = cg_cols(ctx, nc);
  // K7: true residual of the seeded systems, then p = r
  int kern = apply_A(ctx, Xc, ldx, ctx->Q, ld, nc, nullptr);
  launch_cg_init<T>(n, Bc, ldb, (const T *)ctx->Q, ld, (T *)ctx->R, (T *)ctx->P, ld, c, ctx->partials, ctx->tickets,
                    false, ctx->cs);
  ctx->stats.kernel_launches += kern + 1;
  ctx->stats.mvps += nc;

  ReorthRun scg;   // small real CSR problems: the one-launch CG with two barriers per iteration
  if constexpr (std::is_same_v<T, double>) scg = small_cg_shape(ctx, nc);
  const bool persist = scg.grid > 0 || (ctx->allow_persistent_cg && ctx->pgrid_cg > 0 && nc <= kPersistMaxCols);
  const GridSync g = grid_sync_bufs(ctx);
  const int L = 16;
  for (int round = 0;; ++round) {
    if (persist) {
      // one persistent launch runs CG until no column is active
      CU(cudaMemsetAsync(ctx->gsync, 0, sizeof(unsigned) * kGridSyncWords, ctx->cs));
      cudaError_t e;
      if constexpr (sizeof(T) == sizeof(double2))
        e = launch_cg_run_wilson(ctx->wil, ctx->call, (double2 *)ctx->R, (double2 *)ctx->P, (double2 *)ctx->Q,
                                 (double2 *)ctx->T, ld, c, g, ctx->partials, ctx->pgrid_cg, ctx->cs);
      else if (scg.grid > 0)
        e = launch_cg_run_csr_small(ctx->csr, ctx->call, (double *)ctx->R, (double *)ctx->P, (double *)ctx->T,
                                    (double *)ctx->Q, ld, c, g, ctx->partials, scg.rb, scg.grid, ctx->cs);
      else
        e = launch_cg_run_csr(ctx->csr, ctx->call, (double *)ctx->R, (double *)ctx->P, (double *)ctx->Q, ld, c, g,
                              ctx->partials, cg_csr_grid(ctx, nc), ctx->cs);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SEED_ECUDA, std::string("persistent CG launch: ") + cudaGetErrorString(e));
      }
      ctx->stats.kernel_launches += 1;
      CU(cudaMemcpyAsync(ctx->h_gerr, g.error, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->cs));
      CU(cudaStreamSynchronize(ctx->cs));
      if (*ctx->h_gerr) return fail(ctx, SEED_ETIMEOUT, "a grid barrier of the persistent CG kernel timed out");
    } else {
      // CG runs until no column is active (polled one run behind)
      int slot = 0, pending = -1;
      cudaEvent_t evs[2] = {nullptr, nullptr};
      for (;;) {
        TRY(launch_cg_run<T>(ctx, c, L));
        CU(cudaMemcpyAsync(ctx->h_flags + slot * kMaxRhs, c.active, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost,
                           ctx->cs));
        if (!evs[slot]) CU(cudaEventCreateWithFlags(&evs[slot], cudaEventDisableTiming));
        CU(cudaEventRecord(evs[slot], ctx->cs));
        bool any = true;
        if (pending >= 0) {
          CU(cudaEventSynchronize(evs[pending]));
          any = false;
          for (int j = 0; j < nc; ++j) any |= ctx->h_flags[pending * kMaxRhs + j] != 0;
        }
        pending = slot;
        slot ^= 1;
        if (!any) break;
      }
      CU(cudaStreamSynchronize(ctx->cs));
      for (auto &e : evs)
        if (e) cudaEventDestroy(e);
    }
    // true residuals of the columns that stopped; restarts where needed
    kern = apply_A(ctx, Xc, ldx, ctx->Q, ld, nc, c.needs_check);
    launch_cg_check<T>(n, Bc, ldb, (const T *)ctx->Q, ld, (T *)ctx->R, ld, c, ctx->partials, ctx->tickets, ctx->cs);
    launch_cg_init<T>(n, Bc, ldb, (const T *)ctx->Q, ld, (T *)ctx->R, (T *)ctx->P, ld, c, ctx->partials,
                      ctx->tickets, true, ctx->cs);
    ctx->stats.kernel_launches += kern + 2;
    CU(cudaMemcpyAsync(ctx->h_flags, c.active, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, ctx->cs));
    CU(cudaStreamSynchronize(ctx->cs));
    bool any = false;
    for (int j = 0; j < nc; ++j) any |= ctx->h_flags[j] != 0;
    if (!any || round > 64) break;
  }
  CU(cudaEventRecord(ctx->t3, ctx->cs));
  CU(cudaGetLastError());

  std::vector<int32_t> hi(7 * kMaxRhs);
  std::vector<double> hd(5 * kMaxRhs);
  CU(cudaMemcpyAsync(hi.data(), ctx->cg_i, sizeof(int32_t) * 7 * kMaxRhs, cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaMemcpyAsync(hd.data(), ctx->cg_d, sizeof(double) * 5 * kMaxRhs, cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaStreamSynchronize(ctx->cs));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->t2, ctx->t3);
  ctx->stats.ms_rest = ms;
  bool all = true;
  int64_t mv = 0;
  for (int j = 0; j < nc; ++j) {
    const int conv = hi[4 * kMaxRhs + j];
    all &= conv != 0;
    mv += hi[6 * kMaxRhs + j];
    if (info) {
      seed_info &o = info[j];
      o.iters = hi[kMaxRhs + j];
      o.mvps = hi[6 * kMaxRhs + j];
      o.restarts = hi[3 * kMaxRhs + j];
      o.converged = conv;
      o.est_relres = hd[4 * kMaxRhs + j];
      o.true_relres = hd[4 * kMaxRhs + j];
    }
  }
  ctx->stats.mvps += mv - nc;   // the initial residual was counted above
  if (!all) return fail(ctx, SEED_ENOTCONV, "CG did not reach tol_rest on every system within maxit_rest");
  return SEED_OK;
}

template <class T>
seed_status solve_rest_impl(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int nrhs,
                            seed_info *info) {
  const int nc = nrhs - 1;
  if (nc <= 0) {
    if (info && nrhs > 1) std::memset(info + 1, 0, sizeof(seed_info) * (nrhs - 1));
    return SEED_OK;
  }
  TRY(ensure_cols(ctx, nrhs));
  return cg_impl<T>(ctx, (const T *)B + ldb, ldb, (T *)X + ldx, ldx, nc, info ? info + 1 : nullptr);
}

// ---------------------------------------------------------------------------
// CSR launch-shape autotuner: times every shape of kCsrShape on the matrix
// itself (10 launches after 2 untimed ones, CUDA events on the context's
// stream) and keeps the fastest; choices are cached per process by (device,
// n, nnz, precision) so that a batch of equal-sized problems tunes once.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int>, int> g_tune_cache;

template <class R>
seed_status time_csr_shape(seed_ctx *ctx, CsrOpT<R> &op, const R *x, R *y, int shape, float *ms) {
  op.tpr = kCsrShape[shape][0];
  op.block = kCsrShape[shape][1];
  for (int r = 0; r < 12; ++r) {
    if (r == 2) CU(cudaEventRecord(ctx->t0, ctx->cs));
    if constexpr (sizeof(R) == sizeof(double)) launch_csr_spmv(op, x, ctx->ldv, y, ctx->ldv, 1, nullptr, ctx->cs);
    else launch_csr_spmv32(op, x, ctx->ldv, y, ctx->ldv, 1, nullptr, ctx->cs);
  }
  CU(cudaEventRecord(ctx->t1, ctx->cs));
  CU(cudaEventSynchronize(ctx->t1));
  CU(cudaGetLastError());
  CU(cudaEventElapsedTime(ms, ctx->t0, ctx->t1));
  ctx->stats.kernel_launches += 12;
  return SEED_OK;
}

seed_status autotune_csr(seed_ctx *ctx, int64_t nnz) {
  const auto key = std::make_tuple(ctx->device, ctx->n, nnz, ctx->precision);
  int best = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best = it->second;
  }
  if (best < 0) {
    TRY(ensure_cols(ctx, 1));
    float best_ms = 0.f;
    for (int sh = 0; sh < kCsrShapes; ++sh) {
      float ms = 0.f;
      if (ctx->precision == 1) {
        CU(cudaMemsetAsync(ctx->P32, 0, (size_t)ctx->ldv * ctx->vsz, ctx->cs));
        TRY(time_csr_shape<float>(ctx, ctx->csr32, (const float *)ctx->P32, (float *)ctx->Q32, sh, &ms));
      } else {
        CU(cudaMemsetAsync(ctx->P, 0, (size_t)ctx->ldv * ctx->esz, ctx->cs));
        TRY(time_csr_shape<double>(ctx, ctx->csr, (const double *)ctx->P, (double *)ctx->Q, sh, &ms));
      }
      if (best < 0 || ms < best_ms) {
        best = sh;
        best_ms = ms;
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  // the FP64 operator (true residuals) and its FP32 copy share the chosen shape
  ctx->csr.tpr = ctx->csr32.tpr = kCsrShape[best][0];
  ctx->csr.block = ctx->csr32.block = kCsrShape[best][1];
  return SEED_OK;
}

// ---------------------------------------------------------------------------
// Sec. 2.3: single seeding of related right-hand sides
// ---------------------------------------------------------------------------
seed_status ensure_related(seed_ctx *ctx, int nc) {
  if (nc <= ctx->rel_cap) return SEED_OK;
  cudaStreamSynchronize(ctx->cs);
  cudaFree(ctx->Rrel); cudaFree(ctx->xrel); cudaFree(ctx->rrel);
  ctx->Rrel = ctx->xrel = ctx->rrel = nullptr;
  ctx->rel_cap = 0;
  TRY(dalloc(ctx, &ctx->Rrel, (size_t)ctx->ldv * nc * ctx->esz));
  TRY(dalloc(ctx, &ctx->xrel, (size_t)ctx->ldv * ctx->esz));
  TRY(dalloc(ctx, &ctx->rrel, (size_t)ctx->ldv * ctx->esz));
  if (!ctx->reldots) TRY(dalloc(ctx, &ctx->reldots, sizeof(double2) * 2 * kMaxRhs));
  ctx->rel_cap = nc;
  return SEED_OK;
}

// Sec. 2.3 after the seed solve of system 1: project the remaining
// systems over x^1 (x^1_bcg = 0, r^1_bcg = b^1), then for j = 2, 3, ...: CG on
// system j from its current approximation, and project the systems after it
// over that CG's correction.
template <class T>
seed_status solve_related_impl(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int nrhs,
                               seed_info *info) {
  const int64_t n = ctx->n, ld = ctx->ldv;
  const int nc = nrhs - 1;
  if (info && nc > 0) std::memset(info + 1, 0, sizeof(seed_info) * nc);
  if (nc <= 0) return SEED_OK;
  TRY(ensure_cols(ctx, nrhs));
  TRY(ensure_related(ctx, nc));
  const T *Bt = (const T *)B;
  T *Xt = (T *)X;
  T *R = (T *)ctx->Rrel, *xb = (T *)ctx->xrel, *rb = (T *)ctx->rrel;
  double2 *dots = ctx->reldots, *delta = ctx->reldots + kMaxRhs;
  CU(cudaEventRecord(ctx->t2, ctx->cs));
  // residuals of the seeded systems 2..nrhs
  int kern = apply_A(ctx, Xt + ldx, ldx, ctx->Q, ld, nc, nullptr);
  launch_sub_from<T>(Bt + ldb, ldb, (const T *)ctx->Q, ld, R, ld, n, nc, ctx->cs);
  ctx->stats.mvps += nc;
  // projection over system 1: x_cg = x^1, r_bcg = b^1
  launch_related_project<T>(n, Xt, Bt, Xt + ldx, ldx, R, ld, nc, dots, delta, ctx->partials, ctx->tickets, ctx->cs);
  ctx->stats.kernel_launches += kern + 4;
  float ms_total = 0.f;
  for (int j = 0; j < nc; ++j) {
    T *xj = Xt + (int64_t)(1 + j) * ldx;
    // next system: x_bcg, r_bcg of system j + 2, then CG
    launch_copy_cols<T>(xj, ldx, xb, ld, n, 1, ctx->cs);
    launch_copy_cols<T>(R + (int64_t)j * ld, ld, rb, ld, n, 1, ctx->cs);
    ctx->stats.kernel_launches += 2;
    TRY(cg_impl<T>(ctx, Bt + (int64_t)(1 + j) * ldb, ldb, xj, ldx, 1, info ? info + 1 + j : nullptr));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->t2, ctx->t3);
    ms_total += ms;
    if (j + 1 < nc) {
      // x_cg = x^j - x^j_bcg; project the systems after j over it
      launch_sub_from<T>(xj, ldx, xb, ld, xb, ld, n, 1, ctx->cs);
      launch_related_project<T>(n, xb, rb, xj + ldx, ldx, R + (int64_t)(j + 1) * ld, ld, nc - j - 1, dots, delta,
                                ctx->partials, ctx->tickets, ctx->cs);
      ctx->stats.kernel_launches += 4;
    }
  }
  CU(cudaStreamSynchronize(ctx->cs));
  CU(cudaGetLastError());
  ctx->stats.ms_rest = ms_total;
  return SEED_OK;
}

// ---------------------------------------------------------------------------
// Multiple seeding (the comparison method of Sec. 2.1)
// ---------------------------------------------------------------------------
seed_status ensure_multiple(seed_ctx *ctx, int nrhs) {
  if (nrhs <= ctx->ms_cap) return SEED_OK;
  cudaStreamSynchronize(ctx->cs);
  cudaFree(ctx->msX); cudaFree(ctx->msR);
  ctx->msX = ctx->msR = nullptr;
  ctx->ms_cap = 0;
  TRY(dalloc(ctx, &ctx->msX, (size_t)ctx->ldv * nrhs * ctx->esz));
  TRY(dalloc(ctx, &ctx->msR, (size_t)ctx->ldv * nrhs * ctx->esz));
  if (!ctx->reldots) TRY(dalloc(ctx, &ctx->reldots, sizeof(double2) * 2 * kMaxRhs));
  ctx->ms_cap = nrhs;
  return SEED_OK;
}

// Systems solved in order by CG from zero; every CG step of system j projects
// each later system i over its direction p (eta = p^H r^i / p^H q, x^i += eta p,
// r^i -= eta q), with the tracked residuals r^i (b^i at the start).  All on
// internal copies (so the captured graphs stay valid), copied to X at the end.
template <class T>
seed_status solve_multiple_impl(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int nrhs,
                                seed_info *info) {
  const int64_t n = ctx->n, ld = ctx->ldv;
  if (info) std::memset(info, 0, sizeof(seed_info) * nrhs);
  TRY(ensure_cols(ctx, nrhs));
  TRY(ensure_multiple(ctx, nrhs));
  T *Xw = (T *)ctx->msX, *Rw = (T *)ctx->msR;
  const T *Bt = (const T *)B;
  double2 *dots = ctx->reldots, *delta = ctx->reldots + kMaxRhs;
  CU(cudaEventRecord(ctx->t2, ctx->cs));
  launch_zero_cols<T>(Xw, ld, n, nrhs, ctx->cs);
  launch_copy_cols<T>(Bt, ldb, Rw, ld, n, nrhs, ctx->cs);
  ctx->stats.kernel_launches += 2;
  CgCols c = cg_cols(ctx, 1);
  c.max_restarts = 0;
  c.tol_check = 1.5 * c.tol;
  const int L = 16;
  for (int j = 0; j < nrhs; ++j) {
    const CallArgs ca{Xw, ld, j};
    CU(cudaMemcpyAsync(ctx->call, &ca, sizeof(ca), cudaMemcpyHostToDevice, ctx->cs));
    int kern = apply_A(ctx, Xw + (int64_t)j * ld, ld, ctx->Q, ld, 1, nullptr);
    launch_cg_init<T>(n, Bt + (int64_t)j * ldb, ldb, (const T *)ctx->Q, ld, (T *)ctx->R, (T *)ctx->P, ld, c,
                      ctx->partials, ctx->tickets, false, ctx->cs);
    ctx->stats.kernel_launches += kern + 1;
    const int nrem = nrhs - j - 1;
    const std::string key = "MS" + std::to_string(nrhs) + ":" + std::to_string(j) + ":" + std::to_string(L);
    int slot = 0, pending = -1;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    for (;;) {
      TRY(run_graph(ctx, key, [&] {
        int k = 0;
        for (int q = 0; q < L; ++q) {
          k += apply_A(ctx, ctx->P, ld, ctx->Q, ld, 1, c.active);
          launch_cg_alpha<T>(n, (const T *)ctx->P, (const T *)ctx->Q, ld, c, ctx->partials, ctx->tickets, ctx->cs);
          launch_related_project<T>(n, (const T *)ctx->P, (const T *)ctx->Q, Xw + (int64_t)(j + 1) * ld, ld,
                                    Rw + (int64_t)(j + 1) * ld, ld, nrem, dots, delta, ctx->partials, ctx->tickets,
                                    ctx->cs, c.active);
          launch_cg_update<T>(n, ctx->call, (T *)ctx->R, (const T *)ctx->P, (const T *)ctx->Q, ld, c, ctx->partials,
                              ctx->tickets, ctx->cs);
          launch_cg_p<T>(n, (const T *)ctx->R, (T *)ctx->P, ld, c, ctx->cs);
          k += 3 + (nrem > 0 ? 3 : 0);
        }
        return k;
      }));
      CU(cudaMemcpyAsync(ctx->h_flags + slot * kMaxRhs, c.active, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->cs));
      if (!evs[slot]) CU(cudaEventCreateWithFlags(&evs[slot], cudaEventDisableTiming));
      CU(cudaEventRecord(evs[slot], ctx->cs));
      bool any = true;
      if (pending >= 0) {
        CU(cudaEventSynchronize(evs[pending]));
        any = ctx->h_flags[pending * kMaxRhs] != 0;
      }
      pending = slot;
      slot ^= 1;
      if (!any) break;
    }
    CU(cudaStreamSynchronize(ctx->cs));
    for (auto &e : evs)
      if (e) cudaEventDestroy(e);
    // true residual of system j
    kern = apply_A(ctx, Xw + (int64_t)j * ld, ld, ctx->Q, ld, 1, c.needs_check);
    launch_cg_check<T>(n, Bt + (int64_t)j * ldb, ldb, (const T *)ctx->Q, ld, (T *)ctx->R, ld, c, ctx->partials,
                       ctx->tickets, ctx->cs);
    ctx->stats.kernel_launches += kern + 1;
    CgHost h;
    TRY(read_cg(ctx, &h));
    ctx->stats.mvps += h.mvps(0);
    if (info) {
      info[j].iters = h.iters(0);
      info[j].mvps = h.mvps(0);
      info[j].converged = h.converged(0);
      info[j].est_relres = info[j].true_relres = h.relres(0);
    }
  }
  launch_copy_cols<T>(Xw, ld, (T *)X, ldx, n, nrhs, ctx->cs);
  ctx->stats.kernel_launches += 1;
  CU(cudaEventRecord(ctx->t3, ctx->cs));
  CU(cudaStreamSynchronize(ctx->cs));
  CU(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->t2, ctx->t3);
  ctx->stats.ms_rest = ms;
  if (info)
    for (int j = 0; j < nrhs; ++j)
      if (!info[j].converged) return fail(ctx, SEED_ENOTCONV, "multiple seeding: a system did not reach tol_rest");
  return SEED_OK;
}

// ---------------------------------------------------------------------------
// Mixed precision: FP32 iterations, FP64 scalars and reliable updates
// ---------------------------------------------------------------------------

// Capture (once, under `key`) and launch a graph of the work issue() enqueues.
template <class F>
seed_status run_graph(seed_ctx *ctx, const std::string &key, F issue) {
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    GraphEntry g;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(ctx->cs, cudaStreamCaptureModeThreadLocal));
    g.kernels = issue();
    CU(cudaStreamEndCapture(ctx->cs, &graph));
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, SEED_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    it = ctx->graphs.emplace(key, g).first;
  }
  CU(cudaGraphLaunch(it->second.exec, ctx->cs));
  ctx->stats.graph_launches++;
  ctx->stats.kernel_launches += it->second.kernels;
  return SEED_OK;
}

// One lockstep CG iteration in FP32 (the operator's FP32 copy, FP32 vectors,
// FP64 alpha / beta / norms) on the CG columns c0 .. c0 + c.nc - 1 (c: their
// view); x is the FP32 correction E (CallArgs `call`).  Stream, partials and
// tickets as in issue_cg_iter.
template <class T32>
int issue_mixed_iter(seed_ctx *ctx, const CgCols &c, int c0, cudaStream_t s, const CallArgs *call,
                     double *partials, unsigned *tickets) {
  const int64_t n = ctx->nv, ld = ctx->ldv;
  T32 *P = (T32 *)ctx->P32 + (int64_t)c0 * ld, *Q = (T32 *)ctx->Q32 + (int64_t)c0 * ld;
  T32 *R = (T32 *)ctx->R32 + (int64_t)c0 * ld;
  int k;
  if (ctx->kind == 0) {
    launch_csr_spmv32(ctx->csr32, (const float *)P, ld, (float *)Q, ld, c.nc, c.active, s);
    k = 1;
  } else {
    float2 *Tb = (float2 *)ctx->T32 + (int64_t)c0 * ld;
    launch_wilson_dslash32(ctx->wil32, +1, (const float2 *)P, ld, Tb, ld, c.nc, c.active, true, s);
    launch_wilson_dslash32(ctx->wil32, -1, Tb, ld, (float2 *)Q, ld, c.nc, c.active, true, s);
    k = 2;
  }
  launch_cg_alpha<T32>(n, P, Q, ld, c, partials, tickets, s);
  launch_cg_update<T32>(n, call, R, P, Q, ld, c, partials, tickets, s);
  launch_cg_p<T32>(n, R, P, ld, c, s);
  return k + 3;
}

// CG on columns c0..c0+nc-1 of B and X (FP64) to ||b - A x|| <= tol ||b||
// measured with the FP64 operator: runs of 16 FP32 iterations, each run
// followed by the reliable update of the columns that need one.
template <class T64, class T32>
seed_status mixed_cg(seed_ctx *ctx, const T64 *Bc, int64_t ldb, T64 *Xc, int64_t ldx, int c0, int nc, double tol,
                     CgCols *cols_out) {
  const int64_t nv = ctx->nv, ld = ctx->ldv;
  const Layout32 lay = ctx->lay;
  CgCols c = cg_cols(ctx, nc);
  c.tol = tol;
  c.tol_check = tol;
  T32 *E = E_cols<T32>(ctx) + (int64_t)c0 * ld;
  // CG column c corrects system c0 + c + 1; slot 1 + b: branch b of the graphs
  int start[kCgBranches + 1];
  const int nb = cg_branches(nc, start);
  CallArgs ca[kCgBranches];
  for (int b = 0; b < nb; ++b) ca[b] = CallArgs{(void *)E_cols<T32>(ctx), ld, c0 + start[b]};
  CU(cudaMemcpyAsync(ctx->call32 + 1, ca, sizeof(CallArgs) * nb, cudaMemcpyHostToDevice, ctx->cs));
  int kern = apply_A(ctx, Xc, ldx, ctx->Q, ld, nc, nullptr);
  launch_mixed_init<T64, T32>(nv, lay, Bc, ldb, (const T64 *)ctx->Q, ld, (T32 *)ctx->R32, (T32 *)ctx->P32, E, ld, c,
                              ctx->partials, ctx->tickets, ctx->cs);
  ctx->stats.kernel_launches += kern + 1;
  ctx->stats.mvps += nc;
  const int L = 16;
  // the graph bakes in CgCols (tolerance included): system 1 (c0 = 0) and the others have their own
  const std::string key = "M" + std::to_string(nc) + ":" + std::to_string(L) + ":" + std::to_string(c0);
  int slot = 0, pending = -1;
  cudaEvent_t evs[2] = {nullptr, nullptr};
  for (;;) {
    TRY(run_graph(ctx, key, [&] {
      return issue_cg_branches(ctx, c, L, [&](const CgCols &v, int cb0, cudaStream_t s, int b) {
        return issue_mixed_iter<T32>(ctx, v, cb0, s, ctx->call32 + 1 + b, branch_partials(ctx, b), ctx->tickets + cb0);
      });
    }));
    // reliable updates (direct launches: B and X are this call's buffers)
    launch_mixed_flag(c, ctx->cs);
    launch_fold<T64, T32>(Xc, ldx, E, ld, nv, lay, nc, c.upd, ctx->cs);
    kern = apply_A(ctx, Xc, ldx, ctx->Q, ld, nc, c.upd);
    launch_mixed_residual<T64, T32>(nv, lay, Bc, ldb, (const T64 *)ctx->Q, ld, (T32 *)ctx->R32, (T32 *)ctx->P32, ld,
                                    c, ctx->partials, ctx->tickets, ctx->cs);
    ctx->stats.kernel_launches += kern + 3;
    CU(cudaMemcpyAsync(ctx->h_flags + slot * kMaxRhs, c.active, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost,
                       ctx->cs));
    if (!evs[slot]) CU(cudaEventCreateWithFlags(&evs[slot], cudaEventDisableTiming));
    CU(cudaEventRecord(evs[slot], ctx->cs));
    bool any = true;
    if (pending >= 0) {
      CU(cudaEventSynchronize(evs[pending]));
      any = false;
      for (int j = 0; j < nc; ++j) any |= ctx->h_flags[pending * kMaxRhs + j] != 0;
    }
    pending = slot;
    slot ^= 1;
    if (!any) break;
  }
  CU(cudaStreamSynchronize(ctx->cs));
  for (auto &e : evs)
    if (e) cudaEventDestroy(e);
  CU(cudaGetLastError());
  if (cols_out) *cols_out = c;
  return SEED_OK;
}

// The Sec. 3 seed solve with FP32 vectors and operator (FP64 scalars), then system
// 1 finished to tol_seed by mixed CG.
template <class T64, class T32>
seed_status solve_first_mixed(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int nrhs,
                              seed_info *info) {
  const int64_t n = ctx->n, ld = ctx->ldv;
  const seed_params &p = ctx->prm;
  TRY(ensure_cols(ctx, std::max(nrhs, 1)));
  if (blocked_seeding(ctx, nrhs)) TRY(ensure_block(ctx));
  ctx->basis_valid = false;
  ctx->seeded = false;
  // TMA maps of the tensor-core flush over this call's buffers (V, r_0^2.. in FP32)
  ctx->blk.tc = nullptr;
  if (blocked_seeding(ctx, nrhs) && tc_flush_eligible(ctx) && ctx->tc_err) {
    TcFlush &t = ctx->tcf;
    t.err = ctx->tc_err;
    t.grid = tc_grid(ctx->nv);
    t.ok = t.grid >= 1 &&
           tc_make_maps(t.maps.v, ctx->V, ctx->nv, ctx->ldv, (int64_t)ctx->prm.m_max + 1) &&
           tc_make_maps(t.maps.r, (const char *)ctx->R32 + ctx->ldv * ctx->vsz, ctx->nv, ctx->ldv,
                        std::max(ctx->cap_cols - 1, 1));
    if (t.ok) ctx->blk.tc = &ctx->tcf;
  }
  CU(cudaEventRecord(ctx->t0, ctx->cs));
  T32 *E = E_cols<T32>(ctx);
  const CallArgs ca{(void *)E, ld, 0};
  CU(cudaMemcpyAsync(ctx->call32, &ca, sizeof(ca), cudaMemcpyHostToDevice, ctx->cs));
  SeedState s0{};
  s0.tol_rel = p.tol_seed;
  s0.breakdown_rel = p.breakdown_rel;
  s0.m_max = p.m_max;
  s0.extra_iters = p.extra_iters;
  s0.converged_at = -1;
  s0.stop_at = -1;
  s0.blk0 = 1;
  s0.w_last = 0;
  CU(cudaMemcpyAsync(ctx->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, ctx->cs));
  CU(cudaMemsetAsync(ctx->eta, 0, sizeof(double2) * kMaxRhs, ctx->cs));

  // start in FP64: r_0^j = b^j - A x_0^j, rounded to FP32 (column 0 starts the Lanczos run)
  int kern = 0;
  const int64_t nv = ctx->nv;
  if (p.x0_zero) {
    launch_zero_cols<T64>((T64 *)X, ldx, n, nrhs, ctx->cs);
    launch_to_low<T64, T32>((const T64 *)B, ldb, (T32 *)ctx->R32, ld, nv, ctx->lay, nrhs, ctx->cs);
    kern += 2;
  } else {
    kern += apply_A(ctx, X, ldx, ctx->Q, ld, nrhs, nullptr);
    ctx->stats.mvps += nrhs;
    launch_sub_from<T64>((const T64 *)B, ldb, (const T64 *)ctx->Q, ld, (T64 *)ctx->P, ld, n, nrhs, ctx->cs);
    launch_to_low<T64, T32>((const T64 *)ctx->P, ld, (T32 *)ctx->R32, ld, nv, ctx->lay, nrhs, ctx->cs);
    kern += 2;
  }
  launch_zero_cols<T32>(E, ld, nv, nrhs, ctx->cs);
  launch_colnorms<T64>(n, (const T64 *)B, ldb, 1, &ctx->st->bnorm1, ctx->partials, ctx->tickets, ctx->cs);
  SeedBufs<T32> b = seed_bufs<T32>(ctx, nrhs);
  launch_seed_start<T32>(b, (const T32 *)ctx->R32, ctx->cs);
  kern += 3;
  ctx->stats.kernel_launches += kern;
  if (use_persistent_seed(ctx)) {
    TRY(seed_persistent_segments<T32>(ctx, nrhs));
  } else {
    TRY(seed_graph_runs<T32>(ctx, nrhs));
  }
  CU(cudaStreamSynchronize(ctx->cs));
  CU(cudaGetLastError());
  if (ctx->blk.tc) {
    int terr = 0;
    CU(cudaMemcpy(&terr, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (terr) {
      CU(cudaMemset(ctx->tc_err, 0, sizeof(int)));
      return fail(ctx, SEED_ETIMEOUT, "a wait of the tensor-core seeding kernel timed out");
    }
  }
  SeedState st;
  CU(cudaMemcpy(&st, ctx->st, sizeof(st), cudaMemcpyDeviceToHost));
  if (st.stop_reason == STOP_BLOCK) return fail(ctx, SEED_ECUDA, "internal: a seeding block overflowed");
  if (st.stop_reason == STOP_NONFINITE)
    return fail(ctx, SEED_EINVAL, "||b^1 - A x_0^1|| is not finite (NaN or Inf in B, X or the operator)");
  const int steps = (st.beta0 > 0.0 && st.i >= 1) ? st.i : 0;
  ctx->stats.mvps += steps;
  ctx->last_m = steps;
  if (st.stop_reason == STOP_NOTSPD) {
    CU(cudaEventRecord(ctx->t1, ctx->cs));
    return fail(ctx, SEED_ENOTSPD, "delta_i <= 0 at Lanczos step " + std::to_string(st.i) +
                                       ": operator not positive definite in floating point");
  }
  // x^j += e^j (the FP32 Lanczos corrections), then system 1 to tol_seed
  launch_fold<T64, T32>((T64 *)X, ldx, E, ld, nv, ctx->lay, nrhs, nullptr, ctx->cs);
  ctx->stats.kernel_launches += 1;
  TRY((mixed_cg<T64, T32>(ctx, (const T64 *)B, ldb, (T64 *)X, ldx, 0, 1, p.tol_seed, nullptr)));
  CU(cudaEventRecord(ctx->t1, ctx->cs));
  CgHost h;
  TRY(read_cg(ctx, &h));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->t0, ctx->t1);
  ctx->stats.ms_seed = ms;
  ctx->stats.mvps += h.mvps(0) - 1;   // the first true residual was counted by mixed_cg
  if (info) {
    std::memset(info, 0, sizeof(seed_info) * nrhs);
    info[0].iters = steps + h.iters(0);
    info[0].mvps = steps + h.mvps(0) + (p.x0_zero ? 0 : 1);
    info[0].restarts = h.restarts(0);
    info[0].converged = h.converged(0);
    info[0].est_relres = st.bnorm1 > 0.0 ? st.rho / st.bnorm1 : 0.0;
    info[0].true_relres = h.relres(0);
  }
  ctx->seeded = true;
  ctx->basis_valid = false;   // V holds FP32 vectors: no FP64 projection from it
  if (!h.converged(0)) return fail(ctx, SEED_ENOTCONV, "system 1 did not reach tol_seed within maxit_rest");
  return SEED_OK;
}

template <class T64, class T32>
seed_status solve_rest_mixed(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int nrhs,
                             seed_info *info) {
  const int nc = nrhs - 1;
  if (info) std::memset(info + 1, 0, sizeof(seed_info) * (nc > 0 ? nc : 0));
  if (nc <= 0) return SEED_OK;
  TRY(ensure_cols(ctx, nrhs));
  CU(cudaEventRecord(ctx->t2, ctx->cs));
  TRY((mixed_cg<T64, T32>(ctx, (const T64 *)B + ldb, ldb, (T64 *)X + ldx, ldx, 1, nc, ctx->prm.tol_rest, nullptr)));
  CU(cudaEventRecord(ctx->t3, ctx->cs));
  CgHost h;
  TRY(read_cg(ctx, &h));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->t2, ctx->t3);
  ctx->stats.ms_rest = ms;
  bool all = true;
  int64_t mv = 0;
  for (int j = 0; j < nc; ++j) {
    all &= h.converged(j) != 0;
    mv += h.mvps(j);
    if (info) {
      seed_info &o = info[j + 1];
      o.iters = h.iters(j);
      o.mvps = h.mvps(j);
      o.restarts = h.restarts(j);
      o.converged = h.converged(j);
      o.est_relres = h.relres(j);
      o.true_relres = h.relres(j);
    }
  }
  ctx->stats.mvps += mv - nc;
  if (!all) return fail(ctx, SEED_ENOTCONV, "CG did not reach tol_rest on every system within maxit_rest");
  return SEED_OK;
}

seed_status check_block(seed_ctx *ctx, const void *A, int64_t lda, int cols, const char *name) {
  if (cols < 1 || cols > kMaxRhs) return fail(ctx, SEED_EINVAL, std::string("number of columns must be 1..64 (") + name + ")");
  if (lda < ctx->n) return fail(ctx, SEED_EINVAL, std::string("leading dimension < n (") + name + ")");
  if (!is_device_ptr(A, ctx->device)) return fail(ctx, SEED_EINVAL, std::string(name) + " is not a device pointer on the context's device");
  return SEED_OK;
}

bool overlap(const void *a, int64_t lda, const void *b, int64_t ldb, int cols, int64_t n, size_t es) {
  const char *a0 = (const char *)a, *a1 = a0 + ((cols - 1) * lda + n) * es;
  const char *b0 = (const char *)b, *b1 = b0 + ((cols - 1) * ldb + n) * es;
  return a0 < b1 && b0 < a1;
}

// Order the internal stream after the caller's, and back.  Inside
// seed_batch_solve the ordering is done once for the whole batch instead:
// several contexts usually share the caller's stream, and per-call ordering
// through it would make every problem wait for the ones before it.
struct StreamScope {
  seed_ctx *ctx;
  explicit StreamScope(seed_ctx *c) : ctx(c) {
    if (ctx->in_batch) return;
    cudaEventRecord(ctx->ev_in, ctx->user_stream);
    cudaStreamWaitEvent(ctx->cs, ctx->ev_in, 0);
  }
  ~StreamScope() {
    if (ctx->in_batch) return;
    cudaEventRecord(ctx->ev_in, ctx->cs);
    cudaStreamWaitEvent(ctx->user_stream, ctx->ev_in, 0);
  }
};

seed_status create_common(seed_ctx *ctx, const seed_params *p, seed_stream stream) {
  TRY(check_params(ctx, p));
  ctx->prm = *p;
  ctx->allow_persistent = p->kernel_path != 1;
  ctx->allow_persistent_cg = p->kernel_path == 2 && p->precision == 0;
  ctx->allow_small_cg = p->kernel_path != 1;
  ctx->precision = p->precision;
  // mixed precision: persistent seed runs in FP32, no persistent CG
  CU(cudaGetDevice(&ctx->device));
  ctx->user_stream = (cudaStream_t)stream;
  CU(cudaStreamCreateWithFlags(&ctx->cs, cudaStreamNonBlocking));
  for (int b = 0; b < kCgBranches - 1; ++b) {
    CU(cudaStreamCreateWithFlags(&ctx->csb[b], cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&ctx->ev_join[b], cudaEventDisableTiming));
  }
  CU(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&ctx->ev_run[0], cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&ctx->ev_run[1], cudaEventDisableTiming));
  CU(cudaEventCreate(&ctx->t0));
  CU(cudaEventCreate(&ctx->t1));
  CU(cudaEventCreate(&ctx->t2));
  CU(cudaEventCreate(&ctx->t3));
  return SEED_OK;
}

void destroy(seed_ctx *ctx) {
  if (!ctx) return;
  if (ctx->cs) cudaStreamSynchronize(ctx->cs);
  for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
  void *ptrs[] = {ctx->V, ctx->u, ctx->f, ctx->w, ctx->st, ctx->alpha_hist, ctx->beta_hist,
                  ctx->delta_hist, ctx->eta, ctx->partials, ctx->tickets, ctx->Hpart, ctx->H, ctx->call,
                  ctx->colnorm, ctx->R, ctx->P, ctx->Q, ctx->T, ctx->cg_d, ctx->cg_i, ctx->nbr,
                  ctx->gsync, ctx->f2, ctx->tpart, ctx->op32, ctx->R32, ctx->P32, ctx->Q32,
                  ctx->T32, ctx->E32, ctx->call32, ctx->Rrel, ctx->xrel, ctx->rrel, ctx->reldots,
                  ctx->msX, ctx->msR, ctx->Wb, ctx->gamma_hist, ctx->blk.Hpart, ctx->blk.G, ctx->blk.Z,
                  ctx->tc_err, ctx->rhpart, ctx->Hrows};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_gerr) cudaFreeHost(ctx->h_gerr);
  cudaEvent_t evs[] = {ctx->ev_in, ctx->t0, ctx->t1, ctx->t2, ctx->t3, ctx->ev_fork, ctx->ev_run[0], ctx->ev_run[1]};
  for (auto e : evs)
    if (e) cudaEventDestroy(e);
  for (int b = 0; b < kCgBranches - 1; ++b) {
    if (ctx->ev_join[b]) cudaEventDestroy(ctx->ev_join[b]);
    if (ctx->csb[b]) cudaStreamDestroy(ctx->csb[b]);
  }
  if (ctx->cs) cudaStreamDestroy(ctx->cs);
  delete ctx;
}

}  // namespace

namespace seedk {
// lets entry points in other translation units report through seed_last_error(NULL)
void set_last_error_message(const std::string &msg) { g_last_error = msg; }
}  // namespace seedk

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int32_t seed_abi_version(void) { return SEED_ABI_VERSION; }

seed_status seed_params_default(seed_params *p) {
  if (!p) return fail(nullptr, SEED_EINVAL, "params is NULL");
  p->m_max = 1000;
  p->reorth_freq = 0;
  p->reorth_passes = 2;
  p->extra_iters = 0;
  p->keep_basis = 0;
  p->x0_zero = 1;
  p->maxit_rest = 100000;
  p->max_restarts = 3;
  p->tol_seed = 1e-12;
  p->tol_rest = 1e-8;
  p->breakdown_rel = 1e-14;
  p->kernel_path = 0;
  p->precision = 0;
  p->autotune = 0;
  p->reliable_delta = 0.0;
  return SEED_OK;
}

seed_status seed_create_csr(seed_ctx **out, const seed_csr *A, const seed_params *p, seed_stream stream) {
  if (!out) return fail(nullptr, SEED_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A) return fail(nullptr, SEED_EINVAL, "operator is NULL");
  if (A->n < 1 || A->n > ((int64_t)1 << 31) - 1) return fail(nullptr, SEED_EINVAL, "n must be in [1, 2^31)");
  if (A->nnz < 0 || A->nnz > ((int64_t)1 << 31) - 1) return fail(nullptr, SEED_EINVAL, "nnz must be in [0, 2^31)");
  seed_ctx *ctx = new seed_ctx();
  seed_status s = create_common(ctx, p, stream);
  if (s != SEED_OK) { destroy(ctx); return s; }
  if (!is_device_ptr(A->row_ptr, ctx->device) || !is_device_ptr(A->col_idx, ctx->device) ||
      !is_device_ptr(A->vals, ctx->device)) {
    destroy(ctx);
    return fail(nullptr, SEED_EINVAL, "CSR arrays must be device pointers on the current device");
  }
  // structural check on the host before any kernel reads the arrays
  std::vector<int32_t> rp(A->n + 1), ci(A->nnz);
  if (cudaMemcpy(rp.data(), A->row_ptr, sizeof(int32_t) * (A->n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
      (A->nnz && cudaMemcpy(ci.data(), A->col_idx, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost) != cudaSuccess)) {
    cudaGetLastError();
    destroy(ctx);
    return fail(nullptr, SEED_ECUDA, "could not read the CSR arrays");
  }
  if (rp[0] != 0 || rp[A->n] != A->nnz) { destroy(ctx); return fail(nullptr, SEED_EINVAL, "row_ptr[0] != 0 or row_ptr[n] != nnz"); }
  for (int64_t r = 0; r < A->n; ++r)
    if (rp[r + 1] < rp[r]) { destroy(ctx); return fail(nullptr, SEED_EINVAL, "row_ptr is not nondecreasing"); }
  for (int64_t k = 0; k < A->nnz; ++k)
    if (ci[k] < 0 || ci[k] >= A->n) { destroy(ctx); return fail(nullptr, SEED_EINVAL, "col_idx out of range"); }
  ctx->kind = 0;
  ctx->dtype = SEED_F64;
  ctx->n = A->n;
  ctx->esz = sizeof(double);
  ctx->vsz = ctx->precision == 1 ? sizeof(float) : sizeof(double);
  ctx->nv = A->n;
  ctx->lay = Layout32{0};
  ctx->csr = CsrOp{A->n, A->row_ptr, A->col_idx, A->vals};
  s = alloc_common(ctx);
  if (s == SEED_OK && ctx->precision == 1) {
    s = dalloc(ctx, &ctx->op32, sizeof(float) * (size_t)(A->nnz > 0 ? A->nnz : 1));
    if (s == SEED_OK) {
      if (A->nnz > 0)
        launch_to_low<double, float>(A->vals, A->nnz, (float *)ctx->op32, A->nnz, A->nnz, Layout32{0}, 1, ctx->cs);
      ctx->stats.kernel_launches += A->nnz > 0;
      ctx->csr32 = CsrOp32{A->n, A->row_ptr, A->col_idx, (const float *)ctx->op32};
    }
  }
  if (s == SEED_OK && ctx->prm.autotune) s = autotune_csr(ctx, A->nnz);
  if (s == SEED_OK && cudaStreamSynchronize(ctx->cs) != cudaSuccess) s = fail(ctx, SEED_ECUDA, "set-up failed");
  if (s != SEED_OK) { g_last_error = ctx->err; destroy(ctx); return s; }
  *out = ctx;
  return SEED_OK;
}

seed_status seed_create_wilson(seed_ctx **out, const seed_wilson *A, const seed_params *p, seed_stream stream) {
  if (!out) return fail(nullptr, SEED_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A) return fail(nullptr, SEED_EINVAL, "operator is NULL");
  int64_t vol = 1;
  for (int k = 0; k < 4; ++k) {
    if (A->dims[k] < 2 || A->dims[k] > 4096) return fail(nullptr, SEED_EINVAL, "lattice dims must be in [2, 4096]");
    vol *= A->dims[k];
  }
  if (vol * 12 > ((int64_t)1 << 31) - 1) return fail(nullptr, SEED_EINVAL, "lattice too large (12*sites >= 2^31)");
  if (A->bc_t != 0 && A->bc_t != 1) return fail(nullptr, SEED_EINVAL, "bc_t must be 0 or 1");
  if (!std::isfinite(A->kappa)) return fail(nullptr, SEED_EINVAL, "kappa is not finite");
  seed_ctx *ctx = new seed_ctx();
  seed_status s = create_common(ctx, p, stream);
  if (s != SEED_OK) { destroy(ctx); return s; }
  if (!is_device_ptr(A->links, ctx->device)) {
    destroy(ctx);
    return fail(nullptr, SEED_EINVAL, "links must be a device pointer on the current device");
  }
  ctx->kind = 1;
  ctx->dtype = SEED_C128;
  ctx->n = 12 * vol;
  ctx->esz = sizeof(double2);
  ctx->vsz = ctx->precision == 1 ? sizeof(float2) : sizeof(double2);
  ctx->lay = Layout32{ctx->precision == 1 ? vol : 0};
  ctx->nv = ctx->lay.length(ctx->n);
  s = alloc_common(ctx);
  if (s == SEED_OK) s = dalloc(ctx, &ctx->nbr, sizeof(int32_t) * 8 * vol);
  if (s == SEED_OK && ctx->precision == 1) {
    const int64_t nl = 4 * vol * 9;
    s = dalloc(ctx, &ctx->op32, sizeof(float2) * (size_t)nl);
    if (s == SEED_OK) {
      launch_links_soa32((const double2 *)A->links, (float2 *)ctx->op32, vol, ctx->cs);
      ctx->stats.kernel_launches += 1;
    }
  }
  if (s == SEED_OK) {
    launch_wilson_neighbors(A->dims, ctx->nbr, ctx->cs);
    ctx->stats.kernel_launches += 1;
    for (int k = 0; k < 4; ++k) ctx->wil.dims[k] = A->dims[k];
    ctx->wil.sites = vol;
    ctx->wil.kappa = A->kappa;
    ctx->wil.bc_t = A->bc_t;
    ctx->wil.links = (const double2 *)A->links;
    ctx->wil.nbr = ctx->nbr;
    for (int k = 0; k < 4; ++k) ctx->wil32.dims[k] = A->dims[k];
    ctx->wil32.sites = vol;
    ctx->wil32.kappa = A->kappa;
    ctx->wil32.bc_t = A->bc_t;
    ctx->wil32.links = (const float2 *)ctx->op32;
    ctx->wil32.nbr = ctx->nbr;
    if (cudaStreamSynchronize(ctx->cs) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      s = fail(ctx, SEED_ECUDA, "neighbour table build failed");
  }
  if (s != SEED_OK) { g_last_error = ctx->err; destroy(ctx); return s; }
  *out = ctx;
  return SEED_OK;
}

seed_status seed_solve_first(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t nrhs,
                             seed_info *info) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  TRY(check_block(ctx, B, ldb, nrhs, "B"));
  TRY(check_block(ctx, X, ldx, nrhs, "X"));
  if (overlap(B, ldb, X, ldx, nrhs, ctx->n, ctx->esz)) return fail(ctx, SEED_EINVAL, "B and X overlap");
  StreamScope scope(ctx);
  if (ctx->precision == 1) {
    if (ctx->kind == 0) return solve_first_mixed<double, float>(ctx, B, ldb, X, ldx, nrhs, info);
    return solve_first_mixed<double2, float2>(ctx, B, ldb, X, ldx, nrhs, info);
  }
  if (ctx->kind == 0) return solve_first_impl<double>(ctx, B, ldb, X, ldx, nrhs, info);
  return solve_first_impl<double2>(ctx, B, ldb, X, ldx, nrhs, info);
}

seed_status seed_solve_rest(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t nrhs,
                            seed_info *info) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  TRY(check_block(ctx, B, ldb, nrhs, "B"));
  TRY(check_block(ctx, X, ldx, nrhs, "X"));
  if (overlap(B, ldb, X, ldx, nrhs, ctx->n, ctx->esz)) return fail(ctx, SEED_EINVAL, "B and X overlap");
  StreamScope scope(ctx);
  if (ctx->precision == 1) {
    if (ctx->kind == 0) return solve_rest_mixed<double, float>(ctx, B, ldb, X, ldx, nrhs, info);
    return solve_rest_mixed<double2, float2>(ctx, B, ldb, X, ldx, nrhs, info);
  }
  if (ctx->kind == 0) return solve_rest_impl<double>(ctx, B, ldb, X, ldx, nrhs, info);
  return solve_rest_impl<double2>(ctx, B, ldb, X, ldx, nrhs, info);
}

seed_status seed_solve_cg(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t ncols,
                          seed_info *info) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  TRY(check_block(ctx, B, ldb, ncols, "B"));
  TRY(check_block(ctx, X, ldx, ncols, "X"));
  if (overlap(B, ldb, X, ldx, ncols, ctx->n, ctx->esz)) return fail(ctx, SEED_EINVAL, "B and X overlap");
  StreamScope scope(ctx);
  TRY(ensure_cols(ctx, ncols));
  if (ctx->precision == 1) {
    if (info) std::memset(info, 0, sizeof(seed_info) * ncols);
    CU(cudaEventRecord(ctx->t2, ctx->cs));
    seed_status st;
    if (ctx->kind == 0)
      st = mixed_cg<double, float>(ctx, (const double *)B, ldb, (double *)X, ldx, 0, ncols, ctx->prm.tol_rest, nullptr);
    else
      st = mixed_cg<double2, float2>(ctx, (const double2 *)B, ldb, (double2 *)X, ldx, 0, ncols, ctx->prm.tol_rest,
                                     nullptr);
    TRY(st);
    CU(cudaEventRecord(ctx->t3, ctx->cs));
    CgHost h;
    TRY(read_cg(ctx, &h));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->t2, ctx->t3);
    ctx->stats.ms_rest = ms;
    bool all = true;
    for (int j = 0; j < ncols; ++j) {
      all &= h.converged(j) != 0;
      ctx->stats.mvps += h.mvps(j);
      if (info) {
        info[j].iters = h.iters(j);
        info[j].mvps = h.mvps(j);
        info[j].restarts = h.restarts(j);
        info[j].converged = h.converged(j);
        info[j].est_relres = info[j].true_relres = h.relres(j);
      }
    }
    if (!all) return fail(ctx, SEED_ENOTCONV, "CG did not reach tol_rest on every system within maxit_rest");
    return SEED_OK;
  }
  if (ctx->kind == 0) return cg_impl<double>(ctx, (const double *)B, ldb, (double *)X, ldx, ncols, info);
  return cg_impl<double2>(ctx, (const double2 *)B, ldb, (double2 *)X, ldx, ncols, info);
}

seed_status seed_solve_related(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t nrhs,
                               seed_info *info) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  if (ctx->precision != 0) return fail(ctx, SEED_EINVAL, "seed_solve_related runs in FP64 (precision = 0)");
  if (!ctx->prm.x0_zero) return fail(ctx, SEED_EINVAL, "seed_solve_related assumes no initial guesses (x0_zero = 1)");
  if (!ctx->seeded) return fail(ctx, SEED_ESTATE, "seed_solve_related follows seed_solve_first");
  TRY(check_block(ctx, B, ldb, nrhs, "B"));
  TRY(check_block(ctx, X, ldx, nrhs, "X"));
  if (overlap(B, ldb, X, ldx, nrhs, ctx->n, ctx->esz)) return fail(ctx, SEED_EINVAL, "B and X overlap");
  StreamScope scope(ctx);
  if (ctx->kind == 0) return solve_related_impl<double>(ctx, B, ldb, X, ldx, nrhs, info);
  return solve_related_impl<double2>(ctx, B, ldb, X, ldx, nrhs, info);
}

seed_status seed_solve_multiple(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t nrhs,
                                seed_info *info) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  if (ctx->precision != 0) return fail(ctx, SEED_EINVAL, "seed_solve_multiple runs in FP64 (precision = 0)");
  TRY(check_block(ctx, B, ldb, nrhs, "B"));
  TRY(check_block(ctx, X, ldx, nrhs, "X"));
  if (overlap(B, ldb, X, ldx, nrhs, ctx->n, ctx->esz)) return fail(ctx, SEED_EINVAL, "B and X overlap");
  StreamScope scope(ctx);
  if (ctx->kind == 0) return solve_multiple_impl<double>(ctx, B, ldb, X, ldx, nrhs, info);
  return solve_multiple_impl<double2>(ctx, B, ldb, X, ldx, nrhs, info);
}

seed_status seed_grad_kappa(seed_ctx *ctx, const void *Lambda, int64_t ldl, const void *X, int64_t ldx, int32_t ncols,
                            double *out) {
  if (!ctx || !out) return fail(ctx, SEED_EINVAL, "NULL argument");
  if (ctx->kind != 1) return fail(ctx, SEED_EINVAL, "seed_grad_kappa needs a Wilson context");
  TRY(check_block(ctx, Lambda, ldl, ncols, "Lambda"));
  TRY(check_block(ctx, X, ldx, ncols, "X"));
  StreamScope scope(ctx);
  launch_dkappa_inner(ctx->wil, (const double2 *)Lambda, ldl, (const double2 *)X, ldx, ncols, ctx->partials,
                      ctx->tickets, ctx->colnorm, ctx->cs);
  ctx->stats.kernel_launches += 1;
  std::vector<double> v(ncols);
  CU(cudaMemcpyAsync(v.data(), ctx->colnorm, sizeof(double) * ncols, cudaMemcpyDeviceToHost, ctx->cs));
  CU(cudaStreamSynchronize(ctx->cs));
  CU(cudaGetLastError());
  double t = 0.0;
  for (int j = 0; j < ncols; ++j) t += v[j];
  *out = t;
  return SEED_OK;
}

seed_status seed_project(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t ncols) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  if (!ctx->prm.keep_basis || !ctx->basis_valid)
    return fail(ctx, SEED_ESTATE, "seed_project needs keep_basis = 1 and a finished seed_solve_first");
  TRY(check_block(ctx, B, ldb, ncols, "B"));
  TRY(check_block(ctx, X, ldx, ncols, "X"));
  if (overlap(B, ldb, X, ldx, ncols, ctx->n, ctx->esz)) return fail(ctx, SEED_EINVAL, "B and X overlap");
  TRY(ensure_cols(ctx, ncols));
  StreamScope scope(ctx);
  const int64_t n = ctx->n, ld = ctx->ldv;
  int kern = 0;
  if (ctx->kind == 0) {
    if (ctx->prm.x0_zero) {
      launch_zero_cols<double>((double *)X, ldx, n, ncols, ctx->cs);
      launch_copy_cols<double>((const double *)B, ldb, (double *)ctx->R, ld, n, ncols, ctx->cs);
      kern += 2;
    } else {
      kern += apply_A(ctx, X, ldx, ctx->Q, ld, ncols, nullptr);
      launch_sub_from<double>((const double *)B, ldb, (const double *)ctx->Q, ld, (double *)ctx->R, ld, n, ncols, ctx->cs);
      kern += 1;
      ctx->stats.mvps += ncols;
    }
    launch_project<double>(n, (const double *)ctx->V, ctx->ldv, ctx->last_m, ctx->alpha_hist, ctx->beta_hist,
                           (const double *)ctx->R, ld, (double *)X, ldx, ncols, ctx->H, ctx->Hpart, ctx->nrb,
                           ctx->rows_per_item, ctx->cs);
  } else {
    if (ctx->prm.x0_zero) {
      launch_zero_cols<double2>((double2 *)X, ldx, n, ncols, ctx->cs);
      launch_copy_cols<double2>((const double2 *)B, ldb, (double2 *)ctx->R, ld, n, ncols, ctx->cs);
      kern += 2;
    } else {
      kern += apply_A(ctx, X, ldx, ctx->Q, ld, ncols, nullptr);
      launch_sub_from<double2>((const double2 *)B, ldb, (const double2 *)ctx->Q, ld, (double2 *)ctx->R, ld, n, ncols,
                               ctx->cs);
      kern += 1;
      ctx->stats.mvps += ncols;
    }
    launch_project<double2>(n, (const double2 *)ctx->V, ctx->ldv, ctx->last_m, ctx->alpha_hist, ctx->beta_hist,
                            (const double2 *)ctx->R, ld, (double2 *)X, ldx, ncols, ctx->H, ctx->Hpart, ctx->nrb,
                            ctx->rows_per_item, ctx->cs);
  }
  ctx->stats.kernel_launches += kern + 4 * ((ncols + 1) / 2);
  CU(cudaGetLastError());
  return SEED_OK;
}

seed_status seed_apply(seed_ctx *ctx, int32_t op, const void *X, int64_t ldx, void *Y, int64_t ldy, int32_t ncols) {
  if (!ctx) return fail(nullptr, SEED_EINVAL, "ctx is NULL");
  if (op < 0 || op > 7 || ((op == 1 || op == 2 || op >= 4) && ctx->kind != 1))
    return fail(ctx, SEED_EINVAL, "op must be 0 (A), or 1 (D) / 2 (D^H) for Wilson; 3..7 in FP32");
  if (op >= 3 && ctx->precision != 1) return fail(ctx, SEED_EINVAL, "ops 3..7 need a mixed-precision context");
  TRY(check_block(ctx, X, ldx, ncols, "X"));
  TRY(check_block(ctx, Y, ldy, ncols, "Y"));
  const bool tiled = op >= 6;   // the solver's tiled FP32 layout: columns of length nv
  const int64_t len = tiled ? ctx->nv : ctx->n;
  if (tiled && (ldx < len || ldy < len))
    return fail(ctx, SEED_EINVAL, "leading dimension < the tiled column length 384 * ceil(sites / 32)");
  const size_t es = op >= 3 ? ctx->vsz : ctx->esz;
  if (overlap(X, ldx, Y, ldy, ncols, len, es)) return fail(ctx, SEED_EINVAL, "X and Y overlap");
  TRY(ensure_cols(ctx, ncols));
  StreamScope scope(ctx);
  if (op == 3) {
    ctx->stats.kernel_launches += apply_A32(ctx, X, ldx, Y, ldy, ncols, nullptr, false);
  } else if (op >= 4) {
    launch_wilson_dslash32(ctx->wil32, (op == 4 || op == 6) ? +1 : -1, (const float2 *)X, ldx, (float2 *)Y, ldy,
                           ncols, nullptr, tiled, ctx->cs);
    ctx->stats.kernel_launches += 1;
  } else if (op == 0) {
    ctx->stats.kernel_launches += apply_A(ctx, X, ldx, Y, ldy, ncols, nullptr);
    ctx->stats.mvps += ncols;
  } else {
    launch_wilson_dslash(ctx->wil, op == 1 ? +1 : -1, (const double2 *)X, ldx, (double2 *)Y, ldy, ncols, nullptr,
                         ctx->cs);
    ctx->stats.kernel_launches += 1;
  }
  CU(cudaGetLastError());
  return SEED_OK;
}

int32_t seed_inject_alloc_failure(int32_t k) { return g_alloc_countdown.exchange(k > 0 ? k : 0); }

seed_status seed_check_barrier_timeout(seed_stream stream, int32_t *timed_out, double *ms) {
  seed_ctx *ctx = nullptr;   // for CU()
  if (!timed_out || !ms) return fail(nullptr, SEED_EINVAL, "NULL argument");
  int dev = 0, coop = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(nullptr, SEED_ECUDA, "the device has no cooperative launch");
  const cudaStream_t s = (cudaStream_t)stream;
  unsigned *w = nullptr;
  if (cudaMalloc(&w, sizeof(unsigned) * kGridSyncWords) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, SEED_ENOMEM, "cudaMalloc of the barrier words failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  GridSync g;
  g.count = w;
  g.release = w + 1;
  g.error = reinterpret_cast<int *>(w + 2);
  g.owners = w + 3;
  g.sm_slots = w + 4;
  int32_t err = 0;
  float t = 0.f;
  cudaError_t e = cudaMemsetAsync(w, 0, sizeof(unsigned) * kGridSyncWords, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_barrier_timeout_check(g, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&err, g.error, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(w);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, SEED_ECUDA, std::string("barrier self-test: ") + cudaGetErrorString(e));
  }
  *timed_out = err != 0;
  *ms = t;
  return SEED_OK;
}

seed_status seed_wilson_neighbors(const int32_t dims[4], int32_t *nbr, seed_stream stream) {
  seed_ctx *ctx = nullptr;
  if (!dims || !nbr) return fail(nullptr, SEED_EINVAL, "NULL argument");
  for (int k = 0; k < 4; ++k)
    if (dims[k] < 1 || dims[k] > 4096) return fail(nullptr, SEED_EINVAL, "lattice dims must be in [1, 4096]");
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (!is_device_ptr(nbr, dev)) return fail(nullptr, SEED_EINVAL, "nbr must be a device pointer");
  launch_wilson_neighbors(dims, nbr, (cudaStream_t)stream);
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  CU(cudaGetLastError());
  return SEED_OK;
}

seed_status seed_get_tridiag(const seed_ctx *cctx, double *alpha, double *beta, int32_t cap, int32_t *m) {
  seed_ctx *ctx = const_cast<seed_ctx *>(cctx);
  if (!ctx || !m) return fail(ctx, SEED_EINVAL, "NULL argument");
  if (!ctx->seeded) return fail(ctx, SEED_ESTATE, "no finished seed_solve_first");
  *m = ctx->last_m;
  if (!alpha && !beta) return SEED_OK;   // size query
  if (cap < ctx->last_m + 1) return fail(ctx, SEED_EINVAL, "cap < m + 1");
  if (alpha && ctx->last_m > 0)
    CU(cudaMemcpy(alpha, ctx->alpha_hist + 1, sizeof(double) * ctx->last_m, cudaMemcpyDeviceToHost));
  if (beta) CU(cudaMemcpy(beta, ctx->beta_hist, sizeof(double) * (ctx->last_m + 1), cudaMemcpyDeviceToHost));
  return SEED_OK;
}

seed_status seed_get_basis(const seed_ctx *cctx, void *V_host, int32_t ncols) {
  seed_ctx *ctx = const_cast<seed_ctx *>(cctx);
  if (!ctx || !V_host) return fail(ctx, SEED_EINVAL, "NULL argument");
  if (!ctx->seeded || ncols < 0 || ncols > ctx->last_m) return fail(ctx, SEED_EINVAL, "ncols out of range");
  if (ctx->precision == 1) return fail(ctx, SEED_ESTATE, "the basis of a mixed-precision context is FP32");
  CU(cudaMemcpy2D(V_host, ctx->n * ctx->esz, ctx->V, ctx->ldv * ctx->esz, ctx->n * ctx->esz, ncols,
                  cudaMemcpyDeviceToHost));
  return SEED_OK;
}

seed_status seed_time_operator(seed_ctx *ctx, int32_t op, int32_t ncols, int32_t reps, double *ms_per_apply) {
  if (!ctx || !ms_per_apply) return fail(ctx, SEED_EINVAL, "NULL argument");
  if (op < 0 || op > 5 || ((op == 1 || op == 2 || op == 4 || op == 5) && ctx->kind != 1))
    return fail(ctx, SEED_EINVAL, "bad op");
  if (op >= 3 && ctx->precision != 1) return fail(ctx, SEED_EINVAL, "ops 3..5 need a mixed-precision context");
  if (ncols < 1 || ncols > kMaxRhs || reps < 1 || reps > 100000) return fail(ctx, SEED_EINVAL, "bad ncols / reps");
  TRY(ensure_cols(ctx, ncols));
  StreamScope scope(ctx);
  CU(cudaMemsetAsync(ctx->P, 0x3F, (size_t)ctx->ldv * ncols * ctx->esz, ctx->cs));   // normal doubles ~4.8e-4
  if (op >= 3) CU(cudaMemsetAsync(ctx->P32, 0x3F, (size_t)ctx->ldv * ncols * ctx->vsz, ctx->cs));   // floats ~0.75
  // one untimed launch, then the timed ones
  for (int r = 0; r <= reps; ++r) {
    if (r == 1) CU(cudaEventRecord(ctx->t0, ctx->cs));
    if (op == 0) {
      ctx->stats.kernel_launches += apply_A(ctx, ctx->P, ctx->ldv, ctx->Q, ctx->ldv, ncols, nullptr);
    } else if (op == 3) {
      ctx->stats.kernel_launches += apply_A32(ctx, ctx->P32, ctx->ldv, ctx->Q32, ctx->ldv, ncols, nullptr);
    } else if (op >= 4) {
      launch_wilson_dslash32(ctx->wil32, op == 4 ? +1 : -1, (const float2 *)ctx->P32, ctx->ldv, (float2 *)ctx->Q32,
                             ctx->ldv, ncols, nullptr, true, ctx->cs);
      ctx->stats.kernel_launches += 1;
    } else {
      launch_wilson_dslash(ctx->wil, op == 1 ? +1 : -1, (const double2 *)ctx->P, ctx->ldv, (double2 *)ctx->Q,
                           ctx->ldv, ncols, nullptr, ctx->cs);
      ctx->stats.kernel_launches += 1;
    }
  }
  CU(cudaEventRecord(ctx->t1, ctx->cs));
  CU(cudaEventSynchronize(ctx->t1));
  CU(cudaGetLastError());
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, ctx->t0, ctx->t1));
  *ms_per_apply = (double)ms / reps;
  return SEED_OK;
}

seed_status seed_batch_solve(seed_ctx *const *ctxs, const void *const *B, const int64_t *ldb, void *const *X,
                             const int64_t *ldx, const int32_t *nrhs, int32_t nprob, int32_t workers,
                             seed_info *const *info) {
  if (!ctxs || !B || !ldb || !X || !ldx || !nrhs) return fail(nullptr, SEED_EINVAL, "NULL argument");
  if (nprob < 1 || nprob > 4096) return fail(nullptr, SEED_EINVAL, "nprob must be in [1, 4096]");
  if (workers < 0) return fail(nullptr, SEED_EINVAL, "workers must be >= 0");
  std::set<const seed_ctx *> seen;
  for (int i = 0; i < nprob; ++i) {
    if (!ctxs[i]) return fail(nullptr, SEED_EINVAL, "a context is NULL");
    if (!seen.insert(ctxs[i]).second) return fail(nullptr, SEED_EINVAL, "a context appears twice in the batch");
  }
  // largest problems first (longest-processing-time order), so that the small
  // ones fill the GPU around them
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return ctxs[a]->n * (int64_t)nrhs[a] > ctxs[b]->n * (int64_t)nrhs[b];
  });
  const int W = workers > 0 ? std::min<int>(workers, nprob) : std::min<int>(nprob, 32);
  // every context starts after the work already queued on its caller's stream ...
  for (int i = 0; i < nprob; ++i) {
    seed_ctx *c = ctxs[i];
    if (cudaSetDevice(c->device) != cudaSuccess || cudaEventRecord(c->ev_in, c->user_stream) != cudaSuccess ||
        cudaStreamWaitEvent(c->cs, c->ev_in, 0) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, SEED_ECUDA, "stream ordering at the start of the batch failed");
    }
    c->in_batch = true;
  }
  std::vector<seed_status> st(nprob, SEED_OK);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int k = next.fetch_add(1); k < nprob; k = next.fetch_add(1)) {
      const int i = order[k];
      seed_ctx *c = ctxs[i];
      if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        st[i] = fail(c, SEED_ECUDA, "cudaSetDevice failed in a batch worker");
        continue;
      }
      // persistent seed runs and small-problem CG runs of different problems may
      // run side by side (each waits only on its own blocks, every wait is
      // time-bounded); the full-grid persistent CG stays off in a batch
      const bool p0 = c->allow_persistent, p1 = c->allow_persistent_cg, p2 = c->allow_small_cg;
      c->allow_persistent_cg = false;
      seed_info *inf = info ? info[i] : nullptr;
      st[i] = seed_solve_first(c, B[i], ldb[i], X[i], ldx[i], nrhs[i], inf);
      if (st[i] == SEED_OK) st[i] = seed_solve_rest(c, B[i], ldb[i], X[i], ldx[i], nrhs[i], inf);
      c->allow_persistent = p0;
      c->allow_persistent_cg = p1;
      c->allow_small_cg = p2;
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < W; ++w) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  // ... and the callers' streams continue after every context's work
  for (int i = 0; i < nprob; ++i) {
    seed_ctx *c = ctxs[i];
    c->in_batch = false;
    cudaSetDevice(c->device);
    cudaEventRecord(c->ev_in, c->cs);
    cudaStreamWaitEvent(c->user_stream, c->ev_in, 0);
  }
  for (int i = 0; i < nprob; ++i)
    if (st[i] != SEED_OK) {
      g_last_error = "problem " + std::to_string(i) + ": " + ctxs[i]->err;
      return st[i];
    }
  return SEED_OK;
}

seed_status seed_get_stats(const seed_ctx *ctx, seed_stats *out) {
  if (!ctx || !out) return fail(nullptr, SEED_EINVAL, "NULL argument");
  *out = ctx->stats;
  out->csr_tpr = ctx->kind == 0 ? ctx->csr.tpr : 0;
  out->csr_block = ctx->kind == 0 ? ctx->csr.block : 0;
  return SEED_OK;
}

const char *seed_last_error(const seed_ctx *ctx) {
  if (ctx) return ctx->err.c_str();
  return g_last_error.c_str();
}

void seed_destroy(seed_ctx *ctx) { destroy(ctx); }

}  // extern "C"
