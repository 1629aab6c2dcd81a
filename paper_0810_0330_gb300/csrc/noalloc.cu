// noalloc.cu -- Y = D^H D X for the Wilson operator with no device allocation.
//
// Who needs this: code that must not call cudaMalloc once it is running --
// for example a host loop that is being recorded into a CUDA graph (an
// allocation there is not allowed), a latency-critical service whose device
// memory is fixed at start-up, or a plug-in inside a framework that owns the
// whole device heap.  seed_create_wilson allocates a context (the Lanczos basis,
// the neighbour table, work columns), so such callers cannot use it.
//
// This entry point needs two pieces of scratch beyond the caller's X and Y:
// the site -> neighbour table and the intermediate T = D X.  Both live in one
// file-scope device array of fixed size (kNoAllocScratchBytes), which every GPU
// that loads this library holds until the process exits.  Host code may not
// hand the array's name to a kernel (on the host it is only a stand-in
// symbol), so the first call on each device looks up its device address with
// cudaGetSymbolAddress while that device is current and keeps it -- keyed on
// the CUDA context that is current, not only on the device index: a context
// that was reset (cudaDeviceReset) or a different driver context made current
// by the caller holds its own copy of the array at another address, and the
// lookup is then repeated for it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "seed.h"
#include "seed_internal.h"

namespace seedk {
void set_last_error_message(const std::string &msg);   // engine.cu
}

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;   // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
// device address of g_noalloc_scratch, per device, and the id of the context it was looked up in
void *g_scratch_dev[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// The id of the CUDA context current on this thread (unique over the process'
// life, never reused), read through the runtime's driver entry points so the
// library needs no link to the driver library.  0 when unavailable.
typedef int (*PfnCtxGetCurrent)(void **);
typedef int (*PfnCtxGetId)(void *, unsigned long long *);
struct CtxFns {
  PfnCtxGetCurrent get_current = nullptr;
  PfnCtxGetId get_id = nullptr;
};
unsigned long long current_context_id() {
  static const CtxFns fns = [] {   // looked up once (thread-safe static initialisation)
    CtxFns r;
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      r.get_current = (PfnCtxGetCurrent)f1;
      r.get_id = (PfnCtxGetId)f2;
    }
    cudaGetLastError();
    return r;
  }();
  const PfnCtxGetCurrent get_current = fns.get_current;
  const PfnCtxGetId get_id = fns.get_id;
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || ctx == nullptr || get_id(ctx, &id) != 0) return 0;
  return id;
}

seed_status na_fail(seed_status st, const std::string &msg) {
  seedk::set_last_error_message(msg);
  return st;
}

bool na_device_ptr(const void *p, int device) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  return a.type == cudaMemoryTypeManaged;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" seed_status seed_wilson_apply_noalloc(const seed_wilson *A, const void *X, int64_t ldx, void *Y,
                                                 int64_t ldy, int32_t ncols, seed_stream stream) {
  if (!A || !X || !Y) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: NULL argument");
  int64_t vol = 1;
  for (int k = 0; k < 4; ++k) {
    if (A->dims[k] < 2 || A->dims[k] > 4096)
      return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: lattice dims must be in [2, 4096]");
    vol *= A->dims[k];
  }
  if (A->bc_t != 0 && A->bc_t != 1) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: bc_t must be 0 or 1");
  if (!std::isfinite(A->kappa)) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: kappa is not finite");
  if (ncols < 1 || ncols > 64) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: ncols must be 1..64");
  const int64_t n = 12 * vol;
  if (ldx < n || ldy < n) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: leading dimension < n");
  const size_t nbr_bytes = round256((size_t)vol * 8 * sizeof(int32_t));
  const size_t need = nbr_bytes + (size_t)n * ncols * sizeof(double2);
  if (need > kNoAllocScratchBytes)
    return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: needs " + std::to_string(need) +
                                    " bytes of scratch (neighbour table + n*ncols complex), the limit is " +
                                    std::to_string(kNoAllocScratchBytes) + " bytes");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(SEED_ECUDA, "seed_wilson_apply_noalloc: no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: device index >= 64");
  if (!na_device_ptr(A->links, dev) || !na_device_ptr(X, dev) || !na_device_ptr(Y, dev))
    return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: links, X and Y must be device pointers on the current device");
  const char *x0 = (const char *)X, *x1 = x0 + ((ncols - 1) * ldx + n) * sizeof(double2);
  const char *y0 = (const char *)Y, *y1 = y0 + ((ncols - 1) * ldy + n) * sizeof(double2);
  if (x0 < y1 && y0 < x1) return na_fail(SEED_EINVAL, "seed_wilson_apply_noalloc: X and Y overlap");

  // once per device and context, with that device current: the device address of the
  // scratch array (looked up again if the current context is not the one it came from;
  // without a context id the address is looked up on every call)
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    const unsigned long long ctx_id = current_context_id();
    if (g_scratch_dev[dev] == nullptr || ctx_id == 0 || g_scratch_ctx[dev] != ctx_id) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return na_fail(SEED_ECUDA, std::string("seed_wilson_apply_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
      }
      g_scratch_dev[dev] = p;
      g_scratch_ctx[dev] = ctx_id;
    }
    scratch = g_scratch_dev[dev];
  }

  // Both scratch regions are fully overwritten before they are read, so the
  // previous call's contents never leak into this one and nothing needs clearing.
  int32_t *nbr = reinterpret_cast<int32_t *>(scratch);
  double2 *T = reinterpret_cast<double2 *>(reinterpret_cast<char *>(scratch) + nbr_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  seedk::launch_wilson_neighbors(A->dims, nbr, s);
  seedk::WilsonOp op{};
  for (int k = 0; k < 4; ++k) op.dims[k] = A->dims[k];
  op.sites = vol;
  op.kappa = A->kappa;
  op.bc_t = A->bc_t;
  op.links = (const double2 *)A->links;
  op.nbr = nbr;
  seedk::launch_wilson_dslash(op, +1, (const double2 *)X, ldx, T, n, ncols, nullptr, s);
  seedk::launch_wilson_dslash(op, -1, T, n, (double2 *)Y, ldy, ncols, nullptr, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(SEED_ECUDA, std::string("seed_wilson_apply_noalloc: ") + cudaGetErrorString(e));
  return SEED_OK;
}
