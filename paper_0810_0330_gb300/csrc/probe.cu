// probe.cu -- measurement helpers: the FMA rate of the FP64 and FP32 pipes, and
// the rate of the FP64 matrix instructions beside it.
//
// The Wilson operator in FP64 is bound by the FP64 pipe on this GPU, so its
// roofline denominator is the FP64 FMA rate.  The nominal figure follows from
// unit counts (152 SMs x 2 FP64 FMA per clock x 2 flop x clock); this kernel
// measures it: every thread runs kChains independent FMA chains (enough
// independent work per warp scheduler to cover the FMA latency), the grid
// fills every SM several times over, and the time of the launch is taken with
// CUDA events on the launching stream.
#include <cuda_runtime.h>

#include <string>

#include "seed.h"

namespace seedk {
void set_last_error_message(const std::string &msg);   // engine.cu
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kSink = 4096;

// where a result would go if a thread ever met the impossible test below (a valid address either way)
__device__ double g_sink[kSink];

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot drop, taken by no thread for these inputs
  if (s == (T)-1.2345e30) g_sink[blockIdx.x % kSink] = (double)s;
}

template <class T>
seed_status time_chains(cudaStream_t s, int sms, double *tflops, double *ms_out) {
  const int blocks = sms * 8;
  const int iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  seed_status st = SEED_OK;
  float ms = 0.f, best = 1e30f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = SEED_ECUDA;
    goto done;
  }
  // warm-up, then the fastest of five timed launches
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.999999, (T)1e-7);
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = SEED_ECUDA;
      goto done;
    }
    if (ms < best) best = ms;
  }
  {
    const double flops = 2.0 * kChains * (double)iters * kThreads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
  }
done:
  if (cudaGetLastError() != cudaSuccess && st == SEED_OK) st = SEED_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

// ---- FP64 paths: the FMA pipe against the FP64 matrix (DMMA) instructions ----
//
// Roles per warp: 0 idle, 1 FP64 FMA chains (the work of one warp of
// k_fma_chains), 2 chains of mma.sync m8n8k4 f64 (512 flop each), 3 chains of
// mma.sync m16n8k16 f64 (4096 flop each).  Per-warp work is sized so that each
// role's warp does 2^21 flop.  Launching half the warps in one role and half
// in another shows whether the two share a unit: if they do, the mixed launch
// takes the sum of the two half launches; if not, their maximum.
constexpr int kMmaChains = 4;

__device__ __forceinline__ void dmma_m8n8k4(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void dmma_m16n8k16(double (&d)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
      "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
        "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// role_even / role_odd: the role of warps with an even / odd index in the block
__global__ void __launch_bounds__(kThreads) k_fp64_paths(int role_even, int role_odd) {
  const int warp = threadIdx.x >> 5;
  const int role = (warp & 1) ? role_odd : role_even;
  double s = 0.0;
  if (role == 1) {
    const double a = 0.999999, b = 1e-7;
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int it = 0; it < 4096; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
  } else if (role == 2) {
    const double a = 1e-3 * (double)(threadIdx.x & 7), b = 1e-3;
    double d[kMmaChains][2];
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c) d[c][0] = d[c][1] = (double)c;
    for (int it = 0; it < 4096 / kMmaChains; ++it) {   // 4096 x 512 flop per warp
#pragma unroll
      for (int c = 0; c < kMmaChains; ++c) dmma_m8n8k4(d[c][0], d[c][1], a, b);
    }
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c) s += d[c][0] + d[c][1];
  } else if (role == 3) {
    double a[8], b[4], d[kMmaChains][4];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1e-3 * (double)((threadIdx.x + k) & 7);
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = 1e-3;
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) d[c][k] = (double)c;
    for (int it = 0; it < 512 / kMmaChains; ++it) {    // 512 x 4096 flop per warp
#pragma unroll
      for (int c = 0; c < kMmaChains; ++c) dmma_m16n8k16(d[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c) s += (d[c][0] + d[c][1]) + (d[c][2] + d[c][3]);
  }
  if (s == -1.2345e30) g_sink[blockIdx.x % kSink] = s;
}

// fastest of five timed launches (after one warm-up) of k_fp64_paths
seed_status time_paths(cudaStream_t s, int blocks, int role_even, int role_odd, float *best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  seed_status st = SEED_OK;
  float ms = 0.f;
  *best = 1e30f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = SEED_ECUDA;
    goto done;
  }
  k_fp64_paths<<<blocks, kThreads, 0, s>>>(role_even, role_odd);
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, s);
    k_fp64_paths<<<blocks, kThreads, 0, s>>>(role_even, role_odd);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = SEED_ECUDA;
      goto done;
    }
    if (ms < *best) *best = ms;
  }
done:
  if (cudaGetLastError() != cudaSuccess && st == SEED_OK) st = SEED_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

}  // namespace

extern "C" seed_status seed_time_fp64_paths(seed_stream stream, double *out) {
  if (!out) {
    seedk::set_last_error_message("seed_time_fp64_paths: out must not be NULL");
    return SEED_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    seedk::set_last_error_message("seed_time_fp64_paths: no usable CUDA device");
    return SEED_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sms * 8;
  const double warps = (double)blocks * (kThreads / 32), per_warp = 2097152.0;
  // roles for all warps: FMA, DMMA m8n8k4, DMMA m16n8k16; then halves and the mix
  const int cases[6][2] = {{1, 1}, {2, 2}, {3, 3}, {1, 0}, {0, 2}, {1, 2}};
  float t[6];
  for (int c = 0; c < 6; ++c) {
    const seed_status st = time_paths(s, blocks, cases[c][0], cases[c][1], &t[c]);
    if (st != SEED_OK) {
      seedk::set_last_error_message("seed_time_fp64_paths: a CUDA call failed");
      return st;
    }
  }
  for (int c = 0; c < 3; ++c) out[c] = warps * per_warp / (t[c] * 1e-3) / 1e12;
  out[3] = t[5] / (t[3] + t[4]);
  out[4] = t[3];
  out[5] = t[4];
  out[6] = t[5];
  return SEED_OK;
}

extern "C" seed_status seed_time_fma(int32_t dtype, seed_stream stream, double *tflops, double *ms) {
  if (!tflops || (dtype != SEED_F64 && dtype != SEED_F32)) {
    seedk::set_last_error_message("seed_time_fma: dtype must be SEED_F64 or SEED_F32, tflops not NULL");
    return SEED_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    seedk::set_last_error_message("seed_time_fma: no usable CUDA device");
    return SEED_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const seed_status st = dtype == SEED_F64 ? time_chains<double>(s, sms, tflops, ms)
                                           : time_chains<float>(s, sms, tflops, ms);
  if (st != SEED_OK) seedk::set_last_error_message("seed_time_fma: a CUDA call failed");
  return st;
}
