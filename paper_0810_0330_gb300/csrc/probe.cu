// probe.cu -- measurement helper: the FMA rate of the FP64 and FP32 pipes.
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

}  // namespace

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
