// device_common.cuh -- scalar helpers and deterministic reductions shared by
// the sm_103a kernels of this library.
//
// Every reduction here has a fixed shape for a fixed launch configuration, so
// results are bitwise reproducible run to run: warp butterflies, then warps in
// index order, then (grid level) block partials summed in index order by the
// last block to finish.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SEED_DEV __device__ __forceinline__

namespace seedk {

// ---------------------------------------------------------------------------
// scalar types: double (real problems) and double2 (complex, x = re, y = im)
// ---------------------------------------------------------------------------
SEED_DEV double2 c2(double re, double im) { return make_double2(re, im); }
SEED_DEV double2 cadd(double2 a, double2 b) { return c2(a.x + b.x, a.y + b.y); }
SEED_DEV double2 csub(double2 a, double2 b) { return c2(a.x - b.x, a.y - b.y); }
SEED_DEV double2 cmul(double2 a, double2 b) { return c2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)); }
// acc + a * b
SEED_DEV double2 cfma(double2 a, double2 b, double2 acc) {
  return c2(fma(-a.y, b.y, fma(a.x, b.x, acc.x)), fma(a.y, b.x, fma(a.x, b.y, acc.y)));
}
// acc + conj(a) * b
SEED_DEV double2 cfmac(double2 a, double2 b, double2 acc) {
  return c2(fma(a.y, b.y, fma(a.x, b.x, acc.x)), fma(-a.y, b.x, fma(a.x, b.y, acc.y)));
}

// single precision complex (mixed-precision path: FP32 vectors, FP64 scalars)
SEED_DEV float2 c2(float re, float im) { return make_float2(re, im); }
SEED_DEV float2 cadd(float2 a, float2 b) { return c2(a.x + b.x, a.y + b.y); }
SEED_DEV float2 csub(float2 a, float2 b) { return c2(a.x - b.x, a.y - b.y); }
SEED_DEV float2 cmul(float2 a, float2 b) { return c2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }
SEED_DEV float2 cfma(float2 a, float2 b, float2 acc) {
  return c2(fmaf(-a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, acc.y)));
}
SEED_DEV float2 cfmac(float2 a, float2 b, float2 acc) {
  return c2(fmaf(a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(-a.y, b.x, fmaf(a.x, b.y, acc.y)));
}

// Vector element traits.  Scalars of the recurrences are always FP64 (double,
// double2); A / A2 are the per-thread accumulator types of dot products (FP64
// for FP64 vectors; FP32 for FP32 vectors, whose per-thread sums cover a few
// dozen elements and are widened to FP64 before the block and grid sums).
// caxpy2 takes a coefficient already converted to A2 (staged once per block).
template <class T> struct Sc;
template <> struct Sc<double> {
  using A = double;
  using A2 = double2;
  static SEED_DEV double2 zero2() { return c2(0.0, 0.0); }
  static SEED_DEV double2 pair(double re, double im) { return c2(re, im); }
  static SEED_DEV double2 from2(double2 a) { return a; }
  static SEED_DEV double caxpy2(double2 a, double x, double y) { return fma(a.x, x, y); }
  static SEED_DEV double zero() { return 0.0; }
  static SEED_DEV double scale(double s, double x) { return s * x; }
  static SEED_DEV double axpy(double a, double x, double y) { return fma(a, x, y); }          // y + a x
  static SEED_DEV double caxpy(double2 a, double x, double y) { return fma(a.x, x, y); }      // y + a x (a real)
  static SEED_DEV double redot(double a, double b, double acc) { return fma(a, b, acc); }   // acc + Re(conj(a) b)
  static SEED_DEV double2 dotc(double a, double b, double2 acc) { return c2(fma(a, b, acc.x), acc.y); }
  static SEED_DEV double nrm2(double a, double acc) { return fma(a, a, acc); }
  static SEED_DEV double sub(double a, double b) { return a - b; }
  static SEED_DEV double add(double a, double b) { return a + b; }
};
template <> struct Sc<double2> {
  using A = double;
  using A2 = double2;
  static SEED_DEV double2 zero2() { return c2(0.0, 0.0); }
  static SEED_DEV double2 pair(double re, double im) { return c2(re, im); }
  static SEED_DEV double2 from2(double2 a) { return a; }
  static SEED_DEV double2 caxpy2(double2 a, double2 x, double2 y) { return cfma(a, x, y); }
  static SEED_DEV double2 zero() { return c2(0.0, 0.0); }
  static SEED_DEV double2 scale(double s, double2 x) { return c2(s * x.x, s * x.y); }
  static SEED_DEV double2 axpy(double a, double2 x, double2 y) { return c2(fma(a, x.x, y.x), fma(a, x.y, y.y)); }
  static SEED_DEV double2 caxpy(double2 a, double2 x, double2 y) { return cfma(a, x, y); }
  static SEED_DEV double redot(double2 a, double2 b, double acc) { return fma(a.y, b.y, fma(a.x, b.x, acc)); }
  static SEED_DEV double2 dotc(double2 a, double2 b, double2 acc) { return cfmac(a, b, acc); }
  static SEED_DEV double nrm2(double2 a, double acc) { return fma(a.y, a.y, fma(a.x, a.x, acc)); }
  static SEED_DEV double2 sub(double2 a, double2 b) { return csub(a, b); }
  static SEED_DEV double2 add(double2 a, double2 b) { return cadd(a, b); }
};
template <> struct Sc<float> {
  using A = float;
  using A2 = float2;
  static SEED_DEV float2 zero2() { return c2(0.f, 0.f); }
  static SEED_DEV float2 pair(float re, float im) { return c2(re, im); }
  static SEED_DEV float2 from2(double2 a) { return c2((float)a.x, (float)a.y); }
  static SEED_DEV float caxpy2(float2 a, float x, float y) { return fmaf(a.x, x, y); }
  static SEED_DEV float zero() { return 0.f; }
  static SEED_DEV float scale(double s, float x) { return (float)s * x; }
  static SEED_DEV float axpy(double a, float x, float y) { return fmaf((float)a, x, y); }
  static SEED_DEV float caxpy(double2 a, float x, float y) { return fmaf((float)a.x, x, y); }
  static SEED_DEV float redot(float a, float b, float acc) { return fmaf(a, b, acc); }
  static SEED_DEV float2 dotc(float a, float b, float2 acc) { return c2(fmaf(a, b, acc.x), acc.y); }
  static SEED_DEV float nrm2(float a, float acc) { return fmaf(a, a, acc); }
  static SEED_DEV float sub(float a, float b) { return a - b; }
  static SEED_DEV float add(float a, float b) { return a + b; }
};
template <> struct Sc<float2> {
  using A = float;
  using A2 = float2;
  static SEED_DEV float2 zero2() { return c2(0.f, 0.f); }
  static SEED_DEV float2 pair(float re, float im) { return c2(re, im); }
  static SEED_DEV float2 from2(double2 a) { return c2((float)a.x, (float)a.y); }
  static SEED_DEV float2 caxpy2(float2 a, float2 x, float2 y) { return cfma(a, x, y); }
  static SEED_DEV float2 zero() { return c2(0.f, 0.f); }
  static SEED_DEV float2 scale(double s, float2 x) { const float f = (float)s; return c2(f * x.x, f * x.y); }
  static SEED_DEV float2 axpy(double a, float2 x, float2 y) {
    const float f = (float)a;
    return c2(fmaf(f, x.x, y.x), fmaf(f, x.y, y.y));
  }
  static SEED_DEV float2 caxpy(double2 a, float2 x, float2 y) { return cfma(from2(a), x, y); }
  static SEED_DEV float redot(float2 a, float2 b, float acc) { return fmaf(a.y, b.y, fmaf(a.x, b.x, acc)); }
  static SEED_DEV float2 dotc(float2 a, float2 b, float2 acc) { return cfmac(a, b, acc); }
  static SEED_DEV float nrm2(float2 a, float acc) { return fmaf(a.y, a.y, fmaf(a.x, a.x, acc)); }
  static SEED_DEV float2 sub(float2 a, float2 b) { return csub(a, b); }
  static SEED_DEV float2 add(float2 a, float2 b) { return cadd(a, b); }
};

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
SEED_DEV double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum of K values over the block; the result is returned to every thread.
// smem must hold K * (NT/32) doubles.
template <int K, int NT>
SEED_DEV void block_sum(double (&v)[K], double *smem) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) smem[k * NW + warp] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += smem[k * NW + w];
    v[k] = s;
  }
  __syncthreads();
}

// Signals that this block has written its partials; returns true (in every
// thread of the block) for the last of `expected` blocks counted on `ticket`.
// The last block resets the ticket for the next launch.
SEED_DEV bool last_block_done(unsigned *ticket, unsigned expected) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == expected - 1u) ? 1u : 0u;
    if (s_last) *ticket = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0u;
}

// In the last block: sum partial[b*stride + k] over b = 0..nb-1 in a fixed
// order; returned to every thread.  smem: NT/32 doubles.
template <int NT>
SEED_DEV double sum_partials(const double *partial, int nb, int stride, int k, double *smem) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b0 = 0; b0 < nb; b0 += 4 * NT) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * NT + (int)threadIdx.x;
      v[u] = b < nb ? __ldcg(partial + (int64_t)b * stride + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] += v[u];
  }
  double v[1] = {(s[0] + s[1]) + (s[2] + s[3])};
  block_sum<1, NT>(v, smem);
  return v[0];
}

// Lane l ends with the warp sum of v[l] (a reduce-scatter: 31 adds per lane
// for 32 values instead of 160 for 32 butterflies).
SEED_DEV double warp_reduce_scatter32(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const double send = upper ? v[k] : v[k + w];
      const double keep = upper ? v[k + w] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

// One warp: sum of partial[b*stride + k] over b = 0..nb-1 in a fixed order,
// returned to every lane of the warp.  Eight independent loads are in flight
// per lane (GPUs issue in order: a load consumed in the next instruction would
// serialize one L2 round trip per partial).
SEED_DEV double warp_sum_partials(const double *partial, int nb, int stride, int k) {
  const int lane = threadIdx.x & 31;
  double s[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) s[u] = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 256) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < nb ? __ldcg(partial + (int64_t)b * stride + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] += v[u];
  }
  const double t = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
  return warp_sum(t);
}

// Flip the sign of x when the top bit of m is set (an integer op, no FP64 slot).
SEED_DEV double xsign(double x, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(x) ^ m);
}
SEED_DEV float xsign(float x, unsigned m) { return __int_as_float(__float_as_int(x) ^ (int)m); }

// Sign-bit masks of the complex element types (phases by XOR, no FP op).
template <class C> struct CxBits;
template <> struct CxBits<double2> {
  using R = double;
  using U = unsigned long long;
  static constexpr U sign = 0x8000000000000000ull;
};
template <> struct CxBits<float2> {
  using R = float;
  using U = unsigned;
  static constexpr U sign = 0x80000000u;
};

}  // namespace seedk
