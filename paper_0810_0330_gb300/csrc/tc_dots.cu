// tc_dots.cu -- the mixed-precision seeding products G = V_blk^H R_0 on the
// 5th-generation tensor cores (tcgen05, kind::tf32), operands staged by TMA.
//
// In the blocked seeding of systems 2..p (Sec. 3: every Lanczos vector v_i is
// projected onto every r_0^j) one flush forms G[q][j] = v_{blk0+q}^H r_0^j for
// the k <= 128 steps of a block and the p - 1 <= 63 other systems: a
// contraction over the whole vector length n (1.57 M complex on the 16^3 x 32
// lattice) with a tiny k x (p-1) result.  In FP32 that is ~8 flops per byte
// loaded, more than the FP32 pipe sustains at the HBM rate, so it runs here
// on the tensor cores.
//
// Accuracy: TF32 keeps 10 mantissa bits.  Every FP32 operand x is split as
// x = hi + lo (hi = x rounded to TF32, lo = x - hi rounded to TF32), and the
// products hi*hi + hi*lo + lo*hi ("3xTF32") reproduce the FP32 product to
// about 2^-21 -- the FP32 accuracy of the CUDA-core version -- where plain TF32
// would leave ~2e-4 relative error in G.  The tensor cores accumulate in FP32
// over at most 2048 elements (one "item"); each item is then drained from
// tensor memory and added in FP64, and the per-CTA partials are summed over
// CTAs in a fixed order by k_blk_reduce (deterministic).
//
// One MMA instruction computes all four hi/lo combinations at once by stacking
// them in M and N:
//   A (M = 128 rows)  = [V_hi re; V_hi im; V_lo re; V_lo im] x 32 steps
//   B (N = 64 rows)   = [R_hi re; R_hi im; R_lo re; R_lo im] x 16 systems
//   D[row][col] = sum over the stage's elements of A[row][k] B[col][k]
// and the epilogue combines the blocks into Re G = sum Vr Rr + Vi Ri and
// Im G = sum Vr Ri - Vi Rr (keeping hi*hi, hi*lo and lo*hi).  Longer blocks
// and more systems run as more CTAs (grid.y: 32-step tiles, grid.z: 16-system
// tiles).
//
// Warp roles (10 warps, one CTA per SM):
//   warp 0      TMA producer: one thread issues a 2-d cp.async.bulk.tensor per
//               column and stage (64 complex = 512 B of a V or R_0 column)
//               into a 4-stage raw ring
//   warp 1      tensor memory allocation, the MMA issuer (one thread), and
//               deallocation
//   warps 2,3,8,9  converters: raw FP32 (re, im interleaved) -> TF32 hi/lo,
//               deinterleaved, into the UMMA K-major core-matrix layout of a
//               2-stage operand ring
//   warps 4-7   epilogue: warp 4 + q reads tensor-memory lanes 32q..32q+31
//               (rows of A part q), accumulates FP64
// Every wait on an mbarrier gives up after kTcWaitNs, sets *err and lets all
// roles leave; the producer waits for its copies in flight, the issuer for
// its MMAs, and the tensor memory is freed before the CTA exits.
#include <cuda.h>   // CUtensorMap (the type only; the encode call is found through the runtime)
#include <cuda_runtime.h>

#include <string>

#include "seed.h"
#include "seed_internal.h"

namespace seedk {

namespace tc {

constexpr int kThreads = 320;                 // 10 warps
constexpr int kChunk = 64;                    // complex elements of a column per stage
constexpr int kSteps = 32;                    // Lanczos steps per M tile
constexpr int kCols = 16;                     // right-hand sides per N tile
constexpr int kRawStages = 4;
constexpr int kOpStages = 2;
constexpr int kItemChunks = 32;               // stages accumulated in FP32 before a drain
constexpr int kSlot = kChunk * 8;             // 512 B: one column's chunk (64 float2)
constexpr int kRawStage = (kSteps + kCols) * kSlot;   // 24576 B
constexpr int kKGroups = kChunk / 4;          // 16 core-matrix columns of 4 TF32 per stage
constexpr int kM = 128, kN = 64;
// K-major, no swizzle: a core matrix is 8 rows x 16 B; SBO (next 8 rows) = 128 B; LBO
// (next 4 elements of K) = all row groups + 16 B of padding, so that the 8 lanes of a
// shared-memory phase writing one row at 8 consecutive K groups hit 8 different banks.
constexpr int kSBO = 128;
constexpr int kLboA = (kM / 8) * 128 + 16;    // 2064
constexpr int kLboB = (kN / 8) * 128 + 16;    // 1040
constexpr int kOpA = kKGroups * kLboA;        // 33024
constexpr int kOpB = kKGroups * kLboB;        // 16640
constexpr int kOpStage = kOpA + kOpB;         // 49664
constexpr int kRawBytes = kRawStages * kRawStage;   // 98304
constexpr int kOpBytes = kOpStages * kOpStage;      // 99328
constexpr int kBarBytes = 256;
constexpr int kSmemBytes = 1024 + kRawBytes + kOpBytes + kBarBytes;   // + alignment slack
constexpr int kTmemCols = 128;                // two accumulators of N = 64 FP32 columns
constexpr unsigned long long kTcWaitNs = 2000000000ull;
// epilogue combine buffer (aliases the raw ring once every stage is consumed)
constexpr int kCombBytes = 4 * 32 * 2 * kCols * 8;  // 32768
static_assert(kCombBytes <= kRawBytes, "combine buffer must fit in the raw ring");
static_assert(kOpA % 16 == 0 && kOpB % 16 == 0 && kRawStage % 1024 == 0, "alignment");

// instruction descriptor of tcgen05.mma kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

struct Bars {
  uint64_t raw_full[kRawStages];
  uint64_t raw_empty[kRawStages];
  uint64_t op_full[kOpStages];
  uint64_t op_empty[kOpStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_done;
  uint32_t tmem_base;
};
static_assert(sizeof(Bars) <= kBarBytes, "barrier block");

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete.  Gives up (false) when the
// error flag is set by another thread or after kTcWaitNs, setting the flag.
__device__ bool bar_wait(uint64_t *b, uint32_t parity, int *err) {
  unsigned long long t0 = 0;
  for (uint32_t spin = 0;; ++spin) {
    if (bar_try(b, parity)) return true;
    if ((spin & 31u) == 31u) {
      if (*(volatile int *)err) return false;
      const unsigned long long t = gtime();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kTcWaitNs) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
}

// Wait for async work this thread issued (TMA copies, MMAs) before the CTA leaves or
// frees tensor memory: bounded by time only, not cut short by the error flag.
__device__ void bar_drain(uint64_t *b, uint32_t parity, int *err) {
  const unsigned long long t0 = gtime();
  while (!bar_try(b, parity)) {
    if (gtime() - t0 > kTcWaitNs) {
      atomicExch(err, 1);
      return;
    }
  }
}

// 2-d TMA load of one box (128 floats x 1 column) into shared memory, completion on `bar`
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

// shared-memory matrix descriptor (no swizzle): start >> 4, LBO >> 4 at bit 16,
// SBO >> 4 at bit 32, descriptor version 1 at bit 46
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 columns of FP32 from tensor memory (warp-collective)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of (row, K group) in an operand tile (K-major, no swizzle)
__device__ __forceinline__ uint32_t op_off(int row, int kg, int lbo) {
  return (uint32_t)(kg * lbo + (row >> 3) * kSBO + (row & 7) * 16);
}

}  // namespace tc

// Partial products of one CTA: its contiguous range of 64-element chunks, one
// 32-step tile (blockIdx.y) and one 16-system tile (blockIdx.z).  With st set,
// the block is [st->blk0, st->w_last] (column c of V holds v_{c+1}); else
// len_host columns from column vcol_host.  Hpart[(cta * kSeedBlock + q) * kLdG + j]
// receives the CTA's FP64 partial of G[q][j].
__global__ void __launch_bounds__(tc::kThreads, 1)
    k_blk_dots_tc(const __grid_constant__ CUtensorMap vmap, const __grid_constant__ CUtensorMap rmap,
                  const SeedState *st, int len_host, int vcol_host, int nj, int64_t nchunks, double2 *Hpart,
                  int *err) {
  using namespace tc;
  constexpr int kLdG = kMaxRhs - 1;
  int len, vcol0;
  if (st) {
    len = min(st->w_last - st->blk0 + 1, kSeedBlock);
    vcol0 = st->blk0 - 1;
  } else {
    len = len_host;
    vcol0 = vcol_host;
  }
  const int mt = blockIdx.y, nt = blockIdx.z;
  if (len <= 0 || nj <= 0 || mt * kSteps >= len || nt * kCols >= nj) return;   // uniform over the CTA
  const int len_t = min(kSteps, len - mt * kSteps);
  const int nr_t = min(kCols, nj - nt * kCols);
  vcol0 += mt * kSteps;
  const int rcol0 = nt * kCols;
  const int64_t c0 = nchunks * blockIdx.x / gridDim.x, c1 = nchunks * (blockIdx.x + 1) / gridDim.x;
  const int nst = (int)(c1 - c0);                       // >= 1: the host keeps gridDim.x <= nchunks
  const int nitems = (nst + kItemChunks - 1) / kItemChunks;

  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *raw = smem;
  unsigned char *ops = smem + kRawBytes;
  Bars *bars = reinterpret_cast<Bars *>(smem + kRawBytes + kOpBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      tc::bar_init(&bars->raw_full[s], 1);
      tc::bar_init(&bars->raw_empty[s], 4);
    }
    for (int s = 0; s < kOpStages; ++s) {
      tc::bar_init(&bars->op_full[s], 4);
      tc::bar_init(&bars->op_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::bar_init(&bars->acc_full[b], 1);
      tc::bar_init(&bars->acc_empty[b], 4);
    }
    tc::bar_init(&bars->mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // the whole warp: allocate the accumulators in tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::saddr(&bars->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int g = 0; g < nst; ++g) {
        const int r = g % kRawStages;
        if (g >= kRawStages && !tc::bar_wait(&bars->raw_empty[r], ((g / kRawStages) + 1) & 1, err)) break;
        unsigned char *dst = raw + r * kRawStage;
        const int x = (int)((c0 + g) * (kChunk * 2));   // float index of the chunk
        tc::bar_expect_tx(&bars->raw_full[r], (uint32_t)((len_t + nr_t) * kSlot));
        for (int s = 0; s < len_t; ++s) tc::tma_load_2d(dst + s * kSlot, &vmap, x, vcol0 + s, &bars->raw_full[r]);
        for (int c = 0; c < nr_t; ++c)
          tc::tma_load_2d(dst + (kSteps + c) * kSlot, &rmap, x, rcol0 + c, &bars->raw_full[r]);
        issued = g + 1;
      }
      // copies still in flight land before the CTA may leave (their phases are the last ones)
      for (int g = issued - kRawStages > 0 ? issued - kRawStages : 0; g < issued; ++g)
        tc::bar_drain(&bars->raw_full[g % kRawStages], (g / kRawStages) & 1, err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int g = 0; g < nst && ok; ++g) {
        const int s = g % kOpStages;
        const int t = g / kItemChunks;
        const bool first = (g % kItemChunks) == 0;
        const bool last = (g % kItemChunks) == kItemChunks - 1 || g == nst - 1;
        if (first && t >= 2 && !tc::bar_wait(&bars->acc_empty[t & 1], ((t >> 1) + 1) & 1, err)) break;
        if (!tc::bar_wait(&bars->op_full[s], (g / kOpStages) & 1, err)) break;
        tc::tc_fence_after();
        const uint32_t a0 = tc::saddr(ops + s * kOpStage), b0 = a0 + kOpA;
        const uint32_t d = tmem + (uint32_t)((t & 1) * kN);
#pragma unroll
        for (int kk = 0; kk < kKGroups / 2; ++kk) {
          const uint64_t ad = tc::sdesc(a0 + kk * 2 * kLboA, kLboA, kSBO);
          const uint64_t bd = tc::sdesc(b0 + kk * 2 * kLboB, kLboB, kSBO);
          tc::mma_tf32(d, ad, bd, (first && kk == 0) ? 0u : 1u);
        }
        tc::mma_commit(&bars->op_empty[s]);
        if (last) tc::mma_commit(&bars->acc_full[t & 1]);
      }
      // every MMA issued has completed before the accumulators are freed
      tc::mma_commit(&bars->mma_done);
      tc::bar_drain(&bars->mma_done, 0, err);
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------- epilogue: drain the accumulators into FP64 ----------------
    const int q = warp - 4;                  // A part: 0 hi re, 1 hi im, 2 lo re, 3 lo im
    const bool vim = (q & 1) != 0, vlo = (q >> 1) != 0;
    double gre[kCols], gim[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) gre[c] = gim[c] = 0.0;
    for (int t = 0; t < nitems; ++t) {
      if (!tc::bar_wait(&bars->acc_full[t & 1], (t >> 1) & 1, err)) break;
      tc::tc_fence_after();
      float v[64];
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((t & 1) * kN);
      tc::tmem_ld32(ta, v);
      tc::tmem_ld32(ta + 32, v + 32);
      tc::tmem_wait_ld();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::bar_arrive(&bars->acc_empty[t & 1]);
      // columns: [R part hi/lo][re/im][system]; keep hi*hi, hi*lo, lo*hi
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        double pre = (double)v[c], pim = (double)v[kCols + c];
        if (!vlo) {
          pre += (double)v[2 * kCols + c];
          pim += (double)v[3 * kCols + c];
        }
        if (!vim) {
          gre[c] += pre;
          gim[c] += pim;
        } else {
          gre[c] += pim;
          gim[c] -= pre;
        }
      }
    }
    // the four A parts of each step meet in shared memory (the raw ring is idle by now:
    // every stage was consumed before the last accumulator completed)
    double *comb = reinterpret_cast<double *>(raw);
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      comb[((q * 32 + lane) * 2) * kCols + c] = gre[c];
      comb[((q * 32 + lane) * 2 + 1) * kCols + c] = gim[c];
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const int te = threadIdx.x - 128;         // 0..127
    for (int e = te; e < kSteps * kCols; e += 128) {
      const int sq = e / kCols, c = e % kCols;
      if (sq < len_t && c < nr_t) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          re += comb[((qq * 32 + sq) * 2) * kCols + c];
          im += comb[((qq * 32 + sq) * 2 + 1) * kCols + c];
        }
        Hpart[((int64_t)blockIdx.x * kSeedBlock + mt * kSteps + sq) * kLdG + rcol0 + c] = make_double2(re, im);
      }
    }
  } else {
    // ---------------- converters (warps 2, 3, 8, 9) ----------------
    const int cw = warp < 4 ? warp - 2 : warp - 6;      // 0..3
    const int tid = cw * 32 + lane;                      // 0..127
    for (int g = 0; g < nst; ++g) {
      const int r = g % kRawStages, s = g % kOpStages;
      if (!tc::bar_wait(&bars->raw_full[r], (g / kRawStages) & 1, err)) break;
      if (g >= kOpStages && !tc::bar_wait(&bars->op_empty[s], ((g / kOpStages) + 1) & 1, err)) break;
      const unsigned char *src = raw + r * kRawStage;
      unsigned char *opa = ops + s * kOpStage, *opb = opa + kOpA;
      // units (column slot, K group of 4 elements): 16 K groups per slot, 48 slots
#pragma unroll 2
      for (int u = tid; u < (kSteps + kCols) * kKGroups; u += 128) {
        const int slot = u >> 4, kg = u & 15;
        const bool isv = slot < kSteps;
        const int col = isv ? slot : slot - kSteps;
        if (col >= (isv ? len_t : nr_t)) continue;
        const float4 a = *reinterpret_cast<const float4 *>(src + slot * kSlot + kg * 32);
        const float4 b = *reinterpret_cast<const float4 *>(src + slot * kSlot + kg * 32 + 16);
        const float re[4] = {a.x, a.z, b.x, b.z}, im[4] = {a.y, a.w, b.y, b.w};
        float rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          rh[k] = tc::tf32_round(re[k]);
          rl[k] = tc::tf32_round(re[k] - rh[k]);
          ih[k] = tc::tf32_round(im[k]);
          il[k] = tc::tf32_round(im[k] - ih[k]);
        }
        unsigned char *base = isv ? opa : opb;
        const int lbo = isv ? kLboA : kLboB;
        const int stride = isv ? kSteps : kCols;     // rows per (hi/lo, re/im) block
        *reinterpret_cast<float4 *>(base + tc::op_off(col, kg, lbo)) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4 *>(base + tc::op_off(stride + col, kg, lbo)) =
            make_float4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<float4 *>(base + tc::op_off(2 * stride + col, kg, lbo)) =
            make_float4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<float4 *>(base + tc::op_off(3 * stride + col, kg, lbo)) =
            make_float4(il[0], il[1], il[2], il[3]);
      }
      // generic-proxy writes become visible to the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        tc::bar_arrive(&bars->op_full[s]);
        tc::bar_arrive(&bars->raw_empty[r]);
      }
    }
  }
  // everyone is done with the accumulators: free the tensor memory
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {
typedef CUresult (*PfnEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
PfnEncodeTiled encode_fn() {
  static PfnEncodeTiled fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PfnEncodeTiled)p;
    cudaGetLastError();
    looked = true;
  }
  return fn;
}
}  // namespace

// A 2-d map over ncols FP32-complex columns of `len` elements (leading dimension ld
// elements), boxes of 64 complex x 1 column.  False if the map cannot be made.
bool tc_make_map(CUtensorMap *map, const void *base, int64_t len, int64_t ld, int64_t ncols) {
  PfnEncodeTiled enc = encode_fn();
  if (!enc || !base || ncols < 1 || len < tc::kChunk || len % tc::kChunk || ld % 2 ||
      ((uintptr_t)base & 15) || (ld * 8) % 16)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * len), (cuuint64_t)ncols};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 8)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * tc::kChunk), 1u};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_grid(int64_t len) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
      sms = 148;
    cudaGetLastError();
  }
  const int64_t chunks = len / tc::kChunk;
  return (int)(chunks < sms ? chunks : sms);
}

cudaError_t launch_blk_dots_tc(const CUtensorMap &vmap, const CUtensorMap &rmap, const SeedState *st, int len_host,
                               int vcol_host, int nj, int64_t len, double2 *Hpart, int grid, int *err,
                               cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_blk_dots_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int ytiles = (kSeedBlock + tc::kSteps - 1) / tc::kSteps;
  const int ztiles = (nj + tc::kCols - 1) / tc::kCols;
  k_blk_dots_tc<<<dim3((unsigned)grid, (unsigned)ytiles, (unsigned)ztiles), tc::kThreads, tc::kSmemBytes, s>>>(
      vmap, rmap, st, len_host, vcol_host, nj, len / tc::kChunk, Hpart, err);
  return cudaGetLastError();
}

// G[q][j] = sum over CTAs (in CTA order) of the partials, k x nr, row-major
__global__ void k_tc_reduce(const double2 *Hpart, int nchunk, int k, int nr, double2 *G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * nr) return;
  const int q = idx / nr, j = idx - nr * (idx / nr);
  double2 acc = make_double2(0.0, 0.0);
  for (int c = 0; c < nchunk; ++c) {
    const double2 v = Hpart[((int64_t)c * kSeedBlock + q) * (kMaxRhs - 1) + j];
    acc.x += v.x;
    acc.y += v.y;
  }
  G[idx] = acc;
}

void set_last_error_message(const std::string &msg);   // engine.cu

}  // namespace seedk

extern "C" seed_status seed_block_products(const void *V, int64_t ldv, int32_t k, const void *R, int64_t ldr,
                                           int32_t nr, int64_t n, double *G, int32_t reps, double *ms,
                                           seed_stream stream) {
  using namespace seedk;
  auto bad = [](const char *m) {
    set_last_error_message(std::string("seed_block_products: ") + m);
    return SEED_EINVAL;
  };
  if (!V || !R || !G) return bad("NULL argument");
  if (k < 1 || k > kSeedBlock) return bad("k must be in [1, 128]");
  if (nr < 1 || nr > kMaxRhs - 1) return bad("nr must be in [1, 63]");
  if (n < 64 || n % 64) return bad("n must be a positive multiple of 64");
  if (ldv < n || ldr < n || ldv % 2 || ldr % 2) return bad("ldv and ldr must be even and >= n");
  if (((uintptr_t)V & 15) || ((uintptr_t)R & 15)) return bad("V and R must be 16-byte aligned");
  if (reps < 1 || reps > 100000) return bad("reps must be in [1, 100000]");
  CUtensorMap vmap, rmap;
  if (!tc_make_map(&vmap, V, n, ldv, k) || !tc_make_map(&rmap, R, n, ldr, nr)) {
    set_last_error_message("seed_block_products: the TMA maps could not be made (no driver entry point?)");
    return SEED_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = tc_grid(n);
  double2 *Hpart = nullptr, *Gd = nullptr;
  int *err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  seed_status st = SEED_OK;
  float t = 0.f;
  int herr = 0;
  if (cudaMalloc(&Hpart, sizeof(double2) * (size_t)grid * kSeedBlock * (kMaxRhs - 1)) != cudaSuccess ||
      cudaMalloc(&Gd, sizeof(double2) * (size_t)k * nr) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    set_last_error_message("seed_block_products: device allocation failed");
    st = SEED_ENOMEM;
    goto done;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    goto cuda_fail;
  // one untimed launch, then reps timed launches of the product kernel alone
  if (launch_blk_dots_tc(vmap, rmap, nullptr, k, 0, nr, n, Hpart, grid, err, s) != cudaSuccess) goto cuda_fail;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r)
    if (launch_blk_dots_tc(vmap, rmap, nullptr, k, 0, nr, n, Hpart, grid, err, s) != cudaSuccess) goto cuda_fail;
  cudaEventRecord(e1, s);
  k_tc_reduce<<<(k * nr + 127) / 128, 128, 0, s>>>(Hpart, grid, k, nr, Gd);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
      cudaMemcpyAsync(G, Gd, sizeof(double2) * (size_t)k * nr, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    goto cuda_fail;
  if (ms) *ms = (double)t / reps;
  if (herr) {
    set_last_error_message("seed_block_products: a wait of the tensor-core kernel timed out");
    st = SEED_ETIMEOUT;
  }
  goto done;
cuda_fail:
  set_last_error_message(std::string("seed_block_products: ") + cudaGetErrorString(cudaGetLastError()));
  st = SEED_ECUDA;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(Hpart);
  cudaFree(Gd);
  cudaFree(err);
  return st;
}
