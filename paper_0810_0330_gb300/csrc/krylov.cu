// krylov.cu -- the Sec. 3 seed recurrence step by step, its periodic
// reorthogonalization, the Galerkin projection over a kept basis, and lockstep
// CG for the seeded systems, on sm_103a.  Instantiated for FP64 (double,
// double2) and, for the mixed-precision path, FP32 vectors (float, float2)
// whose scalars and reductions stay FP64.
//
// All scalars of the recurrence (alpha_i, beta_i, delta_i, gamma_{i-1},
// zeta_i, eta^j, the step index i and the stop flags) live in device memory
// (SeedState); each kernel reads them at its start and the last block of a
// reducing kernel writes the next values.  The host therefore never waits
// inside an iteration and whole runs of steps can be replayed from one CUDA
// graph.  Every kernel first checks `active` and returns at once when the
// recurrence has stopped, so over-issued steps cost only their launch.
//
// Reductions are deterministic: block partials in a fixed layout, summed in
// block order by the last block (see device_common.cuh).
#include <math.h>

#include <type_traits>

#include "seed_device.cuh"

namespace seedk {

constexpr int NT = kVecThreads;
constexpr int kSeedTicket = 0;     // tickets[0..15]: seed / reorth kernels
constexpr int kGroupTicket = 128;  // tickets[128 + g]: groups of 32 blocks (two-level reductions)
constexpr int kOneLevelBlocks = 152;   // reductions over more blocks than this use two levels

#define GRID_STRIDE(e, n) \
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < (n); e += (int64_t)gridDim.x * NT)

// Single-vector kernels: one block per SM (152) while that leaves each thread
// at most 8 elements -- there the work is a few microseconds and what matters
// is few blocks, independent loads per thread and a short reduction tail --
// and beyond that up to 8 blocks per SM, so that enough loads are in flight to
// keep HBM busy on long vectors.
int vec_blocks(int64_t n) {
  int64_t b = (n + NT * 8 - 1) / (NT * 8);
  if (b < 152) b = 152;
  const int64_t bmax = (n + NT - 1) / NT;
  if (b > bmax) b = bmax;
  if (b > kVecBlocksMax) b = kVecBlocksMax;
  if (b < 1) b = 1;
  return (int)b;
}

// Kernels over nc lockstep columns: up to 8 blocks per SM in total (long
// vectors need that many loads in flight to keep HBM busy), at least 4
// elements per thread.
int col_blocks(int64_t n, int nc) {
  int64_t b = (n + NT * 4 - 1) / (NT * 4);
  int64_t cap = kVecBlocksMax / (nc > 0 ? nc : 1);
  if (cap < 1) cap = 1;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Start of the Lanczos run: f = r_0^1, beta_0 = ||r_0^1||; the first step forms v_1 = f / beta_0.
template <class T>
__global__ void __launch_bounds__(NT) k_seed_start(SeedBufs<T> b, const T *__restrict__ r01) {
  __shared__ double sm[NT / 32];
  typename Sc<T>::A acc = 0;
  GRID_STRIDE(e, b.n) {
    const T r = r01[e];
    b.f[e] = r;
    acc = Sc<T>::nrm2(r, acc);
  }
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  if (threadIdx.x == 0) b.partials[blockIdx.x] = v[0];
  if (!last_block_done(b.tickets + kSeedTicket, gridDim.x)) return;
  const double s = sum_partials<NT>(b.partials, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) {
    SeedState *st = b.st;
    const double b0 = sqrt(s);
    st->beta0 = b0;
    b.beta_hist[0] = b0;
    st->i = 1;
    st->tol_abs = st->tol_rel * st->bnorm1;
    st->tnorm = 0.0;
    st->beta_prev = 0.0;
    st->converged_at = -1;
    st->stop_at = -1;
    st->rho = b0;
    if (b0 > 0.0 && isfinite(b0)) {
      st->active = 1;
      st->stop_reason = STOP_RUNNING;
      st->inv_beta = 1.0 / b0;
    } else {   // r_0 = 0: x_0 solves system 1; NaN or Inf: reported, no step runs
      st->active = 0;
      st->stop_reason = b0 == 0.0 ? STOP_CONVERGED : STOP_NONFINITE;
      st->inv_beta = 0.0;
    }
  }
}

// The dot products of a Lanczos step (alpha_i, g^j) and the scalars of the LU update and seeding, in
// one pass over the elements.  The step's operator was applied to f (not yet
// normalized: beta_{i-1} v_i), so with u = A f:  v_i = f / beta_{i-1} into
// column i-1 of V;  f = u / beta_{i-1} - beta_{i-1} v_{i-1} (A is linear);
// alpha_i = Re(v_i^H f);  g^j = v_i^H r_0^j for j = 2..nrhs.
// Values are packed 32 per chunk (alpha in slot 0 of chunk 0, then 15 complex
// g^j per chunk), reduced per block with a warp reduce-scatter, and the last
// block reduces all chunks warp-parallel and forms alpha_i, gamma_{i-1},
// delta_i, zeta_i and eta^j.
constexpr int kDotsPerChunk = 15;

template <class T>
__global__ void __launch_bounds__(NT) k_seed_dots(SeedBufs<T> b) {
  SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sred[NT / 32][32];
  __shared__ double2 sums[kMaxRhs];
  __shared__ double s_alpha;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = st->i;
  const int nr = b.Wb == nullptr ? b.nrhs : 1;   // blocked seeding: g^j at the flush
  const int nch = nr > 1 ? (nr - 1 + kDotsPerChunk - 1) / kDotsPerChunk : 1;
  T *vi = b.V + (int64_t)(i - 1) * b.ldv;
  const T *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * b.ldv;
  const double bp = (i > 1) ? st->beta_prev : 0.0, inv_b = st->inv_beta;
  for (int ch = 0; ch < nch; ++ch) {
    const int j0 = 1 + kDotsPerChunk * ch;
    const int jn = nr - j0 < kDotsPerChunk ? nr - j0 : kDotsPerChunk;   // may be <= 0
    typename Sc<T>::A acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0;
    GRID_STRIDE(e, b.n) {
      T v;
      if (ch == 0) {   // the same thread reads v_i back in the later chunks
        v = Sc<T>::scale(inv_b, b.f[e]);
        vi[e] = v;
        const T ue = Sc<T>::scale(inv_b, b.u[e]);
        const T fe = (i > 1) ? Sc<T>::axpy(-bp, vm[e], ue) : ue;
        b.f[e] = fe;
        acc[0] = Sc<T>::redot(v, fe, acc[0]);
      } else {
        v = vi[e];
      }
#pragma unroll
      for (int q = 0; q < kDotsPerChunk; ++q) {
        if (q < jn) {
          const auto d = Sc<T>::dotc(v, b.R0[(int64_t)(j0 + q - 1) * b.ldr + e], Sc<T>::pair(acc[1 + 2 * q], acc[2 + 2 * q]));
          acc[1 + 2 * q] = d.x;
          acc[2 + 2 * q] = d.y;
        }
      }
    }
    double accd[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) accd[q] = (double)acc[q];
    const double mine = warp_reduce_scatter32(accd);
    sred[warp][lane] = mine;
    __syncthreads();
    if (threadIdx.x < 32)
      b.partials[((int64_t)ch * gridDim.x + blockIdx.x) * 32 + lane] =
          ((sred[0][lane] + sred[1][lane]) + sred[2][lane]) + sred[3][lane];
    __syncthreads();
  }
  // The last block reduces the block partials; on long vectors (more than one
  // block per SM) in two levels: the last block of every group of 32 blocks
  // sums its group, then the last group sums the group partials, so no single
  // block reads all 32 x gridDim.x partials.  Both orders are fixed.
  const int nb = gridDim.x;
  const double *fin = b.partials;   // partials of the final level: [ch][nfin][32]
  int nfin = nb;
  if (nb > kOneLevelBlocks) {
    const int grp = blockIdx.x >> 5, ngrp = (nb + 31) >> 5, gsz = min(32, nb - grp * 32);
    if (!last_block_done(b.tickets + kGroupTicket + grp, gsz)) return;
    double *gpart = b.partials + (int64_t)nch * nb * 32;
    for (int v0 = warp * 8; v0 < 32 * nch; v0 += (NT / 32) * 8) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int val = v0 + u, ch = val >> 5, q = val & 31;
        x[u] = (val < 32 * nch && lane < gsz) ? __ldcg(b.partials + ((int64_t)ch * nb + grp * 32 + lane) * 32 + q)
                                              : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = warp_sum(x[u]);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int val = v0 + u;
          if (val < 32 * nch) gpart[((int64_t)(val >> 5) * ngrp + grp) * 32 + (val & 31)] = x[u];
        }
      }
    }
    if (!last_block_done(b.tickets + kSeedTicket, ngrp)) return;
    fin = gpart;
    nfin = ngrp;
  } else if (!last_block_done(b.tickets + kSeedTicket, nb)) {
    return;
  }
  for (int val = warp; val < 32 * nch; val += NT / 32) {
    const int ch = val >> 5, q = val & 31;
    const double sv = warp_sum_partials(fin + (int64_t)ch * nfin * 32, nfin, 32, q);
    if (lane == 0) {
      if (q == 0) {
        if (ch == 0) s_alpha = sv;
      } else if (q <= 2 * kDotsPerChunk) {
        const int j = 1 + kDotsPerChunk * ch + (q - 1) / 2;
        if (j < nr) {
          if ((q - 1) % 2 == 0) sums[j].x = sv;
          else sums[j].y = sv;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) seed_step_scalars(b, i, s_alpha, sums);
}

// alpha_i and the LU-update scalars when no g^j is formed here (blocked
// seeding, or system 1 alone): with u = A f as in k_seed_dots, v_i = f /
// beta_{i-1} into V, f = u / beta_{i-1} - beta_{i-1} v_{i-1},
// alpha_i = Re(v_i^H f), one value per block summed in block order by the last.
template <class T>
__global__ void __launch_bounds__(NT) k_seed_alpha(SeedBufs<T> b) {
  SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sm[NT / 32];
  const int i = st->i;
  T *vi = b.V + (int64_t)(i - 1) * b.ldv;
  const T *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * b.ldv;
  const double bp = (i > 1) ? st->beta_prev : 0.0, inv_b = st->inv_beta;
  typename Sc<T>::A acc = 0;
  GRID_STRIDE(e, b.n) {
    const T v = Sc<T>::scale(inv_b, b.f[e]);
    vi[e] = v;
    const T ue = Sc<T>::scale(inv_b, b.u[e]);
    const T fe = (i > 1) ? Sc<T>::axpy(-bp, vm[e], ue) : ue;
    b.f[e] = fe;
    acc = Sc<T>::redot(v, fe, acc);
  }
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  if (threadIdx.x == 0) b.partials[blockIdx.x] = v[0];
  if (!last_block_done(b.tickets + kSeedTicket, gridDim.x)) return;
  const double a = sum_partials<NT>(b.partials, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) seed_step_scalars(b, i, a, nullptr);
}

// f -= alpha_i v_i, the LU update (w_i, x^1) and the seeding (x^j), plus ||f||^2 when this
// step has no reorthogonalization.  Blocked seeding (b.Wb set): w_i also goes
// to column i - blk0 of Wb and x^2..x^p wait for the block's flush.
template <class T, bool NORM>
__global__ void __launch_bounds__(NT) k_seed_update(SeedBufs<T> b) {
  SeedState *st = b.st;
  if (!st->active) return;
  __shared__ typename Sc<T>::A2 s_eta[kMaxRhs];
  __shared__ double sm[NT / 32];
  const int i = st->i;
  T *wcol = nullptr;
  int nx = b.nrhs;   // columns of X updated here
  if (b.Wb != nullptr) {
    const int q = i - st->blk0;
    if (q < 0 || q >= kSeedBlock) {   // the host flushes before a block can fill
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->active = 0;
        st->stop_reason = STOP_BLOCK;
      }
      return;
    }
    wcol = b.Wb + (int64_t)q * b.ldv;
    nx = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->w_last = i;   // read only by later kernels
  }
  for (int j = threadIdx.x; j < nx; j += NT) s_eta[j] = Sc<T>::from2(b.eta[j]);
  __syncthreads();
  const double a = st->alpha, zeta = st->zeta, inv_d = st->inv_delta, bp = st->beta_prev;
  const T *vi = b.V + (int64_t)(i - 1) * b.ldv;
  const int64_t ldx = b.call->ldx;
  T *const X = reinterpret_cast<T *>(b.call->X);
  typename Sc<T>::A acc = 0;
  GRID_STRIDE(e, b.n) {
    const T ve = vi[e];
    const T fe = Sc<T>::axpy(-a, ve, b.f[e]);
    b.f[e] = fe;
    const T we = (i > 1) ? Sc<T>::scale(inv_d, Sc<T>::axpy(-bp, b.w[e], ve)) : Sc<T>::scale(inv_d, ve);
    b.w[e] = we;
    if (wcol != nullptr) wcol[e] = we;
    T *x = X + e;
    x[0] = Sc<T>::axpy(zeta, we, x[0]);
    // x^j += eta^j w_i, four columns at a time with the loads issued before the stores
    int j = 1;
    for (; j + 3 < nx; j += 4) {
      const T x0 = x[j * ldx], x1 = x[(j + 1) * ldx], x2 = x[(j + 2) * ldx], x3 = x[(j + 3) * ldx];
      x[j * ldx] = Sc<T>::caxpy2(s_eta[j], we, x0);
      x[(j + 1) * ldx] = Sc<T>::caxpy2(s_eta[j + 1], we, x1);
      x[(j + 2) * ldx] = Sc<T>::caxpy2(s_eta[j + 2], we, x2);
      x[(j + 3) * ldx] = Sc<T>::caxpy2(s_eta[j + 3], we, x3);
    }
    for (; j < nx; ++j) x[j * ldx] = Sc<T>::caxpy2(s_eta[j], we, x[j * ldx]);
    if (NORM) acc = Sc<T>::nrm2(fe, acc);
  }
  if (!NORM) return;
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  if (threadIdx.x == 0) b.partials[blockIdx.x] = v[0];
  if (!last_block_done(b.tickets + kSeedTicket, gridDim.x)) return;
  const double s = sum_partials<NT>(b.partials, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) seed_finish(b, s);
}

// ---------------------------------------------------------------------------
// Sec. 3 reorthogonalization: reorthonormalize v_i against v_1..v_{i-1}, then
// reorthogonalize f against v_1..v_i.  Classical Gram-Schmidt in blocked form:
// H = V_{<i}^H [v_i f], [v_i f] -= V_{<i} H (repeated `passes` times), then
// v_i /= ||v_i|| and f -= (v_i^H f) v_i (repeated `passes` times).
// ---------------------------------------------------------------------------

// One tile of H partials: rows [rb*R, (rb+1)*R) x columns [c0, c0+8) of V
// against the two vectors F0, F1.  Hpart[(rb*kcap + c)*2 + v].
template <class T>
SEED_DEV void gram_tile(const T *__restrict__ V, int64_t ldv, int64_t n, int rows, int rb, int c0, int nc,
                        const T *__restrict__ F0, const T *__restrict__ F1, double2 *Hpart, int kcap,
                        double (*sred)[32]) {
  typename Sc<T>::A2 acc[8][2];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c][0] = acc[c][1] = Sc<T>::zero2();
  const int64_t r0 = (int64_t)rb * rows;
  const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += NT) {
    const T f0 = F0[row], f1 = F1[row];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < nc) {
        const T v = V[row + (int64_t)(c0 + c) * ldv];
        acc[c][0] = Sc<T>::dotc(v, f0, acc[c][0]);
        acc[c][1] = Sc<T>::dotc(v, f1, acc[c][1]);
      }
    }
  }
  double vals[32];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    vals[4 * c + 0] = acc[c][0].x;
    vals[4 * c + 1] = acc[c][0].y;
    vals[4 * c + 2] = acc[c][1].x;
    vals[4 * c + 3] = acc[c][1].y;
  }
  const double mine = warp_reduce_scatter32(vals);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  sred[warp][lane] = mine;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double s = ((sred[0][lane] + sred[1][lane]) + sred[2][lane]) + sred[3][lane];
    const int c = lane >> 2, vv = (lane >> 1) & 1, ri = lane & 1;
    if (c < nc) reinterpret_cast<double *>(Hpart)[(((int64_t)rb * kcap + c0 + c) * 2 + vv) * 2 + ri] = s;
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(NT) k_reorth_tiles(SeedBufs<T> b, ReorthBufs<T> r) {
  const SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sred[NT / 32][32];
  const int i = st->i, k = i - 1;
  const T *F0 = b.V + (int64_t)(i - 1) * b.ldv;
  const int nck = (k + 7) / 8;
  const int64_t items = (int64_t)r.nrb * nck;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int rb = (int)(it % r.nrb), cb = (int)(it / r.nrb);
    const int c0 = cb * 8;
    const int nc = (k - c0 < 8) ? k - c0 : 8;
    gram_tile<T>(r.V, r.ldv, r.n, r.rows_per_item, rb, c0, nc, F0, b.f, r.Hpart, r.kcap, sred);
  }
}

// Long low-precision vectors: the partial products by row chunks.  Block b
// takes rows [b R, (b + 1) R) (R = r.row_chunk, 4096 to 8192, about two chunks
// per SM) against every column of V_{<i} in tiles of 8; the chunk's v_i and f
// (64 to 128 KB in FP32) are staged in shared memory once for all the block's
// tiles (with one block per (row block, tile) pair they were re-read for every
// tile, and V streamed at a fifth of the HBM rate).
// Hrows[(b kcap + c) 2 + v].
template <class T> constexpr bool kLowT = std::is_same_v<T, float> || std::is_same_v<T, float2>;
constexpr int kRowThreads = 256;

template <class T>
__global__ void __launch_bounds__(kRowThreads) k_reorth_rows(SeedBufs<T> b, ReorthBufs<T> r, double2 *Hrows) {
  const SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sred[kRowThreads / 32][32];
  extern __shared__ unsigned char s_dyn[];
  T *sF = reinterpret_cast<T *>(s_dyn);   // [2][row_chunk]: this chunk of v_i and f
  const int i = st->i, k = i - 1;
  const int64_t r0 = (int64_t)blockIdx.x * r.row_chunk;
  const int64_t r1 = (r0 + r.row_chunk < r.n) ? r0 + r.row_chunk : r.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    const T *vi = b.V + (int64_t)(i - 1) * b.ldv;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += kRowThreads) {
      sF[row - r0] = vi[row];
      sF[r.row_chunk + row - r0] = b.f[row];
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < k; c0 += 8) {
    const int nc = (k - c0 < 8) ? k - c0 : 8;
    typename Sc<T>::A2 acc[8][2];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c][0] = acc[c][1] = Sc<T>::zero2();
    const T *Vc = r.V + (int64_t)c0 * r.ldv;
#pragma unroll 2
    for (int64_t row = r0 + threadIdx.x; row < r1; row += kRowThreads) {
      const T f0 = sF[row - r0], f1 = sF[r.row_chunk + row - r0];
      T v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = c < nc ? Vc[row + (int64_t)c * r.ldv] : Sc<T>::zero();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        acc[c][0] = Sc<T>::dotc(v[c], f0, acc[c][0]);
        acc[c][1] = Sc<T>::dotc(v[c], f1, acc[c][1]);
      }
    }
    double vals[32];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      vals[4 * c + 0] = acc[c][0].x;
      vals[4 * c + 1] = acc[c][0].y;
      vals[4 * c + 2] = acc[c][1].x;
      vals[4 * c + 3] = acc[c][1].y;
    }
    sred[warp][lane] = warp_reduce_scatter32(vals);
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kRowThreads / 32; ++w) t += sred[w][lane];
      const int c = lane >> 2, vv = (lane >> 1) & 1, ri = lane & 1;
      if (c < nc) reinterpret_cast<double *>(Hrows)[(((int64_t)blockIdx.x * r.kcap + c0 + c) * 2 + vv) * 2 + ri] = t;
    }
    __syncthreads();
  }
}

// H[c][v] = sum over the row chunks (in order) of Hrows: one warp per value,
// lane l taking chunks l, l + 32, ... in order, then a fixed shuffle tree.
template <class T>
__global__ void __launch_bounds__(NT) k_reorth_rows_reduce(SeedBufs<T> b, ReorthBufs<T> r, const double2 *Hrows,
                                                           int nchunks) {
  const SeedState *st = b.st;
  if (!st->active) return;
  const int k = st->i - 1, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);   // value: column q / 2, vector q % 2
  if (q >= 2 * (int64_t)k) return;
  double sx = 0.0, sy = 0.0;
  for (int ch = lane; ch < nchunks; ch += 32) {
    const double2 h = __ldcg(Hrows + (int64_t)ch * r.kcap * 2 + q);
    sx += h.x;
    sy += h.y;
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (lane == 0) r.H[q] = c2(sx, sy);
}

// H[c][v] = sum over row blocks (in order) of Hpart
SEED_DEV void gram_reduce(const double2 *Hpart, double2 *H, int k, int nrb, int kcap) {
  for (int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x; q < 2 * (int64_t)k; q += (int64_t)gridDim.x * NT) {
    const int64_t c = q >> 1, v = q & 1;
    double2 s = c2(0.0, 0.0);
    for (int rb = 0; rb < nrb; ++rb) s = cadd(s, Hpart[((int64_t)rb * kcap + c) * 2 + v]);
    H[c * 2 + v] = s;
  }
}

template <class T>
__global__ void __launch_bounds__(NT) k_reorth_reduce(SeedBufs<T> b, ReorthBufs<T> r) {
  const SeedState *st = b.st;
  if (!st->active) return;
  gram_reduce(r.Hpart, r.H, st->i - 1, r.nrb, r.kcap);
}

// F_v += sgn * V[:, 0:k] H[:, v] for the two vectors.  A block covers NT / S
// rows; its S thread groups (S = 1, 2 or 4: one warp each when S = 4) take
// consecutive slices of every 256-column chunk of H, and the S partial sums of
// a row are added in group order (fixed, so the result does not depend on the
// timing).  Short vectors use S = 4 so that a 4096-row vector still spreads
// over 128 blocks instead of 32 serial ones.
template <class T>
SEED_DEV void gram_update(const T *__restrict__ V, int64_t ldv, int64_t n, int k, const double2 *__restrict__ H,
                          T *F0, T *F1, double sgn, int S) {
  __shared__ typename Sc<T>::A2 sH[256][2];
  __shared__ T spart[2][NT];
  const int rb = NT / S, sub = threadIdx.x / rb, rl = threadIdx.x - sub * rb;
  const int64_t row = (int64_t)blockIdx.x * rb + rl;
  const bool valid = row < n;
  T a0 = Sc<T>::zero(), a1 = Sc<T>::zero();
  for (int c0 = 0; c0 < k; c0 += 256) {
    const int cn = (k - c0 < 256) ? k - c0 : 256;
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * cn; q += NT)
      sH[q >> 1][q & 1] = Sc<T>::from2(H[(int64_t)(c0 + (q >> 1)) * 2 + (q & 1)]);
    __syncthreads();
    if (valid) {
      const int ca = cn * sub / S, cb = cn * (sub + 1) / S;
      const T *vr = V + row + (int64_t)c0 * ldv;
#pragma unroll 4
      for (int c = ca; c < cb; ++c) {
        const T v = vr[(int64_t)c * ldv];
        a0 = Sc<T>::caxpy2(sH[c][0], v, a0);
        a1 = Sc<T>::caxpy2(sH[c][1], v, a1);
      }
    }
  }
  if (S > 1) {
    spart[0][threadIdx.x] = a0;
    spart[1][threadIdx.x] = a1;
    __syncthreads();
    if (sub != 0) return;
    for (int q = 1; q < S; ++q) {
      a0 = Sc<T>::add(a0, spart[0][q * rb + rl]);
      a1 = Sc<T>::add(a1, spart[1][q * rb + rl]);
    }
  }
  if (valid) {
    F0[row] = Sc<T>::axpy(sgn, a0, F0[row]);
    if (F1 != nullptr) F1[row] = Sc<T>::axpy(sgn, a1, F1[row]);
  }
}

// column slices per row block of gram_update: 4 below 304 blocks of NT rows
// (two per SM), else 1
inline int gram_splits(int64_t n) { return n < (int64_t)NT * 304 ? 4 : 1; }
inline int gram_blocks(int64_t n) { return (int)((n + NT / gram_splits(n) - 1) / (NT / gram_splits(n))); }

template <class T>
__global__ void __launch_bounds__(NT) k_reorth_sub(SeedBufs<T> b, ReorthBufs<T> r, int S) {
  const SeedState *st = b.st;
  if (!st->active) return;
  const int i = st->i;
  gram_update<T>(r.V, r.ldv, r.n, i - 1, r.H, b.V + (int64_t)(i - 1) * b.ldv, b.f, -1.0, S);
}

// scratch = 1 / ||v_i||
template <class T>
__global__ void __launch_bounds__(NT) k_reorth_norm_vi(SeedBufs<T> b) {
  SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sm[NT / 32];
  const T *vi = b.V + (int64_t)(st->i - 1) * b.ldv;
  typename Sc<T>::A acc = 0;
  GRID_STRIDE(e, b.n) acc = Sc<T>::nrm2(vi[e], acc);
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  if (threadIdx.x == 0) b.partials[blockIdx.x] = v[0];
  if (!last_block_done(b.tickets + kSeedTicket, gridDim.x)) return;
  const double s = sum_partials<NT>(b.partials, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) st->scratch = 1.0 / sqrt(s);
}

// v_i *= scratch; h = v_i^H f
template <class T>
__global__ void __launch_bounds__(NT) k_reorth_scale_dot(SeedBufs<T> b) {
  SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sm[2 * NT / 32];
  T *vi = b.V + (int64_t)(st->i - 1) * b.ldv;
  const double sc = st->scratch;
  typename Sc<T>::A2 acc = Sc<T>::zero2();
  GRID_STRIDE(e, b.n) {
    const T v = Sc<T>::scale(sc, vi[e]);
    vi[e] = v;
    acc = Sc<T>::dotc(v, b.f[e], acc);
  }
  double v[2] = {(double)acc.x, (double)acc.y};
  block_sum<2, NT>(v, sm);
  if (threadIdx.x == 0) {
    b.partials[blockIdx.x * 2] = v[0];
    b.partials[blockIdx.x * 2 + 1] = v[1];
  }
  if (!last_block_done(b.tickets + kSeedTicket, gridDim.x)) return;
  const double re = sum_partials<NT>(b.partials, gridDim.x, 2, 0, sm);
  const double im = sum_partials<NT>(b.partials, gridDim.x, 2, 1, sm);
  if (threadIdx.x == 0) st->h = c2(re, im);
}

// f -= h v_i; then either h = v_i^H f (DOT) or ||f||^2 -> end of the step (seed_finish)
template <class T, bool DOT>
__global__ void __launch_bounds__(NT) k_reorth_axpy(SeedBufs<T> b) {
  SeedState *st = b.st;
  if (!st->active) return;
  __shared__ double sm[2 * NT / 32];
  const T *vi = b.V + (int64_t)(st->i - 1) * b.ldv;
  const double2 h = st->h;
  const double2 mh = c2(-h.x, -h.y);
  typename Sc<T>::A2 acc = Sc<T>::zero2();
  GRID_STRIDE(e, b.n) {
    const T v = vi[e];
    const T fe = Sc<T>::caxpy(mh, v, b.f[e]);
    b.f[e] = fe;
    if (DOT) acc = Sc<T>::dotc(v, fe, acc);
    else acc.x = Sc<T>::nrm2(fe, acc.x);
  }
  double v[2] = {(double)acc.x, (double)acc.y};
  block_sum<2, NT>(v, sm);
  if (threadIdx.x == 0) {
    b.partials[blockIdx.x * 2] = v[0];
    b.partials[blockIdx.x * 2 + 1] = v[1];
  }
  if (!last_block_done(b.tickets + kSeedTicket, gridDim.x)) return;
  const double re = sum_partials<NT>(b.partials, gridDim.x, 2, 0, sm);
  const double im = sum_partials<NT>(b.partials, gridDim.x, 2, 1, sm);
  if (threadIdx.x == 0) {
    if (DOT) st->h = c2(re, im);
    else seed_finish(b, re);
  }
}

template <class T>
void launch_seed_start(const SeedBufs<T> &b, const T *r01, cudaStream_t s) {
  k_seed_start<T><<<b.nblocks, NT, 0, s>>>(b, r01);
}
template <class T>
void launch_seed_dots(const SeedBufs<T> &b, cudaStream_t s) {
  if (b.Wb != nullptr || b.nrhs <= 1) k_seed_alpha<T><<<b.nblocks, NT, 0, s>>>(b);
  else k_seed_dots<T><<<b.nblocks, NT, 0, s>>>(b);
}
template <class T>
void launch_seed_update(const SeedBufs<T> &b, bool with_norm, cudaStream_t s) {
  if (with_norm) k_seed_update<T, true><<<b.nblocks, NT, 0, s>>>(b);
  else k_seed_update<T, false><<<b.nblocks, NT, 0, s>>>(b);
}
template <class T>
void launch_reorth(const SeedBufs<T> &b, const ReorthBufs<T> &r, int passes, cudaStream_t s) {
  const bool rows = kLowT<T> && r.Hrows != nullptr;
  const int nchunks = rows ? (int)((r.n + r.row_chunk - 1) / r.row_chunk) : 0;
  for (int p = 0; p < passes; ++p) {
    if (rows) {
      const size_t smem = 2 * sizeof(T) * (size_t)r.row_chunk;
      // once per instantiation (thread-safe static initialisation: batch workers launch concurrently):
      // allow up to 2 x 8192 rows of shared memory
      static const cudaError_t attr =
          cudaFuncSetAttribute(k_reorth_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (int)sizeof(T) * 8192);
      (void)attr;   // a failure shows as the launch's error
      k_reorth_rows<T><<<nchunks, kRowThreads, smem, s>>>(b, r, r.Hrows);
      k_reorth_rows_reduce<T><<<(2 * r.kcap + NT / 32 - 1) / (NT / 32), NT, 0, s>>>(b, r, r.Hrows, nchunks);
    } else {
      k_reorth_tiles<T><<<r.nitems_grid, NT, 0, s>>>(b, r);
      k_reorth_reduce<T><<<64, NT, 0, s>>>(b, r);
    }
    k_reorth_sub<T><<<gram_blocks(r.n), NT, 0, s>>>(b, r, gram_splits(r.n));
  }
  k_reorth_norm_vi<T><<<b.nblocks, NT, 0, s>>>(b);
  k_reorth_scale_dot<T><<<b.nblocks, NT, 0, s>>>(b);
  for (int p = 1; p < passes; ++p) k_reorth_axpy<T, true><<<b.nblocks, NT, 0, s>>>(b);
  k_reorth_axpy<T, false><<<b.nblocks, NT, 0, s>>>(b);
}
template <class T>
int reorth_kernel_count(int passes) {
  return 3 * passes + 2 + passes;
}

// ---------------------------------------------------------------------------
// Galerkin projection over a kept basis: X += V T^{-1} V^H R
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(NT) k_gram_tiles(const T *V, int64_t ldv, int64_t n, int k, int rows, int nrb,
                                                   const T *F0, const T *F1, double2 *Hpart, int kcap) {
  __shared__ double sred[NT / 32][32];
  const int nck = (k + 7) / 8;
  const int64_t items = (int64_t)nrb * nck;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int rb = (int)(it % nrb), cb = (int)(it / nrb);
    const int c0 = cb * 8;
    const int nc = (k - c0 < 8) ? k - c0 : 8;
    gram_tile<T>(V, ldv, n, rows, rb, c0, nc, F0, F1, Hpart, kcap, sred);
  }
}
__global__ void k_gram_reduce(const double2 *Hpart, double2 *H, int k, int nrb, int kcap) {
  gram_reduce(Hpart, H, k, nrb, kcap);
}
// Solve T y = g for both columns of G in place (Thomas algorithm; T from the
// recorded alpha_1..alpha_m, beta_1..beta_{m-1}; index 1-based).  c' is kept
// in cp[m] per column.
__global__ void k_tridiag_solve(const double *alpha, const double *beta, int m, double2 *G, double *cp) {
  const int v = threadIdx.x;
  if (v >= 2) return;
  double *c = cp + (int64_t)v * m;
  double den = alpha[1];
  c[0] = (m > 1) ? beta[1] / den : 0.0;
  double2 d = G[v];
  d = c2(d.x / den, d.y / den);
  G[v] = d;
  for (int k = 1; k < m; ++k) {
    den = alpha[k + 1] - beta[k] * c[k - 1];
    c[k] = (k + 1 < m) ? beta[k + 1] / den : 0.0;
    const double2 g = G[(int64_t)k * 2 + v];
    d = c2((g.x - beta[k] * d.x) / den, (g.y - beta[k] * d.y) / den);
    G[(int64_t)k * 2 + v] = d;
  }
  for (int k = m - 2; k >= 0; --k) {
    const double2 nx = G[(int64_t)(k + 1) * 2 + v];
    const double2 cur = G[(int64_t)k * 2 + v];
    G[(int64_t)k * 2 + v] = c2(cur.x - c[k] * nx.x, cur.y - c[k] * nx.y);
  }
}
template <class T>
__global__ void __launch_bounds__(NT) k_gram_add(const T *V, int64_t ldv, int64_t n, int k, const double2 *H, T *F0,
                                                 T *F1, int S) {
  gram_update<T>(V, ldv, n, k, H, F0, F1, 1.0, S);
}

template <class T>
void launch_project(int64_t n, const T *V, int64_t ldv, int m, const double *alpha, const double *beta, const T *R,
                    int64_t ldr, T *X, int64_t ldx, int ncols, double2 *G, double2 *Gpart, int nrb,
                    int rows_per_item, cudaStream_t s) {
  for (int j = 0; j < ncols; j += 2) {
    const bool two = j + 1 < ncols;
    const T *F0 = R + (int64_t)j * ldr;
    const T *F1 = two ? R + (int64_t)(j + 1) * ldr : F0;
    k_gram_tiles<T><<<152 * 4, NT, 0, s>>>(V, ldv, n, m, rows_per_item, nrb, F0, F1, Gpart, m + 1);
    k_gram_reduce<<<64, NT, 0, s>>>(Gpart, G, m, nrb, m + 1);
    // the Thomas scratch reuses the (now reduced) partial buffer
    k_tridiag_solve<<<1, 32, 0, s>>>(alpha, beta, m, G, reinterpret_cast<double *>(Gpart));
    k_gram_add<T><<<gram_blocks(n), NT, 0, s>>>(V, ldv, n, m, G, X + (int64_t)j * ldx,
                                                two ? X + (int64_t)(j + 1) * ldx : nullptr, gram_splits(n));
  }
}

// ---------------------------------------------------------------------------
// column utilities
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(NT) k_copy_cols(const T *src, int64_t lds, T *dst, int64_t ldd, int64_t n) {
  const int col = blockIdx.y;
  src += (int64_t)col * lds;
  dst += (int64_t)col * ldd;
  GRID_STRIDE(e, n) dst[e] = src[e];
}
template <class T>
__global__ void __launch_bounds__(NT) k_zero_cols(T *dst, int64_t ldd, int64_t n) {
  dst += (int64_t)blockIdx.y * ldd;
  GRID_STRIDE(e, n) dst[e] = Sc<T>::zero();
}
template <class T>
__global__ void __launch_bounds__(NT) k_sub_from(const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R, int64_t ldr,
                                                 int64_t n) {
  const int col = blockIdx.y;
  B += (int64_t)col * ldb;
  Q += (int64_t)col * ldq;
  R += (int64_t)col * ldr;
  GRID_STRIDE(e, n) R[e] = Sc<T>::sub(B[e], Q[e]);
}
template <class T>
__global__ void __launch_bounds__(NT) k_colnorms(int64_t n, const T *X, int64_t ldx, double *out, double *partials,
                                                 unsigned *tickets) {
  __shared__ double sm[NT / 32];
  const int col = blockIdx.y;
  X += (int64_t)col * ldx;
  typename Sc<T>::A acc = 0;
  GRID_STRIDE(e, n) acc = Sc<T>::nrm2(X[e], acc);
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  if (threadIdx.x == 0) partials[(int64_t)col * gridDim.x + blockIdx.x] = v[0];
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double s = sum_partials<NT>(partials + (int64_t)col * gridDim.x, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) out[col] = sqrt(s);
}

template <class T>
void launch_copy_cols(const T *src, int64_t lds, T *dst, int64_t ldd, int64_t n, int ncols, cudaStream_t s) {
  dim3 g((unsigned)vec_blocks(n), (unsigned)ncols);
  k_copy_cols<T><<<g, NT, 0, s>>>(src, lds, dst, ldd, n);
}
template <class T>
void launch_zero_cols(T *dst, int64_t ldd, int64_t n, int ncols, cudaStream_t s) {
  dim3 g((unsigned)vec_blocks(n), (unsigned)ncols);
  k_zero_cols<T><<<g, NT, 0, s>>>(dst, ldd, n);
}
template <class T>
void launch_sub_from(const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R, int64_t ldr, int64_t n, int ncols,
                     cudaStream_t s) {
  dim3 g((unsigned)vec_blocks(n), (unsigned)ncols);
  k_sub_from<T><<<g, NT, 0, s>>>(B, ldb, Q, ldq, R, ldr, n);
}
template <class T>
void launch_colnorms(int64_t n, const T *X, int64_t ldx, int ncols, double *out, double *partials, unsigned *tickets,
                     cudaStream_t s) {
  dim3 g((unsigned)col_blocks(n, ncols), (unsigned)ncols);
  k_colnorms<T><<<g, NT, 0, s>>>(n, X, ldx, out, partials, tickets);
}

// ---------------------------------------------------------------------------
// Lockstep CG (Hestenes-Stiefel) on nc columns; per-column scalars in CgCols.
// ---------------------------------------------------------------------------

// r = b - q (q = A x), p = r, rho = ||r||^2; a column already within tol is done.
template <class T>
__global__ void __launch_bounds__(NT) k_cg_init(int64_t n, const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R,
                                                T *P, int64_t ld, CgCols c, double *partials, unsigned *tickets) {
  __shared__ double sm[2 * NT / 32];
  const int col = blockIdx.y;
  B += (int64_t)col * ldb;
  Q += (int64_t)col * ldq;
  R += (int64_t)col * ld;
  P += (int64_t)col * ld;
  typename Sc<T>::A rr = 0, bb = 0;
  GRID_STRIDE(e, n) {
    const T bv = B[e];
    const T r = Sc<T>::sub(bv, Q[e]);
    R[e] = r;
    P[e] = r;
    rr = Sc<T>::nrm2(r, rr);
    bb = Sc<T>::nrm2(bv, bb);
  }
  double v[2] = {(double)rr, (double)bb};
  block_sum<2, NT>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x * 2;
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2] = v[0];
    part[blockIdx.x * 2 + 1] = v[1];
  }
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double srr = sum_partials<NT>(part, gridDim.x, 2, 0, sm);
  const double sbb = sum_partials<NT>(part, gridDim.x, 2, 1, sm);
  if (threadIdx.x == 0) {
    const double bn = sqrt(sbb), rn = sqrt(srr);
    c.rho[col] = srr;
    c.bnorm[col] = bn;
    c.relres[col] = bn > 0.0 ? rn / bn : 0.0;
    c.mvps[col] = 1;
    c.iters[col] = 0;
    c.restarts[col] = 0;
    c.needs_check[col] = 0;
    const int done = rn <= c.tol * bn;
    c.active[col] = !done;
    c.reached[col] = done;
    c.converged[col] = done;
  }
}

// alpha = rho / Re(p^H q)
template <class T>
__global__ void __launch_bounds__(NT) k_cg_alpha(int64_t n, const T *P, const T *Q, int64_t ld, CgCols c,
                                                 double *partials, unsigned *tickets) {
  __shared__ double sm[NT / 32];
  const int col = blockIdx.y;
  if (!c.active[col]) return;
  P += (int64_t)col * ld;
  Q += (int64_t)col * ld;
  typename Sc<T>::A acc = 0;
#pragma unroll 4
  GRID_STRIDE(e, n) acc = Sc<T>::redot(P[e], Q[e], acc);
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double pq = sum_partials<NT>(part, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) c.alpha[col] = c.rho[col] / pq;
}

// x += alpha p; r -= alpha q; test ||r|| <= tol ||b||; beta = rho'/rho
template <class T>
__global__ void __launch_bounds__(NT) k_cg_update(int64_t n, const CallArgs *call, T *R, const T *P, const T *Q,
                                                  int64_t ld, CgCols c, double *partials, unsigned *tickets) {
  __shared__ double sm[NT / 32];
  const int col = blockIdx.y;
  if (!c.active[col]) return;
  T *X = reinterpret_cast<T *>(call->X) + (int64_t)(col + call->col0) * call->ldx;
  R += (int64_t)col * ld;
  P += (int64_t)col * ld;
  Q += (int64_t)col * ld;
  const double a = c.alpha[col];
  typename Sc<T>::A acc = 0;
#pragma unroll 4
  GRID_STRIDE(e, n) {
    X[e] = Sc<T>::axpy(a, P[e], X[e]);
    const T r = Sc<T>::axpy(-a, Q[e], R[e]);
    R[e] = r;
    acc = Sc<T>::nrm2(r, acc);
  }
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double rr = sum_partials<NT>(part, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) cg_update_tail(c, col, rr);
}

// p = r + beta p (also used with beta = 0 after a restart: p = r)
template <class T>
__global__ void __launch_bounds__(NT) k_cg_p(int64_t n, const T *R, T *P, int64_t ld, CgCols c, int copy_only) {
  const int col = blockIdx.y;
  if (!c.active[col]) return;
  R += (int64_t)col * ld;
  P += (int64_t)col * ld;
  if (copy_only) {
    GRID_STRIDE(e, n) P[e] = R[e];
  } else {
    const double be = c.beta[col];
#pragma unroll 4
    GRID_STRIDE(e, n) P[e] = Sc<T>::axpy(be, P[e], R[e]);
  }
}

// true residual r = b - A x for columns that stopped; converged if within
// 1.5 tol, otherwise restart (p = r in the next kernel) while restarts remain.
template <class T>
__global__ void __launch_bounds__(NT) k_cg_check(int64_t n, const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R,
                                                 int64_t ld, CgCols c, double *partials, unsigned *tickets) {
  __shared__ double sm[NT / 32];
  const int col = blockIdx.y;
  if (!c.needs_check[col]) return;
  B += (int64_t)col * ldb;
  Q += (int64_t)col * ldq;
  R += (int64_t)col * ld;
  typename Sc<T>::A acc = 0;
  GRID_STRIDE(e, n) {
    const T r = Sc<T>::sub(B[e], Q[e]);
    R[e] = r;
    acc = Sc<T>::nrm2(r, acc);
  }
  double v[1] = {(double)acc};
  block_sum<1, NT>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double rr = sum_partials<NT>(part, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) {
    const double rn = sqrt(rr), bn = c.bnorm[col];
    c.relres[col] = bn > 0.0 ? rn / bn : 0.0;
    c.mvps[col] += 1;
    c.needs_check[col] = 0;
    if (c.reached[col] && rn <= c.tol_check * bn) {
      c.converged[col] = 1;
    } else if (c.reached[col] && c.restarts[col] < c.max_restarts) {
      c.restarts[col] += 1;
      c.active[col] = 1;
      c.reached[col] = 0;
      c.rho[col] = rr;
    }
  }
}

template <class T>
void launch_cg_init(int64_t n, const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R, T *P, int64_t ld,
                    const CgCols &c, double *partials, unsigned *tickets, bool restart_only, cudaStream_t s) {
  dim3 g((unsigned)col_blocks(n, c.nc), (unsigned)c.nc);
  if (restart_only) k_cg_p<T><<<g, NT, 0, s>>>(n, R, P, ld, c, 1);
  else k_cg_init<T><<<g, NT, 0, s>>>(n, B, ldb, Q, ldq, R, P, ld, c, partials, tickets);
}
template <class T>
void launch_cg_alpha(int64_t n, const T *P, const T *Q, int64_t ld, const CgCols &c, double *partials,
                     unsigned *tickets, cudaStream_t s) {
  dim3 g((unsigned)col_blocks(n, c.nc), (unsigned)c.nc);
  k_cg_alpha<T><<<g, NT, 0, s>>>(n, P, Q, ld, c, partials, tickets);
}
template <class T>
void launch_cg_update(int64_t n, const CallArgs *call, T *R, const T *P, const T *Q, int64_t ld, const CgCols &c,
                      double *partials, unsigned *tickets, cudaStream_t s) {
  dim3 g((unsigned)col_blocks(n, c.nc), (unsigned)c.nc);
  k_cg_update<T><<<g, NT, 0, s>>>(n, call, R, P, Q, ld, c, partials, tickets);
}
template <class T>
void launch_cg_p(int64_t n, const T *R, T *P, int64_t ld, const CgCols &c, cudaStream_t s) {
  dim3 g((unsigned)col_blocks(n, c.nc), (unsigned)c.nc);
  k_cg_p<T><<<g, NT, 0, s>>>(n, R, P, ld, c, 0);
}
template <class T>
void launch_cg_check(int64_t n, const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R, int64_t ld, const CgCols &c,
                     double *partials, unsigned *tickets, cudaStream_t s) {
  dim3 g((unsigned)col_blocks(n, c.nc), (unsigned)c.nc);
  k_cg_check<T><<<g, NT, 0, s>>>(n, B, ldb, Q, ldq, R, ld, c, partials, tickets);
}

#define SEED_INSTANTIATE(T)                                                                                        \
  template void launch_seed_start<T>(const SeedBufs<T> &, const T *, cudaStream_t);                              \
  template void launch_seed_dots<T>(const SeedBufs<T> &, cudaStream_t);                                          \
  template void launch_seed_update<T>(const SeedBufs<T> &, bool, cudaStream_t);                                  \
  template void launch_reorth<T>(const SeedBufs<T> &, const ReorthBufs<T> &, int, cudaStream_t);                 \
  template int reorth_kernel_count<T>(int);                                                                      \
  template void launch_project<T>(int64_t, const T *, int64_t, int, const double *, const double *, const T *,   \
                                  int64_t, T *, int64_t, int, double2 *, double2 *, int, int, cudaStream_t);     \
  template void launch_copy_cols<T>(const T *, int64_t, T *, int64_t, int64_t, int, cudaStream_t);               \
  template void launch_zero_cols<T>(T *, int64_t, int64_t, int, cudaStream_t);                                   \
  template void launch_sub_from<T>(const T *, int64_t, const T *, int64_t, T *, int64_t, int64_t, int,           \
                                   cudaStream_t);                                                                \
  template void launch_colnorms<T>(int64_t, const T *, int64_t, int, double *, double *, unsigned *,             \
                                   cudaStream_t);                                                                \
  template void launch_cg_init<T>(int64_t, const T *, int64_t, const T *, int64_t, T *, T *, int64_t,            \
                                  const CgCols &, double *, unsigned *, bool, cudaStream_t);                     \
  template void launch_cg_alpha<T>(int64_t, const T *, const T *, int64_t, const CgCols &, double *, unsigned *, \
                                   cudaStream_t);                                                                \
  template void launch_cg_update<T>(int64_t, const CallArgs *, T *, const T *, const T *, int64_t, const CgCols &, \
                                    double *, unsigned *, cudaStream_t);                                         \
  template void launch_cg_p<T>(int64_t, const T *, T *, int64_t, const CgCols &, cudaStream_t);                  \
  template void launch_cg_check<T>(int64_t, const T *, int64_t, const T *, int64_t, T *, int64_t,                \
                                   const CgCols &, double *, unsigned *, cudaStream_t);

SEED_INSTANTIATE(double)
SEED_INSTANTIATE(double2)
SEED_INSTANTIATE(float)
SEED_INSTANTIATE(float2)

}  // namespace seedk
