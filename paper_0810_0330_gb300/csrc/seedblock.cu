// seedblock.cu -- the Sec. 3 seeding of systems 2..p in
// blocked form.
//
// Each Lanczos step i feeds the other right-hand sides through
//   g_i^j = v_i^H r_0^j,   eta_i^j = g_i^j - gamma_{i-1} eta_{i-1}^j,   x^j += eta_i^j w_i,
// and none of it flows back into the recurrence of system 1 (alpha_i, beta_i,
// delta_i, zeta_i and the stopping test use system 1 only).  So the steps of a
// block only store w_i (column i - blk0 of Wb) and gamma_{i-1}, and one flush
// per block forms
//   G = V_blk^H R_0      k_blk_dots, k_blk_reduce   (k x (p-1), fixed order)
//   eta^j                k_blk_eta                   (the scalar recursion, step order)
//   X_{2..p} += W Z      k_blk_x                     (Z = [eta_i^j], k x (p-1))
// reading the block's v_i and w_i once, instead of reading and writing p-1
// columns of X and forming p-1 dot products in every step.  Blocks end before
// a reorthogonalizing step rewrites v_i (Sec. 3), so V_blk holds the
// vectors the streaming form uses; the two forms differ in summation order
// only.
#include <type_traits>

#include "seed_device.cuh"

namespace seedk {

constexpr int NT = kVecThreads;
constexpr int kBQ = 8;   // steps per tile of G
constexpr int kBJ = 4;   // right-hand sides per tile of G
constexpr int kLdG = kMaxRhs - 1;

#define GRID_STRIDE(e, n) \
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < (n); e += (int64_t)gridDim.x * NT)

// Row chunks of the partial products: at most kBlockChunksMax, at least 1024 rows.
BlockBufs block_layout(int64_t n) {
  BlockBufs k{};
  int64_t nc = (n + 1023) / 1024;
  if (nc > kBlockChunksMax) nc = kBlockChunksMax;
  if (nc < 1) nc = 1;
  int64_t rows = (n + nc - 1) / nc;
  rows = (rows + NT - 1) / NT * NT;
  k.nchunk = (int)((n + rows - 1) / rows);
  k.rows = rows;
  return k;
}

// Partial products of one (row chunk, 8 steps, 4 right-hand sides) tile per
// item; items run chunk by chunk (tiles fastest), so the blocks in flight
// share one chunk of V_blk and R_0 in L2.
template <class T>
__global__ void __launch_bounds__(NT) k_blk_dots(SeedBufs<T> b, BlockBufs k) {
  const SeedState *st = b.st;
  const int blk0 = st->blk0, len = min(st->w_last - blk0 + 1, kSeedBlock), nj = b.nrhs - 1;
  if (len <= 0 || nj <= 0) return;
  __shared__ double sred[NT / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nqt = (len + kBQ - 1) / kBQ, njt = (nj + kBJ - 1) / kBJ, ntile = nqt * njt;
  const int64_t items = (int64_t)k.nchunk * ntile;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int tile = (int)(it % ntile), chunk = (int)(it / ntile);
    const int q0 = (tile % nqt) * kBQ, j0 = (tile / nqt) * kBJ;
    const int nq = min(kBQ, len - q0), njj = min(kBJ, nj - j0);
    const int64_t r0 = (int64_t)chunk * k.rows, r1 = min(b.n, r0 + k.rows);
    const T *Vq = b.V + (int64_t)(blk0 - 1 + q0) * b.ldv;   // column c of V holds v_{c+1}
    const T *Rj = b.R0 + (int64_t)j0 * b.ldr;
    typename Sc<T>::A2 acc[kBQ][kBJ];
#pragma unroll
    for (int qq = 0; qq < kBQ; ++qq)
#pragma unroll
      for (int jj = 0; jj < kBJ; ++jj) acc[qq][jj] = Sc<T>::zero2();
    // two rows per thread and iteration: twice the loads in flight
    for (int64_t row = r0 + threadIdx.x; row < r1; row += 2 * NT) {
      const int64_t row2 = row + NT;
      const bool two = row2 < r1;
      T r[kBJ], r2[kBJ];
#pragma unroll
      for (int jj = 0; jj < kBJ; ++jj) {
        r[jj] = jj < njj ? Rj[(int64_t)jj * b.ldr + row] : Sc<T>::zero();
        r2[jj] = (two && jj < njj) ? Rj[(int64_t)jj * b.ldr + row2] : Sc<T>::zero();
      }
#pragma unroll
      for (int qq = 0; qq < kBQ; ++qq) {
        if (qq < nq) {
          const T v = Vq[(int64_t)qq * b.ldv + row];
          const T v2 = two ? Vq[(int64_t)qq * b.ldv + row2] : Sc<T>::zero();
#pragma unroll
          for (int jj = 0; jj < kBJ; ++jj) {
            acc[qq][jj] = Sc<T>::dotc(v, r[jj], acc[qq][jj]);
            acc[qq][jj] = Sc<T>::dotc(v2, r2[jj], acc[qq][jj]);
          }
        }
      }
    }
    // 8 x 4 complex values: two block reductions of 32 (steps 4h .. 4h+3)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double vals[32];
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4)
#pragma unroll
        for (int jj = 0; jj < kBJ; ++jj) {
          vals[q4 * 8 + jj * 2] = (double)acc[4 * h + q4][jj].x;
          vals[q4 * 8 + jj * 2 + 1] = (double)acc[4 * h + q4][jj].y;
        }
      const double mine = warp_reduce_scatter32(vals);
      sred[warp][lane] = mine;
      __syncthreads();
      if (threadIdx.x < 32) {
        const double s = ((sred[0][lane] + sred[1][lane]) + sred[2][lane]) + sred[3][lane];
        const int qq = 4 * h + (lane >> 3), jj = (lane >> 1) & 3, ri = lane & 1;
        if (qq < nq && jj < njj)
          reinterpret_cast<double *>(k.Hpart)[(((int64_t)chunk * kSeedBlock + q0 + qq) * kLdG + j0 + jj) * 2 + ri] = s;
      }
      __syncthreads();
    }
  }
}

// G[q][j] = sum over chunks of the partials, in chunk order
__global__ void k_blk_reduce(const SeedState *st, int nrhs, BlockBufs k) {
  const int len = min(st->w_last - st->blk0 + 1, kSeedBlock), nj = nrhs - 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = idx / kLdG, j = idx - kLdG * (idx / kLdG);
  if (len <= 0 || q >= len || j >= nj) return;
  double2 s = c2(0.0, 0.0);
  for (int c = 0; c < k.nchunk; ++c) {
    const double2 v = __ldcg(k.Hpart + ((int64_t)c * kSeedBlock + q) * kLdG + j);
    s.x += v.x;
    s.y += v.y;
  }
  k.G[q * kLdG + j] = s;
}

// eta^j over the block, in step order: eta_1 = g_1,
// eta_i = g_i - gamma_{i-1} eta_{i-1}; Z[q][j] = eta at step blk0 + q.
// Then the next block starts after the last stored step.
__global__ void k_blk_eta(SeedState *st, int nrhs, double2 *eta, const double *gamma_hist, BlockBufs k) {
  const int blk0 = st->blk0, w_last = st->w_last, len = min(w_last - blk0 + 1, kSeedBlock);
  const int j = threadIdx.x;   // column j + 1 of X
  if (len > 0 && j < nrhs - 1) {
    double2 e = eta[j + 1];
    for (int q = 0; q < len; ++q) {
      const int i = blk0 + q;
      const double2 g = k.G[q * kLdG + j];
      if (i == 1) {
        e = g;
      } else {
        const double gam = gamma_hist[i];
        e = c2(g.x - gam * e.x, g.y - gam * e.y);
      }
      k.Z[q * kLdG + j] = e;
    }
    eta[j + 1] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->blk_len = len > 0 ? len : 0;
    st->blk0 = w_last + 1;
  }
}

// X[:, 1 + j] += sum_q Z[q][j] W[:, q], for the columns of grid.y's chunk.
// FP64 chunks of 4 columns (the work is bound by the FP64 pipe: more blocks),
// FP32 chunks of 16 (bound by memory: W read once per 16 columns).
template <class T> __host__ __device__ constexpr int blk_xcols() {
  return sizeof(typename Sc<T>::A) == sizeof(double) ? 4 : 16;
}

template <class T>
__global__ void __launch_bounds__(NT) k_blk_x(SeedBufs<T> b, BlockBufs k) {
  constexpr int XC = blk_xcols<T>();
  const int len = min(b.st->blk_len, kSeedBlock), nj = b.nrhs - 1;
  const int j0 = blockIdx.y * XC;
  if (len <= 0 || j0 >= nj) return;
  const int nc = min(XC, nj - j0);
  __shared__ typename Sc<T>::A2 sz[kSeedBlock][XC];
  for (int t = threadIdx.x; t < len * XC; t += NT) {
    const int q = t / XC, c = t - XC * (t / XC);
    sz[q][c] = c < nc ? Sc<T>::from2(k.Z[q * kLdG + j0 + c]) : Sc<T>::zero2();
  }
  __syncthreads();
  T *const X = reinterpret_cast<T *>(b.call->X);
  const int64_t ldx = b.call->ldx;
  GRID_STRIDE(e, b.n) {
    T acc[XC];
#pragma unroll
    for (int c = 0; c < XC; ++c) acc[c] = Sc<T>::zero();
#pragma unroll 4
    for (int q = 0; q < len; ++q) {
      const T w = b.Wb[(int64_t)q * b.ldv + e];
#pragma unroll
      for (int c = 0; c < XC; ++c) acc[c] = Sc<T>::caxpy2(sz[q][c], w, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < XC; ++c) {
      if (c < nc) {
        T *x = X + (int64_t)(1 + j0 + c) * ldx + e;
        *x = Sc<T>::add(*x, acc[c]);
      }
    }
  }
}

template <class T>
int launch_seed_flush(const SeedBufs<T> &b, const BlockBufs &k, cudaStream_t s) {
  if (b.Wb == nullptr || b.nrhs < 2) return 0;
  const int nj = b.nrhs - 1;
  if (std::is_same<T, float2>::value && k.tc && k.tc->ok) {
    // FP32 complex: G = V_blk^H R_0 on the tensor cores (3xTF32), then the same reduction
    launch_blk_dots_tc(k.tc->maps, b.st, 0, 0, nj, b.n, k.Hpart, k.tc->grid, k.tc->err, s);
    BlockBufs kr = k;
    kr.nchunk = k.tc->grid;
    k_blk_reduce<<<(kSeedBlock * kLdG + NT - 1) / NT, NT, 0, s>>>(b.st, b.nrhs, kr);
  } else {
    const int64_t tiles = (int64_t)((kSeedBlock + kBQ - 1) / kBQ) * ((nj + kBJ - 1) / kBJ);
    int64_t grid = (int64_t)k.nchunk * tiles;   // items of a full block; shorter blocks leave blocks idle
    if (grid > 152 * 16) grid = 152 * 16;
    k_blk_dots<T><<<(unsigned)grid, NT, 0, s>>>(b, k);
    k_blk_reduce<<<(kSeedBlock * kLdG + NT - 1) / NT, NT, 0, s>>>(b.st, b.nrhs, k);
  }
  k_blk_eta<<<1, kMaxRhs, 0, s>>>(b.st, b.nrhs, b.eta, b.gamma_hist, k);
  int64_t bx = (b.n + NT - 1) / NT;
  if (bx > 152 * 16) bx = 152 * 16;
  constexpr int XC = blk_xcols<T>();
  k_blk_x<T><<<dim3((unsigned)bx, (unsigned)((nj + XC - 1) / XC)), NT, 0, s>>>(b, k);
  return 4;
}

template int launch_seed_flush<double>(const SeedBufs<double> &, const BlockBufs &, cudaStream_t);
template int launch_seed_flush<double2>(const SeedBufs<double2> &, const BlockBufs &, cudaStream_t);
template int launch_seed_flush<float>(const SeedBufs<float> &, const BlockBufs &, cudaStream_t);
template int launch_seed_flush<float2>(const SeedBufs<float2> &, const BlockBufs &, cudaStream_t);

}  // namespace seedk
