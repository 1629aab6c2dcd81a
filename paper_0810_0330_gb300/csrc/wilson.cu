// wilson.cu -- Wilson-Dirac operator D and D^H on sm_103a (FP64 complex).
//
// Operator (Sec. 4 names the Wilson-Dirac matrix; the textbook form with
// r = 1 is used, gamma matrices in the DeGrand-Rossi basis):
//   (D_s psi)(n) = psi(n) - kappa sum_mu [ (1 - s g_mu) U_mu(n) psi(n+mu)
//                                         + (1 + s g_mu) U_mu(n-mu)^H psi(n-mu) ]
// with s = +1 for D and s = -1 for D^H = g5 D g5.
//
// Spin projection and the hops are in wilson_device.cuh: a hop multiplies only
// a two-spinor by the link (84 FP64 operations instead of 264), and the two
// hops of one direction share their spin algebra: 816 FP64 operations per
// site in all.
//
// GB300 runs FP64 at 1/64 of its FP32 rate (about 1.2 TFLOP/s measured), so
// this kernel is bound by the FP64 pipe, not by HBM: the design minimises FP64
// instructions.  Phase factors and boundary signs are register swaps and
// sign-bit flips (integer ops).  Thread layout: a block of 128 threads covers
// 32 sites; warp mu handles direction mu (forward and backward hop) for all 32
// sites, so every warp runs one uniform code path.  The four per-direction
// partial sums meet in shared memory, then each output is psi - kappa * sum.
#include "wilson_device.cuh"

namespace seedk {

// ---------------------------------------------------------------------------
// neighbour table: nbr[8 s + 2 mu] = s + mu-hat, nbr[8 s + 2 mu + 1] = s - mu-hat
// ---------------------------------------------------------------------------
__global__ void k_wilson_neighbors(int32_t X, int32_t Y, int32_t Z, int32_t T, int64_t vol, int32_t *nbr) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= vol) return;
  const int32_t dims[4] = {X, Y, Z, T};
  int32_t c[4];
  int64_t r = s;
  c[0] = (int32_t)(r % X); r /= X;
  c[1] = (int32_t)(r % Y); r /= Y;
  c[2] = (int32_t)(r % Z); r /= Z;
  c[3] = (int32_t)r;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      int32_t cc[4] = {c[0], c[1], c[2], c[3]};
      if (dir == 0) cc[mu] = (c[mu] + 1 == dims[mu]) ? 0 : c[mu] + 1;
      else cc[mu] = (c[mu] == 0) ? dims[mu] - 1 : c[mu] - 1;
      int64_t t = cc[0] + (int64_t)X * (cc[1] + (int64_t)Y * (cc[2] + (int64_t)Z * cc[3]));
      nbr[8 * s + 2 * mu + dir] = (int32_t)t;
    }
  }
}

void launch_wilson_neighbors(const int32_t dims[4], int32_t *nbr, cudaStream_t s) {
  int64_t vol = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  int blocks = (int)((vol + 255) / 256);
  k_wilson_neighbors<<<blocks, 256, 0, s>>>(dims[0], dims[1], dims[2], dims[3], vol, nbr);
}


// Grid: one block per (32-site tile, column), the column fastest (blockIdx.x,
// tiles on blockIdx.y) while the tiles fit in gridDim.y, so that the columns of
// one tile run together and its links are read from DRAM once per launch even
// when the links do not fit in L2 (with the column slowest every column re-read
// them: 2.3x the algorithmic DRAM bytes at 24^4 x 11 columns).
template <int S, bool COLX, class C>
__global__ void __launch_bounds__(128) k_dslash(WilsonOpT<C> op, const C *__restrict__ in, int64_t ldi,
                                                C *__restrict__ out, int64_t ldo,
                                                const int32_t *__restrict__ col_active) {
  using R = typename CxBits<C>::R;
  const int64_t tile = COLX ? blockIdx.y : blockIdx.x;
  const int col = COLX ? blockIdx.x : blockIdx.y;
  if (col_active != nullptr && col_active[col] == 0) return;
  in += (int64_t)col * ldi;
  out += (int64_t)col * ldo;
  __shared__ R sacc[4][24][kWilsonSites + 1];
  const int64_t s0 = tile * kWilsonSites;
  dslash_tile<S>(op, in, s0, sacc);
  const R *ind = reinterpret_cast<const R *>(in);
  R *outd = reinterpret_cast<R *>(out);
  const R mk = (R)(-op.kappa);
  for (int o = threadIdx.x; o < kWilsonSites * 24; o += 128) {
    const int sl = o / 24, c = o - 24 * (o / 24);
    const int64_t ss = s0 + sl;
    if (ss >= op.sites) continue;
    const R sum = tile_hop_sum(sacc, c, sl);
    outd[24 * ss + c] = fma(mk, sum, __ldg(ind + 24 * ss + c));
  }
}

void launch_wilson_dslash(const WilsonOp &op, int sign, const double2 *in, int64_t ldi, double2 *out, int64_t ldo,
                          int ncols, const int32_t *col_active, cudaStream_t s) {
  if (ncols < 1) return;
  const int64_t tiles = (op.sites + kWilsonSites - 1) / kWilsonSites;
  if (tiles <= 65535) {
    const dim3 grid((unsigned)ncols, (unsigned)tiles);
    if (sign > 0) k_dslash<+1, true><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
    else k_dslash<-1, true><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
  } else {
    const dim3 grid((unsigned)tiles, (unsigned)ncols);
    if (sign > 0) k_dslash<+1, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
    else k_dslash<-1, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
  }
}

}  // namespace seedk
