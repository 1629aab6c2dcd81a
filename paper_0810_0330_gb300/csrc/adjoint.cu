// adjoint.cu -- the kappa derivative of the Wilson normal operator, for the
// adjoint (backward) pass of a solve x = A^{-1} b with A = D^H D:
//
//   out_j = Re <lambda_j, (dA/dkappa) x_j>.
//
// D = 1 - kappa H (H the hopping term of D), so dD/dkappa = -H and
//   dA/dkappa = -(H^H D + D^H H),   Re<l, dA x> = -Re(<H l, D x> + <D l, H x>),
// and D v = v - kappa H v: one hopping sum per vector gives both H v and D v.
// One kernel computes, site by site, the hopping sums of lambda_j and x_j with
// the operator's own hop code (wilson_device.cuh, the S = +1 hop of D), and
// reduces the real inner products (the real part of a complex inner product
// is the dot product of the interleaved real components) in a fixed order.
// The kernel is bound by the FP64 pipe like the operator itself (two hopping
// sums per site and column).
#include "wilson_device.cuh"

namespace seedk {

constexpr int kAdjThreads = 128;   // 4 warps (one per mu) x 32 sites, as the operator kernel

// grid (blocks, ncols); block b of column j handles site tiles b, b + gridDim.x, ...
__global__ void __launch_bounds__(kAdjThreads) k_dkappa_inner(WilsonOp op, const double2 *__restrict__ L, int64_t ldl,
                                                              const double2 *__restrict__ X, int64_t ldx,
                                                              double *partials, unsigned *tickets, double *out) {
  __shared__ double sacc[4][24][kWilsonSites + 1];
  __shared__ double sm[kAdjThreads / 32];
  const int col = blockIdx.y;
  L += (int64_t)col * ldl;
  X += (int64_t)col * ldx;
  const double *Ld = reinterpret_cast<const double *>(L);
  const double *Xd = reinterpret_cast<const double *>(X);
  const int64_t ntiles = (op.sites + kWilsonSites - 1) / kWilsonSites;
  constexpr int kPer = kWilsonSites * 24 / kAdjThreads;   // real components per thread and tile
  double val = 0.0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t s0 = tile * kWilsonSites;
    double hl[kPer];
    dslash_tile<+1>(op, L, s0, sacc);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int o = threadIdx.x + q * kAdjThreads, sl = o / 24, c = o - 24 * (o / 24);
      hl[q] = tile_hop_sum(sacc, c, sl);
    }
    __syncthreads();
    dslash_tile<+1>(op, X, s0, sacc);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int o = threadIdx.x + q * kAdjThreads, sl = o / 24, c = o - 24 * (o / 24);
      const int64_t ss = s0 + sl;
      if (ss < op.sites) {
        const double hx = tile_hop_sum(sacc, c, sl);
        const double l = __ldg(Ld + 24 * ss + c), x = __ldg(Xd + 24 * ss + c);
        const double dl = fma(-op.kappa, hl[q], l), dx = fma(-op.kappa, hx, x);
        val = fma(hl[q], dx, val);
        val = fma(dl, hx, val);
      }
    }
    __syncthreads();
  }
  double v[1] = {val};
  block_sum<1, kAdjThreads>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double t = sum_partials<kAdjThreads>(part, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) out[col] = -t;
}

void launch_dkappa_inner(const WilsonOp &op, const double2 *L, int64_t ldl, const double2 *X, int64_t ldx, int ncols,
                         double *partials, unsigned *tickets, double *out, cudaStream_t s) {
  const int64_t ntiles = (op.sites + kWilsonSites - 1) / kWilsonSites;
  int64_t b = 1520 / (ncols > 0 ? ncols : 1);
  if (b > ntiles) b = ntiles;
  if (b < 1) b = 1;
  k_dkappa_inner<<<dim3((unsigned)b, (unsigned)ncols), kAdjThreads, 0, s>>>(op, L, ldl, X, ldx, partials, tickets,
                                                                            out);
}

}  // namespace seedk
