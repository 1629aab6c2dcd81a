// related.cu -- Sec. 2.3 (single seeding for related right-hand sides), the projection
// on sm_103a: after system j is solved, the remaining systems receive the
// Galerkin projection over the correction x_cg = x^j - x^j_bcg that CG found
// for system j:
//   delta_i = (x_cg^H r^i) / (x_cg^H r^j_bcg),
//   x^i += delta_i x_cg,   r^i -= delta_i r^j_bcg   for every remaining i.
// (r^j_bcg, the residual of system j before its CG, stands for A x_cg: the
// two differ by the final residual of system j, which CG has made small.)
// Reductions are deterministic: block partials summed in block order.
//
// The same two kernels give multiple seeding (the comparison method of Sec.
// 2.1): there every CG step of the current system projects each later system
// over its direction, with (p, q = A p) in place of (x_cg, r^j_bcg).  `gate`
// (NULL = always) is that CG's active flag, so steps issued after it has
// converged change nothing.
#include "seed_device.cuh"

namespace seedk {

constexpr int NT = kVecThreads;

#define GRID_STRIDE(e, n) \
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < (n); e += (int64_t)gridDim.x * NT)

int col_blocks(int64_t n, int nc);

// dots[c] = x_cg^H R[:, c] for c < nrem, dots[nrem] = x_cg^H r_bcg  (grid (blocks, nrem + 1))
template <class T>
__global__ void __launch_bounds__(NT) k_rel_dots(int64_t n, const T *__restrict__ xcg, const T *__restrict__ rbcg,
                                                 const T *__restrict__ R, int64_t ldr, int nrem, double2 *dots,
                                                 double *partials, unsigned *tickets, const int32_t *gate) {
  __shared__ double sm[2 * NT / 32];
  if (gate != nullptr && gate[0] == 0) return;
  const int col = blockIdx.y;
  const T *y = col < nrem ? R + (int64_t)col * ldr : rbcg;
  typename Sc<T>::A2 acc = Sc<T>::zero2();
  GRID_STRIDE(e, n) acc = Sc<T>::dotc(xcg[e], y[e], acc);
  double v[2] = {(double)acc.x, (double)acc.y};
  block_sum<2, NT>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x * 2;
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2] = v[0];
    part[blockIdx.x * 2 + 1] = v[1];
  }
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double re = sum_partials<NT>(part, gridDim.x, 2, 0, sm);
  const double im = sum_partials<NT>(part, gridDim.x, 2, 1, sm);
  if (threadIdx.x == 0) dots[col] = c2(re, im);
}

// delta_c = dots[c] / dots[nrem] (complex division), one thread per column
__global__ void k_rel_delta(int nrem, const double2 *dots, double2 *delta, const int32_t *gate) {
  const int c = threadIdx.x;
  if (c >= nrem || (gate != nullptr && gate[0] == 0)) return;
  const double2 a = dots[c], b = dots[nrem];
  const double d = b.x * b.x + b.y * b.y;
  delta[c] = d > 0.0 ? c2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d) : c2(0.0, 0.0);
}

// X[:, c] += delta_c x_cg;  R[:, c] -= delta_c r_bcg   (grid (blocks, nrem))
template <class T>
__global__ void __launch_bounds__(NT) k_rel_update(int64_t n, const T *__restrict__ xcg, const T *__restrict__ rbcg,
                                                   T *X, int64_t ldx, T *R, int64_t ldr, const double2 *delta,
                                                   const int32_t *gate) {
  if (gate != nullptr && gate[0] == 0) return;
  const int col = blockIdx.y;
  const double2 d = delta[col], md = c2(-d.x, -d.y);
  X += (int64_t)col * ldx;
  R += (int64_t)col * ldr;
  GRID_STRIDE(e, n) {
    X[e] = Sc<T>::caxpy(d, xcg[e], X[e]);
    R[e] = Sc<T>::caxpy(md, rbcg[e], R[e]);
  }
}

template <class T>
void launch_related_project(int64_t n, const T *xcg, const T *rbcg, T *X, int64_t ldx, T *R, int64_t ldr, int nrem,
                            double2 *dots, double2 *delta, double *partials, unsigned *tickets, cudaStream_t s,
                            const int32_t *gate) {
  if (nrem <= 0) return;
  const int b = col_blocks(n, nrem + 1);
  k_rel_dots<T><<<dim3((unsigned)b, (unsigned)(nrem + 1)), NT, 0, s>>>(n, xcg, rbcg, R, ldr, nrem, dots, partials,
                                                                       tickets, gate);
  k_rel_delta<<<1, kMaxRhs, 0, s>>>(nrem, dots, delta, gate);
  const int b2 = col_blocks(n, nrem);
  k_rel_update<T><<<dim3((unsigned)b2, (unsigned)nrem), NT, 0, s>>>(n, xcg, rbcg, X, ldx, R, ldr, delta, gate);
}

template void launch_related_project<double>(int64_t, const double *, const double *, double *, int64_t, double *,
                                             int64_t, int, double2 *, double2 *, double *, unsigned *, cudaStream_t,
                                             const int32_t *);
template void launch_related_project<double2>(int64_t, const double2 *, const double2 *, double2 *, int64_t,
                                              double2 *, int64_t, int, double2 *, double2 *, double *, unsigned *,
                                              cudaStream_t, const int32_t *);

}  // namespace seedk
