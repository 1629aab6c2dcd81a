// mixed.cu -- kernels of the mixed-precision path (FP32 operator applies and
// Krylov vectors, FP64 scalars, reductions and reliable updates).
//
// The FP32 iterations themselves reuse the Krylov kernels instantiated on
// float / float2 (krylov.cu).  What is specific to mixed precision lives
// here: rounding FP64 data to FP32, folding the FP32 correction into the FP64
// solution, and the reliable update of lockstep CG -- every few iterations a
// column whose FP32 recursive residual has fallen far enough (or has met the
// tolerance) gets x += e (FP64), r = b - A x with the FP64 operator, and
// continues from the FP32 rounding of that true residual.  This is the
// residual-replacement strategy of Sleijpen and van der Vorst (reliable
// updates), used in mixed-precision lattice solvers since Clark et al. (2010).
#include "seed_device.cuh"

namespace seedk {

constexpr int NT = kVecThreads;

#define GRID_STRIDE(e, n) \
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < (n); e += (int64_t)gridDim.x * NT)

int col_blocks(int64_t n, int nc);

SEED_DEV float lo(double x) { return (float)x; }
SEED_DEV float2 lo(double2 x) { return make_float2((float)x.x, (float)x.y); }
SEED_DEV double hi(float x) { return (double)x; }
SEED_DEV double2 hi(float2 x) { return make_double2((double)x.x, (double)x.y); }

// In every kernel below t runs over the FP32 vector (length n32, Layout32 L)
// and e = L.to_user(t) is the caller's element (-1: padding, kept zero).

// dst = FP32 rounding of src (grid.y columns; also used once for the CSR values)
template <class T64, class T32>
__global__ void __launch_bounds__(NT) k_to_low(const T64 *src, int64_t lds, T32 *dst, int64_t ldd, int64_t n32,
                                               Layout32 L) {
  src += (int64_t)blockIdx.y * lds;
  dst += (int64_t)blockIdx.y * ldd;
  GRID_STRIDE(t, n32) {
    const int64_t e = L.to_user(t);
    dst[t] = e >= 0 ? lo(src[e]) : Sc<T32>::zero();
  }
}

// X += E (FP64 += FP32), then E = 0; mask: only columns whose flag is set (NULL: all)
template <class T64, class T32>
__global__ void __launch_bounds__(NT) k_fold(T64 *X, int64_t ldx, T32 *E, int64_t lde, int64_t n32, Layout32 L,
                                             const int32_t *mask) {
  const int col = blockIdx.y;
  if (mask != nullptr && mask[col] == 0) return;
  X += (int64_t)col * ldx;
  E += (int64_t)col * lde;
  GRID_STRIDE(t, n32) {
    const int64_t e = L.to_user(t);
    if (e >= 0) X[e] = Sc<T64>::add(X[e], hi(E[t]));
    E[t] = Sc<T32>::zero();
  }
}

// Start of mixed CG on nc columns: r = b - q (q = A x in FP64), R32 = lo(r),
// P32 = R32, E = 0; rho = ||r||^2, ||b||; a column already within tol is done.
template <class T64, class T32>
__global__ void __launch_bounds__(NT) k_mixed_init(int64_t n32, Layout32 L, const T64 *B, int64_t ldb, const T64 *Q,
                                                   int64_t ldq, T32 *R, T32 *P, T32 *E, int64_t ld, CgCols c,
                                                   double *partials, unsigned *tickets) {
  __shared__ double sm[2 * NT / 32];
  const int col = blockIdx.y;
  B += (int64_t)col * ldb;
  Q += (int64_t)col * ldq;
  R += (int64_t)col * ld;
  P += (int64_t)col * ld;
  E += (int64_t)col * ld;
  double rr = 0.0, bb = 0.0;
  GRID_STRIDE(t, n32) {
    const int64_t e = L.to_user(t);
    const T64 bv = e >= 0 ? B[e] : Sc<T64>::zero();
    const T64 r = e >= 0 ? Sc<T64>::sub(bv, Q[e]) : Sc<T64>::zero();
    const T32 r32 = lo(r);
    R[t] = r32;
    P[t] = r32;
    E[t] = Sc<T32>::zero();
    rr = Sc<T64>::nrm2(r, rr);
    bb = Sc<T64>::nrm2(bv, bb);
  }
  double v[2] = {rr, bb};
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
    c.rupd[col] = c.relres[col];
    c.mvps[col] = 1;
    c.iters[col] = 0;
    c.restarts[col] = 0;
    c.needs_check[col] = 0;
    c.upd[col] = 0;
    const int done = rn <= c.tol * bn;
    c.active[col] = !done;
    c.reached[col] = done;
    c.converged[col] = done;
  }
}

// Which columns take a reliable update now: those that stopped (tolerance met
// by the FP32 recursion, or iteration cap) and those whose recursive residual
// fell below delta times its value at the last update.  One thread per column.
__global__ void k_mixed_flag(CgCols c) {
  const int col = threadIdx.x;
  if (col >= c.nc) return;
  int u = 0;
  if (!c.converged[col]) {
    if (c.needs_check[col]) u = 1;
    else if (c.active[col] && c.relres[col] < c.delta * c.rupd[col]) u = 1;
  }
  c.upd[col] = u;
}

// Reliable update, second half (after X += E and Q = A X in FP64 for the
// flagged columns): r = b - q, R32 = lo(r), rho = ||r||^2.  Columns that had
// stopped restart with p = r; the others keep p.  Converged when the FP64
// true residual meets tol.
template <class T64, class T32>
__global__ void __launch_bounds__(NT) k_mixed_residual(int64_t n32, Layout32 L, const T64 *B, int64_t ldb,
                                                       const T64 *Q, int64_t ldq, T32 *R, T32 *P, int64_t ld,
                                                       CgCols c, double *partials, unsigned *tickets) {
  __shared__ double sm[NT / 32];
  const int col = blockIdx.y;
  if (!c.upd[col]) return;
  const bool restart = c.needs_check[col] != 0;
  B += (int64_t)col * ldb;
  Q += (int64_t)col * ldq;
  R += (int64_t)col * ld;
  P += (int64_t)col * ld;
  double rr = 0.0;
  GRID_STRIDE(t, n32) {
    const int64_t e = L.to_user(t);
    const T64 r = e >= 0 ? Sc<T64>::sub(B[e], Q[e]) : Sc<T64>::zero();
    const T32 r32 = lo(r);
    R[t] = r32;
    if (restart) P[t] = r32;
    rr = Sc<T64>::nrm2(r, rr);
  }
  double v[1] = {rr};
  block_sum<1, NT>(v, sm);
  double *part = partials + (int64_t)col * gridDim.x;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (!last_block_done(tickets + kColTicket + col, gridDim.x)) return;
  const double s = sum_partials<NT>(part, gridDim.x, 1, 0, sm);
  if (threadIdx.x == 0) {
    const double rn = sqrt(s), bn = c.bnorm[col];
    const double rel = bn > 0.0 ? rn / bn : 0.0;
    c.relres[col] = rel;
    c.rupd[col] = rel;
    c.mvps[col] += 1;
    c.restarts[col] += 1;
    c.needs_check[col] = 0;
    c.upd[col] = 0;
    c.rho[col] = s;
    if (rn <= c.tol * bn) {
      c.converged[col] = 1;
      c.reached[col] = 1;
      c.active[col] = 0;
    } else if (c.iters[col] >= c.maxit || !isfinite(s)) {   // non-finite: ends unconverged
      c.active[col] = 0;
    } else {
      c.active[col] = 1;
      c.reached[col] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class T64, class T32>
void launch_to_low(const T64 *src, int64_t lds, T32 *dst, int64_t ldd, int64_t n32, Layout32 L, int ncols,
                   cudaStream_t s) {
  int64_t b = (n32 + NT * 4 - 1) / (NT * 4);
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  k_to_low<T64, T32><<<dim3((unsigned)b, (unsigned)ncols), NT, 0, s>>>(src, lds, dst, ldd, n32, L);
}
template <class T64, class T32>
void launch_fold(T64 *X, int64_t ldx, T32 *E, int64_t lde, int64_t n32, Layout32 L, int ncols, const int32_t *mask,
                 cudaStream_t s) {
  k_fold<T64, T32><<<dim3((unsigned)col_blocks(n32, ncols), (unsigned)ncols), NT, 0, s>>>(X, ldx, E, lde, n32, L,
                                                                                         mask);
}
template <class T64, class T32>
void launch_mixed_init(int64_t n32, Layout32 L, const T64 *B, int64_t ldb, const T64 *Q, int64_t ldq, T32 *R, T32 *P,
                       T32 *E, int64_t ld, const CgCols &c, double *partials, unsigned *tickets, cudaStream_t s) {
  k_mixed_init<T64, T32><<<dim3((unsigned)col_blocks(n32, c.nc), (unsigned)c.nc), NT, 0, s>>>(
      n32, L, B, ldb, Q, ldq, R, P, E, ld, c, partials, tickets);
}
void launch_mixed_flag(const CgCols &c, cudaStream_t s) { k_mixed_flag<<<1, kMaxRhs, 0, s>>>(c); }
template <class T64, class T32>
void launch_mixed_residual(int64_t n32, Layout32 L, const T64 *B, int64_t ldb, const T64 *Q, int64_t ldq, T32 *R,
                           T32 *P, int64_t ld, const CgCols &c, double *partials, unsigned *tickets, cudaStream_t s) {
  k_mixed_residual<T64, T32><<<dim3((unsigned)col_blocks(n32, c.nc), (unsigned)c.nc), NT, 0, s>>>(
      n32, L, B, ldb, Q, ldq, R, P, ld, c, partials, tickets);
}

#define MIXED_INSTANTIATE(T64, T32)                                                                              \
  template void launch_to_low<T64, T32>(const T64 *, int64_t, T32 *, int64_t, int64_t, Layout32, int,           \
                                        cudaStream_t);                                                           \
  template void launch_fold<T64, T32>(T64 *, int64_t, T32 *, int64_t, int64_t, Layout32, int, const int32_t *,   \
                                      cudaStream_t);                                                             \
  template void launch_mixed_init<T64, T32>(int64_t, Layout32, const T64 *, int64_t, const T64 *, int64_t, T32 *, \
                                            T32 *, T32 *, int64_t, const CgCols &, double *, unsigned *,        \
                                            cudaStream_t);                                                       \
  template void launch_mixed_residual<T64, T32>(int64_t, Layout32, const T64 *, int64_t, const T64 *, int64_t,    \
                                                T32 *, T32 *, int64_t, const CgCols &, double *, unsigned *,     \
                                                cudaStream_t);

MIXED_INSTANTIATE(double, float)
MIXED_INSTANTIATE(double2, float2)

}  // namespace seedk
