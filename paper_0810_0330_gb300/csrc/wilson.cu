// wilson.cu -- Wilson-Dirac operator D and D^H on sm_103a (FP64 complex).
//
// Operator (Sec. 4 names the Wilson-Dirac matrix; the textbook form with
// r = 1 is used, gamma matrices in the DeGrand-Rossi basis):
//   (D_s psi)(n) = psi(n) - kappa sum_mu [ (1 - s g_mu) U_mu(n) psi(n+mu)
//                                         + (1 + s g_mu) U_mu(n-mu)^H psi(n-mu) ]
// with s = +1 for D and s = -1 for D^H = g5 D g5.
//
// In the chiral basis g_mu = [[0, B_mu], [B_mu^H, 0]] with 2x2 blocks whose
// rows each hold one entry from {1, i, -1, -i}.  Hence (1 - s g_mu) psi has
// upper half h = psi_up - s B_mu psi_dn and lower half -s B_mu^H h: a hop
// multiplies only the two-spinor h by the link (spin projection), 84 FP64
// operations per hop instead of 264.
//
// GB300 runs FP64 at 1/64 of its FP32 rate (about 1.2 TFLOP/s measured), so
// this kernel is bound by the FP64 pipe, not by HBM: the design minimises FP64
// instructions.  Phase factors and boundary signs are register swaps and
// sign-bit flips (integer ops).  Thread layout: a block of 128 threads covers
// 32 sites; warp mu handles direction mu (forward and backward hop) for all 32
// sites, so every warp runs one uniform code path.  The four per-direction
// partial sums meet in shared memory, then each output is psi - kappa * sum.
#include "device_common.cuh"
#include "seed_internal.h"

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

// ---------------------------------------------------------------------------
// phases: code 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
// ---------------------------------------------------------------------------
template <int C> SEED_DEV double2 ph_add(double2 z, double2 w) {   // z + phase(C) w
  if constexpr (C == 0) return c2(z.x + w.x, z.y + w.y);
  else if constexpr (C == 1) return c2(z.x - w.y, z.y + w.x);
  else if constexpr (C == 2) return c2(z.x - w.x, z.y - w.y);
  else return c2(z.x + w.y, z.y - w.x);
}
constexpr unsigned long long kSign = 0x8000000000000000ull;
template <int C> SEED_DEV double2 ph_mul(double2 w) {              // phase(C) w, no FP64 op
  if constexpr (C == 0) return w;
  else if constexpr (C == 1) return c2(xsign(w.y, kSign), w.x);
  else if constexpr (C == 2) return c2(xsign(w.x, kSign), xsign(w.y, kSign));
  else return c2(w.y, xsign(w.x, kSign));
}
__host__ __device__ constexpr int ph_neg(int c) { return (c + 2) & 3; }
__host__ __device__ constexpr int ph_conj(int c) { return (4 - c) & 3; }

// B_mu row k has its one nonzero in column J(mu,k) with phase P(mu,k):
//   B_x = [[0, i], [i, 0]], B_y = [[0, -1], [1, 0]], B_z = [[i, 0], [0, -i]], B_t = 1
__host__ __device__ constexpr int bJ(int mu, int k) { return (mu <= 1) ? 1 - k : k; }
__host__ __device__ constexpr int bP(int mu, int k) {
  return mu == 0 ? 1 : mu == 1 ? (k == 0 ? 2 : 0) : mu == 2 ? (k == 0 ? 1 : 3) : 0;
}

// One hop of (1 - S g_MU) M psi(nb) into acc[spin*3 + colour];  M = U (FWD) or
// U^H.  FIRST: acc is overwritten instead of accumulated.  neg: boundary sign.
template <int MU, int S, bool FWD, bool FIRST>
SEED_DEV void hop(const double2 *__restrict__ psi, const double2 *__restrict__ U, unsigned long long neg,
                  double2 (&acc)[12]) {
  // h_k = psi_k - S * P(k) psi_{2+J(k)}
  constexpr int c0 = S > 0 ? ph_neg(bP(MU, 0)) : bP(MU, 0);
  constexpr int c1 = S > 0 ? ph_neg(bP(MU, 1)) : bP(MU, 1);
  double2 h0[3], h1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double2 p0 = __ldg(psi + a), p1 = __ldg(psi + 3 + a);
    double2 q0 = __ldg(psi + 3 * (2 + bJ(MU, 0)) + a), q1 = __ldg(psi + 3 * (2 + bJ(MU, 1)) + a);
    h0[a] = ph_add<c0>(p0, q0);
    h1[a] = ph_add<c1>(p1, q1);
    h0[a].x = xsign(h0[a].x, neg); h0[a].y = xsign(h0[a].y, neg);
    h1[a].x = xsign(h1[a].x, neg); h1[a].y = xsign(h1[a].y, neg);
  }
  double2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = __ldg(U + k);
  // chi_k = M h_k
  double2 x0[3], x1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if constexpr (FWD) {
      x0[a] = cmul(u[3 * a], h0[0]);
      x1[a] = cmul(u[3 * a], h1[0]);
      x0[a] = cfma(u[3 * a + 1], h0[1], x0[a]);
      x1[a] = cfma(u[3 * a + 1], h1[1], x1[a]);
      x0[a] = cfma(u[3 * a + 2], h0[2], x0[a]);
      x1[a] = cfma(u[3 * a + 2], h1[2], x1[a]);
    } else {
      double2 uc = c2(u[a].x, xsign(u[a].y, kSign));
      x0[a] = cmul(uc, h0[0]);
      x1[a] = cmul(uc, h1[0]);
      x0[a] = cfmac(u[3 + a], h0[1], x0[a]);
      x1[a] = cfmac(u[3 + a], h1[1], x1[a]);
      x0[a] = cfmac(u[6 + a], h0[2], x0[a]);
      x1[a] = cfmac(u[6 + a], h1[2], x1[a]);
    }
  }
  // upper spins get chi; lower spin 2+J(k) gets -S conj(P(k)) chi_k
  constexpr int l0 = S > 0 ? ph_neg(ph_conj(bP(MU, 0))) : ph_conj(bP(MU, 0));
  constexpr int l1 = S > 0 ? ph_neg(ph_conj(bP(MU, 1))) : ph_conj(bP(MU, 1));
  constexpr int s0 = 2 + bJ(MU, 0), s1 = 2 + bJ(MU, 1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if constexpr (FIRST) {
      acc[a] = x0[a];
      acc[3 + a] = x1[a];
      acc[3 * s0 + a] = ph_mul<l0>(x0[a]);
      acc[3 * s1 + a] = ph_mul<l1>(x1[a]);
    } else {
      acc[a] = cadd(acc[a], x0[a]);
      acc[3 + a] = cadd(acc[3 + a], x1[a]);
      acc[3 * s0 + a] = ph_add<l0>(acc[3 * s0 + a], x0[a]);
      acc[3 * s1 + a] = ph_add<l1>(acc[3 * s1 + a], x1[a]);
    }
  }
}

template <int MU, int S>
SEED_DEV void site_mu(const WilsonOp &op, const double2 *__restrict__ in, int64_t s, double2 (&acc)[12]) {
  const int32_t nf = __ldg(op.nbr + 8 * s + 2 * MU);
  const int32_t nb = __ldg(op.nbr + 8 * s + 2 * MU + 1);
  unsigned long long negf = 0ull, negb = 0ull;
  if (MU == 3 && op.bc_t) {
    const int64_t slab = (int64_t)op.dims[0] * op.dims[1] * op.dims[2];
    const int64_t t = s / slab;
    if (t == op.dims[3] - 1) negf = kSign;
    if (t == 0) negb = kSign;
  }
  // forward: (1 - S g) U_mu(s) psi(s + mu); backward: (1 + S g) U_mu(s - mu)^H psi(s - mu)
  hop<MU, S, true, true>(in + 12 * (int64_t)nf, op.links + ((int64_t)MU * op.sites + s) * 9, negf, acc);
  hop<MU, -S, false, false>(in + 12 * (int64_t)nb, op.links + ((int64_t)MU * op.sites + nb) * 9, negb, acc);
}

constexpr int kWilsonSites = 32;   // sites per block; 4 warps (one per mu)

template <int S>
__global__ void __launch_bounds__(128) k_dslash(WilsonOp op, const double2 *__restrict__ in, int64_t ldi,
                                                double2 *__restrict__ out, int64_t ldo,
                                                const int32_t *__restrict__ col_active) {
  const int col = blockIdx.y;
  if (col_active != nullptr && col_active[col] == 0) return;
  in += (int64_t)col * ldi;
  out += (int64_t)col * ldo;
  __shared__ double sacc[4][24][kWilsonSites + 1];
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s0 = (int64_t)blockIdx.x * kWilsonSites;
  const int64_t s = s0 + lane;
  double2 acc[12];
  if (s < op.sites) {
    switch (mu) {
      case 0: site_mu<0, S>(op, in, s, acc); break;
      case 1: site_mu<1, S>(op, in, s, acc); break;
      case 2: site_mu<2, S>(op, in, s, acc); break;
      default: site_mu<3, S>(op, in, s, acc); break;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = c2(0.0, 0.0);
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    sacc[mu][2 * k][lane] = acc[k].x;
    sacc[mu][2 * k + 1][lane] = acc[k].y;
  }
  __syncthreads();
  const double *ind = reinterpret_cast<const double *>(in);
  double *outd = reinterpret_cast<double *>(out);
  for (int o = threadIdx.x; o < kWilsonSites * 24; o += 128) {
    const int sl = o / 24, c = o - 24 * (o / 24);
    const int64_t ss = s0 + sl;
    if (ss >= op.sites) continue;
    const double sum = ((sacc[0][c][sl] + sacc[1][c][sl]) + sacc[2][c][sl]) + sacc[3][c][sl];
    outd[24 * ss + c] = fma(-op.kappa, sum, __ldg(ind + 24 * ss + c));
  }
}

void launch_wilson_dslash(const WilsonOp &op, int sign, const double2 *in, int64_t ldi, double2 *out, int64_t ldo,
                          int ncols, const int32_t *col_active, cudaStream_t s) {
  dim3 grid((unsigned)((op.sites + kWilsonSites - 1) / kWilsonSites), (unsigned)ncols);
  if (sign > 0) k_dslash<+1><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
  else k_dslash<-1><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
}

int wilson_kernels_per_apply() { return 2; }

}  // namespace seedk
