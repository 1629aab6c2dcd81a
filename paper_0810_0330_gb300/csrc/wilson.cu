// wilson.cu -- Wilson-Dirac operator D and D^H on sm_103a (FP64 complex).
//
// Operator (Sec. 4 names the Wilson-Dirac matrix; the textbook form with
// r = 1 is used, gamma matrices in the DeGrand-Rossi basis):
//   (D_s psi)(n) = psi(n) - kappa sum_mu [ (1 - s g_mu) U_mu(n) psi(n+mu)
//                                         + (1 + s g_mu) U_mu(n-mu)^H psi(n-mu) ]
// with s = +1 for D and s = -1 for D^H = g5 D g5.
//
// Spin projection and the hop itself are in wilson_device.cuh: a hop
// multiplies only a two-spinor by the link, 84 FP64 operations instead of 264.
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


template <int S, class C>
__global__ void __launch_bounds__(128) k_dslash(WilsonOpT<C> op, const C *__restrict__ in, int64_t ldi,
                                                C *__restrict__ out, int64_t ldo,
                                                const int32_t *__restrict__ col_active) {
  using R = typename CxBits<C>::R;
  const int col = blockIdx.y;
  if (col_active != nullptr && col_active[col] == 0) return;
  in += (int64_t)col * ldi;
  out += (int64_t)col * ldo;
  __shared__ R sacc[4][24][kWilsonSites + 1];
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s0 = (int64_t)blockIdx.x * kWilsonSites;
  const int64_t s = s0 + lane;
  C acc[12];
  if (s < op.sites) {
    switch (mu) {
      case 0: site_mu<0, S>(op, in, s, acc); break;
      case 1: site_mu<1, S>(op, in, s, acc); break;
      case 2: site_mu<2, S>(op, in, s, acc); break;
      default: site_mu<3, S>(op, in, s, acc); break;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = C{0, 0};
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    sacc[mu][2 * k][lane] = acc[k].x;
    sacc[mu][2 * k + 1][lane] = acc[k].y;
  }
  __syncthreads();
  const R *ind = reinterpret_cast<const R *>(in);
  R *outd = reinterpret_cast<R *>(out);
  const R mk = (R)(-op.kappa);
  for (int o = threadIdx.x; o < kWilsonSites * 24; o += 128) {
    const int sl = o / 24, c = o - 24 * (o / 24);
    const int64_t ss = s0 + sl;
    if (ss >= op.sites) continue;
    const R sum = ((sacc[0][c][sl] + sacc[1][c][sl]) + sacc[2][c][sl]) + sacc[3][c][sl];
    outd[24 * ss + c] = fma(mk, sum, __ldg(ind + 24 * ss + c));
  }
}

void launch_wilson_dslash(const WilsonOp &op, int sign, const double2 *in, int64_t ldi, double2 *out, int64_t ldo,
                          int ncols, const int32_t *col_active, cudaStream_t s) {
  dim3 grid((unsigned)((op.sites + kWilsonSites - 1) / kWilsonSites), (unsigned)ncols);
  if (sign > 0) k_dslash<+1><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
  else k_dslash<-1><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active);
}

// ---------------------------------------------------------------------------
// FP32 operator of the mixed-precision path.  In FP32 the stencil is bound by
// memory traffic (1368 flop per 480 B per site and column against a balance
// point of ~11 flop/B), so this kernel is laid out for traffic instead:
//  * links are an FP32 copy in structure-of-arrays order, links[(mu*9 + k)*sites + s],
//    so a warp's 32 consecutive sites read 256 contiguous bytes per element;
//  * each thread keeps its two links (U_mu(s), U_mu(s - mu)) in registers and
//    applies them to every column of its block's column group, so the links
//    are read once per group instead of once per column;
//  * spinors are read as float4 (two complex numbers) when 16-byte aligned.
// Same thread layout and summation order as the FP64 kernel: warp mu does the
// two hops of direction mu for 32 sites; the partials meet in shared memory.
// ---------------------------------------------------------------------------
template <bool VEC>
SEED_DEV void load_spinor(const float2 *__restrict__ p, float2 (&ps)[12]) {
  if constexpr (VEC) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 v = __ldg(q + k);
      ps[2 * k] = make_float2(v.x, v.y);
      ps[2 * k + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k] = __ldg(p + k);
  }
}

template <int MU, int S, bool VEC>
SEED_DEV void hops32(const float2 *__restrict__ in, int32_t nf, int32_t nb, const float2 (&uf)[9],
                     const float2 (&ub)[9], unsigned negf, unsigned negb, float2 (&acc)[12]) {
  float2 ps[12];
  load_spinor<VEC>(in + 12 * (int64_t)nf, ps);
  hop_r<MU, S, true, true>(ps, uf, negf, acc);
  load_spinor<VEC>(in + 12 * (int64_t)nb, ps);
  hop_r<MU, -S, false, false>(ps, ub, negb, acc);
}

template <int S, bool VEC>
__global__ void __launch_bounds__(128) k_dslash32(WilsonOp32 op, const float2 *__restrict__ in, int64_t ldi,
                                                  float2 *__restrict__ out, int64_t ldo,
                                                  const int32_t *__restrict__ col_active, int ncols, int group) {
  __shared__ float sacc[4][24][kWilsonSites + 1];
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s0 = (int64_t)blockIdx.x * kWilsonSites;
  const int64_t s = s0 + lane;
  const bool valid = s < op.sites;
  const int c_begin = blockIdx.y * group;
  const int c_end = min(ncols, c_begin + group);
  int32_t nf = 0, nb = 0;
  unsigned negf = 0u, negb = 0u;
  float2 uf[9], ub[9];
  if (valid) {
    nf = __ldg(op.nbr + 8 * s + 2 * mu);
    nb = __ldg(op.nbr + 8 * s + 2 * mu + 1);
    if (mu == 3 && op.bc_t) {
      const int64_t t = s / ((int64_t)op.dims[0] * op.dims[1] * op.dims[2]);
      if (t == op.dims[3] - 1) negf = CxBits<float2>::sign;
      if (t == 0) negb = CxBits<float2>::sign;
    }
    const float2 *L = op.links + (int64_t)mu * 9 * op.sites;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      uf[k] = __ldg(L + (int64_t)k * op.sites + s);
      ub[k] = __ldg(L + (int64_t)k * op.sites + nb);
    }
  }
  const float mk = (float)(-op.kappa);
  for (int c = c_begin; c < c_end; ++c) {
    if (col_active != nullptr && col_active[c] == 0) continue;   // uniform over the block
    const float2 *inc = in + (int64_t)c * ldi;
    float2 acc[12];
    if (valid) {
      switch (mu) {
        case 0: hops32<0, S, VEC>(inc, nf, nb, uf, ub, negf, negb, acc); break;
        case 1: hops32<1, S, VEC>(inc, nf, nb, uf, ub, negf, negb, acc); break;
        case 2: hops32<2, S, VEC>(inc, nf, nb, uf, ub, negf, negb, acc); break;
        default: hops32<3, S, VEC>(inc, nf, nb, uf, ub, negf, negb, acc); break;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      sacc[mu][2 * k][lane] = acc[k].x;
      sacc[mu][2 * k + 1][lane] = acc[k].y;
    }
    __syncthreads();
    const float *ind = reinterpret_cast<const float *>(inc);
    float *outd = reinterpret_cast<float *>(out + (int64_t)c * ldo);
    for (int o = threadIdx.x; o < kWilsonSites * 24; o += 128) {
      const int sl = o / 24, cc = o - 24 * (o / 24);
      const int64_t ss = s0 + sl;
      if (ss >= op.sites) continue;
      const float sum = ((sacc[0][cc][sl] + sacc[1][cc][sl]) + sacc[2][cc][sl]) + sacc[3][cc][sl];
      outd[24 * ss + cc] = fmaf(mk, sum, __ldg(ind + 24 * ss + cc));
    }
    __syncthreads();
  }
}

// links (caller's layout [mu][site][3][3], FP64) -> FP32 structure-of-arrays copy
__global__ void k_links_soa32(const double2 *__restrict__ links, float2 *__restrict__ out, int64_t sites) {
  const int64_t total = 36 * sites;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = o % sites, mk = o / sites, mu = mk / 9, k = mk - 9 * mu;
    const double2 v = links[(mu * sites + s) * 9 + k];
    out[o] = make_float2((float)v.x, (float)v.y);
  }
}

void launch_links_soa32(const double2 *links, float2 *out, int64_t sites, cudaStream_t s) {
  int64_t blocks = (36 * sites + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_links_soa32<<<(unsigned)blocks, 256, 0, s>>>(links, out, sites);
}

// Column groups: enough blocks to give every SM about four, otherwise all
// columns of a site block in one group (links read once).
void launch_wilson_dslash32(const WilsonOp32 &op, int sign, const float2 *in, int64_t ldi, float2 *out, int64_t ldo,
                            int ncols, const int32_t *col_active, cudaStream_t s) {
  const int64_t nsb = (op.sites + kWilsonSites - 1) / kWilsonSites;
  int64_t group = (nsb * ncols) / (152 * 4);
  if (group < 1) group = 1;
  if (group > ncols) group = ncols;
  const int ngroups = (int)((ncols + group - 1) / group);
  const dim3 grid((unsigned)nsb, (unsigned)ngroups);
  const bool vec = ((uintptr_t)in % 16 == 0) && (ldi % 2 == 0);
  const int g = (int)group;
  if (sign > 0) {
    if (vec) k_dslash32<+1, true><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
    else k_dslash32<+1, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
  } else {
    if (vec) k_dslash32<-1, true><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
    else k_dslash32<-1, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
  }
}

int wilson_kernels_per_apply() { return 2; }

}  // namespace seedk
