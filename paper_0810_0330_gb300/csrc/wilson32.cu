// wilson32.cu -- the FP32 copy of the Wilson-Dirac operator used by the
// mixed-precision path (seed_params.precision = 1) on sm_103a.
//
// Same operator, spin projection and summation order as the FP64 kernel in
// wilson.cu (the hop itself is shared, wilson_device.cuh), but laid out for
// memory traffic instead of FP64 issue.
#include <stdint.h>

#include "wilson_device.cuh"

namespace seedk {

// ---------------------------------------------------------------------------
// FP32 operator of the mixed-precision path.  In FP32 the stencil is bound by
// memory traffic (1368 flop per 480 B per site and column against a balance
// point of ~11 flop/B), so this kernel is laid out for traffic instead:
//  * links are an FP32 copy in structure-of-arrays order, links[(mu*9 + k)*sites + s],
//    so a warp's 32 consecutive sites read 256 contiguous bytes per element;
//  * each thread keeps its two links (U_mu(s), U_mu(s - mu)) in registers and
//    applies them to every column of its block's column group, so the links
//    are read once per group instead of once per column;
//  * inside the solver the FP32 spinors are tiled by 32 sites (Layout32:
//    component k of site s at ((s/32)*12 + k)*32 + s%32), so the 32 lanes of a
//    warp read each component of their 32 neighbours as one or two 256-byte
//    segments; on the caller's site-major layout (seed_apply) spinors are read
//    as float4 (two complex numbers) when 16-byte aligned.
// Same thread layout and summation order as the FP64 kernel: warp mu does the
// two hops of direction mu for 32 sites; the partials meet in shared memory.
// ---------------------------------------------------------------------------
// Read-only loads; L2ONLY loads skip L1 (ld.global.cg) for data no other
// thread of the SM is likely to want soon.
template <bool L2ONLY, class V>
SEED_DEV V ldro(const V *p) {
  if constexpr (L2ONLY) return __ldcg(p);
  else return __ldg(p);
}

template <bool VEC, bool L2ONLY = false>
SEED_DEV void load_spinor(const float2 *__restrict__ p, float2 (&ps)[12]) {
  if constexpr (VEC) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 v = ldro<L2ONLY>(q + k);
      ps[2 * k] = make_float2(v.x, v.y);
      ps[2 * k + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k] = ldro<L2ONLY>(p + k);
  }
}

// spinor of site q, tiled layout: 12 components 32 complex apart
template <bool L2ONLY = false>
SEED_DEV void load_spinor_tiled(const float2 *__restrict__ in, int64_t q, float2 (&ps)[12]) {
  const float2 *p = in + (q >> 5) * 384 + (q & 31);
#pragma unroll
  for (int k = 0; k < 12; ++k) ps[k] = ldro<L2ONLY>(p + 32 * k);
}

template <int MU, int S, bool VEC, bool TILED>
SEED_DEV void hops32(const float2 *__restrict__ in, int32_t nf, int32_t nb, const float2 (&uf)[9],
                     const float2 (&ub)[9], unsigned negf, unsigned negb, float2 (&acc)[12]) {
  float2 pf[12], pb[12];
  if constexpr (TILED) {
    load_spinor_tiled(in, nf, pf);
    load_spinor_tiled(in, nb, pb);
  } else {
    load_spinor<VEC>(in + 12 * (int64_t)nf, pf);
    load_spinor<VEC>(in + 12 * (int64_t)nb, pb);
  }
  hop_pair_r<MU, S>(pf, uf, negf, pb, ub, negb, acc);
}

template <int S, bool VEC, bool TILED>
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
        case 0: hops32<0, S, VEC, TILED>(inc, nf, nb, uf, ub, negf, negb, acc); break;
        case 1: hops32<1, S, VEC, TILED>(inc, nf, nb, uf, ub, negf, negb, acc); break;
        case 2: hops32<2, S, VEC, TILED>(inc, nf, nb, uf, ub, negf, negb, acc); break;
        default: hops32<3, S, VEC, TILED>(inc, nf, nb, uf, ub, negf, negb, acc); break;
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
    if constexpr (TILED) {
      // this block's tile: 768 contiguous floats, component k at [64 k, 64 k + 64)
      const int64_t base = (s0 >> 5) * 768;
      for (int o = threadIdx.x; o < 768; o += 128) {
        const int k = o >> 6, rem = o & 63, sl = rem >> 1, cc = 2 * k + (rem & 1);
        float v = 0.f;   // padding sites stay zero
        if (s0 + sl < op.sites) {
          const float sum = ((sacc[0][cc][sl] + sacc[1][cc][sl]) + sacc[2][cc][sl]) + sacc[3][cc][sl];
          v = fmaf(mk, sum, __ldg(ind + base + o));
        }
        outd[base + o] = v;
      }
    } else {
      for (int o = threadIdx.x; o < kWilsonSites * 24; o += 128) {
        const int sl = o / 24, cc = o - 24 * (o / 24);
        const int64_t ss = s0 + sl;
        if (ss >= op.sites) continue;
        const float sum = ((sacc[0][cc][sl] + sacc[1][cc][sl]) + sacc[2][cc][sl]) + sacc[3][cc][sl];
        outd[24 * ss + cc] = fmaf(mk, sum, __ldg(ind + 24 * ss + cc));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Large lattices (at least kSiteKernelSites sites): one thread per site runs
// all eight hops of its site, for two columns at a time (blockIdx.y = column
// pair), so the four direction partials never leave registers: no shared
// memory exchange and no CTA barrier.  Each link is loaded once per column
// pair and applied to both columns.  Measured on GB300 against the kernel
// above (11 columns): 16^3 x 32 125 us instead of 152, 16^4 62 us instead of
// 80; on small lattices (8^4: 4096 threads) it leaves most SMs idle, so the
// kernel above stays there.
// ---------------------------------------------------------------------------
constexpr int64_t kSiteKernelSites = 65536;

template <bool TILED, bool VEC, bool L2ONLY>
SEED_DEV void load_site(const float2 *__restrict__ in, int64_t q, float2 (&ps)[12]) {
  if constexpr (TILED) load_spinor_tiled<L2ONLY>(in, q, ps);
  else load_spinor<VEC, L2ONLY>(in + 12 * q, ps);
}

// direction MU of site s for the columns set in jm (bit j: column j of the
// pair); MU == 0 starts the sums.  Cache policy: the x and y neighbours of a
// block's sites lie in the block's own or adjacent 32-site tiles, which its
// other hops and its epilogue read again, so they go through L1; the z and t
// neighbours (another plane of the lattice) and the links are used once per
// thread and are read from L2 only, leaving L1 to the reused tiles.  Measured
// on GB300 (11 columns): 16^3 x 32 114.9 -> 103.3 us and 32^3 x 64 1985 ->
// 1879 us together with the streaming stores of the epilogue; same results
// bit for bit.
template <int MU, int S, bool TILED, bool VEC>
SEED_DEV void site_dir2(const WilsonOp32 &op, const float2 *__restrict__ in, int64_t ldi, int64_t s, int32_t nf,
                        int32_t nb, unsigned negf, unsigned negb, unsigned jm, float2 (&acc)[2][12]) {
  constexpr bool kFar = MU >= 2;
  const float2 *L = op.links + (int64_t)MU * 9 * op.sites;
  {
    float2 u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldcg(L + (int64_t)k * op.sites + s);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (jm & (1u << j)) {
        float2 p[12];
        load_site<TILED, VEC, kFar>(in + j * ldi, nf, p);
        hop_r<MU, S, true, MU == 0>(p, u, negf, acc[j]);
      }
    }
  }
  {
    float2 u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldcg(L + (int64_t)k * op.sites + nb);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (jm & (1u << j)) {
        float2 p[12];
        load_site<TILED, VEC, kFar>(in + j * ldi, nb, p);
        hop_r<MU, -S, false, false>(p, u, negb, acc[j]);
      }
    }
  }
}

// Grid: one block per (128 sites, column pair), the pair fastest, so that the
// pairs of one site block run together and their link loads hit L2.
template <int S, bool TILED, bool VEC>
__global__ void __launch_bounds__(128, 4) k_dslash32_site(WilsonOp32 op, const float2 *__restrict__ in, int64_t ldi,
                                                          float2 *__restrict__ out, int64_t ldo,
                                                          const int32_t *__restrict__ col_active, int ncols) {
  const int npairs = (ncols + 1) / 2;
  const int64_t sblock = (int64_t)blockIdx.x / npairs;
  const int c0 = 2 * (int)(blockIdx.x - sblock * npairs);
  unsigned jm = 0u;
#pragma unroll
  for (int j = 0; j < 2; ++j)
    if (c0 + j < ncols && (col_active == nullptr || col_active[c0 + j] != 0)) jm |= 1u << j;
  if (jm == 0u) return;   // uniform over the block
  const int64_t s = sblock * 128 + threadIdx.x;
  const int64_t send = TILED ? (op.sites + 31) / 32 * 32 : op.sites;
  if (s >= send) return;
  const bool valid = s < op.sites;   // tiled padding sites only write zeros
  in += (int64_t)c0 * ldi;
  out += (int64_t)c0 * ldo;
  float2 acc[2][12];
  if (valid) {
    const int4 *q = reinterpret_cast<const int4 *>(op.nbr + 8 * s);
    const int4 a = __ldg(q), b = __ldg(q + 1);
    unsigned negf = 0u, negb = 0u;
    if (op.bc_t) {
      const int64_t t = s / ((int64_t)op.dims[0] * op.dims[1] * op.dims[2]);
      if (t == op.dims[3] - 1) negf = CxBits<float2>::sign;
      if (t == 0) negb = CxBits<float2>::sign;
    }
    site_dir2<0, S, TILED, VEC>(op, in, ldi, s, a.x, a.y, 0u, 0u, jm, acc);
    site_dir2<1, S, TILED, VEC>(op, in, ldi, s, a.z, a.w, 0u, 0u, jm, acc);
    site_dir2<2, S, TILED, VEC>(op, in, ldi, s, b.x, b.y, 0u, 0u, jm, acc);
    site_dir2<3, S, TILED, VEC>(op, in, ldi, s, b.z, b.w, negf, negb, jm, acc);
  }
  const float mk = (float)(-op.kappa);
  const int64_t so = TILED ? (s >> 5) * 384 + (s & 31) : 12 * s;
  constexpr int kStride = TILED ? 32 : 1;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!(jm & (1u << j))) continue;
    const float2 *ic = in + j * ldi + so;
    float2 *oc = out + j * ldo + so;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      float2 v = make_float2(0.f, 0.f);
      if (valid) {
        const float2 x = __ldg(ic + kStride * k);
        v = make_float2(fmaf(mk, acc[j][k].x, x.x), fmaf(mk, acc[j][k].y, x.y));
      }
      __stcs(oc + kStride * k, v);   // streaming store: this kernel does not read it again
    }
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
                            int ncols, const int32_t *col_active, bool tiled, cudaStream_t s) {
  const int64_t nsb = (op.sites + kWilsonSites - 1) / kWilsonSites;
  int64_t group = (nsb * ncols) / (152 * 4);
  if (group < 1) group = 1;
  if (group > ncols) group = ncols;
  const int ngroups = (int)((ncols + group - 1) / group);
  const dim3 grid((unsigned)nsb, (unsigned)ngroups);
  const bool vec = ((uintptr_t)in % 16 == 0) && (ldi % 2 == 0);
  if (op.sites >= kSiteKernelSites) {
    const int64_t nthreads = tiled ? nsb * kWilsonSites : op.sites;
    const unsigned g2 = (unsigned)(((nthreads + 127) / 128) * ((ncols + 1) / 2));
    if (tiled) {
      if (sign > 0) k_dslash32_site<+1, true, false><<<g2, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols);
      else k_dslash32_site<-1, true, false><<<g2, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols);
    } else if (vec) {
      if (sign > 0) k_dslash32_site<+1, false, true><<<g2, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols);
      else k_dslash32_site<-1, false, true><<<g2, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols);
    } else {
      if (sign > 0) k_dslash32_site<+1, false, false><<<g2, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols);
      else k_dslash32_site<-1, false, false><<<g2, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols);
    }
    return;
  }
  const int g = (int)group;
  if (tiled) {
    if (sign > 0) k_dslash32<+1, false, true><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
    else k_dslash32<-1, false, true><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
  } else if (sign > 0) {
    if (vec) k_dslash32<+1, true, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
    else k_dslash32<+1, false, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
  } else {
    if (vec) k_dslash32<-1, true, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
    else k_dslash32<-1, false, false><<<grid, 128, 0, s>>>(op, in, ldi, out, ldo, col_active, ncols, g);
  }
}

}  // namespace seedk
