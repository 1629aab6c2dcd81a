// wilson_device.cuh -- device code of the Wilson-Dirac hop (spin projection,
// SU(3) multiply, reconstruction), shared by the stand-alone operator kernels
// (wilson.cu) and the persistent solver kernels (persistent.cu).
//
// In the chiral basis g_mu = [[0, B_mu], [B_mu^H, 0]] with 2x2 blocks whose
// rows each hold one entry from {1, i, -1, -i}.  Hence (1 - s g_mu) psi has
// upper half h = psi_up - s B_mu psi_dn and lower half -s B_mu^H h: a hop
// multiplies only the two-spinor h by the link, 84 floating-point operations
// per hop.  Phases and boundary signs are register swaps and sign-bit XORs.
// C = double2 (the FP64 operator) or float2 (its FP32 copy, mixed precision).
//
// NC selects how spinors are loaded: true = the read-only path (__ldg), for
// kernels in which the input does not change; false = ordinary loads, for
// persistent kernels that rewrite the input between grid barriers.  Ordinary
// loads may hit L1 (the 8 hops of a site reuse each neighbour's spinor); they
// see other blocks' writes because every grid barrier is a release (fence +
// arrival) / acquire (acquire load + fence) pair followed by a CTA barrier.
#pragma once
#include "device_common.cuh"
#include "seed_internal.h"

namespace seedk {

template <bool NC, class C> SEED_DEV C ldv(const C *p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// ---------------------------------------------------------------------------
// phases: code 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i  (C = double2 or float2)
// ---------------------------------------------------------------------------
template <int P, class C> SEED_DEV C ph_add(C z, C w) {   // z + phase(P) w
  if constexpr (P == 0) return C{z.x + w.x, z.y + w.y};
  else if constexpr (P == 1) return C{z.x - w.y, z.y + w.x};
  else if constexpr (P == 2) return C{z.x - w.x, z.y - w.y};
  else return C{z.x + w.y, z.y - w.x};
}
template <int P, class C> SEED_DEV C ph_mul(C w) {         // phase(P) w, no FP op
  constexpr auto m = CxBits<C>::sign;
  if constexpr (P == 0) return w;
  else if constexpr (P == 1) return C{xsign(w.y, m), w.x};
  else if constexpr (P == 2) return C{xsign(w.x, m), xsign(w.y, m)};
  else return C{w.y, xsign(w.x, m)};
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
// U^H; psi and U already in registers.  FIRST: acc is overwritten instead of
// accumulated.  neg: boundary sign mask (0 or the sign bit).
template <int MU, int S, bool FWD, bool FIRST, class C>
SEED_DEV void hop_r(const C (&psi)[12], const C (&u)[9], typename CxBits<C>::U neg, C (&acc)[12]) {
  // h_k = psi_k - S * P(k) psi_{2+J(k)}
  constexpr int c0 = S > 0 ? ph_neg(bP(MU, 0)) : bP(MU, 0);
  constexpr int c1 = S > 0 ? ph_neg(bP(MU, 1)) : bP(MU, 1);
  C h0[3], h1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h0[a] = ph_add<c0>(psi[a], psi[3 * (2 + bJ(MU, 0)) + a]);
    h1[a] = ph_add<c1>(psi[3 + a], psi[3 * (2 + bJ(MU, 1)) + a]);
    h0[a].x = xsign(h0[a].x, neg); h0[a].y = xsign(h0[a].y, neg);
    h1[a].x = xsign(h1[a].x, neg); h1[a].y = xsign(h1[a].y, neg);
  }
  // chi_k = M h_k
  C x0[3], x1[3];
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
      C uc = C{u[a].x, xsign(u[a].y, CxBits<C>::sign)};
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

// The two hops of direction MU for one site: forward (1 - S g) U psi_f and
// backward (1 + S g) U^H psi_b, into acc (overwritten).  The lower halves of
// the two hops carry opposite phases, -S conj(P) x_f and +S conj(P) x_b, so
// with the upper half u = x_f + x_b the lower half is 2 (lower of x_f) -
// phase(u): the backward product is chained onto the upper half by FMAs
// instead of being formed and added (12 fewer FP64 operations per pair).
template <int MU, int S, class C>
SEED_DEV void hop_pair_r(const C (&pf)[12], const C (&uf)[9], typename CxBits<C>::U negf, const C (&pb)[12],
                         const C (&ub)[9], typename CxBits<C>::U negb, C (&acc)[12]) {
  using R = typename CxBits<C>::R;
  hop_r<MU, S, true, true>(pf, uf, negf, acc);
  constexpr int c0 = -S > 0 ? ph_neg(bP(MU, 0)) : bP(MU, 0);
  constexpr int c1 = -S > 0 ? ph_neg(bP(MU, 1)) : bP(MU, 1);
  C h0[3], h1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h0[a] = ph_add<c0>(pb[a], pb[3 * (2 + bJ(MU, 0)) + a]);
    h1[a] = ph_add<c1>(pb[3 + a], pb[3 * (2 + bJ(MU, 1)) + a]);
    h0[a].x = xsign(h0[a].x, negb); h0[a].y = xsign(h0[a].y, negb);
    h1[a].x = xsign(h1[a].x, negb); h1[a].y = xsign(h1[a].y, negb);
  }
  // upper half += U^H h
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      acc[a] = cfmac(ub[3 * bb + a], h0[bb], acc[a]);
      acc[3 + a] = cfmac(ub[3 * bb + a], h1[bb], acc[3 + a]);
    }
  }
  // lower half: 2 x (forward lower half) - phase(upper)
  constexpr int l0 = S > 0 ? ph_neg(ph_conj(bP(MU, 0))) : ph_conj(bP(MU, 0));
  constexpr int l1 = S > 0 ? ph_neg(ph_conj(bP(MU, 1))) : ph_conj(bP(MU, 1));
  constexpr int s0 = 2 + bJ(MU, 0), s1 = 2 + bJ(MU, 1);
  const R two = (R)2;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const C p0 = ph_mul<l0>(acc[a]), p1 = ph_mul<l1>(acc[3 + a]);
    acc[3 * s0 + a] = C{fma(two, acc[3 * s0 + a].x, -p0.x), fma(two, acc[3 * s0 + a].y, -p0.y)};
    acc[3 * s1 + a] = C{fma(two, acc[3 * s1 + a].x, -p1.x), fma(two, acc[3 * s1 + a].y, -p1.y)};
  }
}

template <int MU, int S, bool NC = true, class C>
SEED_DEV void site_mu(const WilsonOpT<C> &op, const C *__restrict__ in, int64_t s, C (&acc)[12]) {
  const int32_t nf = __ldg(op.nbr + 8 * s + 2 * MU);
  const int32_t nb = __ldg(op.nbr + 8 * s + 2 * MU + 1);
  typename CxBits<C>::U negf = 0, negb = 0;
  if (MU == 3 && op.bc_t) {
    const int64_t slab = (int64_t)op.dims[0] * op.dims[1] * op.dims[2];
    const int64_t t = s / slab;
    if (t == op.dims[3] - 1) negf = CxBits<C>::sign;
    if (t == 0) negb = CxBits<C>::sign;
  }
  // forward: (1 - S g) U_mu(s) psi(s + mu); backward: (1 + S g) U_mu(s - mu)^H psi(s - mu)
  C pf[12], pb[12], uf[9], ub[9];
  const C *psf = in + 12 * (int64_t)nf, *psb = in + 12 * (int64_t)nb;
  const C *Uf = op.links + ((int64_t)MU * op.sites + s) * 9, *Ub = op.links + ((int64_t)MU * op.sites + nb) * 9;
#pragma unroll
  for (int k = 0; k < 12; ++k) pf[k] = ldv<NC>(psf + k);
#pragma unroll
  for (int k = 0; k < 9; ++k) uf[k] = __ldg(Uf + k);
#pragma unroll
  for (int k = 0; k < 12; ++k) pb[k] = ldv<NC>(psb + k);
#pragma unroll
  for (int k = 0; k < 9; ++k) ub[k] = __ldg(Ub + k);
  hop_pair_r<MU, S>(pf, uf, negf, pb, ub, negb, acc);
}

constexpr int kWilsonSites = 32;   // sites per block; 4 warps (one per mu)

// The hop sums of the 32 sites s0 .. s0+31 (a block of 128 threads: warp mu
// handles direction mu, lane = site), left per direction in
// sacc[mu][real component][lane] for the block's epilogue; sites past the
// lattice contribute zeros.  Ends with a CTA barrier.
template <int S, bool NC = true, class C>
SEED_DEV void dslash_tile(const WilsonOpT<C> &op, const C *__restrict__ in, int64_t s0,
                          typename CxBits<C>::R (*sacc)[24][kWilsonSites + 1]) {
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s = s0 + lane;
  C acc[12];
  if (s < op.sites) {
    switch (mu) {
      case 0: site_mu<0, S, NC>(op, in, s, acc); break;
      case 1: site_mu<1, S, NC>(op, in, s, acc); break;
      case 2: site_mu<2, S, NC>(op, in, s, acc); break;
      default: site_mu<3, S, NC>(op, in, s, acc); break;
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
}

// Sum of the four direction partials of real component c of tile site sl.
template <class R>
SEED_DEV R tile_hop_sum(const R (*sacc)[24][kWilsonSites + 1], int c, int sl) {
  return ((sacc[0][c][sl] + sacc[1][c][sl]) + sacc[2][c][sl]) + sacc[3][c][sl];
}

}  // namespace seedk
