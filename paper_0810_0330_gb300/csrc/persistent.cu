// persistent.cu -- persistent cooperative kernels for the seed solve (runs of
// Sec. 3 Lanczos steps without reorthogonalization; FP64, and FP32 for the
// mixed-precision path) and for the lockstep CG on the seeded systems (FP64).
// One launch runs many steps; grid-wide dependencies are grid barriers instead
// of kernel boundaries.
//
// Why: on the benchmark's 8^4 lattice one Lanczos step is ~6 us of FP64 work
// per SM in each operator half and a few microseconds of vector work; as a
// chain of dependent kernels every step paid launch, ramp-up and tail five
// times, and the small vector kernels ran latency-bound.
//
// Barriers: an arrival counter that only grows during a launch (the host zeroes
// it before each launch); a block waits until it reaches epoch * gridDim.x.  A
// "reducing" barrier lets the last block to arrive run the scalar step (it
// reads every block's partial sums in a fixed order, so results are
// deterministic) and then release the others.  Every wait is bounded: after
// kBarrierTimeoutNs of waiting a block sets GridSync::error and all blocks
// leave; the host turns that into SEED_ETIMEOUT.  The launch is cooperative,
// so all blocks are resident and a barrier can only time out on a fault.
//
// Memory: data written by other blocks during the launch is read with ordinary
// or L2 (__ldcg) loads after a barrier, never through the non-coherent
// read-only path; every barrier is a release (fence, arrival) / acquire
// (acquire load, fence) pair followed by a CTA barrier.
//
// Operator tiles (32 sites, 4 warps) go to at most one block per SM: the first
// block that starts on an SM registers as a tile owner, so two tiles never
// share an SM's FP64 pipe while another SM idles.
#include "seed_device.cuh"
#include "wilson_device.cuh"

namespace seedk {

constexpr int PT = kVecThreads;                          // 4 warps: the Wilson tile layout
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

SEED_DEV unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
SEED_DEV unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
template <class U> SEED_DEV U vload(const U *p) { return *(const volatile U *)p; }

// thread 0: wait until *flag >= target; false on time-out or when another block failed
SEED_DEV bool wait_geq(const unsigned *flag, unsigned target, int *error) {
  unsigned long long t0 = 0;
  for (unsigned spin = 0;; ++spin) {
    if (ld_acquire(flag) >= target) return true;
    if (vload(error)) return false;
    if ((spin & 255u) == 255u) {
      const unsigned long long t = gtimer();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kBarrierTimeoutNs) {
        atomicExch(error, 1);
        return false;
      }
    }
    __nanosleep(32);
  }
}

SEED_DEV bool grid_sync(const GridSync &g, unsigned &epoch) {
  __shared__ int s_ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(g.count, 1u);
    s_ok = wait_geq(g.count, epoch * gridDim.x, g.error) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

template <class F>
SEED_DEV bool grid_reduce_sync(const GridSync &g, unsigned &epoch, F &&last_block_work) {
  __shared__ int s_last, s_ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(g.count, 1u);
    s_last = (prev == epoch * gridDim.x - 1u) ? 1 : 0;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    last_block_work();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(g.release, epoch);
    }
  } else if (threadIdx.x == 0) {
    s_ok = wait_geq(g.release, epoch, g.error) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// Tile ownership: (rank, owners) of this block; the first block on each SM owns
// tiles.  If no block could register (SM ids >= 256), every block owns tiles.
struct Owners {
  int rank, count;
};
SEED_DEV bool register_owner(const GridSync &g, unsigned &epoch, Owners &o) {
  __shared__ int s_rank;
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    int r = -1;
    if (sm < 256u && atomicAdd(g.sm_slots + sm, 1u) == 0u) r = (int)atomicAdd(g.owners, 1u);
    s_rank = r;
  }
  if (!grid_sync(g, epoch)) return false;
  const int n = (int)vload(g.owners);
  if (n > 0) {
    o.rank = s_rank;
    o.count = n;
  } else {
    o.rank = blockIdx.x;
    o.count = gridDim.x;
  }
  return true;
}

// Last block: s_vals[v] = sum over rows b < nrows of part[32 b + v] (v < 32),
// one thread per row (16 independent 16-byte loads), then a block
// reduce-scatter; fixed order, so deterministic.
SEED_DEV void reduce_rows32(const double *part, int nrows, double *s_vals, double (*sred)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) acc[q] = 0.0;
  for (int b = threadIdx.x; b < nrows; b += PT) {
    const double2 *row = reinterpret_cast<const double2 *>(part + (int64_t)b * 32);
    double2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __ldcg(row + k);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      acc[2 * k] += v[k].x;
      acc[2 * k + 1] += v[k].y;
    }
  }
  const double mine = warp_reduce_scatter32(acc);
  sred[warp][lane] = mine;
  __syncthreads();
  if (threadIdx.x < 32) s_vals[lane] = ((sred[0][lane] + sred[1][lane]) + sred[2][lane]) + sred[3][lane];
  __syncthreads();
}

// Hopping sums of one 32-site tile into sacc[mu][component][site] (S = +1: D, -1: D^H).
template <int S>
SEED_DEV void wilson_tile(const WilsonOp &op, const double2 *in, int64_t s0, double (*sacc)[24][kWilsonSites + 1]) {
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s = s0 + lane;
  double2 acc[12];
  if (s < op.sites) {
    switch (mu) {
      case 0: site_mu<0, S, false>(op, in, s, acc); break;
      case 1: site_mu<1, S, false>(op, in, s, acc); break;
      case 2: site_mu<2, S, false>(op, in, s, acc); break;
      default: site_mu<3, S, false>(op, in, s, acc); break;
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
}
// complex component cc of tile-local site sl, summed over the 4 directions in order
SEED_DEV double2 tile_sum(double (*sacc)[24][kWilsonSites + 1], int cc, int sl) {
  return c2(((sacc[0][2 * cc][sl] + sacc[1][2 * cc][sl]) + sacc[2][2 * cc][sl]) + sacc[3][2 * cc][sl],
            ((sacc[0][2 * cc + 1][sl] + sacc[1][2 * cc + 1][sl]) + sacc[2][2 * cc + 1][sl]) + sacc[3][2 * cc + 1][sl]);
}

// ---------------------------------------------------------------------------
// Seed runs (the Lanczos steps of Sec. 3 between two reorthogonalizing steps).  The
// seeding of systems 2..p is blocked (SeedBufs::Wb, seedblock.cu): a step only
// stores w_i, so the recurrence of system 1 is all that runs here.
//
// Wilson, two phases and two grid barriers per step i:
//   phase 1 (tiles): v_i = f / beta_{i-1} into V; t = D v_i; per tile the
//           partial sums of ||t||^2 and Re(v_i^H v_{i-1})
//   barrier; every block: alpha_i = ||D v_i||^2 - beta_{i-1} Re(v_i^H v_{i-1}),
//           then gamma_{i-1}, delta_i, zeta_i (the LU update)
//   phase 2 (tiles): u = D^H t; f = u - beta_{i-1} v_{i-1} - alpha_i v_i (step
//           5); w_i and x^1 += zeta_i w_i (LU update); w_i into Wb; partial ||f||^2
//   barrier; every block: beta_i and the stopping test.
// alpha_i is the paper's v_i^H (A v_i - beta_{i-1} v_{i-1}) with v_i^H A v_i
// written as ||D v_i||^2 (A = D^H D): the same number up to rounding, available
// one barrier earlier, so that the update runs in the D^H tiles' epilogue.
//
// Every block keeps its own shared-memory copy of the recurrence scalars.
// After each barrier every block reduces the same per-tile partials in the same
// fixed order (tile order, not block order) and runs the same scalar code, so
// the copies stay identical; block 0 writes the step histories and, on leaving,
// the state back.
// ---------------------------------------------------------------------------
struct LocalSeed {
  SeedState st;
};

template <class T>
SEED_DEV SeedBufs<T> local_bufs(const SeedBufs<T> &b, LocalSeed &L) {
  SeedBufs<T> l = b;
  l.st = &L.st;
  if (blockIdx.x != 0) l.alpha_hist = l.beta_hist = l.delta_hist = l.gamma_hist = nullptr;
  return l;
}

template <class T>
SEED_DEV void local_load(const SeedBufs<T> &b, LocalSeed &L) {
  if (threadIdx.x == 0) L.st = *b.st;
  __syncthreads();
}

template <class T>
SEED_DEV void local_store(const SeedBufs<T> &b, const LocalSeed &L) {
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) *b.st = L.st;
}

// Stops the run (in every block alike) when step i would not fit in Wb; the
// host caps runs below this, so it only guards the buffer.
template <class T>
SEED_DEV bool block_full(const SeedBufs<T> &b, LocalSeed &L, int i) {
  if (b.Wb == nullptr || i - L.st.blk0 < kSeedBlock) return false;
  __syncthreads();
  if (threadIdx.x == 0) {
    L.st.active = 0;
    L.st.stop_reason = STOP_BLOCK;
  }
  __syncthreads();
  return true;
}

// barrier, then in every block: alpha_i from parts[k * stride] (k < nparts, a
// fixed order that does not depend on which block ran which tile) minus
// beta_{i-1} times parts[k * stride + 1] when `with_vm`, and the step's scalars
template <class T>
SEED_DEV bool seed_alpha_step(const SeedBufs<T> &bl, const double *parts, int nparts, int stride, bool with_vm,
                              int i, LocalSeed &L, const GridSync &g, unsigned &epoch) {
  if (!grid_sync(g, epoch)) return false;
  if (threadIdx.x < 32) {
    double a = warp_sum_partials(parts, nparts, stride, 0);
    if (with_vm) {
      const double vm = warp_sum_partials(parts, nparts, stride, 1);
      a = a - L.st.beta_prev * vm;
    }
    if (threadIdx.x == 0) seed_step_scalars<T, false>(bl, i, a, nullptr);
  }
  __syncthreads();
  return true;
}

// barrier, then in every block: beta_i from the partials of ||f||^2 and the end of the step
template <class T>
SEED_DEV bool seed_beta_step(const SeedBufs<T> &bl, const double *parts, int nparts, int i, LocalSeed &L,
                             const GridSync &g, unsigned &epoch) {
  if (!grid_sync(g, epoch)) return false;
  if (threadIdx.x < 32) {
    const double ss = warp_sum_partials(parts, nparts, 1, 0);
    if (threadIdx.x == 0) {
      if (bl.Wb != nullptr) L.st.w_last = i;
      seed_finish<T, false>(bl, ss);
    }
  }
  __syncthreads();
  return true;
}

// On leaving with i == i_stop (a reorthogonalization step or the end of a
// seeding block follows): the next step starts from f = beta_{i-1} v_i in b.f
// (its first kernel forms v_i), so a run that alternates two f buffers copies
// the current one there.
template <class T>
SEED_DEV void seed_leave(const SeedBufs<T> &b, const LocalSeed &L, const T *f, int i_stop) {
  if (!L.st.active || L.st.i != i_stop || f == b.f) return;
  for (int64_t e = (int64_t)blockIdx.x * PT + threadIdx.x; e < b.n; e += (int64_t)gridDim.x * PT) b.f[e] = __ldcg(f + e);
}

// FP64 Wilson run: five warps per block.  Warps 0-3 are the tile warps of the
// operator (one direction each, as everywhere); warp 4 is a scalar warp.  After
// each grid barrier the stencil of the next phase does not depend on the
// scalars the barrier made available (D f and D^H t need only f and t; v_i =
// f / beta_{i-1} is applied to D f in the epilogue, D being linear), so the
// scalar warp reduces the tiles' partials and runs the recurrence's scalar
// code while the tile warps compute the stencil of the block's first tile;
// one CTA barrier joins them before the epilogue.  On the 8^4 lattice this
// hides the two scalar phases of a step (about 5 of its 29.5 us) behind the
// stencils.  Same arithmetic and summation order as before.
constexpr int PTW = PT + 32;

// named barrier of the four tile warps
SEED_DEV void tile_warps_sync() { asm volatile("bar.sync 1, %0;" ::"n"(PT) : "memory"); }

// wilson_tile for the tile warps alone (ends with their named barrier)
template <int S>
SEED_DEV void wilson_tile4(const WilsonOp &op, const double2 *in, int64_t s0, double (*sacc)[24][kWilsonSites + 1]) {
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s = s0 + lane;
  double2 acc[12];
  if (s < op.sites) {
    switch (mu) {
      case 0: site_mu<0, S, false>(op, in, s, acc); break;
      case 1: site_mu<1, S, false>(op, in, s, acc); break;
      case 2: site_mu<2, S, false>(op, in, s, acc); break;
      default: site_mu<3, S, false>(op, in, s, acc); break;
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
  tile_warps_sync();
}

// The two values of every lane summed over the warp, both returned to every
// lane: the first level trades halves (lanes < 16 keep x, the others y), so
// each lane adds 5 times instead of 10.  Fixed order, deterministic.
SEED_DEV double2 warp_sum_pair(double x, double y) {
  const bool hi = (threadIdx.x & 16) != 0;
  double keep = hi ? y : x;
  keep += __shfl_xor_sync(0xffffffffu, hi ? x : y, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  return c2(__shfl_sync(0xffffffffu, keep, 0), __shfl_sync(0xffffffffu, keep, 16));
}

// One warp: the sum of nb partials with up to 32 PER of them loaded at once
// (lane l adds partial[l], partial[l + 32], ... in order), then the warp tree:
// one FP64 add per value and one round trip to L2 for the short lists of the
// persistent runs, where the scalar warp's FP64 instructions are on the
// critical path.  Longer lists run in chunks.
template <int PER>
SEED_DEV double warp_sum_short(const double *p, int nb) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 32 * PER) {
    double v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < nb ? __ldcg(p + b) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) s += v[u];
  }
  return warp_sum(s);
}
// The same for nb pairs (p[2b], p[2b + 1]); both sums returned to every lane.
template <int PER>
SEED_DEV double2 warp_sum_short_pairs(const double *p, int nb) {
  const int lane = threadIdx.x & 31;
  double sx = 0.0, sy = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 32 * PER) {
    double2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < nb ? __ldcg(reinterpret_cast<const double2 *>(p) + b) : c2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      sx += v[u].x;
      sy += v[u].y;
    }
  }
  return warp_sum_pair(sx, sy);
}
constexpr int kScalarSumPer = 16;   // 512 partials (128 tiles x 4 warps, the 8^4 lattice) in one pass

// Resident form of the run, used when every owner block holds at most one tile
// (lattices with no more 32-site tiles than SMs, e.g. 8^4 with 128 tiles): the
// tile's links (both hops of each direction) stay in shared memory and its
// neighbour indices and boundary signs in registers for the whole run, and the
// tile's own elements of f, t, w_i, x^1, v_i and v_{i-1} are kept in shared
// memory, so that after each grid barrier only the neighbours' spinors come
// from L2.  f, t and v_i still go to global memory every step (other blocks'
// stencils read f and t, V keeps the basis); x^1 and w_i are written back when
// the run ends.  Links: s_lnk[(mu * 18 + k) * 32 + lane], k < 9 the forward
// link U_mu(s), k >= 9 the backward link U_mu(s - mu); vectors:
// s_vec[slot * 384 + o] with o = 12 * (site in tile) + component.
constexpr int kResLinks = 4 * 18 * kWilsonSites;
constexpr int kResTile = 12 * kWilsonSites;
enum { kResF = 0, kResT = 1, kResW = 2, kResX = 3, kResV = 4 };   // kResV + (i & 1): v_i
constexpr size_t kResSmemBytes = (size_t)(kResLinks + 6 * kResTile) * sizeof(double2);

template <int MU, int S>
SEED_DEV void site_mu_res(const double2 *in, int32_t nf, int32_t nb, unsigned long long negf,
                          unsigned long long negb, const double2 *su, double2 (&acc)[12]) {
  double2 pf[12], pb[12], uf[9], ub[9];
  const double2 *psf = in + 12 * (int64_t)nf, *psb = in + 12 * (int64_t)nb;
#pragma unroll
  for (int k = 0; k < 12; ++k) pf[k] = psf[k];
#pragma unroll
  for (int k = 0; k < 12; ++k) pb[k] = psb[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) uf[k] = su[k * 32];
#pragma unroll
  for (int k = 0; k < 9; ++k) ub[k] = su[(9 + k) * 32];
  hop_pair_r<MU, S>(pf, uf, negf, pb, ub, negb, acc);
}

// wilson_tile4 with the links, indices and signs resident (live: the site exists)
template <int S>
SEED_DEV void wilson_tile4_res(const double2 *in, int32_t nf, int32_t nb, unsigned long long negf,
                               unsigned long long negb, bool live, const double2 *s_lnk,
                               double (*sacc)[24][kWilsonSites + 1]) {
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const double2 *su = s_lnk + mu * 18 * 32 + lane;
  double2 acc[12];
  if (live) {
    switch (mu) {
      case 0: site_mu_res<0, S>(in, nf, nb, negf, negb, su, acc); break;
      case 1: site_mu_res<1, S>(in, nf, nb, negf, negb, su, acc); break;
      case 2: site_mu_res<2, S>(in, nf, nb, negf, negb, su, acc); break;
      default: site_mu_res<3, S>(in, nf, nb, negf, negb, su, acc); break;
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
  tile_warps_sync();
}

// tpart: 12 x tiles doubles -- per tile warp (4 per tile) the phase-1 pairs,
// then the phase-2 norms; each tile warp sums its lanes and lane 0 stores, and
// the scalar warp of every block sums all of them in (tile, warp) order.
__global__ void __launch_bounds__(PTW) k_seed_run_wilson(SeedBufs<double2> b, WilsonOp op, double2 *tbuf,
                                                          GridSync g, double *bpart, double *tpart, int i_stop) {
  __shared__ double sacc[4][24][kWilsonSites + 1];
  __shared__ LocalSeed L;
  extern __shared__ double2 s_dyn[];
  (void)bpart;
  const int64_t sites = op.sites;
  const int tiles = (int)((sites + kWilsonSites - 1) / kWilsonSites);
  const double kappa = op.kappa;
  double *part1 = tpart, *part2 = tpart + 8 * (int64_t)tiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool tw = warp < 4;            // tile warp; warp 4 is the scalar warp
  unsigned epoch = 0;
  local_load(b, L);
  const SeedBufs<double2> bl = local_bufs(b, L);
  Owners own;
  if (!register_owner(g, epoch, own)) return;
  double2 *const X = reinterpret_cast<double2 *>(b.call->X);
  const int first_tile = own.rank >= 0 && own.rank < tiles ? own.rank : -1;
  // resident form: one tile per owner block
  const bool res = tiles <= own.count && first_tile >= 0;
  double2 *const s_lnk = s_dyn;
  double2 *const s_vec = s_dyn + kResLinks;
  int32_t r_nf = 0, r_nb = 0;
  unsigned long long r_negf = 0, r_negb = 0;
  const int64_t r_site = (int64_t)(first_tile >= 0 ? first_tile : 0) * kWilsonSites + lane;
  const bool r_live = r_site < sites;
  if (res) {
    const int64_t e0 = (int64_t)first_tile * kResTile;
    const int i0 = L.st.i;
    if (tw && r_live) {
      const int mu = warp;
      r_nf = __ldg(op.nbr + 8 * r_site + 2 * mu);
      r_nb = __ldg(op.nbr + 8 * r_site + 2 * mu + 1);
      if (mu == 3 && op.bc_t) {
        const int64_t t = r_site / ((int64_t)op.dims[0] * op.dims[1] * op.dims[2]);
        if (t == op.dims[3] - 1) r_negf = CxBits<double2>::sign;
        if (t == 0) r_negb = CxBits<double2>::sign;
      }
      const double2 *Uf = op.links + ((int64_t)mu * sites + r_site) * 9;
      const double2 *Ub = op.links + ((int64_t)mu * sites + r_nb) * 9;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        s_lnk[(mu * 18 + k) * 32 + lane] = __ldg(Uf + k);
        s_lnk[(mu * 18 + 9 + k) * 32 + lane] = __ldg(Ub + k);
      }
    }
    const double2 *vprev = b.V + (int64_t)(i0 > 1 ? i0 - 2 : 0) * b.ldv;
    for (int o = threadIdx.x; o < kResTile; o += PTW) {
      const int64_t e = e0 + o;
      if (e < b.n) {
        s_vec[kResF * kResTile + o] = b.f[e];
        s_vec[kResW * kResTile + o] = i0 > 1 ? b.w[e] : c2(0.0, 0.0);
        s_vec[kResX * kResTile + o] = X[e];
        s_vec[(kResV + ((i0 - 1) & 1)) * kResTile + o] = i0 > 1 ? vprev[e] : c2(0.0, 0.0);
      }
    }
    __syncthreads();
  }
  bool pending_beta = false;           // the end of the previous step (beta_{i-1}) is still to run
  for (;;) {
    // ---- phase 1 of step i, overlapped with the end of step i-1 ----
    {
      // the stencil D f of the step that may follow (discarded if the end of step i-1 stops the run)
      const int ip = L.st.i + (pending_beta ? 1 : 0);
      const bool go = L.st.active && ip < i_stop && (b.Wb == nullptr || ip - L.st.blk0 < kSeedBlock);
      __syncthreads();                 // everyone has read L.st before the scalar warp updates it
      if (tw && go && first_tile >= 0) {
        if (res) wilson_tile4_res<+1>(b.f, r_nf, r_nb, r_negf, r_negb, r_live, s_lnk, sacc);
        else wilson_tile4<+1>(op, b.f, (int64_t)first_tile * kWilsonSites, sacc);
      }
      if (!tw && pending_beta) {
        const double ss = warp_sum_short<kScalarSumPer>(part2, 4 * tiles);
        if (threadIdx.x == PT) {
          if (bl.Wb != nullptr) L.st.w_last = L.st.i;
          seed_finish<double2, false>(bl, ss);
        }
      }
      __syncthreads();
      pending_beta = false;
    }
    const int i = L.st.i;
    if (!L.st.active || i >= i_stop) break;
    if (block_full(b, L, i)) break;
    const double inv_b = L.st.inv_beta;
    const double bp = (i > 1) ? L.st.beta_prev : 0.0;
    double2 *vi = b.V + (int64_t)(i - 1) * b.ldv;
    const double2 *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * b.ldv;
    double2 *const s_vi = s_vec + (kResV + (i & 1)) * kResTile;
    double2 *const s_vm = s_vec + (kResV + ((i - 1) & 1)) * kResTile;
    // phase 1 epilogue: v_i, t = D v_i, partials of ||t||^2 and Re(v_i^H v_{i-1})
    if (first_tile >= 0) {
      for (int tile = first_tile; tile < tiles; tile += own.count) {
        const int64_t s0 = (int64_t)tile * kWilsonSites;
        if (tile != first_tile && tw) wilson_tile4<+1>(op, b.f, s0, sacc);
        if (tw) {
          double ptt = 0.0, pvm = 0.0;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int o = threadIdx.x + PT * k, sl = o / 12, cc = o - 12 * (o / 12);
            const int64_t ss = s0 + sl;
            if (ss < sites) {
              const double2 sum = tile_sum(sacc, cc, sl);
              const int64_t e = 12 * ss + cc;
              const double2 fe = res ? s_vec[kResF * kResTile + o] : b.f[e];
              const double2 v = c2(inv_b * fe.x, inv_b * fe.y);
              vi[e] = v;
              const double2 t = c2(fma(-kappa, inv_b * sum.x, v.x), fma(-kappa, inv_b * sum.y, v.y));
              tbuf[e] = t;
              if (res) {
                s_vi[o] = v;
                s_vec[kResT * kResTile + o] = t;
              }
              ptt = fma(t.y, t.y, fma(t.x, t.x, ptt));
              if (i > 1) {
                const double2 m = res ? s_vm[o] : vm[e];
                pvm = fma(v.y, m.y, fma(v.x, m.x, pvm));
              }
            }
          }
          const double2 ws = warp_sum_pair(ptt, pvm);
          if (lane == 0) {
            part1[2 * (4 * tile + warp)] = ws.x;
            part1[2 * (4 * tile + warp) + 1] = ws.y;
          }
        }
        if (tile + own.count < tiles) __syncthreads();   // sacc is reused by the next tile
      }
    }
    if (!grid_sync(g, epoch)) return;
    // ---- phase 2: u = D^H t overlapped with alpha_i and the LU update's scalars ----
    if (tw && first_tile >= 0) {
      if (res) wilson_tile4_res<-1>(tbuf, r_nf, r_nb, r_negf, r_negb, r_live, s_lnk, sacc);
      else wilson_tile4<-1>(op, tbuf, (int64_t)first_tile * kWilsonSites, sacc);
    }
    if (!tw) {
      const double2 s2 = warp_sum_short_pairs<kScalarSumPer>(part1, 4 * tiles);
      const double a = i > 1 ? s2.x - L.st.beta_prev * s2.y : s2.x;
      if (threadIdx.x == PT) seed_step_scalars<double2, false>(bl, i, a, nullptr);
    }
    __syncthreads();
    if (!L.st.active) break;   // delta_i <= 0
    const double a = L.st.alpha, zeta = L.st.zeta, inv_d = L.st.inv_delta;
    double2 *const wcol = b.Wb != nullptr ? b.Wb + (int64_t)(i - L.st.blk0) * b.ldv : nullptr;
    if (first_tile >= 0) {
      for (int tile = first_tile; tile < tiles; tile += own.count) {
        const int64_t s0 = (int64_t)tile * kWilsonSites;
        if (tile != first_tile && tw) wilson_tile4<-1>(op, tbuf, s0, sacc);
        if (tw) {
          double pff = 0.0;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int o = threadIdx.x + PT * k, sl = o / 12, cc = o - 12 * (o / 12);
            const int64_t ss = s0 + sl;
            if (ss < sites) {
              const double2 sum = tile_sum(sacc, cc, sl);
              const int64_t e = 12 * ss + cc;
              const double2 tv = res ? s_vec[kResT * kResTile + o] : tbuf[e];
              const double2 v = res ? s_vi[o] : vi[e];
              double2 f = c2(fma(-kappa, sum.x, tv.x), fma(-kappa, sum.y, tv.y));
              if (i > 1) {
                const double2 m = res ? s_vm[o] : vm[e];
                f = c2(fma(-bp, m.x, f.x), fma(-bp, m.y, f.y));
              }
              f = c2(fma(-a, v.x, f.x), fma(-a, v.y, f.y));
              double2 w;
              if (i > 1) {
                const double2 wp = res ? s_vec[kResW * kResTile + o] : b.w[e];
                w = c2(inv_d * fma(-bp, wp.x, v.x), inv_d * fma(-bp, wp.y, v.y));
              } else {
                w = c2(inv_d * v.x, inv_d * v.y);
              }
              b.f[e] = f;
              if (wcol != nullptr) wcol[e] = w;
              const double2 x = res ? s_vec[kResX * kResTile + o] : X[e];
              const double2 xn = c2(fma(zeta, w.x, x.x), fma(zeta, w.y, x.y));
              if (res) {
                s_vec[kResF * kResTile + o] = f;
                s_vec[kResW * kResTile + o] = w;
                s_vec[kResX * kResTile + o] = xn;
              } else {
                b.w[e] = w;
                X[e] = xn;
              }
              pff = fma(f.y, f.y, fma(f.x, f.x, pff));
            }
          }
          const double ws = warp_sum(pff);
          if (lane == 0) part2[4 * tile + warp] = ws;
        }
        if (tile + own.count < tiles) __syncthreads();
      }
    }
    if (!grid_sync(g, epoch)) return;
    pending_beta = true;               // beta_i and the stopping test run with the next stencil
  }
  if (res) {   // x^1 and w_i back to global memory
    __syncthreads();
    const int64_t e0 = (int64_t)first_tile * kResTile;
    for (int o = threadIdx.x; o < kResTile; o += PTW) {
      const int64_t e = e0 + o;
      if (e < b.n) {
        X[e] = s_vec[kResX * kResTile + o];
        b.w[e] = s_vec[kResW * kResTile + o];
      }
    }
  }
  if (tw) seed_leave<double2>(b, L, b.f, i_stop);
  local_store(b, L);
}

// ---------------------------------------------------------------------------
// The same two-phase Wilson run for the mixed-precision path: FP32 copy of
// the links (structure of arrays), FP32 vectors tiled by 32 sites (component
// k of site s at ((s/32)*12 + k)*32 + s%32, padding sites zero), FP32 sums per
// thread, FP64 block and grid sums and scalars.  Tiles cover the padding too,
// so every element of v_i, t, f, w_i is written (zeros in the padding).
// ---------------------------------------------------------------------------
template <int MU, int S>
SEED_DEV void site_mu32(const WilsonOp32 &op, const float2 *in, int64_t s, float2 (&acc)[12]) {
  const int32_t nf = __ldg(op.nbr + 8 * s + 2 * MU);
  const int32_t nb = __ldg(op.nbr + 8 * s + 2 * MU + 1);
  unsigned negf = 0u, negb = 0u;
  if (MU == 3 && op.bc_t) {
    const int64_t t = s / ((int64_t)op.dims[0] * op.dims[1] * op.dims[2]);
    if (t == op.dims[3] - 1) negf = CxBits<float2>::sign;
    if (t == 0) negb = CxBits<float2>::sign;
  }
  const float2 *L = op.links + (int64_t)MU * 9 * op.sites;
  float2 pf[12], pb[12], uf[9], ub[9];
  // spinors with ordinary loads: the run rewrites them between barriers
  const float2 *qf = in + ((int64_t)nf >> 5) * 384 + (nf & 31), *qb = in + ((int64_t)nb >> 5) * 384 + (nb & 31);
#pragma unroll
  for (int k = 0; k < 12; ++k) pf[k] = qf[32 * k];
#pragma unroll
  for (int k = 0; k < 9; ++k) uf[k] = __ldg(L + (int64_t)k * op.sites + s);
#pragma unroll
  for (int k = 0; k < 12; ++k) pb[k] = qb[32 * k];
#pragma unroll
  for (int k = 0; k < 9; ++k) ub[k] = __ldg(L + (int64_t)k * op.sites + nb);
  hop_pair_r<MU, S>(pf, uf, negf, pb, ub, negb, acc);
}

// hopping sums of the 32-site tile starting at s0 into sacc (zeros for padding
// sites), by the four tile warps (ends with their named barrier)
template <int S>
SEED_DEV void wilson_tile32(const WilsonOp32 &op, const float2 *in, int64_t s0, float (*sacc)[24][kWilsonSites + 1]) {
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const int64_t s = s0 + lane;
  float2 acc[12];
  if (s < op.sites) {
    switch (mu) {
      case 0: site_mu32<0, S>(op, in, s, acc); break;
      case 1: site_mu32<1, S>(op, in, s, acc); break;
      case 2: site_mu32<2, S>(op, in, s, acc); break;
      default: site_mu32<3, S>(op, in, s, acc); break;
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
  tile_warps_sync();
}
SEED_DEV float2 tile_sum32(float (*sacc)[24][kWilsonSites + 1], int cc, int sl) {
  return make_float2(((sacc[0][2 * cc][sl] + sacc[1][2 * cc][sl]) + sacc[2][2 * cc][sl]) + sacc[3][2 * cc][sl],
                     ((sacc[0][2 * cc + 1][sl] + sacc[1][2 * cc + 1][sl]) + sacc[2][2 * cc + 1][sl]) +
                         sacc[3][2 * cc + 1][sl]);
}

// Resident form, as in the FP64 run: s_lnk32[(mu * 18 + k) * 32 + lane] holds
// the tile's links, s_vec32[slot * 384 + o] its elements of f, t, w_i, x^1
// (the FP32 correction), v_i and v_{i-1} (o = the element's offset in the
// tile, the same as in the tiled vectors).
constexpr size_t kResSmemBytes32 = (size_t)(kResLinks + 6 * kResTile) * sizeof(float2);

template <int MU, int S>
SEED_DEV void site_mu32_res(const float2 *in, int32_t nf, int32_t nb, unsigned negf, unsigned negb,
                            const float2 *su, float2 (&acc)[12]) {
  float2 pf[12], pb[12], uf[9], ub[9];
  const float2 *qf = in + ((int64_t)nf >> 5) * 384 + (nf & 31), *qb = in + ((int64_t)nb >> 5) * 384 + (nb & 31);
#pragma unroll
  for (int k = 0; k < 12; ++k) pf[k] = qf[32 * k];
#pragma unroll
  for (int k = 0; k < 12; ++k) pb[k] = qb[32 * k];
#pragma unroll
  for (int k = 0; k < 9; ++k) uf[k] = su[k * 32];
#pragma unroll
  for (int k = 0; k < 9; ++k) ub[k] = su[(9 + k) * 32];
  hop_pair_r<MU, S>(pf, uf, negf, pb, ub, negb, acc);
}

template <int S>
SEED_DEV void wilson_tile32_res(const float2 *in, int32_t nf, int32_t nb, unsigned negf, unsigned negb, bool live,
                                const float2 *s_lnk, float (*sacc)[24][kWilsonSites + 1]) {
  const int lane = threadIdx.x & 31, mu = threadIdx.x >> 5;
  const float2 *su = s_lnk + mu * 18 * 32 + lane;
  float2 acc[12];
  if (live) {
    switch (mu) {
      case 0: site_mu32_res<0, S>(in, nf, nb, negf, negb, su, acc); break;
      case 1: site_mu32_res<1, S>(in, nf, nb, negf, negb, su, acc); break;
      case 2: site_mu32_res<2, S>(in, nf, nb, negf, negb, su, acc); break;
      default: site_mu32_res<3, S>(in, nf, nb, negf, negb, su, acc); break;
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
  tile_warps_sync();
}

// tpart: 12 x tiles doubles, per tile warp as in k_seed_run_wilson.  Five
// warps: four tile warps and the scalar warp, which reduces the partials and
// runs the recurrence's scalar code while the tile warps compute the next
// stencil (the same overlap as the FP64 run).
__global__ void __launch_bounds__(PTW, 1) k_seed_run_wilson32(SeedBufs<float2> b, WilsonOp32 op, float2 *tbuf,
                                                            GridSync g, double *tpart, int i_stop) {
  __shared__ float sacc[4][24][kWilsonSites + 1];
  __shared__ LocalSeed L;
  extern __shared__ float2 s_dyn32[];
  const int tiles = (int)(b.n / 384);
  const float mk = (float)(-op.kappa);
  double *part1 = tpart, *part2 = tpart + 8 * (int64_t)tiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool tw = warp < 4;
  unsigned epoch = 0;
  local_load(b, L);
  const SeedBufs<float2> bl = local_bufs(b, L);
  Owners own;
  if (!register_owner(g, epoch, own)) return;
  float2 *const X = reinterpret_cast<float2 *>(b.call->X);
  const int first_tile = own.rank >= 0 && own.rank < tiles ? own.rank : -1;
  const bool res = tiles <= own.count && first_tile >= 0;
  float2 *const s_lnk = s_dyn32;
  float2 *const s_vec = s_dyn32 + kResLinks;
  int32_t r_nf = 0, r_nb = 0;
  unsigned r_negf = 0u, r_negb = 0u;
  const int64_t r_site = (int64_t)(first_tile >= 0 ? first_tile : 0) * kWilsonSites + lane;
  const bool r_live = r_site < op.sites;
  if (res) {
    const int64_t e0 = (int64_t)first_tile * kResTile;
    const int i0 = L.st.i;
    if (tw && r_live) {
      const int mu = warp;
      r_nf = __ldg(op.nbr + 8 * r_site + 2 * mu);
      r_nb = __ldg(op.nbr + 8 * r_site + 2 * mu + 1);
      if (mu == 3 && op.bc_t) {
        const int64_t t = r_site / ((int64_t)op.dims[0] * op.dims[1] * op.dims[2]);
        if (t == op.dims[3] - 1) r_negf = CxBits<float2>::sign;
        if (t == 0) r_negb = CxBits<float2>::sign;
      }
      const float2 *Lk = op.links + (int64_t)mu * 9 * op.sites;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        s_lnk[(mu * 18 + k) * 32 + lane] = __ldg(Lk + (int64_t)k * op.sites + r_site);
        s_lnk[(mu * 18 + 9 + k) * 32 + lane] = __ldg(Lk + (int64_t)k * op.sites + r_nb);
      }
    }
    const float2 *vprev = b.V + (int64_t)(i0 > 1 ? i0 - 2 : 0) * b.ldv;
    for (int o = threadIdx.x; o < kResTile; o += PTW) {
      const int64_t e = e0 + o;
      s_vec[kResF * kResTile + o] = b.f[e];
      s_vec[kResW * kResTile + o] = i0 > 1 ? b.w[e] : make_float2(0.f, 0.f);
      s_vec[kResX * kResTile + o] = X[e];
      s_vec[(kResV + ((i0 - 1) & 1)) * kResTile + o] = i0 > 1 ? vprev[e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
  }
  bool pending_beta = false;
  for (;;) {
    // ---- phase 1 of step i, overlapped with the end of step i-1 ----
    {
      const int ip = L.st.i + (pending_beta ? 1 : 0);
      const bool go = L.st.active && ip < i_stop && (b.Wb == nullptr || ip - L.st.blk0 < kSeedBlock);
      __syncthreads();                 // everyone has read L.st before the scalar warp updates it
      if (tw && go && first_tile >= 0) {
        if (res) wilson_tile32_res<+1>(b.f, r_nf, r_nb, r_negf, r_negb, r_live, s_lnk, sacc);
        else wilson_tile32<+1>(op, b.f, (int64_t)first_tile * kWilsonSites, sacc);
      }
      if (!tw && pending_beta) {
        const double ss = warp_sum_short<kScalarSumPer>(part2, 4 * tiles);
        if (threadIdx.x == PT) {
          if (bl.Wb != nullptr) L.st.w_last = L.st.i;
          seed_finish<float2, false>(bl, ss);
        }
      }
      __syncthreads();
      pending_beta = false;
    }
    const int i = L.st.i;
    if (!L.st.active || i >= i_stop) break;
    if (block_full(b, L, i)) break;
    const float inv_b = (float)L.st.inv_beta;
    const float bp = (float)((i > 1) ? L.st.beta_prev : 0.0);
    float2 *vi = b.V + (int64_t)(i - 1) * b.ldv;
    const float2 *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * b.ldv;
    float2 *const s_vi = s_vec + (kResV + (i & 1)) * kResTile;
    float2 *const s_vm = s_vec + (kResV + ((i - 1) & 1)) * kResTile;
    // phase 1 epilogue: v_i, t = D v_i, partials of ||t||^2 and Re(v_i^H v_{i-1})
    if (first_tile >= 0) {
      for (int tile = first_tile; tile < tiles; tile += own.count) {
        if (tile != first_tile && tw) wilson_tile32<+1>(op, b.f, (int64_t)tile * kWilsonSites, sacc);
        if (tw) {
          float ptt = 0.f, pvm = 0.f;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int o = threadIdx.x + PT * k, cc = o >> 5, sl = o & 31;
            const int64_t e = (int64_t)tile * 384 + o;
            const float2 sum = tile_sum32(sacc, cc, sl);
            const float2 fe = res ? s_vec[kResF * kResTile + o] : b.f[e];
            const float2 v = make_float2(inv_b * fe.x, inv_b * fe.y);
            vi[e] = v;
            const float2 t = make_float2(fmaf(mk, inv_b * sum.x, v.x), fmaf(mk, inv_b * sum.y, v.y));
            tbuf[e] = t;
            if (res) {
              s_vi[o] = v;
              s_vec[kResT * kResTile + o] = t;
            }
            ptt = fmaf(t.y, t.y, fmaf(t.x, t.x, ptt));
            if (i > 1) {
              const float2 m = res ? s_vm[o] : vm[e];
              pvm = fmaf(v.y, m.y, fmaf(v.x, m.x, pvm));
            }
          }
          const double2 ws = warp_sum_pair((double)ptt, (double)pvm);
          if (lane == 0) {
            part1[2 * (4 * tile + warp)] = ws.x;
            part1[2 * (4 * tile + warp) + 1] = ws.y;
          }
        }
        if (tile + own.count < tiles) __syncthreads();   // sacc is reused by the next tile
      }
    }
    if (!grid_sync(g, epoch)) return;
    // ---- phase 2: u = D^H t overlapped with alpha_i and the LU update's scalars ----
    if (tw && first_tile >= 0) {
      if (res) wilson_tile32_res<-1>(tbuf, r_nf, r_nb, r_negf, r_negb, r_live, s_lnk, sacc);
      else wilson_tile32<-1>(op, tbuf, (int64_t)first_tile * kWilsonSites, sacc);
    }
    if (!tw) {
      const double2 s2 = warp_sum_short_pairs<kScalarSumPer>(part1, 4 * tiles);
      const double a = i > 1 ? s2.x - L.st.beta_prev * s2.y : s2.x;
      if (threadIdx.x == PT) seed_step_scalars<float2, false>(bl, i, a, nullptr);
    }
    __syncthreads();
    if (!L.st.active) break;   // delta_i <= 0
    const float a = (float)L.st.alpha, zeta = (float)L.st.zeta, inv_d = (float)L.st.inv_delta;
    float2 *const wcol = b.Wb != nullptr ? b.Wb + (int64_t)(i - L.st.blk0) * b.ldv : nullptr;
    if (first_tile >= 0) {
      for (int tile = first_tile; tile < tiles; tile += own.count) {
        if (tile != first_tile && tw) wilson_tile32<-1>(op, tbuf, (int64_t)tile * kWilsonSites, sacc);
        if (tw) {
          float pff = 0.f;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int o = threadIdx.x + PT * k, cc = o >> 5, sl = o & 31;
            const int64_t e = (int64_t)tile * 384 + o;
            const float2 sum = tile_sum32(sacc, cc, sl);
            const float2 tv = res ? s_vec[kResT * kResTile + o] : tbuf[e];
            const float2 v = res ? s_vi[o] : vi[e];
            float2 f = make_float2(fmaf(mk, sum.x, tv.x), fmaf(mk, sum.y, tv.y));
            if (i > 1) {
              const float2 m = res ? s_vm[o] : vm[e];
              f = make_float2(fmaf(-bp, m.x, f.x), fmaf(-bp, m.y, f.y));
            }
            f = make_float2(fmaf(-a, v.x, f.x), fmaf(-a, v.y, f.y));
            float2 w;
            if (i > 1) {
              const float2 wp = res ? s_vec[kResW * kResTile + o] : b.w[e];
              w = make_float2(inv_d * fmaf(-bp, wp.x, v.x), inv_d * fmaf(-bp, wp.y, v.y));
            } else {
              w = make_float2(inv_d * v.x, inv_d * v.y);
            }
            b.f[e] = f;
            if (wcol != nullptr) wcol[e] = w;
            const float2 x = res ? s_vec[kResX * kResTile + o] : X[e];
            const float2 xn = make_float2(fmaf(zeta, w.x, x.x), fmaf(zeta, w.y, x.y));
            if (res) {
              s_vec[kResF * kResTile + o] = f;
              s_vec[kResW * kResTile + o] = w;
              s_vec[kResX * kResTile + o] = xn;
            } else {
              b.w[e] = w;
              X[e] = xn;
            }
            pff = fmaf(f.y, f.y, fmaf(f.x, f.x, pff));
          }
          const double ws = warp_sum((double)pff);
          if (lane == 0) part2[4 * tile + warp] = ws;
        }
        if (tile + own.count < tiles) __syncthreads();
      }
    }
    if (!grid_sync(g, epoch)) return;
    pending_beta = true;               // beta_i and the stopping test run with the next stencil
  }
  if (res) {   // x^1 (FP32 correction) and w_i back to global memory
    __syncthreads();
    const int64_t e0 = (int64_t)first_tile * kResTile;
    for (int o = threadIdx.x; o < kResTile; o += PTW) {
      X[e0 + o] = s_vec[kResX * kResTile + o];
      b.w[e0 + o] = s_vec[kResW * kResTile + o];
    }
  }
  if (tw) seed_leave<float2>(b, L, b.f, i_stop);
  local_store(b, L);
}

// ---------------------------------------------------------------------------
// Site form of the FP32 run for lattices with many more sites than threads
// of one wave (from 65536 sites): every thread takes whole sites (all eight
// hops of a site, as the FP32 operator kernel does there), so that each link
// is read once per site and phase and no partial sums cross shared memory;
// sites blockIdx.x * 448 + t, then every 448 * gridDim.x (tiled vectors:
// component k of site s at ((s / 32) 12 + k) 32 + s mod 32); thread 448
// starts the scalar warp.  Each thread accumulates its sites' partial sums in FP64, the
// block adds its warp totals in warp order into one partial per block
// (reproducible grouping).  The first site's stencil of each phase runs
// while the scalar warp works.
// ---------------------------------------------------------------------------
constexpr int kBlockSumPer = 8;     // one partial per block: 256 blocks in one pass
constexpr int kSiteThreads32 = 448;   // 14 site warps + the scalar warp: 15 warps, at most 4 per sub-partition, 128 registers

template <int MU, int S>
SEED_DEV void site32_dir(const WilsonOp32 &op, const float2 *in, int64_t s, int32_t nf, int32_t nb, unsigned negf,
                         unsigned negb, float2 (&acc)[12]) {
  const float2 *L = op.links + (int64_t)MU * 9 * op.sites;
  {
    float2 u[9], p[12];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldcg(L + (int64_t)k * op.sites + s);
    const float2 *q = in + ((int64_t)nf >> 5) * 384 + (nf & 31);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = q[32 * k];
    hop_r<MU, S, true, MU == 0>(p, u, negf, acc);
  }
  {
    float2 u[9], p[12];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldcg(L + (int64_t)k * op.sites + nb);
    const float2 *q = in + ((int64_t)nb >> 5) * 384 + (nb & 31);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = q[32 * k];
    hop_r<MU, -S, false, false>(p, u, negb, acc);
  }
}

// the eight hops of site s (zero for padding sites)
template <int S>
SEED_DEV void site32_hops(const WilsonOp32 &op, const float2 *in, int64_t s, float2 (&acc)[12]) {
  if (s >= op.sites) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = make_float2(0.f, 0.f);
    return;
  }
  const int4 *q = reinterpret_cast<const int4 *>(op.nbr + 8 * s);
  const int4 a = __ldg(q), c = __ldg(q + 1);
  unsigned negf = 0u, negb = 0u;
  if (op.bc_t) {
    const int64_t t = s / ((int64_t)op.dims[0] * op.dims[1] * op.dims[2]);
    if (t == op.dims[3] - 1) negf = CxBits<float2>::sign;
    if (t == 0) negb = CxBits<float2>::sign;
  }
  site32_dir<0, S>(op, in, s, a.x, a.y, 0u, 0u, acc);
  site32_dir<1, S>(op, in, s, a.z, a.w, 0u, 0u, acc);
  site32_dir<2, S>(op, in, s, c.x, c.y, 0u, 0u, acc);
  site32_dir<3, S>(op, in, s, c.z, c.w, negf, negb, acc);
}

// tpart: 3 x blocks doubles (per block: the phase-1 pair, then the phase-2 norm)
__global__ void __launch_bounds__(kSiteThreads32 + 32, 1) k_seed_run_wilson32s(SeedBufs<float2> b, WilsonOp32 op,
                                                                                float2 *tbuf, GridSync g,
                                                                                double *tpart, int i_stop) {
  constexpr int kW = kSiteThreads32 / 32;   // site warps
  __shared__ LocalSeed L;
  __shared__ double s_wp[kW][2];
  const int64_t padded = b.n / 12;          // sites including the padding of the last tile
  const float mk = (float)(-op.kappa);
  const int nb = gridDim.x;
  double *part1 = tpart, *part2 = tpart + 2 * (int64_t)nb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool sw = warp < kW;                // site warp; warp kW is the scalar warp
  const int64_t stride = (int64_t)nb * kSiteThreads32;
  const int64_t first = sw ? (int64_t)blockIdx.x * kSiteThreads32 + threadIdx.x : padded;
  unsigned epoch = 0;
  local_load(b, L);
  const SeedBufs<float2> bl = local_bufs(b, L);
  float2 *const X = reinterpret_cast<float2 *>(b.call->X);
  bool pending_beta = false;
  for (;;) {
    float2 acc[12];
    // ---- phase 1 of step i, overlapped with the end of step i-1 ----
    {
      const int ip = L.st.i + (pending_beta ? 1 : 0);
      const bool go = L.st.active && ip < i_stop && (b.Wb == nullptr || ip - L.st.blk0 < kSeedBlock);
      __syncthreads();                 // everyone has read L.st before the scalar warp updates it
      if (go && first < padded) site32_hops<+1>(op, b.f, first, acc);
      if (!sw && pending_beta) {
        const double ss = warp_sum_short<kBlockSumPer>(part2, nb);
        if (threadIdx.x == kSiteThreads32) {
          if (bl.Wb != nullptr) L.st.w_last = L.st.i;
          seed_finish<float2, false>(bl, ss);
        }
      }
      __syncthreads();
      pending_beta = false;
    }
    const int i = L.st.i;
    if (!L.st.active || i >= i_stop) break;
    if (block_full(b, L, i)) break;
    const float inv_b = (float)L.st.inv_beta;
    const float bp = (float)((i > 1) ? L.st.beta_prev : 0.0);
    float2 *vi = b.V + (int64_t)(i - 1) * b.ldv;
    const float2 *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * b.ldv;
    // phase 1 epilogue: v_i, t = D v_i, partials of ||t||^2 and Re(v_i^H v_{i-1})
    double att = 0.0, avm = 0.0;
    for (int64_t s = first; s < padded; s += stride) {
      if (s != first) site32_hops<+1>(op, b.f, s, acc);
      const int64_t e0 = (s >> 5) * 384 + (s & 31);
      float ptt = 0.f, pvm = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int64_t e = e0 + 32 * k;
        const float2 fe = b.f[e];
        const float2 v = make_float2(inv_b * fe.x, inv_b * fe.y);
        vi[e] = v;
        const float2 t = make_float2(fmaf(mk, inv_b * acc[k].x, v.x), fmaf(mk, inv_b * acc[k].y, v.y));
        tbuf[e] = t;
        ptt = fmaf(t.y, t.y, fmaf(t.x, t.x, ptt));
        if (i > 1) {
          const float2 m = vm[e];
          pvm = fmaf(v.y, m.y, fmaf(v.x, m.x, pvm));
        }
      }
      att += (double)ptt;
      avm += (double)pvm;
    }
    if (sw) {
      const double2 ws = warp_sum_pair(att, avm);
      if (lane == 0) {
        s_wp[warp][0] = ws.x;
        s_wp[warp][1] = ws.y;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < kW; ++w) {
        s0 += s_wp[w][0];
        s1 += s_wp[w][1];
      }
      part1[2 * blockIdx.x] = s0;
      part1[2 * blockIdx.x + 1] = s1;
    }
    if (!grid_sync(g, epoch)) return;
    // ---- phase 2: u = D^H t overlapped with alpha_i and the LU update's scalars ----
    if (first < padded) site32_hops<-1>(op, tbuf, first, acc);
    if (!sw) {
      const double2 s2 = warp_sum_short_pairs<kBlockSumPer>(part1, nb);
      const double a = i > 1 ? s2.x - L.st.beta_prev * s2.y : s2.x;
      if (threadIdx.x == kSiteThreads32) seed_step_scalars<float2, false>(bl, i, a, nullptr);
    }
    __syncthreads();
    if (!L.st.active) break;   // delta_i <= 0
    const float a = (float)L.st.alpha, zeta = (float)L.st.zeta, inv_d = (float)L.st.inv_delta;
    float2 *const wcol = b.Wb != nullptr ? b.Wb + (int64_t)(i - L.st.blk0) * b.ldv : nullptr;
    double aff = 0.0;
    for (int64_t s = first; s < padded; s += stride) {
      if (s != first) site32_hops<-1>(op, tbuf, s, acc);
      const int64_t e0 = (s >> 5) * 384 + (s & 31);
      float pff = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int64_t e = e0 + 32 * k;
        const float2 tv = tbuf[e], v = vi[e];
        float2 f = make_float2(fmaf(mk, acc[k].x, tv.x), fmaf(mk, acc[k].y, tv.y));
        if (i > 1) {
          const float2 m = vm[e];
          f = make_float2(fmaf(-bp, m.x, f.x), fmaf(-bp, m.y, f.y));
        }
        f = make_float2(fmaf(-a, v.x, f.x), fmaf(-a, v.y, f.y));
        float2 w;
        if (i > 1) {
          const float2 wp = b.w[e];
          w = make_float2(inv_d * fmaf(-bp, wp.x, v.x), inv_d * fmaf(-bp, wp.y, v.y));
        } else {
          w = make_float2(inv_d * v.x, inv_d * v.y);
        }
        b.f[e] = f;
        b.w[e] = w;
        if (wcol != nullptr) wcol[e] = w;
        const float2 x = X[e];
        X[e] = make_float2(fmaf(zeta, w.x, x.x), fmaf(zeta, w.y, x.y));
        pff = fmaf(f.y, f.y, fmaf(f.x, f.x, pff));
      }
      aff += (double)pff;
    }
    if (sw) {
      const double ws = warp_sum(aff);
      if (lane == 0) s_wp[warp][0] = ws;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0.0;
      for (int w = 0; w < kW; ++w) s0 += s_wp[w][0];
      part2[blockIdx.x] = s0;
    }
    if (!grid_sync(g, epoch)) return;
    pending_beta = true;
  }
  local_store(b, L);
}

// Phase 3 of the CSR run: f -= alpha_i v_i, w_i (also into column i - blk0 of
// Wb), x^1 and ||f||^2; one value per block, reduced in block order by every
// block after the barrier, then the end of the step.
template <class T>
SEED_DEV bool seed_update_step(const SeedBufs<T> &b, const SeedBufs<T> &bl, T *f, const T *vi, int i, LocalSeed &L,
                               const GridSync &g, unsigned &epoch, double *bpart, double *s_red) {
  const double a = L.st.alpha, zeta = L.st.zeta, inv_d = L.st.inv_delta;
  const double bp = (i > 1) ? L.st.beta_prev : 0.0;
  T *const X = reinterpret_cast<T *>(b.call->X);
  T *const wcol = b.Wb != nullptr ? b.Wb + (int64_t)(i - L.st.blk0) * b.ldv : nullptr;
  typename Sc<T>::A acc = 0;
  for (int64_t e = (int64_t)blockIdx.x * PT + threadIdx.x; e < b.n; e += (int64_t)gridDim.x * PT) {
    const T v = __ldcg(vi + e), f0 = __ldcg(f + e), x0 = __ldcg(X + e);
    const T wp = (i > 1) ? __ldcg(b.w + e) : Sc<T>::zero();
    const T fe = Sc<T>::axpy(-a, v, f0);
    const T we = (i > 1) ? Sc<T>::scale(inv_d, Sc<T>::axpy(-bp, wp, v)) : Sc<T>::scale(inv_d, v);
    f[e] = fe;
    b.w[e] = we;
    if (wcol != nullptr) wcol[e] = we;
    X[e] = Sc<T>::axpy(zeta, we, x0);
    acc = Sc<T>::nrm2(fe, acc);
  }
  double vv[1] = {(double)acc};
  block_sum<1, PT>(vv, s_red);
  if (threadIdx.x == 0) bpart[blockIdx.x] = vv[0];
  return seed_beta_step<T>(bl, bpart, gridDim.x, i, L, g, epoch);
}

// real CSR operator, two barriers per step: the apply reads f_cur (two
// buffers alternate, since a row reads other rows' entries while writing its
// own); alpha_i from block partials; then the update.  T = double, or float
// for the mixed-precision path (FP32 matrix values and vectors; per-thread
// sums in FP32, block and grid sums and every scalar in FP64).
template <class T>
__global__ void __launch_bounds__(PT) k_seed_run_csr(SeedBufs<T> b, CsrOpT<T> op, T *f2, GridSync g, double *bpart,
                                                      int i_stop) {
  __shared__ double s_red[PT / 32];
  __shared__ LocalSeed L;
  unsigned epoch = 0;
  int par = 0;
  local_load(b, L);
  const SeedBufs<T> bl = local_bufs(b, L);
  for (;;) {
    const int i = L.st.i;
    if (!L.st.active || i >= i_stop) break;
    if (block_full(b, L, i)) break;
    const T inv_b = (T)L.st.inv_beta;
    const T bp = (T)((i > 1) ? L.st.beta_prev : 0.0);
    T *fc = par ? f2 : b.f, *fn = par ? b.f : f2;
    T *vi = b.V + (int64_t)(i - 1) * b.ldv;
    const T *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * b.ldv;
    T apart = 0;
    for (int64_t r = (int64_t)blockIdx.x * PT + threadIdx.x; r < b.n; r += (int64_t)gridDim.x * PT) {
      const int32_t k0 = __ldg(op.row_ptr + r), k1 = __ldg(op.row_ptr + r + 1);
      T sum = 0;
      for (int32_t k = k0; k < k1; ++k) sum = fma(__ldg(op.vals + k), fc[__ldg(op.col_idx + k)], sum);
      const T v = inv_b * fc[r];
      vi[r] = v;
      T u = inv_b * sum;
      if (i > 1) u = fma(-bp, vm[r], u);
      fn[r] = u;
      apart = fma(v, u, apart);
    }
    // alpha partials apart from the update partials (every block reads them
    // after the barrier, while a faster block may already be writing its
    // update partial)
    double *apartials = bpart + (int64_t)gridDim.x * 32;
    {
      double vv[1] = {(double)apart};
      block_sum<1, PT>(vv, s_red);
      if (threadIdx.x == 0) apartials[blockIdx.x] = vv[0];   // by blockIdx: fixed order
    }
    if (!seed_alpha_step<T>(bl, apartials, gridDim.x, 1, false, i, L, g, epoch)) return;
    if (!L.st.active) break;
    if (!seed_update_step<T>(b, bl, fn, vi, i, L, g, epoch, bpart, s_red)) return;
    par ^= 1;
  }
  seed_leave<T>(b, L, par ? f2 : b.f, i_stop);
  local_store(b, L);
}

// ---------------------------------------------------------------------------
// Small real CSR problems that reorthogonalize every few steps (Sec. 3 with a
// reorthogonalization frequency of 1 to 7, where the seeding of systems 2..p
// runs in its streaming form): every step -- the apply, alpha_i and
// g^j = v_i^H r_0^j, the LU update with x^1 += zeta_i w_i and
// x^j += eta^j w_i, and on reorthogonalizing steps the classical Gram-Schmidt
// passes over V_{<i}, the renormalization of v_i and the projections of f on
// it -- in one cooperative launch, instead of 10 to 14 kernels per step.
//
// Block b owns rows [b RB, (b + 1) RB) (RB = 16 or 32, so that the grid spans
// most SMs even for n = 4096); thread t < RB holds row b RB + t in every row
// phase.  The products with V_{<i} run with one thread per basis column
// (columns t, t + PT, ...): a thread loads its column's RB rows (one or two
// 128-byte lines), so the whole grid streams V with many loads in flight.
//   H = V_{<i}^H [v_i f]: per block and column the dot products over the
//   block's rows, written to hpart[(2 c + v) G + b]; after a barrier block b
//   sums the values [2 k b / G, 2 k (b + 1) / G) over the blocks in block order
//   into H; after a second barrier each thread adds x_rc H_c of its columns
//   into 2 RB row sums, the block combines them (warp reduce-scatter, then the
//   warps in order), and the rows subtract them.  When a second pass follows,
//   its dot products use the same lines again (from L1) in the same phase.
// Scalar sums (alpha_i with the g^j, ||v_i||^2, v_i^H f, ||f||^2): one row of
// block partials per block in one of two alternating regions -- a block that
// has run ahead writes the other region while slower blocks still read this
// one -- reduced by every block in block order, so the blocks' shared-memory
// copies of the recurrence's scalars stay identical.
// ---------------------------------------------------------------------------
constexpr int kRunRegion = 32;                 // doubles per block in a scalar partial region
constexpr int kRunMaxRhs = kReorthRunMaxRhs;   // alpha_i and g^2..g^16 in one region row

// block sums of v[0..nv) into row[0..nv) (warp sums, then the four warps in order)
template <int NV>
SEED_DEV void block_row(const double (&v)[NV], int nv, double *row, double (*s)[kRunRegion]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    if (q < nv) {
      const double t = warp_sum(v[q]);
      if (lane == 0) s[warp][q] = t;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < nv)
    row[threadIdx.x] = ((s[0][threadIdx.x] + s[1][threadIdx.x]) + s[2][threadIdx.x]) + s[3][threadIdx.x];
}

// after the barrier: S[q] = sum over blocks (in block order) of region[b * kRunRegion + q], q < nv
SEED_DEV void reduce_region(const double *region, int nv, double *S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < nv; q += PT / 32) {
    const double t = warp_sum_partials(region, gridDim.x, kRunRegion, q);
    if (lane == 0) S[q] = t;
  }
  __syncthreads();
}

// hpart[(2 c + v) G + b] = sum over the block's rows r of V[c][row0 + r] y_v[r], c < k
template <int RB>
SEED_DEV void col_dots(const double *V, int64_t ldv, int64_t row0, int rows, int k, const double (*y)[RB],
                       double *hpart) {
  const int G = gridDim.x;
  for (int c = threadIdx.x; c < k; c += PT) {
    const double *vc = V + (int64_t)c * ldv + row0;
    double x[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) x[r] = r < rows ? vc[r] : 0.0;
    double hv = 0.0, hf = 0.0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      hv = fma(x[r], y[0][r], hv);
      hf = fma(x[r], y[1][r], hf);
    }
    hpart[(int64_t)(2 * c) * G + blockIdx.x] = hv;
    hpart[(int64_t)(2 * c + 1) * G + blockIdx.x] = hf;
  }
}

// H[q] = sum over blocks (block order) of hpart[q G + b], for this block's slice of q < 2k
SEED_DEV void slice_reduce(const double *hpart, int k, double *H) {
  const int G = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q0 = (int)((int64_t)2 * k * blockIdx.x / G), q1 = (int)((int64_t)2 * k * (blockIdx.x + 1) / G);
  for (int q = q0 + warp; q < q1; q += PT / 32) {
    const double t = warp_sum_partials(hpart + (int64_t)q * G, G, 1, 0);
    if (lane == 0) H[q] = t;
  }
}

// sub[v][r] = sum over c < k of V[c][row0 + r] H[2 c + v]: thread (r, g) of the
// block (r = t mod RB, g = t / RB) sums the columns c = g, g + G, ... (G = PT /
// RB groups) of row r, then each output adds its G group sums in group order --
// G - 1 FP64 adds per output instead of a 31-add warp reduce-scatter per lane
// (FP64 adds run at 2 per clock per SM on this part).
template <int RB>
SEED_DEV void rows_times_h(const double *V, int64_t ldv, int64_t row0, int rows, int k, const double *H,
                           double (*sub)[RB], double (*sred)[2 * RB]) {
  constexpr int kGroups = PT / RB;
  const int r = threadIdx.x % RB, grp = threadIdx.x / RB;
  double pv = 0.0, pf = 0.0;
  if (r < rows) {
    const double *vr = V + row0 + r;
#pragma unroll 4
    for (int c = grp; c < k; c += kGroups) {
      const double x = vr[(int64_t)c * ldv];
      pv = fma(x, __ldcg(H + 2 * c), pv);
      pf = fma(x, __ldcg(H + 2 * c + 1), pf);
    }
  }
  sred[grp][r] = pv;
  sred[grp][RB + r] = pf;
  __syncthreads();
  if ((int)threadIdx.x < 2 * RB) {
    const int q = threadIdx.x;
    double t = sred[0][q];
#pragma unroll
    for (int g2 = 1; g2 < kGroups; ++g2) t += sred[g2][q];
    sub[q / RB][q % RB] = t;
  }
  __syncthreads();
}

template <int RB>
__global__ void __launch_bounds__(PT) k_seed_run_csr_reorth(SeedBufs<double> b, CsrOp op, double *f2, GridSync g,
                                                            double *bpart, double *hpart, double *H, int freq,
                                                            int passes, int i_stop) {
  static_assert(2 * RB % 32 == 0 && 2 * RB <= PT, "rows per block");
  __shared__ double s_w[PT / 32][kRunRegion];
  __shared__ double s_sum[kRunRegion];
  __shared__ double2 s_g[kRunMaxRhs];
  __shared__ double2 s_eta[kRunMaxRhs];
  __shared__ double s_y[2][RB];
  __shared__ double s_sub[2][RB];
  __shared__ double s_red[PT / RB][2 * RB];
  __shared__ LocalSeed L;
  unsigned epoch = 0;
  int par = 0, reg = 0;
  local_load(b, L);
  const int nr = b.nrhs;   // <= kRunMaxRhs (checked by the host)
  for (int j = threadIdx.x; j < nr; j += PT) s_eta[j] = b.eta[j];
  __syncthreads();
  SeedBufs<double> bl = local_bufs(b, L);
  bl.eta = s_eta;
  const int G = gridDim.x;
  const int64_t n = b.n, ldv = b.ldv;
  const int64_t row0 = (int64_t)blockIdx.x * RB;
  const int rows = (int)(n - row0 < RB ? n - row0 : RB);   // >= 1: the grid is ceil(n / RB)
  const int64_t e = row0 + threadIdx.x;                     // this thread's row in the row phases
  const bool own = (int)threadIdx.x < rows;
  double *const X = reinterpret_cast<double *>(b.call->X);
  const int64_t ldx = b.call->ldx;
  // this thread's matrix row, held in registers for the whole run when it has
  // at most kRowCache entries (every step's apply then waits on one round trip)
  constexpr int kRowCache = 8;
  int32_t k0 = 0, k1 = 0, rc_col[kRowCache];
  double rc_val[kRowCache];
  if (own) {
    k0 = __ldg(op.row_ptr + e);
    k1 = __ldg(op.row_ptr + e + 1);
  }
  const bool cached = k1 - k0 <= kRowCache;
#pragma unroll
  for (int q = 0; q < kRowCache; ++q) {
    const bool in = cached && q < k1 - k0;
    rc_col[q] = in ? __ldg(op.col_idx + k0 + q) : (int32_t)e;
    rc_val[q] = in ? __ldg(op.vals + k0 + q) : 0.0;
  }
  auto region = [&]() {   // the next scalar partial region (alternating)
    double *r = bpart + (int64_t)reg * G * kRunRegion;
    reg ^= 1;
    return r;
  };
  for (;;) {
    const int i = L.st.i;
    if (!L.st.active || i >= i_stop) break;
    const double inv_b = L.st.inv_beta;
    const double bp = (i > 1) ? L.st.beta_prev : 0.0;
    const double *fc = par ? f2 : b.f;
    double *fn = par ? b.f : f2;
    double *vi = b.V + (int64_t)(i - 1) * ldv;
    const double *vm = b.V + (int64_t)(i > 1 ? i - 2 : 0) * ldv;
    // ---- v_i = f / beta_{i-1}; f = A v_i - beta_{i-1} v_{i-1}; alpha_i and g^j ----
    double acc[kRunMaxRhs];
#pragma unroll
    for (int q = 0; q < kRunMaxRhs; ++q) acc[q] = 0.0;
    double v = 0.0, fe = 0.0;
    if (own) {
      double sum = 0.0;
      if (cached) {
        double xv[kRowCache];
#pragma unroll
        for (int q = 0; q < kRowCache; ++q) xv[q] = q < k1 - k0 ? __ldcg(fc + rc_col[q]) : 0.0;
#pragma unroll
        for (int q = 0; q < kRowCache; ++q)
          if (q < k1 - k0) sum = fma(rc_val[q], xv[q], sum);
      } else {
        for (int32_t q = k0; q < k1; ++q) sum = fma(__ldg(op.vals + q), __ldcg(fc + __ldg(op.col_idx + q)), sum);
      }
      v = inv_b * __ldcg(fc + e);
      vi[e] = v;
      double u = inv_b * sum;
      if (i > 1) u = fma(-bp, vm[e], u);
      fe = u;
      acc[0] = v * u;
#pragma unroll
      for (int q = 1; q < kRunMaxRhs; ++q)
        if (q < nr) acc[q] = v * b.R0[(int64_t)(q - 1) * b.ldr + e];
    }
    {
      double *r = region();
      block_row<kRunMaxRhs>(acc, nr, r + (int64_t)blockIdx.x * kRunRegion, s_w);
      if (!grid_sync(g, epoch)) return;
      reduce_region(r, nr, s_sum);
    }
    if (threadIdx.x == 0) {
      for (int j = 1; j < nr; ++j) s_g[j] = c2(s_sum[j], 0.0);
      seed_step_scalars<double, false>(bl, i, s_sum[0], s_g);
    }
    __syncthreads();
    if (!L.st.active) break;   // delta_i <= 0
    // ---- f -= alpha_i v_i; w_i; x^1 += zeta_i w_i; x^j += eta^j w_i ----
    const bool ro = freq > 0 && i >= 2 && i % freq == 0;
    {
      const double a = L.st.alpha, zeta = L.st.zeta, inv_d = L.st.inv_delta;
      double nf = 0.0;
      if (own) {
        fe = fma(-a, v, fe);
        const double we = (i > 1) ? inv_d * fma(-bp, b.w[e], v) : inv_d * v;
        b.w[e] = we;
        X[e] = fma(zeta, we, X[e]);
        for (int j = 1; j < nr; ++j) X[e + j * ldx] = fma(s_eta[j].x, we, X[e + j * ldx]);
        nf = fe * fe;
        if (!ro) fn[e] = fe;
      }
      if (!ro) {
        double vv[1] = {nf};
        double *r = region();
        block_row<1>(vv, 1, r + (int64_t)blockIdx.x * kRunRegion, s_w);
        if (!grid_sync(g, epoch)) return;
        reduce_region(r, 1, s_sum);
        if (threadIdx.x == 0) seed_finish<double, false>(bl, s_sum[0]);
        __syncthreads();
        par ^= 1;
        continue;
      }
    }
    // ---- reorthogonalization of v_i and f against V_{<i} (classical Gram-Schmidt, `passes` times) ----
    const int k = i - 1;
    if ((int)threadIdx.x < RB) {
      s_y[0][threadIdx.x] = own ? v : 0.0;
      s_y[1][threadIdx.x] = own ? fe : 0.0;
    }
    __syncthreads();
    col_dots<RB>(b.V, ldv, row0, rows, k, s_y, hpart);
    for (int pass = 0; pass < passes; ++pass) {
      if (!grid_sync(g, epoch)) return;
      slice_reduce(hpart, k, H);
      if (!grid_sync(g, epoch)) return;
      rows_times_h<RB>(b.V, ldv, row0, rows, k, H, s_sub, s_red);
      if ((int)threadIdx.x < RB) {
        s_y[0][threadIdx.x] = fma(-1.0, s_sub[0][threadIdx.x], s_y[0][threadIdx.x]);
        s_y[1][threadIdx.x] = fma(-1.0, s_sub[1][threadIdx.x], s_y[1][threadIdx.x]);
      }
      __syncthreads();
      if (pass + 1 < passes) col_dots<RB>(b.V, ldv, row0, rows, k, s_y, hpart);
    }
    v = own ? s_y[0][threadIdx.x] : 0.0;
    fe = own ? s_y[1][threadIdx.x] : 0.0;
    // ---- v_i /= ||v_i||, then f -= (v_i^H f) v_i, `passes` times; ||f||^2 ends the step.
    // ||v_i||^2 and v_i^H f come from one reduction (h = (v_i^H f) / ||v_i|| before
    // the scaling: the first projection's coefficient, rounded in another order) ----
    {
      double vv[2] = {v * v, v * fe};
      double *r = region();
      block_row<2>(vv, 2, r + (int64_t)blockIdx.x * kRunRegion, s_w);
      if (!grid_sync(g, epoch)) return;
      reduce_region(r, 2, s_sum);
    }
    {
      const double inv = 1.0 / sqrt(s_sum[0]);
      v = inv * v;
      fe = fma(-(s_sum[1] * inv), v, fe);
    }
    if (own) vi[e] = v;
    for (int pass = 1; pass <= passes; ++pass) {
      // pass < passes: h = v_i^H f, then f -= h v_i; pass == passes: ||f||^2 (f final: stored first)
      if (pass == passes && own) fn[e] = fe;
      double vv[1] = {pass < passes ? v * fe : fe * fe};
      double *r = region();
      block_row<1>(vv, 1, r + (int64_t)blockIdx.x * kRunRegion, s_w);
      if (!grid_sync(g, epoch)) return;
      reduce_region(r, 1, s_sum);
      if (pass < passes) {
        fe = fma(-s_sum[0], v, fe);
      } else {
        if (threadIdx.x == 0) seed_finish<double, false>(bl, s_sum[0]);
        __syncthreads();
      }
    }
    par ^= 1;
  }
  seed_leave<double>(b, L, par ? f2 : b.f, i_stop);
  __syncthreads();
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < nr; j += PT) b.eta[j] = s_eta[j];
  local_store(b, L);
}

// ---------------------------------------------------------------------------
// lockstep CG (Hestenes-Stiefel) on nc columns, per-column scalars in CgCols:
//   phase 1: t = D p;  phase 2: q = D^H t, p^H q;  alpha = rho / Re(p^H q)
//   phase 3: x += alpha p, r -= alpha q, ||r||^2;  convergence, beta
//   phase 4: p = r + beta p
// ---------------------------------------------------------------------------
// elements per thread of a vector work item: all loads of an item are in
// flight together (8 real or 4 complex per thread and vector)
template <class T> __host__ __device__ constexpr int elems_per_thread() { return sizeof(T) == sizeof(double) ? 8 : 4; }

// (runs in the last block of a reducing barrier, on any SM: L2 loads, all
// issued before use)
SEED_DEV void cg_update_fin(const CgCols &c, int j, double rr) {
  const int act = __ldcg(c.active + j), it = __ldcg(c.iters + j), mv = __ldcg(c.mvps + j);
  const double bn = __ldcg(c.bnorm + j), rho = __ldcg(c.rho + j);
  if (!act) return;
  const double rn = sqrt(rr);
  c.iters[j] = it + 1;
  c.mvps[j] = mv + 1;
  c.relres[j] = bn > 0.0 ? rn / bn : 0.0;
  if (rn <= c.tol * bn) {
    c.active[j] = 0;
    c.reached[j] = 1;
    c.needs_check[j] = 1;
  } else if (it + 1 >= c.maxit || !isfinite(rr)) {   // non-finite: ends unconverged
    c.active[j] = 0;
    c.needs_check[j] = 1;
  } else {
    c.beta[j] = rr / rho;
    c.rho[j] = rr;
  }
}

SEED_DEV void cg_alpha_fin(const CgCols &c, int j, double pq) {
  const int act = __ldcg(c.active + j);
  const double rho = __ldcg(c.rho + j);
  if (act) c.alpha[j] = rho / pq;
}

// per-column block partials (s_colacc) -> one row of bpart -> reducing barrier;
// the last block reduces all rows and applies fin(j, sum) per column
template <class F>
SEED_DEV bool col_reduce_barrier(const GridSync &g, unsigned &epoch, double *bpart, const double *s_colacc, int nc,
                                 double (*sred)[32], double *s_vals, F &&fin) {
  if (threadIdx.x < 32) bpart[(int64_t)blockIdx.x * 32 + threadIdx.x] = threadIdx.x < nc ? s_colacc[threadIdx.x] : 0.0;
  return grid_reduce_sync(g, epoch, [&]() {
    reduce_rows32(bpart, gridDim.x, s_vals, sred);
    if ((int)threadIdx.x < nc) fin(threadIdx.x, s_vals[threadIdx.x]);
  });
}

// phases 3 and 4 for both operators
template <class T>
SEED_DEV bool cg_vector_phases(const CallArgs *call, T *R, T *P, const T *Q, int64_t ld, int64_t n, const CgCols &c,
                               const GridSync &g, unsigned &epoch, double *bpart, int *s_act, double *s_a,
                               double *s_colacc, double *s_red, double (*sred)[32], double *s_vals) {
  constexpr int kElem = elems_per_thread<T>(), kChunk = PT * kElem;
  const int nc = c.nc;
  const int nchunks = (int)((n + kChunk - 1) / kChunk);
  T *const X = reinterpret_cast<T *>(call->X) + call->col0 * call->ldx;   // CG column c is column c + col0 of X
  const int64_t ldx = call->ldx;
  for (int j = threadIdx.x; j < nc; j += PT) {
    s_a[j] = __ldcg(c.alpha + j);
    s_colacc[j] = 0.0;
  }
  __syncthreads();
  for (int item = blockIdx.x; item < nchunks * nc; item += gridDim.x) {
    const int j = item / nchunks, ch = item - j * nchunks;
    if (!s_act[j]) continue;
    const double a = s_a[j];
    T *x = X + j * ldx;
    T *r = R + j * ld;
    const T *p = P + j * ld, *q = Q + j * ld;
    T pv[kElem], qv[kElem], xv[kElem], rv[kElem];
#pragma unroll
    for (int k = 0; k < kElem; ++k) {
      const int64_t e = (int64_t)ch * kChunk + k * PT + threadIdx.x;
      if (e < n) {
        pv[k] = p[e];
        qv[k] = q[e];
        xv[k] = x[e];
        rv[k] = r[e];
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kElem; ++k) {
      const int64_t e = (int64_t)ch * kChunk + k * PT + threadIdx.x;
      if (e < n) {
        x[e] = Sc<T>::axpy(a, pv[k], xv[k]);
        const T rn = Sc<T>::axpy(-a, qv[k], rv[k]);
        r[e] = rn;
        acc = Sc<T>::nrm2(rn, acc);
      }
    }
    double vv[1] = {acc};
    block_sum<1, PT>(vv, s_red);
    if (threadIdx.x == 0) s_colacc[j] += vv[0];
  }
  __syncthreads();
  if (!col_reduce_barrier(g, epoch, bpart, s_colacc, nc, sred, s_vals, [&](int j, double s) { cg_update_fin(c, j, s); }))
    return false;
  // phase 4 on the columns still active
  for (int j = threadIdx.x; j < nc; j += PT) {
    s_act[j] = __ldcg(c.active + j);
    s_a[j] = __ldcg(c.beta + j);
  }
  __syncthreads();
  for (int item = blockIdx.x; item < nchunks * nc; item += gridDim.x) {
    const int j = item / nchunks, ch = item - j * nchunks;
    if (!s_act[j]) continue;
    const double be = s_a[j];
    const T *r = R + j * ld;
    T *p = P + j * ld;
    T pv[kElem], rv[kElem];
#pragma unroll
    for (int k = 0; k < kElem; ++k) {
      const int64_t e = (int64_t)ch * kChunk + k * PT + threadIdx.x;
      if (e < n) {
        pv[k] = p[e];
        rv[k] = r[e];
      }
    }
#pragma unroll
    for (int k = 0; k < kElem; ++k) {
      const int64_t e = (int64_t)ch * kChunk + k * PT + threadIdx.x;
      if (e < n) p[e] = Sc<T>::axpy(be, pv[k], rv[k]);
    }
  }
  return grid_sync(g, epoch);
}

SEED_DEV bool cg_load_active(const CgCols &c, int *s_act) {
  for (int j = threadIdx.x; j < c.nc; j += PT) s_act[j] = __ldcg(c.active + j);
  __syncthreads();
  int any = 0;
  for (int j = 0; j < c.nc; ++j) any |= s_act[j];
  return any != 0;
}

__global__ void __launch_bounds__(PT) k_cg_run_wilson(WilsonOp op, const CallArgs *call, double2 *R, double2 *P,
                                                       double2 *Q, double2 *tbuf, int64_t ld, CgCols c, GridSync g,
                                                       double *bpart) {
  __shared__ double sacc[4][24][kWilsonSites + 1];
  __shared__ double sred[PT / 32][32];
  __shared__ double s_vals[32];
  __shared__ int s_act[kPersistMaxCols];
  __shared__ double s_a[kPersistMaxCols];
  __shared__ double s_colacc[kPersistMaxCols];
  __shared__ double s_red[PT / 32];
  const int64_t sites = op.sites, n = 12 * op.sites;
  const int tiles = (int)((sites + kWilsonSites - 1) / kWilsonSites);
  const int nc = c.nc;
  const double kappa = op.kappa;
  unsigned epoch = 0;
  while (cg_load_active(c, s_act)) {
    for (int item = blockIdx.x; item < tiles * nc; item += gridDim.x) {
      const int j = item / tiles, tile = item - j * tiles;
      if (!s_act[j]) continue;
      const int64_t s0 = (int64_t)tile * kWilsonSites;
      const double2 *p = P + j * ld;
      double2 *t = tbuf + j * ld;
      wilson_tile<+1>(op, p, s0, sacc);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int o = threadIdx.x + PT * k, sl = o / 12, cc = o - 12 * (o / 12);
        const int64_t ss = s0 + sl;
        if (ss < sites) {
          const double2 sum = tile_sum(sacc, cc, sl);
          const int64_t e = 12 * ss + cc;
          const double2 pv = p[e];
          t[e] = c2(fma(-kappa, sum.x, pv.x), fma(-kappa, sum.y, pv.y));
        }
      }
      __syncthreads();
    }
    if (!grid_sync(g, epoch)) return;
    for (int j = threadIdx.x; j < nc; j += PT) s_colacc[j] = 0.0;
    __syncthreads();
    for (int item = blockIdx.x; item < tiles * nc; item += gridDim.x) {
      const int j = item / tiles, tile = item - j * tiles;
      if (!s_act[j]) continue;
      const int64_t s0 = (int64_t)tile * kWilsonSites;
      const double2 *t = tbuf + j * ld, *p = P + j * ld;
      double2 *q = Q + j * ld;
      wilson_tile<-1>(op, t, s0, sacc);
      double pq = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int o = threadIdx.x + PT * k, sl = o / 12, cc = o - 12 * (o / 12);
        const int64_t ss = s0 + sl;
        if (ss < sites) {
          const double2 sum = tile_sum(sacc, cc, sl);
          const int64_t e = 12 * ss + cc;
          const double2 tv = t[e], pv = p[e];
          const double2 qv = c2(fma(-kappa, sum.x, tv.x), fma(-kappa, sum.y, tv.y));
          q[e] = qv;
          pq = fma(pv.y, qv.y, fma(pv.x, qv.x, pq));
        }
      }
      double vv[1] = {pq};
      block_sum<1, PT>(vv, s_red);
      if (threadIdx.x == 0) s_colacc[j] += vv[0];
    }
    __syncthreads();
    if (!col_reduce_barrier(g, epoch, bpart, s_colacc, nc, sred, s_vals,
                            [&](int j, double s) { cg_alpha_fin(c, j, s); }))
      return;
    if (!cg_vector_phases<double2>(call, R, P, Q, ld, n, c, g, epoch, bpart, s_act, s_a, s_colacc, s_red, sred,
                                   s_vals))
      return;
  }
}

__global__ void __launch_bounds__(PT) k_cg_run_csr(CsrOp op, const CallArgs *call, double *R, double *P, double *Q,
                                                    int64_t ld, CgCols c, GridSync g, double *bpart) {
  __shared__ double sred[PT / 32][32];
  __shared__ double s_vals[32];
  __shared__ int s_act[kPersistMaxCols];
  __shared__ double s_a[kPersistMaxCols];
  __shared__ double s_colacc[kPersistMaxCols];
  __shared__ double s_red[PT / 32];
  constexpr int kElem = elems_per_thread<double>(), kChunk = PT * kElem;
  const int64_t n = op.n;
  const int nc = c.nc;
  const int nchunks = (int)((n + kChunk - 1) / kChunk);
  unsigned epoch = 0;
  while (cg_load_active(c, s_act)) {
    for (int j = threadIdx.x; j < nc; j += PT) s_colacc[j] = 0.0;
    __syncthreads();
    for (int item = blockIdx.x; item < nchunks * nc; item += gridDim.x) {
      const int j = item / nchunks, ch = item - j * nchunks;
      if (!s_act[j]) continue;
      const double *p = P + j * ld;
      double *q = Q + j * ld;
      double pq = 0.0;
#pragma unroll
      for (int k = 0; k < kElem; ++k) {
        const int64_t r = (int64_t)ch * kChunk + k * PT + threadIdx.x;
        if (r < n) {
          const int32_t k0 = __ldg(op.row_ptr + r), k1 = __ldg(op.row_ptr + r + 1);
          double s = 0.0;
          for (int32_t kk = k0; kk < k1; ++kk) s = fma(__ldg(op.vals + kk), p[__ldg(op.col_idx + kk)], s);
          q[r] = s;
          pq = fma(p[r], s, pq);
        }
      }
      double vv[1] = {pq};
      block_sum<1, PT>(vv, s_red);
      if (threadIdx.x == 0) s_colacc[j] += vv[0];
    }
    __syncthreads();
    if (!col_reduce_barrier(g, epoch, bpart, s_colacc, nc, sred, s_vals,
                            [&](int j, double s) { cg_alpha_fin(c, j, s); }))
      return;
    if (!cg_vector_phases<double>(call, R, P, Q, ld, n, c, g, epoch, bpart, s_act, s_a, s_colacc, s_red, sred,
                                  s_vals))
      return;
  }
}

// ---------------------------------------------------------------------------
// Lockstep CG on small real CSR problems (n <= kReorthRunMaxN, at most
// kSmallCgCols columns): the row layout of k_seed_run_csr_reorth (block b owns
// RB rows; here thread t of a block holds row t % RB of column slot t / RB),
// each thread's matrix row kept in registers, and two grid barriers per
// iteration instead of three: the direction update p = r + beta p of the
// previous iteration is formed inside the apply, for the block's own rows
// (written to the other of two p buffers) and, redundantly and with the same
// arithmetic, for the neighbour rows the row reads -- so no barrier is needed
// between the p update and the apply.  The first iteration of a launch takes
// beta = 0 (p = r after the initialisation or a restart).
//   apply: p = r + beta p (own rows), q = A p, partial p^H q
//   barrier; every block: alpha_j = rho_j / (p^H q)_j
//   update: x += alpha p, r -= alpha q, partial ||r||^2
//   barrier; every block: the column's count, relres, stop test, beta, rho
// Every block keeps its own shared-memory copy of the per-column scalars and
// computes them from the same partials in the same order; block 0 writes them
// to the CgCols arrays.  Arithmetic as in the step kernels (the same fma for p,
// x and r; dot products in a different order).
// ---------------------------------------------------------------------------
constexpr int kSmallCgCols = 16;

template <int RB>
__global__ void __launch_bounds__(PT) k_cg_run_csr_small(CsrOp op, const CallArgs *call, double *R, double *P,
                                                         double *P2, double *Q, int64_t ld, CgCols c, GridSync g,
                                                         double *bpart) {
  constexpr int kSlots = PT / RB;   // column slots per block
  __shared__ double s_sum[kRunRegion];
  __shared__ double s_part[kSmallCgCols][RB];
  __shared__ double s_rho[kSmallCgCols], s_alpha[kSmallCgCols], s_beta[kSmallCgCols], s_bn[kSmallCgCols];
  __shared__ int s_act[kSmallCgCols], s_it[kSmallCgCols], s_mv[kSmallCgCols];
  __shared__ int s_any;
  unsigned epoch = 0;
  int reg = 0, par = 0;
  const int nc = c.nc;   // <= kSmallCgCols (checked by the host)
  const int G = gridDim.x;
  const int64_t n = op.n;
  const int rl = threadIdx.x % RB, slot = threadIdx.x / RB;
  const int64_t row0 = (int64_t)blockIdx.x * RB;
  const int rows = (int)(n - row0 < RB ? n - row0 : RB);
  const int64_t e = row0 + rl;
  const bool own = rl < rows;
  double *const X = reinterpret_cast<double *>(call->X) + call->col0 * call->ldx;
  const int64_t ldx = call->ldx;
  constexpr int kRowCache = 8;
  int32_t k0 = 0, k1 = 0, rc_col[kRowCache];
  double rc_val[kRowCache];
  if (own) {
    k0 = __ldg(op.row_ptr + e);
    k1 = __ldg(op.row_ptr + e + 1);
  }
  const bool cached = k1 - k0 <= kRowCache;
#pragma unroll
  for (int q = 0; q < kRowCache; ++q) {
    const bool in = cached && q < k1 - k0;
    rc_col[q] = in ? __ldg(op.col_idx + k0 + q) : 0;
    rc_val[q] = in ? __ldg(op.vals + k0 + q) : 0.0;
  }
  for (int j = threadIdx.x; j < nc; j += PT) {
    s_act[j] = __ldcg(c.active + j);
    s_rho[j] = __ldcg(c.rho + j);
    s_bn[j] = __ldcg(c.bnorm + j);
    s_it[j] = __ldcg(c.iters + j);
    s_mv[j] = __ldcg(c.mvps + j);
    s_beta[j] = 0.0;
  }
  auto region = [&]() {
    double *r = bpart + (int64_t)reg * G * kRunRegion;
    reg ^= 1;
    return r;
  };
  // per-column block sums of the threads' values (s_part[j][rl]) into a region row, then the grid sums
  auto column_sums = [&](double *r) -> bool {
    __syncthreads();
    if ((int)threadIdx.x < nc) {
      double t = 0.0;
      for (int q = 0; q < RB; ++q) t += s_part[threadIdx.x][q];
      r[(int64_t)blockIdx.x * kRunRegion + threadIdx.x] = t;
    }
    if (!grid_sync(g, epoch)) return false;
    reduce_region(r, nc, s_sum);
    return true;
  };
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int any = 0;
      for (int j = 0; j < nc; ++j) any |= s_act[j];
      s_any = any;
    }
    __syncthreads();
    if (!s_any) break;
    const double *Po = par ? P2 : P;
    double *Pn = par ? P : P2;
    // ---- p = r + beta p; q = A p; partial p^H q ----
    for (int j0 = 0; j0 < nc; j0 += kSlots) {
      const int j = j0 + slot;
      if (j < nc) {
        double pq = 0.0;
        if (own && s_act[j]) {
          const double be = s_beta[j];
          const double *rj = R + j * ld, *pj = Po + j * ld;
          double sum = 0.0;
          if (cached) {
            double xr[kRowCache], xp[kRowCache];
#pragma unroll
            for (int q = 0; q < kRowCache; ++q) {
              xr[q] = q < k1 - k0 ? __ldcg(rj + rc_col[q]) : 0.0;
              xp[q] = q < k1 - k0 ? __ldcg(pj + rc_col[q]) : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kRowCache; ++q)
              if (q < k1 - k0) sum = fma(rc_val[q], fma(be, xp[q], xr[q]), sum);
          } else {
            for (int32_t q = k0; q < k1; ++q) {
              const int32_t col = __ldg(op.col_idx + q);
              sum = fma(__ldg(op.vals + q), fma(be, __ldcg(pj + col), __ldcg(rj + col)), sum);
            }
          }
          const double pe = fma(be, __ldcg(pj + e), __ldcg(rj + e));
          Pn[j * ld + e] = pe;
          Q[j * ld + e] = sum;
          pq = pe * sum;
        }
        s_part[j][rl] = pq;
      }
    }
    if (!column_sums(region())) return;
    if ((int)threadIdx.x < nc && s_act[threadIdx.x]) {
      const int j = threadIdx.x;
      s_alpha[j] = s_rho[j] / s_sum[j];
      if (blockIdx.x == 0) c.alpha[j] = s_alpha[j];
    }
    __syncthreads();
    // ---- x += alpha p; r -= alpha q; partial ||r||^2 ----
    for (int j0 = 0; j0 < nc; j0 += kSlots) {
      const int j = j0 + slot;
      if (j < nc) {
        double rr = 0.0;
        if (own && s_act[j]) {
          const double a = s_alpha[j];
          const double pe = Pn[j * ld + e], qe = Q[j * ld + e];
          X[j * ldx + e] = fma(a, pe, X[j * ldx + e]);
          const double rn = fma(-a, qe, R[j * ld + e]);
          R[j * ld + e] = rn;
          rr = rn * rn;
        }
        s_part[j][rl] = rr;
      }
    }
    if (!column_sums(region())) return;
    if ((int)threadIdx.x < nc && s_act[threadIdx.x]) {
      const int j = threadIdx.x;
      const double rr = s_sum[j], rn = sqrt(rr), bn = s_bn[j];
      const int it = s_it[j] + 1;
      s_it[j] = it;
      s_mv[j] += 1;
      int act = 1, reached = 0, check = 0;
      if (rn <= c.tol * bn) {
        act = 0;
        reached = 1;
        check = 1;
      } else if (it >= c.maxit || !isfinite(rr)) {   // non-finite: ends unconverged
        act = 0;
        check = 1;
      } else {
        s_beta[j] = rr / s_rho[j];
        s_rho[j] = rr;
      }
      s_act[j] = act;
      if (blockIdx.x == 0) {
        c.iters[j] = it;
        c.mvps[j] = s_mv[j];
        c.relres[j] = bn > 0.0 ? rn / bn : 0.0;
        c.beta[j] = s_beta[j];
        c.rho[j] = s_rho[j];
        if (!act) {
          c.active[j] = 0;
          if (reached) c.reached[j] = 1;
          c.needs_check[j] = check;
        }
      }
    }
    par ^= 1;
  }
}

int small_cg_grid_cap(int sm_count, int rb) {
  int per_sm = 0;
  const void *k = rb == 16 ? (const void *)k_cg_run_csr_small<16> : (const void *)k_cg_run_csr_small<32>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PT, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm > 2) per_sm = 2;
  return per_sm * sm_count;
}

cudaError_t launch_cg_run_csr_small(const CsrOp &op, const CallArgs *call, double *R, double *P, double *P2,
                                    double *Q, int64_t ld, const CgCols &c, GridSync g, double *bpart, int rb,
                                    int grid, cudaStream_t s) {
  CsrOp o = op;
  CgCols cc = c;
  void *args[] = {&o, &call, &R, &P, &P2, &Q, &ld, &cc, &g, &bpart};
  const void *k = rb == 16 ? (const void *)k_cg_run_csr_small<16> : (const void *)k_cg_run_csr_small<32>;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(PT), args, 0, s);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// The Wilson runs' dynamic shared memory (resident links and tile vectors)
// is above the default 48 KB limit: raise it once per process.
cudaError_t seed_run_wilson_smem_attr() {
  static const cudaError_t attr = [] {
    const cudaError_t e = cudaFuncSetAttribute((const void *)k_seed_run_wilson,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResSmemBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_seed_run_wilson32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kResSmemBytes32);
  }();
  return attr;
}

// Up to 2 blocks per SM (3 for the seed runs, with the kernel bounded to fit,
// measured no faster on the 8^4 workload); 0 when the occupancy query fails.
int persistent_grid(int kind, int sm_count, bool cg, bool fp32) {
  int per_sm = 0;
  const void *k;
  if (cg) k = kind == 0 ? (const void *)k_cg_run_csr : (const void *)k_cg_run_wilson;
  else if (fp32) k = kind == 0 ? (const void *)k_seed_run_csr<float> : (const void *)k_seed_run_wilson32;
  else k = kind == 0 ? (const void *)k_seed_run_csr<double> : (const void *)k_seed_run_wilson;
  const bool wil = !cg && kind == 1;   // the Wilson seed runs: five warps, resident tiles
  const int threads = wil ? PTW : PT;
  if (wil && seed_run_wilson_smem_attr() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t dyn = !wil ? 0 : fp32 ? kResSmemBytes32 : kResSmemBytes;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (wil && fp32) {   // the site form of large lattices must fit once per SM too
    int per_sm_g = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_g, (const void *)k_seed_run_wilson32s,
                                                      kSiteThreads32 + 32, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (per_sm_g < per_sm) per_sm = per_sm_g;
  }
  // the Wilson seed runs work in operator tiles only (one owner block per SM):
  // more blocks would only add barrier arrivals
  const int cap = (!cg && kind == 1) ? 1 : 2;
  if (per_sm > cap) per_sm = cap;
  return per_sm * sm_count;
}

cudaError_t launch_seed_run_wilson(const SeedBufs<double2> &b, const WilsonOp &op, double2 *tbuf, GridSync g,
                                   double *bpart, double *tpart, int i_stop, int grid, cudaStream_t s) {
  SeedBufs<double2> bb = b;
  WilsonOp o = op;
  void *args[] = {&bb, &o, &tbuf, &g, &bpart, &tpart, &i_stop};
  const cudaError_t attr = seed_run_wilson_smem_attr();
  if (attr != cudaSuccess) return attr;
  return cudaLaunchCooperativeKernel((const void *)k_seed_run_wilson, dim3(grid), dim3(PTW), args, kResSmemBytes, s);
}
cudaError_t launch_seed_run_csr(const SeedBufs<double> &b, const CsrOp &op, double *f2, GridSync g, double *bpart,
                                int i_stop, int grid, cudaStream_t s) {
  SeedBufs<double> bb = b;
  CsrOp o = op;
  void *args[] = {&bb, &o, &f2, &g, &bpart, &i_stop};
  return cudaLaunchCooperativeKernel((const void *)k_seed_run_csr<double>, dim3(grid), dim3(PT), args, 0, s);
}
cudaError_t launch_seed_run_csr32(const SeedBufs<float> &b, const CsrOp32 &op, float *f2, GridSync g, double *bpart,
                                  int i_stop, int grid, cudaStream_t s) {
  SeedBufs<float> bb = b;
  CsrOp32 o = op;
  void *args[] = {&bb, &o, &f2, &g, &bpart, &i_stop};
  return cudaLaunchCooperativeKernel((const void *)k_seed_run_csr<float>, dim3(grid), dim3(PT), args, 0, s);
}
cudaError_t launch_seed_run_wilson32(const SeedBufs<float2> &b, const WilsonOp32 &op, float2 *tbuf, GridSync g,
                                     double *tpart, int i_stop, int grid, cudaStream_t s) {
  SeedBufs<float2> bb = b;
  WilsonOp32 o = op;
  void *args[] = {&bb, &o, &tbuf, &g, &tpart, &i_stop};
  const cudaError_t attr = seed_run_wilson_smem_attr();
  if (attr != cudaSuccess) return attr;
  if (b.n / 384 > grid)   // more tiles than blocks: the site form
    return cudaLaunchCooperativeKernel((const void *)k_seed_run_wilson32s, dim3(grid), dim3(kSiteThreads32 + 32), args,
                                       0, s);
  return cudaLaunchCooperativeKernel((const void *)k_seed_run_wilson32, dim3(grid), dim3(PTW), args, kResSmemBytes32,
                                     s);
}
cudaError_t launch_cg_run_wilson(const WilsonOp &op, const CallArgs *call, double2 *R, double2 *P, double2 *Q,
                                 double2 *tbuf, int64_t ld, const CgCols &c, GridSync g, double *bpart, int grid,
                                 cudaStream_t s) {
  WilsonOp o = op;
  CgCols cc = c;
  void *args[] = {&o, &call, &R, &P, &Q, &tbuf, &ld, &cc, &g, &bpart};
  return cudaLaunchCooperativeKernel((const void *)k_cg_run_wilson, dim3(grid), dim3(PT), args, 0, s);
}
// Self-test of the bounded barrier wait: the epoch starts one ahead, so the
// barrier's target (2 x gridDim.x arrivals) is never reached, every block's
// wait runs out after kBarrierTimeoutNs (or ends when another block has
// flagged the error) and the kernel returns with GridSync::error set.
__global__ void k_barrier_timeout_check(GridSync g) {
  unsigned epoch = 1;
  grid_sync(g, epoch);
}

cudaError_t launch_barrier_timeout_check(GridSync g, cudaStream_t s) {
  GridSync gg = g;
  void *args[] = {&gg};
  return cudaLaunchCooperativeKernel((const void *)k_barrier_timeout_check, dim3(2), dim3(PT), args, 0, s);
}

int reorth_run_grid_cap(int sm_count, int rb) {
  int per_sm = 0;
  const void *k = rb == 16 ? (const void *)k_seed_run_csr_reorth<16> : (const void *)k_seed_run_csr_reorth<32>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PT, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm > 2) per_sm = 2;
  return per_sm * sm_count;
}

cudaError_t launch_seed_run_csr_reorth(const SeedBufs<double> &b, const CsrOp &op, double *f2, GridSync g,
                                       double *bpart, double *hpart, double *H, int freq, int passes, int i_stop,
                                       int rb, int grid, cudaStream_t s) {
  SeedBufs<double> bb = b;
  CsrOp o = op;
  void *args[] = {&bb, &o, &f2, &g, &bpart, &hpart, &H, &freq, &passes, &i_stop};
  const void *k = rb == 16 ? (const void *)k_seed_run_csr_reorth<16> : (const void *)k_seed_run_csr_reorth<32>;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(PT), args, 0, s);
}

cudaError_t launch_cg_run_csr(const CsrOp &op, const CallArgs *call, double *R, double *P, double *Q, int64_t ld,
                              const CgCols &c, GridSync g, double *bpart, int grid, cudaStream_t s) {
  CsrOp o = op;
  CgCols cc = c;
  void *args[] = {&o, &call, &R, &P, &Q, &ld, &cc, &g, &bpart};
  return cudaLaunchCooperativeKernel((const void *)k_cg_run_csr, dim3(grid), dim3(PT), args, 0, s);
}

}  // namespace seedk
