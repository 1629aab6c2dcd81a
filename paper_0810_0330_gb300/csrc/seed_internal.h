// seed_internal.h -- declarations shared by the kernel translation units and
// the engine (host).  Not part of the public ABI.
#pragma once
#include <cuda.h>   // CUtensorMap (type only)
#include <cuda_runtime.h>
#include <stdint.h>

namespace seedk {

constexpr int kMaxRhs = 64;       // right-hand sides per call
constexpr int kColTicket = 16;    // tickets[16 + c]: last-block tickets of per-column reductions
constexpr int kVecThreads = 128;  // threads per block of the vector kernels
constexpr int kVecBlocksMax = 152 * 8;   // blocks of the single-vector kernels on long vectors
// device scratch for block partials: the seed dot kernel's 5 chunks x 32 values per block
// (plus its group partials, 5 chunks x ceil(kVecBlocksMax / 32) x 32)
constexpr int kPartials = 5 * kVecBlocksMax * 32 + 5 * ((kVecBlocksMax + 31) / 32) * 32 + 4096;

// Stop reasons of the seed recurrence (SeedState::stop_reason)
enum { STOP_RUNNING = 0, STOP_CONVERGED = 1, STOP_BREAKDOWN = 2, STOP_MMAX = 3, STOP_NOTSPD = 4, STOP_TIMEOUT = 5,
       STOP_BLOCK = 6 /* internal: a step found its seeding block full (never expected) */,
       STOP_NONFINITE = 7 /* ||r_0^1|| is NaN or infinite */ };

// Device-resident scalars of the Sec. 3 recurrence (paper notation).
struct SeedState {
  double alpha;       // alpha_i
  double beta;        // beta_i of the last finished step
  double beta_prev;   // beta_{i-1}
  double delta;       // delta_i (delta_{i-1} until the LU update of step i runs)
  double inv_delta;   // 1 / delta_i, formed once by the LU update's scalar code
  double zeta;        // zeta_i
  double gamma;       // gamma_{i-1}
  double rho;         // beta_i |zeta_i| / delta_i
  double tnorm;       // max row sum of |T|
  double inv_beta;    // 1 / beta_i, used to form v_{i+1}
  double beta0;       // ||r_0^1||
  double bnorm1;      // ||b^1||
  double tol_rel;     // tol_seed
  double tol_abs;     // tol_seed * ||b^1||
  double breakdown_rel;
  double scratch;     // reorthogonalization: 1 / ||v_i||
  double2 h;          // reorthogonalization: v_i^H f
  int32_t i;          // current step (1-based)
  int32_t active;     // 1 while the recurrence runs
  int32_t stop_reason;
  int32_t converged_at;
  int32_t stop_at;
  int32_t m_max;
  int32_t extra_iters;
  // blocked seeding of systems 2..p (SeedBufs::Wb set): the current block
  // starts at step blk0; w_last is the last step whose w_i is stored in Wb;
  // blk_len is the length of the block a flush is folding into X
  int32_t blk0;
  int32_t w_last;
  int32_t blk_len;
};

// Caller buffers of the current call, read by the kernels from device memory so
// that captured CUDA graphs stay valid across calls with other buffers.
struct CallArgs {
  void *X;             // x^1..x^nrhs, column-major
  int64_t ldx;
  int64_t col0;        // lockstep CG: CG column c updates column c + col0 of X
};

// Buffers of one seed solve; T = double (real) or double2 (complex).
template <class T>
struct SeedBufs {
  int64_t n;
  int32_t nrhs;        // columns of X (1 = seed system only)
  int32_t nblocks;     // blocks of the vector kernels (fixed for n)
  T *V;                // n x (m_max+1), column c holds v_{c+1}
  int64_t ldv;
  T *u;                // A v_i
  T *f;                // the Lanczos residual vector
  T *w;                // w_i
  const T *R0;         // r_0^j for j = 2..nrhs, column j-2
  int64_t ldr;
  const CallArgs *call;  // X (x^j in column j-1) and ldx
  SeedState *st;
  double *alpha_hist;  // [m_max+1], alpha_i at index i
  double *beta_hist;   // [m_max+1], beta_i at index i (beta_0 at 0)
  double *delta_hist;  // [m_max+1]
  double2 *eta;        // [kMaxRhs]
  double *partials;    // kPartials doubles
  unsigned *tickets;   // >= 4 counters, zero between launches
  // Blocked seeding (the Sec. 3 seeding of systems 2..p deferred over a block of steps):
  // NULL = the streaming form (g^j, eta^j and x^j every step).  Otherwise each
  // step stores w_i in column i - blk0 of Wb and gamma_{i-1} in gamma_hist[i],
  // and launch_seed_flush folds the block into x^2..x^p.
  T *Wb;               // n x kSeedBlock, leading dimension ldv
  double *gamma_hist;  // [m_max+2]
};

// Steps per block of the blocked seeding (columns of SeedBufs::Wb).
constexpr int kSeedBlock = 128;

// Tensor-core form of the FP32 complex flush products (tc_dots.cu): TMA maps
// over V and R_0 and the CTA count of its grid; a host-side descriptor.
// TMA maps of one FP32 complex block, one per box height: v[h] loads 16 >> h columns
// (16, 8, 4, 2, 1) of 128 complex each; a height above the block's column count is never used.
struct TcMaps {
  CUtensorMap v[5];   // V: columns of the FP32 basis (len nv, leading dimension ldv)
  CUtensorMap r[5];   // R_0: r_0^2.. in FP32
};
struct TcFlush {
  TcMaps maps;
  int *err;           // device flag: a wait of the kernel ran out (reported as SEED_ETIMEOUT)
  int grid;           // CTAs along the vector (<= SMs, <= nv / 128); also the partials' chunk count
  bool ok;            // maps valid for the current buffers
};

// Workspace of the block flush (seedblock.cu).
struct BlockBufs {
  double2 *Hpart;   // [max(nchunk, tc grid)][kSeedBlock][kMaxRhs - 1] partial products v_i^H r_0^j
  double2 *G;       // [kSeedBlock][kMaxRhs - 1]   g_i^j
  double2 *Z;       // [kSeedBlock][kMaxRhs - 1]   eta_i^j
  int32_t nchunk;   // row chunks of the partial products
  int64_t rows;     // rows per chunk
  const TcFlush *tc;   // host pointer, NULL or !ok: CUDA-core products (only read by the launcher)
};
constexpr int kBlockChunksMax = 64;

// tc_dots.cu
bool tc_make_maps(CUtensorMap maps[5], const void *base, int64_t len, int64_t ld, int64_t ncols);
int tc_grid(int64_t len);
cudaError_t launch_blk_dots_tc(const TcMaps &maps, const SeedState *st, int len_host, int vcol_host, int nj,
                               int64_t len, double2 *Hpart, int grid, int *err, cudaStream_t s);

// Buffers of the blocked reorthogonalization (Sec. 3).
template <class T>
struct ReorthBufs {
  int64_t n;
  int32_t rows_per_item;   // rows of one partial product tile
  int32_t nrb;             // row blocks = ceil(n / rows_per_item)
  int32_t nitems_grid;     // persistent grid size of the tile kernel
  int32_t kcap;            // column capacity of Hpart / H (m_max + 1)
  const T *V;
  int64_t ldv;
  double2 *Hpart;          // [nrb][m_max+1][2]
  double2 *H;              // [m_max+1][2]
  double2 *Hrows;          // long FP32 vectors: [ceil(n / 4096)][m_max+1][2] partials by row chunks, else NULL
  int32_t row_chunk;       // rows per chunk of Hrows: 4096..8192, a multiple of 256
};

// Per-column CG state (lockstep CG over nc columns).  rupd, upd and delta are
// used by the mixed-precision reliable updates only.
struct CgCols {
  int32_t nc;
  double *rho, *alpha, *beta, *bnorm, *relres, *rupd;
  int32_t *active, *iters, *reached, *restarts, *converged, *needs_check, *mvps, *upd;
  double tol, tol_check, delta;
  int32_t maxit, max_restarts;
};
constexpr int kCgDoubles = 6;   // arrays of kMaxRhs doubles in CgCols
constexpr int kCgInts = 8;      // arrays of kMaxRhs int32 in CgCols

// Grid barrier of the persistent kernels (all zeroed before every launch).
constexpr int kGridSyncWords = 4 + 256;
struct GridSync {
  unsigned *count;       // arrivals, monotonic within a launch
  unsigned *release;     // last epoch released by a reducing barrier
  int *error;            // 1 after a barrier wait ran past its time limit
  unsigned *owners;      // number of blocks that own operator tiles
  unsigned *sm_slots;    // [256] blocks seen per SM id
};

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------

// Wilson-Dirac (wilson.cu).  sign = +1 applies D, -1 applies D^H.
// C = double2 (FP64 links) or float2 (FP32 copy of the links, mixed precision)
template <class C>
struct WilsonOpT {
  int32_t dims[4];
  int64_t sites;
  double kappa;
  int32_t bc_t;
  const C *links;         // FP64: [4][sites][3][3];  FP32 copy: [4][9][sites]
  const int32_t *nbr;     // [sites][8]
};
using WilsonOp = WilsonOpT<double2>;
using WilsonOp32 = WilsonOpT<float2>;
void launch_wilson_neighbors(const int32_t dims[4], int32_t *nbr, cudaStream_t s);
void launch_wilson_dslash(const WilsonOp &op, int sign, const double2 *in, int64_t ldi, double2 *out,
                          int64_t ldo, int ncols, const int32_t *col_active, cudaStream_t s);
// FP32 copy (links in structure-of-arrays order, see wilson.cu).  tiled: the
// spinor vectors use the mixed path's 32-site tiled layout (Layout32), else the
// caller's site-major layout.
void launch_wilson_dslash32(const WilsonOp32 &op, int sign, const float2 *in, int64_t ldi, float2 *out, int64_t ldo,
                            int ncols, const int32_t *col_active, bool tiled, cudaStream_t s);
void launch_links_soa32(const double2 *links, float2 *out, int64_t sites, cudaStream_t s);

// CSR (csr.cu)
template <class R>
struct CsrOpT {
  int64_t n;
  const int32_t *row_ptr, *col_idx;
  const R *vals;
  int32_t tpr = 1;        // threads per row (1, 2, 4 or 8); see csr.cu
  int32_t block = 256;    // threads per block
};
using CsrOp = CsrOpT<double>;
using CsrOp32 = CsrOpT<float>;
void launch_csr_spmv(const CsrOp &op, const double *in, int64_t ldi, double *out, int64_t ldo, int ncols,
                     const int32_t *col_active, cudaStream_t s);
void launch_csr_spmv32(const CsrOp32 &op, const float *in, int64_t ldi, float *out, int64_t ldo, int ncols,
                       const int32_t *col_active, cudaStream_t s);
// launch shapes the CSR autotuner chooses from: {threads per row, block size}
constexpr int kCsrShapes = 6;
extern const int32_t kCsrShape[kCsrShapes][2];

// Seed recurrence, reorthogonalization, CG (krylov.cu)
int vec_blocks(int64_t n);
template <class T> void launch_seed_start(const SeedBufs<T> &b, const T *r01, cudaStream_t s);
template <class T> void launch_seed_dots(const SeedBufs<T> &b, cudaStream_t s);
template <class T> void launch_seed_update(const SeedBufs<T> &b, bool with_norm, cudaStream_t s);
template <class T> void launch_reorth(const SeedBufs<T> &b, const ReorthBufs<T> &r, int passes, cudaStream_t s);
// Blocked seeding: fold the steps blk0..w_last into x^2..x^p (G = V_blk^H R_0,
// the eta recursion, X += W Z) and start the next block.  Returns the kernel count.
template <class T> int launch_seed_flush(const SeedBufs<T> &b, const BlockBufs &k, cudaStream_t s);
BlockBufs block_layout(int64_t n);
template <class T> int reorth_kernel_count(int passes);

template <class T> void launch_sub_from(const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R, int64_t ldr,
                                        int64_t n, int ncols, cudaStream_t s);   // R = B - Q
template <class T> void launch_cg_init(int64_t n, const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R, T *P,
                                       int64_t ld, const CgCols &c, double *partials, unsigned *tickets,
                                       bool restart_only, cudaStream_t s);
template <class T> void launch_cg_alpha(int64_t n, const T *P, const T *Q, int64_t ld, const CgCols &c,
                                        double *partials, unsigned *tickets, cudaStream_t s);
template <class T> void launch_cg_update(int64_t n, const CallArgs *call, T *R, const T *P, const T *Q, int64_t ld,
                                         const CgCols &c, double *partials, unsigned *tickets, cudaStream_t s);
template <class T> void launch_cg_p(int64_t n, const T *R, T *P, int64_t ld, const CgCols &c, cudaStream_t s);
template <class T> void launch_cg_check(int64_t n, const T *B, int64_t ldb, const T *Q, int64_t ldq, T *R,
                                        int64_t ld, const CgCols &c, double *partials, unsigned *tickets,
                                        cudaStream_t s);
template <class T> void launch_colnorms(int64_t n, const T *X, int64_t ldx, int ncols, double *out,
                                        double *partials, unsigned *tickets, cudaStream_t s);
template <class T> void launch_project(int64_t n, const T *V, int64_t ldv, int m, const double *alpha,
                                       const double *beta, const T *R, int64_t ldr, T *X, int64_t ldx,
                                       int ncols, double2 *G, double2 *Gpart, int nrb, int rows_per_item,
                                       cudaStream_t s);
template <class T> void launch_copy_cols(const T *src, int64_t lds, T *dst, int64_t ldd, int64_t n, int ncols,
                                         cudaStream_t s);
template <class T> void launch_zero_cols(T *dst, int64_t ldd, int64_t n, int ncols, cudaStream_t s);

// Index map from the mixed path's FP32 vectors to the caller's vectors.  For a
// Wilson operator the FP32 vectors are tiled by 32 sites: component k (0..11)
// of site s lives at ((s / 32) * 12 + k) * 32 + s % 32, so that a warp reading
// one component of 32 consecutive sites reads 256 contiguous bytes; the
// vector length is 12 * 32 * ceil(sites / 32) and sites beyond the lattice are
// zero padding.  For CSR (sites == 0) the map is the identity.
struct Layout32 {
  int64_t sites;
  __host__ __device__ int64_t to_user(int64_t t) const {   // -1 for padding
    if (sites == 0) return t;
    const int64_t blk = t / 384, rem = t - blk * 384, s = blk * 32 + (rem & 31);
    return s < sites ? 12 * s + (rem >> 5) : -1;
  }
  __host__ __device__ int64_t length(int64_t n) const { return sites == 0 ? n : 384 * ((sites + 31) / 32); }
};

// Sec. 2.3 projection (related.cu): X[:, c] += delta_c xcg, R[:, c] -= delta_c rbcg with
// delta_c = (xcg^H R[:, c]) / (xcg^H rbcg), c < nrem.  dots: nrem + 1, delta: nrem device scratch.
template <class T>
void launch_related_project(int64_t n, const T *xcg, const T *rbcg, T *X, int64_t ldx, T *R, int64_t ldr, int nrem,
                            double2 *dots, double2 *delta, double *partials, unsigned *tickets, cudaStream_t s,
                            const int32_t *gate = nullptr);

// Adjoint (adjoint.cu): out[j] = Re <L_j, (dA/dkappa) X_j> for the Wilson normal
// operator A = D^H D (device array of ncols doubles).
void launch_dkappa_inner(const WilsonOp &op, const double2 *L, int64_t ldl, const double2 *X, int64_t ldx, int ncols,
                         double *partials, unsigned *tickets, double *out, cudaStream_t s);

// Mixed precision (mixed.cu): T64 / T32 = double / float or double2 / float2.
// n32: length of the FP32 vectors (Layout32::length); user vectors follow L.
template <class T64, class T32>
void launch_to_low(const T64 *src, int64_t lds, T32 *dst, int64_t ldd, int64_t n32, Layout32 L, int ncols,
                   cudaStream_t s);
template <class T64, class T32>   // X += E, E = 0 (columns with mask set; mask NULL = all)
void launch_fold(T64 *X, int64_t ldx, T32 *E, int64_t lde, int64_t n32, Layout32 L, int ncols, const int32_t *mask,
                 cudaStream_t s);
template <class T64, class T32>
void launch_mixed_init(int64_t n32, Layout32 L, const T64 *B, int64_t ldb, const T64 *Q, int64_t ldq, T32 *R, T32 *P,
                       T32 *E, int64_t ld, const CgCols &c, double *partials, unsigned *tickets, cudaStream_t s);
void launch_mixed_flag(const CgCols &c, cudaStream_t s);
template <class T64, class T32>
void launch_mixed_residual(int64_t n32, Layout32 L, const T64 *B, int64_t ldb, const T64 *Q, int64_t ldq, T32 *R,
                           T32 *P, int64_t ld, const CgCols &c, double *partials, unsigned *tickets, cudaStream_t s);

// Persistent cooperative kernels (persistent.cu).  Seed: runs Lanczos steps
// i < i_stop (none of which reorthogonalizes) while the recurrence is active;
// on leaving with i == i_stop it leaves f = beta_{i-1} v_i in SeedBufs::f, from
// which the step-by-step path continues.  CG: runs lockstep iterations until no column is active.  Both return
// cudaErrorCooperativeLaunchTooLarge and friends from the launch, and report a
// barrier time-out through GridSync::error.  CG: nc <= 32.
constexpr int kPersistMaxCols = 32;
int persistent_grid(int kind, int sm_count, bool cg, bool fp32 = false);
// two blocks wait at a grid barrier that can never complete; g zeroed by the caller
cudaError_t launch_barrier_timeout_check(GridSync g, cudaStream_t s);
// tpart: three doubles per 32-site tile
cudaError_t launch_seed_run_wilson(const SeedBufs<double2> &b, const WilsonOp &op, double2 *tbuf, GridSync g,
                                   double *bpart, double *tpart, int i_stop, int grid, cudaStream_t s);
cudaError_t launch_seed_run_csr(const SeedBufs<double> &b, const CsrOp &op, double *f2, GridSync g, double *bpart,
                                int i_stop, int grid, cudaStream_t s);
// Small real CSR problems reorthogonalizing every freq (1..7) steps, streaming
// seeding, nrhs <= 16: the whole seed run in one launch of ceil(n / rb) blocks
// (rb = 16 or 32 rows per block).  bpart: 2 x grid x 32 doubles; hpart:
// 2 x (m_max + 1) x grid doubles; H: 2 x (m_max + 1) doubles.
constexpr int64_t kReorthRunMaxN = 32 * 304;
constexpr int kReorthRunMaxRhs = 16;
int reorth_run_grid_cap(int sm_count, int rb);
cudaError_t launch_seed_run_csr_reorth(const SeedBufs<double> &b, const CsrOp &op, double *f2, GridSync g,
                                       double *bpart, double *hpart, double *H, int freq, int passes, int i_stop,
                                       int rb, int grid, cudaStream_t s);
// mixed precision (FP32 vectors and operator copy, FP64 scalars)
cudaError_t launch_seed_run_csr32(const SeedBufs<float> &b, const CsrOp32 &op, float *f2, GridSync g, double *bpart,
                                  int i_stop, int grid, cudaStream_t s);
cudaError_t launch_seed_run_wilson32(const SeedBufs<float2> &b, const WilsonOp32 &op, float2 *tbuf, GridSync g,
                                     double *tpart, int i_stop, int grid, cudaStream_t s);
cudaError_t launch_cg_run_wilson(const WilsonOp &op, const CallArgs *call, double2 *R, double2 *P, double2 *Q,
                                 double2 *tbuf, int64_t ld, const CgCols &c, GridSync g, double *bpart, int grid,
                                 cudaStream_t s);
// Lockstep CG on small real CSR problems (n <= kReorthRunMaxN, nc <= 16): one
// launch of ceil(n / rb) blocks, two grid barriers per iteration; P2 is a
// second n x nc p buffer (ld).
int small_cg_grid_cap(int sm_count, int rb);
cudaError_t launch_cg_run_csr_small(const CsrOp &op, const CallArgs *call, double *R, double *P, double *P2,
                                    double *Q, int64_t ld, const CgCols &c, GridSync g, double *bpart, int rb,
                                    int grid, cudaStream_t s);
cudaError_t launch_cg_run_csr(const CsrOp &op, const CallArgs *call, double *R, double *P, double *Q, int64_t ld,
                              const CgCols &c, GridSync g, double *bpart, int grid, cudaStream_t s);

}  // namespace seedk
