/*
 * seed_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * improved seed method of Abdel-Rehim, Morgan and Wilcox ("Improved Seed
 * Methods for Symmetric Positive Definite Linear Equations with Multiple
 * Right-hand Sides").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * Everything is complex double (a real problem is embedded with zero
 * imaginary parts; the real parts then follow exactly the real arithmetic).
 * Reductions run in index order.  Build with -ffp-contract=off so that x86
 * and Arm hosts give the same bits.
 *
 * Contents and the passage each part follows:
 *   orc_csr_apply ........ y = A x for a CSR matrix (Sec. 1 problem A x = b)
 *   orc_wilson_dslash .... Wilson-Dirac D (sign=+1) or D^H (sign=-1); the
 *                          paper (Sec. 4) names D but does not define it, so
 *                          the textbook Wilson operator with r = 1 is used
 *   orc_op_apply ......... A = D^H D (Sec. 4: the system multiplied by
 *                          D^H to make it Hermitian), or CSR, or dense
 *   orc_seed_first ....... Sec. 3, the Lanczos form of single-seed CG with
 *                          periodic reorthogonalization
 *   orc_cg ............... plain CG (Hestenes-Stiefel) for the seeded systems
 *                          (Sec. 1, Sec. 2.2)
 *   orc_related_project .. Sec. 2.3 (single seeding for related right-hand
 *                          sides): the projection over one CG correction
 *   orc_cholesky_solve ... dense Hermitian Cholesky (pin only)
 *   orc_tridiag_eigs ..... eigenvalues of the Lanczos tridiagonal by Sturm
 *                          bisection (pin only)
 *   orc_wilson_neighbors . site -> 8 neighbour table (x fastest, periodic)
 *   orc_seed_multiple .... multiple seeding, the seed CG that Sec. 2.1 compares
 *                          against: systems solved in order by CG, each CG
 *                          step also projecting every later system
 *   orc_wilson_dA_dkappa . y = (dA/dkappa) x for A = D^H D (no passage: the
 *                          chain rule for the adjoint of a solve; pinned by
 *                          finite differences of the operator and of a loss)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* All-cores build (-fopenmp -DORC_OMP, used only to time the oracle on every
 * host core): the loops whose iterations are independent -- operator applies
 * row by row or site by site, axpys and scalings -- are split over threads;
 * every reduction (dot product, norm) keeps its one-thread index order, so the
 * results are bit-identical to the one-thread build. */
#ifdef ORC_OMP
#include <omp.h>
#define ORC_PAR _Pragma("omp parallel for schedule(static)")
int orc_threads(int k) {
  if (k > 0) omp_set_num_threads(k);
  return omp_get_max_threads();
}
#else
#define ORC_PAR
int orc_threads(int k) {
  (void)k;
  return 1;
}
#endif

typedef struct { double re, im; } zc;

static inline zc zmk(double re, double im) { zc r; r.re = re; r.im = im; return r; }
static inline zc zadd(zc a, zc b) { return zmk(a.re + b.re, a.im + b.im); }
static inline zc zsub(zc a, zc b) { return zmk(a.re - b.re, a.im - b.im); }
static inline zc zmul(zc a, zc b) { return zmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static inline zc zconj(zc a) { return zmk(a.re, -a.im); }
static inline zc zscale(double s, zc a) { return zmk(s * a.re, s * a.im); }

/* status codes (same numbering as the library's public ones) */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOTSPD = 4, ORC_ENOTCONV = 5 };

/* ------------------------------------------------------------------------ */
/* length-n vector operations (the vector operations Table 2.1 counts)  */
/* ------------------------------------------------------------------------ */

/* a^H b, summed in index order */
static zc vdot(int64_t n, const zc *a, const zc *b) {
  zc s = zmk(0.0, 0.0);
  for (int64_t k = 0; k < n; ++k) s = zadd(s, zmul(zconj(a[k]), b[k]));
  return s;
}

static double vnorm(int64_t n, const zc *a) {
  double s = 0.0;
  for (int64_t k = 0; k < n; ++k) s += a[k].re * a[k].re + a[k].im * a[k].im;
  return sqrt(s);
}

/* y += alpha x */
static void vaxpy(int64_t n, zc alpha, const zc *x, zc *y) {
  ORC_PAR
  for (int64_t k = 0; k < n; ++k) y[k] = zadd(y[k], zmul(alpha, x[k]));
}

/* ------------------------------------------------------------------------ */
/* Operators                                                                */
/* ------------------------------------------------------------------------ */

/* y = A x, A real CSR (row_ptr[n+1], col_idx[nnz], vals[nnz]) */
void orc_csr_apply(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                   const double *vals, const zc *x, zc *y) {
  ORC_PAR
  for (int64_t r = 0; r < n; ++r) {
    zc s = zmk(0.0, 0.0);
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k)
      s = zadd(s, zscale(vals[k], x[col_idx[k]]));
    y[r] = s;
  }
}

/* Lattice site s = x + X*(y + Y*(z + Z*t)); nbr[8*s + 2*mu] = s + mu-hat,
 * nbr[8*s + 2*mu + 1] = s - mu-hat, periodic wrap in every direction. */
void orc_wilson_neighbors(const int32_t dims[4], int32_t *nbr) {
  int64_t vol = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  ORC_PAR
  for (int64_t s = 0; s < vol; ++s) {
    int32_t c[4];
    int64_t rem = s;
    for (int mu = 0; mu < 4; ++mu) { c[mu] = (int32_t)(rem % dims[mu]); rem /= dims[mu]; }
    for (int mu = 0; mu < 4; ++mu) {
      for (int dir = 0; dir < 2; ++dir) {
        int32_t cc[4] = {c[0], c[1], c[2], c[3]};
        cc[mu] = dir == 0 ? (c[mu] + 1) % dims[mu] : (c[mu] - 1 + dims[mu]) % dims[mu];
        int64_t t = cc[0] + (int64_t)dims[0] * (cc[1] + (int64_t)dims[1] * (cc[2] + (int64_t)dims[2] * cc[3]));
        nbr[8 * s + 2 * mu + dir] = (int32_t)t;
      }
    }
  }
}

/* Euclidean gamma matrices in the DeGrand-Rossi (chiral) basis, mu = x,y,z,t;
 * Hermitian, mutually anticommuting, gamma_x gamma_y gamma_z gamma_t =
 * diag(1,1,-1,-1). */
static zc GAMMA[4][4][4];
static int gamma_ready = 0;
static void gamma_init(void) {
  if (gamma_ready) return;
  memset(GAMMA, 0, sizeof(GAMMA));
  /* gamma_x */
  GAMMA[0][0][3] = zmk(0, 1);  GAMMA[0][1][2] = zmk(0, 1);
  GAMMA[0][2][1] = zmk(0, -1); GAMMA[0][3][0] = zmk(0, -1);
  /* gamma_y */
  GAMMA[1][0][3] = zmk(-1, 0); GAMMA[1][1][2] = zmk(1, 0);
  GAMMA[1][2][1] = zmk(1, 0);  GAMMA[1][3][0] = zmk(-1, 0);
  /* gamma_z */
  GAMMA[2][0][2] = zmk(0, 1);  GAMMA[2][1][3] = zmk(0, -1);
  GAMMA[2][2][0] = zmk(0, -1); GAMMA[2][3][1] = zmk(0, 1);
  /* gamma_t */
  GAMMA[3][0][2] = zmk(1, 0);  GAMMA[3][1][3] = zmk(1, 0);
  GAMMA[3][2][0] = zmk(1, 0);  GAMMA[3][3][1] = zmk(1, 0);
  gamma_ready = 1;
}

/*
 * Wilson-Dirac operator (Wilson parameter r = 1), hopping form:
 *   (D_s psi)(n) = psi(n) - kappa * sum_mu [ (1 - s*gamma_mu) U_mu(n) psi(n+mu)
 *                                          + (1 + s*gamma_mu) U_mu(n-mu)^H psi(n-mu) ]
 * s = +1 gives D, s = -1 gives D^H (= gamma5 D gamma5).  bc_t = 1 multiplies
 * hops across the t boundary by -1 (antiperiodic), otherwise periodic.
 * Spinor layout [site][spin][colour]; links [mu][site][a][b].
 */
void orc_wilson_dslash(const int32_t dims[4], double kappa, int32_t bc_t, int32_t sign,
                       const zc *links, const zc *in, zc *out) {
  gamma_init();
  int64_t vol = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * 8 * vol);
  orc_wilson_neighbors(dims, nbr);
  ORC_PAR
  for (int64_t s = 0; s < vol; ++s) {
    int32_t t_coord = (int32_t)(s / ((int64_t)dims[0] * dims[1] * dims[2]));
    zc acc[4][3];
    memset(acc, 0, sizeof(acc));
    for (int mu = 0; mu < 4; ++mu) {
      for (int dir = 0; dir < 2; ++dir) {
        int64_t nb = nbr[8 * s + 2 * mu + dir];
        /* link for this hop: U_mu(n) forward, U_mu(n-mu)^H backward */
        const zc *u = links + ((int64_t)mu * vol + (dir == 0 ? s : nb)) * 9;
        double bc = 1.0;
        if (mu == 3 && bc_t) {
          if (dir == 0 && t_coord == dims[3] - 1) bc = -1.0;
          if (dir == 1 && t_coord == 0) bc = -1.0;
        }
        /* colour: c[sp][a] = (U or U^H) psi(nb)[sp] */
        zc c[4][3];
        for (int sp = 0; sp < 4; ++sp) {
          for (int a = 0; a < 3; ++a) {
            zc v = zmk(0.0, 0.0);
            for (int b = 0; b < 3; ++b) {
              zc uab = dir == 0 ? u[3 * a + b] : zconj(u[3 * b + a]);
              v = zadd(v, zmul(uab, in[12 * nb + 3 * sp + b]));
            }
            c[sp][a] = zscale(bc, v);
          }
        }
        /* spin: (1 -/+ s*gamma_mu) */
        double sg = (dir == 0 ? -1.0 : 1.0) * (double)sign;
        for (int sp = 0; sp < 4; ++sp) {
          for (int a = 0; a < 3; ++a) {
            zc v = c[sp][a];
            for (int q = 0; q < 4; ++q) v = zadd(v, zscale(sg, zmul(GAMMA[mu][sp][q], c[q][a])));
            acc[sp][a] = zadd(acc[sp][a], v);
          }
        }
      }
    }
    for (int sp = 0; sp < 4; ++sp)
      for (int a = 0; a < 3; ++a)
        out[12 * s + 3 * sp + a] = zsub(in[12 * s + 3 * sp + a], zscale(kappa, acc[sp][a]));
  }
  free(nbr);
}

/* y = (dA/dkappa) x for A = D^H D.  D = 1 - kappa H with H the hopping sum
 * of orc_wilson_dslash (sign +1); D^H = 1 - kappa H^H with H^H the sign -1
 * sum.  So dA/dkappa = -(H^H D + D^H H).  H v is formed as v - D(kappa=1) v
 * and H^H v as v - D^H(kappa=1) v.  Returns 0 or ORC_ENOMEM. */
int orc_wilson_dA_dkappa(const int32_t dims[4], double kappa, int32_t bc_t, const zc *links, const zc *x, zc *y) {
  int64_t n = 12 * (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  zc *t1 = (zc *)malloc(sizeof(zc) * n), *t2 = (zc *)malloc(sizeof(zc) * n);
  if (!t1 || !t2) { free(t1); free(t2); return 2; }
  orc_wilson_dslash(dims, kappa, bc_t, +1, links, x, t1);       /* t1 = D x */
  orc_wilson_dslash(dims, 1.0, bc_t, -1, links, t1, t2);        /* t2 = D x - H^H D x */
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) y[i] = zsub(t2[i], t1[i]);    /* y = -H^H D x */
  orc_wilson_dslash(dims, 1.0, bc_t, +1, links, x, t1);         /* t1 = x - H x */
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) t1[i] = zsub(x[i], t1[i]);    /* t1 = H x */
  orc_wilson_dslash(dims, kappa, bc_t, -1, links, t1, t2);      /* t2 = D^H H x */
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) y[i] = zsub(y[i], t2[i]);
  free(t1);
  free(t2);
  return 0;
}

/* Operator description passed from the test harness. */
typedef struct {
  int32_t kind;          /* 0 = real CSR, 1 = Wilson normal A = D^H D, 2 = dense Hermitian */
  int32_t pad_;
  int64_t n;
  const int32_t *row_ptr, *col_idx;
  const double *vals;
  int32_t dims[4];
  double kappa;
  int32_t bc_t, pad2_;
  const zc *links;
  const zc *dense;       /* row-major n x n */
} orc_op;

/* y = A x; returns 0 or ORC_ENOMEM */
int orc_op_apply(const orc_op *A, const zc *x, zc *y) {
  int64_t n = A->n;
  if (A->kind == 0) {
    orc_csr_apply(n, A->row_ptr, A->col_idx, A->vals, x, y);
  } else if (A->kind == 1) {
    zc *t = (zc *)malloc(sizeof(zc) * n);
    if (!t) return ORC_ENOMEM;
    orc_wilson_dslash(A->dims, A->kappa, A->bc_t, +1, A->links, x, t);
    orc_wilson_dslash(A->dims, A->kappa, A->bc_t, -1, A->links, t, y);
    free(t);
  } else {
    ORC_PAR
    for (int64_t r = 0; r < n; ++r) {
      zc s = zmk(0.0, 0.0);
      for (int64_t c = 0; c < n; ++c) s = zadd(s, zmul(A->dense[r * n + c], x[c]));
      y[r] = s;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3: Lanczos version of single seed CG with periodic reorthogonalization */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t m_max;          /* m: maximum number of Lanczos steps (subspace size) */
  int32_t reorth_freq;    /* frequency of reorthogonalization; 0 = never */
  int32_t reorth_passes;  /* classical Gram-Schmidt passes per reorth (1 or 2) */
  int32_t extra_iters;    /* steps taken after the stopping test first holds */
  int32_t x0_zero;        /* 1: initial guesses are zero (no mvp for r_0) */
  int32_t pad_;
  double tol;             /* stop when beta_i |zeta_i| / delta_i <= tol * ||b^1|| */
  double breakdown_rel;   /* stop when beta_i <= breakdown_rel * max_k(|alpha_k| + beta_k + beta_{k-1}) */
} orc_seed_params;

typedef struct {
  int32_t iters;          /* Lanczos steps taken (i at exit) */
  int32_t mvps;           /* operator applies */
  int32_t converged_at;   /* first step at which the stopping test held, or -1 */
  int32_t breakdown;      /* 1 if stopped by a (lucky) breakdown */
  double rho;             /* last residual estimate beta_i |zeta_i| / delta_i */
  double bnorm1;          /* ||b^1|| */
} orc_seed_out;

/* Classical Gram-Schmidt of x against columns 0..k-1 of V (ld = n), repeated
 * `passes` times: h = V^H x computed from the same x, then x -= V h. */
static void cgs(int64_t n, const zc *V, int32_t k, int32_t passes, zc *x, zc *h) {
  for (int32_t p = 0; p < passes; ++p) {
    for (int32_t c = 0; c < k; ++c) h[c] = vdot(n, V + (int64_t)c * n, x);
    for (int32_t c = 0; c < k; ++c) vaxpy(n, zmk(-h[c].re, -h[c].im), V + (int64_t)c * n, x);
  }
}

/*
 * The seed solve of Sec. 3, written as what it is: the Lanczos process on
 * r_0^1 builds the orthonormal basis V and the tridiagonal T (diagonal alpha,
 * off-diagonal beta); CG is the solution of T y = beta_0 e_1 through the LU
 * factorisation T = L U, whose pivots delta_i and multipliers gamma_i are
 * formed one step at a time, with W = V U^{-1} (the w_i) so that
 * x^1 = x_0^1 + W L^{-1} beta_0 e_1 (the zeta_i) grows by one term per step.
 * The other right-hand sides receive the same Galerkin projection over the
 * growing space, x^j = x_0^j + V T^{-1} V^H r_0^j, also one term per step: the
 * eta^j are the entries of L^{-1} V^H r_0^j.  Every few steps the newest
 * basis vector and the next Lanczos direction are made orthogonal again to
 * all stored vectors.
 *
 * B, X: column-major n x nrhs (ld = n).  X holds the initial guesses on entry
 * (ignored when x0_zero) and on exit x^1 (solved) and x^2..x^nrhs (seeded).
 * alpha[m_max], beta[m_max+1] (beta[0] = beta_0), rho_hist[m_max] may be NULL.
 * V may be NULL or n x (m_max+1) to receive the Lanczos vectors as stored.
 * Returns ORC_OK, ORC_ENOTSPD (delta_i <= 0 or not finite), ORC_ENOMEM.
 *
 * Readings where the paper is silent: the second basis vector is f / beta_1,
 * formed exactly as every later one; the first reorthogonalization can come
 * at i = 2 (the first step has none); alpha_i is the real part of v_i^H f;
 * after a reorthogonalization the corrected v_i is what V keeps and what the
 * next step's three-term recurrence uses as v_{i-1}, while alpha_i, w_i and
 * eta^j keep the values computed from v_i before the correction.
 */
int orc_seed_first(const orc_op *A, int32_t nrhs, const zc *B, zc *X,
                   const orc_seed_params *P, orc_seed_out *out,
                   double *alpha, double *beta, double *rho_hist, zc *V_out) {
  int64_t n = A->n;
  int32_t m = P->m_max;
  if (n <= 0 || nrhs < 1 || m < 1) return ORC_EINVAL;
  memset(out, 0, sizeof(*out));
  out->converged_at = -1;
  int status = ORC_OK;

  zc *V = V_out ? V_out : (zc *)malloc(sizeof(zc) * n * ((int64_t)m + 1));
  zc *R0 = (zc *)malloc(sizeof(zc) * n * nrhs);
  zc *f = (zc *)malloc(sizeof(zc) * n);
  zc *w = (zc *)malloc(sizeof(zc) * n);
  zc *tmp = (zc *)malloc(sizeof(zc) * n);
  zc *h = (zc *)malloc(sizeof(zc) * ((int64_t)m + 1));
  zc *eta = (zc *)malloc(sizeof(zc) * nrhs);
  if (!V || !R0 || !f || !w || !tmp || !h || !eta) { status = ORC_ENOMEM; goto done; }

  /* initial residuals of every system */
  for (int32_t j = 0; j < nrhs; ++j) {
    zc *xj = X + (int64_t)j * n, *rj = R0 + (int64_t)j * n;
    const zc *bj = B + (int64_t)j * n;
    if (P->x0_zero) {
      memset(xj, 0, sizeof(zc) * n);
      memcpy(rj, bj, sizeof(zc) * n);
    } else {
      orc_op_apply(A, xj, tmp);
      out->mvps++;
      ORC_PAR
      for (int64_t k = 0; k < n; ++k) rj[k] = zsub(bj[k], tmp[k]);
    }
  }
  out->bnorm1 = vnorm(n, B);

  /* first basis vector from the seed system's residual, first diagonal entry of T */
  double beta0 = vnorm(n, R0);
  if (beta) beta[0] = beta0;
  if (beta0 == 0.0) { out->iters = 0; goto done; }
  zc *v1 = V;
  ORC_PAR
  for (int64_t k = 0; k < n; ++k) v1[k] = zmk(R0[k].re / beta0, R0[k].im / beta0);
  orc_op_apply(A, v1, f);
  out->mvps++;
  double ai = vdot(n, v1, f).re;
  ORC_PAR
  for (int64_t k = 0; k < n; ++k) f[k] = zsub(f[k], zscale(ai, v1[k]));
  if (alpha) alpha[0] = ai;

  /* the LU factorisation starts with the pivot alpha_1; first term of x^1 */
  double delta = ai;
  if (!(delta > 0.0) || !isfinite(delta)) { status = ORC_ENOTSPD; out->iters = 1; goto done; }
  ORC_PAR
  for (int64_t k = 0; k < n; ++k) w[k] = zmk(v1[k].re / delta, v1[k].im / delta);
  double zeta = beta0;
  vaxpy(n, zmk(zeta, 0.0), w, X);

  /* first projection coefficient of every other system */
  for (int32_t j = 1; j < nrhs; ++j) {
    eta[j] = vdot(n, v1, R0 + (int64_t)j * n);
    vaxpy(n, eta[j], w, X + (int64_t)j * n);
  }

  int32_t i = 1;
  double beta_im1 = 0.0;   /* off-diagonal of T above row i (none for i = 1) */
  double tnorm = 0.0;      /* max_k (|alpha_k| + beta_{k-1} + beta_k): row sums of |T| */
  int32_t stop_at = -1;
  for (;;) {
    /* off-diagonal entry beta_i, residual estimate, stopping tests */
    double bi = vnorm(n, f);
    if (beta) beta[i] = bi;
    double row = fabs(ai) + beta_im1 + bi;
    if (row > tnorm) tnorm = row;
    double rho = bi * fabs(zeta) / delta;
    if (rho_hist) rho_hist[i - 1] = rho;
    out->rho = rho;
    out->iters = i;
    if (out->converged_at < 0 && rho <= P->tol * out->bnorm1) {
      out->converged_at = i;
      stop_at = i + P->extra_iters;
    }
    if (bi <= P->breakdown_rel * tnorm) { out->breakdown = 1; break; }
    if (stop_at >= 0 && i >= stop_at) break;
    if (i >= m) break;
    /* next basis vector */
    zc *vnext = V + (int64_t)i * n;
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) vnext[k] = zmk(f[k].re / bi, f[k].im / bi);
    beta_im1 = bi;
    i += 1;
    zc *vi = V + (int64_t)(i - 1) * n, *vim1 = V + (int64_t)(i - 2) * n;

    /* three-term recurrence: diagonal entry alpha_i and the unnormalised next direction */
    orc_op_apply(A, vi, f);
    out->mvps++;
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) f[k] = zsub(f[k], zscale(beta_im1, vim1[k]));
    ai = vdot(n, vi, f).re;
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) f[k] = zsub(f[k], zscale(ai, vi[k]));
    if (alpha) alpha[i - 1] = ai;

    /* one more row of T = L U: multiplier, pivot (positive for a definite T), the new
     * column of W and the new term of x^1 */
    double gam = beta_im1 / delta;
    delta = ai - gam * beta_im1;
    if (!(delta > 0.0) || !isfinite(delta)) { status = ORC_ENOTSPD; out->iters = i; goto done; }
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) {
      zc t = zsub(vi[k], zscale(beta_im1, w[k]));
      w[k] = zmk(t.re / delta, t.im / delta);
    }
    zeta = -gam * zeta;
    vaxpy(n, zmk(zeta, 0.0), w, X);

    /* the same forward substitution for the other systems' projections */
    for (int32_t j = 1; j < nrhs; ++j) {
      zc g = vdot(n, vi, R0 + (int64_t)j * n);
      eta[j] = zsub(g, zscale(gam, eta[j]));
      vaxpy(n, eta[j], w, X + (int64_t)j * n);
    }

    /* periodic reorthogonalization: the newest basis vector against the older ones
     * (then renormalised), and the next direction against all of them */
    if (P->reorth_freq > 0 && i % P->reorth_freq == 0) {
      cgs(n, V, i - 1, P->reorth_passes, vi, h);
      double nv = vnorm(n, vi);
      ORC_PAR
      for (int64_t k = 0; k < n; ++k) vi[k] = zmk(vi[k].re / nv, vi[k].im / nv);
      cgs(n, V, i, P->reorth_passes, f, h);
    }
  }
done:
  if (!V_out) free(V);
  free(R0); free(f); free(w); free(tmp); free(h); free(eta);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Plain CG (Hestenes-Stiefel) on one system, from the given x              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t iters;       /* CG iterations (one mvp each) */
  int32_t mvps;        /* including the true-residual applies */
  int32_t restarts;
  int32_t converged;
  double true_relres;  /* ||b - A x|| / ||b|| at exit */
} orc_cg_out;

/*
 * r = b - A x; stop at once if ||r|| <= tol ||b||.  Otherwise p = r and the
 * Hestenes-Stiefel iteration runs until the recursive residual satisfies
 * ||r_k|| <= tol ||b||.  The true residual is then recomputed; if it exceeds
 * 1.5 tol ||b||, CG restarts from it (at most max_restarts times).
 * Returns ORC_OK or ORC_ENOTCONV.
 */
int orc_cg(const orc_op *A, const zc *b, zc *x, double tol, int32_t maxit,
           int32_t max_restarts, orc_cg_out *out) {
  int64_t n = A->n;
  memset(out, 0, sizeof(*out));
  zc *r = (zc *)malloc(sizeof(zc) * n), *p = (zc *)malloc(sizeof(zc) * n),
     *q = (zc *)malloc(sizeof(zc) * n);
  if (!r || !p || !q) { free(r); free(p); free(q); return ORC_ENOMEM; }
  double bn = vnorm(n, b);
  int status = ORC_ENOTCONV;
  orc_op_apply(A, x, q);
  out->mvps++;
  ORC_PAR
  for (int64_t k = 0; k < n; ++k) r[k] = zsub(b[k], q[k]);
  double rr = vnorm(n, r);
  out->true_relres = bn > 0.0 ? rr / bn : 0.0;
  if (rr <= tol * bn) { out->converged = 1; status = ORC_OK; goto done; }
  for (;;) {
    memcpy(p, r, sizeof(zc) * n);
    double rho = rr * rr;
    int reached = 0;
    while (out->iters < maxit) {
      orc_op_apply(A, p, q);
      out->mvps++;
      out->iters++;
      double pq = vdot(n, p, q).re;
      double al = rho / pq;
      vaxpy(n, zmk(al, 0.0), p, x);
      vaxpy(n, zmk(-al, 0.0), q, r);
      double rn = vnorm(n, r);
      if (rn <= tol * bn) { reached = 1; break; }
      double be = (rn * rn) / rho;
      ORC_PAR
      for (int64_t k = 0; k < n; ++k) p[k] = zadd(r[k], zscale(be, p[k]));
      rho = rn * rn;
    }
    /* true residual */
    orc_op_apply(A, x, q);
    out->mvps++;
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) r[k] = zsub(b[k], q[k]);
    rr = vnorm(n, r);
    out->true_relres = bn > 0.0 ? rr / bn : 0.0;
    if (!reached) break;
    if (rr <= 1.5 * tol * bn) { out->converged = 1; status = ORC_OK; break; }
    if (out->restarts >= max_restarts) break;
    out->restarts++;
  }
done:
  free(r); free(p); free(q);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Multiple seeding (Sec. 2.1, the comparison method)                       */
/* ------------------------------------------------------------------------ */

/* No initial guesses.  For j = 1..nrhs: CG on system j from its current x^j
 * (residual recomputed, one mvp); every CG step, with direction p and
 * q = A p, first projects each later system i over p:
 *   eta = (p^H r^i) / (p^H q),  x^i += eta p,  r^i -= eta q,
 * where r^i is the tracked residual of system i (r^i = b^i at the start).
 * CG stops at ||r^j|| <= tol ||b^j||, then the true residual is computed
 * (one mvp).  iters[j], mvps[j] and relres[j] receive each system's counts;
 * X_seeded (NULL or n x nrhs) receives x^j as it stands when system j's own
 * CG starts, i.e. after the projections over the earlier systems' steps. */
int orc_seed_multiple(const orc_op *A, int32_t nrhs, const zc *B, zc *X, double tol, int32_t maxit,
                      int32_t *iters, int32_t *mvps, double *relres, zc *X_seeded) {
  int64_t n = A->n;
  zc *R = (zc *)malloc(sizeof(zc) * n * nrhs), *r = (zc *)malloc(sizeof(zc) * n),
     *p = (zc *)malloc(sizeof(zc) * n), *q = (zc *)malloc(sizeof(zc) * n);
  if (!R || !r || !p || !q) { free(R); free(r); free(p); free(q); return ORC_ENOMEM; }
  memset(X, 0, sizeof(zc) * n * nrhs);
  memcpy(R, B, sizeof(zc) * n * nrhs);
  int status = ORC_OK;
  for (int32_t j = 0; j < nrhs; ++j) {
    const zc *b = B + (int64_t)j * n;
    zc *x = X + (int64_t)j * n;
    double bn = vnorm(n, b);
    if (X_seeded) memcpy(X_seeded + (int64_t)j * n, x, sizeof(zc) * n);
    iters[j] = 0;
    mvps[j] = 1;
    orc_op_apply(A, x, q);
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) r[k] = zsub(b[k], q[k]);
    double rn = vnorm(n, r);
    if (rn > tol * bn) {
      memcpy(p, r, sizeof(zc) * n);
      double rho = rn * rn;
      while (iters[j] < maxit) {
        orc_op_apply(A, p, q);
        mvps[j]++;
        iters[j]++;
        zc pqz = vdot(n, p, q);
        double al = rho / pqz.re;
        for (int32_t i = j + 1; i < nrhs; ++i) {
          zc *xi = X + (int64_t)i * n, *ri = R + (int64_t)i * n;
          zc num = vdot(n, p, ri);
          double d = pqz.re * pqz.re + pqz.im * pqz.im;
          zc eta = zmk((num.re * pqz.re + num.im * pqz.im) / d, (num.im * pqz.re - num.re * pqz.im) / d);
          vaxpy(n, eta, p, xi);
          vaxpy(n, zmk(-eta.re, -eta.im), q, ri);
        }
        vaxpy(n, zmk(al, 0.0), p, x);
        vaxpy(n, zmk(-al, 0.0), q, r);
        rn = vnorm(n, r);
        if (rn <= tol * bn) break;
        double be = (rn * rn) / rho;
        ORC_PAR
        for (int64_t k = 0; k < n; ++k) p[k] = zadd(r[k], zscale(be, p[k]));
        rho = rn * rn;
      }
    }
    orc_op_apply(A, x, q);
    mvps[j]++;
    ORC_PAR
    for (int64_t k = 0; k < n; ++k) r[k] = zsub(b[k], q[k]);
    relres[j] = bn > 0.0 ? vnorm(n, r) / bn : 0.0;
    if (relres[j] > 1.5 * tol) status = ORC_ENOTCONV;
  }
  free(R); free(r); free(p); free(q);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: Galerkin projection of a later system over x_cg              */
/* ------------------------------------------------------------------------ */

/* delta = x_cg^H r_bpr / x_cg^H r_bcg; x_bpr += delta x_cg; r_bpr -= delta r_bcg */
void orc_related_project(int64_t n, const zc *x_cg, const zc *r_bcg, zc *x_bpr, zc *r_bpr) {
  zc num = vdot(n, x_cg, r_bpr), den = vdot(n, x_cg, r_bcg);
  double dd = den.re * den.re + den.im * den.im;
  zc d = zmk((num.re * den.re + num.im * den.im) / dd, (num.im * den.re - num.re * den.im) / dd);
  vaxpy(n, d, x_cg, x_bpr);
  vaxpy(n, zmk(-d.re, -d.im), r_bcg, r_bpr);
}

/* ------------------------------------------------------------------------ */
/* Pins: dense Cholesky solve and tridiagonal eigenvalues                   */
/* ------------------------------------------------------------------------ */

/* Solve A x = b for Hermitian positive definite A (row-major n x n) by
 * A = L L^H.  Returns ORC_ENOTSPD if a pivot is not positive. */
int orc_cholesky_solve(int64_t n, const zc *A, const zc *b, zc *x) {
  zc *L = (zc *)calloc((size_t)(n * n), sizeof(zc));
  zc *y = (zc *)malloc(sizeof(zc) * n);
  if (!L || !y) { free(L); free(y); return ORC_ENOMEM; }
  for (int64_t j = 0; j < n; ++j) {
    double d = A[j * n + j].re;
    for (int64_t k = 0; k < j; ++k) d -= L[j * n + k].re * L[j * n + k].re + L[j * n + k].im * L[j * n + k].im;
    if (!(d > 0.0)) { free(L); free(y); return ORC_ENOTSPD; }
    double ljj = sqrt(d);
    L[j * n + j] = zmk(ljj, 0.0);
    for (int64_t r = j + 1; r < n; ++r) {
      zc s = A[r * n + j];
      for (int64_t k = 0; k < j; ++k) s = zsub(s, zmul(L[r * n + k], zconj(L[j * n + k])));
      L[r * n + j] = zscale(1.0 / ljj, s);
    }
  }
  for (int64_t r = 0; r < n; ++r) {            /* L y = b */
    zc s = b[r];
    for (int64_t k = 0; k < r; ++k) s = zsub(s, zmul(L[r * n + k], y[k]));
    y[r] = zscale(1.0 / L[r * n + r].re, s);
  }
  for (int64_t r = n - 1; r >= 0; --r) {       /* L^H x = y */
    zc s = y[r];
    for (int64_t k = r + 1; k < n; ++k) s = zsub(s, zmul(zconj(L[k * n + r]), x[k]));
    x[r] = zscale(1.0 / L[r * n + r].re, s);
  }
  free(L); free(y);
  return ORC_OK;
}

/* number of eigenvalues of the symmetric tridiagonal (a[m], b[m-1]) below x */
static int32_t sturm_count(int32_t m, const double *a, const double *b, double x) {
  int32_t count = 0;
  double d = 1.0;
  for (int32_t k = 0; k < m; ++k) {
    double off = k > 0 ? b[k - 1] * b[k - 1] : 0.0;
    d = (a[k] - x) - (k > 0 ? off / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) count++;
  }
  return count;
}

/* All eigenvalues (ascending) of the symmetric tridiagonal with diagonal
 * a[0..m-1] and off-diagonal b[0..m-2], by bisection on Sturm counts. */
void orc_tridiag_eigs(int32_t m, const double *a, const double *b, double *eig) {
  double lo = a[0], hi = a[0];
  for (int32_t k = 0; k < m; ++k) {
    double r = (k > 0 ? fabs(b[k - 1]) : 0.0) + (k < m - 1 ? fabs(b[k]) : 0.0);
    if (a[k] - r < lo) lo = a[k] - r;
    if (a[k] + r > hi) hi = a[k] + r;
  }
  double span = hi - lo;
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
  for (int32_t k = 0; k < m; ++k) {
    double l = lo, h = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (l + h);
      if (mid <= l || mid >= h) break;
      if (sturm_count(m, a, b, mid) > k) h = mid; else l = mid;
    }
    eig[k] = 0.5 * (l + h);
  }
}
