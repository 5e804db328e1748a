/*
 * ppgmres.h -- C ABI of libppgmres, a GB300 (sm_103a) implementation of
 * polynomial-preconditioned GMRES with the GMRES polynomial in root form
 * (Loe & Morgan, "Toward Efficient Polynomial Preconditioning for GMRES").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Sparse matrices are CSR with int32 indices (ppg_csr).  Column indices
 *    are sorted within a row and lie in [0, n).  All CSR arrays and all
 *    vectors passed to device entry points are DEVICE pointers owned by the
 *    caller; the library never frees them and never keeps them after the
 *    call returns.
 *  - Vectors have n entries of the CSR's dtype unless stated otherwise
 *    (double for PPG_F64, float for PPG_F32).  Input and output vectors of
 *    one call must not alias.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it.  Entry points that need a result on
 *    the host (build_poly, solve, stability_check, csr_validate)
 *    synchronise the stream before returning; apply_poly, apply_phi, spmv,
 *    csr_transpose and adjoint_vals_grad are asynchronous.
 *  - Scratch memory is taken stream-ordered (cudaMallocAsync) and returned
 *    (cudaFreeAsync) before the call returns.
 *  - Return codes: 0 = success, > 0 = soft status, < 0 = error (see
 *    PPG_* below; ppg_strerror gives a message).  No C++ exception crosses
 *    this interface.  After PPG_ERR_CUDA the CUDA error is also reported by
 *    ppg_last_cuda_error().
 *
 * Host-only entry points (marked HOST) run on the CPU and need no GPU.
 */
#ifndef PPGMRES_H
#define PPGMRES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPG_ABI_VERSION 2

/* status codes */
#define PPG_OK                0
#define PPG_NOT_CONVERGED     1   /* max_cycles reached; x holds the last iterate */
#define PPG_LUCKY_BREAKDOWN   2   /* build_poly: Krylov space invariant before d steps */
#define PPG_ERR_ARG          -1   /* bad argument (NULL, size, aliasing, dtype) */
#define PPG_ERR_CSR          -2   /* CSR structure invalid */
#define PPG_ERR_SINGULAR_H   -3   /* H_dd singular: harmonic Ritz values undefined */
#define PPG_ERR_NONFINITE    -4   /* NaN or Inf met in a residual or in H */
#define PPG_ERR_CUDA         -5   /* a CUDA runtime call failed */
#define PPG_ERR_CAPACITY     -6   /* ppg_roots arrays too small; n_total = needed */
#define PPG_ERR_EIG          -7   /* Hessenberg QR did not converge */
#define PPG_ERR_NOMEM        -8   /* device scratch allocation failed */
#define PPG_ERR_TOO_LARGE    -9   /* n above PPG_NOALLOC_MAX_N (ppg_apply_poly_noalloc) */
#define PPG_ERR_TIMEOUT     -10   /* a bounded wait inside a kernel gave up (data staging or
                                     a grid-wide barrier did not complete in time) */

/* Largest n that ppg_apply_poly_noalloc accepts (its fixed work area). */
#define PPG_NOALLOC_MAX_N 1048576

/* dtypes */
#define PPG_F64 0
#define PPG_F32 1

/* CSR matrix (Algorithms 1 and 3 take "sparse matrix A"): device pointers. */
typedef struct ppg_csr {
    int32_t n;              /* rows = columns */
    int32_t nnz;
    const int32_t* rowptr;  /* [n+1], rowptr[0] = 0, rowptr[n] = nnz */
    const int32_t* colind;  /* [nnz] */
    const void* vals;       /* [nnz] double (PPG_F64) or float (PPG_F32) */
    int32_t dtype;
} ppg_csr;

/* Roots of the GMRES residual polynomial pi (eq 2.1), Leja-ordered, with
 * the copies added by the stability control of Algorithm 2.  HOST arrays
 * owned by the caller, each of `capacity` entries.  Conjugate pairs are
 * adjacent, +Im member first, and are exact conjugates; a root is real iff
 * im == 0.  log10_pof (may be NULL) receives log10 pof(k) of the n_orig
 * original roots in Leja order. */
typedef struct ppg_roots {
    int32_t n_orig;     /* original degree d actually reached */
    int32_t n_added;    /* roots added by Algorithm 2 */
    int32_t n_total;    /* n_orig + n_added = degree of pi and phi */
    int32_t capacity;   /* entries available in re/im */
    double* re;
    double* im;
    double* log10_pof;  /* optional, n_orig entries */
} ppg_roots;

typedef struct ppg_opts {
    int32_t max_cycles;            /* restart cap (default 10000) */
    int32_t stability_control;     /* 1: add roots by Algorithm 2 (default 1) */
    double  pof_threshold_log10;   /* default 4  (pof > 1e4 adds a root) */
    double  pof_step_log10;        /* default 14 (one more per factor 1e14) */
    int32_t timing;                /* 1: record CUDA-event times into stats */
    int32_t x0_given;              /* 1: x holds the initial guess (default 0: x0 = 0) */
    int32_t batch_mode;            /* ppg_solve_batched: 0 = every restart cycle of every
                                      solve in one persistent cooperative launch (default),
                                      1 = one CUDA graph per restart cycle, replayed by a
                                      host loop */
    int32_t cgs2_fused;            /* 1: run CGS2's second update and dot pass as one fused
                                      pass over the basis (3/4 of the bytes, the same FP64
                                      multiply-adds; measured slower on GB300, where the
                                      FP64 pipe bounds CGS2); default 0 */
    double  wait_timeout_ms;       /* limit of each grid-wide barrier wait of the persistent
                                      launch (default 5000); a wait that runs out ends the
                                      launch with PPG_ERR_TIMEOUT */
} ppg_opts;

typedef struct ppg_stats {
    int64_t iters;          /* Arnoldi steps of the outer (F)GMRES */
    int64_t cycles;         /* restarts + 1 */
    int64_t mvps;           /* every SpMV: d per phi(A)v, d-1 per p(A)v, 1 per residual */
    int64_t dots;           /* dot products and norms of length n */
    int64_t launches;       /* kernels this call launched */
    double  true_relres;    /* ||b - A x|| / ||b|| at return */
    double  est_relres;     /* last shortcut residual |g_{j+1}| / ||b|| */
    int32_t converged;
    int32_t pad_;
    /* filled when opts.timing = 1: the fused SpMV-root kernels of the
     * polynomial chains (Algorithms 1 and 3) */
    double  poly_ms;        /* summed CUDA-event time of those launches */
    int64_t poly_launches;
    double  poly_bytes;     /* algorithmic bytes of those launches */
    double  ortho_ms;       /* CGS2 + Givens kernels */
} ppg_stats;

/* ---- library ---------------------------------------------------------- */

int32_t     ppg_abi_version(void);
const char* ppg_strerror(int32_t code);
const char* ppg_last_cuda_error(void);
void        ppg_default_opts(ppg_opts* opts);
/* Kernels launched so far by the calling host thread (all entry points). */
int64_t     ppg_launch_count(void);

/* ---- HOST: polynomial construction steps (Algorithm 4 step 1(b)-(c)) ---- */

/* Harmonic Ritz values theta_1..theta_d (Algorithm 4 step 1(b)): the
 * eigenvalues of H_dd + h_{d+1,d}^2 f e_d^T with H_dd^T f = e_d.  Hbar is
 * the (d+1) x d upper Hessenberg matrix of the Arnoldi relation
 * A V_d = V_{d+1} Hbar, column-major with leading dimension ldh >= d+1.
 * re/im receive d values (unordered).  HOST.  Errors: PPG_ERR_ARG,
 * PPG_ERR_SINGULAR_H, PPG_ERR_EIG, PPG_ERR_NONFINITE. */
int32_t ppg_harmonic_ritz(const double* Hbar, int32_t ldh, int32_t d,
                          double* re, double* im);

/* Modified Leja ordering (Section 2; Algorithm 2 step 1) of k roots closed
 * under conjugation: largest modulus first, then each next root maximises
 * the sum of log-distances to those chosen; a non-real root is followed by
 * its conjugate (+Im first); ties go to the larger real part, then the
 * larger imaginary part.  HOST.  Errors: PPG_ERR_ARG (not conjugation
 * closed). */
int32_t ppg_leja_order(int32_t k, const double* re, const double* im,
                       double* re_out, double* im_out);

/* Algorithm 2 steps 2-3 on k Leja-ordered roots: pof(k) =
 * prod_{i != k} |1 - theta_k/theta_i|; ceil((log10 pof - thr)/step) copies
 * when positive; the first copy is appended, further copies spread evenly
 * between the root and the end of the list (pairs kept together).  Writes
 * out->re/im/n_*.  HOST.  Errors: PPG_ERR_ARG, PPG_ERR_CAPACITY. */
int32_t ppg_add_roots(int32_t k, const double* re, const double* im,
                      double thr_log10, double step_log10, ppg_roots* out);

/* Steps 1(b) and 1(c) together: harmonic Ritz values of Hbar, Leja order,
 * and (if opts->stability_control) root adding.  HOST. */
int32_t ppg_roots_from_hessenberg(const double* Hbar, int32_t ldh, int32_t d,
                                  const ppg_opts* opts, ppg_roots* out);

/* HOST: check CSR structure held in host memory (rowptr monotone from 0 to
 * nnz, colind sorted within rows and in range).  Returns PPG_OK or
 * PPG_ERR_CSR. */
int32_t ppg_csr_validate_host(int32_t n, int32_t nnz, const int32_t* rowptr,
                              const int32_t* colind);

/* ---- DEVICE entry points ---------------------------------------------- */

/* Algorithm 4 step 1: one cycle of GMRES(d) (d Arnoldi steps, CGS2) from
 * the device vector v0 (FP64, need not be normalised), then harmonic Ritz
 * values, Leja order and root adding on the host in FP64.  A must be
 * PPG_F64.  Hbar_host (nullable) receives the (d+1) x d Hessenberg matrix,
 * column-major, ld = d+1.  Returns PPG_LUCKY_BREAKDOWN (with
 * out->n_orig < d) if h_{j+1,j} <= 1e-13 ||A v_j|| at some step.
 * Synchronises `stream`. */
int32_t ppg_build_poly(const ppg_csr* A, int32_t d, const double* v0,
                       const ppg_opts* opts, ppg_roots* out, double* Hbar_host,
                       void* stream);

/* y = p(A) v by Algorithm 3: d-1 fused SpMV-root passes (two per conjugate
 * pair, the last pair's second one omitted), vectors in A's dtype.  For
 * PPG_F32 the root coefficients 1/theta, 2a and 1/(a^2+b^2) are rounded to
 * float.  Asynchronous.
 *
 * L2: the chains of this call (and of ppg_apply_phi and the solvers) set
 * the persisting-L2 set-aside of the current device's CUDA context -- a
 * limit of this process's context, never a device setting: when the matrix
 * and three vectors fit in 80 % of L2, a set-aside sized for the matrix,
 * which then stays resident across the roots; otherwise 48 MB, which holds
 * the nonzeros of the matrix's leading rows while the rest streams. */
int32_t ppg_apply_poly(const ppg_csr* A, const ppg_roots* r, const void* v,
                       void* y, void* stream);

/* y = p(A) v exactly as ppg_apply_poly computes it, for callers that cannot
 * allocate device memory at call time: their GPU memory is already held by
 * another allocator (for example a framework's caching allocator that has
 * reserved the whole device), or an allocation or free would synchronise
 * the device or could fail under memory pressure in the middle of their
 * work.  The paper has no counterpart: this is a deployment variant.
 *
 * It allocates nothing.  Its three work vectors live in one fixed array of
 * 3 * PPG_NOALLOC_MAX_N doubles (24 MiB) compiled into the library; every
 * GPU that loads the library holds that array until the process exits.
 * n > PPG_NOALLOC_MAX_N is rejected with PPG_ERR_TOO_LARGE before any work
 * is enqueued.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture (a first call made while `stream`
 * is capturing returns PPG_ERR_ARG and enqueues nothing).  Unlike
 * ppg_apply_poly it never reserves an L2 set-aside for the matrix, so
 * apart from that lookup it changes no state of the CUDA context.  The
 * argument checks are those of ppg_apply_poly (PPG_ERR_ARG for a NULL or
 * aliased vector, a bad CSR descriptor, or a root list that is not finite,
 * has a zero root or an unpaired complex root).  All calls share the one array and
 * it keeps the last call's contents (nothing in it needs to start at zero:
 * each call writes every slot before reading it), so calls whose GPU work
 * overlaps -- on different streams or host threads -- race and give wrong
 * results; serialise them.  v and y are caller-owned device vectors as for
 * ppg_apply_poly.  Asynchronous on `stream`. */
int32_t ppg_apply_poly_noalloc(const ppg_csr* A, const ppg_roots* r,
                               const void* v, void* y, void* stream);

/* y = phi(A) v = v - pi(A) v by Algorithm 1: d fused SpMV-root passes.
 * Asynchronous. */
int32_t ppg_apply_phi(const ppg_csr* A, const ppg_roots* r, const void* v,
                      void* y, void* stream);

/* y = A x.  Asynchronous. */
int32_t ppg_spmv(const ppg_csr* A, const void* x, void* y, void* stream);

/* Algorithm 4 step 2: restarted GMRES(m) on phi(A) y = b with phi applied
 * by Algorithm 1, and x = p(A) y by Algorithm 3 at each restart; the next
 * cycle starts from the true residual b - A x.  r == NULL or
 * r->n_total == 0 runs plain GMRES(m) on A.  CGS2 orthogonalisation,
 * Givens least squares; a cycle ends at m steps or when the shortcut
 * residual |g_{j+1}| <= tol ||b||; the solve converges when the true
 * residual ||b - A x|| <= tol ||b||.  A PPG_F64; b, x device double.
 * Returns PPG_OK, PPG_NOT_CONVERGED or an error.  Synchronises. */
int32_t ppg_solve(const ppg_csr* A, const ppg_roots* r, const double* b,
                  double* x, int32_t m, double tol, const ppg_opts* opts,
                  ppg_stats* stats, void* stream);

/* Precision form: flexible GMRES(m) in FP64 with the right preconditioner
 * z_j = p(A) v_j computed by Algorithm 3 in FP32 on A32 (the same matrix
 * with float values; rowptr/colind may be shared with A64).  The Arnoldi
 * orthogonalisation, Givens least squares, w = A64 z_j and the true
 * residual are FP64.  x = x0 + Z y.  Synchronises. */
int32_t ppg_solve_flex(const ppg_csr* A64, const ppg_csr* A32,
                       const ppg_roots* r, const double* b, double* x,
                       int32_t m, double tol, const ppg_opts* opts,
                       ppg_stats* stats, void* stream);

/* Polynomial construction on a composite operator (Section 6): one cycle of
 * GMRES(d) with the operator phi_inner(A) (phi_inner applied by Algorithm 1
 * with the roots `inner`) from v0, harmonic Ritz values, Leja order and
 * root adding: the roots of the outer polynomial phi_2 in double
 * polynomial preconditioning.  inner == NULL gives ppg_build_poly.
 * Synchronises. */
int32_t ppg_build_poly_composite(const ppg_csr* A, const ppg_roots* inner, int32_t d,
                                 const double* v0, const ppg_opts* opts, ppg_roots* out,
                                 double* Hbar_host, void* stream);

/* Double polynomial preconditioning (Section 6): restarted GMRES(m) on
 * phi_2(phi_1(A)) z = b with phi_1 from r1 and phi_2 from r2 (built by
 * ppg_build_poly_composite), x = p_1(A) p_2(phi_1(A)) z.  Each restart
 * starts from the true residual b - phi_1(A) x' of the accumulated
 * x' = p_2(phi_1(A)) z; the returned x is p_1(A) x'.  stats.mvps counts every
 * SpMV (d_1 per product with phi_1(A)).  x0_given is not supported.
 * Synchronises. */
int32_t ppg_solve_double(const ppg_csr* A, const ppg_roots* r1, const ppg_roots* r2,
                         const double* b, double* x, int32_t m, double tol,
                         const ppg_opts* opts, ppg_stats* stats, void* stream);

/* PP-GMRES with the polynomial changed at every restart (Section 5.2): at the
 * start of each cycle a degree-d polynomial is built by GMRES(d) from the
 * current residual (the first cycle from b), then one GMRES(m) cycle runs on
 * phi(A) and x += p(A) y.  stats.mvps includes the d SpMVs of every
 * construction.  x0_given is not supported.  Synchronises. */
int32_t ppg_solve_chpoly(const ppg_csr* A, int32_t d, const double* b, double* x,
                         int32_t m, double tol, const ppg_opts* opts, ppg_stats* stats,
                         void* stream);

/* Batching form: nsys independent systems A_s x = b_s with nrhs (1 or 4)
 * right-hand sides each, solved together.  Each system gets its own
 * polynomial from one batched GMRES(d) run (Algorithm 4 step 1; v0[s] is
 * system s's random start vector) and is solved by flexible GMRES(m) in
 * FP64 with z = p(A_s) v applied by Algorithm 3 in FP32 (the precision
 * form of ppg_solve_flex).  All systems and right-hand sides advance in the
 * same launches: the systems are packed block-diagonally (each padded to
 * 256-row tiles) and the right-hand sides interleaved.  With
 * opts->batch_mode = 0 (default) every restart cycle of every solve runs
 * in ONE persistent cooperative kernel launch (captured as a one-node CUDA
 * graph on `stream`, launched directly on the legacy default stream), its
 * phases separated by grid-wide barriers whose waits are bounded by
 * opts->wait_timeout_ms (PPG_ERR_TIMEOUT when one runs out); with
 * batch_mode = 1 a restart cycle of the whole batch is captured as a CUDA
 * graph of many kernels and replayed once per cycle from a host loop.  The
 * rows per group of the FP32 root step (64, 128 or 256) are chosen by
 * timing the candidates on the batch (cached per batch shape).
 *   As      host array of nsys CSR descriptors (PPG_F64, device pointers)
 *   B, X    host arrays of nsys device pointers, each n_s * nrhs doubles,
 *           column-major (right-hand side k at offset k * n_s)
 *   v0      host array of nsys device pointers (n_s doubles each)
 *   roots_out (nullable) nsys caller-owned ppg_roots receiving each
 *           system's roots; relres_out / iters_out (nullable) host arrays
 *           of nsys * nrhs entries (solve s * nrhs + k): final true relative
 *           residual and Arnoldi steps.
 * Packed sizes must stay below 2^31 entries.  Returns PPG_OK when every
 * solve converged, PPG_NOT_CONVERGED otherwise.  Synchronises. */
int32_t ppg_solve_batched(int32_t nsys, const ppg_csr* As, int32_t nrhs,
                          const double* const* B, double* const* X,
                          const double* const* v0, int32_t d, int32_t m, double tol,
                          const ppg_opts* opts, ppg_roots* roots_out, ppg_stats* stats,
                          double* relres_out, int32_t* iters_out, void* stream);

/* Stability check StCh of Section 3.5: ||r1 - r2|| with r1 = b - A p(A) b
 * (Algorithm 3) and r2 = pi(A) b = b - phi(A) b (Algorithm 1).  A PPG_F64,
 * b device double.  Writes the host double *stch.  Synchronises. */
int32_t ppg_stability_check(const ppg_csr* A, const ppg_roots* r,
                            const double* b, double* stch, void* stream);

/* Outcome of ppg_build_poly_checked. */
typedef struct ppg_poly_check {
    int32_t d_requested;   /* degree asked for */
    int32_t d_chosen;      /* original degree of the returned polynomial */
    int32_t n_tried;       /* degrees checked, the requested one first */
    int32_t pad_;
    double  stch;          /* StCh of the returned polynomial */
    double  stch_first;    /* StCh at the first degree checked */
} ppg_poly_check;

/* Algorithm 4 step 1 followed by the stability check of Section 3.5, which
 * the paper applies once the polynomial is determined and before the
 * solve, lowering the degree when instability is predicted.  The degree-d
 * polynomial is built as by ppg_build_poly; then, with the unit vector
 * u = b / ||b|| (u = v0 / ||v0|| when b is NULL), StCh = ||(u - A p(A) u) -
 * pi(A) u|| is computed (Algorithms 3 and 1, as ppg_stability_check).
 * While StCh > stch_tol and the degree is above d_min, the degree is
 * halved (d' = max(d_min, d / 2); the paper does not say by how much) and
 * the roots of GMRES(d') from the same v0 -- the leading (d'+1) x d' block
 * of the same Arnoldi run, so no further Arnoldi steps -- are formed,
 * ordered, augmented by Algorithm 2 (opts) and checked in turn.  `out`
 * receives the last polynomial checked; info (nullable) the degrees and
 * StCh values.  A StCh that overflows counts as above any tolerance.  If
 * the floor is reached with StCh still above stch_tol the call returns
 * PPG_OK with info->stch > stch_tol.  A PPG_F64; v0, b device double.
 * Returns PPG_OK, PPG_LUCKY_BREAKDOWN (as ppg_build_poly) or an error.
 * Synchronises. */
int32_t ppg_build_poly_checked(const ppg_csr* A, int32_t d, const double* v0,
                               const double* b, double stch_tol, int32_t d_min,
                               const ppg_opts* opts, ppg_roots* out,
                               ppg_poly_check* info, void* stream);

/* ---- Multi-root fused sweep (the matrix-powers idea of Section 1) ------- */

/* A plan for applying Algorithm 3 in FP32 with both SpMV passes of each
 * conjugate pair in one pass over the matrix.  The matrix is reordered
 * symmetrically (row i of the plan's matrix is row perm[i] of A, its
 * entries in their stored order, columns relabelled) so that consecutive
 * tiles of tile_rows rows are compact; each tile's halo (the rows outside
 * it that its rows reference) is listed.  A pair then runs as one launch:
 * tmp = 2a prod - A prod over the tile and its halo into shared memory,
 * then A tmp for the tile's rows.  Every row keeps the unfused arithmetic,
 * so results are bit-identical to ppg_apply_poly on A.
 *   A          PPG_F32 CSR (device), structurally suited to tiling (the
 *              plan copies what it needs; A may be freed afterwards)
 *   perm_host  HOST array of n row indices (new -> old), a permutation, or
 *              NULL: rows are grouped by breadth-first growth over the
 *              pattern of A from the lowest-numbered row not yet placed
 *   tile_rows  rows per tile, a multiple of 32 in [32, 16384]
 *   fuse       1: fuse pairs when the halos total at most 60 % of n and a
 *              tile fits in shared memory; 0: never (the plain chain on the
 *              reordered matrix, for comparison)
 * The plan owns device memory (cudaMalloc, about the size of A plus 8n
 * bytes) until ppg_sweep_plan_destroy.  Synchronises `stream`.  Errors:
 * PPG_ERR_ARG (bad perm, tile_rows), PPG_ERR_CSR, PPG_ERR_NOMEM. */
typedef struct ppg_sweep_plan ppg_sweep_plan;

typedef struct ppg_sweep_info {
    int32_t n, nnz, tile_rows, ntiles;
    int32_t max_halo;       /* largest halo of one tile */
    int32_t fused;          /* 1 when pairs run fused */
    int64_t halo_total;     /* sum of the tiles' halo sizes */
    double  halo_fraction;  /* halo_total / n */
} ppg_sweep_info;

int32_t ppg_sweep_plan_create(const ppg_csr* A, const int32_t* perm_host, int32_t tile_rows,
                              int32_t fuse, ppg_sweep_plan** out, void* stream);
int32_t ppg_sweep_plan_info(const ppg_sweep_plan* plan, ppg_sweep_info* info);
void    ppg_sweep_plan_destroy(ppg_sweep_plan* plan);

/* y = p(A) v (Algorithm 3, FP32 vectors in A's original ordering) through a
 * plan: v is permuted into the plan's ordering, the chain runs with each
 * non-final pair fused, and the result is permuted back.  Bit-identical to
 * ppg_apply_poly on the plan's A.  Asynchronous. */
int32_t ppg_apply_poly_sweep(const ppg_sweep_plan* plan, const ppg_roots* r, const void* v,
                             void* y, void* stream);

/* The precision form (as ppg_solve_flex) with z_j = p(A) v_j applied
 * through a plan of the FP32 matrix: identical iterates to ppg_solve_flex
 * with that matrix.  A64 PPG_F64 with the plan's n.  Synchronises. */
int32_t ppg_solve_flex_sweep(const ppg_csr* A64, const ppg_sweep_plan* plan,
                             const ppg_roots* r, const double* b, double* x, int32_t m,
                             double tol, const ppg_opts* opts, ppg_stats* stats,
                             void* stream);

/* Transposed CSR of A (for the adjoint solve with A^T): rowptr_t [n+1],
 * colind_t [nnz], vals_t [nnz] in A's dtype, all device, caller-owned.
 * perm (nullable, [nnz]) receives for each entry of A^T the index of the
 * same entry in A.  Columns of A^T come out sorted.  Asynchronous. */
int32_t ppg_csr_transpose(const ppg_csr* A, int32_t* rowptr_t,
                          int32_t* colind_t, void* vals_t, int32_t* perm,
                          void* stream);

/* Adjoint gradient on the sparsity pattern: for x solving A x = b and
 * lambda solving A^T lambda = dL/dx, dL/dvals[k] = -lambda[row(k)] *
 * x[colind[k]] (dL/db = lambda needs no kernel).  FP64.  Asynchronous. */
int32_t ppg_adjoint_vals_grad(const ppg_csr* A, const double* lambda,
                              const double* x, double* gvals, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PPGMRES_H */
