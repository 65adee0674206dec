/* feti.h -- C ABI of the GB300 FETI dual-operator library.
 *
 * The library assembles and applies the FETI dual operator
 *     F = sum_i B_i K_i^+ B_i^T                       (arXiv 2502.08382, Sec. II, eqs. 6-9)
 * explicitly on one GPU: for every subdomain i it regularises K_i with fixing
 * DOFs (K^+ = K_reg^{-1}, Sec. III), factorises K_reg = L L^T (Sec. III), forms
 * X_i = L^{-1} P B_i^T with a pruned triangular solve and F_i = X_i^T X_i
 * (the SYRK path of Sec. IV, Table I), and applies F p every PCPG iteration
 * (Algorithm 1) as a batched packed-tile SYMV with the scatter/gather of
 * Algorithm 2 fused in.
 *
 * Conventions for every entry point:
 *  - Host pointers are borrowed for the duration of the call and deep-copied;
 *    the caller keeps ownership.
 *  - Device pointers (suffix _dev) are caller-owned, hold FP64 values, and are
 *    used on the context's stream (feti_options.stream); calls are ordered on
 *    that stream and return before the GPU work completes unless stated.
 *  - Every call returns a feti_status; nothing is thrown across the ABI.
 *    The first error is sticky: later calls on the same context return
 *    FETI_ERR_STATE until feti_destroy.  FETI_ERR_NOT_CONVERGED is
 *    informative and not sticky.  feti_last_error gives the message.
 *  - Dual vectors have n_lambda entries in the global multiplier order.
 */
#ifndef FETI_GB300_H
#define FETI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FETI_OK = 0,
  FETI_ERR_ARG = 1,           /* invalid argument (shape, index, missing pointer) */
  FETI_ERR_ALLOC = 2,         /* device allocation failed */
  FETI_ERR_NOT_SPD = 3,       /* a Cholesky pivot of some K_reg,i was not positive */
  FETI_ERR_NOT_CONVERGED = 4, /* PCPG stopped at maxit or broke down (informative) */
  FETI_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  FETI_ERR_STATE = 6,         /* call out of order, or an earlier error is sticky */
  FETI_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up */
} feti_status;

typedef enum {
  FETI_PREC_FP64 = 0,       /* FP64 everywhere; F_i stored as FP64 tiles */
  FETI_PREC_TF32 = 1,       /* TRSM updates / SYRK on tensor cores in TF32, F_i as FP32 tiles */
  FETI_PREC_SPLIT_BF16 = 2  /* as TF32 but each FP32 operand split into two bf16 halves */
} feti_precision;

/* One subdomain (Sec. II, eq. 2 block i).  All arrays are host memory. */
typedef struct {
  int32_t n;                  /* DOFs of the subdomain */
  int64_t nnz;                /* entries of K_i */
  const int64_t* K_rowptr;    /* [n+1] CSR row pointers of the FULL symmetric K_i */
  const int32_t* K_col;       /* [nnz] column indices, sorted within each row */
  const double* K_val;        /* [nnz] values */
  int32_t m;                  /* rows of B_i (multipliers touching this subdomain) */
  const int64_t* B_rowptr;    /* [m+1] CSR of B_i (m x n); exactly one entry per row */
  const int32_t* B_col;       /* [m] local DOF of each row */
  const double* B_val;        /* [m] +1 or -1 */
  const int32_t* B_lambda;    /* [m] global multiplier id of each row (strictly increasing) */
  int32_t d;                  /* dimension of ker K_i (0: not floating, no regularisation) */
  const double* R;            /* [n*d] column-major basis of ker K_i (eq. 4) */
  const double* f;            /* [n] load vector */
  int32_t nfix;               /* fixing DOFs; must equal d (a generalised inverse needs it) */
  const int32_t* fix_dofs;    /* [nfix] DOFs penalised by rho = max diag K_i */
  const double* coords;       /* [n*3] node coordinates of each DOF, or NULL (ordering hint) */
  int32_t nelem, edofs;       /* optional element data for feti_adjoint (0 if unused; edofs <= 32) */
  const int32_t* elem_dofs;   /* [nelem*edofs] local DOFs of each element */
  const double* dKe;          /* [nelem*edofs*edofs] d K_e / d theta_e of each element, row-major in the
                                 element's DOF order; when NULL, the compact form below is used */
  const double* dKe_ref;      /* [edofs*edofs] shared reference element derivative (compact form) */
  const double* dKe_scale;    /* [nelem] compact form: d K_e / d theta_e = dKe_scale[e] * dKe_ref */
} feti_subdomain;

typedef struct {
  int32_t nsub;
  const feti_subdomain* sub;  /* [nsub] */
  int32_t n_lambda;           /* length of the dual vectors */
  const double* c;            /* [n_lambda] right-hand side of the gluing/Dirichlet rows (eq. 2) */
} feti_problem;

typedef struct {
  feti_precision prec;
  int32_t refine_every;       /* PCPG: recompute the FP64 residual every k iterations (0 = never) */
  double tol;                 /* PCPG: stop when ||P r|| <= tol * ||P r_0||, or at the rounding level
                                 ||P r|| <= 64 eps (||d|| + ||F lambda_0||) */
  int32_t maxit;
  int32_t recompute_X;        /* 1 = do not keep X_i = L_i^{-1} P B_i^T after feti_assemble (it is an
                                 intermediate of the assembly) nor the FP64 X_i of feti_adjoint after that
                                 call: both are released and recomputed from L_i when next needed, for
                                 problems where HBM is short; 0 = keep both buffers for reuse */
  void* (*dev_alloc)(size_t bytes, void* ctx);  /* optional device allocator (NULL: cudaMalloc) */
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  void* stream;               /* cudaStream_t; NULL = legacy default stream */
  int32_t leaf_dofs;          /* nested-dissection leaf size (0 = 16) */
  int32_t use_coords;         /* 1 = coordinate bisection when coords are given */
  double refine_drop;         /* PCPG: also recompute the FP64 residual once ||P r|| has dropped by this
                                 factor since the last recomputation (0 = off) */
  int32_t refine_restart;     /* PCPG: 1 = restart the search direction after each recomputation
                                 (iterative refinement with inner CG solves); 0 = keep it */
  int32_t precond;            /* PCPG preconditioner M of Algorithm 1 (the paper leaves it open):
                                 0 = none (M = I); 1 = lumped, M = W (sum_i B_i K_i B_i^T) W with
                                 W = (B B^T)^{-1}, rebuilt from K at every feti_assemble */
  int64_t adjoint_work_bytes; /* device work budget of one feti_adjoint batch (dense n_i x 2 m_i arrays
                                 of the subdomains in the batch); 0 = min(24 GiB, 45% of free memory) */
  int32_t assembly_route;     /* how F_i is formed (Sec. III-IV):
                                 0 = the SYRK path: nested-dissection ordering, pruned TRSM
                                     X_i = L_i^{-1} P B_i^T, F_i = X_i^T X_i;
                                 1 = Schur complement (eq. 13, the augmented-matrix route): the DOFs B_i
                                     touches are ordered last as one root supernode, so eliminating the
                                     interior forms their Schur complement S_i in the root front, the
                                     root's factor is L_T with L_T L_T^T = S_i, and
                                     F_i = (L_T^{-1} D_i)^T (L_T^{-1} D_i) (D_i: the signed B columns);
                                     the same TRSM and SYRK kernels run on that single dense block;
                                 2 = the TRSM path (Sec. IV, Table I): X_i = L_i^{-1} P B_i^T, then the
                                     backward solve Z_i = P^T L_i^{-T} X_i on all m_i columns (FP64, in
                                     batches like feti_adjoint) and F_i = B_i Z_i (the rows of Z_i at the
                                     B DOFs), stored in the precision's tiles;
                                 3 = autotuned: the first feti_assemble times route 0 against route 2 on
                                     the problem and keeps the faster (feti_stats.assembly_route) */
  int32_t chol_split;         /* work items of the batched Cholesky: 0 = autotuned at the first
                                 feti_assemble; 1 = one subdomain per CTA; 2 = subtree tasks (heavy
                                 subtrees of the supernodal tree factored by CTAs of their own, a parent
                                 task after its children), so that large subdomains spread over several
                                 SMs.  The factor is the same bit for bit either way */
  int32_t syrk_kernel;        /* split-bf16 SYRK kernel: 0 = autotuned at the first feti_assemble; 1, 2, 3 =
                                 feti_stats.syrk_variant 0, 1, 2 (the same F bit for bit) */
  int32_t chol_tc;            /* 0 = the rank-32 and rank-128 updates of the fronts at least 384 wide run on
                                 the tensor cores by exact slicing of FP64 into bf16 integers (integer partial
                                 sums exact in FP32; error below FP64's own normwise bound); 1 = all of the
                                 Cholesky on the FP64 pipe */
  int32_t chol_tc_front;      /* with chol_tc = 0: the narrowest front (w + r) taken by the tensor-core kernel,
                                 with all its ancestors (0 = 384, the fastest measured on the 3D elasticity
                                 workload; values below 128 act as 128) */
} feti_options;

typedef struct {
  int32_t iterations;
  int32_t refinements;
  double rel_residual;        /* ||P r|| / ||P r_0|| at exit (FP64 residual when refinement is on) */
  int32_t converged;
  double initial_residual;    /* ||P r_0|| (FP64) */
} feti_solve_info;

typedef struct {
  /* sizes */
  int32_t nsub, n_lambda, npatterns, nbplans;
  int64_t sum_n, sum_m, L_doubles, X_elems, F_elems, workspace_bytes, device_bytes;
  /* algorithmic work (counted by the symbolic phase) */
  double chol_flops, trsm_flops, syrk_flops, syrk_exec_flops;
  double apply_bytes;         /* algorithmic bytes of one explicit apply */
  double implicit_bytes;      /* factor bytes read by one implicit apply */
  /* last feti_assemble, CUDA-event times on the context's stream (ms) */
  double t_chol_ms, t_trsm_ms, t_syrk_ms, t_coarse_ms, t_assemble_ms;
  double t_chol_tc_ms;        /* the part of t_chol_ms spent in the tensor-core kernel of the large fronts */
  double t_symbolic_ms;       /* host analysis time in feti_create */
  /* measurement counters since the last feti_set_profiling(ctx, 1) */
  int64_t launches;           /* kernel launches issued by this context */
  int64_t apply_calls;        /* explicit applications: feti_apply calls and PCPG iterations */
  double apply_ms;            /* CUDA-event time of those applications (feti_apply: scatter, tiles and
                                 gather; a PCPG iteration: tiles and gather) */
  double apply_tiles_ms;      /* CUDA-event time of their F-streaming kernel only */
  int64_t implicit_calls;     /* implicit-operator applications (feti_apply_implicit and inside feti_solve) */
  double implicit_ms;         /* CUDA-event time of those applications */
  /* autotuner choice for the apply (after the first feti_assemble) */
  int32_t apply_variant, apply_grid;  /* tile-kernel variant (0-2: register batches of 4, 8, 16 loads;
                                         3-5: bulk-copy rings of 4x3, 8x3, 2x6 warps x stages) and grid */
  /* autotuner choice for the pruned TRSM (after the first feti_assemble) */
  int32_t trsm_cols;          /* sorted columns per CTA work item (0: a whole subdomain per item) */
  int32_t trsm_grid;          /* persistent CTAs of the TRSM launch */
  int32_t chol_tasks;         /* Cholesky work items the autotuner kept: the subdomains, or the tasks of the
                                 subtree split when that was faster */
  int32_t syrk_variant;       /* split-bf16 SYRK kernel picked by the autotuner (0: all threads load, one issues;
                                 1: warp-specialised producers / issuer / epilogue; 2: as 0 with 32-deep chunks
                                 and two CTAs per SM) */
  int32_t assembly_route;     /* route of the last feti_assemble (0 SYRK path, 1 Schur complement, 2 TRSM path) */
  double route_ms[3];         /* route 3: time of the TRSM + SYRK (0) and of the TRSM path (2) at the first call */
} feti_stats;

typedef struct feti_ctx feti_ctx;

/* Analyse, copy inputs to the device and plan memory (Algorithm 2,
 * "preparation").  Symbolic analysis runs on host threads once per distinct
 * sparsity pattern.  Errors: FETI_ERR_ARG (malformed CSR, B row without a
 * single +-1, nfix != d, non-increasing B_lambda), FETI_ERR_ALLOC, FETI_ERR_CUDA. */
feti_status feti_create(const feti_problem* prob, const feti_options* opt, feti_ctx** out);

/* Replace the values of K_i (same pattern) for the next feti_assemble
 * (Algorithm 2: numeric values change between steps).  K_val is host memory. */
feti_status feti_update_values(feti_ctx* ctx, int32_t sub, const double* K_val);

/* Numeric phase (Algorithm 2, "preprocessing"): regularise, factorise,
 * pruned TRSM, SYRK into packed F_i tiles, and set up the coarse problem
 * G^T G (eqs. 6-8).  Synchronises the stream.  Errors: FETI_ERR_NOT_SPD. */
feti_status feti_assemble(feti_ctx* ctx);

/* Explicit application q = F p (eq. 12 summed over subdomains; scatter,
 * per-subdomain SYMV and gather of Algorithm 2) with the stored F_i.
 * p_dev, q_dev: [n_lambda] device FP64. */
feti_status feti_apply(feti_ctx* ctx, const double* p_dev, double* q_dev);

/* Implicit application q = sum_i B_i L_i^{-T} L_i^{-1} B_i^T p (eq. 11) in FP64. */
feti_status feti_apply_implicit(feti_ctx* ctx, const double* p_dev, double* q_dev);

/* Projected PCPG (Algorithm 1; M = I, or the lumped preconditioner of options.precond) for the
 * dual problem (eq. 7), then
 * alpha (eq. 8) and u (eq. 5).  lambda_dev [n_lambda], alpha_dev [sum d_i],
 * u_dev [sum n_i] (subdomains concatenated in order); any may be NULL except
 * lambda_dev.  The iteration runs on the device with the explicit F_i; the
 * host reads a small control block once per chunk of iterations.  With
 * refine_every = k > 0 the residual is recomputed with the FP64 implicit
 * operator (eq. 11) every k iterations, with refine_drop = f > 0 whenever
 * ||P r|| has dropped by f since the last recomputation; with either on, the
 * stopping rule is met only on such an FP64 residual.  Synchronises.
 * Returns FETI_ERR_NOT_CONVERGED (informative) at maxit or on a breakdown
 * (p.F p <= 0). */
feti_status feti_solve(feti_ctx* ctx, double* lambda_dev, double* alpha_dev, double* u_dev,
                       feti_solve_info* info);

/* feti_solve started from a guess: on entry lambda_dev [n_lambda] holds
 * lambda_g (for instance the previous step's solution in a multi-step
 * simulation, Algorithm 2, after feti_update_values + feti_assemble), and the
 * iteration starts from lambda_0 = lambda_I + P lambda_g, which satisfies
 * G^T lambda_0 = e (eq. 4) for any guess.  The stopping rule keeps the
 * reference norm of a cold start, ||P (d - F lambda_I)|| (one more FP64
 * implicit application), so a good guess reaches the same accuracy in fewer
 * iterations.  Outputs and errors as feti_solve; lambda_dev is overwritten
 * with the solution. */
feti_status feti_solve_warm(feti_ctx* ctx, double* lambda_dev, double* alpha_dev, double* u_dev,
                            feti_solve_info* info);

/* Adjoint of L = sum_i <W_i, F_i>: dtheta[e] = -<Z_i^T dK_e Z_i, W_i> with
 * Z_i = K_reg,i^{-1} B_i^T (derivative of the inverse, rho held fixed), in
 * FP64.  With K_reg = P^T L L^T P and L = L_u D (unit lower L_u):
 * Z_i = P^T L_u^{-T} D^{-2} X_u and Y_i = Z_i W_i = P^T L_u^{-T} D^{-2} (X_u W_i)
 * with X_u = L_u^{-1} P B_i^T from the pruned forward solve (recomputed here in
 * FP64 from L), and dtheta_e = -sum_{a,b in e} (dK_e)_ab Y_i[b,:] . Z_i[a,:].
 * Subdomains are processed in batches whose dense n_i x 2 m_i work arrays fit
 * a device budget.  W_dev: per subdomain m_i x m_i row-major FP64 in B-row
 * order, concatenated (W_i symmetric); dtheta_dev: [sum nelem_i] device FP64.
 * Needs element data at create and a preceding feti_assemble.  Synchronises.
 * Errors: FETI_ERR_ARG (no element data), FETI_ERR_STATE, FETI_ERR_ALLOC. */
feti_status feti_adjoint(feti_ctx* ctx, const double* W_dev, double* dtheta_dev);

/* Weighted trace L = sum_i <W_i, F_i> of the assembled local operators (the
 * loss whose gradient feti_adjoint returns).  W_dev as in feti_adjoint;
 * L_dev: one device FP64 value, written (summed in a fixed order, so the
 * result is reproducible).  Errors: FETI_ERR_ARG, FETI_ERR_STATE (before
 * feti_assemble). */
feti_status feti_weighted_trace(feti_ctx* ctx, const double* W_dev, double* L_dev);

/* Copy F_i (m_i x m_i, row-major, B-row order, FP64) to host memory. */
feti_status feti_get_F(feti_ctx* ctx, int32_t sub, double* out_host);

/* Measurement aid: enable (1) or disable (0) CUDA-event timing of feti_apply
 * and of the implicit operator on the context's stream, and reset the
 * counters reported by feti_get_stats (which synchronises the stream). */
feti_status feti_set_profiling(feti_ctx* ctx, int32_t enable);

feti_status feti_get_stats(feti_ctx* ctx, feti_stats* out);
const char* feti_last_error(feti_ctx* ctx);
void feti_destroy(feti_ctx* ctx);

/* Host-only symbolic analysis of one subdomain (no GPU needed): fills
 * info[0..15] = {n, nsn, max_front, max_width, nnzL, chol_flops, Lsize,
 * m, Xsize, trsm_flops, syrk_flops, ntile_contrib, chol_stack, rhs_stack,
 * nroots, nlast} (nlast: columns of the root supernode that holds the DOFs
 * B touches when opt->assembly_route = 1, else 0) and, if perm_out is not
 * NULL, the fill-reducing permutation
 * (perm_out[new] = old DOF).  sn_out, if not NULL (room for 4 n ints),
 * receives [nsn first columns..., nsn widths..., nsn parents (-1: root)...,
 * nsn counts of rows below the diagonal block...] of the supernodes in
 * postorder.  Errors: FETI_ERR_ARG for NULL sub/info or an invalid pattern. */
feti_status feti_analyse(const feti_subdomain* sub, const feti_options* opt, double* info,
                         int32_t* perm_out, int32_t* sn_out);

/* Host-only plan of the lumped preconditioner (options.precond = 1), for
 * inspection; no device is touched.  M = W M_core W with W = (B B^T)^{-1}
 * (CSR over multipliers: w_off [n_lambda + 1], w_col / w_val [sizes[0]]) and
 * M_core = sum_i B_i K_i B_i^T (CSR: m_off [n_lambda + 1], m_col [sizes[1]];
 * entry e's value is sum over k in [c_off[e], c_off[e + 1]) of
 * c_sign[k] * K[c_kidx[k]], with K the subdomains' CSR values concatenated in
 * order; c_off [sizes[1] + 1], c_kidx / c_sign [sizes[2]]).  Call with NULL
 * arrays to get sizes = {nnz(W), nnz(M_core), contributions}; arrays are
 * caller-owned host memory.  Errors: FETI_ERR_ARG for invalid input or a
 * singular B B^T block (redundant multipliers). */
feti_status feti_analyse_lumped(const feti_problem* prob, int64_t* sizes, int32_t* w_off, int32_t* w_col,
                                double* w_val, int32_t* m_off, int32_t* m_col, int64_t* c_off, int64_t* c_kidx,
                                double* c_sign);

/* Largest m accepted by feti_apply_one_static. */
#define FETI_STATIC_MAX_M 8192

/* Apply ONE local dual operator without allocating device memory:
 *     q[map[j]] += sum_k F[j][k] p[map[k]]      for j, k < m.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at the point where they apply the operator,
 * for example a framework that has reserved all device memory for its own
 * pool and forbids other allocations, or a latency-critical loop in which
 * cudaMalloc (which synchronises the device) is not acceptable.  It calls no
 * cudaMalloc, cudaFree or other allocating routine; all intermediates live in
 * fixed device arrays of this library (12 MiB plus small tables), which every
 * GPU that loads the library holds until the process exits.
 *
 * F_dev: F_i in this library's tile layout, FP32 (fp32 = 1) or FP64 (fp32 = 0),
 *        device memory, 16-byte aligned: 64 x 64 tiles (bi, bj) with bj <= bi
 *        stored one after another in the order bi (bi + 1) / 2 + bj.  An
 *        off-diagonal tile is row-major, 64 values per row; a diagonal tile
 *        keeps, for each row r, only its first w ceil((r + 1) / w) values
 *        (w = 16 / sizeof(value)), rows packed back to back, with zeros right
 *        of the diagonal.  The last block row bi = nb - 1 (nb = ceil(m / 64))
 *        holds only m - 64 (nb - 1) rows per tile; columns beyond m hold zeros.
 * map_dev: [m] int32 device array, distinct multiplier ids (rows of F_i).
 * p_dev, q_dev: FP64 device dual vectors; q is accumulated into, not cleared.
 * stream: cudaStream_t or NULL.  The call is synchronous (it waits for the
 *        stream).
 * Errors: FETI_ERR_ARG for m <= 0, m > FETI_STATIC_MAX_M or a NULL pointer;
 *        FETI_ERR_CUDA for a failed CUDA call, and also, without launching
 *        anything, when a CUDA error left by earlier work on the calling
 *        thread is pending (it is not cleared, so its owner still sees it).
 * The first call on each device looks up the device addresses of the fixed
 * arrays (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  CUDA loads this library's device code lazily, so
 * the fixed arrays and the kernels become resident on a device at that first
 * call: a caller that later reserves all free device memory for its own pool
 * should make the first call before it does; from then on no call takes device
 * memory.  All calls share the same arrays and leave the last call's contents
 * in them, so calls that overlap on the GPU (other streams or host threads)
 * race: order them. */
feti_status feti_apply_one_static(int32_t m, int32_t fp32, const void* F_dev, const int32_t* map_dev,
                                  const double* p_dev, double* q_dev, void* stream);

/* Library version string. */
const char* feti_version(void);

#ifdef __cplusplus
}
#endif
#endif
