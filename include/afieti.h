/*
 * afieti.h - C ABI of the GB300 (sm_103a) inexact All-Floating IETI solver for
 * multi-patch isogeometric compressible linear elasticity
 * (Bosy, Montardini, Sangalli, Tani, arXiv 2001.09626).
 *
 * The library solves the saddle-point system of eq. (4.5),
 *     [A B^T; B 0] [u; lambda] = [f; 0],
 * by MINRES on the projected system of eq. (4.7) preconditioned by the
 * block-diagonal operator of eq. (4.9) with the inexact local solvers of
 * Section 5.2 (fast diagonalization, Algorithm 1) and the non-redundant
 * Schur-type multiplier preconditioner of Remark 1.
 *
 * Conventions shared by every entry point
 *  - "torn" vectors (length n_dof): patches stacked in input order; inside a
 *    patch the d displacement components are stacked; each component is an
 *    n3*n2*n1 block in colexicographic order, i1 fastest (Section 2.2).
 *  - multiplier vectors (length n_c): one entry per row of B, rows ordered
 *    component-major, then by geometric node (nodes ordered by their first
 *    copy (patch, local index)); a node on the Dirichlet boundary has one row
 *    per copy, any other node has rows u_{c1} - u_{cj}, j = 2..m.
 *  - every *_dev pointer is device memory of the current CUDA device, FP64,
 *    contiguous, owned by the caller; with nrhs > 1 vectors are stacked
 *    [nrhs][length].  Host pointers (afi_problem fields) are read during the
 *    call and not retained.
 *  - the context owns all setup data and workspaces; one context may be used
 *    by one host thread and one stream at a time.
 *  - errors are reported through the returned status, never by aborting;
 *    afi_last_error() gives a message for the most recent failure.
 */
#ifndef AFIETI_H
#define AFIETI_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AFI_OK = 0,
  AFI_EINVAL = 1,          /* invalid argument or geometry (e.g. det J <= 0) */
  AFI_ENOMEM = 2,          /* device allocation failed */
  AFI_ECUDA = 3,           /* a CUDA runtime call failed */
  AFI_ESINGULAR = 4,       /* G^T G or a pencil is not positive definite */
  AFI_ENOT_CONVERGED = 5,  /* maxit reached before the tolerance */
  AFI_EBREAKDOWN = 6,      /* MINRES breakdown (non-finite or negative norm) */
  AFI_ETIMEOUT = 7         /* a bounded mbarrier wait of a tensor-core or bulk-copy
                              kernel ran out; reported by ieti_solve and
                              ieti_solve_adjoint at the end of the solve */
} afi_status;

/* Arithmetic of the local solvers (fast diagonalization and the parametric
 * stiffness products inside the Schur preconditioner).  The jumps,
 * projectors, Krylov algebra and true residual are FP64 always; the
 * stiffness matvec of the iterations is FP64 or double-FP32, see
 * AFI_VARIANT_STENCIL_F64. */
typedef enum {
  AFI_FD_FP64 = 0,   /* plain form: FP64 throughout */
  AFI_FD_FP32 = 1,   /* FP32 contractions, FP32 accumulate */
  AFI_FD_TF32 = 2,   /* TF32 tensor-core contractions, FP32 accumulate */
  AFI_FD_BF16 = 3    /* BF16 tensor-core contractions, FP32 accumulate */
} afi_fd_precision;

typedef struct afi_ctx afi_ctx;   /* opaque, owned by the library */

/* Problem description (Sections 2-4), host memory.
 *   dim            2 or 3
 *   npatch         number of patches
 *   degree[k]      spline degree of patch k (same in every direction)
 *   nel[k*dim+l]   elements of patch k in direction l: open uniform knot
 *                  vector with single interior knots (C^{p-1} splines),
 *                  n_l = nel + degree basis functions
 *   ctrl           control points of all patches concatenated, each patch
 *                  [i3][i2][i1][dim] (i1 fastest); the geometry map is the
 *                  isoparametric spline map of Section 2.2.  Shared interface
 *                  control points of conforming faces must coincide; they
 *                  are matched by coordinates (relative tolerance 1e-10).
 *                  A face whose knot vectors refine the neighbour's (nested
 *                  non-conforming interface, Section 2) is found by its
 *                  corners: same corners in the same tangential order, one
 *                  degree, element counts that divide, the fine control net
 *                  equal to the refined coarse net, and face edges on the
 *                  Dirichlet boundary.  Each of its fine coefficients off
 *                  the Dirichlet boundary gets the row
 *                  u_fine - sum W u_coarse (W the knot-insertion weights);
 *                  these rows follow the node rows, by (fine patch, fine
 *                  face), then component, then fine point
 *   lame[2k+0,1]   (lambda_k, mu_k) of patch k (eq. 3.1)
 *   dirichlet_face[k*2*dim + 2*l + side]  1 if the face eta_l = side of
 *                  patch k carries the homogeneous Dirichlet condition      */
typedef struct {
  int dim, npatch;
  const int *degree;
  const int *nel;
  const double *ctrl;
  const double *lame;
  const unsigned char *dirichlet_face;
} afi_problem;

/* afi_options.variant bits */
#define AFI_VARIANT_LOCAL_ONLY 1   /* set up the local solvers, constraints and
                                      projectors only: no quadrature geometry,
                                      no stiffness (whose stencil can exceed
                                      device memory); ieti_solve, afi_apply of
                                      STIFFNESS/SADDLE, afi_load_vector and
                                      afi_lame_grad then return AFI_EINVAL */
#define AFI_VARIANT_FD_SLAB 2      /* TF32/BF16 local solvers: send every 3D
                                      tensor through the three-pass kernels
                                      used for tensors larger than one CTA
                                      (same operator; for testing and
                                      measuring that path on small patches) */
#define AFI_VARIANT_STENCIL_F64 4  /* apply the stiffness with FP64 FMAs
                                      everywhere.  By default, when every patch
                                      has one degree (at most 5 in 3D, 3 in
                                      2D) and rows of at most 128 nodes, and a
                                      second, row-compressed copy of the
                                      stencil fits in device memory (with a
                                      tenth of it to spare), each coefficient
                                      is also stored as a sum of two FP32
                                      numbers (relative error <= 2^-48), and
                                      the MINRES iterations and
                                      afi_apply(AFI_OP_STIFFNESS / SADDLE) run
                                      the matvec in double-FP32 arithmetic on
                                      the FP32 pipe (inputs and results within
                                      the FP32 range); the true residual is
                                      always FP64 */
#define AFI_VARIANT_FORCE_RESTART 8 /* with the double-FP32 stiffness: take the
                                      FP64 restart at the first true-residual
                                      check, as if the iteration had stalled
                                      (same converged answer; for testing and
                                      timing that path) */
#define AFI_VARIANT_EXACT 16       /* EXACT local solvers (Section 5.1), the
                                      paper's iteration-count reference:
                                      P_A^ex = A^(k) + H_k^{-2} M^(k) (eq. 5.1)
                                      and P_S^{ex-nr} with the Schur
                                      complements S^(k) of A^(k) (Remark 1),
                                      applied with dense per-patch FP64
                                      inverses built at setup; every patch
                                      must have d N^(k) <= 4096 (else
                                      AFI_EINVAL).  afi_apply's AFI_OP_PA_INV
                                      and AFI_OP_SCHUR then apply these;
                                      fd_apply stays the FD of Algorithm 1,
                                      and afi_options.prec has no effect */
#define AFI_VARIANT_GEO 32         /* geometry-inclusion inexact local solvers
                                      (Section 5.2.3), the variant of the
                                      paper's experiments: per (patch,
                                      component l) the diagonal of the
                                      elasticity coefficient C_l and |det J|
                                      are fitted at the Gauss points by
                                      products of univariate factors (in the
                                      logarithm, by Diliberto-Straus
                                      mid-range sweeps until no factor moves
                                      by more than 1e-14, at most 500), which
                                      give the univariate K~_{l,m}, M~_{l,m}
                                      of eq. 5.11; then
                                      P_A^{-1} = D_A^{-1/2} (A~_l +
                                      H^{-2} M~_l)^{-1} D_A^{-1/2} (eq. 5.12)
                                      by Algorithm 1 on the eigenpairs of
                                      (K~_{l,m}, M~_{l,m}), and the Schur
                                      block is D_S^{1/2} S~_l D_S^{1/2} with
                                      S~_l the Schur complement of A~_l
                                      (eq. 5.13), D_A and D_S the diagonal
                                      scalings that restore the diagonals of
                                      A_ll + H^{-2} M and A_ll.  Applies to
                                      fd_apply (interior = 0 and 1),
                                      AFI_OP_PA_INV, AFI_OP_SCHUR, AFI_OP_PS,
                                      AFI_OP_PRECOND and the solves, at every
                                      afi_options.prec.  Needs the geometry:
                                      with AFI_VARIANT_LOCAL_ONLY or
                                      AFI_VARIANT_EXACT it returns
                                      AFI_EINVAL.  The fit and the per-(patch,
                                      component) tables count as local-solver
                                      setup (afi_info.t_fd_setup_ms). */
#define AFI_VARIANT_FD_FIXED 64    /* TF32/BF16 local solvers on 3D tensors of
                                      several shapes: keep every tensor that
                                      fits one CTA in the single-CTA kernel.
                                      By default the split between it and the
                                      three-pass kernels is chosen at setup by
                                      timing one application per candidate
                                      (each distinct shared-memory need of the
                                      tensors is a candidate threshold), so two
                                      contexts of one problem may split
                                      differently and round differently; this
                                      bit makes the split a fixed rule.  A
                                      batch of tensors of one shape has a
                                      single candidate and is never timed. */

#define AFI_VARIANT_MATRIX_FREE 128 /* 3D problems with one degree (1..5) for
                                      every patch: apply the stiffness A^(k)
                                      (eq. 3.1) and the mass of
                                      afi_load_vector without storing them,
                                      by sum factorisation over each element
                                      with the same Gauss rule (p + 1 points
                                      per element and direction) and the
                                      Jacobian recomputed from the control
                                      points in every product.  Nothing per
                                      quadrature point is stored, so problems
                                      whose stencil exceeds device memory can
                                      be solved.  The MINRES iterations use
                                      FP32 products (input and sums in FP32)
                                      and refine against the FP64 true
                                      residual: each run stops when its
                                      estimate has fallen by 1e-4 (or reached
                                      tol) and the next solves for the
                                      correction, at most 12 more runs
                                      (afi_info.fp64_restarts counts them).
                                      The true residual is always FP64, and
                                      with AFI_VARIANT_STENCIL_F64 every
                                      product is.  afi_apply(AFI_OP_STIFFNESS /
                                      AFI_OP_SADDLE) uses the FP32 form unless
                                      AFI_VARIANT_STENCIL_F64 is set.  Several
                                      right-hand sides are solved one after
                                      the other.  Excludes
                                      AFI_VARIANT_LOCAL_ONLY, AFI_VARIANT_EXACT
                                      and AFI_VARIANT_GEO; afi_lame_grad
                                      returns AFI_EINVAL. */

/* prec: local-solver arithmetic; tol: relative tolerance (the MINRES
 * preconditioned residual estimate and then the true FP64 residual
 * ||b - A x|| / ||b|| of eq. (4.7) must both reach it; when the
 * double-FP32 stiffness of the iterations keeps the true residual from
 * falling, MINRES restarts once from the current iterate with the FP64
 * stiffness, see afi_info.fp64_restarts); maxit: iteration cap;
 * use_graph: 1 runs the MINRES iterations as replays of a CUDA graph of six
 * captured iterations (same iterates and iteration count as 0, which
 * launches every kernel from the host); variant: 0 or a combination of the
 * AFI_VARIANT_* bits. */
typedef struct {
  afi_fd_precision prec;
  double tol;
  int maxit;
  int use_graph;
  int variant;
} afi_options;

/* Filled by ieti_solve / ieti_solve_adjoint (for the last right-hand side):
 * iterations (of both runs when restarted), the MINRES estimate, the true
 * relative residual (FP64 stiffness), the setup
 * time of the context, the wall time of this solve (device events) and the
 * part of the setup that builds the local solvers of Algorithm 1 (univariate
 * matrices, generalised eigensolves of eq. 5.8, tensor-core operand tables,
 * FD work splits; the paper counts this part in its solve times). */
typedef struct {
  int iters;
  double relres_est, relres_true;
  double t_setup_ms, t_solve_ms;
  double t_fd_setup_ms;
  int fp64_restarts;   /* 1 if the solve restarted with the FP64 stiffness;
                          with AFI_VARIANT_MATRIX_FREE the number of
                          refinement runs after the first */
} afi_info;

/* Operators of the hot path, for afi_apply (each is one row of the solve):
 *  AFI_OP_STIFFNESS  y = A x                 (torn -> torn), eqs. 3.1, 4.2;
 *                    double-FP32 unless AFI_VARIANT_STENCIL_F64
 *  AFI_OP_B          y = B x                 (torn -> multipliers), Sec. 4
 *  AFI_OP_BT         y = B^T x               (multipliers -> torn)
 *  AFI_OP_PCHI       y = P_chi x             (multipliers), eq. 4.6
 *  AFI_OP_PU         y = P_u x               (torn), Sec. 4 after eq. 4.9
 *  AFI_OP_PA_INV     y = P_A^{-1} x          (torn), eq. 5.6 by Algorithm 1
 *                    (AFI_VARIANT_EXACT: (A + D_H M)^{-1} x, eq. 5.1)
 *  AFI_OP_SCHUR      y = blkdiag H^{d-2} S_hat x (torn shell -> torn shell)
 *                    (AFI_VARIANT_EXACT: blkdiag S x, Section 5.1),
 *                    eqs. 5.4-5.5; interior entries of y are written as zero
 *  AFI_OP_PS         y = (B B^T)^{-1} B S_hat_H B^T (B B^T)^{-1} x  (Remark 1)
 *  AFI_OP_PRECOND    y = calB^{-1} x         ([torn; multipliers]), eq. 4.9
 *  AFI_OP_SADDLE     y = calA x              ([torn; multipliers]), eq. 4.7 */
typedef enum {
  AFI_OP_STIFFNESS = 0, AFI_OP_B = 1, AFI_OP_BT = 2, AFI_OP_PCHI = 3,
  AFI_OP_PU = 4, AFI_OP_PA_INV = 5, AFI_OP_SCHUR = 6, AFI_OP_PS = 7,
  AFI_OP_PRECOND = 8, AFI_OP_SADDLE = 9
} afi_operator;

/* Setup (Section 2.1 knots and B-splines, Section 4 constraints, rigid modes
 * and G^T G, Section 5.2.1 step 1 generalised eigendecompositions, and the
 * assembly of every patch stiffness A^(k) by Gauss quadrature with p+1
 * points per element and direction).  Runs on the current device, returns
 * after the work is complete.  *out receives a new context on success.
 * Errors: AFI_EINVAL (bad sizes, faces that neither match nor nest as
 * described above, det J <= 0), AFI_ESINGULAR (G^T G or the B B^T block of
 * a nested face not positive definite), AFI_ENOMEM, AFI_ECUDA. */
afi_status af_ieti_setup(const afi_problem *prob, const afi_options *opt, afi_ctx **out);

/* Algorithm 1 (steps 2-4) on every (patch, component) block:
 *  interior = 0: s = P_A^{inex,-1} r = blkdiag [H^{d-2}(A_hat_l + M_hat_l)]^{-1} r
 *               over torn vectors (eqs. 5.6, 5.9);
 *  interior = 1: s = (A_hat_l)_II^{-1} r over the compact interior blocks
 *               (each block (n3-2)(n2-2)(n1-2), i1 fastest, patches and
 *               components stacked like torn vectors; eq. 5.10).
 * Uses the context's precision.  Stream-ordered, asynchronous. */
afi_status fd_apply(afi_ctx *ctx, int interior, const double *r_dev, double *s_dev,
                    int nrhs, void *stream);

/* AF-IETI solve: lambda_0 = G (G^T G)^{-1} R^T f, MINRES on eq. (4.7) from a
 * zero guess, recovery u = w - R (G^T G)^{-1} G^T B w, lambda = lambda_0 + chi
 * (Section 4).  f_dev, u_dev: [nrhs][n_dof]; lambda_dev: [nrhs][n_c] or NULL.
 * The call returns when the solve has finished (the host polls the
 * convergence flag).  info may be NULL.  Returns AFI_ENOT_CONVERGED if maxit
 * was reached (u is still the last iterate's recovery).
 * nrhs > 1: the right-hand sides are solved in batches of up to 8 whose
 * MINRES recurrences run in lockstep, sharing one batched stiffness launch
 * per iteration (each solution is bitwise the one a separate call gives);
 * info then holds the largest iteration count and residuals over all
 * right-hand sides, the summed solve time and the number of FP64 restarts.
 * The first multi-right-hand-side solve of a context allocates 8 sets of
 * MINRES vectors (96 (n_dof + n_c) doubles). */
afi_status ieti_solve(afi_ctx *ctx, const double *f_dev, double *u_dev, double *lambda_dev,
                      int nrhs, afi_info *info, void *stream);

/* Adjoint solve.  The saddle matrix of eq. (4.5) is symmetric, so the
 * adjoint state (z, z_lambda) for an objective gradient g = dJ/du solves the
 * same system with right-hand side g.  Same layout and errors as ieti_solve.
 * (The paper has no differentiation; this entry point extends it.) */
afi_status ieti_solve_adjoint(afi_ctx *ctx, const double *g_dev, double *z_dev,
                              double *zlambda_dev, int nrhs, afi_info *info, void *stream);

/* Gradient with respect to the Lame values: A^(k) is linear in
 * (lambda_k, mu_k) (eq. 3.1), so dJ/dlambda_k = -z_k^T A_lambda^(k) u_k and
 * dJ/dmu_k = -z_k^T A_mu^(k) u_k, with A_lambda = int div div and
 * A_mu = int 2 eps:eps.  grad_dev: [npatch][2] (lambda, mu).  For the
 * compliance J = f^T u pass z = u. */
afi_status afi_lame_grad(afi_ctx *ctx, const double *u_dev, const double *z_dev,
                         double *grad_dev, void *stream);

/* Load vector of a body force with nodal coefficients c (torn layout):
 * f^(k) = M^(k) c^(k), M^(k) the mapped mass matrix of eq. (4.8). */
afi_status afi_load_vector(afi_ctx *ctx, const double *c_dev, double *f_dev, void *stream);

/* One hot-path operator (see afi_operator) applied to x_dev, result in
 * y_dev (lengths as listed there).  Stream-ordered, asynchronous. */
afi_status afi_apply(afi_ctx *ctx, afi_operator op, const double *x_dev, double *y_dev,
                     void *stream);

/* The same operator applied to nrhs vectors stacked in x_dev ([nrhs][input
 * length]) into y_dev ([nrhs][output length]).  AFI_OP_STIFFNESS runs the
 * batched double-FP32 stencil kernel on up to 8 vectors per launch (each
 * coefficient streamed once for all of them; bitwise the same results as
 * separate applications) when the pair copy exists, FP64 launches
 * otherwise; AFI_OP_PA_INV is one batched FD launch; the other operators
 * are applied one vector after the other.  (The batching has no
 * counterpart in the paper: it serves several right-hand sides, eqs. 3.1,
 * 4.7, 4.9.)  Errors as afi_apply, AFI_EINVAL for nrhs < 1. */
afi_status afi_apply_batch(afi_ctx *ctx, afi_operator op, const double *x_dev, double *y_dev,
                           int nrhs, void *stream);

/* Change the local-solver arithmetic of an existing context (the low
 * precision copies of the eigenvectors are built at setup). */
afi_status afi_set_precision(afi_ctx *ctx, afi_fd_precision prec);

/* Allocation-free fast diagonalization.  The paper has no counterpart: this
 * entry point serves callers that may not allocate device memory where they
 * need a local solve, e.g. code being recorded into a CUDA graph that must
 * contain no allocation, real-time loops on a fixed memory budget, or
 * plug-ins whose host framework owns all device memory.  For nblk FP64
 * tensors of one shape stacked in r and s ([nblk][n3][n2][n1], i1 fastest,
 * device memory) it computes
 *     s = (U3 x U2 x U1) Lambda^{-1} (U3 x U2 x U1)^T r,
 *     Lambda[i1,i2,i3] = scale * (coef[0] D1[i1] + coef[1] D2[i2]
 *                                 + coef[2] D3[i3] + shift),
 * where U_l is n_l x n_l row-major (row = basis index, column = mode) and
 * D_l has n_l entries, all in device memory; coef is a host array of three.
 * With U_l, D_l the generalised eigenvectors (U^T M U = I) and eigenvalues
 * of a pair of univariate matrices (K_l, M_l), s solves the Kronecker-sum
 * system whose matrix is scale * (sum_l coef[l] K_l (x) the M's of the other
 * directions + shift * M_3 x M_2 x M_1).
 * Three directions are used exactly when U3 and D3 are both given (n3 may
 * then be 1); pass U3 = D3 = NULL with n3 = 1 for two directions (coef[2]
 * is then ignored).  One of U3, D3 alone, or n3 > 1 without them, returns
 * AFI_EINVAL.
 * Scratch: a file-scope device array of 2^21 doubles (16 MiB) that every GPU
 * loading the library holds until the process exits; 2 * nblk * n1*n2*n3
 * must not exceed 2^21 (checked without overflow), larger requests return
 * AFI_EINVAL without running.
 * The first call on a device looks up the array's address (with that device
 * current); make that first call before any stream capture.  All calls share
 * the array, so calls whose executions overlap on the GPU (different streams
 * or devices' concurrent work on one device) race; every scratch element is
 * written before it is read, so nothing needs clearing.  Calls no cudaMalloc,
 * cudaFree or other allocating routine.  Stream-ordered, asynchronous. */
afi_status afi_fd_apply_static(int n1, int n2, int n3, const double *U1, const double *U2,
                               const double *U3, const double *D1, const double *D2,
                               const double *D3, const double coef[3], double shift, double scale,
                               const double *r, double *s, int nblk, void *stream);

/* n_dof (torn length) and n_c (number of constraints). */
afi_status afi_sizes(const afi_ctx *ctx, long *n_dof, long *n_c);

/* Device bytes held by the context and the stiffness storage alone (the
 * FP64 stencil plus its FP32-pair copy when there is one). */
afi_status afi_memory(const afi_ctx *ctx, long long *total_bytes, long long *stiffness_bytes);

void af_ieti_destroy(afi_ctx *ctx);
const char *afi_status_string(afi_status s);

/* Message of the most recent failure in this process (not thread-specific). */
const char *afi_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts, all threads); the difference of two readings counts the
 * launches in between. */
long long afi_kernel_launches(void);

/* Self-test of the library's failure path for tensor-core waits (no
 * counterpart in the paper).  Every tcgen05 and bulk-copy kernel waits on
 * mbarriers (TMA and MMA completion) with a bounded number of polls; when a
 * wait runs out the kernel waits (bounded) for its own copies, frees its
 * tensor memory, returns, and the solve reports AFI_ETIMEOUT instead of
 * hanging the GPU.  This entry point runs that path
 * on purpose: one CTA allocates tensor memory, waits at most `polls` polls
 * (1 <= polls <= 2^22) on an mbarrier that nothing ever arrives on, frees
 * the tensor memory and returns.  Returns AFI_ETIMEOUT when the wait ran out
 * (the expected outcome), AFI_OK if it completed, AFI_EINVAL for polls out
 * of range, AFI_ECUDA on a CUDA error.  *polls_used (may be NULL) receives
 * the number of polls made.  Synchronous on the legacy default stream;
 * allocates and frees 16 bytes of device memory. */
afi_status afi_selftest_bounded_wait(long long polls, long long *polls_used);

#ifdef __cplusplus
}
#endif
#endif /* AFIETI_H */
