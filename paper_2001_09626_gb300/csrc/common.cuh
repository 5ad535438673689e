// Internal definitions of the AF-IETI library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <array>
#include <atomic>
#include <cstdint>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "../../include/afieti.h"

namespace afi {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);

#define AFI_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::afi::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      return AFI_ECUDA;                                                       \
    }                                                                         \
  } while (0)

#define AFI_TRY(expr)                                                         \
  do {                                                                        \
    afi_status s_ = (expr);                                                   \
    if (s_ != AFI_OK) return s_;                                              \
  } while (0)

#define AFI_LAUNCH_CHECK() AFI_CUDA(cudaGetLastError())

// Every kernel launch of the library goes through launch(), which counts it
// (afi_kernel_launches) before the ordinary <<<>>> launch.
extern std::atomic<long long> g_launches;

template <typename Kernel, typename... Args>
inline void launch(Kernel kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                   Args... args) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  kernel<<<grid, block, smem, stream>>>(args...);
}

// ------------------------------------------- FP64 <-> FP32 on the integer pipes
// The mixed-precision kernels convert every FP64 input to FP32 and every
// FP32 result back to FP64.  The hardware conversions issue on the FP64
// pipe, which on this GPU has a small fraction of the FP32 and integer
// issue rate, so these do the same conversions with integer operations on
// the IEEE-754 bit fields.
//
// f64 -> f32: round to nearest even; results below the FP32 normal range
// flush to signed zero, finite values above it become +-inf, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int ein = (int)((hi >> 20) & 0x7FFu);
  const int e = ein - 1023 + 127;
  unsigned r = sign | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rbit = (lo >> 28) & 1u, sticky = lo & 0x0FFFFFFFu;
  r += rbit & ((sticky != 0u) | (r & 1u));   // a carry into the exponent is correct
  r = (e <= 0) ? sign : r;
  r = (e >= 255 || ((r >> 23) & 0xFFu) == 0xFFu) ? (sign | 0x7F800000u) : r;
  r = (ein == 0x7FF && (((hi & 0xFFFFFu) | lo) != 0u)) ? 0x7FC00000u : r;
  return __uint_as_float(r);
}

// f32 -> f64: exact for normal numbers, zero and infinities; FP32
// subnormals flush to signed zero, NaN becomes the quiet NaN.  Written
// without branches: the magnitude's bits shifted into place and the
// exponent rebiased by 1023 - 127 in one add, then selects for the ends.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f), mag = u & 0x7FFFFFFFu;
  unsigned hi = (mag >> 3) + (896u << 20), lo = u << 29;
  const bool tiny = mag < 0x00800000u, special = mag >= 0x7F800000u;
  hi = tiny ? 0u : hi;
  lo = (tiny || special) ? 0u : lo;
  hi = special ? (mag > 0x7F800000u ? 0x7FF80000u : 0x7FF00000u) : hi;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}

// ------------------------------------------------------- 1D spline tables
// One table per distinct (nel, p) pair (open uniform knots).  Offsets index
// the context's FP64 pool (and FP32 / BF16 pools for the low-precision
// copies of the eigenvectors).  A "dummy" table (n = 1) stands for the third
// direction of 2D problems: basis value 1, K = 0, M = 1, U = 1, D = 0.
struct Tab1D {
  int nel, p, n, nq, ni;       // ni = interior count (n - 2, or 1 for dummy)
  long long knots;             // [nel + 2p + 1]
  long long qw;                // [nq] Gauss weights (times span length)
  long long val, der;          // [nq][p+1] active basis values / derivatives
  long long K, M;              // [n][n] univariate stiffness and mass
  long long U, D;              // [n][n] (row i = basis, col a = mode), [n]
  long long Ui, Di;            // interior pencil [ni][ni], [ni]
  long long Uf, Uif;           // FP32 copies (float pool)
  long long Ub, Uib;           // BF16 copies (bf16 pool), row-major like U
  int ld, ldi;                 // padded leading dimensions (multiples of 4)
  long long Up, Upt;           // U and U^T padded to [n][ld] (zero padding)
  long long Uip, Uipt;         // interior U and U^T padded to [ni][ldi]
  long long Kb, Mb;            // bands by diagonal: Kb[t*n + i] = K[i][i + t - p], t = 0..2p
  long long tcB[2][2][2];      // tensor-core B operands, byte offsets in tcpool:
                               // [bf16][interior][back]; forward B[a][k] = U[k][a],
                               // back B[i][k] = U[i][k], canonical K-major layout
  long long wK, wM;            // geometry-inclusion tables: per-quadrature-point factors
                               // nu (in K) and beta (in M) of eq. 5.11; -1 for the
                               // plain univariate K_hat, M_hat
};

// Per-patch descriptor (device-side POD).
struct DevPatch {
  int n[3];         // basis functions per direction (n3 = 1 in 2D)
  int ni[3];        // interior counts (n - 2; 1 for a dummy direction)
  int nq[3];        // quadrature points per direction (1 for dummy)
  int W[3];         // stencil widths 2p+1 (1 for dummy)
  int tab[3];       // 1D table per direction
  int p, N, Ni, S;  // degree, nodes, interior nodes, stencil offsets
  int NQ;           // quadrature points of the patch
  int n1p, NP;      // stencil planes: rows padded to even length n1p, NP = n1p*n2*n3
  long long off;    // torn offset of component 0
  long long ioff;   // compact interior offset of component 0
  long long soff;   // stiffness stencil offset (doubles)
  long long roff;   // offset in the row-compressed pair copy (pairs)
  long long rstride;  // pairs per row group of the pair copy
  long long qoff;   // quadrature geometry offset (points)
  long long xoff;   // control point offset (doubles)
  double lam, mu, Hs;  // Lame values, H^{d-2}
  double H;            // patch diameter H^(k)
  // Local solvers of component l (FD of P_A and of the interior block, the
  // Schur block): univariate table per direction m, the coefficient of the
  // stiffness term in direction m, the mass shift and the overall scale:
  //   Lambda_l = lscale (sum_m lcf[l][m] D_m + lshift),  S scaled by lscale.
  // Plain parametric solvers (eqs. 5.6, 5.7): ltab[l][m] = tab[m],
  // lcf = 2 mu + lambda on m = l and mu elsewhere, lshift = 1, lscale =
  // H^{d-2}.  Geometry inclusion (eqs. 5.12, 5.13): tables of the fitted
  // K~_{l,m}, M~_{l,m}, lcf = 1, lshift = H^{-2}, lscale = 1.
  int ltab[3][3];
  double lcf[3][3];
  double lshift, lscale;
  long long qloff;     // geometry-inclusion fit: first per-direction Gauss-point slot
};

// Split of the patches between the tensor-core FD (tensors that fit one CTA)
// and the SIMT FD, per (interior, operand format); built on first use.
struct TcSplit {
  bool ready = false;
  int *d_tc = nullptr, *d_simt = nullptr;   // patch index lists (device)
  int ntc = 0, nsimt = 0;
  int cap = 0, bsz = 0, tcols = 32;
  size_t smem = 0;
  int simt_maxN = 0;
  // three-pass tensor-core FD for tensors larger than one CTA (fd_slab.cu)
  void *d_plane = nullptr, *d_line = nullptr;   // int4 / int2 work lists
  int nplane = 0, nline = 0;
  int *d_pbounds = nullptr, *d_lbounds = nullptr;   // persistent CTAs' ranges of the lists
  int pgrid = 0, lgrid = 0;                         // persistent CTAs per (component, rhs)
  int per = 2;                                      // three-pass work items per CTA (tuned)
  int cap_p = 0, bsz_p = 0, tcols_p = 32, cap_l = 0, bsz_l = 0, tcols_l = 32;
  size_t smem_p = 0, smem_l = 0;
};

struct afi_ctx_impl;

}  // namespace afi

// The opaque context.
struct afi_ctx {
  int dim = 0, npatch = 0, nm = 0;   // nm = rigid modes per patch
  int device = 0;
  long n_dof = 0, n_c = 0, n_int = 0;
  long n_c0 = 0;                     // rows of the conforming nodes (the first n_c0 of n_c)
  afi_options opt{};
  double t_setup_ms = 0.0;
  double t_fd_setup_ms = 0.0;        // local-solver part of the setup (Algorithm 1 step 1)

  // host copies
  std::vector<afi::DevPatch> hp;
  std::vector<afi::Tab1D> htab;
  int max_N = 0, max_n = 0;
  int smem_optin = 0;                // opt-in dynamic shared memory per block
  int nsm = 0;                       // streaming multiprocessors of the device

  // device data
  afi::DevPatch *patches = nullptr;
  afi::Tab1D *tabs = nullptr;
  double *dpool = nullptr;  long long dpool_n = 0;
  float *fpool = nullptr;   long long fpool_n = 0;
  __nv_bfloat16 *bpool = nullptr; long long bpool_n = 0;
  unsigned char *tcpool = nullptr; long long tcpool_n = 0;   // tensor-core B operands
  double *ctrl = nullptr;                     // all control points
  double *stencil = nullptr; long long stencil_n = 0;
  float2 *stencil2 = nullptr;                 // row-compressed (hi, lo) FP32-pair copy, or null
  long long stencil2_n = 0;                   // its size in pairs
  float2 *xsplit = nullptr;                   // (hi, lo) FP32 pairs of the matvec input
  float2 *xsplit_multi = nullptr;             // the same for up to kMaxRhs inputs
  int mv_width = 0;                           // vectors per batched stiffness launch (0: not tuned)
  // EXACT local solvers (AFI_VARIANT_EXACT): dense per-patch inverses
  bool exact = false;
  double *ex_Kinv = nullptr, *ex_AIIinv = nullptr;   // (A + H^-2 M)^{-1}, A_II^{-1}
  long long *ex_koff = nullptr, *ex_aoff = nullptr;  // their per-patch offsets
  bool mv_exact = false;                      // apply the FP64 stencil even if pairs exist
  double *qgeo = nullptr; long long nqp = 0;  // [DIM*DIM + 1][nqp] SoA
  // matrix-free stiffness and mass (AFI_VARIANT_MATRIX_FREE, mf.cu)
  bool mf = false;
  int mf_p = 0;                               // the common degree
  long long mf_ne = 0;                        // elements of all patches
  long long *mf_eoff = nullptr;               // [npatch + 1] first element of each patch
  float *mf_ctrlf = nullptr;                  // FP32 control points, patch-relative
  float *mf_xf = nullptr, *mf_yf = nullptr;   // FP32 input and sums of the FP32 form
  int mf_grid[4] = {0, 0, 0, 0};              // [fp32 / fp64 stiffness, fp32 / fp64 mass]
  int mf_wpc[4] = {0, 0, 0, 0};
  int mf_smem[4] = {0, 0, 0, 0};
  // geometry-inclusion local solvers (AFI_VARIANT_GEO, Section 5.2.3)
  bool geo = false;
  int nbase_tab = 0;                          // tables before the per-(patch, component) ones
  double *geo_dA = nullptr;                   // D_A^{-1/2} per dof (eq. 5.12)
  double *geo_dS = nullptr;                   // D_S^{1/2} per dof (eq. 5.13)
  double *geo_tmp = nullptr;                  // n_dof scratch of the scaled FD

  // constraints
  int2 *row_copy = nullptr;      // (dofA, dofB or -1) per row
  int2 *row_grp = nullptr;       // (group start, copies m; m = 0 -> Dirichlet)
  int2 *row_patch = nullptr;     // (patch of copy A, patch of copy B or -1)
  int *shell_dof = nullptr;      // torn index of each shell copy-dof
  int *bt_ptr = nullptr;         // CSR over shell dofs
  int *bt_ent = nullptr;         // row*2 + (sign < 0)
  long n_shell = 0;
  int *prow_ptr = nullptr;       // per patch: rows touching the patch
  int2 *prow_ent = nullptr;      // (row*2 + neg, dof); the dof becomes its component
                                 // once rigid_tables has run
  double2 *prow_coef = nullptr;  // rotation coefficients (v1, v2) of each entry
  int2 *row_cp = nullptr;        // per row: (patch*4 + component) of copy A, of copy B or -1
  double4_32a *row_cv = nullptr;     // per row: (v1, v2) of copy A, (v1, v2) of copy B
  // nested non-conforming faces (rows n_c0 .. n_c - 1): row r is
  // u_fine - sum W u_coarse; entries CSR, the fine dof first
  long n_nest = 0, n_nd = 0;         // nested rows, dofs they touch
  int n_nblk = 0;                    // (face, component) blocks of B B^T
  int *nest_ptr = nullptr, *nest_ent = nullptr;   // row CSR: entry dofs
  double *nest_w = nullptr;                       // entry weights (+1, -W)
  int4 *nest_eki = nullptr;          // per entry: (patch, component, local index, side)
  int *nd_dof = nullptr, *nd_ptr = nullptr, *nd_ent = nullptr;   // transposed CSR
  double *nd_w = nullptr;
  int *nblk_ptr = nullptr;           // block row ranges (nested-local rows)
  long long *nblk_off = nullptr;     // offsets of the blocks' dense inverses in nest_binv
  double *nest_binv = nullptr;       // (B B^T)^{-1} of each block, row-major
  int2 *nest_gk = nullptr;           // per row: (fine patch, coarse patch)
  double *nest_gc = nullptr;         // per row: G coefficients [2][nm] (fine, coarse)
  int *pn_ptr = nullptr, *pn_ent = nullptr;   // per patch: nested rows touching it (row*2 + side)
  double *nest_tmp = nullptr;        // n_nest scratch of the Schur-type block
  int *pair_ptr = nullptr;       // G^T G off-diagonal pair blocks
  int2 *pair_kk = nullptr;       // (k, k')
  int4 *pair_ent = nullptr;      // (dofA, dofB, sign product, unused)
  int npairs = 0;
  double *GtG = nullptr;         // [ng][ng] then overwritten by the inverse
  double *GtG_inv = nullptr;
  double *RtR_inv = nullptr;     // [npatch][nm][nm]
  int ng = 0;

  // workspaces
  double *ws = nullptr; long long ws_n = 0;     // general FP64 workspace
  double *fdscratch = nullptr; long long fdscratch_n = 0;
  double *ps_buf = nullptr;                     // Schur block: 4 n_dof doubles (v, o, t1, t2)
  double *ps_rint = nullptr, *ps_vint = nullptr;   // Schur block: interior right side, solution
  double *small = nullptr;                      // reduction / scalar area
  double *part = nullptr;                       // per-patch partial sums
  double *host_small = nullptr;                 // pinned host mirror
  int *dflag = nullptr;

  long long bytes = 0;

  // captured MINRES iterations (cudaGraphExec_t), rebuilt when prec changes
  void *graph_exec = nullptr;
  void *cap_stream = nullptr;        // private stream used only for capture
  void *aux_stream = nullptr;        // second stream for independent operator branches
  void *ev_fork = nullptr, *ev_join = nullptr;   // fork / join events of aux_stream
  const double *gate = nullptr;      // while enqueueing MINRES: device 'active' flag
  afi::TcSplit tcsplit[2][2];        // [interior][bf16]
  long long graph_nodes = 0;
  int graph_prec = -1;
  // several right-hand sides solved in lockstep (ieti_solve with nrhs > 1):
  // per right-hand side MINRES vectors and scalars, the captured iterations
  double *mws = nullptr;             // [kMaxRhs][kKrylov][n_dof + n_c]
  double *mst = nullptr;             // [kMaxRhs][kStStride] scalars, then the any-active flag
  double *host_mst = nullptr;        // pinned mirror of mst
  void *mgraph_exec = nullptr;
  int mgraph_nr = 0, mgraph_prec = -1;
  long long mgraph_nodes = 0;
};

namespace afi {

constexpr int kMaxRhs = 8;               // right-hand sides per lockstep solve / batched matvec
constexpr int kStStride = 128;           // doubles of MINRES scalars per right-hand side
constexpr int kSmallDoubles = 1 << 16;   // reduction scratch (partials + scalars)
constexpr int kOpScratch = 5;            // operator scratch, in units of (n_dof + n_c)
constexpr int kKrylov = 12;              // MINRES vectors of length n_dof + n_c

// allocation helper that records bytes
afi_status dalloc(afi_ctx *c, void **p, size_t bytes);

// ----------------------------------------------------------- kernels API
// setup.cu
afi_status setup_context(const afi_problem *prob, const afi_options *opt, afi_ctx *c);
void free_context(afi_ctx *c);

// ops.cu (FP64 operators on the hot path)
afi_status op_stiffness(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status stencil_to_pairs(afi_ctx *c);
bool stiffness_has_pairs(const afi_ctx *c);
afi_status op_stiffness_fp64(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_stiffness_multi(afi_ctx *c, const double *x, long long xstride, double *y,
                              long long ystride, int nr, cudaStream_t s);
afi_status stiffness_multi_prepare(afi_ctx *c, cudaStream_t s);
// mf.cu (matrix-free stiffness and mass)
afi_status mf_setup(afi_ctx *c);
afi_status mf_stiffness(afi_ctx *c, const double *x, double *y, bool exact, cudaStream_t s);
afi_status mf_mass(afi_ctx *c, const double *coef, double *f, cudaStream_t s);
afi_status solve_multi(afi_ctx *c, const double *f, double *u, double *lam, int nr,
                       afi_info *info, cudaStream_t s);
// exact.cu (EXACT local solvers, Section 5.1)
afi_status exact_setup(afi_ctx *c);
afi_status exact_PA_inv(afi_ctx *c, const double *r, double *s, cudaStream_t st);
afi_status exact_schur(afi_ctx *c, const double *t, double *y, cudaStream_t st);
long long pair_layout(std::vector<afi::DevPatch> &hp, int dim);
afi_status op_B(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_Bt(afi_ctx *c, const double *x, double *y, bool accumulate, bool zero_first,
                 cudaStream_t s);
afi_status op_Pchi(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_Pu(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_BBt_inv(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_Gt_rows(afi_ctx *c, const double *x, double *g, cudaStream_t s);
afi_status op_Rt(afi_ctx *c, const double *x, double *g, cudaStream_t s);
afi_status op_dense_inv(afi_ctx *c, const double *g, double *y, cudaStream_t s);
afi_status op_G(afi_ctx *c, const double *y, double *out, bool subtract, cudaStream_t s);
afi_status op_R_sub(afi_ctx *c, const double *y, double *v, cudaStream_t s);
afi_status rigid_tables(afi_ctx *c);
// nested non-conforming faces (nested.cu: detection, rows, blocks; ops.cu:
// the G coefficients of the rows)
struct NestedFace {
  int kc, fc, kf, ff;            // coarse patch and face, fine patch and face (face = 2 l + side)
  std::vector<int> pc, pf;       // face points (local indices, increasing)
  std::vector<double> W;         // [pf.size()][pc.size()]: fine = W coarse
};
afi_status nested_detect(afi_ctx *c, const afi_problem *prob, double quant,
                         std::vector<NestedFace> &faces, std::set<std::pair<int, int>> &apart);
afi_status nested_build(afi_ctx *c, const afi_problem *prob, const std::vector<NestedFace> &faces);
afi_status nested_gcoef(afi_ctx *c);
afi_status nested_gtg(afi_ctx *c);
afi_status op_PS(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_precond(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_saddle(afi_ctx *c, const double *x, double *y, cudaStream_t s);
afi_status op_load(afi_ctx *c, const double *coef, double *f, cudaStream_t s);
afi_status op_lame_grad(afi_ctx *c, const double *u, const double *z, double *g,
                        cudaStream_t s);
afi_status solve_one(afi_ctx *c, const double *f, double *u, double *lam, afi_info *info,
                     cudaStream_t s);

// fd.cu (local solvers: Algorithm 1 and the parametric Schur complement)
afi_status fd_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                  int nrhs = 1);
afi_status schur_run(afi_ctx *c, const double *t, double *y, cudaStream_t st);
afi_status fd_prepare(afi_ctx *c);
// fd_tc.cu (tensor-core FD over the patches that fit; the others go to the
// SIMT kernel through simt_list)
afi_status fd_tc_prepare(afi_ctx *c);
afi_status fd_tc_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                     int nrhs);
afi_status fd_simt_list(afi_ctx *c, int interior, const int *list, int count, int maxN,
                        const double *r, double *s, cudaStream_t st, int nrhs);
afi_status fd_tc_ready(afi_ctx *c);
// true when the local-solver FD (full or interior tensors) at the context's
// precision uses the shared local-solver scratch slab
bool fd_uses_scratch(afi_ctx *c, int interior);
afi_status fd_tc_tables(afi_ctx *c);
// geo.cu (geometry-inclusion local solvers, Section 5.2.3)
afi_status geo_setup(afi_ctx *c);
afi_status geo_scale(afi_ctx *c, const double *x, const double *d, double *y, long n, int nrhs,
                     cudaStream_t st);
// fd_slab.cu (three-pass tensor-core FD for tensors larger than one CTA)
afi_status slab_prepare(afi_ctx *c, int *dyn_max);
afi_status slab_build(afi_ctx *c, int interior, int fmt, const std::vector<int> &cand,
                      std::vector<int> &rest, TcSplit &sp, int dyn_max, int per);
afi_status slab_run(afi_ctx *c, int interior, int fmt, const TcSplit &sp, const double *r,
                    double *s, cudaStream_t st, int nrhs);

// reductions (ops.cu)
afi_status dot(afi_ctx *c, const double *a, const double *b, long n, double *dst,
               cudaStream_t s);

}  // namespace afi
