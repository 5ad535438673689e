// FP64 operators of the AF-IETI iteration (Section 4) and the preconditioned
// MINRES driver:
//  * stiffness matvec y = A x from the assembled per-node stencil (eq. 4.2);
//  * jump operators B x (row gather) and B^T x (gather over the rows that
//    touch each interface copy), (B B^T)^{-1} per geometric node (closed form
//    of the block I + 1 1^T, Remark 1);
//  * rigid modes R (Section 4), G = B R, P_chi (eq. 4.6), P_u, lambda_0 and
//    the recovery of (u, lambda);
//  * the saddle operator of eq. (4.7) and the preconditioner of eq. (4.9);
//  * deterministic two-stage reductions and the MINRES recurrences
//    (Paige-Saunders, zero initial guess).
#include "common.cuh"

#include <cmath>

namespace afi {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ double rigid(int a, int comp, const double *X, int dim) {
  // translations, then (0, x3, -x2), (x3, 0, -x1), (x2, -x1, 0) in 3D and
  // (x2, -x1) in 2D, evaluated at the control point X.
  if (a < dim) return (a == comp) ? 1.0 : 0.0;
  if (dim == 2) return (comp == 0) ? X[1] : -X[0];
  switch (a) {
    case 3: return comp == 1 ? X[2] : (comp == 2 ? -X[1] : 0.0);
    case 4: return comp == 0 ? X[2] : (comp == 2 ? -X[0] : 0.0);
    default: return comp == 0 ? X[1] : (comp == 1 ? -X[0] : 0.0);
  }
}

// decode a torn dof of patch k into (component, node) and fetch its point
__device__ __forceinline__ const double *dof_point(const DevPatch &pt, const double *ctrl,
                                                   long long dof, int dim, int &comp) {
  long long r = dof - pt.off;
  comp = (int)(r / pt.N);
  int node = (int)(r - (long long)comp * pt.N);
  return ctrl + pt.xoff + (long long)node * dim;
}

template <int NT>
__device__ __forceinline__ void block_sum_multi(double *vals, int nv, double *sh) {
  // sums vals[0..nv) over the block in a fixed order; result in vals on
  // thread 0.  sh: NT * nv doubles of shared scratch.
  for (int i = 0; i < nv; ++i) sh[i * NT + threadIdx.x] = vals[i];
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int i = 0; i < nv; ++i) sh[i * NT + threadIdx.x] += sh[i * NT + threadIdx.x + s];
    __syncthreads();
  }
  for (int i = 0; i < nv; ++i) vals[i] = sh[i * NT];
  __syncthreads();
}

// ------------------------------------------------------- stiffness matvec
template <int DIM>
__global__ void __launch_bounds__(128) k_stencil_mv(const DevPatch *P, const double *__restrict__ A,
                                                    const double *__restrict__ x,
                                                    double *__restrict__ y) {
  const DevPatch pt = P[blockIdx.y];
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= pt.N) return;
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2], p = pt.p;
  const int i1 = node % n1, i2 = (node / n1) % n2, i3 = node / (n1 * n2);
  const int W1 = pt.W[0], W2 = pt.W[1], W3 = pt.W[2];
  double acc[DIM];
#pragma unroll
  for (int l = 0; l < DIM; ++l) acc[l] = 0.0;
  const long long N = pt.N, S = pt.S;
  const double *Ab = A + pt.soff + node;
  for (int m = 0; m < DIM; ++m) {
    const double *xm = x + pt.off + m * N;
    for (int o3 = 0; o3 < W3; ++o3) {
      const int j3 = (DIM == 3) ? i3 + o3 - p : i3;
      if (j3 < 0 || j3 >= n3) continue;
      for (int o2 = 0; o2 < W2; ++o2) {
        const int j2 = i2 + o2 - p;
        if (j2 < 0 || j2 >= n2) continue;
        const int orow = W1 * (o2 + W2 * o3);
        const long long jrow = (long long)n1 * (j2 + (long long)n2 * j3);
        for (int o1 = 0; o1 < W1; ++o1) {
          const int j1 = i1 + o1 - p;
          const double xv = (j1 >= 0 && j1 < n1) ? xm[jrow + j1] : 0.0;
          const long long o = orow + o1;
#pragma unroll
          for (int l = 0; l < DIM; ++l) acc[l] += Ab[((long long)(l * DIM + m) * S + o) * N] * xv;
        }
      }
    }
  }
  for (int l = 0; l < DIM; ++l) y[pt.off + l * N + node] = acc[l];
}

afi_status op_stiffness(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  dim3 g((c->max_N + 127) / 128, c->npatch);
  if (c->dim == 3) launch(k_stencil_mv<3>, g, 128, 0, s, c->patches, c->stencil, x, y);
  else launch(k_stencil_mv<2>, g, 128, 0, s, c->patches, c->stencil, x, y);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// ------------------------------------------------------------------ jumps
__global__ void k_B(const int2 *rc, long n_c, const double *x, double *y, double alpha, int acc) {
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  int2 e = rc[r];
  double v = x[e.x] - (e.y >= 0 ? x[e.y] : 0.0);
  y[r] = acc ? y[r] + alpha * v : alpha * v;
}

__global__ void k_Bt(const int *shell, const int *ptr, const int *ent, long ns, const double *x,
                     double *y, double alpha, int acc) {
  long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (s >= ns) return;
  double v = 0.0;
  for (int e = ptr[s]; e < ptr[s + 1]; ++e) {
    int code = ent[e];
    double xv = x[code >> 1];
    v += (code & 1) ? -xv : xv;
  }
  int dof = shell[s];
  y[dof] = acc ? y[dof] + alpha * v : alpha * v;
}

__global__ void k_BBt_inv(const int2 *grp, long n_c, const double *x, double *y) {
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  int2 g = grp[r];
  if (g.y == 0) { y[r] = x[r]; return; }
  double s = 0.0;
  for (int j = 0; j < g.y - 1; ++j) s += x[g.x + j];
  y[r] = x[r] - s / (double)g.y;
}

afi_status op_B(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  if (c->n_c == 0) return AFI_OK;
  launch(k_B, (unsigned)((c->n_c + 255) / 256), 256, 0, s, c->row_copy, c->n_c, x, y, 1.0, 0);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

static afi_status op_Bt_scaled(afi_ctx *c, const double *x, double *y, double alpha, bool acc,
                               bool zero_first, cudaStream_t s) {
  if (zero_first) AFI_CUDA(cudaMemsetAsync(y, 0, c->n_dof * sizeof(double), s));
  if (c->n_shell == 0) return AFI_OK;
  launch(k_Bt, (unsigned)((c->n_shell + 255) / 256), 256, 0, s, c->shell_dof, c->bt_ptr, c->bt_ent,
                                                            c->n_shell, x, y, alpha, acc ? 1 : 0);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_Bt(afi_ctx *c, const double *x, double *y, bool accumulate, bool zero_first,
                 cudaStream_t s) {
  return op_Bt_scaled(c, x, y, 1.0, accumulate, zero_first, s);
}

afi_status op_BBt_inv(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  if (c->n_c == 0) return AFI_OK;
  launch(k_BBt_inv, (unsigned)((c->n_c + 255) / 256), 256, 0, s, c->row_grp, c->n_c, x, y);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// ------------------------------------------------------ rigid-mode algebra
// g[k][a] = sum over the rows touching patch k of (+-x_row) R_k(copy)[a],
// i.e. (G^T x) restricted to patch k.
template <int NM>
__global__ void __launch_bounds__(256) k_Gt(const DevPatch *P, const double *ctrl, const int *ptr,
                                            const int2 *ent, const double *x, double *g, int dim) {
  __shared__ double sh[256 * NM];
  const int k = blockIdx.x;
  const DevPatch pt = P[k];
  double acc[NM];
  for (int a = 0; a < NM; ++a) acc[a] = 0.0;
  for (int e = ptr[k] + threadIdx.x; e < ptr[k + 1]; e += blockDim.x) {
    int2 en = ent[e];
    double xv = x[en.x >> 1];
    if (en.x & 1) xv = -xv;
    int comp;
    const double *X = dof_point(pt, ctrl, en.y, dim, comp);
    for (int a = 0; a < NM; ++a) acc[a] += xv * rigid(a, comp, X, dim);
  }
  block_sum_multi<256>(acc, NM, sh);
  if (threadIdx.x == 0)
    for (int a = 0; a < NM; ++a) g[k * NM + a] = acc[a];
}

// g[k][a] = R_k^T v over all dofs of patch k.
template <int NM>
__global__ void __launch_bounds__(256) k_Rt(const DevPatch *P, const double *ctrl, const double *v,
                                            double *g, int dim) {
  __shared__ double sh[256 * NM];
  const int k = blockIdx.x;
  const DevPatch pt = P[k];
  double acc[NM];
  for (int a = 0; a < NM; ++a) acc[a] = 0.0;
  const long long n = (long long)dim * pt.N;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    int comp = (int)(i / pt.N), node = (int)(i - (long long)comp * pt.N);
    const double *X = ctrl + pt.xoff + (long long)node * dim;
    double xv = v[pt.off + i];
    for (int a = 0; a < NM; ++a) acc[a] += xv * rigid(a, comp, X, dim);
  }
  block_sum_multi<256>(acc, NM, sh);
  if (threadIdx.x == 0)
    for (int a = 0; a < NM; ++a) g[k * NM + a] = acc[a];
}

// v[dof] -= sum_a R(dof)[a] y_k[a], with y_k = Minv_k g_k if Minv != null
// (per-patch NM x NM matrices) or y_k = g_k otherwise.
__global__ void k_Rsub(const DevPatch *P, const double *ctrl, const double *src, double *dst,
                       const double *g, const double *Minv, int dim, int nm) {
  const int k = blockIdx.y;
  const DevPatch pt = P[k];
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)dim * pt.N) return;
  double y[6];
  for (int a = 0; a < nm; ++a) {
    if (Minv) {
      double s = 0.0;
      for (int b = 0; b < nm; ++b) s += Minv[(k * nm + a) * nm + b] * g[k * nm + b];
      y[a] = s;
    } else {
      y[a] = g[k * nm + a];
    }
  }
  int comp = (int)(i / pt.N), node = (int)(i - (long long)comp * pt.N);
  const double *X = ctrl + pt.xoff + (long long)node * dim;
  double s = 0.0;
  for (int a = 0; a < nm; ++a) s += rigid(a, comp, X, dim) * y[a];
  dst[pt.off + i] = src[pt.off + i] - s;
}

// dense y = M g (M: n x n), one warp per row.
__global__ void k_dense_mv(const double *M, const double *g, double *y, int n) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += M[(long long)row * n + j] * g[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// out[r] (= or -=) sum over the row's copies of sign * (R_k y_k)(copy).
__global__ void k_G(const DevPatch *P, const double *ctrl, const int2 *rc, const int2 *rk, long n_c,
                    const double *y, double *out, int dim, int nm, int subtract, const double *src) {
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  int2 e = rc[r], kk = rk[r];
  double v = 0.0;
  {
    const DevPatch pa = P[kk.x];
    int comp;
    const double *X = dof_point(pa, ctrl, e.x, dim, comp);
    for (int a = 0; a < nm; ++a) v += rigid(a, comp, X, dim) * y[kk.x * nm + a];
  }
  if (e.y >= 0) {
    const DevPatch pb = P[kk.y];
    int comp;
    const double *X = dof_point(pb, ctrl, e.y, dim, comp);
    for (int a = 0; a < nm; ++a) v -= rigid(a, comp, X, dim) * y[kk.y * nm + a];
  }
  out[r] = subtract ? src[r] - v : v;
}

afi_status op_Gt_rows(afi_ctx *c, const double *x, double *g, cudaStream_t s) {
  if (c->nm == 6) launch(k_Gt<6>, c->npatch, 256, 0, s, c->patches, c->ctrl, c->prow_ptr, c->prow_ent, x, g, c->dim);
  else launch(k_Gt<3>, c->npatch, 256, 0, s, c->patches, c->ctrl, c->prow_ptr, c->prow_ent, x, g, c->dim);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_Rt(afi_ctx *c, const double *x, double *g, cudaStream_t s) {
  if (c->nm == 6) launch(k_Rt<6>, c->npatch, 256, 0, s, c->patches, c->ctrl, x, g, c->dim);
  else launch(k_Rt<3>, c->npatch, 256, 0, s, c->patches, c->ctrl, x, g, c->dim);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_dense_inv(afi_ctx *c, const double *g, double *y, cudaStream_t s) {
  launch(k_dense_mv, (c->ng * 32 + 255) / 256, 256, 0, s, c->GtG_inv, g, y, c->ng);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

static afi_status G_apply(afi_ctx *c, const double *y, double *out, const double *src, cudaStream_t s);

// scratch for small vectors lives in c->small
static double *gbuf(afi_ctx *c, int i) { return c->small + 4096 + (long long)i * c->ng; }

afi_status op_Pchi(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  if (c->n_c == 0) return AFI_OK;
  double *g = gbuf(c, 0), *gy = gbuf(c, 1);
  AFI_TRY(op_Gt_rows(c, x, g, s));
  AFI_TRY(op_dense_inv(c, g, gy, s));
  return G_apply(c, gy, y, x, s);
}

static afi_status G_apply(afi_ctx *c, const double *y, double *out, const double *src, cudaStream_t s) {
  launch(k_G, (unsigned)((c->n_c + 255) / 256), 256, 0, s, c->patches, c->ctrl, c->row_copy,
                                                       c->row_patch, c->n_c, y, out, c->dim,
                                                       c->nm, src ? 1 : 0, src);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_G(afi_ctx *c, const double *y, double *out, bool subtract, cudaStream_t s) {
  return G_apply(c, y, out, subtract ? out : nullptr, s);
}

afi_status op_Pu(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  double *g = gbuf(c, 0);
  AFI_TRY(op_Rt(c, x, g, s));
  dim3 gr((unsigned)((c->dim * c->max_N + 255) / 256), c->npatch);
  launch(k_Rsub, gr, 256, 0, s, c->patches, c->ctrl, x, y, g, c->RtR_inv, c->dim, c->nm);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_R_sub(afi_ctx *c, const double *y, double *v, cudaStream_t s) {
  dim3 gr((unsigned)((c->dim * c->max_N + 255) / 256), c->npatch);
  launch(k_Rsub, gr, 256, 0, s, c->patches, c->ctrl, v, v, y, nullptr, c->dim, c->nm);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// --------------------------------------------------------- reductions
__global__ void k_dot_partial(const double *a, const double *b, long n, double *part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double *part, int nb, double *dst) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *dst = sh[0];
}

constexpr int kDotBlocks = 1216;   // 8 per SM on 152 SMs
constexpr int kPart = 1024;        // offset of the partials in c->small

afi_status dot(afi_ctx *c, const double *a, const double *b, long n, double *dst, cudaStream_t s) {
  launch(k_dot_partial, kDotBlocks, 256, 0, s, a, b, n, c->small + kPart);
  launch(k_sum_final, 1, 1024, 0, s, c->small + kPart, kDotBlocks, dst);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// ------------------------------------------------- composite operators
afi_status op_PS(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  // (B B^T)^{-1} B [blkdiag H^{d-2} S_hat] B^T (B B^T)^{-1} x  (Remark 1)
  double *t1 = c->ws, *t2 = c->ws + c->n_dof, *m1 = c->ws + 2 * c->n_dof;
  AFI_TRY(op_BBt_inv(c, x, m1, s));
  AFI_TRY(op_Bt(c, m1, t1, false, false, s));
  AFI_TRY(schur_run(c, t1, t2, s));
  AFI_TRY(op_B(c, t2, m1, s));
  return op_BBt_inv(c, m1, y, s);
}

afi_status op_precond(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  // calB^{-1} = blkdiag(P_u P_A^{-1} P_u^T, P_chi P_S P_chi^T), eq. (4.9)
  const long n = c->n_dof;
  double *t1 = c->ws + 3 * n + c->n_c, *m2 = c->ws + 4 * n + c->n_c;
  AFI_TRY(op_Pu(c, x, t1, s));
  AFI_TRY(fd_run(c, 0, t1, y, s));
  AFI_TRY(op_Pu(c, y, y, s));
  if (c->n_c > 0) {
    AFI_TRY(op_Pchi(c, x + n, m2, s));
    AFI_TRY(op_PS(c, m2, y + n, s));
    AFI_TRY(op_Pchi(c, y + n, y + n, s));
  }
  return AFI_OK;
}

afi_status op_saddle(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  // [A w + B^T P_chi chi ; P_chi B w], eq. (4.7)
  const long n = c->n_dof;
  double *m2 = c->ws + 4 * n + 2 * c->n_c, *m3 = m2 + c->n_c;
  AFI_TRY(op_stiffness(c, x, y, s));
  if (c->n_c > 0) {
    AFI_TRY(op_Pchi(c, x + n, m2, s));
    AFI_TRY(op_Bt(c, m2, y, true, false, s));
    AFI_TRY(op_B(c, x, m3, s));
    AFI_TRY(op_Pchi(c, m3, y + n, s));
  }
  return AFI_OK;
}

// -------------------------------------------------------------- MINRES
enum { S_BETA1 = 0, S_BETA, S_OLDB, S_ALFA, S_DBAR, S_EPSLN, S_OLDEPS, S_PHIBAR, S_CS, S_SN,
       S_DELTA, S_GAMMA, S_PHI, S_REL, S_BETA2, S_FLAG, S_DOT, S_BNORM2, S_RES2, S_COUNT };

__global__ void k_minres_init(double *st) {
  double b2 = st[S_BETA2];
  double beta1 = (b2 >= 0.0 && isfinite(b2)) ? sqrt(b2) : -1.0;
  st[S_BETA1] = beta1;
  st[S_BETA] = beta1;
  st[S_OLDB] = 0.0;
  st[S_DBAR] = 0.0;
  st[S_EPSLN] = 0.0;
  st[S_PHIBAR] = beta1;
  st[S_CS] = -1.0;
  st[S_SN] = 0.0;
  st[S_REL] = 1.0;
  st[S_FLAG] = (beta1 < 0.0) ? 2.0 : (beta1 == 0.0 ? 1.0 : 0.0);
}

__global__ void k_v_from_y(const double *y, double *v, long n, const double *st) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  v[i] = y[i] / st[S_BETA];
}

// y -= (beta/oldb) r1 (unless first), partial dots of v.y
__global__ void k_y_upd1(double *y, const double *r1, const double *v, long n, const double *st,
                         int first, double *part) {
  __shared__ double sh[256];
  double coef = first ? 0.0 : st[S_BETA] / st[S_OLDB];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double yi = y[i];
    if (!first) yi -= coef * r1[i];
    y[i] = yi;
    s += v[i] * yi;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_y_upd2(double *y, const double *r2, long n, const double *st) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] -= (st[S_ALFA] / st[S_BETA]) * r2[i];
}

__global__ void k_minres_scalars(double *st, double tol) {
  double beta2 = st[S_BETA2];
  if (!(beta2 >= 0.0) || !isfinite(beta2)) { st[S_FLAG] = 2.0; return; }
  double beta = st[S_BETA], alfa = st[S_ALFA];
  double cs = st[S_CS], sn = st[S_SN], dbar = st[S_DBAR], phibar = st[S_PHIBAR];
  st[S_OLDB] = beta;
  beta = sqrt(beta2);
  st[S_BETA] = beta;
  st[S_OLDEPS] = st[S_EPSLN];
  double delta = cs * dbar + sn * alfa;
  double gbar = sn * dbar - cs * alfa;
  st[S_EPSLN] = sn * beta;
  st[S_DBAR] = -cs * beta;
  double gamma = hypot(gbar, beta);
  if (gamma < 2.2250738585072014e-308) gamma = 2.2250738585072014e-308;
  cs = gbar / gamma;
  sn = beta / gamma;
  double phi = cs * phibar;
  phibar = sn * phibar;
  st[S_DELTA] = delta;
  st[S_GAMMA] = gamma;
  st[S_CS] = cs;
  st[S_SN] = sn;
  st[S_PHI] = phi;
  st[S_PHIBAR] = phibar;
  double rel = phibar / st[S_BETA1];
  st[S_REL] = rel;
  if (!isfinite(rel)) st[S_FLAG] = 2.0;
  else if (rel <= tol) st[S_FLAG] = 1.0;
}

__global__ void k_w_upd(const double *v, const double *w1, const double *w2, double *wn, double *x,
                        long n, const double *st) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double w = (v[i] - st[S_OLDEPS] * w1[i] - st[S_DELTA] * w2[i]) / st[S_GAMMA];
  wn[i] = w;
  x[i] += st[S_PHI] * w;
}

__global__ void k_sub(const double *a, const double *b, double *out, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = a[i] - b[i];
}

__global__ void k_add(const double *a, const double *b, double *out, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = a[i] + b[i];
}

static inline unsigned nblk(long n) { return (unsigned)((n + 255) / 256); }

// one right-hand side
afi_status solve_one(afi_ctx *c, const double *f, double *u, double *lam_out, afi_info *info,
                     cudaStream_t s) {
  const long n = c->n_dof, m = c->n_c, nt = n + m;
  double *V = c->ws + kOpScratch * (n + m);   // Krylov vectors after the operator scratch
  double *b = V, *x = V + nt, *v = V + 2 * nt;
  double *buf[3] = {V + 3 * nt, V + 4 * nt, V + 5 * nt};   // r1, r2, y rotation
  double *wb[2] = {V + 6 * nt, V + 7 * nt};                 // older / newer w
  double *tmp = V + 9 * nt, *lam0 = V + 10 * nt;
  double *st = c->small;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  // lambda_0 = G (G^T G)^{-1} R^T f and b = [f - B^T lambda_0; 0]
  if (m > 0) {
    AFI_TRY(op_Rt(c, f, gbuf(c, 0), s));
    AFI_TRY(op_dense_inv(c, gbuf(c, 0), gbuf(c, 1), s));
    AFI_TRY(G_apply(c, gbuf(c, 1), lam0, nullptr, s));
  }
  AFI_CUDA(cudaMemcpyAsync(b, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (m > 0) {
    AFI_TRY(op_Bt_scaled(c, lam0, b, -1.0, true, false, s));
    AFI_CUDA(cudaMemsetAsync(b + n, 0, m * sizeof(double), s));
  }
  AFI_CUDA(cudaMemsetAsync(x, 0, nt * sizeof(double), s));
  AFI_CUDA(cudaMemsetAsync(wb[0], 0, nt * sizeof(double), s));
  AFI_CUDA(cudaMemsetAsync(wb[1], 0, nt * sizeof(double), s));
  double *r1 = buf[0], *r2 = buf[1], *y = buf[2];
  AFI_CUDA(cudaMemcpyAsync(r1, b, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AFI_CUDA(cudaMemcpyAsync(r2, b, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AFI_TRY(op_precond(c, r1, y, s));
  AFI_TRY(dot(c, r1, y, nt, st + S_BETA2, s));
  AFI_TRY(dot(c, b, b, nt, st + S_BNORM2, s));
  launch(k_minres_init, 1, 1, 0, s, st);
  AFI_LAUNCH_CHECK();
  double *hs = c->host_small;
  AFI_CUDA(cudaMemcpyAsync(hs, st, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  AFI_CUDA(cudaStreamSynchronize(s));
  int itn = 0;
  afi_status status = AFI_OK;
  const double tol = c->opt.tol;
  const double bnorm = sqrt(hs[S_BNORM2]);
  double relres_true = 0.0;
  int last_check = -1000000;
  if (hs[S_FLAG] == 2.0) status = AFI_EBREAKDOWN;
  bool done = (hs[S_FLAG] != 0.0);
  double *w1 = wb[0], *w2 = wb[1];
  while (!done && itn < c->opt.maxit) {
    ++itn;
    launch(k_v_from_y, nblk(nt), 256, 0, s, y, v, nt, st);
    AFI_TRY(op_saddle(c, v, y, s));
    launch(k_y_upd1, kDotBlocks, 256, 0, s, y, r1, v, nt, st, itn == 1, c->small + kPart);
    launch(k_sum_final, 1, 1024, 0, s, c->small + kPart, kDotBlocks, st + S_ALFA);
    launch(k_y_upd2, nblk(nt), 256, 0, s, y, r2, nt, st);
    AFI_LAUNCH_CHECK();
    double *t = r1; r1 = r2; r2 = y; y = t;
    AFI_TRY(op_precond(c, r2, y, s));
    AFI_TRY(dot(c, r2, y, nt, st + S_BETA2, s));
    launch(k_minres_scalars, 1, 1, 0, s, st, tol);
    // w update uses the rotated buffers: new w overwrites w1's storage
    launch(k_w_upd, nblk(nt), 256, 0, s, v, w1, w2, w1, x, nt, st);
    AFI_LAUNCH_CHECK();
    double *tw = w1; w1 = w2; w2 = tw;   // (w1, w2) <- (old w2, new w)
    AFI_CUDA(cudaMemcpyAsync(hs, st, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFI_CUDA(cudaStreamSynchronize(s));
    if (hs[S_FLAG] == 2.0) { status = AFI_EBREAKDOWN; break; }
    if (hs[S_FLAG] == 1.0 && itn - last_check >= 5) {
      last_check = itn;
      AFI_TRY(op_saddle(c, x, tmp, s));
      launch(k_sub, nblk(nt), 256, 0, s, b, tmp, tmp, nt);
      AFI_TRY(dot(c, tmp, tmp, nt, st + S_RES2, s));
      AFI_CUDA(cudaMemcpyAsync(hs, st, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
      AFI_CUDA(cudaStreamSynchronize(s));
      relres_true = sqrt(hs[S_RES2]) / (bnorm > 0 ? bnorm : 1.0);
      if (relres_true <= tol) done = true;
    }
  }
  if (!done && status == AFI_OK) status = AFI_ENOT_CONVERGED;
  // true residual of the final iterate if not just measured
  if (last_check != itn) {
    AFI_TRY(op_saddle(c, x, tmp, s));
    launch(k_sub, nblk(nt), 256, 0, s, b, tmp, tmp, nt);
    AFI_TRY(dot(c, tmp, tmp, nt, st + S_RES2, s));
    AFI_CUDA(cudaMemcpyAsync(hs, st, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFI_CUDA(cudaStreamSynchronize(s));
    relres_true = sqrt(hs[S_RES2]) / (bnorm > 0 ? bnorm : 1.0);
  }
  // recovery: u = w - R (G^T G)^{-1} G^T B w, lambda = lambda_0 + chi
  AFI_CUDA(cudaMemcpyAsync(u, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (m > 0) {
    double *t = tmp;   // B w
    AFI_TRY(op_B(c, x, t, s));
    AFI_TRY(op_Gt_rows(c, t, gbuf(c, 0), s));
    AFI_TRY(op_dense_inv(c, gbuf(c, 0), gbuf(c, 1), s));
    AFI_TRY(op_R_sub(c, gbuf(c, 1), u, s));
    if (lam_out) {
      launch(k_add, nblk(m), 256, 0, s, lam0, x + n, lam_out, m);
      AFI_LAUNCH_CHECK();
    }
  }
  cudaEventRecord(e1, s);
  AFI_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iters = itn;
    info->relres_est = hs[S_REL];
    info->relres_true = relres_true;
    info->t_setup_ms = c->t_setup_ms;
    info->t_solve_ms = ms;
  }
  if (status == AFI_EBREAKDOWN) set_error("MINRES breakdown (non-finite or negative norm)");
  if (status == AFI_ENOT_CONVERGED) set_error("MINRES reached maxit before the tolerance");
  return status;
}

}  // namespace afi
