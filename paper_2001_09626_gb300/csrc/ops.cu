// FP64 operators of the AF-IETI iteration (Section 4) and the preconditioned
// MINRES driver (the stiffness matvec is in stencil.cu):
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
  const int r = (int)(dof - pt.off);   // within one patch: fits in 32 bits
  comp = r / pt.N;
  const int node = r - comp * pt.N;
  return ctrl + pt.xoff + (long long)node * dim;
}

template <int NT>
__device__ __forceinline__ void block_sum_multi(double *vals, int nv, double *sh) {
  // sums vals[0..nv) over the block in a fixed order (warp shuffles, then
  // the per-warp sums in warp order); result in vals on thread 0.
  // sh: (NT / 32) * nv doubles of shared scratch.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    double v = vals[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[i * (NT / 32) + warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < nv; ++i) {
      double v = 0.0;
      for (int w = 0; w < NT / 32; ++w) v += sh[i * (NT / 32) + w];
      vals[i] = v;
    }
  __syncthreads();
}

// the nested-face rows (defined below, with their kernels)
static void nest_B(afi_ctx *c, const double *x, double *yr, double alpha, int acc, cudaStream_t s);
static void nest_Bt(afi_ctx *c, const double *xr, double *y, double alpha, int acc, cudaStream_t s);
static void nest_blockinv(afi_ctx *c, const double *xr, double *yr, cudaStream_t s);

// ------------------------------------------------------------------ jumps
__global__ void k_B(const int2 *rc, long n_c, const double *x, double *y, double alpha, int acc, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  int2 e = rc[r];
  double v = x[e.x] - (e.y >= 0 ? x[e.y] : 0.0);
  y[r] = acc ? y[r] + alpha * v : alpha * v;
}

__global__ void k_Bt(const int *shell, const int *ptr, const int *ent, long ns, const double *x,
                     double *y, double alpha, int acc, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
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

__global__ void k_BBt_inv(const int2 *grp, long n_c, const double *x, double *y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  int2 g = grp[r];
  if (g.y == 0) { y[r] = x[r]; return; }
  double s = 0.0;
  for (int j = 0; j < g.y - 1; ++j) s += x[g.x + j];
  y[r] = x[r] - s / (double)g.y;
}

// y = B^T (B B^T)^{-1} x over the shell dofs (other entries of y untouched).
// The rows touching one dof all belong to its node's group, whose block of
// B B^T is inverted in closed form (I - 1 1^T / m for a star of m copies).
__global__ void k_Bt_inv(const int *shell, const int *ptr, const int *ent, const int2 *grp, long ns,
                         const double *x, double *y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int e0 = ptr[s], e1 = ptr[s + 1];
  const int2 g = grp[ent[e0] >> 1];
  double corr = 0.0;
  if (g.y > 0) {
    double sum = 0.0;
    for (int j = 0; j < g.y - 1; ++j) sum += x[g.x + j];
    corr = sum / (double)g.y;
  }
  double v = 0.0;
  for (int e = e0; e < e1; ++e) {
    const int code = ent[e];
    const double xv = x[code >> 1] - corr;
    v += (code & 1) ? -xv : xv;
  }
  y[shell[s]] = v;
}

// y = (B B^T)^{-1} B x: each row recomputes the jumps of its group's rows.
__global__ void k_B_inv(const int2 *rc, const int2 *grp, long n_c, const double *x, double *y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  const int2 e = rc[r], g = grp[r];
  const double own = x[e.x] - (e.y >= 0 ? x[e.y] : 0.0);
  if (g.y == 0) { y[r] = own; return; }
  double sum = 0.0;
  for (int j = 0; j < g.y - 1; ++j) {
    const int2 f = rc[g.x + j];
    sum += x[f.x] - (f.y >= 0 ? x[f.y] : 0.0);
  }
  y[r] = own - sum / (double)g.y;
}

afi_status op_B(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  if (c->n_c == 0) return AFI_OK;
  if (c->n_c0)
    launch(k_B, (unsigned)((c->n_c0 + 255) / 256), 256, 0, s, c->row_copy, c->n_c0, x, y, 1.0, 0,
           (const double *)c->gate);
  if (c->n_nest) nest_B(c, x, y + c->n_c0, 1.0, 0, s);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

static afi_status op_Bt_scaled(afi_ctx *c, const double *x, double *y, double alpha, bool acc,
                               bool zero_first, cudaStream_t s) {
  if (zero_first) AFI_CUDA(cudaMemsetAsync(y, 0, c->n_dof * sizeof(double), s));
  if (c->n_shell)
    launch(k_Bt, (unsigned)((c->n_shell + 255) / 256), 256, 0, s, c->shell_dof, c->bt_ptr, c->bt_ent,
           c->n_shell, x, y, alpha, acc ? 1 : 0, (const double *)c->gate);
  if (c->n_nest) nest_Bt(c, x + c->n_c0, y, alpha, acc ? 1 : 0, s);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_Bt(afi_ctx *c, const double *x, double *y, bool accumulate, bool zero_first,
                 cudaStream_t s) {
  return op_Bt_scaled(c, x, y, 1.0, accumulate, zero_first, s);
}

afi_status op_BBt_inv(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  if (c->n_c == 0) return AFI_OK;
  if (c->n_c0)
    launch(k_BBt_inv, (unsigned)((c->n_c0 + 255) / 256), 256, 0, s, c->row_grp, c->n_c0, x, y,
           (const double *)c->gate);
  if (c->n_nest) nest_blockinv(c, x + c->n_c0, y + c->n_c0, s);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// ------------------------------------------------------ rigid-mode algebra
// The rigid modes of a component-`comp` dof at point X: the translation
// `comp` (value 1) and two rotations (3D) or one (2D), see rigid().
struct RigidNZ { int m1, m2; double v1, v2; };
__device__ __forceinline__ RigidNZ rigid_nz(int comp, const double *X, int dim) {
  RigidNZ r;
  if (dim == 2) {
    r.m1 = 2; r.v1 = (comp == 0) ? X[1] : -X[0];
    r.m2 = 2; r.v2 = 0.0;
  } else if (comp == 0) {
    r.m1 = 4; r.v1 = X[2]; r.m2 = 5; r.v2 = X[1];
  } else if (comp == 1) {
    r.m1 = 3; r.v1 = X[2]; r.m2 = 5; r.v2 = -X[0];
  } else {
    r.m1 = 3; r.v1 = -X[1]; r.m2 = 4; r.v2 = -X[0];
  }
  return r;
}

constexpr int kCounters = 3072;  // block tickets of the last-block reductions, in c->small
constexpr int kGtBlocks = 4;    // blocks per patch for the row-list reduction
constexpr int kRtChunksMax = 16;   // blocks per (patch, component) for R^T v, at most
                                   // (partials: dim * 16 * 3 <= the 320 per patch of
                                   // the P_u slice); about one per 8192 nodes, at least 4

// After each block has written its partials: true (in every thread) in the
// block that finishes last, which then combines all partials; it resets the
// ticket counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned *counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    last = atomicAdd(counter, 1u) == nb - 1;
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Partial sums of (G^T x) over a strided part of the rows touching patch k:
// part[(k * kGtBlocks + b) * NM + a].  Each entry touches its translation
// and two rotations only, with the rotation coefficients precomputed per
// entry (ent[e] = (row*2 + neg, component), coef[e] = (v1, v2), see
// rigid_nz); the lists are sorted by dof, so a warp mostly sees one
// component.
template <int NM>
__global__ void __launch_bounds__(256) k_Gt_part(const int *ptr, const int2 *ent, const double2 *coef,
                                                 const double *x, double *part, unsigned *counter,
                                                 double *g, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  __shared__ double sh[8 * NM];
  const int k = blockIdx.y, b = blockIdx.x;
  double acc[NM];
#pragma unroll
  for (int a = 0; a < NM; ++a) acc[a] = 0.0;
#pragma unroll 4
  for (int e = ptr[k] + b * blockDim.x + threadIdx.x; e < ptr[k + 1]; e += gridDim.x * blockDim.x) {
    const int2 en = ent[e];
    const double2 cf = coef[e];
    double xv = x[en.x >> 1];
    if (en.x & 1) xv = -xv;
    if (NM == 6) {
      if (en.y == 0) { acc[0] += xv; acc[4] += xv * cf.x; acc[5] += xv * cf.y; }
      else if (en.y == 1) { acc[1] += xv; acc[3] += xv * cf.x; acc[5] += xv * cf.y; }
      else { acc[2] += xv; acc[3] += xv * cf.x; acc[4] += xv * cf.y; }
    } else {
      if (en.y == 0) { acc[0] += xv; acc[2] += xv * cf.x; }
      else { acc[1] += xv; acc[2] += xv * cf.x; }
    }
  }
  block_sum_multi<256>(acc, NM, sh);
  if (threadIdx.x == 0)
    for (int a = 0; a < NM; ++a) part[((long long)k * gridDim.x + b) * NM + a] = acc[a];
  // g[k][a] = sum over the blocks of patch k, in block order
  if (!last_block(counter)) return;
  // (L2 loads: the partials were written by other blocks of this launch)
  const int npatch = gridDim.y;
  for (int e = threadIdx.x; e < npatch * NM; e += blockDim.x) {
    const int kk = e / NM, a = e - kk * NM;
    double sum = 0.0;
    for (int bb = 0; bb < (int)gridDim.x; ++bb) sum += __ldcg(part + ((long long)kk * gridDim.x + bb) * NM + a);
    g[e] = sum;
  }
}

// Partial sums of R_k^T v over one chunk of one component block: the
// translation and the two rotation products, part[((k*dim + comp)*CH + ch)*3].
__global__ void __launch_bounds__(256) k_Rt_part(const DevPatch *P, const double *ctrl,
                                                 const double *v, double *part, int dim,
                                                 unsigned *counter, int nm, double *g,
                                                 const double *Minv, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  __shared__ double sh[8 * 3];
  const int ch = blockIdx.x, comp = blockIdx.y, k = blockIdx.z;
  const DevPatch pt = P[k];
  const double *vc = v + pt.off + (long long)comp * pt.N;
  const double *Xb = ctrl + pt.xoff;
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll 4
  for (int i = ch * blockDim.x + threadIdx.x; i < pt.N; i += gridDim.x * blockDim.x) {
    const double xv = vc[i];
    const RigidNZ r = rigid_nz(comp, Xb + (long long)i * dim, dim);
    acc[0] += xv;
    acc[1] += xv * r.v1;
    acc[2] += xv * r.v2;
  }
  block_sum_multi<256>(acc, 3, sh);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) part[(((long long)k * dim + comp) * gridDim.x + ch) * 3 + a] = acc[a];
  // per patch: the modes' sums over components and chunks (fixed order),
  // then optionally Minv_k times them
  if (!last_block(counter)) return;
  const int nch = gridDim.x;
  for (int kk = threadIdx.x; kk < (int)gridDim.z; kk += blockDim.x) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    const double X0[3] = {0.0, 0.0, 0.0};
    for (int cp = 0; cp < dim; ++cp) {
      const RigidNZ r = rigid_nz(cp, X0, dim);   // only the mode indices are used
      double q[3] = {0.0, 0.0, 0.0};
      for (int c2 = 0; c2 < nch; ++c2)
        for (int a = 0; a < 3; ++a) q[a] += __ldcg(part + (((long long)kk * dim + cp) * nch + c2) * 3 + a);
      t[cp] += q[0];
      t[r.m1] += q[1];
      if (dim == 3) t[r.m2] += q[2];
    }
    for (int a = 0; a < nm; ++a) {
      double val = t[a];
      if (Minv) {
        val = 0.0;
        for (int b2 = 0; b2 < nm; ++b2) val += Minv[((long long)kk * nm + a) * nm + b2] * t[b2];
      }
      g[kk * nm + a] = val;
    }
  }
}

// dst = src - R_k y_k on every dof (y per patch, NM entries).
__global__ void k_Rsub(const DevPatch *P, const double *ctrl, const double *src, double *dst,
                       const double *y, int dim, int nm, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const int comp = blockIdx.y, k = blockIdx.z;
  const DevPatch pt = P[k];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pt.N) return;
  const RigidNZ r = rigid_nz(comp, ctrl + pt.xoff + (long long)i * dim, dim);
  const double *yk = y + k * nm;
  double sub = yk[comp] + r.v1 * yk[r.m1];
  if (dim == 3) sub += r.v2 * yk[r.m2];
  const long long at = pt.off + (long long)comp * pt.N + i;
  dst[at] = src[at] - sub;
}

// ------------------------------------------------ nested faces (rows n_c0..)
// The rows of nested non-conforming faces (nested.cu): row r is
// u_fine - sum W u_coarse, CSR entries (dof, weight); xr / yr point at the
// first nested row of a multiplier vector.

// G coefficients of every nested row (setup): per side (fine, coarse) the
// row's products with the patch's rigid modes, sum over the entries of
// weight x R(dof, mode).
__global__ void k_nest_gcoef(const DevPatch *P, const double *ctrl, const int *ptr, const double *w,
                             const int4 *eki, int nr, int dim, int nm, double *gc) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  double g[2][6] = {{0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) {
    const int4 q = eki[e];
    const RigidNZ rz = rigid_nz(q.y, ctrl + P[q.x].xoff + (long long)q.z * dim, dim);
    const double we = w[e];
    g[q.w][q.y] += we;
    g[q.w][rz.m1] += we * rz.v1;
    if (dim == 3) g[q.w][rz.m2] += we * rz.v2;
  }
  for (int sd = 0; sd < 2; ++sd)
    for (int a = 0; a < nm; ++a) gc[((long long)r * 2 + sd) * nm + a] = g[sd][a];
}

// yr[r] (= or += alpha *) sum over the row's entries of weight * x[dof]
__global__ void k_nest_B(const int *ptr, const int *ent, const double *w, long nr, const double *x,
                         double *yr, double alpha, int acc, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  double v = 0.0;
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) v += w[e] * x[ent[e]];
  yr[r] = acc ? yr[r] + alpha * v : alpha * v;
}

// y[dof] (= or += alpha *) sum over the nested rows touching the dof of
// weight * xr[row], for the dofs the nested rows touch
__global__ void k_nest_Bt(const int *dofs, const int *ptr, const int *ent, const double *w, long nd,
                          const double *xr, double *y, double alpha, int acc, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= nd) return;
  double v = 0.0;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) v += w[e] * xr[ent[e]];
  const int d = dofs[i];
  y[d] = acc ? y[d] + alpha * v : alpha * v;
}

// yr = blockdiag((B B^T)^{-1}) xr over the (face, component) blocks: one CTA
// per block, one warp per row of the block's dense inverse
__global__ void k_nest_blockinv(const int *bptr, const long long *boff, const double *binv,
                                const double *xr, double *yr, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const int b = blockIdx.x, r0 = bptr[b], m = bptr[b + 1] - r0;
  const double *M = binv + boff[b];
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x >> 5; i < m; i += nw) {
    double v = 0.0;
    for (int j = lane; j < m; j += 32) v += M[(long long)i * m + j] * xr[r0 + j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) yr[r0 + i] = v;
  }
}

// outr[r] = (src ? srcr[r] - : ) (G y)[row r]
__global__ void k_nest_G(const int2 *gk, const double *gc, long nr, int nm, const double *y,
                         double *outr, const double *srcr, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const int2 k = gk[r];
  const double *g = gc + r * 2 * nm;
  double v = 0.0;
  for (int a = 0; a < nm; ++a) v += g[a] * y[k.x * nm + a] + g[nm + a] * y[k.y * nm + a];
  outr[r] = srcr ? srcr[r] - v : v;
}

// g[k nm + a] += sum over the nested rows touching patch k of their
// coefficient of mode a times xr[row]: one CTA per patch, fixed order
template <int NM>
__global__ void __launch_bounds__(256) k_nest_Gt(const int *pptr, const int *pent, const double *gc,
                                                 const double *xr, double *g, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  __shared__ double sh[8 * NM];
  const int k = blockIdx.x;
  double acc[NM];
#pragma unroll
  for (int a = 0; a < NM; ++a) acc[a] = 0.0;
  for (int e = pptr[k] + threadIdx.x; e < pptr[k + 1]; e += blockDim.x) {
    const int code = pent[e], r = code >> 1, sd = code & 1;
    const double xv = xr[r];
#pragma unroll
    for (int a = 0; a < NM; ++a) acc[a] += gc[((long long)r * 2 + sd) * NM + a] * xv;
  }
  block_sum_multi<256>(acc, NM, sh);
  if (threadIdx.x == 0 && pptr[k + 1] > pptr[k])
    for (int a = 0; a < NM; ++a) g[k * NM + a] += acc[a];
}

afi_status nested_gcoef(afi_ctx *c) {
  if (!c->n_nest) return AFI_OK;
  launch(k_nest_gcoef, (unsigned)((c->n_nest + 127) / 128), 128, 0, 0, (const DevPatch *)c->patches,
         (const double *)c->ctrl, (const int *)c->nest_ptr, (const double *)c->nest_w,
         (const int4 *)c->nest_eki, (int)c->n_nest, c->dim, c->nm, c->nest_gc);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

static void nest_B(afi_ctx *c, const double *x, double *yr, double alpha, int acc, cudaStream_t s) {
  launch(k_nest_B, (unsigned)((c->n_nest + 255) / 256), 256, 0, s, (const int *)c->nest_ptr,
         (const int *)c->nest_ent, (const double *)c->nest_w, c->n_nest, x, yr, alpha, acc,
         (const double *)c->gate);
}

static void nest_Bt(afi_ctx *c, const double *xr, double *y, double alpha, int acc, cudaStream_t s) {
  launch(k_nest_Bt, (unsigned)((c->n_nd + 255) / 256), 256, 0, s, (const int *)c->nd_dof,
         (const int *)c->nd_ptr, (const int *)c->nd_ent, (const double *)c->nd_w, c->n_nd, xr, y,
         alpha, acc, (const double *)c->gate);
}

static void nest_blockinv(afi_ctx *c, const double *xr, double *yr, cudaStream_t s) {
  launch(k_nest_blockinv, (unsigned)c->n_nblk, 256, 0, s, (const int *)c->nblk_ptr,
         (const long long *)c->nblk_off, (const double *)c->nest_binv, xr, yr, (const double *)c->gate);
}

// dense y = M g (M: n x n), one warp per row.
__global__ void k_dense_mv(const double *M, const double *g, double *y, int n, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += M[(long long)row * n + j] * g[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// (R_k y_k) at one dof: its translation plus two rotations (one in 2D).
__device__ __forceinline__ double rigid_apply(int comp, const double *X, const double *y, int dim) {
  const RigidNZ r = rigid_nz(comp, X, dim);
  double v = y[comp] + r.v1 * y[r.m1];
  if (dim == 3) v += r.v2 * y[r.m2];
  return v;
}

// out[r] (= or -=) sum over the row's copies of sign * (R_k y_k)(copy).
// out[r] (= or -=) sum over the row's copies of sign * (R_k y_k)(copy), with
// the copies' (patch * 4 + component) in cp[r] and their rotation
// coefficients (v1, v2 per copy) in cv[r].
__global__ void k_G(const int2 *cp, const double4_32a *cv, long n_c, const double *y, double *out, int dim,
                    int nm, int subtract, const double *src, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  const int2 e = cp[r];
  const double4_32a v4 = cv[r];
  const double X0[3] = {0.0, 0.0, 0.0};
  const double *ya = y + (e.x >> 2) * nm;
  RigidNZ ra = rigid_nz(e.x & 3, X0, dim);   // mode indices only
  double v = ya[e.x & 3] + v4.x * ya[ra.m1] + v4.y * ya[ra.m2];
  if (e.y >= 0) {
    const double *yb = y + (e.y >> 2) * nm;
    RigidNZ rb = rigid_nz(e.y & 3, X0, dim);
    v -= yb[e.y & 3] + v4.z * yb[rb.m1] + v4.w * yb[rb.m2];
  }
  out[r] = subtract ? src[r] - v : v;
}

// Rotation coefficients of G = B R, once at setup: per constraint row the
// (patch * 4 + component) and (v1, v2) of both copies, and per entry of the
// per-patch row lists the component and (v1, v2) of its dof.
__global__ void k_rigid_tables(const DevPatch *P, const double *ctrl, const int2 *rc, const int2 *rk,
                               long n_c, int2 *cp, double4_32a *cv, const int *pptr, int2 *pent,
                               double2 *pcoef, int npatch, int dim) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < n_c) {
    const int2 e = rc[t], kk = rk[t];
    int ca, cb;
    const double *Xa = dof_point(P[kk.x], ctrl, e.x, dim, ca);
    const RigidNZ a = rigid_nz(ca, Xa, dim);
    double4_32a v = make_double4_32a(a.v1, dim == 3 ? a.v2 : 0.0, 0.0, 0.0);
    int2 c2 = make_int2(kk.x * 4 + ca, -1);
    if (e.y >= 0) {
      const double *Xb = dof_point(P[kk.y], ctrl, e.y, dim, cb);
      const RigidNZ b = rigid_nz(cb, Xb, dim);
      v.z = b.v1;
      v.w = dim == 3 ? b.v2 : 0.0;
      c2.y = kk.y * 4 + cb;
    }
    cp[t] = c2;
    cv[t] = v;
  }
  // entries of the per-patch lists: patch k owns [pptr[k], pptr[k+1])
  const long ne = pptr[npatch];
  for (long e = t; e < ne; e += (long)gridDim.x * blockDim.x) {
    int lo = 0, hi = npatch;   // the patch of entry e
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pptr[mid] <= e) lo = mid; else hi = mid;
    }
    int comp;
    const double *X = dof_point(P[lo], ctrl, pent[e].y, dim, comp);
    const RigidNZ r = rigid_nz(comp, X, dim);
    pcoef[e] = make_double2(r.v1, dim == 3 ? r.v2 : 0.0);
    pent[e].y = comp;
  }
}

afi_status rigid_tables(afi_ctx *c) {
  if (c->n_c0 == 0) return AFI_OK;
  AFI_TRY(dalloc(c, (void **)&c->row_cp, (size_t)c->n_c0 * sizeof(int2)));
  AFI_TRY(dalloc(c, (void **)&c->row_cv, (size_t)c->n_c0 * sizeof(double4_32a)));
  int ne = 0;
  AFI_CUDA(cudaMemcpy(&ne, c->prow_ptr + c->npatch, sizeof(int), cudaMemcpyDeviceToHost));
  AFI_TRY(dalloc(c, (void **)&c->prow_coef, (size_t)std::max(ne, 1) * sizeof(double2)));
  const long nt = std::max((long)ne, c->n_c0);
  launch(k_rigid_tables, (unsigned)((nt + 255) / 256), 256, 0, 0, (const DevPatch *)c->patches,
         (const double *)c->ctrl, (const int2 *)c->row_copy, (const int2 *)c->row_patch, c->n_c0,
         c->row_cp, c->row_cv, (const int *)c->prow_ptr, c->prow_ent, c->prow_coef, c->npatch, c->dim);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_Gt_rows(afi_ctx *c, const double *x, double *g, cudaStream_t s) {
  dim3 gr(kGtBlocks, c->npatch);
  unsigned *cnt = reinterpret_cast<unsigned *>(c->small + kCounters) + 2;
  if (c->nm == 6)
    launch(k_Gt_part<6>, gr, 256, 0, s, (const int *)c->prow_ptr, (const int2 *)c->prow_ent,
           (const double2 *)c->prow_coef, x, c->part, cnt, g, (const double *)c->gate);
  else
    launch(k_Gt_part<3>, gr, 256, 0, s, (const int *)c->prow_ptr, (const int2 *)c->prow_ent,
           (const double2 *)c->prow_coef, x, c->part, cnt, g, (const double *)c->gate);
  if (c->n_nest) {   // the nested rows' share, added after the node rows' sums
    if (c->nm == 6)
      launch(k_nest_Gt<6>, c->npatch, 256, 0, s, (const int *)c->pn_ptr, (const int *)c->pn_ent,
             (const double *)c->nest_gc, x + c->n_c0, g, (const double *)c->gate);
    else
      launch(k_nest_Gt<3>, c->npatch, 256, 0, s, (const int *)c->pn_ptr, (const int *)c->pn_ent,
             (const double *)c->nest_gc, x + c->n_c0, g, (const double *)c->gate);
  }
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// g = R^T v per patch; with Minv, g = Minv_k (R_k^T v) instead.
// The P_u reductions use their own slice of c->part, ticket and g buffer, so
// that they can run concurrently with the P_chi reductions (op_precond).
static double *pu_part(afi_ctx *c) { return c->part + 64LL * c->npatch; }

static afi_status Rt_apply(afi_ctx *c, const double *x, double *g, const double *Minv, cudaStream_t s) {
  unsigned *cnt = reinterpret_cast<unsigned *>(c->small + kCounters) + 3;
  const int chunks = std::min(kRtChunksMax, std::max(4, (int)((c->max_N + 8191) / 8192)));
  launch(k_Rt_part, dim3(chunks, c->dim, c->npatch), 256, 0, s, c->patches, c->ctrl, x, pu_part(c),
         c->dim, cnt, c->nm, g, Minv, (const double *)c->gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_Rt(afi_ctx *c, const double *x, double *g, cudaStream_t s) {
  return Rt_apply(c, x, g, nullptr, s);
}

afi_status op_dense_inv(afi_ctx *c, const double *g, double *y, cudaStream_t s) {
  launch(k_dense_mv, (c->ng * 32 + 255) / 256, 256, 0, s, c->GtG_inv, g, y, c->ng, (const double *)c->gate);
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
  if (c->n_c0)
    launch(k_G, (unsigned)((c->n_c0 + 255) / 256), 256, 0, s, (const int2 *)c->row_cp,
           (const double4_32a *)c->row_cv, c->n_c0, y, out, c->dim, c->nm, src ? 1 : 0, src,
           (const double *)c->gate);
  if (c->n_nest)
    launch(k_nest_G, (unsigned)((c->n_nest + 255) / 256), 256, 0, s, (const int2 *)c->nest_gk,
           (const double *)c->nest_gc, c->n_nest, c->nm, y, out + c->n_c0,
           src ? src + c->n_c0 : (const double *)nullptr, (const double *)c->gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_G(afi_ctx *c, const double *y, double *out, bool subtract, cudaStream_t s) {
  return G_apply(c, y, out, subtract ? out : nullptr, s);
}

afi_status op_Pu(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  // P_u x = x - R (R^T R)^{-1} R^T x, patch by patch
  double *g = gbuf(c, 2);
  AFI_TRY(Rt_apply(c, x, g, c->RtR_inv, s));
  launch(k_Rsub, dim3((c->max_N + 255) / 256, c->dim, c->npatch), 256, 0, s, c->patches, c->ctrl, x,
         y, (const double *)g, c->dim, c->nm, (const double *)c->gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status op_R_sub(afi_ctx *c, const double *y, double *v, cudaStream_t s) {
  launch(k_Rsub, dim3((c->max_N + 255) / 256, c->dim, c->npatch), 256, 0, s, c->patches, c->ctrl,
         (const double *)v, v, y, c->dim, c->nm, (const double *)c->gate);
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
  double *t1 = c->ws, *t2 = c->ws + c->n_dof;
  if (c->n_c == 0) return AFI_OK;
  // shell dofs on a natural-boundary face and on no interface have no
  // constraint row: B^T leaves them zero, and the Schur block reads them
  AFI_CUDA(cudaMemsetAsync(t1, 0, (size_t)c->n_dof * sizeof(double), s));
  if (c->n_shell)
    launch(k_Bt_inv, (unsigned)((c->n_shell + 255) / 256), 256, 0, s, (const int *)c->shell_dof,
           (const int *)c->bt_ptr, (const int *)c->bt_ent, (const int2 *)c->row_grp, c->n_shell, x, t1, (const double *)c->gate);
  if (c->n_nest) {   // nested rows: their block inverse, then B^T onto their dofs
    nest_blockinv(c, x + c->n_c0, c->nest_tmp, s);
    nest_Bt(c, c->nest_tmp, t1, 1.0, 0, s);
  }
  if (c->exact) AFI_TRY(exact_schur(c, t1, t2, s));
  else AFI_TRY(schur_run(c, t1, t2, s));
  if (c->n_c0)
    launch(k_B_inv, (unsigned)((c->n_c0 + 255) / 256), 256, 0, s, (const int2 *)c->row_copy,
           (const int2 *)c->row_grp, c->n_c0, (const double *)t2, y, (const double *)c->gate);
  if (c->n_nest) {
    nest_B(c, t2, c->nest_tmp, 1.0, 0, s);
    nest_blockinv(c, c->nest_tmp, y + c->n_c0, s);
  }
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// Independent branches of an operator run on the context's second stream:
// fork() makes it wait for everything enqueued on s so far, join() makes s
// wait for the branch.  Under stream capture this records a fork and a join
// in the graph.
static afi_status fork_aux(afi_ctx *c, cudaStream_t s, cudaStream_t *aux) {
  *aux = (cudaStream_t)c->aux_stream;
  AFI_CUDA(cudaEventRecord((cudaEvent_t)c->ev_fork, s));
  AFI_CUDA(cudaStreamWaitEvent(*aux, (cudaEvent_t)c->ev_fork, 0));
  return AFI_OK;
}

static afi_status join_aux(afi_ctx *c, cudaStream_t s, cudaStream_t aux) {
  AFI_CUDA(cudaEventRecord((cudaEvent_t)c->ev_join, aux));
  AFI_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)c->ev_join, 0));
  return AFI_OK;
}

// The multiplier branch of the preconditioner (whose Schur block solves on
// the interior tensors) may run beside the primal one (FD on the full
// tensors) unless both local solves would use the local-solver scratch slab.
static bool precond_branches_independent(afi_ctx *c) {
  return c->exact || !(fd_uses_scratch(c, 0) && fd_uses_scratch(c, 1));
}

afi_status op_precond(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  // calB^{-1} = blkdiag(P_u P_A^{-1} P_u^T, P_chi P_S P_chi^T), eq. (4.9); the
  // two diagonal blocks are independent
  const long n = c->n_dof;
  double *t1 = c->ws + 3 * n + c->n_c, *m2 = c->ws + 4 * n + c->n_c;
  cudaStream_t a = s;
  const bool two = c->n_c > 0 && precond_branches_independent(c);
  if (two) AFI_TRY(fork_aux(c, s, &a));
  if (c->n_c > 0) {
    AFI_TRY(op_Pchi(c, x + n, m2, a));
    AFI_TRY(op_PS(c, m2, y + n, a));
    AFI_TRY(op_Pchi(c, y + n, y + n, a));
  }
  AFI_TRY(op_Pu(c, x, t1, s));
  if (c->exact) AFI_TRY(exact_PA_inv(c, t1, y, s));
  else AFI_TRY(fd_run(c, 0, t1, y, s));
  AFI_TRY(op_Pu(c, y, y, s));
  if (two) AFI_TRY(join_aux(c, s, a));
  return AFI_OK;
}

afi_status op_saddle(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  // [A w + B^T P_chi chi ; P_chi B w], eq. (4.7); the multiplier products
  // run beside the stiffness matvec
  const long n = c->n_dof;
  double *m2 = c->ws + 4 * n + 2 * c->n_c, *m3 = m2 + c->n_c;
  cudaStream_t a = s;
  if (c->n_c > 0) {
    AFI_TRY(fork_aux(c, s, &a));
    AFI_TRY(op_Pchi(c, x + n, m2, a));
    AFI_TRY(op_B(c, x, m3, a));
    AFI_TRY(op_Pchi(c, m3, y + n, a));
  }
  AFI_TRY(op_stiffness(c, x, y, s));
  if (c->n_c > 0) {
    AFI_TRY(join_aux(c, s, a));
    AFI_TRY(op_Bt(c, m2, y, true, false, s));
  }
  return AFI_OK;
}

// -------------------------------------------------------------- MINRES
// Scalars of the recurrences live on the device (c->small); every kernel of
// one iteration reads S_ACTIVE, set by k_iter_begin, so that iterations after
// convergence (inside a replayed graph) leave the state untouched.
enum { S_BETA1 = 0, S_BETA, S_OLDB, S_ALFA, S_DBAR, S_EPSLN, S_OLDEPS, S_PHIBAR, S_CS, S_SN,
       S_DELTA, S_GAMMA, S_PHI, S_REL, S_BETA2, S_FLAG, S_DOT, S_BNORM2, S_RES2, S_INVBETA,
       S_BOVERO, S_INVGAMMA, S_ACTIVE, S_ITN, S_NEXTCHECK, S_MAXIT, S_TOL, S_COUNT };

constexpr int kRelHist = 64;   // st[64 + itn % 8]: estimate of the last 8 iterations
constexpr int kHostStats = kRelHist + 8;

__global__ void k_minres_init(double *st, double maxit, double tol) {
  for (int i = 0; i < 8; ++i) st[kRelHist + i] = 1.0;
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
  st[S_INVBETA] = (beta1 > 0.0) ? 1.0 / beta1 : 0.0;
  st[S_BOVERO] = 0.0;   // the first iteration has no r1 term
  st[S_ACTIVE] = 0.0;
  st[S_ITN] = 0.0;
  st[S_NEXTCHECK] = 0.0;
  st[S_MAXIT] = maxit;
  st[S_TOL] = tol;
  st[S_FLAG] = (beta1 < 0.0) ? 2.0 : (beta1 == 0.0 ? 1.0 : 0.0);
}

__global__ void k_iter_begin(double *st) {
  const bool act = st[S_FLAG] == 0.0 && st[S_ITN] < st[S_MAXIT];
  st[S_ACTIVE] = act ? 1.0 : 0.0;
  if (act) st[S_ITN] += 1.0;
}

__global__ void k_set(double *st, int idx, double v) { st[idx] = v; }

// v = y / beta_1 before the first iteration
__global__ void k_v_from_y(const double *y, double *v, long n, const double *st) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  v[i] = y[i] * st[S_INVBETA];
}

// Block partial of a grid-wide sum; the last block to finish (ticket on
// *counter) adds the gridDim.x partials in block order, writes *dst and resets
// the counter.  Deterministic: the order of the final sum does not depend on
// which block finishes last.
__device__ __forceinline__ void grid_sum_last(double s, double *part, unsigned *counter, double *dst) {
  __shared__ double sh[256];
  __shared__ bool last;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sh[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) t += __ldcg(part + i);
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) { *dst = sh[0]; *counter = 0u; }
}

// y = A v - (beta/oldb) r1 (A v given in av), partial dots of v.y
__global__ void k_y_upd1(const double *av, double *y, const double *r1, const double *v, long n,
                         double *st, double *part, unsigned *counter) {
  if (st[S_ACTIVE] == 0.0) return;
  const double coef = st[S_BOVERO];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double yi = av[i] - coef * r1[i];
    y[i] = yi;
    s += v[i] * yi;
  }
  grid_sum_last(s, part, counter, st + S_ALFA);   // alfa = v . y
}

__global__ void k_y_upd2(double *y, const double *r2, long n, const double *st) {
  if (st[S_ACTIVE] == 0.0) return;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] -= (st[S_ALFA] * st[S_INVBETA]) * r2[i];
}

// beta2 = r2 . y with y = M^{-1} r2 already in place
__global__ void k_dot_active(const double *r2, const double *y, long n, double *st, double *part,
                             unsigned *counter) {
  if (st[S_ACTIVE] == 0.0) return;
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += r2[i] * y[i];
  grid_sum_last(s, part, counter, st + S_BETA2);
}

__global__ void k_minres_scalars(double *st) {
  if (st[S_ACTIVE] == 0.0) return;
  const double tol = st[S_TOL];
  double beta2 = st[S_BETA2];
  if (!(beta2 >= 0.0) || !isfinite(beta2)) { st[S_FLAG] = 2.0; return; }
  double beta = st[S_BETA], alfa = st[S_ALFA];
  double cs = st[S_CS], sn = st[S_SN], dbar = st[S_DBAR], phibar = st[S_PHIBAR];
  st[S_OLDB] = beta;
  const double oldb = beta;
  beta = sqrt(beta2);
  st[S_BETA] = beta;
  st[S_INVBETA] = 1.0 / beta;
  st[S_BOVERO] = beta / oldb;
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
  st[S_INVGAMMA] = 1.0 / gamma;
  st[S_CS] = cs;
  st[S_SN] = sn;
  st[S_PHI] = phi;
  st[S_PHIBAR] = phibar;
  double rel = phibar / st[S_BETA1];
  st[S_REL] = rel;
  st[kRelHist + ((long)st[S_ITN] % 8)] = rel;
  if (!isfinite(rel)) st[S_FLAG] = 2.0;
  else if (rel <= tol && st[S_ITN] >= st[S_NEXTCHECK]) st[S_FLAG] = 1.0;
}

// w = (v - oldeps w1 - delta w2) / gamma, x += phi w, and the next Lanczos
// vector v = y_next / beta_next (S_INVBETA already holds 1 / beta_next)
__global__ void k_w_upd(double *v, const double *w1, const double *w2, double *wn, double *x,
                        const double *ynext, long n, const double *st) {
  if (st[S_ACTIVE] == 0.0) return;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double w = (v[i] - st[S_OLDEPS] * w1[i] - st[S_DELTA] * w2[i]) * st[S_INVGAMMA];
  wn[i] = w;
  x[i] += st[S_PHI] * w;
  v[i] = ynext[i] * st[S_INVBETA];
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

// Buffers of the iteration: three rotating Krylov vectors B (r1, r2, y), two
// rotating search directions W, and fixed v, x, the operator output tA and
// the iterate x0 kept across an FP64 restart.
struct MinresBufs { double *b, *x, *v, *B[3], *W[2], *tA, *x0, *tmp, *lam0; };

static MinresBufs minres_bufs(afi_ctx *c) {
  const long nt = c->n_dof + c->n_c;
  double *V = c->ws + kOpScratch * nt;
  MinresBufs M;
  M.b = V; M.x = V + nt; M.v = V + 2 * nt;
  M.B[0] = V + 3 * nt; M.B[1] = V + 4 * nt; M.B[2] = V + 5 * nt;
  M.W[0] = V + 6 * nt; M.W[1] = V + 7 * nt;
  M.tA = V + 8 * nt; M.x0 = V + 9 * nt; M.tmp = V + 10 * nt; M.lam0 = V + 11 * nt;
  return M;
}

// Enqueue one MINRES iteration after t completed ones (roles rotate with t),
// recurrence scalars in st.
static afi_status enqueue_iteration(afi_ctx *c, const MinresBufs &M, double *st, long t,
                                    cudaStream_t s) {
  const long nt = c->n_dof + c->n_c;
  double *r1 = M.B[t % 3], *r2 = M.B[(t + 1) % 3], *y = M.B[(t + 2) % 3];
  double *w1 = M.W[t % 2], *w2 = M.W[(t + 1) % 2];
  unsigned *cnt = reinterpret_cast<unsigned *>(c->small + kCounters);
  launch(k_iter_begin, 1, 1, 0, s, st);
  // the heavy operator kernels skip their work in inactive iterations
  struct GateScope {
    afi_ctx *c;
    GateScope(afi_ctx *cc, const double *g) : c(cc) { c->gate = g; }
    ~GateScope() { c->gate = nullptr; }
  } gate_scope(c, st + S_ACTIVE);
  AFI_TRY(op_saddle(c, M.v, M.tA, s));
  launch(k_y_upd1, kDotBlocks, 256, 0, s, (const double *)M.tA, y, (const double *)r1,
         (const double *)M.v, nt, st, c->small + kPart, cnt);
  launch(k_y_upd2, nblk(nt), 256, 0, s, y, (const double *)r2, nt, (const double *)st);
  // roles now: r1' = r2, r2' = y, y' = r1 (r1 is free: the preconditioner
  // writes y' there directly)
  AFI_TRY(op_precond(c, y, r1, s));
  launch(k_dot_active, kDotBlocks, 256, 0, s, (const double *)y, (const double *)r1, nt, st,
         c->small + kPart, cnt + 1);
  launch(k_minres_scalars, 1, 1, 0, s, st);
  launch(k_w_upd, nblk(nt), 256, 0, s, M.v, (const double *)w1, (const double *)w2, w1, M.x,
         (const double *)r1, nt, (const double *)st);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

constexpr int kGraphIters = 6;   // lcm of the rotation periods 3 and 2

// Capture kGraphIters iterations on the context's private stream (the caller's
// stream may be the legacy default stream, which cannot be captured); the
// graph is then launched on the caller's stream.
static afi_status ensure_graph(afi_ctx *c, const MinresBufs &M) {
  if (c->graph_exec && c->graph_prec == (int)c->opt.prec) return AFI_OK;
  cudaStream_t s = (cudaStream_t)c->cap_stream;
  if (c->graph_exec) { cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec); c->graph_exec = nullptr; }
  cudaGraph_t g = nullptr;
  const long long before = g_launches.load();
  AFI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  afi_status st = AFI_OK;
  for (int i = 0; i < kGraphIters && st == AFI_OK; ++i) st = enqueue_iteration(c, M, c->small, i, s);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  g_launches.fetch_sub(g_launches.load() - before);
  if (st != AFI_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) { set_error(std::string("graph capture: ") + cudaGetErrorString(e)); return AFI_ECUDA; }
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { set_error(std::string("graph instantiate: ") + cudaGetErrorString(e)); return AFI_ECUDA; }
  c->graph_exec = ex;
  c->graph_nodes = (long long)nodes;
  c->graph_prec = (int)c->opt.prec;
  return AFI_OK;
}

// The stiffness runs with FP64 products inside this scope (the true
// residual), whatever stencil form the iterations use.
struct ExactStiffness {
  afi_ctx *c;
  bool old;
  explicit ExactStiffness(afi_ctx *cc) : c(cc), old(cc->mv_exact) { c->mv_exact = true; }
  ~ExactStiffness() { c->mv_exact = old; }
};

// ||b - calA x||^2 with the FP64 stiffness into st[S_RES2]; hs refreshed
static afi_status true_residual2(afi_ctx *c, const MinresBufs &M, double *st, double *hs,
                                 cudaStream_t s) {
  const long nt = c->n_dof + c->n_c;
  {
    ExactStiffness ex(c);
    AFI_TRY(op_saddle(c, M.x, M.tmp, s));
  }
  launch(k_sub, nblk(nt), 256, 0, s, (const double *)M.b, (const double *)M.tmp, M.tmp, nt);
  AFI_TRY(dot(c, M.tmp, M.tmp, nt, st + S_RES2, s));
  AFI_CUDA(cudaMemcpyAsync(hs, st, kHostStats * sizeof(double), cudaMemcpyDeviceToHost, s));
  AFI_CUDA(cudaStreamSynchronize(s));
  return AFI_OK;
}

// MINRES from x = 0 on the right-hand side in M.b: r1 = r2 = b,
// y = M^{-1} b, beta_1, ||b||^2, the recurrence scalars (estimate tolerance
// tol_est, iteration cap maxit) and v = y / beta_1; hs refreshed
static afi_status minres_start(afi_ctx *c, const MinresBufs &M, double *st, double tol_est,
                               long maxit, double *hs, cudaStream_t s) {
  const long nt = c->n_dof + c->n_c;
  AFI_CUDA(cudaMemsetAsync(M.x, 0, nt * sizeof(double), s));
  AFI_CUDA(cudaMemsetAsync(M.W[0], 0, nt * sizeof(double), s));
  AFI_CUDA(cudaMemsetAsync(M.W[1], 0, nt * sizeof(double), s));
  AFI_CUDA(cudaMemcpyAsync(M.B[0], M.b, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AFI_CUDA(cudaMemcpyAsync(M.B[1], M.b, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AFI_TRY(op_precond(c, M.B[0], M.B[2], s));
  AFI_TRY(dot(c, M.B[0], M.B[2], nt, st + S_BETA2, s));
  AFI_TRY(dot(c, M.b, M.b, nt, st + S_BNORM2, s));
  launch(k_minres_init, 1, 1, 0, s, st, (double)maxit, tol_est);
  launch(k_v_from_y, nblk(nt), 256, 0, s, (const double *)M.B[2], M.v, nt, (const double *)st);
  AFI_LAUNCH_CHECK();
  AFI_CUDA(cudaMemcpyAsync(hs, st, kHostStats * sizeof(double), cudaMemcpyDeviceToHost, s));
  AFI_CUDA(cudaStreamSynchronize(s));
  return AFI_OK;
}

struct LoopResult {
  afi_status status = AFI_OK;
  bool converged = false;
  bool stalled = false;     // the true residual stopped falling (stiffness rounding floor)
  double relres_true = 0.0;
  long checked_at = -1;     // iteration of the last true-residual check
};

// Iterate until the estimate and the FP64 true residual (relative to bnorm)
// both reach tol.  With stop_on_stall, return as soon as a failed check
// shows the true residual nearly flat since the previous failed check while
// the estimate kept falling: the iteration's stiffness rounding then sets a
// floor, and the caller restarts with the FP64 stiffness.  force_stall
// treats the first check as such a stall.
static LoopResult minres_loop(afi_ctx *c, const MinresBufs &M, double *st, bool use_graph,
                              double bnorm, bool stop_on_stall, bool force_stall, double *hs,
                              cudaStream_t s) {
  LoopResult R;
  const double tol = c->opt.tol;
  long t = 0;   // completed iterations (buffer roles)
  double last_fail = 0.0, last_est = 0.0;   // true residual and estimate at the last failed check
  auto fail = [&](afi_status e) { R.status = e; return R; };
  if (hs[S_FLAG] == 2.0) return fail(AFI_EBREAKDOWN);
  if (hs[S_FLAG] != 0.0) { R.converged = true; }   // b = 0
  while (!R.converged) {
    afi_status e = AFI_OK;
    if (use_graph && t % kGraphIters == 0) {
      if (cudaGraphLaunch((cudaGraphExec_t)c->graph_exec, s) != cudaSuccess) return fail(AFI_ECUDA);
      g_launches.fetch_add(c->graph_nodes);
      t += kGraphIters;
    } else {
      e = enqueue_iteration(c, M, st, t, s);
      if (e != AFI_OK) return fail(e);
      t += 1;
    }
    if (cudaMemcpyAsync(hs, st, kHostStats * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(AFI_ECUDA);
    const long itn = (long)hs[S_ITN];
    if (hs[S_FLAG] == 2.0) return fail(AFI_EBREAKDOWN);
    if (hs[S_FLAG] == 1.0) {
      // estimate converged at iteration itn: confirm with the true residual
      e = true_residual2(c, M, st, hs, s);
      if (e != AFI_OK) return fail(e);
      R.relres_true = sqrt(hs[S_RES2]) / (bnorm > 0 ? bnorm : 1.0);
      R.checked_at = itn;
      if (force_stall) { R.stalled = true; break; }
      if (R.relres_true <= tol) { R.converged = true; break; }
      // stall: since the previous failed check the estimate has fallen by
      // more than 4x while the true residual fell by less than 1.5x
      const double est = hs[S_REL];
      if (stop_on_stall && last_fail > 0.0 && est < 0.25 * last_est && R.relres_true > last_fail / 1.5) {
        R.stalled = true;
        break;
      }
      last_fail = R.relres_true;
      last_est = est;
      // continue from iteration itn; next check where the estimate's recent
      // reduction rate would bring the true residual to tol (5..50 later)
      long extra = 5;
      if (itn >= 5) {
        const double rn = hs[kRelHist + itn % 8], r5 = hs[kRelHist + (itn - 5) % 8];
        if (rn > 0.0 && r5 > 0.0) {
          const double q = pow(rn / r5, 0.2);
          if (q > 0.0 && q < 1.0) extra = (long)ceil(log(R.relres_true / tol) / (-log(q)));
        }
      }
      extra = std::min(std::max(extra, 5L), 50L);
      launch(k_set, 1, 1, 0, s, st, (int)S_NEXTCHECK, (double)(itn + extra));
      launch(k_set, 1, 1, 0, s, st, (int)S_FLAG, 0.0);
      if (cudaGetLastError() != cudaSuccess) return fail(AFI_ECUDA);
    }
    t = itn;   // the data state corresponds to the executed iterations
    if (itn >= (long)hs[S_MAXIT]) { R.status = AFI_ENOT_CONVERGED; break; }
  }
  if (R.checked_at != (long)hs[S_ITN]) {   // true residual of the final iterate
    afi_status e = true_residual2(c, M, st, hs, s);
    if (e != AFI_OK) return fail(e);
    R.relres_true = sqrt(hs[S_RES2]) / (bnorm > 0 ? bnorm : 1.0);
  }
  return R;
}

// lambda_0 = G (G^T G)^{-1} R^T f into M.lam0 and b = [f - B^T lambda_0; 0]
// into M.b (Section 4)
static afi_status rhs_setup(afi_ctx *c, const MinresBufs &M, const double *f, cudaStream_t s) {
  const long n = c->n_dof, m = c->n_c;
  if (m > 0) {
    AFI_TRY(op_Rt(c, f, gbuf(c, 0), s));
    AFI_TRY(op_dense_inv(c, gbuf(c, 0), gbuf(c, 1), s));
    AFI_TRY(G_apply(c, gbuf(c, 1), M.lam0, nullptr, s));
  }
  AFI_CUDA(cudaMemcpyAsync(M.b, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (m > 0) {
    AFI_TRY(op_Bt_scaled(c, M.lam0, M.b, -1.0, true, false, s));
    AFI_CUDA(cudaMemsetAsync(M.b + n, 0, m * sizeof(double), s));
  }
  return AFI_OK;
}

// recovery: u = w - R (G^T G)^{-1} G^T B w, lambda = lambda_0 + chi
static afi_status recover(afi_ctx *c, const MinresBufs &M, double *u, double *lam_out,
                          cudaStream_t s) {
  const long n = c->n_dof, m = c->n_c;
  AFI_CUDA(cudaMemcpyAsync(u, M.x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (m > 0) {
    AFI_TRY(op_B(c, M.x, M.tmp, s));
    AFI_TRY(op_Gt_rows(c, M.tmp, gbuf(c, 0), s));
    AFI_TRY(op_dense_inv(c, gbuf(c, 0), gbuf(c, 1), s));
    AFI_TRY(op_R_sub(c, gbuf(c, 1), u, s));
    if (lam_out) {
      launch(k_add, nblk(m), 256, 0, s, (const double *)M.lam0, (const double *)(M.x + n), lam_out, m);
      AFI_LAUNCH_CHECK();
    }
  }
  return AFI_OK;
}

// FP64 restart from the iterate in M.x, whose residual b - calA x is in
// M.tmp (reading 19 of the stopping rule): solve calA d = b - calA x with the
// FP64 stiffness (host-launched iterations, scalars in c->small), then
// x = x + d.  R is replaced by the restarted run's result; its iterations
// are added to *iters.
static afi_status fp64_restart(afi_ctx *c, const MinresBufs &M, double bnorm, LoopResult &R,
                               long *iters, cudaStream_t s) {
  const long nt = c->n_dof + c->n_c;
  double *hs = c->host_small;
  AFI_CUDA(cudaMemcpyAsync(M.x0, M.x, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AFI_CUDA(cudaMemcpyAsync(M.b, M.tmp, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  c->mv_exact = true;
  const double rnorm = R.relres_true * bnorm;
  afi_status e = minres_start(c, M, c->small, c->opt.tol * bnorm / (rnorm > 0 ? rnorm : 1.0),
                              std::max(1L, (long)c->opt.maxit - *iters), hs, s);
  if (e == AFI_OK) {
    R = minres_loop(c, M, c->small, false, bnorm, false, false, hs, s);
    *iters += (long)hs[S_ITN];
  } else {
    R.status = e;
  }
  c->mv_exact = false;
  launch(k_add, nblk(nt), 256, 0, s, (const double *)M.x0, (const double *)M.x, M.x, nt);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// Iterative refinement of the matrix-free FP32 form (AFI_VARIANT_MATRIX_FREE
// without AFI_VARIANT_STENCIL_F64): each MINRES run on b' = b - calA x (FP32
// products) stops once its estimate has fallen by kRefineDrop or reached
// the tolerance, takes one FP64 true residual, and the next run solves for
// the correction from x; at most kRefineMax runs after the first.
constexpr double kRefineDrop = 1e-4;
constexpr int kRefineMax = 12;

static bool refines(const afi_ctx *c) {
  return c->mf && !(c->opt.variant & AFI_VARIANT_STENCIL_F64);
}

// one refinement run from the iterate in M.x, whose residual b - calA x is
// in M.tmp: x0 = x, solve calA d = b - calA x0, x = x0 + d; R is replaced by
// the run's result and its iterations are added to *iters
static afi_status refine_restart(afi_ctx *c, const MinresBufs &M, double bnorm, bool use_graph,
                                 LoopResult &R, long *iters, cudaStream_t s) {
  const long nt = c->n_dof + c->n_c;
  double *hs = c->host_small;
  AFI_CUDA(cudaMemcpyAsync(M.x0, M.x, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AFI_CUDA(cudaMemcpyAsync(M.b, M.tmp, nt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const double rnorm = R.relres_true * bnorm;
  const double tol_est = std::max(c->opt.tol * bnorm / (rnorm > 0 ? rnorm : 1.0), kRefineDrop);
  afi_status e = minres_start(c, M, c->small, tol_est, std::max(1L, (long)c->opt.maxit - *iters), hs, s);
  if (e == AFI_OK) {
    R = minres_loop(c, M, c->small, use_graph, bnorm, true, true, hs, s);
    *iters += (long)hs[S_ITN];
  } else {
    R.status = e;
  }
  launch(k_add, nblk(nt), 256, 0, s, (const double *)M.x0, (const double *)M.x, M.x, nt);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// one right-hand side
afi_status solve_one(afi_ctx *c, const double *f, double *u, double *lam_out, afi_info *info,
                     cudaStream_t s) {
  const MinresBufs M = minres_bufs(c);
  cudaEvent_t e0, e1;
  AFI_CUDA(cudaEventCreate(&e0));
  AFI_CUDA(cudaEventCreate(&e1));
  AFI_CUDA(cudaEventRecord(e0, s));
  c->mv_exact = false;
  AFI_TRY(rhs_setup(c, M, f, s));
  double *hs = c->host_small;
  const double tol = c->opt.tol;
  const bool refine = refines(c);
  AFI_TRY(minres_start(c, M, c->small, refine ? std::max(tol, kRefineDrop) : tol, c->opt.maxit, hs, s));
  const double bnorm = sqrt(hs[S_BNORM2]);
  const bool use_graph = c->opt.use_graph != 0;
  if (use_graph) {
    AFI_TRY(fd_tc_ready(c));   // no allocation or host copy during capture
    AFI_TRY(ensure_graph(c, M));
  }
  const bool pairs = stiffness_has_pairs(c);
  LoopResult R = minres_loop(c, M, c->small, use_graph, bnorm, pairs || refine,
                             refine || (pairs && (c->opt.variant & AFI_VARIANT_FORCE_RESTART)), hs, s);
  long iters = (long)hs[S_ITN];
  int restarts = 0;
  if (refine) {
    while (R.status == AFI_OK && R.stalled && R.relres_true > tol && restarts < kRefineMax &&
           iters < (long)c->opt.maxit) {
      AFI_TRY(refine_restart(c, M, bnorm, use_graph, R, &iters, s));
      ++restarts;
    }
    if (R.status == AFI_OK && R.relres_true > tol) R.status = AFI_ENOT_CONVERGED;
  } else if (R.status == AFI_OK && R.stalled) {
    AFI_TRY(fp64_restart(c, M, bnorm, R, &iters, s));
    restarts = 1;
  }
  afi_status status = R.status;
  AFI_TRY(recover(c, M, u, lam_out, s));
  AFI_CUDA(cudaEventRecord(e1, s));
  AFI_CUDA(cudaEventSynchronize(e1));
  int tc_timeout = 0;   // set by a tensor-core or bulk-copy kernel whose bounded wait ran out
  AFI_CUDA(cudaMemcpy(&tc_timeout, c->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (tc_timeout && status == AFI_OK) status = AFI_ETIMEOUT;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iters = (int)iters;
    info->relres_est = hs[S_REL];
    info->relres_true = R.relres_true;
    info->t_setup_ms = c->t_setup_ms;
    info->t_fd_setup_ms = c->t_fd_setup_ms;
    info->t_solve_ms = ms;
    info->fp64_restarts = restarts;
  }
  if (status == AFI_EBREAKDOWN) set_error("MINRES breakdown (non-finite or negative norm)");
  if (status == AFI_ENOT_CONVERGED) set_error("MINRES reached maxit before the tolerance");
  if (status == AFI_ETIMEOUT) set_error("a tensor-core or bulk-copy kernel timed out on a bounded wait");
  return status;
}


// ------------------------------------------- several right-hand sides
// ieti_solve with nrhs > 1 runs up to kMaxRhs MINRES recurrences in
// lockstep: each right-hand side has its own vectors (c->mws) and scalars
// (c->mst), and every iteration applies the stiffness to all of their
// Lanczos vectors in one batched launch (op_stiffness_multi: the stencil is
// streamed once for all of them); the rest of each iteration (multiplier
// products, preconditioner, dots, updates) runs per right-hand side, gated
// by that right-hand side's own active flag.  The buffer roles rotate with
// the common iteration count t; a right-hand side that paused for a
// true-residual check and then continues has its rotating buffers moved to
// the roles of t (k_rotate_roles), so one captured graph serves all of them;
// the host keeps, per right-hand side, the offset between the common index
// its buffers are arranged for and its own iteration count.
static MinresBufs multi_bufs(afi_ctx *c, int j) {
  const long nt = c->n_dof + c->n_c;
  double *V = c->mws + (long long)j * kKrylov * nt;
  MinresBufs M;
  M.b = V; M.x = V + nt; M.v = V + 2 * nt;
  M.B[0] = V + 3 * nt; M.B[1] = V + 4 * nt; M.B[2] = V + 5 * nt;
  M.W[0] = V + 6 * nt; M.W[1] = V + 7 * nt;
  M.tA = V + 8 * nt; M.x0 = V + 9 * nt; M.tmp = V + 10 * nt; M.lam0 = V + 11 * nt;
  return M;
}

static double *multi_st(afi_ctx *c, int j) { return c->mst + (long long)j * kStStride; }
static double *multi_any(afi_ctx *c) { return c->mst + (long long)kMaxRhs * kStStride; }

// any[0] = 1 if some right-hand side is active in this iteration
__global__ void k_any_active(const double *mst, int nr, double *any) {
  if (threadIdx.x != 0) return;
  double a = 0.0;
  for (int j = 0; j < nr; ++j) a = fmax(a, mst[(long long)j * kStStride + S_ACTIVE]);
  *any = a;
}

// new B[k] = old B[(k - d3) mod 3], new W[k] = old W[(k - d2) mod 2]
__global__ void k_rotate_roles(double *B0, double *B1, double *B2, double *W0, double *W1, long n,
                               int d3, int d2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double b[3] = {B0[i], B1[i], B2[i]}, w[2] = {W0[i], W1[i]};
    B0[i] = b[(3 - d3) % 3];
    B1[i] = b[(4 - d3) % 3];
    B2[i] = b[(5 - d3) % 3];
    W0[i] = w[(2 - d2) % 2];
    W1[i] = w[(3 - d2) % 2];
  }
}

// [A w + B^T P_chi chi ; P_chi B w] given A w already in y (eq. 4.7)
static afi_status saddle_multipliers(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  const long n = c->n_dof;
  if (c->n_c == 0) return AFI_OK;
  double *m2 = c->ws + 4 * n + 2 * c->n_c, *m3 = m2 + c->n_c;
  AFI_TRY(op_Pchi(c, x + n, m2, s));
  AFI_TRY(op_B(c, x, m3, s));
  AFI_TRY(op_Pchi(c, m3, y + n, s));
  AFI_TRY(op_Bt(c, m2, y, true, false, s));
  return AFI_OK;
}

// one lockstep iteration of nr recurrences after t completed ones
static afi_status enqueue_iteration_multi(afi_ctx *c, int nr, long t, cudaStream_t s) {
  const long nt = c->n_dof + c->n_c;
  unsigned *cnt = reinterpret_cast<unsigned *>(c->small + kCounters);
  struct GateScope {
    afi_ctx *c;
    GateScope(afi_ctx *cc, const double *g) : c(cc) { c->gate = g; }
    ~GateScope() { c->gate = nullptr; }
  };
  for (int j = 0; j < nr; ++j) launch(k_iter_begin, 1, 1, 0, s, multi_st(c, j));
  launch(k_any_active, 1, 32, 0, s, (const double *)c->mst, nr, multi_any(c));
  {
    GateScope g(c, multi_any(c));
    const MinresBufs M0 = multi_bufs(c, 0);
    const long long stride = (long long)kKrylov * nt;
    AFI_TRY(op_stiffness_multi(c, M0.v, stride, M0.tA, stride, nr, s));
  }
  for (int j = 0; j < nr; ++j) {
    const MinresBufs M = multi_bufs(c, j);
    double *st = multi_st(c, j);
    double *r1 = M.B[t % 3], *r2 = M.B[(t + 1) % 3], *y = M.B[(t + 2) % 3];
    double *w1 = M.W[t % 2], *w2 = M.W[(t + 1) % 2];
    GateScope g(c, st + S_ACTIVE);
    AFI_TRY(saddle_multipliers(c, M.v, M.tA, s));
    launch(k_y_upd1, kDotBlocks, 256, 0, s, (const double *)M.tA, y, (const double *)r1,
           (const double *)M.v, nt, st, c->small + kPart, cnt);
    launch(k_y_upd2, nblk(nt), 256, 0, s, y, (const double *)r2, nt, (const double *)st);
    AFI_TRY(op_precond(c, y, r1, s));
    launch(k_dot_active, kDotBlocks, 256, 0, s, (const double *)y, (const double *)r1, nt, st,
           c->small + kPart, cnt + 1);
    launch(k_minres_scalars, 1, 1, 0, s, st);
    launch(k_w_upd, nblk(nt), 256, 0, s, M.v, (const double *)w1, (const double *)w2, w1, M.x,
           (const double *)r1, nt, (const double *)st);
  }
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

static afi_status ensure_multi_graph(afi_ctx *c, int nr) {
  if (c->mgraph_exec && c->mgraph_prec == (int)c->opt.prec && c->mgraph_nr == nr) return AFI_OK;
  cudaStream_t s = (cudaStream_t)c->cap_stream;
  if (c->mgraph_exec) { cudaGraphExecDestroy((cudaGraphExec_t)c->mgraph_exec); c->mgraph_exec = nullptr; }
  cudaGraph_t g = nullptr;
  const long long before = g_launches.load();
  AFI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  afi_status st = AFI_OK;
  for (int i = 0; i < kGraphIters && st == AFI_OK; ++i) st = enqueue_iteration_multi(c, nr, i, s);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  g_launches.fetch_sub(g_launches.load() - before);
  if (st != AFI_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) { set_error(std::string("graph capture: ") + cudaGetErrorString(e)); return AFI_ECUDA; }
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { set_error(std::string("graph instantiate: ") + cudaGetErrorString(e)); return AFI_ECUDA; }
  c->mgraph_exec = ex;
  c->mgraph_nodes = (long long)nodes;
  c->mgraph_prec = (int)c->opt.prec;
  c->mgraph_nr = nr;
  return AFI_OK;
}

static afi_status multi_alloc(afi_ctx *c) {
  const long nt = c->n_dof + c->n_c;
  if (!c->mws) AFI_TRY(dalloc(c, (void **)&c->mws, (size_t)kMaxRhs * kKrylov * nt * sizeof(double)));
  if (!c->mst) {
    AFI_TRY(dalloc(c, (void **)&c->mst, (size_t)(kMaxRhs + 1) * kStStride * sizeof(double)));
    AFI_CUDA(cudaMemset(c->mst, 0, (size_t)(kMaxRhs + 1) * kStStride * sizeof(double)));
  }
  if (!c->host_mst)
    AFI_CUDA(cudaMallocHost((void **)&c->host_mst, (size_t)kMaxRhs * kStStride * sizeof(double)));
  return AFI_OK;
}

// nr (2 .. kMaxRhs) right-hand sides f_j = f + j n_dof in lockstep; u_j and
// lambda_j (optional) likewise.  info: the largest iteration count and true
// residual over the right-hand sides, the number of FP64 restarts.
afi_status solve_multi(afi_ctx *c, const double *f, double *u, double *lam_out, int nr,
                       afi_info *info, cudaStream_t s) {
  const long n = c->n_dof, m = c->n_c;
  if (nr < 2 || nr > kMaxRhs) { set_error("solve_multi: 2 <= nrhs <= 8 per batch"); return AFI_EINVAL; }
  AFI_TRY(multi_alloc(c));
  AFI_TRY(stiffness_multi_prepare(c, s));
  cudaEvent_t e0, e1;
  AFI_CUDA(cudaEventCreate(&e0));
  AFI_CUDA(cudaEventCreate(&e1));
  AFI_CUDA(cudaEventRecord(e0, s));
  c->mv_exact = false;
  const double tol = c->opt.tol;
  const bool pairs = stiffness_has_pairs(c);
  const bool force_stall = pairs && (c->opt.variant & AFI_VARIANT_FORCE_RESTART);
  struct Run {
    LoopResult R;
    double bnorm = 0.0, last_fail = 0.0, last_est = 0.0;
    bool done = false;
    long lag = 0;   // (common index its buffers are arranged for) - (its own iteration count)
  };
  std::vector<Run> run(nr);
  for (int j = 0; j < nr; ++j) {
    const MinresBufs M = multi_bufs(c, j);
    double *hs = c->host_mst + (long long)j * kStStride;
    AFI_TRY(rhs_setup(c, M, f + (long long)j * n, s));
    AFI_TRY(minres_start(c, M, multi_st(c, j), tol, c->opt.maxit, hs, s));
    run[j].bnorm = sqrt(hs[S_BNORM2]);
    if (hs[S_FLAG] == 2.0) { run[j].R.status = AFI_EBREAKDOWN; run[j].done = true; }
    else if (hs[S_FLAG] != 0.0) {   // b = 0
      run[j].R.converged = true;
      run[j].done = true;
      run[j].R.checked_at = 0;
    }
  }
  const bool use_graph = c->opt.use_graph != 0;
  if (use_graph) {
    AFI_TRY(fd_tc_ready(c));
    AFI_TRY(ensure_multi_graph(c, nr));
  }
  long t = 0;
  auto all_done = [&]() {
    for (auto &r : run)
      if (!r.done) return false;
    return true;
  };
  while (!all_done()) {
    if (use_graph && t % kGraphIters == 0) {
      if (cudaGraphLaunch((cudaGraphExec_t)c->mgraph_exec, s) != cudaSuccess) {
        set_error("graph launch failed");
        return AFI_ECUDA;
      }
      g_launches.fetch_add(c->mgraph_nodes);
      t += kGraphIters;
    } else {
      AFI_TRY(enqueue_iteration_multi(c, nr, t, s));
      t += 1;
    }
    AFI_CUDA(cudaMemcpyAsync(c->host_mst, c->mst, (size_t)nr * kStStride * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    AFI_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < nr; ++j) {
      Run &r = run[j];
      if (r.done) continue;
      const MinresBufs M = multi_bufs(c, j);
      double *st = multi_st(c, j), *hs = c->host_mst + (long long)j * kStStride;
      const long itn = (long)hs[S_ITN];
      if (hs[S_FLAG] == 2.0) { r.R.status = AFI_EBREAKDOWN; r.done = true; continue; }
      if (hs[S_FLAG] == 1.0) {
        // estimate converged at iteration itn: confirm with the true residual
        AFI_TRY(true_residual2(c, M, st, hs, s));
        r.R.relres_true = sqrt(hs[S_RES2]) / (r.bnorm > 0 ? r.bnorm : 1.0);
        r.R.checked_at = itn;
        if (force_stall) { r.R.stalled = true; r.done = true; continue; }
        if (r.R.relres_true <= tol) { r.R.converged = true; r.done = true; continue; }
        const double est = hs[S_REL];
        if (pairs && r.last_fail > 0.0 && est < 0.25 * r.last_est &&
            r.R.relres_true > r.last_fail / 1.5) {
          r.R.stalled = true;
          r.done = true;
          continue;
        }
        r.last_fail = r.R.relres_true;
        r.last_est = est;
        long extra = 5;
        if (itn >= 5) {
          const double rn = hs[kRelHist + itn % 8], r5 = hs[kRelHist + (itn - 5) % 8];
          if (rn > 0.0 && r5 > 0.0) {
            const double q = pow(rn / r5, 0.2);
            if (q > 0.0 && q < 1.0) extra = (long)ceil(log(r.R.relres_true / tol) / (-log(q)));
          }
        }
        extra = std::min(std::max(extra, 5L), 50L);
        launch(k_set, 1, 1, 0, s, st, (int)S_NEXTCHECK, (double)(itn + extra));
        launch(k_set, 1, 1, 0, s, st, (int)S_FLAG, 0.0);
        // the data state of this right-hand side is that of itn own
        // iterations, arranged for the common index itn + lag: move its
        // rotating buffers to the roles of the common count t
        const long shift = t - itn - r.lag;
        r.lag = t - itn;
        const int d3 = (int)((shift % 3 + 3) % 3), d2 = (int)((shift % 2 + 2) % 2);
        if (d3 || d2)
          launch(k_rotate_roles, (unsigned)std::min<long>(nblk(n + m), 8L * c->nsm), 256, 0, s,
                 M.B[0], M.B[1], M.B[2], M.W[0], M.W[1], n + m, d3, d2);
        AFI_LAUNCH_CHECK();
      }
      if (itn >= (long)hs[S_MAXIT]) { r.R.status = AFI_ENOT_CONVERGED; r.done = true; }
    }
  }
  // final true residuals, FP64 restarts of stalled right-hand sides, recovery
  int restarts = 0;
  long max_it = 0;
  double max_res = 0.0, max_est = 0.0;
  afi_status status = AFI_OK;
  for (int j = 0; j < nr; ++j) {
    Run &r = run[j];
    const MinresBufs M = multi_bufs(c, j);
    double *st = multi_st(c, j), *hs = c->host_mst + (long long)j * kStStride;
    AFI_CUDA(cudaMemcpyAsync(hs, st, kHostStats * sizeof(double), cudaMemcpyDeviceToHost, s));
    AFI_CUDA(cudaStreamSynchronize(s));
    long iters = (long)hs[S_ITN];
    max_est = std::max(max_est, hs[S_REL]);
    if ((r.R.status == AFI_OK || r.R.status == AFI_ENOT_CONVERGED) && r.R.checked_at != iters) {
      AFI_TRY(true_residual2(c, M, st, hs, s));
      r.R.relres_true = sqrt(hs[S_RES2]) / (r.bnorm > 0 ? r.bnorm : 1.0);
    }
    if (r.R.status == AFI_OK && r.R.stalled) {
      AFI_TRY(fp64_restart(c, M, r.bnorm, r.R, &iters, s));
      ++restarts;
    }
    if (r.R.status != AFI_OK && status == AFI_OK) status = r.R.status;
    AFI_TRY(recover(c, M, u + (long long)j * n, lam_out ? lam_out + (long long)j * m : nullptr, s));
    max_it = std::max(max_it, iters);
    max_res = std::max(max_res, r.R.relres_true);
  }
  AFI_CUDA(cudaEventRecord(e1, s));
  AFI_CUDA(cudaEventSynchronize(e1));
  int tc_timeout = 0;
  AFI_CUDA(cudaMemcpy(&tc_timeout, c->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (tc_timeout && status == AFI_OK) status = AFI_ETIMEOUT;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iters = (int)max_it;
    info->relres_est = max_est;
    info->relres_true = max_res;
    info->t_setup_ms = c->t_setup_ms;
    info->t_fd_setup_ms = c->t_fd_setup_ms;
    info->t_solve_ms = ms;
    info->fp64_restarts = restarts;
  }
  if (status == AFI_EBREAKDOWN) set_error("MINRES breakdown (non-finite or negative norm)");
  if (status == AFI_ENOT_CONVERGED) set_error("MINRES reached maxit before the tolerance");
  if (status == AFI_ETIMEOUT) set_error("a tensor-core or bulk-copy kernel timed out on a bounded wait");
  return status;
}

}  // namespace afi
