// EXACT local solvers (Section 5.1), the iteration-count reference of the
// paper's tables, for small patches:
//   P_A^ex = A^(k) + H_k^{-2} M^(k)  (eq. 5.1 with D_H = H^{-2} I, the scalar
//            mapped mass on every component), applied through its inverse;
//   S^(k)   the Schur complement of A^(k) on the patch interface, applied as
//            S theta = (A v)_Gamma with v_Gamma = theta and
//            v_I = -A_II^{-1} (A v^0)_I, inside P_S^{ex-nr} (Remark 1).
// The dense per-patch matrices are built column by column from the library's
// own FP64 operators (stiffness stencil, quadrature mass), with the unit
// vector of column j placed in every patch at once, and inverted in FP64 by
// Gauss-Jordan.  Only for patches with d N^(k) <= kExactMax.
#include "common.cuh"

#include <algorithm>

namespace afi {

afi_status dense_spd_inverse(afi_ctx *c, double *A, double *Ainv, int n, double *scratch);
afi_status op_stiffness_fp64(afi_ctx *c, const double *x, double *y, cudaStream_t s);

constexpr int kExactMax = 4096;

// position of interior node (a1, a2, a3) of patch pt in its component block of
// the compact interior layout, and the node index in the full layout
__device__ __forceinline__ int interior_node(const DevPatch &pt, int q) {
  const int a1 = q % pt.ni[0], a2 = (q / pt.ni[0]) % pt.ni[1], a3 = q / (pt.ni[0] * pt.ni[1]);
  const int o3 = pt.n[2] > 1 ? 1 : 0;   // 2D: the dummy third direction has no boundary
  return (a1 + 1) + pt.n[0] * ((a2 + 1) + pt.n[1] * (a3 + o3));
}

// x = e_j in the dof block of every patch with j < d N_k
__global__ void k_unit_col(const DevPatch *P, int npatch, int dim, int j, double *x) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npatch) return;
  if (j < dim * P[k].N) x[P[k].off + j] = 1.0;
}

// column j of K_k = A_k + H_k^{-2} M_k from y = A e_j and z = M e_j, and of
// A_II,k when j is an interior dof (rows and columns in the compact interior
// order [component][interior node])
__global__ void k_exact_col(const DevPatch *P, int dim, int j, const double *y, const double *z,
                            const long long *koff, const long long *aoff, double *K, double *AII) {
  const DevPatch pt = P[blockIdx.y];
  const int n = dim * pt.N, ni = dim * pt.Ni;
  if (j >= n) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double h2 = 1.0 / (pt.H * pt.H);
  if (i < n) K[koff[blockIdx.y] + (long long)i * n + j] = y[pt.off + i] + h2 * z[pt.off + i];
  // interior column index of j, if any
  const int cj = j / pt.N, nj = j - cj * pt.N;
  const int j1 = nj % pt.n[0], j2 = (nj / pt.n[0]) % pt.n[1], j3 = nj / (pt.n[0] * pt.n[1]);
  const bool in3 = pt.n[2] == 1 || (j3 > 0 && j3 < pt.n[2] - 1);
  if (!(j1 > 0 && j1 < pt.n[0] - 1 && j2 > 0 && j2 < pt.n[1] - 1 && in3)) return;
  const int qj = (j1 - 1) + pt.ni[0] * ((j2 - 1) + pt.ni[1] * (pt.n[2] > 1 ? j3 - 1 : 0));
  const int cidx = cj * pt.Ni + qj;
  if (i < ni) {
    const int ci = i / pt.Ni, qi = i - ci * pt.Ni;
    AII[aoff[blockIdx.y] + (long long)i * ni + cidx] = y[pt.off + (long long)ci * pt.N + interior_node(pt, qi)];
  }
}

// y_k = M_k x_k for every patch (dense row-major blocks, one warp per row)
__global__ void k_block_mv(const DevPatch *P, int dim, int interior, const long long *moff, const double *M,
                           const double *x, double *y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const DevPatch pt = P[blockIdx.y];
  const int n = dim * (interior ? pt.Ni : pt.N);
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  const long long vo = interior ? pt.ioff : pt.off;
  const double *m = M + moff[blockIdx.y] + (long long)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += m[j] * x[vo + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[vo + row] = s;
}

// compact interior entries of a torn vector: out[ioff + c Ni + q] = x[off + c N + node(q)]
__global__ void k_take_interior(const DevPatch *P, int dim, const double *x, double *out, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const DevPatch pt = P[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim * pt.Ni) return;
  const int c = i / pt.Ni, q = i - c * pt.Ni;
  out[pt.ioff + i] = x[pt.off + (long long)c * pt.N + interior_node(pt, q)];
}

// v (torn, zero in the interior) gets -w on its interior entries
__global__ void k_put_interior(const DevPatch *P, int dim, const double *w, double *v, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const DevPatch pt = P[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim * pt.Ni) return;
  const int c = i / pt.Ni, q = i - c * pt.Ni;
  v[pt.off + (long long)c * pt.N + interior_node(pt, q)] = -w[pt.ioff + i];
}

// y = z on the shell, 0 in the interior
__global__ void k_shell_only(const DevPatch *P, int dim, const double *z, double *y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const DevPatch pt = P[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim * pt.N) return;
  const int node = i % pt.N;
  const int i1 = node % pt.n[0], i2 = (node / pt.n[0]) % pt.n[1], i3 = node / (pt.n[0] * pt.n[1]);
  const bool in3 = pt.n[2] == 1 || (i3 > 0 && i3 < pt.n[2] - 1);
  const bool inner = i1 > 0 && i1 < pt.n[0] - 1 && i2 > 0 && i2 < pt.n[1] - 1 && in3;
  y[pt.off + i] = inner ? 0.0 : z[pt.off + i];
}

afi_status exact_setup(afi_ctx *c) {
  const int D = c->dim, NP = c->npatch;
  if (!c->stencil) { set_error("AFI_VARIANT_EXACT needs the stiffness (not AFI_VARIANT_LOCAL_ONLY)"); return AFI_EINVAL; }
  std::vector<long long> koff(NP), aoff(NP);
  long long kt = 0, at = 0;
  int nmax = 0, nimax = 0;
  for (int k = 0; k < NP; ++k) {
    const int n = D * c->hp[k].N, ni = D * c->hp[k].Ni;
    if (n > kExactMax) { set_error("AFI_VARIANT_EXACT: a patch has more than 4096 dofs"); return AFI_EINVAL; }
    koff[k] = kt; kt += (long long)n * n;
    aoff[k] = at; at += (long long)ni * ni;
    nmax = std::max(nmax, n);
    nimax = std::max(nimax, ni);
  }
  struct Tmp {   // setup temporaries, freed on every return path
    double *p = nullptr;
    ~Tmp() { if (p) cudaFree(p); }
  } tK, tA, tS, tx, ty, tz;
  AFI_TRY(dalloc(c, (void **)&c->ex_Kinv, (size_t)kt * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->ex_AIIinv, (size_t)std::max(1LL, at) * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->ex_koff, NP * sizeof(long long)));
  AFI_TRY(dalloc(c, (void **)&c->ex_aoff, NP * sizeof(long long)));
  AFI_CUDA(cudaMemcpy(c->ex_koff, koff.data(), NP * sizeof(long long), cudaMemcpyHostToDevice));
  AFI_CUDA(cudaMemcpy(c->ex_aoff, aoff.data(), NP * sizeof(long long), cudaMemcpyHostToDevice));
  // temporaries: the matrices before inversion, GJ scratch, column vectors
  AFI_CUDA(cudaMalloc((void **)&tK.p, (size_t)kt * sizeof(double)));
  AFI_CUDA(cudaMalloc((void **)&tA.p, (size_t)std::max(1LL, at) * sizeof(double)));
  AFI_CUDA(cudaMalloc((void **)&tS.p, ((size_t)nmax * nmax + nmax) * sizeof(double)));
  AFI_CUDA(cudaMalloc((void **)&tx.p, (size_t)c->n_dof * sizeof(double)));
  AFI_CUDA(cudaMalloc((void **)&ty.p, (size_t)c->n_dof * sizeof(double)));
  AFI_CUDA(cudaMalloc((void **)&tz.p, (size_t)c->n_dof * sizeof(double)));
  double *K = tK.p, *AII = tA.p, *scratch = tS.p, *x = tx.p, *y = ty.p, *z = tz.p;
  afi_status st = AFI_OK;
  for (int j = 0; j < nmax && st == AFI_OK; ++j) {
    AFI_CUDA(cudaMemsetAsync(x, 0, (size_t)c->n_dof * sizeof(double), 0));
    launch(k_unit_col, (NP + 127) / 128, 128, 0, 0, (const DevPatch *)c->patches, NP, D, j, x);
    st = op_stiffness_fp64(c, x, y, 0);
    if (st == AFI_OK) st = op_load(c, x, z, 0);
    if (st == AFI_OK)
      launch(k_exact_col, dim3((nmax + 127) / 128, NP), 128, 0, 0, (const DevPatch *)c->patches, D, j,
             (const double *)y, (const double *)z, (const long long *)c->ex_koff,
             (const long long *)c->ex_aoff, K, AII);
  }
  AFI_LAUNCH_CHECK();
  for (int k = 0; k < NP && st == AFI_OK; ++k) {
    const int n = D * c->hp[k].N, ni = D * c->hp[k].Ni;
    st = dense_spd_inverse(c, K + koff[k], c->ex_Kinv + koff[k], n, scratch);
    if (st == AFI_OK && ni > 0) st = dense_spd_inverse(c, AII + aoff[k], c->ex_AIIinv + aoff[k], ni, scratch);
  }
  AFI_CUDA(cudaDeviceSynchronize());
  if (st == AFI_ESINGULAR) set_error("AFI_VARIANT_EXACT: a local matrix is not positive definite");
  c->exact = (st == AFI_OK);
  return st;
}

static int max_patch_n(const afi_ctx *c, bool interior) {
  int m = 1;
  for (auto &p : c->hp) m = std::max(m, c->dim * (interior ? p.Ni : p.N));
  return m;
}

// s = (A^(k) + H_k^{-2} M^(k))^{-1} r, every patch
afi_status exact_PA_inv(afi_ctx *c, const double *r, double *s, cudaStream_t st) {
  const int n = max_patch_n(c, false);
  launch(k_block_mv, dim3((n * 32 + 255) / 256, c->npatch), 256, 0, st, (const DevPatch *)c->patches, c->dim, 0,
         (const long long *)c->ex_koff, (const double *)c->ex_Kinv, r, s, (const double *)c->gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// y = blkdiag S^(k) t for t supported on the shell (zero in the interior)
afi_status exact_schur(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  const int D = c->dim;
  double *v = c->ps_buf, *a = c->ps_buf + c->n_dof;
  double *yi = c->ps_rint, *wi = c->ps_vint;
  const int ni = max_patch_n(c, true), n = max_patch_n(c, false);
  const double *gate = c->gate;
  AFI_CUDA(cudaMemcpyAsync(v, t, (size_t)c->n_dof * sizeof(double), cudaMemcpyDeviceToDevice, st));
  AFI_TRY(op_stiffness_fp64(c, v, a, st));
  const dim3 gi((ni + 127) / 128, c->npatch);
  launch(k_take_interior, gi, 128, 0, st, (const DevPatch *)c->patches, D, (const double *)a, yi, gate);
  launch(k_block_mv, dim3((ni * 32 + 255) / 256, c->npatch), 256, 0, st, (const DevPatch *)c->patches, D, 1,
         (const long long *)c->ex_aoff, (const double *)c->ex_AIIinv, (const double *)yi, wi, gate);
  launch(k_put_interior, gi, 128, 0, st, (const DevPatch *)c->patches, D, (const double *)wi, v, gate);
  AFI_TRY(op_stiffness_fp64(c, v, a, st));
  launch(k_shell_only, dim3((n + 127) / 128, c->npatch), 128, 0, st, (const DevPatch *)c->patches, D,
         (const double *)a, y, gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

}  // namespace afi
