// Local solvers of Section 5.2 on every (patch, component) block:
//  * fast diagonalization, Algorithm 1: s = (U3 x U2 x U1) Lambda^{-1}
//    (U3 x U2 x U1)^T r with Lambda_l of eq. (5.9) (P_A^{inex}, eq. 5.6) or
//    Lambda~_l of eq. (5.10) (interior block (A_hat_l)_II);
//  * the parametric Schur complement S_hat_l of eqs. (5.4)-(5.5),
//    S theta = (A_hat v)_Gamma with v_Gamma = theta and
//    v_I = -(A_hat_l)_II^{-1} (A_hat [theta; 0])_I, scaled by H^{d-2} (eq. 5.7),
//    where A_hat_l (Section 5.2) is applied through its Kronecker form with the
//    banded univariate K_hat, M_hat.
// One CTA owns one (patch, component) tensor; the tensor lives in shared
// memory when it fits and in a global scratch slab otherwise.  Arithmetic is
// FP64 (plain form) or FP32 (mixed form), inputs and outputs FP64.
#include "common.cuh"

namespace afi {

template <typename T> struct Pool;
template <> struct Pool<double> { static const double *get(const afi_ctx *c) { return c->dpool; } };
template <> struct Pool<float> { static const float *get(const afi_ctx *c) { return c->fpool; } };

// dst = op(U) applied along direction d.  TRANS: dst[a] = sum_i U[i][a] src[i]
// (forward transform), else dst[i] = sum_a U[i][a] src[a].
template <typename T, bool TRANS>
__device__ __forceinline__ void mode_dense(const T *__restrict__ src, T *__restrict__ dst,
                                           const T *__restrict__ U, int n, int d, int n1, int n2,
                                           int n3) {
  const int tot = n1 * n2 * n3;
  const int stride = (d == 0) ? 1 : (d == 1 ? n1 : n1 * n2);
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int io = (d == 0) ? idx % n1 : (d == 1 ? (idx / n1) % n2 : idx / (n1 * n2));
    const T *base = src + idx - io * stride;
    T acc = 0;
    if (TRANS) {
#pragma unroll 4
      for (int j = 0; j < n; ++j) acc += U[j * n + io] * base[j * stride];
    } else {
      const T *row = U + io * n;
#pragma unroll 4
      for (int j = 0; j < n; ++j) acc += row[j] * base[j * stride];
    }
    dst[idx] = acc;
  }
}

// dst = alpha * Mat1(src1) [+ beta * Mat2(src2)] along direction d, with the
// banded (half-bandwidth p) n x n matrices of the univariate pencil.
template <typename T>
__device__ __forceinline__ void mode_band2(const T *__restrict__ src1, const T *__restrict__ M1,
                                           T alpha, const T *__restrict__ src2,
                                           const T *__restrict__ M2, T beta, T *__restrict__ dst,
                                           int p, int d, int n1, int n2, int n3) {
  const int tot = n1 * n2 * n3;
  const int n = (d == 0) ? n1 : (d == 1 ? n2 : n3);
  const int stride = (d == 0) ? 1 : (d == 1 ? n1 : n1 * n2);
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int io = (d == 0) ? idx % n1 : (d == 1 ? (idx / n1) % n2 : idx / (n1 * n2));
    const int lo = max(io - p, 0), hi = min(io + p, n - 1);
    const long long base = idx - (long long)io * stride;
    T a1 = 0, a2 = 0;
    for (int j = lo; j <= hi; ++j) {
      a1 += M1[io * n + j] * src1[base + (long long)j * stride];
      if (src2) a2 += M2[io * n + j] * src2[base + (long long)j * stride];
    }
    dst[idx] = alpha * a1 + (src2 ? beta * a2 : T(0));
  }
}

struct Dims { int n[3]; int N; };

__device__ __forceinline__ Dims dims_of(const DevPatch &pt, int interior) {
  Dims D;
  for (int d = 0; d < 3; ++d) D.n[d] = interior ? pt.ni[d] : pt.n[d];
  D.N = D.n[0] * D.n[1] * D.n[2];
  return D;
}

// Algorithm 1 on the tensor in `cur` (ping-pong with `oth`).  The final mode
// product goes to `dst` (FP64, contiguous) or, if scatter_full is given, is
// negated and scattered to the interior positions of a full patch tensor
// (the interior solve inside the Schur complement).
template <typename T>
__device__ void fd_tensor(T *cur, T *oth, const DevPatch &pt, const Tab1D *tabs,
                          const double *dpool, const T *upool, int dim, int l, int interior,
                          double *dst, T *scatter_full) {
  const Dims D = dims_of(pt, interior);
  const T *U[3];
  const double *Dv[3];
  for (int d = 0; d < 3; ++d) {
    const Tab1D tb = tabs[pt.tab[d]];
    U[d] = upool + (interior ? tb.Ui : tb.U);
    Dv[d] = dpool + (interior ? tb.Di : tb.D);
  }
  // forward: r~ = (U^T x ... x U^T) r
  for (int d = 0; d < dim; ++d) {
    mode_dense<T, true>(cur, oth, U[d], D.n[d], d, D.n[0], D.n[1], D.n[2]);
    __syncthreads();
    T *t = cur; cur = oth; oth = t;
  }
  // scale by Lambda^{-1}
  const double cl = 2.0 * pt.mu + pt.lam;
  const double c0 = (l == 0) ? cl : pt.mu, c1 = (l == 1) ? cl : pt.mu, c2 = (l == 2) ? cl : pt.mu;
  for (int idx = threadIdx.x; idx < D.N; idx += blockDim.x) {
    const int i1 = idx % D.n[0], i2 = (idx / D.n[0]) % D.n[1], i3 = idx / (D.n[0] * D.n[1]);
    double lam = c0 * Dv[0][i1] + c1 * Dv[1][i2] + (dim == 3 ? c2 * Dv[2][i3] : 0.0);
    if (!interior) lam = pt.Hs * (lam + 1.0);
    cur[idx] = (T)((double)cur[idx] / lam);
  }
  __syncthreads();
  // back: s = (U x ... x U) q~, last direction first
  for (int d = dim - 1; d >= 1; --d) {
    mode_dense<T, false>(cur, oth, U[d], D.n[d], d, D.n[0], D.n[1], D.n[2]);
    __syncthreads();
    T *t = cur; cur = oth; oth = t;
  }
  // direction 1 straight to the destination
  const T *U0 = U[0];
  const int n0 = D.n[0];
  for (int idx = threadIdx.x; idx < D.N; idx += blockDim.x) {
    const int io = idx % n0;
    const T *base = cur + idx - io;
    const T *row = U0 + io * n0;
    T acc = 0;
    for (int j = 0; j < n0; ++j) acc += row[j] * base[j];
    if (scatter_full) {
      const int i2 = (idx / n0) % D.n[1], i3 = idx / (n0 * D.n[1]);
      const int full = (io + 1) + pt.n[0] * ((i2 + 1) + pt.n[1] * (i3 + (dim == 3 ? 1 : 0)));
      scatter_full[full] = -acc;
    } else {
      dst[idx] = (double)acc;
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_fd(const DevPatch *P, const Tab1D *tabs,
                                            const double *dpool, const T *upool, int dim,
                                            int interior, const double *r, double *s,
                                            T *gscratch, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int k = blockIdx.x, l = blockIdx.y;
  const DevPatch pt = P[k];
  const Dims D = dims_of(pt, interior);
  const long long base = (interior ? pt.ioff : pt.off) + (long long)l * D.N;
  T *b0, *b1;
  if (use_smem) {
    b0 = reinterpret_cast<T *>(smraw);
    b1 = b0 + D.N;
  } else {
    b0 = gscratch + 2 * base;
    b1 = b0 + D.N;
  }
  for (int i = threadIdx.x; i < D.N; i += blockDim.x) b0[i] = (T)r[base + i];
  __syncthreads();
  fd_tensor<T>(b0, b1, pt, tabs, dpool, upool, dim, l, interior, s + base, nullptr);
}

// A_hat_l v (Kronecker form) from buffer v into `out`, using two temporaries.
template <typename T>
__device__ void ahat_apply(const T *v, T *out, T *t1, T *t2, const DevPatch &pt,
                           const Tab1D *tabs, const T *upool, int dim, int l) {
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2];
  const Tab1D A0 = tabs[pt.tab[0]], A1 = tabs[pt.tab[1]], A2 = tabs[pt.tab[2]];
  const T cl = (T)(2.0 * pt.mu + pt.lam), mu = (T)pt.mu;
  const T c0 = (l == 0) ? cl : mu, c1 = (l == 1) ? cl : mu, c2 = (l == 2) ? cl : mu;
  const int p = pt.p;
  // t1 = M1 v (dir 0), t2 = K1 v (dir 0): done as one pass each
  mode_band2<T>(v, upool + A0.M, T(1), nullptr, nullptr, T(0), t1, p, 0, n1, n2, n3);
  mode_band2<T>(v, upool + A0.K, T(1), nullptr, nullptr, T(0), t2, p, 0, n1, n2, n3);
  __syncthreads();
  if (dim == 2) {
    // out = c0 M2 (K1 v) + c1 K2 (M1 v)
    mode_band2<T>(t2, upool + A1.M, c0, t1, upool + A1.K, c1, out, p, 1, n1, n2, n3);
    __syncthreads();
    return;
  }
  // out = Ta = c0 M2 t2 + c1 K2 t1  (dir 1)
  mode_band2<T>(t2, upool + A1.M, c0, t1, upool + A1.K, c1, out, p, 1, n1, n2, n3);
  __syncthreads();
  // t2 = Tb = M2 t1 (dir 1)
  mode_band2<T>(t1, upool + A1.M, T(1), nullptr, nullptr, T(0), t2, p, 1, n1, n2, n3);
  __syncthreads();
  // t1 = M3 Ta + c2 K3 Tb (dir 2)
  mode_band2<T>(out, upool + A2.M, T(1), t2, upool + A2.K, c2, t1, p, 2, n1, n2, n3);
  __syncthreads();
  for (int i = threadIdx.x; i < n1 * n2 * n3; i += blockDim.x) out[i] = t1[i];
  __syncthreads();
}

__device__ __forceinline__ bool on_shell(int idx, const DevPatch &pt, int dim) {
  const int i1 = idx % pt.n[0], i2 = (idx / pt.n[0]) % pt.n[1], i3 = idx / (pt.n[0] * pt.n[1]);
  bool s = (i1 == 0 || i1 == pt.n[0] - 1 || i2 == 0 || i2 == pt.n[1] - 1);
  if (dim == 3) s = s || (i3 == 0 || i3 == pt.n[2] - 1);
  return s;
}

// y = H^{d-2} S_hat_l theta for every (patch, component); t, y torn vectors,
// only shell entries of t are read, interior entries of y are zero.
template <typename T>
__global__ void __launch_bounds__(256) k_schur(const DevPatch *P, const Tab1D *tabs,
                                               const double *dpool, const T *upool, int dim,
                                               const double *t, double *y, T *gscratch,
                                               int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int k = blockIdx.x, l = blockIdx.y;
  const DevPatch pt = P[k];
  const int N = pt.N;
  const long long base = pt.off + (long long)l * N;
  T *B0;
  if (use_smem) B0 = reinterpret_cast<T *>(smraw);
  else B0 = gscratch + 4 * base;
  T *B1 = B0 + N, *B2 = B1 + N, *B3 = B2 + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    B0[i] = on_shell(i, pt, dim) ? (T)t[base + i] : T(0);
  __syncthreads();
  // first product: out = A_hat [theta; 0]
  T *out = B1;
  ahat_apply<T>(B0, out, B2, B3, pt, tabs, upool, dim, l);
  // interior solve v_I = -(A_hat)_II^{-1} out_I, compact in B2/B3
  Dims Di = dims_of(pt, 1);
  for (int idx = threadIdx.x; idx < Di.N; idx += blockDim.x) {
    const int j1 = idx % Di.n[0], j2 = (idx / Di.n[0]) % Di.n[1], j3 = idx / (Di.n[0] * Di.n[1]);
    const int full = (j1 + 1) + pt.n[0] * ((j2 + 1) + pt.n[1] * (j3 + (dim == 3 ? 1 : 0)));
    B2[idx] = out[full];
  }
  __syncthreads();
  fd_tensor<T>(B2, B3, pt, tabs, dpool, upool, dim, l, 1, nullptr, B0);
  // second product on [theta; v_I]
  ahat_apply<T>(B0, out, B2, B3, pt, tabs, upool, dim, l);
  const double hs = pt.Hs;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    y[base + i] = on_shell(i, pt, dim) ? hs * (double)out[i] : 0.0;
}

static int smem_limit() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

template <typename T>
static afi_status fd_launch(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st) {
  int maxN = 1;
  for (auto &p : c->hp) maxN = std::max(maxN, interior ? p.Ni : p.N);
  size_t smem = 2ull * maxN * sizeof(T);
  int use_smem = smem <= (size_t)smem_limit();
  if (use_smem) AFI_CUDA(cudaFuncSetAttribute(k_fd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  else smem = 0;
  launch(k_fd<T>, dim3(c->npatch, c->dim), 256, smem, st, c->patches, c->tabs, c->dpool, Pool<T>::get(c),
                                                     c->dim, interior, r, s,
                                                     reinterpret_cast<T *>(c->fdscratch), use_smem);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

template <typename T>
static afi_status schur_launch(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  size_t smem = 4ull * c->max_N * sizeof(T);
  int use_smem = smem <= (size_t)smem_limit();
  if (use_smem) AFI_CUDA(cudaFuncSetAttribute(k_schur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  else smem = 0;
  launch(k_schur<T>, dim3(c->npatch, c->dim), 256, smem, st, c->patches, c->tabs, c->dpool, Pool<T>::get(c),
                                                         c->dim, t, y,
                                                         reinterpret_cast<T *>(c->fdscratch), use_smem);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status fd_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st) {
  switch (c->opt.prec) {
    case AFI_FD_FP64: return fd_launch<double>(c, interior, r, s, st);
    case AFI_FD_FP32: return fd_launch<float>(c, interior, r, s, st);
    default: set_error("local-solver precision not available"); return AFI_EINVAL;
  }
}

afi_status schur_run(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  switch (c->opt.prec) {
    case AFI_FD_FP64: return schur_launch<double>(c, t, y, st);
    case AFI_FD_FP32: return schur_launch<float>(c, t, y, st);
    default: set_error("local-solver precision not available"); return AFI_EINVAL;
  }
}

}  // namespace afi
