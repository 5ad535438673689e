// Fast diagonalization, Algorithm 1, on every (patch, component) block with
// SIMT arithmetic: s = (U3 x U2 x U1) Lambda^{-1} (U3 x U2 x U1)^T r with
// Lambda_l of eq. (5.9) (P_A^{inex}, eq. 5.6) or Lambda~_l of eq. (5.10)
// (interior block (A_hat_l)_II).  (The tensor-core versions are in fd_tc.cu
// and fd_slab.cu, the Schur block in schur.cu.)
// One CTA owns one (patch, component) tensor; the tensor lives in shared
// memory when it fits and in a global scratch slab otherwise.  Arithmetic is
// FP64 (plain form) or FP32 (mixed form), inputs and outputs FP64.
//
// Mode products are register blocked: a thread computes RA = 4 consecutive
// outputs of one line, loading each input once and the 4 coefficients of a
// row of the (zero-padded) U or U^T copy with one vector load.
#include "common.cuh"

namespace afi {

template <typename T> struct Pool;
template <> struct Pool<double> { static const double *get(const afi_ctx *c) { return c->dpool; } };
template <> struct Pool<float> { static const float *get(const afi_ctx *c) { return c->fpool; } };

template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void load(const float *p, float *o) {
    float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void load(const double *p, double *o) {
    double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
};

// FP64 vector entries to and from the working precision (integer-pipe
// conversions for FP32)
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return f64_to_f32(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }

// dst[i] = src[i] (converted) for i < n, block-strided; the global loads of
// a batch are issued before its stores so that they overlap
template <typename T>
__device__ __forceinline__ void load_block(const double *__restrict__ src, T *dst, int n) {
  constexpr int LB = 8;
  for (int i0 = threadIdx.x; i0 < n; i0 += LB * blockDim.x) {
    double v[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < n ? __ldg(src + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n) dst[i] = from_f64<T>(v[u]);
    }
  }
}

constexpr int RA = 4;

// dst[.., a, ..] = sum_j Mp[j][a] src[.., j, ..] along direction d, Mp padded
// to leading dimension ld (multiple of 4).  Forward transforms pass U
// (Mp[j][a] = U[j][a]); back transforms pass U^T.
template <typename T>
__device__ __forceinline__ void mode_rb(const T *__restrict__ src, T *__restrict__ dst,
                                        const T *__restrict__ Mp, int ld, int n, int d, int n1,
                                        int n2, int n3) {
  const int N = n1 * n2 * n3;
  const int nl = N / n, nab = (n + RA - 1) / RA;
  const int stride = (d == 0) ? 1 : (d == 1 ? n1 : n1 * n2);
  for (int item = threadIdx.x; item < nl * nab; item += blockDim.x) {
    const int line = item % nl, a0 = (item / nl) * RA;
    int base;
    if (d == 0) base = line * n1;
    else if (d == 1) base = (line % n1) + (line / n1) * n1 * n2;
    else base = line;
    T acc[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) acc[r] = T(0);
    const T *row = Mp + a0;
    for (int j = 0; j < n; ++j) {
      const T x = src[base + j * stride];
      T m[RA];
      Vec4<T>::load(row + j * ld, m);
#pragma unroll
      for (int r = 0; r < RA; ++r) acc[r] += m[r] * x;
    }
#pragma unroll
    for (int r = 0; r < RA; ++r)
      if (a0 + r < n) dst[base + (a0 + r) * stride] = acc[r];
  }
}

struct Dims { int n[3]; int N; };

__device__ __forceinline__ Dims dims_of(const DevPatch &pt, int interior) {
  Dims D;
  for (int d = 0; d < 3; ++d) D.n[d] = interior ? pt.ni[d] : pt.n[d];
  D.N = D.n[0] * D.n[1] * D.n[2];
  return D;
}

// Algorithm 1 on the tensor in `cur` (ping-pong with `oth`).  Returns the
// buffer that holds the result.
template <typename T>
__device__ T *fd_tensor(T *cur, T *oth, const DevPatch &pt, const DevPatch *pglob,
                        const Tab1D *tabs, const T *tpool, int dim, int l, int interior) {
  const Dims D = dims_of(pt, interior);
  const T *Uf[3], *Ub[3], *Dv[3];
  int ld[3];
  // component-indexed fields straight from global memory (pt is a local
  // copy, which a runtime index would move to local memory)
  const DevPatch &pg = *pglob;
  const int lt[3] = {pg.ltab[l][0], pg.ltab[l][1], pg.ltab[l][2]};
  for (int d = 0; d < 3; ++d) {
    const Tab1D tb = tabs[lt[d]];
    Uf[d] = tpool + (interior ? tb.Uip : tb.Up);
    Ub[d] = tpool + (interior ? tb.Uipt : tb.Upt);
    Dv[d] = tpool + (interior ? tb.Di : tb.D);
    ld[d] = interior ? tb.ldi : tb.ld;
  }
  for (int d = 0; d < dim; ++d) {   // r~ = (U^T x ... x U^T) r
    mode_rb<T>(cur, oth, Uf[d], ld[d], D.n[d], d, D.n[0], D.n[1], D.n[2]);
    __syncthreads();
    T *t = cur; cur = oth; oth = t;
  }
  const T hs = (T)pt.lscale, sh = (T)pt.lshift;
  const T c0 = (T)pg.lcf[l][0], c1 = (T)pg.lcf[l][1], c2 = (T)pg.lcf[l][2];
  for (int idx = threadIdx.x; idx < D.N; idx += blockDim.x) {   // q~ = Lambda^{-1} r~
    const int i1 = idx % D.n[0], i2 = (idx / D.n[0]) % D.n[1], i3 = idx / (D.n[0] * D.n[1]);
    T lam = c0 * Dv[0][i1] + c1 * Dv[1][i2] + (dim == 3 ? c2 * Dv[2][i3] : T(0));
    if (!interior) lam = hs * (lam + sh);
    cur[idx] = cur[idx] / lam;
  }
  __syncthreads();
  for (int d = dim - 1; d >= 0; --d) {   // s = (U x ... x U) q~
    mode_rb<T>(cur, oth, Ub[d], ld[d], D.n[d], d, D.n[0], D.n[1], D.n[2]);
    __syncthreads();
    T *t = cur; cur = oth; oth = t;
  }
  return cur;
}

template <typename T>
__global__ void __launch_bounds__(512) k_fd(const DevPatch *P, const Tab1D *tabs, const T *tpool,
                                            int dim, int interior, const double *r, double *s,
                                            T *gscratch, int use_smem, const double *gate,
                                            long long rhs_stride, const int *plist) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  extern __shared__ __align__(16) unsigned char smraw[];
  const int k = plist ? plist[blockIdx.x] : blockIdx.x, l = blockIdx.y;
  const DevPatch pt = P[k];
  const Dims D = dims_of(pt, interior);
  const long long tbase = (interior ? pt.ioff : pt.off) + (long long)l * D.N;
  const long long base = tbase + (long long)blockIdx.z * rhs_stride;
  // the global fallback slab is per tensor of one right-hand side: the
  // launch uses grid.z = 1 whenever shared memory is too small
  T *b0 = use_smem ? reinterpret_cast<T *>(smraw) : gscratch + 2 * tbase;
  T *b1 = b0 + D.N;
  load_block<T>(r + base, b0, D.N);
  __syncthreads();
  const T *res = fd_tensor<T>(b0, b1, pt, P + k, tabs, tpool, dim, l, interior);
  for (int i = threadIdx.x; i < D.N; i += blockDim.x) s[base + i] = to_f64(res[i]);
}

// Opt the local-solver kernels into the device's full dynamic shared memory
// once per context (outside any stream capture).
afi_status fd_prepare(afi_ctx *c) {
  int dev = 0, v = 0;
  AFI_CUDA(cudaGetDevice(&dev));
  AFI_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  c->smem_optin = v;
  AFI_CUDA(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
  // these kernels have no static shared memory: the whole opt-in size is dynamic
  AFI_CUDA(cudaFuncSetAttribute(k_fd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
  AFI_CUDA(cudaFuncSetAttribute(k_fd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
  return AFI_OK;
}

template <typename T>
static afi_status fd_launch(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                            int nrhs, const int *list = nullptr, int count = 0, int maxN = 0) {
  if (!list) {
    count = c->npatch;
    maxN = 1;
    for (auto &p : c->hp) maxN = std::max(maxN, interior ? p.Ni : p.N);
  }
  size_t smem = 2ull * maxN * sizeof(T);
  const int use_smem = smem <= (size_t)c->smem_optin;
  if (!use_smem) smem = 0;
  const long long stride = interior ? c->n_int : c->n_dof;
  // with the global scratch slab the right-hand sides go one launch each
  const int per_launch = use_smem ? nrhs : 1;
  for (int j = 0; j < nrhs; j += per_launch) {
    launch(k_fd<T>, dim3(count, c->dim, per_launch), 512, smem, st, c->patches,
           (const Tab1D *)c->tabs, Pool<T>::get(c), c->dim, interior, r + j * stride, s + j * stride,
           reinterpret_cast<T *>(c->fdscratch), use_smem, (const double *)c->gate, stride, list);
  }
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

static afi_status fd_dispatch(afi_ctx *c, int interior, const double *r, double *s,
                              cudaStream_t st, int nrhs) {
  switch (c->opt.prec) {
    case AFI_FD_FP64: return fd_launch<double>(c, interior, r, s, st, nrhs);
    case AFI_FD_FP32: return fd_launch<float>(c, interior, r, s, st, nrhs);
    case AFI_FD_TF32:
    case AFI_FD_BF16:
      // tensor cores: the single-CTA kernel for the tensors that fit one
      // CTA, the three-pass kernels for larger ones, and FP32 SIMT only for
      // tensors that neither takes
      return fd_tc_run(c, interior, r, s, st, nrhs);
    default: set_error("local-solver precision not available"); return AFI_EINVAL;
  }
}

afi_status fd_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                  int nrhs) {
  if (c->geo && !interior) {
    // geometry inclusion (eq. 5.12): D_A^{-1/2} (A~_l + H^{-2} M~_l)^{-1} D_A^{-1/2}
    const long n = c->n_dof;
    for (int j = 0; j < nrhs; ++j) {
      AFI_TRY(geo_scale(c, r + (long long)j * n, c->geo_dA, c->geo_tmp, n, 1, st));
      AFI_TRY(fd_dispatch(c, 0, c->geo_tmp, s + (long long)j * n, st, 1));
      AFI_TRY(geo_scale(c, s + (long long)j * n, c->geo_dA, s + (long long)j * n, n, 1, st));
    }
    return AFI_OK;
  }
  return fd_dispatch(c, interior, r, s, st, nrhs);
}

afi_status fd_simt_list(afi_ctx *c, int interior, const int *list, int count, int maxN,
                        const double *r, double *s, cudaStream_t st, int nrhs) {
  return fd_launch<float>(c, interior, r, s, st, nrhs, list, count, maxN);
}

}  // namespace afi
