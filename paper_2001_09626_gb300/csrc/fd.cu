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

// dst = alpha * Mat1(src1) [+ beta * Mat2(src2)] along direction d, with the
// banded (half-bandwidth p) univariate matrices stored by diagonal:
// Mb[t*n + i] = Mat[i][i + t - p].  One thread per line along d: the line
// base is decoded once, then the thread walks the line.  PC > 0 fixes the
// half-bandwidth at compile time.
template <typename T, int PC>
__device__ __forceinline__ void mode_band2_lines(const T *__restrict__ src1,
                                                 const T *__restrict__ Mb1, T alpha,
                                                 const T *__restrict__ src2,
                                                 const T *__restrict__ Mb2, T beta,
                                                 T *__restrict__ dst, int p_rt, int d, int n1,
                                                 int n2, int n3) {
  const int p = PC > 0 ? PC : p_rt;
  const int n = (d == 0) ? n1 : (d == 1 ? n2 : n3);
  const int stride = (d == 0) ? 1 : (d == 1 ? n1 : n1 * n2);
  const int nlines = n1 * n2 * n3 / n;
  for (int line = threadIdx.x; line < nlines; line += blockDim.x) {
    int base;
    if (d == 0) base = line * n1;
    else if (d == 1) base = (line % n1) + (line / n1) * n1 * n2;
    else base = line;
    for (int io = 0; io < n; ++io) {
      T a1 = 0, a2 = 0;
      const int j0 = io - p;
#pragma unroll
      for (int t = 0; t < (PC > 0 ? 2 * PC + 1 : 1); ++t) {
        if (PC == 0) break;
        const int j = j0 + t;
        if (j >= 0 && j < n) {
          a1 += Mb1[t * n + io] * src1[base + j * stride];
          if (src2) a2 += Mb2[t * n + io] * src2[base + j * stride];
        }
      }
      if (PC == 0)
        for (int t = 0; t <= 2 * p; ++t) {
          const int j = j0 + t;
          if (j >= 0 && j < n) {
            a1 += Mb1[t * n + io] * src1[base + j * stride];
            if (src2) a2 += Mb2[t * n + io] * src2[base + j * stride];
          }
        }
      dst[base + io * stride] = alpha * a1 + (src2 ? beta * a2 : T(0));
    }
  }
}

template <typename T>
__device__ __forceinline__ void mode_band2(const T *src1, const T *Mb1, T alpha, const T *src2,
                                           const T *Mb2, T beta, T *dst, int p, int d, int n1,
                                           int n2, int n3) {
  switch (p) {
    case 1: mode_band2_lines<T, 1>(src1, Mb1, alpha, src2, Mb2, beta, dst, p, d, n1, n2, n3); break;
    case 2: mode_band2_lines<T, 2>(src1, Mb1, alpha, src2, Mb2, beta, dst, p, d, n1, n2, n3); break;
    case 3: mode_band2_lines<T, 3>(src1, Mb1, alpha, src2, Mb2, beta, dst, p, d, n1, n2, n3); break;
    case 4: mode_band2_lines<T, 4>(src1, Mb1, alpha, src2, Mb2, beta, dst, p, d, n1, n2, n3); break;
    case 5: mode_band2_lines<T, 5>(src1, Mb1, alpha, src2, Mb2, beta, dst, p, d, n1, n2, n3); break;
    default: mode_band2_lines<T, 0>(src1, Mb1, alpha, src2, Mb2, beta, dst, p, d, n1, n2, n3);
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
__device__ T *fd_tensor(T *cur, T *oth, const DevPatch &pt, const Tab1D *tabs, const T *tpool,
                        int dim, int l, int interior) {
  const Dims D = dims_of(pt, interior);
  const T *Uf[3], *Ub[3], *Dv[3];
  int ld[3];
  for (int d = 0; d < 3; ++d) {
    const Tab1D tb = tabs[pt.tab[d]];
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
  const T cl = (T)(2.0 * pt.mu + pt.lam), mu = (T)pt.mu, hs = (T)pt.Hs;
  const T c0 = (l == 0) ? cl : mu, c1 = (l == 1) ? cl : mu, c2 = (l == 2) ? cl : mu;
  for (int idx = threadIdx.x; idx < D.N; idx += blockDim.x) {   // q~ = Lambda^{-1} r~
    const int i1 = idx % D.n[0], i2 = (idx / D.n[0]) % D.n[1], i3 = idx / (D.n[0] * D.n[1]);
    T lam = c0 * Dv[0][i1] + c1 * Dv[1][i2] + (dim == 3 ? c2 * Dv[2][i3] : T(0));
    if (!interior) lam = hs * (lam + T(1));
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
  const T *res = fd_tensor<T>(b0, b1, pt, tabs, tpool, dim, l, interior);
  for (int i = threadIdx.x; i < D.N; i += blockDim.x) s[base + i] = to_f64(res[i]);
}

// One banded pass along direction d: dst = alpha Mat_A srcA (+ beta Mat_B srcB)
// with the half-bandwidth P fixed at compile time (diagonal-major bands,
// Mb[t*n + i] = Mat[i][i + t - P]).  Work items are (line, block of OB
// consecutive outputs): each loads its window of OB + 2P inputs once into
// registers, so a line is split over several threads and every thread has
// several independent accumulations.  With DUAL, srcB is ignored and the
// same window feeds two bands into two outputs (dst = Mat_A src, dst2 =
// Mat_B src).
template <typename T, int P, bool DUAL>
__device__ __forceinline__ void band_pass(const T *__restrict__ srcA, const T *__restrict__ MbA, T alpha,
                                          const T *__restrict__ srcB, const T *__restrict__ MbB,
                                          T beta, T *__restrict__ dst, T *__restrict__ dst2, int d,
                                          int n1, int n2, int n3) {
  constexpr int OB = 4, WN = OB + 2 * P;
  const int n = (d == 0) ? n1 : (d == 1 ? n2 : n3);
  const int stride = (d == 0) ? 1 : (d == 1 ? n1 : n1 * n2);
  const int nlines = n1 * n2 * n3 / n, nob = (n + OB - 1) / OB;
  for (int item = threadIdx.x; item < nlines * nob; item += blockDim.x) {
    const int line = item % nlines, i0 = (item / nlines) * OB;
    int base;
    if (d == 0) base = line * n1;
    else if (d == 1) base = (line % n1) + (line / n1) * n1 * n2;
    else base = line;
    T wa[WN], wb[WN];
#pragma unroll
    for (int t = 0; t < WN; ++t) {
      const int j = i0 - P + t;
      const bool in = j >= 0 && j < n;
      wa[t] = in ? srcA[base + j * stride] : T(0);
      if (!DUAL && srcB) wb[t] = in ? srcB[base + j * stride] : T(0);
    }
#pragma unroll
    for (int o = 0; o < OB; ++o) {
      const int io = i0 + o;
      if (io >= n) break;
      T a = 0, b = 0;
#pragma unroll
      for (int t = 0; t <= 2 * P; ++t) {
        a += MbA[t * n + io] * wa[o + t];
        if (DUAL) b += MbB[t * n + io] * wa[o + t];
        else if (srcB) b += MbB[t * n + io] * wb[o + t];
      }
      if (DUAL) {
        dst[base + io * stride] = a;
        dst2[base + io * stride] = b;
      } else {
        dst[base + io * stride] = alpha * a + (srcB ? beta * b : T(0));
      }
    }
  }
}

// A_hat_l v (Kronecker form, Section 5.2) from buffer v; out, t1, t2 are
// scratch.  Returns the buffer that holds the result (t1 in 3D, out in 2D).
// P > 0: half-bandwidth (degree) fixed at compile time; P = 0: any degree.
template <typename T, int P>
__device__ __noinline__ T *ahat_apply(const T *v, T *out, T *t1, T *t2, const DevPatch &pt,
                                      const Tab1D *tabs, const T *tpool, int dim, int l) {
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2];
  const Tab1D &A0 = tabs[pt.tab[0]], &A1 = tabs[pt.tab[1]], &A2 = tabs[pt.tab[2]];
  const T cl = (T)(2.0 * pt.mu + pt.lam), mu = (T)pt.mu;
  const T c0 = (l == 0) ? cl : mu, c1 = (l == 1) ? cl : mu, c2 = (l == 2) ? cl : mu;
  const int p = pt.p;
  // t1 = M_1 v, t2 = K_1 v (direction 1)
  if (P > 0) {
    band_pass<T, P, true>(v, tpool + A0.Mb, T(1), nullptr, tpool + A0.Kb, T(0), t1, t2, 0, n1, n2, n3);
  } else {
    mode_band2<T>(v, tpool + A0.Mb, T(1), nullptr, nullptr, T(0), t1, p, 0, n1, n2, n3);
    mode_band2<T>(v, tpool + A0.Kb, T(1), nullptr, nullptr, T(0), t2, p, 0, n1, n2, n3);
  }
  __syncthreads();
  // out = c0 M_2 t2 + c1 K_2 t1 (direction 2): the 2D result, Ta in 3D
  if (P > 0) band_pass<T, P, false>(t2, tpool + A1.Mb, c0, t1, tpool + A1.Kb, c1, out, nullptr, 1, n1, n2, n3);
  else mode_band2<T>(t2, tpool + A1.Mb, c0, t1, tpool + A1.Kb, c1, out, p, 1, n1, n2, n3);
  __syncthreads();
  if (dim == 2) return out;
  // t2 = Tb = M_2 t1 (direction 2)
  if (P > 0) band_pass<T, P, false>(t1, tpool + A1.Mb, T(1), nullptr, nullptr, T(0), t2, nullptr, 1, n1, n2, n3);
  else mode_band2<T>(t1, tpool + A1.Mb, T(1), nullptr, nullptr, T(0), t2, p, 1, n1, n2, n3);
  __syncthreads();
  // t1 = M_3 Ta + c2 K_3 Tb (direction 3)
  if (P > 0) band_pass<T, P, false>(out, tpool + A2.Mb, T(1), t2, tpool + A2.Kb, c2, t1, nullptr, 2, n1, n2, n3);
  else mode_band2<T>(out, tpool + A2.Mb, T(1), t2, tpool + A2.Kb, c2, t1, p, 2, n1, n2, n3);
  __syncthreads();
  return t1;
}

// y = H^{d-2} S_hat_l theta for every (patch, component); t, y torn vectors,
// only shell entries of t are read, interior entries of y are zero.
// (eqs. 5.4-5.5: S theta = (A_hat v)_Gamma, v_Gamma = theta,
// v_I = -(A_hat)_II^{-1} (A_hat [theta; 0])_I.)
template <typename T, int P>
__global__ void __launch_bounds__(512, 2) k_schur(const DevPatch *P_, const Tab1D *tabs,
                                               const T *tpool, int dim, const double *t, double *y,
                                               T *gscratch, int use_smem, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  extern __shared__ __align__(16) unsigned char smraw[];
  const int k = blockIdx.x, l = blockIdx.y;
  const DevPatch pt = P_[k];
  const int N = pt.N;
  const long long base = pt.off + (long long)l * N;
  T *B0 = use_smem ? reinterpret_cast<T *>(smraw) : gscratch + 4 * base;
  T *B1 = B0 + N, *B2 = B1 + N, *B3 = B2 + N;
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2];
  // theta on the shell: the whole block is read (interior entries of t are
  // finite: zero or stale operator output) and the interior is zeroed after
  load_block<T>(t + base, B0, N);
  __syncthreads();
  const Dims Di = dims_of(pt, 1);
  const int zo = (dim == 3) ? 1 : 0;
  for (int idx = threadIdx.x; idx < Di.N; idx += blockDim.x) {
    const int j1 = idx % Di.n[0], j2 = (idx / Di.n[0]) % Di.n[1], j3 = idx / (Di.n[0] * Di.n[1]);
    B0[(j1 + 1) + n1 * ((j2 + 1) + n2 * (j3 + zo))] = T(0);
  }
  __syncthreads();
  T *R = ahat_apply<T, P>(B0, B1, B2, B3, pt, tabs, tpool, dim, l);   // A_hat [theta; 0]
  // interior solve v_I = -(A_hat)_II^{-1} R_I on compact tensors in B3 and a free buffer
  T *F = (R == B1) ? B2 : B1;
  for (int idx = threadIdx.x; idx < Di.N; idx += blockDim.x) {
    const int j1 = idx % Di.n[0], j2 = (idx / Di.n[0]) % Di.n[1], j3 = idx / (Di.n[0] * Di.n[1]);
    B3[idx] = R[(j1 + 1) + n1 * ((j2 + 1) + n2 * (j3 + zo))];
  }
  __syncthreads();
  const T *vI = fd_tensor<T>(B3, F, pt, tabs, tpool, dim, l, 1);
  for (int idx = threadIdx.x; idx < Di.N; idx += blockDim.x) {
    const int j1 = idx % Di.n[0], j2 = (idx / Di.n[0]) % Di.n[1], j3 = idx / (Di.n[0] * Di.n[1]);
    B0[(j1 + 1) + n1 * ((j2 + 1) + n2 * (j3 + zo))] = -vI[idx];
  }
  __syncthreads();
  R = ahat_apply<T, P>(B0, B1, B2, B3, pt, tabs, tpool, dim, l);   // A_hat [theta; v_I]
  const T hs = (T)pt.Hs;
  for (int line = threadIdx.x; line < n2 * n3; line += blockDim.x) {
    const int i2 = line % n2, i3 = line / n2;
    const bool face = i2 == 0 || i2 == n2 - 1 || (dim == 3 && (i3 == 0 || i3 == n3 - 1));
    for (int i1 = 0; i1 < n1; ++i1) {
      const int i = i1 + n1 * line;
      y[base + i] = (face || i1 == 0 || i1 == n1 - 1) ? to_f64(hs * R[i]) : 0.0;
    }
  }
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
  const void *schur[] = {(const void *)k_schur<float, 0>, (const void *)k_schur<float, 1>,
                         (const void *)k_schur<float, 2>, (const void *)k_schur<float, 3>,
                         (const void *)k_schur<float, 4>, (const void *)k_schur<float, 5>,
                         (const void *)k_schur<double, 0>, (const void *)k_schur<double, 1>,
                         (const void *)k_schur<double, 2>, (const void *)k_schur<double, 3>,
                         (const void *)k_schur<double, 4>, (const void *)k_schur<double, 5>};
  for (const void *f : schur)
    AFI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
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

template <typename T>
static afi_status schur_launch(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  size_t smem = 4ull * c->max_N * sizeof(T);
  const int use_smem = smem <= (size_t)c->smem_optin;
  if (!use_smem) smem = 0;
  int pu = c->hp[0].p;   // one degree for every patch -> degree-specialised kernel
  for (auto &q : c->hp)
    if (q.p != pu) pu = 0;
  auto go = [&](auto kern) {
    launch(kern, dim3(c->npatch, c->dim), 512, smem, st, (const DevPatch *)c->patches,
           (const Tab1D *)c->tabs, Pool<T>::get(c), c->dim, t, y, reinterpret_cast<T *>(c->fdscratch),
           use_smem, (const double *)c->gate);
  };
  switch (pu) {
    case 1: go(k_schur<T, 1>); break;
    case 2: go(k_schur<T, 2>); break;
    case 3: go(k_schur<T, 3>); break;
    case 4: go(k_schur<T, 4>); break;
    case 5: go(k_schur<T, 5>); break;
    default: go(k_schur<T, 0>);
  }
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status fd_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                  int nrhs) {
  switch (c->opt.prec) {
    case AFI_FD_FP64: return fd_launch<double>(c, interior, r, s, st, nrhs);
    case AFI_FD_FP32: return fd_launch<float>(c, interior, r, s, st, nrhs);
    case AFI_FD_TF32:
    case AFI_FD_BF16:
      // tensor cores for the patches whose tensors fit one CTA, FP32 SIMT
      // for the others
      return fd_tc_run(c, interior, r, s, st, nrhs);
    default: set_error("local-solver precision not available"); return AFI_EINVAL;
  }
}

afi_status fd_simt_list(afi_ctx *c, int interior, const int *list, int count, int maxN,
                        const double *r, double *s, cudaStream_t st, int nrhs) {
  return fd_launch<float>(c, interior, r, s, st, nrhs, list, count, maxN);
}

// The Schur block (banded A_hat products and the interior FD between them)
// runs in FP64 for the plain form and in FP32 for every mixed form.
afi_status schur_run(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  if (c->opt.prec == AFI_FD_FP64) return schur_launch<double>(c, t, y, st);
  return schur_launch<float>(c, t, y, st);
}

}  // namespace afi
