// The parametric Schur complement of Section 5.2, eqs. (5.4)-(5.5), in the
// H^{d-2}-scaled non-redundant preconditioner P_S (eq. 5.7, Remark 1), for
// every (patch, component) block at once:
//
//   S_hat theta = (A_hat v)_Gamma,  v_Gamma = theta,
//   v_I = -(A_hat_l)_II^{-1} (A_hat [theta; 0])_I,
//
// where A_hat_l is applied through its Kronecker form with the banded
// univariate K_hat, M_hat (Section 5.2):
//   A_hat_1 = c1 M3 x M2 x K1 + c2 M3 x K2 x M1 + c3 K3 x M2 x M1   (3D)
// evaluated as four banded directional passes:
//   t1 = M1 v, t2 = K1 v;  o = c1 M2 t2 + c2 K2 t1;  t2 = M2 t1;
//   t1 = M3 o + c3 K3 t2.
//
// Each pass is one launch over all tensors (kOB consecutive outputs per
// thread from a register window, consecutive threads along the contiguous
// index, L2-resident buffers).  The first pass builds v from theta (and v_I)
// on the fly and the last pass writes the interior right-hand side or the
// scaled shell output directly.  The interior solve goes through the
// local-solver FD (fd_run with interior = 1: tensor cores for TF32/BF16,
// SIMT for FP32/FP64).  Buffers are FP32 in the mixed forms and FP64 in the
// plain form; inputs and outputs are FP64 torn vectors.
#include "common.cuh"

#include <algorithm>

namespace afi {

namespace {

template <typename T> struct SPool;
template <> struct SPool<double> { static const double *get(const afi_ctx *c) { return c->dpool; } };
template <> struct SPool<float> { static const float *get(const afi_ctx *c) { return c->fpool; } };

template <typename T> __device__ __forceinline__ T in64(double x);
template <> __device__ __forceinline__ double in64<double>(double x) { return x; }
template <> __device__ __forceinline__ float in64<float>(double x) { return f64_to_f32(x); }
__device__ __forceinline__ double out64(double x) { return x; }
__device__ __forceinline__ double out64(float x) { return f32_to_f64(x); }

// Per-CTA data of one (patch, component) tensor, loaded once into shared
// memory by thread 0.
template <typename T>
struct PsMeta {
  int n[3], ni[3], N, p, zo;
  long long off, ioff;   // this component's first entry, full and compact interior
  const T *Mb, *Kb;      // bands of the pass direction
  T cf0, cf1, cf2, hs;
};

template <typename T>
__device__ __forceinline__ void load_meta(PsMeta<T> &m, const DevPatch *P, const Tab1D *tabs,
                                          const T *tpool, int dim, int d) {
  if (threadIdx.x == 0) {
    const int k = blockIdx.y / dim, l = blockIdx.y - k * dim;
    const DevPatch &pt = P[k];
    for (int q = 0; q < 3; ++q) { m.n[q] = pt.n[q]; m.ni[q] = pt.ni[q]; }
    m.N = pt.N;
    m.p = pt.p;
    m.zo = (dim == 3) ? 1 : 0;
    m.off = pt.off + (long long)l * pt.N;
    m.ioff = pt.ioff + (long long)l * pt.Ni;
    const Tab1D &tb = tabs[pt.ltab[l][d]];
    m.Mb = tpool + tb.Mb;
    m.Kb = tpool + tb.Kb;
    m.cf0 = (T)pt.lcf[l][0];
    m.cf1 = (T)pt.lcf[l][1];
    m.cf2 = (T)pt.lcf[l][2];
    m.hs = (T)pt.lscale;
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ bool shell_node(const PsMeta<T> &m, int i1, int i2, int i3, int dim) {
  return i1 == 0 || i1 == m.n[0] - 1 || i2 == 0 || i2 == m.n[1] - 1 ||
         (dim == 3 && (i3 == 0 || i3 == m.n[2] - 1));
}

// compact interior index of an interior node (interior sizes n - 2; a 2D
// problem's dummy third direction keeps its single layer)
template <typename T>
__device__ __forceinline__ long long interior_at(const PsMeta<T> &m, int i1, int i2, int i3) {
  return m.ioff + (i1 - 1) + (long long)m.ni[0] * ((i2 - 1) + (long long)m.ni[1] * (i3 - m.zo));
}

}  // namespace

constexpr int kOB = 4;   // consecutive outputs along the pass direction per thread

// One banded pass of A_hat (see the file comment) for every (patch,
// component) tensor: blockIdx.y = patch * dim + component; each thread
// computes kOB consecutive outputs along the pass direction from a register
// window of kOB + 2p inputs.
//   PASS 0 (direction 1): t1 = M1 v, t2 = K1 v, with v built on the fly:
//          theta (from t) on the shell, 0 (CALL 0) or -v_I (CALL 1) inside;
//   PASS 1 (direction 2): o = c1 M2 t2 + c2 K2 t1 (the last pass in 2D);
//   PASS 2 (direction 2): t2 = M2 t1;
//   PASS 3 (direction 3): t1 = M3 o + c3 K3 t2 (the last pass in 3D).
// The last pass writes, for CALL 0, the interior entries of A_hat [theta; 0]
// to rint (compact, FP64) and, for CALL 1, y = H^{d-2} (A_hat v) on the
// shell and 0 inside.  With the geometry-inclusion solvers (dS non-null, the
// per-dof D_S^{1/2} of eq. 5.13) theta enters as D_S^{1/2} theta and the
// shell output leaves times D_S^{1/2}; the tables are then those of A~_l,
// with unit coefficients and unit scale.
template <typename T, int PC, int PASS, int CALL>
__global__ void __launch_bounds__(256) k_ps_band(const DevPatch *P, const Tab1D *tabs, const T *tpool,
                                                 int dim, const double *t, const double *vint, T *O,
                                                 T *T1, T *T2, double *rint, double *y,
                                                 const double *dS, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  constexpr int d = (PASS == 0) ? 0 : (PASS == 3 ? 2 : 1);
  __shared__ PsMeta<T> m;
  load_meta<T>(m, P, tabs, tpool, dim, d);
  const int n1 = m.n[0], n2 = m.n[1], n = m.n[d];
  const int p = PC > 0 ? PC : m.p;
  const int nbd = (n + kOB - 1) / kOB;
  const int groups = m.N / n * nbd;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  int i1, i2, i3, b;
  if (d == 0) { b = g % nbd; const int r = g / nbd; i2 = r % n2; i3 = r / n2; i1 = 0; }
  else if (d == 1) { i1 = g % n1; const int r = g / n1; b = r % nbd; i3 = r / nbd; i2 = 0; }
  else { i1 = g % n1; const int r = g / n1; i2 = r % n2; b = r / n2; i3 = 0; }
  const int io0 = b * kOB;
  const long long stride = (d == 0) ? 1 : (d == 1 ? n1 : (long long)n1 * n2);
  const long long base = m.off + i1 + (long long)n1 * (i2 + (long long)n2 * i3);   // io = 0
  constexpr int WMAX = kOB + 2 * (PC > 0 ? PC : 5);
  const int WN = kOB + 2 * p;
  T wa[WMAX], wb[WMAX];
  const T *sa = (PASS == 1) ? T2 : (PASS == 2 ? T1 : O);
  const T *sb = (PASS == 1) ? T1 : T2;
#pragma unroll
  for (int w = 0; w < WMAX; ++w) {
    wa[w] = T(0);
    wb[w] = T(0);
    if (w >= WN) continue;
    const int j = io0 - p + w;
    if (j < 0 || j >= n) continue;
    const long long at = base + j * stride;
    if (PASS == 0) {
      const int a1 = (d == 0) ? j : i1;
      if (shell_node(m, a1, i2, i3, dim)) wa[w] = in64<T>(dS ? t[at] * dS[at] : t[at]);
      else if (CALL == 1) wa[w] = in64<T>(-vint[interior_at(m, a1, i2, i3)]);
    } else {
      wa[w] = sa[at];
      if (PASS != 2) wb[w] = sb[at];
    }
  }
  const bool last = (PASS == 3) || (PASS == 1 && dim == 2);
#pragma unroll
  for (int o = 0; o < kOB; ++o) {
    const int io = io0 + o;
    if (io >= n) break;
    T a = 0, c2 = 0;
#pragma unroll
    for (int q = 0; q < (PC > 0 ? 2 * PC + 1 : 11); ++q) {
      if (PC == 0 && q > 2 * p) break;
      const T mq = m.Mb[q * n + io];
      a += mq * wa[o + q];
      if (PASS == 0) c2 += m.Kb[q * n + io] * wa[o + q];
      else if (PASS != 2) c2 += m.Kb[q * n + io] * wb[o + q];
    }
    const long long at = base + io * stride;
    T val;
    if (PASS == 0) { T1[at] = a; T2[at] = c2; continue; }
    else if (PASS == 1) val = m.cf0 * a + m.cf1 * c2;
    else if (PASS == 2) { T2[at] = a; continue; }
    else val = a + m.cf2 * c2;
    if (!last) { O[at] = val; continue; }
    const int a1 = (d == 0) ? io : i1, a2 = (d == 1) ? io : i2, a3 = (d == 2) ? io : i3;
    const bool sh = shell_node(m, a1, a2, a3, dim);
    if (CALL == 0) {
      if (!sh) rint[interior_at(m, a1, a2, a3)] = out64(val);
    } else {
      y[at] = sh ? (dS ? out64(m.hs * val) * dS[at] : out64(m.hs * val)) : 0.0;
    }
  }
}

template <typename T, int PC, int CALL>
static void ahat_passes(afi_ctx *c, const double *t, const double *vint, T *O, T *T1, T *T2,
                        double *rint, double *y, cudaStream_t st) {
  const DevPatch *P = c->patches;
  const Tab1D *tabs = c->tabs;
  const T *tp = SPool<T>::get(c);
  const double *gate = c->gate;
  const double *dS = c->geo ? c->geo_dS : nullptr;
  // groups per tensor <= N / n_d * ceil(n_d / kOB) <= max_N / kOB + max_N / min(n)
  int gmax = 1;
  for (auto &q : c->hp)
    for (int d = 0; d < c->dim; ++d)
      gmax = std::max(gmax, q.N / q.n[d] * ((q.n[d] + kOB - 1) / kOB));
  const dim3 g((gmax + 255) / 256, c->npatch * c->dim);
  launch(k_ps_band<T, PC, 0, CALL>, g, 256, 0, st, P, tabs, tp, c->dim, t, vint, O, T1, T2, rint, y, dS, gate);
  launch(k_ps_band<T, PC, 1, CALL>, g, 256, 0, st, P, tabs, tp, c->dim, t, vint, O, T1, T2, rint, y, dS, gate);
  if (c->dim == 3) {
    launch(k_ps_band<T, PC, 2, CALL>, g, 256, 0, st, P, tabs, tp, c->dim, t, vint, O, T1, T2, rint, y, dS, gate);
    launch(k_ps_band<T, PC, 3, CALL>, g, 256, 0, st, P, tabs, tp, c->dim, t, vint, O, T1, T2, rint, y, dS, gate);
  }
}

template <typename T, int PC>
static afi_status schur_pc(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  T *O = reinterpret_cast<T *>(c->ps_buf);
  T *T1 = O + c->n_dof, *T2 = T1 + c->n_dof;
  ahat_passes<T, PC, 0>(c, t, nullptr, O, T1, T2, c->ps_rint, nullptr, st);   // (A_hat [theta; 0])_I
  AFI_LAUNCH_CHECK();
  AFI_TRY(fd_run(c, 1, c->ps_rint, c->ps_vint, st));   // v_I = -(A_hat)_II^{-1} (...)
  ahat_passes<T, PC, 1>(c, t, c->ps_vint, O, T1, T2, nullptr, y, st);   // (A_hat [theta; v_I])_Gamma
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

template <typename T>
static afi_status schur_pipeline(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  int pu = c->hp[0].p;   // one degree for every patch -> degree-specialised passes
  for (auto &q : c->hp)
    if (q.p != pu) pu = 0;
  switch (pu) {
    case 1: return schur_pc<T, 1>(c, t, y, st);
    case 2: return schur_pc<T, 2>(c, t, y, st);
    case 3: return schur_pc<T, 3>(c, t, y, st);
    case 4: return schur_pc<T, 4>(c, t, y, st);
    case 5: return schur_pc<T, 5>(c, t, y, st);
    default: return schur_pc<T, 0>(c, t, y, st);
  }
}

// y = blkdiag_k H_k^{d-2} S_hat^(k) t on the shell (interior entries of y are
// zero; only shell entries of t are read).  FP64 buffers in the plain form,
// FP32 in the mixed forms; the interior solve uses the context's local-solver
// precision.
afi_status schur_run(afi_ctx *c, const double *t, double *y, cudaStream_t st) {
  if (c->opt.prec == AFI_FD_FP64) return schur_pipeline<double>(c, t, y, st);
  return schur_pipeline<float>(c, t, y, st);
}

}  // namespace afi
