// Stiffness matvec y = A x (eqs. 3.1, 4.2) from the assembled per-node
// stencil A[l][m][o][node] over the (2p+1)^d neighbour offsets o, in three
// forms:
//  * k_stencil_mv: FP64 coefficients and FMAs (the true residual, contexts
//    set up with AFI_VARIANT_STENCIL_F64, and contexts where the pair copy
//    does not fit);
//  * k_stencil_mv_rows: the MINRES iterations' form, on a row-compressed
//    copy of the stencil as (hi, lo) FP32 pairs in double-FP32 arithmetic,
//    the coefficient rows of a tile of nodes streamed into shared memory by
//    bulk (TMA) copies through a ring of mbarrier stages.
#include "tc.cuh"

#include <algorithm>
#include <vector>

namespace afi {

using tc::bulk_g2s;
using tc::expect_tx;
using tc::smem_u32;
using tc::wait_phase;

// ------------------------------------------------------- stiffness matvec
// One thread per node: y_l(node) = sum_m sum_o A[l][m][o][node] x_m(node + o).
// Stencil planes have rows padded to even length n1p (padding coefficients
// are zero); x and y use the torn layout.  Consecutive threads read
// consecutive coefficients of one plane (coalesced).
// PC > 0: degree known at compile time (fully unrolled neighbour rows);
// PC = 0: any degree.
template <int DIM, int PC>
__global__ void __launch_bounds__(128) k_stencil_mv(const DevPatch *P, const double *__restrict__ A,
                                                    const double *__restrict__ x,
                                                    double *__restrict__ y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const DevPatch pt = P[blockIdx.y];
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= pt.N) return;
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2], p = PC > 0 ? PC : pt.p;
  const int i1 = node % n1, i2 = (node / n1) % n2, i3 = node / (n1 * n2);
  const int W1 = PC > 0 ? 2 * PC + 1 : pt.W[0], W2 = PC > 0 ? 2 * PC + 1 : pt.W[1];
  const int W3 = (DIM == 3) ? W2 : 1;
  double acc[DIM];
#pragma unroll
  for (int l = 0; l < DIM; ++l) acc[l] = 0.0;
  const long long N = pt.N, S = pt.S, NP = pt.NP;
  const double *Ab = A + pt.soff + i1 + (long long)pt.n1p * (i2 + (long long)n2 * i3);
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
#pragma unroll
        for (int o1 = 0; o1 < W1; ++o1) {
          const int j1 = i1 + o1 - p;
          const double xv = (j1 >= 0 && j1 < n1) ? xm[jrow + j1] : 0.0;
          const long long o = orow + o1;
#pragma unroll
          for (int l = 0; l < DIM; ++l) acc[l] += Ab[((long long)(l * DIM + m) * S + o) * NP] * xv;
        }
      }
    }
  }
  for (int l = 0; l < DIM; ++l) y[pt.off + l * N + node] = acc[l];
}

// ------------------------------------ stiffness matvec, double-FP32 form
// GB300 runs FP64 FMAs at 1/64 of the FP32 rate, so the FP64 form above is
// bound by the FP64 pipe (one FMA per 8-byte coefficient) rather than by
// HBM.  The MINRES iterations therefore use a second copy of the stencil in
// which every coefficient a is held, in 8 bytes, as the unevaluated sum of
// two FP32 numbers, hi = rn(a) and lo = rn(a - hi), so that
// |a - hi - lo| <= 2^-48 |a| (Dekker's double-length representation); x is
// split the same way by k_split_x.  A product
// a x = hi_a hi_x + e + hi_a lo_x + lo_a hi_x (+ lo_a lo_x, dropped) takes
// its rounding error e exactly from an FMA; each addition of hi_a hi_x to the
// running sum is made error free by Knuth's TwoSum, and the addition errors,
// e and the cross terms collect in a second FP32 sum.  The result is the
// FP64 value hi + lo.  Twelve FP32 operations per coefficient (and a
// renormalisation per neighbour row) leave the product bound by HBM.  Values
// must stay within the FP32 range.  The true residual of the solver always
// uses the FP64 form.

__global__ void k_split_x(const double *__restrict__ x, float2 *__restrict__ xs, long n, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float hi = __double2float_rn(v);
  xs[i] = make_float2(hi, __double2float_rn(v - (double)hi));
}

// the same for gridDim.y vectors x_j = x + j xstride into xs + j n
__global__ void k_split_x_multi(const double *__restrict__ x, long long xstride,
                                float2 *__restrict__ xs, long n, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration(s)
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[(long long)blockIdx.y * xstride + i];
  const float hi = __double2float_rn(v);
  xs[(long long)blockIdx.y * n + i] = make_float2(hi, __double2float_rn(v - (double)hi));
}

// sum += a x in double-FP32; the rounding steps are spelled out so that no
// contraction or reassociation can change them
__device__ __forceinline__ void df_madd(float &sh, float &sl, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float e = __fmaf_rn(a.x, x.x, -p);                     // hi_a hi_x - p, exact
  const float t = __fmaf_rn(a.y, x.x, __fmaf_rn(a.x, x.y, e));
  const float s = __fadd_rn(sh, p);                            // TwoSum(sh, p)
  const float b = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, b)), __fsub_rn(p, b));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, t));
}

// ------------------------------------- the pair copy: row-compressed layout
// The pair copy drops what the FP64 stencil stores only for regularity: the
// row padding and, for each in-row offset o1, the coefficients whose
// neighbour i1 + o1 - p falls outside the row (zeros).  Per patch, for each
// row group g = (l, m, o3, o2) (in 2D (l, m, o2)) and each o1, the sub-plane
// holds, row by row (row r = i2 + n2 i3), the len(o1) = n1 - |o1 - p|
// coefficients of the nodes i1 in [max(0, p - o1), min(n1, n1 + p - o1)),
// padded to an even count; sub-planes follow each other (rstride elements
// per group).  Every sub-plane therefore starts on a 16-byte boundary.
struct RowLayout {
  int s[11], len[11], cum[11];   // first node, length and offset of each o1 sub-plane
};

__host__ __device__ __forceinline__ void row_layout(int n1, int rows, int p, RowLayout &L) {
  const int W = 2 * p + 1;
  int c = 0;
  for (int o1 = 0; o1 < W; ++o1) {
    const int d = o1 > p ? o1 - p : p - o1;
    L.s[o1] = o1 < p ? p - o1 : 0;
    L.len[o1] = n1 - d;
    L.cum[o1] = c;
    const long long sz = (long long)rows * L.len[o1];
    c += (int)(sz + (sz & 1));
  }
}

// pair copy element e of patch blockIdx.y from the FP64 stencil
template <int DIM>
__global__ void k_stencil_pack(const DevPatch *P, const double *__restrict__ A, float2 *__restrict__ A2) {
  const DevPatch pt = P[blockIdx.y];
  const int p = pt.p, W = 2 * p + 1, n1 = pt.n[0], n2 = pt.n[1];
  const int rows = n2 * pt.n[2];
  const int G = DIM * DIM * (DIM == 3 ? W * W : W);
  const long long total = (long long)G * pt.rstride;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= total) return;
  RowLayout L;
  row_layout(n1, rows, p, L);
  const int g = (int)(e / pt.rstride), rem = (int)(e - (long long)g * pt.rstride);
  int o1 = W - 1;
  while (o1 > 0 && L.cum[o1] > rem) --o1;
  const int idx = rem - L.cum[o1];
  float2 out = make_float2(0.0f, 0.0f);
  if (idx < rows * L.len[o1]) {
    const int r = idx / L.len[o1], i1 = L.s[o1] + idx - r * L.len[o1];
    const int gpl = DIM == 3 ? W * W : W;   // row groups per (l, m)
    const int lm = g / gpl, orow = g - lm * gpl;
    const int o = o1 + W * orow;
    const int i2 = r % n2, i3 = r / n2;
    const double a = A[pt.soff + ((long long)lm * pt.S + o) * pt.NP + i1 + (long long)pt.n1p * (i2 + (long long)n2 * i3)];
    const float hi = __double2float_rn(a);
    out = make_float2(hi, __double2float_rn(a - (double)hi));
  }
  A2[pt.roff + e] = out;
}

// Rows [first, last] of the tile's rows [r0, rl] whose neighbour row
// (i2 + o2 - p, i3 + o3 - p) lies in the patch (i2 in [A2, B2], i3 in
// [A3, B3]); false if there is none.  (i3a, i2a) and (i3b, i2b) are the
// coordinates of r0 and rl.  The rows in between may include unneeded ones
// (a tile crossing an i3 plane).
__host__ __device__ __forceinline__ bool row_hull(int r0, int rl, int i3a, int i2a, int i3b, int i2b, int n2,
                                                  int A2, int B2, int A3, int B3, int &first, int &last) {
  if (A2 > B2 || A3 > B3) return false;
  if (i3a < A3) first = A3 * n2 + A2;
  else if (i3a > B3) return false;
  else if (i2a < A2) first = i3a * n2 + A2;
  else if (i2a > B2) { if (i3a + 1 > B3) return false; first = (i3a + 1) * n2 + A2; }
  else first = r0;
  if (i3b > B3) last = B3 * n2 + B2;
  else if (i3b < A3) return false;
  else if (i2b > B2) last = i3b * n2 + B2;
  else if (i2b < A2) { if (i3b - 1 < A3) return false; last = (i3b - 1) * n2 + B2; }
  else last = rl;
  return first <= last && first <= rl && last >= r0;
}

// ------------------------------- double-FP32 matvec, bulk-copy pipeline
// One CTA per tile of whole rows of a patch (as many as fit 128 threads,
// one thread per node) plus a producer warp.  A stage is one neighbour row
// (m, o3, o2): for each (l, o1), the rows of the tile that need it (their
// hull) arrive from the o1 sub-plane of group (l, m, o3, o2) by one bulk
// copy into a slot of kSlot pairs; the consumers add their products, release
// the stage and move on while the copies of the next NST - 1 stages are in
// flight.  Stages that no row of the tile needs are neither copied nor
// visited (producer and consumers decide that from the tile alone).  Every
// mbarrier wait is bounded; a wait that runs out sets *err, and the
// producer waits (bounded) for the copies it issued before the CTA exits.
constexpr int kRowsTN = 128;
constexpr int kSlot = kRowsTN + 2;   // a hull of <= 128 pairs, shifted to an even start

template <int DIM, int PC>
struct RowsCfg {
  static constexpr int W = 2 * PC + 1;
  static constexpr int W3 = DIM == 3 ? W : 1;
  static constexpr int NROW = DIM * W * W3;        // stages: (m, o3, o2)
  static constexpr int CH = DIM * W;               // copies per stage: (l, o1)
  static constexpr int STAGE = CH * kSlot * 8;     // bytes per stage
  static constexpr int NST0 = 49152 / STAGE;
  static constexpr int NST = NST0 < 2 ? 2 : (NST0 > 6 ? 6 : NST0);
  static constexpr int SMEM = NST * STAGE;
};

// NR > 1: up to NR right-hand sides per launch (nrhs of them: x_j at
// xs + j n_dof, y_j at y + j ystride); every coefficient pair brought into
// shared memory serves all of them.
template <int DIM, int PC, int NR>
__global__ void __launch_bounds__(kRowsTN + 32) k_stencil_mv_rows(const DevPatch *P, const float2 *__restrict__ A2,
                                                                  const float2 *__restrict__ xs,
                                                                  double *__restrict__ y, const double *gate,
                                                                  int *err, int nrhs, long ndof,
                                                                  long long ystride) {
  using C = RowsCfg<DIM, PC>;
  constexpr int W = C::W, W3 = C::W3, NROW = C::NROW, NST = C::NST;
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  extern __shared__ __align__(128) unsigned char sm_raw[];
  float2 *stage = reinterpret_cast<float2 *>(sm_raw);   // [NST][DIM][W][kSlot]
  __shared__ uint64_t full[NST], empty[NST];
  const DevPatch pt = P[blockIdx.y];
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2], rows = n2 * n3;
  const int R = kRowsTN / n1;   // rows per tile (n1 <= 128 for contexts with a pair copy)
  const int r0 = blockIdx.x * R;
  if (r0 >= rows) return;       // the whole CTA: the grid covers the patch with most tiles
  const int nr = min(R, rows - r0), rl = r0 + nr - 1;
  const int i3a = r0 / n2, i2a = r0 - i3a * n2, i3b = rl / n2, i2b = rl - i3b * n2;
  const int tid = threadIdx.x, lane = tid & 31;
  RowLayout L;
  row_layout(n1, rows, PC, L);
  const float2 *Ap = A2 + pt.roff;
  const long long gstride = pt.rstride;
  // slots are read at clamped positions for nodes without a neighbour there
  // (their x is zero): zero the ring once so that every value read is finite
  for (int i = tid; i < C::SMEM / 16; i += blockDim.x) reinterpret_cast<float4 *>(sm_raw)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("fence.proxy.async.shared::cta;");
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(kRowsTN / 32));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  // valid neighbour-row ranges of stage (o2, o3): i2 in [A2, B2], i3 in [A3, B3]
  auto bounds = [&](int o2, int o3, int &a2, int &b2, int &a3, int &b3) {
    a2 = max(0, PC - o2); b2 = min(n2 - 1, n2 - 1 + PC - o2);
    if (DIM == 3) { a3 = max(0, PC - o3); b3 = min(n3 - 1, n3 - 1 + PC - o3); }
    else { a3 = 0; b3 = 0; }
  };

  if (tid >= kRowsTN) {   // producer warp: one lane issues every copy
    if (lane != 0) return;
    int k = 0;
    bool failed = false;
    for (int r = 0; r < NROW; ++r) {
      const int m = r / (W * W3), o3 = (r / W) % W3, o2 = r % W;
      int a2, b2, a3, b3, first, last;
      bounds(o2, o3, a2, b2, a3, b3);
      if (!row_hull(r0, rl, i3a, i2a, i3b, i2b, n2, a2, b2, a3, b3, first, last)) continue;
      const int s = k % NST;
      if (k >= NST && !wait_phase(&empty[s], (uint32_t)((k / NST - 1) & 1))) { failed = true; break; }
      uint32_t bytes = 0;
#pragma unroll
      for (int o1 = 0; o1 < W; ++o1) {
        const int st0 = first * L.len[o1], cnt = (last - first + 1) * L.len[o1];
        bytes += (uint32_t)((cnt + (st0 & 1) + ((st0 + cnt) & 1)) * 8);
      }
      expect_tx(&full[s], bytes * DIM);
      float2 *dst = stage + (size_t)s * C::CH * kSlot;
      const int grow = DIM == 3 ? o3 * W + o2 : o2;
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        const long long g = (long long)(l * DIM + m) * (W3 * W) + grow;
#pragma unroll
        for (int o1 = 0; o1 < W; ++o1) {
          const int st0 = first * L.len[o1], cnt = (last - first + 1) * L.len[o1];
          const int a = st0 & ~1, b = st0 + cnt + ((st0 + cnt) & 1);
          bulk_g2s(dst + (l * W + o1) * kSlot, Ap + g * gstride + L.cum[o1] + a, (uint32_t)(b - a) * 8u,
                   &full[s]);
        }
      }
      ++k;
    }
    // the copies issued must land before the CTA's shared memory goes away
    for (int s = 0; s < NST && s < k; ++s) {
      const int kl = s + ((k - 1 - s) / NST) * NST;
      if (!wait_phase(&full[s], (uint32_t)((kl / NST) & 1))) failed = true;
    }
    if (failed) atomicExch(err, 1);
    return;
  }

  // consumers: thread = (row of the tile, i1)
  const int tr = tid / n1, i1 = tid - tr * n1;
  const bool act = tr < nr;
  const int rr = r0 + tr, i3 = rr / n2, i2 = rr - i3 * n2;
  const int N = pt.N;
  float sh[NR][DIM], sl[NR][DIM];
#pragma unroll
  for (int j = 0; j < NR; ++j)
#pragma unroll
    for (int l = 0; l < DIM; ++l) sh[j][l] = sl[j][l] = 0.0f;
  int k = 0;
  bool failed = false;
  for (int r = 0; r < NROW; ++r) {
    const int m = r / (W * W3), o3 = (r / W) % W3, o2 = r % W;
    int a2, b2, a3, b3, first, last;
    bounds(o2, o3, a2, b2, a3, b3);
    if (!row_hull(r0, rl, i3a, i2a, i3b, i2b, n2, a2, b2, a3, b3, first, last)) continue;
    const int s = k % NST;
    if (!wait_phase(&full[s], (uint32_t)((k / NST) & 1))) { failed = true; break; }
    const bool rowok = act && rr >= first && rr <= last && i2 >= a2 && i2 <= b2 && i3 >= a3 && i3 <= b3;
    if (rowok) {
      const int j2 = i2 + o2 - PC, j3 = DIM == 3 ? i3 + o3 - PC : 0;
      const float2 *xm = xs + pt.off + (long long)m * N + (long long)n1 * (j2 + (long long)n2 * j3);
      const float2 *st = stage + (size_t)s * C::CH * kSlot;
      const int dr = rr - first;
#pragma unroll
      for (int o1 = 0; o1 < W; ++o1) {
        // a node without this neighbour multiplies x = 0 by a finite value
        // read at a clamped slot position
        const int j1 = i1 + o1 - PC;
        const bool in = j1 >= 0 && j1 < n1;
        const int at = min(max(((first * L.len[o1]) & 1) + dr * L.len[o1] + i1 - L.s[o1], 0), kSlot - 1);
        float2 av[DIM];
#pragma unroll
        for (int l = 0; l < DIM; ++l) av[l] = st[(l * W + o1) * kSlot + at];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (NR > 1 && j >= nrhs) break;
          const float2 xv = in ? xm[(long long)j * ndof + j1] : make_float2(0.0f, 0.0f);
#pragma unroll
          for (int l = 0; l < DIM; ++l) df_madd(sh[j][l], sl[j][l], av[l], xv);
        }
      }
#pragma unroll
      for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int l = 0; l < DIM; ++l) {   // renormalise (Fast2Sum) after each neighbour row
          const float t = __fadd_rn(sh[j][l], sl[j][l]);
          sl[j][l] = __fsub_rn(sl[j][l], __fsub_rn(t, sh[j][l]));
          sh[j][l] = t;
        }
    }
    __syncwarp();
    if (lane == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    ++k;
  }
  if (failed) {
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  if (act) {
    const int node = i1 + n1 * rr;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (NR > 1 && j >= nrhs) break;
#pragma unroll
      for (int l = 0; l < DIM; ++l)
        y[(long long)j * ystride + pt.off + (long long)l * N + node] = (double)sh[j][l] + (double)sl[j][l];
    }
  }
}

// degree shared by every patch (0: mixed)
static int uniform_degree(const afi_ctx *c) {
  int pu = c->hp[0].p;
  for (auto &p : c->hp)
    if (p.p != pu) pu = 0;
  return pu;
}

// nr right-hand sides x_j = x + j xstride, y_j = y + j ystride (nr = 1:
// the single-vector kernel; 2..kMaxRhs: the batched one)
template <int DIM, int PC>
static afi_status rows_launch(afi_ctx *c, const double *x, long long xstride, double *y,
                              long long ystride, int nr, cudaStream_t s, bool set_attr) {
  using C = RowsCfg<DIM, PC>;
  auto kern1 = k_stencil_mv_rows<DIM, PC, 1>;
  auto kern2 = k_stencil_mv_rows<DIM, PC, 2>;
  auto kern4 = k_stencil_mv_rows<DIM, PC, 4>;
  auto kern8 = k_stencil_mv_rows<DIM, PC, 8>;
  if (set_attr) {
    AFI_CUDA(cudaFuncSetAttribute(kern1, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    AFI_CUDA(cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    AFI_CUDA(cudaFuncSetAttribute(kern4, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    AFI_CUDA(cudaFuncSetAttribute(kern8, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    return AFI_OK;
  }
  auto kernm = nr <= 2 ? kern2 : (nr <= 4 ? kern4 : kern8);
  int tiles = 0;
  for (auto &p : c->hp) {
    const int R = kRowsTN / p.n[0], rows = p.n[1] * p.n[2];
    tiles = std::max(tiles, (rows + R - 1) / R);
  }
  float2 *xs = nr > 1 ? c->xsplit_multi : c->xsplit;
  launch(k_split_x_multi, dim3((unsigned)((c->n_dof + 255) / 256), nr), 256, 0, s, x, xstride, xs,
         c->n_dof, (const double *)c->gate);
  if (nr == 1)
    launch(kern1, dim3(tiles, c->npatch), kRowsTN + 32, C::SMEM, s, (const DevPatch *)c->patches,
           (const float2 *)c->stencil2, (const float2 *)xs, y, (const double *)c->gate, c->dflag + 1,
           1, c->n_dof, ystride);
  else
    launch(kernm, dim3(tiles, c->npatch), kRowsTN + 32, C::SMEM, s, (const DevPatch *)c->patches,
           (const float2 *)c->stencil2, (const float2 *)xs, y, (const double *)c->gate, c->dflag + 1,
           nr, c->n_dof, ystride);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// the instantiation for (dim, uniform degree); false if there is none
static bool rows_dispatch(afi_ctx *c, const double *x, long long xstride, double *y,
                          long long ystride, int nr, cudaStream_t s, bool set_attr, afi_status *st) {
  const int pu = uniform_degree(c);
  if (c->dim == 3) {
    switch (pu) {
      case 1: *st = rows_launch<3, 1>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
      case 2: *st = rows_launch<3, 2>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
      case 3: *st = rows_launch<3, 3>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
      case 4: *st = rows_launch<3, 4>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
      case 5: *st = rows_launch<3, 5>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
      default: return false;
    }
  }
  switch (pu) {
    case 1: *st = rows_launch<2, 1>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
    case 2: *st = rows_launch<2, 2>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
    case 3: *st = rows_launch<2, 3>(c, x, xstride, y, ystride, nr, s, set_attr); return true;
    default: return false;
  }
}

// Sizes of the pair copy (DevPatch.roff, .rstride), set on the host
// patches before they are uploaded; returns the total in pairs.
long long pair_layout(std::vector<DevPatch> &hp, int dim) {
  long long off = 0;
  for (auto &P : hp) {
    const int W = 2 * P.p + 1, rows = P.n[1] * P.n[2];
    RowLayout L;
    row_layout(P.n[0], rows, P.p, L);
    const long long last = (long long)rows * L.len[W - 1];
    P.rstride = L.cum[W - 1] + last + (last & 1);
    P.roff = off;
    off += (long long)dim * dim * (dim == 3 ? W * W : W) * P.rstride;
  }
  return off;
}

// The pair copy of the stencil: for patches of one degree up to 5 (3D; 3
// in 2D) with rows of at most 128 nodes, when it fits beside the FP64
// stencil with a tenth of the device memory to spare.  Without it every
// product is FP64.
afi_status stencil_to_pairs(afi_ctx *c) {
  if (!c->stencil || c->stencil_n == 0 || c->stencil2_n == 0) return AFI_OK;
  const int pu = uniform_degree(c);
  if (pu < 1 || pu > (c->dim == 3 ? 5 : 3)) return AFI_OK;
  for (auto &p : c->hp)
    if (p.n[0] > kRowsTN) return AFI_OK;
  size_t free_b = 0, total_b = 0;
  AFI_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t bytes = (size_t)c->stencil2_n * sizeof(float2) + (size_t)c->n_dof * sizeof(float2);
  if (free_b < bytes + total_b / 10) return AFI_OK;
  AFI_TRY(dalloc(c, (void **)&c->stencil2, (size_t)c->stencil2_n * sizeof(float2)));
  AFI_TRY(dalloc(c, (void **)&c->xsplit, (size_t)c->n_dof * sizeof(float2)));
  long long maxsz = 0;
  for (auto &p : c->hp) {
    const int W = 2 * p.p + 1;
    maxsz = std::max(maxsz, (long long)c->dim * c->dim * (c->dim == 3 ? W * W : W) * p.rstride);
  }
  dim3 g((unsigned)((maxsz + 255) / 256), c->npatch);
  if (c->dim == 3) launch(k_stencil_pack<3>, g, 256, 0, 0, (const DevPatch *)c->patches, (const double *)c->stencil, c->stencil2);
  else launch(k_stencil_pack<2>, g, 256, 0, 0, (const DevPatch *)c->patches, (const double *)c->stencil, c->stencil2);
  AFI_LAUNCH_CHECK();
  afi_status st = AFI_OK;
  rows_dispatch(c, nullptr, 0, nullptr, 0, 1, 0, true, &st);
  return st;
}

bool stiffness_has_pairs(const afi_ctx *c) { return c->stencil2 != nullptr; }

afi_status op_stiffness_fp64(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  const bool old = c->mv_exact;
  c->mv_exact = true;
  const afi_status st = op_stiffness(c, x, y, s);
  c->mv_exact = old;
  return st;
}

// y_j = A x_j for nr <= kMaxRhs vectors at the given strides: one launch of
// the batched double-FP32 kernel when the pair copy exists (the coefficients
// stream once for all of them), else one FP64 launch per vector.
static afi_status multi_launches(afi_ctx *c, const double *x, long long xstride, double *y,
                                 long long ystride, int nr, int width, cudaStream_t s) {
  for (int j = 0; j < nr; j += width) {
    afi_status st = AFI_OK;
    if (!rows_dispatch(c, x + j * xstride, xstride, y + j * ystride, ystride,
                       std::min(width, nr - j), s, false, &st)) {
      set_error("op_stiffness_multi: no batched kernel for this degree");
      return AFI_EINVAL;
    }
    AFI_TRY(st);
  }
  return AFI_OK;
}

// The number of vectors per launch of the batched kernel, chosen once per
// context by timing 8 vectors in launches of 1, 2, 4 and 8 (best of three
// after a warm-up) on scratch data: more vectors per launch share each
// coefficient but hold more accumulators per thread (fewer resident CTAs).
static afi_status tune_multi_width(afi_ctx *c, cudaStream_t s) {
  if (c->mv_width > 0) return AFI_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  AFI_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) { c->mv_width = kMaxRhs; return AFI_OK; }
  double *buf = nullptr;
  AFI_TRY(dalloc(c, (void **)&buf, (size_t)2 * kMaxRhs * c->n_dof * sizeof(double)));
  AFI_CUDA(cudaMemsetAsync(buf, 0, (size_t)2 * kMaxRhs * c->n_dof * sizeof(double), s));
  cudaEvent_t e0, e1;
  AFI_CUDA(cudaEventCreate(&e0));
  AFI_CUDA(cudaEventCreate(&e1));
  const double *gate = c->gate;
  c->gate = nullptr;
  afi_status st = AFI_OK;
  float best = 1e30f;
  int bw = kMaxRhs;
  for (int w : {1, 2, 4, 8}) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 4 && st == AFI_OK; ++rep) {
      cudaEventRecord(e0, s);
      st = multi_launches(c, buf, c->n_dof, buf + (long long)kMaxRhs * c->n_dof, c->n_dof,
                          kMaxRhs, w, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    if (tmin < best) { best = tmin; bw = w; }
  }
  c->gate = gate;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  c->bytes -= (long long)2 * kMaxRhs * c->n_dof * sizeof(double);
  AFI_TRY(st);
  c->mv_width = bw;
  return AFI_OK;
}

// Buffers and launch width of the batched stiffness, set up before any
// stream capture.
afi_status stiffness_multi_prepare(afi_ctx *c, cudaStream_t s) {
  if (!c->stencil2 || uniform_degree(c) == 0) return AFI_OK;
  if (!c->xsplit_multi)
    AFI_TRY(dalloc(c, (void **)&c->xsplit_multi, (size_t)kMaxRhs * c->n_dof * sizeof(float2)));
  return tune_multi_width(c, s);
}

afi_status op_stiffness_multi(afi_ctx *c, const double *x, long long xstride, double *y,
                              long long ystride, int nr, cudaStream_t s) {
  if (nr < 1 || nr > kMaxRhs) { set_error("op_stiffness_multi: bad batch"); return AFI_EINVAL; }
  if (c->stencil2 && !c->mv_exact && nr > 1 && uniform_degree(c) > 0) {
    if (!c->xsplit_multi)
      AFI_TRY(dalloc(c, (void **)&c->xsplit_multi, (size_t)kMaxRhs * c->n_dof * sizeof(float2)));
    AFI_TRY(tune_multi_width(c, s));
    return multi_launches(c, x, xstride, y, ystride, nr, c->mv_width, s);
  }
  for (int j = 0; j < nr; ++j) AFI_TRY(op_stiffness(c, x + j * xstride, y + j * ystride, s));
  return AFI_OK;
}

afi_status op_stiffness(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  if (c->mf)
    return mf_stiffness(c, x, y, c->mv_exact || (c->opt.variant & AFI_VARIANT_STENCIL_F64), s);
  if (c->stencil2 && !c->mv_exact) {
    afi_status st = AFI_OK;
    if (rows_dispatch(c, x, 0, y, 0, 1, s, false, &st)) return st;
  }
  dim3 g((c->max_N + 127) / 128, c->npatch);
  const int pu = uniform_degree(c);   // one degree for every patch -> specialised kernel
  const double *A = c->stencil;
  const DevPatch *P = c->patches;
#define AFI_MV(D, PC) launch(k_stencil_mv<D, PC>, g, 128, 0, s, P, A, x, y, c->gate)
  if (c->dim == 3) {
    switch (pu) {
      case 1: AFI_MV(3, 1); break;
      case 2: AFI_MV(3, 2); break;
      case 3: AFI_MV(3, 3); break;
      case 4: AFI_MV(3, 4); break;
      case 5: AFI_MV(3, 5); break;
      default: AFI_MV(3, 0);
    }
  } else {
    switch (pu) {
      case 1: AFI_MV(2, 1); break;
      case 2: AFI_MV(2, 2); break;
      case 3: AFI_MV(2, 3); break;
      default: AFI_MV(2, 0);
    }
  }
#undef AFI_MV
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

}  // namespace afi
