// Stiffness matvec y = A x (eqs. 3.1, 4.2) from the assembled per-node
// stencil A[l][m][o][node] over the (2p+1)^d neighbour offsets o, in three
// forms:
//  * k_stencil_mv: FP64 coefficients and FMAs (AFI_VARIANT_STENCIL_F64);
//  * k_stencil_mv_bulk: (hi, lo) FP32-pair coefficients in double-FP32
//    arithmetic, the coefficient planes of a tile of nodes streamed into
//    shared memory by bulk (TMA) copies through a ring of mbarrier stages;
//  * k_stencil_mv_df: the same arithmetic with plain loads, for patches of
//    mixed degree.
#include "tc.cuh"

#include <algorithm>

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
// HBM.  In the default form every coefficient a is held, in the same 8
// bytes, as the unevaluated sum of two FP32 numbers, hi = rn(a) and
// lo = rn(a - hi), so |a - hi - lo| <= 2^-48 |a| (Dekker's double-length
// representation); x is split the same way by k_split_x.  A product
// a x = hi_a hi_x + e + hi_a lo_x + lo_a hi_x (+ lo_a lo_x, dropped) takes
// its rounding error e exactly from an FMA; each addition of hi_a hi_x to the
// running sum is made error free by Knuth's TwoSum, and the addition errors,
// e and the cross terms collect in a second FP32 sum.  The result is the
// FP64 value hi + lo.  Twelve FP32 operations per coefficient (and a
// renormalisation per neighbour row) leave the product bound by HBM.  Values
// must stay within the FP32 range.

__global__ void k_stencil_split(double *A, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = A[i];
  const float hi = __double2float_rn(a);
  const float lo = __double2float_rn(a - (double)hi);
  reinterpret_cast<float2 *>(A)[i] = make_float2(hi, lo);   // same 8 bytes, in place
}

__global__ void k_split_x(const double *__restrict__ x, float2 *__restrict__ xs, long n, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float hi = __double2float_rn(v);
  xs[i] = make_float2(hi, __double2float_rn(v - (double)hi));
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

// The loop nest of k_stencil_mv with (hi, lo) coefficients and inputs.
template <int DIM, int PC>
__global__ void __launch_bounds__(128) k_stencil_mv_df(const DevPatch *P, const float2 *__restrict__ A,
                                                       const float2 *__restrict__ xs,
                                                       double *__restrict__ y, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const DevPatch pt = P[blockIdx.y];
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= pt.N) return;
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2], p = PC > 0 ? PC : pt.p;
  const int i1 = node % n1, i2 = (node / n1) % n2, i3 = node / (n1 * n2);
  const int W1 = PC > 0 ? 2 * PC + 1 : pt.W[0], W2 = PC > 0 ? 2 * PC + 1 : pt.W[1];
  const int W3 = (DIM == 3) ? W2 : 1;
  float sh[DIM], sl[DIM];
#pragma unroll
  for (int l = 0; l < DIM; ++l) sh[l] = sl[l] = 0.0f;
  const long long N = pt.N, S = pt.S, NP = pt.NP;
  const float2 *Ab = A + pt.soff + i1 + (long long)pt.n1p * (i2 + (long long)n2 * i3);
  for (int m = 0; m < DIM; ++m) {
    const float2 *xm = xs + pt.off + m * N;
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
          const float2 xv = (j1 >= 0 && j1 < n1) ? xm[jrow + j1] : make_float2(0.0f, 0.0f);
          const long long o = orow + o1;
#pragma unroll
          for (int l = 0; l < DIM; ++l) df_madd(sh[l], sl[l], Ab[((long long)(l * DIM + m) * S + o) * NP], xv);
        }
        // renormalise after each neighbour row (Fast2Sum): sl stays within
        // one FP32 ulp of sh, so the additions to sl keep their precision
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
          const float t = __fadd_rn(sh[l], sl[l]);
          sl[l] = __fsub_rn(sl[l], __fsub_rn(t, sh[l]));
          sh[l] = t;
        }
      }
    }
  }
  for (int l = 0; l < DIM; ++l) y[pt.off + l * N + node] = (double)sh[l] + (double)sl[l];
}

// ------------------------------- double-FP32 matvec, bulk-copy pipeline
// One CTA per tile of TN consecutive positions of a patch's padded stencil
// plane (position = i1 + n1p (i2 + n2 i3); threads on row padding idle), one
// thread per position, plus a producer warp.  A stage is one neighbour row
// (m, o3, o2): the DIM x W coefficient planes (l, o1) of the tile, TN pairs
// of 8 bytes each, arrive by one bulk copy per plane; the consumers add their
// W x DIM products, release the stage and move on.  The copies of the next
// NST - 1 rows are in flight meanwhile, so the coefficient stream does not
// depend on how many loads a thread keeps in registers.  Rows that lie
// outside the patch for every node of the tile are neither copied nor
// visited (producer and consumers decide that from the tile's extent alone).
// Every mbarrier wait is bounded; a wait that runs out sets *err, and the
// producer waits (bounded) for the copies it issued before the CTA exits.
template <int DIM, int PC, int TN>
struct BulkCfg {
  static constexpr int W = 2 * PC + 1;
  static constexpr int W3 = DIM == 3 ? W : 1;
  static constexpr int NROW = DIM * W * W3;   // stages of a tile: (m, o3, o2)
  static constexpr int CH = DIM * W;          // copies per stage: (l, o1)
  static constexpr int STAGE = CH * TN * 8;   // bytes per stage
  static constexpr int NST0 = 65536 / STAGE;
  static constexpr int NST = NST0 < 2 ? 2 : (NST0 > 6 ? 6 : NST0);
  static constexpr int SMEM = NST * STAGE;
};

template <int DIM, int PC, int TN>
__global__ void __launch_bounds__(TN + 32) k_stencil_mv_bulk(const DevPatch *P, const float2 *__restrict__ A,
                                                            const float2 *__restrict__ xs,
                                                            double *__restrict__ y, const double *gate,
                                                            int *err) {
  using C = BulkCfg<DIM, PC, TN>;
  constexpr int W = C::W, W3 = C::W3, NROW = C::NROW, NST = C::NST;
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  extern __shared__ __align__(128) unsigned char sm_raw[];
  float2 *stage = reinterpret_cast<float2 *>(sm_raw);   // [NST][DIM][W][TN]
  __shared__ uint64_t full[NST], empty[NST];
  const DevPatch pt = P[blockIdx.y];
  const int base = blockIdx.x * TN;
  if (base >= pt.NP) return;   // the whole CTA: the grid covers the largest patch
  const int tid = threadIdx.x, lane = tid & 31;
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2], n1p = pt.n1p;
  const int npos = min(TN, pt.NP - base);   // even: NP and TN are even
  const int last = base + npos - 1;
  const int i3lo = base / (n1p * n2), i3hi = last / (n1p * n2);
  const int i2lo = (base / n1p) % n2, i2hi = (last / n1p) % n2;
  // is neighbour row (o2, o3) inside the patch for some node of the tile?
  auto needed = [&](int o2, int o3) {
    if (DIM == 3) {
      if (i3hi + o3 - PC < 0 || i3lo + o3 - PC >= n3) return false;
      if (i3lo != i3hi) return true;
    }
    return !(i2hi + o2 - PC < 0 || i2lo + o2 - PC >= n2);
  };
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(TN / 32));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();

  if (tid >= TN) {   // producer warp: one lane issues every copy
    if (lane != 0) return;
    const long long NP = pt.NP, S = pt.S;
    const float2 *Ab = A + pt.soff + base;
    const uint32_t bytes = (uint32_t)npos * 8u;
    int k = 0;
    bool failed = false;
    for (int r = 0; r < NROW; ++r) {
      const int m = r / (W * W3), o3 = (r / W) % W3, o2 = r % W;
      if (!needed(o2, o3)) continue;
      const int s = k % NST;
      if (k >= NST && !wait_phase(&empty[s], (uint32_t)((k / NST - 1) & 1))) { failed = true; break; }
      expect_tx(&full[s], bytes * C::CH);
      const int orow = W * (o2 + W * o3);
      float2 *dst = stage + (size_t)s * C::CH * TN;
#pragma unroll
      for (int l = 0; l < DIM; ++l)
#pragma unroll
        for (int o1 = 0; o1 < W; ++o1)
          bulk_g2s(dst + (l * W + o1) * TN, Ab + ((long long)(l * DIM + m) * S + orow + o1) * NP, bytes,
                   &full[s]);
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

  // consumers
  const int pos = base + tid;
  const int i1 = pos % n1p, i2 = (pos / n1p) % n2, i3 = pos / (n1p * n2);
  const bool act = tid < npos && i1 < n1;
  const int N = pt.N;
  float sh[DIM], sl[DIM];
#pragma unroll
  for (int l = 0; l < DIM; ++l) sh[l] = sl[l] = 0.0f;
  int k = 0;
  bool failed = false;
  for (int r = 0; r < NROW; ++r) {
    const int m = r / (W * W3), o3 = (r / W) % W3, o2 = r % W;
    if (!needed(o2, o3)) continue;
    const int s = k % NST;
    if (!wait_phase(&full[s], (uint32_t)((k / NST) & 1))) { failed = true; break; }
    const int j2 = i2 + o2 - PC, j3 = DIM == 3 ? i3 + o3 - PC : 0;
    const bool rowok = act && j2 >= 0 && j2 < n2 && j3 >= 0 && j3 < n3;
    const float2 *xm = xs + pt.off + (long long)m * N + (long long)n1 * (j2 + (long long)n2 * j3);
    const float2 *st = stage + (size_t)s * C::CH * TN + tid;
#pragma unroll
    for (int o1 = 0; o1 < W; ++o1) {
      const int j1 = i1 + o1 - PC;
      const float2 xv = (rowok && j1 >= 0 && j1 < n1) ? xm[j1] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int l = 0; l < DIM; ++l) df_madd(sh[l], sl[l], st[(l * W + o1) * TN], xv);
    }
#pragma unroll
    for (int l = 0; l < DIM; ++l) {   // renormalise (Fast2Sum), as in k_stencil_mv_df
      const float t = __fadd_rn(sh[l], sl[l]);
      sl[l] = __fsub_rn(sl[l], __fsub_rn(t, sh[l]));
      sh[l] = t;
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
    const int node = i1 + n1 * (i2 + n2 * i3);
#pragma unroll
    for (int l = 0; l < DIM; ++l) y[pt.off + (long long)l * N + node] = (double)sh[l] + (double)sl[l];
  }
}

constexpr int kBulkTN = 128;

// degree shared by every patch (0: mixed)
static int uniform_degree(const afi_ctx *c) {
  int pu = c->hp[0].p;
  for (auto &p : c->hp)
    if (p.p != pu) pu = 0;
  return pu;
}

template <int DIM, int PC>
static afi_status bulk_launch(afi_ctx *c, const double *x, double *y, cudaStream_t s, bool set_attr) {
  using C = BulkCfg<DIM, PC, kBulkTN>;
  auto kern = k_stencil_mv_bulk<DIM, PC, kBulkTN>;
  if (set_attr) {
    AFI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    return AFI_OK;
  }
  int maxNP = 0;
  for (auto &p : c->hp) maxNP = std::max(maxNP, p.NP);
  launch(k_split_x, (unsigned)((c->n_dof + 255) / 256), 256, 0, s, x, c->xsplit, c->n_dof,
         (const double *)c->gate);
  dim3 g((maxNP + kBulkTN - 1) / kBulkTN, c->npatch);
  launch(kern, g, kBulkTN + 32, C::SMEM, s, (const DevPatch *)c->patches,
         reinterpret_cast<const float2 *>(c->stencil), (const float2 *)c->xsplit, y,
         (const double *)c->gate, c->dflag + 1);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// the bulk-pipeline instantiation for (dim, uniform degree); false if none
static bool bulk_dispatch(afi_ctx *c, const double *x, double *y, cudaStream_t s, bool set_attr,
                          afi_status *st) {
  const int pu = uniform_degree(c);
  if (c->dim == 3) {
    switch (pu) {
      case 1: *st = bulk_launch<3, 1>(c, x, y, s, set_attr); return true;
      case 2: *st = bulk_launch<3, 2>(c, x, y, s, set_attr); return true;
      case 3: *st = bulk_launch<3, 3>(c, x, y, s, set_attr); return true;
      case 4: *st = bulk_launch<3, 4>(c, x, y, s, set_attr); return true;
      case 5: *st = bulk_launch<3, 5>(c, x, y, s, set_attr); return true;
      default: return false;
    }
  }
  switch (pu) {
    case 1: *st = bulk_launch<2, 1>(c, x, y, s, set_attr); return true;
    case 2: *st = bulk_launch<2, 2>(c, x, y, s, set_attr); return true;
    case 3: *st = bulk_launch<2, 3>(c, x, y, s, set_attr); return true;
    default: return false;
  }
}

afi_status stencil_to_pairs(afi_ctx *c) {
  if (!c->stencil || c->stencil_n == 0) return AFI_OK;
  launch(k_stencil_split, (unsigned)((c->stencil_n + 255) / 256), 256, 0, 0, c->stencil, c->stencil_n);
  AFI_LAUNCH_CHECK();
  afi_status st = AFI_OK;
  bulk_dispatch(c, nullptr, nullptr, 0, true, &st);
  if (st != AFI_OK) return st;
  c->stencil_pairs = true;
  return AFI_OK;
}

afi_status op_stiffness(afi_ctx *c, const double *x, double *y, cudaStream_t s) {
  dim3 g((c->max_N + 127) / 128, c->npatch);
  const int pu = uniform_degree(c);   // one degree for every patch -> specialised kernel
  const double *A = c->stencil;
  const DevPatch *P = c->patches;
  if (c->stencil_pairs) {
    afi_status st = AFI_OK;
    if (bulk_dispatch(c, x, y, s, false, &st)) return st;
    launch(k_split_x, (unsigned)((c->n_dof + 255) / 256), 256, 0, s, x, c->xsplit, c->n_dof,
           (const double *)c->gate);
    const float2 *A2 = reinterpret_cast<const float2 *>(A), *xs = c->xsplit;
    if (c->dim == 3) launch(k_stencil_mv_df<3, 0>, g, 128, 0, s, P, A2, xs, y, (const double *)c->gate);
    else launch(k_stencil_mv_df<2, 0>, g, 128, 0, s, P, A2, xs, y, (const double *)c->gate);
    AFI_LAUNCH_CHECK();
    return AFI_OK;
  }
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
