// Fast diagonalization (Algorithm 1, eqs. 5.6, 5.9, 5.10) on tcgen05 tensor
// cores for tensors too large for one CTA's shared memory.  The six mode
// products are grouped into three passes over an FP32 scratch copy of the
// tensor X[i3][i2][i1]:
//
//   pass A (k_fd_plane<.., 0>): for a group of consecutive i3 planes, the
//     products with U_1^T and U_2^T (both in one CTA, shared memory between
//     them); reads FP64, writes FP32;
//   pass B (k_fd_line): for a tile of 128 (a1, a2) lines, the product with
//     U_3^T along i3, the scaling by Lambda^{-1}, and the product with U_3,
//     in place in the scratch;
//   pass C (k_fd_plane<.., 1>): for a group of planes, the products with U_1
//     and U_2; reads FP32, writes FP64.
//
// Every pass reads and writes whole rows of 128-byte sectors, so the traffic
// is 8 + 4 + 4 + 4 + 4 + 8 = 32 bytes per DoF (TF32/BF16 operands, FP32
// scratch) against the 16 of a single-pass kernel.  Each MMA is a GEMM
// D[line][j] = sum_k A[line][k] B[j][k] with the tensor as the K-major A
// operand (lines on the 128 TMEM lanes, one slab per 16-byte K chunk with
// rows 16 bytes apart) and U^T or U as B, staged by TMA.  Each CTA works
// through a short range of the pass's work list (about two items, ranges of
// equal cost), allocating tensor memory, initialising its barriers and
// loading the B operands once per range; one thread issues and waits for
// the MMAs while the others wait at the CTA barrier.
#include "tc.cuh"

#include <algorithm>
#include <type_traits>

namespace afi {

using namespace tc;

namespace {

// Issue the MMAs of one product: ntile tiles of 128 lines of the tensor
// operand A (K-major, one slab per 16-byte K chunk: rows 16 bytes apart,
// chunks lbo bytes apart), against the canonical B operand (Np x Kp) at b,
// accumulating into TMEM columns t * Np.
template <int FMT>
__device__ __forceinline__ void issue_product(uint32_t tmem, const void *A, const void *B, int ntile,
                                              int Kp, int Np, uint32_t lbo) {
  constexpr int KSTEP = Op<FMT>::KSTEP, T16 = Op<FMT>::T16;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t id = idesc(FMT, 128, Np);
  const uint32_t sboB = (uint32_t)(Kp / T16) * 128u;
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
  for (int t = 0; t < ntile; ++t)
    for (int ks = 0; ks < Kp / KSTEP; ++ks)
      mma<FMT>(tmem + (uint32_t)(t * Np), sdesc(a0 + t * 2048u + ks * 2u * lbo, lbo, 128u),
               sdesc(b0 + ks * 256, 128, sboB), id, ks > 0 ? 1u : 0u);
}

// Stage the B operands of two products (prebuilt canonical layout in
// tcpool) into slots bm and bm + bsz.
template <typename T>
__device__ __forceinline__ void stage_b(uint64_t *bar, T *bm, int bsz, const unsigned char *tcpool,
                                        long long off0, uint32_t bytes0, long long off1,
                                        uint32_t bytes1) {
  expect_tx(bar, bytes0 + bytes1);
  bulk_g2s(bm, tcpool + off0, bytes0, bar);
  bulk_g2s(bm + bsz, tcpool + off1, bytes1, bar);
}

// four consecutive inputs (16-byte aligned) as FP32
__device__ __forceinline__ void ld4(const double *p, float *v) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
  v[0] = f64_to_op(a.x); v[1] = f64_to_op(a.y); v[2] = f64_to_op(b.x); v[3] = f64_to_op(b.y);
}
__device__ __forceinline__ void ld4(const float *p, float *v) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
// two consecutive inputs (aligned to their pair size) as FP32
__device__ __forceinline__ void ld2(const double *p, float *v) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  v[0] = f64_to_op(a.x); v[1] = f64_to_op(a.y);
}
__device__ __forceinline__ void ld2(const float *p, float *v) {
  const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ float ld_in(const double *p) { return f64_to_op(__ldg(p)); }
__device__ __forceinline__ float ld_in(const float *p) { return __ldg(p); }
__device__ __forceinline__ void st_out(double *p, float v) { *p = f32_to_f64(v); }
__device__ __forceinline__ void st_out(float *p, float v) { *p = v; }

}  // namespace

// Passes A (BACK = 0: U_1^T then U_2^T, FP64 in, FP32 out) and C (BACK = 1:
// U_1 then U_2, FP32 in, FP64 out).  Work items (patch, first plane, nz
// planes) of one component (blockIdx.y) and right-hand side (blockIdx.z); a
// CTA takes the items [bounds[x], bounds[x + 1]) (ranges of equal cost) and
// keeps its tensor memory, barriers and, while the tables stay the same, its
// B operands from one item to the next.
template <int FMT, int BACK>
__global__ void __launch_bounds__(256, 3) k_fd_plane(const DevPatch *P, const Tab1D *tabs,
                                                     const int4 *work, const int *bounds,
                                                     int interior, const double *r, float *scr,
                                                     double *s, long long rhs_stride, int cap,
                                                     int bsz, int tcols, const double *gate,
                                                     int *err, const unsigned char *tcpool) {
  using T = typename Op<FMT>::T;
  using TIn = typename std::conditional<BACK == 0, double, float>::type;
  constexpr int KSTEP = Op<FMT>::KSTEP, T16 = Op<FMT>::T16;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  T *A = reinterpret_cast<T *>(smraw);
  T *bm = A + cap;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double gv = gate ? *gate : 1.0;
  const int w0 = bounds[blockIdx.x], w1 = bounds[blockIdx.x + 1];
  const int l = blockIdx.y;
  if (gv == 0.0 || w0 >= w1) return;   // inactive MINRES iteration / empty range

  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tma_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const int q = warp & 3, half = warp >> 2;
  int key = -1;            // tables of the B operands held in shared memory
  uint32_t tma_phase = 0;

  for (int wi = w0; wi < w1; ++wi) {
    const int4 w = work[wi];
    const DevPatch &pg = P[w.x];
    const int n1 = interior ? pg.ni[0] : pg.n[0], n2 = interior ? pg.ni[1] : pg.n[1];
    const int n3 = interior ? pg.ni[2] : pg.n[2];
    const int z0 = w.y, nz = w.z;
    const long long plane = (long long)n1 * n2;
    const long long base = (interior ? pg.ioff : pg.off) + (long long)l * plane * n3 +
                           (long long)blockIdx.z * rhs_stride + z0 * plane;
    const TIn *in = BACK ? (const TIn *)(const void *)(scr + base) : (const TIn *)(const void *)(r + base);
    // this component's tables, read from global memory (a runtime index
    // into a local copy would move it to local memory)
    const int lt0 = pg.ltab[l][0], lt1 = pg.ltab[l][1];
    const int slot1 = (lt0 == lt1) ? 0 : 1;
    const int nkey = lt0 * 65536 + lt1;
    const bool reload = nkey != key;
    if (reload && tid == 0) {   // both products use one slot when the tables agree
      const uint32_t b0 = (uint32_t)(rup(n1, 16) * rup(n1, KSTEP) * (int)sizeof(T));
      const uint32_t b1 = (uint32_t)(rup(n2, 16) * rup(n2, KSTEP) * (int)sizeof(T));
      expect_tx(&tma_bar, slot1 ? b0 + b1 : b0);
      bulk_g2s(bm, tcpool + tabs[lt0].tcB[FMT == 1][interior][BACK], b0, &tma_bar);
      if (slot1) bulk_g2s(bm + bsz, tcpool + tabs[lt1].tcB[FMT == 1][interior][BACK], b1, &tma_bar);
    }
    // a fresh zero operand per item: no value of the previous item (a NaN
    // included) may reach this item's K padding
    {
      uint4 *zp = reinterpret_cast<uint4 *>(A);
      const int nzero = cap * (int)sizeof(T) / 16;
      for (int i = tid; i < nzero; i += 256) zp[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    // first operand: row = i2 + n2 * zl, k = i1 (the slice is contiguous)
    const int lbo0 = (rup(n2 * nz, 128) + 1) * T16, N = (int)(plane * nz);
    const float inv = 1.0f / (float)n1;
    if ((n1 & 3) == 0 && ((uintptr_t)in & 15) == 0) {
      // four consecutive i1 of one row per thread: 16-byte global loads and
      // one 16-byte (TF32) or 8-byte (BF16) shared store
      constexpr int LB = 4;
      const int N4 = N >> 2;
      for (int g0 = tid; g0 < N4; g0 += LB * 256) {
        float v[LB][4];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int g = g0 + u * 256;
          if (g < N4) ld4(in + 4 * g, v[u]);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int g = g0 + u * 256;
          if (g < N4) {
            const int idx = 4 * g;
            const int row = __float2int_rz(__fmul_rn(__fadd_rn((float)idx, 0.5f), inv));
            st4<FMT>(&A[kslab<FMT>(row, idx - row * n1, lbo0)], v[u]);
          }
        }
      }
    } else if ((n1 & 1) == 0 && ((uintptr_t)in & (2 * sizeof(TIn) - 1)) == 0) {
      // two consecutive i1 of one row per thread (even rows): 2-element
      // global loads and one 8-byte (TF32) or 4-byte (BF16) shared store
      constexpr int LB = 4;
      const int N2 = N >> 1;
      for (int g0 = tid; g0 < N2; g0 += LB * 256) {
        float v[LB][2];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int g = g0 + u * 256;
          if (g < N2) ld2(in + 2 * g, v[u]);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int g = g0 + u * 256;
          if (g < N2) {
            const int idx = 2 * g;
            const int row = __float2int_rz(__fmul_rn(__fadd_rn((float)idx, 0.5f), inv));
            st2<FMT>(&A[kslab<FMT>(row, idx - row * n1, lbo0)], v[u]);
          }
        }
      }
    } else {
      constexpr int LB = 8;
      for (int i0 = tid; i0 < N; i0 += LB * 256) {
        float v[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int idx = i0 + u * 256;
          v[u] = idx < N ? ld_in(in + idx) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int idx = i0 + u * 256;
          if (idx < N) {
            const int row = __float2int_rz(__fmul_rn(__fadd_rn((float)idx, 0.5f), inv));
            A[kslab<FMT>(row, idx - row * n1, lbo0)] = Op<FMT>::cvt(v[u]);
          }
        }
      }
    }
    if (reload) {   // the B operands have landed
      if (tid == 0 && !wait_phase_backoff(&tma_bar, tma_phase)) failed = 1;
      tma_phase ^= 1u;
      key = nkey;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (failed) break;

    for (int m = 0; m < 2; ++m) {
      const int na = m ? n2 : n1, nb = m ? n1 : n2;   // contracted size, other in-plane size
      const int L = nb * nz, ntile = rup(L, 128) / 128;
      const int Kp = rup(na, KSTEP), Np = rup(na, 16);
      // one thread issues the MMAs and waits for them (two commits per item:
      // phase parity m); the others wait at the CTA barrier
      if (tid == 0 && !failed) {
        issue_product<FMT>(tmem, A, bm + (m ? slot1 : 0) * bsz, ntile, Kp, Np,
                           (uint32_t)(ntile * 128 + 1) * 16u);
        commit(&mbar);
        if (!wait_phase_backoff(&mbar, (uint32_t)m)) failed = 1;
        asm volatile("tcgen05.fence::before_thread_sync;");
      }
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (failed) break;
      // m = 0: D[line = i2 + n2 zl][j = a1] -> A[row = a1 + n1 zl][k = i2]
      // m = 1: D[line = a1 + n1 zl][j = a2] -> out[zl][a2][a1]
      // items (t, ch) = (it / nch, it % nch), it = half, half + 2, ...; the
      // lane's line = b + nb zl is stepped without divisions
      const int lbo1 = (rup(n1 * nz, 128) + 1) * T16;
      const int nch = (na + 7) >> 3;
      int t = 0, ch = half;
      while (ch >= nch) { ch -= nch; ++t; }
      int line = t * 128 + q * 32 + lane;
      int zl = line / nb, b = line - zl * nb;
      const int dq = 128 / nb, dr = 128 - dq * nb;
      while (t < ntile) {
        const int j0 = ch * 8;
        uint32_t raw[8];
        ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * Np + j0), raw);
        ld_wait();
        if (line < L) {
          const int jn = min(8, na - j0);
          if (m == 0) {
            T *dst = A + kslab<FMT>(j0 + n1 * zl, b, lbo1);
            if (jn == 8) {   // a full chunk: no per-column predicate
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) dst[jj * T16] = Op<FMT>::cvt(__uint_as_float(raw[jj]));
            } else {
#pragma unroll
              for (int jj = 0; jj < 8; ++jj)
                if (jj < jn) dst[jj * T16] = Op<FMT>::cvt(__uint_as_float(raw[jj]));
            }
          } else {
            const long long ob = base + (long long)zl * plane + b + (long long)j0 * n1;
            if (jn == 8) {
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                if (BACK) st_out(s + ob + (long long)jj * n1, __uint_as_float(raw[jj]));
                else st_out(scr + ob + (long long)jj * n1, __uint_as_float(raw[jj]));
              }
            } else {
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                if (jj < jn) {
                  if (BACK) st_out(s + ob + (long long)jj * n1, __uint_as_float(raw[jj]));
                  else st_out(scr + ob + (long long)jj * n1, __uint_as_float(raw[jj]));
                }
              }
            }
          }
        }
        ch += 2;
        while (ch >= nch) {   // next tile: line += 128
          ch -= nch;
          ++t;
          line += 128;
          zl += dq;
          b += dr;
          if (b >= nb) { b -= nb; ++zl; }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
    if (failed) break;
  }
  if (failed) {   // one more bounded wait for MMAs in flight before freeing TMEM
    if (tid == 0)
      for (int ph = 0; ph < 2; ++ph) wait_phase(&mbar, (uint32_t)ph);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
  if (tid == 0 && failed) atomicExch(err, 1);
}

// Pass B: for 128 consecutive lines (a1 + n1 a2) of one tensor in the FP32
// scratch, t = U_3^T x along i3, t /= Lambda, x = U_3 t, in place.  Work
// items (patch, first line) of one component (blockIdx.y) and right-hand
// side (blockIdx.z); a CTA takes the items [bounds[x], bounds[x + 1]) and
// keeps its tensor memory, barriers and, while the table stays the same, its
// B operands.
template <int FMT>
__global__ void __launch_bounds__(256, 3) k_fd_line(const DevPatch *P, const Tab1D *tabs,
                                                    const float *fpool, const int2 *work,
                                                    const int *bounds, int interior, float *scr,
                                                    long long rhs_stride, int cap, int bsz,
                                                    int tcols, const double *gate, int *err,
                                                    const unsigned char *tcpool) {
  using T = typename Op<FMT>::T;
  constexpr int KSTEP = Op<FMT>::KSTEP, T16 = Op<FMT>::T16;
  constexpr int lbo = 129 * T16;   // one 128-line tile: K chunks (128 + 1) x 16 bytes apart
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  T *A = reinterpret_cast<T *>(smraw);
  T *bm = A + cap;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double gv = gate ? *gate : 1.0;
  const int w0 = bounds[blockIdx.x], w1 = bounds[blockIdx.x + 1];
  const int l = blockIdx.y;
  if (gv == 0.0 || w0 >= w1) return;   // inactive MINRES iteration / empty range

  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tma_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const int q = warp & 3, half = warp >> 2;
  const int row = q * 32 + lane;
  int key = -1;            // table of the B operands held in shared memory
  uint32_t tma_phase = 0;

  for (int wi = w0; wi < w1; ++wi) {
    const int2 w = work[wi];
    const DevPatch &pg = P[w.x];   // component-indexed fields straight from global memory
    const int n1 = interior ? pg.ni[0] : pg.n[0], n2 = interior ? pg.ni[1] : pg.n[1];
    const int n3 = interior ? pg.ni[2] : pg.n[2];
    const int LN = n1 * n2, line0 = w.y, nl = min(128, LN - line0);
    float *X = scr + (interior ? pg.ioff : pg.off) + (long long)l * LN * n3 +
               (long long)blockIdx.z * rhs_stride + line0;
    const int t0 = pg.ltab[l][0], t1 = pg.ltab[l][1], t2 = pg.ltab[l][2];
    const bool reload = t2 != key;
    const uint32_t bbytes = (uint32_t)(rup(n3, 16) * rup(n3, KSTEP) * (int)sizeof(T));
    if (reload && tid == 0) {
      const Tab1D &tb = tabs[t2];
      stage_b(&tma_bar, bm, bsz, tcpool, tb.tcB[FMT == 1][interior][0], bbytes,
              tb.tcB[FMT == 1][interior][1], bbytes);
    }
    {   // a fresh zero operand per item (no value of the previous item may reach the K padding)
      uint4 *zp = reinterpret_cast<uint4 *>(A);
      const int nzero = cap * (int)sizeof(T) / 16;
      for (int i = tid; i < nzero; i += 256) zp[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int Kp = rup(n3, KSTEP), Np = rup(n3, 16);
    // operand: row = line (128), k = i3
    if ((LN & 3) == 0 && ((uintptr_t)X & 15) == 0) {
      // aligned planes: a lane moves 4 consecutive lines of one plane with a
      // 16-byte load (a warp: 16 lines x 8 planes per instruction)
      const int l4 = lane & 3, k8 = lane >> 2;
      const int nk8 = (n3 + 7) / 8, nitem = 8 * nk8;
      constexpr int LB = 4;
      for (int i0 = warp; i0 < nitem; i0 += 8 * LB) {
        float v[LB][4];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int it = i0 + u * 8;
          const int rg = it % 8, kg = it / 8;
          const int r0 = rg * 16 + l4 * 4, k = kg * 8 + k8;
          const bool in = it < nitem && k < n3;
          if (in && r0 + 3 < nl) {
            ld4(X + (long long)k * LN + r0, v[u]);
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              v[u][e] = (in && r0 + e < nl) ? __ldg(X + (long long)k * LN + r0 + e) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int it = i0 + u * 8;
          const int rg = it % 8, kg = it / 8;
          const int r0 = rg * 16 + l4 * 4, k = kg * 8 + k8;
          if (it < nitem && k < n3)
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (r0 + e < nl) A[kslab<FMT>(r0 + e, k, lbo)] = Op<FMT>::cvt(v[u][e]);
        }
      }
    } else {
      const int r8 = lane & 7, k4 = lane >> 3;
      const int nk4 = (n3 + 3) / 4, nitem = 16 * nk4;
      constexpr int LB = 8;
      for (int i0 = warp; i0 < nitem; i0 += 8 * LB) {
        float v[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int it = i0 + u * 8;
          const int rg = it % 16, kg = it / 16;
          const int r0 = rg * 8 + r8, k = kg * 4 + k4;
          v[u] = (it < nitem && r0 < nl && k < n3) ? __ldg(X + (long long)k * LN + r0) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int it = i0 + u * 8;
          const int rg = it % 16, kg = it / 16;
          const int r0 = rg * 8 + r8, k = kg * 4 + k4;
          if (it < nitem && r0 < nl && k < n3) A[kslab<FMT>(r0, k, lbo)] = Op<FMT>::cvt(v[u]);
        }
      }
    }
    if (reload) {   // the B operands have landed
      if (tid == 0 && !wait_phase_backoff(&tma_bar, tma_phase)) failed = 1;
      tma_phase ^= 1u;
      key = t2;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (failed) break;
    // Lambda = c1 D1[a1] + c2 D2[a2] + c3 D3[a3] (+ shift, times H^{d-2}, for P_A)
    const float hs = interior ? 1.f : (float)pg.lscale, shf = interior ? 0.f : (float)pg.lshift;
    const float c0 = (float)pg.lcf[l][0], c1 = (float)pg.lcf[l][1], c2 = (float)pg.lcf[l][2];
    const float *D0 = fpool + (interior ? tabs[t0].Di : tabs[t0].D);
    const float *D1 = fpool + (interior ? tabs[t1].Di : tabs[t1].D);
    const float *D2 = fpool + (interior ? tabs[t2].Di : tabs[t2].D);
    float lab = 0.f;
    if (row < nl) {
      const int ln = line0 + row, a2 = ln / n1, a1 = ln - a2 * n1;
      lab = hs * (c0 * D0[a1] + c1 * D1[a2] + shf);
    }
    const float c2s = hs * c2;
    const int nch = Np / 8;

    for (int m = 0; m < 2; ++m) {
      // one thread issues the MMAs and waits for them (two commits per item:
      // phase parity m); the others wait at the CTA barrier
      if (tid == 0 && !failed) {
        issue_product<FMT>(tmem, A, bm + m * bsz, 1, Kp, Np, (uint32_t)lbo * (uint32_t)sizeof(T));
        commit(&mbar);
        if (!wait_phase_backoff(&mbar, (uint32_t)m)) failed = 1;
        asm volatile("tcgen05.fence::before_thread_sync;");
      }
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (failed) break;
      for (int c0i = half; c0i < nch; c0i += 2) {
        uint32_t raw[8];
        ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c0i * 8), raw);
        ld_wait();
        if (row >= nl) continue;
        const int j0 = c0i * 8;
        if (m == 0) {   // scale by Lambda^{-1}, write back as the next operand
          float x[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = j0 + jj;
            x[jj] = (j < n3) ? __fdividef(__uint_as_float(raw[jj]), lab + c2s * D2[j]) : 0.f;
          }
          if (j0 < Kp) {
            if (FMT == 2) {
              *reinterpret_cast<float4 *>(&A[kslab<FMT>(row, j0, lbo)]) = make_float4(x[0], x[1], x[2], x[3]);
              if (j0 + 4 < Kp)
                *reinterpret_cast<float4 *>(&A[kslab<FMT>(row, j0 + 4, lbo)]) =
                    make_float4(x[4], x[5], x[6], x[7]);
            } else {
              __nv_bfloat162 h[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
              *reinterpret_cast<uint4 *>(&A[kslab<FMT>(row, j0, lbo)]) =
                  *reinterpret_cast<const uint4 *>(h);
            }
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = j0 + jj;
            if (j < n3) X[(long long)j * LN + row] = __uint_as_float(raw[jj]);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
    if (failed) break;
  }
  if (failed) {   // one more bounded wait for MMAs in flight before freeing TMEM
    if (tid == 0)
      for (int ph = 0; ph < 2; ++ph) wait_phase(&mbar, (uint32_t)ph);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
  if (tid == 0 && failed) atomicExch(err, 1);
}

// ------------------------------------------------------------------ host
namespace {

int tc_cols(int c) {
  int t = 32;
  while (t < c) t *= 2;
  return t;
}

struct SlabNeed {
  bool ok;
  int nz;                              // planes per pass-A/C CTA
  int cap_p, bsz_p, tcols_p;           // plane kernel
  int cap_l, bsz_l, tcols_l;           // line kernel
};

SlabNeed slab_need(const DevPatch &p, int interior, int fmt, int dim) {
  const int kstep = (fmt == 2) ? 8 : 16;
  SlabNeed s{};
  int n[3];
  for (int d = 0; d < 3; ++d) n[d] = interior ? p.ni[d] : p.n[d];
  s.ok = dim == 3;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 1 || rup(n[d], 16) > 256) s.ok = false;
  if (!s.ok) return s;
  const int nmax = std::max(n[0], n[1]);
  s.nz = std::max(1, std::min(n[2], 128 / nmax));
  int ntile = 1;
  for (int m = 0; m < 2; ++m) {
    const int na = m ? n[1] : n[0], nb = m ? n[0] : n[1];
    const int Lp = rup(nb * s.nz, 128), Kp = rup(na, kstep), Np = rup(na, 16);
    s.cap_p = std::max(s.cap_p, Kp * (Lp + 1));   // K-chunk slabs of Lp + 1 rows
    s.bsz_p = std::max(s.bsz_p, Np * Kp);
    ntile = std::max(ntile, Lp / 128);
    s.tcols_p = std::max(s.tcols_p, tc_cols((Lp / 128) * Np));
  }
  if (s.tcols_p > 512 || ntile > 2) s.ok = false;
  const int Kp3 = rup(n[2], kstep), Np3 = rup(n[2], 16);
  s.cap_l = Kp3 * (128 + 1);
  s.bsz_l = Np3 * Kp3;
  s.tcols_l = tc_cols(Np3);
  return s;
}

size_t slab_smem(int cap, int bsz, int tcols, int fmt, int nslot = 2) {
  const int esz = (fmt == 2) ? 4 : 2;
  const size_t smem = (size_t)(rup(cap, 256) + nslot * rup(bsz, 256)) * esz + 1024;
  // at most 512 / tcols CTAs per SM (see tc_smem in fd_tc.cu)
  const size_t floor_smem = (size_t)228 * 1024 * (size_t)tcols / 512 - 2048;
  return std::max(smem, floor_smem);
}

// Bounds of nb contiguous ranges of the items with about equal total cost
// (empty ranges allowed).
std::vector<int> balanced_ranges(const std::vector<long long> &cost, int nb) {
  long long total = 0;
  for (long long c : cost) total += c;
  std::vector<int> b(nb + 1, (int)cost.size());
  b[0] = 0;
  long long acc = 0;
  int k = 1;
  for (int i = 0; i < (int)cost.size() && k < nb; ++i) {
    acc += cost[i];
    while (k < nb && acc * nb >= total * (long long)k) b[k++] = i + 1;
  }
  return b;
}

// CTAs per (component, right-hand side): at least the resident CTAs of the
// whole GPU shared over the components, and about `per` items per CTA, so
// that a CTA's setup (tensor memory, barriers, B operands) is shared by a few
// items while CTAs that finish early are replaced by waiting ones (a single
// wave of long ranges measured 35% slower with one right-hand side; 2 to 4
// items did best, which of them depends on the shapes: the FD split tuner
// times both).
template <typename K>
afi_status persistent_grid(afi_ctx *c, K kern, size_t smem, int nitems, int per, int *grid) {
  int occ = 0;
  AFI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem));
  const int wave = c->nsm * std::max(occ, 1) / std::max(c->dim, 1);
  per = std::max(1, per);
  *grid = std::max(1, std::min(nitems, std::max(wave, (nitems + per - 1) / per)));
  return AFI_OK;
}

}  // namespace

// Decide which of the given patches the slab path takes (the rest stay with
// the SIMT kernel) and build the pass work lists and the persistent CTAs'
// ranges of them.
afi_status slab_build(afi_ctx *c, int interior, int fmt, const std::vector<int> &cand,
                      std::vector<int> &rest, TcSplit &sp, int dyn_max, int per) {
  std::vector<int4> pw;
  std::vector<int2> lw;
  std::vector<long long> pcost, lcost;
  int cap_p = 0, bsz_p = 0, tcols_p = 32, cap_l = 0, bsz_l = 0, tcols_l = 32, nslot_p = 1;
  for (int k : cand) {
    const DevPatch &p = c->hp[k];
    const SlabNeed s = slab_need(p, interior, fmt, c->dim);
    const int ncp = std::max(cap_p, s.cap_p), nbp = std::max(bsz_p, s.bsz_p);
    const int ntp = std::max(tcols_p, s.tcols_p);
    const int ncl = std::max(cap_l, s.cap_l), nbl = std::max(bsz_l, s.bsz_l);
    const int ntl = std::max(tcols_l, s.tcols_l);
    int nsp = nslot_p;
    for (int l = 0; l < c->dim; ++l) nsp = std::max(nsp, p.ltab[l][0] == p.ltab[l][1] ? 1 : 2);
    if (!s.ok || slab_smem(ncp, nbp, ntp, fmt, nsp) > (size_t)dyn_max ||
        slab_smem(ncl, nbl, ntl, fmt) > (size_t)dyn_max) {
      rest.push_back(k);
      continue;
    }
    cap_p = ncp; bsz_p = nbp; tcols_p = ntp; cap_l = ncl; bsz_l = nbl; tcols_l = ntl;
    nslot_p = nsp;
    const int n1 = interior ? p.ni[0] : p.n[0], n2 = interior ? p.ni[1] : p.n[1];
    const int n3 = interior ? p.ni[2] : p.n[2];
    for (int z = 0; z < n3; z += s.nz) {
      pw.push_back(make_int4(k, z, std::min(s.nz, n3 - z), 0));
      pcost.push_back((long long)n1 * n2 * std::min(s.nz, n3 - z));
    }
    for (int ln = 0; ln < n1 * n2; ln += 128) {
      lw.push_back(make_int2(k, ln));
      lcost.push_back((long long)std::min(128, n1 * n2 - ln) * n3);
    }
  }
  sp.nplane = (int)pw.size();
  sp.nline = (int)lw.size();
  sp.cap_p = rup(std::max(cap_p, 256), 256);
  sp.bsz_p = rup(std::max(bsz_p, 256), 256);
  sp.tcols_p = tcols_p;
  sp.cap_l = rup(std::max(cap_l, 256), 256);
  sp.bsz_l = rup(std::max(bsz_l, 256), 256);
  sp.tcols_l = tcols_l;
  sp.smem_p = slab_smem(sp.cap_p, sp.bsz_p, sp.tcols_p, fmt, nslot_p);
  sp.smem_l = slab_smem(sp.cap_l, sp.bsz_l, sp.tcols_l, fmt);
  if (sp.nplane) {
    AFI_TRY(dalloc(c, (void **)&sp.d_plane, pw.size() * sizeof(int4)));
    AFI_CUDA(cudaMemcpy(sp.d_plane, pw.data(), pw.size() * sizeof(int4), cudaMemcpyHostToDevice));
    AFI_TRY(dalloc(c, (void **)&sp.d_line, lw.size() * sizeof(int2)));
    AFI_CUDA(cudaMemcpy(sp.d_line, lw.data(), lw.size() * sizeof(int2), cudaMemcpyHostToDevice));
    if (fmt == 2) {
      AFI_TRY(persistent_grid(c, k_fd_plane<2, 0>, sp.smem_p, sp.nplane, per, &sp.pgrid));
      AFI_TRY(persistent_grid(c, k_fd_line<2>, sp.smem_l, sp.nline, per, &sp.lgrid));
    } else {
      AFI_TRY(persistent_grid(c, k_fd_plane<1, 0>, sp.smem_p, sp.nplane, per, &sp.pgrid));
      AFI_TRY(persistent_grid(c, k_fd_line<1>, sp.smem_l, sp.nline, per, &sp.lgrid));
    }
    const std::vector<int> pb = balanced_ranges(pcost, sp.pgrid), lb = balanced_ranges(lcost, sp.lgrid);
    AFI_TRY(dalloc(c, (void **)&sp.d_pbounds, pb.size() * sizeof(int)));
    AFI_CUDA(cudaMemcpy(sp.d_pbounds, pb.data(), pb.size() * sizeof(int), cudaMemcpyHostToDevice));
    AFI_TRY(dalloc(c, (void **)&sp.d_lbounds, lb.size() * sizeof(int)));
    AFI_CUDA(cudaMemcpy(sp.d_lbounds, lb.data(), lb.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  return AFI_OK;
}

// Opt the slab kernels into the largest dynamic shared memory the device
// allows next to their static shared memory; returns that size.
afi_status slab_prepare(afi_ctx *c, int *dyn_max) {
  const void *fns[] = {(const void *)k_fd_plane<2, 0>, (const void *)k_fd_plane<2, 1>,
                       (const void *)k_fd_plane<1, 0>, (const void *)k_fd_plane<1, 1>,
                       (const void *)k_fd_line<2>, (const void *)k_fd_line<1>};
  size_t stat = 0;
  for (const void *f : fns) {
    cudaFuncAttributes fa;
    AFI_CUDA(cudaFuncGetAttributes(&fa, f));
    stat = std::max(stat, fa.sharedSizeBytes);
  }
  *dyn_max = c->smem_optin - (int)stat;
  for (const void *f : fns)
    AFI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, *dyn_max));
  return AFI_OK;
}

// The three passes over the slab patches, right-hand sides in chunks that
// fit the FP32 scratch (the context's local-solver scratch slab).
afi_status slab_run(afi_ctx *c, int interior, int fmt, const TcSplit &sp, const double *r,
                    double *s, cudaStream_t st, int nrhs) {
  if (!sp.nplane) return AFI_OK;
  const long long stride = interior ? c->n_int : c->n_dof;
  float *scr = reinterpret_cast<float *>(c->fdscratch);
  const int chunk = (int)std::max(1LL, (2 * c->fdscratch_n) / std::max(1LL, stride));
  const Tab1D *tabs = c->tabs;
  const DevPatch *P = c->patches;
  const int4 *pw = (const int4 *)sp.d_plane;
  const int2 *lw = (const int2 *)sp.d_line;
  for (int j = 0; j < nrhs; j += chunk) {
    const int nb = std::min(chunk, nrhs - j);
    const double *rj = r + (long long)j * stride;
    double *sj = s + (long long)j * stride;
    const dim3 gp(sp.pgrid, c->dim, nb), gl(sp.lgrid, c->dim, nb);
    const int *pb = sp.d_pbounds, *lb = sp.d_lbounds;
    if (fmt == 2) {
      launch(k_fd_plane<2, 0>, gp, 256, sp.smem_p, st, P, tabs, pw, pb, interior, rj, scr, sj, stride,
             sp.cap_p, sp.bsz_p, sp.tcols_p, c->gate, c->dflag + 1, (const unsigned char *)c->tcpool);
      launch(k_fd_line<2>, gl, 256, sp.smem_l, st, P, tabs, (const float *)c->fpool, lw, lb, interior,
             scr, stride, sp.cap_l, sp.bsz_l, sp.tcols_l, c->gate, c->dflag + 1,
             (const unsigned char *)c->tcpool);
      launch(k_fd_plane<2, 1>, gp, 256, sp.smem_p, st, P, tabs, pw, pb, interior, rj, scr, sj, stride,
             sp.cap_p, sp.bsz_p, sp.tcols_p, c->gate, c->dflag + 1, (const unsigned char *)c->tcpool);
    } else {
      launch(k_fd_plane<1, 0>, gp, 256, sp.smem_p, st, P, tabs, pw, pb, interior, rj, scr, sj, stride,
             sp.cap_p, sp.bsz_p, sp.tcols_p, c->gate, c->dflag + 1, (const unsigned char *)c->tcpool);
      launch(k_fd_line<1>, gl, 256, sp.smem_l, st, P, tabs, (const float *)c->fpool, lw, lb, interior,
             scr, stride, sp.cap_l, sp.bsz_l, sp.tcols_l, c->gate, c->dflag + 1,
             (const unsigned char *)c->tcpool);
      launch(k_fd_plane<1, 1>, gp, 256, sp.smem_p, st, P, tabs, pw, pb, interior, rj, scr, sj, stride,
             sp.cap_p, sp.bsz_p, sp.tcols_p, c->gate, c->dflag + 1, (const unsigned char *)c->tcpool);
    }
    AFI_LAUNCH_CHECK();
  }
  return AFI_OK;
}

}  // namespace afi
