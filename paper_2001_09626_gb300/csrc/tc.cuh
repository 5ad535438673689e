// tcgen05 building blocks shared by the tensor-core FD kernels: shared
// memory and instruction descriptors, MMA issue and commit, bounded mbarrier
// waits, tensor-memory loads, bulk (TMA) copies and the operand layouts.
#pragma once

#include "common.cuh"

namespace afi {

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: FP32 accumulate, A/B format fmt (2 = TF32, 1 = BF16),
// both K-major, N and M dimensions
__device__ __forceinline__ uint32_t idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (FMT == 2)
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d), "l"(a),
                 "l"(b), "r"(id), "r"(acc));
  else
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d), "l"(a),
                 "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

// bounded wait for the given phase of an mbarrier: at most `limit` polls
// (each try_wait may suspend the thread for a short hardware-defined time);
// false on timeout, *used = polls made
__device__ __forceinline__ bool wait_phase_n(uint64_t *mbar, uint32_t phase, long long limit,
                                             long long *used) {
  uint32_t done = 0;
  long long it = 0;
  for (; it < limit && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(mbar)), "r"(phase));
  *used = it;
  return done != 0;
}

// the waits of the tensor-core kernels: at most 2^22 polls
__device__ __forceinline__ bool wait_phase(uint64_t *mbar, uint32_t phase) {
  long long used;
  return wait_phase_n(mbar, phase, 1LL << 22, &used);
}

// The same with a 64 ns sleep between polls, for a single thread waiting on
// MMAs or bulk copies while the rest of its CTA waits at a barrier: the polls
// then take fewer issue slots from the other CTAs on the SM (at most 2^22
// polls).
__device__ __forceinline__ bool wait_phase_backoff(uint64_t *mbar, uint32_t phase) {
  uint32_t done = 0;
  for (long long it = 0; it < (1LL << 22) && !done; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(mbar)), "r"(phase));
    if (!done) __nanosleep(64);
  }
  return done != 0;
}

// 32 lanes x 8 columns of 32 bits from tensor memory; completes at ld_wait()
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// mbarrier expecting `bytes` of asynchronous copies (one arrival)
__device__ __forceinline__ void expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes));
}

// 1D bulk copy global -> shared (TMA), completion counted on mbar; 16-byte
// aligned addresses, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

template <int FMT> struct Op;
template <> struct Op<2> {   // TF32: FP32 storage, 4 elements per 16 bytes, 8 per MMA
  using T = float;
  static constexpr int T16 = 4, KSTEP = 8;
  static __device__ __forceinline__ T cvt(float x) { return x; }
};
template <> struct Op<1> {   // BF16: 8 elements per 16 bytes, 16 per MMA
  using T = __nv_bfloat16;
  static constexpr int T16 = 8, KSTEP = 16;
  static __device__ __forceinline__ T cvt(float x) { return __float2bfloat16(x); }
};

__host__ __device__ __forceinline__ int rup(int x, int m) { return (x + m - 1) / m * m; }

// FP64 -> FP32 for a value that only becomes a tensor-core operand, on the
// integer pipes and from the high word alone: the FP32 significand keeps the
// top 20 bits of the FP64 one (truncated), which the operand rounding to
// TF32 (10 stored bits) or BF16 (7) makes immaterial.  The exponent is
// clamped: magnitudes below 2^-127 give signed zero, those in [2^-127,
// 2^-126) an FP32 subnormal below 2^-126, those of 2^128 and above +-inf;
// NaN stays NaN.
__device__ __forceinline__ float f64_to_op(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned mag = hi & 0x7FFFFFFFu;
  const unsigned m = min(max(mag, 0x38000000u), 0x47F00000u);
  unsigned r = ((m - 0x38000000u) << 3) | (hi & 0x80000000u);
  if (mag > 0x7FF00000u) r |= 0x00400000u;
  return __uint_as_float(r);
}

// four (two) consecutive K entries of one operand row, 16-byte (8-byte)
// aligned for TF32, 8-byte (4-byte) for BF16
template <int FMT> __device__ __forceinline__ void st4(typename Op<FMT>::T *p, const float *v);
template <> __device__ __forceinline__ void st4<2>(float *p, const float *v) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void st4<1>(__nv_bfloat16 *p, const float *v) {
  __nv_bfloat162 h[2] = {__floats2bfloat162_rn(v[0], v[1]), __floats2bfloat162_rn(v[2], v[3])};
  *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(h);
}
template <int FMT> __device__ __forceinline__ void st2(typename Op<FMT>::T *p, const float *v);
template <> __device__ __forceinline__ void st2<2>(float *p, const float *v) {
  *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
template <> __device__ __forceinline__ void st2<1>(__nv_bfloat16 *p, const float *v) {
  *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v[0], v[1]);
}

// element offset of (row, k) in the canonical K-major core-matrix layout with
// Kp columns (core matrices 128 bytes apart); used for the prebuilt B operands
template <int FMT>
__device__ __forceinline__ int cm(int row, int k, int Kp) {
  constexpr int T16 = Op<FMT>::T16;
  return (((row >> 3) * (Kp / T16) + k / T16) * 8 + (row & 7)) * T16 + (k % T16);
}

// The tensor operands of the FD kernels store each 16-byte K chunk of all
// their rows as one slab: rows 16 bytes apart (8-row groups 128 bytes apart)
// and chunks lbo = (Lp + 1) x 16 bytes apart, Lp = rows padded to the
// 128-row tile.  An element's offset is then linear in its row, and the
// extra 16 bytes per slab put a warp writing one row across its K chunks on
// distinct shared-memory banks.  Element offset of (row, k), lbo in elements:
template <int FMT>
__device__ __forceinline__ int kslab(int row, int k, int lbo) {
  constexpr int T16 = Op<FMT>::T16;
  return (k / T16) * lbo + row * T16 + (k % T16);
}

}  // namespace tc

}  // namespace afi
