// Fast diagonalization (Algorithm 1, eqs. 5.6, 5.9, 5.10) on the 5th
// generation tensor cores: tcgen05.mma with TF32 or BF16 operands in shared
// memory and FP32 accumulators in tensor memory.
//
// One CTA owns one (patch, component) tensor X[i3][i2][i1].  Each of the six
// mode products (U_1^T, U_2^T, U_3^T, then U_1, U_2, U_3) is a GEMM
//     D[line][a] = sum_k A[line][k] B[a][k],
// where the rows ("lines") run over the two uncontracted indices and k over
// the contracted one, which is always the fastest index of the operand: the
// epilogue of every mode writes its result with the axes rotated
// ([c][b][a] -> [a'][c][b]), so the next contraction is again over the
// contiguous index and A stays K-major.  After three rotations the axes are
// back in their original order.  The scaling by Lambda^{-1} is fused into the
// epilogue of the third product, and the last epilogue writes FP64 straight
// to global memory.
//
// Operands use the no-swizzle K-major canonical layout of core matrices
// (8 rows x 16 bytes); one elected thread issues the MMAs (M = 128 lines per
// tile, N = output modes padded to 16, K in steps of 32 bytes) and commits
// them to an mbarrier that all threads wait on with a bounded spin.
#include "common.cuh"

#include <algorithm>

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

// bounded wait for the given phase of an mbarrier; false on timeout
__device__ __forceinline__ bool wait_phase(uint64_t *mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(mbar)), "r"(phase));
  return done != 0;
}

__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                 "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

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

// element offset of (row, k) in the K-major core-matrix layout with Kp columns
template <int FMT>
__device__ __forceinline__ int cm(int row, int k, int Kp) {
  constexpr int T16 = Op<FMT>::T16;
  return (((row >> 3) * (Kp / T16) + k / T16) * 8 + (row & 7)) * T16 + (k % T16);
}

}  // namespace tc

template <int FMT>
__global__ void __launch_bounds__(256) k_fd_tc(const DevPatch *P, const Tab1D *tabs,
                                               const float *fpool, int dim, int interior,
                                               const double *r, double *s, int cap, int bsz,
                                               int tcols, const double *gate, int *err,
                                               long long rhs_stride, const int *plist,
                                               const unsigned char *tcpool) {
  using namespace tc;
  using T = typename Op<FMT>::T;
  constexpr int KSTEP = Op<FMT>::KSTEP, T16 = Op<FMT>::T16;
  if (gate && *gate == 0.0) return;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  T *buf[2] = {reinterpret_cast<T *>(smraw), reinterpret_cast<T *>(smraw) + cap};
  T *bm = reinterpret_cast<T *>(smraw) + 2 * cap;   // 6 B operands, bsz elements each
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = plist[blockIdx.x], l = blockIdx.y;
  const DevPatch pt = P[k];
  int n[3];
  for (int d = 0; d < 3; ++d) n[d] = interior ? pt.ni[d] : pt.n[d];
  const int N = n[0] * n[1] * n[2];
  const long long base =
      (interior ? pt.ioff : pt.off) + (long long)l * N + (long long)blockIdx.z * rhs_stride;

  // stage the six B operands (prebuilt in the canonical layout) with TMA
  // bulk copies while the threads zero the operand buffers
  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tma_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t bytes[6], total = 0;
    for (int m = 0; m < 6; ++m) {
      const int nd = n[m % 3];
      bytes[m] = (uint32_t)(rup(nd, 16) * rup(nd, KSTEP) * (int)sizeof(T));
      total += bytes[m];
    }
    expect_tx(&tma_bar, total);
    for (int m = 0; m < 6; ++m) {
      const Tab1D tb = tabs[pt.tab[m % 3]];
      bulk_g2s(bm + m * bsz, tcpool + tb.tcB[FMT == 1][interior][m >= 3], bytes[m], &tma_bar);
    }
  }
  for (int i = tid; i < 2 * cap; i += blockDim.x) buf[0][i] = Op<FMT>::cvt(0.f);
  __syncthreads();
  // load the tensor as the first operand: line = i2 + n2 i3, k = i1
  {
    const int Kp = rup(n[0], KSTEP);
    for (int idx = tid; idx < N; idx += blockDim.x)
      buf[0][cm<FMT>(idx / n[0], idx % n[0], Kp)] = Op<FMT>::cvt((float)r[base + idx]);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (!wait_phase(&tma_bar, 0)) failed = 1;   // B operands have landed
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;

  // Lambda for this (patch, component)
  const float cl = (float)(2.0 * pt.mu + pt.lam), mu = (float)pt.mu, hs = (float)pt.Hs;
  const float c0 = (l == 0) ? cl : mu, c1 = (l == 1) ? cl : mu, c2 = (l == 2) ? cl : mu;
  const float *Dv[3];
  for (int d = 0; d < 3; ++d) {
    const Tab1D tb = tabs[pt.tab[d]];
    Dv[d] = fpool + (interior ? tb.Di : tb.D);
  }

  int na = n[0], nb = n[1], nc = n[2];   // current operand dims, a fastest
  for (int m = 0; m < 6; ++m) {
    const int L = nb * nc, ntile = rup(L, 128) / 128;
    const int Kp = rup(na, KSTEP), Np = rup(na, 16);
    T *A = buf[m & 1];
    if (tid == 0 && !failed) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t id = idesc(FMT, 128, Np);
      const uint32_t sbo = (uint32_t)(Kp / T16) * 128u;
      const uint32_t a0 = smem_u32(A), b0 = smem_u32(bm + m * bsz);
      for (int t = 0; t < ntile; ++t)
        for (int ks = 0; ks < Kp / KSTEP; ++ks)
          mma<FMT>(tmem + (uint32_t)(t * Np), sdesc(a0 + t * 16 * sbo + ks * 256, 128, sbo),
                   sdesc(b0 + ks * 256, 128, sbo), id, ks > 0 ? 1u : 0u);
      commit(&mbar);
    }
    if (!wait_phase(&mbar, (uint32_t)(m & 1))) failed = 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (failed) break;
    // epilogue: D[line][j] -> next operand (rotated) or the FP64 output
    const int q = warp & 3, half = warp >> 2;
    const int nnb = nc, nKp = rup(nb, KSTEP);   // next operand: K = nb, lines = nc * na
    T *An = buf[(m + 1) & 1];
    for (int t = 0; t < ntile; ++t) {
      const int line = t * 128 + q * 32 + lane;
      const int b = line % nb, c = line / nb;
      for (int j0 = half * 16; j0 < Np; j0 += 32) {
        float v[16];
        ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * Np + j0), v);
        if (line >= L) continue;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = j0 + jj;
          if (j >= na) continue;
          float x = v[jj];
          if (m == 2) {   // element r~(a1 = b, a2 = c, a3 = j): scale by Lambda^{-1}
            float lam = c0 * Dv[0][b] + c1 * Dv[1][c] + c2 * Dv[2][j];
            if (dim != 3) lam = c0 * Dv[0][b] + c1 * Dv[1][c];
            if (!interior) lam = hs * (lam + 1.f);
            x = x / lam;
          }
          if (m == 5) s[base + b + (long long)n[0] * (c + (long long)n[1] * j)] = (double)x;
          else An[cm<FMT>(c + nnb * j, b, nKp)] = Op<FMT>::cvt(x);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // rotate dims: (na, nb, nc) -> (nb, nc, na)
    const int t0 = na;
    na = nb; nb = nc; nc = t0;
  }
  if (failed) {   // give MMAs still in flight one more bounded wait before freeing TMEM
    for (int ph = 0; ph < 2; ++ph) wait_phase(&mbar, (uint32_t)ph);
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
  if (tid == 0 && failed) atomicExch(err, 1);
}

static int g_tc_dyn_max;

// Shared memory, B-operand size and TMEM columns the kernel needs for one
// patch (operand format fmt: 2 = TF32, 1 = BF16).
struct TcNeed { int cap, bsz, tcols; bool ok; };

static TcNeed tc_need(const DevPatch &p, int interior, int fmt) {
  const int kstep = (fmt == 2) ? 8 : 16;
  TcNeed t{0, 0, 32, true};
  int n[3];
  for (int d = 0; d < 3; ++d) n[d] = interior ? p.ni[d] : p.n[d];
  for (int d = 0; d < 3; ++d) {
    const int na = n[d], nb = n[(d + 1) % 3], nc = n[(d + 2) % 3];
    const int Lp = tc::rup(nb * nc, 128), Kp = tc::rup(na, kstep), Np = tc::rup(na, 16);
    t.cap = std::max(t.cap, Lp * Kp);
    t.bsz = std::max(t.bsz, Np * Kp);
    const int cols = (Lp / 128) * Np;
    while (t.tcols < cols) t.tcols *= 2;
    if (Np > 256) t.ok = false;
  }
  if (t.tcols > 512) t.ok = false;
  return t;
}

static size_t tc_smem(int cap, int bsz, int tcols, int fmt) {
  const int esz = (fmt == 2) ? 4 : 2;
  size_t smem = (size_t)(2 * tc::rup(cap, 256) + 6 * tc::rup(bsz, 256)) * esz + 1024;
  // at most 512 / tcols CTAs per SM, so tensor-memory allocation never waits long
  const size_t floor_smem = (size_t)228 * 1024 * (size_t)tcols / 512 + 1024;
  return std::max(smem, floor_smem);
}

// Patches in increasing order of need join the tensor-core list while the
// combined launch still fits; the rest go to the SIMT kernel.
static afi_status build_split(afi_ctx *c, int interior, int fmt, TcSplit &sp) {
  std::vector<std::pair<size_t, int>> order;
  for (int k = 0; k < c->npatch; ++k) {
    const TcNeed t = tc_need(c->hp[k], interior, fmt);
    if (t.ok) order.push_back({tc_smem(t.cap, t.bsz, t.tcols, fmt), k});
  }
  std::sort(order.begin(), order.end());
  std::vector<int> tc, simt;
  std::vector<char> in(c->npatch, 0);
  int cap = 0, bsz = 0, tcols = 32;
  for (auto &o : order) {
    const TcNeed t = tc_need(c->hp[o.second], interior, fmt);
    const int ncap = std::max(cap, t.cap), nbsz = std::max(bsz, t.bsz), ncols = std::max(tcols, t.tcols);
    if (tc_smem(ncap, nbsz, ncols, fmt) > (size_t)g_tc_dyn_max) continue;
    cap = ncap; bsz = nbsz; tcols = ncols;
    in[o.second] = 1;
  }
  int maxN = 1;
  for (int k = 0; k < c->npatch; ++k) {
    if (in[k]) tc.push_back(k);
    else {
      simt.push_back(k);
      maxN = std::max(maxN, interior ? c->hp[k].Ni : c->hp[k].N);
    }
  }
  sp.ntc = (int)tc.size();
  sp.nsimt = (int)simt.size();
  sp.cap = tc::rup(cap, 256);
  sp.bsz = tc::rup(bsz, 256);
  sp.tcols = tcols;
  sp.smem = tc_smem(cap, bsz, tcols, fmt);
  sp.simt_maxN = maxN;
  if (sp.ntc) {
    AFI_TRY(dalloc(c, (void **)&sp.d_tc, tc.size() * sizeof(int)));
    AFI_CUDA(cudaMemcpy(sp.d_tc, tc.data(), tc.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  if (sp.nsimt) {
    AFI_TRY(dalloc(c, (void **)&sp.d_simt, simt.size() * sizeof(int)));
    AFI_CUDA(cudaMemcpy(sp.d_simt, simt.data(), simt.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  sp.ready = true;
  return AFI_OK;
}

afi_status fd_tc_prepare(afi_ctx *c) {
  cudaFuncAttributes fa2, fa1;
  AFI_CUDA(cudaFuncGetAttributes(&fa2, k_fd_tc<2>));
  AFI_CUDA(cudaFuncGetAttributes(&fa1, k_fd_tc<1>));
  const int stat = (int)std::max(fa2.sharedSizeBytes, fa1.sharedSizeBytes);
  g_tc_dyn_max = c->smem_optin - stat;
  AFI_CUDA(cudaFuncSetAttribute(k_fd_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, g_tc_dyn_max));
  AFI_CUDA(cudaFuncSetAttribute(k_fd_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, g_tc_dyn_max));
  return AFI_OK;
}

// Tensor-core FD on the patches that fit, SIMT FP32 FD on the others.  The
// splits are built outside stream capture: the first solve builds them
// before capturing (see fd_tc_ready).
afi_status fd_tc_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                     int nrhs) {
  const int fmt = (c->opt.prec == AFI_FD_BF16) ? 1 : 2;
  TcSplit &sp = c->tcsplit[interior][fmt == 1];
  if (!sp.ready) AFI_TRY(build_split(c, interior, fmt, sp));
  const long long stride = interior ? c->n_int : c->n_dof;
  if (sp.ntc) {
    const dim3 grid(sp.ntc, c->dim, nrhs);
    if (fmt == 2)
      launch(k_fd_tc<2>, grid, 256, sp.smem, st, (const DevPatch *)c->patches,
             (const Tab1D *)c->tabs, (const float *)c->fpool, c->dim, interior, r, s, sp.cap,
             sp.bsz, sp.tcols, c->gate, c->dflag + 1, stride, (const int *)sp.d_tc,
             (const unsigned char *)c->tcpool);
    else
      launch(k_fd_tc<1>, grid, 256, sp.smem, st, (const DevPatch *)c->patches,
             (const Tab1D *)c->tabs, (const float *)c->fpool, c->dim, interior, r, s, sp.cap,
             sp.bsz, sp.tcols, c->gate, c->dflag + 1, stride, (const int *)sp.d_tc,
             (const unsigned char *)c->tcpool);
    AFI_LAUNCH_CHECK();
  }
  if (sp.nsimt) AFI_TRY(fd_simt_list(c, interior, sp.d_simt, sp.nsimt, sp.simt_maxN, r, s, st, nrhs));
  return AFI_OK;
}

// The B operands of every table in the canonical K-major layout, for both
// operand formats, full and interior pencils, forward (U^T) and back (U).
__global__ void k_tc_bops(const Tab1D *tabs, int ntab, const double *pool, unsigned char *tcpool) {
  const int t = blockIdx.y, v = blockIdx.z;   // v = bf16 * 4 + interior * 2 + back
  if (t >= ntab) return;
  const Tab1D T = tabs[t];
  const int bf = v >> 2, in = (v >> 1) & 1, back = v & 1;
  const int n = in ? T.ni : T.n;
  const double *U = pool + (in ? T.Ui : T.U);
  const int Np = tc::rup(n, 16), Kp = tc::rup(n, bf ? 16 : 8);
  unsigned char *dst = tcpool + T.tcB[bf][in][back];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Np * Kp; i += gridDim.x * blockDim.x) {
    const int a = i / Kp, k = i % Kp;
    double val = 0.0;
    if (a < n && k < n) val = back ? U[a * n + k] : U[k * n + a];
    if (bf) reinterpret_cast<__nv_bfloat16 *>(dst)[tc::cm<1>(a, k, Kp)] = __double2bfloat16(val);
    else reinterpret_cast<float *>(dst)[tc::cm<2>(a, k, Kp)] = (float)val;
  }
}

afi_status fd_tc_tables(afi_ctx *c) {
  long long off = 0;
  for (auto &T : c->htab)
    for (int bf = 0; bf < 2; ++bf)
      for (int in = 0; in < 2; ++in)
        for (int back = 0; back < 2; ++back) {
          const int n = in ? T.ni : T.n;
          const long long bytes = (long long)tc::rup(n, 16) * tc::rup(n, bf ? 16 : 8) * (bf ? 2 : 4);
          T.tcB[bf][in][back] = off;
          off += (bytes + 127) / 128 * 128;
        }
  c->tcpool_n = off;
  AFI_TRY(dalloc(c, (void **)&c->tcpool, (size_t)off));
  AFI_CUDA(cudaMemcpy(c->tabs, c->htab.data(), c->htab.size() * sizeof(Tab1D), cudaMemcpyHostToDevice));
  const int nt = (int)c->htab.size();
  launch(k_tc_bops, dim3(4, nt, 8), 256, 0, 0, (const Tab1D *)c->tabs, nt, (const double *)c->dpool,
         c->tcpool);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// Build every split up front (called before a CUDA graph is captured).
afi_status fd_tc_ready(afi_ctx *c) {
  for (int in = 0; in < 2; ++in)
    for (int f = 1; f <= 2; ++f) {
      TcSplit &sp = c->tcsplit[in][f == 1];
      if (!sp.ready) AFI_TRY(build_split(c, in, f, sp));
    }
  return AFI_OK;
}

}  // namespace afi
