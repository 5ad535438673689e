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
// Operands use the no-swizzle K-major layout of core matrices (8 rows x 16
// bytes).  The tensor operand stores each 16-byte K chunk of all its rows as
// one slab, rows 16 bytes apart (stride between 8-row groups 128 bytes) and
// chunks (Lp + 1) x 16 bytes apart (Lp = lines padded to the 128-line
// tile), so an element's offset is linear in its row and a warp writing one
// row across its K chunks touches distinct banks.  One elected thread issues
// the MMAs (M = 128 lines per tile, N = output modes padded to 16, K in steps
// of 32 bytes), commits them to an mbarrier and waits on it with a bounded
// spin while the other threads wait at the CTA barrier.  The tensor operand
// lives in a single shared-memory buffer that each epilogue overwrites in
// place, so three to four CTAs share an SM; FP64 <-> FP32 conversions of the
// input and output run on the integer pipes (f64_to_op / f32_to_f64).
#include "tc.cuh"

#include <algorithm>

namespace afi {

// Slots of the B operands in shared memory: one per distinct (table, back)
// pair of the six mode products, packed 4 bits per product (bits 24.. hold
// the number of slots).
__host__ __device__ __forceinline__ unsigned b_slots(int t0, int t1, int t2) {
  const int tab[3] = {t0, t1, t2};
  unsigned packed = 0;
  int nslot = 0;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int sl = -1;
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (q < m && sl < 0 && q / 3 == m / 3 && tab[q % 3] == tab[m % 3])
        sl = (int)((packed >> (4 * q)) & 15u);
    if (sl < 0) sl = nslot++;
    packed |= (unsigned)sl << (4 * m);
  }
  return packed | ((unsigned)nslot << 24);
}
__host__ __device__ __forceinline__ int bslot(unsigned packed, int m) {
  return (int)((packed >> (4 * m)) & 15u);
}

// Epilogue of one mode product: D[line][j] from tensor memory to registers,
// then (KIND 0) into the next operand with the axes rotated, in place;
// (KIND 1) the same after the scaling by Lambda^{-1}; (KIND 2) as FP64 into
// the output.  Work items are (128-line tile, 8 columns), split between the
// NT / 128 warps that share a tensor-memory lane quarter.  The current operand is [c][b][a] (a = na fastest); line =
// b + nb c, j = a; the next operand row is c + nc j with K index b.
struct Scale {   // lambda(b, c, j) = s0 + sb D0[b] + sc D1[c] + sj D2[j]
  const float *D0, *D1, *D2;
  float s0, sb, sc, sj;
};

template <int FMT, int NT, int KIND>
__device__ __forceinline__ void fd_epilogue(uint32_t tmem, typename tc::Op<FMT>::T *A, int na, int nb,
                                            int nc, int Np, int ntile, const Scale &sc, double *so,
                                            long long jstride) {
  using namespace tc;
  constexpr int G = NT / 128, T16 = Op<FMT>::T16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
  const int L = nb * nc, nch = (na + 7) >> 3;
  const int lbo = (rup(nc * na, 128) + 1) * T16;   // K-chunk stride of the next operand
  const int jstep = nc * T16;                       // next-operand offset per column j
  // the warp's items (t, ch) = (it / nch, it % nch), it = half, half + G,
  // ..., and its lane's line = b + nb c, stepped without divisions
  int t = 0, ch = half;
  while (ch >= nch) { ch -= nch; ++t; }
  int line = t * 128 + q * 32 + lane;
  int c = line / nb, b = line - c * nb;
  const int dq = 128 / nb, dr = 128 - dq * nb;
  while (t < ntile) {
    const int j0 = ch * 8;
    uint32_t raw[8];
    ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * Np + j0), raw);
    ld_wait();
    if (line < L) {
      const int jn = min(8, na - j0);
      if (KIND == 2) {
        double *o = so + line + jstride * j0;
        if (jn == 8) {   // a full chunk: no per-column predicate
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) o[jstride * jj] = f32_to_f64(__uint_as_float(raw[jj]));
        } else {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            if (jj < jn) o[jstride * jj] = f32_to_f64(__uint_as_float(raw[jj]));
        }
      } else {
        // element (row = c + nc j, k = b) of the next operand
        typename Op<FMT>::T *dst = A + kslab<FMT>(c + nc * j0, b, lbo);
        float lb = 0.f;
        if (KIND == 1) lb = sc.s0 + sc.sb * sc.D0[b] + sc.sc * sc.D1[c];
        if (jn == 8) {   // a full chunk: no per-column predicate
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            float x = __uint_as_float(raw[jj]);
            if (KIND == 1) x = __fdividef(x, lb + sc.sj * sc.D2[j0 + jj]);
            dst[jj * jstep] = Op<FMT>::cvt(x);
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            if (jj < jn) {
              float x = __uint_as_float(raw[jj]);
              if (KIND == 1) x = __fdividef(x, lb + sc.sj * sc.D2[j0 + jj]);
              dst[jj * jstep] = Op<FMT>::cvt(x);
            }
          }
        }
      }
    }
    ch += G;
    while (ch >= nch) {   // next tile: line += 128
      ch -= nch;
      ++t;
      line += 128;
      c += dq;
      b += dr;
      if (b >= nb) { b -= nb; ++c; }
    }
  }
}

template <int FMT, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_fd_tc(const DevPatch *P, const Tab1D *tabs,
                                               const float *fpool, int dim, int interior,
                                               const double *r, double *s, int cap, int bsz,
                                               int tcols, const double *gate, int *err,
                                               long long rhs_stride, const int *plist,
                                               const unsigned char *tcpool) {
  using namespace tc;
  using T = typename Op<FMT>::T;
  constexpr int KSTEP = Op<FMT>::KSTEP, T16 = Op<FMT>::T16;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  // one operand buffer, rewritten in place by every epilogue (the MMAs that
  // read it have completed by then), followed by the B operands
  T *A = reinterpret_cast<T *>(smraw);
  T *bm = A + cap;
  const int tid = threadIdx.x, warp = tid >> 5;
  // the gate load overlaps the patch-descriptor loads
  const double gv = gate ? *gate : 1.0;
  const int k = plist[blockIdx.x], l = blockIdx.y;
  const DevPatch pt = P[k];
  if (gv == 0.0) return;   // inactive MINRES iteration
  int n[3];
  for (int d = 0; d < 3; ++d) n[d] = interior ? pt.ni[d] : pt.n[d];
  const int N = n[0] * n[1] * n[2];
  const long long base =
      (interior ? pt.ioff : pt.off) + (long long)l * N + (long long)blockIdx.z * rhs_stride;
  // this component's tables and coefficients, read from global memory
  // (indexing the local copy by the runtime component would move it to
  // local memory)
  const int lt0 = P[k].ltab[l][0], lt1 = P[k].ltab[l][1], lt2 = P[k].ltab[l][2];
  const unsigned bs = b_slots(lt0, lt1, lt2);

  // stage the B operands (prebuilt in the canonical layout) with TMA bulk
  // copies while the threads zero the operand buffer
  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tma_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (tid == 0) {
    // a product copies its B operand when it is the first user of its slot
    uint32_t total = 0;
    unsigned first = 0;
    int seen = 0;
    for (int m = 0; m < 6; ++m) {
      const int sl = bslot(bs, m);
      if (seen & (1 << sl)) continue;
      seen |= 1 << sl;
      first |= 1u << m;
      const int nd = n[m % 3];
      total += (uint32_t)(rup(nd, 16) * rup(nd, KSTEP) * (int)sizeof(T));
    }
    expect_tx(&tma_bar, total);
    for (int m = 0; m < 6; ++m) {
      if (!(first & (1u << m))) continue;
      const int nd = n[m % 3];
      const int tm = (m % 3 == 0) ? lt0 : (m % 3 == 1 ? lt1 : lt2);
      const long long off = tabs[tm].tcB[FMT == 1][interior][m >= 3];
      bulk_g2s(bm + bslot(bs, m) * bsz, tcpool + off,
               (uint32_t)(rup(nd, 16) * rup(nd, KSTEP) * (int)sizeof(T)), &tma_bar);
    }
  }
  {
    uint4 *z = reinterpret_cast<uint4 *>(A);
    const int nz = cap * (int)sizeof(T) / 16;
    for (int i = tid; i < nz; i += NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();
  // load the tensor as the first operand (line = i2 + n2 i3, k = i1) in
  // chunks of four K entries, chunk g = line * kq + kc; the (line, kc) of a
  // thread's chunks step by NT without a division, and the loads of two
  // steps are issued before their stores
  {
    const int kq = (n[0] + 3) >> 2, nq = (N / n[0]) * kq;
    const int lbo = (rup(N / n[0], 128) + 1) * T16;
    const int dl = NT / kq, dk = NT - dl * kq;
    int line = tid / kq, kc = tid - (tid / kq) * kq;
    const double *rb = r + base;
    for (int g0 = tid; g0 < nq; g0 += 2 * NT) {
      double v[2][4];
      int ln[2], kk[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        ln[u] = line;
        kk[u] = kc;
        const bool in = g0 + u * NT < nq;
        const double *p = rb + (long long)line * n[0] + 4 * kc;
#pragma unroll
        for (int e = 0; e < 4; ++e) v[u][e] = (in && 4 * kc + e < n[0]) ? __ldg(p + e) : 0.0;
        line += dl;
        kc += dk;
        if (kc >= kq) { kc -= kq; ++line; }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (g0 + u * NT < nq) {
          float f[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) f[e] = f64_to_op(v[u][e]);
          st4<FMT>(&A[kslab<FMT>(ln[u], 4 * kk[u], lbo)], f);
        }
      }
    }
  }
  if (tid == 0 && !wait_phase_backoff(&tma_bar, 0)) failed = 1;   // B operands have landed
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

  int na = n[0], nb = n[1], nc = n[2];   // current operand dims, a fastest
#pragma unroll 1
  for (int m = 0; m < 6; ++m) {
    const int ntile = rup(nb * nc, 128) / 128;
    const int Kp = rup(na, KSTEP), Np = rup(na, 16);
    // one thread issues the MMAs and waits for them; the others wait at the
    // CTA barrier, which costs no issue slots
    if (tid == 0 && !failed) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t id = idesc(FMT, 128, Np);
      const uint32_t lboA = (uint32_t)(ntile * 128 + 1) * 16u, sboB = (uint32_t)(Kp / T16) * 128u;
      const uint32_t a0 = smem_u32(A), b0 = smem_u32(bm + bslot(bs, m) * bsz);
      for (int t = 0; t < ntile; ++t)
        for (int ks = 0; ks < Kp / KSTEP; ++ks)
          mma<FMT>(tmem + (uint32_t)(t * Np), sdesc(a0 + t * 2048u + ks * 2u * lboA, lboA, 128u),
                   sdesc(b0 + ks * 256, 128, sboB), id, ks > 0 ? 1u : 0u);
      commit(&mbar);
      if (!wait_phase_backoff(&mbar, (uint32_t)(m & 1))) failed = 1;
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (failed) break;
    if (m == 5)
      fd_epilogue<FMT, NT, 2>(tmem, A, na, nb, nc, Np, ntile, Scale{}, s + base,
                              (long long)n[0] * n[1]);
    else if (m == 2) {
      // Lambda for this (patch, component), element (a1 = b, a2 = c,
      // a3 = j): hs (c0 D0[b] + c1 D1[c] + c2 D2[j] + shift) for the full
      // pencil, without hs and shift for the interior one; 2D problems have
      // no third term (their third table is the one-function dummy)
      const float hs = interior ? 1.f : (float)pt.lscale, shf = interior ? 0.f : (float)pt.lshift;
      const float c0 = (float)P[k].lcf[l][0], c1 = (float)P[k].lcf[l][1];
      const float c2 = dim == 3 ? (float)P[k].lcf[l][2] : 0.f;
      const float *Dv[3];
      for (int d = 0; d < 3; ++d) {
        const Tab1D &tb = tabs[d == 0 ? lt0 : (d == 1 ? lt1 : lt2)];
        Dv[d] = fpool + (interior ? tb.Di : tb.D);
      }
      const Scale sc{Dv[0], Dv[1], Dv[2], hs * shf, hs * c0, hs * c1, hs * c2};
      fd_epilogue<FMT, NT, 1>(tmem, A, na, nb, nc, Np, ntile, sc, nullptr, 0);
    } else {
      fd_epilogue<FMT, NT, 0>(tmem, A, na, nb, nc, Np, ntile, Scale{}, nullptr, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // rotate dims: (na, nb, nc) -> (nb, nc, na)
    const int t0 = na;
    na = nb; nb = nc; nc = t0;
  }
  if (failed) {   // give MMAs still in flight one more bounded wait before freeing TMEM
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

static int g_tc_dyn_max, g_slab_dyn_max;

// Shared memory (operand buffer and B slots), B-operand size and TMEM
// columns the kernel needs for one patch (fmt: 2 = TF32, 1 = BF16).
struct TcNeed { int cap, bsz, tcols, nslot; bool ok; };

static TcNeed tc_need(const DevPatch &p, int interior, int fmt) {
  const int kstep = (fmt == 2) ? 8 : 16;
  TcNeed t{0, 0, 32, 1, true};
  for (int l = 0; l < 3; ++l)
    t.nslot = std::max(t.nslot, (int)(b_slots(p.ltab[l][0], p.ltab[l][1], p.ltab[l][2]) >> 24));
  int n[3];
  for (int d = 0; d < 3; ++d) n[d] = interior ? p.ni[d] : p.n[d];
  for (int d = 0; d < 3; ++d) {
    const int na = n[d], nb = n[(d + 1) % 3], nc = n[(d + 2) % 3];
    const int Lp = tc::rup(nb * nc, 128), Kp = tc::rup(na, kstep), Np = tc::rup(na, 16);
    t.cap = std::max(t.cap, Kp * (Lp + 1));   // K-chunk slabs of Lp + 1 rows
    if (Lp + 1 >= (1 << 14)) t.ok = false;    // chunk stride within the descriptor field
    t.bsz = std::max(t.bsz, Np * Kp);
    const int cols = (Lp / 128) * Np;
    while (t.tcols < cols) t.tcols *= 2;
    if (Np > 256) t.ok = false;
  }
  if (t.tcols > 512) t.ok = false;
  return t;
}

static size_t tc_smem(int cap, int bsz, int tcols, int nslot, int fmt) {
  const int esz = (fmt == 2) ? 4 : 2;
  size_t smem = (size_t)(tc::rup(cap, 256) + nslot * tc::rup(bsz, 256)) * esz + 1024;
  // at most 512 / tcols CTAs per SM, so tensor-memory allocation never waits
  // long: the SM's 228 KiB hold 512 / tcols CTAs of this size (with their
  // 1 KiB reserve and static shared memory) but not one more
  const size_t floor_smem = (size_t)228 * 1024 * (size_t)tcols / 512 - 2048;
  return std::max(smem, floor_smem);
}

// Patches in increasing order of need join the single-CTA tensor-core list
// while the combined launch still fits and their own need is at most thr;
// the rest go to the three-pass kernels, else to the SIMT kernel.  One launch
// gives every CTA the shared memory of the largest tensor in the list, so a
// low thr keeps the small tensors' residency high.
static afi_status build_split_thr(afi_ctx *c, int interior, int fmt, size_t thr, TcSplit &sp,
                                  int per) {
  std::vector<std::pair<size_t, int>> order;
  const bool force_slab = (c->opt.variant & AFI_VARIANT_FD_SLAB) != 0;
  for (int k = 0; k < c->npatch; ++k) {
    const TcNeed t = tc_need(c->hp[k], interior, fmt);
    const size_t need = tc_smem(t.cap, t.bsz, t.tcols, t.nslot, fmt);
    if (t.ok && !force_slab && need <= thr) order.push_back({need, k});
  }
  std::sort(order.begin(), order.end());
  std::vector<int> tc, simt;
  std::vector<char> in(c->npatch, 0);
  int cap = 0, bsz = 0, tcols = 32, nslot = 1;
  for (auto &o : order) {
    const TcNeed t = tc_need(c->hp[o.second], interior, fmt);
    const int ncap = std::max(cap, t.cap), nbsz = std::max(bsz, t.bsz), ncols = std::max(tcols, t.tcols);
    const int nsl = std::max(nslot, t.nslot);
    if (tc_smem(ncap, nbsz, ncols, nsl, fmt) > (size_t)g_tc_dyn_max) continue;
    cap = ncap; bsz = nbsz; tcols = ncols; nslot = nsl;
    in[o.second] = 1;
  }
  std::vector<int> big;
  for (int k = 0; k < c->npatch; ++k) {
    if (in[k]) tc.push_back(k);
    else big.push_back(k);
  }
  // tensors too large for one CTA: three-pass slab kernels, else SIMT
  AFI_TRY(slab_build(c, interior, fmt, big, simt, sp, g_slab_dyn_max, per));
  sp.per = per;
  int maxN = 1;
  for (int k : simt) maxN = std::max(maxN, interior ? c->hp[k].Ni : c->hp[k].N);
  sp.ntc = (int)tc.size();
  sp.nsimt = (int)simt.size();
  sp.cap = tc::rup(cap, 256);
  sp.bsz = tc::rup(bsz, 256);
  sp.tcols = tcols;
  sp.smem = tc_smem(cap, bsz, tcols, nslot, fmt);
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

static void free_split(TcSplit &sp) {
  void *p[] = {sp.d_tc, sp.d_simt, sp.d_plane, sp.d_line, sp.d_pbounds, sp.d_lbounds};
  for (void *q : p)
    if (q) cudaFree(q);
  sp = TcSplit{};
}

static afi_status run_split(afi_ctx *c, int interior, int fmt, const TcSplit &sp, const double *r,
                            double *s, cudaStream_t st, int nrhs);

// Project-written autotuner of the FD work split, per (interior, operand
// format): every distinct shared-memory need of the tensors that fit one CTA
// is a candidate threshold (tensors above it take the three-pass kernels),
// and the three-pass kernels take 2 or 4 work items per CTA; each
// combination with work for the three-pass kernels (or the single-CTA split
// alone) is timed on one application (best of three after a warm-up) and
// the fastest kept.  A batch with one combination needs no timing.
// AFI_VARIANT_FD_FIXED keeps every tensor that fits one CTA in the
// single-CTA kernel and two items per three-pass CTA instead.
static afi_status build_split(afi_ctx *c, int interior, int fmt, TcSplit &sp) {
  const size_t all = (size_t)-1;
  std::vector<size_t> cand;
  for (int k = 0; k < c->npatch; ++k) {
    const TcNeed t = tc_need(c->hp[k], interior, fmt);
    const size_t need = tc_smem(t.cap, t.bsz, t.tcols, t.nslot, fmt);
    if (t.ok && need <= (size_t)g_tc_dyn_max) cand.push_back(need);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  const bool fixed = (c->opt.variant & (AFI_VARIANT_FD_FIXED | AFI_VARIANT_FD_SLAB)) != 0 ||
                     c->dim != 3;
  if (fixed) return build_split_thr(c, interior, fmt, all, sp, 2);
  std::vector<size_t> thrs;
  if (cand.size() > 1) {
    thrs.push_back(0);   // every 3D tensor through the three-pass kernels
    thrs.insert(thrs.end(), cand.begin(), cand.end());
  } else {
    thrs.push_back(all);
  }
  if (thrs.size() == 1) {   // one split: time the items per CTA only if it has three-pass work
    AFI_TRY(build_split_thr(c, interior, fmt, all, sp, 2));
    if (sp.nplane == 0) return AFI_OK;
    free_split(sp);
  }
  const long long n = interior ? c->n_int : c->n_dof;
  double *buf = nullptr;
  AFI_CUDA(cudaMalloc(&buf, (size_t)2 * n * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemset(buf, 0, (size_t)2 * n * sizeof(double));
  const double *gate = c->gate;
  c->gate = nullptr;
  afi_status st = AFI_OK;
  float best = 1e30f;
  size_t bthr = all;
  int bper = 2;
  for (size_t thr : thrs)
    for (int per : {2, 4}) {
      TcSplit tmp;
      st = build_split_thr(c, interior, fmt, thr, tmp, per);
      if (st == AFI_OK && per != 2 && tmp.nplane == 0) {   // no three-pass work: same split as per 2
        free_split(tmp);
        continue;
      }
      float tmin = 1e30f;
      for (int rep = 0; rep < 4 && st == AFI_OK; ++rep) {
        cudaEventRecord(e0, 0);
        st = run_split(c, interior, fmt, tmp, buf, buf + n, 0, 1);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tmin = std::min(tmin, ms);
      }
      free_split(tmp);
      if (st != AFI_OK) break;
      if (tmin < best) { best = tmin; bthr = thr; bper = per; }
    }
  c->gate = gate;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  AFI_TRY(st);
  return build_split_thr(c, interior, fmt, bthr, sp, bper);
}

afi_status fd_tc_prepare(afi_ctx *c) {
  const void *fns[] = {(const void *)k_fd_tc<2, 256>, (const void *)k_fd_tc<2, 512>,
                       (const void *)k_fd_tc<1, 256>, (const void *)k_fd_tc<1, 512>};
  size_t stat = 0;
  for (const void *f : fns) {
    cudaFuncAttributes fa;
    AFI_CUDA(cudaFuncGetAttributes(&fa, f));
    stat = std::max(stat, fa.sharedSizeBytes);
  }
  g_tc_dyn_max = c->smem_optin - (int)stat;
  for (const void *f : fns)
    AFI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, g_tc_dyn_max));
  return slab_prepare(c, &g_slab_dyn_max);
}

// Tensor-core FD on the patches that fit, SIMT FP32 FD on the others.  The
// splits are built outside stream capture: the first solve builds them
// before capturing (see fd_tc_ready).
afi_status fd_tc_run(afi_ctx *c, int interior, const double *r, double *s, cudaStream_t st,
                     int nrhs) {
  const int fmt = (c->opt.prec == AFI_FD_BF16) ? 1 : 2;
  TcSplit &sp = c->tcsplit[interior][fmt == 1];
  if (!sp.ready) AFI_TRY(build_split(c, interior, fmt, sp));
  return run_split(c, interior, fmt, sp, r, s, st, nrhs);
}

static afi_status run_split(afi_ctx *c, int interior, int fmt, const TcSplit &sp, const double *r,
                            double *s, cudaStream_t st, int nrhs) {
  const long long stride = interior ? c->n_int : c->n_dof;
  if (sp.ntc) {
    const dim3 grid(sp.ntc, c->dim, nrhs);
    // a grid that fills the SMs at most twice: 512 threads per tensor to
    // shorten each CTA's chain of mode products; else 256 (more CTAs per SM)
    const bool wide = (long long)sp.ntc * c->dim * nrhs <= 2LL * c->nsm;
    auto args = [&](auto kern, int nt) {
      launch(kern, grid, nt, sp.smem, st, (const DevPatch *)c->patches, (const Tab1D *)c->tabs,
             (const float *)c->fpool, c->dim, interior, r, s, sp.cap, sp.bsz, sp.tcols, c->gate,
             c->dflag + 1, stride, (const int *)sp.d_tc, (const unsigned char *)c->tcpool);
    };
    if (fmt == 2) {
      if (wide) args(k_fd_tc<2, 512>, 512);
      else args(k_fd_tc<2, 256>, 256);
    } else {
      if (wide) args(k_fd_tc<1, 512>, 512);
      else args(k_fd_tc<1, 256>, 256);
    }
    AFI_LAUNCH_CHECK();
  }
  AFI_TRY(slab_run(c, interior, fmt, sp, r, s, st, nrhs));
  if (sp.nsimt) AFI_TRY(fd_simt_list(c, interior, sp.d_simt, sp.nsimt, sp.simt_maxN, r, s, st, nrhs));
  return AFI_OK;
}

// The B operands of every table in the canonical K-major layout, for both
// operand formats, full and interior pencils, forward (U^T) and back (U).
__global__ void k_tc_bops(const Tab1D *tabs, int ntab, const double *pool, unsigned char *tcpool) {
  const int t = blockIdx.y, v = blockIdx.z;   // v = bf16 * 4 + interior * 2 + back
  if (t >= ntab) return;
  const Tab1D &T = tabs[t];
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

bool fd_uses_scratch(afi_ctx *c, int interior) {
  int maxN = 1;
  for (auto &p : c->hp) maxN = std::max(maxN, interior ? p.Ni : p.N);
  switch (c->opt.prec) {
    case AFI_FD_FP64: return 2ull * maxN * sizeof(double) > (size_t)c->smem_optin;
    case AFI_FD_FP32: return 2ull * maxN * sizeof(float) > (size_t)c->smem_optin;
    default: {
      const TcSplit &sp = c->tcsplit[interior][c->opt.prec == AFI_FD_BF16];
      if (!sp.ready) return true;   // not known yet: assume it does
      return sp.nplane > 0 ||
             (sp.nsimt > 0 && 2ull * sp.simt_maxN * sizeof(float) > (size_t)c->smem_optin);
    }
  }
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
