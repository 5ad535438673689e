// Geometry-inclusion inexact local solvers (Section 5.2.3, eqs. 5.11-5.13).
//
// For patch k and displacement component l the diagonal block of the
// elasticity stiffness is int grad B_i^T C_l grad B_j over the parametric
// domain, with
//     C_l = [mu J^{-1} J^{-T} + (mu + lambda) J^{-1} e_l e_l^T J^{-T}] |det J|.
// Each diagonal entry of C_l is replaced by a product of univariate factors,
//     [C_l]_aa ~ nu_{l,a}(eta_a) prod_{j != a} beta_{l,j}(eta_j),
// and |det J| ~ prod_j beta_{l,j}(eta_j) (the mass M~_l uses the same beta),
// which gives K~_{l,m} = int nu_{l,m} b_i' b_j' and M~_{l,m} = int beta_{l,m}
// b_i b_j per direction m and the Kronecker forms
//     A~_l = sum_m K~_{l,m} (x) M~_{l,j != m},   M~_l = (x)_m M~_{l,m}.
// The fit (the paper cites it without stating it) is made in the logarithm
// at the Gauss points, where products become sums of univariate functions,
// by Diliberto-Straus sweeps: each factor in turn is set to the mid-range
// (max + min) / 2 of its residual over the other variables, a shared factor
// over every target it enters, until no factor moves by more than 1e-14
// (at most 500 sweeps).  The local solvers are then
//     P_A^{-1} = D_A^{-1/2} (A~_l + H^{-2} M~_l)^{-1} D_A^{-1/2}   (eq. 5.12),
//     S = D_S^{1/2} S~_l D_S^{1/2},  S~_l the Schur complement of A~_l (eq. 5.13),
// with D_A = diag(A_ll + H^{-2} M) / diag(A~_l + H^{-2} M~_l) and
// D_S = diag(A_ll) / diag(A~_l), applied by Algorithm 1 with the eigenpairs
// of (K~_{l,m}, M~_{l,m}) through the same FD and Schur kernels as the plain
// solvers: every (patch, component, direction) gets its own univariate table.
//
// GPU layout of the fit: the targets log [C_l]_aa and log |det J| live on
// the patch's Gauss-point grid (the quadrature geometry's order, q1
// fastest); the factors of fit (k, l) live in per-direction slots.  A sweep
// is eight launches: the nu update (all directions at once, they do not
// depend on each other), then beta_1, beta_2, beta_3 in order, each followed
// by a small kernel that turns the reduced max / min into the new factor.
// The sweeps run in 64-bit fixed point: every logarithm is held as the
// integer round(x 2^52) (|x| < 2^6), so the sums, differences, maxima and
// minima of a sweep are exact integer operations on the integer pipes (this
// GPU's FP64 pipe is a small fraction of its integer rate), independent of
// the reduction order, and the mid-range (hi + lo) / 2 and the stopping rule
// (no factor moves by more than 1e-14 = 45 units of 2^-52) differ from
// double-precision arithmetic only by rounding at the 2^-52 level.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>

namespace afi {

afi_status build_1d_tables_range(afi_ctx *c, int t0, int t1, bool basis);

namespace {

constexpr int kGeoMaxSweeps = 500;
constexpr double kFix = 4503599627370496.0;   // 2^52
constexpr long long kGeoTolFix = 45;           // floor(1e-14 * 2^52)
constexpr double kGeoMaxLog = 64.0;            // |log| < 2^6: |value| < 2^58, every sum < 2^61

struct Fit {
  long long *LD;   // [DIM * DIM][nqp]: log [C_l]_aa in fixed point, (l * DIM + a) * nqp + gq
  long long *L0;   // [nqp]: log |det J| in fixed point
  long long *fa, *fb;   // log nu, log beta: [DIM][Qs] slots, l * Qs + qloff + dir offset + q
  long long *mx, *mn;   // reduction slots, same layout
  long long *move;      // per fit (k * DIM + l): largest factor change this sweep
  int *done;            // per fit
  int *remaining;       // fits not done after the last sweep
  int *bad;             // a logarithm out of the fixed-point range
  long long Qs;
};

__device__ __forceinline__ long long slot(const Fit &F, const DevPatch &pt, int l, int dir, int q) {
  const int off = (dir == 0) ? 0 : (dir == 1 ? pt.nq[0] : pt.nq[0] + pt.nq[1]);
  return (long long)l * F.Qs + pt.qloff + off + q;
}

__device__ __forceinline__ long long to_fix(double x, int *bad) {
  if (!(fabs(x) < kGeoMaxLog)) { atomicExch(bad, 1); return 0; }
  return __double2ll_rn(x * kFix);
}

// targets at every Gauss point: log of the DIM diagonal entries of C_l for
// every component l, and log |det J| (= log(w |det J| / w))
template <int DIM>
__global__ void k_geo_targets(const DevPatch *P, const Tab1D *tabs, const double *pool,
                              const double *qgeo, long long nqp, Fit F) {
  const DevPatch pt = P[blockIdx.y];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= pt.NQ) return;
  const int q1 = q % pt.nq[0], q2 = (q / pt.nq[0]) % pt.nq[1], q3 = q / (pt.nq[0] * pt.nq[1]);
  const double w = pool[tabs[pt.tab[0]].qw + q1] * pool[tabs[pt.tab[1]].qw + q2] *
                   pool[tabs[pt.tab[2]].qw + q3];
  const long long gq = pt.qoff + q;
  double Q[DIM][DIM];
  for (int a = 0; a < DIM; ++a)
    for (int x = 0; x < DIM; ++x) Q[a][x] = qgeo[(long long)(a * DIM + x) * nqp + gq];
  const double det = qgeo[(long long)(DIM * DIM) * nqp + gq] / w;
  F.L0[gq] = to_fix(log(det), F.bad);
  for (int l = 0; l < DIM; ++l)
    for (int a = 0; a < DIM; ++a) {
      double s2 = 0.0;
      for (int x = 0; x < DIM; ++x) s2 += Q[a][x] * Q[a][x];
      const double cval = (pt.mu * s2 + (pt.mu + pt.lam) * Q[a][l] * Q[a][l]) * det;
      F.LD[(long long)(l * DIM + a) * nqp + gq] = to_fix(log(cval), F.bad);
    }
}

__device__ __forceinline__ void red_pair(long long &hi, long long &lo, long long v) {
  hi = max(hi, v);
  lo = min(lo, v);
}

__device__ __forceinline__ void warp_pair(long long &hi, long long &lo) {
  for (int o = 16; o > 0; o >>= 1) {
    hi = max(hi, (long long)__shfl_xor_sync(0xffffffffu, hi, o));
    lo = min(lo, (long long)__shfl_xor_sync(0xffffffffu, lo, o));
  }
}

// max / min over the CTA (256 threads) added to the slot (thread 0)
__device__ __forceinline__ void block_to_slot(long long hi, long long lo, long long *mx,
                                              long long *mn, long long s) {
  __shared__ long long sh[2][8];
  warp_pair(hi, lo);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][w] = hi; sh[1][w] = lo; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { hi = max(hi, sh[0][i]); lo = min(lo, sh[1][i]); }
    atomicMax(mx + s, hi);
    atomicMin(mn + s, lo);
  }
  __syncthreads();
}

constexpr long long kLo = -0x7FFFFFFFFFFFFFFFLL, kHi = 0x7FFFFFFFFFFFFFFFLL;

// One plane q3 of one fit (k, l) per CTA (blockIdx.y = k * DIM + l).
// PHASE 0: the nu_a residuals log[C_l]_aa - sum_{j != a} log beta_j reduced
// per q_a; PHASE 1 + j: the residuals of every target that contains beta_j
// (log |det J| - sum_{j' != j} log beta_j' and, for a != j,
// log[C_l]_aa - log nu_a - sum_{j' != a, j} log beta_j') reduced per q_j.
template <int DIM, int PHASE>
__global__ void __launch_bounds__(256) k_geo_sweep(const DevPatch *P, long long nqp, Fit F) {
  const int f = blockIdx.y, k = f / DIM, l = f - k * DIM;
  if (F.done[f]) return;
  const DevPatch pt = P[k];
  const int n1 = pt.nq[0], n2 = pt.nq[1], n3 = pt.nq[2];
  const int q3 = blockIdx.x;
  if (q3 >= n3) return;
  const long long g0 = pt.qoff + (long long)q3 * n1 * n2;
  const long long *b[3], *a[3];
  for (int d = 0; d < 3; ++d) {
    b[d] = F.fb + slot(F, pt, l, d, 0);
    a[d] = F.fa + slot(F, pt, l, d, 0);
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (PHASE == 0) {
    // residual of target a = dir at (q1, q2, q3): factors beta_j, j != dir
    auto val = [&](int dir, int q1, int q2) -> long long {
      const int qq[3] = {q1, q2, q3};
      long long s = 0;
      for (int j = 0; j < DIM; ++j)
        if (j != dir) s += b[j][qq[j]];
      return F.LD[(long long)(l * DIM + dir) * nqp + g0 + q1 + (long long)n1 * q2] - s;
    };
    for (int dir = 0; dir < DIM; ++dir) {
      if (dir == 0) {
        for (int q1 = tid; q1 < n1; q1 += blockDim.x) {
          long long hi = kLo, lo = kHi;
          for (int q2 = 0; q2 < n2; ++q2) red_pair(hi, lo, val(0, q1, q2));
          atomicMax(F.mx + slot(F, pt, l, 0, q1), hi);
          atomicMin(F.mn + slot(F, pt, l, 0, q1), lo);
        }
      } else if (dir == 1) {
        for (int q2 = warp; q2 < n2; q2 += (blockDim.x >> 5)) {
          long long hi = kLo, lo = kHi;
          for (int q1 = lane; q1 < n1; q1 += 32) red_pair(hi, lo, val(1, q1, q2));
          warp_pair(hi, lo);
          if (lane == 0) {
            atomicMax(F.mx + slot(F, pt, l, 1, q2), hi);
            atomicMin(F.mn + slot(F, pt, l, 1, q2), lo);
          }
        }
      } else {
        long long hi = kLo, lo = kHi;
        for (int i = tid; i < n1 * n2; i += blockDim.x) red_pair(hi, lo, val(2, i % n1, i / n1));
        block_to_slot(hi, lo, F.mx, F.mn, slot(F, pt, l, 2, q3));
      }
    }
    return;
  }
  constexpr int j = PHASE - 1;   // the beta being updated
  // max / min over every target containing beta_j at one point
  auto bval = [&](int q1, int q2, long long &hi, long long &lo) {
    const long long gq = g0 + q1 + (long long)n1 * q2;
    const int qq[3] = {q1, q2, q3};
    long long s = 0;
    for (int jj = 0; jj < DIM; ++jj)
      if (jj != j) s += b[jj][qq[jj]];
    red_pair(hi, lo, F.L0[gq] - s);
    for (int i = 0; i < DIM; ++i) {
      if (i == j) continue;
      long long t = a[i][qq[i]];
      for (int jj = 0; jj < DIM; ++jj)
        if (jj != i && jj != j) t += b[jj][qq[jj]];   // at most one in 3D, none in 2D
      red_pair(hi, lo, F.LD[(long long)(l * DIM + i) * nqp + gq] - t);
    }
  };
  if (j == 0) {
    for (int q1 = tid; q1 < n1; q1 += blockDim.x) {
      long long hi = kLo, lo = kHi;
      for (int q2 = 0; q2 < n2; ++q2) bval(q1, q2, hi, lo);
      atomicMax(F.mx + slot(F, pt, l, 0, q1), hi);
      atomicMin(F.mn + slot(F, pt, l, 0, q1), lo);
    }
  } else if (j == 1) {
    for (int q2 = warp; q2 < n2; q2 += (blockDim.x >> 5)) {
      long long hi = kLo, lo = kHi;
      for (int q1 = lane; q1 < n1; q1 += 32) bval(q1, q2, hi, lo);
      warp_pair(hi, lo);
      if (lane == 0) {
        atomicMax(F.mx + slot(F, pt, l, 1, q2), hi);
        atomicMin(F.mn + slot(F, pt, l, 1, q2), lo);
      }
    }
  } else {
    long long hi = kLo, lo = kHi;
    for (int i = tid; i < n1 * n2; i += blockDim.x) bval(i % n1, i / n1, hi, lo);
    block_to_slot(hi, lo, F.mx, F.mn, slot(F, pt, l, 2, q3));
  }
}

// New factors from the reduced slots (PHASE 0: nu in every direction;
// PHASE 1 + j: beta_j), the largest change per fit, and the slots reset.
// The mid-range of two fixed-point values is their sum shifted right once
// (targets and factors stay below 2^58 in magnitude, residuals of three
// terms below 2^60, so hi + lo cannot overflow).
template <int DIM, int PHASE>
__global__ void k_geo_fin(const DevPatch *P, Fit F) {
  const int f = blockIdx.y, k = f / DIM, l = f - k * DIM;
  const DevPatch pt = P[k];
  const bool live = !F.done[f];
  long long mv = 0;
  for (int dir = (PHASE == 0 ? 0 : PHASE - 1); dir < (PHASE == 0 ? DIM : PHASE); ++dir)
    for (int q = threadIdx.x; q < pt.nq[dir]; q += blockDim.x) {
      const long long s = slot(F, pt, l, dir, q);
      if (live) {
        const long long nw = (F.mx[s] + F.mn[s]) >> 1;
        long long *fac = (PHASE == 0 ? F.fa : F.fb) + s;
        mv = max(mv, nw > *fac ? nw - *fac : *fac - nw);
        *fac = nw;
      }
      F.mx[s] = kLo;
      F.mn[s] = kHi;
    }
  if (live) atomicMax(F.move + f, mv);
}

// End of a sweep: fits whose factors all moved by at most 1e-14 are done.
__global__ void k_geo_done(Fit F, int nfit) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int f = threadIdx.x; f < nfit; f += blockDim.x) {
    if (!F.done[f] && F.move[f] <= kGeoTolFix) F.done[f] = 1;
    F.move[f] = 0;
    mine += F.done[f] ? 0 : 1;
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) *F.remaining = cnt;
}

// nu = exp(log nu), beta = exp(log beta) into the per-(patch, component,
// direction) tables (weights of the univariate K~ and M~).
template <int DIM>
__global__ void k_geo_weights(const DevPatch *P, const Tab1D *tabs, double *pool, Fit F) {
  const int f = blockIdx.y, k = f / DIM, l = f - k * DIM;
  const DevPatch pt = P[k];
  for (int m = 0; m < DIM; ++m) {
    const Tab1D T = tabs[pt.ltab[l][m]];
    for (int q = threadIdx.x; q < pt.nq[m]; q += blockDim.x) {
      const long long s = slot(F, pt, l, m, q);
      pool[T.wK + q] = exp((double)F.fa[s] / kFix);
      pool[T.wM + q] = exp((double)F.fb[s] / kFix);
    }
  }
}

// Per node of a patch: the diagonal of the scalar mass M (quadrature over
// the node's support), then per component l the scalings
//   D_A = (A_ll,ii + M_ii / H^2) / (A~_l + M~_l / H^2)_ii,  D_A^{-1/2} stored;
//   D_S = A_ll,ii / (A~_l)_ii,                            D_S^{1/2} stored.
// The Kronecker diagonals are products of the univariate diagonals.
template <int DIM>
__global__ void k_geo_diag(const DevPatch *P, const Tab1D *tabs, const double *pool,
                           const double *qgeo, long long nqp, const double *stencil, double *dA,
                           double *dS) {
  const DevPatch pt = P[blockIdx.y];
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= pt.N) return;
  const int id[3] = {node % pt.n[0], (node / pt.n[0]) % pt.n[1], node / (pt.n[0] * pt.n[1])};
  int lo[3], hi[3], ng[3];
  Tab1D T[3] = {tabs[pt.tab[0]], tabs[pt.tab[1]], tabs[pt.tab[2]]};
  for (int d = 0; d < 3; ++d) {
    ng[d] = T[d].p + 1;
    lo[d] = max(id[d] - T[d].p, 0);
    hi[d] = min(id[d], max(T[d].nel - 1, 0));
  }
  double mii = 0.0;
  for (int e2 = lo[2]; e2 <= hi[2]; ++e2)
    for (int g2 = 0; g2 < ng[2]; ++g2) {
      const int q2 = e2 * ng[2] + g2;
      const double v2 = pool[T[2].val + (long long)q2 * ng[2] + id[2] - e2];
      for (int e1 = lo[1]; e1 <= hi[1]; ++e1)
        for (int g1 = 0; g1 < ng[1]; ++g1) {
          const int q1 = e1 * ng[1] + g1;
          const double v1 = v2 * pool[T[1].val + (long long)q1 * ng[1] + id[1] - e1];
          for (int e0 = lo[0]; e0 <= hi[0]; ++e0)
            for (int g0 = 0; g0 < ng[0]; ++g0) {
              const int q0 = e0 * ng[0] + g0;
              const double bb = v1 * pool[T[0].val + (long long)q0 * ng[0] + id[0] - e0];
              const long long gq = pt.qoff + q0 + (long long)pt.nq[0] * (q1 + (long long)pt.nq[1] * q2);
              mii += qgeo[(long long)(DIM * DIM) * nqp + gq] * bb * bb;
            }
        }
    }
  const double ih2 = 1.0 / (pt.H * pt.H);
  const int oc = pt.p + pt.W[0] * (pt.p + pt.W[1] * (DIM == 3 ? pt.p : 0));
  const long long np = id[0] + (long long)pt.n1p * (id[1] + (long long)pt.n[1] * id[2]);
  for (int l = 0; l < DIM; ++l) {
    double kd[3], md[3];
    for (int m = 0; m < DIM; ++m) {
      const Tab1D G = tabs[pt.ltab[l][m]];
      kd[m] = pool[G.K + (long long)id[m] * G.n + id[m]];
      md[m] = pool[G.M + (long long)id[m] * G.n + id[m]];
    }
    // Kronecker diagonals, products formed from direction 1 up
    double at = 0.0, mt = 1.0;
    for (int m = 0; m < DIM; ++m) {
      double t = 1.0;
      for (int j = 0; j < DIM; ++j) t = (j == m ? kd[j] : md[j]) * t;
      at = (m == 0) ? t : at + t;
    }
    for (int j = 0; j < DIM; ++j) mt = md[j] * mt;
    const double all = stencil[pt.soff + ((long long)(l * DIM + l) * pt.S + oc) * pt.NP + np];
    const double DA = (all + mii * ih2) / (at + mt * ih2);
    const double DS = all / at;
    const long long i = pt.off + (long long)l * pt.N + node;
    dA[i] = 1.0 / sqrt(DA);
    dS[i] = sqrt(DS);
  }
}

__global__ void k_geo_scale(const double *x, const double *d, double *y, long n, int nrhs,
                            const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  const long long tot = (long long)n * nrhs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * d[i % n];
}

template <int DIM>
afi_status geo_fit(afi_ctx *c, Fit &F) {
  const int nfit = c->npatch * DIM;
  int maxq = 1, maxNQ = 1;
  for (auto &p : c->hp) { maxq = std::max(maxq, p.nq[2]); maxNQ = std::max(maxNQ, p.NQ); }
  launch(k_geo_targets<DIM>, dim3((maxNQ + 127) / 128, c->npatch), 128, 0, 0,
         (const DevPatch *)c->patches, (const Tab1D *)c->tabs, (const double *)c->dpool,
         (const double *)c->qgeo, c->nqp, F);
  AFI_LAUNCH_CHECK();
  {
    int bad = 0;
    AFI_CUDA(cudaMemcpy(&bad, F.bad, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) {
      set_error("AFI_VARIANT_GEO: an elasticity coefficient or |det J| outside exp(+-64)");
      return AFI_EINVAL;
    }
  }
  const dim3 gs(maxq, nfit), gf(1, nfit);
  for (int sw = 0; sw < kGeoMaxSweeps; ++sw) {
    launch(k_geo_sweep<DIM, 0>, gs, 256, 0, 0, (const DevPatch *)c->patches, c->nqp, F);
    launch(k_geo_fin<DIM, 0>, gf, 256, 0, 0, (const DevPatch *)c->patches, F);
    launch(k_geo_sweep<DIM, 1>, gs, 256, 0, 0, (const DevPatch *)c->patches, c->nqp, F);
    launch(k_geo_fin<DIM, 1>, gf, 256, 0, 0, (const DevPatch *)c->patches, F);
    launch(k_geo_sweep<DIM, 2>, gs, 256, 0, 0, (const DevPatch *)c->patches, c->nqp, F);
    launch(k_geo_fin<DIM, 2>, gf, 256, 0, 0, (const DevPatch *)c->patches, F);
    if (DIM == 3) {
      launch(k_geo_sweep<DIM, 3>, gs, 256, 0, 0, (const DevPatch *)c->patches, c->nqp, F);
      launch(k_geo_fin<DIM, 3>, gf, 256, 0, 0, (const DevPatch *)c->patches, F);
    }
    launch(k_geo_done, 1, 256, 0, 0, F, nfit);
    AFI_LAUNCH_CHECK();
    if (sw % 8 == 7 || sw == kGeoMaxSweeps - 1) {
      int rem = 0;
      AFI_CUDA(cudaMemcpy(&rem, F.remaining, sizeof(int), cudaMemcpyDeviceToHost));
      if (rem == 0) break;
    }
  }
  launch(k_geo_weights<DIM>, gf, 256, 0, 0, (const DevPatch *)c->patches, (const Tab1D *)c->tabs,
         c->dpool, F);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

}  // namespace

// y = x * d elementwise over nrhs stacked vectors of length n (d repeats).
afi_status geo_scale(afi_ctx *c, const double *x, const double *d, double *y, long n, int nrhs,
                     cudaStream_t st) {
  const long long tot = (long long)n * nrhs;
  const unsigned nb = (unsigned)std::min<long long>((tot + 255) / 256, 8LL * c->nsm);
  launch(k_geo_scale, nb, 256, 0, st, x, d, y, n, nrhs, c->gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

// Setup of the geometry-inclusion local solvers, after the quadrature
// geometry and the stiffness exist: the fit, the per-(patch, component,
// direction) univariate matrices and their eigenpairs, and the scalings.
afi_status geo_setup(afi_ctx *c) {
  const int D = c->dim;
  if (!c->qgeo || !c->stencil) {
    set_error("AFI_VARIANT_GEO needs the geometry and the stiffness (not AFI_VARIANT_LOCAL_ONLY)");
    return AFI_EINVAL;
  }
  Fit F{};
  F.Qs = 0;
  for (auto &p : c->hp) F.Qs += p.nq[0] + p.nq[1] + p.nq[2];
  const size_t nslot = (size_t)D * F.Qs, nfit = (size_t)c->npatch * D;
  std::vector<void *> tmp;
  auto talloc = [&](void **p, size_t bytes) -> afi_status {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMalloc(geometry-inclusion fit, ") + std::to_string(bytes) +
                "): " + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? AFI_ENOMEM : AFI_ECUDA;
    }
    tmp.push_back(*p);
    return AFI_OK;
  };
  afi_status st = AFI_OK;
  auto run = [&]() -> afi_status {
    AFI_TRY(talloc((void **)&F.LD, (size_t)D * D * c->nqp * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.L0, (size_t)c->nqp * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.fa, nslot * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.fb, nslot * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.mx, nslot * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.mn, nslot * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.move, nfit * sizeof(long long)));
    AFI_TRY(talloc((void **)&F.done, (nfit + 2) * sizeof(int)));
    F.remaining = F.done + nfit;
    F.bad = F.done + nfit + 1;
    AFI_CUDA(cudaMemset(F.fa, 0, nslot * sizeof(long long)));
    AFI_CUDA(cudaMemset(F.fb, 0, nslot * sizeof(long long)));
    {   // empty reduction slots: max = lowest, min = highest
      std::vector<long long> lo(nslot, -0x7FFFFFFFFFFFFFFFLL), hi(nslot, 0x7FFFFFFFFFFFFFFFLL);
      AFI_CUDA(cudaMemcpy(F.mx, lo.data(), nslot * sizeof(long long), cudaMemcpyHostToDevice));
      AFI_CUDA(cudaMemcpy(F.mn, hi.data(), nslot * sizeof(long long), cudaMemcpyHostToDevice));
    }
    AFI_CUDA(cudaMemset(F.move, 0, nfit * sizeof(long long)));
    AFI_CUDA(cudaMemset(F.done, 0, (nfit + 2) * sizeof(int)));
    AFI_TRY(D == 3 ? geo_fit<3>(c, F) : geo_fit<2>(c, F));
    // univariate K~, M~ and their eigenpairs for the per-(patch, component,
    // direction) tables
    AFI_TRY(build_1d_tables_range(c, c->nbase_tab, (int)c->htab.size(), false));
    AFI_TRY(dalloc(c, (void **)&c->geo_dA, (size_t)c->n_dof * sizeof(double)));
    AFI_TRY(dalloc(c, (void **)&c->geo_dS, (size_t)c->n_dof * sizeof(double)));
    AFI_TRY(dalloc(c, (void **)&c->geo_tmp, (size_t)c->n_dof * sizeof(double)));
    int maxN = 1;
    for (auto &p : c->hp) maxN = std::max(maxN, p.N);
    const dim3 g((maxN + 127) / 128, c->npatch);
    if (D == 3)
      launch(k_geo_diag<3>, g, 128, 0, 0, (const DevPatch *)c->patches, (const Tab1D *)c->tabs,
             (const double *)c->dpool, (const double *)c->qgeo, c->nqp,
             (const double *)c->stencil, c->geo_dA, c->geo_dS);
    else
      launch(k_geo_diag<2>, g, 128, 0, 0, (const DevPatch *)c->patches, (const Tab1D *)c->tabs,
             (const double *)c->dpool, (const double *)c->qgeo, c->nqp,
             (const double *)c->stencil, c->geo_dA, c->geo_dS);
    AFI_LAUNCH_CHECK();
    AFI_CUDA(cudaDeviceSynchronize());
    return AFI_OK;
  };
  st = run();
  for (void *p : tmp) cudaFree(p);
  return st;
}

}  // namespace afi
