// Geometry at the quadrature points and assembly of the patch stiffness
// matrices A^(k) of the elasticity form (eq. 3.1),
//     A[(l,i),(m,j)] = int mu (delta_lm grad B_i . grad B_j + d_m B_i d_l B_j)
//                          + lambda d_l B_i d_m B_j  dx,
// stored as a per-node stencil over the (2p+1)^d neighbours, in FP64.  In
// parametric variables, with Q = J^{-1} and wd = w |det J|,
//     A_lm[i][j] = sum_q sum_{a,b} C^{lm}_{ab}(q) dB_i/deta_a dB_j/deta_b,
//     C^{lm}_{ab} = wd [mu delta_lm (Q Q^T)_ab + mu Q_am Q_bl + lambda Q_al Q_bm].
// The sum over the tensor-product quadrature is factorised direction by
// direction (three passes).  Also: load vectors f = M c (mapped mass, eq. 4.8)
// and the Lame-parameter gradient quadrature.
#include "common.cuh"

namespace afi {

__device__ __forceinline__ const double *tab_val(const Tab1D &T, const double *pool, int q) {
  return pool + T.val + (long long)q * (T.p + 1);
}
__device__ __forceinline__ const double *tab_der(const Tab1D &T, const double *pool, int q) {
  return pool + T.der + (long long)q * (T.p + 1);
}

// --------------------------------------------------------------- geometry
// Q = J^{-1} ([a][x]) and w|det J| at every quadrature point; flag on det <= 0.
template <int DIM>
__global__ void k_geometry(const DevPatch *P, const Tab1D *tabs, const double *pool,
                           const double *ctrl, double *qgeo, long long nqp, int *flag) {
  const DevPatch pt = P[blockIdx.y];
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= pt.NQ) return;
  int qd[3] = {q % pt.nq[0], (q / pt.nq[0]) % pt.nq[1], q / (pt.nq[0] * pt.nq[1])};
  const Tab1D T0 = tabs[pt.tab[0]], T1 = tabs[pt.tab[1]], T2 = tabs[pt.tab[2]];
  const int ng0 = T0.p + 1, ng1 = T1.p + 1, ng2 = T2.p + 1;
  const int e0 = qd[0] / ng0, e1 = qd[1] / ng1, e2 = qd[2] / ng2;
  const double *v0 = tab_val(T0, pool, qd[0]), *d0 = tab_der(T0, pool, qd[0]);
  const double *v1 = tab_val(T1, pool, qd[1]), *d1 = tab_der(T1, pool, qd[1]);
  const double *v2 = tab_val(T2, pool, qd[2]), *d2 = tab_der(T2, pool, qd[2]);
  double J[DIM][DIM];
  for (int x = 0; x < DIM; ++x)
    for (int a = 0; a < DIM; ++a) J[x][a] = 0.0;
  const double *X = ctrl + pt.xoff;
  for (int t2 = 0; t2 < ng2; ++t2)
    for (int t1 = 0; t1 < ng1; ++t1)
      for (int t0 = 0; t0 < ng0; ++t0) {
        int node = (e0 + t0) + pt.n[0] * ((e1 + t1) + pt.n[1] * (e2 + t2));
        double g[3];
        g[0] = d0[t0] * v1[t1] * v2[t2];
        g[1] = v0[t0] * d1[t1] * v2[t2];
        g[2] = v0[t0] * v1[t1] * d2[t2];
        for (int x = 0; x < DIM; ++x) {
          double xv = X[(long long)node * DIM + x];
          for (int a = 0; a < DIM; ++a) J[x][a] += xv * g[a];
        }
      }
  double det, Q[DIM][DIM];
  if (DIM == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double id = 1.0 / det;
    // Q = J^{-1}: Q[a][x]
    Q[0][0] = J[1][1] * id;  Q[0][1] = -J[0][1] * id;
    Q[1][0] = -J[1][0] * id; Q[1][1] = J[0][0] * id;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    double id = 1.0 / det;
    Q[0][0] = c00 * id;
    Q[1][0] = c01 * id;
    Q[2][0] = c02 * id;
    Q[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Q[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Q[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Q[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Q[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Q[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  }
  if (!(det > 0.0)) atomicExch(flag, 1);
  const double w = pool[T0.qw + qd[0]] * pool[T1.qw + qd[1]] * pool[T2.qw + qd[2]];
  const long long gq = pt.qoff + q;
  for (int a = 0; a < DIM; ++a)
    for (int x = 0; x < DIM; ++x) qgeo[(long long)(a * DIM + x) * nqp + gq] = Q[a][x];
  qgeo[(long long)(DIM * DIM) * nqp + gq] = w * fabs(det);
}

// ----------------------------------------------------- stiffness assembly
// channel index of the pair (l <= m)
template <int DIM> struct LM;
template <> struct LM<2> { static constexpr int n = 3; };
template <> struct LM<3> { static constexpr int n = 6; };
__device__ __forceinline__ void lm_of(int DIMv, int c, int &l, int &m) {
  if (DIMv == 2) { const int L[3] = {0, 0, 1}, M[3] = {0, 1, 1}; l = L[c]; m = M[c]; }
  else { const int L[6] = {0, 0, 0, 1, 1, 2}, M[6] = {0, 1, 2, 1, 2, 2}; l = L[c]; m = M[c]; }
}

// Pass 1: contract direction 1.  T1[lm][q3][q2][o1*n1 + i1] for one (a, b).
template <int DIM>
__global__ void k_asm1(const DevPatch *P, const int *batch, const Tab1D *tabs,
                       const double *pool, const double *qgeo, long long nqp, double *T1,
                       const long long *t1off, int a, int b) {
  constexpr int NLM = LM<DIM>::n;
  const int k = batch[blockIdx.y];
  const DevPatch pt = P[k];
  const int line = blockIdx.x;
  if (line >= pt.nq[1] * pt.nq[2]) return;
  const int q2 = line % pt.nq[1], q3 = line / pt.nq[1];
  const int nq1 = pt.nq[0];
  extern __shared__ double Cs[];   // [NLM][nq1]
  for (int q1 = threadIdx.x; q1 < nq1; q1 += blockDim.x) {
    long long gq = pt.qoff + q1 + (long long)nq1 * (q2 + (long long)pt.nq[1] * q3);
    double Q[DIM][DIM];
    for (int aa = 0; aa < DIM; ++aa)
      for (int x = 0; x < DIM; ++x) Q[aa][x] = qgeo[(long long)(aa * DIM + x) * nqp + gq];
    double wd = qgeo[(long long)(DIM * DIM) * nqp + gq];
    double qq = 0.0;
    for (int x = 0; x < DIM; ++x) qq += Q[a][x] * Q[b][x];
    for (int c = 0; c < NLM; ++c) {
      int l, m;
      lm_of(DIM, c, l, m);
      double v = pt.mu * Q[a][m] * Q[b][l] + pt.lam * Q[a][l] * Q[b][m];
      if (l == m) v += pt.mu * qq;
      Cs[c * nq1 + q1] = wd * v;
    }
  }
  __syncthreads();
  const Tab1D T = tabs[pt.tab[0]];
  const int p = T.p, ng = p + 1, n1 = pt.n[0], W1 = pt.W[0], cols = W1 * n1;
  const int nel = T.nel;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    int o = c / n1, i1 = c % n1, j1 = i1 + o - p;
    double acc[NLM];
    for (int t = 0; t < NLM; ++t) acc[t] = 0.0;
    if (j1 >= 0 && j1 < n1) {
      int elo = max(max(i1, j1) - p, 0), ehi = min(min(i1, j1), nel - 1);
      for (int e = elo; e <= ehi; ++e)
        for (int g = 0; g < ng; ++g) {
          int q1 = e * ng + g;
          const double *vv = tab_val(T, pool, q1), *dd = tab_der(T, pool, q1);
          double f = (a == 0 ? dd[i1 - e] : vv[i1 - e]) * (b == 0 ? dd[j1 - e] : vv[j1 - e]);
          for (int t = 0; t < NLM; ++t) acc[t] += Cs[t * nq1 + q1] * f;
        }
    }
    for (int t = 0; t < NLM; ++t)
      T1[t1off[blockIdx.y] + (((long long)t * pt.nq[2] + q3) * pt.nq[1] + q2) * cols + c] = acc[t];
  }
}

// Pass 2: contract direction 2, accumulate into the direction-3 derivative
// pattern pat = 2*(a == 3rd) + (b == 3rd).  T2[pat][lm][q3][o2*n2+i2][c1].
template <int DIM>
__global__ void k_asm2(const DevPatch *P, const int *batch, const Tab1D *tabs,
                       const double *pool, const double *T1, const long long *t1off,
                       double *T2, const long long *t2off, int a, int b) {
  constexpr int NLM = LM<DIM>::n;
  const int k = batch[blockIdx.y];
  const DevPatch pt = P[k];
  const int q3 = blockIdx.x;
  if (q3 >= pt.nq[2]) return;
  const Tab1D T = tabs[pt.tab[1]];
  const int p = T.p, ng = p + 1, nel = T.nel;
  const int n2 = pt.n[1], cols1 = pt.W[0] * pt.n[0], cols2 = pt.W[1] * n2, nq2 = pt.nq[1];
  const int pat = (DIM == 3) ? ((a == 2) * 2 + (b == 2)) : 0;
  const double *t1 = T1 + t1off[blockIdx.y];
  double *t2 = T2 + t2off[blockIdx.y];
  for (int c = threadIdx.x; c < cols1; c += blockDim.x) {
    for (int c2 = 0; c2 < cols2; ++c2) {
      int o = c2 / n2, i2 = c2 % n2, j2 = i2 + o - p;
      if (j2 < 0 || j2 >= n2) continue;
      double acc[NLM];
      for (int t = 0; t < NLM; ++t) acc[t] = 0.0;
      int elo = max(max(i2, j2) - p, 0), ehi = min(min(i2, j2), nel - 1);
      for (int e = elo; e <= ehi; ++e)
        for (int g = 0; g < ng; ++g) {
          int q2 = e * ng + g;
          const double *vv = tab_val(T, pool, q2), *dd = tab_der(T, pool, q2);
          double f = (a == 1 ? dd[i2 - e] : vv[i2 - e]) * (b == 1 ? dd[j2 - e] : vv[j2 - e]);
          for (int t = 0; t < NLM; ++t)
            acc[t] += t1[(((long long)t * pt.nq[2] + q3) * nq2 + q2) * cols1 + c] * f;
        }
      for (int t = 0; t < NLM; ++t)
        t2[((((long long)pat * NLM + t) * pt.nq[2] + q3) * cols2 + c2) * cols1 + c] += acc[t];
    }
  }
}

// Pass 3: contract direction 3 and write the upper blocks (l <= m) of the
// stencil A[l][m][o][node], o = o1 + W1 (o2 + W2 o3).
template <int DIM>
__global__ void k_asm3(const DevPatch *P, const int *batch, const Tab1D *tabs,
                       const double *pool, const double *T2, const long long *t2off,
                       double *A) {
  constexpr int NLM = LM<DIM>::n;
  const int k = batch[blockIdx.y];
  const DevPatch pt = P[k];
  const int n1 = pt.n[0], n2 = pt.n[1], n3 = pt.n[2];
  const int cols1 = pt.W[0] * n1, cols2 = pt.W[1] * n2;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)cols1 * cols2) return;
  const int c = (int)(idx % cols1), c2 = (int)(idx / cols1);
  const int p = pt.p;
  const int o1 = c / n1, i1 = c % n1, o2 = c2 / n2, i2 = c2 % n2;
  const int j1 = i1 + o1 - p, j2 = i2 + o2 - p;
  const bool v12 = (j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < n2);
  const double *t2 = T2 + t2off[blockIdx.y];
  const Tab1D T = tabs[pt.tab[2]];
  const int ng = T.p + 1, nel = T.nel, nq3 = pt.nq[2], W3 = pt.W[2];
  for (int i3 = 0; i3 < n3; ++i3)
    for (int o3 = 0; o3 < W3; ++o3) {
      int j3 = (DIM == 3) ? i3 + o3 - p : i3;
      double acc[NLM];
      for (int t = 0; t < NLM; ++t) acc[t] = 0.0;
      if (v12 && j3 >= 0 && j3 < n3) {
        if (DIM == 2) {
          for (int t = 0; t < NLM; ++t)
            acc[t] = t2[(((long long)t * nq3) * cols2 + c2) * cols1 + c];
        } else {
          int elo = max(max(i3, j3) - T.p, 0), ehi = min(min(i3, j3), nel - 1);
          for (int e = elo; e <= ehi; ++e)
            for (int g = 0; g < ng; ++g) {
              int q3 = e * ng + g;
              const double *vv = tab_val(T, pool, q3), *dd = tab_der(T, pool, q3);
              double fv[4];
              fv[0] = vv[i3 - e] * vv[j3 - e];
              fv[1] = vv[i3 - e] * dd[j3 - e];
              fv[2] = dd[i3 - e] * vv[j3 - e];
              fv[3] = dd[i3 - e] * dd[j3 - e];
              for (int pat = 0; pat < 4; ++pat)
                for (int t = 0; t < NLM; ++t)
                  acc[t] += t2[((((long long)pat * NLM + t) * nq3 + q3) * cols2 + c2) * cols1 + c] *
                            fv[pat];
            }
        }
      }
      const int o = o1 + pt.W[0] * (o2 + pt.W[1] * o3);
      const long long node = i1 + (long long)pt.n1p * (i2 + (long long)n2 * i3);
      for (int t = 0; t < NLM; ++t) {
        int l, m;
        lm_of(DIM, t, l, m);
        A[pt.soff + (((long long)(l * DIM + m) * pt.S + o) * pt.NP) + node] = acc[t];
      }
    }
}

// Lower blocks by symmetry: A_lm[i][o] = A_ml[i+o][-o].
template <int DIM>
__global__ void k_asm_fill(const DevPatch *P, double *A) {
  const DevPatch pt = P[blockIdx.y];
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long tot = (long long)pt.S * pt.NP;
  if (idx >= tot) return;
  const int node = (int)(idx % pt.NP), o = (int)(idx / pt.NP);
  const int i1 = node % pt.n1p, i2 = (node / pt.n1p) % pt.n[1], i3 = node / (pt.n1p * pt.n[1]);
  if (i1 >= pt.n[0]) return;   // row padding stays zero
  const int o1 = o % pt.W[0], o2 = (o / pt.W[0]) % pt.W[1], o3 = o / (pt.W[0] * pt.W[1]);
  const int p = pt.p;
  const int j1 = i1 + o1 - p, j2 = i2 + o2 - p, j3 = (DIM == 3) ? i3 + o3 - p : i3;
  const bool valid = j1 >= 0 && j1 < pt.n[0] && j2 >= 0 && j2 < pt.n[1] && j3 >= 0 && j3 < pt.n[2];
  const int orf = (pt.W[0] - 1 - o1) + pt.W[0] * ((pt.W[1] - 1 - o2) + pt.W[1] * (pt.W[2] - 1 - o3));
  const long long jn = j1 + (long long)pt.n1p * (j2 + (long long)pt.n[1] * j3);
  for (int l = 1; l < DIM; ++l)
    for (int m = 0; m < l; ++m) {
      double v = valid ? A[pt.soff + ((long long)(m * DIM + l) * pt.S + orf) * pt.NP + jn] : 0.0;
      A[pt.soff + ((long long)(l * DIM + m) * pt.S + o) * pt.NP + node] = v;
    }
}

afi_status assemble_stiffness(afi_ctx *c) {
  const int D = c->dim, NLM = (D == 3) ? 6 : 3, NPAT = (D == 3) ? 4 : 1;
  // scratch per patch
  std::vector<long long> s1(c->npatch), s2(c->npatch);
  long long maxs = 0;
  for (int k = 0; k < c->npatch; ++k) {
    const DevPatch &p = c->hp[k];
    long long cols1 = (long long)p.W[0] * p.n[0], cols2 = (long long)p.W[1] * p.n[1];
    s1[k] = (long long)NLM * p.nq[2] * p.nq[1] * cols1;
    s2[k] = (long long)NPAT * NLM * p.nq[2] * cols2 * cols1;
    maxs = std::max(maxs, s1[k] + s2[k]);
  }
  size_t freeb = 0, totb = 0;
  AFI_CUDA(cudaMemGetInfo(&freeb, &totb));
  long long budget = std::min<long long>((long long)(freeb * 0.5) / 8, 2000000000LL);
  budget = std::max(budget, maxs);
  double *scratch = nullptr;
  long long scratch_n = 0;
  for (int k = 0; k < c->npatch; ++k) scratch_n += s1[k] + s2[k];
  scratch_n = std::min(scratch_n, budget);
  AFI_CUDA(cudaMalloc(&scratch, scratch_n * sizeof(double)));
  int *dbatch = nullptr;
  long long *doff = nullptr;
  AFI_CUDA(cudaMalloc(&dbatch, c->npatch * sizeof(int)));
  AFI_CUDA(cudaMalloc(&doff, 2 * c->npatch * sizeof(long long)));
  afi_status st = AFI_OK;
  int k0 = 0;
  while (k0 < c->npatch && st == AFI_OK) {
    std::vector<int> batch;
    std::vector<long long> o1, o2;
    long long used = 0;
    int maxline = 1, maxq3 = 1, maxnq1 = 1;
    long long maxcols = 1;
    for (int k = k0; k < c->npatch; ++k) {
      if (!batch.empty() && used + s1[k] + s2[k] > scratch_n) break;
      batch.push_back(k);
      o1.push_back(used);
      o2.push_back(used + s1[k]);
      used += s1[k] + s2[k];
      const DevPatch &p = c->hp[k];
      maxline = std::max(maxline, p.nq[1] * p.nq[2]);
      maxq3 = std::max(maxq3, p.nq[2]);
      maxnq1 = std::max(maxnq1, p.nq[0]);
      maxcols = std::max(maxcols, (long long)p.W[0] * p.n[0] * p.W[1] * p.n[1]);
    }
    const int nb = (int)batch.size();
    std::vector<long long> offs(o1);
    offs.insert(offs.end(), o2.begin(), o2.end());
    cudaMemcpy(dbatch, batch.data(), nb * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(doff, offs.data(), 2 * nb * sizeof(long long), cudaMemcpyHostToDevice);
    cudaMemset(scratch, 0, used * sizeof(double));
    size_t smem1 = (size_t)NLM * maxnq1 * sizeof(double);
    for (int a = 0; a < D && st == AFI_OK; ++a)
      for (int b = 0; b < D; ++b) {
        if (D == 3) {
          launch(k_asm1<3>, dim3(maxline, nb), 128, smem1, 0, c->patches, dbatch, c->tabs, c->dpool,
                                                       c->qgeo, c->nqp, scratch, doff, a, b);
          launch(k_asm2<3>, dim3(maxq3, nb), 128, 0, 0, c->patches, dbatch, c->tabs, c->dpool, scratch,
                                              doff, scratch, doff + nb, a, b);
        } else {
          launch(k_asm1<2>, dim3(maxline, nb), 128, smem1, 0, c->patches, dbatch, c->tabs, c->dpool,
                                                       c->qgeo, c->nqp, scratch, doff, a, b);
          launch(k_asm2<2>, dim3(maxq3, nb), 128, 0, 0, c->patches, dbatch, c->tabs, c->dpool, scratch,
                                              doff, scratch, doff + nb, a, b);
        }
        if (cudaGetLastError() != cudaSuccess) { st = AFI_ECUDA; break; }
      }
    if (st != AFI_OK) break;
    unsigned g3 = (unsigned)((maxcols + 127) / 128);
    if (D == 3)
      launch(k_asm3<3>, dim3(g3, nb), 128, 0, 0, c->patches, dbatch, c->tabs, c->dpool, scratch, doff + nb,
                                       c->stencil);
    else
      launch(k_asm3<2>, dim3(g3, nb), 128, 0, 0, c->patches, dbatch, c->tabs, c->dpool, scratch, doff + nb,
                                       c->stencil);
    if (cudaGetLastError() != cudaSuccess) st = AFI_ECUDA;
    k0 += nb;
  }
  if (st == AFI_OK) {
    long long maxSN = 1;
    for (auto &p : c->hp) maxSN = std::max(maxSN, (long long)p.S * p.NP);
    dim3 g((unsigned)((maxSN + 255) / 256), c->npatch);
    if (D == 3) launch(k_asm_fill<3>, g, 256, 0, 0, c->patches, c->stencil);
    else launch(k_asm_fill<2>, g, 256, 0, 0, c->patches, c->stencil);
    if (cudaGetLastError() != cudaSuccess) st = AFI_ECUDA;
  }
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(scratch);
  cudaFree(dbatch);
  cudaFree(doff);
  if (e != cudaSuccess) { set_error(std::string("stiffness assembly: ") + cudaGetErrorString(e)); return AFI_ECUDA; }
  if (st != AFI_OK) set_error("stiffness assembly launch failed");
  return st;
}

afi_status compute_geometry(afi_ctx *c) {
  int maxNQ = 1;
  for (auto &p : c->hp) maxNQ = std::max(maxNQ, p.NQ);
  dim3 g((maxNQ + 127) / 128, c->npatch);
  AFI_CUDA(cudaMemset(c->dflag, 0, sizeof(int)));
  if (c->dim == 3) launch(k_geometry<3>, g, 128, 0, 0, c->patches, c->tabs, c->dpool, c->ctrl, c->qgeo, c->nqp, c->dflag);
  else launch(k_geometry<2>, g, 128, 0, 0, c->patches, c->tabs, c->dpool, c->ctrl, c->qgeo, c->nqp, c->dflag);
  AFI_LAUNCH_CHECK();
  int h = 0;
  AFI_CUDA(cudaMemcpy(&h, c->dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) { set_error("geometry map has det J <= 0 at a quadrature point"); return AFI_EINVAL; }
  return AFI_OK;
}

// --------------------------------------------------------- qp evaluation
// Field values (grad = 0) or parametric gradients at every quadrature point:
// out[comp][q] (grad = 0) or out[comp*DIM + a][q] for the torn vector u.
template <int DIM>
__global__ void k_eval_qp(const DevPatch *P, const Tab1D *tabs, const double *pool,
                          const double *u, double *out, long long nqp, int grad) {
  const DevPatch pt = P[blockIdx.y];
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= pt.NQ) return;
  int qd[3] = {q % pt.nq[0], (q / pt.nq[0]) % pt.nq[1], q / (pt.nq[0] * pt.nq[1])};
  const Tab1D T0 = tabs[pt.tab[0]], T1 = tabs[pt.tab[1]], T2 = tabs[pt.tab[2]];
  const int ng0 = T0.p + 1, ng1 = T1.p + 1, ng2 = T2.p + 1;
  const int e0 = qd[0] / ng0, e1 = qd[1] / ng1, e2 = qd[2] / ng2;
  const double *v0 = tab_val(T0, pool, qd[0]), *d0 = tab_der(T0, pool, qd[0]);
  const double *v1 = tab_val(T1, pool, qd[1]), *d1 = tab_der(T1, pool, qd[1]);
  const double *v2 = tab_val(T2, pool, qd[2]), *d2 = tab_der(T2, pool, qd[2]);
  double acc[DIM][DIM + 1];
  for (int l = 0; l < DIM; ++l)
    for (int a = 0; a <= DIM; ++a) acc[l][a] = 0.0;
  for (int t2 = 0; t2 < ng2; ++t2)
    for (int t1 = 0; t1 < ng1; ++t1)
      for (int t0 = 0; t0 < ng0; ++t0) {
        int node = (e0 + t0) + pt.n[0] * ((e1 + t1) + pt.n[1] * (e2 + t2));
        double g[4] = {v0[t0] * v1[t1] * v2[t2], d0[t0] * v1[t1] * v2[t2],
                       v0[t0] * d1[t1] * v2[t2], v0[t0] * v1[t1] * d2[t2]};
        for (int l = 0; l < DIM; ++l) {
          double uv = u[pt.off + (long long)l * pt.N + node];
          for (int a = 0; a <= DIM; ++a) acc[l][a] += uv * g[a];
        }
      }
  const long long gq = pt.qoff + q;
  for (int l = 0; l < DIM; ++l) {
    if (grad)
      for (int a = 0; a < DIM; ++a) out[(long long)(l * DIM + a) * nqp + gq] = acc[l][a + 1];
    else
      out[(long long)l * nqp + gq] = acc[l][0];
  }
}

// f_i = sum_q w|det J| B_i(q) c(q): node-wise gather over the support.
template <int DIM>
__global__ void k_mass_gather(const DevPatch *P, const Tab1D *tabs, const double *pool,
                              const double *qgeo, const double *cq, double *f, long long nqp) {
  const DevPatch pt = P[blockIdx.y];
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= pt.N) return;
  int id[3] = {node % pt.n[0], (node / pt.n[0]) % pt.n[1], node / (pt.n[0] * pt.n[1])};
  int lo[3], hi[3], ng[3];
  Tab1D T[3] = {tabs[pt.tab[0]], tabs[pt.tab[1]], tabs[pt.tab[2]]};
  for (int d = 0; d < 3; ++d) {
    ng[d] = T[d].p + 1;
    lo[d] = max(id[d] - T[d].p, 0);
    hi[d] = min(id[d], max(T[d].nel - 1, 0));
  }
  double acc[DIM];
  for (int l = 0; l < DIM; ++l) acc[l] = 0.0;
  for (int e2 = lo[2]; e2 <= hi[2]; ++e2)
    for (int g2 = 0; g2 < ng[2]; ++g2) {
      int q2 = e2 * ng[2] + g2;
      double b2 = tab_val(T[2], pool, q2)[id[2] - e2];
      for (int e1 = lo[1]; e1 <= hi[1]; ++e1)
        for (int g1 = 0; g1 < ng[1]; ++g1) {
          int q1 = e1 * ng[1] + g1;
          double b1 = b2 * tab_val(T[1], pool, q1)[id[1] - e1];
          for (int e0 = lo[0]; e0 <= hi[0]; ++e0)
            for (int g0 = 0; g0 < ng[0]; ++g0) {
              int q0 = e0 * ng[0] + g0;
              double bb = b1 * tab_val(T[0], pool, q0)[id[0] - e0];
              long long gq = pt.qoff + q0 + (long long)pt.nq[0] * (q1 + (long long)pt.nq[1] * q2);
              double wd = qgeo[(long long)(DIM * DIM) * nqp + gq];
              for (int l = 0; l < DIM; ++l) acc[l] += wd * bb * cq[(long long)l * nqp + gq];
            }
        }
    }
  for (int l = 0; l < DIM; ++l) f[pt.off + (long long)l * pt.N + node] = acc[l];
}

// Per-quadrature-point Lame gradient densities, reduced per block:
//   div z div u  and  2 eps(z):eps(u)  times w|det J|.
template <int DIM>
__global__ void k_lame_density(const DevPatch *P, const double *qgeo, const double *gu,
                               const double *gz, long long nqp, double *partial, int nblk) {
  const DevPatch pt = P[blockIdx.y];
  double sl = 0.0, sm = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < pt.NQ; q += gridDim.x * blockDim.x) {
    const long long gq = pt.qoff + q;
    double Q[DIM][DIM];
    for (int a = 0; a < DIM; ++a)
      for (int x = 0; x < DIM; ++x) Q[a][x] = qgeo[(long long)(a * DIM + x) * nqp + gq];
    double wd = qgeo[(long long)(DIM * DIM) * nqp + gq];
    double Gu[DIM][DIM], Gz[DIM][DIM];  // [component][x]
    for (int l = 0; l < DIM; ++l)
      for (int x = 0; x < DIM; ++x) {
        double su = 0.0, sz = 0.0;
        for (int a = 0; a < DIM; ++a) {
          su += Q[a][x] * gu[(long long)(l * DIM + a) * nqp + gq];
          sz += Q[a][x] * gz[(long long)(l * DIM + a) * nqp + gq];
        }
        Gu[l][x] = su;
        Gz[l][x] = sz;
      }
    double du = 0.0, dz = 0.0, ee = 0.0;
    for (int l = 0; l < DIM; ++l) { du += Gu[l][l]; dz += Gz[l][l]; }
    for (int l = 0; l < DIM; ++l)
      for (int x = 0; x < DIM; ++x) {
        double eu = 0.5 * (Gu[l][x] + Gu[x][l]), ez = 0.5 * (Gz[l][x] + Gz[x][l]);
        ee += eu * ez;
      }
    sl += wd * du * dz;
    sm += wd * 2.0 * ee;
  }
  __shared__ double rl[256], rm[256];
  rl[threadIdx.x] = sl;
  rm[threadIdx.x] = sm;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) { rl[threadIdx.x] += rl[threadIdx.x + s]; rm[threadIdx.x] += rm[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[((long long)blockIdx.y * nblk + blockIdx.x) * 2 + 0] = rl[0];
    partial[((long long)blockIdx.y * nblk + blockIdx.x) * 2 + 1] = rm[0];
  }
}

__global__ void k_lame_final(const double *partial, int nblk, int npatch, double *grad) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npatch) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += partial[((long long)k * nblk + i) * 2];
    b += partial[((long long)k * nblk + i) * 2 + 1];
  }
  grad[2 * k] = -a;
  grad[2 * k + 1] = -b;
}

afi_status op_load(afi_ctx *c, const double *coef, double *f, cudaStream_t s) {
  if (c->mf) return mf_mass(c, coef, f, s);
  const int D = c->dim;
  int maxNQ = 1, maxN = 1;
  for (auto &p : c->hp) { maxNQ = std::max(maxNQ, p.NQ); maxN = std::max(maxN, p.N); }
  double *cq = nullptr;
  AFI_CUDA(cudaMallocAsync((void **)&cq, (size_t)D * c->nqp * sizeof(double), s));
  dim3 g((maxNQ + 127) / 128, c->npatch), g2((maxN + 127) / 128, c->npatch);
  if (D == 3) {
    launch(k_eval_qp<3>, g, 128, 0, s, c->patches, c->tabs, c->dpool, coef, cq, c->nqp, 0);
    launch(k_mass_gather<3>, g2, 128, 0, s, c->patches, c->tabs, c->dpool, c->qgeo, cq, f, c->nqp);
  } else {
    launch(k_eval_qp<2>, g, 128, 0, s, c->patches, c->tabs, c->dpool, coef, cq, c->nqp, 0);
    launch(k_mass_gather<2>, g2, 128, 0, s, c->patches, c->tabs, c->dpool, c->qgeo, cq, f, c->nqp);
  }
  AFI_LAUNCH_CHECK();
  AFI_CUDA(cudaFreeAsync(cq, s));
  return AFI_OK;
}

afi_status op_lame_grad(afi_ctx *c, const double *u, const double *z, double *grad,
                        cudaStream_t s) {
  const int D = c->dim;
  int maxNQ = 1;
  for (auto &p : c->hp) maxNQ = std::max(maxNQ, p.NQ);
  const int nblk = 8;
  double *gu = nullptr;
  AFI_CUDA(cudaMallocAsync((void **)&gu, (2ull * D * D * c->nqp + 2ull * c->npatch * nblk) * sizeof(double), s));
  double *gz = gu + (long long)D * D * c->nqp, *part = gz + (long long)D * D * c->nqp;
  dim3 g((maxNQ + 127) / 128, c->npatch);
  if (D == 3) {
    launch(k_eval_qp<3>, g, 128, 0, s, c->patches, c->tabs, c->dpool, u, gu, c->nqp, 1);
    launch(k_eval_qp<3>, g, 128, 0, s, c->patches, c->tabs, c->dpool, z, gz, c->nqp, 1);
    launch(k_lame_density<3>, dim3(nblk, c->npatch), 256, 0, s, c->patches, c->qgeo, gu, gz, c->nqp, part, nblk);
  } else {
    launch(k_eval_qp<2>, g, 128, 0, s, c->patches, c->tabs, c->dpool, u, gu, c->nqp, 1);
    launch(k_eval_qp<2>, g, 128, 0, s, c->patches, c->tabs, c->dpool, z, gz, c->nqp, 1);
    launch(k_lame_density<2>, dim3(nblk, c->npatch), 256, 0, s, c->patches, c->qgeo, gu, gz, c->nqp, part, nblk);
  }
  launch(k_lame_final, (c->npatch + 127) / 128, 128, 0, s, part, nblk, c->npatch, grad);
  AFI_LAUNCH_CHECK();
  AFI_CUDA(cudaFreeAsync(gu, s));
  return AFI_OK;
}

}  // namespace afi
