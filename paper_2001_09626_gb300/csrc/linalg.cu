// Small dense FP64 linear algebra on the device, used by the setup:
//  * 1D spline data: knots, Gauss-Legendre rules, B-spline values and
//    derivatives at the quadrature points (Cox-de Boor, Section 2.1) and the
//    univariate stiffness / mass matrices K_hat, M_hat (Section 5.2);
//  * the generalised eigendecomposition U^T K U = D, U^T M U = I of eq. (5.8)
//    by Cholesky reduction plus parallel cyclic Jacobi;
//  * explicit inverses of G^T G (eq. 4.6, Gauss-Jordan over the whole grid)
//    and of the per-patch R^T R (projection P_u).
#include "common.cuh"

#include <cmath>

namespace afi {

// ------------------------------------------------------------------ 1D data
// One block per table: knots, Gauss-Legendre nodes (Newton on the Legendre
// three-term recurrence), quadrature weights scaled to each element.
__global__ void k_knots_quad(Tab1D *tabs, int ntab, double *pool) {
  int t = blockIdx.x;
  if (t >= ntab) return;
  Tab1D T = tabs[t];
  if (T.n == 1) {  // dummy direction of 2D problems
    if (threadIdx.x == 0) {
      pool[T.qw] = 1.0;
      pool[T.val] = 1.0;
      pool[T.der] = 0.0;
      pool[T.K] = 0.0;
      pool[T.M] = 1.0;
    }
    return;
  }
  const int p = T.p, nel = T.nel, nk = nel + 2 * p + 1, ng = p + 1;
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    double v;
    if (j <= p) v = 0.0;
    else if (j >= nel + p) v = 1.0;
    else v = (double)(j - p) / (double)nel;
    pool[T.knots + j] = v;
  }
  __shared__ double gw[16];
  if (threadIdx.x < ng) {
    int i = threadIdx.x;
    // root i of P_ng on (-1, 1), descending order, Newton from the
    // Chebyshev-like initial guess
    double x = cos(M_PI * (i + 0.75) / (ng + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= ng; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (ng == 1) { p1 = x; p0 = 1.0; }
      dp = ng * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= ng; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = ng * (x * p1 - p0) / (x * x - 1.0);
    }
    double w = 2.0 / ((1.0 - x * x) * dp * dp);
    // roots come in descending x; store ascending on [0, 1]
    gw[ng - 1 - i] = 0.5 * w;
  }
  __syncthreads();
  // uniform elements of length 1/nel
  for (int q = threadIdx.x; q < T.nq; q += blockDim.x) pool[T.qw + q] = gw[q % ng] / nel;
}

// quadrature point coordinate (same ordering as k_knots_quad)
__device__ __forceinline__ double gl_node(int ng, int g) {
  // recompute node g of the ng-point rule on [0, 1]
  int i = ng - 1 - g;
  double x = cos(M_PI * (i + 0.75) / (ng + 0.5));
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= ng; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (ng == 1) { p1 = x; p0 = 1.0; }
    double dp = ng * (x * p1 - p0) / (x * x - 1.0);
    double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  return 0.5 * (x + 1.0);
}

// Values and first derivatives of the p+1 B-splines active on the element of
// every quadrature point (Cox-de Boor recursion with the 0/0 = 0 rule).
__global__ void k_basis(Tab1D *tabs, int ntab, double *pool) {
  int t = blockIdx.y;
  if (t >= ntab) return;
  Tab1D T = tabs[t];
  if (T.n == 1) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= T.nq) return;
  const int p = T.p, ng = p + 1;
  const int e = q / ng, g = q % ng;
  const double *kn = pool + T.knots;
  const int span = p + e;
  const double a = kn[span], b = kn[span + 1];
  const double x = a + (b - a) * gl_node(ng, g);
  double N[16], left[16], right[16], Np1[16];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - kn[span + 1 - j];
    right[j] = kn[span + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double den = right[r + 1] + left[j - r];
      double tmp = (den == 0.0) ? 0.0 : N[r] / den;
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
    if (j == p - 1)
      for (int r = 0; r <= j; ++r) Np1[r] = N[r];
  }
  if (p == 1) Np1[0] = 1.0;
  for (int r = 0; r <= p; ++r) {
    pool[T.val + (long long)q * (p + 1) + r] = N[r];
    int i = span - p + r;  // global basis index
    double d = 0.0;
    if (r >= 1) {
      double den = kn[i + p] - kn[i];
      if (den != 0.0) d += p * Np1[r - 1] / den;
    }
    if (r <= p - 1) {
      double den = kn[i + p + 1] - kn[i + 1];
      if (den != 0.0) d -= p * Np1[r] / den;
    }
    pool[T.der + (long long)q * (p + 1) + r] = d;
  }
}

// K_hat_ij = sum_q w b_i' b_j',  M_hat_ij = sum_q w b_i b_j (dense n x n).
// Geometry-inclusion tables (wK, wM >= 0) weight the points by the fitted
// factors: K~_ij = sum_q w nu_q b_i' b_j',  M~_ij = sum_q w beta_q b_i b_j.
__global__ void k_kmass(Tab1D *tabs, int ntab, double *pool) {
  int t = blockIdx.y;
  if (t >= ntab) return;
  Tab1D T = tabs[t];
  if (T.n == 1) return;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T.n * T.n) return;
  const int i = idx / T.n, j = idx % T.n, p = T.p, ng = p + 1;
  double k = 0.0, m = 0.0;
  if (abs(i - j) <= p) {
    int elo = max(max(i, j) - p, 0), ehi = min(min(i, j), T.nel - 1);
    for (int e = elo; e <= ehi; ++e)
      for (int g = 0; g < ng; ++g) {
        int q = e * ng + g;
        const double w = pool[T.qw + q];
        const double wk = T.wK >= 0 ? w * pool[T.wK + q] : w;
        const double wm = T.wM >= 0 ? w * pool[T.wM + q] : w;
        const double *v = pool + T.val + (long long)q * ng;
        const double *d = pool + T.der + (long long)q * ng;
        k += wk * d[i - e] * d[j - e];
        m += wm * v[i - e] * v[j - e];
      }
  }
  pool[T.K + idx] = k;
  pool[T.M + idx] = m;
}

// --------------------------------------------------- generalised eigensolve
// One block per pencil.  K, M: n x n row-major (n <= 96).  Writes U (row i =
// basis index, column a = mode, U^T M U = I) and D.  interior = 1 takes the
// pencil with the first and last index removed.  flag[0] is set on failure.
__global__ void k_geneig(Tab1D *tabs, int ntab, double *pool, int interior, int *flag) {
  int t = blockIdx.x;
  if (t >= ntab) return;
  Tab1D T = tabs[t];
  const int n = interior ? T.ni : T.n;
  double *Uo = pool + (interior ? T.Ui : T.U);
  double *Do = pool + (interior ? T.Di : T.D);
  if (T.n == 1) {  // dummy: U = 1, D = 0
    if (threadIdx.x == 0) { Uo[0] = 1.0; Do[0] = 0.0; }
    return;
  }
  extern __shared__ double sm[];
  double *L = sm;            // n*n
  double *C = sm + n * n;    // n*n
  double *V = sm + 2 * n * n;
  __shared__ double cs_c[64], cs_s[64];
  __shared__ int bad;
  __shared__ double red[32];
  const int off = interior ? 1 : 0, ld = T.n;
  const double *K = pool + T.K, *M = pool + T.M;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int i = idx / n, j = idx % n;
    L[idx] = M[(i + off) * ld + j + off];
    C[idx] = K[(i + off) * ld + j + off];
    V[idx] = (i == j) ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // Cholesky of M in place (lower triangle)
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = L[j * n + j];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      L[j * n + j] = sqrt(d);
    }
    __syncthreads();
    double d = L[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) L[i * n + j] /= d;
    __syncthreads();
    int m = n - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = j + 1 + idx / m, k = j + 1 + idx % m;
      if (k <= i) L[i * n + k] -= L[i * n + j] * L[k * n + j];
    }
    __syncthreads();
  }
  // C := L^{-1} K  (forward substitution, one column per thread)
  for (int col = threadIdx.x; col < n; col += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double s = C[i * n + col];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * C[k * n + col];
      C[i * n + col] = s / L[i * n + i];
    }
  }
  __syncthreads();
  // C := C L^{-T}  (one row per thread)
  for (int row = threadIdx.x; row < n; row += blockDim.x) {
    for (int j = 0; j < n; ++j) {
      double s = C[row * n + j];
      for (int k = 0; k < j; ++k) s -= C[row * n + k] * L[j * n + k];
      C[row * n + j] = s / L[j * n + j];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int i = idx / n, j = idx % n;
    if (i < j) {
      double a = 0.5 * (C[i * n + j] + C[j * n + i]);
      C[i * n + j] = a;
      C[j * n + i] = a;
    }
  }
  __syncthreads();
  // parallel cyclic Jacobi, round-robin pairing of n' = n rounded up to even
  const int np = (n + 1) & ~1, npair = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // off-diagonal norm
    double off2 = 0.0, tot = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      double v = C[idx] * C[idx];
      tot += v;
      if (idx / n != idx % n) off2 += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off2 += __shfl_down_sync(0xffffffffu, off2, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      red[0] = s;
    }
    __syncthreads();
    double offn = red[0];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      red[0] = s;
    }
    __syncthreads();
    double totn = red[0];
    __syncthreads();
    if (offn <= 1e-30 * totn) break;
    for (int r = 0; r < np - 1; ++r) {
      // rotation parameters, one pair per thread
      for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        int a, b;
        if (k == 0) { a = 0; b = 1 + (r % (np - 1)); }
        else { a = 1 + (r + k) % (np - 1); b = 1 + (r - k + np - 1) % (np - 1); }
        if (a > b) { int tmp = a; a = b; b = tmp; }
        double c = 1.0, s = 0.0;
        if (b < n) {
          double apq = C[a * n + b];
          if (apq != 0.0) {
            double tau = (C[b * n + b] - C[a * n + a]) / (2.0 * apq);
            double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        cs_c[k] = c;
        cs_s[k] = s;
      }
      __syncthreads();
      // columns: C := C J, V := V J
      for (int idx = threadIdx.x; idx < npair * n; idx += blockDim.x) {
        int k = idx / n, row = idx % n;
        int a, b;
        if (k == 0) { a = 0; b = 1 + (r % (np - 1)); }
        else { a = 1 + (r + k) % (np - 1); b = 1 + (r - k + np - 1) % (np - 1); }
        if (a > b) { int tmp = a; a = b; b = tmp; }
        if (b >= n) continue;
        double c = cs_c[k], s = cs_s[k];
        double xa = C[row * n + a], xb = C[row * n + b];
        C[row * n + a] = c * xa - s * xb;
        C[row * n + b] = s * xa + c * xb;
        double va = V[row * n + a], vb = V[row * n + b];
        V[row * n + a] = c * va - s * vb;
        V[row * n + b] = s * va + c * vb;
      }
      __syncthreads();
      // rows: C := J^T C
      for (int idx = threadIdx.x; idx < npair * n; idx += blockDim.x) {
        int k = idx / n, col = idx % n;
        int a, b;
        if (k == 0) { a = 0; b = 1 + (r % (np - 1)); }
        else { a = 1 + (r + k) % (np - 1); b = 1 + (r - k + np - 1) % (np - 1); }
        if (a > b) { int tmp = a; a = b; b = tmp; }
        if (b >= n) continue;
        double c = cs_c[k], s = cs_s[k];
        double xa = C[a * n + col], xb = C[b * n + col];
        C[a * n + col] = c * xa - s * xb;
        C[b * n + col] = s * xa + c * xb;
      }
      __syncthreads();
    }
  }
  // U = L^{-T} V (back substitution per column), D = diag(C)
  for (int col = threadIdx.x; col < n; col += blockDim.x) {
    for (int i = n - 1; i >= 0; --i) {
      double s = V[i * n + col];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * Uo[k * n + col];
      Uo[i * n + col] = s / L[i * n + i];
    }
    Do[col] = C[col * n + col];
  }
  if (threadIdx.x == 0 && bad) atomicExch(flag, 1);
}

// Zero-padded copies U[i][a] -> Up[i*ld + a] and Upt[a*ld + i] (and the
// interior pencil), so that mode products can load 4 coefficients at once.
__global__ void k_pad_u(Tab1D *tabs, int ntab, double *pool) {
  const int t = blockIdx.y;
  if (t >= ntab) return;
  const Tab1D T = tabs[t];
  for (int part = 0; part < 2; ++part) {
    const int n = part ? T.ni : T.n, ld = part ? T.ldi : T.ld;
    const double *U = pool + (part ? T.Ui : T.U);
    double *Up = pool + (part ? T.Uip : T.Up), *Upt = pool + (part ? T.Uipt : T.Upt);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * ld; idx += gridDim.x * blockDim.x) {
      const int i = idx / ld, a = idx % ld;
      Up[idx] = (a < n) ? U[i * n + a] : 0.0;
      Upt[idx] = (a < n) ? U[a * n + i] : 0.0;
    }
  }
}

// Diagonal-major band copies of K_hat and M_hat (half-bandwidth p), so that
// neighbouring output indices read neighbouring addresses.
__global__ void k_band(Tab1D *tabs, int ntab, double *pool) {
  const int t = blockIdx.y;
  if (t >= ntab) return;
  const Tab1D T = tabs[t];
  const int W = 2 * T.p + 1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < W * T.n; idx += gridDim.x * blockDim.x) {
    const int tt = idx / T.n, i = idx % T.n, j = i + tt - T.p;
    const bool in = j >= 0 && j < T.n;
    pool[T.Kb + idx] = in ? pool[T.K + (long long)i * T.n + j] : 0.0;
    pool[T.Mb + idx] = in ? pool[T.M + (long long)i * T.n + j] : 0.0;
  }
}

__global__ void k_to_low(const double *src, float *f, __nv_bfloat16 *b, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  f[i] = (float)src[i];
  b[i] = __double2bfloat16(src[i]);
}

// ---------------------------------------------------- dense SPD inverse
// Gauss-Jordan elimination without pivoting (the pivots of an SPD matrix
// are the diagonals of its successive Schur complements, all positive), one
// grid-wide launch per pivot k, ping-pong src -> dst:
//   row k:    dst[k][j] = src[k][j] / src[k][k]   (and 1 / src[k][k] at j = k)
//   row i!=k: dst[i][j] = src[i][j] - src[i][k] dst[k][j]   (0 - ... at j = k)
// After the n steps the buffer holds A^{-1}.  pinv[k] = 1 / pivot k is
// written by the thread that computes that diagonal entry one step earlier,
// so each step divides once.
__global__ void k_gj_first(const double *A, double *pinv, int *flag) {
  const double d = A[0];
  if (!(d > 0.0) || !isfinite(d)) { atomicExch(flag, 1); pinv[0] = 0.0; }
  else pinv[0] = 1.0 / d;
}

__global__ void k_gj_step(const double *src, double *dst, int n, int k, double *pinv, int *flag) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const double p = pinv[k];
  const long long at = (long long)i * n + j;
  const double rk = (j == k) ? p : src[(long long)k * n + j] * p;
  const double v = (i == k) ? rk : ((j == k) ? 0.0 : src[at]) - src[(long long)i * n + k] * rk;
  dst[at] = v;
  if (i == k + 1 && j == k + 1) {
    if (!(v > 0.0) || !isfinite(v)) { atomicExch(flag, 1); pinv[k + 1] = 0.0; }
    else pinv[k + 1] = 1.0 / v;
  }
}

// Per patch nm x nm SPD inverse by Gauss-Jordan (one thread per patch).
__global__ void k_small_inv(double *A, int nm, int count, int *flag) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  double a[6][12];
  double *M = A + (long long)k * nm * nm;
  for (int i = 0; i < nm; ++i)
    for (int j = 0; j < nm; ++j) {
      a[i][j] = M[i * nm + j];
      a[i][nm + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int c = 0; c < nm; ++c) {
    int piv = c;
    for (int r = c + 1; r < nm; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (!(fabs(a[piv][c]) > 0.0)) { atomicExch(flag, 1); return; }
    if (piv != c)
      for (int j = 0; j < 2 * nm; ++j) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
    double d = a[c][c];
    for (int j = 0; j < 2 * nm; ++j) a[c][j] /= d;
    for (int r = 0; r < nm; ++r)
      if (r != c) {
        double f = a[r][c];
        for (int j = 0; j < 2 * nm; ++j) a[r][j] -= f * a[c][j];
      }
  }
  for (int i = 0; i < nm; ++i)
    for (int j = 0; j < nm; ++j) M[i * nm + j] = a[i][nm + j];
}

// ------------------------------------------------------------ host entry
// Tables [t0, t1): knots, Gauss rules and basis tables (basis = true; the
// geometry-inclusion tables share those of their base table), univariate
// matrices, generalised eigenpairs (full and interior pencils), padded and
// banded copies, and the low-precision mirrors of the whole pool.
afi_status build_1d_tables_range(afi_ctx *c, int t0, int t1, bool basis) {
  const int nt = t1 - t0;
  if (nt <= 0) return AFI_OK;
  Tab1D *tb = c->tabs + t0;
  int maxq = 1, maxn = 1;
  for (int t = t0; t < t1; ++t) {
    maxq = std::max(maxq, c->htab[t].nq);
    maxn = std::max(maxn, c->htab[t].n);
  }
  if (basis) {
    launch(k_knots_quad, nt, 64, 0, 0, tb, nt, c->dpool);
    AFI_LAUNCH_CHECK();
    launch(k_basis, dim3((maxq + 127) / 128, nt), 128, 0, 0, tb, nt, c->dpool);
    AFI_LAUNCH_CHECK();
  }
  launch(k_kmass, dim3((maxn * maxn + 127) / 128, nt), 128, 0, 0, tb, nt, c->dpool);
  AFI_LAUNCH_CHECK();
  size_t smem = 3ull * maxn * maxn * sizeof(double);
  AFI_CUDA(cudaFuncSetAttribute(k_geneig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  launch(k_geneig, nt, 256, smem, 0, tb, nt, c->dpool, 0, c->dflag);
  AFI_LAUNCH_CHECK();
  launch(k_geneig, nt, 256, smem, 0, tb, nt, c->dpool, 1, c->dflag);
  AFI_LAUNCH_CHECK();
  int h = 0;
  AFI_CUDA(cudaMemcpy(&h, c->dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) { set_error("univariate mass pencil not positive definite"); return AFI_ESINGULAR; }
  launch(k_pad_u, dim3(16, nt), 256, 0, 0, tb, nt, c->dpool);
  launch(k_band, dim3(16, nt), 256, 0, 0, tb, nt, c->dpool);
  // low-precision copies of the eigenvectors: the pools mirror the FP64 pool
  launch(k_to_low, (unsigned)((c->dpool_n + 255) / 256), 256, 0, 0, c->dpool, c->fpool, c->bpool, c->dpool_n);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status build_1d_tables(afi_ctx *c) {
  return build_1d_tables_range(c, 0, c->nbase_tab, true);
}

// Ainv = A^{-1} for SPD A (n x n); scratch holds n*n + n doubles.  A is
// left unchanged.
afi_status dense_spd_inverse(afi_ctx *c, double *A, double *Ainv, int n, double *scratch) {
  double *buf[2] = {Ainv, scratch};
  double *pinv = scratch + (long long)n * n;
  AFI_CUDA(cudaMemcpy(Ainv, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice));
  launch(k_gj_first, 1, 1, 0, 0, (const double *)Ainv, pinv, c->dflag);
  const dim3 grid((n + 255) / 256, n);
  for (int k = 0; k < n; ++k)
    launch(k_gj_step, grid, 256, 0, 0, (const double *)buf[k & 1], buf[(k + 1) & 1], n, k, pinv, c->dflag);
  AFI_LAUNCH_CHECK();
  if (n & 1)
    AFI_CUDA(cudaMemcpy(Ainv, scratch, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice));
  int h = 0;
  AFI_CUDA(cudaMemcpy(&h, c->dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) { set_error("G^T G is not positive definite (too few constraints?)"); return AFI_ESINGULAR; }
  return AFI_OK;
}

afi_status small_inverses(afi_ctx *c, double *A, int nm, int count) {
  launch(k_small_inv, (count + 63) / 64, 64, 0, 0, A, nm, count, c->dflag);
  AFI_LAUNCH_CHECK();
  int h = 0;
  AFI_CUDA(cudaMemcpy(&h, c->dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) { set_error("R^T R is singular"); return AFI_ESINGULAR; }
  return AFI_OK;
}

}  // namespace afi
