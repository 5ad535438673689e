// Context setup: problem validation, univariate tables, patch descriptors,
// geometry and stiffness assembly, interface connectivity, the constraint
// matrix B (Section 4, non-redundant rows: one row per copy on the Dirichlet
// boundary, star rows u_{c1} - u_{cj} elsewhere, then the rows of nested
// non-conforming faces, nested.cu), rigid modes, R^T R and G^T G with their
// inverses.  Integer bookkeeping (which copies form a
// geometric node, the row lists) is done on the host; all floating-point
// work runs in kernels.
#include "common.cuh"

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>

namespace afi {

std::atomic<long long> g_launches{0};

static std::mutex g_err_mu;
static std::string g_err;

void set_error(const std::string &msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = msg;
}
const char *last_error_cstr() {
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err.c_str();
}

afi_status dalloc(afi_ctx *c, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? AFI_ENOMEM : AFI_ECUDA;
  }
  c->bytes += (long long)bytes;
  return AFI_OK;
}

template <typename T>
static afi_status upload(afi_ctx *c, T **dst, const std::vector<T> &src) {
  AFI_TRY(dalloc(c, (void **)dst, src.size() * sizeof(T)));
  if (!src.empty()) AFI_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return AFI_OK;
}

afi_status build_1d_tables(afi_ctx *c);
afi_status dense_spd_inverse(afi_ctx *c, double *A, double *Ainv, int n, double *scratch);
afi_status small_inverses(afi_ctx *c, double *A, int nm, int count);
afi_status compute_geometry(afi_ctx *c);
afi_status assemble_stiffness(afi_ctx *c);

// ----------------------------------------------------------------- kernels
// H^(k): diagonal of the control-point bounding box; Hs = H^{d-2}.
__global__ void k_patch_H(DevPatch *P, const double *ctrl, int dim) {
  const int k = blockIdx.x;
  DevPatch pt = P[k];
  __shared__ double lo[3][256], hi[3][256];
  double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
  for (int i = threadIdx.x; i < pt.N; i += blockDim.x)
    for (int d = 0; d < dim; ++d) {
      double v = ctrl[pt.xoff + (long long)i * dim + d];
      l[d] = fmin(l[d], v);
      h[d] = fmax(h[d], v);
    }
  for (int d = 0; d < 3; ++d) { lo[d][threadIdx.x] = l[d]; hi[d][threadIdx.x] = h[d]; }
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        lo[d][threadIdx.x] = fmin(lo[d][threadIdx.x], lo[d][threadIdx.x + s]);
        hi[d][threadIdx.x] = fmax(hi[d][threadIdx.x], hi[d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int d = 0; d < dim; ++d) s2 += (hi[d][0] - lo[d][0]) * (hi[d][0] - lo[d][0]);
    double H = sqrt(s2);
    P[k].H = H;
    P[k].Hs = (dim == 3) ? H : 1.0;
  }
}

__device__ __forceinline__ double rigid_s(int a, int comp, const double *X, int dim) {
  if (a < dim) return (a == comp) ? 1.0 : 0.0;
  if (dim == 2) return (comp == 0) ? X[1] : -X[0];
  switch (a) {
    case 3: return comp == 1 ? X[2] : (comp == 2 ? -X[1] : 0.0);
    case 4: return comp == 0 ? X[2] : (comp == 2 ? -X[0] : 0.0);
    default: return comp == 0 ? X[1] : (comp == 1 ? -X[0] : 0.0);
  }
}

// Sum over a list of (dofA of patch ka, dofB of patch kb, sign) of
// sign * R_ka(dofA)[a] R_kb(dofB)[b], written to block (ka, kb) of M (ld),
// and its transpose to (kb, ka) if transpose_too.  One block per list.
__global__ void k_rr_blocks(const DevPatch *P, const double *ctrl, const int *ptr,
                            const int2 *kk, const int4 *ent, double *M, int ld, int nm, int dim,
                            int transpose_too) {
  const int b = blockIdx.x;
  const int2 kp = kk[b];
  const DevPatch pa = P[kp.x], pb = P[kp.y];
  __shared__ double sh[256];
  double acc[36];
  for (int i = 0; i < nm * nm; ++i) acc[i] = 0.0;
  for (int e = ptr[b] + threadIdx.x; e < ptr[b + 1]; e += blockDim.x) {
    int4 en = ent[e];
    long long ra = en.x - pa.off, rb = en.y - pb.off;
    int ca = (int)(ra / pa.N), cb = (int)(rb / pb.N);
    const double *Xa = ctrl + pa.xoff + (ra - (long long)ca * pa.N) * dim;
    const double *Xb = ctrl + pb.xoff + (rb - (long long)cb * pb.N) * dim;
    double va[6], vb[6];
    for (int a = 0; a < nm; ++a) { va[a] = rigid_s(a, ca, Xa, dim); vb[a] = rigid_s(a, cb, Xb, dim); }
    for (int a = 0; a < nm; ++a)
      for (int bb = 0; bb < nm; ++bb) acc[a * nm + bb] += en.z * va[a] * vb[bb];
  }
  for (int i = 0; i < nm * nm; ++i) {
    sh[threadIdx.x] = acc[i];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      int a = i / nm, bb = i % nm;
      M[(long long)(kp.x * nm + a) * ld + kp.y * nm + bb] = sh[0];
      if (transpose_too) M[(long long)(kp.y * nm + bb) * ld + kp.x * nm + a] = sh[0];
    }
    __syncthreads();
  }
}

// R_k^T R_k over all dofs of each patch (one block per patch).
__global__ void k_RtR(const DevPatch *P, const double *ctrl, double *out, int dim, int nm) {
  const int k = blockIdx.x;
  const DevPatch pt = P[k];
  __shared__ double sh[256];
  double acc[36];
  for (int i = 0; i < nm * nm; ++i) acc[i] = 0.0;
  for (long long i = threadIdx.x; i < (long long)dim * pt.N; i += blockDim.x) {
    int comp = (int)(i / pt.N);
    const double *X = ctrl + pt.xoff + (i - (long long)comp * pt.N) * dim;
    double v[6];
    for (int a = 0; a < nm; ++a) v[a] = rigid_s(a, comp, X, dim);
    for (int a = 0; a < nm; ++a)
      for (int b = 0; b < nm; ++b) acc[a * nm + b] += v[a] * v[b];
  }
  for (int i = 0; i < nm * nm; ++i) {
    sh[threadIdx.x] = acc[i];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(long long)k * nm * nm + i] = sh[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------------- host
static int idx3(int i1, int i2, int i3, const int *n) { return i1 + n[0] * (i2 + n[1] * i3); }

afi_status setup_context(const afi_problem *prob, const afi_options *opt, afi_ctx *c) {
  auto t0 = std::chrono::steady_clock::now();
  if (!prob || !opt) { set_error("null problem or options"); return AFI_EINVAL; }
  const int D = prob->dim, NP = prob->npatch;
  if ((D != 2 && D != 3) || NP < 1 || !prob->degree || !prob->nel || !prob->ctrl || !prob->lame ||
      !prob->dirichlet_face) {
    set_error("invalid problem description");
    return AFI_EINVAL;
  }
  if (opt->prec < AFI_FD_FP64 || opt->prec > AFI_FD_BF16 || !(opt->tol > 0.0) || opt->maxit < 1) {
    set_error("invalid options");
    return AFI_EINVAL;
  }
  if ((opt->variant & AFI_VARIANT_GEO) &&
      (opt->variant & (AFI_VARIANT_LOCAL_ONLY | AFI_VARIANT_EXACT))) {
    set_error("AFI_VARIANT_GEO needs the geometry and excludes AFI_VARIANT_LOCAL_ONLY and "
              "AFI_VARIANT_EXACT");
    return AFI_EINVAL;
  }
  if ((opt->variant & AFI_VARIANT_MATRIX_FREE) &&
      (opt->variant & (AFI_VARIANT_LOCAL_ONLY | AFI_VARIANT_EXACT | AFI_VARIANT_GEO))) {
    set_error("AFI_VARIANT_MATRIX_FREE excludes AFI_VARIANT_LOCAL_ONLY, AFI_VARIANT_EXACT and "
              "AFI_VARIANT_GEO");
    return AFI_EINVAL;
  }
  c->dim = D;
  c->npatch = NP;
  c->geo = (opt->variant & AFI_VARIANT_GEO) != 0;
  c->nm = (D == 3) ? 6 : 3;
  c->opt = *opt;
  cudaGetDevice(&c->device);

  // ---- univariate tables, one per distinct (nel, p)
  std::map<std::pair<int, int>, int> tabidx;
  long long dn = 0;
  auto take = [&](long long n) { long long o = dn; dn += (n + 3) & ~3LL; return o; };
  auto make_tab = [&](int nel, int p) {
    Tab1D T{};
    if (nel == 0) {
      T.nel = 0; T.p = 0; T.n = 1; T.nq = 1; T.ni = 1;
      T.knots = take(1); T.qw = take(1); T.val = take(1); T.der = take(1);
      T.K = take(1); T.M = take(1); T.U = take(1); T.D = take(1); T.Ui = take(1); T.Di = take(1);
    } else {
      T.nel = nel; T.p = p; T.n = nel + p; T.nq = nel * (p + 1); T.ni = T.n - 2;
      T.knots = take(nel + 2 * p + 1); T.qw = take(T.nq);
      T.val = take((long long)T.nq * (p + 1)); T.der = take((long long)T.nq * (p + 1));
      T.K = take((long long)T.n * T.n); T.M = take((long long)T.n * T.n);
      T.U = take((long long)T.n * T.n); T.D = take(T.n);
      T.Ui = take((long long)T.ni * T.ni); T.Di = take(T.ni);
    }
    T.ld = (T.n + 3) & ~3;
    T.ldi = (T.ni + 3) & ~3;
    T.Up = take((long long)T.n * T.ld); T.Upt = take((long long)T.n * T.ld);
    T.Uip = take((long long)T.ni * T.ldi); T.Uipt = take((long long)T.ni * T.ldi);
    T.Kb = take((long long)(2 * T.p + 1) * T.n); T.Mb = take((long long)(2 * T.p + 1) * T.n);
    T.Uf = T.U; T.Uif = T.Ui; T.Ub = T.U; T.Uib = T.Ui;   // low-precision pools mirror offsets
    T.wK = T.wM = -1;
    c->htab.push_back(T);
    return (int)c->htab.size() - 1;
  };
  // a geometry-inclusion table: the knots, Gauss rule and basis tables of its
  // base table, its own weights, matrices, eigenpairs and copies
  auto make_geo_tab = [&](int base) {
    Tab1D T = c->htab[base];
    T.K = take((long long)T.n * T.n); T.M = take((long long)T.n * T.n);
    T.U = take((long long)T.n * T.n); T.D = take(T.n);
    T.Ui = take((long long)T.ni * T.ni); T.Di = take(T.ni);
    T.Up = take((long long)T.n * T.ld); T.Upt = take((long long)T.n * T.ld);
    T.Uip = take((long long)T.ni * T.ldi); T.Uipt = take((long long)T.ni * T.ldi);
    T.Kb = take((long long)(2 * T.p + 1) * T.n); T.Mb = take((long long)(2 * T.p + 1) * T.n);
    T.Uf = T.U; T.Uif = T.Ui; T.Ub = T.U; T.Uib = T.Ui;
    T.wK = take(T.nq); T.wM = take(T.nq);
    c->htab.push_back(T);
    return (int)c->htab.size() - 1;
  };
  int dummy = -1;
  for (int k = 0; k < NP; ++k) {
    int p = prob->degree[k];
    if (p < 1 || p > 10) { set_error("degree must be in [1, 10]"); return AFI_EINVAL; }
    for (int l = 0; l < D; ++l) {
      int ne = prob->nel[k * D + l];
      if (ne < 1 || ne + p < 3 || ne + p > 96) {
        set_error("need 3 <= nel + p <= 96 in every direction");
        return AFI_EINVAL;
      }
      auto key = std::make_pair(ne, p);
      if (!tabidx.count(key)) tabidx[key] = make_tab(ne, p);
    }
  }
  if (D == 2) dummy = make_tab(0, 0);
  c->nbase_tab = (int)c->htab.size();

  // ---- patch descriptors
  long long off = 0, ioff = 0, soff = 0, qoff = 0, xoff = 0;
  c->hp.resize(NP);
  for (int k = 0; k < NP; ++k) {
    DevPatch &P = c->hp[k];
    P = DevPatch{};
    const int p = prob->degree[k];
    P.p = p;
    for (int d = 0; d < 3; ++d) {
      if (d < D) {
        int t = tabidx[std::make_pair(prob->nel[k * D + d], p)];
        const Tab1D &T = c->htab[t];
        P.tab[d] = t; P.n[d] = T.n; P.ni[d] = T.ni; P.nq[d] = T.nq; P.W[d] = 2 * p + 1;
      } else {
        P.tab[d] = dummy; P.n[d] = 1; P.ni[d] = 1; P.nq[d] = 1; P.W[d] = 1;
      }
    }
    P.N = P.n[0] * P.n[1] * P.n[2];
    P.Ni = P.ni[0] * P.ni[1] * P.ni[2];
    P.S = P.W[0] * P.W[1] * P.W[2];
    P.NQ = P.nq[0] * P.nq[1] * P.nq[2];
    P.off = off; off += (long long)D * P.N;
    P.ioff = ioff; ioff += (long long)D * P.Ni;
    P.n1p = P.n[0] + (P.n[0] & 1);
    P.NP = P.n1p * P.n[1] * P.n[2];
    P.soff = soff; soff += (long long)D * D * P.S * P.NP;
    P.qoff = qoff; qoff += P.NQ;
    P.xoff = xoff; xoff += (long long)D * P.N;
    P.lam = prob->lame[2 * k];
    P.mu = prob->lame[2 * k + 1];
    if (!(P.mu > 0.0) || !(P.lam + 2.0 * P.mu / D > 0.0)) { set_error("invalid Lame values"); return AFI_EINVAL; }
    c->max_N = std::max(c->max_N, P.N);
    for (int d = 0; d < D; ++d) c->max_n = std::max(c->max_n, P.n[d]);
  }
  // local-solver descriptors per (patch, component): the plain parametric
  // tables and coefficients (eqs. 5.6, 5.7), or one geometry-inclusion table
  // per (patch, component, direction) with unit coefficients (eqs. 5.12,
  // 5.13); shift and scale follow once H is known
  long long qlo = 0;
  for (int k = 0; k < NP; ++k) {
    DevPatch &P = c->hp[k];
    P.qloff = qlo;
    qlo += P.nq[0] + P.nq[1] + P.nq[2];
    for (int l = 0; l < 3; ++l)
      for (int d = 0; d < 3; ++d) {
        if (c->geo && l < D && d < D) {
          P.ltab[l][d] = make_geo_tab(P.tab[d]);
          P.lcf[l][d] = 1.0;
        } else {
          P.ltab[l][d] = P.tab[d];
          P.lcf[l][d] = c->geo ? 1.0 : ((l == d) ? 2.0 * P.mu + P.lam : P.mu);
        }
      }
    P.lshift = 1.0;
    P.lscale = 1.0;
  }
  if (off >= (1LL << 31)) { set_error("n_dof exceeds 2^31"); return AFI_EINVAL; }
  c->n_dof = (long)off;
  c->n_int = (long)ioff;
  c->nqp = qoff;
  c->stencil_n = soff;
  c->stencil2_n = pair_layout(c->hp, D);
  c->dpool_n = dn;

  // ---- device allocations for tables, patches, geometry
  AFI_TRY(dalloc(c, (void **)&c->dflag, 16));
  AFI_CUDA(cudaMemset(c->dflag, 0, 16));
  AFI_TRY(dalloc(c, (void **)&c->dpool, dn * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->fpool, dn * sizeof(float)));
  AFI_TRY(dalloc(c, (void **)&c->bpool, dn * sizeof(__nv_bfloat16)));
  AFI_CUDA(cudaMemset(c->dpool, 0, dn * sizeof(double)));
  AFI_TRY(upload(c, &c->tabs, c->htab));
  AFI_TRY(upload(c, &c->patches, c->hp));
  std::vector<double> hctrl(prob->ctrl, prob->ctrl + xoff);
  AFI_TRY(upload(c, &c->ctrl, hctrl));
  AFI_CUDA(cudaDeviceSynchronize());
  const auto tf0 = std::chrono::steady_clock::now();
  AFI_TRY(fd_prepare(c));
  AFI_TRY(fd_tc_prepare(c));
  AFI_TRY(build_1d_tables(c));
  if (!c->geo) AFI_TRY(fd_tc_tables(c));   // geometry inclusion: after its tables exist
  AFI_CUDA(cudaDeviceSynchronize());
  c->t_fd_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf0).count();
  launch(k_patch_H, NP, 256, 0, 0, c->patches, c->ctrl, D);
  AFI_LAUNCH_CHECK();
  AFI_CUDA(cudaMemcpy(c->hp.data(), c->patches, NP * sizeof(DevPatch), cudaMemcpyDeviceToHost));
  for (auto &P : c->hp) {   // Lambda = lscale (sum_m lcf D_m + lshift)
    P.lshift = c->geo ? 1.0 / (P.H * P.H) : 1.0;
    P.lscale = c->geo ? 1.0 : P.Hs;
  }
  AFI_CUDA(cudaMemcpy(c->patches, c->hp.data(), NP * sizeof(DevPatch), cudaMemcpyHostToDevice));
  if (opt->variant & AFI_VARIANT_MATRIX_FREE) {
    c->nqp = 0;
    c->stencil_n = 0;
    c->stencil2_n = 0;
    AFI_TRY(mf_setup(c));
  } else if (!(opt->variant & AFI_VARIANT_LOCAL_ONLY)) {
    AFI_TRY(dalloc(c, (void **)&c->qgeo, (size_t)(D * D + 1) * qoff * sizeof(double)));
    AFI_TRY(compute_geometry(c));
    AFI_TRY(dalloc(c, (void **)&c->stencil, (size_t)soff * sizeof(double)));
    AFI_CUDA(cudaMemset(c->stencil, 0, (size_t)soff * sizeof(double)));   // padded nodes stay 0
    AFI_TRY(assemble_stiffness(c));
    if (c->geo) {   // local-solver setup: the fit, its tables, the scalings
      AFI_CUDA(cudaDeviceSynchronize());
      const auto tg0 = std::chrono::steady_clock::now();
      AFI_TRY(geo_setup(c));
      AFI_TRY(fd_tc_tables(c));
      AFI_CUDA(cudaDeviceSynchronize());
      c->t_fd_setup_ms +=
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tg0).count();
    }
    if (!(opt->variant & AFI_VARIANT_STENCIL_F64)) AFI_TRY(stencil_to_pairs(c));
  } else {
    c->nqp = 0;
    c->stencil_n = 0;
  }

  // ---- connectivity: group interface control points by coordinates
  double scale = 0.0;
  {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (long long i = 0; i < xoff; ++i) {
      int d = (int)(i % D);
      lo[d] = std::min(lo[d], prob->ctrl[i]);
      hi[d] = std::max(hi[d], prob->ctrl[i]);
    }
    for (int d = 0; d < D; ++d) scale = std::max(scale, hi[d] - lo[d]);
    if (!(scale > 0.0)) scale = 1.0;
  }
  const double quant = 1e-10 * scale;
  // nested non-conforming faces: their points off the Dirichlet boundary are
  // glued by the nested rows (nested.cu), not by coordinates
  std::vector<NestedFace> nfaces;
  std::set<std::pair<int, int>> apart;
  AFI_TRY(nested_detect(c, prob, quant, nfaces, apart));
  struct Item { std::array<long long, 3> key; int k, i; };
  std::vector<Item> items;
  for (int k = 0; k < NP; ++k) {
    const DevPatch &P = c->hp[k];
    for (int i3 = 0; i3 < P.n[2]; ++i3)
      for (int i2 = 0; i2 < P.n[1]; ++i2)
        for (int i1 = 0; i1 < P.n[0]; ++i1) {
          bool sh = i1 == 0 || i1 == P.n[0] - 1 || i2 == 0 || i2 == P.n[1] - 1;
          if (D == 3) sh = sh || i3 == 0 || i3 == P.n[2] - 1;
          if (!sh) continue;
          int i = idx3(i1, i2, i3, P.n);
          if (!apart.empty() && apart.count({k, i})) continue;
          Item it;
          it.key = {0, 0, 0};
          for (int d = 0; d < D; ++d)
            it.key[d] = std::llround(prob->ctrl[P.xoff + (long long)i * D + d] / quant);
          it.k = k;
          it.i = i;
          items.push_back(it);
        }
  }
  std::sort(items.begin(), items.end(), [](const Item &a, const Item &b) {
    if (a.key != b.key) return a.key < b.key;
    if (a.k != b.k) return a.k < b.k;
    return a.i < b.i;
  });
  std::vector<std::vector<std::pair<int, int>>> nodes;
  for (size_t s = 0; s < items.size();) {
    size_t e = s;
    std::vector<std::pair<int, int>> cp;
    while (e < items.size() && items[e].key == items[s].key) { cp.push_back({items[e].k, items[e].i}); ++e; }
    for (size_t q = 1; q < cp.size(); ++q)
      if (cp[q].first == cp[q - 1].first) { set_error("two control points of one patch coincide"); return AFI_EINVAL; }
    nodes.push_back(cp);
    s = e;
  }
  std::sort(nodes.begin(), nodes.end(), [](const auto &a, const auto &b) { return a[0] < b[0]; });
  auto on_dirichlet = [&](int k, int i) {
    const DevPatch &P = c->hp[k];
    int id[3] = {i % P.n[0], (i / P.n[0]) % P.n[1], i / (P.n[0] * P.n[1])};
    for (int l = 0; l < D; ++l)
      for (int side = 0; side < 2; ++side)
        if (prob->dirichlet_face[k * 2 * D + 2 * l + side] && id[l] == (side ? P.n[l] - 1 : 0))
          return true;
    return false;
  };
  auto dof = [&](int k, int comp, int i) { return (int)(c->hp[k].off + (long long)comp * c->hp[k].N + i); };

  // ---- constraint rows
  std::vector<int2> rc, grp, rpatch;
  for (int comp = 0; comp < D; ++comp)
    for (const auto &cp : nodes) {
      bool dir = false;
      for (auto &q : cp) dir = dir || on_dirichlet(q.first, q.second);
      if (dir) {
        for (auto &q : cp) {
          rc.push_back(make_int2(dof(q.first, comp, q.second), -1));
          grp.push_back(make_int2((int)rc.size() - 1, 0));
          rpatch.push_back(make_int2(q.first, -1));
        }
      } else if (cp.size() >= 2) {
        int start = (int)rc.size();
        for (size_t j = 1; j < cp.size(); ++j) {
          rc.push_back(make_int2(dof(cp[0].first, comp, cp[0].second), dof(cp[j].first, comp, cp[j].second)));
          grp.push_back(make_int2(start, (int)cp.size()));
          rpatch.push_back(make_int2(cp[0].first, cp[j].first));
        }
      }
    }
  c->n_c = (long)rc.size();
  c->n_c0 = c->n_c;
  // B^T CSR over shell dofs, per-patch row lists, pair lists for G^T G
  std::map<int, std::vector<int>> by_dof;
  std::vector<std::vector<int4>> plist(NP);
  std::map<std::pair<int, int>, std::vector<int4>> pairs;
  for (int r = 0; r < (int)rc.size(); ++r) {
    by_dof[rc[r].x].push_back(2 * r);
    plist[rpatch[r].x].push_back(make_int4(rc[r].x, rc[r].x, 1, 2 * r));
    if (rc[r].y >= 0) {
      by_dof[rc[r].y].push_back(2 * r + 1);
      plist[rpatch[r].y].push_back(make_int4(rc[r].y, rc[r].y, 1, 2 * r + 1));
      int ka = rpatch[r].x, kb = rpatch[r].y;
      if (ka < kb) pairs[{ka, kb}].push_back(make_int4(rc[r].x, rc[r].y, -1, 0));
      else pairs[{kb, ka}].push_back(make_int4(rc[r].y, rc[r].x, -1, 0));
    }
  }
  std::vector<int> shell, btp(1, 0), bte;
  for (auto &kv : by_dof) {
    shell.push_back(kv.first);
    for (int e : kv.second) bte.push_back(e);
    btp.push_back((int)bte.size());
  }
  c->n_shell = (long)shell.size();
  std::vector<int> pptr(1, 0);
  std::vector<int2> pent;
  for (int k = 0; k < NP; ++k) {
    std::vector<int4> lst = plist[k];
    std::sort(lst.begin(), lst.end(), [](const int4 &a, const int4 &b) {   // by dof: by component
      return a.x != b.x ? a.x < b.x : a.w < b.w;
    });
    for (auto &e : lst) pent.push_back(make_int2(e.w, e.x));
    pptr.push_back((int)pent.size());
  }
  AFI_TRY(upload(c, &c->row_copy, rc));
  AFI_TRY(upload(c, &c->row_grp, grp));
  AFI_TRY(upload(c, &c->row_patch, rpatch));
  AFI_TRY(upload(c, &c->shell_dof, shell));
  AFI_TRY(upload(c, &c->bt_ptr, btp));
  AFI_TRY(upload(c, &c->bt_ent, bte));
  AFI_TRY(upload(c, &c->prow_ptr, pptr));
  AFI_TRY(upload(c, &c->prow_ent, pent));
  AFI_TRY(rigid_tables(c));
  // rows of the nested faces after the node rows, and their G coefficients
  AFI_TRY(nested_build(c, prob, nfaces));
  AFI_TRY(nested_gcoef(c));

  // ---- G^T G (diagonal blocks from the per-patch lists, off-diagonal from
  //      the patch pairs) and its inverse; R^T R per patch and its inverse
  const int nm = c->nm;
  c->ng = nm * NP;
  AFI_TRY(dalloc(c, (void **)&c->GtG, (size_t)c->ng * c->ng * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->GtG_inv, (size_t)c->ng * c->ng * sizeof(double)));
  AFI_CUDA(cudaMemset(c->GtG, 0, (size_t)c->ng * c->ng * sizeof(double)));
  {
    std::vector<int> bptr(1, 0);
    std::vector<int2> bkk;
    std::vector<int4> bent;
    for (int k = 0; k < NP; ++k) {
      for (auto &e : plist[k]) bent.push_back(make_int4(e.x, e.y, 1, 0));
      bptr.push_back((int)bent.size());
      bkk.push_back(make_int2(k, k));
    }
    int ndiag = NP;
    for (auto &kv : pairs) {
      for (auto &e : kv.second) bent.push_back(e);
      bptr.push_back((int)bent.size());
      bkk.push_back(make_int2(kv.first.first, kv.first.second));
    }
    int *dptr; int2 *dkk; int4 *dent;
    AFI_CUDA(cudaMalloc(&dptr, bptr.size() * sizeof(int)));
    AFI_CUDA(cudaMalloc(&dkk, std::max<size_t>(1, bkk.size()) * sizeof(int2)));
    AFI_CUDA(cudaMalloc(&dent, std::max<size_t>(1, bent.size()) * sizeof(int4)));
    cudaMemcpy(dptr, bptr.data(), bptr.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(dkk, bkk.data(), bkk.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (!bent.empty()) cudaMemcpy(dent, bent.data(), bent.size() * sizeof(int4), cudaMemcpyHostToDevice);
    launch(k_rr_blocks, ndiag, 256, 0, 0, c->patches, c->ctrl, dptr, dkk, dent, c->GtG, c->ng, nm, D, 0);
    int npair = (int)bkk.size() - ndiag;
    if (npair > 0)
      launch(k_rr_blocks, npair, 256, 0, 0, c->patches, c->ctrl, dptr + ndiag, dkk + ndiag, dent, c->GtG, c->ng, nm, D, 1);
    AFI_LAUNCH_CHECK();
    AFI_TRY(nested_gtg(c));
    // R^T R per patch
    AFI_TRY(dalloc(c, (void **)&c->RtR_inv, (size_t)NP * nm * nm * sizeof(double)));
    launch(k_RtR, NP, 256, 0, 0, c->patches, c->ctrl, c->RtR_inv, D, nm);
    AFI_LAUNCH_CHECK();
    AFI_TRY(small_inverses(c, c->RtR_inv, nm, NP));
    afi_status st = AFI_OK;
    double *lscratch = nullptr;
    AFI_CUDA(cudaMalloc(&lscratch, ((size_t)c->ng * c->ng + c->ng) * sizeof(double)));
    if (c->n_c > 0) st = dense_spd_inverse(c, c->GtG, c->GtG_inv, c->ng, lscratch);
    cudaFree(lscratch);
    cudaFree(dptr); cudaFree(dkk); cudaFree(dent);
    AFI_TRY(st);
  }

  // ---- workspaces
  const long long nt = c->n_dof + c->n_c;
  c->ws_n = (long long)(kOpScratch + kKrylov) * nt + 16;
  AFI_TRY(dalloc(c, (void **)&c->ws, c->ws_n * sizeof(double)));
  // local-solver scratch for tensors that do not fit in shared memory:
  // 4 slabs per (patch, component) block in the widest precision
  c->fdscratch_n = 4LL * c->n_dof + 16;
  AFI_TRY(dalloc(c, (void **)&c->fdscratch, c->fdscratch_n * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->ps_buf, (size_t)4 * c->n_dof * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->ps_rint, (size_t)std::max(1L, c->n_int) * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->ps_vint, (size_t)std::max(1L, c->n_int) * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->small, kSmallDoubles * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->part, (size_t)NP * 64 * 6 * sizeof(double)));
  AFI_CUDA(cudaMemset(c->small, 0, kSmallDoubles * sizeof(double)));
  AFI_CUDA(cudaMallocHost((void **)&c->host_small, 128 * sizeof(double)));
  {
    cudaStream_t cs = nullptr, as = nullptr;
    AFI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    c->cap_stream = cs;
    AFI_CUDA(cudaStreamCreateWithFlags(&as, cudaStreamNonBlocking));
    c->aux_stream = as;
    cudaEvent_t ef = nullptr, ej = nullptr;
    AFI_CUDA(cudaEventCreateWithFlags(&ef, cudaEventDisableTiming));
    AFI_CUDA(cudaEventCreateWithFlags(&ej, cudaEventDisableTiming));
    c->ev_fork = ef;
    c->ev_join = ej;
  }
  {   // the FD work splits (tensor-core / three-pass / SIMT), part of the FD setup
    const auto ts0 = std::chrono::steady_clock::now();
    AFI_TRY(fd_tc_ready(c));
    AFI_CUDA(cudaDeviceSynchronize());
    c->t_fd_setup_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts0).count();
  }
  if (opt->variant & AFI_VARIANT_EXACT) {   // exact local solvers: also local-solver setup
    const auto ts0 = std::chrono::steady_clock::now();
    AFI_TRY(exact_setup(c));
    c->t_fd_setup_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts0).count();
  }
  AFI_CUDA(cudaDeviceSynchronize());
  auto t1 = std::chrono::steady_clock::now();
  c->t_setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  return AFI_OK;
}

void free_context(afi_ctx *c) {
  if (c->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
  if (c->mgraph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->mgraph_exec);
  if (c->cap_stream) cudaStreamDestroy((cudaStream_t)c->cap_stream);
  if (c->aux_stream) cudaStreamDestroy((cudaStream_t)c->aux_stream);
  if (c->ev_fork) cudaEventDestroy((cudaEvent_t)c->ev_fork);
  if (c->ev_join) cudaEventDestroy((cudaEvent_t)c->ev_join);
  void *ptrs[] = {c->patches, c->tabs, c->dpool, c->fpool, c->bpool, c->tcpool, c->ctrl, c->stencil,
                  c->qgeo, c->row_copy, c->row_grp, c->row_patch, c->shell_dof, c->bt_ptr,
                  c->bt_ent, c->prow_ptr, c->prow_ent, c->pair_ptr, c->pair_kk, c->pair_ent,
                  c->GtG, c->GtG_inv, c->RtR_inv, c->ws, c->fdscratch, c->small, c->part,
                  c->dflag, c->tcsplit[0][0].d_tc, c->tcsplit[0][0].d_simt, c->tcsplit[0][1].d_tc,
                  c->tcsplit[0][1].d_simt, c->tcsplit[1][0].d_tc, c->tcsplit[1][0].d_simt,
                  c->tcsplit[1][1].d_tc, c->tcsplit[1][1].d_simt, c->tcsplit[0][0].d_plane,
                  c->tcsplit[0][0].d_line, c->tcsplit[0][1].d_plane, c->tcsplit[0][1].d_line,
                  c->tcsplit[1][0].d_plane, c->tcsplit[1][0].d_line, c->tcsplit[1][1].d_plane,
                  c->tcsplit[1][1].d_line, c->prow_coef, c->row_cp, c->row_cv, c->ps_buf,
                  c->ps_rint, c->ps_vint, c->xsplit, c->stencil2, c->ex_Kinv, c->ex_AIIinv,
                  c->ex_koff, c->ex_aoff, c->geo_dA, c->geo_dS, c->geo_tmp, c->mws, c->mst,
                  c->xsplit_multi, c->nest_ptr, c->nest_ent, c->nest_w, c->nest_eki, c->nd_dof,
                  c->nd_ptr, c->nd_ent, c->nd_w, c->nblk_ptr, c->nblk_off, c->nest_binv, c->nest_gk,
                  c->nest_gc, c->pn_ptr, c->pn_ent, c->nest_tmp, c->tcsplit[0][0].d_pbounds,
                  c->tcsplit[0][0].d_lbounds, c->tcsplit[0][1].d_pbounds, c->tcsplit[0][1].d_lbounds,
                  c->tcsplit[1][0].d_pbounds, c->tcsplit[1][0].d_lbounds, c->tcsplit[1][1].d_pbounds,
                  c->tcsplit[1][1].d_lbounds, c->mf_eoff, c->mf_ctrlf, c->mf_xf, c->mf_yf};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->host_small) cudaFreeHost(c->host_small);
  if (c->host_mst) cudaFreeHost(c->host_mst);
}

}  // namespace afi
