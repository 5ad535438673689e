// Nested non-conforming interfaces (Section 2): a face whose knot vectors
// refine the neighbouring patch's.  The coarse side's splines are linear
// combinations of the fine side's, so instead of matching control points
// the gluing rows tie every fine face coefficient off the Dirichlet boundary
// to that combination of the coarse ones (the knot-insertion property used
// in the paper's non-conforming test, Section 6):
//     row:  u_fine(i) - sum_j W[i][j] u_coarse(j),
// W = E_t1 (x) E_t2 the refinement matrices of the two tangential directions,
// computed here by Boehm's knot insertion, one knot at a time.
//
// Host-side detection and bookkeeping: faces whose corners coincide in the
// same tangential order but whose point counts differ; checks (one degree,
// element counts that divide, the fine net equal to the refined coarse net,
// face edges on the Dirichlet boundary); the rows in CSR and transposed
// CSR; the (face, component) blocks of B B^T (these rows share no dof with
// the node rows) and their dense inverses.  The kernels that apply the rows
// live in ops.cu.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <map>

namespace afi {

namespace {

// Local indices (increasing) of the points of face f = 2 l + side of a patch
// with basis counts n[3], and their tangential indices (directions != l in
// increasing order; the third direction of a 2D patch has n = 1).
void face_points(const int *n, int dim, int f, std::vector<int> &pts, std::vector<std::array<int, 2>> &ti,
                 int tang[2]) {
  const int l = f / 2, side = f % 2;
  int q = 0;
  for (int t = 0; t < dim; ++t)
    if (t != l) tang[q++] = t;
  if (dim == 2) tang[1] = 2;
  pts.clear();
  ti.clear();
  for (int i3 = 0; i3 < n[2]; ++i3)
    for (int i2 = 0; i2 < n[1]; ++i2)
      for (int i1 = 0; i1 < n[0]; ++i1) {
        const int im[3] = {i1, i2, i3};
        if (im[l] != (side ? n[l] - 1 : 0)) continue;
        pts.push_back(i1 + n[0] * (i2 + n[1] * i3));
        ti.push_back({im[tang[0]], im[tang[1]]});
      }
}

// Refinement matrix E [(nel_f + p) x (nel_c + p)], row-major: fine
// coefficients = E coarse coefficients, for the open uniform knot vectors of
// nel_c and nel_f elements (nel_f a multiple of nel_c).  Boehm's insertion
// of each fine knot that is not a coarse knot, in increasing order.
std::vector<double> refinement(int nel_c, int nel_f, int p) {
  std::vector<double> U;
  for (int j = 0; j <= p; ++j) U.push_back(0.0);
  for (int j = 1; j < nel_c; ++j) U.push_back((double)j / nel_c);
  for (int j = 0; j <= p; ++j) U.push_back(1.0);
  const int nc = nel_c + p;
  std::vector<std::vector<double>> C(nc, std::vector<double>(nc, 0.0));
  for (int i = 0; i < nc; ++i) C[i][i] = 1.0;
  const int r = nel_f / nel_c;
  for (int j = 1; j < nel_f; ++j) {
    if (j % r == 0) continue;   // already a coarse knot
    const double u = (double)j / nel_f;
    const int n = (int)C.size();
    int k = p;
    while (k + 1 < n && U[k + 1] <= u) ++k;   // U[k] <= u < U[k + 1]
    std::vector<std::vector<double>> D(n + 1, std::vector<double>(nc, 0.0));
    for (int i = 0; i <= n; ++i) {
      if (i <= k - p) {
        D[i] = C[i];
      } else if (i >= k + 1) {
        D[i] = C[i - 1];
      } else {
        const double a = (u - U[i]) / (U[i + p] - U[i]);
        for (int m = 0; m < nc; ++m) D[i][m] = a * C[i][m] + (1.0 - a) * C[i - 1][m];
      }
    }
    U.insert(U.begin() + k + 1, u);
    C.swap(D);
  }
  std::vector<double> E;
  for (auto &row : C) E.insert(E.end(), row.begin(), row.end());
  return E;
}

}  // namespace

afi_status nested_detect(afi_ctx *c, const afi_problem *prob, double quant,
                         std::vector<NestedFace> &faces, std::set<std::pair<int, int>> &apart) {
  const int D = c->dim, NP = c->npatch, nfaces = 2 * D;
  auto on_dirichlet = [&](int k, int i) {
    const DevPatch &P = c->hp[k];
    const int id[3] = {i % P.n[0], (i / P.n[0]) % P.n[1], i / (P.n[0] * P.n[1])};
    for (int l = 0; l < D; ++l)
      for (int side = 0; side < 2; ++side)
        if (prob->dirichlet_face[k * 2 * D + 2 * l + side] && id[l] == (side ? P.n[l] - 1 : 0))
          return true;
    return false;
  };
  auto key = [&](int k, int i) {
    std::array<long long, 3> kk{0, 0, 0};
    for (int d = 0; d < D; ++d) kk[d] = std::llround(prob->ctrl[c->hp[k].xoff + (long long)i * D + d] / quant);
    return kk;
  };
  // corners of every face, in tangential order
  struct FaceC { int k, f; std::vector<std::array<long long, 3>> corner; int tang[2]; int nt[2]; };
  std::vector<FaceC> fc;
  std::map<std::vector<std::array<long long, 3>>, std::vector<int>> by_set;
  for (int k = 0; k < NP; ++k)
    for (int f = 0; f < nfaces; ++f) {
      const DevPatch &P = c->hp[k];
      FaceC F{k, f, {}, {0, 0}, {1, 1}};
      std::vector<int> pts;
      std::vector<std::array<int, 2>> ti;
      face_points(P.n, D, f, pts, ti, F.tang);
      for (int t = 0; t < D - 1; ++t) F.nt[t] = P.n[F.tang[t]];
      for (size_t q = 0; q < pts.size(); ++q) {
        const bool end0 = ti[q][0] == 0 || ti[q][0] == F.nt[0] - 1;
        const bool end1 = D == 2 || ti[q][1] == 0 || ti[q][1] == F.nt[1] - 1;
        if (end0 && end1) F.corner.push_back(key(k, pts[q]));
      }
      auto set = F.corner;
      std::sort(set.begin(), set.end());
      by_set[set].push_back((int)fc.size());
      fc.push_back(F);
    }
  for (auto &kv : by_set) {
    const auto &ids = kv.second;
    for (size_t a = 0; a < ids.size(); ++a)
      for (size_t b = a + 1; b < ids.size(); ++b) {
        const FaceC &A = fc[ids[a]], &B = fc[ids[b]];
        if (A.k == B.k) continue;
        const bool same = A.nt[0] == B.nt[0] && A.nt[1] == B.nt[1];
        if (same) continue;   // a conforming face: matched by coordinates
        if (A.corner != B.corner) {
          set_error("nested interface between faces of different orientation");
          return AFI_EINVAL;
        }
        const DevPatch &PA = c->hp[A.k], &PB = c->hp[B.k];
        if (PA.p != PB.p) {
          set_error("nested interface between patches of different degree");
          return AFI_EINVAL;
        }
        // the fine side has at least as many points in both tangential directions
        const bool afine = A.nt[0] >= B.nt[0] && A.nt[1] >= B.nt[1];
        const bool bfine = B.nt[0] >= A.nt[0] && B.nt[1] >= A.nt[1];
        if (!afine && !bfine) {
          set_error("interface that neither matches nor nests");
          return AFI_EINVAL;
        }
        const FaceC &Fc = afine ? B : A, &Ff = afine ? A : B;
        NestedFace nf;
        nf.kc = Fc.k; nf.fc = Fc.f; nf.kf = Ff.k; nf.ff = Ff.f;
        const int p = PA.p;
        std::vector<double> E[2];
        for (int t = 0; t < D - 1; ++t) {
          const int nec = Fc.nt[t] - p, nef = Ff.nt[t] - p;
          if (nec < 1 || nef % nec != 0) {
            set_error("nested interface whose knot vectors do not refine one another");
            return AFI_EINVAL;
          }
          E[t] = refinement(nec, nef, p);
        }
        std::vector<std::array<int, 2>> tc_, tf_;
        int tg[2];
        face_points(c->hp[nf.kc].n, D, nf.fc, nf.pc, tc_, tg);
        face_points(c->hp[nf.kf].n, D, nf.ff, nf.pf, tf_, tg);
        const int ncp = (int)nf.pc.size(), nfp = (int)nf.pf.size();
        nf.W.assign((size_t)nfp * ncp, 0.0);
        for (int i = 0; i < nfp; ++i)
          for (int j = 0; j < ncp; ++j) {
            double w = E[0][(size_t)tf_[i][0] * Fc.nt[0] + tc_[j][0]];
            if (D == 3) w *= E[1][(size_t)tf_[i][1] * Fc.nt[1] + tc_[j][1]];
            nf.W[(size_t)i * ncp + j] = w;
          }
        // the fine net must be the refined coarse net
        double err = 0.0;
        for (int i = 0; i < nfp; ++i)
          for (int d = 0; d < D; ++d) {
            double v = 0.0;
            for (int j = 0; j < ncp; ++j)
              v += nf.W[(size_t)i * ncp + j] * prob->ctrl[c->hp[nf.kc].xoff + (long long)nf.pc[j] * D + d];
            err = std::max(err, std::fabs(v - prob->ctrl[c->hp[nf.kf].xoff + (long long)nf.pf[i] * D + d]));
          }
        if (err > 1e3 * quant) {
          set_error("nested interface whose fine control net is not the refined coarse net");
          return AFI_EINVAL;
        }
        // face edges on the Dirichlet boundary; the other face points are
        // glued by the nested rows, not by coordinates
        for (int side = 0; side < 2; ++side) {
          const int k = side ? nf.kf : nf.kc;
          const std::vector<int> &pts = side ? nf.pf : nf.pc;
          const std::vector<std::array<int, 2>> &ti = side ? tf_ : tc_;
          const int *nt = side ? Ff.nt : Fc.nt;
          for (size_t q = 0; q < pts.size(); ++q) {
            const bool edge = ti[q][0] == 0 || ti[q][0] == nt[0] - 1 ||
                              (D == 3 && (ti[q][1] == 0 || ti[q][1] == nt[1] - 1));
            const bool dir = on_dirichlet(k, pts[q]);
            if (edge && !dir) {
              set_error("nested interface whose edges are not on the Dirichlet boundary");
              return AFI_EINVAL;
            }
            if (!dir) apart.insert({k, pts[q]});
          }
        }
        faces.push_back(std::move(nf));
      }
  }
  std::sort(faces.begin(), faces.end(), [](const NestedFace &a, const NestedFace &b) {
    return a.kf != b.kf ? a.kf < b.kf : a.ff < b.ff;
  });
  return AFI_OK;
}

namespace {

// Inverse of a dense symmetric positive definite matrix (row-major, n x n)
// by Cholesky: A = L L^T, A^{-1} = L^{-T} L^{-1}.  False if A is not SPD.
bool spd_inverse_host(std::vector<double> &A, int n) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  // columns of L^{-1}
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c)
    for (int i = c; i < n; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[(size_t)i * n + k] * Li[(size_t)k * n + c];
      Li[(size_t)i * n + c] = v / L[(size_t)i * n + i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = 0.0;
      for (int k = i; k < n; ++k) v += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      A[(size_t)i * n + j] = v;
      A[(size_t)j * n + i] = v;
    }
  return true;
}

template <typename T>
afi_status upload_vec(afi_ctx *c, T **dst, const std::vector<T> &src) {
  AFI_TRY(dalloc(c, (void **)dst, std::max<size_t>(1, src.size()) * sizeof(T)));
  if (!src.empty())
    AFI_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return AFI_OK;
}

}  // namespace

// Rows n_c0 .. n_c0 + n_nest - 1: faces in the given order, then component,
// then free fine point (increasing local index).  Each (face, component)
// block of rows touches dofs no other row touches, so B B^T is block
// diagonal over the node groups and these blocks.
afi_status nested_build(afi_ctx *c, const afi_problem *prob, const std::vector<NestedFace> &faces) {
  c->n_c0 = c->n_c;
  if (faces.empty()) return AFI_OK;
  const int D = c->dim, NP = c->npatch;
  auto on_dirichlet = [&](int k, int i) {
    const DevPatch &P = c->hp[k];
    const int id[3] = {i % P.n[0], (i / P.n[0]) % P.n[1], i / (P.n[0] * P.n[1])};
    for (int l = 0; l < D; ++l)
      for (int side = 0; side < 2; ++side)
        if (prob->dirichlet_face[k * 2 * D + 2 * l + side] && id[l] == (side ? P.n[l] - 1 : 0))
          return true;
    return false;
  };
  auto dof = [&](int k, int comp, int i) { return (int)(c->hp[k].off + (long long)comp * c->hp[k].N + i); };
  std::vector<int> ptr(1, 0), ent, bptr(1, 0);
  std::vector<double> w;
  std::vector<int4> eki;
  std::vector<int2> gk;
  for (const NestedFace &F : faces) {
    const int ncp = (int)F.pc.size();
    std::vector<int> cfree;
    for (int j = 0; j < ncp; ++j)
      if (!on_dirichlet(F.kc, F.pc[j])) cfree.push_back(j);
    for (int comp = 0; comp < D; ++comp) {
      for (size_t a = 0; a < F.pf.size(); ++a) {
        if (on_dirichlet(F.kf, F.pf[a])) continue;
        ent.push_back(dof(F.kf, comp, F.pf[a]));
        w.push_back(1.0);
        eki.push_back(make_int4(F.kf, comp, F.pf[a], 0));
        for (int j : cfree) {
          const double v = F.W[a * ncp + j];
          if (v == 0.0) continue;
          ent.push_back(dof(F.kc, comp, F.pc[j]));
          w.push_back(-v);
          eki.push_back(make_int4(F.kc, comp, F.pc[j], 1));
        }
        ptr.push_back((int)ent.size());
        gk.push_back(make_int2(F.kf, F.kc));
      }
      bptr.push_back((int)gk.size());
    }
  }
  const int nr = (int)gk.size();
  // transposed lists: per dof, its (row, weight)
  std::map<int, std::vector<std::pair<int, double>>> T;
  for (int r = 0; r < nr; ++r)
    for (int e = ptr[r]; e < ptr[r + 1]; ++e) T[ent[e]].push_back({r, w[e]});
  std::vector<int> nd_dof, nd_ptr(1, 0), nd_ent;
  std::vector<double> nd_w;
  for (auto &kv : T) {
    nd_dof.push_back(kv.first);
    for (auto &q : kv.second) { nd_ent.push_back(q.first); nd_w.push_back(q.second); }
    nd_ptr.push_back((int)nd_ent.size());
  }
  // dense (B B^T)^{-1} per block
  std::vector<long long> boff(1, 0);
  std::vector<double> binv;
  const int nblk = (int)bptr.size() - 1;
  std::vector<int> blk_of(nr);
  for (int b = 0; b < nblk; ++b)
    for (int r = bptr[b]; r < bptr[b + 1]; ++r) blk_of[r] = b;
  for (int b = 0; b < nblk; ++b) {
    const int r0 = bptr[b], m = bptr[b + 1] - r0;
    std::vector<double> M((size_t)m * m, 0.0);
    for (auto &kv : T)
      for (auto &q1 : kv.second) {
        if (blk_of[q1.first] != b) continue;
        for (auto &q2 : kv.second) {
          if (blk_of[q2.first] != b) {
            set_error("nested rows of two blocks share a dof");
            return AFI_EINVAL;
          }
          M[(size_t)(q1.first - r0) * m + (q2.first - r0)] += q1.second * q2.second;
        }
      }
    if (!spd_inverse_host(M, m)) {
      set_error("B B^T of a nested face is not positive definite");
      return AFI_ESINGULAR;
    }
    binv.insert(binv.end(), M.begin(), M.end());
    boff.push_back((long long)binv.size());
  }
  // per patch: the rows touching it (row * 2 + side, side 1 = coarse)
  std::vector<std::vector<int>> pl(NP);
  for (int r = 0; r < nr; ++r) {
    pl[gk[r].x].push_back(2 * r);
    pl[gk[r].y].push_back(2 * r + 1);
  }
  std::vector<int> pn_ptr(1, 0), pn_ent;
  for (int k = 0; k < NP; ++k) {
    pn_ent.insert(pn_ent.end(), pl[k].begin(), pl[k].end());
    pn_ptr.push_back((int)pn_ent.size());
  }
  AFI_TRY(upload_vec(c, &c->nest_ptr, ptr));
  AFI_TRY(upload_vec(c, &c->nest_ent, ent));
  AFI_TRY(upload_vec(c, &c->nest_w, w));
  AFI_TRY(upload_vec(c, &c->nest_eki, eki));
  AFI_TRY(upload_vec(c, &c->nest_gk, gk));
  AFI_TRY(upload_vec(c, &c->nd_dof, nd_dof));
  AFI_TRY(upload_vec(c, &c->nd_ptr, nd_ptr));
  AFI_TRY(upload_vec(c, &c->nd_ent, nd_ent));
  AFI_TRY(upload_vec(c, &c->nd_w, nd_w));
  AFI_TRY(upload_vec(c, &c->nblk_ptr, bptr));
  AFI_TRY(upload_vec(c, &c->nblk_off, boff));
  AFI_TRY(upload_vec(c, &c->nest_binv, binv));
  AFI_TRY(upload_vec(c, &c->pn_ptr, pn_ptr));
  AFI_TRY(upload_vec(c, &c->pn_ent, pn_ent));
  AFI_TRY(dalloc(c, (void **)&c->nest_gc, (size_t)nr * 2 * c->nm * sizeof(double)));
  AFI_TRY(dalloc(c, (void **)&c->nest_tmp, (size_t)nr * sizeof(double)));
  c->n_nest = nr;
  c->n_nd = (long)nd_dof.size();
  c->n_nblk = nblk;
  c->n_c = c->n_c0 + nr;
  return AFI_OK;
}

// G^T G += sum over the nested rows of g_r g_r^T (g_r: the row's G
// coefficients on its fine and coarse patch), added on the host in FP64.
afi_status nested_gtg(afi_ctx *c) {
  if (!c->n_nest) return AFI_OK;
  const int nm = c->nm, ng = c->ng, nr = (int)c->n_nest;
  std::vector<double> G((size_t)ng * ng), gc((size_t)nr * 2 * nm);
  std::vector<int2> gk(nr);
  AFI_CUDA(cudaDeviceSynchronize());
  AFI_CUDA(cudaMemcpy(G.data(), c->GtG, G.size() * sizeof(double), cudaMemcpyDeviceToHost));
  AFI_CUDA(cudaMemcpy(gc.data(), c->nest_gc, gc.size() * sizeof(double), cudaMemcpyDeviceToHost));
  AFI_CUDA(cudaMemcpy(gk.data(), c->nest_gk, gk.size() * sizeof(int2), cudaMemcpyDeviceToHost));
  for (int r = 0; r < nr; ++r) {
    const int kk[2] = {gk[r].x, gk[r].y};
    const double *g = gc.data() + (size_t)r * 2 * nm;
    for (int s1 = 0; s1 < 2; ++s1)
      for (int s2 = 0; s2 < 2; ++s2)
        for (int a = 0; a < nm; ++a)
          for (int b = 0; b < nm; ++b)
            G[(size_t)(kk[s1] * nm + a) * ng + kk[s2] * nm + b] += g[s1 * nm + a] * g[s2 * nm + b];
  }
  AFI_CUDA(cudaMemcpy(c->GtG, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice));
  return AFI_OK;
}

}  // namespace afi
