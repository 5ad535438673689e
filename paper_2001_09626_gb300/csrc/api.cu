// extern "C" entry points declared in include/afieti.h.
#include "common.cuh"

#include <algorithm>

namespace afi {
const char *last_error_cstr();
}

using namespace afi;

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// entry points that need the assembled stiffness or the quadrature geometry
static bool has_operator(afi_ctx *c) {
  if (c->stencil || c->mf) return true;
  set_error("context set up with AFI_VARIANT_LOCAL_ONLY: no stiffness or geometry");
  return false;
}

extern "C" {

afi_status af_ieti_setup(const afi_problem *prob, const afi_options *opt, afi_ctx **out) {
  if (!out) { set_error("out is null"); return AFI_EINVAL; }
  *out = nullptr;
  afi_ctx *c = new (std::nothrow) afi_ctx();
  if (!c) { set_error("host allocation failed"); return AFI_ENOMEM; }
  afi_status st = setup_context(prob, opt, c);
  if (st != AFI_OK) {
    free_context(c);
    delete c;
    return st;
  }
  *out = c;
  return AFI_OK;
}

void af_ieti_destroy(afi_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  free_context(c);
  delete c;
}

afi_status fd_apply(afi_ctx *c, int interior, const double *r, double *s, int nrhs, void *stream) {
  if (!c || !r || !s || nrhs < 1 || (interior != 0 && interior != 1)) {
    set_error("fd_apply: invalid argument");
    return AFI_EINVAL;
  }
  return fd_run(c, interior, r, s, as_stream(stream), nrhs);
}

static afi_status solve_many(afi_ctx *c, const double *f, double *u, double *lam, int nrhs,
                             afi_info *info, void *stream) {
  if (!c || !f || !u || nrhs < 1) { set_error("solve: invalid argument"); return AFI_EINVAL; }
  if (!has_operator(c)) return AFI_EINVAL;
  // batches of up to kMaxRhs right-hand sides solved in lockstep (one
  // stiffness pass per iteration for the whole batch); info aggregates the
  // batches: largest iteration count and residuals, summed solve time
  afi_status worst = AFI_OK;
  afi_info agg{};
  for (int j = 0; j < nrhs; j += kMaxRhs) {
    const int nb = std::min(kMaxRhs, nrhs - j);
    afi_info bi{};
    const double *fj = f + (long long)j * c->n_dof;
    double *uj = u + (long long)j * c->n_dof;
    double *lj = lam ? lam + (long long)j * c->n_c : nullptr;
    afi_status st = AFI_OK;
    if (nb == 1) {
      st = solve_one(c, fj, uj, lj, &bi, as_stream(stream));
    } else if (c->mf) {
      // matrix-free products gain nothing from lockstep (no shared
      // coefficient stream): one solve per right-hand side
      for (int r = 0; r < nb && st != AFI_EBREAKDOWN && st != AFI_ECUDA; ++r) {
        afi_info ri{};
        const afi_status sr = solve_one(c, fj + (long long)r * c->n_dof, uj + (long long)r * c->n_dof,
                                        lj ? lj + (long long)r * c->n_c : nullptr, &ri, as_stream(stream));
        bi.iters = std::max(bi.iters, ri.iters);
        bi.relres_est = std::max(bi.relres_est, ri.relres_est);
        bi.relres_true = std::max(bi.relres_true, ri.relres_true);
        bi.t_setup_ms = ri.t_setup_ms;
        bi.t_fd_setup_ms = ri.t_fd_setup_ms;
        bi.t_solve_ms += ri.t_solve_ms;
        bi.fp64_restarts += ri.fp64_restarts;
        if (sr != AFI_OK && (st == AFI_OK || sr == AFI_EBREAKDOWN || sr == AFI_ECUDA)) st = sr;
      }
    } else {
      st = solve_multi(c, fj, uj, lj, nb, &bi, as_stream(stream));
    }
    agg.iters = std::max(agg.iters, bi.iters);
    agg.relres_est = std::max(agg.relres_est, bi.relres_est);
    agg.relres_true = std::max(agg.relres_true, bi.relres_true);
    agg.t_setup_ms = bi.t_setup_ms;
    agg.t_fd_setup_ms = bi.t_fd_setup_ms;
    agg.t_solve_ms += bi.t_solve_ms;
    agg.fp64_restarts += bi.fp64_restarts;
    if (st == AFI_EBREAKDOWN || st == AFI_ECUDA || st == AFI_EINVAL || st == AFI_ENOMEM) {
      if (info) *info = agg;
      return st;
    }
    if (st != AFI_OK) worst = st;
  }
  if (info) *info = agg;
  return worst;
}

afi_status ieti_solve(afi_ctx *c, const double *f, double *u, double *lam, int nrhs,
                      afi_info *info, void *stream) {
  return solve_many(c, f, u, lam, nrhs, info, stream);
}

afi_status ieti_solve_adjoint(afi_ctx *c, const double *g, double *z, double *zl, int nrhs,
                              afi_info *info, void *stream) {
  return solve_many(c, g, z, zl, nrhs, info, stream);
}

afi_status afi_lame_grad(afi_ctx *c, const double *u, const double *z, double *grad, void *stream) {
  if (!c || !u || !z || !grad) { set_error("afi_lame_grad: invalid argument"); return AFI_EINVAL; }
  if (!has_operator(c)) return AFI_EINVAL;
  if (c->mf) { set_error("afi_lame_grad: not available with AFI_VARIANT_MATRIX_FREE"); return AFI_EINVAL; }
  return op_lame_grad(c, u, z, grad, as_stream(stream));
}

afi_status afi_load_vector(afi_ctx *c, const double *coef, double *f, void *stream) {
  if (!c || !coef || !f) { set_error("afi_load_vector: invalid argument"); return AFI_EINVAL; }
  if (!has_operator(c)) return AFI_EINVAL;
  return op_load(c, coef, f, as_stream(stream));
}

afi_status afi_apply(afi_ctx *c, afi_operator op, const double *x, double *y, void *stream) {
  if (!c || !x || !y) { set_error("afi_apply: invalid argument"); return AFI_EINVAL; }
  cudaStream_t s = as_stream(stream);
  if ((op == AFI_OP_STIFFNESS || op == AFI_OP_SADDLE) && !has_operator(c)) return AFI_EINVAL;
  switch (op) {
    case AFI_OP_STIFFNESS: return op_stiffness(c, x, y, s);
    case AFI_OP_B: return op_B(c, x, y, s);
    case AFI_OP_BT: return op_Bt(c, x, y, false, true, s);
    case AFI_OP_PCHI: return op_Pchi(c, x, y, s);
    case AFI_OP_PU: return op_Pu(c, x, y, s);
    case AFI_OP_PA_INV: return c->exact ? exact_PA_inv(c, x, y, s) : fd_run(c, 0, x, y, s);
    case AFI_OP_SCHUR: return c->exact ? exact_schur(c, x, y, s) : schur_run(c, x, y, s);
    case AFI_OP_PS: return op_PS(c, x, y, s);
    case AFI_OP_PRECOND: return op_precond(c, x, y, s);
    case AFI_OP_SADDLE: return op_saddle(c, x, y, s);
    default: set_error("afi_apply: unknown operator"); return AFI_EINVAL;
  }
}

static long op_in_len(const afi_ctx *c, afi_operator op) {
  switch (op) {
    case AFI_OP_BT: case AFI_OP_PCHI: case AFI_OP_PS: return c->n_c;
    case AFI_OP_PRECOND: case AFI_OP_SADDLE: return c->n_dof + c->n_c;
    default: return c->n_dof;
  }
}

static long op_out_len(const afi_ctx *c, afi_operator op) {
  switch (op) {
    case AFI_OP_B: case AFI_OP_PCHI: case AFI_OP_PS: return c->n_c;
    case AFI_OP_PRECOND: case AFI_OP_SADDLE: return c->n_dof + c->n_c;
    default: return c->n_dof;
  }
}

afi_status afi_apply_batch(afi_ctx *c, afi_operator op, const double *x, double *y, int nrhs,
                           void *stream) {
  if (!c || !x || !y || nrhs < 1) { set_error("afi_apply_batch: invalid argument"); return AFI_EINVAL; }
  cudaStream_t s = as_stream(stream);
  const long ni = op_in_len(c, op), no = op_out_len(c, op);
  if (op == AFI_OP_STIFFNESS) {
    if (!has_operator(c)) return AFI_EINVAL;
    for (int j = 0; j < nrhs; j += kMaxRhs)
      AFI_TRY(op_stiffness_multi(c, x + (long long)j * ni, ni, y + (long long)j * no, no,
                                 std::min(kMaxRhs, nrhs - j), s));
    return AFI_OK;
  }
  if (op == AFI_OP_PA_INV && !c->exact) return fd_run(c, 0, x, y, s, nrhs);
  for (int j = 0; j < nrhs; ++j)
    AFI_TRY(afi_apply(c, op, x + (long long)j * ni, y + (long long)j * no, stream));
  return AFI_OK;
}

afi_status afi_set_precision(afi_ctx *c, afi_fd_precision prec) {
  if (!c || prec < AFI_FD_FP64 || prec > AFI_FD_BF16) { set_error("afi_set_precision: invalid"); return AFI_EINVAL; }
  c->opt.prec = prec;
  return AFI_OK;
}

afi_status afi_sizes(const afi_ctx *c, long *n_dof, long *n_c) {
  if (!c) { set_error("afi_sizes: null context"); return AFI_EINVAL; }
  if (n_dof) *n_dof = c->n_dof;
  if (n_c) *n_c = c->n_c;
  return AFI_OK;
}

afi_status afi_memory(const afi_ctx *c, long long *total, long long *stiff) {
  if (!c) { set_error("afi_memory: null context"); return AFI_EINVAL; }
  if (total) *total = c->bytes;
  if (stiff) *stiff = c->stencil_n * (long long)sizeof(double) * (c->stencil2 ? 2 : 1);
  return AFI_OK;
}

const char *afi_status_string(afi_status s) {
  switch (s) {
    case AFI_OK: return "ok";
    case AFI_EINVAL: return "invalid argument";
    case AFI_ENOMEM: return "out of device memory";
    case AFI_ECUDA: return "CUDA error";
    case AFI_ESINGULAR: return "singular or indefinite matrix";
    case AFI_ENOT_CONVERGED: return "not converged";
    case AFI_EBREAKDOWN: return "MINRES breakdown";
    case AFI_ETIMEOUT: return "timeout";
    default: return "unknown status";
  }
}

const char *afi_last_error(void) { return last_error_cstr(); }

long long afi_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
