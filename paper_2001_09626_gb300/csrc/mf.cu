// Matrix-free patch stiffness (eq. 3.1, the blocks A^(k) of Section 4) and
// mapped mass (eq. 4.8) by element-wise sum factorisation, for problems whose
// stored stiffness stencil would not fit in device memory
// (AFI_VARIANT_MATRIX_FREE).
//
// With Q = J^{-1}, wd = w |det J| at the problem's Gauss points (p + 1 per
// element and direction) and the parametric gradient Ghat[l][a] = d u_l /
// d eta_a,
//     grad u = Ghat Q,   sigma = mu (grad u + grad u^T) + lambda (div u) I,
//     (A^(k) u)_(l,i) = sum_q wd sum_a (sigma Q^T)[l][a] dB_i / d eta_a,
//     (M^(k) c)_(l,i) = sum_q wd c_l(q) B_i(q),
// which is the bilinear form of the stored stencil, integrated with the same
// rule.  J comes from the control points (isoparametric map, Section 2.2) in
// every application, so nothing per quadrature point is stored.
//
// One warp owns one element at a time (a grid-stride loop over all elements
// of all patches).  Six fields enter: the three coordinates of the element's
// (p+1)^3 control points and the three displacement components.  Three
// direction passes contract them to the Gauss points (the value and
// derivative tables of direction 1, then 2, then 3), the pointwise stress is
// formed in place, three transposed passes contract back to the element's
// nodes, and the results are added to y with atomics (neighbouring elements
// share nodes).  Each lane holds one direction's (p+1) x (p+1) value and
// derivative tables in registers during a pass and works through lines of
// p+1 entries, so every shared-memory operand feeds p+1 FMAs.
//
// FP64 form: FP64 throughout (the true residual and the plain form).  FP32
// form: the input converted once to FP32 and the results summed in FP32,
// then widened (the MINRES iterations, which refine against the FP64 true
// residual).
#include "common.cuh"

#include <algorithm>

namespace afi {

constexpr int kMfMaxWarps = 4;   // warps (elements in flight) per CTA

template <int P>
struct MfShape {
  static constexpr int NB = P + 1, NB2 = NB * NB, NB3 = NB2 * NB;
  static constexpr int TABS = 6 * NB2 + 3 * NB;   // V, D of each direction, then the weights
  static constexpr int REG = 18 * NB3;            // each of the two work regions
  static constexpr int PER_WARP = TABS + 2 * REG;
};

// one direction's tables into registers: v[g][t] = B_{e+t}(x_g), d = B'
template <typename T, int NB>
__device__ __forceinline__ void mf_tabs(const T *tb, int dir, T (&v)[NB][NB], T (&d)[NB][NB]) {
#pragma unroll
  for (int g = 0; g < NB; ++g)
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      v[g][t] = tb[(2 * dir) * NB * NB + g * NB + t];
      d[g][t] = tb[(2 * dir + 1) * NB * NB + g * NB + t];
    }
}

// patch and element coordinates of element ge (eoff[k] <= ge < eoff[k + 1])
template <int P>
__device__ __forceinline__ int mf_locate(const DevPatch *__restrict__ Pp,
                                         const long long *__restrict__ eoff, int npatch,
                                         long long ge, int (&e)[3]) {
  int lo = 0, hi = npatch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (eoff[mid] <= ge) lo = mid; else hi = mid - 1;
  }
  const int ne1 = Pp[lo].n[0] - P, ne2 = Pp[lo].n[1] - P;
  const long long le = ge - eoff[lo];
  e[0] = (int)(le % ne1);
  e[1] = (int)((le / ne1) % ne2);
  e[2] = (int)(le / ((long long)ne1 * ne2));
  return lo;
}

// one element's tables (tv, entries lane + 32 j of tb's layout) and fields
// (fv, entries lane + 32 j of [f][t3][t2][t1]: f = 0..2 control-point
// coordinates, 3..5 x) into registers
template <typename T, int P, int NT, int NF>
__device__ __forceinline__ void mf_fetch(const DevPatch &pt, const Tab1D *__restrict__ tabs,
                                         const T *__restrict__ pool, const T *__restrict__ ctrl,
                                         const T *__restrict__ x, const int (&e)[3], int lane,
                                         T (&tv)[NT], T (&fv)[NF]) {
  constexpr int NB = P + 1, NB2 = NB * NB, NB3 = NB2 * NB;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int i = lane + 32 * j;
    if (i < 6 * NB2) {
      const int dir = i / (2 * NB2), rem = i - dir * 2 * NB2, vd = rem / NB2, gt = rem - vd * NB2;
      const Tab1D &Tt = tabs[pt.tab[dir]];
      tv[j] = pool[(vd ? Tt.der : Tt.val) + (long long)e[dir] * NB2 + gt];
    } else if (i < 6 * NB2 + 3 * NB) {
      const int jj = i - 6 * NB2, dir = jj / NB, g = jj - dir * NB;
      tv[j] = pool[tabs[pt.tab[dir]].qw + (long long)e[dir] * NB + g];
    }
  }
  const int n1 = pt.n[0], n2 = pt.n[1];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const int i = lane + 32 * j;
    if (i < 6 * NB3) {
      const int f = i / NB3, r = i - f * NB3;
      const int t1 = r % NB, t2 = (r / NB) % NB, t3 = r / NB2;
      const long long node = (e[0] + t1) + (long long)n1 * ((e[1] + t2) + (long long)n2 * (e[2] + t3));
      fv[j] = f < 3 ? ctrl[pt.xoff + node * 3 + f] : x[pt.off + (long long)(f - 3) * pt.N + node];
    }
  }
}

// y += A x (MASS = false) or y += M x (MASS = true) over every element.
// pool, ctrl, x and y are in the arithmetic type T; eoff[k] is the first
// element of patch k (eoff[npatch] = ne).  *flag is set where det J <= 0.
// The FP32 form fetches the warp's next element into registers while it
// works on the current one (the element's global loads are otherwise
// waited on at every element); the FP64 form, bound by the FP64 pipe,
// fetches each element when it starts.
template <typename T, int P, bool MASS>
__global__ void __launch_bounds__(32 * kMfMaxWarps)
k_mf(const DevPatch *__restrict__ Pp, const Tab1D *__restrict__ tabs, const T *__restrict__ pool,
     const T *__restrict__ ctrl, const T *__restrict__ x, T *__restrict__ y,
     const long long *__restrict__ eoff, int npatch, long long ne, int *flag, const double *gate) {
  if (gate && *gate == 0.0) return;   // inactive MINRES iteration
  using S = MfShape<P>;
  constexpr int NB = S::NB, NB2 = S::NB2, NB3 = S::NB3;
  extern __shared__ __align__(16) unsigned char mf_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  T *tb = reinterpret_cast<T *>(mf_smem) + (size_t)wib * S::PER_WARP;
  T *R0 = tb + S::TABS, *R1 = R0 + S::REG;
  constexpr bool PF = sizeof(T) == 4;
  constexpr int NT = (6 * NB2 + 3 * NB + 31) / 32, NF = (6 * NB3 + 31) / 32;
  T tv[NT], fv[NF];
  const long long nw = (long long)gridDim.x * wpc;
  long long ge = (long long)blockIdx.x * wpc + wib;
  int en[3] = {0, 0, 0}, kn = 0;   // the fetched element
  if (PF && ge < ne) {
    kn = mf_locate<P>(Pp, eoff, npatch, ge, en);
    mf_fetch<T, P, NT, NF>(Pp[kn], tabs, pool, ctrl, x, en, lane, tv, fv);
  }
  for (; ge < ne; ge += nw) {
    if (!PF) {
      kn = mf_locate<P>(Pp, eoff, npatch, ge, en);
      mf_fetch<T, P, NT, NF>(Pp[kn], tabs, pool, ctrl, x, en, lane, tv, fv);
    }
    const DevPatch &pt = Pp[kn];
    const int n1 = pt.n[0], n2 = pt.n[1], N = pt.N;
    const int e[3] = {en[0], en[1], en[2]};
    // tables of the element: tb[(2 dir + vd) NB2 + g NB + t], weights at
    // 6 NB2; fields [f][t3][t2][t1] at R0
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (lane + 32 * j < 6 * NB2 + 3 * NB) tb[lane + 32 * j] = tv[j];
#pragma unroll
    for (int j = 0; j < NF; ++j)
      if (lane + 32 * j < 6 * NB3) R0[lane + 32 * j] = fv[j];
    __syncwarp();
    if (PF && ge + nw < ne) {   // the next element's loads run during this one
      kn = mf_locate<P>(Pp, eoff, npatch, ge + nw, en);
      mf_fetch<T, P, NT, NF>(Pp[kn], tabs, pool, ctrl, x, en, lane, tv, fv);
    }

    // pass 1 (direction 1): S1[f][vd][t3][t2][g1] at R0 + 6 NB3
    {
      T v[NB][NB], d[NB][NB];
      mf_tabs<T, NB>(tb, 0, v, d);
      for (int t = lane; t < 6 * NB2; t += 32) {
        const int f = t / NB2, r = t - f * NB2;
        const T *in = R0 + f * NB3 + r * NB;
        T a[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) a[j] = in[j];
        T *o = R0 + 6 * NB3 + 2 * f * NB3 + r * NB;
#pragma unroll
        for (int g = 0; g < NB; ++g) {
          T sv = 0, sd = 0;
#pragma unroll
          for (int j = 0; j < NB; ++j) { sv += v[g][j] * a[j]; sd += d[g][j] * a[j]; }
          o[g] = sv;
          o[NB3 + g] = sd;
        }
      }
    }
    __syncwarp();
    // pass 2 (direction 2): S2[f][k][t3][g2][g1] at R1, k = 0 vv, 1 vd, 2 dv
    {
      T v[NB][NB], d[NB][NB];
      mf_tabs<T, NB>(tb, 1, v, d);
      for (int t = lane; t < 6 * NB2; t += 32) {
        const int f = t / NB2, r = t - f * NB2, g1 = r % NB, t3 = r / NB;
        const T *in = R0 + 6 * NB3 + 2 * f * NB3 + g1 + NB2 * t3;
        T av[NB], ad[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) { av[j] = in[NB * j]; ad[j] = in[NB3 + NB * j]; }
        T *o = R1 + 3 * f * NB3 + g1 + NB2 * t3;
#pragma unroll
        for (int g = 0; g < NB; ++g) {
          T vv = 0, vd = 0, dv = 0;
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            vv += v[g][j] * av[j];
            vd += d[g][j] * av[j];
            dv += v[g][j] * ad[j];
          }
          o[NB * g] = vv;
          o[NB3 + NB * g] = vd;
          o[2 * NB3 + NB * g] = dv;
        }
      }
    }
    __syncwarp();
    // pass 3 (direction 3): OUT[f][a][g3][g2][g1] at R0, a = parametric
    // derivative direction (mass: the value of fields 3..5 in slot a = 0)
    {
      T v[NB][NB], d[NB][NB];
      mf_tabs<T, NB>(tb, 2, v, d);
      for (int t = lane; t < 6 * NB2; t += 32) {
        const int f = t / NB2, r = t - f * NB2;
        const T *in = R1 + 3 * f * NB3 + r;
        T avv[NB], avd[NB], adv[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          avv[j] = in[NB2 * j];
          avd[j] = in[NB3 + NB2 * j];
          adv[j] = in[2 * NB3 + NB2 * j];
        }
        T *o = R0 + 3 * f * NB3 + r;
        if (MASS && f >= 3) {
#pragma unroll
          for (int g = 0; g < NB; ++g) {
            T s0 = 0;
#pragma unroll
            for (int j = 0; j < NB; ++j) s0 += v[g][j] * avv[j];
            o[NB2 * g] = s0;
          }
        } else {
#pragma unroll
          for (int g = 0; g < NB; ++g) {
            T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
              s0 += v[g][j] * adv[j];
              s1 += v[g][j] * avd[j];
              s2 += d[g][j] * avv[j];
            }
            o[NB2 * g] = s0;
            o[NB3 + NB2 * g] = s1;
            o[2 * NB3 + NB2 * g] = s2;
          }
        }
      }
    }
    __syncwarp();
    // pointwise: J[x][a] = OUT[x][a], then the flux (sigma Q^T) wd (or wd c)
    // in place of the displacement gradients
    {
      const T *w = tb + 6 * NB2;
      for (int q = lane; q < NB3; q += 32) {
        const int g1 = q % NB, g2 = (q / NB) % NB, g3 = q / NB2;
        T J[3][3];
#pragma unroll
        for (int xx = 0; xx < 3; ++xx)
#pragma unroll
          for (int a = 0; a < 3; ++a) J[xx][a] = R0[(3 * xx + a) * NB3 + q];
        const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        if (!(det > T(0)) && flag) atomicExch(flag, 1);
        const T wd = w[g1] * w[NB + g2] * w[2 * NB + g3] * (det < T(0) ? -det : det);
        if (MASS) {
#pragma unroll
          for (int c = 0; c < 3; ++c) R0[(3 * (3 + c)) * NB3 + q] *= wd;
        } else {
          const T id = T(1) / det;
          T Q[3][3];   // Q[a][x] = (J^{-1})_{a x}
          Q[0][0] = c00 * id;
          Q[1][0] = c01 * id;
          Q[2][0] = c02 * id;
          Q[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
          Q[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
          Q[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
          Q[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
          Q[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
          Q[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
          T G[3][3];   // physical gradient G[l][x] = d u_l / d x_x
#pragma unroll
          for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int xx = 0; xx < 3; ++xx) {
              T s = 0;
#pragma unroll
              for (int a = 0; a < 3; ++a) s += R0[(3 * (3 + l) + a) * NB3 + q] * Q[a][xx];
              G[l][xx] = s;
            }
          const T lam_tr = T(pt.lam) * (G[0][0] + G[1][1] + G[2][2]);
          const T mu = T(pt.mu);
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            T sg[3];
#pragma unroll
            for (int xx = 0; xx < 3; ++xx) sg[xx] = mu * (G[l][xx] + G[xx][l]) + (l == xx ? lam_tr : T(0));
#pragma unroll
            for (int a = 0; a < 3; ++a)
              R0[(3 * (3 + l) + a) * NB3 + q] = wd * (sg[0] * Q[a][0] + sg[1] * Q[a][1] + sg[2] * Q[a][2]);
          }
        }
      }
    }
    __syncwarp();
    // back pass 3 (direction 3): R2[c][k][t3][g2][g1] at R1; k = 0 pairs with
    // the direction-1 derivative, 1 with direction 2, 2 with direction 3
    // (mass: slot 2 only)
    {
      T v[NB][NB], d[NB][NB];
      mf_tabs<T, NB>(tb, 2, v, d);
      for (int t = lane; t < 3 * NB2; t += 32) {
        const int c = t / NB2, r = t - c * NB2;
        const T *in = R0 + 3 * (3 + c) * NB3 + r;
        T *o = R1 + 3 * c * NB3 + r;
        if (MASS) {
          T a0[NB];
#pragma unroll
          for (int j = 0; j < NB; ++j) a0[j] = in[NB2 * j];
#pragma unroll
          for (int tt = 0; tt < NB; ++tt) {
            T s = 0;
#pragma unroll
            for (int g = 0; g < NB; ++g) s += v[g][tt] * a0[g];
            o[2 * NB3 + NB2 * tt] = s;
          }
        } else {
          T a0[NB], a1[NB], a2[NB];
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            a0[j] = in[NB2 * j];
            a1[j] = in[NB3 + NB2 * j];
            a2[j] = in[2 * NB3 + NB2 * j];
          }
#pragma unroll
          for (int tt = 0; tt < NB; ++tt) {
            T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
            for (int g = 0; g < NB; ++g) {
              s0 += v[g][tt] * a0[g];
              s1 += v[g][tt] * a1[g];
              s2 += d[g][tt] * a2[g];
            }
            o[NB2 * tt] = s0;
            o[NB3 + NB2 * tt] = s1;
            o[2 * NB3 + NB2 * tt] = s2;
          }
        }
      }
    }
    __syncwarp();
    // back pass 2 (direction 2): R1b[c][vd][t3][t2][g1] at R0; vd = 0 carries
    // the direction-1 derivative term, vd = 1 the rest
    {
      T v[NB][NB], d[NB][NB];
      mf_tabs<T, NB>(tb, 1, v, d);
      for (int t = lane; t < 3 * NB2; t += 32) {
        const int c = t / NB2, r = t - c * NB2, g1 = r % NB, t3 = r / NB;
        const T *in = R1 + 3 * c * NB3 + g1 + NB2 * t3;
        T *o = R0 + 2 * c * NB3 + g1 + NB2 * t3;
        T a0[NB], a1[NB], a2[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          a0[j] = MASS ? T(0) : in[NB * j];
          a1[j] = MASS ? T(0) : in[NB3 + NB * j];
          a2[j] = in[2 * NB3 + NB * j];
        }
#pragma unroll
        for (int tt = 0; tt < NB; ++tt) {
          T s0 = 0, s1 = 0;
#pragma unroll
          for (int g = 0; g < NB; ++g) {
            if (!MASS) {
              s0 += v[g][tt] * a0[g];
              s1 += d[g][tt] * a1[g];
            }
            s1 += v[g][tt] * a2[g];
          }
          o[NB * tt] = s0;
          o[NB3 + NB * tt] = s1;
        }
      }
    }
    __syncwarp();
    // back pass 1 (direction 1) and the scatter-add into y
    {
      T v[NB][NB], d[NB][NB];
      mf_tabs<T, NB>(tb, 0, v, d);
      for (int t = lane; t < 3 * NB2; t += 32) {
        const int c = t / NB2, r = t - c * NB2, t2 = r % NB, t3 = r / NB;
        const T *in = R0 + 2 * c * NB3 + NB * r;
        T ad[NB], av[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) { ad[j] = in[j]; av[j] = in[NB3 + j]; }
        T *yo = y + pt.off + (long long)c * N + e[0] +
                (long long)n1 * ((e[1] + t2) + (long long)n2 * (e[2] + t3));
#pragma unroll
        for (int tt = 0; tt < NB; ++tt) {
          T s = 0;
#pragma unroll
          for (int g = 0; g < NB; ++g) {
            if (!MASS) s += d[g][tt] * ad[g];
            s += v[g][tt] * av[g];
          }
          atomicAdd(yo + tt, s);
        }
      }
    }
    __syncwarp();   // R0 is reloaded for the next element
  }
}

// FP32 form: xf = x in FP32 and yf = 0; afterwards y = yf in FP64
__global__ void k_mf_pre(const double *__restrict__ x, float *__restrict__ xf,
                         float *__restrict__ yf, long n, const double *gate) {
  if (gate && *gate == 0.0) return;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    xf[i] = f64_to_f32(x[i]);
    yf[i] = 0.f;
  }
}
__global__ void k_mf_post(const float *__restrict__ yf, double *__restrict__ y, long n,
                          const double *gate) {
  if (gate && *gate == 0.0) return;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = f32_to_f64(yf[i]);
}
__global__ void k_mf_zero(double *__restrict__ y, long n, const double *gate) {
  if (gate && *gate == 0.0) return;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = 0.0;
}
// the float copy of the control points, each patch relative to its first
// control point (J is unchanged: the derivative tables sum to zero)
__global__ void k_mf_ctrl(const DevPatch *P, const double *ctrl, float *cf) {
  const DevPatch pt = P[blockIdx.y];
  const double *X = ctrl + pt.xoff;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3LL * pt.N;
       i += (long long)gridDim.x * blockDim.x)
    cf[pt.xoff + i] = f64_to_f32(X[i] - X[i % 3]);
}

namespace {

template <typename T> constexpr int prec_index() { return sizeof(T) == 8 ? 1 : 0; }

template <typename T, int P, bool MASS>
afi_status mf_config(afi_ctx *c) {
  const size_t per = (size_t)MfShape<P>::PER_WARP * sizeof(T);
  int wpc = (int)std::min<size_t>(kMfMaxWarps, (size_t)c->smem_optin / per);
  if (wpc < 1) { set_error("matrix-free stiffness: element work area exceeds shared memory"); return AFI_EINVAL; }
  const size_t smem = per * wpc;
  AFI_CUDA(cudaFuncSetAttribute(k_mf<T, P, MASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  AFI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mf<T, P, MASS>, 32 * wpc, smem));
  const long long need = (c->mf_ne + wpc - 1) / wpc;
  const int i = prec_index<T>() + 2 * (MASS ? 1 : 0);
  c->mf_wpc[i] = wpc;
  c->mf_smem[i] = (int)smem;
  c->mf_grid[i] = (int)std::max<long long>(1, std::min<long long>(need, (long long)c->nsm * std::max(occ, 1)));
  return AFI_OK;
}

template <typename T, int P, bool MASS>
void mf_launch(afi_ctx *c, const T *pool, const T *ctrl, const T *x, T *y, cudaStream_t s) {
  const int i = prec_index<T>() + 2 * (MASS ? 1 : 0);
  launch(k_mf<T, P, MASS>, c->mf_grid[i], 32 * c->mf_wpc[i], (size_t)c->mf_smem[i], s,
         (const DevPatch *)c->patches, (const Tab1D *)c->tabs, pool, ctrl, x, y,
         (const long long *)c->mf_eoff, c->npatch, c->mf_ne, c->dflag + 2, c->gate);
}

template <typename T, bool MASS>
afi_status mf_dispatch(afi_ctx *c, const T *pool, const T *ctrl, const T *x, T *y, cudaStream_t s,
                       bool config) {
  switch (c->mf_p) {
#define AFI_MF_CASE(PP)                                            \
    case PP:                                                       \
      if (config) return mf_config<T, PP, MASS>(c);                \
      mf_launch<T, PP, MASS>(c, pool, ctrl, x, y, s);              \
      break;
    AFI_MF_CASE(1)
    AFI_MF_CASE(2)
    AFI_MF_CASE(3)
    AFI_MF_CASE(4)
    AFI_MF_CASE(5)
#undef AFI_MF_CASE
    default:
      set_error("matrix-free stiffness: degree outside 1..5");
      return AFI_EINVAL;
  }
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

unsigned vec_blocks(const afi_ctx *c, long n) {
  return (unsigned)std::max<long>(1, std::min<long>((n + 255) / 256, (long)c->nsm * 8));
}

}  // namespace

afi_status mf_setup(afi_ctx *c) {
  if (c->dim != 3) { set_error("AFI_VARIANT_MATRIX_FREE needs a 3D problem"); return AFI_EINVAL; }
  const int p = c->hp[0].p;
  std::vector<long long> eoff(c->npatch + 1, 0);
  for (int k = 0; k < c->npatch; ++k) {
    const DevPatch &P = c->hp[k];
    if (P.p != p) { set_error("AFI_VARIANT_MATRIX_FREE needs one degree for every patch"); return AFI_EINVAL; }
    for (int d = 0; d < 3; ++d)
      if (c->htab[P.tab[d]].p != p || P.n[d] - p < 1) {
        set_error("AFI_VARIANT_MATRIX_FREE: inconsistent patch tables");
        return AFI_EINVAL;
      }
    eoff[k + 1] = eoff[k] + (long long)(P.n[0] - p) * (P.n[1] - p) * (P.n[2] - p);
  }
  if (p < 1 || p > 5) { set_error("AFI_VARIANT_MATRIX_FREE: degree outside 1..5"); return AFI_EINVAL; }
  c->mf = true;
  c->mf_p = p;
  c->mf_ne = eoff[c->npatch];
  long long nx = 0;
  for (auto &P : c->hp) nx = std::max(nx, P.xoff + 3LL * P.N);
  AFI_TRY(dalloc(c, (void **)&c->mf_eoff, eoff.size() * sizeof(long long)));
  AFI_CUDA(cudaMemcpy(c->mf_eoff, eoff.data(), eoff.size() * sizeof(long long), cudaMemcpyHostToDevice));
  AFI_TRY(dalloc(c, (void **)&c->mf_ctrlf, (size_t)nx * sizeof(float)));
  AFI_TRY(dalloc(c, (void **)&c->mf_xf, (size_t)c->n_dof * sizeof(float)));
  AFI_TRY(dalloc(c, (void **)&c->mf_yf, (size_t)c->n_dof * sizeof(float)));
  launch(k_mf_ctrl, dim3(64, c->npatch), 256, 0, 0, (const DevPatch *)c->patches,
         (const double *)c->ctrl, c->mf_ctrlf);
  AFI_LAUNCH_CHECK();
  AFI_TRY((mf_dispatch<float, false>(c, nullptr, nullptr, nullptr, nullptr, 0, true)));
  AFI_TRY((mf_dispatch<double, false>(c, nullptr, nullptr, nullptr, nullptr, 0, true)));
  AFI_TRY((mf_dispatch<double, true>(c, nullptr, nullptr, nullptr, nullptr, 0, true)));
  // geometry check: one FP32 application to zero flags det J <= 0
  AFI_CUDA(cudaMemset(c->dflag + 2, 0, sizeof(int)));
  AFI_CUDA(cudaMemset(c->mf_xf, 0, (size_t)c->n_dof * sizeof(float)));
  AFI_CUDA(cudaMemset(c->mf_yf, 0, (size_t)c->n_dof * sizeof(float)));
  const double *gate = c->gate;
  c->gate = nullptr;
  const afi_status st = mf_dispatch<float, false>(c, c->fpool, c->mf_ctrlf, c->mf_xf, c->mf_yf, 0, false);
  c->gate = gate;
  AFI_TRY(st);
  AFI_CUDA(cudaDeviceSynchronize());
  int h = 0;
  AFI_CUDA(cudaMemcpy(&h, c->dflag + 2, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) { set_error("geometry map has det J <= 0 at a quadrature point"); return AFI_EINVAL; }
  return AFI_OK;
}

afi_status mf_stiffness(afi_ctx *c, const double *x, double *y, bool exact, cudaStream_t s) {
  const long n = c->n_dof;
  if (exact) {
    launch(k_mf_zero, vec_blocks(c, n), 256, 0, s, y, n, c->gate);
    AFI_LAUNCH_CHECK();
    return mf_dispatch<double, false>(c, c->dpool, c->ctrl, x, y, s, false);
  }
  launch(k_mf_pre, vec_blocks(c, n), 256, 0, s, x, c->mf_xf, c->mf_yf, n, c->gate);
  AFI_LAUNCH_CHECK();
  AFI_TRY((mf_dispatch<float, false>(c, c->fpool, c->mf_ctrlf, c->mf_xf, c->mf_yf, s, false)));
  launch(k_mf_post, vec_blocks(c, n), 256, 0, s, (const float *)c->mf_yf, y, n, c->gate);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}

afi_status mf_mass(afi_ctx *c, const double *coef, double *f, cudaStream_t s) {
  const double *gate = c->gate;
  c->gate = nullptr;
  launch(k_mf_zero, vec_blocks(c, c->n_dof), 256, 0, s, f, c->n_dof, (const double *)nullptr);
  afi_status st = AFI_OK;
  if (cudaGetLastError() != cudaSuccess) { set_error("matrix-free mass: launch failed"); st = AFI_ECUDA; }
  if (st == AFI_OK) st = mf_dispatch<double, true>(c, c->dpool, c->ctrl, coef, f, s, false);
  c->gate = gate;
  return st;
}

}  // namespace afi
