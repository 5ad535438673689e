// Allocation-free fast diagonalization for callers that cannot allocate
// device memory.
//
// Some callers may not call cudaMalloc at the point where they need the
// local solve: code recorded into a CUDA graph whose capture must not
// contain allocations, real-time loops that run on a fixed, pre-committed
// memory budget, or plug-ins whose host framework owns every device byte
// through its own allocator.  afi_fd_apply_static serves them: it runs the
// fast diagonalization on caller-provided eigen data and keeps its
// intermediate tensors in the file-scope array below, which the CUDA runtime
// creates when the library is loaded and every GPU that loads the library
// holds until the process exits.  The entry point itself calls no
// allocating routine.
#include "common.cuh"

#include <mutex>

namespace afi {

// Maximum scratch: 2^21 doubles = 16 MiB per device (two ping-pong tensors
// per block, so nblk * n1 * n2 * n3 <= 2^20).
constexpr long long kFdStaticMaxDoubles = 1LL << 21;

static __device__ __align__(256) double g_fd_static_scratch[kFdStaticMaxDoubles];

// dst[.., a, ..] = sum_i U[i][a] src[.., i, ..] (forward) or
// dst[.., i, ..] = sum_a U[i][a] src[.., a, ..] (back) along direction d.
__device__ __forceinline__ void fds_mode(const double *src, double *dst, const double *U, int n,
                                         int d, int n1, int n2, int n3, bool forward) {
  const int tot = n1 * n2 * n3;
  const int stride = (d == 0) ? 1 : (d == 1 ? n1 : n1 * n2);
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int io = (d == 0) ? idx % n1 : (d == 1 ? (idx / n1) % n2 : idx / (n1 * n2));
    const double *base = src + idx - io * stride;
    double acc = 0.0;
    if (forward)
      for (int j = 0; j < n; ++j) acc += U[j * n + io] * base[j * stride];
    else
      for (int j = 0; j < n; ++j) acc += U[io * n + j] * base[j * stride];
    dst[idx] = acc;
  }
}

// One block per tensor; the two ping-pong tensors of block b live at
// scratch + 2 b N.
__global__ void __launch_bounds__(256) k_fd_static(int n1, int n2, int n3, const double *U1,
                                                   const double *U2, const double *U3,
                                                   const double *D1, const double *D2,
                                                   const double *D3, double c1, double c2,
                                                   double c3, double shift, double scale,
                                                   int nd, const double *r, double *s,
                                                   double *scratch) {
  const int N = n1 * n2 * n3;
  const long long blk = blockIdx.x;
  double *cur = scratch + 2 * blk * N, *oth = cur + N;
  const double *in = r + blk * N;
  double *out = s + blk * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) cur[i] = in[i];
  __syncthreads();
  const double *U[3] = {U1, U2, U3};
  const int n[3] = {n1, n2, n3};
  for (int d = 0; d < nd; ++d) {
    fds_mode(cur, oth, U[d], n[d], d, n1, n2, n3, true);
    __syncthreads();
    double *t = cur; cur = oth; oth = t;
  }
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const int i1 = idx % n1, i2 = (idx / n1) % n2, i3 = idx / (n1 * n2);
    double lam = c1 * D1[i1] + c2 * D2[i2] + (nd == 3 ? c3 * D3[i3] : 0.0) + shift;
    cur[idx] /= scale * lam;
  }
  __syncthreads();
  for (int d = nd - 1; d >= 1; --d) {
    fds_mode(cur, oth, U[d], n[d], d, n1, n2, n3, false);
    __syncthreads();
    double *t = cur; cur = oth; oth = t;
  }
  fds_mode(cur, out, U1, n1, 0, n1, n2, n3, false);
}

// Device address of the scratch array, looked up once per device with that
// device current (the array's name is only a host-side stand-in in host code).
static afi_status static_scratch(double **out) {
  static std::mutex mu;
  static double *addr[128] = {nullptr};
  int dev = 0;
  AFI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) { set_error("device index out of range"); return AFI_EINVAL; }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fd_static_scratch);
    if (e != cudaSuccess) {
      set_error(std::string("cudaGetSymbolAddress(fd scratch): ") + cudaGetErrorString(e));
      return AFI_ECUDA;
    }
    addr[dev] = static_cast<double *>(p);
  }
  *out = addr[dev];
  return AFI_OK;
}

}  // namespace afi

using namespace afi;

extern "C" afi_status afi_fd_apply_static(int n1, int n2, int n3, const double *U1,
                                          const double *U2, const double *U3, const double *D1,
                                          const double *D2, const double *D3, const double coef[3],
                                          double shift, double scale, const double *r, double *s,
                                          int nblk, void *stream) {
  // three directions exactly when the third direction's eigen data is given
  const bool has3 = (U3 != nullptr) || (D3 != nullptr);
  if (n1 < 1 || n2 < 1 || n3 < 1 || nblk < 1 || !coef || !r || !s || !U1 || !U2 || !D1 || !D2 ||
      (has3 && (!U3 || !D3)) || (!has3 && n3 != 1)) {
    set_error("afi_fd_apply_static: invalid argument (3D data needs both U3 and D3; "
              "2D data needs n3 == 1)");
    return AFI_EINVAL;
  }
  // 2 * nblk * n1 * n2 * n3 <= kFdStaticMaxDoubles, checked factor by factor
  // so that no product can overflow
  long long room = kFdStaticMaxDoubles / 2;
  const long long f[4] = {n1, n2, n3, nblk};
  for (long long x : f) {
    if (x > room) {
      set_error("afi_fd_apply_static: 2 * nblk * n1 * n2 * n3 exceeds the static scratch of " +
                std::to_string(kFdStaticMaxDoubles) + " doubles");
      return AFI_EINVAL;
    }
    room /= x;
  }
  double *scratch = nullptr;
  AFI_TRY(static_scratch(&scratch));
  launch(k_fd_static, nblk, 256, 0, reinterpret_cast<cudaStream_t>(stream), n1, n2, n3, U1, U2,
         has3 ? U3 : U1, D1, D2, has3 ? D3 : D1, coef[0], coef[1], coef[2], shift, scale,
         has3 ? 3 : 2, r, s, scratch);
  AFI_LAUNCH_CHECK();
  return AFI_OK;
}
