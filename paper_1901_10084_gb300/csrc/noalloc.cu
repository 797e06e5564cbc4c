// cc_check_noalloc: the convergence check (largest metric-row violation and
// the objective sums) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they want this number:
// a host program whose device memory is already reserved in full by another
// allocator (a framework's memory pool, a fixed-budget plugin host), or a
// latency-critical loop where cudaMalloc/cudaFree may synchronize the whole
// device.  This entry point reads the caller's arrays, writes the caller's
// output array, and keeps its only scratch (one partial result per object) in
// a fixed array in the library's own device memory, so it allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ccdyk.h"

namespace {

// Six partial results per object: metric violation max, pair violation max,
// sum w|x-d|, sum w f, sum w (x^2 + f^2), sum d (y+ - y-).  Every GPU that
// loads the library holds this array (6 * CC_NOALLOC_MAX_N doubles) until
// the process exits.
constexpr int kParts = 6;
static __device__ __align__(256) double g_noalloc_scratch[kParts * CC_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

__host__ __device__ inline int64_t packed(int64_t n, int64_t i, int64_t j) {
  return i * n - i * (i + 1) / 2 + (j - i - 1);
}

__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA per object i: the violation of every triplet whose smallest index
// is i, and the pair terms of the pairs (i, j > i).  Writes the six partials
// of row i; the final step reads exactly the rows 0..n-1 written here.
__global__ void __launch_bounds__(256) k_noalloc_rows(int n, const double* __restrict__ x,
                                                     const double* __restrict__ f,
                                                     const double* __restrict__ d,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ yp, double* scratch) {
  const int i = blockIdx.x;
  __shared__ double red[kParts][8];
  double mv = 0.0, pv = 0.0, lp = 0.0, wf = 0.0, quad = 0.0, by = 0.0;
  const int64_t m = n - 1 - i;                   // objects j > i
  const int64_t pairs_jk = m * (m - 1) / 2;      // (j, k) with i < j < k
  for (int64_t q = threadIdx.x; q < pairs_jk; q += blockDim.x) {
    // q-th pair (j, k) of the objects i+1..n-1, row-major
    int64_t lo = 0, hi = m - 2;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (mid * m - mid * (mid + 1) / 2 <= q) lo = mid; else hi = mid - 1;
    }
    const int64_t j = i + 1 + lo;
    const int64_t k = j + 1 + (q - (lo * m - lo * (lo + 1) / 2));
    const double xij = x[packed(n, i, j)], xik = x[packed(n, i, k)], xjk = x[packed(n, j, k)];
    const double v0 = (xij - xik) - xjk, v1 = (xik - xij) - xjk, v2 = (xjk - xij) - xik;
    mv = fmax(mv, fmax(v0, fmax(v1, v2)));
  }
  for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
    const int64_t p = packed(n, i, j);
    const double xv = x[p], fv = f[p], dv = d[p], wv = w[p];
    lp += wv * fabs(xv - dv);
    wf += wv * fv;
    quad += wv * (xv * xv + fv * fv);
    by += dv * (yp[2 * p] - yp[2 * p + 1]);
    pv = fmax(pv, fmax(xv - fv - dv, dv - xv - fv));
  }
  mv = warp_max(mv);
  pv = warp_max(pv);
  lp = warp_sum(lp);
  wf = warp_sum(wf);
  quad = warp_sum(quad);
  by = warp_sum(by);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = mv;
    red[1][wid] = pv;
    red[2][wid] = lp;
    red[3][wid] = wf;
    red[4][wid] = quad;
    red[5][wid] = by;
  }
  __syncthreads();
  if (threadIdx.x < kParts) {
    const int r = threadIdx.x;
    const int nw = blockDim.x >> 5;
    double v = red[r][0];
    for (int t = 1; t < nw; ++t) v = (r < 2) ? fmax(v, red[r][t]) : v + red[r][t];
    scratch[(int64_t)r * CC_NOALLOC_MAX_N + i] = v;
  }
}

// Single CTA: fold the n row partials in a fixed order and write
// out[0..7] = {max_violation, pair_violation, lp_objective, wf, qp_primal,
//              dual_objective, gap, 0}.
__global__ void __launch_bounds__(256) k_noalloc_final(int n, double eps, const double* scratch, double* out) {
  __shared__ double red[kParts][8];
  double acc[kParts];
  for (int r = 0; r < kParts; ++r) acc[r] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int r = 0; r < kParts; ++r) {
      const double v = scratch[(int64_t)r * CC_NOALLOC_MAX_N + i];
      acc[r] = (r < 2) ? fmax(acc[r], v) : acc[r] + v;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = 0; r < kParts; ++r) {
    acc[r] = (r < 2) ? warp_max(acc[r]) : warp_sum(acc[r]);
    if (lane == 0) red[r][wid] = acc[r];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double v[kParts];
    for (int r = 0; r < kParts; ++r) {
      v[r] = red[r][0];
      for (int t = 1; t < nw; ++t) v[r] = (r < 2) ? fmax(v[r], red[r][t]) : v[r] + red[r][t];
    }
    const double qp = v[3] + 0.5 * eps * v[4];
    const double dual = -v[5] - 0.5 * eps * v[4];
    out[0] = v[0];
    out[1] = fmax(v[1], 0.0);
    out[2] = v[2];
    out[3] = v[3];
    out[4] = qp;
    out[5] = dual;
    out[6] = qp - dual;
    out[7] = 0.0;
  }
}

// Address of the scratch array on the current device, looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

// defined in ccdyk.cu: sets the message cc_last_error(NULL) returns
void ccd_set_global_error(const char* msg);

extern "C" int cc_check_noalloc(int64_t n, double eps, const double* x, const double* f, const double* d,
                                const double* w, const double* y_pair, double* out, void* stream) {
  if (!x || !f || !d || !w || !y_pair || !out) {
    ccd_set_global_error("cc_check_noalloc: NULL array");
    return CC_ERR_ARG;
  }
  if (n < 3) {
    ccd_set_global_error("cc_check_noalloc: n must be >= 3");
    return CC_ERR_ARG;
  }
  if (n > CC_NOALLOC_MAX_N) {
    ccd_set_global_error("cc_check_noalloc: n exceeds CC_NOALLOC_MAX_N (4096), the size of the "
                         "fixed scratch array; use cc_check on a handle instead");
    return CC_ERR_ARG;
  }
  if (!(eps > 0.0)) {
    ccd_set_global_error("cc_check_noalloc: eps must be > 0");
    return CC_ERR_ARG;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    ccd_set_global_error("cc_check_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return CC_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_noalloc_rows<<<(unsigned)n, 256, 0, st>>>((int)n, x, f, d, w, y_pair, scratch);
  k_noalloc_final<<<1, 256, 0, st>>>((int)n, eps, scratch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    ccd_set_global_error(cudaGetErrorString(e));
    return CC_ERR_CUDA;
  }
  return CC_OK;
}
