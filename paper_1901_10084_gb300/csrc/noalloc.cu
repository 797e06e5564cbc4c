// cc_check_noalloc: the convergence check (largest metric-row violation and
// the objective sums) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they want this number:
// a host program whose device memory is already reserved in full by another
// allocator (a framework's memory pool, a fixed-budget plugin host), or a
// latency-critical loop where cudaMalloc/cudaFree may synchronize the whole
// device.  This entry point reads the caller's arrays, writes the caller's
// output array, and keeps its only scratch (the partial results of at most
// CC_NOALLOC_MAX_N equal chunks of the work) in a fixed array in the
// library's own device memory, so it allocates nothing.  It serves the CC LP
// problem (metric rows, pair rows and the objectives of Eq. qp with
// c = (0, w)); l2 nearness handles report through cc_check.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "ccdyk.h"

namespace {

// Six partial results per chunk of work: metric violation max, pair violation
// max, sum w|x-d|, sum w f, sum w (x^2 + f^2), sum d (y+ - y-).  Every GPU
// that loads the library holds this array (6 * CC_NOALLOC_MAX_N doubles)
// until the process exits.  A call cuts its work into at most
// CC_NOALLOC_MAX_N chunks, one CTA each, and uses one column per chunk.
constexpr int kParts = 6;
constexpr int kSlots = CC_NOALLOC_MAX_N;
constexpr int kThreads = 256;
constexpr int64_t kMinTripletsPerChunk = 1 << 16;
static __device__ __align__(256) double g_noalloc_scratch[kParts * kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
  double* addr;
  unsigned long long ctx_id;   // context the address belongs to (0: unknown)
};
ScratchSlot g_scratch[kMaxDevices] = {};

__host__ __device__ inline int64_t packed(int64_t n, int64_t i, int64_t j) {
  return i * n - i * (i + 1) / 2 + (j - i - 1);
}
__host__ __device__ inline int64_t choose2(int64_t m) { return m < 2 ? 0 : m * (m - 1) / 2; }
__host__ __device__ inline int64_t choose3(int64_t m) { return m < 3 ? 0 : m * (m - 1) * (m - 2) / 6; }

// First triplet (i, j, k), i < j < k, of lexicographic rank r among the
// triplets of {0..n-1}: i is the largest index whose earlier first indices
// hold at most r triplets, j likewise inside i's block, then k.
__device__ inline void unrank_triplet(int64_t n, int64_t r, int64_t& i, int64_t& j, int64_t& k) {
  const int64_t T = choose3(n);
  int64_t lo = 0, hi = n - 3;
  while (lo < hi) {   // triplets with first index < i: T - C(n - i, 3)
    const int64_t mid = (lo + hi + 1) >> 1;
    if (T - choose3(n - mid) <= r) lo = mid; else hi = mid - 1;
  }
  i = lo;
  int64_t q = r - (T - choose3(n - i));
  const int64_t m = n - 1 - i;     // objects after i; pairs (j, k) among them
  lo = 0;
  hi = m - 2;
  while (lo < hi) {   // pairs with local first index < a: C(m, 2) - C(m - a, 2)
    const int64_t mid = (lo + hi + 1) >> 1;
    if (choose2(m) - choose2(m - mid) <= q) lo = mid; else hi = mid - 1;
  }
  j = i + 1 + lo;
  q -= choose2(m) - choose2(m - lo);
  k = j + 1 + q;
}

__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA b of `chunks`: the triplets of lexicographic ranks [b T / chunks,
// (b+1) T / chunks) and the pairs [b P / chunks, (b+1) P / chunks), so every
// CTA gets the same amount of work whatever n.  The triplets of a chunk form
// runs of consecutive k for fixed (i, j) (a row); the warps take the rows in
// turn and their lanes consecutive k, so the reads of x_ik and x_jk are
// contiguous.  Writes the six partials of column b; the final step reads
// exactly the columns 0..chunks-1 written by this launch.
__global__ void __launch_bounds__(kThreads) k_noalloc_chunks(int n, int chunks, const double* __restrict__ x,
                                                            const double* __restrict__ f,
                                                            const double* __restrict__ d,
                                                            const double* __restrict__ w,
                                                            const double* __restrict__ yp, double* scratch) {
  constexpr int NW = kThreads / 32;
  __shared__ double red[kParts][NW];
  __shared__ long long start[3];
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t T = choose3(n), P = choose2(n);
  const int64_t r0 = T * b / chunks, r1 = T * (b + 1) / chunks;
  if (threadIdx.x == 0 && r1 > r0) {
    int64_t i, j, k;
    unrank_triplet(n, r0, i, j, k);
    start[0] = i;
    start[1] = j;
    start[2] = k;
  }
  __syncthreads();
  double mv = 0.0, pv = 0.0, lp = 0.0, wf = 0.0, quad = 0.0, by = 0.0;
  if (r1 > r0) {
    int64_t i = start[0], j = start[1], k0 = start[2], left = r1 - r0;
    for (int64_t row = 0; left > 0; ++row) {
      const int64_t len = min(left, (int64_t)n - k0);   // k = k0 .. k0 + len - 1 of row (i, j)
      if (len <= 0) break;                               // not reached: r1 <= T
      if (row % NW == wid) {
        const double xij = x[packed(n, i, j)];
        const double* xi = x + packed(n, i, k0);   // x_ik for consecutive k are consecutive
        const double* xj = x + packed(n, j, k0);
        for (int64_t t = lane; t < len; t += 32) {
          const double xik = xi[t], xjk = xj[t];
          const double v0 = (xij - xik) - xjk, v1 = (xik - xij) - xjk, v2 = (xjk - xij) - xik;
          mv = fmax(mv, fmax(v0, fmax(v1, v2)));
        }
      }
      left -= len;
      if (++j == n - 1) {   // next row: (i, j + 1), or the first row of i + 1
        ++i;
        j = i + 1;
      }
      k0 = j + 1;
    }
  }
  for (int64_t p = P * b / chunks + threadIdx.x; p < P * (b + 1) / chunks; p += kThreads) {
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
    double v = red[r][0];
    for (int t = 1; t < NW; ++t) v = (r < 2) ? fmax(v, red[r][t]) : v + red[r][t];
    scratch[(int64_t)r * kSlots + b] = v;
  }
}

// Single CTA: fold the partials of the `chunks` columns in a fixed order and
// write out[0..7] = {max_violation, pair_violation, lp_objective, wf,
// qp_primal, dual_objective, gap, 0}.
__global__ void __launch_bounds__(kThreads) k_noalloc_final(int chunks, double eps, const double* scratch,
                                                           double* out) {
  constexpr int NW = kThreads / 32;
  __shared__ double red[kParts][NW];
  double acc[kParts];
  for (int r = 0; r < kParts; ++r) acc[r] = 0.0;
  for (int c = threadIdx.x; c < chunks; c += kThreads) {
    for (int r = 0; r < kParts; ++r) {
      const double v = scratch[(int64_t)r * kSlots + c];
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
    double v[kParts];
    for (int r = 0; r < kParts; ++r) {
      v[r] = red[r][0];
      for (int t = 1; t < NW; ++t) v[r] = (r < 2) ? fmax(v[r], red[r][t]) : v[r] + red[r][t];
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

// Identifier of the current context (cuCtxGetId through the runtime's driver
// entry-point lookup, so the library needs no link against the driver
// library); 0 when there is no current context or the driver lacks the call.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(p);
  });
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return 0;
  unsigned long long id = 0;
  return get_id(ctx, &id) == 0 ? id : 0;
}

// Address of the scratch array in the current device's context.  The set-up
// (cudaGetSymbolAddress, with the device current) runs on the first call on
// a device, and again only when that device's current context differs from
// the one the address was taken in (after cudaDeviceReset the module is
// loaded anew and the array may move).  Where the context cannot be
// identified the address is looked up on every call.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  ScratchSlot& slot = g_scratch[dev];
  const unsigned long long id = current_context_id();
  if (!slot.addr || id == 0 || id != slot.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    slot.addr = static_cast<double*>(p);
    slot.ctx_id = id ? id : current_context_id();   // the lookup made the primary context current
  }
  *out = slot.addr;
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
  const int64_t per = kMinTripletsPerChunk;
  const int chunks = (int)std::min<int64_t>(kSlots, std::max<int64_t>(1, (choose3(n) + per - 1) / per));
  k_noalloc_chunks<<<(unsigned)chunks, kThreads, 0, st>>>((int)n, chunks, x, f, d, w, y_pair, scratch);
  k_noalloc_final<<<1, kThreads, 0, st>>>(chunks, eps, scratch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    ccd_set_global_error(cudaGetErrorString(e));
    return CC_ERR_CUDA;
  }
  return CC_OK;
}
