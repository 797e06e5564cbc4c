// Device building blocks shared by the sweep kernels: packed-pair and tile
// index arithmetic, the per-row Dykstra update (Algorithm 1) in a fused and in
// a row-by-row form, and a grid barrier whose wait is bounded in time.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ccdyk.h"

namespace ccd {

// ---------------------------------------------------------------- indices

__host__ __device__ __forceinline__ int64_t ch2(int64_t m) { return m < 2 ? 0 : m * (m - 1) / 2; }
__host__ __device__ __forceinline__ int64_t ch3(int64_t m) { return m < 3 ? 0 : m * (m - 1) * (m - 2) / 6; }

// lexicographic rank of i<j<k among the triplets of {0..n-1}
__host__ __device__ __forceinline__ int64_t tri_rank(int64_t n, int64_t i, int64_t j, int64_t k) {
  return (ch3(n) - ch3(n - i)) + (ch2(n - 1 - i) - ch2(n - j)) + (k - j - 1);
}

// inverse of tri_rank (binary searches on the two leading indices)
__host__ __device__ __forceinline__ void tri_unrank(int64_t n, int64_t r, int& i, int& j, int& k) {
  const int64_t T = ch3(n);
  int lo = 0, hi = (int)n - 3;                  // largest i with T - C3(n-i) <= r
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (T - ch3(n - mid) <= r) lo = mid; else hi = mid - 1;
  }
  i = lo;
  int64_t rem = r - (T - ch3(n - i));
  const int64_t base = ch2(n - 1 - i);
  lo = i + 1; hi = (int)n - 2;                  // largest j with base - C2(n-j) <= rem
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base - ch2(n - mid) <= rem) lo = mid; else hi = mid - 1;
  }
  j = lo;
  k = (int)(j + 1 + (rem - (base - ch2(n - j))));
}

// packed pair index p(i,j), i<j, row-major
__host__ __device__ __forceinline__ int64_t pair_index(int64_t n, int64_t i, int64_t j) {
  return i * n - i * (i + 1) / 2 + (j - i - 1);
}

// Tile (I,J), I<=J, of the B x B tiling of the strict upper triangle.
__host__ __device__ __forceinline__ int64_t tile_index(int64_t nb, int64_t I, int64_t J) {
  return I * nb - I * (I - 1) / 2 + (J - I);
}

// element offset of pair (i,j), i<j, in the tile-major layout
__host__ __device__ __forceinline__ int64_t tiled_offset(int64_t nb, int B, int64_t i, int64_t j) {
  int64_t I = i / B, J = j / B;
  return tile_index(nb, I, J) * (int64_t)B * B + (i % B) * B + (j % B);
}

// ---------------------------------------------------------------- loads

template <typename T>
__device__ __forceinline__ T ld_l2(const T* p) { return __ldcg(p); }    // skip L1: data written by other CTAs
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// ---------------------------------------------------------------- updates

// One metric row x_h - x_a - x_b <= 0 in fused form.  z is the scaled dual
// y/eps; r = 1 / (a^T W^{-1} a) = 1 / (w_h^-1 + w_a^-1 + w_b^-1).  Algebraically
// the correction, projection and dual update of Algorithm 1 collapse to:
//   z' = max(z + r (x_h - x_a - x_b), 0),  c = z - z',
//   x_h += c w_h^-1,  x_a -= c w_a^-1,  x_b -= c w_b^-1,  z = z'.
// v > 0 by an integer test of the sign and magnitude bits (for doubles this
// keeps the comparison off the FP64 unit): a non-NaN float or double is > 0
// exactly when its bit pattern, read as a signed integer, is > 0 (-0.0 reads
// as the most negative integer).
__device__ __forceinline__ bool positive(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool positive(float v) { return __float_as_int(v) > 0; }

template <typename T, bool UNITW>
__device__ __forceinline__ void metric_row_fused(T& xh, T& xa, T& xb, T wh, T wa, T wb, T r, T& z) {
  T d0 = (xh - xa) - xb;
  T zn = fma(d0, r, z);
  zn = positive(zn) ? zn : T(0);
  T c = z - zn;
  if (UNITW) {
    xh = xh + c;
    xa = xa - c;
    xb = xb - c;
  } else {
    xh = fma(c, wh, xh);
    xa = fma(-c, wa, xa);
    xb = fma(-c, wb, xb);
  }
  z = zn;
}

// The same row step by step as Algorithm 1 states it (correction, theta,
// projection, dual update), each operation rounded on its own; y is the dual
// of Algorithm 1 itself.
__device__ __forceinline__ void metric_row_exact(double& xh, double& xa, double& xb, double wh,
                                                 double wa, double wb, double eps, double& y) {
  double corr = __ddiv_rn(y, eps);
  xh = __dadd_rn(xh, __dmul_rn(corr, wh));
  xa = __dsub_rn(xa, __dmul_rn(corr, wa));
  xb = __dsub_rn(xb, __dmul_rn(corr, wb));
  double delta = __dsub_rn(__dsub_rn(xh, xa), xb);
  double aWa = __dadd_rn(__dadd_rn(wh, wa), wb);
  double theta = __ddiv_rn(__dmul_rn(eps, fmax(delta, 0.0)), aWa);
  double step = __ddiv_rn(theta, eps);
  xh = __dsub_rn(xh, __dmul_rn(step, wh));
  xa = __dadd_rn(xa, __dmul_rn(step, wa));
  xb = __dadd_rn(xb, __dmul_rn(step, wb));
  y = theta;
}

// The three rows of a triplet in the order hypotenuse = ij, ik, jk.
template <typename T, bool EXACT, bool UNITW>
__device__ __forceinline__ void triplet_rows(T& xij, T& xik, T& xjk, T wij, T wik, T wjk,
                                             T eps, T r_unit, T& z0, T& z1, T& z2) {
  if constexpr (EXACT) {
    metric_row_exact(xij, xik, xjk, wij, wik, wjk, eps, z0);
    metric_row_exact(xik, xij, xjk, wik, wij, wjk, eps, z1);
    metric_row_exact(xjk, xij, xik, wjk, wij, wik, eps, z2);
  } else {
    T r;
    if (UNITW) r = r_unit;
    else r = T(1) / ((wij + wik) + wjk);
    metric_row_fused<T, UNITW>(xij, xik, xjk, wij, wik, wjk, r, z0);
    metric_row_fused<T, UNITW>(xik, xij, xjk, wik, wij, wjk, r, z1);
    metric_row_fused<T, UNITW>(xjk, xij, xik, wjk, wij, wik, r, z2);
  }
}

// The two rows of a pair: x - f <= d, then d - x <= f.  a^T W^{-1} a = 2 w^-1.
template <typename T, bool EXACT>
__device__ __forceinline__ void pair_rows(T& x, T& f, T d, T wv, T eps, T& zp, T& zm) {
  if constexpr (EXACT) {
    double corr = __ddiv_rn(zp, eps);
    x = __dadd_rn(x, __dmul_rn(corr, wv));
    f = __dsub_rn(f, __dmul_rn(corr, wv));
    double delta = __dsub_rn(__dsub_rn(x, f), d);
    double theta = __ddiv_rn(__dmul_rn(eps, fmax(delta, 0.0)), __dadd_rn(wv, wv));
    double step = __ddiv_rn(theta, eps);
    x = __dsub_rn(x, __dmul_rn(step, wv));
    f = __dadd_rn(f, __dmul_rn(step, wv));
    zp = theta;
    corr = __ddiv_rn(zm, eps);
    x = __dsub_rn(x, __dmul_rn(corr, wv));
    f = __dsub_rn(f, __dmul_rn(corr, wv));
    delta = __dadd_rn(__dsub_rn(-x, f), d);
    theta = __ddiv_rn(__dmul_rn(eps, fmax(delta, 0.0)), __dadd_rn(wv, wv));
    step = __ddiv_rn(theta, eps);
    x = __dadd_rn(x, __dmul_rn(step, wv));
    f = __dadd_rn(f, __dmul_rn(step, wv));
    zm = theta;
  } else {
    T r = T(1) / (wv + wv);
    T d0 = (x - f) - d;                 // row +: a = (+1, -1), b = d
    T zn = fma(d0, r, zp);
    zn = positive(zn) ? zn : T(0);
    T c = zp - zn;
    x = fma(c, wv, x);
    f = fma(-c, wv, f);
    zp = zn;
    d0 = (d - x) - f;                   // row -: a = (-1, -1), b = -d
    zn = fma(d0, r, zm);
    zn = positive(zn) ? zn : T(0);
    c = zm - zn;
    x = fma(-c, wv, x);
    f = fma(-c, wv, f);
    zm = zn;
  }
}

// ---------------------------------------------------------------- barrier

struct Ctl {            // device control block (scratch)
  unsigned int arrive;  // grid-barrier arrivals of the running launch
  int err;              // first error code raised by any CTA
  int err_phase;        // phase at which the error was raised
  int pad;
};

// A block triple I <= J <= K of the tiled schedule, packed in 64 bits (21 bits
// per block index).
typedef unsigned long long btpk;
__host__ __device__ __forceinline__ btpk pack_bt(int I, int J, int K) {
  return (btpk)I | ((btpk)J << 21) | ((btpk)K << 42);
}

// Checked build (CCD_CHECKED): CCD_IN_BOUNDS(cond, ctl) records CC_ERR_BOUNDS
// in the control block when cond is false and returns cond, so the caller
// skips the access; in the normal build it is `true` and compiles away.
#ifdef CCD_CHECKED
__device__ __forceinline__ bool ccd_in_bounds(bool ok, Ctl* ctl) {
  if (!ok) atomicCAS(&ctl->err, 0, CC_ERR_BOUNDS);
  return ok;
}
#define CCD_IN_BOUNDS(cond, ctl) ccd_in_bounds((cond), (ctl))
#else
#define CCD_IN_BOUNDS(cond, ctl) true
#endif

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch.  The wait is bounded by
// timeout_ns; on expiry the CTA records CC_ERR_TIMEOUT and every CTA leaves.
// `skip` makes this CTA leave without arriving (fault injection for tests:
// the other CTAs then run into the time limit).  Returns false when the
// kernel must stop.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned target, long long timeout_ns,
                                             int phase, bool skip, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (skip) {
      ok = 0;
    } else {
      __threadfence();
      atomicAdd(&ctl->arrive, 1u);
      unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (true) {
        if (ld_acquire_u32(&ctl->arrive) >= target) break;
        if (ld_relaxed_s32(&ctl->err) != 0) { ok = 0; break; }
        if ((++spins & 63u) == 0 && (long long)(global_ns() - t0) > timeout_ns) {
          if (atomicCAS(&ctl->err, 0, CC_ERR_TIMEOUT) == 0) ctl->err_phase = phase;
          ok = 0;
          break;
        }
      }
      __threadfence();
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

}  // namespace ccd
