// Schedules 0 and 1 on the GPU (Sec. III-B): one cooperative launch per
// sweep, a bounded grid barrier between phases, the pair rows after the last
// phase.  x, f, d and W^{-1} use the same tile-major layout as the tiled
// schedule; only the triangle phases and the dual store differ.
//
// Schedule 1 (phase s: triplets with (i+j+k) mod n = s): one thread per
// triplet.  Inside a phase the triplets are numbered in ascending (i, j); the
// first index of thread t comes from a per-phase prefix table over i (an
// n x (n+1) table, no triplet list), the middle index from the at most three
// runs of j with i+j+k = s, s+n, s+2n.  Duals: phase-major, 3 per triplet.
//
// Schedule 0 (the paper's diagonal schedule: the sets S_{i,k}, one phase per
// anti-diagonal i + k of the (i, k) grid): one thread
// per set; the set's triplets run serially in ascending j, carrying x_ik in a
// register.  Duals: set by set in schedule order, 3 per triplet.
#pragma once
#include "tiled.cuh"

namespace ccd {

struct ListArgs {
  int sched;             // 0 or 1
  int nphases;           // 2n-5 or n
  int B;                 // tile size of the x layout
  const int* pre1;       // schedule 1: (n+1) entries per phase
  const int64_t* phoff;  // schedule 1: triplet offsets of the phases (n+1);
                         // schedule 0: set offsets of the phases (nphases+1)
  const int* sets;       // schedule 0: sets in schedule order, packed i | k<<16
  const int64_t* setoff; // schedule 0: triplet offset of each set
  const int* setidx;     // schedule 0: set number of (i, k), n*n (for layout moves)
};

// floor((m - i - 1) / 2) for m - i - 1 >= -1
__device__ __forceinline__ int half_floor(int v) { return v >= 0 ? v / 2 : -1; }

// k-th triplet (thread t) of phase s of schedule 1
__device__ __forceinline__ void summod_decode(int n, int s, const int* pre, int64_t t, int& i, int& j, int& k) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  i = lo;
  int64_t rem = t - pre[i];
  j = k = -1;
  for (int q = 0; q < 3; ++q) {
    const int m = s + q * n;
    const int jlo = max(i + 1, m - i - n + 1), jhi = half_floor(m - i - 1);
    const int c = jhi - jlo + 1;
    if (c <= 0) continue;
    if (rem < c) {
      j = jlo + (int)rem;
      k = m - i - j;
      return;
    }
    rem -= c;
  }
}

// position of (i, j, k) inside its phase of schedule 1
__device__ __forceinline__ int64_t summod_position(int n, const int* pre1, int i, int j, int k, int& s) {
  const int m = i + j + k;
  s = m % n;
  const int* pre = pre1 + (int64_t)s * (n + 1);
  int64_t pos = pre[i];
  for (int q = 0; q < 3; ++q) {
    const int mm = s + q * n;
    const int jlo = max(i + 1, mm - i - n + 1), jhi = half_floor(mm - i - 1);
    if (mm == m) return pos + (j - jlo);
    pos += max(0, jhi - jlo + 1);
  }
  return pos;  // not reached for a valid triplet
}

template <typename T>
__device__ __forceinline__ T* xat(const TiledArgs<T>& a, int B, int i, int j) {
  return a.x + tiled_offset(a.nb, B, i, j);
}
template <typename T>
__device__ __forceinline__ T wat(const TiledArgs<T>& a, int B, int i, int j) {
  return a.winv[tiled_offset(a.nb, B, i, j)];
}

// pair rows of every pair, grid-stride (runtime tile size)
template <typename T, bool EXACT>
__device__ __forceinline__ void list_pair_phase(const TiledArgs<T>& a, int B) {
  const int BB = B * B;
  const int64_t total = (int64_t)a.ntiles * BB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int tl = (int)(e / BB), slot = (int)(e % BB);
    const int pk = a.tile_list[tl];
    const int I = pk & 0xffff, J = pk >> 16;
    const int la = slot / B, lb = slot % B;
    if (!((I < J || la < lb) && J * B + lb < a.n)) continue;
    T* zq = a.zp + (int64_t)tl * (2 * BB) + slot;
    T x = ld_l2(a.x + e), f = a.f[e];
    T zp = zq[0], zm = zq[BB];
    pair_rows<T, EXACT>(x, f, a.d[e], a.winv[e], a.eps, zp, zm);
    a.x[e] = x;
    a.f[e] = f;
    zq[0] = zp;
    zq[BB] = zm;
  }
}

template <typename T, bool EXACT, bool UNITW>
__device__ __forceinline__ void list_triplet(const TiledArgs<T>& a, int B, int i, int j, int k, T* z) {
  T* pij = xat(a, B, i, j);
  T* pik = xat(a, B, i, k);
  T* pjk = xat(a, B, j, k);
  T xij = ld_l2(pij), xik = ld_l2(pik), xjk = ld_l2(pjk);
  T vij = T(1), vik = T(1), vjk = T(1);
  if (!UNITW) {
    vij = wat(a, B, i, j);
    vik = wat(a, B, i, k);
    vjk = wat(a, B, j, k);
  }
  T z0 = z[0], z1 = z[1], z2 = z[2];
  triplet_rows<T, EXACT, UNITW>(xij, xik, xjk, vij, vik, vjk, a.eps, a.r_unit, z0, z1, z2);
  *pij = xij;
  *pik = xik;
  *pjk = xjk;
  z[0] = z0;
  z[1] = z1;
  z[2] = z2;
}

template <typename T, bool EXACT, bool UNITW>
__global__ void __launch_bounds__(256) k_sweep_summod(TiledArgs<T> a, ListArgs L) {
  __shared__ int s_flag;
  unsigned target = 0;
  const int n = a.n;
  for (int s = 0; s < n; ++s) {
    const int64_t cnt = L.phoff[s + 1] - L.phoff[s];
    const int* pre = L.pre1 + (int64_t)s * (n + 1);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
      int i, j, k;
      summod_decode(n, s, pre, t, i, j, k);
      list_triplet<T, EXACT, UNITW>(a, L.B, i, j, k, a.zt + 3 * (L.phoff[s] + t));
    }
    target += gridDim.x;
    const bool skip = (s == 0) && ((int)blockIdx.x == a.skip_cta);
    if (!grid_barrier(a.ctl, target, a.timeout_ns, s, skip, &s_flag)) return;
  }
  if (a.pairs) list_pair_phase<T, EXACT>(a, L.B);
}

template <typename T, bool EXACT, bool UNITW>
__global__ void __launch_bounds__(256) k_sweep_diagonal(TiledArgs<T> a, ListArgs L) {
  __shared__ int s_flag;
  unsigned target = 0;
  for (int p = 0; p < L.nphases; ++p) {
    for (int64_t c = L.phoff[p] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < L.phoff[p + 1];
         c += (int64_t)gridDim.x * blockDim.x) {
      const int pk = L.sets[c];
      const int i = pk & 0xffff, k = pk >> 16;
      T* z = a.zt + 3 * L.setoff[c];
      T* pik = xat(a, L.B, i, k);
      T xik = ld_l2(pik);
      const T vik = UNITW ? T(1) : wat(a, L.B, i, k);
      for (int j = i + 1; j < k; ++j, z += 3) {
        T* pij = xat(a, L.B, i, j);
        T* pjk = xat(a, L.B, j, k);
        T xij = ld_l2(pij), xjk = ld_l2(pjk);
        T vij = T(1), vjk = T(1);
        if (!UNITW) {
          vij = wat(a, L.B, i, j);
          vjk = wat(a, L.B, j, k);
        }
        T z0 = z[0], z1 = z[1], z2 = z[2];
        triplet_rows<T, EXACT, UNITW>(xij, xik, xjk, vij, vik, vjk, a.eps, a.r_unit, z0, z1, z2);
        *pij = xij;
        *pjk = xjk;
        z[0] = z0;
        z[1] = z1;
        z[2] = z2;
      }
      *pik = xik;
    }
    target += gridDim.x;
    const bool skip = (p == 0) && ((int)blockIdx.x == a.skip_cta);
    if (!grid_barrier(a.ctl, target, a.timeout_ns, p, skip, &s_flag)) return;
  }
  if (a.pairs) list_pair_phase<T, EXACT>(a, L.B);
}

// Triangle duals between the schedule-0/1 store and canonical order.
// dir 0: buf[3q + r] = scale * z;  dir 1: z = buf[3q + r] / scale.
template <typename T>
__global__ void k_tri_duals_list(T* zt, ListArgs L, int n, int64_t first, int64_t count, double* buf,
                                 double scale, int dir) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    tri_unrank(n, first + q, i, j, k);
    int64_t pos;
    if (L.sched == 1) {
      int s;
      const int64_t p = summod_position(n, L.pre1, i, j, k, s);
      pos = L.phoff[s] + p;
    } else {
      pos = L.setoff[L.setidx[(int64_t)i * n + k]] + (j - i - 1);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (dir == 0) buf[3 * q + r] = scale * (double)zt[3 * pos + r];
      else zt[3 * pos + r] = (T)(buf[3 * q + r] / scale);
    }
  }
}

}  // namespace ccd
