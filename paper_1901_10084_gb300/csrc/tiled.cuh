// Tiled schedule: sweep, convergence-check and layout kernels.
//
// The index set is cut into blocks of B consecutive objects (Nb = ceil(n/B)
// blocks).  x, f, d and W^{-1} live in B x B tiles (I,J), I<=J, of the strict
// upper triangle, each tile contiguous (tile_index order), so that a CTA moves
// whole tiles between HBM/L2 and shared memory (the b x b tiles of Sec. III-C).
//
// A sweep is one cooperative launch.  Phase g = 0..Nb-1 holds the block triples
// I<=J<=K with (I+J+K) mod Nb = g; two of them share at most one block, so they
// touch disjoint tiles and run on different CTAs without locks (the two-triplet
// lemma of Sec. III-A lifted to blocks).  Inside a block triple the CTA walks
// sub-phases t = 0..B-1; sub-phase t holds the local offsets (a,b,c) with
// (a+b+c) mod B = t, and any two of those share at most one global index, so
// one sub-phase runs with one triplet per thread on tiles held in shared memory.
// A bounded grid barrier separates phases; the pair rows run after the last one.
//
// Triangle duals are stored in schedule order: block triple w (its rank in the
// concatenated phase lists) owns 3 B^3 slots, sub-phase-major, then row, then
// local slot a*B+b, so each thread's three duals of a sub-phase sit at a fixed
// stride and consecutive threads read consecutive words.
#pragma once
#include "common.cuh"

namespace ccd {

template <int B>
struct TileCfg {
  static constexpr int BB = B * B;
  static constexpr int NT = BB < 256 ? BB : 256;   // threads per CTA
  static constexpr int SPT = BB / NT;              // slots per thread and sub-phase
};

template <typename T>
struct TiledArgs {
  int n, nb, ntiles;
  T* x;                 // tile-major distances
  T* f;                 // tile-major slacks
  const T* d;           // tile-major dissimilarities
  const T* winv;        // tile-major 1/w
  T* zt;                // triangle duals, 3 B^3 per block triple
  T* zp;                // pair duals, 2 B^2 per tile (row +, row -)
  const btpk* bt_list;  // block triples in schedule order, packed by pack_bt
  const int* bt_off;    // nb+1 offsets of the phases in bt_list
  const int* tile_list; // tiles in tile_index order, packed I | J<<16
  Ctl* ctl;
  long long timeout_ns;
  T eps;                // eps of Eq. (qp)
  T r_unit;             // 1/3: 1/(a^T W^{-1} a) for unit weights
  int skip_cta;         // fault-injection hook (-1 = off)
  uint32_t* mask;       // nonzero-dual bits, same schedule order as zt (filtered form)
  int nbt;              // block triples per sweep
  unsigned long long* trace;  // optional per-item timestamps (nullptr = off)
  int* cnt;             // per-tile visit counters of this instance (batched sweep)
  int pairs;            // 1: the pair rows of the CC LP follow the metric rows; 0: l2 nearness
  int compact;          // FP64 CTA items: 1 = compacted update lists per sub-phase
  int nofilter;         // 1: update every triplet and row (reference for the filters)
  // sparse dual store (Sec. III-D): per block triple w, entries
  // [sp_off[w], sp_off[w] + sp_cnt[w]) of (local index, value), local index =
  // the dense offset inside the block triple's 3 B^3 slots, ascending; a sweep
  // reads the current pool and writes the next one (bump allocator sp_top)
  int sparse;
  const uint32_t* sp_idx;
  const T* sp_val;
  const long long* sp_off;
  const int* sp_cnt;
  uint32_t* sp_idx_next;
  T* sp_val_next;
  long long* sp_off_next;
  int* sp_cnt_next;
  unsigned long long* sp_top;
  long long sp_cap;     // entries the next pool holds
  T* sp_scratch;        // 3 B^3 values per CTA, all zero between items
  // buffer sizes, for the checked build's offset tests
  long long zt_elems, mask_words, sp_cap_cur, scratch_ctas;
};

__host__ __device__ __forceinline__ void unpack_bt(btpk pk, int& I, int& J, int& K) {
  I = (int)(pk & 0x1fffffull);
  J = (int)((pk >> 21) & 0x1fffffull);
  K = (int)(pk >> 42);
}

// Project every triplet of block triple number w (schedule rank).
template <typename T, bool EXACT, bool UNITW, int B>
__device__ __forceinline__ void tiled_block_triple(const TiledArgs<T>& a, int w, T* s0, T* s1,
                                                   T* s2, T* q0, T* q1, T* q2) {
  using C = TileCfg<B>;
  int I, J, K;
  unpack_bt(a.bt_list[w], I, J, K);
  const int64_t oIJ = tile_index(a.nb, I, J) * C::BB;
  const int64_t oIK = tile_index(a.nb, I, K) * C::BB;
  const int64_t oJK = tile_index(a.nb, J, K) * C::BB;
  const bool kj = (K == J), ij = (I == J);
  // tile (I,K) is tile (I,J) when K == J; tile (J,K) is tile (I,K) when I == J
  T* pIJ = s0;
  T* pIK = kj ? s0 : s1;
  T* pJK = ij ? pIK : s2;
  T* wIJ = q0;
  T* wIK = kj ? q0 : q1;
  T* wJK = ij ? wIK : q2;
  for (int e = threadIdx.x; e < C::BB; e += C::NT) {
    s0[e] = ld_l2(a.x + oIJ + e);
    if (!kj) s1[e] = ld_l2(a.x + oIK + e);
    if (!ij) s2[e] = ld_l2(a.x + oJK + e);
    if (!UNITW) {
      q0[e] = a.winv[oIJ + e];
      if (!kj) q1[e] = a.winv[oIK + e];
      if (!ij) q2[e] = a.winv[oJK + e];
    }
  }
  __syncthreads();
  T* zb = a.zt + (int64_t)w * (3 * B * C::BB);
  const int kB = K * B;
  for (int t = 0; t < B; ++t) {
    T* zs = zb + (int64_t)t * (3 * C::BB);
#pragma unroll
    for (int q = 0; q < C::SPT; ++q) {
      const int slot = threadIdx.x + q * C::NT;
      const int la = slot / B, lb = slot % B;
      const int lc = (t - la - lb) & (B - 1);
      const bool valid = (!ij || la < lb) && (!kj || lb < lc) && (kB + lc < a.n);
      if (valid) {
        T z0 = ld_stream(zs + slot);
        T z1 = ld_stream(zs + C::BB + slot);
        T z2 = ld_stream(zs + 2 * C::BB + slot);
        const int eij = la * B + lb, eik = la * B + lc, ejk = lb * B + lc;
        T xij = pIJ[eij], xik = pIK[eik], xjk = pJK[ejk];
        T vij = T(1), vik = T(1), vjk = T(1);
        if (!UNITW) {
          vij = wIJ[eij];
          vik = wIK[eik];
          vjk = wJK[ejk];
        }
        triplet_rows<T, EXACT, UNITW>(xij, xik, xjk, vij, vik, vjk, a.eps, a.r_unit, z0, z1, z2);
        pIJ[eij] = xij;
        pIK[eik] = xik;
        pJK[ejk] = xjk;
        st_stream(zs + slot, z0);
        st_stream(zs + C::BB + slot, z1);
        st_stream(zs + 2 * C::BB + slot, z2);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < C::BB; e += C::NT) {
    a.x[oIJ + e] = s0[e];
    if (!kj) a.x[oIK + e] = s1[e];
    if (!ij) a.x[oJK + e] = s2[e];
  }
  __syncthreads();
}

// The two rows of every pair (the last phase of a sweep).
template <typename T, bool EXACT, int B>
__device__ __forceinline__ void tiled_pair_phase(const TiledArgs<T>& a) {
  using C = TileCfg<B>;
  for (int tl = blockIdx.x; tl < a.ntiles; tl += gridDim.x) {
    const int pk = a.tile_list[tl];
    const int I = pk & 0xffff, J = pk >> 16;
    for (int slot = threadIdx.x; slot < C::BB; slot += C::NT) {
      const int la = slot / B, lb = slot % B;
      if ((I < J || la < lb) && J * B + lb < a.n) {
        const int64_t e = (int64_t)tl * C::BB + slot;
        T* zq = a.zp + (int64_t)tl * (2 * C::BB) + slot;
        T x = ld_l2(a.x + e), f = a.f[e];
        T zp = zq[0], zm = zq[C::BB];
        pair_rows<T, EXACT>(x, f, a.d[e], a.winv[e], a.eps, zp, zm);
        a.x[e] = x;
        a.f[e] = f;
        zq[0] = zp;
        zq[C::BB] = zm;
      }
    }
  }
}

template <typename T, bool EXACT, bool UNITW, int B>
__global__ void __launch_bounds__(TileCfg<B>::NT) k_sweep_tiled(TiledArgs<T> a) {
  using C = TileCfg<B>;
  __shared__ T sx[3][C::BB];
  __shared__ T sw[UNITW ? 1 : 3][C::BB];
  __shared__ int s_flag;
  unsigned target = 0;
  for (int g = 0; g < a.nb; ++g) {
    const int beg = a.bt_off[g], end = a.bt_off[g + 1];
    for (int w = beg + (int)blockIdx.x; w < end; w += gridDim.x)
      tiled_block_triple<T, EXACT, UNITW, B>(a, w, sx[0], sx[1], sx[2], sw[0], sw[UNITW ? 0 : 1],
                                             sw[UNITW ? 0 : 2]);
    target += gridDim.x;
    const bool skip = (g == 0) && ((int)blockIdx.x == a.skip_cta);
    if (!grid_barrier(a.ctl, target, a.timeout_ns, g, skip, &s_flag)) return;
  }
  if (a.pairs) tiled_pair_phase<T, EXACT, B>(a);
}

// ------------------------------------------------------------ filtered sweep
//
// Most metric rows are inactive at any time: their dual is zero and the row
// is satisfied (x_h - x_a - x_b <= 0), and then the fused update changes
// nothing (z' = max(0 + r*delta, 0) = 0, c = 0).  The filtered sweep proves a
// row inactive cheaply and skips it:
//   * a bit per row records whether its dual is nonzero (same schedule order
//     as the dual store; the store itself stays exact, zeros included), so
//     zero duals are never read from HBM;
//   * for FP64 state, a float copy of the x tiles in shared memory gives
//     delta_f = (x_h - x_a) - x_b in float; with S = |x_h| + |x_a| + |x_b|
//     (float), |delta_f - delta| <= 3.1 * 2^-24 * S (three conversions and two
//     additions rounded to nearest), so delta_f <= -(2^-21 S + 2^-100)
//     proves delta < 0 for the double evaluation as well;
//   * for FP32 state the test is the fused form's own delta <= 0.
// A triplet whose three rows are proved inactive is skipped; any other
// triplet runs the fused form unchanged, so the result equals the unfiltered
// sweep's in value.  Warps whose 32 triplets are all inactive skip the FP64
// work entirely (a warp vote).

// Float copy of a double for the filters: sign, exponent and the leading 23
// bits of the significand (truncated), built with integer operations only (a
// double-to-float conversion instruction would occupy the FP64 unit, which
// issues one warp instruction per 64 cycles).  |f - x| < 2^-23 |x| for
// 2^-126 <= |x| < 2^128; below, f = +-0 and |f - x| < 2^-126.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);      // biased double exponent
  if (e < 897) return __uint_as_float(sign);      // below 2^-126
  if (e > 1150) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m);
}

// All three rows of a triplet proved satisfied from float values.  The
// largest row delta is 2 max(x) - sum(x); evaluated in float from values
// within 2^-23 |x| of the doubles (f32_trunc; rounding to nearest is closer)
// or exact (FP32 state), it is within 11 * 2^-24 * S + 2^-123 of the exact
// one (S = |x_ij| + |x_ik| + |x_jk|; three conversions, two additions and one
// fused multiply-add), so dmax <= -(2^-20 S + 2^-100) proves every row delta
// < 0 with a margin far above the rounding of the double (or float) row
// evaluation itself.
__device__ __forceinline__ bool inactive_fast(float a, float b, float c) {
  const float sum = (a + b) + c;
  const float mx = fmaxf(fmaxf(a, b), c);
  const float dmax = fmaf(2.0f, mx, -sum);
  const float S = (fabsf(a) + fabsf(b)) + fabsf(c);
  return dmax <= -fmaf(S, 0x1p-20f, 0x1p-100f);
}

// Tests on dual values by their bit patterns (integer instructions; an FP64
// comparison would take 64 issue cycles of the FP64 unit).  Duals are never
// NaN; nz() treats -0.0 as zero like the value test, differs() compares bit
// patterns (a +-0 change would count as a change, and only costs a store).
__device__ __forceinline__ bool nz(double v) { return (__double_as_longlong(v) << 1) != 0; }
__device__ __forceinline__ bool nz(float v) { return (__float_as_int(v) << 1) != 0; }
__device__ __forceinline__ bool differs(double a, double b) { return __double_as_longlong(a) != __double_as_longlong(b); }
__device__ __forceinline__ bool differs(float a, float b) { return __float_as_int(a) != __float_as_int(b); }

__device__ __forceinline__ float to_shadow(double v) { return f32_trunc(v); }
__device__ __forceinline__ float to_shadow(float v) { return v; }

// One row (x_h against x_a, x_b) proved satisfied from float values: its
// delta (x_h - x_a) - x_b in float is within 10 * 2^-24 * S + 2^-123 of the
// exact one (three conversions as above, two additions), so the same test
// proves delta < 0; with a zero dual the fused row update is then a no-op.
__device__ __forceinline__ bool row_inactive(float h, float a, float b) {
  const float d = (h - a) - b;
  const float S = (fabsf(h) + fabsf(a)) + fabsf(b);
  return d <= -fmaf(S, 0x1p-20f, 0x1p-100f);
}

// The three rows of a triplet in FP64 state, skipping each row that is
// proved a no-op (zero dual, row satisfied in the float test above); the
// float copies follow every executed row.  Executing a skipped row would
// give z' = max(r * delta, 0) = 0 and c = 0, so the values equal those of
// triplet_rows; only the FP64 instructions of the skipped rows are saved
// (each costs 64 issue cycles of the warp whatever its active lanes).
template <bool UNITW>
__device__ __forceinline__ int triplet_rows_skip(double& xij, double& xik, double& xjk, float& fij, float& fik,
                                                  float& fjk, double vij, double vik, double vjk, double r,
                                                  double& z0, double& z1, double& z2, bool all = false) {
  int rows = 0;
  if (all || nz(z0) || !row_inactive(fij, fik, fjk)) {
    ++rows;
    metric_row_fused<double, UNITW>(xij, xik, xjk, vij, vik, vjk, r, z0);
    fij = f32_trunc(xij);
    fik = f32_trunc(xik);
    fjk = f32_trunc(xjk);
  }
  if (all || nz(z1) || !row_inactive(fik, fij, fjk)) {
    ++rows;
    metric_row_fused<double, UNITW>(xik, xij, xjk, vik, vij, vjk, r, z1);
    fij = f32_trunc(xij);
    fik = f32_trunc(xik);
    fjk = f32_trunc(xjk);
  }
  if (all || nz(z2) || !row_inactive(fjk, fij, fik)) {
    ++rows;
    metric_row_fused<double, UNITW>(xjk, xij, xik, vjk, vij, vik, r, z2);
    fij = f32_trunc(xij);
    fik = f32_trunc(xik);
    fjk = f32_trunc(xjk);
  }
  return rows;
}

template <int B>
struct MaskCfg {
  static constexpr int WPR = (B * B) / 32;          // mask words per row and sub-phase
  static constexpr int PER_BT = 3 * B * WPR;        // mask words per block triple
  static constexpr int CAP = 2 * B * B;             // nonzero duals staged per block triple
  static_assert((PER_BT * 4) % 16 == 0, "a block triple's bits are copied and prefetched in 16-byte units");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_ca(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared-memory layout of one CTA of the dataflow sweep (dynamic shared memory).
template <typename T, int B>
struct alignas(16) FlowSmem {
  static constexpr int BB = B * B;
  static constexpr int NSH = sizeof(T) == 8 ? 3 : 1;
  T x[3][BB];
  float f[NSH][BB];
  uint32_t mask[MaskCfg<B>::PER_BT];
  int pre[MaskCfg<B>::PER_BT];
  T dual[MaskCfg<B>::CAP];
  T lz[3][BB];              // compacted list of a sub-phase: current duals
  int lslot[BB];            //   and slots of the triplets to update
  int lcnt[B];              // list length per sub-phase
  int scan[32];
  int item, flag, total, dirty;
  int ready;                // the item's tiles were ready at the first look
  int t0;                   // first sub-phase with an update (items without nonzero duals)
  uint32_t nmask[MaskCfg<B>::PER_BT];   // sparse store: nonzero-dual bits after the item
  unsigned long long base;              //   and its place in the next pool
  int ntrip, nrows, nsub;   // trace counters: triplets updated, rows executed, sub-phases with updates
  unsigned subbits;         //   sub-phases with updates (per-warp form)
};

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait (thread 0) until each listed tile has been visited `need` times: the
// (up to three) counters are polled together with relaxed loads, then an
// acquire fence orders the item's reads after the visits it waited for.
// Bounded in time; on expiry records CC_ERR_TIMEOUT.  Returns false when the
// kernel must stop.
__device__ __forceinline__ bool wait_tiles(const int* cnt, int64_t t0, int64_t t1, int64_t t2, int need,
                                           Ctl* ctl, long long timeout_ns, int tag) {
  unsigned long long start = 0;
  unsigned spins = 0;
  while (true) {
    const int c0 = ld_relaxed_i32(cnt + t0);
    const int c1 = t1 >= 0 ? ld_relaxed_i32(cnt + t1) : need;
    const int c2 = t2 >= 0 ? ld_relaxed_i32(cnt + t2) : need;
    if (c0 >= need && c1 >= need && c2 >= need) break;
    if (ld_relaxed_s32(&ctl->err) != 0) return false;
    if (start == 0) start = global_ns();
    if ((++spins & 15u) == 0 && (long long)(global_ns() - start) > timeout_ns) {
      if (atomicCAS(&ctl->err, 0, CC_ERR_TIMEOUT) == 0) ctl->err_phase = tag;
      return false;
    }
    if (spins > 4) __nanosleep(64);
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return true;
}

// One look at the tile counters (thread 0): true when every listed tile has
// been visited `need` times.
__device__ __forceinline__ bool tiles_ready(const int* cnt, int64_t t0, int64_t t1, int64_t t2, int need) {
  const int c0 = ld_relaxed_i32(cnt + t0);
  const int c1 = t1 >= 0 ? ld_relaxed_i32(cnt + t1) : need;
  const int c2 = t2 >= 0 ? ld_relaxed_i32(cnt + t2) : need;
  return c0 >= need && c1 >= need && c2 >= need;
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Bring `bytes` (a multiple of 16, 16-byte aligned) into L2 without waiting.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// While an item waits for its tiles, bring into L2 what its staging will read
// from HBM: the nonzero-dual bits of block triple w and the 128-byte lines
// that hold its nonzero duals (dense store), or its entry list (sparse
// store).  Threads t0, t0 + nt, ... share the work.  Prefetches only: no value
// is kept, and the item's own writes come after its wait, so the staging
// reads what it reads without them.
template <typename T, int B>
__device__ __forceinline__ void warm_item(const TiledArgs<T>& a, int w, int t0, int nt) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  if (a.sparse) {
    const int cnt = a.sp_cnt[w];
    const long long off = a.sp_off[w];
    if (cnt <= 0 || off < 0 || off + cnt > a.sp_cap_cur) return;
    constexpr long long IL = 128 / sizeof(uint32_t), VL = 128 / sizeof(T);   // entries per line
    for (long long l = off / IL + t0; l <= (off + cnt - 1) / IL; l += nt) prefetch_l2(a.sp_idx + l * IL);
    for (long long l = off / VL + t0; l <= (off + cnt - 1) / VL; l += nt) prefetch_l2(a.sp_val + l * VL);
    return;
  }
  if ((long long)(w + 1) * M::PER_BT > a.mask_words || (long long)(w + 1) * (3 * B * C::BB) > a.zt_elems) return;
  const uint32_t* mb = a.mask + (int64_t)w * M::PER_BT;
  const T* zb = a.zt + (int64_t)w * (3 * B * C::BB);
  for (int q = t0; q < M::PER_BT; q += nt) {
    const uint32_t bits = __ldcg(mb + q);
    if (!bits) continue;
    // word q holds the bits of 32 consecutive duals (sub-phase t, row r, word wd)
    const int t = q / (3 * M::WPR), r = (q / M::WPR) % 3, wd = q % M::WPR;
    const T* src = zb + (int64_t)t * (3 * C::BB) + r * C::BB + wd * 32;
    if constexpr (sizeof(T) == 8) {
      if (bits & 0xffffu) prefetch_l2(src);
      if (bits >> 16) prefetch_l2(src + 16);
    } else {
      prefetch_l2(src);
    }
  }
}

// Release (thread 0, after a CTA barrier): make the item's writes visible at
// GPU scope, then count one visit on each of its tiles.
__device__ __forceinline__ void release_tiles(int* cnt, int64_t t0, int64_t t1, int64_t t2) {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  atomicAdd(cnt + t0, 1);
  if (t1 >= 0) atomicAdd(cnt + t1, 1);
  if (t2 >= 0) atomicAdd(cnt + t2, 1);
}

template <bool WARP>
__device__ __forceinline__ void item_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

// Barrier of the NTHG threads staging an item: the whole item group
// (CTA or warp), or, with NAMED, warps 1.. of the CTA on named barrier 1
// while warp 0 waits for the item's tiles.
template <int NTHG, bool NAMED>
__device__ __forceinline__ void group_sync() {
  if constexpr (NAMED) asm volatile("bar.sync 1, %0;" ::"n"(NTHG) : "memory");
  else item_sync<NTHG == 32>();
}

// The item's staging plan from its nonzero-dual bits (sm.mask, loaded):
// exclusive prefix of the word popcounts (the staging slot of every nonzero
// dual, sm.pre), the count (sm.total) and, when they fit, asynchronous copies
// of the nonzero duals of the dense store into sm.dual (or, for the sparse
// store, the starting copy of the item's new bits).  Run by the NTHG threads
// of a group, thread gtid; returns the count.  The dual copies are in flight
// on return.
template <typename T, int B, int NTHG, bool NAMED>
__device__ __forceinline__ int stage_duals(const TiledArgs<T>& a, FlowSmem<T, B>& sm, const T* zb, int gtid) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  constexpr int NWG = NTHG / 32;
  constexpr int CH = (M::PER_BT + NTHG - 1) / NTHG;
  const int lane = gtid & 31, gw = gtid >> 5;
  int cnt = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int q = gtid * CH + c;
    if (q < M::PER_BT) cnt += __popc(sm.mask[q]);
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) sm.scan[gw] = incl;
  group_sync<NTHG, NAMED>();
  if (gw == 0) {
    int v = lane < NWG ? sm.scan[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < NWG) sm.scan[lane] = v;
  }
  group_sync<NTHG, NAMED>();
  int run = (gw ? sm.scan[gw - 1] : 0) + incl - cnt;
  const int total = sm.scan[NWG - 1];
  if (gtid == 0) sm.total = total;
  const bool staged = total <= M::CAP;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int q = gtid * CH + c;
    if (q < M::PER_BT) {
      uint32_t bits = sm.mask[q];
      sm.pre[q] = run;
      if (a.sparse) sm.nmask[q] = bits;
      if (staged && bits && !a.sparse) {
        const int t = q / (3 * M::WPR), r = (q / M::WPR) % 3, wd = q % M::WPR;
        const T* src = zb + (int64_t)t * (3 * C::BB) + r * C::BB + wd * 32;
        int idx = run;
        while (bits) {
          const int l = __ffs(bits) - 1;
          bits &= bits - 1;
          cp_async_ca<sizeof(T)>(&sm.dual[idx++], src + l);
        }
      }
      run += __popc(sm.mask[q]);
    }
  }
  return total;
}

// While warp 0 waits for block triple w's tiles, warps 1.. stage what the
// item owns alone (its nonzero-dual bits, their prefix and its nonzero duals
// of the dense store: written only by this item's visit of the previous
// sweep), so that after the wait only the x tiles remain to be loaded.
// Returns with the dual copies complete for the calling thread; a CTA
// barrier must follow before other threads read them.
template <typename T, int B, int NT>
__device__ __noinline__ void prestage_item(const TiledArgs<T>& a, int w, FlowSmem<T, B>& sm) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  constexpr int NTHG = NT - 32;
  const int gtid = (int)threadIdx.x - 32;
  const uint32_t* mb = a.mask + (int64_t)w * M::PER_BT;
  const T* zb = a.zt + (int64_t)w * (3 * B * C::BB);
  constexpr int MCH = M::PER_BT * 4 / 16;
  for (int e = gtid; e < MCH; e += NTHG)
    cp_async16(reinterpret_cast<char*>(sm.mask) + 16 * e, reinterpret_cast<const char*>(mb) + 16 * e);
  cp_async_wait_all();
  group_sync<NTHG, true>();
  stage_duals<T, B, NTHG, true>(a, sm, zb, gtid);
  cp_async_wait_all();
}

// The B sub-phases of one staged block triple.  FULL: I < J < K and no
// ragged block, so every slot is a triplet and the thread owns its x_ij
// (tile (I,J) entry (a,b) is touched only by slot (a,b)): x_ij and its float
// value stay in registers for the whole item.  HASMASK = false: the item has
// no nonzero dual, so no mask word is read.  Returns whether this thread
// updated anything.
template <typename T, bool UNITW, int B, int NTH_, bool FULL, bool HASMASK>
__device__ __forceinline__ int flow_subphases(const TiledArgs<T>& a, int w, FlowSmem<T, B>& sm, T* pIJ, T* pIK,
                                              T* pJK, float* gIJ, float* gIK, float* gJK, int64_t oIJ,
                                              int64_t oIK, int64_t oJK, bool ij, bool kj, int kB, bool staged,
                                              int tid, int lane, T* zb) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  constexpr bool SHADOW = sizeof(T) == 8;
  constexpr bool WARP = NTH_ == 32;
  constexpr int NTH = NTH_;
  constexpr int SPT = C::BB / NTH;
  const uint32_t below = (1u << lane) - 1u;
  int la[SPT], lb[SPT];
  T xr[SPT];
  float fr[SPT];
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    const int slot = tid + q * NTH;
    la[q] = slot / B;
    lb[q] = slot % B;
    if constexpr (FULL) {
      xr[q] = pIJ[slot];
      fr[q] = gIJ[slot];
    }
  }
  int touched = 0;
  int t_start = 0;
  if constexpr (FULL && !HASMASK) {
    // no nonzero dual: until the first sub-phase in which some triplet
    // fails the filter nothing changes, so that sub-phase is found from the
    // staged tiles in one pass without barriers, and the walk starts there
    // (an item with no such sub-phase changes nothing at all)
    if (!a.nofilter) {
      // a thread stops at the first sub-phase it needs, or at one that some
      // thread already found to need an update (the minimum only falls, and
      // a thread stopping at t saw no need before t, so the minimum found is
      // the first sub-phase with any need)
      int first = B;
      volatile int* t0v = &sm.t0;
      for (int t = 0; t < B && first == B && t < *t0v; ++t) {
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
          const int lc = (t - la[q] - lb[q]) & (B - 1);
          if (!inactive_fast(fr[q], gIK[la[q] * B + lc], gJK[lb[q] * B + lc])) first = t;
        }
      }
      if (first < B) atomicMin(&sm.t0, first);
      item_sync<WARP>();
      t_start = sm.t0;
    }
  }
  for (int t = t_start; t < B; ++t) {
    T* zs = zb + (int64_t)t * (3 * C::BB);
    const int qt = t * (3 * M::WPR);
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      const int slot = tid + q * NTH;
      const int lc = (t - la[q] - lb[q]) & (B - 1);
      const int eij = slot, eik = la[q] * B + lc, ejk = lb[q] * B + lc;
      bool valid = true;
      if constexpr (!FULL) valid = (!ij || la[q] < lb[q]) && (!kj || lb[q] < lc) && (kB + lc < a.n);
      const int wd = slot >> 5;
      const int q0 = qt + wd, q1 = qt + M::WPR + wd, q2 = qt + 2 * M::WPR + wd;
      uint32_t m0 = 0u, m1 = 0u, m2 = 0u;
      if constexpr (HASMASK) {
        m0 = sm.mask[q0];
        m1 = sm.mask[q1];
        m2 = sm.mask[q2];
      }
      const bool b0 = (m0 >> lane) & 1u, b1 = (m1 >> lane) & 1u, b2 = (m2 >> lane) & 1u;
      bool need = false;
      if (valid) {
        const float fij = FULL ? fr[q] : gIJ[eij];
        need = a.nofilter || (b0 | b1 | b2) || !inactive_fast(fij, gIK[eik], gJK[ejk]);
      }
      if (__any_sync(0xffffffffu, need)) {
        if (a.trace && lane == 0) atomicOr(&sm.subbits, 1u << t);
        T z0 = T(0), z1 = T(0), z2 = T(0);
        if (need) {
          if (staged) {
            if (b0) z0 = sm.dual[sm.pre[q0] + __popc(m0 & below)];
            if (b1) z1 = sm.dual[sm.pre[q1] + __popc(m1 & below)];
            if (b2) z2 = sm.dual[sm.pre[q2] + __popc(m2 & below)];
          } else {
            if (b0) z0 = ld_stream(zs + slot);
            if (b1) z1 = ld_stream(zs + C::BB + slot);
            if (b2) z2 = ld_stream(zs + 2 * C::BB + slot);
          }
          const T o0 = z0, o1 = z1, o2 = z2;
          T xij = FULL ? xr[q] : pIJ[eij];
          T xik = pIK[eik], xjk = pJK[ejk];
          T vij = T(1), vik = T(1), vjk = T(1);
          if (!UNITW) {
            vij = a.winv[oIJ + eij];
            vik = a.winv[oIK + eik];
            vjk = a.winv[oJK + ejk];
          }
          if constexpr (SHADOW) {
            float fij = FULL ? fr[q] : gIJ[eij], fik = gIK[eik], fjk = gJK[ejk];
            const T r = UNITW ? a.r_unit : T(1) / ((vij + vik) + vjk);
            const int rows = triplet_rows_skip<UNITW>(xij, xik, xjk, fij, fik, fjk, vij, vik, vjk, r, z0, z1, z2,
                                                     a.nofilter != 0);
            if (a.trace) {
              atomicAdd(&sm.ntrip, 1);
              atomicAdd(&sm.nrows, rows);
            }
            if constexpr (FULL) fr[q] = fij;
            else gIJ[eij] = fij;
            gIK[eik] = fik;
            gJK[ejk] = fjk;
          } else {
            triplet_rows<T, false, UNITW>(xij, xik, xjk, vij, vik, vjk, a.eps, a.r_unit, z0, z1, z2);
            if constexpr (FULL) fr[q] = xij;   // FP32 state: the filter reads x_ij itself
          }
          if constexpr (FULL) xr[q] = xij;
          else pIJ[eij] = xij;
          pIK[eik] = xik;
          pJK[ejk] = xjk;
          if (differs(z0, o0)) st_stream(zs + slot, z0);
          if (differs(z1, o1)) st_stream(zs + C::BB + slot, z1);
          if (differs(z2, o2)) st_stream(zs + 2 * C::BB + slot, z2);
          // a dual that became zero or nonzero flips its bit in the item's
          // shared-memory mask, written back once at the end of the item
          // (the words of sub-phase t belong to one warp and are read only
          // at the top of sub-phase t, before any flip)
          uint32_t* mw = a.sparse ? sm.nmask : sm.mask;
          const uint32_t bit = 1u << lane;
          const bool f0 = nz(z0) != b0, f1 = nz(z1) != b1, f2 = nz(z2) != b2;
          if (f0) atomicXor(&mw[q0], bit);
          if (f1) atomicXor(&mw[q1], bit);
          if (f2) atomicXor(&mw[q2], bit);
          if ((f0 | f1 | f2) && !a.sparse) sm.dirty = 1;
          touched = 1;
        }
      }
    }
    item_sync<WARP>();
  }
  if constexpr (FULL) {
#pragma unroll
    for (int q = 0; q < SPT; ++q) pIJ[tid + q * NTH] = xr[q];
  }
  return touched;
}

// The B sub-phases with compaction (CTA per item).  A filter pass lists, in
// shared memory, the triplets of the sub-phase that need the update together
// with their current duals; the first threads of the CTA then process the
// list, so the FP64 work of a sub-phase occupies as few warps as possible
// (the triplets of a sub-phase are independent, so which thread handles which
// triplet does not change the result).  Mask bits are updated in shared
// memory and written back once per item.  FULL / HASMASK as above.
template <typename T, bool UNITW, int B, int NTH_, bool FULL, bool HASMASK>
__device__ __forceinline__ int flow_subphases_compact(const TiledArgs<T>& a, FlowSmem<T, B>& sm, T* pIJ, T* pIK,
                                                      T* pJK, float* gIJ, float* gIK, float* gJK, int64_t oIJ,
                                                      int64_t oIK, int64_t oJK, bool ij, bool kj, int kB,
                                                      bool staged, int tid, int lane, T* zb) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  constexpr bool SHADOW = sizeof(T) == 8;
  constexpr bool WARP = NTH_ == 32;
  constexpr int NTH = NTH_;
  constexpr int SPT = C::BB / NTH;
  const uint32_t below = (1u << lane) - 1u;
  int touched = 0;
  for (int t = 0; t < B; ++t) {
    T* zs = zb + (int64_t)t * (3 * C::BB);
    const int qt = t * (3 * M::WPR);
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      const int slot = tid + q * NTH;
      const int la = slot / B, lb = slot % B, lc = (t - la - lb) & (B - 1);
      bool valid = true;
      if constexpr (!FULL) valid = (!ij || la < lb) && (!kj || lb < lc) && (kB + lc < a.n);
      const int wd = slot >> 5;
      const int q0 = qt + wd, q1 = qt + M::WPR + wd, q2 = qt + 2 * M::WPR + wd;
      uint32_t m0 = 0u, m1 = 0u, m2 = 0u;
      if constexpr (HASMASK) {
        m0 = sm.mask[q0];
        m1 = sm.mask[q1];
        m2 = sm.mask[q2];
      }
      const bool b0 = (m0 >> lane) & 1u, b1 = (m1 >> lane) & 1u, b2 = (m2 >> lane) & 1u;
      if (valid && (a.nofilter || (b0 | b1 | b2) || !inactive_fast(gIJ[slot], gIK[la * B + lc], gJK[lb * B + lc]))) {
        T z0 = T(0), z1 = T(0), z2 = T(0);
        if (staged) {
          if (b0) z0 = sm.dual[sm.pre[q0] + __popc(m0 & below)];
          if (b1) z1 = sm.dual[sm.pre[q1] + __popc(m1 & below)];
          if (b2) z2 = sm.dual[sm.pre[q2] + __popc(m2 & below)];
        } else {
          if (b0) z0 = ld_stream(zs + slot);
          if (b1) z1 = ld_stream(zs + C::BB + slot);
          if (b2) z2 = ld_stream(zs + 2 * C::BB + slot);
        }
        const int pos = atomicAdd(&sm.lcnt[t], 1);
        sm.lslot[pos] = slot;
        sm.lz[0][pos] = z0;
        sm.lz[1][pos] = z1;
        sm.lz[2][pos] = z2;
      }
    }
    item_sync<WARP>();
    const int cnt = sm.lcnt[t];
    if (cnt > 0) {
      // list entry p goes to warp p % NW: a few updates land on different
      // warps (different SM sub-partitions, each with its own FP64 issue)
      constexpr int NWL = NTH / 32;
      if (a.trace && tid == 0) ++sm.nsub;
      for (int p = (tid & 31) * NWL + (tid >> 5); p < cnt; p += NTH) {
        const int slot = sm.lslot[p];
        const int la = slot / B, lb = slot % B, lc = (t - la - lb) & (B - 1);
        const int eij = slot, eik = la * B + lc, ejk = lb * B + lc;
        T z0 = sm.lz[0][p], z1 = sm.lz[1][p], z2 = sm.lz[2][p];
        const T o0 = z0, o1 = z1, o2 = z2;
        T xij = pIJ[eij], xik = pIK[eik], xjk = pJK[ejk];
        T vij = T(1), vik = T(1), vjk = T(1);
        if (!UNITW) {
          vij = a.winv[oIJ + eij];
          vik = a.winv[oIK + eik];
          vjk = a.winv[oJK + ejk];
        }
        if constexpr (SHADOW) {
          float fij = gIJ[eij], fik = gIK[eik], fjk = gJK[ejk];
          const T r = UNITW ? a.r_unit : T(1) / ((vij + vik) + vjk);
          const int rows = triplet_rows_skip<UNITW>(xij, xik, xjk, fij, fik, fjk, vij, vik, vjk, r, z0, z1, z2,
                                                     a.nofilter != 0);
          if (a.trace) {
            atomicAdd(&sm.ntrip, 1);
            atomicAdd(&sm.nrows, rows);
          }
          gIJ[eij] = fij;
          gIK[eik] = fik;
          gJK[ejk] = fjk;
        } else {
          triplet_rows<T, false, UNITW>(xij, xik, xjk, vij, vik, vjk, a.eps, a.r_unit, z0, z1, z2);
        }
        pIJ[eij] = xij;
        pIK[eik] = xik;
        pJK[ejk] = xjk;
        const uint32_t bit = 1u << (slot & 31);
        const int wq = qt + (slot >> 5);
        if (differs(z0, o0)) {
          st_stream(zs + slot, z0);
          if (nz(z0) != nz(o0)) {
            if (nz(z0)) atomicOr(&sm.mask[wq], bit); else atomicAnd(&sm.mask[wq], ~bit);
            sm.dirty = 1;
          }
        }
        if (differs(z1, o1)) {
          st_stream(zs + C::BB + slot, z1);
          if (nz(z1) != nz(o1)) {
            if (nz(z1)) atomicOr(&sm.mask[wq + M::WPR], bit); else atomicAnd(&sm.mask[wq + M::WPR], ~bit);
            sm.dirty = 1;
          }
        }
        if (differs(z2, o2)) {
          st_stream(zs + 2 * C::BB + slot, z2);
          if (nz(z2) != nz(o2)) {
            if (nz(z2)) atomicOr(&sm.mask[wq + 2 * M::WPR], bit); else atomicAnd(&sm.mask[wq + 2 * M::WPR], ~bit);
            sm.dirty = 1;
          }
        }
        touched = 1;
      }
      item_sync<WARP>();
    }
  }
  return touched;
}

// One block triple, processed by one CTA (WARP = false) or by one warp alone
// (WARP = true): stage tiles, mask and nonzero duals in shared memory
// (asynchronous copies, one round of memory latency per item), then walk
// the B sub-phases.
template <typename T, bool UNITW, int B, int NTH_>
__device__ __forceinline__ void flow_block_triple(const TiledArgs<T>& a, int w, int I, int J, int K,
                                                  FlowSmem<T, B>& sm, bool prestaged = false) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  constexpr bool SHADOW = sizeof(T) == 8;
  constexpr bool WARP = NTH_ == 32;
  constexpr int NTH = NTH_;                      // threads working on the item
  constexpr int SPT = C::BB / NTH;               // slots per thread and sub-phase
  constexpr int NW = NTH / 32;
  const int tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t oIJ = tile_index(a.nb, I, J) * C::BB;
  const int64_t oIK = tile_index(a.nb, I, K) * C::BB;
  const int64_t oJK = tile_index(a.nb, J, K) * C::BB;
  const bool kj = (K == J), ij = (I == J);
  T* pIJ = sm.x[0];
  T* pIK = kj ? sm.x[0] : sm.x[1];
  T* pJK = ij ? pIK : sm.x[2];
  // float values the pre-filter reads: a float copy of FP64 tiles, the
  // tiles themselves for FP32 state
  float* gIJ;
  float* gIK;
  float* gJK;
  if constexpr (SHADOW) {
    gIJ = sm.f[0];
    gIK = kj ? sm.f[0] : sm.f[SHADOW ? 1 : 0];
    gJK = ij ? gIK : sm.f[SHADOW ? 2 : 0];
  } else {
    gIJ = reinterpret_cast<float*>(pIJ);
    gIK = reinterpret_cast<float*>(pIK);
    gJK = reinterpret_cast<float*>(pJK);
  }
  T* zb = a.sparse ? a.sp_scratch + (int64_t)blockIdx.x * (3 * B * C::BB) : a.zt + (int64_t)w * (3 * B * C::BB);
  const uint32_t* mb = a.sparse ? nullptr : a.mask + (int64_t)w * M::PER_BT;
  {
    // checked build: every offset this item uses, tested once (the same
    // result in every thread, so the item is skipped as a whole)
    const long long te = (long long)a.ntiles * C::BB;
    bool ok = w >= 0 && w < a.nbt && oIJ >= 0 && oIJ + C::BB <= te && oIK >= 0 && oIK + C::BB <= te &&
              oJK >= 0 && oJK + C::BB <= te;
    if (a.sparse) {
      ok = ok && (long long)blockIdx.x < a.scratch_ctas && a.sp_off[w] >= 0 && a.sp_cnt[w] >= 0 &&
           a.sp_off[w] + a.sp_cnt[w] <= a.sp_cap_cur;
    } else {
      ok = ok && ((long long)w + 1) * (3 * B * C::BB) <= a.zt_elems && ((long long)w + 1) * M::PER_BT <= a.mask_words;
    }
    if (!CCD_IN_BOUNDS(ok, a.ctl)) return;
  }
  int sp_n = 0;
  long long sp_o = 0;
  if (a.sparse) {   // the item's bits are rebuilt from its entries below
    sp_n = a.sp_cnt[w];
    sp_o = a.sp_off[w];
    for (int e = tid; e < M::PER_BT; e += NTH) sm.mask[e] = 0u;
    item_sync<WARP>();
  }

  // first memory round trip: x tiles and mask words (16-byte copies, L2 only)
  constexpr int XCH = C::BB * (int)sizeof(T) / 16;     // 16-byte chunks per tile
  for (int e = tid; e < XCH; e += NTH) {
    cp_async16(reinterpret_cast<char*>(sm.x[0]) + 16 * e, reinterpret_cast<const char*>(a.x + oIJ) + 16 * e);
    if (!kj) cp_async16(reinterpret_cast<char*>(sm.x[1]) + 16 * e, reinterpret_cast<const char*>(a.x + oIK) + 16 * e);
    if (!ij) cp_async16(reinterpret_cast<char*>(sm.x[2]) + 16 * e, reinterpret_cast<const char*>(a.x + oJK) + 16 * e);
  }
  constexpr int MCH = M::PER_BT * 4 / 16;
  if (!a.sparse) {
    if (!prestaged)
      for (int e = tid; e < MCH; e += NTH)
        cp_async16(reinterpret_cast<char*>(sm.mask) + 16 * e, reinterpret_cast<const char*>(mb) + 16 * e);
  } else {
    // entries: set the bit, place the value in the CTA's scratch block and,
    // when they fit, in the staging array (ascending index = bit order)
    for (int e = tid; e < sp_n; e += NTH) {
      const uint32_t ix = a.sp_idx[sp_o + e];
      const T v = a.sp_val[sp_o + e];
      if (!CCD_IN_BOUNDS(ix < (uint32_t)(3 * B * C::BB), a.ctl)) continue;
      atomicOr(&sm.mask[ix >> 5], 1u << (ix & 31));
      zb[ix] = v;
      if (sp_n <= M::CAP) sm.dual[e] = v;
    }
  }
  for (int e = tid; e < B; e += NTH) sm.lcnt[e] = 0;
  if (tid == 0) {
    sm.dirty = 0;
    sm.t0 = B;
    sm.ntrip = 0;
    sm.nrows = 0;
    sm.nsub = 0;
    sm.subbits = 0u;
  }
  cp_async_wait_all();
  item_sync<WARP>();

  // exclusive prefix of the mask popcounts (the staging slot of each nonzero
  // dual) and the staging copies, unless warps 1.. did this during the wait
  const int total = prestaged ? sm.total : stage_duals<T, B, NTH, false>(a, sm, zb, tid);
  const bool staged = total <= M::CAP;
  constexpr int CH = (M::PER_BT + NTH - 1) / NTH;
  if constexpr (SHADOW) {
    for (int e = tid; e < C::BB; e += NTH) {
      sm.f[0][e] = f32_trunc(sm.x[0][e]);
      if (!kj) sm.f[SHADOW ? 1 : 0][e] = f32_trunc(sm.x[1][e]);
      if (!ij) sm.f[SHADOW ? 2 : 0][e] = f32_trunc(sm.x[2][e]);
    }
  }
  cp_async_wait_all();
  item_sync<WARP>();

  const int kB = K * B;
  const bool full = (I < J) && (J < K) && (kB + B <= a.n);
  int touched = 0;
  // per-warp form (filter and update in the same thread, one barrier per
  // sub-phase); compact = 1 selects compacted update lists for FP64 state
  if (WARP || !SHADOW || a.compact == 0) {
    if (full && total == 0)
      touched = flow_subphases<T, UNITW, B, NTH_, true, false>(a, w, sm, pIJ, pIK, pJK, gIJ, gIK, gJK, oIJ, oIK,
                                                               oJK, false, false, kB, staged, tid, lane, zb);
    else if (full)
      touched = flow_subphases<T, UNITW, B, NTH_, true, true>(a, w, sm, pIJ, pIK, pJK, gIJ, gIK, gJK, oIJ, oIK,
                                                              oJK, false, false, kB, staged, tid, lane, zb);
    else
      touched = flow_subphases<T, UNITW, B, NTH_, false, true>(a, w, sm, pIJ, pIK, pJK, gIJ, gIK, gJK, oIJ, oIK,
                                                               oJK, ij, kj, kB, staged, tid, lane, zb);
  } else {
    if constexpr (SHADOW && !WARP) {
      if (full && total == 0)
        touched = flow_subphases_compact<T, UNITW, B, NTH_, true, false>(a, sm, pIJ, pIK, pJK, gIJ, gIK, gJK, oIJ,
                                                                         oIK, oJK, false, false, kB, staged, tid,
                                                                         lane, zb);
      else if (full)
        touched = flow_subphases_compact<T, UNITW, B, NTH_, true, true>(a, sm, pIJ, pIK, pJK, gIJ, gIK, gJK, oIJ,
                                                                        oIK, oJK, false, false, kB, staged, tid,
                                                                        lane, zb);
      else
        touched = flow_subphases_compact<T, UNITW, B, NTH_, false, true>(a, sm, pIJ, pIK, pJK, gIJ, gIK, gJK, oIJ,
                                                                         oIK, oJK, ij, kj, kB, staged, tid, lane,
                                                                         zb);
    }
  }
  bool any_touched;
  if constexpr (WARP) any_touched = __any_sync(0xffffffffu, touched);
  else any_touched = __syncthreads_or(touched);
  if (sm.dirty && !a.sparse) {   // the item's mask words, once, if any bit flipped
    uint32_t* mw = a.mask + (int64_t)w * M::PER_BT;
    for (int e = tid; e < M::PER_BT; e += NTH) mw[e] = sm.mask[e];
  }
  if (any_touched) {
    for (int e = tid; e < C::BB; e += NTH) {
      a.x[oIJ + e] = sm.x[0][e];
      if (!kj) a.x[oIK + e] = sm.x[1][e];
      if (!ij) a.x[oJK + e] = sm.x[2][e];
    }
  }
  if (a.sparse) {
    // the item's nonzero duals into the next pool, in bit (index) order;
    // then the scratch block back to zero (every other slot already is)
    int mine = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int q = tid * CH + c;
      if (q < M::PER_BT) mine += __popc(sm.nmask[q]);
    }
    int inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) sm.scan[wid] = inc;
    item_sync<WARP>();
    if (wid == 0) {
      int v = lane < NW ? sm.scan[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (lane < NW) sm.scan[lane] = v;
    }
    item_sync<WARP>();
    const int cnt_new = sm.scan[NW - 1];
    if (tid == 0) {
      sm.base = cnt_new ? atomicAdd(a.sp_top, (unsigned long long)cnt_new) : 0ull;
      a.sp_cnt_next[w] = cnt_new;
    }
    item_sync<WARP>();
    const unsigned long long base = sm.base;
    const bool fits = base + (unsigned long long)cnt_new <= (unsigned long long)a.sp_cap;
    if (tid == 0) a.sp_off_next[w] = fits ? (long long)base : -1ll;
    long long pos = (long long)base + (wid ? sm.scan[wid - 1] : 0) + inc - mine;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int q = tid * CH + c;
      if (q < M::PER_BT) {
        uint32_t bits = sm.nmask[q];
        while (bits) {
          const int l = __ffs(bits) - 1;
          bits &= bits - 1;
          const uint32_t ix = (uint32_t)q * 32u + (uint32_t)l;
          if (fits) {
            a.sp_idx_next[pos] = ix;
            a.sp_val_next[pos] = zb[ix];
          }
          ++pos;
          zb[ix] = T(0);
        }
      }
    }
  }
  item_sync<WARP>();
}

// The pair rows of one tile (a pair item of the dataflow sweep).
template <typename T, int B, int NTH_>
__device__ __forceinline__ void flow_pair_tile(const TiledArgs<T>& a, int tl) {
  using C = TileCfg<B>;
  constexpr bool WARP = NTH_ == 32;
  constexpr int NTH = NTH_;
  const int tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
  const int pk = a.tile_list[tl];
  const int I = pk & 0xffff, J = pk >> 16;
  for (int slot = tid; slot < C::BB; slot += NTH) {
    const int la = slot / B, lb = slot % B;
    if ((I < J || la < lb) && J * B + lb < a.n) {
      const int64_t e = (int64_t)tl * C::BB + slot;
      T* zq = a.zp + (int64_t)tl * (2 * C::BB) + slot;
      T x = ld_l2(a.x + e), f = a.f[e];
      T zp = zq[0], zm = zq[C::BB];
      pair_rows<T, false>(x, f, a.d[e], a.winv[e], a.eps, zp, zm);
      a.x[e] = x;
      a.f[e] = f;
      zq[0] = zp;
      zq[C::BB] = zm;
    }
  }
}

// `passes` visits of every pair's two rows and nothing else (Hildreth's
// coordinate ascent restricted to the pair block of the dual, Sec. II-B).
// The pair rows of different pairs share no variable, so the passes of one
// pair run in registers one after the other, which is the same as `passes`
// pair-only sweeps one after the other.
template <typename T, bool EXACT, int B>
__global__ void k_pair_passes(TiledArgs<T> a, int passes) {
  using C = TileCfg<B>;
  const int64_t total = (int64_t)a.ntiles * C::BB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int tl = (int)(e / C::BB), slot = (int)(e % C::BB);
    const int pk = a.tile_list[tl];
    const int I = pk & 0xffff, J = pk >> 16;
    const int la = slot / B, lb = slot % B;
    if (!((I < J || la < lb) && J * B + lb < a.n)) continue;
    T* zq = a.zp + (int64_t)tl * (2 * C::BB) + slot;
    T x = a.x[e], f = a.f[e], zp = zq[0], zm = zq[C::BB];
    const T d = a.d[e], wv = a.winv[e];
    for (int k = 0; k < passes; ++k) pair_rows<T, EXACT>(x, f, d, wv, a.eps, zp, zm);
    a.x[e] = x;
    a.f[e] = f;
    zq[0] = zp;
    zq[C::BB] = zm;
  }
}

// One sweep as a dataflow over tiles.  Work items, taken in order from one
// counter: the block triples in schedule order (phase-major, largest first
// inside a phase), then one pair item per tile.  Every phase visits every
// tile exactly once, so a block triple of phase g may start once each of its
// tiles has g visits (counters in `tile_cnt`), and a tile's pair item once it
// has Nb.  No grid-wide barrier: a CTA waits only for the items it depends
// on, which were taken earlier by resident CTAs.
template <typename T, bool UNITW, int B, int NT>
__global__ void __launch_bounds__(NT) k_sweep_flow(TiledArgs<T> a, int* flow) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FlowSmem<T, B>& sm = *reinterpret_cast<FlowSmem<T, B>*>(smem_raw);
  int* const next = flow;            // item counter
  int* const tile_cnt = flow + 1;    // visits per tile in this sweep
  const int total = a.nbt + (a.pairs ? a.ntiles : 0);
  bool first = true;
  if (threadIdx.x == 0) sm.item = atomicAdd(next, 1);
  __syncthreads();
  int w = sm.item;
  while (w < total) {
    int nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(next, 1);   // the following item, fetched while this one runs
    unsigned long long* tr = a.trace ? a.trace + 6 * (int64_t)w : nullptr;
    if (tr && threadIdx.x == 0) {
      tr[0] = global_ns();
      tr[5] = (unsigned long long)blockIdx.x;
    }
    if (w < a.nbt) {
      int I, J, K;
      unpack_bt(a.bt_list[w], I, J, K);
      const int g = (I + J + K) % a.nb;
      const int64_t tIJ = tile_index(a.nb, I, J), tIK = tile_index(a.nb, I, K), tJK = tile_index(a.nb, J, K);
      const int64_t u1 = (K == J) ? -1 : tIK, u2 = (I == J) ? -1 : tJK;
      // one look at the tiles; if they are not ready, warp 0 waits while the
      // other warps stage what the item owns alone (dense store: its bits,
      // their prefix and its nonzero duals) or, for the sparse store in FP64
      // state, bring its entry list toward L2
      if (threadIdx.x == 0) {
        const bool rdy = tiles_ready(tile_cnt, tIJ, u1, u2, g);
        if (rdy) asm volatile("fence.acq_rel.gpu;" ::: "memory");
        sm.ready = rdy;
        sm.flag = rdy;
      }
      __syncthreads();
      bool pre = false;
      if (!sm.ready) {
        if (threadIdx.x >= 32) {
          if (!a.sparse) prestage_item<T, B, NT>(a, w, sm);
          else if (sizeof(T) == 8) warm_item<T, B>(a, w, (int)threadIdx.x - 32, NT - 32);
        } else if (threadIdx.x == 0) {
          sm.flag = wait_tiles(tile_cnt, tIJ, u1, u2, g, a.ctl, a.timeout_ns, g);
        }
        __syncthreads();
        pre = !a.sparse;
      }
      if (tr && threadIdx.x == 0) tr[1] = global_ns();
      if (!sm.flag) return;
      flow_block_triple<T, UNITW, B, NT>(a, w, I, J, K, sm, pre);
      if (tr && threadIdx.x == 0) {
        tr[2] = global_ns();
        tr[4] = (unsigned long long)min(sm.total, 0xffffff) | ((unsigned long long)min(sm.ntrip, 0xffff) << 24) |
                ((unsigned long long)min(sm.nrows, 0xffff) << 40) | ((unsigned long long)min(sm.nsub + __popc(sm.subbits), 0xff) << 56);
      }
      if (first && (int)blockIdx.x == a.skip_cta) return;   // fault injection: never release
      if (threadIdx.x == 0) {
        release_tiles(tile_cnt, tIJ, u1, u2);
        // the next item's bits, on their way to L2 while it waits or stages
        using M = MaskCfg<B>;
        if (sizeof(T) == 8 && !a.sparse && nxt < a.nbt && (long long)(nxt + 1) * M::PER_BT <= a.mask_words)
          prefetch_l2_bulk(a.mask + (int64_t)nxt * M::PER_BT, M::PER_BT * 4);
      }
      if (tr && threadIdx.x == 0) tr[3] = global_ns();
    } else {
      const int tl = w - a.nbt;
      if (threadIdx.x == 0) sm.flag = wait_tiles(tile_cnt, tl, -1, -1, a.nb, a.ctl, a.timeout_ns, a.nb);
      __syncthreads();
      if (!sm.flag) return;
      flow_pair_tile<T, B, NT>(a, tl);
    }
    first = false;
    if (threadIdx.x == 0) sm.item = nxt;
    __syncthreads();
    w = sm.item;
    __syncthreads();
  }
}

// Many instances in one launch (the batched form).  `items` lists (instance,
// local item) pairs; each instance's local items are its block triples in
// schedule order, then its pair tiles, and the list keeps every instance's
// items in that order, so each item depends only on items listed before it
// and the dataflow argument above carries over.  Instances are independent,
// so the items of one fill the dependency waits of another.  The arguments of
// an item's instance are read from global memory, which costs registers the
// single-instance kernel does not spend; for B = 16 the kernel is held to 64
// registers so that four CTAs share an SM (80 registers gave three).  The
// batch keeps the FP64 pipe busy (its instances keep many rows active), and
// the fourth CTA outweighs the few spilled bytes the cap costs.
template <typename T, bool UNITW, int B, int NT>
__global__ void __launch_bounds__(NT, (B == 16 && NT == 256) ? 4 : 1) k_sweep_batch(const TiledArgs<T>* __restrict__ args,
                                                    const int2* __restrict__ items, int total, int* next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FlowSmem<T, B>& sm = *reinterpret_cast<FlowSmem<T, B>*>(smem_raw);
  if (threadIdx.x == 0) sm.item = atomicAdd(next, 1);
  __syncthreads();
  int w = sm.item;
  while (w < total) {
    int nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(next, 1);
    const int2 it = items[w];
    const TiledArgs<T>& a = args[it.x];
    const int lw = it.y;
    if (lw < a.nbt) {
      int I, J, K;
      unpack_bt(a.bt_list[lw], I, J, K);
      const int g = (I + J + K) % a.nb;
      const int64_t tIJ = tile_index(a.nb, I, J), tIK = tile_index(a.nb, I, K), tJK = tile_index(a.nb, J, K);
      const int64_t u1 = (K == J) ? -1 : tIK, u2 = (I == J) ? -1 : tJK;
      if (threadIdx.x == 0) sm.flag = wait_tiles(a.cnt, tIJ, u1, u2, g, a.ctl, a.timeout_ns, g);
      __syncthreads();
      if (!sm.flag) return;
      flow_block_triple<T, UNITW, B, NT>(a, lw, I, J, K, sm);
      if (threadIdx.x == 0) release_tiles(a.cnt, tIJ, u1, u2);
    } else {
      const int tl = lw - a.nbt;
      if (threadIdx.x == 0) sm.flag = wait_tiles(a.cnt, tl, -1, -1, a.nb, a.ctl, a.timeout_ns, a.nb);
      __syncthreads();
      if (!sm.flag) return;
      flow_pair_tile<T, B, NT>(a, tl);
    }
    if (threadIdx.x == 0) sm.item = nxt;
    __syncthreads();
    w = sm.item;
    __syncthreads();
  }
}

// The same dataflow sweep with one warp per work item: the warps of a CTA
// are independent (each has its own shared-memory slice and synchronizes
// only with __syncwarp), so no CTA-wide barrier is ever needed.
template <typename T, bool UNITW, int B>
__global__ void __launch_bounds__(256) k_sweep_warpflow(TiledArgs<T> a, int* flow) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  FlowSmem<T, B>& sm = reinterpret_cast<FlowSmem<T, B>*>(smem_raw)[wid];
  int* const next = flow;
  int* const tile_cnt = flow + 1;
  const int total = a.nbt + (a.pairs ? a.ntiles : 0);
  bool first = true;
  while (true) {
    int w = 0;
    if (lane == 0) w = atomicAdd(next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= total) break;
    if (w < a.nbt) {
      int I, J, K;
      unpack_bt(a.bt_list[w], I, J, K);
      const int g = (I + J + K) % a.nb;
      const int64_t tIJ = tile_index(a.nb, I, J), tIK = tile_index(a.nb, I, K), tJK = tile_index(a.nb, J, K);
      const int64_t u1 = (K == J) ? -1 : tIK, u2 = (I == J) ? -1 : tJK;
      int ok = 0;
      if (lane == 0) ok = wait_tiles(tile_cnt, tIJ, u1, u2, g, a.ctl, a.timeout_ns, g);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) return;
      flow_block_triple<T, UNITW, B, 32>(a, w, I, J, K, sm);
      if (first && (int)blockIdx.x == a.skip_cta) return;   // fault injection: never release
      if (lane == 0) release_tiles(tile_cnt, tIJ, u1, u2);
    } else {
      const int tl = w - a.nbt;
      int ok = 0;
      if (lane == 0) ok = wait_tiles(tile_cnt, tl, -1, -1, a.nb, a.ctl, a.timeout_ns, a.nb);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) return;
      flow_pair_tile<T, B, 32>(a, tl);
      __syncwarp();
    }
    first = false;
  }
}

// Rebuild the nonzero bits from the dual store (after the store was written
// from outside a sweep).  One thread per mask word.
template <typename T, int B>
__global__ void k_rebuild_mask(const T* zt, uint32_t* mask, int64_t nwords) {
  using M = MaskCfg<B>;
  constexpr int BB = B * B;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nwords; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = q / M::PER_BT;
    const int rem = (int)(q % M::PER_BT);
    const int t = rem / (3 * M::WPR), r = (rem / M::WPR) % 3, wd = rem % M::WPR;
    const T* z = zt + w * (3 * B * BB) + (int64_t)t * (3 * BB) + r * BB + wd * 32;
    uint32_t bits = 0;
    for (int l = 0; l < 32; ++l) bits |= (z[l] != T(0) ? 1u : 0u) << l;
    mask[q] = bits;
  }
}

// ------------------------------------------------------------ reductions

template <typename V, typename Op>
__device__ __forceinline__ V block_reduce(V v, Op op, V* sred, V identity) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sred[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < nw ? sred[lane] : identity;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

struct MaxOp {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
};
struct SumOp {
  __device__ double operator()(double a, double b) const { return a + b; }
};

// Largest metric-row violation max(0, x_h - x_a - x_b) over all triplets,
// evaluated in FP64; one partial maximum per CTA.  A triplet's rows are
// evaluated in FP64 only when their float estimate can still exceed the
// running maximum m.  The largest row delta of a triplet is 2 max(x) - sum(x);
// from float copies of its three values (for FP64 state truncated with
// integer operations, f32_trunc: within 2^-23 |x|; a conversion instruction
// would occupy the FP64 unit) that estimate is within 11 * 2^-24 S + 2^-123
// of the exact one (S = |x_h| + |x_a| + |x_b|; three copies, two additions,
// one fused multiply-add).  Skipping when RN(dmax_f + tau) <= m_f (tau =
// RN(2^-19 S + 2^-100), m_f = m rounded down to float) never skips a row
// above m: either S >= m / 21, and the margin tau - 11 * 2^-24 S covers m_f's
// half ulp, or every row delta <= S < m.  The maximum is order-free, so the
// result equals a serial FP64 evaluation.  Each CTA walks block triples with
// the next one's three tiles already on their way (asynchronous copies into
// a second buffer).
template <typename T, int B>
__global__ void __launch_bounds__(TileCfg<B>::NT) k_maxviol_tiled(const T* __restrict__ x, int n, int nb,
                                                                   const btpk* __restrict__ bt_list, int nbt,
                                                                   double* part) {
  using C = TileCfg<B>;
  // two tile buffers where they fit in the 48 KB of static shared memory
  constexpr int NBUF = (3 * C::BB * (int)sizeof(T) * 2 + 3 * C::BB * 4 <= 40 * 1024) ? 2 : 1;
  __shared__ __align__(16) T sx[NBUF][3][C::BB];
  __shared__ float sf[3][C::BB];
  __shared__ double sred[32];
  constexpr int XCH = C::BB * (int)sizeof(T) / 16;     // 16-byte chunks per tile
  double m = 0.0;
  float mf = 0.0f;
  auto issue = [&](int w, int buf) {
    int I, J, K;
    unpack_bt(bt_list[w], I, J, K);
    const int64_t o0 = tile_index(nb, I, J) * C::BB, o1 = tile_index(nb, I, K) * C::BB,
                  o2 = tile_index(nb, J, K) * C::BB;
    for (int e = threadIdx.x; e < 3 * XCH; e += C::NT) {
      const int t = e / XCH, c = e % XCH;
      const int64_t ot = t == 0 ? o0 : (t == 1 ? o1 : o2);
      cp_async16(reinterpret_cast<char*>(sx[buf][t]) + 16 * c, reinterpret_cast<const char*>(x + ot) + 16 * c);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int buf = 0;
  if (NBUF == 2 && (int)blockIdx.x < nbt) issue(blockIdx.x, 0);
  for (int w = blockIdx.x; w < nbt; w += gridDim.x) {
    const int wn = w + gridDim.x;
    if (NBUF == 1) {
      issue(w, 0);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (wn < nbt) {
      issue(wn, buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    for (int e = threadIdx.x; e < C::BB; e += C::NT) {
      sf[0][e] = to_shadow(sx[buf][0][e]);
      sf[1][e] = to_shadow(sx[buf][1][e]);
      sf[2][e] = to_shadow(sx[buf][2][e]);
    }
    __syncthreads();
    int I, J, K;
    unpack_bt(bt_list[w], I, J, K);
    const bool kj = (K == J), ij = (I == J);
    const int kB = K * B;
    for (int slot = threadIdx.x; slot < C::BB; slot += C::NT) {
      const int la = slot / B, lb = slot % B;
      if (ij && la >= lb) continue;
      const float fij = sf[0][la * B + lb];
      const float* fik_row = sf[1] + la * B;
      const float* fjk_row = sf[2] + lb * B;
      auto triplet = [&](int lc) {
        const float fik = fik_row[lc], fjk = fjk_row[lc];
        const float mx = fmaxf(fmaxf(fij, fik), fjk);
        const float dmax = fmaf(2.0f, mx, -((fij + fik) + fjk));
        const float S = (fabsf(fij) + fabsf(fik)) + fabsf(fjk);
        if (dmax + fmaf(S, 0x1p-19f, 0x1p-100f) > mf) {
          const double xij = (double)sx[buf][0][la * B + lb];
          const double xik = (double)sx[buf][1][la * B + lc], xjk = (double)sx[buf][2][lb * B + lc];
          const double v0 = (xij - xik) - xjk, v1 = (xik - xij) - xjk, v2 = (xjk - xij) - xik;
          const double v = fmax(v0, fmax(v1, v2));
          if (v > m) {
            m = v;
            mf = __double2float_rd(m);
          }
        }
      };
      if (!kj && kB + B <= n) {   // every c of the K block: an unrolled run
#pragma unroll
        for (int lc = 0; lc < B; ++lc) triplet(lc);
      } else {
        for (int lc = kj ? lb + 1 : 0; lc < B && kB + lc < n; ++lc) triplet(lc);
      }
    }
    __syncthreads();   // buffer buf is refilled two items on (one with a single buffer)
    if (NBUF == 2) buf ^= 1;
  }
  m = block_reduce(m, MaxOp(), sred, 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// Pair sums: lp = sum w|x-d|, wf = sum w f, quad = sum w (x^2 + f^2),
// by = sum d (y+ - y-) (y = yscale * stored dual), pv = max pair violation.
template <typename T, int B>
__global__ void __launch_bounds__(256) k_pairsums_tiled(const T* __restrict__ x, const T* __restrict__ f,
                                                         const double* __restrict__ d, const double* __restrict__ winv,
                                                         const T* __restrict__ zp, const int* __restrict__ tile_list,
                                                         int ntiles, int n, double yscale, int l2, double* part) {
  using C = TileCfg<B>;
  __shared__ double sred[32];
  double lp = 0, wf = 0, quad = 0, by = 0, pv = 0;
  const int64_t total = (int64_t)ntiles * C::BB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int tl = (int)(e / C::BB), slot = (int)(e % C::BB);
    const int pk = tile_list[tl];
    const int I = pk & 0xffff, J = pk >> 16;
    const int la = slot / B, lb = slot % B;
    if (!((I < J || la < lb) && J * B + lb < n)) continue;
    const double xv = x[e], fv = f[e], dv = d[e], wv = 1.0 / winv[e];
    if (l2) {   // sum w (x - d)^2 and sum w d (d - x)
      lp += wv * ((xv - dv) * (xv - dv));
      wf += wv * (dv * (dv - xv));
      continue;
    }
    const double yp = yscale * (double)zp[(int64_t)tl * 2 * C::BB + slot];
    const double ym = yscale * (double)zp[(int64_t)tl * 2 * C::BB + C::BB + slot];
    lp += wv * fabs(xv - dv);
    wf += wv * fv;
    quad += wv * (xv * xv + fv * fv);
    by += dv * (yp - ym);
    pv = fmax(pv, fmax(xv - fv - dv, dv - xv - fv));
  }
  lp = block_reduce(lp, SumOp(), sred, 0.0);
  if (threadIdx.x == 0) part[5 * blockIdx.x + 0] = lp;
  wf = block_reduce(wf, SumOp(), sred, 0.0);
  if (threadIdx.x == 0) part[5 * blockIdx.x + 1] = wf;
  quad = block_reduce(quad, SumOp(), sred, 0.0);
  if (threadIdx.x == 0) part[5 * blockIdx.x + 2] = quad;
  by = block_reduce(by, SumOp(), sred, 0.0);
  if (threadIdx.x == 0) part[5 * blockIdx.x + 3] = by;
  pv = block_reduce(pv, MaxOp(), sred, 0.0);
  if (threadIdx.x == 0) part[5 * blockIdx.x + 4] = fmax(pv, 0.0);
}

// ------------------------------------------------------------ layout moves

// packed pair p -> (i, j)
__device__ __forceinline__ void pair_unrank(int64_t n, int64_t p, int& i, int& j) {
  int lo = 0, hi = (int)n - 2;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pair_index(n, mid, mid + 1) <= p) lo = mid; else hi = mid - 1;
  }
  i = lo;
  j = (int)(p - pair_index(n, i, i + 1)) + i + 1;
}

// Caller labels -> internal labels.  `lab` (n ints, or null for the
// identity) is the relabeling of the tiled schedule; the pair comes back in
// increasing internal order.
__device__ __forceinline__ void map_pair(const int* lab, int& i, int& j) {
  if (lab) {
    const int a = lab[i], b = lab[j];
    i = min(a, b);
    j = max(a, b);
  }
}

// Same for a triplet i<j<k; rowmap[r] is the internal row (0: hyp uv,
// 1: hyp uw, 2: hyp vw of the sorted internal labels u<v<w) of the caller's
// row r (0: hyp ij, 1: hyp ik, 2: hyp jk).  A row is named by its hypotenuse
// pair, i.e. by the label it leaves out: leaving out the largest is row 0,
// the middle one row 1, the smallest row 2.
__device__ __forceinline__ void map_triplet(const int* lab, int& i, int& j, int& k, int* rowmap) {
  if (!lab) {
    rowmap[0] = 0;
    rowmap[1] = 1;
    rowmap[2] = 2;
    return;
  }
  const int a = lab[i], b = lab[j], c = lab[k];
  const int u = min(a, min(b, c)), w = max(a, max(b, c)), v = a + b + c - u - w;
  auto out = [&](int third) { return third == w ? 0 : (third == v ? 1 : 2); };
  rowmap[0] = out(c);   // hyp ij leaves out k
  rowmap[1] = out(b);   // hyp ik leaves out j
  rowmap[2] = out(a);   // hyp jk leaves out i
  i = u;
  j = v;
  k = w;
}

// dir 0: tile-major (x, f) -> packed double buffers; dir 1: the reverse.
template <typename T>
__global__ void k_pairs_layout(T* x, T* f, int n, int nb, int B, double* px, double* pf, int dir,
                               const int* lab) {
  const int64_t P = ch2(n);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    pair_unrank(n, p, i, j);
    map_pair(lab, i, j);
    const int64_t e = tiled_offset(nb, B, i, j);
    if (dir == 0) {
      if (px) px[p] = (double)x[e];
      if (pf) pf[p] = (double)f[e];
    } else {
      if (px) x[e] = (T)px[p];
      if (pf) f[e] = (T)pf[p];
    }
  }
}

// Packed d, w (device, double) -> tile-major d and W^{-1}.
template <typename T>
__global__ void k_load_problem(const double* pd, const double* pw, int n, int nb, int B, T* d, T* winv,
                               const int* lab) {
  const int64_t P = ch2(n);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    pair_unrank(n, p, i, j);
    map_pair(lab, i, j);
    const int64_t e = tiled_offset(nb, B, i, j);
    d[e] = (T)pd[p];
    winv[e] = (T)(1.0 / pw[p]);
  }
}

// Input checks on device: flags[0] += non-finite d, flags[1] += w not finite
// or <= 0, flags[2] += w != 1.
__global__ void k_validate(const double* pd, const double* pw, int64_t P, int* flags) {
  int bad_d = 0, bad_w = 0, nonunit = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const double dv = pd[p], wv = pw[p];
    bad_d |= !isfinite(dv);
    bad_w |= !(isfinite(wv) && wv > 0.0);
    nonunit |= (wv != 1.0);
  }
  if (__syncthreads_or(bad_d) && threadIdx.x == 0) atomicAdd(&flags[0], 1);
  if (__syncthreads_or(bad_w) && threadIdx.x == 0) atomicAdd(&flags[1], 1);
  if (__syncthreads_or(nonunit) && threadIdx.x == 0) atomicAdd(&flags[2], 1);
}

template <typename T>
__global__ void k_fill(T* p, int64_t count, T v) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = v;
}

// Triangle duals between the tiled store and canonical order.
// dir 0: buf[3q + r] = scale * z;  dir 1: z = buf[3q + r] / scale.
template <typename T, int B>
__global__ void k_tri_duals_tiled(T* zt, const int* bt_rank, int n, int nb, int64_t first, int64_t count,
                                  double* buf, double scale, int dir, const int* lab) {
  constexpr int BB = B * B;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k, rm[3];
    tri_unrank(n, first + q, i, j, k);
    map_triplet(lab, i, j, k, rm);
    const int I = i / B, J = j / B, K = k / B;
    const int la = i % B, lb = j % B, lc = k % B;
    const int t = (la + lb + lc) % B;
    const int64_t w = bt_rank[((int64_t)I * nb + J) * nb + K];
    const int64_t base = w * (3 * B * BB) + (int64_t)t * (3 * BB) + la * B + lb;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (dir == 0) buf[3 * q + r] = scale * (double)zt[base + rm[r] * BB];
      else zt[base + rm[r] * BB] = (T)(buf[3 * q + r] / scale);
    }
  }
}

// Pair duals between the tiled store and packed order (2 per pair).
template <typename T>
__global__ void k_pair_duals_tiled(T* zp, int n, int nb, int B, double* buf, double scale, int dir,
                                   const int* lab) {
  const int64_t P = ch2(n);
  const int BB = B * B;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    pair_unrank(n, p, i, j);
    map_pair(lab, i, j);
    const int64_t tl = tile_index(nb, i / B, j / B);
    const int64_t e = tl * (2 * BB) + (i % B) * B + (j % B);
    if (dir == 0) {
      buf[2 * p] = scale * (double)zp[e];
      buf[2 * p + 1] = scale * (double)zp[e + BB];
    } else {
      zp[e] = (T)(buf[2 * p] / scale);
      zp[e + BB] = (T)(buf[2 * p + 1] / scale);
    }
  }
}

// ------------------------------------------------------------ resync
//
// Dykstra keeps v = v0 - W^{-1} A^T z (z = y/eps) at every step.  After the
// duals change precision (FP32 bulk -> FP64 refinement) or are set from
// outside, x and f are rebuilt from that identity in FP64:
//   acc_p = sum over metric rows of z_r * (+1 if p is a leg, -1 if p is the
//           hypotenuse),
//   x_p = w_p^-1 (acc_p - z+_p + z-_p),   f_p = -1/eps + w_p^-1 (z+_p + z-_p).
// Pass 1 visits the block triples phase by phase (tiles of one phase are
// disjoint) and inside a block triple sub-phase by sub-phase, so the sums are
// formed in one fixed order (deterministic); block triples without a nonzero
// dual are skipped through the bitmask.
// Sparse-store input of the resync (idx == nullptr: the dense store is used).
struct SparseIn {
  const uint32_t* idx;
  const double* val;
  const long long* off;
  const int* cnt;
  double* scratch;      // 3 B^3 doubles per CTA, zero
};

template <int B>
__global__ void __launch_bounds__(TileCfg<B>::NT) k_resync_metric(const double* __restrict__ zt,
                                                                   const uint32_t* __restrict__ mask, double* acc,
                                                                   int n, int nb, const btpk* __restrict__ bt_list,
                                                                   const int* __restrict__ bt_off, Ctl* ctl,
                                                                   long long timeout_ns, SparseIn sp) {
  using C = TileCfg<B>;
  using M = MaskCfg<B>;
  __shared__ double sx[3][C::BB];
  __shared__ uint32_t smask[M::PER_BT];   // sparse store: the item's bits rebuilt from its entries
  __shared__ int s_flag;
  unsigned target = 0;
  const int lane = threadIdx.x & 31;
  double* scratch = sp.idx ? sp.scratch + (int64_t)blockIdx.x * (3 * B * C::BB) : nullptr;
  for (int g = 0; g < nb; ++g) {
    for (int w = bt_off[g] + (int)blockIdx.x; w < bt_off[g + 1]; w += gridDim.x) {
      const uint32_t* mb;
      const double* zb;
      if (sp.idx) {
        const int m = sp.cnt[w];
        if (m == 0) continue;   // the same in every thread
        const long long o = sp.off[w];
        for (int e = threadIdx.x; e < M::PER_BT; e += C::NT) smask[e] = 0u;
        __syncthreads();
        for (int e = threadIdx.x; e < m; e += C::NT) {
          const uint32_t ix = sp.idx[o + e];
          atomicOr(&smask[ix >> 5], 1u << (ix & 31));
          scratch[ix] = sp.val[o + e];
        }
        __syncthreads();
        mb = smask;
        zb = scratch;
      } else {
        mb = mask + (int64_t)w * M::PER_BT;
        zb = zt + (int64_t)w * (3 * B * C::BB);
        int any = 0;
        for (int e = threadIdx.x; e < M::PER_BT; e += C::NT) any |= (mb[e] != 0u);
        if (!__syncthreads_or(any)) continue;
      }
      int I, J, K;
      unpack_bt(bt_list[w], I, J, K);
      const int64_t oIJ = tile_index(nb, I, J) * C::BB, oIK = tile_index(nb, I, K) * C::BB,
                    oJK = tile_index(nb, J, K) * C::BB;
      const bool kj = (K == J), ij = (I == J);
      double* pIJ = sx[0];
      double* pIK = kj ? sx[0] : sx[1];
      double* pJK = ij ? pIK : sx[2];
      for (int e = threadIdx.x; e < C::BB; e += C::NT) {
        sx[0][e] = ld_l2(acc + oIJ + e);
        if (!kj) sx[1][e] = ld_l2(acc + oIK + e);
        if (!ij) sx[2][e] = ld_l2(acc + oJK + e);
      }
      __syncthreads();
      for (int t = 0; t < B; ++t) {
        for (int q = 0; q < C::SPT; ++q) {
          const int slot = threadIdx.x + q * C::NT;
          const int la = slot / B, lb = slot % B, lc = (t - la - lb) & (B - 1);
          const int qw = t * (3 * M::WPR) + (slot >> 5);
          const bool b0 = (mb[qw] >> lane) & 1u, b1 = (mb[qw + M::WPR] >> lane) & 1u,
                     b2 = (mb[qw + 2 * M::WPR] >> lane) & 1u;
          if (b0 | b1 | b2) {
            const double* zs = zb + (int64_t)t * (3 * C::BB) + slot;
            const double z0 = b0 ? zs[0] : 0.0, z1 = b1 ? zs[C::BB] : 0.0, z2 = b2 ? zs[2 * C::BB] : 0.0;
            const int eij = la * B + lb, eik = la * B + lc, ejk = lb * B + lc;
            double aij = pIJ[eij], aik = pIK[eik], ajk = pJK[ejk];
            aij = ((aij - z0) + z1) + z2;   // hypotenuse of row 0, leg of rows 1 and 2
            aik = ((aik + z0) - z1) + z2;   // hypotenuse of row 1
            ajk = ((ajk + z0) + z1) - z2;   // hypotenuse of row 2
            pIJ[eij] = aij;
            pIK[eik] = aik;
            pJK[ejk] = ajk;
          }
        }
        __syncthreads();
      }
      for (int e = threadIdx.x; e < C::BB; e += C::NT) {
        acc[oIJ + e] = sx[0][e];
        if (!kj) acc[oIK + e] = sx[1][e];
        if (!ij) acc[oJK + e] = sx[2][e];
      }
      if (sp.idx) {   // the scratch block back to zero
        const long long o = sp.off[w];
        for (int e = threadIdx.x; e < sp.cnt[w]; e += C::NT) scratch[sp.idx[o + e]] = 0.0;
      }
      __syncthreads();
    }
    target += gridDim.x;
    if (!grid_barrier(ctl, target, timeout_ns, g, false, &s_flag)) return;
  }
}

// Pass 2: x and f from acc and the pair duals (in place: acc is x).
__global__ void k_resync_finish(double* x, double* f, const double* __restrict__ winv,
                                const double* __restrict__ zp, int64_t ntiles, int BB, double eps) {
  const int64_t total = ntiles * BB;
  const double f0 = -(1.0 / eps);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tl = e / BB, slot = e % BB;
    const double zpv = zp[tl * 2 * BB + slot], zmv = zp[tl * 2 * BB + BB + slot];
    x[e] = winv[e] * ((x[e] - zpv) + zmv);
    f[e] = f0 + winv[e] * (zpv + zmv);
  }
}

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* dst, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (D)src[e];
}

}  // namespace ccd

namespace ccd {

// Triangle duals of the sparse store in canonical order (caller labels):
// every entry of every block triple is mapped to its triplet and row and,
// when the triplet's rank lies in [first, first + count), written as
// buf[3 (rank - first) + row] = scale * value.  buf must be zeroed first.
// ilab maps internal to caller labels (nullptr: identity).  A row is named by
// the object it leaves out: row 0 (hypotenuse ij) leaves out k, 1 leaves out
// j, 2 leaves out i.
template <typename T, int B>
__global__ void k_tri_duals_sparse(const uint32_t* __restrict__ idx, const T* __restrict__ val,
                                   const long long* __restrict__ off, const int* __restrict__ cnt,
                                   const btpk* __restrict__ bt_list, int nbt, int n, const int* __restrict__ ilab,
                                   int64_t first, int64_t count, double* buf, double scale) {
  constexpr int BB = B * B;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nbt; w += gridDim.x * blockDim.x) {
    int I, J, K;
    unpack_bt(bt_list[w], I, J, K);
    const long long o = off[w];
    const int m = cnt[w];
    for (int e = 0; e < m; ++e) {
      const uint32_t ix = idx[o + e];
      const int t = (int)(ix / (3 * BB)), r = (int)((ix / BB) % 3), slot = (int)(ix % BB);
      const int la = slot / B, lb = slot % B, lc = (t - la - lb) & (B - 1);
      int a = I * B + la, b = J * B + lb, c = K * B + lc;       // internal labels, a < b < c
      const int out = r == 0 ? c : (r == 1 ? b : a);
      int co = out;
      if (ilab) {
        a = ilab[a];
        b = ilab[b];
        c = ilab[c];
        co = ilab[out];
      }
      const int u = min(a, min(b, c)), z = max(a, max(b, c)), v = a + b + c - u - z;
      const int row = co == z ? 0 : (co == v ? 1 : 2);
      const int64_t rank = tri_rank(n, u, v, z);
      if (rank >= first && rank < first + count) buf[3 * (rank - first) + row] = scale * (double)val[o + e];
    }
  }
}

}  // namespace ccd
