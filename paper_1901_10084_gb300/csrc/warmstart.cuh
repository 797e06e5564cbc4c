// Learned dual warm start (not in the paper).  A small MLP predicts the three
// triangle duals of a triplet from ten features; the predicted duals are
// written into the dual store and x, f are rebuilt from them through the
// identity v = v0 - W^{-1} A^T y / eps that Dykstra's method keeps, so the
// solve continues from a consistent state and converges to the same optimum
// (Dykstra on halfspaces is dual coordinate ascent from any nonnegative
// start).  Included at the end of ccdyk.cu (it uses the handle's internals).
//
// Candidates: triplets with at least one edge (d = 0) among their three
// pairs; every other triplet keeps dual 0 (three non-edges give rows with a
// slack near 1).  Features of a candidate (a, b, c), internal labels a<b<c,
// edges from d = 0:
//   d_ab, d_ac, d_bc; log(1 + deg u / mean degree) for u = a, b, c;
//   log(1 + common neighbours) of ab, ac, bc and of all three.
// Network: 10 -> 64 -> 64 -> 3, ReLU, softplus output, BF16 weights and
// activations, FP32 accumulation (mma.sync m16n8k16 on the tensor cores).
// After the rebuild, a few passes over the pair rows alone let the pair
// duals (not predicted, started at 0) settle to the predicted triangle duals.
#pragma once

namespace ccd {

constexpr int WS_IN = 10, WS_H = 64, WS_OUT = 3;
// parameter layout (floats): W1[10][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3]
constexpr int WS_W1 = 0, WS_B1 = WS_W1 + WS_IN * WS_H, WS_W2 = WS_B1 + WS_H, WS_B2 = WS_W2 + WS_H * WS_H,
              WS_W3 = WS_B2 + WS_H, WS_B3 = WS_W3 + WS_H * WS_OUT, WS_NPARAM = WS_B3 + WS_OUT;
constexpr int WS_FEAT = 12;  // feature row stride (10 used)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat16 l = __float2bfloat16_rn(lo), h = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(l) | ((uint32_t)__bfloat16_as_ushort(h) << 16);
}

// D = A * B + C for one 16x8x16 tile: A row-major bf16 (4 regs), B col-major
// bf16 (2 regs), C/D fp32 (4 regs).
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Weights staged in shared memory as bf16, K padded to multiples of 16 and
// the output width of layer 3 to 8.
struct WsSmem {
  __nv_bfloat16 w1[16][WS_H];
  __nv_bfloat16 w2[WS_H][WS_H];
  __nv_bfloat16 w3[WS_H][8];
  float b1[WS_H], b2[WS_H], b3[8];
};

__device__ __forceinline__ void ws_stage_weights(const float* __restrict__ p, WsSmem& s) {
  for (int e = threadIdx.x; e < 16 * WS_H; e += blockDim.x) {
    const int k = e / WS_H, n = e % WS_H;
    s.w1[k][n] = __float2bfloat16_rn(k < WS_IN ? p[WS_W1 + k * WS_H + n] : 0.f);
  }
  for (int e = threadIdx.x; e < WS_H * WS_H; e += blockDim.x) s.w2[e / WS_H][e % WS_H] = __float2bfloat16_rn(p[WS_W2 + e]);
  for (int e = threadIdx.x; e < WS_H * 8; e += blockDim.x) {
    const int k = e / 8, n = e % 8;
    s.w3[k][n] = __float2bfloat16_rn(n < WS_OUT ? p[WS_W3 + k * WS_OUT + n] : 0.f);
  }
  for (int e = threadIdx.x; e < WS_H; e += blockDim.x) {
    s.b1[e] = p[WS_B1 + e];
    s.b2[e] = p[WS_B2 + e];
  }
  if (threadIdx.x < 8) s.b3[threadIdx.x] = threadIdx.x < WS_OUT ? p[WS_B3 + threadIdx.x] : 0.f;
}

// B fragment (16x8, k rows kb.., n columns nb..) of a row-major [k][n] bf16 matrix.
template <int LD>
__device__ __forceinline__ void ws_bfrag(const __nv_bfloat16* w, int kb, int nb, int lane, uint32_t* b) {
  const int g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* col = w + nb + g;
  b[0] = (uint32_t)__bfloat16_as_ushort(col[(kb + 2 * t) * LD]) |
         ((uint32_t)__bfloat16_as_ushort(col[(kb + 2 * t + 1) * LD]) << 16);
  b[1] = (uint32_t)__bfloat16_as_ushort(col[(kb + 2 * t + 8) * LD]) |
         ((uint32_t)__bfloat16_as_ushort(col[(kb + 2 * t + 9) * LD]) << 16);
}

// Forward pass of 16 rows held by one warp.  x: the warp's 16 feature rows
// (row r at x + r * WS_FEAT).  Hidden activations come back in accumulator
// layout (h1[j][4], h2[j][4] for n-tile j; pre-activation values) for the
// backward pass; out[4]: outputs of layer 3 (pre-softplus) for rows g and
// g+8, columns 2t, 2t+1.
__device__ __forceinline__ void ws_forward(const float* x, const WsSmem& s, int lane, float (*h1)[4],
                                           float (*h2)[4], float* out) {
  const int g = lane >> 2, t = lane & 3;
  uint32_t a[4];
  // layer 1: A = x (16 x 16, columns >= 5 zero)
  auto xv = [&](int r, int c) { return c < WS_IN ? x[r * WS_FEAT + c] : 0.f; };
  a[0] = pack_bf16(xv(g, 2 * t), xv(g, 2 * t + 1));
  a[1] = pack_bf16(xv(g + 8, 2 * t), xv(g + 8, 2 * t + 1));
  a[2] = pack_bf16(xv(g, 2 * t + 8), xv(g, 2 * t + 9));
  a[3] = pack_bf16(xv(g + 8, 2 * t + 8), xv(g + 8, 2 * t + 9));
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h1[j][0] = h1[j][2] = s.b1[8 * j + 2 * t];
    h1[j][1] = h1[j][3] = s.b1[8 * j + 2 * t + 1];
    uint32_t b[2];
    ws_bfrag<WS_H>(&s.w1[0][0], 0, 8 * j, lane, b);
    mma_bf16(h1[j], a, b);
  }
  // layer 2: A = relu(h1) in bf16; accumulator tiles 2kk, 2kk+1 form k-step kk
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h2[j][0] = h2[j][2] = s.b2[8 * j + 2 * t];
    h2[j][1] = h2[j][3] = s.b2[8 * j + 2 * t + 1];
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const float* p = h1[2 * kk];
    const float* q = h1[2 * kk + 1];
    a[0] = pack_bf16(fmaxf(p[0], 0.f), fmaxf(p[1], 0.f));
    a[1] = pack_bf16(fmaxf(p[2], 0.f), fmaxf(p[3], 0.f));
    a[2] = pack_bf16(fmaxf(q[0], 0.f), fmaxf(q[1], 0.f));
    a[3] = pack_bf16(fmaxf(q[2], 0.f), fmaxf(q[3], 0.f));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t b[2];
      ws_bfrag<WS_H>(&s.w2[0][0], 16 * kk, 8 * j, lane, b);
      mma_bf16(h2[j], a, b);
    }
  }
  // layer 3
  out[0] = out[2] = s.b3[2 * t];
  out[1] = out[3] = s.b3[2 * t + 1];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const float* p = h2[2 * kk];
    const float* q = h2[2 * kk + 1];
    a[0] = pack_bf16(fmaxf(p[0], 0.f), fmaxf(p[1], 0.f));
    a[1] = pack_bf16(fmaxf(p[2], 0.f), fmaxf(p[3], 0.f));
    a[2] = pack_bf16(fmaxf(q[0], 0.f), fmaxf(q[1], 0.f));
    a[3] = pack_bf16(fmaxf(q[2], 0.f), fmaxf(q[3], 0.f));
    uint32_t b[2];
    ws_bfrag<8>(&s.w3[0][0], 16 * kk, 0, lane, b);
    mma_bf16(out, a, b);
  }
}

__device__ __forceinline__ float softplus(float v) { return v > 20.f ? v : log1pf(expf(v)); }

}  // namespace ccd

namespace ccd {

// ------------------------------------------------------------ features

// Adjacency bitsets adj[u][n_words] (internal labels): an edge is d == 0.
__global__ void k_ws_adjacency(const double* __restrict__ d, const int* __restrict__ tile_list, int ntiles, int n,
                               int B, uint32_t* adj, int words) {
  const int BB = B * B;
  const int64_t total = (int64_t)ntiles * BB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int tl = (int)(e / BB), slot = (int)(e % BB);
    const int pk = tile_list[tl];
    const int I = pk & 0xffff, J = pk >> 16;
    const int i = I * B + slot / B, j = J * B + slot % B;
    if (i < j && j < n && d[e] == 0.0) {
      atomicOr(&adj[(int64_t)i * words + (j >> 5)], 1u << (j & 31));
      atomicOr(&adj[(int64_t)j * words + (i >> 5)], 1u << (i & 31));
    }
  }
}

__global__ void k_ws_degree(const uint32_t* __restrict__ adj, int n, int words, int* deg) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    int s = 0;
    for (int q = 0; q < words; ++q) s += __popc(adj[(int64_t)u * words + q]);
    deg[u] = s;
  }
}

__device__ __forceinline__ bool ws_edge(const uint32_t* adj, int words, int u, int v) {
  return (adj[(int64_t)u * words + (v >> 5)] >> (v & 31)) & 1u;
}

// Candidates with smallest pair (a, b) = pair p: c > b with an edge among
// ab, ac, bc.  mode 0: count them into cnt[p]; mode 1: write them at
// off[p].., packed a | b << 21 | c << 42.
__global__ void k_ws_candidates(const uint32_t* __restrict__ adj, int n, int words, int mode, int* cnt,
                                const int64_t* __restrict__ off, int64_t* out) {
  const int64_t P = ch2(n);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    int a, b;
    pair_unrank(n, p, a, b);
    const bool eab = ws_edge(adj, words, a, b);
    int64_t pos = mode ? off[p] : 0;
    int count = 0;
    for (int q = (b + 1) >> 5; q < words; ++q) {
      uint32_t m = eab ? 0xffffffffu : (adj[(int64_t)a * words + q] | adj[(int64_t)b * words + q]);
      const int base = q * 32;
      if (base <= b) m &= ~((b - base + 1 >= 32) ? 0xffffffffu : ((1u << (b - base + 1)) - 1u));   // c > b
      if (base + 32 > n) m &= (n - base >= 32) ? 0xffffffffu : ((1u << (n - base)) - 1u);       // c < n
      if (mode == 0) {
        count += __popc(m);
      } else {
        while (m) {
          const int c = base + __ffs(m) - 1;
          m &= m - 1;
          out[pos++] = (int64_t)a | ((int64_t)b << 21) | ((int64_t)c << 42);
        }
      }
    }
    if (mode == 0) cnt[p] = count;
  }
}

// Features of each candidate (row stride WS_FEAT).
__global__ void k_ws_features(const int64_t* __restrict__ cand, int64_t count, const double* __restrict__ d,
                              const uint32_t* __restrict__ adj, const int* __restrict__ deg, int n, int nb, int B,
                              int words, float inv_mean_deg, float* feat) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pk = cand[q];
    const int a = (int)(pk & 0x1fffff), b = (int)((pk >> 21) & 0x1fffff), c = (int)(pk >> 42);
    int cab = 0, cac = 0, cbc = 0, c3 = 0;   // common neighbours of each pair and of all three
    for (int w = 0; w < words; ++w) {
      const uint32_t na = adj[(int64_t)a * words + w], nb_ = adj[(int64_t)b * words + w],
                     nc = adj[(int64_t)c * words + w];
      cab += __popc(na & nb_);
      cac += __popc(na & nc);
      cbc += __popc(nb_ & nc);
      c3 += __popc(na & nb_ & nc);
    }
    float* f = feat + q * WS_FEAT;
    f[0] = (float)d[tiled_offset(nb, B, a, b)];
    f[1] = (float)d[tiled_offset(nb, B, a, c)];
    f[2] = (float)d[tiled_offset(nb, B, b, c)];
    f[3] = log1pf((float)deg[a] * inv_mean_deg);
    f[4] = log1pf((float)deg[b] * inv_mean_deg);
    f[5] = log1pf((float)deg[c] * inv_mean_deg);
    f[6] = log1pf((float)cab);
    f[7] = log1pf((float)cac);
    f[8] = log1pf((float)cbc);
    f[9] = log1pf((float)c3);
    f[10] = f[11] = 0.f;
  }
}

// Storage slot (row 0) of internal triplet a<b<c in the tiled dual store;
// rows 1 and 2 follow at +B^2 and +2B^2.
__device__ __forceinline__ int64_t tiled_dual_slot(const int* bt_rank, int nb, int B, int a, int b, int c) {
  const int I = a / B, J = b / B, K = c / B;
  const int la = a % B, lb = b % B, lc = c % B;
  const int t = (la + lb + lc) % B;
  const int64_t w = bt_rank[((int64_t)I * nb + J) * nb + K];
  return w * (3 * (int64_t)B * B * B) + (int64_t)t * (3 * B * B) + la * B + lb;
}

// Every dual whose nonzero bit is set back to zero, and the bits cleared: the
// dense store all zero again after a pass over the bits alone (one thread
// per mask word; bit b of word q is slot 32 q + b of the store).
template <typename T>
__global__ void k_ws_clear_by_mask(uint32_t* mask, T* zt, int64_t nwords) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nwords; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bits = mask[q];
    if (!bits) continue;
    while (bits) {
      const int l = __ffs(bits) - 1;
      bits &= bits - 1;
      zt[q * 32 + l] = T(0);
    }
    mask[q] = 0u;
  }
}

// The duals whose bit is set rounded from an FP64 store into an FP32 store
// (same layout); the other slots of the FP32 store are left as they are.
__global__ void k_ws_round_by_mask(const uint32_t* __restrict__ mask, const double* __restrict__ z64, float* z32,
                                   int64_t nwords) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nwords; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bits = mask[q];
    while (bits) {
      const int l = __ffs(bits) - 1;
      bits &= bits - 1;
      z32[q * 32 + l] = (float)z64[q * 32 + l];
    }
  }
}

// ------------------------------------------------------------ inference

// One warp per 16 candidates.  mode 0: out[3q + r] = softplus(mlp(feat_q))_r;
// mode 1: the same values, below `threshold` set to 0, written as scaled duals
// z = y / eps into the dual store (FP64) at the candidate's slots; with mask
// non-null the nonzero-dual bit of every dual written nonzero is set (the
// mask holds one bit per slot of the store, in the same order).
__global__ void __launch_bounds__(256) k_ws_infer(const float* __restrict__ params, const float* __restrict__ feat,
                                                 int64_t count, int mode, float* out, const int64_t* __restrict__ cand,
                                                 double* zt, const int* __restrict__ bt_rank, int nb, int B,
                                                 double eps, float threshold, uint32_t* mask = nullptr) {
  __shared__ WsSmem s;
  __shared__ float xs[8][16 * WS_FEAT];
  ws_stage_weights(params, s);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t tiles = (count + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * 8 + wid; tile < tiles; tile += (int64_t)gridDim.x * 8) {
    const int64_t r0 = tile * 16;
    for (int e = lane; e < 16 * WS_FEAT; e += 32) {
      const int64_t r = r0 + e / WS_FEAT;
      xs[wid][e] = r < count ? feat[r * WS_FEAT + e % WS_FEAT] : 0.f;
    }
    __syncwarp();
    float h1[8][4], h2[8][4], o[4];
    ws_forward(xs[wid], s, lane, h1, h2, o);
    __syncwarp();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t r = r0 + g + 8 * half;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col = 2 * t + cc;
        if (r >= count || col >= WS_OUT) continue;
        float y = softplus(o[2 * half + cc]);
        if (mode == 0) {
          out[3 * r + col] = y;
        } else {
          if (y < threshold) y = 0.f;
          const int64_t pk = cand[r];
          const int a = (int)(pk & 0x1fffff), b = (int)((pk >> 21) & 0x1fffff), c = (int)(pk >> 42);
          const int64_t gi = tiled_dual_slot(bt_rank, nb, B, a, b, c) + (int64_t)col * B * B;
          zt[gi] = (double)y / eps;
          if (mask && y > 0.f) atomicOr(mask + (gi >> 5), 1u << (gi & 31));
        }
      }
    }
  }
}

// Training targets: the current duals y = eps * z of each candidate.
__global__ void k_ws_targets(const int64_t* __restrict__ cand, int64_t count, const double* __restrict__ zt,
                             const int* __restrict__ bt_rank, int nb, int B, double eps, float* target) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pk = cand[q];
    const int a = (int)(pk & 0x1fffff), b = (int)((pk >> 21) & 0x1fffff), c = (int)(pk >> 42);
    const int64_t s0 = tiled_dual_slot(bt_rank, nb, B, a, b, c);
#pragma unroll
    for (int r = 0; r < 3; ++r) target[3 * q + r] = (float)(eps * zt[s0 + (int64_t)r * B * B]);
  }
}

}  // namespace ccd

namespace ccd {

// ------------------------------------------------------------ training

constexpr int WS_TRAIN_WARPS = 4;

struct WsWarpStage {                 // one warp's 16 rows for the backward pass
  __nv_bfloat16 r1[16][WS_H];        // relu(h1)
  __nv_bfloat16 r2[16][WS_H];        // relu(h2)
  __nv_bfloat16 dh1[16][WS_H];
  __nv_bfloat16 dh2[16][WS_H];
  __nv_bfloat16 dout[16][8];
  __nv_bfloat16 x[16][16];           // features, padded
};

struct WsTrainSmem {
  WsSmem w;
  WsWarpStage st[WS_TRAIN_WARPS];
  float xin[WS_TRAIN_WARPS][16 * WS_FEAT];
  int64_t rowi[WS_TRAIN_WARPS][16];
  float grad[WS_NPARAM];
  float loss;
};

__device__ __forceinline__ uint64_t ws_hash(uint64_t v) {   // SplitMix64 finalizer
  v += 0x9E3779B97F4A7C15ull;
  v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
  v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
  return v ^ (v >> 31);
}

__device__ __forceinline__ uint32_t pk2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A fragment of M^T for a [16 rows][LD] bf16 matrix M: rows of the fragment
// are columns mb.. of M, its k dimension the 16 rows of M.
template <int LD>
__device__ __forceinline__ void ws_afrag_t(const __nv_bfloat16* m, int mb, int lane, uint32_t* a) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = pk2(m[(2 * t) * LD + mb + g], m[(2 * t + 1) * LD + mb + g]);
  a[1] = pk2(m[(2 * t) * LD + mb + g + 8], m[(2 * t + 1) * LD + mb + g + 8]);
  a[2] = pk2(m[(2 * t + 8) * LD + mb + g], m[(2 * t + 9) * LD + mb + g]);
  a[3] = pk2(m[(2 * t + 8) * LD + mb + g + 8], m[(2 * t + 9) * LD + mb + g + 8]);
}

// B fragment (k = the 16 rows, n = columns nb..nb+7) of a [16][LD] bf16 matrix.
template <int LD>
__device__ __forceinline__ void ws_bfrag_rows(const __nv_bfloat16* m, int nb, int lane, uint32_t* b) {
  const int g = lane >> 2, t = lane & 3;
  b[0] = pk2(m[(2 * t) * LD + nb + g], m[(2 * t + 1) * LD + nb + g]);
  b[1] = pk2(m[(2 * t + 8) * LD + nb + g], m[(2 * t + 9) * LD + nb + g]);
}

// One minibatch: gradients of the mean squared error of softplus outputs
// against the targets, summed into grad (global), loss into *loss.
__global__ void __launch_bounds__(32 * WS_TRAIN_WARPS) k_ws_train_grad(
    const float* __restrict__ params, const float* __restrict__ feat, const float* __restrict__ target,
    int64_t count, int64_t rows, int sample, uint64_t seed, float pos_weight, float* grad, float* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WsTrainSmem& S = *reinterpret_cast<WsTrainSmem*>(smem_raw);
  ws_stage_weights(params, S.w);
  for (int e = threadIdx.x; e < WS_NPARAM; e += blockDim.x) S.grad[e] = 0.f;
  if (threadIdx.x == 0) S.loss = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  WsWarpStage& W = S.st[wid];
  float* xs = S.xin[wid];
  const float scale = 1.f / (3.f * (float)rows);
  const int64_t chunks = (rows + 15) / 16;
  int64_t* rowi = S.rowi[wid];
  for (int64_t ch = (int64_t)blockIdx.x * WS_TRAIN_WARPS + wid; ch < chunks; ch += (int64_t)gridDim.x * WS_TRAIN_WARPS) {
    // the chunk's 16 rows: drawn uniformly (sample) or taken in order; -1 past the end
    if (lane < 16) {
      const int64_t idx = ch * 16 + lane;
      rowi[lane] = idx >= rows ? -1
                   : sample ? (int64_t)(ws_hash(seed * 0x100000001B3ull + (uint64_t)idx) % (uint64_t)count)
                            : idx;
    }
    __syncwarp();
    for (int e = lane; e < 16 * WS_FEAT; e += 32) {
      const int64_t r = rowi[e / WS_FEAT];
      xs[e] = r >= 0 ? feat[r * WS_FEAT + e % WS_FEAT] : 0.f;
    }
    __syncwarp();
    float h1[8][4], h2[8][4], o[4];
    ws_forward(xs, S.w, lane, h1, h2, o);
    // output gradient (columns 2t, 2t+1 of rows g, g+8; only the first 3 columns are outputs)
    float dO[4];
    float lsum = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = g + 8 * (q >> 1), col = 2 * t + (q & 1);
      dO[q] = 0.f;
      if (col < WS_OUT && rowi[row] >= 0) {
        const float y = target[rowi[row] * 3 + col];
        const float p = softplus(o[q]);
        const float sig = 1.f / (1.f + expf(-o[q]));
        const float wt = y > 0.f ? pos_weight : 1.f;   // weight of the nonzero targets
        dO[q] = 2.f * (p - y) * scale * sig * wt;
        lsum += wt * (p - y) * (p - y) * scale;
      }
    }
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) atomicAdd(&S.loss, lsum);
    // stage relu activations, output gradient and inputs (bf16)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      W.r1[g][8 * j + 2 * t] = __float2bfloat16_rn(fmaxf(h1[j][0], 0.f));
      W.r1[g][8 * j + 2 * t + 1] = __float2bfloat16_rn(fmaxf(h1[j][1], 0.f));
      W.r1[g + 8][8 * j + 2 * t] = __float2bfloat16_rn(fmaxf(h1[j][2], 0.f));
      W.r1[g + 8][8 * j + 2 * t + 1] = __float2bfloat16_rn(fmaxf(h1[j][3], 0.f));
      W.r2[g][8 * j + 2 * t] = __float2bfloat16_rn(fmaxf(h2[j][0], 0.f));
      W.r2[g][8 * j + 2 * t + 1] = __float2bfloat16_rn(fmaxf(h2[j][1], 0.f));
      W.r2[g + 8][8 * j + 2 * t] = __float2bfloat16_rn(fmaxf(h2[j][2], 0.f));
      W.r2[g + 8][8 * j + 2 * t + 1] = __float2bfloat16_rn(fmaxf(h2[j][3], 0.f));
    }
    W.dout[g][2 * t] = __float2bfloat16_rn(dO[0]);
    W.dout[g][2 * t + 1] = __float2bfloat16_rn(dO[1]);
    W.dout[g + 8][2 * t] = __float2bfloat16_rn(dO[2]);
    W.dout[g + 8][2 * t + 1] = __float2bfloat16_rn(dO[3]);
    for (int e = lane; e < 16 * 16; e += 32) {
      const int r = e / 16, c = e % 16;
      W.x[r][c] = __float2bfloat16_rn(c < WS_IN ? xs[r * WS_FEAT + c] : 0.f);
    }
    __syncwarp();
    // dH2 = (dO W3^T) * relu'(h2)
    float dh2[8][4];
    {
      uint32_t a[4];
      a[0] = pack_bf16(dO[0], dO[1]);
      a[1] = pack_bf16(dO[2], dO[3]);
      a[2] = a[3] = 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        dh2[j][0] = dh2[j][1] = dh2[j][2] = dh2[j][3] = 0.f;
        uint32_t b[2];
        b[0] = pk2(S.w.w3[8 * j + g][2 * t], S.w.w3[8 * j + g][2 * t + 1]);
        b[1] = 0u;
        mma_bf16(dh2[j], a, b);
#pragma unroll
        for (int q = 0; q < 4; ++q) dh2[j][q] = h2[j][q] > 0.f ? dh2[j][q] : 0.f;
      }
    }
    // dH1 = (dH2 W2^T) * relu'(h1)
    float dh1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) dh1[j][0] = dh1[j][1] = dh1[j][2] = dh1[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t a[4];
      a[0] = pack_bf16(dh2[2 * kk][0], dh2[2 * kk][1]);
      a[1] = pack_bf16(dh2[2 * kk][2], dh2[2 * kk][3]);
      a[2] = pack_bf16(dh2[2 * kk + 1][0], dh2[2 * kk + 1][1]);
      a[3] = pack_bf16(dh2[2 * kk + 1][2], dh2[2 * kk + 1][3]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b[2];
        b[0] = pk2(S.w.w2[8 * j + g][16 * kk + 2 * t], S.w.w2[8 * j + g][16 * kk + 2 * t + 1]);
        b[1] = pk2(S.w.w2[8 * j + g][16 * kk + 2 * t + 8], S.w.w2[8 * j + g][16 * kk + 2 * t + 9]);
        mma_bf16(dh1[j], a, b);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int q = 0; q < 4; ++q) dh1[j][q] = h1[j][q] > 0.f ? dh1[j][q] : 0.f;
      W.dh2[g][8 * j + 2 * t] = __float2bfloat16_rn(dh2[j][0]);
      W.dh2[g][8 * j + 2 * t + 1] = __float2bfloat16_rn(dh2[j][1]);
      W.dh2[g + 8][8 * j + 2 * t] = __float2bfloat16_rn(dh2[j][2]);
      W.dh2[g + 8][8 * j + 2 * t + 1] = __float2bfloat16_rn(dh2[j][3]);
      W.dh1[g][8 * j + 2 * t] = __float2bfloat16_rn(dh1[j][0]);
      W.dh1[g][8 * j + 2 * t + 1] = __float2bfloat16_rn(dh1[j][1]);
      W.dh1[g + 8][8 * j + 2 * t] = __float2bfloat16_rn(dh1[j][2]);
      W.dh1[g + 8][8 * j + 2 * t + 1] = __float2bfloat16_rn(dh1[j][3]);
    }
    __syncwarp();
    // bias gradients: column sums over the 16 rows
    for (int c = lane; c < WS_H; c += 32) {
      float s1 = 0.f, s2 = 0.f;
      for (int r = 0; r < 16; ++r) {
        s1 += __bfloat162float(W.dh1[r][c]);
        s2 += __bfloat162float(W.dh2[r][c]);
      }
      atomicAdd(&S.grad[WS_B1 + c], s1);
      atomicAdd(&S.grad[WS_B2 + c], s2);
    }
    if (lane < WS_OUT) {
      float s3 = 0.f;
      for (int r = 0; r < 16; ++r) s3 += __bfloat162float(W.dout[r][lane]);
      atomicAdd(&S.grad[WS_B3 + lane], s3);
    }
    // dW3 = relu(h2)^T dO   (64 x 8)
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      uint32_t a[4], b[2];
      ws_afrag_t<WS_H>(&W.r2[0][0], 16 * mt, lane, a);
      ws_bfrag_rows<8>(&W.dout[0][0], 0, lane, b);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, a, b);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = 16 * mt + g + 8 * (q >> 1), col = 2 * t + (q & 1);
        if (col < WS_OUT) atomicAdd(&S.grad[WS_W3 + row * WS_OUT + col], c[q]);
      }
    }
    // dW2 = relu(h1)^T dH2   (64 x 64)
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      uint32_t a[4];
      ws_afrag_t<WS_H>(&W.r1[0][0], 16 * mt, lane, a);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b[2];
        ws_bfrag_rows<WS_H>(&W.dh2[0][0], 8 * j, lane, b);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(c, a, b);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = 16 * mt + g + 8 * (q >> 1), col = 8 * j + 2 * t + (q & 1);
          atomicAdd(&S.grad[WS_W2 + row * WS_H + col], c[q]);
        }
      }
    }
    // dW1 = x^T dH1   (16 (5 used) x 64)
    {
      uint32_t a[4];
      ws_afrag_t<16>(&W.x[0][0], 0, lane, a);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b[2];
        ws_bfrag_rows<WS_H>(&W.dh1[0][0], 8 * j, lane, b);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(c, a, b);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = g + 8 * (q >> 1), col = 8 * j + 2 * t + (q & 1);
          if (row < WS_IN) atomicAdd(&S.grad[WS_W1 + row * WS_H + col], c[q]);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < WS_NPARAM; e += blockDim.x) atomicAdd(&grad[e], S.grad[e]);
  if (threadIdx.x == 0) atomicAdd(loss, S.loss);
}

// Adam on the FP32 master parameters; clears the gradient.
__global__ void k_ws_adam(float* params, float* m, float* v, float* grad, float lr, float b1, float b2, float eps,
                          int step) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < WS_NPARAM; e += gridDim.x * blockDim.x) {
    const float gr = grad[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr, vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    params[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    grad[e] = 0.f;
  }
}

}  // namespace ccd
