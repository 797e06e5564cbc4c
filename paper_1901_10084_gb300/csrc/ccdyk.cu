// C ABI of the GPU Dykstra solver (declared in include/ccdyk.h): handle
// state, device memory, schedule tables and kernel launches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ccdyk.h"
#include "common.cuh"
#include "tiled.cuh"
#include "listsched.cuh"
#include "warmstart.cuh"

using namespace ccd;

namespace {

thread_local std::string g_create_error;

struct Alloc {
  void* p;
  size_t bytes;
};

}  // namespace

struct cc_handle {
  int64_t n = 0, P = 0, T3 = 0;
  int B = 16, nb = 0, ntiles = 0, nbt = 0, max_bt_phase = 0;
  cc_opts o{};
  cudaStream_t st = nullptr;
  int dev = 0, sms = 0;
  bool unitw = true;
  bool fp32 = false;   // state currently held in FP32 (bulk phase of CC_PREC_FP32_REFINE)
  size_t esz = 8;      // element size of the state
  // device state (element type double, or float while fp32)
  void* x = nullptr;
  void* f = nullptr;
  void* d = nullptr;         // current precision (aliases d64 in FP64)
  void* winv = nullptr;
  double* d64 = nullptr;     // FP64 problem data, kept for the whole solve
  double* winv64 = nullptr;
  int64_t fp32_sweeps = 0;
  int64_t fp64_from = -1;   // sweep count when the state left FP32 (-1: never in this state)
  int var = 0;               // sweep form in use (opts.variant, or the automatic choice)
  void* zt = nullptr;
  void* zp = nullptr;
  int64_t tile_elems = 0;   // ntiles * B * B
  int64_t zt_elems = 0;     // nbt * 3 * B^3
  // schedule tables
  btpk* bt_list = nullptr;
  int* bt_off = nullptr;
  int* tile_list = nullptr;
  int* bt_rank = nullptr;
  uint32_t* mask = nullptr;  // nonzero-dual bits (fused form)
  int64_t mask_words = 0;
  int* flow = nullptr;       // dataflow sweep: item counter + visits per tile
  unsigned long long* trace = nullptr;   // per-item timestamps of the last sweep (opts.trace)
  int* lab = nullptr;        // caller label -> internal label (tiled schedule, opts.interleave)
  int* ilab = nullptr;       // internal label -> caller label (sparse store export)
  // sparse dual store (opts.store = CC_STORE_SPARSE): two pools of entries
  bool sparse = false;
  uint32_t* sp_idx[2] = {nullptr, nullptr};
  void* sp_val[2] = {nullptr, nullptr};      // values in the state's type (float in the FP32 phase)
  long long* sp_off[2] = {nullptr, nullptr};
  int* sp_cnt[2] = {nullptr, nullptr};
  int64_t sp_cap[2] = {0, 0};
  int sp_cur = 0;            // pool read by the next sweep
  unsigned long long* sp_top = nullptr;
  double* sp_scratch = nullptr;   // 3 B^3 doubles per CTA of the sweep
  int sp_scratch_ctas = 0;        // CTAs the scratch holds blocks for
  double* snap = nullptr;    // x, f, pair duals before a sparse sweep
  int64_t sp_nnz = 0;        // entries in the current pool
  int64_t sp_retries = 0;    // sweeps run again after the next pool grew
  bool fresh = false;        // CC state still Algorithm 1's start (x = 0, all duals 0)
  std::vector<int> h_bt_off; // host copy of the phase offsets of the block triples
  // schedules 0 and 1 (device tables)
  ListArgs la{};
  int* l_pre1 = nullptr;
  int64_t* l_phoff = nullptr;
  int* l_sets = nullptr;
  int64_t* l_setoff = nullptr;
  int* l_setidx = nullptr;
  int64_t max_units_phase = 0;
  size_t dyn_smem = 0;       // dynamic shared memory of the sweep kernel
  // scratch
  Ctl* ctl = nullptr;
  double* part = nullptr;    // reduction partials
  int part_cap = 0;
  double* stage = nullptr;   // layout staging
  int64_t stage_elems = 0;
  double* h_pin = nullptr;   // pinned host mirror of the check partials (part_cap * 6)
  int chk_gtri = 0, chk_gpair = 0;
  // launch config
  int sweep_grid = 0, sweep_threads = 0;
  // bookkeeping
  int64_t sweeps = 0;
  cc_stats last{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool ev_recorded = false;
  std::vector<Alloc> allocs;
  int64_t dev_bytes = 0;
  std::string err;
};

namespace {

int fail(cc_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(cc_handle* h, cudaError_t e, const char* what) {
  return fail(h, CC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

void* dalloc(cc_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h->o.alloc) {
    p = h->o.alloc(h->o.alloc_ctx, bytes, h->st);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    h->allocs.push_back({p, bytes});
    h->dev_bytes += (int64_t)bytes;
  }
  return p;
}

void dfree(cc_handle* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    if (h->allocs[i].p == p) {
      h->dev_bytes -= (int64_t)h->allocs[i].bytes;
      h->allocs.erase(h->allocs.begin() + (long)i);
      break;
    }
  }
  if (h->o.free) h->o.free(h->o.alloc_ctx, p, h->st);
  else cudaFree(p);
}

int grid_for(cc_handle* h, int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  g = std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)h->sms * 8));
  return (int)g;
}

// ------------------------------------------------------------ dispatch

template <typename T, bool EXACT, bool UNITW, int B>
void* sweep_kernel_ptr() {
  return (void*)k_sweep_tiled<T, EXACT, UNITW, B>;
}

template <typename T, bool EXACT, bool UNITW>
void* sweep_kernel_b(int B) {
  switch (B) {
    case 8: return sweep_kernel_ptr<T, EXACT, UNITW, 8>();
    case 16: return sweep_kernel_ptr<T, EXACT, UNITW, 16>();
    default: return sweep_kernel_ptr<T, EXACT, UNITW, 32>();
  }
}

int threads_for_tile(int B) { return B * B < 256 ? B * B : 256; }

// warp-per-item kernel: warps per CTA
int warps_per_cta(int B) { return B == 8 ? 8 : 4; }

// CTA-per-item kernel: threads per CTA (variant 3: half of the default for
// B >= 16, so that twice as many block triples are in flight per SM)
int flow_threads(const cc_handle* h) {
  const int full = threads_for_tile(h->B);
  return (h->var == 3 && h->B >= 16) ? full / 2 : full;
}

bool use_warp_kernel(const cc_handle* h) {
  if (h->o.exact || h->B > 16) return false;
  return h->var == 2;
}

template <typename T, bool UNITW>
void* filtered_kernel_b(int B, bool warp, bool half) {
  if (warp) return B == 8 ? (void*)k_sweep_warpflow<T, UNITW, 8> : (void*)k_sweep_warpflow<T, UNITW, 16>;
  switch (B) {
    case 8: return (void*)k_sweep_flow<T, UNITW, 8, 64>;
    case 16: return half ? (void*)k_sweep_flow<T, UNITW, 16, 128> : (void*)k_sweep_flow<T, UNITW, 16, 256>;
    default: return half ? (void*)k_sweep_flow<T, UNITW, 32, 128> : (void*)k_sweep_flow<T, UNITW, 32, 256>;
  }
}

size_t flow_smem(bool fp32, int B) {
  if (fp32) return B == 8 ? sizeof(FlowSmem<float, 8>) : B == 16 ? sizeof(FlowSmem<float, 16>) : sizeof(FlowSmem<float, 32>);
  return B == 8 ? sizeof(FlowSmem<double, 8>) : B == 16 ? sizeof(FlowSmem<double, 16>) : sizeof(FlowSmem<double, 32>);
}

template <typename T, bool EXACT, bool UNITW>
void* list_kernel(int sched) {
  return sched == CC_SCHED_SUMMOD ? (void*)k_sweep_summod<T, EXACT, UNITW> : (void*)k_sweep_diagonal<T, EXACT, UNITW>;
}

// exact form: row-by-row kernel with grid barriers; fused form: filtered dataflow kernel
void* sweep_kernel(cc_handle* h) {
  if (h->o.schedule != CC_SCHED_TILED) {
    const int sc = h->o.schedule;
    if (h->o.exact) return h->unitw ? list_kernel<double, true, true>(sc) : list_kernel<double, true, false>(sc);
    if (h->fp32) return h->unitw ? list_kernel<float, false, true>(sc) : list_kernel<float, false, false>(sc);
    return h->unitw ? list_kernel<double, false, true>(sc) : list_kernel<double, false, false>(sc);
  }
  if (h->o.exact) return h->unitw ? sweep_kernel_b<double, true, true>(h->B) : sweep_kernel_b<double, true, false>(h->B);
  const bool wk = use_warp_kernel(h);
  const bool half = flow_threads(h) != threads_for_tile(h->B);
  if (h->fp32) return h->unitw ? filtered_kernel_b<float, true>(h->B, wk, half) : filtered_kernel_b<float, false>(h->B, wk, half);
  return h->unitw ? filtered_kernel_b<double, true>(h->B, wk, half) : filtered_kernel_b<double, false>(h->B, wk, half);
}


template <typename T>
TiledArgs<T> tiled_args(cc_handle* h) {
  TiledArgs<T> a;
  a.n = (int)h->n;
  a.nb = h->nb;
  a.ntiles = h->ntiles;
  a.x = (T*)h->x;
  a.f = (T*)h->f;
  a.d = (const T*)h->d;
  a.winv = (const T*)h->winv;
  a.zt = (T*)h->zt;
  a.zp = (T*)h->zp;
  a.bt_list = h->bt_list;
  a.bt_off = h->bt_off;
  a.tile_list = h->tile_list;
  a.ctl = h->ctl;
  a.timeout_ns = (long long)(h->o.barrier_timeout_s * 1e9);
  a.eps = (T)h->o.eps;
  a.r_unit = (T)(1.0 / 3.0);
  a.skip_cta = h->o.debug_skip_cta;
  a.mask = h->mask;
  a.nbt = h->nbt;
  a.trace = h->trace;
  a.pairs = h->o.problem == CC_PROB_CC ? 1 : 0;
  a.compact = h->var == 1 ? 1 : 0;
  a.nofilter = h->var == 4 ? 1 : 0;
  a.sparse = h->sparse ? 1 : 0;
  a.zt_elems = (long long)h->zt_elems;
  a.mask_words = (long long)h->mask_words;
  a.sp_cap_cur = h->sparse ? (long long)h->sp_cap[h->sp_cur] : 0;
  a.scratch_ctas = h->sparse ? (long long)h->sp_scratch_ctas : 0;
  if (h->sparse) {
    const int c = h->sp_cur, nx = 1 - c;
    a.sp_idx = h->sp_idx[c];
    a.sp_val = (const T*)h->sp_val[c];
    a.sp_off = h->sp_off[c];
    a.sp_cnt = h->sp_cnt[c];
    a.sp_idx_next = h->sp_idx[nx];
    a.sp_val_next = (T*)h->sp_val[nx];
    a.sp_off_next = h->sp_off[nx];
    a.sp_cnt_next = h->sp_cnt[nx];
    a.sp_top = h->sp_top;
    a.sp_cap = (long long)h->sp_cap[nx];
    a.sp_scratch = (T*)h->sp_scratch;
  } else {
    a.sp_idx = nullptr;
    a.sp_val = nullptr;
    a.sp_off = nullptr;
    a.sp_cnt = nullptr;
    a.sp_idx_next = nullptr;
    a.sp_val_next = nullptr;
    a.sp_off_next = nullptr;
    a.sp_cnt_next = nullptr;
    a.sp_top = nullptr;
    a.sp_cap = 0;
    a.sp_scratch = nullptr;
  }
  return a;
}

// CTAs of the dataflow sweep that stay resident: per-SM occupancy of the
// kernel (at most 8) times the SMs.
int resident_ctas(cc_handle* h, void* k, int threads, size_t smem, int* out) {
  if (smem) CK(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem));
  *out = std::min(per_sm, 8) * h->sms;
  return CC_OK;
}

// opts.variant < 0: the sweep form for this instance and precision.  While a
// phase holds about as many block triples as there are resident CTAs, the
// sweep is paced by the chain of dependent items on each tile, and full-size
// CTAs walk each item fastest (form 0).  When a phase holds at least twice
// as many block triples as form 0 keeps resident, the CTAs are busy with
// items more than they wait, so the form that keeps more CTAs resident wins:
// half-size CTAs (form 3), if more of them fit.  Measured with the Chung-Lu
// instances: n = 1000 form 0 (form 3 11 % slower); n = 2000 form 3 6 % faster
// in FP64, 12 % in FP32; n = 3000 weighted: FP32 21 % faster with form 3, FP64
// form 0 (the weighted half-size FP64 kernel holds no more CTAs).
int choose_variant(cc_handle* h) {
  h->var = 0;
  if (h->o.exact || h->o.schedule != CC_SCHED_TILED || h->B < 16) return CC_OK;
  const size_t smem = flow_smem(h->fp32, h->B);
  const int full = threads_for_tile(h->B);
  int slots0 = 0, slots3 = 0;
  void* k0 = h->fp32 ? (h->unitw ? filtered_kernel_b<float, true>(h->B, false, false)
                                 : filtered_kernel_b<float, false>(h->B, false, false))
                     : (h->unitw ? filtered_kernel_b<double, true>(h->B, false, false)
                                 : filtered_kernel_b<double, false>(h->B, false, false));
  void* k3 = h->fp32 ? (h->unitw ? filtered_kernel_b<float, true>(h->B, false, true)
                                 : filtered_kernel_b<float, false>(h->B, false, true))
                     : (h->unitw ? filtered_kernel_b<double, true>(h->B, false, true)
                                 : filtered_kernel_b<double, false>(h->B, false, true));
  int rc = resident_ctas(h, k0, full, smem, &slots0);
  if (rc) return rc;
  rc = resident_ctas(h, k3, full / 2, smem, &slots3);
  if (rc) return rc;
  if ((int64_t)h->max_bt_phase >= 2 * (int64_t)slots0 && slots3 > slots0) h->var = 3;
  return CC_OK;
}

int configure_sweep(cc_handle* h) {
  h->var = h->o.variant < 0 ? 0 : h->o.variant;
  void* k = sweep_kernel(h);
  if (h->o.schedule != CC_SCHED_TILED) {
    int per_sm = 0;
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0));
    if (per_sm < 1) return fail(h, CC_ERR_CUDA, "sweep kernel does not fit on an SM");
    const int64_t need = std::max<int64_t>(1, (std::max<int64_t>(h->max_units_phase, h->tile_elems / 4) + 255) / 256);
    int g = (int)std::min<int64_t>((int64_t)per_sm * h->sms, need);
    if (h->o.grid > 0) g = std::min(h->o.grid, per_sm * h->sms);
    h->sweep_grid = g;
    h->sweep_threads = 256;
    h->dyn_smem = 0;
    return CC_OK;
  }
  if (h->o.variant < 0) {
    int rc = choose_variant(h);
    if (rc) return rc;
    k = sweep_kernel(h);
  }
  const bool wk = use_warp_kernel(h);
  const int threads = wk ? 32 * warps_per_cta(h->B) : flow_threads(h);
  h->dyn_smem = h->o.exact ? 0 : flow_smem(h->fp32, h->B) * (wk ? warps_per_cta(h->B) : 1);
  if (h->dyn_smem) CK(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->dyn_smem));
  int per_sm = 0;
  CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, h->dyn_smem));
  if (per_sm < 1) return fail(h, CC_ERR_CUDA, "sweep kernel does not fit on an SM");
  int cap = per_sm * h->sms;
  int g;
  if (h->o.grid > 0) g = std::min(h->o.grid, cap);
  else if (h->o.exact) g = std::min(cap, std::max(1, h->max_bt_phase));   // static: one item per CTA
  else g = std::min(per_sm, 8) * h->sms;                                 // dataflow: all resident
  h->sweep_grid = g;
  h->sweep_threads = threads;
  return CC_OK;
}

int read_ctl_error(cc_handle* h);

// Dataflow counters before a sweep.  From Algorithm 1's start of the CC
// problem (x = 0, every dual 0) every metric row has delta = 0 and z = 0, so
// its update is exactly a no-op (z' = max(0 + r * 0, 0) = 0, c = 0, x + 0 = x):
// the first sweep then starts with every tile visited Nb times and the item
// counter past the block triples, and only the pair items run.
int reset_flow(cc_handle* h) {
  if (h->fresh) {
    k_fill<int><<<1, 1, 0, h->st>>>(h->flow, 1, h->nbt);
    k_fill<int><<<grid_for(h, h->ntiles, 256), 256, 0, h->st>>>(h->flow + 1, h->ntiles, h->nb);
    CK(h, cudaGetLastError());
  } else {
    CK(h, cudaMemsetAsync(h->flow, 0, (size_t)(1 + h->ntiles) * sizeof(int), h->st));
  }
  return CC_OK;
}

// One sweep with the sparse store: the current pool is only read, so a sweep
// whose next pool overflows is undone (x, f and the pair duals back from the
// snapshot), the next pool grows to the size the sweep reported, and the sweep
// runs again.  Synchronizes once per sweep.
template <typename T>
int sweep_sparse_t(cc_handle* h) {
  const size_t te = (size_t)h->tile_elems * sizeof(T);
  char* snap = (char*)h->snap;
  void* k = sweep_kernel(h);
  for (int attempt = 0; attempt < 4; ++attempt) {
    CK(h, cudaMemcpyAsync(snap, h->x, te, cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaMemcpyAsync(snap + te, h->f, te, cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaMemcpyAsync(snap + 2 * te, h->zp, 2 * te, cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaMemsetAsync(h->sp_top, 0, sizeof(unsigned long long), h->st));
    int rc0 = reset_flow(h);
    if (rc0) return rc0;
    int* flow = h->flow;
    TiledArgs<T> a = tiled_args<T>(h);
    void* args[] = {&a, &flow};
    CK(h, cudaLaunchCooperativeKernel(k, h->sweep_grid, h->sweep_threads, args, h->dyn_smem, h->st));
    unsigned long long top = 0;
    CK(h, cudaMemcpyAsync(&top, h->sp_top, sizeof top, cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    const int nx = 1 - h->sp_cur;
    if (top <= (unsigned long long)h->sp_cap[nx]) {
      h->sp_cur = nx;
      h->sp_nnz = (int64_t)top;
      return CC_OK;
    }
    int rc = read_ctl_error(h);
    if (rc) return rc;
    CK(h, cudaMemcpyAsync(h->x, snap, te, cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->f, snap + te, te, cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->zp, snap + 2 * te, 2 * te, cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    dfree(h, h->sp_idx[nx]);
    dfree(h, h->sp_val[nx]);
    const int64_t cap = (int64_t)top + (int64_t)top / 2 + 1024;
    h->sp_idx[nx] = (uint32_t*)dalloc(h, (size_t)cap * sizeof(uint32_t));
    h->sp_val[nx] = dalloc(h, (size_t)cap * sizeof(T));
    if (!h->sp_idx[nx] || !h->sp_val[nx]) {
      // capacity 0: a later sweep overflows again and writes nothing
      dfree(h, h->sp_idx[nx]);
      dfree(h, h->sp_val[nx]);
      h->sp_idx[nx] = nullptr;
      h->sp_val[nx] = nullptr;
      h->sp_cap[nx] = 0;
      return fail(h, CC_ERR_OOM, "sparse dual pool");
    }
    h->sp_cap[nx] = cap;
    ++h->sp_retries;
  }
  return fail(h, CC_ERR_OOM, "sparse dual pool keeps overflowing");
}

int sweep_sparse(cc_handle* h) { return h->fp32 ? sweep_sparse_t<float>(h) : sweep_sparse_t<double>(h); }

int launch_sweep(cc_handle* h) {
  void* k = sweep_kernel(h);
  if (h->o.schedule != CC_SCHED_TILED) {
    CK(h, cudaMemsetAsync(&h->ctl->arrive, 0, sizeof(unsigned), h->st));
    ListArgs L = h->la;
    if (h->fp32) {
      TiledArgs<float> a = tiled_args<float>(h);
      void* args[] = {&a, &L};
      CK(h, cudaLaunchCooperativeKernel(k, h->sweep_grid, h->sweep_threads, args, 0, h->st));
    } else {
      TiledArgs<double> a = tiled_args<double>(h);
      void* args[] = {&a, &L};
      CK(h, cudaLaunchCooperativeKernel(k, h->sweep_grid, h->sweep_threads, args, 0, h->st));
    }
    return CC_OK;
  }
  if (h->o.exact) {
    CK(h, cudaMemsetAsync(&h->ctl->arrive, 0, sizeof(unsigned), h->st));
    TiledArgs<double> a = tiled_args<double>(h);
    void* args[] = {&a};
    CK(h, cudaLaunchCooperativeKernel(k, h->sweep_grid, h->sweep_threads, args, 0, h->st));
    return CC_OK;
  }
  if (h->sparse) return sweep_sparse(h);
  int rc0 = reset_flow(h);
  if (rc0) return rc0;
  int* flow = h->flow;
  if (h->fp32) {
    TiledArgs<float> a = tiled_args<float>(h);
    void* args[] = {&a, &flow};
    CK(h, cudaLaunchCooperativeKernel(k, h->sweep_grid, h->sweep_threads, args, h->dyn_smem, h->st));
  } else {
    TiledArgs<double> a = tiled_args<double>(h);
    void* args[] = {&a, &flow};
    CK(h, cudaLaunchCooperativeKernel(k, h->sweep_grid, h->sweep_threads, args, h->dyn_smem, h->st));
  }
  return CC_OK;
}

// ------------------------------------------------------------ tables

int build_tables(cc_handle* h) {
  const int nb = h->nb, B = h->B;
  // the rank table (O(nb^3)) serves the dense store only
  const bool dense = h->o.store == CC_STORE_DENSE;
  std::vector<btpk> list;
  std::vector<int> off(nb + 1, 0), rank(dense ? (size_t)nb * nb * nb : 1, -1), tiles;
  // triplets in block triple (I,J,K): products of block sizes, with
  // binomials where blocks coincide
  auto bsize = [&](int I) { return (int64_t)std::min<int64_t>(B, h->n - (int64_t)I * B); };
  auto count = [&](int I, int J, int K) -> int64_t {
    if (I == J && J == K) return ch3(bsize(I));
    if (I == J) return ch2(bsize(I)) * bsize(K);
    if (J == K) return bsize(I) * ch2(bsize(J));
    return bsize(I) * bsize(J) * bsize(K);
  };
  std::vector<std::pair<int64_t, btpk>> ph;
  for (int g = 0; g < nb; ++g) {
    off[g] = (int)list.size();
    ph.clear();
    for (int I = 0; I < nb; ++I)
      for (int J = I; J < nb; ++J) {
        int K = ((g - I - J) % nb + 2 * nb) % nb;
        if (K < J) continue;
        ph.push_back({-count(I, J, K), pack_bt(I, J, K)});
      }
    // largest first, so that the dynamic distribution ends the phase with
    // the smallest items
    std::stable_sort(ph.begin(), ph.end(),
                     [](const std::pair<int64_t, btpk>& x, const std::pair<int64_t, btpk>& y) { return x.first < y.first; });
    for (auto& e : ph) {
      int I, J, K;
      unpack_bt(e.second, I, J, K);
      if (dense) rank[((size_t)I * nb + J) * nb + K] = (int)list.size();
      list.push_back(e.second);
    }
    h->max_bt_phase = std::max(h->max_bt_phase, (int)list.size() - off[g]);
  }
  off[nb] = (int)list.size();
  h->h_bt_off = off;
  for (int I = 0; I < nb; ++I)
    for (int J = I; J < nb; ++J) tiles.push_back(I | (J << 16));
  h->nbt = (int)list.size();
  h->ntiles = (int)tiles.size();
  h->tile_elems = (int64_t)h->ntiles * B * B;
  h->zt_elems = (int64_t)h->nbt * 3 * B * B * B;
  h->bt_list = (btpk*)dalloc(h, list.size() * sizeof(btpk));
  h->bt_off = (int*)dalloc(h, off.size() * sizeof(int));
  h->bt_rank = (int*)dalloc(h, rank.size() * sizeof(int));
  h->tile_list = (int*)dalloc(h, tiles.size() * sizeof(int));
  if (!h->bt_list || !h->bt_off || !h->bt_rank || !h->tile_list) return fail(h, CC_ERR_OOM, "schedule tables");
  CK(h, cudaMemcpyAsync(h->bt_list, list.data(), list.size() * sizeof(btpk), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaMemcpyAsync(h->bt_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaMemcpyAsync(h->bt_rank, rank.data(), rank.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaMemcpyAsync(h->tile_list, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaStreamSynchronize(h->st));  // host vectors go out of scope
  return CC_OK;
}

// Relabeling of the tiled schedule: the objects are dealt over the blocks in
// rounds (round r gives one object to every block with more than r slots),
// so that objects that are close in the caller's order (e.g. sorted by
// degree) land in different blocks and no tile collects all the activity of
// a dense group.  Caller label i -> internal label lab[i].
int build_labels(cc_handle* h) {
  const int n = (int)h->n, B = h->B, nb = h->nb;
  std::vector<int> lab(n);
  int i = 0;
  for (int r = 0; r < B; ++r)
    for (int b = 0; b < nb; ++b)
      if (std::min<int64_t>(B, h->n - (int64_t)b * B) > r) lab[i++] = b * B + r;
  if (i != n) return fail(h, CC_ERR_ARG, "relabeling does not cover every object");
  h->lab = (int*)dalloc(h, (size_t)n * sizeof(int));
  if (!h->lab) return fail(h, CC_ERR_OOM, "relabeling");
  CK(h, cudaMemcpyAsync(h->lab, lab.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return CC_OK;
}

// Tables of schedules 0 and 1 (O(n^2) integers; no triplet lists).
int build_list_tables(cc_handle* h) {
  const int n = (int)h->n;
  ListArgs& L = h->la;
  L.sched = h->o.schedule;
  L.B = h->B;
  if (L.sched == CC_SCHED_SUMMOD) {
    L.nphases = n;
    std::vector<int> pre1((size_t)n * (n + 1));
    std::vector<int64_t> phoff(n + 1, 0);
    for (int s = 0; s < n; ++s) {
      int run = 0;
      for (int i = 0; i < n; ++i) {
        pre1[(size_t)s * (n + 1) + i] = run;
        for (int q = 0; q < 3; ++q) {
          const int m = s + q * n;
          const int jlo = std::max(i + 1, m - i - n + 1);
          const int jhi = (m - i - 1) >= 0 ? (m - i - 1) / 2 : -1;
          if (jhi >= jlo) run += jhi - jlo + 1;
        }
      }
      pre1[(size_t)s * (n + 1) + n] = run;
      phoff[s + 1] = phoff[s] + run;
      h->max_units_phase = std::max<int64_t>(h->max_units_phase, run);
    }
    if (phoff[n] != h->T3) return fail(h, CC_ERR_ARG, "schedule 1 table does not cover every triplet");
    h->l_pre1 = (int*)dalloc(h, pre1.size() * sizeof(int));
    h->l_phoff = (int64_t*)dalloc(h, phoff.size() * sizeof(int64_t));
    if (!h->l_pre1 || !h->l_phoff) return fail(h, CC_ERR_OOM, "schedule tables");
    CK(h, cudaMemcpyAsync(h->l_pre1, pre1.data(), pre1.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->l_phoff, phoff.data(), phoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
  } else {
    // the sets S_{i,k} (outer pair i < k - 1, 0-based here) grouped by the
    // anti-diagonal i + k: the paper's phases are the 1-based sums n+1 down
    // to 4, then n+2 up to 2n-2, i.e. 0-based sums n-1 down to 2, then n up to
    // 2n-4; inside a phase ascending i, inside a set ascending j
    std::vector<int> sets, setidx((size_t)n * n, -1);
    std::vector<int64_t> setoff, phoff;
    int64_t run = 0;
    auto add_diagonal = [&](int sum) {
      phoff.push_back((int64_t)sets.size());
      int units = 0;
      for (int i = std::max(0, sum - (n - 1)); sum - 2 * i >= 2; ++i, ++units) {
        const int k = sum - i;
        setidx[(size_t)i * n + k] = (int)sets.size();
        sets.push_back(i | (k << 16));
        setoff.push_back(run);
        run += k - i - 1;
      }
      h->max_units_phase = std::max<int64_t>(h->max_units_phase, units);
    };
    for (int sum = n - 1; sum >= 2; --sum) add_diagonal(sum);
    for (int sum = n; sum <= 2 * n - 4; ++sum) add_diagonal(sum);
    L.nphases = (int)phoff.size();
    phoff.push_back((int64_t)sets.size());
    if (run != h->T3) return fail(h, CC_ERR_ARG, "schedule 0 table does not cover every triplet");
    h->l_sets = (int*)dalloc(h, sets.size() * sizeof(int));
    h->l_setoff = (int64_t*)dalloc(h, setoff.size() * sizeof(int64_t));
    h->l_phoff = (int64_t*)dalloc(h, phoff.size() * sizeof(int64_t));
    h->l_setidx = (int*)dalloc(h, setidx.size() * sizeof(int));
    if (!h->l_sets || !h->l_setoff || !h->l_phoff || !h->l_setidx) return fail(h, CC_ERR_OOM, "schedule tables");
    CK(h, cudaMemcpyAsync(h->l_sets, sets.data(), sets.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->l_setoff, setoff.data(), setoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->l_phoff, phoff.data(), phoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->l_setidx, setidx.data(), setidx.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
  }
  L.pre1 = h->l_pre1;
  L.phoff = h->l_phoff;
  L.sets = h->l_sets;
  L.setoff = h->l_setoff;
  L.setidx = h->l_setidx;
  return CC_OK;
}

int ensure_stage(cc_handle* h, int64_t elems) {
  if (h->stage_elems >= elems) return CC_OK;
  dfree(h, h->stage);
  h->stage = (double*)dalloc(h, (size_t)elems * sizeof(double));
  h->stage_elems = h->stage ? elems : 0;
  return h->stage ? CC_OK : fail(h, CC_ERR_OOM, "staging buffer");
}

int read_ctl_error(cc_handle* h) {
  Ctl c;
  CK(h, cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  if (c.err != 0) {
    CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->st));
    CK(h, cudaStreamSynchronize(h->st));
    char buf[160];
    if (c.err == CC_ERR_BOUNDS)
      snprintf(buf, sizeof buf, "an offset outside its buffer was caught by the checked build; the state is undefined");
    else
      snprintf(buf, sizeof buf, "grid barrier time limit hit in phase %d of a sweep; the state is undefined",
               c.err_phase);
    return fail(h, c.err, buf);
  }
  return CC_OK;
}

template <typename T>
int init_state(cc_handle* h) {
  const int th = 256;
  if (h->o.problem == CC_PROB_L2) {
    // Algorithm 1's start -(1/eps) W^{-1} c = d for c = -W d, eps = 1 (FP64 state only)
    CK(h, cudaMemcpyAsync(h->x, h->d64, (size_t)h->tile_elems * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    k_fill<T><<<grid_for(h, h->tile_elems, th), th, 0, h->st>>>((T*)h->f, h->tile_elems, T(0));
  } else {
    k_fill<T><<<grid_for(h, h->tile_elems, th), th, 0, h->st>>>((T*)h->x, h->tile_elems, T(0));
    k_fill<T><<<grid_for(h, h->tile_elems, th), th, 0, h->st>>>((T*)h->f, h->tile_elems, (T)(-1.0 / h->o.eps));
  }
  CK(h, cudaMemsetAsync(h->zt, 0, (size_t)h->zt_elems * sizeof(T), h->st));
  CK(h, cudaMemsetAsync(h->zp, 0, (size_t)h->ntiles * 2 * h->B * h->B * sizeof(T), h->st));
  CK(h, cudaGetLastError());
  return CC_OK;
}

// Sparse store: two pools (entries), their tables, the per-CTA scratch
// blocks (zero), the snapshot for undoing a sweep, and the inverse labels.
int alloc_sparse(cc_handle* h) {
  const int64_t cap = h->o.pool_entries > 0 ? h->o.pool_entries : std::max<int64_t>((int64_t)1 << 20, (int64_t)h->nbt / 2);
  for (int p = 0; p < 2; ++p) {
    h->sp_idx[p] = (uint32_t*)dalloc(h, (size_t)cap * sizeof(uint32_t));
    h->sp_val[p] = dalloc(h, (size_t)cap * h->esz);
    h->sp_off[p] = (long long*)dalloc(h, (size_t)h->nbt * sizeof(long long));
    h->sp_cnt[p] = (int*)dalloc(h, (size_t)h->nbt * sizeof(int));
    if (!h->sp_idx[p] || !h->sp_val[p] || !h->sp_off[p] || !h->sp_cnt[p]) return fail(h, CC_ERR_OOM, "sparse dual pools");
    h->sp_cap[p] = cap;
    CK(h, cudaMemsetAsync(h->sp_cnt[p], 0, (size_t)h->nbt * sizeof(int), h->st));
    CK(h, cudaMemsetAsync(h->sp_off[p], 0, (size_t)h->nbt * sizeof(long long), h->st));
  }
  const size_t scratch = (size_t)h->sweep_grid * 3 * h->B * h->B * h->B;
  h->sp_scratch = (double*)dalloc(h, scratch * sizeof(double));
  h->sp_scratch_ctas = h->sweep_grid;
  h->sp_top = (unsigned long long*)dalloc(h, sizeof(unsigned long long));
  h->snap = (double*)dalloc(h, (size_t)h->tile_elems * 4 * sizeof(double));
  if (!h->sp_scratch || !h->sp_top || !h->snap) return fail(h, CC_ERR_OOM, "sparse store scratch");
  CK(h, cudaMemsetAsync(h->sp_scratch, 0, scratch * sizeof(double), h->st));
  if (h->lab) {
    std::vector<int> lab((size_t)h->n), inv((size_t)h->n);
    CK(h, cudaMemcpyAsync(lab.data(), h->lab, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    for (int64_t i = 0; i < h->n; ++i) inv[(size_t)lab[(size_t)i]] = (int)i;
    h->ilab = (int*)dalloc(h, (size_t)h->n * sizeof(int));
    if (!h->ilab) return fail(h, CC_ERR_OOM, "inverse labels");
    CK(h, cudaMemcpyAsync(h->ilab, inv.data(), (size_t)h->n * sizeof(int), cudaMemcpyHostToDevice, h->st));
  }
  CK(h, cudaStreamSynchronize(h->st));
  h->sp_cur = 0;
  h->sp_nnz = 0;
  return CC_OK;
}

int create_common(cc_handle** out, int64_t n, const double* d_dev, const double* w_dev, const cc_opts* opts,
                  cc_handle* h) {
  h->n = n;
  h->P = ch2(n);
  h->T3 = ch3(n);
  h->B = h->o.tile;
  h->nb = (int)((n + h->B - 1) / h->B);
  // the rank table of the dense store has nb^3 entries; the sparse store has none
  if (h->o.store == CC_STORE_DENSE && h->nb > 1023) return fail(h, CC_ERR_ARG, "n / tile exceeds 1023 blocks");
  if (h->nb > 2047) return fail(h, CC_ERR_ARG, "n / tile exceeds 2047 blocks");
  (void)opts;
  // validate inputs on device
  int* flags = (int*)dalloc(h, 4 * sizeof(int));
  if (!flags) return fail(h, CC_ERR_OOM, "flags");
  CK(h, cudaMemsetAsync(flags, 0, 4 * sizeof(int), h->st));
  k_validate<<<grid_for(h, h->P, 256), 256, 0, h->st>>>(d_dev, w_dev, h->P, flags);
  int hf[4];
  CK(h, cudaMemcpyAsync(hf, flags, sizeof hf, cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  dfree(h, flags);
  if (hf[0]) return fail(h, CC_ERR_ARG, "d has non-finite entries");
  if (hf[1]) return fail(h, CC_ERR_ARG, "w must be finite and > 0");
  h->unitw = hf[2] == 0;
  int rc = build_tables(h);
  if (rc) return rc;
  if (h->o.schedule != CC_SCHED_TILED) {
    rc = build_list_tables(h);
    if (rc) return rc;
    h->zt_elems = 3 * h->T3;   // compact store in schedule order
  } else if (h->o.interleave) {
    rc = build_labels(h);
    if (rc) return rc;
  }
  h->fp32 = h->o.precision == CC_PREC_FP32_REFINE;
  h->esz = h->fp32 ? 4 : 8;
  const size_t te = (size_t)h->tile_elems;
  h->x = dalloc(h, te * h->esz);
  h->f = dalloc(h, te * h->esz);
  h->d64 = (double*)dalloc(h, te * sizeof(double));
  h->winv64 = (double*)dalloc(h, te * sizeof(double));
  if (h->fp32) {
    h->d = dalloc(h, te * sizeof(float));
    h->winv = dalloc(h, te * sizeof(float));
  } else {
    h->d = h->d64;
    h->winv = h->winv64;
  }
  h->zp = dalloc(h, te * 2 * h->esz);
  h->sparse = h->o.store == CC_STORE_SPARSE;
  if (h->sparse) h->zt_elems = 0;
  else h->zt = dalloc(h, (size_t)h->zt_elems * h->esz);
  h->ctl = (Ctl*)dalloc(h, sizeof(Ctl));
  if (!h->o.exact && h->o.schedule == CC_SCHED_TILED) {
    h->mask_words = h->sparse ? 0 : (int64_t)h->nbt * 3 * h->B * ((h->B * h->B) / 32);
    if (!h->sparse) h->mask = (uint32_t*)dalloc(h, (size_t)h->mask_words * sizeof(uint32_t));
    h->flow = (int*)dalloc(h, (size_t)(1 + h->ntiles) * sizeof(int));
    if (h->o.trace) {
      h->trace = (unsigned long long*)dalloc(h, (size_t)(h->nbt + h->ntiles) * 6 * sizeof(unsigned long long));
      if (!h->trace) return fail(h, CC_ERR_OOM, "trace buffer");
      CK(h, cudaMemsetAsync(h->trace, 0, (size_t)(h->nbt + h->ntiles) * 6 * sizeof(unsigned long long), h->st));
    }
    if ((!h->sparse && !h->mask) || !h->flow) return fail(h, CC_ERR_OOM, "dual bitmask");
    if (h->mask) CK(h, cudaMemsetAsync(h->mask, 0, (size_t)h->mask_words * sizeof(uint32_t), h->st));
  }
  h->part_cap = std::max(8 * h->sms, 64);
  h->part = (double*)dalloc(h, (size_t)h->part_cap * 6 * sizeof(double));  // maxima, then 5 sums each
  if (!h->x || !h->f || !h->d64 || !h->winv64 || !h->d || !h->winv || !h->zp || (!h->zt && !h->sparse) || !h->ctl ||
      !h->part)
    return fail(h, CC_ERR_OOM, "device state");
  CK(h, cudaMallocHost((void**)&h->h_pin, (size_t)h->part_cap * 6 * sizeof(double)));
  CK(h, cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->st));
  CK(h, cudaMemsetAsync(h->d64, 0, te * sizeof(double), h->st));
  k_fill<double><<<grid_for(h, te, 256), 256, 0, h->st>>>(h->winv64, te, 1.0);
  k_load_problem<double><<<grid_for(h, h->P, 256), 256, 0, h->st>>>(d_dev, w_dev, (int)n, h->nb, h->B, h->d64,
                                                                     h->winv64, h->lab);
  if (h->fp32) {
    k_convert<double, float><<<grid_for(h, te, 256), 256, 0, h->st>>>(h->d64, (float*)h->d, te);
    k_convert<double, float><<<grid_for(h, te, 256), 256, 0, h->st>>>(h->winv64, (float*)h->winv, te);
    rc = init_state<float>(h);
  } else {
    rc = init_state<double>(h);
  }
  if (rc) return rc;
  // (not while the fault-injection hook is armed: it acts on block triples)
  h->fresh = h->o.problem == CC_PROB_CC && h->o.schedule == CC_SCHED_TILED && !h->o.exact && h->o.debug_skip_cta < 0;
  CK(h, cudaEventCreate(&h->ev0));
  CK(h, cudaEventCreate(&h->ev1));
  rc = configure_sweep(h);
  if (rc) return rc;
  if (h->sparse) {
    rc = alloc_sparse(h);
    if (rc) return rc;
  }
  CK(h, cudaStreamSynchronize(h->st));
  *out = h;
  return CC_OK;
}

int check_opts(const cc_opts& o) {
  if (!(o.eps > 0.0) || !std::isfinite(o.eps)) return fail(nullptr, CC_ERR_ARG, "eps must be finite and > 0");
  if (o.tile != 8 && o.tile != 16 && o.tile != 32) return fail(nullptr, CC_ERR_ARG, "tile must be 8, 16 or 32");
  if (o.schedule != CC_SCHED_TILED && o.schedule != CC_SCHED_SUMMOD && o.schedule != CC_SCHED_DIAGONAL)
    return fail(nullptr, CC_ERR_ARG, "unknown schedule");
  if (o.precision != CC_PREC_FP64 && o.precision != CC_PREC_FP32_REFINE)
    return fail(nullptr, CC_ERR_ARG, "unknown precision");
  if (o.exact && o.precision != CC_PREC_FP64) return fail(nullptr, CC_ERR_ARG, "exact mode needs FP64");
  if (o.precision == CC_PREC_FP32_REFINE && o.schedule != CC_SCHED_TILED)
    return fail(nullptr, CC_ERR_ARG, "the FP32 bulk form runs on the tiled schedule");
  if (o.check_every < 1) return fail(nullptr, CC_ERR_ARG, "check_every must be >= 1");
  if (o.variant < -1 || o.variant > 4) return fail(nullptr, CC_ERR_ARG, "variant must be -1 (automatic) or 0..4");
  if (!(o.barrier_timeout_s > 0.0)) return fail(nullptr, CC_ERR_ARG, "barrier_timeout_s must be > 0");
  if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(nullptr, CC_ERR_ARG, "alloc and free go together");
  if (o.problem != CC_PROB_CC && o.problem != CC_PROB_L2) return fail(nullptr, CC_ERR_ARG, "unknown problem");
  if (o.problem == CC_PROB_L2 && o.precision != CC_PREC_FP64)
    return fail(nullptr, CC_ERR_UNSUPPORTED, "l2 metric nearness runs in FP64");
  if (o.store != CC_STORE_DENSE && o.store != CC_STORE_SPARSE) return fail(nullptr, CC_ERR_ARG, "unknown store");
  if (o.pool_entries < 0) return fail(nullptr, CC_ERR_ARG, "pool_entries must be >= 0");
  if (o.refine_sweeps < 1) return fail(nullptr, CC_ERR_ARG, "refine_sweeps must be >= 1");
  if (o.store == CC_STORE_SPARSE &&
      (o.schedule != CC_SCHED_TILED || o.exact || (o.variant != -1 && o.variant != 0 && o.variant != 3 && o.variant != 4)))
    return fail(nullptr, CC_ERR_UNSUPPORTED, "the sparse store runs the tiled schedule, fused form, variant -1, 0, 3 or 4");
  return CC_OK;
}

int new_handle(cc_handle** out, int64_t n, const cc_opts* opts, cc_handle** hp) {
  if (!out) return fail(nullptr, CC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 3) return fail(nullptr, CC_ERR_ARG, "n must be >= 3");
  if (n > 100000) return fail(nullptr, CC_ERR_ARG, "n too large");
  cc_opts o;
  cc_opts_default(&o);
  if (opts) o = *opts;
  int rc = check_opts(o);
  if (rc) return rc;
  cc_handle* h = new (std::nothrow) cc_handle();
  if (!h) return fail(nullptr, CC_ERR_OOM, "handle");
  h->o = o;
  if (o.problem == CC_PROB_L2) h->o.eps = 1.0;   // Eq. qp with eps = 1, c = -W d
  h->st = (cudaStream_t)o.stream;
  h->dev = o.device;
  cudaError_t e = cudaSetDevice(h->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, CC_ERR_CUDA, std::string("device: ") + cudaGetErrorString(e));
  }
  *hp = h;
  return CC_OK;
}

}  // namespace

// x, f <- v0 - W^{-1} A^T z from the FP64 duals (tiled schedule, fused form).
int resync_fp64(cc_handle* h) {
  const int B = h->B;
  double* x = (double*)h->x;
  CK(h, cudaMemsetAsync(x, 0, (size_t)h->tile_elems * sizeof(double), h->st));
  CK(h, cudaMemsetAsync(&h->ctl->arrive, 0, sizeof(unsigned), h->st));
  const double* zt = (const double*)h->zt;
  const uint32_t* mask = h->mask;
  int nb = h->nb;
  int n = (int)h->n;
  const btpk* bl = h->bt_list;
  const int* bo = h->bt_off;
  Ctl* ctl = h->ctl;
  long long tns = (long long)(h->o.barrier_timeout_s * 1e9);
  SparseIn sp{};
  if (h->sparse) {
    const int c = h->sp_cur;
    sp.idx = h->sp_idx[c];
    sp.val = (const double*)h->sp_val[c];
    sp.off = h->sp_off[c];
    sp.cnt = h->sp_cnt[c];
    sp.scratch = (double*)h->sp_scratch;
  }
  void* args[] = {(void*)&zt, (void*)&mask, (void*)&x, &n, &nb, (void*)&bl, (void*)&bo, (void*)&ctl, &tns, &sp};
  void* k = B == 8 ? (void*)k_resync_metric<8> : B == 16 ? (void*)k_resync_metric<16> : (void*)k_resync_metric<32>;
  const int threads = threads_for_tile(B);
  int per_sm = 0;
  CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0));
  int grid = std::max(1, std::min(per_sm * h->sms, std::max(1, h->max_bt_phase)));
  if (h->sparse) grid = std::min(grid, h->sweep_grid);   // one scratch block per CTA
  CK(h, cudaLaunchCooperativeKernel(k, grid, threads, args, 0, h->st));
  k_resync_finish<<<grid_for(h, h->tile_elems, 256), 256, 0, h->st>>>(x, (double*)h->f, h->winv64,
                                                                       (const double*)h->zp, h->ntiles, B * B,
                                                                       h->o.eps);
  CK(h, cudaGetLastError());
  return read_ctl_error(h);
}

// Leave the FP32 bulk phase: duals to FP64, x and f rebuilt from them in FP64.
int switch_to_fp64(cc_handle* h) {
  if (!h->fp32) return CC_OK;
  int rc = read_ctl_error(h);
  if (rc) return rc;
  const size_t te = (size_t)h->tile_elems;
  double* zt = h->sparse ? nullptr : (double*)dalloc(h, (size_t)h->zt_elems * sizeof(double));
  double* zp = (double*)dalloc(h, te * 2 * sizeof(double));
  double* x = (double*)dalloc(h, te * sizeof(double));
  double* f = (double*)dalloc(h, te * sizeof(double));
  double* pv[2] = {nullptr, nullptr};
  if (h->sparse) {
    pv[0] = (double*)dalloc(h, (size_t)h->sp_cap[0] * sizeof(double));
    pv[1] = (double*)dalloc(h, (size_t)h->sp_cap[1] * sizeof(double));
  }
  if ((!zt && !h->sparse) || !zp || !x || !f || (h->sparse && (!pv[0] || !pv[1]))) {
    dfree(h, zt); dfree(h, zp); dfree(h, x); dfree(h, f); dfree(h, pv[0]); dfree(h, pv[1]);
    return fail(h, CC_ERR_OOM, "FP64 refinement state");
  }
  if (h->sparse) {   // the current pool's values to FP64; the other pool is rewritten by the next sweep
    const int c = h->sp_cur;
    if (h->sp_nnz > 0)
      k_convert<float, double><<<grid_for(h, h->sp_nnz, 256), 256, 0, h->st>>>((const float*)h->sp_val[c], pv[c],
                                                                             h->sp_nnz);
  } else {
    k_convert<float, double><<<grid_for(h, h->zt_elems, 256), 256, 0, h->st>>>((const float*)h->zt, zt, h->zt_elems);
  }
  k_convert<float, double><<<grid_for(h, 2 * te, 256), 256, 0, h->st>>>((const float*)h->zp, zp, 2 * (int64_t)te);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->st));
  dfree(h, h->zt); dfree(h, h->zp); dfree(h, h->x); dfree(h, h->f); dfree(h, h->d); dfree(h, h->winv);
  h->zt = zt; h->zp = zp; h->x = x; h->f = f; h->d = h->d64; h->winv = h->winv64;
  if (h->sparse) {
    dfree(h, h->sp_val[0]);
    dfree(h, h->sp_val[1]);
    h->sp_val[0] = pv[0];
    h->sp_val[1] = pv[1];
  }
  h->fp32 = false;
  h->esz = 8;
  h->fp64_from = h->sweeps;
  rc = resync_fp64(h);
  if (rc) return rc;
  rc = configure_sweep(h);
  if (rc) return rc;
  if (h->sparse && h->sweep_grid > h->sp_scratch_ctas) {   // FP64 grid wider than the FP32 one
    const size_t scratch = (size_t)h->sweep_grid * 3 * h->B * h->B * h->B;
    dfree(h, h->sp_scratch);
    h->sp_scratch = (double*)dalloc(h, scratch * sizeof(double));
    if (!h->sp_scratch) return fail(h, CC_ERR_OOM, "sparse store scratch");
    h->sp_scratch_ctas = h->sweep_grid;
    CK(h, cudaMemsetAsync(h->sp_scratch, 0, scratch * sizeof(double), h->st));
  }
  return CC_OK;
}

// FP64 refinement done: the state never left FP32 in this solve, or has run
// opts.refine_sweeps FP64 sweeps since it did.
static bool refined(const cc_handle* h) {
  return !h->fp32 && (h->fp64_from < 0 || h->sweeps - h->fp64_from >= h->o.refine_sweeps);
}

// Message for cc_last_error(NULL) from entry points outside this file.
void ccd_set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }

// ====================================================================== ABI

extern "C" {

void cc_opts_default(cc_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->eps = 0.2;
  o->schedule = CC_SCHED_TILED;
  o->tile = 16;
  o->precision = CC_PREC_FP64;
  o->exact = 0;
  o->check_every = 10;
  o->device = 0;
  o->barrier_timeout_s = 2.0;
  o->stream = nullptr;
  o->alloc = nullptr;
  o->free = nullptr;
  o->alloc_ctx = nullptr;
  o->grid = 0;
  o->debug_skip_cta = -1;
  o->variant = -1;
  o->refine_at = 1e-5;
  o->trace = 0;
  o->interleave = 1;
  o->batch_order = 0;
  o->problem = CC_PROB_CC;
  o->store = CC_STORE_DENSE;
  o->pool_entries = 0;
  o->refine_sweeps = 5;
}

int cc_create_device(cc_handle** out, int64_t n, const double* d_dev, const double* w_dev, const cc_opts* opts) {
  cc_handle* h = nullptr;
  int rc = new_handle(out, n, opts, &h);
  if (rc) return rc;
  if (!d_dev || !w_dev) {
    cc_destroy(h);
    return fail(nullptr, CC_ERR_ARG, "d or w is NULL");
  }
  rc = create_common(out, n, d_dev, w_dev, opts, h);
  if (rc) {
    g_create_error = h->err;
    cc_destroy(h);
    *out = nullptr;
  }
  return rc;
}

int cc_create(cc_handle** out, int64_t n, const double* d, const double* w, const cc_opts* opts) {
  cc_handle* h = nullptr;
  int rc = new_handle(out, n, opts, &h);
  if (rc) return rc;
  if (!d || !w) {
    cc_destroy(h);
    return fail(nullptr, CC_ERR_ARG, "d or w is NULL");
  }
  const int64_t P = ch2(n);
  double* buf = (double*)dalloc(h, (size_t)P * 2 * sizeof(double));
  if (!buf) {
    cc_destroy(h);
    return fail(nullptr, CC_ERR_OOM, "input staging");
  }
  cudaError_t e = cudaMemcpyAsync(buf, d, P * sizeof(double), cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + P, w, P * sizeof(double), cudaMemcpyHostToDevice, h->st);
  if (e != cudaSuccess) {
    cc_destroy(h);
    return fail(nullptr, CC_ERR_CUDA, std::string("input upload: ") + cudaGetErrorString(e));
  }
  rc = create_common(out, n, buf, buf + P, opts, h);
  if (rc) {
    g_create_error = h->err;
    cc_destroy(h);
    *out = nullptr;
    return rc;
  }
  dfree(h, buf);
  return CC_OK;
}

int cc_pair_passes(cc_handle* h, int32_t passes) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (passes < 0) return fail(h, CC_ERR_ARG, "passes must be >= 0");
  if (h->o.schedule != CC_SCHED_TILED) return fail(h, CC_ERR_UNSUPPORTED, "pair passes need the tiled schedule");
  if (h->o.problem == CC_PROB_L2 || passes == 0) return CC_OK;   // l2 nearness has no pair rows
  CK(h, cudaSetDevice(h->dev));
  const int grid = grid_for(h, (int64_t)h->ntiles * h->B * h->B, 256);
  if (h->fp32) {
    TiledArgs<float> a = tiled_args<float>(h);
    if (h->B == 8) k_pair_passes<float, false, 8><<<grid, 256, 0, h->st>>>(a, passes);
    else if (h->B == 16) k_pair_passes<float, false, 16><<<grid, 256, 0, h->st>>>(a, passes);
    else k_pair_passes<float, false, 32><<<grid, 256, 0, h->st>>>(a, passes);
  } else {
    TiledArgs<double> a = tiled_args<double>(h);
    if (h->o.exact) {
      if (h->B == 8) k_pair_passes<double, true, 8><<<grid, 256, 0, h->st>>>(a, passes);
      else if (h->B == 16) k_pair_passes<double, true, 16><<<grid, 256, 0, h->st>>>(a, passes);
      else k_pair_passes<double, true, 32><<<grid, 256, 0, h->st>>>(a, passes);
    } else {
      if (h->B == 8) k_pair_passes<double, false, 8><<<grid, 256, 0, h->st>>>(a, passes);
      else if (h->B == 16) k_pair_passes<double, false, 16><<<grid, 256, 0, h->st>>>(a, passes);
      else k_pair_passes<double, false, 32><<<grid, 256, 0, h->st>>>(a, passes);
    }
  }
  CK(h, cudaGetLastError());
  h->fresh = false;
  return CC_OK;
}

int cc_sweep(cc_handle* h, int64_t k) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (k < 0) return fail(h, CC_ERR_ARG, "k must be >= 0");
  CK(h, cudaSetDevice(h->dev));
  for (int64_t s = 0; s < k; ++s) {
    const bool last = (s == k - 1);
    if (last) CK(h, cudaEventRecord(h->ev0, h->st));
    int rc = launch_sweep(h);
    if (rc) return rc;
    h->fresh = false;
    if (last) {
      CK(h, cudaEventRecord(h->ev1, h->st));
      h->ev_recorded = true;
    }
    h->sweeps++;
    h->fresh = false;
    if (h->fp32) h->fp32_sweeps++;
  }
  return CC_OK;
}

}  // extern "C"

namespace {

// Convergence check in two halves: the launch queues the reduction kernels and
// the copy of their partials into pinned host memory on the handle's stream;
// the finish (after the stream is synchronized) folds the partials.
int check_launch(cc_handle* h) {
  const int B = h->B;
  const int gtri = std::min(h->part_cap, h->sms * 4);
  const int gpair = std::min(h->part_cap, grid_for(h, h->tile_elems, 256));
  h->chk_gtri = gtri;
  h->chk_gpair = gpair;
  double* pm = h->part;                        // gtri maxima
  double* ps = h->part + h->part_cap;          // gpair x 5 sums
  const double yscale = h->o.exact ? 1.0 : h->o.eps;
#define LAUNCH_CHECK(T, BV)                                                                                   \
  k_maxviol_tiled<T, BV><<<gtri, threads_for_tile(BV), 0, h->st>>>((const T*)h->x, (int)h->n, h->nb,      \
                                                                    h->bt_list, h->nbt, pm);                \
  k_pairsums_tiled<T, BV><<<gpair, 256, 0, h->st>>>((const T*)h->x, (const T*)h->f, h->d64,                 \
                                                    h->winv64, (const T*)h->zp, h->tile_list,              \
                                                    h->ntiles, (int)h->n, yscale,                \
                                                    h->o.problem == CC_PROB_L2 ? 1 : 0, ps);
  if (h->fp32) {
    if (B == 8) { LAUNCH_CHECK(float, 8) } else if (B == 16) { LAUNCH_CHECK(float, 16) } else { LAUNCH_CHECK(float, 32) }
  } else {
    if (B == 8) { LAUNCH_CHECK(double, 8) } else if (B == 16) { LAUNCH_CHECK(double, 16) } else { LAUNCH_CHECK(double, 32) }
  }
#undef LAUNCH_CHECK
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(h->h_pin, pm, gtri * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(h->h_pin + h->part_cap, ps, (size_t)gpair * 5 * sizeof(double), cudaMemcpyDeviceToHost,
                        h->st));
  return CC_OK;
}

void check_finish(cc_handle* h, cc_stats* st) {
  const double* hm = h->h_pin;
  const double* hs = h->h_pin + h->part_cap;
  double mv = 0, lp = 0, wf = 0, quad = 0, by = 0, pv = 0;
  for (int i = 0; i < h->chk_gtri; ++i) mv = std::max(mv, hm[i]);
  for (int i = 0; i < h->chk_gpair; ++i) {
    lp += hs[5 * i];
    wf += hs[5 * i + 1];
    quad += hs[5 * i + 2];
    by += hs[5 * i + 3];
    pv = std::max(pv, hs[5 * i + 4]);
  }
  cc_stats& s = h->last;
  s.sweeps = h->sweeps;
  s.fp32_sweeps = h->fp32_sweeps;
  s.dual_nnz = h->sparse ? h->sp_nnz : -1;
  s.pool_retries = h->sp_retries;
  s.variant = h->var;
  s.state_fp32 = h->fp32 ? 1 : 0;
  s.max_violation = mv;
  s.pair_violation = pv;
  if (h->o.problem == CC_PROB_L2) {
    // lp = sum w (x - d)^2, wf = sum w d (d - x); dual through A^T y = W (d - x)
    s.lp_objective = lp;
    s.wf = 0.0;
    s.pair_violation = 0.0;
    s.qp_primal = 0.5 * lp;
    s.dual_objective = wf - 0.5 * lp;
  } else {
    s.lp_objective = lp;
    s.wf = wf;
    s.qp_primal = wf + 0.5 * h->o.eps * quad;
    s.dual_objective = -by - 0.5 * h->o.eps * quad;
  }
  s.gap = s.qp_primal - s.dual_objective;
  if (h->ev_recorded) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) s.last_sweep_ms = ms;
  }
  if (st) *st = s;
}

}  // namespace

extern "C" {

int cc_check(cc_handle* h, cc_stats* st) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  rc = check_launch(h);
  if (rc) return rc;
  CK(h, cudaStreamSynchronize(h->st));
  check_finish(h, st);
  return CC_OK;
}

int cc_solve(cc_handle* h, double tol, int64_t max_sweeps, int64_t* sweeps_done) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (!std::isfinite(tol) || tol < 0) return fail(h, CC_ERR_ARG, "tol must be finite and >= 0");
  if (max_sweeps < 0) return fail(h, CC_ERR_ARG, "max_sweeps must be >= 0");
  int64_t done = 0;
  if (sweeps_done) *sweeps_done = 0;
  double prev_fp32 = INFINITY;
  while (done < max_sweeps) {
    int64_t k = std::min<int64_t>(h->o.check_every, max_sweeps - done);
    int rc = cc_sweep(h, k);
    if (rc) return rc;
    done += k;
    if (sweeps_done) *sweeps_done = done;
    cc_stats s;
    rc = cc_check(h, &s);
    if (rc) return rc;
    if (h->fp32) {
      // FP32 bulk phase: go to FP64 (duals converted, x and f rebuilt from
      // them) once the violation is small enough for FP32, or stops
      // decreasing near that level (early plateaus of Dykstra's violation
      // are not FP32's floor); then run the refinement sweeps in FP64 at
      // once: the rebuilt point carries the FP32 duals' rounding (its LP
      // objective about 1e-5 off), which a few FP64 sweeps remove
      const double at = std::max(tol, h->o.refine_at);
      const bool small = s.max_violation <= at;
      const bool stalled = s.max_violation <= 100.0 * at && s.max_violation > 0.99 * prev_fp32;
      prev_fp32 = s.max_violation;
      if (!(small || stalled)) continue;
      rc = switch_to_fp64(h);
      if (rc) return rc;
      k = std::min<int64_t>(h->o.refine_sweeps, max_sweeps - done);
      rc = cc_sweep(h, k);
      if (rc) return rc;
      done += k;
      if (sweeps_done) *sweeps_done = done;
      rc = cc_check(h, &s);
      if (rc) return rc;
    }
    // l2 nearness also needs the gap closed: Dykstra's iterate is often
    // feasible long before it is optimal (gap = sum w x (x - d) >= 0 at the optimum)
    if (s.max_violation <= tol && refined(h) &&
        (h->o.problem != CC_PROB_L2 || std::fabs(s.gap) <= tol * std::max(s.qp_primal, 1e-300)))
      return CC_OK;
  }
  return fail(h, CC_ERR_NOT_CONVERGED, "max_sweeps reached before the tolerance");
}

int cc_get_x(cc_handle* h, double* x, double* f) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (!x && !f) return fail(h, CC_ERR_ARG, "x and f are both NULL");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  rc = ensure_stage(h, 2 * h->P);
  if (rc) return rc;
  double* sx = h->stage;
  double* sf = h->stage + h->P;
  const int g = grid_for(h, h->P, 256);
  if (h->fp32)
    k_pairs_layout<float><<<g, 256, 0, h->st>>>((float*)h->x, (float*)h->f, (int)h->n, h->nb, h->B, sx, sf, 0, h->lab);
  else
    k_pairs_layout<double><<<g, 256, 0, h->st>>>((double*)h->x, (double*)h->f, (int)h->n, h->nb, h->B, sx, sf, 0, h->lab);
  CK(h, cudaGetLastError());
  if (x) CK(h, cudaMemcpyAsync(x, sx, h->P * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (f) CK(h, cudaMemcpyAsync(f, sf, h->P * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return CC_OK;
}

static int move_duals(cc_handle* h, double* y_tri, double* y_pair, int64_t first, int64_t count, int dir) {
  const double scale = h->o.exact ? 1.0 : h->o.eps;
  if (h->sparse && dir == 1 && y_tri) return fail(h, CC_ERR_UNSUPPORTED, "the sparse store does not import duals");
  const int64_t chunk = std::min<int64_t>(std::max<int64_t>(count, 1), (int64_t)1 << 22);
  int rc = ensure_stage(h, std::max<int64_t>(3 * chunk, 2 * h->P));
  if (rc) return rc;
  if (y_tri) {
    for (int64_t c0 = 0; c0 < count; c0 += chunk) {
      const int64_t m = std::min(chunk, count - c0);
      if (dir == 1)
        CK(h, cudaMemcpyAsync(h->stage, y_tri + 3 * c0, 3 * m * sizeof(double), cudaMemcpyHostToDevice, h->st));
      const int g = grid_for(h, m, 256);
      if (h->sparse) {
        CK(h, cudaMemsetAsync(h->stage, 0, 3 * m * sizeof(double), h->st));
        const int gw = grid_for(h, h->nbt, 128);
        const int c = h->sp_cur;
#define LAUNCH_SP(T, BV)                                                                                       \
  k_tri_duals_sparse<T, BV><<<gw, 128, 0, h->st>>>(h->sp_idx[c], (const T*)h->sp_val[c], h->sp_off[c],          \
                                                  h->sp_cnt[c], h->bt_list, h->nbt, (int)h->n, h->ilab,         \
                                                  first + c0, m, h->stage, scale);
        if (h->fp32) {
          if (h->B == 8) { LAUNCH_SP(float, 8) } else if (h->B == 16) { LAUNCH_SP(float, 16) } else { LAUNCH_SP(float, 32) }
        } else {
          if (h->B == 8) { LAUNCH_SP(double, 8) } else if (h->B == 16) { LAUNCH_SP(double, 16) } else { LAUNCH_SP(double, 32) }
        }
#undef LAUNCH_SP
        CK(h, cudaGetLastError());
        CK(h, cudaMemcpyAsync(y_tri + 3 * c0, h->stage, 3 * m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        continue;
      }
      if (h->o.schedule != CC_SCHED_TILED) {
        if (h->fp32)
          k_tri_duals_list<float><<<g, 256, 0, h->st>>>((float*)h->zt, h->la, (int)h->n, first + c0, m, h->stage, scale, dir);
        else
          k_tri_duals_list<double><<<g, 256, 0, h->st>>>((double*)h->zt, h->la, (int)h->n, first + c0, m, h->stage, scale, dir);
        CK(h, cudaGetLastError());
        if (dir == 0)
          CK(h, cudaMemcpyAsync(y_tri + 3 * c0, h->stage, 3 * m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        continue;
      }
#define LAUNCH_TD(T, BV) \
  k_tri_duals_tiled<T, BV><<<g, 256, 0, h->st>>>((T*)h->zt, h->bt_rank, (int)h->n, h->nb, first + c0, m, h->stage, scale, dir, h->lab);
      if (h->fp32) {
        if (h->B == 8) { LAUNCH_TD(float, 8) } else if (h->B == 16) { LAUNCH_TD(float, 16) } else { LAUNCH_TD(float, 32) }
      } else {
        if (h->B == 8) { LAUNCH_TD(double, 8) } else if (h->B == 16) { LAUNCH_TD(double, 16) } else { LAUNCH_TD(double, 32) }
      }
#undef LAUNCH_TD
      CK(h, cudaGetLastError());
      if (dir == 0)
        CK(h, cudaMemcpyAsync(y_tri + 3 * c0, h->stage, 3 * m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(h, cudaStreamSynchronize(h->st));
    }
  }
  if (y_pair) {
    if (dir == 1)
      CK(h, cudaMemcpyAsync(h->stage, y_pair, 2 * h->P * sizeof(double), cudaMemcpyHostToDevice, h->st));
    const int g = grid_for(h, h->P, 256);
    if (h->fp32)
      k_pair_duals_tiled<float><<<g, 256, 0, h->st>>>((float*)h->zp, (int)h->n, h->nb, h->B, h->stage, scale, dir, h->lab);
    else
      k_pair_duals_tiled<double><<<g, 256, 0, h->st>>>((double*)h->zp, (int)h->n, h->nb, h->B, h->stage, scale, dir, h->lab);
    CK(h, cudaGetLastError());
    if (dir == 0)
      CK(h, cudaMemcpyAsync(y_pair, h->stage, 2 * h->P * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
  }
  return CC_OK;
}

int cc_get_duals(cc_handle* h, double* y_tri, double* y_pair, int64_t tri_first, int64_t tri_count) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (y_tri && (tri_first < 0 || tri_count < 0 || tri_first + tri_count > h->T3))
    return fail(h, CC_ERR_ARG, "triplet range out of bounds");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  return move_duals(h, y_tri, y_pair, tri_first, tri_count, 0);
}

int cc_set_state(cc_handle* h, const double* x, const double* f, const double* y_tri, const double* y_pair) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (!x || !f || !y_tri || !y_pair) return fail(h, CC_ERR_ARG, "all four arrays are required");
  if (h->sparse) return fail(h, CC_ERR_UNSUPPORTED, "the sparse store does not import duals");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  rc = ensure_stage(h, 2 * h->P);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(h->stage, x, h->P * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaMemcpyAsync(h->stage + h->P, f, h->P * sizeof(double), cudaMemcpyHostToDevice, h->st));
  const int g = grid_for(h, h->P, 256);
  if (h->fp32)
    k_pairs_layout<float><<<g, 256, 0, h->st>>>((float*)h->x, (float*)h->f, (int)h->n, h->nb, h->B, h->stage,
                                                h->stage + h->P, 1, h->lab);
  else
    k_pairs_layout<double><<<g, 256, 0, h->st>>>((double*)h->x, (double*)h->f, (int)h->n, h->nb, h->B, h->stage,
                                                 h->stage + h->P, 1, h->lab);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->st));
  rc = move_duals(h, const_cast<double*>(y_tri), const_cast<double*>(y_pair), 0, h->T3, 1);
  if (rc) return rc;
  if (h->mask) {
    const int g2 = grid_for(h, h->mask_words, 256);
#define LAUNCH_RM(T, BV) k_rebuild_mask<T, BV><<<g2, 256, 0, h->st>>>((const T*)h->zt, h->mask, h->mask_words);
    if (h->fp32) {
      if (h->B == 8) { LAUNCH_RM(float, 8) } else if (h->B == 16) { LAUNCH_RM(float, 16) } else { LAUNCH_RM(float, 32) }
    } else {
      if (h->B == 8) { LAUNCH_RM(double, 8) } else if (h->B == 16) { LAUNCH_RM(double, 16) } else { LAUNCH_RM(double, 32) }
    }
#undef LAUNCH_RM
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->st));
  }
  h->sweeps = 0;
  h->fp64_from = -1;   // a state set by the caller needs no refinement sweeps
  h->fresh = false;
  return CC_OK;
}

int cc_refine_fp64(cc_handle* h) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  CK(h, cudaSetDevice(h->dev));
  return switch_to_fp64(h);
}

int cc_set_duals(cc_handle* h, const double* y_tri, const double* y_pair) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (!y_tri || !y_pair) return fail(h, CC_ERR_ARG, "y_tri and y_pair are required");
  if (h->o.schedule != CC_SCHED_TILED || h->o.exact || h->fp32 || h->o.problem != CC_PROB_CC || h->sparse)
    return fail(h, CC_ERR_UNSUPPORTED,
                "cc_set_duals needs the CC problem, tiled schedule, fused form, FP64 state, dense store");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  rc = move_duals(h, const_cast<double*>(y_tri), const_cast<double*>(y_pair), 0, h->T3, 1);
  if (rc) return rc;
  const int g2 = grid_for(h, h->mask_words, 256);
  if (h->B == 8) k_rebuild_mask<double, 8><<<g2, 256, 0, h->st>>>((const double*)h->zt, h->mask, h->mask_words);
  else if (h->B == 16) k_rebuild_mask<double, 16><<<g2, 256, 0, h->st>>>((const double*)h->zt, h->mask, h->mask_words);
  else k_rebuild_mask<double, 32><<<g2, 256, 0, h->st>>>((const double*)h->zt, h->mask, h->mask_words);
  CK(h, cudaGetLastError());
  rc = resync_fp64(h);
  if (rc) return rc;
  h->sweeps = 0;
  h->fp64_from = -1;   // a state set by the caller needs no refinement sweeps
  h->fresh = false;
  h->fp32_sweeps = 0;
  return CC_OK;
}

int64_t cc_get_trace(cc_handle* h, uint64_t* out, int64_t cap) {
  if (!h || !h->trace) return 0;
  const int64_t items = (int64_t)h->nbt + h->ntiles;
  if (!out) return items;
  const int64_t m = std::min(cap, items);
  if (cudaMemcpyAsync(out, h->trace, (size_t)m * 6 * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return -1;
  return m;
}

int cc_get_stats(cc_handle* h, cc_stats* st) {
  if (!h || !st) return fail(h, CC_ERR_ARG, "NULL argument");
  *st = h->last;
  st->sweeps = h->sweeps;
  st->fp32_sweeps = h->fp32_sweeps;
  st->state_fp32 = h->fp32 ? 1 : 0;
  st->dual_nnz = h->sparse ? h->sp_nnz : -1;
  st->pool_retries = h->sp_retries;
  st->variant = h->var;
  return CC_OK;
}

int64_t cc_device_bytes(const cc_handle* h) { return h ? h->dev_bytes : 0; }

void cc_destroy(cc_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
  while (!h->allocs.empty()) dfree(h, h->allocs.back().p);
  if (h->h_pin) cudaFreeHost(h->h_pin);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

const char* cc_last_error(const cc_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

}  // extern "C"

// ====================================================================== batch
//
// Many instances of uneven size in one launch per sweep (k_sweep_batch): a
// batch owns ordinary handles (same options: tiled schedule, fused form,
// same tile) and drains one queue of work items from all instances that are
// still active.  Instances in FP32 state and in FP64 state run in separate
// launches of the same sweep.

struct cc_batch {
  std::vector<cc_handle*> hs;
  std::vector<char> active;
  std::vector<double> prev_fp32;       // last FP32 violation per instance (stall test)
  cc_opts o{};
  cudaStream_t st = nullptr;
  int dev = 0, sms = 0;
  bool unitw = true;
  // device buffers, allocated through hs[0]'s allocator
  void* args[2] = {nullptr, nullptr};  // TiledArgs<double>, TiledArgs<float> per instance
  int2* items[2] = {nullptr, nullptr};
  int nitems[2] = {0, 0};
  bool stale[2] = {true, true};
  int* cnt = nullptr;                  // [0]: item counter; then every instance's tile counters
  std::vector<int64_t> cnt_off;
  int64_t cnt_total = 0;
  int64_t sweeps = 0;
  std::string err;
};

namespace {

int bfail(cc_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg; else g_create_error = msg;
  return code;
}

#define BCK(b, call)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return bfail(b, CC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Work-item list of one precision group: (instance, local item).  Order 0
// ("phase-major"): phase g of every instance, g = 0, 1, ..., then all pair
// tiles; order 1 ("instance-major"): every instance's items in turn.  Both
// keep each instance's items in its own order.
void build_items(cc_batch* b, bool fp32, std::vector<int2>& out) {
  out.clear();
  std::vector<int> ids;
  int maxnb = 0;
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (b->active[i] && b->hs[i]->fp32 == fp32) {
      ids.push_back((int)i);
      maxnb = std::max(maxnb, b->hs[i]->nb);
    }
  if (b->o.batch_order == 1) {
    for (int i : ids) {
      const cc_handle* h = b->hs[i];
      for (int w = 0; w < h->nbt + h->ntiles; ++w) out.push_back(make_int2(i, w));
    }
    return;
  }
  for (int g = 0; g < maxnb; ++g)
    for (int i : ids) {
      const cc_handle* h = b->hs[i];
      if (g >= h->nb) continue;
      for (int w = h->h_bt_off[g]; w < h->h_bt_off[g + 1]; ++w) out.push_back(make_int2(i, w));
    }
  for (int i : ids) {
    const cc_handle* h = b->hs[i];
    for (int tl = 0; tl < h->ntiles; ++tl) out.push_back(make_int2(i, h->nbt + tl));
  }
}

template <typename T>
int upload_group(cc_batch* b, int gi) {
  const bool fp32 = gi == 1;
  std::vector<TiledArgs<T>> args(b->hs.size());
  for (size_t i = 0; i < b->hs.size(); ++i) {
    cc_handle* h = b->hs[i];
    if (h->fp32 != fp32) continue;
    args[i] = tiled_args<T>(h);
    args[i].cnt = b->cnt + b->cnt_off[i];
    args[i].trace = nullptr;
    args[i].skip_cta = -1;
  }
  std::vector<int2> items;
  build_items(b, fp32, items);
  cc_handle* h0 = b->hs[0];
  if (!b->args[gi]) {
    b->args[gi] = dalloc(h0, args.size() * sizeof(TiledArgs<T>));
    if (!b->args[gi]) return bfail(b, CC_ERR_OOM, "batch arguments");
  }
  if (b->items[gi]) dfree(h0, b->items[gi]);
  b->items[gi] = (int2*)dalloc(h0, std::max<size_t>(1, items.size()) * sizeof(int2));
  if (!b->items[gi]) return bfail(b, CC_ERR_OOM, "batch work list");
  BCK(b, cudaMemcpyAsync(b->args[gi], args.data(), args.size() * sizeof(TiledArgs<T>), cudaMemcpyHostToDevice, b->st));
  if (!items.empty())
    BCK(b, cudaMemcpyAsync(b->items[gi], items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, b->st));
  BCK(b, cudaStreamSynchronize(b->st));
  b->nitems[gi] = (int)items.size();
  b->stale[gi] = false;
  return CC_OK;
}

template <typename T, bool UNITW, int B>
void* batch_kernel() {
  return (void*)k_sweep_batch<T, UNITW, B, TileCfg<B>::NT>;
}

template <typename T>
void* batch_kernel_b(bool unitw, int B) {
  if (unitw) return B == 8 ? batch_kernel<T, true, 8>() : B == 16 ? batch_kernel<T, true, 16>() : batch_kernel<T, true, 32>();
  return B == 8 ? batch_kernel<T, false, 8>() : B == 16 ? batch_kernel<T, false, 16>() : batch_kernel<T, false, 32>();
}

// One sweep of every active instance of one precision group.
int batch_launch(cc_batch* b, int gi) {
  int rc = CC_OK;
  if (b->stale[gi]) rc = gi ? upload_group<float>(b, gi) : upload_group<double>(b, gi);
  if (rc) return rc;
  if (b->nitems[gi] == 0) return CC_OK;
  const int B = b->o.tile;
  void* k = gi ? batch_kernel_b<float>(b->unitw, B) : batch_kernel_b<double>(b->unitw, B);
  const size_t smem = flow_smem(gi == 1, B);
  const int threads = threads_for_tile(B);
  BCK(b, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem));
  if (per_sm < 1) return bfail(b, CC_ERR_CUDA, "batch kernel does not fit on an SM");
  int grid = std::min(per_sm, 8) * b->sms;
  if (b->o.grid > 0) grid = std::min(b->o.grid, per_sm * b->sms);
  grid = std::min(grid, std::max(1, b->nitems[gi]));   // the tail of a solve has few items left
  BCK(b, cudaMemsetAsync(b->cnt, 0, (size_t)b->cnt_total * sizeof(int), b->st));
  void* a = b->args[gi];
  int2* items = b->items[gi];
  int total = b->nitems[gi];
  int* next = b->cnt;
  void* kargs[] = {&a, &items, &total, &next};
  BCK(b, cudaLaunchCooperativeKernel(k, grid, threads, kargs, smem, b->st));
  for (size_t i = 0; i < b->hs.size(); ++i) {
    cc_handle* h = b->hs[i];
    if (!b->active[i] || h->fp32 != (gi == 1)) continue;
    h->sweeps++;
    h->fresh = false;
    if (h->fp32) h->fp32_sweeps++;
  }
  return CC_OK;
}

int batch_sweep(cc_batch* b, int64_t k) {
  BCK(b, cudaSetDevice(b->dev));
  for (int64_t s = 0; s < k; ++s) {
    int rc = batch_launch(b, 0);
    if (rc) return rc;
    rc = batch_launch(b, 1);
    if (rc) return rc;
    b->sweeps++;
  }
  return CC_OK;
}

}  // namespace

extern "C" {

void cc_batch_destroy(cc_batch* b) {
  if (!b) return;
  if (!b->hs.empty()) {
    cc_handle* h0 = b->hs[0];
    cudaSetDevice(h0->dev);
    cudaStreamSynchronize(b->st);
    for (int g = 0; g < 2; ++g) {
      dfree(h0, b->args[g]);
      dfree(h0, b->items[g]);
    }
    dfree(h0, b->cnt);
  }
  for (cc_handle* h : b->hs) cc_destroy(h);
  delete b;
}

int cc_batch_create(cc_batch** out, int32_t count, const int64_t* ns, const double* const* ds,
                    const double* const* ws, const cc_opts* opts) {
  if (!out) return bfail(nullptr, CC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !ns || !ds || !ws) return bfail(nullptr, CC_ERR_ARG, "count >= 1 and ns, ds, ws required");
  cc_opts o;
  cc_opts_default(&o);
  if (opts) o = *opts;
  if (o.schedule != CC_SCHED_TILED || o.exact)
    return bfail(nullptr, CC_ERR_ARG, "a batch runs the tiled schedule in the fused form");
  if (o.problem != CC_PROB_CC) return bfail(nullptr, CC_ERR_UNSUPPORTED, "a batch holds CC instances");
  if (o.store != CC_STORE_DENSE) return bfail(nullptr, CC_ERR_UNSUPPORTED, "a batch uses the dense store");
  cc_batch* b = new (std::nothrow) cc_batch();
  if (!b) return bfail(nullptr, CC_ERR_OOM, "batch");
  b->o = o;
  b->st = (cudaStream_t)o.stream;
  b->dev = o.device;
  for (int32_t i = 0; i < count; ++i) {
    cc_handle* h = nullptr;
    int rc = cc_create(&h, ns[i], ds[i], ws[i], &o);
    if (rc) {
      std::string msg = "instance " + std::to_string(i) + ": " + g_create_error;
      cc_batch_destroy(b);
      return bfail(nullptr, rc, msg);
    }
    b->hs.push_back(h);
    b->unitw = b->unitw && h->unitw;
  }
  b->sms = b->hs[0]->sms;
  b->active.assign(count, 1);
  b->prev_fp32.assign(count, INFINITY);
  b->cnt_off.resize(count);
  int64_t off = 1;
  for (int32_t i = 0; i < count; ++i) {
    b->cnt_off[i] = off;
    off += b->hs[i]->ntiles;
  }
  b->cnt_total = off;
  b->cnt = (int*)dalloc(b->hs[0], (size_t)off * sizeof(int));
  if (!b->cnt) {
    cc_batch_destroy(b);
    return bfail(nullptr, CC_ERR_OOM, "batch counters");
  }
  *out = b;
  return CC_OK;
}

int32_t cc_batch_size(const cc_batch* b) { return b ? (int32_t)b->hs.size() : 0; }

cc_handle* cc_batch_handle(cc_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->hs.size()) return nullptr;
  return b->hs[i];
}

int cc_batch_sweep(cc_batch* b, int64_t k) {
  if (!b) return bfail(nullptr, CC_ERR_ARG, "batch is NULL");
  if (k < 0) return bfail(b, CC_ERR_ARG, "k must be >= 0");
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (!b->active[i]) {
      b->active.assign(b->hs.size(), 1);
      b->stale[0] = b->stale[1] = true;
      break;
    }
  return batch_sweep(b, k);
}

int cc_batch_solve(cc_batch* b, double tol, int64_t max_sweeps, int64_t* sweeps_done, int64_t* per_instance) {
  if (!b) return bfail(nullptr, CC_ERR_ARG, "batch is NULL");
  if (!std::isfinite(tol) || tol < 0 || max_sweeps < 0) return bfail(b, CC_ERR_ARG, "bad tol or max_sweeps");
  const size_t m = b->hs.size();
  b->active.assign(m, 1);
  b->prev_fp32.assign(m, INFINITY);
  b->stale[0] = b->stale[1] = true;
  if (per_instance)
    for (size_t i = 0; i < m; ++i) per_instance[i] = -1;
  int64_t done = 0;
  size_t left = m;
  while (left > 0 && done < max_sweeps) {
    const int64_t k = std::min<int64_t>(b->o.check_every, max_sweeps - done);
    int rc = batch_sweep(b, k);
    if (rc) return rc;
    done += k;
    // checks of all active instances, one synchronization
    for (size_t i = 0; i < m; ++i)
      if (b->active[i]) {
        rc = check_launch(b->hs[i]);
        if (rc) return bfail(b, rc, b->hs[i]->err);
      }
    BCK(b, cudaStreamSynchronize(b->st));
    for (size_t i = 0; i < m; ++i) {
      if (!b->active[i]) continue;
      cc_handle* h = b->hs[i];
      rc = read_ctl_error(h);
      if (rc) return bfail(b, rc, "instance " + std::to_string(i) + ": " + h->err);
      cc_stats s;
      check_finish(h, &s);
      if (h->fp32) {
        const double at = std::max(tol, b->o.refine_at);
        const bool small = s.max_violation <= at;
        const bool stalled = s.max_violation <= 100.0 * at && s.max_violation > 0.99 * b->prev_fp32[i];
        b->prev_fp32[i] = s.max_violation;
        if (!(small || stalled)) continue;
        rc = switch_to_fp64(h);   // its FP64 refinement sweeps come with the next batch sweeps
        if (rc) return bfail(b, rc, h->err);
        b->stale[0] = b->stale[1] = true;
        continue;
      }
      if (s.max_violation <= tol && refined(h)) {
        b->active[i] = 0;
        b->stale[0] = b->stale[1] = true;
        --left;
        if (per_instance) per_instance[i] = h->sweeps;
      }
    }
  }
  if (sweeps_done) *sweeps_done = done;
  b->active.assign(m, 1);
  b->stale[0] = b->stale[1] = true;
  return left == 0 ? CC_OK : bfail(b, CC_ERR_NOT_CONVERGED, "max_sweeps reached before every instance converged");
}

int cc_batch_autotune(int32_t count, const int64_t* ns, const double* const* ds, const double* const* ws,
                      const cc_opts* base, int32_t trial_sweeps, cc_opts* best, double* best_ms) {
  if (!best || trial_sweeps < 1) return bfail(nullptr, CC_ERR_ARG, "best is NULL or trial_sweeps < 1");
  cc_opts o;
  cc_opts_default(&o);
  if (base) o = *base;
  const int tiles[3] = {8, 16, 32};
  double best_t = INFINITY;
  cc_opts pick = o;
  const int nvar = o.precision == CC_PREC_FP64 ? 2 : 1;   // variant 1 differs from 0 in FP64 only
  for (int ti = 0; ti < 3; ++ti)
    for (int order = 0; order < 2; ++order)
    for (int var = 0; var < nvar; ++var) {
      cc_opts c = o;
      c.tile = tiles[ti];
      c.batch_order = order;
      c.variant = var;
      cc_batch* b = nullptr;
      int rc = cc_batch_create(&b, count, ns, ds, ws, &c);
      if (rc) return rc;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      rc = cc_batch_sweep(b, trial_sweeps);                    // warm-up: the first sweeps are the busiest
      if (!rc) {
        cudaEventRecord(e0, b->st);
        rc = cc_batch_sweep(b, trial_sweeps);
        cudaEventRecord(e1, b->st);
      }
      float ms = 0;
      if (!rc) {
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::string err = b->err;
      cc_batch_destroy(b);
      if (rc) return bfail(nullptr, rc, err);
      const double per = ms / trial_sweeps;
      if (per < best_t) {
        best_t = per;
        pick = c;
      }
    }
  *best = pick;
  if (best_ms) *best_ms = best_t;
  return CC_OK;
}

const char* cc_batch_last_error(const cc_batch* b) {
  if (!b) return g_create_error.c_str();
  return b->err.c_str();
}

}  // extern "C"

// ====================================================================== warm start

namespace {

// Candidates (triplets with an edge), their features, and the adjacency the
// features come from; device buffers owned by the caller of this helper.
struct WsCands {
  int64_t* cand = nullptr;
  float* feat = nullptr;
  int64_t count = 0;
};

int ws_build(cc_handle* h, WsCands& c, bool features) {
  const int n = (int)h->n, words = (n + 31) / 32;
  uint32_t* adj = (uint32_t*)dalloc(h, (size_t)n * words * sizeof(uint32_t));
  int* deg = (int*)dalloc(h, (size_t)n * sizeof(int));
  int* cnt = (int*)dalloc(h, (size_t)h->P * sizeof(int));
  int64_t* off = (int64_t*)dalloc(h, (size_t)h->P * sizeof(int64_t));
  auto cleanup = [&]() { dfree(h, adj); dfree(h, deg); dfree(h, cnt); dfree(h, off); };
  if (!adj || !deg || !cnt || !off) {
    cleanup();
    return fail(h, CC_ERR_OOM, "warm-start buffers");
  }
  CK(h, cudaMemsetAsync(adj, 0, (size_t)n * words * sizeof(uint32_t), h->st));
  k_ws_adjacency<<<grid_for(h, h->tile_elems, 256), 256, 0, h->st>>>(h->d64, h->tile_list, h->ntiles, n, h->B, adj, words);
  k_ws_degree<<<grid_for(h, n, 256), 256, 0, h->st>>>(adj, n, words, deg);
  k_ws_candidates<<<grid_for(h, h->P, 256), 256, 0, h->st>>>(adj, n, words, 0, cnt, nullptr, nullptr);
  CK(h, cudaGetLastError());
  std::vector<int> hc((size_t)h->P), hd(n);
  CK(h, cudaMemcpyAsync(hc.data(), cnt, (size_t)h->P * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(hd.data(), deg, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  std::vector<int64_t> ho((size_t)h->P);
  int64_t total = 0;
  for (int64_t p = 0; p < h->P; ++p) {
    ho[p] = total;
    total += hc[p];
  }
  int64_t degsum = 0;
  for (int v : hd) degsum += v;
  const float inv_mean = degsum > 0 ? (float)((double)n / (double)degsum) : 0.f;
  c.count = total;
  c.cand = (int64_t*)dalloc(h, (size_t)std::max<int64_t>(total, 1) * sizeof(int64_t));
  if (features) c.feat = (float*)dalloc(h, (size_t)std::max<int64_t>(total, 1) * WS_FEAT * sizeof(float));
  if (!c.cand || (features && !c.feat)) {
    cleanup();
    return fail(h, CC_ERR_OOM, "warm-start candidates");
  }
  CK(h, cudaMemcpyAsync(off, ho.data(), (size_t)h->P * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
  k_ws_candidates<<<grid_for(h, h->P, 256), 256, 0, h->st>>>(adj, n, words, 1, nullptr, off, c.cand);
  if (features && total > 0)
    k_ws_features<<<grid_for(h, total, 256), 256, 0, h->st>>>(c.cand, total, h->d64, adj, deg, n, h->nb, h->B, words,
                                                              inv_mean, c.feat);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->st));
  cleanup();
  return CC_OK;
}

void ws_release(cc_handle* h, WsCands& c) {
  dfree(h, c.cand);
  dfree(h, c.feat);
  c.cand = nullptr;
  c.feat = nullptr;
}

bool ws_usable(const cc_handle* h) {
  return h->o.schedule == CC_SCHED_TILED && !h->o.exact && h->mask && h->o.problem == CC_PROB_CC;
}

}  // namespace

extern "C" {

int cc_warm_start_mlp(cc_handle* h, const float* params, double threshold, int64_t* candidates) {
  if (!h) return fail(nullptr, CC_ERR_ARG, "handle is NULL");
  if (!params) return fail(h, CC_ERR_ARG, "params is NULL");
  if (!ws_usable(h)) return fail(h, CC_ERR_UNSUPPORTED, "warm start needs the tiled schedule, fused form, dense store");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  WsCands c;
  rc = ws_build(h, c, true);
  if (rc) return rc;
  float* pd = (float*)dalloc(h, WS_NPARAM * sizeof(float));
  if (!pd) {
    ws_release(h, c);
    return fail(h, CC_ERR_OOM, "parameters");
  }
  // FP32 bulk state: the same steps run on FP64 copies of the state, which
  // are rounded to FP32 at the end (the bulk phase's precision).  The FP32
  // store is cleared through its bits first; the FP64 copy of the store is
  // read and rounded only where the prediction leaves a bit set (the resync
  // too reads only those slots), so it is never cleared as a whole
  const bool f32 = h->fp32;
  void* keep[6] = {h->zt, h->zp, h->x, h->f, h->d, h->winv};
  if (f32) {
    const size_t te = (size_t)h->tile_elems;
    void* t[4] = {dalloc(h, (size_t)h->zt_elems * sizeof(double)), dalloc(h, te * 2 * sizeof(double)),
                  dalloc(h, te * sizeof(double)), dalloc(h, te * sizeof(double))};
    if (!t[0] || !t[1] || !t[2] || !t[3]) {
      for (void* q : t) dfree(h, q);
      dfree(h, pd);
      ws_release(h, c);
      return fail(h, CC_ERR_OOM, "FP64 warm-start state");
    }
    k_ws_clear_by_mask<float><<<grid_for(h, h->mask_words, 256), 256, 0, h->st>>>(h->mask, (float*)keep[0],
                                                                                h->mask_words);
    h->zt = t[0];
    h->zp = t[1];
    h->x = t[2];
    h->f = t[3];
    h->d = h->d64;
    h->winv = h->winv64;
    h->fp32 = false;
    h->esz = 8;
  }
  // errors from here on fall through to the restore below.  FP64 state:
  // the store is cleared through its nonzero bits (the bits describe it
  // exactly); in both states the inference sets the bits of what it writes,
  // so neither a pass over the whole store nor a rebuild of the bits is
  // needed
  cudaError_t ce = cudaMemcpyAsync(pd, params, WS_NPARAM * sizeof(float), cudaMemcpyHostToDevice, h->st);
  if (ce == cudaSuccess && !f32) {
    k_ws_clear_by_mask<double><<<grid_for(h, h->mask_words, 256), 256, 0, h->st>>>(h->mask, (double*)h->zt,
                                                                                 h->mask_words);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->zp, 0, (size_t)h->tile_elems * 2 * sizeof(double), h->st);
  if (ce == cudaSuccess && c.count > 0) {
    const int grid = (int)std::min<int64_t>((c.count + 127) / 128, (int64_t)h->sms * 8);
    k_ws_infer<<<grid, 256, 0, h->st>>>(pd, c.feat, c.count, 1, nullptr, c.cand, (double*)h->zt, h->bt_rank, h->nb,
                                        h->B, h->o.eps, (float)threshold, h->mask);
  }
  if (ce == cudaSuccess) ce = cudaGetLastError();
  rc = ce == cudaSuccess ? CC_OK : fail(h, CC_ERR_CUDA, "warm-start inference");
  if (rc == CC_OK) rc = resync_fp64(h);
  if (rc == CC_OK) rc = cc_pair_passes(h, CC_WS_PAIR_PASSES);
  if (f32) {   // round to FP32, back to the FP32 arrays; bits from the rounded duals
    const size_t te = (size_t)h->tile_elems;
    if (rc == CC_OK) {
      // a nonzero prediction is at least the smallest normal float over eps,
      // so its rounding stays nonzero and the bits describe the FP32 store
      k_ws_round_by_mask<<<grid_for(h, h->mask_words, 256), 256, 0, h->st>>>(h->mask, (const double*)h->zt,
                                                                            (float*)keep[0], h->mask_words);
      k_convert<double, float><<<grid_for(h, 2 * te, 256), 256, 0, h->st>>>((const double*)h->zp, (float*)keep[1],
                                                                          2 * (int64_t)te);
      k_convert<double, float><<<grid_for(h, te, 256), 256, 0, h->st>>>((const double*)h->x, (float*)keep[2], te);
      k_convert<double, float><<<grid_for(h, te, 256), 256, 0, h->st>>>((const double*)h->f, (float*)keep[3], te);
    }
    cudaStreamSynchronize(h->st);
    dfree(h, h->zt);
    dfree(h, h->zp);
    dfree(h, h->x);
    dfree(h, h->f);
    h->zt = keep[0];
    h->zp = keep[1];
    h->x = keep[2];
    h->f = keep[3];
    h->d = keep[4];
    h->winv = keep[5];
    h->fp32 = true;
    h->esz = 4;
    if (rc != CC_OK) {   // after a failure the FP32 store may hold part of the prediction
      CK(h, cudaMemsetAsync(h->zt, 0, (size_t)h->zt_elems * sizeof(float), h->st));
      CK(h, cudaMemsetAsync(h->mask, 0, (size_t)h->mask_words * sizeof(uint32_t), h->st));
    }
    const int r2 = cudaGetLastError() == cudaSuccess ? CC_OK : fail(h, CC_ERR_CUDA, "FP32 warm-start state");
    if (rc == CC_OK) rc = r2;
  }
  CK(h, cudaStreamSynchronize(h->st));
  dfree(h, pd);
  ws_release(h, c);
  if (rc) return rc;
  h->sweeps = 0;
  h->fp64_from = -1;   // a state set by the caller needs no refinement sweeps
  h->fresh = false;
  h->fp32_sweeps = 0;
  if (candidates) *candidates = c.count;
  return CC_OK;
}

int cc_ws_samples(cc_handle* h, float* feat, float* target, int64_t cap, int64_t* count) {
  if (!h || !count) return fail(h, CC_ERR_ARG, "handle or count is NULL");
  if (!ws_usable(h) || h->fp32)
    return fail(h, CC_ERR_UNSUPPORTED, "samples need the tiled schedule, fused form, dense store, FP64 state");
  CK(h, cudaSetDevice(h->dev));
  int rc = read_ctl_error(h);
  if (rc) return rc;
  WsCands c;
  rc = ws_build(h, c, true);
  if (rc) return rc;
  *count = c.count;
  if (feat && target && c.count <= cap && c.count > 0) {
    CK(h, cudaMemcpyAsync(feat, c.feat, (size_t)c.count * WS_FEAT * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    k_ws_targets<<<grid_for(h, c.count, 256), 256, 0, h->st>>>(c.cand, c.count, (const double*)h->zt, h->bt_rank,
                                                               h->nb, h->B, h->o.eps, target);
    CK(h, cudaGetLastError());
  }
  CK(h, cudaStreamSynchronize(h->st));
  ws_release(h, c);
  if ((feat || target) && c.count > cap) return fail(h, CC_ERR_ARG, "cap is smaller than the sample count");
  return CC_OK;
}

int cc_mlp_forward(const float* params, const float* feat, float* out, int64_t count, void* stream) {
  if (!params || !feat || !out || count < 0) return fail(nullptr, CC_ERR_ARG, "NULL argument or count < 0");
  if (count == 0) return CC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  float* pd = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&pd, WS_NPARAM * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pd, params, WS_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>((count + 127) / 128, (int64_t)sms * 8);
    k_ws_infer<<<grid, 256, 0, st>>>(pd, feat, count, 0, out, nullptr, nullptr, nullptr, 0, 8, 1.0, 0.f);
    e = cudaGetLastError();
  }
  if (pd) cudaFreeAsync(pd, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, CC_ERR_CUDA, std::string("cc_mlp_forward: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // extern "C"

namespace {

// Device copies of the parameters, Adam moments, gradient and per-step loss.
struct WsTrainBufs {
  float* p = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;
  float* loss = nullptr;
};

cudaError_t ws_train_alloc(WsTrainBufs& b, int steps, cudaStream_t st) {
  const size_t np = WS_NPARAM * sizeof(float);
  cudaError_t e = cudaMallocAsync((void**)&b.p, 4 * np + (size_t)std::max(steps, 1) * sizeof(float), st);
  if (e != cudaSuccess) return e;
  b.m = b.p + WS_NPARAM;
  b.v = b.m + WS_NPARAM;
  b.g = b.v + WS_NPARAM;
  b.loss = b.g + WS_NPARAM;
  return cudaMemsetAsync(b.m, 0, 3 * np + (size_t)std::max(steps, 1) * sizeof(float), st);
}

cudaError_t ws_train_launch(const WsTrainBufs& b, const float* feat, const float* target, int64_t count, int64_t rows,
                            float pos_weight,
                            int sample, uint64_t seed, float* loss, cudaStream_t st) {
  const size_t smem = sizeof(WsTrainSmem);
  cudaError_t e = cudaFuncSetAttribute(k_ws_train_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t chunks = (rows + 15) / 16;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + WS_TRAIN_WARPS - 1) / WS_TRAIN_WARPS, sms));
  k_ws_train_grad<<<grid, 32 * WS_TRAIN_WARPS, smem, st>>>(b.p, feat, target, count, rows, sample, seed, pos_weight,
                                                           b.g, loss);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int cc_mlp_grad(const float* params, const float* feat, const float* target, int64_t count, float pos_weight,
                float* grad, float* loss, void* stream) {
  if (!params || !feat || !target || !grad || count <= 0) return fail(nullptr, CC_ERR_ARG, "NULL argument or count <= 0");
  if (!(pos_weight > 0.f && pos_weight < INFINITY)) return fail(nullptr, CC_ERR_ARG, "pos_weight not positive and finite");
  cudaStream_t st = (cudaStream_t)stream;
  WsTrainBufs b;
  cudaError_t e = ws_train_alloc(b, 1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.p, params, WS_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = ws_train_launch(b, feat, target, count, count, pos_weight, 0, 0, b.loss, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, b.g, WS_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st);
  float l = 0.f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, b.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (b.p) cudaFreeAsync(b.p, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, CC_ERR_CUDA, std::string("cc_mlp_grad: ") + cudaGetErrorString(e));
  if (loss) *loss = l;
  return CC_OK;
}

int cc_mlp_train(float* params, const float* feat, const float* target, int64_t count, int32_t batch, int32_t steps,
                 float lr, uint64_t seed, float pos_weight, float* loss, void* stream) {
  if (!params || !feat || !target || count <= 0 || batch <= 0 || steps < 0 || !(lr > 0.f))
    return fail(nullptr, CC_ERR_ARG, "NULL argument, count/batch <= 0, steps < 0 or lr <= 0");
  if (!(pos_weight > 0.f && pos_weight < INFINITY)) return fail(nullptr, CC_ERR_ARG, "pos_weight not positive and finite");
  if (steps == 0) return CC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  WsTrainBufs b;
  cudaError_t e = ws_train_alloc(b, steps, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.p, params, WS_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st);
  for (int s = 0; s < steps && e == cudaSuccess; ++s) {
    e = ws_train_launch(b, feat, target, count, batch, pos_weight, 1, seed * 1000003ull + (uint64_t)s, b.loss + s, st);
    if (e == cudaSuccess) {
      k_ws_adam<<<(WS_NPARAM + 255) / 256, 256, 0, st>>>(b.p, b.m, b.v, b.g, lr, 0.9f, 0.999f, 1e-8f, s + 1);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(params, b.p, WS_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, b.loss, (size_t)steps * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (b.p) cudaFreeAsync(b.p, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, CC_ERR_CUDA, std::string("cc_mlp_train: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // extern "C"
