// batch.cu -- many densities of uneven size and wavenumber in one persistent
// launch (a batched form of the apply of Section 4; not in the paper).
//
// Every pass of every density becomes a list of tiles.  All lists are laid out
// pass-major in one global item range: first pass of every density, then the
// second pass of every density, and so on.  Persistent CTAs take items from a
// global counter; before running a tile of pass p of density i a CTA waits
// until every tile of pass p-1 of density i has completed (per-pass completion
// counters).  Every item a CTA waits on was taken earlier by a resident CTA,
// so the batch always makes progress; each wait is still bounded by a clock
// limit after which the kernel records VP_ERR_TIMEOUT in an error word and goes
// on, so a lost dependency can never hang the device.  Intermediate data is
// produced inside the kernel, so tiles read it with ld.global.cg (L2) instead
// of the non-coherent read-only path.
//
// The host driver captures [reset counters, batch kernel] into a CUDA graph and
// replays it; density pointers travel as kernel parameters updated per replay.
// An autotuner times the persistent kernel at two grid sizes against
// per-density launches and caches the fastest choice per device and batch.
#include <cuda_runtime.h>
#include <sys/stat.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vp.h"
#include "fourstep.cuh"
#include "vp_internal.cuh"

namespace vp {

constexpr int BATCH_MAX = 128;
constexpr int BATCH_THREADS = 256;

// Per-(density, pass) description of the tiles.
struct BatchPass {
  PassArgs<float> a;
  int n;                 // FFT length 2N
  int kind;              // PassKind
  int density;           // index into the pointer tables
  int io;                // 1: input is the density's f, 2: output is the density's phi
  long long ntiles;
  long long item_base;   // first tile of this pass in the pass-major order
  int dep;               // completion counter to wait on (-1: none)
  long long dep_need;    // tiles that counter must reach
  long long dep_need_orig;
  int done;              // completion counter this pass increments
};

struct BatchLaunch {
  const BatchPass* passes;
  int npasses;
  long long total_items;
  unsigned long long* next_item;
  long long* done;
  int* err;
  long long timeout_cycles;
  int chunk;  // tiles per work item
  const void* f[BATCH_MAX];
  void* phi[BATCH_MAX];
};

// Uniform 256-thread configuration per FFT length: E = 16 (12 with a factor 3),
// W = 256 / (n / E) pencils per tile.
template <int n> struct BatchE {
  static constexpr int E = (n % 3 == 0) ? 12 : 16;
};
template <int n, bool CONTIG, int MODE>
using BatchCfg = PassCfg<float, n, CONTIG, MODE, BatchE<n>::E, BATCH_THREADS / (n / BatchE<n>::E), 1, 2>;

// Lengths whose tiles run the four-step code (fourstep.cuh) with W = 256 / Q
// pencils per tile; the others run the Stockham tiles of pencil_fft.cuh.
__host__ __device__ constexpr bool batch_fourstep(int n) { return n == 64 || n == 128 || n == 256; }
template <int n> constexpr int batch_fs_W() { return BATCH_THREADS / (n / fs::fs_P(n)); }
template <int n, bool CONTIG, int MODE> using BatchFs = fs::Cfg<n, CONTIG, MODE, batch_fs_W<n>(), 2>;

#define VP_BATCH_LENGTHS(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256)
#define VP_BATCH_STOCKHAM(X) X(16) X(24) X(32) X(48) X(96) X(192)

// shared memory: the exchange buffer (either engine), two input staging
// slots, the four-step twiddle tables
template <int n> constexpr size_t batch_xs_n() {
  if constexpr (batch_fourstep(n))
    return std::max((size_t)BatchFs<n, true, MODE_FWD>::XELEMS, (size_t)BatchFs<n, false, MODE_FWD>::XELEMS) * 8;
  else
    return std::max(BatchCfg<n, true, MODE_FWD>::xchg_bytes, BatchCfg<n, false, MODE_FWD>::xchg_bytes);
}
template <int n> constexpr size_t batch_slot_n() {
  if constexpr (batch_fourstep(n))
    return std::max({BatchFs<n, true, MODE_FWD>::in_bytes, BatchFs<n, false, MODE_FWD>::in_bytes,
                     BatchFs<n, true, MODE_INV>::in_bytes, BatchFs<n, false, MODE_INV>::in_bytes});
  else
    return std::max({BatchCfg<n, true, MODE_FWD>::slot_bytes, BatchCfg<n, false, MODE_FWD>::slot_bytes,
                     BatchCfg<n, true, MODE_INV>::slot_bytes, BatchCfg<n, false, MODE_INV>::slot_bytes});
}
constexpr size_t r128(size_t b) { return (b + 127) / 128 * 128; }
constexpr size_t batch_xs_bytes() {
  size_t m = 0;
#define VP_M(N) m = std::max(m, batch_xs_n<N>());
  VP_BATCH_LENGTHS(VP_M)
#undef VP_M
  return r128(m);
}
constexpr size_t batch_slot_bytes() {
  size_t m = 0;
#define VP_M(N) m = std::max(m, batch_slot_n<N>());
  VP_BATCH_LENGTHS(VP_M)
#undef VP_M
  return r128(m);
}
// four-step twiddle tables, (Q x (P + 2)) each: 2N = 256, 128, 64
__host__ __device__ constexpr int batch_tw_off(int li) { return li == 0 ? 0 : (li == 1 ? 16 * 18 : 16 * 18 + 8 * 18); }
constexpr int BATCH_TW_TOTAL = 16 * 18 + 8 * 18 + 8 * 10;
__host__ __device__ constexpr int batch_tw_index(int n) { return n == 256 ? 0 : (n == 128 ? 1 : 2); }
constexpr size_t batch_smem_bytes() { return batch_xs_bytes() + 2 * batch_slot_bytes() + (size_t)BATCH_TW_TOTAL * 8; }
// two CTAs per SM (228 KB of shared memory per SM, 1 KB reserved per CTA, the
// kernel's static arrays about 3 KB)
static_assert(2 * (batch_smem_bytes() + 3072 + 1024) <= 233472, "two batch CTAs per SM");

bool batch_length_built(int n) {
  switch (n) {
#define VP_C(N) \
  case N: return true;
    VP_BATCH_LENGTHS(VP_C)
#undef VP_C
  }
  return false;
}

// Stockham tiles: stage the input of a tile into a slot, or run a tile (from
// the slot when given, else from global memory through L2)
template <int n>
__device__ __noinline__ void bt_stage_st(int kind, const PassArgs<float>& a, long long tile, float2* slot) {
  unsigned char* sl = reinterpret_cast<unsigned char*>(slot);
  switch (kind) {
    case FWD_CONTIG: stage_tile<float, n, true, MODE_FWD, BatchCfg<n, true, MODE_FWD>>(a, tile, sl); break;
    case FWD_STRIDED: stage_tile<float, n, false, MODE_FWD, BatchCfg<n, false, MODE_FWD>>(a, tile, sl); break;
    case INV_CONTIG: stage_tile<float, n, true, MODE_INV, BatchCfg<n, true, MODE_INV>>(a, tile, sl); break;
    case INV_STRIDED: stage_tile<float, n, false, MODE_INV, BatchCfg<n, false, MODE_INV>>(a, tile, sl); break;
    default: stage_tile<float, n, false, MODE_FUSED1, BatchCfg<n, false, MODE_FUSED1>>(a, tile, sl); break;
  }
}
template <int n>
__device__ __noinline__ void bt_run_st(int kind, const PassArgs<float>& a, long long tile, float2* sm,
                                       const float2* slot) {
  const unsigned char* sl = reinterpret_cast<const unsigned char*>(slot);
  const bool st = slot != nullptr;
  switch (kind) {
    case FWD_CONTIG: process_tile<float, n, true, MODE_FWD, BatchCfg<n, true, MODE_FWD>, true>(a, tile, sm, sl, st); break;
    case FWD_STRIDED: process_tile<float, n, false, MODE_FWD, BatchCfg<n, false, MODE_FWD>, true>(a, tile, sm, sl, st); break;
    case INV_CONTIG: process_tile<float, n, true, MODE_INV, BatchCfg<n, true, MODE_INV>, true>(a, tile, sm, sl, st); break;
    case INV_STRIDED: process_tile<float, n, false, MODE_INV, BatchCfg<n, false, MODE_INV>, true>(a, tile, sm, sl, st); break;
    default: process_tile<float, n, false, MODE_FUSED1, BatchCfg<n, false, MODE_FUSED1>, true>(a, tile, sm, sl, st); break;
  }
}
// four-step tiles
template <int n>
__device__ __noinline__ void bt_stage_fs(int kind, const PassArgs<float>& a, int tile, float2* slot) {
  const float2* i2 = reinterpret_cast<const float2*>(a.in);
  switch (kind) {
    case FWD_CONTIG: fs::stage_input_from<BatchFs<n, true, MODE_FWD>>(a, i2, tile, slot); break;
    case FWD_STRIDED: fs::stage_input_from<BatchFs<n, false, MODE_FWD>>(a, i2, tile, slot); break;
    case INV_CONTIG: fs::stage_input_from<BatchFs<n, true, MODE_INV>>(a, i2, tile, slot); break;
    case INV_STRIDED: fs::stage_input_from<BatchFs<n, false, MODE_INV>>(a, i2, tile, slot); break;
    default: fs::stage_input_from<BatchFs<n, false, MODE_FUSED1>>(a, i2, tile, slot); break;
  }
}
template <int n>
__device__ __noinline__ void bt_run_fs(int kind, const PassArgs<float>& a, int tile, float2* xs, const float2* tws,
                                       const float2* slot) {
  constexpr int W = batch_fs_W<n>();
  const float2* i2 = reinterpret_cast<const float2*>(a.in);
  float2* o2 = reinterpret_cast<float2*>(a.out);
  switch (kind) {
    case FWD_CONTIG: fs::batch_tile<n, true, MODE_FWD, W>(a, i2, o2, tile, xs, tws, slot); break;
    case FWD_STRIDED: fs::batch_tile<n, false, MODE_FWD, W>(a, i2, o2, tile, xs, tws, slot); break;
    case INV_CONTIG: fs::batch_tile<n, true, MODE_INV, W>(a, i2, o2, tile, xs, tws, slot); break;
    case INV_STRIDED: fs::batch_tile<n, false, MODE_INV, W>(a, i2, o2, tile, xs, tws, slot); break;
    default: fs::batch_tile<n, false, MODE_FUSED1, W>(a, i2, o2, tile, xs, tws, slot); break;
  }
}

constexpr int BATCH_MAX_PASSES = BATCH_MAX * 5;

// The persistent kernel.  Work items are chunks of up to L.chunk consecutive
// tiles of one pass, laid out pass-major; CTAs take them from a
// global counter.  Per chunk: thread 0 takes the next chunk, finds its pass and
// waits (bounded) until every tile of the pass it depends on has completed;
// one barrier publishes the chunk; its tiles then run like a standalone pass,
// each tile's input staged into shared memory by cp.async while the tile
// before it is computed (two slots); a barrier, and thread 0 adds the chunk's
// tiles to the pass's completion counter (fence, then atomic add).  Every chunk
// a CTA waits on was taken earlier by a resident CTA, so the batch always
// makes progress.  Data written inside the launch is read through L2
// (cp.async.cg, ld.global.cg).
constexpr int BATCH_CHUNKS[4] = {4, 8, 16, 32};  // chunk sizes the autotuner tries

__device__ __forceinline__ int batch_find_pass(const int* base, int npasses, long long item) {
  int lo = 0, hi = npasses - 1;  // last pass whose first item <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (base[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void batch_stage(int n, int kind, const PassArgs<float>& a, long long tile, float2* slot) {
  switch (n) {
    case 256: bt_stage_fs<256>(kind, a, (int)tile, slot); break;
    case 128: bt_stage_fs<128>(kind, a, (int)tile, slot); break;
    case 64: bt_stage_fs<64>(kind, a, (int)tile, slot); break;
#define VP_C(N) \
  case N: bt_stage_st<N>(kind, a, tile, slot); break;
    VP_BATCH_STOCKHAM(VP_C)
#undef VP_C
  }
}

__global__ void __launch_bounds__(BATCH_THREADS, 2) batch_kernel(const BatchLaunch L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* slots = reinterpret_cast<float2*>(smem_raw + batch_xs_bytes());
  float2* tws = reinterpret_cast<float2*>(smem_raw + batch_xs_bytes() + 2 * batch_slot_bytes());
  constexpr int SLOT = (int)(batch_slot_bytes() / 8);
  __shared__ int s_base[BATCH_MAX_PASSES];  // first chunk of every pass (< 2^31, checked at creation)
  __shared__ long long s_item;
  __shared__ int s_pass;
  __shared__ __align__(16) PassArgs<float> s_a;  // the chunk's pass arguments, density pointers patched in
  __shared__ const float2* s_twsrc[3];
  if (threadIdx.x < 3) s_twsrc[threadIdx.x] = nullptr;
  __syncthreads();
  if (threadIdx.x == 0) {  // first chunk of every pass
    long long b = 0;
    for (int i = 0; i < L.npasses; ++i) {
      s_base[i] = (int)b;
      b += (L.passes[i].ntiles + L.chunk - 1) / L.chunk;
    }
  }
  for (int i = threadIdx.x; i < L.npasses; i += blockDim.x) {
    const int n = L.passes[i].n;
    if (batch_fourstep(n)) s_twsrc[batch_tw_index(n)] = reinterpret_cast<const float2*>(L.passes[i].a.tw);
  }
  __syncthreads();
  // four-step twiddle tables w_n^(t k1) (any pass of that length has the table exp(-2 pi i q / n))
#pragma unroll
  for (int li = 0; li < 3; ++li) {
    const float2* src = s_twsrc[li];
    if (!src) continue;
    const int n = li == 0 ? 256 : (li == 1 ? 128 : 64);
    const int P = fs::fs_P(n), Q = n / P, TP = P + 2;
    for (int i = threadIdx.x; i < Q * P; i += blockDim.x) {
      const int t = i / P, k1 = i % P;
      tws[batch_tw_off(li) + t * TP + k1] = src[(t * k1) % n];
    }
  }
  for (;;) {
    if (threadIdx.x < 32) {
      // warp 0: lane 0 takes the next chunk and waits for its dependency; the
      // warp copies the pass arguments into shared memory
      long long item = 0;
      int pi = -1;
      if (threadIdx.x == 0) {
        item = (long long)atomicAdd(L.next_item, 1ULL);
        if (item < L.total_items) {
          pi = batch_find_pass(s_base, L.npasses, item);
          const int dep = L.passes[pi].dep;
          if (dep >= 0) {
            const long long need = L.passes[pi].dep_need;
            const long long c0 = clock64();
            volatile long long* cnt = L.done + dep;
            while (*cnt < need) {
              if (clock64() - c0 > L.timeout_cycles) {
                atomicOr(L.err, 1);
                break;
              }
              __nanosleep(64);
            }
            __threadfence();
          }
        }
        s_item = item;
        s_pass = pi;
      }
      pi = __shfl_sync(0xffffffffu, pi, 0);
      if (pi >= 0) {
        const unsigned* src = reinterpret_cast<const unsigned*>(&L.passes[pi].a);
        unsigned* dst = reinterpret_cast<unsigned*>(&s_a);
        for (int i = threadIdx.x; i < (int)(sizeof(PassArgs<float>) / 4); i += 32) dst[i] = src[i];
        __syncwarp();
        if (threadIdx.x == 0) {
          const BatchPass& bp = L.passes[pi];
          if (bp.io == 1) s_a.in = L.f[bp.density];
          if (bp.io == 2) s_a.out = L.phi[bp.density];
        }
      }
    }
    __syncthreads();  // the chunk, its dependency and its arguments are ready for every thread
    const int pi = s_pass;
    if (pi < 0) break;
    const BatchPass& bp = L.passes[pi];
    const int n = bp.n, kind = bp.kind;
    const long long t0 = (s_item - s_base[pi]) * L.chunk;
    const long long t1 = t0 + L.chunk < bp.ntiles ? t0 + L.chunk : bp.ntiles;
    // the first pass reads the caller's density: staged only when 16-byte aligned
    const bool stage = !(reinterpret_cast<uintptr_t>(s_a.in) & 15);
    if (stage) batch_stage(n, kind, s_a, t0, slots);
    cp_async_commit();
    for (long long tile = t0; tile < t1; ++tile) {
      const int si = (int)(tile - t0) & 1;
      if (stage && tile + 1 < t1) batch_stage(n, kind, s_a, tile + 1, slots + (si ^ 1) * SLOT);
      cp_async_commit();
      cp_async_wait<1>();  // this tile's input
      __syncthreads();
      const float2* sl = stage ? slots + si * SLOT : nullptr;
      switch (n) {
        case 256: bt_run_fs<256>(kind, s_a, (int)tile, sm, tws + batch_tw_off(0), sl); break;
        case 128: bt_run_fs<128>(kind, s_a, (int)tile, sm, tws + batch_tw_off(1), sl); break;
        case 64: bt_run_fs<64>(kind, s_a, (int)tile, sm, tws + batch_tw_off(2), sl); break;
#define VP_C(N) \
  case N: bt_run_st<N>(kind, s_a, tile, sm, sl); break;
          VP_BATCH_STOCKHAM(VP_C)
#undef VP_C
      }
      __syncthreads();  // the slot, the exchange buffer and s_a are free; the tile's stores are issued
    }
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(reinterpret_cast<unsigned long long*>(L.done + bp.done), (unsigned long long)(t1 - t0));
    }
  }
  cp_async_wait<0>();
}

// tiles of one pass under the batch configuration
long long batch_tiles(int n, int kind, const PassArgs<float>& a, int* nblk) {
  int W;
  if (batch_fourstep(n)) {
    W = BATCH_THREADS / (n / fs::fs_P(n));
  } else {
    const int Tp = n / ((n % 3 == 0) ? 12 : 16);
    W = BATCH_THREADS / Tp;
  }
  if (kind == FWD_CONTIG || kind == INV_CONTIG) {
    *nblk = 1;
    return (a.O + W - 1) / W;
  }
  *nblk = (a.I + W - 1) / W;
  return (long long)a.O * (*nblk);
}

// On-disk autotuner cache: lines "key value"; the last line of a key wins.
// VP_AUTOTUNE_CACHE overrides the path ($HOME/.cache/vp_autotune.txt).
std::string autotune_cache_path() {
  const char* p = getenv("VP_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/vp_autotune.txt";
}

int autotune_cache_lookup(const std::string& key) {
  FILE* fh = fopen(autotune_cache_path().c_str(), "r");
  if (!fh) return 0;
  char line[4096];
  int found = 0;
  while (fgets(line, sizeof(line), fh)) {
    char* sp = strrchr(line, ' ');
    if (!sp) continue;
    *sp = 0;
    if (key == line) found = atoi(sp + 1);
  }
  fclose(fh);
  return found;
}

void autotune_cache_store(const std::string& key, int s) {
  const std::string path = autotune_cache_path();
  // best effort: create the missing directories of the path, then append
  FILE* fh = fopen(path.c_str(), "a");
  if (!fh) {
    for (size_t i = path.find('/', 1); i != std::string::npos; i = path.find('/', i + 1))
      mkdir(path.substr(0, i).c_str(), 0755);
    fh = fopen(path.c_str(), "a");
  }
  if (!fh) return;
  fprintf(fh, "%s %d\n", key.c_str(), s);
  fclose(fh);
}

}  // namespace vp

using namespace vp;

namespace {

enum Strategy { S_PERSISTENT = 1, S_PERSISTENT_1 = 2, S_SEQUENTIAL = 3, S_STREAMS = 4 };
constexpr int kSideStreams = 8;

}  // namespace

struct vp_batch_s {
  int count = 0;
  std::vector<vp_plan> plans;
  int device = 0;
  cudaStream_t stream = nullptr;
  int strategy = 0;  // 0 = not tuned yet
  int forced = 0;    // strategy set by the caller
  int chunk = 8;     // tiles per work item of the persistent kernel (the autotuner's choice)
  int forced_chunk = 0;
  std::vector<BatchPass> host_passes;
  BatchPass* passes = nullptr;
  long long total_items = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  unsigned long long* next_item = nullptr;  // followed by the completion counters and the error word
  long long* done = nullptr;
  int* err = nullptr;
  void* ctrl = nullptr;
  size_t ctrl_bytes = 0;
  int grid_full = 0, grid_one = 0;
  long long timeout_cycles = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr;
  int graph_grid = 0;
  // per-density launches forked over side streams, captured as one graph
  cudaStream_t side[8] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[8] = {};
  cudaGraph_t sgraph = nullptr;
  cudaGraphExec_t sexec = nullptr;
  std::vector<const void*> sgraph_f;
  std::vector<void*> sgraph_phi;
  std::string last_error;
  std::string signature;
};

namespace {

vp_status bfail(vp_batch b, vp_status st, const std::string& m) {
  vp::log_line(1, "batch", m);
  if (b) b->last_error = m;
  return st;
}

BatchLaunch make_launch(vp_batch b, const void* const* f, void* const* phi) {
  BatchLaunch L;
  memset(&L, 0, sizeof(L));
  L.passes = b->passes;
  L.npasses = (int)b->host_passes.size();
  L.chunk = b->forced_chunk ? b->forced_chunk : b->chunk;
  L.total_items = 0;
  for (const BatchPass& bp : b->host_passes) L.total_items += (bp.ntiles + L.chunk - 1) / L.chunk;
  L.next_item = b->next_item;
  L.done = b->done;
  L.err = b->err;
  L.timeout_cycles = b->timeout_cycles;
  for (int i = 0; i < b->count; ++i) {
    L.f[i] = f[i];
    L.phi[i] = phi[i];
  }
  return L;
}

// counters and item cursor reset (the error word is kept until vp_batch_status)
cudaError_t reset_counters(vp_batch b) {
  return cudaMemsetAsync(b->ctrl, 0, b->ctrl_bytes - sizeof(int) * 4, b->stream);
}

cudaError_t launch_persistent(vp_batch b, const BatchLaunch& L, int grid) {
  cudaError_t e = reset_counters(b);
  if (e != cudaSuccess) return e;
  batch_kernel<<<grid, BATCH_THREADS, batch_smem_bytes(), b->stream>>>(L);
  return cudaGetLastError();
}

vp_status run_sequential(vp_batch b, const void* const* f, void* const* phi) {
  for (int i = 0; i < b->count; ++i) {
    cudaStream_t saved = plan_stream(b->plans[i]);
    vp_plan_set_stream(b->plans[i], b->stream);
    vp_status st = vp_apply(b->plans[i], f[i], phi[i], VP_C64);
    vp_plan_set_stream(b->plans[i], saved);
    if (st != VP_OK) return bfail(b, st, std::string("density apply: ") + vp_last_error(b->plans[i]));
  }
  return VP_OK;
}

// graph of [reset, batch kernel] for a grid size; kernel params updated per replay
vp_status graph_launch(vp_batch b, const BatchLaunch& L, int grid) {
  if (!b->exec || b->graph_grid != grid) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bfail(b, VP_ERR_CUDA, "stream");
    cudaStream_t saved = b->stream;
    b->stream = cap;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = launch_persistent(b, L, grid);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    b->stream = saved;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, VP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    b->knode = nullptr;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      if (ty == cudaGraphNodeTypeKernel) b->knode = nd;
    }
    if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess)
      return bfail(b, VP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->graph_grid = grid;
  }
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  BatchLaunch Lc = L;
  void* args[1] = {&Lc};
  kp.func = (void*)batch_kernel;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(BATCH_THREADS);
  kp.sharedMemBytes = (unsigned)batch_smem_bytes();
  kp.kernelParams = args;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
  if (e != cudaSuccess) return bfail(b, VP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return VP_OK;
}

// Per-density applies spread over side streams, captured once per pointer set
// into a graph and replayed.  Densities are placed largest first, each on the
// stream with the least work so far (work = N^d), so the streams finish together.
vp_status run_streams(vp_batch b, const void* const* f, void* const* phi) {
  bool same = b->sexec && (int)b->sgraph_f.size() == b->count;
  for (int i = 0; same && i < b->count; ++i) same = b->sgraph_f[i] == f[i] && b->sgraph_phi[i] == phi[i];
  if (!same) {
    if (b->sexec) cudaGraphExecDestroy(b->sexec);
    if (b->sgraph) cudaGraphDestroy(b->sgraph);
    b->sexec = nullptr;
    b->sgraph = nullptr;
    if (!b->fork_ev) {
      cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
      for (int k = 0; k < kSideStreams; ++k) {
        cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming);
      }
    }
    // one uncaptured run so every workspace and kernel attribute exists before capture
    vp_status st = run_sequential(b, f, phi);
    if (st != VP_OK) return st;
    cudaStream_t origin;
    cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    cudaStreamSynchronize(b->stream);
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork_ev, origin);
    for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork_ev, 0);
    std::vector<int> order(b->count);
    std::vector<double> work(b->count, 1.0);
    for (int i = 0; i < b->count; ++i) {
      order[i] = i;
      work[i] = (double)plan_points(b->plans[i]);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    double load[kSideStreams] = {0.0};
    for (int j = 0; j < b->count && e == cudaSuccess && st == VP_OK; ++j) {
      const int i = order[j];
      int k = 0;
      for (int c = 1; c < kSideStreams; ++c)
        if (load[c] < load[k]) k = c;
      load[k] += work[i];
      cudaStream_t saved = plan_stream(b->plans[i]);
      vp_plan_set_stream(b->plans[i], b->side[k]);
      st = vp_apply(b->plans[i], f[i], phi[i], VP_C64);
      vp_plan_set_stream(b->plans[i], saved);
    }
    for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) {
      e = cudaEventRecord(b->join_ev[k], b->side[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, b->join_ev[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(origin, &g);
    cudaStreamDestroy(origin);
    if (e != cudaSuccess || e2 != cudaSuccess || st != VP_OK) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, st != VP_OK ? st : VP_ERR_CUDA, "stream graph capture failed");
    }
    if ((e = cudaGraphInstantiate(&b->sexec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return bfail(b, VP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    b->sgraph = g;
    b->sgraph_f.assign(f, f + b->count);
    b->sgraph_phi.assign(phi, phi + b->count);
  }
  cudaError_t e = cudaGraphLaunch(b->sexec, b->stream);
  return e == cudaSuccess ? VP_OK : bfail(b, VP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
}

vp_status run_strategy(vp_batch b, int s, const void* const* f, void* const* phi) {
  if (s == S_SEQUENTIAL) return run_sequential(b, f, phi);
  if (s == S_STREAMS) return run_streams(b, f, phi);
  const BatchLaunch L = make_launch(b, f, phi);
  return graph_launch(b, L, s == S_PERSISTENT ? b->grid_full : b->grid_one);
}

// Times each candidate on the batch (2 warm-ups, 3 timed runs on the batch's
// stream with CUDA events) and keeps the fastest: the persistent kernel with
// every chunk size of BATCH_CHUNKS (all resident CTAs) and with 8-tile chunks
// at one CTA per SM, the per-density launches and their graph over side
// streams.  The choice is cached per device, driver and batch shape as
// strategy + 100 x chunk.
vp_status autotune(vp_batch b, const void* const* f, void* const* phi) {
  struct Cand { int s, chunk; };
  std::vector<Cand> cands;
  for (int c : BATCH_CHUNKS) cands.push_back({S_PERSISTENT, c});
  cands.push_back({S_PERSISTENT_1, 8});
  cands.push_back({S_SEQUENTIAL, 8});
  cands.push_back({S_STREAMS, 8});
  float best = 1e30f;
  Cand bestc = {S_PERSISTENT, 8};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved_forced_chunk = b->forced_chunk;
  for (const Cand& c : cands) {
    b->forced_chunk = c.chunk;
    vp_status st = VP_OK;
    for (int r = 0; r < 2 && st == VP_OK; ++r) st = run_strategy(b, c.s, f, phi);
    if (st != VP_OK) continue;
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < 3 && st == VP_OK; ++r) st = run_strategy(b, c.s, f, phi);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || st != VP_OK) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bestc = c;
    }
  }
  b->forced_chunk = saved_forced_chunk;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->strategy = bestc.s;
  b->chunk = bestc.chunk;
  vp::autotune_cache_store(b->signature, bestc.s + 100 * bestc.chunk);
  return VP_OK;
}

}  // namespace

extern "C" {

vp_status vp_batch_create(vp_batch* out, int count, const vp_plan* plans) {
  if (!out) return VP_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || count > BATCH_MAX || !plans) return VP_ERR_INVALID_ARG;
  static_assert(sizeof(BatchPass) % 4 == 0, "pass descriptor is copied as words");
  vp_batch b = new vp_batch_s();
  b->count = count;
  b->plans.assign(plans, plans + count);
  // the batch runs on its plans' device (they must share one)
  b->device = plans[0] ? plan_device(plans[0]) : 0;
  for (int i = 1; i < count; ++i)
    if (plans[i] && plan_device(plans[i]) != b->device) {
      delete b;
      return VP_ERR_INVALID_ARG;
    }
  vp::DeviceGuard dg_(b->device);
  if (dg_.error() != cudaSuccess) {
    delete b;
    return VP_ERR_CUDA;
  }
  // pass tables and workspace layout
  size_t ws_elems = 0;
  std::vector<size_t> ws_off(count);
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !plan_is_fp32(plans[i])) {
      delete b;
      return VP_ERR_INVALID_ARG;
    }
    int d, N, dims[3];
    vp_plan_info(plans[i], &d, &N, nullptr, nullptr, nullptr);
    plan_dims(plans[i], dims);
    for (int a = 0; a < d; ++a)
      if (!batch_length_built(2 * dims[a])) {
        delete b;
        return VP_ERR_UNSUPPORTED;
      }
    const size_t U = (size_t)plan_points(plans[i]);
    ws_off[i] = ws_elems;
    ws_elems += (d == 3 ? 6 : 2) * U;
  }
  cudaError_t e = cudaMalloc(&b->ws, ws_elems * sizeof(float2));
  if (e != cudaSuccess) {
    delete b;
    return VP_ERR_OOM;
  }
  b->ws_bytes = ws_elems * sizeof(float2);
  // pass-major ordering: pass level 0 of every density, then level 1, ...
  std::vector<std::vector<BatchPass>> per(count);
  int counter = 0;
  for (int i = 0; i < count; ++i) {
    PassArgs<float> args[5];
    int kinds[5], lens[5];
    int np = plan_pass_args_f32(plans[i], reinterpret_cast<float2*>(b->ws) + ws_off[i], args, kinds, lens);
    for (int p = 0; p < np; ++p) {
      BatchPass bp;
      memset(&bp, 0, sizeof(bp));
      bp.a = args[p];
      bp.n = lens[p];
      bp.kind = kinds[p];
      bp.density = i;
      bp.io = (p == 0) ? 1 : (p == np - 1 ? 2 : 0);
      int nblk = 1;
      bp.ntiles = batch_tiles(bp.n, bp.kind, bp.a, &nblk);
      bp.a.nblk_i = nblk;
      bp.a.async_ok = 0;
      bp.done = counter++;
      bp.dep = (p == 0) ? -1 : bp.done - 1;
      per[i].push_back(bp);
    }
  }
  for (int i = 0; i < count; ++i)
    for (size_t p = 1; p < per[i].size(); ++p) per[i][p].dep_need = per[i][p].dep_need_orig = per[i][p - 1].ntiles;
  // within a level, the largest densities first: their longer dependency
  // chains start early and the small ones fill the tail
  std::vector<int> order(count);
  std::vector<double> work(count);
  for (int i = 0; i < count; ++i) {
    order[i] = i;
    work[i] = (double)plan_points(plans[i]);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  long long base = 0;
  for (int level = 0; level < 5; ++level)
    for (int i : order)
      if (level < (int)per[i].size()) {
        BatchPass bp = per[i][level];
        bp.item_base = base;
        base += bp.ntiles;
        b->host_passes.push_back(bp);
      }
  b->total_items = base;
  if (base >= (1LL << 31)) {
    vp_batch_destroy(b);
    return VP_ERR_UNSUPPORTED;
  }
  const size_t npass = b->host_passes.size();
  e = cudaMalloc(&b->passes, npass * sizeof(BatchPass));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->passes, b->host_passes.data(), npass * sizeof(BatchPass), cudaMemcpyHostToDevice);
  b->ctrl_bytes = sizeof(unsigned long long) + npass * sizeof(long long) + sizeof(int) * 4;
  if (e == cudaSuccess) e = cudaMalloc(&b->ctrl, b->ctrl_bytes);
  if (e == cudaSuccess) e = cudaMemset(b->ctrl, 0, b->ctrl_bytes);
  if (e != cudaSuccess) {
    vp_batch_destroy(b);
    return VP_ERR_CUDA;
  }
  b->next_item = reinterpret_cast<unsigned long long*>(b->ctrl);
  b->done = reinterpret_cast<long long*>(b->next_item + 1);
  b->err = reinterpret_cast<int*>(b->done + npass);
  // persistent grids: all resident CTAs, or one per SM
  int sms = 0, per_sm = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, b->device);  // kHz
  cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, BATCH_THREADS, batch_smem_bytes());
  b->grid_full = sms * std::max(1, per_sm);
  b->grid_one = sms;
  b->timeout_cycles = (long long)std::max(clk, 1000000) * 1000LL * 2;  // about 2 s
  // autotuner key: device, driver and the batch's (d, N) multiset
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, b->device);
  int drv = 0;
  cudaDriverGetVersion(&drv);
  std::vector<std::string> parts;
  for (int i = 0; i < count; ++i) {
    int d, N, dims[3];
    vp_plan_info(plans[i], &d, &N, nullptr, nullptr, nullptr);
    plan_dims(plans[i], dims);
    std::string g = std::to_string(dims[0]);
    for (int a = 1; a < d; ++a) g += "x" + std::to_string(dims[a]);
    parts.push_back(std::to_string(d) + "d" + g);
  }
  std::sort(parts.begin(), parts.end());
  std::string sig = std::string(prop.name) + "|drv" + std::to_string(drv) + "|";
  for (auto& s : parts) sig += s + ",";
  for (auto& c : sig)
    if (c == ' ') c = '_';
  b->signature = sig;
  const int cached = vp::autotune_cache_lookup(sig);
  b->strategy = cached % 100;
  if (cached >= 100) b->chunk = cached / 100;
  if (const double secs = vp::env_timeout_seconds()) vp_batch_set_timeout(b, secs);
  *out = b;
  return VP_OK;
}

vp_status vp_batch_set_stream(vp_batch b, void* stream) {
  if (!b) return VP_ERR_INVALID_ARG;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  return VP_OK;
}

vp_status vp_batch_set_strategy(vp_batch b, int strategy) {
  if (!b || strategy < 0 || strategy > 4) return VP_ERR_INVALID_ARG;
  b->forced = strategy;
  return VP_OK;
}

vp_status vp_batch_set_chunk(vp_batch b, int chunk) {
  if (!b || chunk < 0 || chunk > 256) return VP_ERR_INVALID_ARG;
  b->forced_chunk = chunk;
  return VP_OK;
}

vp_status vp_batch_get_chunk(vp_batch b, int* chunk) {
  if (!b || !chunk) return VP_ERR_INVALID_ARG;
  *chunk = b->forced_chunk ? b->forced_chunk : b->chunk;
  return VP_OK;
}

vp_status vp_batch_get_strategy(vp_batch b, int* strategy) {
  if (!b || !strategy) return VP_ERR_INVALID_ARG;
  *strategy = b->forced ? b->forced : b->strategy;
  return VP_OK;
}

vp_status vp_batch_set_timeout(vp_batch b, double seconds) {
  if (!b || !(seconds > 0)) return VP_ERR_INVALID_ARG;
  int clk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, b->device);
  b->timeout_cycles = (long long)(seconds * std::max(clk, 1000000) * 1000.0);
  return VP_OK;
}

vp_status vp_batch_withhold(vp_batch b, int density, int pass) {
  if (!b) return VP_ERR_INVALID_ARG;
  if (pass <= 0) {  // restore every dependency
    for (size_t k = 0; k < b->host_passes.size(); ++k) {
      BatchPass& bp = b->host_passes[k];
      if (bp.dep >= 0 && bp.dep_need != bp.dep_need_orig) {
        bp.dep_need = bp.dep_need_orig;
        if (cudaMemcpy(b->passes + k, &bp, sizeof(BatchPass), cudaMemcpyHostToDevice) != cudaSuccess)
          return VP_ERR_CUDA;
      }
    }
    return VP_OK;
  }
  if (density < 0 || density >= b->count) return VP_ERR_INVALID_ARG;
  int level = 0;
  for (size_t k = 0; k < b->host_passes.size(); ++k) {
    BatchPass& bp = b->host_passes[k];
    if (bp.density != density) continue;
    if (level == pass) {
      // this pass now waits for one tile more than its predecessor has
      bp.dep_need = bp.dep_need_orig + 1;
      return cudaMemcpy(b->passes + k, &bp, sizeof(BatchPass), cudaMemcpyHostToDevice) == cudaSuccess ? VP_OK
                                                                                                   : VP_ERR_CUDA;
    }
    ++level;
  }
  return VP_ERR_INVALID_ARG;
}

vp_status vp_batch_apply(vp_batch b, const void* const* f, void* const* phi) {
  vp::NvtxRange range("vp_batch_apply");
  if (!b || !f || !phi) return VP_ERR_INVALID_ARG;
  for (int i = 0; i < b->count; ++i)
    if (!f[i] || !phi[i]) return bfail(b, VP_ERR_INVALID_ARG, "NULL density pointer");
  vp::DeviceGuard dg_(b->device);
  if (dg_.error() != cudaSuccess) return VP_ERR_CUDA;
  int s = b->forced;
  if (!s) {
    if (!b->strategy) {
      vp_status st = autotune(b, f, phi);
      if (st != VP_OK) return st;
    }
    s = b->strategy;
  }
  return run_strategy(b, s, f, phi);
}

vp_status vp_batch_status(vp_batch b) {
  if (!b) return VP_ERR_INVALID_ARG;
  vp::DeviceGuard dg_(b->device);
  if (dg_.error() != cudaSuccess) return VP_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, VP_ERR_CUDA, "stream sync");
  int err = 0;
  if (cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return VP_ERR_CUDA;
  if (err) {
    cudaMemset(b->err, 0, sizeof(int));
    return bfail(b, VP_ERR_TIMEOUT, "a batch tile gave up waiting for the pass it depends on");
  }
  return VP_OK;
}

vp_status vp_batch_info(vp_batch b, long long* items, int* passes, size_t* device_bytes) {
  if (!b) return VP_ERR_INVALID_ARG;
  if (items) *items = b->total_items;
  if (passes) *passes = (int)b->host_passes.size();
  if (device_bytes) *device_bytes = b->ws_bytes + b->ctrl_bytes + b->host_passes.size() * sizeof(BatchPass);
  return VP_OK;
}

const char* vp_batch_last_error(vp_batch b) { return b ? b->last_error.c_str() : ""; }

vp_status vp_batch_destroy(vp_batch b) {
  if (!b) return VP_OK;
  vp::DeviceGuard dg_(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->sexec) cudaGraphExecDestroy(b->sexec);
  if (b->sgraph) cudaGraphDestroy(b->sgraph);
  for (int k = 0; k < kSideStreams; ++k) {
    if (b->side[k]) {
      cudaStreamSynchronize(b->side[k]);
      cudaStreamDestroy(b->side[k]);
    }
    if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  cudaFree(b->passes);
  cudaFree(b->ctrl);
  cudaFree(b->ws);
  delete b;
  return VP_OK;
}

}  // extern "C"
