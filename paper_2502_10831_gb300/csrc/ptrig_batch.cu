// ptrig_batch.cu -- ragged batch: thousands of arrays, each with its own
// function selector, evaluated by one kernel launch.
//
// The plan cuts every array into tiles of block * items_per_thread elements
// and uploads a table of 32-byte tile descriptors (pointers already offset to
// the tile, and its length), grouped by selector.  k_batch_tiles runs one
// block per tile: a single broadcast load finds the tile, the block index
// range gives its selector (uniform over the block), and the block streams the
// tile with the inline vector code of the elementwise kernels (a ring of four
// 16-byte loads per thread).  Many small resident blocks hide the memory
// latency, as in the one-shot elementwise kernels, and no per-tile call
// remains.  An array whose pointers share one misalignment inside a
// 16-byte line gets a separate head tile of at most three elements, so that
// its other tiles start aligned.  With PTRIG_BATCH_GRAPH the launch is
// captured once into a CUDA graph and ptrig_batch_run replays it.
//
// The no-allocation entry point further below keeps a persistent kernel over
// a per-array tile table that it builds on the device.
#include <algorithm>
#include <mutex>
#include <vector>

#include "ptrig_map.cuh"

namespace ptrig {
// One tile of one array: pointers offset to the tile's first element.
struct BatchTile {
  const float *x;
  float *y0;
  float *y1;  // sincos only
  uint32_t len;
  uint32_t pad;
};
static_assert(sizeof(BatchTile) == 32, "BatchTile layout");
}  // namespace ptrig

struct ptrig_batch_plan {
  int device = -1;
  unsigned flags = 0;
  std::vector<ptrig_desc> host;
  ptrig::BatchTile *d_tiles = nullptr;
  size_t tiles_cap = 0;
  uint64_t op_off[4] = {};  // first tile of each selector in d_tiles
  uint64_t op_cnt[4] = {};  // tiles of each selector
  uint64_t ntiles = 0;
  int block = 128;
  int items = 16;
  int grid = 0;  // blocks launched per run (one per tile)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace ptrig {

static_assert(sizeof(ptrig_desc) == 40, "ptrig_desc layout");

// Vectors v, v + blockDim, ... < nv of one tile with the full reduction (out
// of line; reached only when the tile holds an angle beyond the FP32
// reduction range).
template <int OP>
static __device__ __noinline__ void batch_resume_full(const float *x, float *y0, float *y1, uint32_t v,
                                                      uint32_t nv, const STab *tab) {
  using F = Proposed<OP>;
  for (; v < nv; v += blockDim.x) {
    float f[4], o0[4], o1[4];
    Storage<float>::unpack(ld_stream(reinterpret_cast<const uint4 *>(x) + v), f);
    for (int e = 0; e < 4; ++e) F::template eval<true>(f[e], tab, o0[e], o1[e]);
    st_stream(reinterpret_cast<uint4 *>(y0) + v, Storage<float>::pack(o0));
    if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + v, Storage<float>::pack(o1));
  }
}

// Elements [from, len) of a tile one at a time (unaligned arrays, n % 4 tails);
// out of line like the full-reduction path.
template <int OP>
static __device__ __noinline__ void batch_elements(const float *x, float *y0, float *y1, uint32_t from,
                                                   uint32_t len, const STab *tab) {
  using F = Proposed<OP>;
  for (uint32_t i = from + threadIdx.x; i < len; i += blockDim.x) {
    float o0, o1;
    F::template eval<true>(__ldg(x + i), tab, o0, o1);
    y0[i] = o0;
    if constexpr (F::NOUT == 2) y1[i] = o1;
  }
}

// One tile (len elements from `start` of array d).  Vector path when the
// tile's pointers are 16-byte aligned: each thread issues up to four loads,
// then computes one vector at a time; element path otherwise and for the
// n % 4 tail.
template <int OP>
static __device__ __noinline__ void batch_tile(const ptrig_desc d, uint64_t start, uint32_t len,
                                               const STab *tab) {
  using F = Proposed<OP>;
  const float *x = d.x + start;
  float *y0 = d.y0 + start;
  float *y1 = (OP == OP_SINCOS) ? d.y1 + start : nullptr;
  // A common offset inside the 16-byte line (arrays packed at arbitrary
  // element offsets): peel up to three elements, then vectors.
  const uint32_t ox = (uint32_t)((uintptr_t)x & 15u);
  const bool same = ((uint32_t)((uintptr_t)y0 & 15u) == ox) &&
                    (OP != OP_SINCOS || (uint32_t)((uintptr_t)y1 & 15u) == ox) && (ox & 3u) == 0;
  uint32_t head = 0, done = 0;
  if (same) {
    head = ox ? (16u - ox) / 4u : 0u;
    if (head > len) head = len;
    constexpr int U = 4;
    const uint32_t nv = (len - head) / 4;
    const float *xa = x + head;
    float *y0a = y0 + head;
    float *y1a = (OP == OP_SINCOS) ? y1 + head : nullptr;
    const uint4 *xv = reinterpret_cast<const uint4 *>(xa);
    uint32_t resume = 0;
    for (uint32_t v0 = threadIdx.x; v0 < nv; v0 += blockDim.x * U) {
      uint4 buf[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = v0 + u * blockDim.x;
        if (i < nv) buf[u] = ld_stream(xv + i);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = v0 + u * blockDim.x;
        if (i < nv && !map_vector_fast<float, F>(buf[u], i, y0a, y1a, tab)) {
          resume = i + 1;
          goto full;
        }
      }
    }
  full:
    if (resume) batch_resume_full<OP>(xa, y0a, y1a, resume - 1, nv, tab);
    done = head + nv * 4;
  }
  if (head > 0) batch_elements<OP>(x, y0, y1, 0, head, tab);
  if (done < len) batch_elements<OP>(x, y0, y1, done, len, tab);
}

// One tile of selector OP by one block.  Vector path when the tile's pointers
// are 16-byte aligned (a ring of four 16-byte loads per thread, the next load
// of a slot issued before the slot's vector is computed); element path
// otherwise and for the len % 4 tail; out-of-line full reduction after an
// angle beyond the FP32 reduction range, as in the elementwise kernels.
template <int OP>
__device__ __forceinline__ void batch_block(const BatchTile &t, STab *s_tab) {
  using F = Proposed<OP>;
  float *y1 = (OP == OP_SINCOS) ? t.y1 : nullptr;
  uintptr_t a = (uintptr_t)t.x | (uintptr_t)t.y0;
  if (OP == OP_SINCOS) a |= (uintptr_t)y1;
  const uint32_t nv = (a & 15u) ? 0u : t.len / 4u;
  constexpr int R = 4;
  const uint4 *xv = reinterpret_cast<const uint4 *>(t.x);
  uint4 buf[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = threadIdx.x + r * blockDim.x;
    if (i < nv) buf[r] = ld_stream(xv + i);
  }
  // the table is staged while the first loads are in flight (the selector is
  // uniform over the block, so every thread reaches this barrier)
  stage_stab(s_tab);
  __syncthreads();
  uint32_t resume = 0;
  for (uint32_t v0 = threadIdx.x; v0 < nv; v0 += R * blockDim.x) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t i = v0 + r * blockDim.x;
      if (i < nv) {
        const uint4 cur = buf[r];
        const uint32_t nx = i + R * blockDim.x;
        if (nx < nv) buf[r] = ld_stream(xv + nx);
        if (!map_vector_fast<float, F>(cur, i, t.y0, y1, s_tab)) {
          resume = i + 1;
          goto full;
        }
      }
    }
  }
  goto tail;
full:
  batch_resume_full<OP>(t.x, t.y0, y1, resume - 1, nv, s_tab);
tail:
  if (nv * 4u < t.len) batch_elements<OP>(t.x, t.y0, y1, nv * 4u, t.len, s_tab);
}

// One launch for the whole batch: the tiles are stored by selector (sin,
// cos, tan, sincos), and block b takes tile b with the selector whose range
// holds b -- uniform over the block, so the branch never diverges.
__global__ void __launch_bounds__(512) k_batch_tiles(const BatchTile *__restrict__ tiles, uint32_t end_sin,
                                                     uint32_t end_cos, uint32_t end_tan) {
  __shared__ STab s_tab;
  const uint32_t b = blockIdx.x;
  const BatchTile t = tiles[b];
  if (b < end_sin)
    batch_block<OP_SIN>(t, &s_tab);
  else if (b < end_cos)
    batch_block<OP_COS>(t, &s_tab);
  else if (b < end_tan)
    batch_block<OP_TAN>(t, &s_tab);
  else
    batch_block<OP_SINCOS>(t, &s_tab);
}

// ---------------------------------------------------------------------------
// Batch entry point that allocates nothing (ptrig_batch_run_noalloc).
//
// Its only scratch is the table below: the first tile of each array plus the
// total tile count, rewritten by every call.  A file-scope __device__ array
// is reserved when the library loads on a device and stays until the process
// exits, so a call needs no cudaMalloc.  Host code cannot use the name
// g_noalloc_first_tile as a device address; the address is looked up once per
// device with cudaGetSymbolAddress (noalloc_scratch()).
#define PTRIG_NOALLOC_MAX_ARRAYS 16384
static __device__ __align__(256) uint64_t g_noalloc_first_tile[PTRIG_NOALLOC_MAX_ARRAYS + 1];

// A descriptor the batch can use: known selector, reserved == 0 and non-NULL
// pointers for a non-empty array.  Others count as empty and are skipped.
__device__ __forceinline__ bool noalloc_desc_ok(const ptrig_desc &d) {
  if (d.func > PTRIG_SINCOS || d.reserved != 0) return false;
  if (d.n == 0) return true;
  return d.x && d.y0 && (d.func != PTRIG_SINCOS || d.y1);
}

// One block of 1024 threads: tiles per array and their exclusive prefix sum
// into first_tile[0 .. count] (first_tile[count] = total tiles).
__global__ void __launch_bounds__(1024) k_noalloc_prefix(const ptrig_desc *__restrict__ descs, uint32_t count,
                                                         uint32_t tile_elems, uint64_t *first_tile) {
  __shared__ uint64_t s_part[1024];
  const uint32_t per = (count + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = threadIdx.x * per;
  const uint32_t hi = min(count, lo + per);
  uint64_t sum = 0;
  for (uint32_t i = lo; i < hi; ++i) {
    const ptrig_desc d = descs[i];
    if (noalloc_desc_ok(d)) sum += (d.n + tile_elems - 1) / tile_elems;
  }
  s_part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan of the 1024 partial sums
    uint64_t run = 0;
    for (uint32_t t = 0; t < blockDim.x; ++t) {
      const uint64_t v = s_part[t];
      s_part[t] = run;
      run += v;
    }
    first_tile[count] = run;
  }
  __syncthreads();
  uint64_t run = s_part[threadIdx.x];
  for (uint32_t i = lo; i < hi; ++i) {
    first_tile[i] = run;
    const ptrig_desc d = descs[i];
    if (noalloc_desc_ok(d)) run += (d.n + tile_elems - 1) / tile_elems;
  }
}

// Persistent batch kernel over the table above: a tile finds its array by
// binary search on first_tile (the largest i with first_tile[i] <= tile),
// then runs the same per-tile code as k_batch.
__global__ void __launch_bounds__(512, 2) k_batch_noalloc(const ptrig_desc *__restrict__ descs, uint32_t count,
                                                          const uint64_t *__restrict__ first_tile,
                                                          uint32_t tile_elems) {
  __shared__ STab s_tab;
  stage_stab(&s_tab);
  __syncthreads();
  const uint64_t ntiles = first_tile[count];
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint32_t lo = 0, hi = count;  // first_tile[lo] <= tile < first_tile[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (first_tile[mid] <= tile)
        lo = mid;
      else
        hi = mid;
    }
    const ptrig_desc d = descs[lo];
    const uint64_t start = (tile - first_tile[lo]) * (uint64_t)tile_elems;
    const uint64_t rem = d.n - start;
    const uint32_t len = rem < tile_elems ? (uint32_t)rem : tile_elems;
    switch (d.func) {
      case PTRIG_SIN:
        batch_tile<OP_SIN>(d, start, len, &s_tab);
        break;
      case PTRIG_COS:
        batch_tile<OP_COS>(d, start, len, &s_tab);
        break;
      case PTRIG_TAN:
        batch_tile<OP_TAN>(d, start, len, &s_tab);
        break;
      default:
        batch_tile<OP_SINCOS>(d, start, len, &s_tab);
        break;
    }
  }
}

// Device address of g_noalloc_first_tile on the current device, looked up on
// the first call per device and cached.
static ptrig_status noalloc_scratch(uint64_t **out) {
  static std::mutex mu;
  static uint64_t *cache[64] = {};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= 64) return PTRIG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_first_tile);
    if (e != cudaSuccess) return cuda_fail(e);
    cache[dev] = static_cast<uint64_t *>(ptr);
  }
  *out = cache[dev];
  return PTRIG_OK;
}

static void free_graph(ptrig_batch_plan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

static ptrig_status launch_batch(ptrig_batch_plan *p, cudaStream_t s) {
  if (p->ntiles == 0) return PTRIG_OK;
  k_batch_tiles<<<(unsigned)p->ntiles, p->block, 0, s>>>(
      p->d_tiles, (uint32_t)p->op_cnt[0], (uint32_t)(p->op_cnt[0] + p->op_cnt[1]),
      (uint32_t)(p->op_cnt[0] + p->op_cnt[1] + p->op_cnt[2]));
  return finish_launch();
}

static ptrig_status capture_graph(ptrig_batch_plan *p) {
  free_graph(p);
  if (!(p->flags & PTRIG_BATCH_GRAPH) || p->ntiles == 0) return PTRIG_OK;
  cudaError_t e;
  if (!p->cap_stream) {
    e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e);
  const ptrig_status st = launch_batch(p, p->cap_stream);
  e = cudaStreamEndCapture(p->cap_stream, &p->graph);
  if (st != PTRIG_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e);
  return PTRIG_OK;
}

// Rebuilds the per-selector tile lists for the plan's (block, items) and
// uploads them (synchronous).
static ptrig_status build_tiles(ptrig_batch_plan *p) {
  const uint64_t tile = (uint64_t)p->block * (uint64_t)p->items;
  std::vector<BatchTile> lists[4];
  for (const ptrig_desc &d : p->host) {
    if (d.n == 0) continue;
    const int op = (int)d.func;
    float *y1 = (op == OP_SINCOS) ? d.y1 : nullptr;
    uint64_t off = 0;
    const uintptr_t ox = (uintptr_t)d.x & 15u;
    if (ox != 0 && (ox & 3u) == 0 && ((uintptr_t)d.y0 & 15u) == ox && (!y1 || ((uintptr_t)y1 & 15u) == ox)) {
      off = std::min<uint64_t>(d.n, (16u - ox) / 4u);  // head tile up to the 16-byte boundary
      lists[op].push_back(BatchTile{d.x, d.y0, y1, (uint32_t)off, 0u});
    }
    for (; off < d.n; off += tile) {
      const uint64_t len = std::min<uint64_t>(tile, d.n - off);
      lists[op].push_back(BatchTile{d.x + off, d.y0 + off, y1 ? y1 + off : nullptr, (uint32_t)len, 0u});
    }
  }
  uint64_t nt = 0;
  for (int op = 0; op < 4; ++op) {
    p->op_off[op] = nt;
    p->op_cnt[op] = lists[op].size();
    nt += lists[op].size();
  }
  if (nt > 0x7fffffffull) return PTRIG_ERR_INVALID_ARG;  // one block per tile: grid limit
  cudaError_t e;
  if (nt > p->tiles_cap) {
    if (p->d_tiles) cudaFree(p->d_tiles);
    p->d_tiles = nullptr;
    p->tiles_cap = 0;
    e = cudaMalloc(&p->d_tiles, (size_t)nt * sizeof(BatchTile));
    if (e != cudaSuccess) return cuda_fail(e);
    p->tiles_cap = (size_t)nt;
  }
  for (int op = 0; op < 4; ++op) {
    if (lists[op].empty()) continue;
    e = cudaMemcpy(p->d_tiles + p->op_off[op], lists[op].data(), lists[op].size() * sizeof(BatchTile),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  p->ntiles = nt;
  p->grid = (int)std::min<uint64_t>(nt, 0x7fffffffull);
  return capture_graph(p);
}

}  // namespace ptrig

using namespace ptrig;

extern "C" {

ptrig_status ptrig_batch_plan_create(ptrig_batch_plan **plan, const ptrig_desc *host_descs, size_t count,
                                     int flags) {
  if (!plan) return PTRIG_ERR_INVALID_ARG;
  *plan = nullptr;
  if (count > 0 && !host_descs) return PTRIG_ERR_INVALID_ARG;
  if (count > 0xffffffffull) return PTRIG_ERR_INVALID_ARG;
  if (flags & ~(int)PTRIG_BATCH_GRAPH) return PTRIG_ERR_INVALID_ARG;
  for (size_t i = 0; i < count; ++i) {
    const ptrig_desc &d = host_descs[i];
    if (d.func > PTRIG_SINCOS || d.reserved != 0) return PTRIG_ERR_INVALID_ARG;
    if (d.n > 0 && (!d.x || !d.y0 || (d.func == PTRIG_SINCOS && !d.y1))) return PTRIG_ERR_INVALID_ARG;
    if (d.n > (1ull << 62)) return PTRIG_ERR_INVALID_ARG;
  }
  if (sm_count() <= 0) return PTRIG_ERR_NO_DEVICE;
  ptrig_batch_plan *p = new ptrig_batch_plan();
  p->flags = (unsigned)flags;
  cudaGetDevice(&p->device);
  p->host.assign(host_descs, host_descs + count);
  const ptrig_status st = build_tiles(p);
  if (st != PTRIG_OK) {
    ptrig_batch_plan_destroy(p);
    return st;
  }
  *plan = p;
  return PTRIG_OK;
}

ptrig_status ptrig_batch_run(ptrig_batch_plan *plan, ptrig_stream stream) {
  if (!plan) return PTRIG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (plan->exec) {
    const cudaError_t e = cudaGraphLaunch(plan->exec, s);
    return e == cudaSuccess ? PTRIG_OK : cuda_fail(e);
  }
  return launch_batch(plan, s);
}

ptrig_status ptrig_batch_run_per_array(ptrig_batch_plan *plan, ptrig_stream stream) {
  if (!plan) return PTRIG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (const ptrig_desc &d : plan->host) {
    if (d.n == 0) continue;
    const ptrig_status st = launch_proposed_f32((int)d.func, d.x, d.y0, d.y1, (size_t)d.n, s);
    if (st != PTRIG_OK) return st;
  }
  return PTRIG_OK;
}

ptrig_status ptrig_batch_plan_set_config(ptrig_batch_plan *plan, int block, int items_per_thread) {
  if (!plan) return PTRIG_ERR_INVALID_ARG;
  const int b = block ? block : plan->block;
  const int it = items_per_thread ? items_per_thread : plan->items;
  if (b < 64 || b > 512 || b % 32 != 0 || it < 4 || it > 256 || it % 4 != 0) return PTRIG_ERR_INVALID_ARG;
  plan->block = b;
  plan->items = it;
  return build_tiles(plan);
}

ptrig_status ptrig_batch_plan_get_config(const ptrig_batch_plan *plan, int *block, int *items_per_thread,
                                         uint64_t *tiles, int *grid) {
  if (!plan) return PTRIG_ERR_INVALID_ARG;
  if (block) *block = plan->block;
  if (items_per_thread) *items_per_thread = plan->items;
  if (tiles) *tiles = plan->ntiles;
  if (grid) *grid = plan->grid;
  return PTRIG_OK;
}

ptrig_status ptrig_batch_plan_autotune(ptrig_batch_plan *plan, ptrig_stream stream, int reps,
                                       const int *cand_block, const int *cand_items, int ncand,
                                       int *best_block, int *best_items, float *best_ms) {
  if (!plan || reps < 1 || ncand < 0 || (ncand > 0 && (!cand_block || !cand_items))) return PTRIG_ERR_INVALID_ARG;
  static const int kBlocks[] = {128, 128, 256, 256, 128, 512, 256, 128};
  static const int kItems[] = {16, 32, 16, 32, 64, 16, 8, 8};
  const int nc = ncand ? ncand : (int)(sizeof(kBlocks) / sizeof(kBlocks[0]));
  const int *cb = ncand ? cand_block : kBlocks;
  const int *ci = ncand ? cand_items : kItems;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(e);
  }
  const unsigned saved_flags = plan->flags;
  plan->flags &= ~PTRIG_BATCH_GRAPH;  // time plain launches while searching
  float best = -1.0f;
  int bb = plan->block, bi = plan->items;
  ptrig_status st = PTRIG_OK;
  for (int c = 0; c < nc && st == PTRIG_OK; ++c) {
    st = ptrig_batch_plan_set_config(plan, cb[c], ci[c]);
    if (st != PTRIG_OK) break;
    st = launch_batch(plan, s);
    if (st != PTRIG_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == PTRIG_OK; ++r) st = launch_batch(plan, s);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e);
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (best < 0.0f || ms < best) {
      best = ms;
      bb = plan->block;
      bi = plan->items;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->flags = saved_flags;
  if (st != PTRIG_OK) return st;
  st = ptrig_batch_plan_set_config(plan, bb, bi);
  if (st != PTRIG_OK) return st;
  if (best_block) *best_block = bb;
  if (best_items) *best_items = bi;
  if (best_ms) *best_ms = best;
  return PTRIG_OK;
}

ptrig_status ptrig_batch_run_noalloc(const ptrig_desc *device_descs, size_t count, ptrig_stream stream) {
  if (count == 0) return PTRIG_OK;
  if (!device_descs) return PTRIG_ERR_INVALID_ARG;
  if (count > PTRIG_NOALLOC_MAX_ARRAYS) return PTRIG_ERR_INVALID_ARG;
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  uint64_t *first_tile = nullptr;
  const ptrig_status st = noalloc_scratch(&first_tile);
  if (st != PTRIG_OK) return st;
  const int block = 256, items = 32;
  const uint32_t tile_elems = (uint32_t)(block * items);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_noalloc_prefix<<<1, 1024, 0, s>>>(device_descs, (uint32_t)count, tile_elems, first_tile);
  ptrig_status ls = finish_launch();
  if (ls != PTRIG_OK) return ls;
  const int occ = occupancy((const void *)k_batch_noalloc, block);
  const int grid = sms * (occ > 0 ? occ : 1);
  k_batch_noalloc<<<grid, block, 0, s>>>(device_descs, (uint32_t)count, first_tile, tile_elems);
  return finish_launch();
}

void ptrig_batch_plan_destroy(ptrig_batch_plan *plan) {
  if (!plan) return;
  free_graph(plan);
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  if (plan->d_tiles) cudaFree(plan->d_tiles);
  delete plan;
}

}  // extern "C"
