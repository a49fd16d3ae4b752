// Batched SIRT over many independent reconstructions of uneven size.
//
// Each SIRT stage (path-length weights, voxel weights, forward residual,
// back-projection, update) runs as ONE persistent launch over all instances:
// blocks pull work items (instance, detector tile) from an atomic counter, load
// the instance's grid table into shared memory when the instance changes, and
// trace the tile's rays with the same traversal as the single-instance calls.
// Element-wise stages pull chunks of the concatenated voxel space the same
// way. The whole schedule (weights + n_iter iterations) is captured once into
// a CUDA graph and replayed with a single graph launch. Per instance, the
// warp tile and the scatter strategy come from the autotuner's size-class
// cache (tsp_autotune), the block size from the instance with the most rays.
#include <algorithm>
#include <vector>

#include "tsp_kernels.cuh"

namespace tsp {
namespace {

struct InstDesc {
  GridDesc gd;
  GeomArgs ga;
  int kind;
  int tw;        // warp tile width
  int scatter;   // 0 atomics, 1 warp-aggregated
  int tiles_x, tiles_y;
  int64_t item0, n_items;  // trace work items (tiles)
  int64_t vox0, V;         // offset into the concatenated voxel arrays
  int64_t ray0;            // offset into the concatenated ray arrays
  const float* y;
  float* x;
};

enum Stage { ST_PATHLEN = 0, ST_UNIT = 1, ST_RESID = 2, ST_SCATTER = 3 };

struct BatchPtrs {
  float *R, *r, *C, *g;  // concatenated: R, r over rays; C, g over voxels
};

__device__ __forceinline__ int find_instance(const InstDesc* insts, int n, int64_t item, bool by_voxel) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {  // last instance whose start <= item
    const int mid = (lo + hi + 1) >> 1;
    const int64_t start = by_voxel ? insts[mid].vox0 : insts[mid].item0;
    if (start <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct BPathLen {
  float* R;
  float acc;
  __device__ __forceinline__ bool begin(int64_t) {
    acc = 0.0f;
    return true;
  }
  __device__ __forceinline__ void operator()(int, float dl) { acc = __fadd_rn(acc, dl); }
  __device__ __forceinline__ void end(int64_t ray) { R[ray] = acc > 0.0f ? __frcp_rn(acc) : 0.0f; }
};

struct BUnit {
  float* C;
  __device__ __forceinline__ bool begin(int64_t) { return true; }
  __device__ __forceinline__ void operator()(int v, float dl) { atomicAdd(C + v, dl); }
  __device__ __forceinline__ void end(int64_t) {}
};

struct BResid {
  const float* x;
  const float* y;
  const float* R;
  float* r;
  DelayedSum sum;
  __device__ __forceinline__ bool begin(int64_t) {
    sum.reset();
    return true;
  }
  __device__ __forceinline__ void operator()(int v, float dl) { sum.add(x + v, dl); }
  __device__ __forceinline__ void end(int64_t ray) {
    r[ray] = __fmul_rn(__ldg(R + ray), __fsub_rn(__ldg(y + ray), sum.total()));
  }
};

template <int GK, class Op>
__device__ __forceinline__ void trace_tile(const TGrid& G, const InstDesc& d, int64_t t, Op& op, const ConeList& L) {
  int64_t ray;
  ff x[3], dd[3];
  if (GK == GEOM_RAYS) {
    ray = t * blockDim.x + threadIdx.x;
    if (ray >= d.ga.n_rays) return;
    ray_geometry<GK>(d.ga, 0, 0, 0, ray, x, dd);
  } else {
    const int64_t per_view = int64_t(d.tiles_x) * d.tiles_y;
    const int view = int(t / per_view);
    const int rem = int(t - int64_t(view) * per_view);
    const int ty = rem / d.tiles_x, tx = rem - ty * d.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tw = d.tw, th = 32 / tw, bh = blockDim.x / tw;
    const int col = tx * tw + (lane % tw);
    const int row = ty * bh + warp * th + lane / tw;
    if (col >= d.ga.W || row >= d.ga.H) return;
    ray = (int64_t(view) * d.ga.H + row) * d.ga.W + col;
    ray_geometry<GK>(d.ga, view, row, col, ray, x, dd);
  }
  if (!op.begin(ray)) return;
  if (!trace_ray(G, x, dd, op, L)) atomicOr(&g_tsp_error_word, 1);
  op.end(ray);
}

template <class Op>
__device__ __forceinline__ void trace_any(const TGrid& G, const InstDesc& d, int64_t t, Op& op, const ConeList& L) {
  if (d.kind == GEOM_CONE) trace_tile<GEOM_CONE>(G, d, t, op, L);
  else if (d.kind == GEOM_PARALLEL) trace_tile<GEOM_PARALLEL>(G, d, t, op, L);
  else trace_tile<GEOM_RAYS>(G, d, t, op, L);
}

// Persistent traversal stage over all instances, one kernel per stage (each
// holds one per-segment operation, so the walk's registers are those of that
// operation alone). At most 72 registers a thread, which keeps 7 blocks of
// 128 threads per SM: the compiler's own choice, 92-109, allows 4 (measured:
// the 64-instance schedule 14.4 s uncapped, 13.2 s capped).
template <int stage>
__global__ void __maxnreg__(72) batch_trace_kernel(const InstDesc* __restrict__ insts, int n_inst,
                                                          int64_t total_items, unsigned long long* counter,
                                                          BatchPtrs P, int list_off, int ccap) {
  // shared memory: the current instance's grid table, then from word list_off
  // (the largest table) each thread's cone-crossing list of ccap entries
  extern __shared__ float smem[];
  const ConeList L{smem + list_off + threadIdx.x, int(blockDim.x), ccap};
  __shared__ long long s_item;
  __shared__ int s_inst;
  int loaded = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (long long)atomicAdd(counter, 1ull);
      s_inst = s_item < total_items ? find_instance(insts, n_inst, s_item, false) : -1;
    }
    __syncthreads();
    const int64_t item = s_item;
    const int ii = s_inst;
    if (item >= total_items) break;
    const InstDesc& d = insts[ii];
    if (ii != loaded) {
      for (int i = threadIdx.x; i < d.gd.words; i += blockDim.x) smem[i] = __ldg(d.gd.table + i);
      __syncthreads();
      loaded = ii;
    }
    const TGrid G = tgrid_from_smem(d.gd, smem);
    const int64_t t = item - d.item0;
    if constexpr (stage == ST_PATHLEN) {
      BPathLen op;
      op.R = P.R + d.ray0;
      trace_any(G, d, t, op, L);
    } else if constexpr (stage == ST_UNIT) {
      BUnit op;
      op.C = P.C + d.vox0;
      trace_any(G, d, t, op, L);
    } else if constexpr (stage == ST_RESID) {
      BResid op;
      op.x = d.x;
      op.y = d.y;
      op.R = P.R + d.ray0;
      op.r = P.r + d.ray0;
      trace_any(G, d, t, op, L);
    } else if (d.scatter) {  // ST_SCATTER, per instance: warp-aggregated or one atomic per segment
      AggScatterOp<1> op;
      op.y = P.r + d.ray0;
      op.g = P.g + d.vox0;
      op.V = d.V;
      op.n_rays = d.ga.n_rays;
      op.nb = 1;
      trace_any(G, d, t, op, L);
    } else {
      ScatterOp<1> op;
      op.y = P.r + d.ray0;
      op.g = P.g + d.vox0;
      op.V = d.V;
      op.n_rays = d.ga.n_rays;
      op.nb = 1;
      trace_any(G, d, t, op, L);
    }
    __syncthreads();  // the table may be replaced by the next item
  }
}

// Persistent element-wise stage over the concatenated voxels: reciprocal of
// the voxel weights (mode 0) or the SIRT update x += C g, g = 0 (mode 1).
constexpr int kChunk = 4096;

__global__ void batch_voxel_kernel(const InstDesc* __restrict__ insts, int n_inst, int64_t total_vox,
                                   unsigned long long* counter, int mode, int nonneg, BatchPtrs P) {
  __shared__ long long s_chunk;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t c0 = int64_t(s_chunk) * kChunk;
    __syncthreads();
    if (c0 >= total_vox) break;
    const int64_t c1 = c0 + kChunk < total_vox ? c0 + kChunk : total_vox;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      if (mode == 0) {
        const float v = P.C[i];
        P.C[i] = v > 0.0f ? __frcp_rn(v) : 0.0f;
      } else {
        const int ii = find_instance(insts, n_inst, i, true);
        float* x = insts[ii].x + (i - insts[ii].vox0);
        float v = fmaf(__ldg(P.C + i), P.g[i], *x);
        if (nonneg) v = fmaxf(v, 0.0f);
        *x = v;
        P.g[i] = 0.0f;
      }
    }
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace tsp

using namespace tsp;

struct tsp_batch_s {
  std::vector<InstDesc> h;
  InstDesc* d = nullptr;
  int n = 0;
  int64_t total_items = 0, total_rays = 0, total_vox = 0;
  int block = 128;
  int max_words = 0;
  int grid_stage[4] = {152, 152, 152, 152};  // persistent grid per traversal stage (resident blocks x SMs)
  int grid_vox = 608;
  int device = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_iters = -1;
};

namespace {

size_t batch_ws_bytes(const tsp_batch_s* b, int n_stage_counters) {
  return 2 * align256(sizeof(float) * size_t(b->total_rays)) + 2 * align256(sizeof(float) * size_t(b->total_vox)) +
         align256(sizeof(unsigned long long) * size_t(n_stage_counters));
}

int counters_for(int n_iter) { return 3 + 3 * n_iter; }

// Enqueue the whole batched SIRT schedule on st (capturable).
tsp_status enqueue_batch(tsp_batch b, int n_iter, int flags, void* ws, cudaStream_t st) {
  char* p = static_cast<char*>(ws);
  BatchPtrs P;
  const size_t nr = align256(sizeof(float) * size_t(b->total_rays));
  const size_t nv = align256(sizeof(float) * size_t(b->total_vox));
  P.R = reinterpret_cast<float*>(p);
  P.r = reinterpret_cast<float*>(p + nr);
  P.C = reinterpret_cast<float*>(p + 2 * nr);
  P.g = reinterpret_cast<float*>(p + 2 * nr + nv);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p + 2 * nr + 2 * nv);
  const int n_ctr = counters_for(n_iter);
  const int ccap = cone_cap(b->block);
  const size_t smem = sizeof(float) * (size_t(b->max_words) + size_t(ccap) * size_t(b->block));
  const int grid_vox = b->grid_vox;
  const int nonneg = flags & TSP_SIRT_NONNEG;
  int c = 0;
  TSP_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * size_t(n_ctr), st));
  TSP_CUDA(cudaMemsetAsync(P.C, 0, sizeof(float) * size_t(b->total_vox), st));
  TSP_CUDA(cudaMemsetAsync(P.g, 0, sizeof(float) * size_t(b->total_vox), st));
  batch_trace_kernel<ST_PATHLEN><<<b->grid_stage[ST_PATHLEN], b->block, smem, st>>>(b->d, b->n, b->total_items,
                                                                                    ctr + c++, P, b->max_words, ccap);
  batch_trace_kernel<ST_UNIT><<<b->grid_stage[ST_UNIT], b->block, smem, st>>>(b->d, b->n, b->total_items, ctr + c++,
                                                                              P, b->max_words, ccap);
  batch_voxel_kernel<<<grid_vox, 256, 0, st>>>(b->d, b->n, b->total_vox, ctr + c++, 0, 0, P);
  for (int it = 0; it < n_iter; ++it) {
    batch_trace_kernel<ST_RESID><<<b->grid_stage[ST_RESID], b->block, smem, st>>>(b->d, b->n, b->total_items,
                                                                                  ctr + c++, P, b->max_words, ccap);
    batch_trace_kernel<ST_SCATTER><<<b->grid_stage[ST_SCATTER], b->block, smem, st>>>(b->d, b->n, b->total_items,
                                                                                      ctr + c++, P, b->max_words, ccap);
    batch_voxel_kernel<<<grid_vox, 256, 0, st>>>(b->d, b->n, b->total_vox, ctr + c++, 1, nonneg, P);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

void drop_graph(tsp_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_iters = -1;
}

}  // namespace

extern "C" tsp_status tsp_batch_create(const tsp_batch_item* items, int n_items, tsp_batch* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_batch_create: out is NULL");
  *out = nullptr;
  if (!items || n_items <= 0) return fail(TSP_EINVAL, "tsp_batch_create: no items");
  tsp_batch b = new (std::nothrow) tsp_batch_s();
  if (!b) return fail(TSP_ENOMEM, "tsp_batch_create: host allocation");
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaGetDevice");
  }
  int64_t most_rays = -1;
  tsp_launch lead = default_launch();
  for (int i = 0; i < n_items; ++i) {
    const tsp_batch_item& it = items[i];
    tsp_status st = check_trace_args(it.grid, it.geom, it.y, it.x, 1, nullptr, "tsp_batch_create");
    if (st != TSP_OK) {
      delete b;
      return st;
    }
    tsp_launch lf = preferred_launch(it.grid, it.geom, false), la = preferred_launch(it.grid, it.geom, true);
    if (it.geom->n_rays > most_rays) {
      most_rays = it.geom->n_rays;
      lead = lf;
    }
    InstDesc d;
    d.gd = it.grid->desc();
    d.ga = geom_args(it.geom);
    d.kind = it.geom->kind;
    d.tw = la.warp_tile_w;
    d.scatter = la.scatter;
    d.V = it.grid->voxels();
    d.y = it.y;
    d.x = it.x;
    b->max_words = std::max(b->max_words, it.grid->words);
    b->h.push_back(d);
  }
  b->block = lead.block_threads;
  for (InstDesc& d : b->h) {
    if (d.kind == GEOM_RAYS) {
      d.tiles_x = d.tiles_y = 0;
      d.n_items = (d.ga.n_rays + b->block - 1) / b->block;
    } else {
      const int bh = b->block / d.tw;
      d.tiles_x = (d.ga.W + d.tw - 1) / d.tw;
      d.tiles_y = (d.ga.H + bh - 1) / bh;
      d.n_items = int64_t(d.tiles_x) * d.tiles_y * (d.ga.n_rays / (int64_t(d.ga.H) * d.ga.W));
    }
    d.item0 = b->total_items;
    d.ray0 = b->total_rays;
    d.vox0 = b->total_vox;
    b->total_items += d.n_items;
    b->total_rays += d.ga.n_rays;
    b->total_vox += d.V;
  }
  b->n = n_items;
  e = cudaMalloc(&b->d, sizeof(InstDesc) * b->h.size());
  if (e == cudaSuccess) e = cudaMemcpy(b->d, b->h.data(), sizeof(InstDesc) * b->h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (b->d) cudaFree(b->d);
    delete b;
    return cuda_fail(e, "tsp_batch_create: upload");
  }
  const size_t smem = sizeof(float) * (size_t(b->max_words) + size_t(cone_cap(b->block)) * size_t(b->block));
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
  if (smem + 1024 > size_t(optin)) {
    cudaFree(b->d);
    delete b;
    return fail(TSP_ENOTSUP, "tsp_batch_create: grid tables and cone lists exceed a block's shared memory");
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  auto persistent_grid = [&](auto kernel) {
    allow_smem(kernel, smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, b->block, smem);
    return std::max(1, per_sm) * sms;
  };
  b->grid_stage[ST_PATHLEN] = persistent_grid(batch_trace_kernel<ST_PATHLEN>);
  b->grid_stage[ST_UNIT] = persistent_grid(batch_trace_kernel<ST_UNIT>);
  b->grid_stage[ST_RESID] = persistent_grid(batch_trace_kernel<ST_RESID>);
  b->grid_stage[ST_SCATTER] = persistent_grid(batch_trace_kernel<ST_SCATTER>);
  b->grid_vox = 4 * sms;
  *out = b;
  return TSP_OK;
}

extern "C" tsp_status tsp_batch_workspace_bytes(tsp_batch b, int n_iter, size_t* bytes) {
  if (!b || !bytes || n_iter < 0) return fail(TSP_EINVAL, "tsp_batch_workspace_bytes: bad argument");
  *bytes = batch_ws_bytes(b, counters_for(n_iter));
  return TSP_OK;
}

static tsp_status check_ws(tsp_batch b, int n_iter, int flags, void* ws, size_t bytes, const char* who) {
  if (!b) return fail(TSP_EINVAL, std::string(who) + ": NULL batch");
  if (n_iter < 0) return fail(TSP_EINVAL, std::string(who) + ": n_iter must be >= 0");
  if (flags & ~TSP_SIRT_NONNEG) return fail(TSP_EINVAL, std::string(who) + ": only TSP_SIRT_NONNEG is accepted");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(TSP_EINVAL, std::string(who) + ": workspace NULL or not 256-byte aligned");
  if (bytes < batch_ws_bytes(b, counters_for(n_iter)))
    return fail(TSP_EINVAL, std::string(who) + ": workspace smaller than tsp_batch_workspace_bytes()");
  return check_device(b->device);
}

extern "C" tsp_status tsp_batch_sirt(tsp_batch b, int n_iter, int flags, void* ws, size_t bytes, void* stream) {
  TSP_RANGE("tsp_batch_sirt");
  tsp_status st = check_ws(b, n_iter, flags, ws, bytes, "tsp_batch_sirt");
  if (st != TSP_OK) return st;
  return enqueue_batch(b, n_iter, flags, ws, static_cast<cudaStream_t>(stream));
}

extern "C" tsp_status tsp_batch_sirt_capture(tsp_batch b, int n_iter, int flags, void* ws, size_t bytes) {
  tsp_status st = check_ws(b, n_iter, flags, ws, bytes, "tsp_batch_sirt_capture");
  if (st != TSP_OK) return st;
  drop_graph(b);
  cudaStream_t cs = nullptr;
  TSP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "tsp_batch_sirt_capture: begin");
  }
  st = enqueue_batch(b, n_iter, flags, ws, cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st != TSP_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "tsp_batch_sirt_capture: end");
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    drop_graph(b);
    return cuda_fail(e, "tsp_batch_sirt_capture: instantiate");
  }
  b->graph_iters = n_iter;
  return TSP_OK;
}

extern "C" tsp_status tsp_batch_sirt_launch(tsp_batch b, void* stream) {
  if (!b) return fail(TSP_EINVAL, "tsp_batch_sirt_launch: NULL batch");
  if (!b->exec) return fail(TSP_EINVAL, "tsp_batch_sirt_launch: no captured schedule (call tsp_batch_sirt_capture)");
  tsp_status st = check_device(b->device);
  if (st != TSP_OK) return st;
  TSP_CUDA(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return TSP_OK;
}

extern "C" tsp_status tsp_batch_info(tsp_batch b, int64_t* total_rays, int64_t* total_voxels, int* block_threads) {
  if (!b) return fail(TSP_EINVAL, "tsp_batch_info: NULL batch");
  if (total_rays) *total_rays = b->total_rays;
  if (total_voxels) *total_voxels = b->total_vox;
  if (block_threads) *block_threads = b->block;
  return TSP_OK;
}

extern "C" void tsp_batch_destroy(tsp_batch b) {
  if (!b) return;
  drop_graph(b);
  if (b->d) cudaFree(b->d);
  delete b;
}
