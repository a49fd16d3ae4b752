// SIRT with library-owned static scratch: an entry point that allocates no
// device memory. Some callers cannot call cudaMalloc: onboard or real-time
// reconstruction code that must run inside a fixed memory budget fixed at
// start-up, code that runs where a device allocation's implicit
// synchronisation would stall a latency-critical pipeline, and host
// frameworks that own the whole device memory pool through their own
// allocator. They call tsp_sirt_noalloc, which keeps its scratch (ray
// weights, residual, voxel weights, back-projection) in the file-scope array
// below, sized once at module load.
//
// Every call on a device shares that one array and leaves its contents behind;
// everything that must start at zero is cleared by each call, so a call never
// depends on an earlier one. Calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array and must not be issued.
#include <mutex>

#include "tsp_kernels.cuh"

namespace {

// 32 MiB of scratch: enough for n_rays + voxels up to 4,194,240 (rounded to
// 256-byte sections). Every GPU that loads the library holds it until exit.
static __device__ __align__(256) float g_noalloc_scratch[TSP_NOALLOC_SCRATCH_BYTES / sizeof(float)];

std::mutex g_scratch_mutex;
void* g_scratch_addr[128] = {nullptr};

// Device address of the scratch array for the current device. The host-side
// name of the array is only a stand-in for the symbol, so its address is taken
// once per device, with that device current, and cached.
tsp_status scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tsp::cuda_fail(e, "tsp_sirt_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 128) return tsp::fail(TSP_ENOTSUP, "tsp_sirt_noalloc: device ordinal above 127");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return tsp::cuda_fail(e, "tsp_sirt_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TSP_OK;
}

}  // namespace

extern "C" tsp_status tsp_sirt_noalloc(tsp_grid grid, tsp_geom geom, const float* y, float* x, int n_iter,
                                       int flags, void* stream) {
  TSP_RANGE("tsp_sirt_noalloc");
  tsp_status st = tsp::check_trace_args(grid, geom, y, x, 1, nullptr, "tsp_sirt_noalloc");
  if (st != TSP_OK) return st;
  if (n_iter < 0) return tsp::fail(TSP_EINVAL, "tsp_sirt_noalloc: n_iter must be >= 0");
  if (flags & ~TSP_SIRT_NONNEG)
    return tsp::fail(TSP_EINVAL, "tsp_sirt_noalloc: only TSP_SIRT_NONNEG is accepted (weights are always recomputed)");
  const size_t need = tsp::sirt_workspace_bytes(grid, geom);
  if (need > TSP_NOALLOC_SCRATCH_BYTES)
    return tsp::fail(TSP_ENOTSUP, "tsp_sirt_noalloc: this grid and geometry need " + std::to_string(need) +
                                      " bytes of scratch; the static scratch holds " +
                                      std::to_string(size_t(TSP_NOALLOC_SCRATCH_BYTES)) +
                                      " (use tsp_sirt with a caller workspace)");
  void* ws = nullptr;
  st = scratch_for_current_device(&ws);
  if (st != TSP_OK) return st;
  return tsp::sirt_enqueue(grid, geom, y, x, n_iter, flags, ws, tsp::default_launch(), tsp::default_launch(),
                           static_cast<cudaStream_t>(stream));
}
