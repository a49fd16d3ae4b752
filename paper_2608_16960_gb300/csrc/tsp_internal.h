// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tsp.h"
#include "tsp_trace.cuh"

struct tsp_grid_s {
  int Nr = 0, Ne = 0, Na = 0, M = 0;
  bool wrap = false;
  float pa0 = 0.0f;
  int words = 0;
  float* d_table = nullptr;  // the grid table of tsp_table.h (radii, cones, half-planes, sector maps)
  float* d_centres = nullptr;  // voxel centres: r [Nr] | sin t [Ne] | cos t [Ne] | cos p [Na] | sin p [Na]
  int device = 0;
  std::vector<double> r, th, ph;
  tsp::GridDesc desc() const {
    tsp::GridDesc d;
    d.table = d_table;
    d.Nr = Nr;
    d.Ne = Ne;
    d.Na = Na;
    d.M = M;
    d.words = words;
    d.pa0 = pa0;
    return d;
  }
  int64_t voxels() const { return int64_t(Nr) * Ne * Na; }
};

enum GeomKind { GEOM_CONE = 0, GEOM_PARALLEL = 1, GEOM_RAYS = 2 };

// Per-view parameters as float-float pairs split from host double arithmetic.
// cone:     origin = o; dir(u,v) = a + u*bu + v*bv, u = 2(j+.5)/W - 1, v = 1 - 2(i+.5)/H
// parallel: origin(u,v) = o + u*bu + v*bv, u = (j+.5)/W - .5, v = .5 - (i+.5)/H; dir = a
struct ViewParams {
  tsp::ff o[3], a[3], bu[3], bv[3];
};

struct tsp_geom_s {
  GeomKind kind = GEOM_CONE;
  int n_views = 0, H = 0, W = 0;
  int64_t n_rays = 0;
  ViewParams* d_views = nullptr;
  std::vector<ViewParams> h_views;
  const float* starts = nullptr;  // [3][n] device (free-form rays)
  const float* dirs = nullptr;
  float* owned = nullptr;
  int device = 0;
};

namespace tsp {

tsp_status fail(tsp_status st, const std::string& msg);
tsp_status cuda_fail(cudaError_t e, const char* what);
tsp_status check_device(int device);

// Autotuner cache lookup (tsp_autotune.cu).
bool tuned_launch(const tsp_grid_s* grid, const tsp_geom_s* geom, tsp_launch* fwd, tsp_launch* adj);

// SIRT enqueue shared by the single and batched entry points (tsp_sirt.cu).
// lf drives the gathering traversals, la the scattering ones (its scatter
// field picks the strategy).
tsp_status sirt_enqueue(tsp_grid grid, tsp_geom geom, const float* y, float* x, int n_iter, int flags, void* ws,
                        const tsp_launch& lf, const tsp_launch& la, cudaStream_t st);
size_t sirt_workspace_bytes(const tsp_grid_s* grid, const tsp_geom_s* geom);

// Readers of the per-translation-unit device error words (tsp_core.cu).
typedef cudaError_t (*error_reader)(int* out, cudaStream_t st);
void register_error_reader(error_reader r);
const std::vector<error_reader>& error_readers();

inline bool valid_launch(const tsp_launch& l) {
  const int b = l.block_threads, w = l.warp_tile_w;
  return (b == 64 || b == 128 || b == 256 || b == 512) && (w == 4 || w == 8 || w == 16 || w == 32) &&
         (l.scatter == 0 || l.scatter == 1);
}

inline tsp_launch default_launch() {
  tsp_launch l;
  l.block_threads = 128;
  l.warp_tile_w = 8;
  l.scatter = 0;
  return l;
}

// NVTX range over one library call: it names the call's kernels in a
// profiler's timeline and costs nothing measurable when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define TSP_RANGE(name) const tsp::NvtxRange tsp_nvtx_range_(name)

// cudaMalloc with the test hook of tsp_debug_fail_allocation (one injected
// out-of-memory failure after a countdown); used by the stored-list code.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

}  // namespace tsp

#define TSP_CUDA(call)                                     \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) return tsp::cuda_fail(e__, #call); \
  } while (0)
