// Autotuner for the traversal launches: times candidate block sizes, warp
// tiles (detector pixels per warp row) and, for the adjoint, the scatter
// strategy (one atomic per segment vs warp-aggregated), on the caller's grid
// and geometry, and caches the fastest per size class. tsp_forward /
// tsp_adjoint / tsp_sirt use a cached choice when they are called without
// explicit launch knobs.
#include <map>
#include <mutex>
#include <tuple>

#include "tsp_kernels.cuh"

namespace tsp {
namespace {

// Size class: grid shape rounded to a power of two per dimension, geometry kind,
// detector shape rounded likewise, views rounded likewise.
typedef std::tuple<int, int, int, int, int, int, int> Key;

int bucket(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

Key key_of(const tsp_grid_s* g, const tsp_geom_s* geom) {
  return Key(bucket(g->Nr), bucket(g->Ne), bucket(g->Na), int(geom->kind), bucket(geom->n_views), bucket(geom->H),
             bucket(geom->kind == GEOM_RAYS ? geom->n_rays : geom->W));
}

std::mutex g_mu;
std::map<Key, std::pair<tsp_launch, tsp_launch>> g_cache;

__global__ void fill_kernel(float* p, int64_t n, float v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

}  // namespace

bool tuned_launch(const tsp_grid_s* grid, const tsp_geom_s* geom, tsp_launch* fwd, tsp_launch* adj) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(key_of(grid, geom));
  if (it == g_cache.end()) return false;
  if (fwd) *fwd = it->second.first;
  if (adj) *adj = it->second.second;
  return true;
}

}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_autotune(tsp_grid grid, tsp_geom geom, tsp_launch* fwd_out, tsp_launch* adj_out,
                                   void* stream) {
  TSP_RANGE("tsp_autotune");
  tsp_status st = check_trace_args(grid, geom, grid, geom, 1, nullptr, "tsp_autotune");
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int64_t V = grid->voxels(), R = geom->n_rays;
  float *rho = nullptr, *y = nullptr, *g = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (rho) cudaFree(rho);
    if (y) cudaFree(y);
    if (g) cudaFree(g);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t e = cudaMalloc(&rho, sizeof(float) * size_t(V));
  if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(float) * size_t(R));
  if (e == cudaSuccess) e = cudaMalloc(&g, sizeof(float) * size_t(V));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "tsp_autotune: scratch");
  }
  fill_kernel<<<512, 256, 0, cs>>>(rho, V, 1.0f);
  fill_kernel<<<512, 256, 0, cs>>>(y, R, 1.0f);

  const int blocks[] = {64, 128, 256, 512};
  const int tiles_det[] = {4, 8, 16, 32};
  const int tiles_rays[] = {8};
  const int* tiles = geom->kind == GEOM_RAYS ? tiles_rays : tiles_det;
  const int n_tiles = geom->kind == GEOM_RAYS ? 1 : 4;

  float* yf = nullptr;  // forward output, kept apart so the adjoint input stays 1
  e = cudaMalloc(&yf, sizeof(float) * size_t(R));
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "tsp_autotune: scratch");
  }
  // Average time of two launches after one warm-up launch.
  auto time_it = [&](bool adjoint, const tsp_launch& l, float* ms) -> tsp_status {
    tsp_status s2 = TSP_OK;
    for (int rep = 0; rep < 3 && s2 == TSP_OK; ++rep) {
      if (rep == 1) cudaEventRecord(e0, cs);
      s2 = adjoint ? tsp_adjoint_ex(grid, geom, y, g, 1, 0, &l, cs) : tsp_forward_ex(grid, geom, rho, yf, 1, &l, cs);
    }
    if (s2 != TSP_OK) return s2;
    cudaEventRecord(e1, cs);
    const cudaError_t e2 = cudaEventSynchronize(e1);
    if (e2 != cudaSuccess) return cuda_fail(e2, "tsp_autotune: timing");
    cudaEventElapsedTime(ms, e0, e1);
    return TSP_OK;
  };

  tsp_launch best_f = default_launch(), best_a = default_launch();
  float tf = 1e30f, ta = 1e30f;
  tsp_status s2 = TSP_OK;
  for (int b : blocks) {
    for (int i = 0; i < n_tiles && s2 == TSP_OK; ++i) {
      tsp_launch l;
      l.block_threads = b;
      l.warp_tile_w = tiles[i];
      l.scatter = 0;
      if (check_trace_args(grid, geom, rho, yf, 1, &l, "tsp_autotune") != TSP_OK) continue;
      float ms = 0;
      s2 = time_it(false, l, &ms);
      if (s2 == TSP_OK && ms < tf) {
        tf = ms;
        best_f = l;
      }
      for (int sc = 0; sc < 2 && s2 == TSP_OK; ++sc) {
        l.scatter = sc;
        s2 = time_it(true, l, &ms);
        if (s2 == TSP_OK && ms < ta) {
          ta = ms;
          best_a = l;
        }
      }
    }
  }
  if (s2 != TSP_OK) {
    cudaFree(yf);
    cleanup();
    return s2;
  }
  cudaFree(yf);
  cleanup();
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key_of(grid, geom)] = std::make_pair(best_f, best_a);
  }
  if (fwd_out) *fwd_out = best_f;
  if (adj_out) *adj_out = best_a;
  return TSP_OK;
}

extern "C" tsp_status tsp_autotune_lookup(tsp_grid grid, tsp_geom geom, tsp_launch* fwd, tsp_launch* adj) {
  if (!grid || !geom) return fail(TSP_EINVAL, "tsp_autotune_lookup: NULL handle");
  if (!tuned_launch(grid, geom, fwd, adj)) return fail(TSP_ENOTSUP, "tsp_autotune_lookup: size class not tuned");
  return TSP_OK;
}

extern "C" tsp_status tsp_autotune_store(tsp_grid grid, tsp_geom geom, const tsp_launch* fwd, const tsp_launch* adj) {
  if (!grid || !geom) return fail(TSP_EINVAL, "tsp_autotune_store: NULL handle");
  if (!fwd || !adj) return fail(TSP_EINVAL, "tsp_autotune_store: NULL knobs");
  if (!valid_launch(*fwd) || !valid_launch(*adj)) return fail(TSP_EINVAL, "tsp_autotune_store: invalid launch knobs");
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache[key_of(grid, geom)] = std::make_pair(*fwd, *adj);
  return TSP_OK;
}

extern "C" void tsp_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
}
