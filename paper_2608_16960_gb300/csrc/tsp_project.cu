// Forward projection F (Eq. 5) and its adjoint F^T (Sec. 4.4), fused with the
// per-ray traversal (tsp_trace.cuh): one thread per ray, a warp per detector
// tile, grid tables in shared memory, density gathered through the read-only
// path (the volume stays resident in L2), adjoint scattered with L2 atomics.
//
// Built with -fmad=false and explicit fmaf/__f*_rn in the traversal, so the
// forward and adjoint kernels compute bit-identical segments.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "tsp_internal.h"

namespace cg = cooperative_groups;

__device__ int g_tsp_error_word;

namespace tsp {

int* device_error_word() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tsp_error_word) != cudaSuccess) return nullptr;
  return static_cast<int*>(p);
}

struct GeomArgs {
  const ViewParams* views;
  const float* starts;
  const float* dirs;
  int H, W;
  int64_t n_rays;
};

// Map this thread to a ray: detector geometries tile a warp over tw x (32/tw)
// pixels and stack the block's warps vertically; free-form rays are linear.
template <int GK>
__device__ __forceinline__ bool ray_of_thread(const GeomArgs& ga, int tw, int64_t& ray, float x[3], float d[3]) {
  if (GK == GEOM_RAYS) {
    ray = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (ray >= ga.n_rays) return false;
    const int64_t n = ga.n_rays;
    x[0] = __ldg(ga.starts + ray);
    x[1] = __ldg(ga.starts + n + ray);
    x[2] = __ldg(ga.starts + 2 * n + ray);
    d[0] = __ldg(ga.dirs + ray);
    d[1] = __ldg(ga.dirs + n + ray);
    d[2] = __ldg(ga.dirs + 2 * n + ray);
    return true;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int th = 32 / tw, bh = blockDim.x / tw;
  const int col = blockIdx.x * tw + (lane % tw);
  const int row = blockIdx.y * bh + warp * th + lane / tw;
  if (col >= ga.W || row >= ga.H) return false;
  const int view = blockIdx.z;
  ray = (int64_t(view) * ga.H + row) * ga.W + col;
  const ViewParams& p = ga.views[view];
  if (GK == GEOM_CONE) {
    const float u = __fdiv_rn(float(2 * col + 1 - ga.W), float(ga.W));
    const float v = __fdiv_rn(float(ga.H - 2 * row - 1), float(ga.H));
    for (int i = 0; i < 3; ++i) {
      x[i] = p.o[i];
      d[i] = fmaf(v, p.bv[i], fmaf(u, p.bu[i], p.a[i]));
    }
  } else {
    const float u = __fdiv_rn(float(2 * col + 1 - ga.W), float(2 * ga.W));
    const float v = __fdiv_rn(float(ga.H - 2 * row - 1), float(2 * ga.H));
    for (int i = 0; i < 3; ++i) {
      x[i] = fmaf(v, p.bv[i], fmaf(u, p.bu[i], p.o[i]));
      d[i] = p.a[i];
    }
  }
  return true;
}

template <int NB>
struct FwdOp {
  const float* __restrict__ rho;
  int64_t V;
  int nb;
  float acc[NB];
  __device__ __forceinline__ void operator()(int v, float dl) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < nb) acc[b] = fmaf(__ldg(rho + b * V + v), dl, acc[b]);
  }
};

template <int NB, int AGG>
struct AdjOp {
  float* __restrict__ g;
  int64_t V;
  int nb;
  float yv[NB];
  __device__ __forceinline__ void operator()(int v, float dl) {
    if (AGG) {
      cg::coalesced_group act = cg::coalesced_threads();
      cg::coalesced_group grp = cg::labeled_partition(act, v);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (b < nb) {
          const float s = cg::reduce(grp, __fmul_rn(yv[b], dl), cg::plus<float>());
          if (grp.thread_rank() == 0) atomicAdd(g + b * V + v, s);
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < nb && yv[b] != 0.0f) atomicAdd(g + b * V + v, __fmul_rn(yv[b], dl));
    }
  }
};

template <int GK, int NB>
__global__ void __launch_bounds__(512) forward_kernel(GridDesc gd, GeomArgs ga, const float* __restrict__ rho,
                                                      float* __restrict__ y, int nb, int tw) {
  extern __shared__ float smem[];
  load_table(gd, smem);
  const TGrid G = tgrid_from_smem(gd, smem);
  int64_t ray;
  float x[3], d[3];
  if (!ray_of_thread<GK>(ga, tw, ray, x, d)) return;
  FwdOp<NB> op;
  op.rho = rho;
  op.V = int64_t(gd.Nr) * gd.Ne * gd.Na;
  op.nb = nb;
#pragma unroll
  for (int b = 0; b < NB; ++b) op.acc[b] = 0.0f;
  if (!trace_ray(G, x[0], x[1], x[2], d[0], d[1], d[2], op)) atomicOr(&g_tsp_error_word, 1);
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b < nb) y[b * ga.n_rays + ray] = op.acc[b];
}

template <int GK, int NB, int AGG>
__global__ void __launch_bounds__(512) adjoint_kernel(GridDesc gd, GeomArgs ga, const float* __restrict__ y,
                                                      float* __restrict__ g, int nb, int tw) {
  extern __shared__ float smem[];
  load_table(gd, smem);
  const TGrid G = tgrid_from_smem(gd, smem);
  int64_t ray;
  float x[3], d[3];
  if (!ray_of_thread<GK>(ga, tw, ray, x, d)) return;
  AdjOp<NB, AGG> op;
  op.g = g;
  op.V = int64_t(gd.Nr) * gd.Ne * gd.Na;
  op.nb = nb;
  bool any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    op.yv[b] = b < nb ? __ldg(y + b * ga.n_rays + ray) : 0.0f;
    any |= op.yv[b] != 0.0f;
  }
  if (!any && !AGG) return;
  if (!trace_ray(G, x[0], x[1], x[2], d[0], d[1], d[2], op)) atomicOr(&g_tsp_error_word, 1);
}

struct CountOp {
  int n;
  __device__ __forceinline__ void operator()(int, float) { ++n; }
};

// Number of valid segments of each ray (the pieces with an in-range voxel index).
template <int GK>
__global__ void __launch_bounds__(512) count_kernel(GridDesc gd, GeomArgs ga, int* __restrict__ counts, int tw) {
  extern __shared__ float smem[];
  load_table(gd, smem);
  const TGrid G = tgrid_from_smem(gd, smem);
  int64_t ray;
  float x[3], d[3];
  if (!ray_of_thread<GK>(ga, tw, ray, x, d)) return;
  CountOp op{0};
  if (!trace_ray(G, x[0], x[1], x[2], d[0], d[1], d[2], op)) atomicOr(&g_tsp_error_word, 1);
  counts[ray] = op.n;
}

struct LaunchShape {
  dim3 grid, block;
  size_t smem;
};

LaunchShape shape_for(const tsp_grid_s* grid, const tsp_geom_s* geom, const tsp_launch& l) {
  LaunchShape s;
  s.block = dim3(l.block_threads);
  s.smem = sizeof(float) * size_t(grid->words);
  if (geom->kind == GEOM_RAYS) {
    s.grid = dim3(unsigned((geom->n_rays + l.block_threads - 1) / l.block_threads));
  } else {
    const int bh = l.block_threads / l.warp_tile_w;
    s.grid = dim3((geom->W + l.warp_tile_w - 1) / l.warp_tile_w, (geom->H + bh - 1) / bh, geom->n_views);
  }
  return s;
}

GeomArgs geom_args(const tsp_geom_s* g) {
  GeomArgs a;
  a.views = g->d_views;
  a.starts = g->starts;
  a.dirs = g->dirs;
  a.H = g->H;
  a.W = g->W;
  a.n_rays = g->n_rays;
  return a;
}

template <int GK, int NB>
void launch_forward(const LaunchShape& s, const GridDesc& gd, const GeomArgs& ga, const float* rho, float* y,
                    int nb, int tw, cudaStream_t st) {
  forward_kernel<GK, NB><<<s.grid, s.block, s.smem, st>>>(gd, ga, rho, y, nb, tw);
}

template <int GK, int NB, int AGG>
void launch_adjoint(const LaunchShape& s, const GridDesc& gd, const GeomArgs& ga, const float* y, float* g,
                    int nb, int tw, cudaStream_t st) {
  adjoint_kernel<GK, NB, AGG><<<s.grid, s.block, s.smem, st>>>(gd, ga, y, g, nb, tw);
}

template <int GK>
void dispatch_forward(const LaunchShape& s, const GridDesc& gd, const GeomArgs& ga, const float* rho, float* y,
                      int nb, int tw, cudaStream_t st) {
  if (nb == 1) launch_forward<GK, 1>(s, gd, ga, rho, y, nb, tw, st);
  else if (nb == 2) launch_forward<GK, 2>(s, gd, ga, rho, y, nb, tw, st);
  else if (nb <= 4) launch_forward<GK, 4>(s, gd, ga, rho, y, nb, tw, st);
  else launch_forward<GK, 8>(s, gd, ga, rho, y, nb, tw, st);
}

template <int GK, int AGG>
void dispatch_adjoint(const LaunchShape& s, const GridDesc& gd, const GeomArgs& ga, const float* y, float* g,
                      int nb, int tw, cudaStream_t st) {
  if (nb == 1) launch_adjoint<GK, 1, AGG>(s, gd, ga, y, g, nb, tw, st);
  else if (nb == 2) launch_adjoint<GK, 2, AGG>(s, gd, ga, y, g, nb, tw, st);
  else if (nb <= 4) launch_adjoint<GK, 4, AGG>(s, gd, ga, y, g, nb, tw, st);
  else launch_adjoint<GK, 8, AGG>(s, gd, ga, y, g, nb, tw, st);
}

tsp_status check_args(tsp_grid grid, tsp_geom geom, const void* a, const void* b, int batch, const tsp_launch* l,
                      const char* who) {
  if (!grid || !geom) return fail(TSP_EINVAL, std::string(who) + ": NULL handle");
  if (!a || !b) return fail(TSP_EINVAL, std::string(who) + ": NULL array");
  if (batch <= 0) return fail(TSP_EINVAL, std::string(who) + ": batch must be >= 1");
  if (l && !valid_launch(*l)) return fail(TSP_EINVAL, std::string(who) + ": invalid launch knobs");
  tsp_status st = check_device(grid->device);
  if (st != TSP_OK) return st;
  st = check_device(geom->device);
  if (st != TSP_OK) return st;
  const tsp_launch lc = l ? *l : default_launch();
  const LaunchShape s = shape_for(grid, geom, lc);
  if (s.grid.y > 65535u || s.grid.z > 65535u || s.grid.x > 2147483647u)
    return fail(TSP_ENOTSUP, std::string(who) + ": detector too large for one launch");
  return TSP_OK;
}

}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_forward_ex(tsp_grid grid, tsp_geom geom, const float* rho, float* y, int batch,
                                     const tsp_launch* launch, void* stream) {
  tsp_status st = check_args(grid, geom, rho, y, batch, launch, "tsp_forward");
  if (st != TSP_OK) return st;
  const tsp_launch l = launch ? *launch : default_launch();
  const LaunchShape s = shape_for(grid, geom, l);
  const GridDesc gd = grid->desc();
  const GeomArgs ga = geom_args(geom);
  const int64_t V = grid->voxels();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  for (int b0 = 0; b0 < batch; b0 += 8) {
    const int nb = std::min(8, batch - b0);
    const float* r = rho + b0 * V;
    float* yy = y + b0 * geom->n_rays;
    if (geom->kind == GEOM_CONE) dispatch_forward<GEOM_CONE>(s, gd, ga, r, yy, nb, l.warp_tile_w, cs);
    else if (geom->kind == GEOM_PARALLEL) dispatch_forward<GEOM_PARALLEL>(s, gd, ga, r, yy, nb, l.warp_tile_w, cs);
    else dispatch_forward<GEOM_RAYS>(s, gd, ga, r, yy, nb, l.warp_tile_w, cs);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_forward(tsp_grid grid, tsp_geom geom, const float* rho, float* y, int batch,
                                  void* stream) {
  return tsp_forward_ex(grid, geom, rho, y, batch, nullptr, stream);
}

extern "C" tsp_status tsp_adjoint_ex(tsp_grid grid, tsp_geom geom, const float* y, float* rho, int batch,
                                     int accumulate, const tsp_launch* launch, void* stream) {
  tsp_status st = check_args(grid, geom, y, rho, batch, launch, "tsp_adjoint");
  if (st != TSP_OK) return st;
  const tsp_launch l = launch ? *launch : default_launch();
  const LaunchShape s = shape_for(grid, geom, l);
  const GridDesc gd = grid->desc();
  const GeomArgs ga = geom_args(geom);
  const int64_t V = grid->voxels();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (!accumulate) TSP_CUDA(cudaMemsetAsync(rho, 0, sizeof(float) * size_t(V) * batch, cs));
  for (int b0 = 0; b0 < batch; b0 += 8) {
    const int nb = std::min(8, batch - b0);
    const float* yy = y + b0 * geom->n_rays;
    float* g = rho + b0 * V;
    const int tw = l.warp_tile_w;
    if (l.scatter == 1) {
      if (geom->kind == GEOM_CONE) dispatch_adjoint<GEOM_CONE, 1>(s, gd, ga, yy, g, nb, tw, cs);
      else if (geom->kind == GEOM_PARALLEL) dispatch_adjoint<GEOM_PARALLEL, 1>(s, gd, ga, yy, g, nb, tw, cs);
      else dispatch_adjoint<GEOM_RAYS, 1>(s, gd, ga, yy, g, nb, tw, cs);
    } else {
      if (geom->kind == GEOM_CONE) dispatch_adjoint<GEOM_CONE, 0>(s, gd, ga, yy, g, nb, tw, cs);
      else if (geom->kind == GEOM_PARALLEL) dispatch_adjoint<GEOM_PARALLEL, 0>(s, gd, ga, yy, g, nb, tw, cs);
      else dispatch_adjoint<GEOM_RAYS, 0>(s, gd, ga, yy, g, nb, tw, cs);
    }
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_adjoint(tsp_grid grid, tsp_geom geom, const float* y, float* rho, int batch,
                                  int accumulate, void* stream) {
  return tsp_adjoint_ex(grid, geom, y, rho, batch, accumulate, nullptr, stream);
}

extern "C" tsp_status tsp_count_segments(tsp_grid grid, tsp_geom geom, int* counts, void* stream) {
  tsp_status st = check_args(grid, geom, counts, counts, 1, nullptr, "tsp_count_segments");
  if (st != TSP_OK) return st;
  const tsp_launch l = default_launch();
  const LaunchShape s = shape_for(grid, geom, l);
  const GridDesc gd = grid->desc();
  const GeomArgs ga = geom_args(geom);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (geom->kind == GEOM_CONE) count_kernel<GEOM_CONE><<<s.grid, s.block, s.smem, cs>>>(gd, ga, counts, l.warp_tile_w);
  else if (geom->kind == GEOM_PARALLEL)
    count_kernel<GEOM_PARALLEL><<<s.grid, s.block, s.smem, cs>>>(gd, ga, counts, l.warp_tile_w);
  else count_kernel<GEOM_RAYS><<<s.grid, s.block, s.smem, cs>>>(gd, ga, counts, l.warp_tile_w);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_device_status(void* stream, int* code) {
  if (!code) return fail(TSP_EINVAL, "tsp_device_status: NULL code");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  int v = 0;
  TSP_CUDA(cudaMemcpyFromSymbolAsync(&v, g_tsp_error_word, sizeof(int), 0, cudaMemcpyDeviceToHost, cs));
  TSP_CUDA(cudaStreamSynchronize(cs));
  const int zero = 0;
  TSP_CUDA(cudaMemcpyToSymbolAsync(g_tsp_error_word, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, cs));
  TSP_CUDA(cudaStreamSynchronize(cs));
  *code = v;
  if (v != 0) return fail(TSP_EDEVICE, "a kernel set the device error word: " + std::to_string(v));
  return TSP_OK;
}
