// Forward projection F (Eq. 5) and its adjoint F^T (Sec. 4.4), fused with the
// per-ray traversal (tsp_trace.cuh) through the generic trace_kernel
// (tsp_kernels.cuh): one thread per ray, a warp per detector tile, grid tables
// in shared memory, density gathered through the read-only path (the volume
// stays resident in L2), adjoint scattered with L2 atomics.
//
// Built with -fmad=false and explicit fmaf/__f*_rn in the traversal, so the
// forward and adjoint kernels compute bit-identical segments.
#include "tsp_kernels.cuh"

namespace tsp {
namespace {

struct CountOp {
  int* __restrict__ counts;
  int n;
  __device__ __forceinline__ bool begin(int64_t) {
    n = 0;
    return true;
  }
  __device__ __forceinline__ void operator()(int, float) { ++n; }
  __device__ __forceinline__ void end(int64_t ray) { counts[ray] = n; }
};

// Dynamic object (Sec. 4.4: a 4D object seen by a collection of sequential
// views): view k of the geometry sees volume k. The ray's view is its index
// divided by the rays per view; all lanes of a warp share a view.
struct DynGatherOp {
  const float* __restrict__ rho;
  float* __restrict__ y;
  int64_t V, per_view;
  const float* base;
  DelayedSum sum;
  __device__ __forceinline__ bool begin(int64_t ray) {
    base = rho + (ray / per_view) * V;
    sum.reset();
    return true;
  }
  __device__ __forceinline__ void operator()(int v, float dl) { sum.add(base + v, dl); }
  __device__ __forceinline__ void end(int64_t ray) { y[ray] = sum.total(); }
};

// Adjoint of DynGatherOp: g[view][v] += y dl, one atomic add per segment, or
// (AGG) one per pair of neighbouring lanes (lane, lane ^ 1) that hit the same
// voxel in a step.
template <bool AGG>
struct DynScatterOp {
  static constexpr bool wide_registers = true;
  const float* __restrict__ y;
  float* __restrict__ g;
  int64_t V, per_view;
  float* base;
  float w;
  __device__ __forceinline__ bool begin(int64_t ray) {
    base = g + (ray / per_view) * V;
    w = __ldg(y + ray);
    return w != 0.0f;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    float c = __fmul_rn(w, dl);
    if (AGG) {
      // the neighbour's voxel index is per view: compare the addresses
      const unsigned m = __activemask();
      const int lane = threadIdx.x & 31;
      float* const a = base + v;
      const unsigned long long pa = __shfl_xor_sync(m, reinterpret_cast<unsigned long long>(a), 1);
      const float pc = __shfl_xor_sync(m, c, 1);
      if (((m >> (lane ^ 1)) & 1u) && pa == reinterpret_cast<unsigned long long>(a)) {
        if (lane & 1) return;
        c = __fadd_rn(c, pc);
      }
    }
    atomicAdd(base + v, c);
  }
  __device__ __forceinline__ void end(int64_t) {}
};

template <int NB>
void forward_chunk(tsp_grid grid, tsp_geom geom, const tsp_launch& l, const float* rho, float* y, int nb,
                   cudaStream_t st) {
  GatherOp<NB> op;
  op.rho = rho;
  op.y = y;
  op.V = grid->voxels();
  op.n_rays = geom->n_rays;
  op.nb = nb;
  launch_trace(grid, geom, l, op, st);
}

template <int NB, class OpT>
void adjoint_chunk(tsp_grid grid, tsp_geom geom, const tsp_launch& l, const float* y, float* g, int nb,
                   cudaStream_t st) {
  OpT op;
  op.y = y;
  op.g = g;
  op.V = grid->voxels();
  op.n_rays = geom->n_rays;
  op.nb = nb;
  launch_trace(grid, geom, l, op, st);
}

}  // namespace
}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_forward_ex(tsp_grid grid, tsp_geom geom, const float* rho, float* y, int batch,
                                     const tsp_launch* launch, void* stream) {
  TSP_RANGE("tsp_forward_ex");
  tsp_status st = check_trace_args(grid, geom, rho, y, batch, launch, "tsp_forward");
  if (st != TSP_OK) return st;
  const tsp_launch l = launch ? *launch : preferred_launch(grid, geom, false);
  const int64_t V = grid->voxels();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  for (int b0 = 0; b0 < batch; b0 += 8) {
    const int nb = std::min(8, batch - b0);
    const float* r = rho + b0 * V;
    float* yy = y + b0 * geom->n_rays;
    if (nb == 1) forward_chunk<1>(grid, geom, l, r, yy, nb, cs);
    else if (nb == 2) forward_chunk<2>(grid, geom, l, r, yy, nb, cs);
    else if (nb <= 4) forward_chunk<4>(grid, geom, l, r, yy, nb, cs);
    else forward_chunk<8>(grid, geom, l, r, yy, nb, cs);
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
  TSP_RANGE("tsp_adjoint_ex");
  tsp_status st = check_trace_args(grid, geom, y, rho, batch, launch, "tsp_adjoint");
  if (st != TSP_OK) return st;
  const tsp_launch l = launch ? *launch : preferred_launch(grid, geom, true);
  const int64_t V = grid->voxels();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (!accumulate) TSP_CUDA(cudaMemsetAsync(rho, 0, sizeof(float) * size_t(V) * batch, cs));
  for (int b0 = 0; b0 < batch; b0 += 8) {
    const int nb = std::min(8, batch - b0);
    const float* yy = y + b0 * geom->n_rays;
    float* g = rho + b0 * V;
    if (l.scatter == 1) {
      if (nb == 1) adjoint_chunk<1, AggScatterOp<1>>(grid, geom, l, yy, g, nb, cs);
      else if (nb == 2) adjoint_chunk<2, AggScatterOp<2>>(grid, geom, l, yy, g, nb, cs);
      else if (nb <= 4) adjoint_chunk<4, AggScatterOp<4>>(grid, geom, l, yy, g, nb, cs);
      else adjoint_chunk<8, AggScatterOp<8>>(grid, geom, l, yy, g, nb, cs);
    } else {
      if (nb == 1) adjoint_chunk<1, ScatterOp<1>>(grid, geom, l, yy, g, nb, cs);
      else if (nb == 2) adjoint_chunk<2, ScatterOp<2>>(grid, geom, l, yy, g, nb, cs);
      else if (nb <= 4) adjoint_chunk<4, ScatterOp<4>>(grid, geom, l, yy, g, nb, cs);
      else adjoint_chunk<8, ScatterOp<8>>(grid, geom, l, yy, g, nb, cs);
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
  tsp_status st = check_trace_args(grid, geom, counts, counts, 1, nullptr, "tsp_count_segments");
  if (st != TSP_OK) return st;
  CountOp op;
  op.counts = counts;
  launch_trace(grid, geom, default_launch(), op, static_cast<cudaStream_t>(stream));
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_forward_dynamic(tsp_grid grid, tsp_geom geom, const float* rho, float* y, void* stream) {
  TSP_RANGE("tsp_forward_dynamic");
  tsp_status st = check_trace_args(grid, geom, rho, y, 1, nullptr, "tsp_forward_dynamic");
  if (st != TSP_OK) return st;
  const tsp_launch l = preferred_launch(grid, geom, false);
  DynGatherOp op;
  op.rho = rho;
  op.y = y;
  op.V = grid->voxels();
  op.per_view = geom->n_rays / std::max(1, geom->n_views);
  launch_trace(grid, geom, l, op, static_cast<cudaStream_t>(stream));
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_adjoint_dynamic(tsp_grid grid, tsp_geom geom, const float* y, float* rho, int accumulate,
                                          void* stream) {
  TSP_RANGE("tsp_adjoint_dynamic");
  tsp_status st = check_trace_args(grid, geom, y, rho, 1, nullptr, "tsp_adjoint_dynamic");
  if (st != TSP_OK) return st;
  const tsp_launch l = preferred_launch(grid, geom, true);
  const int64_t V = grid->voxels();
  const int nv = std::max(1, geom->n_views);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (!accumulate) TSP_CUDA(cudaMemsetAsync(rho, 0, sizeof(float) * size_t(V) * nv, cs));
  if (l.scatter == 1) {
    DynScatterOp<true> op;
    op.y = y;
    op.g = rho;
    op.V = V;
    op.per_view = geom->n_rays / nv;
    launch_trace(grid, geom, l, op, cs);
  } else {
    DynScatterOp<false> op;
    op.y = y;
    op.g = rho;
    op.V = V;
    op.per_view = geom->n_rays / nv;
    launch_trace(grid, geom, l, op, cs);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}
