// SIRT on the spherical-grid projector (the simultaneous iterative
// reconstruction technique the paper cites among the algorithms its operator
// serves, Sec. 1 ref. [10]):
//   R = 1 / (F 1),  C = 1 / (F^T 1)   (0 where the sum is 0)
//   x <- x + C * F^T( R * (y - F x) ),  optionally clamped at 0.
// Per iteration: one fused forward+residual traversal, one scatter traversal,
// one element-wise update that also clears the scatter target for the next
// iteration. All traversals share trace_kernel, so segments are bit-identical
// to tsp_forward / tsp_adjoint.
#include "tsp_kernels.cuh"

namespace tsp {
namespace {

// R[ray] = 1 / (in-grid path length), 0 for rays that miss the grid.
struct PathLenOp {
  float* __restrict__ R;
  float acc;
  __device__ __forceinline__ bool begin(int64_t) {
    acc = 0.0f;
    return true;
  }
  __device__ __forceinline__ void operator()(int, float dl) { acc = __fadd_rn(acc, dl); }
  __device__ __forceinline__ void end(int64_t ray) { R[ray] = acc > 0.0f ? __frcp_rn(acc) : 0.0f; }
};

// c[v] += dl for every segment of every ray (F^T 1).
struct UnitScatterOp {
  static constexpr bool wide_registers = true;
  float* __restrict__ c;
  __device__ __forceinline__ bool begin(int64_t) { return true; }
  __device__ __forceinline__ void operator()(int v, float dl) { atomicAdd(c + v, dl); }
  __device__ __forceinline__ void end(int64_t) {}
};

// r[ray] = R[ray] * (y[ray] - sum x[v] dl)
struct ResidualOp {
  const float* __restrict__ x;
  const float* __restrict__ y;
  const float* __restrict__ R;
  float* __restrict__ r;
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

__global__ void reciprocal_kernel(float* __restrict__ c, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float v = c[i];
    c[i] = v > 0.0f ? __frcp_rn(v) : 0.0f;
  }
}

// x += C * g (clamped at 0 if asked); g is cleared for the next scatter.
__global__ void update_kernel(float* __restrict__ x, float* __restrict__ g, const float* __restrict__ C, int64_t n,
                              int nonneg) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float v = fmaf(__ldg(C + i), g[i], x[i]);
    if (nonneg) v = fmaxf(v, 0.0f);
    x[i] = v;
    g[i] = 0.0f;
  }
}

int elementwise_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return int(std::min<int64_t>(b, 152 * 16));
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Workspace {
  float *R, *r, *C, *g;
};

size_t workspace_bytes(const tsp_grid_s* grid, const tsp_geom_s* geom) {
  return 2 * align256(sizeof(float) * size_t(geom->n_rays)) + 2 * align256(sizeof(float) * size_t(grid->voxels()));
}

Workspace carve(void* ws, const tsp_grid_s* grid, const tsp_geom_s* geom) {
  char* p = static_cast<char*>(ws);
  const size_t nr = align256(sizeof(float) * size_t(geom->n_rays));
  const size_t nv = align256(sizeof(float) * size_t(grid->voxels()));
  Workspace w;
  w.R = reinterpret_cast<float*>(p);
  w.r = reinterpret_cast<float*>(p + nr);
  w.C = reinterpret_cast<float*>(p + 2 * nr);
  w.g = reinterpret_cast<float*>(p + 2 * nr + nv);
  return w;
}

}  // namespace

// Enqueue SIRT on `st`. Shared by the public entry points; the workspace must
// hold workspace_bytes(grid, geom) bytes, 256-byte aligned.
tsp_status sirt_enqueue(tsp_grid grid, tsp_geom geom, const float* y, float* x, int n_iter, int flags, void* ws,
                        const tsp_launch& lf, const tsp_launch& la, cudaStream_t st) {
  const Workspace w = carve(ws, grid, geom);
  const int64_t V = grid->voxels();
  const int nonneg = flags & TSP_SIRT_NONNEG;
  if (!(flags & TSP_SIRT_REUSE_WEIGHTS)) {
    PathLenOp lop;
    lop.R = w.R;
    launch_trace(grid, geom, lf, lop, st);
    TSP_CUDA(cudaMemsetAsync(w.C, 0, sizeof(float) * size_t(V), st));
    UnitScatterOp uop;
    uop.c = w.C;
    launch_trace(grid, geom, la, uop, st);
    reciprocal_kernel<<<elementwise_blocks(V), 256, 0, st>>>(w.C, V);
  }
  TSP_CUDA(cudaMemsetAsync(w.g, 0, sizeof(float) * size_t(V), st));
  for (int it = 0; it < n_iter; ++it) {
    ResidualOp rop;
    rop.x = x;
    rop.y = y;
    rop.R = w.R;
    rop.r = w.r;
    launch_trace(grid, geom, lf, rop, st);
    if (la.scatter == 1) {
      AggScatterOp<1> sop;
      sop.y = w.r;
      sop.g = w.g;
      sop.V = V;
      sop.n_rays = geom->n_rays;
      sop.nb = 1;
      launch_trace(grid, geom, la, sop, st);
    } else {
      ScatterOp<1> sop;
      sop.y = w.r;
      sop.g = w.g;
      sop.V = V;
      sop.n_rays = geom->n_rays;
      sop.nb = 1;
      launch_trace(grid, geom, la, sop, st);
    }
    update_kernel<<<elementwise_blocks(V), 256, 0, st>>>(x, w.g, w.C, V, nonneg);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

size_t sirt_workspace_bytes(const tsp_grid_s* grid, const tsp_geom_s* geom) { return workspace_bytes(grid, geom); }

}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_sirt_weights(tsp_grid grid, tsp_geom geom, float* R, float* C, void* stream) {
  tsp_status st = check_trace_args(grid, geom, R, C, 1, nullptr, "tsp_sirt_weights");
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int64_t V = grid->voxels();
  PathLenOp lop;
  lop.R = R;
  launch_trace(grid, geom, preferred_launch(grid, geom, false), lop, cs);
  TSP_CUDA(cudaMemsetAsync(C, 0, sizeof(float) * size_t(V), cs));
  UnitScatterOp uop;
  uop.c = C;
  launch_trace(grid, geom, preferred_launch(grid, geom, true), uop, cs);
  reciprocal_kernel<<<elementwise_blocks(V), 256, 0, cs>>>(C, V);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_sirt_workspace_bytes(tsp_grid grid, tsp_geom geom, size_t* bytes) {
  if (!grid || !geom || !bytes) return fail(TSP_EINVAL, "tsp_sirt_workspace_bytes: NULL argument");
  *bytes = workspace_bytes(grid, geom);
  return TSP_OK;
}

extern "C" tsp_status tsp_sirt(tsp_grid grid, tsp_geom geom, const float* y, float* x, int n_iter, int flags,
                               void* workspace, size_t workspace_bytes_given, const tsp_launch* launch,
                               void* stream) {
  TSP_RANGE("tsp_sirt");
  tsp_status st = check_trace_args(grid, geom, y, x, 1, launch, "tsp_sirt");
  if (st != TSP_OK) return st;
  if (n_iter < 0) return fail(TSP_EINVAL, "tsp_sirt: n_iter must be >= 0");
  if (flags & ~(TSP_SIRT_NONNEG | TSP_SIRT_REUSE_WEIGHTS)) return fail(TSP_EINVAL, "tsp_sirt: unknown flag");
  if (!workspace) return fail(TSP_EINVAL, "tsp_sirt: NULL workspace");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(TSP_EINVAL, "tsp_sirt: workspace not 256-byte aligned");
  if (workspace_bytes_given < workspace_bytes(grid, geom))
    return fail(TSP_EINVAL, "tsp_sirt: workspace smaller than tsp_sirt_workspace_bytes()");
  const tsp_launch lf = launch ? *launch : preferred_launch(grid, geom, false);
  const tsp_launch la = launch ? *launch : preferred_launch(grid, geom, true);
  return sirt_enqueue(grid, geom, y, x, n_iter, flags, workspace, lf, la, static_cast<cudaStream_t>(stream));
}
