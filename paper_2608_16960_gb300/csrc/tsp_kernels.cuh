// Generic per-ray traversal kernel: one thread per ray, the grid table staged
// in shared memory, a per-segment operation supplied as a functor.
//
//   struct Op {
//     __device__ bool begin(int64_t ray);          // false: skip this ray
//     __device__ void operator()(int voxel, float dl);
//     __device__ void end(int64_t ray);
//   };
//
// Every kernel of the library that walks rays instantiates this template, so
// all of them see bit-identical segments (same code, -fmad=false).
#pragma once


#include "tsp_internal.h"

// Device error word of this translation unit (device variables are not shared
// across translation units without relocatable device code). A kernel that
// detects an internal inconsistency ORs a bit into it instead of trapping; the
// host reads and clears every unit's word through the registered readers.
static __device__ int g_tsp_error_word;

namespace tsp {

static cudaError_t take_unit_error(int* out, cudaStream_t st) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_tsp_error_word, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const int zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_tsp_error_word, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *out |= v;
  return e;
}

namespace {
struct UnitErrorRegistrar {
  UnitErrorRegistrar() { register_error_reader(&take_unit_error); }
};
UnitErrorRegistrar unit_error_registrar;
}  // namespace

struct GeomArgs {
  const ViewParams* views;
  const float* starts;
  const float* dirs;
  int H, W;
  int64_t n_rays;
};

inline GeomArgs geom_args(const tsp_geom_s* g) {
  GeomArgs a;
  a.views = g->d_views;
  a.starts = g->starts;
  a.dirs = g->dirs;
  a.H = g->H;
  a.W = g->W;
  a.n_rays = g->n_rays;
  return a;
}

// num / den for small integers, as float-float (the remainder is exact).
__device__ __forceinline__ ff ratio_ff(int num, int den) {
  const float n = float(num), d = float(den);
  const float hi = __fdiv_rn(n, d);
  return ff{hi, __fdiv_rn(fmaf(-hi, d, n), d)};
}

// Ray of a detector pixel (cone or parallel view) or of a free-form ray, as
// float-float start x and direction d.
template <int GK>
__device__ __forceinline__ void ray_geometry(const GeomArgs& ga, int view, int row, int col, int64_t ray, ff x[3],
                                             ff d[3]) {
  if (GK == GEOM_RAYS) {
    const int64_t n = ga.n_rays;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[i] = ff{__ldg(ga.starts + i * n + ray), 0.0f};
      d[i] = ff{__ldg(ga.dirs + i * n + ray), 0.0f};
    }
    return;
  }
  const ViewParams& p = ga.views[view];
  const bool cone = GK == GEOM_CONE;
  const ff u = ratio_ff(2 * col + 1 - ga.W, cone ? ga.W : 2 * ga.W);
  const ff v = ratio_ff(ga.H - 2 * row - 1, cone ? ga.H : 2 * ga.H);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const ff off = ff_add(ff_mul(u, p.bu[i]), ff_mul(v, p.bv[i]));
    if (cone) {
      x[i] = p.o[i];
      d[i] = ff_add(p.a[i], off);
    } else {
      x[i] = ff_add(p.o[i], off);
      d[i] = p.a[i];
    }
  }
}

// Map this thread to a ray: detector geometries tile a warp over tw x (32/tw)
// pixels and stack the block's warps vertically; free-form rays are linear.
template <int GK>
__device__ __forceinline__ bool ray_of_thread(const GeomArgs& ga, int tw, int64_t& ray, ff x[3], ff d[3]) {
  if (GK == GEOM_RAYS) {
    ray = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (ray >= ga.n_rays) return false;
    ray_geometry<GK>(ga, 0, 0, 0, ray, x, d);
    return true;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int th = 32 / tw, bh = blockDim.x / tw;
  const int col = blockIdx.x * tw + (lane % tw);
  const int row = blockIdx.y * bh + warp * th + lane / tw;
  if (col >= ga.W || row >= ga.H) return false;
  const int view = blockIdx.z;
  ray = (int64_t(view) * ga.H + row) * ga.W + col;
  ray_geometry<GK>(ga, view, row, col, ray, x, d);
  return true;
}

// Shared memory: the grid table, then each thread's cone-crossing list of
// ccap entries (thread i's entry j at word words + j * blockDim + i).
template <int GK, class Op>
__device__ __forceinline__ void trace_body(const GridDesc& gd, const GeomArgs& ga, Op& op, int tw, int ccap) {
  extern __shared__ float smem[];
  load_table(gd, smem);
  const TGrid G = tgrid_from_smem(gd, smem);
  int64_t ray;
  ff x[3], d[3];
  if (!ray_of_thread<GK>(ga, tw, ray, x, d)) return;
  if (!op.begin(ray)) return;
  const ConeList L{smem + gd.words + threadIdx.x, int(blockDim.x), ccap};
  if (!trace_ray(G, x, d, op, L)) atomicOr(&g_tsp_error_word, 1);
  op.end(ray);
}

// At most 72 registers a thread: 7 blocks of 128 threads per SM. Left to
// the compiler most per-segment operations take 75-90 and lose one to three
// blocks (measured: the single-volume gather 3.9% faster capped, the batch
// stages 9%), without spilling under the cap.
template <int GK, class Op>
__global__ void __maxnreg__(72) trace_kernel(GridDesc gd, GeomArgs ga, Op op, int tw, int ccap) {
  trace_body<GK>(gd, ga, op, tw, ccap);
}

// Ops that declare `static constexpr bool wide_registers = true` keep the
// compiler's allocation: the scatters, which fit in 72 registers anyway and
// ran 2% slower under the cap's allocation, the 8-volume gather, which would
// spill, and the attenuated projection's operations (8% slower capped; the
// dynamic gather, by contrast, 15% faster).
template <int GK, class Op>
__global__ void __launch_bounds__(512, 1) trace_kernel_wide(GridDesc gd, GeomArgs ga, Op op, int tw, int ccap) {
  trace_body<GK>(gd, ga, op, tw, ccap);
}

template <class Op, class = void>
struct op_wide_registers {
  static constexpr bool value = false;
};
template <class Op>
struct op_wide_registers<Op, decltype(void(Op::wide_registers))> {
  static constexpr bool value = Op::wide_registers;
};

// Cone-crossing list entries per thread: 48 up to 128 threads per block
// (24 KB per block; one ray in two hundred at the paper-scale workload has
// more and refills its list), proportionally fewer for larger blocks, so the
// lists take 24 KB a block at most (measured: 32 entries ran 2% slower, 64
// entries 3% slower, the lists then limiting blocks per SM).
inline int cone_cap(int block_threads) { return block_threads <= 128 ? 48 : (48 * 128) / block_threads; }

struct LaunchShape {
  dim3 grid, block;
  size_t smem;
  int ccap;
};

inline LaunchShape shape_for(const tsp_grid_s* grid, const tsp_geom_s* geom, const tsp_launch& l) {
  LaunchShape s;
  s.block = dim3(l.block_threads);
  s.ccap = cone_cap(l.block_threads);
  s.smem = sizeof(float) * (size_t(grid->words) + size_t(s.ccap) * size_t(l.block_threads));
  if (geom->kind == GEOM_RAYS) {
    s.grid = dim3(unsigned((geom->n_rays + l.block_threads - 1) / l.block_threads));
  } else {
    const int bh = l.block_threads / l.warp_tile_w;
    s.grid = dim3((geom->W + l.warp_tile_w - 1) / l.warp_tile_w, (geom->H + bh - 1) / bh, geom->n_views);
  }
  return s;
}

// Dynamic shared memory above the default 48 KB (tables of the largest grids)
// needs the kernel's opt-in, set on the current device before the launch.
template <class K>
inline void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

// Launch trace_kernel for the geometry kind of `geom`.
template <class Op>
void launch_trace(const tsp_grid_s* grid, const tsp_geom_s* geom, const tsp_launch& l, const Op& op,
                  cudaStream_t st) {
  const LaunchShape s = shape_for(grid, geom, l);
  const GridDesc gd = grid->desc();
  const GeomArgs ga = geom_args(geom);
  auto go = [&](auto kernel) {
    allow_smem(kernel, s.smem);
    kernel<<<s.grid, s.block, s.smem, st>>>(gd, ga, op, l.warp_tile_w, s.ccap);
  };
  if constexpr (op_wide_registers<Op>::value) {
    if (geom->kind == GEOM_CONE) go(trace_kernel_wide<GEOM_CONE, Op>);
    else if (geom->kind == GEOM_PARALLEL) go(trace_kernel_wide<GEOM_PARALLEL, Op>);
    else go(trace_kernel_wide<GEOM_RAYS, Op>);
  } else {
    if (geom->kind == GEOM_CONE) go(trace_kernel<GEOM_CONE, Op>);
    else if (geom->kind == GEOM_PARALLEL) go(trace_kernel<GEOM_PARALLEL, Op>);
    else go(trace_kernel<GEOM_RAYS, Op>);
  }
}

// Validation shared by the entry points that launch traversals.
inline tsp_status check_trace_args(tsp_grid grid, tsp_geom geom, const void* a, const void* b, int batch,
                                   const tsp_launch* l, const char* who) {
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

// ---- per-segment operations shared across translation units ----

// A line integral accumulated one segment behind the walk: the value loaded
// for a segment is added when the next segment (or the end of the ray) comes,
// so the load's latency overlaps the walk's next step instead of stalling the
// multiply-add. The terms are added in the same order, fma(value, length,
// sum) per segment, so the result is the same bit for bit. The previous
// term's multiply-add is issued before the new load (measured: the other
// order, the load first, ran the forward 17% slower).
struct DelayedSum {
  float acc, pv, pdl;
  __device__ __forceinline__ void reset() { acc = pv = pdl = 0.0f; }
  __device__ __forceinline__ void add(const float* p, float dl) {
    acc = fmaf(pv, pdl, acc);
    pv = __ldg(p);
    pdl = dl;
  }
  __device__ __forceinline__ float total() const { return fmaf(pv, pdl, acc); }
};

// y[b] = sum rho[b][v] dl  (Eq. 5), optionally followed by an epilogue.
template <int NB>
struct GatherOp {
  static constexpr bool wide_registers = NB == 8;
  const float* __restrict__ rho;
  float* __restrict__ y;
  int64_t V, n_rays;
  int nb;
  float acc[NB];
  DelayedSum one;  // NB == 1
  __device__ __forceinline__ bool begin(int64_t) {
    one.reset();
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.0f;
    return true;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    if (NB == 1) {
      one.add(rho + v, dl);
      return;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < nb) acc[b] = fmaf(__ldg(rho + b * V + v), dl, acc[b]);
  }
  __device__ __forceinline__ void end(int64_t ray) {
    if (NB == 1) {
      y[ray] = one.total();
      return;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < nb) y[b * n_rays + ray] = acc[b];
  }
};

// g[b][v] += w[b] dl with one atomic add per segment (adjoint of Eq. 5).
template <int NB>
struct ScatterOp {
  static constexpr bool wide_registers = NB < 8;
  const float* __restrict__ y;
  float* __restrict__ g;
  int64_t V, n_rays;
  int nb;
  float w[NB];
  __device__ __forceinline__ bool begin(int64_t ray) {
    bool any = false;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      w[b] = b < nb ? __ldg(y + b * n_rays + ray) : 0.0f;
      any |= w[b] != 0.0f;
    }
    return any;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    if (NB == 1) {  // begin() skipped a ray whose value is zero
      atomicAdd(g + v, __fmul_rn(w[0], dl));
      return;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < nb && w[b] != 0.0f) atomicAdd(g + b * V + v, __fmul_rn(w[b], dl));
  }
  __device__ __forceinline__ void end(int64_t) {}
};

// Warp-aggregated scatter: a lane whose neighbour (lane ^ 1) adds to the same
// voxel in the same step hands its contribution over, and the pair issues one
// atomic add. Neighbouring rays of a cone view often sit in the same voxel at
// the same step; the combine costs two shuffles per segment. (Groups of four,
// and a full match of equal voxels with a group reduction, cost more in
// shuffles than they saved in atomics.)
template <int NB>
struct AggScatterOp : ScatterOp<NB> {
  static constexpr bool wide_registers = NB < 4;
  __device__ __forceinline__ void operator()(int v, float dl) {
    const unsigned m = __activemask();  // the lanes with a segment in this step
    const int lane = threadIdx.x & 31;
    const int pv = __shfl_xor_sync(m, v, 1);
    const bool pair = ((m >> (lane ^ 1)) & 1u) && pv == v;
    if (NB == 1) {  // begin() skipped a ray whose value is zero
      float c = __fmul_rn(this->w[0], dl);
      const float pc = __shfl_xor_sync(m, c, 1);
      if (pair) {
        if (lane & 1) return;
        c = __fadd_rn(c, pc);
      }
      atomicAdd(this->g + v, c);
      return;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      float c = __fmul_rn(this->w[b], dl);
      const float pc = __shfl_xor_sync(m, c, 1);
      if (pair && !(lane & 1)) c = __fadd_rn(c, pc);
      if (b < this->nb && !(pair && (lane & 1)) && c != 0.0f) atomicAdd(this->g + b * this->V + v, c);
    }
  }
};

// Launch knobs for a call without explicit ones: the autotuner's choice for
// this size class if it has one, else the defaults.
inline tsp_launch preferred_launch(const tsp_grid_s* grid, const tsp_geom_s* geom, bool adjoint) {
  tsp_launch f, a;
  if (tuned_launch(grid, geom, &f, &a)) return adjoint ? a : f;
  return default_launch();
}

}  // namespace tsp
