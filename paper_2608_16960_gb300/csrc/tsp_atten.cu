// Attenuated projection (Sec. 9.3, Eq. 14-18): the first-order corrections of
// the optically thin model for photons lost on their way from the sun to the
// scattering point (tau_1) and from there to the observer (tau_2).
//
//   y    = sum_i rho[v_i] e^{-tau_1[v_i]} e^{-tau_2,i} dl_i           (Eq. 16-17)
//   tau_2,i = sum_{j <= i} sigma[v_j] rho[v_j] dl_j                   (Eq. 18, inclusive)
//   tau_1 = F_1(sigma rho), F_1 one ray per voxel from its centroid    (Eq. 14, Fig. 16b)
//           toward the sun
//
// The sums run over the maximal runs of a ray in one voxel: consecutive
// traversal pieces in the same voxel with no voxel-free gap between them are
// joined before the running sum (a traversal may cut a run at points that are
// no grid boundary, and the inclusive running sum would see the cut). Every
// kernel here is the generic traversal (tsp_kernels.cuh) with a per-segment
// operation: tau_2 and the contributions are carried in registers along the
// ray, rho, sigma and tau_1 are gathered from L2, gradients are scattered with
// L2 atomics. Built with -fmad=false like every other traversal unit.
#include <cmath>

#include "tsp_kernels.cuh"

namespace tsp {
namespace {

// Joins consecutive pieces of one voxel into runs. The voxel's rho, sigma
// and tau_1 are gathered when its run starts and used when it ends (at the
// next traversal step at the earliest), so the gathers overlap the search
// for the next crossing.
struct RunJoin {
  int pv;
  float pdl, r, s, t1;
  __device__ __forceinline__ void reset() {
    pv = -1;
    pdl = 0.0f;
  }
  __device__ __forceinline__ void start(int v, float dl, const float* __restrict__ rho,
                                        const float* __restrict__ sigma, const float* __restrict__ tau1) {
    pv = v;
    pdl = dl;
    r = __ldg(rho + v);
    s = __ldg(sigma + v);
    t1 = __ldg(tau1 + v);
  }
};

// y_1[ray] = sum sigma[v] rho[v] dl over the sunward ray of each voxel
// (tau_1 = F_1(sigma rho); the product is formed per segment). Each
// segment's loads are used at the next segment, as in DelayedSum.
struct ProductGatherOp {
  static constexpr bool wide_registers = true;  // (8% slower under the 72-register cap)
  const float* __restrict__ rho;
  const float* __restrict__ sigma;
  float* __restrict__ out;
  float acc, ps, pr, pdl;
  __device__ __forceinline__ bool begin(int64_t) {
    acc = ps = pr = pdl = 0.0f;
    return true;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    acc = fmaf(__fmul_rn(ps, pr), pdl, acc);
    ps = __ldg(sigma + v);
    pr = __ldg(rho + v);
    pdl = dl;
  }
  __device__ __forceinline__ void end(int64_t ray) { out[ray] = fmaf(__fmul_rn(ps, pr), pdl, acc); }
};

// Add x to *p; with AGG a lane whose neighbour (lane ^ 1) adds to the same
// key in this step hands its value over and the pair issues one atomic add.
template <bool AGG>
__device__ __forceinline__ void scatter_add(float* p, int key, float x) {
  if (AGG) {
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31;
    const int pk = __shfl_xor_sync(m, key, 1);
    const float px = __shfl_xor_sync(m, x, 1);
    if (((m >> (lane ^ 1)) & 1u) && pk == key) {
      if (lane & 1) return;
      x = __fadd_rn(x, px);
    }
  }
  atomicAdd(p, x);
}

// Adjoint of ProductGatherOp: with w = g_tau1[ray], g_rho[v] += w sigma[v] dl
// and g_sigma[v] += w rho[v] dl.
template <bool AGG>
struct ProductScatterOp {
  static constexpr bool wide_registers = true;
  const float* __restrict__ rho;
  const float* __restrict__ sigma;
  const float* __restrict__ g_tau1;
  float* __restrict__ g_rho;
  float* __restrict__ g_sigma;  // may be null
  float w;
  __device__ __forceinline__ bool begin(int64_t ray) {
    w = __ldg(g_tau1 + ray);
    return w != 0.0f;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    const float wd = __fmul_rn(w, dl);
    scatter_add<AGG>(g_rho + v, v, __fmul_rn(wd, __ldg(sigma + v)));
    if (g_sigma) scatter_add<AGG>(g_sigma + v, v, __fmul_rn(wd, __ldg(rho + v)));
  }
  __device__ __forceinline__ void end(int64_t) {}
};

// Attenuated forward (Eq. 17-18) of one density.
struct AttenFwdOp {
  static constexpr bool wide_registers = true;  // (8% slower under the 72-register cap)
  const float* __restrict__ rho;
  const float* __restrict__ sigma;
  const float* __restrict__ tau1;
  float* __restrict__ y;
  RunJoin run;
  float tau2, acc;
  __device__ __forceinline__ void flush() {
    if (run.pv >= 0) {
      const float r = run.r, dl = run.pdl;
      tau2 = fmaf(__fmul_rn(run.s, r), dl, tau2);
      acc = fmaf(__fmul_rn(r, expf(-__fadd_rn(run.t1, tau2))), dl, acc);
    }
    run.reset();
  }
  __device__ __forceinline__ bool begin(int64_t) {
    run.reset();
    tau2 = acc = 0.0f;
    return true;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    if (v == run.pv) {
      run.pdl = __fadd_rn(run.pdl, dl);
    } else {
      flush();
      run.start(v, dl, rho, sigma, tau1);
    }
  }
  __device__ __forceinline__ void gap() { flush(); }
  __device__ __forceinline__ void end(int64_t ray) {
    flush();
    y[ray] = acc;
  }
};

// Gradient of sum_ray gy[ray] y[ray] (AttenFwdOp's y) with respect to rho,
// sigma and tau_1. Along a ray, with c_i the contribution of segment i and
// S_i = sum_{k >= i} c_k = Y - (c_0 + ... + c_{i-1}) (Y = the forward's y):
//   dy/d(e^{-tau_1} rho)[v_i] = e^{-tau_2,i} dl_i,  dy/d(sigma rho)[v_i] = -dl_i S_i.
// The running prefix repeats the forward's arithmetic, so S of the last
// segment is that segment's own contribution. AGG: warp-aggregated adds.
template <bool AGG>
struct AttenBwdOp {
  static constexpr bool wide_registers = true;  // (8% slower under the 72-register cap)
  const float* __restrict__ rho;
  const float* __restrict__ sigma;
  const float* __restrict__ tau1;
  const float* __restrict__ y;
  const float* __restrict__ gy;
  float* __restrict__ g_rho;
  float* __restrict__ g_sigma;  // may be null
  float* __restrict__ g_tau1;   // may be null
  RunJoin run;
  float tau2, pre, Y, w;
  __device__ __forceinline__ void step(int v, float dl, float r, float s, float t1) {
    tau2 = fmaf(__fmul_rn(s, r), dl, tau2);
    const float S = __fsub_rn(Y, pre);  // contributions from this segment on
    pre = fmaf(__fmul_rn(r, expf(-__fadd_rn(t1, tau2))), dl, pre);
    const float e1 = expf(-t1);
    const float ga = __fmul_rn(__fmul_rn(w, expf(-tau2)), dl);  // d/d(e^{-tau_1} rho)
    const float gb = -__fmul_rn(__fmul_rn(w, dl), S);           // d/d(sigma rho)
    scatter_add<AGG>(g_rho + v, v, fmaf(ga, e1, __fmul_rn(gb, s)));
    if (g_sigma) scatter_add<AGG>(g_sigma + v, v, __fmul_rn(gb, r));
    if (g_tau1) scatter_add<AGG>(g_tau1 + v, v, -__fmul_rn(__fmul_rn(ga, r), e1));
  }
  __device__ __forceinline__ void flush() {
    if (run.pv >= 0) step(run.pv, run.pdl, run.r, run.s, run.t1);
    run.reset();
  }
  __device__ __forceinline__ bool begin(int64_t ray) {
    w = __ldg(gy + ray);
    Y = __ldg(y + ray);
    run.reset();
    tau2 = pre = 0.0f;
    return w != 0.0f;
  }
  __device__ __forceinline__ void operator()(int v, float dl) {
    if (v == run.pv) {
      run.pdl = __fadd_rn(run.pdl, dl);
    } else {
      flush();
      run.start(v, dl, rho, sigma, tau1);
    }
  }
  __device__ __forceinline__ void gap() { flush(); }
  __device__ __forceinline__ void end(int64_t) { flush(); }
};

// Sunward rays: voxel v = (ir, ie, ia) starts at its centroid (the midpoints
// of its edges, from the grid's centre table) and runs along the unit sun
// direction. starts / dirs: [3][V] (component-major).
__global__ void sunward_rays_kernel(const float* __restrict__ centres, int Nr, int Ne, int Na, float sx, float sy,
                                    float sz, float* __restrict__ starts, float* __restrict__ dirs) {
  const int64_t V = int64_t(Nr) * Ne * Na;
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < V; v += int64_t(gridDim.x) * blockDim.x) {
    const int ia = int(v % Na), ie = int((v / Na) % Ne), ir = int(v / (int64_t(Na) * Ne));
    const float r = centres[ir], st = centres[Nr + ie], ct = centres[Nr + Ne + ie];
    const float cp = centres[Nr + 2 * Ne + ia], sp = centres[Nr + 2 * Ne + Na + ia];
    const float rs = __fmul_rn(r, st);
    starts[v] = __fmul_rn(rs, cp);
    starts[V + v] = __fmul_rn(rs, sp);
    starts[2 * V + v] = __fmul_rn(r, ct);
    dirs[v] = sx;
    dirs[V + v] = sy;
    dirs[2 * V + v] = sz;
  }
}

template <bool AGG>
void launch_product_scatter(tsp_grid grid, tsp_geom sun, const tsp_launch& l, const float* rho, const float* sigma,
                            const float* g_tau1, float* g_rho, float* g_sigma, int b, cudaStream_t cs) {
  const int64_t V = grid->voxels();
  ProductScatterOp<AGG> op;
  op.rho = rho + b * V;
  op.sigma = sigma + b * V;
  op.g_tau1 = g_tau1 + b * V;
  op.g_rho = g_rho + b * V;
  op.g_sigma = g_sigma ? g_sigma + b * V : nullptr;
  launch_trace(grid, sun, l, op, cs);
}

template <bool AGG>
void launch_atten_bwd(tsp_grid grid, tsp_geom geom, const tsp_launch& l, const float* rho, const float* sigma,
                      const float* tau1, const float* y, const float* gy, float* g_rho, float* g_sigma,
                      float* g_tau1, int b, cudaStream_t cs) {
  const int64_t V = grid->voxels(), n = geom->n_rays;
  AttenBwdOp<AGG> op;
  op.rho = rho + b * V;
  op.sigma = sigma + b * V;
  op.tau1 = tau1 + b * V;
  op.y = y + b * n;
  op.gy = gy + b * n;
  op.g_rho = g_rho + b * V;
  op.g_sigma = g_sigma ? g_sigma + b * V : nullptr;
  op.g_tau1 = g_tau1 ? g_tau1 + b * V : nullptr;
  launch_trace(grid, geom, l, op, cs);
}

tsp_status check_sunward(tsp_grid grid, tsp_geom sun, const char* who) {
  if (sun->n_rays != grid->voxels())
    return fail(TSP_EINVAL, std::string(who) + ": the sunward geometry must have one ray per voxel");
  return TSP_OK;
}

}  // namespace
}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_sunward_rays(tsp_grid grid, const double* sun, float* starts, float* dirs, void* stream) {
  if (!grid || !sun || !starts || !dirs) return fail(TSP_EINVAL, "tsp_sunward_rays: NULL argument");
  const double n = std::sqrt(sun[0] * sun[0] + sun[1] * sun[1] + sun[2] * sun[2]);
  if (!(n > 0.0) || !std::isfinite(n)) return fail(TSP_EINVAL, "tsp_sunward_rays: the sun direction must be non-zero");
  tsp_status st = check_device(grid->device);
  if (st != TSP_OK) return st;
  const int64_t V = grid->voxels();
  const unsigned blocks = unsigned(std::min<int64_t>((V + 255) / 256, 152 * 16));
  sunward_rays_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      grid->d_centres, grid->Nr, grid->Ne, grid->Na, float(sun[0] / n), float(sun[1] / n), float(sun[2] / n), starts,
      dirs);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_atten_optical_depth(tsp_grid grid, tsp_geom sun, const float* rho, const float* sigma,
                                              float* tau1, int batch, void* stream) {
  tsp_status st = check_trace_args(grid, sun, rho, tau1, batch, nullptr, "tsp_atten_optical_depth");
  if (st != TSP_OK) return st;
  if (!sigma) return fail(TSP_EINVAL, "tsp_atten_optical_depth: NULL array");
  st = check_sunward(grid, sun, "tsp_atten_optical_depth");
  if (st != TSP_OK) return st;
  const tsp_launch l = preferred_launch(grid, sun, false);
  const int64_t V = grid->voxels();
  for (int b = 0; b < batch; ++b) {
    ProductGatherOp op;
    op.rho = rho + b * V;
    op.sigma = sigma + b * V;
    op.out = tau1 + b * V;
    launch_trace(grid, sun, l, op, static_cast<cudaStream_t>(stream));
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_atten_optical_depth_adjoint(tsp_grid grid, tsp_geom sun, const float* rho,
                                                      const float* sigma, const float* g_tau1, float* g_rho,
                                                      float* g_sigma, int batch, int accumulate, void* stream) {
  tsp_status st = check_trace_args(grid, sun, g_tau1, g_rho, batch, nullptr, "tsp_atten_optical_depth_adjoint");
  if (st != TSP_OK) return st;
  if (!rho || !sigma) return fail(TSP_EINVAL, "tsp_atten_optical_depth_adjoint: NULL array");
  st = check_sunward(grid, sun, "tsp_atten_optical_depth_adjoint");
  if (st != TSP_OK) return st;
  const tsp_launch l = preferred_launch(grid, sun, true);
  const int64_t V = grid->voxels();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (!accumulate) {
    TSP_CUDA(cudaMemsetAsync(g_rho, 0, sizeof(float) * size_t(V) * batch, cs));
    if (g_sigma) TSP_CUDA(cudaMemsetAsync(g_sigma, 0, sizeof(float) * size_t(V) * batch, cs));
  }
  for (int b = 0; b < batch; ++b) {
    if (l.scatter == 1) launch_product_scatter<true>(grid, sun, l, rho, sigma, g_tau1, g_rho, g_sigma, b, cs);
    else launch_product_scatter<false>(grid, sun, l, rho, sigma, g_tau1, g_rho, g_sigma, b, cs);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_atten_forward(tsp_grid grid, tsp_geom geom, const float* rho, const float* sigma,
                                        const float* tau1, float* y, int batch, void* stream) {
  TSP_RANGE("tsp_atten_forward");
  tsp_status st = check_trace_args(grid, geom, rho, y, batch, nullptr, "tsp_atten_forward");
  if (st != TSP_OK) return st;
  if (!sigma || !tau1) return fail(TSP_EINVAL, "tsp_atten_forward: NULL array");
  const tsp_launch l = preferred_launch(grid, geom, false);
  const int64_t V = grid->voxels();
  for (int b = 0; b < batch; ++b) {
    AttenFwdOp op;
    op.rho = rho + b * V;
    op.sigma = sigma + b * V;
    op.tau1 = tau1 + b * V;
    op.y = y + b * geom->n_rays;
    launch_trace(grid, geom, l, op, static_cast<cudaStream_t>(stream));
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_atten_backward(tsp_grid grid, tsp_geom geom, const float* rho, const float* sigma,
                                         const float* tau1, const float* y, const float* gy, float* g_rho,
                                         float* g_sigma, float* g_tau1, int batch, int accumulate, void* stream) {
  TSP_RANGE("tsp_atten_backward");
  tsp_status st = check_trace_args(grid, geom, gy, g_rho, batch, nullptr, "tsp_atten_backward");
  if (st != TSP_OK) return st;
  if (!rho || !sigma || !tau1 || !y) return fail(TSP_EINVAL, "tsp_atten_backward: NULL array");
  const tsp_launch l = preferred_launch(grid, geom, true);
  const int64_t V = grid->voxels();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (!accumulate) {
    const size_t bytes = sizeof(float) * size_t(V) * batch;
    TSP_CUDA(cudaMemsetAsync(g_rho, 0, bytes, cs));
    if (g_sigma) TSP_CUDA(cudaMemsetAsync(g_sigma, 0, bytes, cs));
    if (g_tau1) TSP_CUDA(cudaMemsetAsync(g_tau1, 0, bytes, cs));
  }
  for (int b = 0; b < batch; ++b) {
    if (l.scatter == 1) launch_atten_bwd<true>(grid, geom, l, rho, sigma, tau1, y, gy, g_rho, g_sigma, g_tau1, b, cs);
    else launch_atten_bwd<false>(grid, geom, l, rho, sigma, tau1, y, gy, g_rho, g_sigma, g_tau1, b, cs);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}
