// Data pipeline of the learned warm start: synthetic phantoms rendered on the
// grid's voxel centres, measurement noise from a counter-based generator, and
// the normalisations that turn measurements into the network's input.
//
// Noise: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) on the counter
// seed + (i+1) * 0x9E3779B97F4A7C15, 53-bit uniforms, Box-Muller
// z_i = sqrt(-2 ln(1 - u_i)) cos(2 pi u_{n+i}) for a sample of n values: the
// same stream the synthetic-input module draws on the host.
#include "tsp_internal.h"

namespace tsp {
namespace {

__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + counter * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform53(uint64_t z) { return double(z >> 11) * (1.0 / 9007199254740992.0); }

// rho[b][v] = exp(-r/H_b) + sum_j A exp(-|p - c|^2 / (2 s^2)); params [B][rows][5]
__global__ void phantom_kernel(const float* __restrict__ centres, int Nr, int Ne, int Na,
                               const float* __restrict__ params, int rows, int B, float* __restrict__ rho) {
  const int64_t V = int64_t(Nr) * Ne * Na;
  const int64_t gi = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gi >= V * B) return;
  const int b = int(gi / V);
  const int64_t v = gi - int64_t(b) * V;
  const int ia = int(v % Na), ie = int((v / Na) % Ne), ir = int(v / (int64_t(Na) * Ne));
  const float r = centres[ir];
  const float st = centres[Nr + ie], ct = centres[Nr + Ne + ie];
  const float cp = centres[Nr + 2 * Ne + ia], sp = centres[Nr + 2 * Ne + Na + ia];
  const float x = r * st * cp, y = r * st * sp, z = r * ct;
  const float* P = params + size_t(b) * rows * 5;
  float acc = expf(-r / P[0]);
  for (int j = 1; j < rows; ++j) {
    const float dx = x - P[5 * j], dy = y - P[5 * j + 1], dz = z - P[5 * j + 2];
    const float s = P[5 * j + 4];
    acc += P[5 * j + 3] * expf(-(dx * dx + dy * dy + dz * dz) / (2.0f * s * s));
  }
  rho[gi] = acc;
}

__global__ void batch_max_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ out) {
  const int b = blockIdx.y;
  float m = -INFINITY;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = fmaxf(m, x[int64_t(b) * n + i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) {
    // float max via ordered integer compare (all values compared as signed ints for >= 0, else flipped)
    int* addr = reinterpret_cast<int*>(out + b);
    const int mi = __float_as_int(m);
    if (mi >= 0) atomicMax(addr, mi);
    else atomicMin(reinterpret_cast<unsigned int*>(addr), static_cast<unsigned int>(mi));
  }
}

__global__ void noise_kernel(float* __restrict__ y, int64_t n, const uint64_t* __restrict__ seeds, float frac,
                             const float* __restrict__ ymax) {
  const int b = blockIdx.y;
  const float sigma = frac * ymax[b];
  const uint64_t seed = seeds[b];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double u1 = 1.0 - uniform53(splitmix(seed, uint64_t(i) + 1));
    const double u2 = uniform53(splitmix(seed, uint64_t(n + i) + 1));
    const float z = sqrtf(-2.0f * logf(float(u1))) * cosf(6.28318530717958647692f * float(u2));
    y[int64_t(b) * n + i] += sigma * z;
  }
}

// x[b][i] *= s[i] (s broadcast over the batch)
__global__ void mul_bcast_kernel(float* __restrict__ x, const float* __restrict__ s, int64_t n, int B) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * B; i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= s[i % n];
}

// x[b][i] = divide ? x / scale[b] : x * scale[b]  (scale 0 leaves x)
__global__ void scale_batch_kernel(float* __restrict__ x, const float* __restrict__ scale, int64_t n, int B,
                                   int divide) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * B; i += int64_t(gridDim.x) * blockDim.x) {
    const float s = scale[i / n];
    if (s != 0.0f) x[i] = divide ? x[i] / s : x[i] * s;
  }
}

__global__ void fill_kernel(float* p, int n, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

int eblocks(int64_t n) { return int(std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace
}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_phantoms(tsp_grid grid, const float* params, int rows, int batch, float* rho, void* stream) {
  if (!grid || !params || !rho || rows < 1 || batch <= 0) return fail(TSP_EINVAL, "tsp_phantoms: bad argument");
  tsp_status st = check_device(grid->device);
  if (st != TSP_OK) return st;
  const int64_t n = grid->voxels() * batch;
  phantom_kernel<<<int((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      grid->d_centres, grid->Nr, grid->Ne, grid->Na, params, rows, batch, rho);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_batch_max(const float* x, int64_t n, int batch, float* out, void* stream) {
  if (!x || !out || n <= 0 || batch <= 0 || batch > 65535) return fail(TSP_EINVAL, "tsp_batch_max: bad argument");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  fill_kernel<<<(batch + 255) / 256, 256, 0, cs>>>(out, batch, -INFINITY);
  const int bx = int(std::min<int64_t>((n + 255) / 256, 512));
  batch_max_kernel<<<dim3(bx, batch), 256, 0, cs>>>(x, n, out);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_add_noise(float* y, int64_t n, int batch, const uint64_t* seeds, float frac, float* ymax,
                                    void* stream) {
  if (!y || !seeds || !ymax || n <= 0 || batch <= 0) return fail(TSP_EINVAL, "tsp_add_noise: bad argument");
  tsp_status st = tsp_batch_max(y, n, batch, ymax, stream);
  if (st != TSP_OK) return st;
  const int bx = int(std::min<int64_t>((n + 255) / 256, 2048));
  noise_kernel<<<dim3(bx, batch), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, n, seeds, frac, ymax);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_mul_bcast(float* x, const float* s, int64_t n, int batch, void* stream) {
  if (!x || !s || n <= 0 || batch <= 0) return fail(TSP_EINVAL, "tsp_mul_bcast: bad argument");
  mul_bcast_kernel<<<eblocks(n * batch), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, s, n, batch);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_scale_batch(float* x, const float* scale, int64_t n, int batch, int divide, void* stream) {
  if (!x || !scale || n <= 0 || batch <= 0) return fail(TSP_EINVAL, "tsp_scale_batch: bad argument");
  scale_batch_kernel<<<eblocks(n * batch), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, scale, n, batch, divide);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}
