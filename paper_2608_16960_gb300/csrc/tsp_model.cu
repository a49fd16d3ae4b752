// Parametric density model and optimiser kernels for reconstructions that
// differentiate through the projector (Sec. 4.5 Eq. 7 / Listing 8; Sec. 6
// Eq. 10 uses spherical harmonics per shell).
//
// Model: rho[ir, ie, ia] = sum_j sum_q B[ir, j] c[j, q] Y[(ie, ia), q]
//   B: clamped cubic B-splines in r (Cox-de Boor recursion, de Boor 1972),
//   Y: real orthonormal spherical harmonics, q = l^2 + l + m, |m| <= l <= L,
//      from the normalised associated Legendre recurrence:
//        Y_l0 = N_l0 P_l(cos t), Y_lm = sqrt(2) N_lm P_l^m(cos t) cos(m p) (m > 0),
//        Y_l,-m = sqrt(2) N_lm P_l^m(cos t) sin(m p), N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
//      (no Condon-Shortley phase in P_l^m).
// Both bases are evaluated on the host in double at the voxel centres and
// uploaded as float32 tables (B as [Nr][nb], Y transposed as [nq][Ne*Na]).
//
// Also here: Adam (Kingma and Ba, 2015) and the squared-residual loss.
#include <cmath>
#include <vector>

#include "tsp_internal.h"

struct tsp_shbs_s {
  int Nr = 0, nang = 0, nb = 0, L = 0, nq = 0;
  float* B = nullptr;   // [Nr][nb]
  float* Yt = nullptr;  // [nq][nang]
  float* T = nullptr;   // [Nr][nq] scratch for the render and its adjoint
  int device = 0;
};

namespace tsp {
namespace {

const double kPi = 3.14159265358979323846;

// Clamped cubic B-spline basis values at x (nb functions, uniform interior knots).
void bspline_row(double x, double x0, double x1, int nb, double* out) {
  const int deg = 3, nk = nb + deg + 1;
  std::vector<double> t(nk);
  const int n_int = nb - deg - 1;  // interior knots
  for (int i = 0; i <= deg; ++i) {
    t[i] = x0;
    t[nk - 1 - i] = x1;
  }
  for (int i = 1; i <= n_int; ++i) t[deg + i] = x0 + (x1 - x0) * i / (n_int + 1);
  // degree-0 indicators; the right end belongs to the last non-empty interval
  std::vector<double> N(nk - 1, 0.0);
  for (int i = 0; i + 1 < nk; ++i) {
    if (t[i] < t[i + 1] && ((x >= t[i] && x < t[i + 1]) || (x == x1 && t[i + 1] == x1 && i + 1 == nk - 1 - deg)))
      N[i] = 1.0;
  }
  for (int k = 1; k <= deg; ++k) {
    for (int i = 0; i + k + 1 < nk; ++i) {
      double a = 0.0, b = 0.0;
      if (t[i + k] > t[i]) a = (x - t[i]) / (t[i + k] - t[i]) * N[i];
      if (t[i + k + 1] > t[i + 1]) b = (t[i + k + 1] - x) / (t[i + k + 1] - t[i + 1]) * N[i + 1];
      N[i] = a + b;
    }
  }
  for (int j = 0; j < nb; ++j) out[j] = N[j];
}

// Real orthonormal spherical harmonics up to degree L at (theta, phi).
void sh_row(double theta, double phi, int L, double* out) {
  const double x = std::cos(theta), s = std::sin(theta);
  // normalised associated Legendre functions Pbar_l^m = N_lm P_l^m (no CS phase)
  std::vector<double> P((L + 1) * (L + 1), 0.0);
  auto at = [&](int l, int m) -> double& { return P[l * (L + 1) + m]; };
  at(0, 0) = std::sqrt(1.0 / (4.0 * kPi));
  for (int m = 1; m <= L; ++m) at(m, m) = std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * at(m - 1, m - 1);
  for (int m = 0; m < L; ++m) at(m + 1, m) = std::sqrt(2.0 * m + 3.0) * x * at(m, m);
  for (int m = 0; m <= L; ++m) {
    for (int l = m + 2; l <= L; ++l) {
      const double a = std::sqrt((4.0 * l * l - 1.0) / (double(l) * l - double(m) * m));
      const double b = std::sqrt(((l - 1.0) * (l - 1.0) - double(m) * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      at(l, m) = a * (x * at(l - 1, m) - b * at(l - 2, m));
    }
  }
  for (int l = 0; l <= L; ++l) {
    out[l * l + l] = at(l, 0);
    for (int m = 1; m <= l; ++m) {
      const double v = std::sqrt(2.0) * at(l, m);
      out[l * l + l + m] = v * std::cos(m * phi);
      out[l * l + l - m] = v * std::sin(m * phi);
    }
  }
}

// T[ir][q] = sum_j B[ir][j] c[j][q]
__global__ void shbs_t_kernel(const float* __restrict__ B, const float* __restrict__ c, float* __restrict__ T, int Nr,
                              int nb, int nq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nr * nq) return;
  const int ir = i / nq, q = i - ir * nq;
  float acc = 0.0f;
  for (int j = 0; j < nb; ++j) acc = fmaf(B[ir * nb + j], c[j * nq + q], acc);
  T[i] = acc;
}

// rho[ir][a] = sum_q T[ir][q] Yt[q][a]; block (ir, a-chunk), T row in shared memory.
__global__ void shbs_render_kernel(const float* __restrict__ T, const float* __restrict__ Yt, float* __restrict__ rho,
                                   int nang, int nq) {
  extern __shared__ float tr[];
  const int ir = blockIdx.y;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) tr[q] = T[ir * nq + q];
  __syncthreads();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nang) return;
  float acc = 0.0f;
  for (int q = 0; q < nq; ++q) acc = fmaf(tr[q], __ldg(Yt + size_t(q) * nang + a), acc);
  rho[size_t(ir) * nang + a] = acc;
}

// dT[ir][q] = sum_a G[ir][a] Yt[q][a]; block (ir, q), reduction over a.
__global__ void shbs_dt_kernel(const float* __restrict__ G, const float* __restrict__ Yt, float* __restrict__ dT,
                               int nang, int nq) {
  const int ir = blockIdx.y, q = blockIdx.x;
  float acc = 0.0f;
  for (int a = threadIdx.x; a < nang; a += blockDim.x) acc = fmaf(G[size_t(ir) * nang + a], Yt[size_t(q) * nang + a], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) dT[ir * nq + q] = v;
  }
}

// dc[j][q] = sum_ir B[ir][j] dT[ir][q]
__global__ void shbs_dc_kernel(const float* __restrict__ B, const float* __restrict__ dT, float* __restrict__ dc, int Nr,
                               int nb, int nq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * nq) return;
  const int j = i / nq, q = i - j * nq;
  float acc = 0.0f;
  for (int ir = 0; ir < Nr; ++ir) acc = fmaf(B[ir * nb + j], dT[ir * nq + q], acc);
  dc[i] = acc;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd,
                            float c1, float c2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = fmaf(wd, p[i], g[i]);
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// grad = 2 (yhat - y) (if grad != NULL); loss += sum (yhat - y)^2 in double.
__global__ void sq_residual_kernel(const float* __restrict__ yhat, const float* __restrict__ y, int64_t n,
                                   float* __restrict__ grad, double* __restrict__ loss) {
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float r = yhat[i] - y[i];
    if (grad) grad[i] = 2.0f * r;
    acc += double(r) * double(r);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, v);
  }
}

// loss += lambda sum_{ir < Nr-1, q} (c[ir+1][q] - c[ir][q])^2 (double) and
// grad[ir][q] += its derivative: one thread per coefficient.
__global__ void tikhonov_radial_kernel(const float* __restrict__ c, int Nr, int nq, float lambda,
                                       float* __restrict__ grad, double* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  if (i < Nr * nq) {
    const int ir = i / nq;
    const float here = c[i];
    float g = 0.0f;
    if (ir > 0) g = fmaf(2.0f * lambda, here - c[i - nq], g);
    if (ir + 1 < Nr) {
      const float d = c[i + nq] - here;
      g = fmaf(-2.0f * lambda, d, g);
      part = double(lambda) * double(d) * double(d);
    }
    if (grad) grad[i] += g;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, part);
}

// loss += sum (w yhat - y)^2 (double); grad = 2 w (w yhat - y).
__global__ void weighted_residual_kernel(const float* __restrict__ yhat, const float* __restrict__ w,
                                         const float* __restrict__ y, int64_t n, float* __restrict__ grad,
                                         double* __restrict__ loss) {
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float wi = w[i];
    const float r = fmaf(wi, yhat[i], -y[i]);
    if (grad) grad[i] = 2.0f * wi * r;
    acc += double(r) * double(r);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, v);
  }
}

// out += sum x y (double), grid-stride with a block reduction.
__global__ void vec_dot_kernel(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                               double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(x[i]) * double(y[i]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}

// y = a x + b y
__global__ void vec_axpby_kernel(float a, const float* __restrict__ x, float b, float* __restrict__ y, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = fmaf(a, x[i], b * y[i]);
}

// out = w x (elementwise)
__global__ void vec_mul_kernel(const float* __restrict__ w, const float* __restrict__ x, float* __restrict__ out,
                               int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = w[i] * x[i];
}

int vec_blocks(int64_t n) { return int(std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace
}  // namespace tsp

using namespace tsp;

extern "C" tsp_status tsp_shbs_create(int n_basis_r, int L, const double* r_centres, int Nr, const double* theta_centres,
                                      int Ne, const double* phi_centres, int Na, double r_min, double r_max,
                                      tsp_shbs* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_shbs_create: out is NULL");
  *out = nullptr;
  if (n_basis_r < 4 || L < 0 || L > 32 || Nr <= 0 || Ne <= 0 || Na <= 0 || !r_centres || !theta_centres || !phi_centres ||
      !(r_max > r_min))
    return fail(TSP_EINVAL, "tsp_shbs_create: bad argument");
  tsp_shbs h = new (std::nothrow) tsp_shbs_s();
  if (!h) return fail(TSP_ENOMEM, "tsp_shbs_create: host allocation");
  h->Nr = Nr;
  h->nang = Ne * Na;
  h->nb = n_basis_r;
  h->L = L;
  h->nq = (L + 1) * (L + 1);
  std::vector<float> B(size_t(Nr) * h->nb), Yt(size_t(h->nq) * h->nang);
  std::vector<double> row(std::max(h->nb, h->nq));
  for (int ir = 0; ir < Nr; ++ir) {
    bspline_row(std::min(std::max(r_centres[ir], r_min), r_max), r_min, r_max, h->nb, row.data());
    for (int j = 0; j < h->nb; ++j) B[size_t(ir) * h->nb + j] = float(row[j]);
  }
  for (int ie = 0; ie < Ne; ++ie) {
    for (int ia = 0; ia < Na; ++ia) {
      sh_row(theta_centres[ie], phi_centres[ia], L, row.data());
      for (int q = 0; q < h->nq; ++q) Yt[size_t(q) * h->nang + ie * Na + ia] = float(row[q]);
    }
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->B, sizeof(float) * B.size());
  if (e == cudaSuccess) e = cudaMalloc(&h->Yt, sizeof(float) * Yt.size());
  if (e == cudaSuccess) e = cudaMalloc(&h->T, sizeof(float) * size_t(Nr) * h->nq);
  if (e == cudaSuccess) e = cudaMemcpy(h->B, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->Yt, Yt.data(), sizeof(float) * Yt.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tsp_shbs_destroy(h);
    return cuda_fail(e, "tsp_shbs_create: upload");
  }
  *out = h;
  return TSP_OK;
}

extern "C" tsp_status tsp_shbs_create_shells(int L, int Nr, const double* theta_centres, int Ne,
                                             const double* phi_centres, int Na, tsp_shbs* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_shbs_create_shells: out is NULL");
  *out = nullptr;
  if (L < 0 || L > 32 || Nr <= 0 || Ne <= 0 || Na <= 0 || !theta_centres || !phi_centres)
    return fail(TSP_EINVAL, "tsp_shbs_create_shells: bad argument");
  tsp_shbs h = new (std::nothrow) tsp_shbs_s();
  if (!h) return fail(TSP_ENOMEM, "tsp_shbs_create_shells: host allocation");
  h->Nr = Nr;
  h->nang = Ne * Na;
  h->nb = Nr;
  h->L = L;
  h->nq = (L + 1) * (L + 1);
  std::vector<float> B(size_t(Nr) * Nr, 0.0f), Yt(size_t(h->nq) * h->nang);
  for (int ir = 0; ir < Nr; ++ir) B[size_t(ir) * Nr + ir] = 1.0f;  // one coefficient set per shell
  std::vector<double> row(h->nq);
  for (int ie = 0; ie < Ne; ++ie) {
    for (int ia = 0; ia < Na; ++ia) {
      sh_row(theta_centres[ie], phi_centres[ia], L, row.data());
      for (int q = 0; q < h->nq; ++q) Yt[size_t(q) * h->nang + ie * Na + ia] = float(row[q]);
    }
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->B, sizeof(float) * B.size());
  if (e == cudaSuccess) e = cudaMalloc(&h->Yt, sizeof(float) * Yt.size());
  if (e == cudaSuccess) e = cudaMalloc(&h->T, sizeof(float) * size_t(Nr) * h->nq);
  if (e == cudaSuccess) e = cudaMemcpy(h->B, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->Yt, Yt.data(), sizeof(float) * Yt.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tsp_shbs_destroy(h);
    return cuda_fail(e, "tsp_shbs_create_shells: upload");
  }
  *out = h;
  return TSP_OK;
}

extern "C" void tsp_shbs_destroy(tsp_shbs h) {
  if (!h) return;
  if (h->B) cudaFree(h->B);
  if (h->Yt) cudaFree(h->Yt);
  if (h->T) cudaFree(h->T);
  delete h;
}

extern "C" tsp_status tsp_shbs_tables(tsp_shbs h, float* B_host, float* Yt_host) {
  if (!h) return fail(TSP_EINVAL, "tsp_shbs_tables: NULL handle");
  if (B_host) TSP_CUDA(cudaMemcpy(B_host, h->B, sizeof(float) * size_t(h->Nr) * h->nb, cudaMemcpyDeviceToHost));
  if (Yt_host) TSP_CUDA(cudaMemcpy(Yt_host, h->Yt, sizeof(float) * size_t(h->nq) * h->nang, cudaMemcpyDeviceToHost));
  return TSP_OK;
}

extern "C" tsp_status tsp_shbs_render(tsp_shbs h, const float* coeffs, float* rho, void* stream) {
  if (!h || !coeffs || !rho) return fail(TSP_EINVAL, "tsp_shbs_render: NULL argument");
  tsp_status st = check_device(h->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int n = h->Nr * h->nq;
  shbs_t_kernel<<<(n + 127) / 128, 128, 0, cs>>>(h->B, coeffs, h->T, h->Nr, h->nb, h->nq);
  dim3 grid((h->nang + 255) / 256, h->Nr);
  shbs_render_kernel<<<grid, 256, sizeof(float) * h->nq, cs>>>(h->T, h->Yt, rho, h->nang, h->nq);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_shbs_render_adjoint(tsp_shbs h, const float* grad_rho, float* grad_coeffs, void* stream) {
  if (!h || !grad_rho || !grad_coeffs) return fail(TSP_EINVAL, "tsp_shbs_render_adjoint: NULL argument");
  tsp_status st = check_device(h->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  shbs_dt_kernel<<<dim3(h->nq, h->Nr), 256, 0, cs>>>(grad_rho, h->Yt, h->T, h->nang, h->nq);
  const int n = h->nb * h->nq;
  shbs_dc_kernel<<<(n + 127) / 128, 128, 0, cs>>>(h->B, h->T, grad_coeffs, h->Nr, h->nb, h->nq);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_adam(float* params, const float* grads, float* m, float* v, int64_t n, float lr, float beta1,
                               float beta2, float eps, float weight_decay, int step, void* stream) {
  if (!params || !grads || !m || !v || n <= 0 || step < 1) return fail(TSP_EINVAL, "tsp_adam: bad argument");
  const float c1 = float(1.0 - std::pow(double(beta1), step));
  const float c2 = float(1.0 - std::pow(double(beta2), step));
  const int blocks = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
  adam_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grads, m, v, n, lr, beta1, beta2, eps,
                                                                     weight_decay, c1, c2);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_sq_residual(const float* yhat, const float* y, int64_t n, float* grad, double* loss,
                                      void* stream) {
  if (!yhat || !y || n <= 0) return fail(TSP_EINVAL, "tsp_sq_residual: bad argument");
  const int blocks = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
  sq_residual_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(yhat, y, n, grad, loss);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_tikhonov_radial(const float* coeffs, int n_r, int n_q, float lambda, float* grad,
                                          double* loss, void* stream) {
  if (!coeffs || n_r <= 0 || n_q <= 0 || !(lambda >= 0.0f))
    return fail(TSP_EINVAL, "tsp_tikhonov_radial: bad argument");
  const int n = n_r * n_q;
  tikhonov_radial_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(coeffs, n_r, n_q, lambda,
                                                                                          grad, loss);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_sq_residual_weighted(const float* yhat, const float* w, const float* y, int64_t n,
                                               float* grad, double* loss, void* stream) {
  if (!yhat || !w || !y || n <= 0) return fail(TSP_EINVAL, "tsp_sq_residual_weighted: bad argument");
  const int blocks = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
  weighted_residual_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(yhat, w, y, n, grad, loss);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_vec_dot(const float* x, const float* y, int64_t n, double* out, void* stream) {
  if (!x || !y || !out || n < 0) return fail(TSP_EINVAL, "tsp_vec_dot: bad argument");
  if (n == 0) return TSP_OK;
  vec_dot_kernel<<<vec_blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n, out);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_vec_axpby(float a, const float* x, float b, float* y, int64_t n, void* stream) {
  if (!x || !y || n < 0) return fail(TSP_EINVAL, "tsp_vec_axpby: bad argument");
  if (n == 0) return TSP_OK;
  vec_axpby_kernel<<<vec_blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, x, b, y, n);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_vec_mul(const float* w, const float* x, float* out, int64_t n, void* stream) {
  if (!w || !x || !out || n < 0) return fail(TSP_EINVAL, "tsp_vec_mul: bad argument");
  if (n == 0) return TSP_OK;
  vec_mul_kernel<<<vec_blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(w, x, out, n);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}
