// Handles, validation and error reporting of the C ABI (include/tsp.h).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "tsp_internal.h"
#include "tsp_table.h"

namespace {
thread_local std::string g_last_error;
const double kPi = 3.14159265358979323846;
const double kTwoPi = 2.0 * kPi;
}  // namespace

namespace tsp {

tsp_status fail(tsp_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

tsp_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky: clear it so the context stays usable
    return TSP_ENOMEM;
  }
  return TSP_ECUDA;
}

namespace {
std::atomic<long long> g_fail_alloc{-1};  // allocations left before the injected failure (-1: none)
std::atomic<long long> g_alloc_count{0};  // allocations made through dev_malloc_raw
}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  g_alloc_count.fetch_add(1);
  long long c = g_fail_alloc.load();
  while (c >= 0 && !g_fail_alloc.compare_exchange_weak(c, c - 1)) {
  }
  if (c == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

tsp_status check_device(int device) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != device)
    return fail(TSP_EINVAL, "handle was created on device " + std::to_string(device) +
                                " but the current device is " + std::to_string(cur));
  return TSP_OK;
}

std::vector<error_reader>& reader_list() {
  static std::vector<error_reader> v;
  return v;
}

void register_error_reader(error_reader r) { reader_list().push_back(r); }

const std::vector<error_reader>& error_readers() { return reader_list(); }

}  // namespace tsp

using tsp::fail;

extern "C" tsp_status tsp_device_status(void* stream, int* code) {
  if (!code) return fail(TSP_EINVAL, "tsp_device_status: NULL code");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  int v = 0;
  for (tsp::error_reader r : tsp::error_readers()) {
    cudaError_t e = r(&v, cs);
    if (e != cudaSuccess) return tsp::cuda_fail(e, "tsp_device_status");
  }
  *code = v;
  if (v & TSP_DEVERR_WAIT_TIMEOUT)
    return fail(TSP_ETIMEOUT, "a tensor-core kernel's bounded wait gave up (device error word " + std::to_string(v) +
                                  ")");
  if (v != 0) return fail(TSP_EDEVICE, "a kernel set the device error word: " + std::to_string(v));
  return TSP_OK;
}

extern "C" const char* tsp_last_error(void) { return g_last_error.c_str(); }

extern "C" int tsp_version(void) { return 1; }

static bool strictly_increasing(const double* v, int n) {
  for (int i = 0; i + 1 < n; ++i)
    if (!(v[i] < v[i + 1])) return false;
  return true;
}

namespace tsp {

}  // namespace tsp

extern "C" tsp_status tsp_grid_create(const double* r_edges, int n_r_edges, const double* theta_edges,
                                      int n_theta_edges, const double* phi_edges, int n_phi_edges,
                                      tsp_grid* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_grid_create: out is NULL");
  *out = nullptr;
  if (!r_edges || !theta_edges || !phi_edges) return fail(TSP_EINVAL, "tsp_grid_create: NULL edge array");
  if (n_r_edges < 2 || n_theta_edges < 2 || n_phi_edges < 2)
    return fail(TSP_EINVAL, "tsp_grid_create: each dimension needs at least 2 edges");
  const int Nr = n_r_edges - 1, Ne = n_theta_edges - 1, Na = n_phi_edges - 1;
  if (Nr > 1024 || Ne > 1024 || Na > 2048)
    return fail(TSP_ENOTSUP, "tsp_grid_create: grid larger than 1024 x 1024 x 2048");
  if (int64_t(Nr) * Ne * Na >= (int64_t(1) << 31))
    return fail(TSP_ENOTSUP, "tsp_grid_create: more than 2^31 - 1 voxels");
  for (int i = 0; i < n_r_edges; ++i)
    if (!std::isfinite(r_edges[i])) return fail(TSP_EINVAL, "tsp_grid_create: non-finite radial edge");
  for (int i = 0; i < n_theta_edges; ++i)
    if (!std::isfinite(theta_edges[i])) return fail(TSP_EINVAL, "tsp_grid_create: non-finite polar edge");
  for (int i = 0; i < n_phi_edges; ++i)
    if (!std::isfinite(phi_edges[i])) return fail(TSP_EINVAL, "tsp_grid_create: non-finite azimuth edge");
  if (!strictly_increasing(r_edges, n_r_edges) || !strictly_increasing(theta_edges, n_theta_edges) ||
      !strictly_increasing(phi_edges, n_phi_edges))
    return fail(TSP_ENOTMONO, "tsp_grid_create: edges must be strictly increasing");
  if (r_edges[0] < 0) return fail(TSP_EINVAL, "tsp_grid_create: negative radius");
  if (theta_edges[0] < -1e-9 || theta_edges[n_theta_edges - 1] > kPi + 1e-9)
    return fail(TSP_EINVAL, "tsp_grid_create: polar edges must lie in [0, pi]");
  const double span = phi_edges[n_phi_edges - 1] - phi_edges[0];
  if (span > kTwoPi + 1e-9) return fail(TSP_EINVAL, "tsp_grid_create: azimuth span exceeds 2 pi");

  tsp_grid g = new (std::nothrow) tsp_grid_s();
  if (!g) return fail(TSP_ENOMEM, "tsp_grid_create: host allocation");
  g->r.assign(r_edges, r_edges + n_r_edges);
  g->th.assign(theta_edges, theta_edges + n_theta_edges);
  g->ph.assign(phi_edges, phi_edges + n_phi_edges);
  std::vector<float> table;
  tsp::build_grid_table(r_edges, n_r_edges, theta_edges, n_theta_edges, phi_edges, n_phi_edges, &table, g);
  // Kernels stage the table in shared memory beside the cone lists (24 KB a
  // block): at most 227 KB a block on this GPU. The grid limits keep the table
  // under 107 KB, so this only guards the layout's arithmetic.
  if (g->words > (232448 - 24576 - 4096) / 4) {
    delete g;
    return fail(TSP_ENOTSUP, "tsp_grid_create: boundary tables exceed the shared memory of a block (too many edges)");
  }
  // voxel centres at the arithmetic midpoints of the edges (for phantoms and models)
  std::vector<float> centres(size_t(Nr + 2 * Ne + 2 * Na));
  for (int k = 0; k < Nr; ++k) centres[k] = float(0.5 * (r_edges[k] + r_edges[k + 1]));
  for (int k = 0; k < Ne; ++k) {
    const double t = 0.5 * (theta_edges[k] + theta_edges[k + 1]);
    centres[Nr + k] = float(std::sin(t));
    centres[Nr + Ne + k] = float(std::cos(t));
  }
  for (int k = 0; k < Na; ++k) {
    const double p = 0.5 * (phi_edges[k] + phi_edges[k + 1]);
    centres[Nr + 2 * Ne + k] = float(std::cos(p));
    centres[Nr + 2 * Ne + Na + k] = float(std::sin(p));
  }
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_table, sizeof(float) * table.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_table, table.data(), sizeof(float) * table.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_centres, sizeof(float) * centres.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_centres, centres.data(), sizeof(float) * centres.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tsp_status st = tsp::cuda_fail(e, "tsp_grid_create: upload");
    if (g->d_table) cudaFree(g->d_table);
    if (g->d_centres) cudaFree(g->d_centres);
    delete g;
    return st;
  }
  *out = g;
  return TSP_OK;
}

extern "C" tsp_status tsp_grid_shape(tsp_grid g, int* n_r, int* n_e, int* n_a) {
  if (!g) return fail(TSP_EINVAL, "tsp_grid_shape: NULL grid");
  if (n_r) *n_r = g->Nr;
  if (n_e) *n_e = g->Ne;
  if (n_a) *n_a = g->Na;
  return TSP_OK;
}

extern "C" void tsp_grid_destroy(tsp_grid g) {
  if (!g) return;
  if (g->d_table) cudaFree(g->d_table);
  if (g->d_centres) cudaFree(g->d_centres);
  delete g;
}

// ---------------------------------------------------------------------------
// geometries
// ---------------------------------------------------------------------------
namespace {

void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

tsp::ff split_ff(double v) {
  const float hi = float(v);
  return tsp::ff{hi, float(v - double(hi))};
}

double norm3(const double a[3]) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

// Detector frame: look toward look_at (origin by default), right = look x up_hint
// (up_hint +Z, or +Y when +Z is along the view axis), up = right x look.
bool view_frame(const double* pos, const double* look_at, const double* up_hint, double look[3],
                double right[3], double up[3]) {
  double d[3] = {-pos[0], -pos[1], -pos[2]};
  if (look_at) {
    d[0] += look_at[0];
    d[1] += look_at[1];
    d[2] += look_at[2];
  }
  const double dn = norm3(d);
  if (!(dn > 0) || !std::isfinite(dn)) return false;
  for (int i = 0; i < 3; ++i) look[i] = d[i] / dn;
  double uh[3] = {0, 0, 1};
  if (up_hint) std::memcpy(uh, up_hint, sizeof uh);
  double rt[3];
  cross3(look, uh, rt);
  double s = norm3(rt);
  if (s < 1e-9) {
    const double alt[3] = {0, 1, 0};
    cross3(look, alt, rt);
    s = norm3(rt);
  }
  if (!(s > 0)) return false;
  for (int i = 0; i < 3; ++i) right[i] = rt[i] / s;
  cross3(right, look, up);
  return true;
}

tsp_status upload_views(tsp_geom g) {
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_views, sizeof(ViewParams) * g->h_views.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_views, g->h_views.data(), sizeof(ViewParams) * g->h_views.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return tsp::cuda_fail(e, "geometry upload");
  return TSP_OK;
}

}  // namespace

extern "C" tsp_status tsp_geom_cone(int n_views, const double* pos, const double* look_at, const double* up,
                                    int H, int W, double fov_h_deg, double fov_w_deg, tsp_geom* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_geom_cone: out is NULL");
  *out = nullptr;
  if (n_views <= 0 || H <= 0 || W <= 0 || !pos) return fail(TSP_EINVAL, "tsp_geom_cone: bad size or NULL pos");
  if (H > 65535 * 8 || W > (1 << 20) || n_views > 65535)
    return fail(TSP_ENOTSUP, "tsp_geom_cone: detector or view count too large");
  if (!(fov_h_deg > 0 && fov_h_deg < 180) || !(fov_w_deg > 0 && fov_w_deg < 180))
    return fail(TSP_EINVAL, "tsp_geom_cone: field of view must be in (0, 180) degrees");
  tsp_geom g = new (std::nothrow) tsp_geom_s();
  if (!g) return fail(TSP_ENOMEM, "tsp_geom_cone: host allocation");
  g->kind = GEOM_CONE;
  g->n_views = n_views;
  g->H = H;
  g->W = W;
  g->n_rays = int64_t(n_views) * H * W;
  const double th = std::tan(0.5 * fov_h_deg * kPi / 180.0), tw = std::tan(0.5 * fov_w_deg * kPi / 180.0);
  g->h_views.resize(n_views);
  for (int v = 0; v < n_views; ++v) {
    double look[3], right[3], upv[3];
    if (!view_frame(pos + 3 * v, look_at ? look_at + 3 * v : nullptr, up ? up + 3 * v : nullptr, look, right,
                    upv)) {
      delete g;
      return fail(TSP_EINVAL, "tsp_geom_cone: degenerate view (pos equals look_at?)");
    }
    ViewParams& p = g->h_views[v];
    for (int i = 0; i < 3; ++i) {
      p.o[i] = split_ff(pos[3 * v + i]);
      p.a[i] = split_ff(look[i]);
      p.bu[i] = split_ff(right[i] * tw);
      p.bv[i] = split_ff(upv[i] * th);
    }
  }
  tsp_status st = upload_views(g);
  if (st != TSP_OK) {
    tsp_geom_destroy(g);
    return st;
  }
  *out = g;
  return TSP_OK;
}

namespace {
// Polar-binned detector rays (Sec. 6): tab = per view [pos | look | right | up]
// (12 floats), then cos/sin of the n_rad bin angles and of the n_az bin
// azimuths. Ray (v, i, j) = pos_v + l (cos t_i look + sin t_i (cos p_j right
// + sin p_j up)); out = starts [3][n] | dirs [3][n].
__global__ void polar_rays_kernel(const float* __restrict__ tab, int n_views, int n_rad, int n_az,
                                  float* __restrict__ out) {
  const int64_t n = int64_t(n_views) * n_rad * n_az;
  const float* ct = tab + 12 * n_views;
  const float* st = ct + n_rad;
  const float* cp = st + n_rad;
  const float* sp = cp + n_az;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(k % n_az), i = int((k / n_az) % n_rad), v = int(k / (int64_t(n_az) * n_rad));
    const float* f = tab + 12 * v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float side = fmaf(cp[j], f[6 + c], __fmul_rn(sp[j], f[9 + c]));
      out[c * n + k] = f[c];
      out[(3 + c) * n + k] = fmaf(ct[i], f[3 + c], __fmul_rn(st[i], side));
    }
  }
}
}  // namespace

extern "C" tsp_status tsp_geom_polar(int n_views, const double* pos, const double* look_at, const double* up,
                                     int n_rad, int n_az, double fov_deg, tsp_geom* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_geom_polar: out is NULL");
  *out = nullptr;
  if (n_views <= 0 || n_rad <= 0 || n_az <= 0 || !pos) return fail(TSP_EINVAL, "tsp_geom_polar: bad size or NULL pos");
  if (!(fov_deg > 0 && fov_deg < 180)) return fail(TSP_EINVAL, "tsp_geom_polar: field of view must be in (0, 180)");
  const int64_t n = int64_t(n_views) * n_rad * n_az;
  if (n >= (int64_t(1) << 40)) return fail(TSP_ENOTSUP, "tsp_geom_polar: too many rays");
  std::vector<float> tab(size_t(12) * n_views + 2 * size_t(n_rad) + 2 * size_t(n_az));
  for (int v = 0; v < n_views; ++v) {
    double look[3], right[3], upv[3];
    if (!view_frame(pos + 3 * v, look_at ? look_at + 3 * v : nullptr, up ? up + 3 * v : nullptr, look, right, upv))
      return fail(TSP_EINVAL, "tsp_geom_polar: degenerate view (pos equals look_at?)");
    for (int c = 0; c < 3; ++c) {
      tab[12 * v + c] = float(pos[3 * v + c]);
      tab[12 * v + 3 + c] = float(look[c]);
      tab[12 * v + 6 + c] = float(right[c]);
      tab[12 * v + 9 + c] = float(upv[c]);
    }
  }
  const double half = 0.5 * fov_deg * kPi / 180.0;
  float* t = tab.data() + 12 * size_t(n_views);
  for (int i = 0; i < n_rad; ++i) {
    const double a = (i + 0.5) / n_rad * half;
    t[i] = float(std::cos(a));
    t[n_rad + i] = float(std::sin(a));
  }
  for (int j = 0; j < n_az; ++j) {
    const double a = 2.0 * kPi * (j + 0.5) / n_az;
    t[2 * n_rad + j] = float(std::cos(a));
    t[2 * n_rad + n_az + j] = float(std::sin(a));
  }
  tsp_geom g = new (std::nothrow) tsp_geom_s();
  if (!g) return fail(TSP_ENOMEM, "tsp_geom_polar: host allocation");
  g->kind = GEOM_RAYS;
  g->n_views = n_views;
  g->H = n_rad;
  g->W = n_az;
  g->n_rays = n;
  float* d_tab = nullptr;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaMalloc(&g->owned, sizeof(float) * 6 * size_t(n));
  if (e == cudaSuccess) e = cudaMalloc(&d_tab, sizeof(float) * tab.size());
  if (e == cudaSuccess) e = cudaMemcpy(d_tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned blocks = unsigned(std::min<int64_t>((n + 255) / 256, 152 * 16));
    polar_rays_kernel<<<blocks, 256>>>(d_tab, n_views, n_rad, n_az, g->owned);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (d_tab) cudaFree(d_tab);
  if (e != cudaSuccess) {
    tsp_geom_destroy(g);
    return tsp::cuda_fail(e, "tsp_geom_polar");
  }
  g->starts = g->owned;
  g->dirs = g->owned + 3 * n;
  *out = g;
  return TSP_OK;
}

extern "C" tsp_status tsp_geom_parallel(int n_views, const double* pos, const double* up, int H, int W,
                                        double size_h, double size_w, tsp_geom* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_geom_parallel: out is NULL");
  *out = nullptr;
  if (n_views <= 0 || H <= 0 || W <= 0 || !pos) return fail(TSP_EINVAL, "tsp_geom_parallel: bad size or NULL pos");
  if (H > 65535 * 8 || W > (1 << 20) || n_views > 65535)
    return fail(TSP_ENOTSUP, "tsp_geom_parallel: detector or view count too large");
  if (!(size_h > 0) || !(size_w > 0)) return fail(TSP_EINVAL, "tsp_geom_parallel: detector size must be > 0");
  tsp_geom g = new (std::nothrow) tsp_geom_s();
  if (!g) return fail(TSP_ENOMEM, "tsp_geom_parallel: host allocation");
  g->kind = GEOM_PARALLEL;
  g->n_views = n_views;
  g->H = H;
  g->W = W;
  g->n_rays = int64_t(n_views) * H * W;
  g->h_views.resize(n_views);
  for (int v = 0; v < n_views; ++v) {
    double look[3], right[3], upv[3];
    if (!view_frame(pos + 3 * v, nullptr, up ? up + 3 * v : nullptr, look, right, upv)) {
      delete g;
      return fail(TSP_EINVAL, "tsp_geom_parallel: degenerate view (pos at the origin?)");
    }
    ViewParams& p = g->h_views[v];
    for (int i = 0; i < 3; ++i) {
      p.o[i] = split_ff(pos[3 * v + i]);
      p.a[i] = split_ff(look[i]);
      p.bu[i] = split_ff(right[i] * size_w);
      p.bv[i] = split_ff(upv[i] * size_h);
    }
  }
  tsp_status st = upload_views(g);
  if (st != TSP_OK) {
    tsp_geom_destroy(g);
    return st;
  }
  *out = g;
  return TSP_OK;
}

extern "C" tsp_status tsp_geom_rays(int64_t n_rays, const float* starts, const float* dirs, int copy,
                                    tsp_geom* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_geom_rays: out is NULL");
  *out = nullptr;
  if (n_rays <= 0 || !starts || !dirs) return fail(TSP_EINVAL, "tsp_geom_rays: bad size or NULL array");
  if (n_rays >= (int64_t(1) << 40)) return fail(TSP_ENOTSUP, "tsp_geom_rays: too many rays");
  tsp_geom g = new (std::nothrow) tsp_geom_s();
  if (!g) return fail(TSP_ENOMEM, "tsp_geom_rays: host allocation");
  g->kind = GEOM_RAYS;
  g->n_views = 1;
  g->H = 1;
  g->W = 0;
  g->n_rays = n_rays;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    delete g;
    return tsp::cuda_fail(e, "cudaGetDevice");
  }
  if (copy) {
    e = cudaMalloc(&g->owned, sizeof(float) * 6 * size_t(n_rays));
    if (e == cudaSuccess)
      e = cudaMemcpy(g->owned, starts, sizeof(float) * 3 * size_t(n_rays), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(g->owned + 3 * n_rays, dirs, sizeof(float) * 3 * size_t(n_rays), cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
      if (g->owned) cudaFree(g->owned);
      delete g;
      return tsp::cuda_fail(e, "tsp_geom_rays: copy");
    }
    g->starts = g->owned;
    g->dirs = g->owned + 3 * n_rays;
  } else {
    g->starts = starts;
    g->dirs = dirs;
  }
  *out = g;
  return TSP_OK;
}

extern "C" tsp_status tsp_geom_num_rays(tsp_geom g, int64_t* n) {
  if (!g || !n) return fail(TSP_EINVAL, "tsp_geom_num_rays: NULL argument");
  *n = g->n_rays;
  return TSP_OK;
}

extern "C" void tsp_geom_destroy(tsp_geom g) {
  if (!g) return;
  if (g->d_views) cudaFree(g->d_views);
  if (g->owned) cudaFree(g->owned);
  delete g;
}

extern "C" tsp_status tsp_debug_fail_allocation(int64_t after) {
  tsp::g_fail_alloc.store(after < 0 ? -1 : (long long)after);
  return TSP_OK;
}

extern "C" tsp_status tsp_debug_allocation_count(int64_t* count) {
  if (!count) return fail(TSP_EINVAL, "tsp_debug_allocation_count: count is NULL");
  *count = (int64_t)tsp::g_alloc_count.load();
  return TSP_OK;
}
