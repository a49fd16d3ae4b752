// FP64 CPU oracle for the spherical-grid projector F and its adjoint F^T.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
// execute this file; only the tests, the smoke check and the benchmark's CPU
// baseline leg use it. It shares no code, headers or tables with the CUDA path.
//
// What it computes (TomoSphero, Sec. 2.1, Eq. 3-5): for a ray p(l) = x + l n,
// n normalised, l >= 0, the line integral of the piecewise-constant density
// defined on a spherical grid (zero outside the grid, Sec. 4.6):
//     y = sum_i rho[r_i, e_i, a_i] * dl_i.
// The adjoint is F^T y [v] = sum_rays y_ray * |ray  intersect  voxel v|.
//
// Two independent derivations of the per-ray segment list live here:
//   trace_definition: every crossing with every boundary (Sec. 3.1), sorted
//     (Sec. 3.3), each piece classified by its midpoint. This is the plain
//     definition of Eq. 4 and is what forward/adjoint use.
//   trace_paper: the paper's steps 1-3 literally - crossing directions by
//     Eq. 11-13, region = boundary index minus one for a negative crossing,
//     sort, forward fill from the start voxel, zero invalid rows (Table 2).
// The tests check that the two agree, and pin the first against closed forms.
//
// Readings of points where the paper is silent (listed in the design notes):
//   * polar index e grows with the polar angle measured from +Z (Eq. 12);
//   * azimuth boundaries spanning exactly 2 pi form N_a distinct half-planes
//     and region indices wrap modulo N_a;
//   * crossings at l <= 0 (behind the start) are dropped (Eq. 3 integrates
//     from l = 0);
//   * bins are half-open [edge_k, edge_{k+1});
//   * the theta = pi/2 "cone" is the plane z = 0; theta = 0 or pi is the axis,
//     which a ray only grazes, so it contributes no crossing.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;
const double kTwoPi = 2.0 * kPi;
const double kInf = std::numeric_limits<double>::infinity();

struct Grid {
  std::vector<double> r, th, ph;  // boundary locations
  int Nr = 0, Ne = 0, Na = 0;
  bool wrap = false;              // azimuth covers the full circle
};

bool make_grid(const double* r, int nr1, const double* th, int ne1, const double* ph, int na1,
               Grid* g) {
  if (nr1 < 2 || ne1 < 2 || na1 < 2) return false;
  g->r.assign(r, r + nr1);
  g->th.assign(th, th + ne1);
  g->ph.assign(ph, ph + na1);
  g->Nr = nr1 - 1;
  g->Ne = ne1 - 1;
  g->Na = na1 - 1;
  for (int i = 0; i + 1 < nr1; ++i) if (!(r[i] < r[i + 1])) return false;
  for (int i = 0; i + 1 < ne1; ++i) if (!(th[i] < th[i + 1])) return false;
  for (int i = 0; i + 1 < na1; ++i) if (!(ph[i] < ph[i + 1])) return false;
  if (r[0] < 0) return false;
  const double span = ph[na1 - 1] - ph[0];
  if (span > kTwoPi + 1e-9) return false;
  g->wrap = std::fabs(span - kTwoPi) <= 1e-9;
  return true;
}

// Index of the half-open bin [e_k, e_{k+1}) holding v: upper_bound - 1, so -1
// below the first edge and N (= edges.size() - 1) at or above the last.
int bin_of(const std::vector<double>& e, double v) {
  return int(std::upper_bound(e.begin(), e.end(), v) - e.begin()) - 1;
}

// Azimuth of (x, y) mapped into [ph_0, ph_0 + 2 pi).
double azimuth(const Grid& g, double x, double y) {
  double d = std::atan2(y, x) - g.ph[0];
  d = std::fmod(d, kTwoPi);
  if (d < 0) d += kTwoPi;
  if (d >= kTwoPi) d -= kTwoPi;
  return g.ph[0] + d;
}

// Raw (possibly out-of-range) region indices of a point.
void regions_of(const Grid& g, const double m[3], int* ir, int* ie, int* ia) {
  const double r = std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  *ir = bin_of(g.r, r);
  double ct = r > 0 ? m[2] / r : 1.0;
  ct = std::min(1.0, std::max(-1.0, ct));
  *ie = bin_of(g.th, std::acos(ct));
  const double a = azimuth(g, m[0], m[1]);
  if (g.wrap) {
    int k = bin_of(g.ph, a);
    *ia = std::min(k, g.Na - 1);
  } else {
    *ia = bin_of(g.ph, a);
  }
}

int64_t flat_index(const Grid& g, int ir, int ie, int ia) {
  if (ir < 0 || ir >= g.Nr || ie < 0 || ie >= g.Ne || ia < 0 || ia >= g.Na) return -1;
  return (int64_t(ir) * g.Ne + ie) * g.Na + ia;
}

// Real roots of a t^2 + 2 bh t + c = 0 by the cancellation-free form
// q = -(bh + sign(bh) sqrt(bh^2 - a c)), roots q/a and c/q (Numerical Recipes 5.6).
int quad_roots(double a, double bh, double c, double out[2]) {
  if (a == 0.0) {
    if (bh == 0.0) return 0;
    out[0] = -c / (2.0 * bh);
    return 1;
  }
  const double d = bh * bh - a * c;
  if (d < 0) return 0;
  const double s = std::sqrt(d);
  const double q = -(bh + (bh >= 0 ? s : -s));
  if (q == 0.0) {  // bh == 0 and d == 0: double root at 0
    out[0] = 0.0;
    out[1] = 0.0;
    return 2;
  }
  out[0] = q / a;
  out[1] = c / q;
  return 2;
}

struct Seg {
  int64_t v;
  double len;
  double l0 = 0.0;  // start of the piece along the unit-direction line (definition method)
};

void normalise(const double n_in[3], double n[3]) {
  const double s = std::sqrt(n_in[0] * n_in[0] + n_in[1] * n_in[1] + n_in[2] * n_in[2]);
  n[0] = n_in[0] / s;
  n[1] = n_in[1] / s;
  n[2] = n_in[2] / s;
}

// ---------------------------------------------------------------------------
// Crossing candidates (Sec. 3.1): spheres (refs [30]), cones (refs [28],[29]),
// half-planes. Each callback receives the distance l and the boundary kind/index.
// ---------------------------------------------------------------------------
template <class F>
void all_crossings(const Grid& g, const double x[3], const double n[3], F&& emit) {
  const double xn = x[0] * n[0] + x[1] * n[1] + x[2] * n[2];
  const double xx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  double roots[2];
  // spheres |x + l n|^2 = R^2  ->  l^2 + 2 (x.n) l + |x|^2 - R^2 = 0
  for (int k = 0; k <= g.Nr; ++k) {
    const double R = g.r[k];
    if (R <= 0) continue;
    const int nr = quad_roots(1.0, xn, xx - R * R, roots);
    for (int i = 0; i < nr; ++i) emit(roots[i], 0, k);
  }
  // cones: points with p_z = cos(theta_k) |p|; squared:
  // (n_z^2 - c^2) l^2 + 2 (x_z n_z - c^2 x.n) l + (x_z^2 - c^2 |x|^2) = 0,
  // keeping the nappe with sign(p_z) = sign(c).
  for (int k = 0; k <= g.Ne; ++k) {
    const double c = std::cos(g.th[k]);
    if (std::fabs(c) < 1e-12) {  // theta = pi/2: the plane z = 0
      if (n[2] != 0.0) emit(-x[2] / n[2], 1, k);
      continue;
    }
    if (std::fabs(c) >= 1.0 - 1e-15) continue;  // the polar axis: grazed, never crossed
    const double c2 = c * c;
    const int nr = quad_roots(n[2] * n[2] - c2, x[2] * n[2] - c2 * xn, x[2] * x[2] - c2 * xx, roots);
    for (int i = 0; i < nr; ++i) {
      const double pz = x[2] + roots[i] * n[2];
      if (pz * c > 0) emit(roots[i], 1, k);
    }
  }
  // half-planes through the z axis at azimuth phi_k, on the side cos/sin(phi_k)
  const int nplanes = g.wrap ? g.Na : g.Na + 1;
  for (int k = 0; k < nplanes; ++k) {
    const double cp = std::cos(g.ph[k]), sp = std::sin(g.ph[k]);
    const double den = n[0] * sp - n[1] * cp;
    if (den == 0.0) continue;
    const double l = (x[1] * cp - x[0] * sp) / den;
    const double px = x[0] + l * n[0], py = x[1] + l * n[1];
    if (px * cp + py * sp > 0) emit(l, 2, k);
  }
}

// Definition: sorted crossings, each piece classified at its midpoint.
void trace_definition(const Grid& g, const double x[3], const double n_in[3], std::vector<Seg>* out) {
  out->clear();
  double n[3];
  normalise(n_in, n);
  std::vector<double> ls;
  ls.reserve(2 * (g.Nr + g.Ne + 2) + g.Na + 4);
  ls.push_back(0.0);
  all_crossings(g, x, n, [&](double l, int, int) {
    if (l > 0 && std::isfinite(l)) ls.push_back(l);
  });
  // Extra breakpoints that are not boundaries but where the polar/azimuthal
  // angle jumps: the closest approach to the origin and to the z axis. Adding a
  // breakpoint never changes the integral; it keeps every piece on one side.
  const double lo = -(x[0] * n[0] + x[1] * n[1] + x[2] * n[2]);
  if (lo > 0) ls.push_back(lo);
  const double nxy = n[0] * n[0] + n[1] * n[1];
  if (nxy > 0) {
    const double la = -(x[0] * n[0] + x[1] * n[1]) / nxy;
    if (la > 0) ls.push_back(la);
  }
  std::sort(ls.begin(), ls.end());
  for (size_t i = 0; i + 1 < ls.size(); ++i) {
    const double l0 = ls[i], l1 = ls[i + 1];
    if (!(l1 > l0)) continue;
    const double lm = 0.5 * (l0 + l1);
    const double m[3] = {x[0] + lm * n[0], x[1] + lm * n[1], x[2] + lm * n[2]};
    int ir, ie, ia;
    regions_of(g, m, &ir, &ie, &ia);
    const int64_t v = flat_index(g, ir, ie, ia);
    if (v >= 0) out->push_back({v, l1 - l0, l0});
  }
}

// Paper, steps 1-3 (Sec. 3.1-3.3, Eq. 11-13, Table 2).
struct Row {
  double l;
  int kind;    // 0 radial, 1 polar, 2 azimuthal
  int region;  // region index set by this crossing
};

void trace_paper(const Grid& g, const double x[3], const double n_in[3], std::vector<Seg>* out) {
  out->clear();
  double n[3];
  normalise(n_in, n);
  std::vector<Row> rows;
  all_crossings(g, x, n, [&](double l, int kind, int k) {
    if (!(l > 0) || !std::isfinite(l)) return;  // behind the start: never reached
    const double p[3] = {x[0] + l * n[0], x[1] + l * n[1], x[2] + l * n[2]};
    bool negative;
    if (kind == 0) {  // Eq. 11
      negative = (p[0] * n[0] + p[1] * n[1] + p[2] * n[2]) < 0;
    } else if (kind == 1) {  // Eq. 12: m = p x (-p_y, p_x, 0)
      const double m0 = -p[2] * p[0], m1 = -p[2] * p[1], m2 = p[0] * p[0] + p[1] * p[1];
      negative = (m0 * n[0] + m1 * n[1] + m2 * n[2]) > 0;
    } else {  // Eq. 13: m = p x n
      negative = (p[0] * n[1] - p[1] * n[0]) < 0;
    }
    int reg = negative ? k - 1 : k;
    if (kind == 2 && g.wrap) reg = (reg + g.Na) % g.Na;
    rows.push_back({l, kind, reg});
  });
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) { return a.l < b.l; });
  int idx[3];
  regions_of(g, x, &idx[0], &idx[1], &idx[2]);  // start voxel (Sec. 3.3)
  double lcur = 0.0;
  for (size_t i = 0; i <= rows.size(); ++i) {
    const double lnext = i < rows.size() ? rows[i].l : kInf;
    const double dl = lnext - lcur;
    const int64_t v = flat_index(g, idx[0], idx[1], idx[2]);
    if (v >= 0 && std::isfinite(dl) && dl > 0) out->push_back({v, dl});  // Table 2(c)
    if (i < rows.size()) {
      idx[rows[i].kind] = rows[i].region;  // Table 2(b): other coordinates carry over
      lcur = lnext;
    }
  }
}

// ---------------------------------------------------------------------------
// Detector models (Sec. 4.2). Cone: pinhole at pos looking at look_at; pixel
// centres uniform in tangent space over the full field of view; row 0 at +up,
// column 0 at -right. Parallel: same raster on a plane through pos, rays along
// the look direction.
// ---------------------------------------------------------------------------
void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

void view_basis(const double pos[3], const double* look_at, const double* up_hint, double look[3],
                double right[3], double up[3]) {
  double la[3] = {0, 0, 0};
  if (look_at) std::memcpy(la, look_at, sizeof la);
  double d[3] = {la[0] - pos[0], la[1] - pos[1], la[2] - pos[2]};
  normalise(d, look);
  double uh[3] = {0, 0, 1};
  if (up_hint) std::memcpy(uh, up_hint, sizeof uh);
  double rt[3];
  cross(look, uh, rt);
  double s = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
  if (s < 1e-9) {
    const double alt[3] = {0, 1, 0};
    cross(look, alt, rt);
    s = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
  }
  for (int i = 0; i < 3; ++i) right[i] = rt[i] / s;
  cross(right, look, up);
}

template <class Body>
void parallel_for(int64_t n, int threads, Body&& body) {
  if (threads <= 0) threads = int(std::max(1u, std::thread::hardware_concurrency()));
  if (n < 64) threads = 1;
  std::vector<std::thread> pool;
  const int64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    const int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([&, t, lo, hi] { body(t, lo, hi); });
  }
  for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

int oracle_threads(void) { return int(std::max(1u, std::thread::hardware_concurrency())); }

// Segment list of one ray by the definition (method 0) or the paper's steps
// (method 1). Returns the number of segments (may exceed cap; only cap written),
// or -1 for an invalid grid.
int oracle_ray_segments(const double* r, int nr1, const double* th, int ne1, const double* ph,
                        int na1, const double* x, const double* n, int method, int cap,
                        int64_t* vox, double* len) {
  Grid g;
  if (!make_grid(r, nr1, th, ne1, ph, na1, &g)) return -1;
  std::vector<Seg> segs;
  if (method == 0) trace_definition(g, x, n, &segs);
  else trace_paper(g, x, n, &segs);
  for (int i = 0; i < int(segs.size()) && i < cap; ++i) {
    vox[i] = segs[i].v;
    len[i] = segs[i].len;
  }
  return int(segs.size());
}

// Pieces of one ray by the definition (method 0), with their start distance
// along the normalised direction: vox, start l0, length. Returns the count
// (may exceed cap; only cap written), or -1 for an invalid grid.
int oracle_ray_pieces(const double* r, int nr1, const double* th, int ne1, const double* ph, int na1,
                      const double* x, const double* n, int cap, int64_t* vox, double* l0, double* len) {
  Grid g;
  if (!make_grid(r, nr1, th, ne1, ph, na1, &g)) return -1;
  std::vector<Seg> segs;
  trace_definition(g, x, n, &segs);
  for (int i = 0; i < int(segs.size()) && i < cap; ++i) {
    vox[i] = segs[i].v;
    l0[i] = segs[i].l0;
    len[i] = segs[i].len;
  }
  return int(segs.size());
}

// Forward projection y[b, i] = sum_seg rho[b, v] * len for rays given as
// (n_rays, 3) starts and directions. method as above. Returns 0 or -1.
int oracle_forward(const double* r, int nr1, const double* th, int ne1, const double* ph, int na1,
                   int64_t n_rays, const double* starts, const double* dirs, const double* rho,
                   int batch, double* y, int method, int threads) {
  Grid g;
  if (!make_grid(r, nr1, th, ne1, ph, na1, &g)) return -1;
  const int64_t V = int64_t(g.Nr) * g.Ne * g.Na;
  parallel_for(n_rays, threads, [&](int, int64_t lo, int64_t hi) {
    std::vector<Seg> segs;
    for (int64_t i = lo; i < hi; ++i) {
      if (method == 0) trace_definition(g, starts + 3 * i, dirs + 3 * i, &segs);
      else trace_paper(g, starts + 3 * i, dirs + 3 * i, &segs);
      for (int b = 0; b < batch; ++b) {
        double acc = 0.0;
        for (const Seg& s : segs) acc += rho[b * V + s.v] * s.len;
        y[b * n_rays + i] = acc;
      }
    }
  });
  return 0;
}

// Adjoint g[b, v] = sum_rays y[b, i] * |ray i in voxel v| (overwrites g).
int oracle_adjoint(const double* r, int nr1, const double* th, int ne1, const double* ph, int na1,
                   int64_t n_rays, const double* starts, const double* dirs, const double* y,
                   int batch, double* gout, int threads) {
  Grid g;
  if (!make_grid(r, nr1, th, ne1, ph, na1, &g)) return -1;
  const int64_t V = int64_t(g.Nr) * g.Ne * g.Na;
  if (threads <= 0) threads = oracle_threads();
  std::vector<std::vector<double>> part(threads);
  parallel_for(n_rays, threads, [&](int t, int64_t lo, int64_t hi) {
    std::vector<double>& acc = part[t];
    acc.assign(size_t(batch * V), 0.0);
    std::vector<Seg> segs;
    for (int64_t i = lo; i < hi; ++i) {
      trace_definition(g, starts + 3 * i, dirs + 3 * i, &segs);
      for (int b = 0; b < batch; ++b) {
        const double yi = y[b * n_rays + i];
        for (const Seg& s : segs) acc[b * V + s.v] += yi * s.len;
      }
    }
  });
  std::fill(gout, gout + batch * V, 0.0);
  for (auto& p : part)
    for (size_t j = 0; j < p.size(); ++j) gout[j] += p[j];
  return 0;
}

// Cone-beam rays (n_views * H * W, 3), row-major (view, row, col).
// look_at / up may be NULL (origin / +Z). fov in degrees, full angle.
void oracle_cone_rays(int n_views, const double* pos, const double* look_at, const double* up_hint,
                      int H, int W, double fov_h_deg, double fov_w_deg, double* starts, double* dirs) {
  const double th = std::tan(0.5 * fov_h_deg * kPi / 180.0);
  const double tw = std::tan(0.5 * fov_w_deg * kPi / 180.0);
  for (int v = 0; v < n_views; ++v) {
    double look[3], right[3], up[3];
    view_basis(pos + 3 * v, look_at ? look_at + 3 * v : nullptr, up_hint ? up_hint + 3 * v : nullptr,
               look, right, up);
    for (int i = 0; i < H; ++i) {
      const double vv = th * (1.0 - 2.0 * (i + 0.5) / H);
      for (int j = 0; j < W; ++j) {
        const double uu = tw * (2.0 * (j + 0.5) / W - 1.0);
        const int64_t k = (int64_t(v) * H + i) * W + j;
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = look[c] + uu * right[c] + vv * up[c];
        normalise(d, dirs + 3 * k);
        for (int c = 0; c < 3; ++c) starts[3 * k + c] = pos[3 * v + c];
      }
    }
  }
}

// Parallel-beam rays: detector plane through pos, extent size_h x size_w,
// all rays along the direction from pos to the origin.
void oracle_parallel_rays(int n_views, const double* pos, const double* up_hint, int H, int W,
                          double size_h, double size_w, double* starts, double* dirs) {
  for (int v = 0; v < n_views; ++v) {
    double look[3], right[3], up[3];
    view_basis(pos + 3 * v, nullptr, up_hint ? up_hint + 3 * v : nullptr, look, right, up);
    for (int i = 0; i < H; ++i) {
      const double vv = size_h * (0.5 - (i + 0.5) / H);
      for (int j = 0; j < W; ++j) {
        const double uu = size_w * ((j + 0.5) / W - 0.5);
        const int64_t k = (int64_t(v) * H + i) * W + j;
        for (int c = 0; c < 3; ++c) {
          starts[3 * k + c] = pos[3 * v + c] + uu * right[c] + vv * up[c];
          dirs[3 * k + c] = look[c];
        }
      }
    }
  }
}

// Table 2 logic on a hand-built sorted table: blank entries (INT32_MIN) are
// forward-filled from the previous row (2b); rows with an index outside
// [0, N) or a non-finite length get length 0 (2c).
void oracle_fill_zero(int n_rows, int* r, int* e, int* a, double* len, int Nr, int Ne, int Na) {
  const int blank = INT32_MIN;
  for (int i = 0; i < n_rows; ++i) {
    if (i > 0) {
      if (r[i] == blank) r[i] = r[i - 1];
      if (e[i] == blank) e[i] = e[i - 1];
      if (a[i] == blank) a[i] = a[i - 1];
    }
    const bool bad = r[i] < 0 || r[i] >= Nr || e[i] < 0 || e[i] >= Ne || a[i] < 0 || a[i] >= Na ||
                     !std::isfinite(len[i]);
    if (bad) len[i] = 0.0;
  }
}

// Crossing direction of one boundary crossing by Eq. 11 (kind 0), 12 (kind 1)
// or 13 (kind 2): returns 1 if negative.
int oracle_is_negative(int kind, const double* p, const double* n) {
  if (kind == 0) return (p[0] * n[0] + p[1] * n[1] + p[2] * n[2]) < 0;
  if (kind == 1) {
    const double m0 = -p[2] * p[0], m1 = -p[2] * p[1], m2 = p[0] * p[0] + p[1] * p[1];
    return (m0 * n[0] + m1 * n[1] + m2 * n[2]) > 0;
  }
  return (p[0] * n[1] - p[1] * n[0]) < 0;
}

}  // extern "C"
