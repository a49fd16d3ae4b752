// Per-ray traversal of a spherical grid (TomoSphero Sec. 3, steps 1-3, fused).
//
// The paper computes every crossing of a ray with every boundary (Sec. 3.1),
// turns each into a region index by its crossing direction (Sec. 3.2,
// Eq. 11-13), sorts them and forward-fills the voxel index (Sec. 3.3,
// Table 2). Along a line, r(l) and the polar angle theta(l) are unimodal and
// the azimuth phi(l) is monotone, so the sorted crossing list is a merge of at
// most five monotone runs. This routine walks that merge lazily: for each
// family (spheres, cones, half-planes) it keeps only the next crossing in the
// direction the ray is moving, chosen from the two boundaries bounding the
// current region. Each crossing sets one coordinate of the voxel index exactly
// as Eq. 11-13 + forward fill do; a segment whose index is out of range (inside
// the inner sphere, outside the outer sphere or outside a wedge) is skipped
// (Table 2c). No buffers, no sort.
//
// Parameterisation: p(t) = q + t n with n the unit direction and q the point of
// closest approach to the origin (q . n = 0, |q|^2 = b2). The start is t0 = x.n.
//   sphere k:  t = -+ sqrt(R_k^2 - b2)                          (inbound / outbound)
//   cone k (c = cos theta_k), with Q = q_z, w = Q^2 + b2 n_z^2, W = sqrt(w - c^2 b2):
//     theta decreasing through it:  t = (b2 n_z c - Q W) / (Q c + n_z W)
//     theta increasing through it:  t = (b2 n_z c + Q W) / (Q c - n_z W)
//     (the roots of the cone quadratic of refs [28],[29], each tagged with its
//      Eq. 12 direction; a non-positive denominator puts the root at infinity)
//   half-plane j at azimuth psi_j, w_j = (cos psi_j, sin psi_j): measured from
//     t_a, where the line's horizontal projection passes closest to the z axis,
//     t = t_a - (m_z / |n_xy|^2) (n_xy . w_j) / den_j,  den_j = n_xy x w_j
//     = n_x sin psi_j - n_y cos psi_j, on the half-plane iff den_j m_z < 0 where
//     m_z = (q x n)_z (Eq. 13: the azimuth grows iff m_z > 0). A plane parallel
//     to the line within rounding (den_j ~ 0) is stepped across at the start
//     if the line comes from its direction (n_xy . w_j < 0), never crossed if
//     it heads along it.
// cos(theta) along the line peaks (Q > 0) or dips (Q < 0) once, at
// t_e = b2 n_z / Q, with value sign(Q) sqrt(Q^2/b2 + n_z^2); before/after that
// point theta moves monotonically, which fixes which cone comes next.
//
// Every choice is made from the current region, so a start index that is off
// by one because the start lies within rounding of a boundary corrects itself
// at the first crossing (that crossing is then "just behind" and fires at once).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <utility>

namespace tsp {

// Explicitly rounded arithmetic: the device build uses the round-to-nearest
// intrinsics so no multiply-add is ever contracted implicitly; the host build
// (used only to check the index logic on a CPU) maps them to plain operations.
#if defined(__CUDA_ARCH__)
#define TSP_HD __host__ __device__ __forceinline__
#define T_MUL(a, b) __fmul_rn(a, b)
#define T_ADD(a, b) __fadd_rn(a, b)
#define T_SUB(a, b) __fsub_rn(a, b)
#define T_SQRT(a) __fsqrt_rn(a)
#define T_RCP(a) __frcp_rn(a)
#define T_DIV(a, b) __fdividef(a, b)
#define T_SQRTA(a) sqrt_approx_(a)
#else
#define TSP_HD __host__ __device__ inline
#define T_MUL(a, b) ((a) * (b))
#define T_ADD(a, b) ((a) + (b))
#define T_SUB(a, b) ((a) - (b))
#define T_SQRT(a) sqrtf(a)
#define T_RCP(a) (1.0f / (a))
#define T_DIV(a, b) ((a) / (b))
#define T_SQRTA(a) sqrtf(a)
#endif

#if defined(__CUDA_ARCH__)
// Hardware square root (sqrt.approx.f32, about 1 ulp) for the per-crossing
// formulas: every crossing of every ray takes one, and the correctly rounded
// square root costs several more instructions on paths that diverge within a
// warp. The once-per-ray float-float set-up keeps the rounded one (T_SQRT).
__device__ __forceinline__ float sqrt_approx_(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
#endif

// Grid tables as seen by a kernel (pointers into shared memory).
struct TGrid {
  const float2* RR; // [Nr+1] squared sphere radii (high, low): R_k^2 = x + y to ~2^-48;
                    // RR[-1] = (-inf, 0)
  const float4* CR; // [Ne+1] (cos theta_k decreasing, sin^2 and cos^2 theta_k high parts, 0);
                    // CR[-1].x = +inf, CR[Ne+1].x = -inf
  const float* S2L; // [Ne+1] low part of sin^2(theta_k)
  const float* K2L; // [Ne+1] low part of cos^2(theta_k)
  const float4* PR; // [2M] half-plane records (cos psi_j, sin psi_j, sector beyond, next record)
                    // as int bits: record j for azimuth growing (the sector
                    // counter-clockwise of plane j, then record j+1 mod M), record M + j
                    // for azimuth falling (the sector clockwise of it, then M + (j-1 mod M))
  const float* PA;  // [M] half-plane azimuth minus PA0, increasing in [0, 2 pi)
  int Nr, Ne, Na, M;
  float pa0;
};

// Device-side description of a grid's table in global memory.
struct GridDesc {
  const float* table;  // PR | CR | (-inf, 0) RR | S2L | K2L | PA (16-byte aligned)
  int Nr, Ne, Na, M;
  int words;           // table length in 32-bit words
  float pa0;
};

TSP_HD TGrid tgrid_from_smem(const GridDesc& d, const float* s) {
  TGrid g;
  g.PR = reinterpret_cast<const float4*>(s);
  g.RR = reinterpret_cast<const float2*>(s + 8 * d.M + 4 * (d.Ne + 3) + 2);
  g.CR = reinterpret_cast<const float4*>(s + 8 * d.M + 4);
  g.S2L = s + 8 * d.M + 4 * (d.Ne + 3) + 2 + 2 * (d.Nr + 1);
  g.K2L = g.S2L + (d.Ne + 1);
  g.PA = g.K2L + (d.Ne + 1);
  g.Nr = d.Nr;
  g.Ne = d.Ne;
  g.Na = d.Na;
  g.M = d.M;
  g.pa0 = d.pa0;
  return g;
}

#if defined(__CUDACC__)
// Cooperative copy of the grid table into shared memory (whole block).
__device__ __forceinline__ void load_table(const GridDesc& d, float* s) {
  for (int i = threadIdx.x; i < d.words; i += blockDim.x) s[i] = __ldg(d.table + i);
  __syncthreads();
}
#endif

// ---- classification of one point (only at the ray's first in-grid point) ----

// Radial region: number of k with R_k^2 (high part) <= r2, minus one.
TSP_HD int classify_r(const TGrid& G, float r2) {
  int lo = 0, hi = G.Nr + 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (G.RR[mid].x <= r2) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// Polar region of a point with z component pz and norm pn: number of k with
// cos(theta_k) >= pz / pn (a prefix, the table decreasing), minus one.
TSP_HD int classify_theta(const TGrid& G, float pz, float pn) {
  int lo = 0, hi = G.Ne + 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (G.CR[mid].x * pn >= pz) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// Azimuth sector of a direction (px, py): the last plane j with PA[j] <= angle.
TSP_HD int classify_sector(const TGrid& G, float px, float py) {
  const float two_pi = 6.28318530717958647692f;
  float a = atan2f(py, px) - G.pa0;
  a = a - two_pi * floorf(a * (1.0f / two_pi));
  int lo = 0, hi = G.M;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (G.PA[mid] <= a) lo = mid + 1;
    else hi = mid;
  }
  int s = lo - 1;
  return s < 0 ? G.M - 1 : s;
}

// ---- next-crossing rules per family ----

// The int stored in a float's bits (the table's integer fields).
TSP_HD int bits_i(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_int(f);
#else
  int v;
  memcpy(&v, &f, sizeof v);
  return v;
#endif
}

TSP_HD int imin_(int a, int b) { return a < b ? a : b; }

// ---- float-float (unevaluated sum hi + lo) arithmetic ----
// Error-free products and sums (Dekker; Knuth's TwoSum; FMA-based TwoProduct,
// as in Ogita, Rump and Oishi, "Accurate sum and dot product", SISC 2005).
// Used once per ray for the impact parameter and per sphere/cone crossing for
// the discriminant R^2 - b^2, whose cancellation near tangency float32 alone
// cannot resolve.
struct ff {
  float hi, lo;
};
TSP_HD ff two_prod(float a, float b) {
  const float p = T_MUL(a, b);
  return ff{p, fmaf(a, b, -p)};
}
TSP_HD ff two_sum(float a, float b) {
  const float s = T_ADD(a, b);
  const float bb = T_SUB(s, a);
  return ff{s, T_ADD(T_SUB(a, T_SUB(s, bb)), T_SUB(b, bb))};
}
TSP_HD ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, T_ADD(s.lo, T_ADD(a.lo, b.lo)));
}
TSP_HD ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
TSP_HD ff ff_mul(ff a, ff b) {
  const ff p = two_prod(a.hi, b.hi);
  return two_sum(p.hi, T_ADD(p.lo, T_ADD(T_MUL(a.hi, b.lo), T_MUL(a.lo, b.hi))));
}
TSP_HD ff ff_div(ff a, ff b) {
  const float q1 = T_DIV(a.hi, b.hi);
  const ff r = ff_add(a, ff_neg(ff_mul(ff{q1, 0.0f}, b)));
  return two_sum(q1, T_DIV(r.hi, b.hi));
}
TSP_HD ff ff_sqrt(ff a) {
  const float r = T_SQRT(a.hi);
  if (!(r > 0.0f)) return ff{0.0f, 0.0f};
  const ff r2 = two_prod(r, r);
  const float e = T_ADD(T_SUB(T_SUB(a.hi, r2.hi), r2.lo), a.lo);
  return two_sum(r, T_DIV(e, T_ADD(r, r)));
}
// a*d - b*c exactly rounded to float-float
TSP_HD ff ff_cross(float a, float d, float b, float c) { return ff_add(two_prod(a, d), ff_neg(two_prod(b, c))); }

struct RayState {
  // line
  float qx, qy, qz, nx, ny, nz, b2;
  float b2lo;          // b2 + b2lo = squared impact parameter to ~2^-46
  float b2nz;          // b2 n_z (the cone numerators)
  ff mxy2, mz2;        // |(q cross n)_xy|^2 and (q cross n)_z^2 in float-float
  // radial
  int ir, ir_next;
  bool r_out;
  float tr;
  // polar
  int ie;
  int gie;       // the cone generator's region (after the last crossing it produced)
  bool th_br2;   // the generator is past the extremum of theta
  int cn, ci;    // crossings in the cone list, index of the next one
  int cturn;     // crossings (counted from the list's first entry) before the polar direction turns
  int cdir;      // +1: the polar index rises at crossings before the turn, -1: it falls
  bool cmore;    // the list filled up: more crossings may follow
  float tgen;    // the last crossing produced (each is clamped to it)
  float th_sg, th_fe, th_te;
  float tth;
  // azimuth
  int ia;        // azimuth voxel index of the current sector (-1 outside a wedge)
  int pj;        // record of the half-plane the next azimuth crossing is on
  int psec, pnx; // its sector beyond and next record
  float nxs, nys;   // n_x, n_y times the sign of m_z (0, 0: no crossing ahead)
  float pk;      // m_z / |n_xy|^2
  float ptax;    // t_a: closest approach of the horizontal projection to the z axis
  int pstop;     // record of the half-plane the line heads along (parallel within rounding):
                 // never crossed; -1 none
  float tph;
};

// R_k^2 - b^2 from the two-part table and impact parameter (-inf for k = -1).
TSP_HD float sphere_disc(const TGrid& G, const RayState& s, int k) {
  const float2 r = G.RR[k];
  return T_ADD(T_SUB(r.x, s.b2), T_SUB(r.y, s.b2lo));
}

TSP_HD void radial_next(const TGrid& G, RayState& s) {
  if (!s.r_out) {
    const int k = s.ir;  // inner sphere of the current shell (-1 inside the innermost)
    const float dk = sphere_disc(G, s, k);
    if (dk > 0.0f) {
      s.tr = -T_SQRTA(dk);
      s.ir_next = k - 1;
      return;
    }
    s.r_out = true;  // passed the closest approach: from now on outward
  }
  // outer sphere of the current shell: k <= N_r, as the walk stops once it
  // leaves through sphere N_r
  const int k = s.ir + 1;
  s.tr = T_SQRTA(fmaxf(sphere_disc(G, s, k), 0.0f));
  s.ir_next = k;
}

// W = sqrt(b2 sin^2 theta_k - m_z^2) = sqrt(|m_xy|^2 sin^2 - m_z^2 cos^2) with
// m = q x n, the difference taken in float-float (it cancels at tangency).
TSP_HD float cone_w(const TGrid& G, const RayState& s, int k, const float4& cr) {
  // Far from tangency (the difference keeps at least a quarter of its terms'
  // magnitude) float32 already gives W to about an ulp.
  const float a0 = T_MUL(s.mxy2.hi, cr.y);
  const float b0 = T_MUL(s.mz2.hi, cr.z);
  const float w2f = T_SUB(a0, b0);
  if (w2f >= T_MUL(0.25f, T_ADD(a0, b0))) return T_SQRTA(w2f);
  const ff a = ff_mul(s.mxy2, ff{cr.y, G.S2L[k]});
  const ff b = ff_mul(s.mz2, ff{cr.z, G.K2L[k]});
  const float w2 = T_ADD(T_SUB(a.hi, b.hi), T_SUB(a.lo, b.lo));
  return T_SQRTA(fmaxf(w2, 0.0f));
}

// Cone crossings are produced ahead of the walk, up to L.cap at a time, into
// a per-ray list (shared memory on the device: entry i at t[i * stride]).
// Every lane of a warp fills its list in the same loop, so the crossing
// arithmetic runs in lockstep instead of inside the walk's divergent
// three-way step, where a lane needs a cone crossing in about one step in
// eight. Each crossing is clamped to the one before, as the walk clamps a
// next crossing to where it stands.
struct ConeList {
  float* t;
  int stride, cap;
};

// theta(t) along a line is unimodal, so the polar index moves one way until
// the extremum (phase s.th_br2 false) and the other way after it (true). The
// fill runs the phases in turn from the generator's region s.gie: the next
// cone is the region's small-theta side (k = gie) while theta decreases, its
// large-theta side (k = gie + 1) while it increases, as long as that cone is
// reached before the phase's limit on cos theta (the +-inf records end the
// run at the axis). The list keeps the direction of the phase it started in
// and the number of crossings made in it (after them the direction is
// reversed). A crossing at t = +inf ends the sequence.
TSP_HD void cone_fill(const TGrid& G, RayState& s, const ConeList& L) {
  int n = 0, n0 = 0, d0 = 0;
  float prev = s.tgen;
  bool more = true;
#pragma unroll 1
  for (int phase = 0; phase < 2; ++phase) {
    const bool dec = s.th_br2 ? (s.th_sg < 0.0f) : (s.th_sg > 0.0f);
    const float lim = s.th_br2 ? s.nz : s.th_fe;
    // the cone test c < lim (decreasing) or c > lim (increasing) as one
    // compare, and the root's signs, of the phase
    const float csg = dec ? 1.0f : -1.0f, lims = dec ? lim : -lim;
    const float qzs = dec ? -s.qz : s.qz, nzs = dec ? s.nz : -s.nz;
    const float tden = s.th_br2 ? INFINITY : -INFINITY;  // a non-positive denominator
    const int koff = dec ? 0 : 1, kstep = dec ? -1 : 1;
    if (phase == 0) d0 = kstep;
#pragma unroll 1
    for (; n < L.cap; ++n) {
      const int k = s.gie + koff;
      const float4 cr = G.CR[k];
      if (!(T_MUL(csg, cr.x) < lims)) break;
      const float c = cr.x;
      const float W = cone_w(G, s, k, cr);
      const float num = fmaf(qzs, W, T_MUL(s.b2nz, c));
      const float den = fmaf(nzs, W, T_MUL(s.qz, c));
      float t = den > 0.0f ? T_DIV(num, den) : tden;
      s.gie += kstep;
      if (!(t < INFINITY)) {
        more = false;
        break;
      }
      t = fmaxf(t, prev);
      prev = t;
      L.t[n * L.stride] = t;
    }
    if (phase == 0) n0 = n;
    if (n == L.cap || !more || s.th_br2) break;
    s.th_br2 = true;  // no more crossings before the extremum: continue past it
  }
  s.cmore = n == L.cap;
  s.cn = n;
  s.ci = 0;
  s.cturn = n0;
  s.cdir = d0;
  s.tgen = prev;
  s.tth = n > 0 ? L.t[0] : INFINITY;
}

// Crossing of half-plane pj, if the line meets it: the sign of m_z is folded
// into (nxs, nys), so den = sign(m_z) (n_xy x w_j) is negative exactly when
// the crossing is on the half-plane (Eq. 13), and nw / den equals the
// unsigned ratio (n_xy . w_j) / (n_xy x w_j) bit for bit.
TSP_HD void phi_next(const TGrid& G, RayState& s) {
  const float4 r = G.PR[s.pj];
  s.psec = bits_i(r.z);
  s.pnx = bits_i(r.w);
  const float den = fmaf(s.nxs, r.y, -T_MUL(s.nys, r.x));
  if (den < 0.0f && s.pj != s.pstop) {
    const float nw = fmaf(s.nxs, r.x, T_MUL(s.nys, r.y));
    s.tph = fmaf(-s.pk, T_DIV(nw, den), s.ptax);
  } else {
    s.tph = INFINITY;
  }
}

// Ops that define gap() are told of every piece of the ray that holds no
// voxel (inside the inner sphere, outside a wedge) between valid segments.
template <class Op, class = void>
struct op_has_gap {
  static constexpr bool value = false;
};
template <class Op>
struct op_has_gap<Op, decltype(void(std::declval<Op&>().gap()))> {
  static constexpr bool value = true;
};

// Trace one ray from start x along direction d (need not be unit); L is the
// ray's cone-crossing list (at least one entry).
// op(voxel, dl) is called for every valid segment in order along the ray
// (and op.gap() for the pieces in between that hold no voxel, if Op has it).
// Returns false if the step cap was hit (an internal inconsistency).
template <class Op>
TSP_HD bool trace_ray(const TGrid& G, const ff x[3], const ff d_in[3], Op& op, const ConeList& L) {
  const float xx = x[0].hi, xy = x[1].hi, xz = x[2].hi;
  // The direction is first scaled by a power of two that puts its largest
  // component in [0.5, 1). The scaling is exact, so every quantity below is the
  // same as without it (up to that power of two, which cancels in q and n),
  // while |d|^2 can neither overflow (float32 directions up to 3.4e38) nor lose
  // precision as a subnormal (directions down to the smallest floats).
  const float dm = fmaxf(fabsf(d_in[0].hi), fmaxf(fabsf(d_in[1].hi), fabsf(d_in[2].hi)));
  if (!(dm > 0.0f) || !(dm < INFINITY)) return true;  // zero or non-finite direction: y = 0
  ff d[3] = {d_in[0], d_in[1], d_in[2]};
  int ex = 0;
  frexpf(dm, &ex);
  for (int k = -ex; k != 0;) {  // multiply by 2^-ex in steps that stay representable
    const int step = k > 100 ? 100 : (k < -100 ? -100 : k);
    const float sc = ldexpf(1.0f, step);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = ff{T_MUL(d[i].hi, sc), T_MUL(d[i].lo, sc)};
    k -= step;
  }
  // The line arrives as float-float start and direction (exact for float32
  // inputs; carrying the rounding residue of detector-generated rays).
  // Its closest point to the origin, q = (d x (x x d)) / |d|^2, is formed in
  // float-float: accurate to ~2^-46 |x| absolute, where x - (x.n) n in float32
  // would carry an ulp of |x|. Every other quantity is then derived from
  // (q, n) alone, n the unit direction (float-float; its float32 part drives
  // the crossing formulas), so spheres, cones and half-planes all see the same
  // line: m = q x n, b^2 = |m_xy|^2 + m_z^2. Near
  // tangency R^2 - b^2 and the cone discriminant cancel; both are formed from
  // these float-float parts.
  const ff mx = ff_add(ff_mul(x[1], d[2]), ff_neg(ff_mul(x[2], d[1])));
  const ff my = ff_add(ff_mul(x[2], d[0]), ff_neg(ff_mul(x[0], d[2])));
  const ff mzf = ff_add(ff_mul(x[0], d[1]), ff_neg(ff_mul(x[1], d[0])));
  const ff D = ff_add(ff_add(ff_mul(d[0], d[0]), ff_mul(d[1], d[1])), ff_mul(d[2], d[2]));
  if (!(D.hi > 0.0f) || !(D.hi < INFINITY)) return true;  // zero or non-finite direction: y = 0
  const ff qxf = ff_div(ff_add(ff_mul(d[1], mzf), ff_neg(ff_mul(d[2], my))), D);
  const ff qyf = ff_div(ff_add(ff_mul(d[2], mx), ff_neg(ff_mul(d[0], mzf))), D);
  const ff qzf = ff_div(ff_add(ff_mul(d[0], my), ff_neg(ff_mul(d[1], mx))), D);
  RayState s;
  const ff dn = ff_sqrt(D);
  const ff nxf = ff_div(d[0], dn), nyf = ff_div(d[1], dn), nzf = ff_div(d[2], dn);  // unit to ~2^-44
  s.nx = nxf.hi;
  s.ny = nyf.hi;
  s.nz = nzf.hi;
  const ff mnx = ff_add(ff_mul(qyf, nzf), ff_neg(ff_mul(qzf, nyf)));
  const ff mny = ff_add(ff_mul(qzf, nxf), ff_neg(ff_mul(qxf, nzf)));
  const ff mnz = ff_add(ff_mul(qxf, nyf), ff_neg(ff_mul(qyf, nxf)));
  s.mxy2 = ff_add(ff_mul(mnx, mnx), ff_mul(mny, mny));
  s.mz2 = ff_mul(mnz, mnz);
  const ff b2 = ff_add(s.mxy2, s.mz2);
  s.b2 = b2.hi;
  s.b2lo = b2.lo;
  s.b2nz = T_MUL(s.b2, s.nz);
  // m_z = (q x n)_z: its sign gives the azimuth's direction along the ray (it
  // grows iff m_z > 0, Eq. 13); |m_z| / |n_xy| is the line's distance from the z axis
  const float mz = mnz.hi;
  s.qx = qxf.hi;
  s.qy = qyf.hi;
  s.qz = qzf.hi;
  const float t0 = T_ADD(T_ADD(T_MUL(xx, s.nx), T_MUL(xy, s.ny)), T_MUL(xz, s.nz));

  const float dout = sphere_disc(G, s, G.Nr);
  if (!(dout > 0.0f)) return true;  // misses the outer sphere
  const float sout = T_SQRT(dout);
  if (!(t0 < sout)) return true;     // starts beyond the grid, moving away

  float tcur;
  if (t0 <= -sout) {  // enters through the outer sphere
    tcur = -sout;
    s.ir = G.Nr - 1;
    s.r_out = false;
  } else {            // starts inside the outer sphere
    tcur = t0;
    s.ir = imin_(classify_r(G, fmaf(t0, t0, s.b2)), G.Nr - 1);
    s.r_out = t0 >= 0.0f;
  }
  const float px = fmaf(tcur, s.nx, s.qx), py = fmaf(tcur, s.ny, s.qy), pz = fmaf(tcur, s.nz, s.qz);
  const float pn = T_SQRT(fmaf(tcur, tcur, s.b2));

  // polar set-up
  s.ie = classify_theta(G, pz, pn);
  int th_mode;  // 0 walk, 1 no crossings, 2 one jump (the line passes through the origin)
  if (s.b2 == 0.0f) {              // through the origin: theta jumps there
    th_mode = tcur < 0.0f ? 2 : 1;
    if (tcur >= 0.0f) s.ie = classify_theta(G, s.nz, 1.0f);  // at or past the apex: the direction's bin
  } else if (s.qz != 0.0f) {
    th_mode = 0;
    s.th_sg = s.qz > 0.0f ? 1.0f : -1.0f;
    // |cos theta| at the extremum: sqrt(|m_xy|^2 / |m|^2)
    const float rho2 = fminf(T_DIV(s.mxy2.hi, T_ADD(s.mxy2.hi, s.mz2.hi)), 1.0f);
    s.th_fe = s.th_sg * T_SQRT(rho2);
    s.th_te = T_DIV(T_MUL(s.b2, s.nz), s.qz);
    s.th_br2 = !(tcur < s.th_te);
  } else if (s.nz != 0.0f) {       // q in the plane z = 0: cos(theta) monotone
    th_mode = 0;
    s.th_sg = s.nz > 0.0f ? 1.0f : -1.0f;
    s.th_fe = s.nz;
    s.th_te = INFINITY;
    s.th_br2 = false;
  } else {                         // horizontal line in the plane z = 0
    th_mode = 1;
  }

  // azimuth set-up
  int sec = classify_sector(G, px, py);
  int ph_mode;  // 0 walk, 1 no crossings, 2 one jump (the line meets the z axis)
  float t_ax = INFINITY;
  int sec_ax = 0;
  // Half-plane crossings are measured from t_a, where the line's horizontal
  // projection passes closest to the z axis (t_a in float-float from q and n):
  // their offsets from it, (m_z / |n_xy|^2) (n_xy . w) / (n_xy x w), keep
  // float32 relative precision however close the line passes to the axis,
  // where a crossing formed from q alone loses it to cancellation (near the
  // axis the whole azimuth sweep happens within |m_z| / |n_xy|^2 of t_a). A
  // line whose sweep is shorter than an ulp of its half-chord meets the axis
  // as far as float32 can tell: its azimuth jumps by pi there.
  const float nxy = fmaf(s.nx, s.nx, T_MUL(s.ny, s.ny));
  if (nxy > 0.0f) {
    const ff nn = ff_add(ff_mul(nxf, nxf), ff_mul(nyf, nyf));
    s.ptax = -ff_div(ff_add(ff_mul(qxf, nxf), ff_mul(qyf, nyf)), nn).hi;
    s.pk = T_DIV(mz, nn.hi);
  }
  s.pstop = -1;
  if (nxy > 0.0f && fabsf(s.pk) > T_MUL(0x1p-24f, sout)) {
    ph_mode = 0;
    // Half-planes parallel to the line within rounding of n and of the table
    // (|n_xy x w| <= 2^-21 |n_xy|) can only sit at the two ends of the sweep,
    // where their crossing test sees noise. The one the line comes from
    // (n_xy . w < 0) can only be the first plane ahead, and the line lies on
    // it there: the walk steps across it at once. The one the line heads
    // along (n_xy . w > 0) is never crossed.
    const float pde = T_MUL(0x1p-21f, T_SQRT(nxy));
    const bool ccw = mz > 0.0f;
    const int j0 = ccw ? (sec + 1 == G.M ? 0 : sec + 1) : sec;
    if (fabsf(fmaf(s.nx, G.PR[j0].y, -T_MUL(s.ny, G.PR[j0].x))) <= pde &&
        fmaf(s.nx, G.PR[j0].x, T_MUL(s.ny, G.PR[j0].y)) < 0.0f)
      sec = ccw ? j0 : (sec == 0 ? G.M - 1 : sec - 1);
    const int se = classify_sector(G, s.nx, s.ny);  // the sector of the direction of travel
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = e == 0 ? se : (se + 1 == G.M ? 0 : se + 1);
      if (fabsf(fmaf(s.nx, G.PR[j].y, -T_MUL(s.ny, G.PR[j].x))) <= pde &&
          fmaf(s.nx, G.PR[j].x, T_MUL(s.ny, G.PR[j].y)) > 0.0f)
        s.pstop = j;
    }
  } else {
    if (nxy > 0.0f) {  // the line meets the z axis: azimuth jumps by pi there
      t_ax = s.ptax;
      ph_mode = t_ax > tcur ? 2 : 1;
      sec_ax = classify_sector(G, s.nx, s.ny);
      if (t_ax <= tcur) sec = sec_ax;  // at or past the axis: the direction's azimuth
    } else {
      ph_mode = 1;  // vertical line: constant azimuth
    }
  }

  radial_next(G, s);
  s.tr = fmaxf(s.tr, tcur);
  s.gie = s.ie;
  s.tgen = tcur;
  s.cn = s.ci = 0;
  s.cturn = 0;
  s.cdir = 1;
  s.cmore = false;
  if (th_mode == 2) {  // through the origin: one list entry, the jump to the direction's bin
    L.t[0] = 0.0f;
    s.tth = 0.0f;
    s.cn = 1;
    s.cturn = L.cap;
    s.cdir = classify_theta(G, s.nz, 1.0f) - s.ie;
  } else if (th_mode == 0) {
    cone_fill(G, s, L);
  } else {
    s.tth = INFINITY;
  }
  s.ia = bits_i(G.PR[sec].z);
  if (ph_mode == 0) {
    const bool ccw = mz > 0.0f;
    s.nxs = ccw ? s.nx : -s.nx;
    s.nys = ccw ? s.ny : -s.ny;
    s.pj = ccw ? (sec + 1 == G.M ? 0 : sec + 1) : G.M + sec;
    if (s.pstop >= 0 && !ccw) s.pstop += G.M;
    phi_next(G, s);
    s.tph = fmaxf(s.tph, tcur);
  } else {  // no half-plane crossing, or the one jump to the sector of sec_ax
    s.nxs = s.nys = 0.0f;  // no crossing after it: den = 0
    s.pj = 0;
    s.psec = bits_i(G.PR[sec_ax].z);
    s.pnx = 0;
    s.tph = ph_mode == 2 ? t_ax : INFINITY;
  }

  const int cap = 2 * (G.Nr + G.Ne + 2) + G.M + 8;
#pragma unroll 1
  for (int it = 0; it < cap; ++it) {
    const float tn = fminf(s.tr, fminf(s.tth, s.tph));
    if ((unsigned)s.ir < (unsigned)G.Nr && (unsigned)s.ie < (unsigned)G.Ne && s.ia >= 0) {
      op((s.ir * G.Ne + s.ie) * G.Na + s.ia, T_SUB(tn, tcur));
    } else {
      if constexpr (op_has_gap<Op>::value) op.gap();
    }
    tcur = tn;
    if (s.tr == tn) {  // the smallest (ties go to the sphere, then the cone)
      s.ir = s.ir_next;
      if (s.ir >= G.Nr) return true;  // left through the outer sphere
      radial_next(G, s);
      s.tr = fmaxf(s.tr, tcur);
    } else if (s.tth <= s.tph) {
      s.ie += s.ci < s.cturn ? s.cdir : -s.cdir;
      if (++s.ci < s.cn) s.tth = L.t[s.ci * L.stride];
      else if (s.cmore) cone_fill(G, s, L);
      else s.tth = INFINITY;
    } else {
      s.ia = s.psec;
      s.pj = s.pnx;
      phi_next(G, s);
      s.tph = fmaxf(s.tph, tcur);
    }
  }
  return false;
}

}  // namespace tsp
