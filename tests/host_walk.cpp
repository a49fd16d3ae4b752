// Host build of the library's per-ray walk (tsp_trace.cuh) over the library's
// own boundary table (tsp_table.h), for CPU tests of the traversal logic
// against the oracle. The host build rounds divisions and square roots
// correctly where the device uses approximate instructions, so its lengths
// are not bit-identical to the GPU's; the index logic is the same code.
#include <vector>

#include "tsp_table.h"

namespace {
struct Record {
  int* vox;
  float* len;
  int cap, n = 0;
  void operator()(int v, float dl) {
    if (n < cap) {
      vox[n] = v;
      len[n] = dl;
    }
    ++n;
  }
};
}  // namespace

// Walks n rays (float32 starts / directions, [n][3]) through the grid given
// by its edges, with a cone-crossing list of 32 entries. Ray i writes at most cap (voxel, length) pairs at i * cap and
// its full segment count to cnt[i]. Returns the number of rays that hit the
// walk's step cap (an internal inconsistency), or -1 for an empty grid.
extern "C" int host_walk_list(const double* r, int nr, const double* th, int nt, const double* ph, int np, long n,
                              const float* x, const float* d, int cap, int* vox, float* len, int* cnt, int ccap);

extern "C" int host_walk(const double* r, int nr, const double* th, int nt, const double* ph, int np, long n,
                         const float* x, const float* d, int cap, int* vox, float* len, int* cnt) {
  return host_walk_list(r, nr, th, nt, ph, np, n, x, d, cap, vox, len, cnt, 32);
}

// As host_walk, with a cone-crossing list of ccap entries (1..32): lists
// shorter than a ray's cone crossings are refilled during the walk.
extern "C" int host_walk_list(const double* r, int nr, const double* th, int nt, const double* ph, int np, long n,
                              const float* x, const float* d, int cap, int* vox, float* len, int* cnt, int ccap) {
  if (ccap < 1 || ccap > 32) return -1;
  if (nr < 2 || nt < 2 || np < 2) return -1;
  tsp_grid_s g;
  std::vector<float> table;
  tsp::build_grid_table(r, nr, th, nt, ph, np, &table, &g);
  tsp::GridDesc gd;
  gd.table = nullptr;
  gd.Nr = g.Nr;
  gd.Ne = g.Ne;
  gd.Na = g.Na;
  gd.M = g.M;
  gd.words = g.words;
  gd.pa0 = g.pa0;
  const tsp::TGrid G = tsp::tgrid_from_smem(gd, table.data());
  int bad = 0;
  for (long i = 0; i < n; ++i) {
    tsp::ff xx[3], dd[3];
    for (int c = 0; c < 3; ++c) {
      xx[c] = tsp::ff{x[3 * i + c], 0.0f};
      dd[c] = tsp::ff{d[3 * i + c], 0.0f};
    }
    Record rec{vox + i * cap, len + i * cap, cap};
    float cone_buf[32];
    if (!tsp::trace_ray(G, xx, dd, rec, tsp::ConeList{cone_buf, 1, ccap})) ++bad;
    cnt[i] = rec.n;
  }
  return bad;
}

// The boundary table of a grid as the kernels stage it in shared memory:
// copies up to cap words to out, and writes the table's length, M and the
// word offsets of its parts (half-plane records, cone records, radius pairs,
// low parts of sin^2 and cos^2, plane angles) as read through TGrid to
// info[0..7]. Returns the length in words, -1 for a grid with no cells.
extern "C" int host_table(const double* r, int nr, const double* th, int nt, const double* ph, int np, float* out,
                          int cap, int* info) {
  if (nr < 2 || nt < 2 || np < 2) return -1;
  tsp_grid_s g;
  std::vector<float> table;
  tsp::build_grid_table(r, nr, th, nt, ph, np, &table, &g);
  tsp::GridDesc gd;
  gd.table = nullptr;
  gd.Nr = g.Nr;
  gd.Ne = g.Ne;
  gd.Na = g.Na;
  gd.M = g.M;
  gd.words = g.words;
  gd.pa0 = g.pa0;
  const tsp::TGrid G = tsp::tgrid_from_smem(gd, table.data());
  const float* base = table.data();
  info[0] = g.words;
  info[1] = g.M;
  info[2] = int(reinterpret_cast<const float*>(G.PR) - base);
  info[3] = int(reinterpret_cast<const float*>(G.CR) - base);
  info[4] = int(reinterpret_cast<const float*>(G.RR) - base);
  info[5] = int(G.S2L - base);
  info[6] = int(G.K2L - base);
  info[7] = int(G.PA - base);
  for (int i = 0; i < g.words && i < cap; ++i) out[i] = table[size_t(i)];
  return g.words;
}
