// Host construction of a grid's boundary table (the layout tsp::TGrid reads
// from shared memory). A header of its own so that a host build of the
// traversal can use the same table.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "tsp_internal.h"

namespace tsp {

constexpr double kTablePi = 3.14159265358979323846;
constexpr double kTableTwoPi = 2.0 * kTablePi;

// Shared-memory table of a grid (layout PR | CR | RR | S2L | K2L | PA; the *L arrays hold the float32 rounding residue of the
// preceding high parts, computed in double). Pure host
// arithmetic: radii squared, cosines of the polar edges, and the azimuth
// half-planes with their sector-to-voxel map. Fills the grid's dimensions.
inline void build_grid_table(const double* r_edges, int n_r_edges, const double* theta_edges,
                             int n_theta_edges, const double* phi_edges, int n_phi_edges,
                             std::vector<float>* table_out, tsp_grid_s* g) {
  const int Nr = n_r_edges - 1, Ne = n_theta_edges - 1, Na = n_phi_edges - 1;
  const double span = phi_edges[n_phi_edges - 1] - phi_edges[0];
  g->Nr = Nr;
  g->Ne = Ne;
  g->Na = Na;
  g->wrap = std::fabs(span - kTableTwoPi) <= 1e-9;
  // Azimuth half-planes: the real boundaries (N_a distinct ones when the grid
  // wraps), plus the gap sector of a wedge grid, plus virtual planes that split
  // any sector wider than pi/2 (they keep the sector's voxel index on both
  // sides), so that every sector is narrower than the half-turn a line sweeps.
  std::vector<double> planes;
  std::vector<int> sec;
  const int nreal = g->wrap ? Na : Na + 1;
  for (int k = 0; k < nreal; ++k) {
    const double a0 = phi_edges[k];
    const double a1 = (k + 1 < nreal) ? phi_edges[k + 1] : phi_edges[0] + kTableTwoPi;
    const int vox = (k < Na) ? k : -1;
    const double w = a1 - a0;
    const int pieces = std::max(1, int(std::ceil(w / (0.5 * kTablePi) - 1e-12)));
    for (int m = 0; m < pieces; ++m) {
      planes.push_back(a0 + w * m / pieces);
      sec.push_back(vox);
    }
  }
  g->M = int(planes.size());
  g->pa0 = float(planes[0]);
  const int M = g->M;
  g->words = 8 * M + 4 * (Ne + 3) + 2 * (Nr + 2) + 2 * (Ne + 1) + M;
  std::vector<float>& table = *table_out;
  table.assign(size_t(g->words), 0.0f);
  // Half-plane records first (16-byte aligned): record j < M serves a line
  // whose azimuth grows, record M + j one whose azimuth falls. Each holds
  // plane j's (cos, sin), the voxel index of the sector beyond it in that
  // direction and the record of the plane after it.
  float* PR = table.data();
  auto put_int = [](float* dst, int v) { std::memcpy(dst, &v, sizeof v); };
  for (int j = 0; j < M; ++j) {
    const float c = float(std::cos(planes[j])), sn = float(std::sin(planes[j]));
    const int jp = j + 1 == M ? 0 : j + 1, jm = j == 0 ? M - 1 : j - 1;
    float* up = PR + 4 * j;
    float* dn = PR + 4 * (M + j);
    up[0] = dn[0] = c;
    up[1] = dn[1] = sn;
    put_int(up + 2, sec[j]);
    put_int(up + 3, jp);
    put_int(dn + 2, sec[jm]);
    put_int(dn + 3, M + jm);
  }
  // Cone records (cos theta_k, sin^2 theta_k, cos^2 theta_k, 0), k = 0..N_e,
  // between records for k = -1 (cos = +inf) and k = N_e + 1 (cos = -inf) that
  // end a cone run without a range test
  float* CR = table.data() + 8 * M + 4;
  CR[-4] = std::numeric_limits<float>::infinity();
  CR[4 * (Ne + 1)] = -std::numeric_limits<float>::infinity();
  // Squared radii as (high, low) pairs, starting with a pair for k = -1 (the
  // hole inside the innermost sphere: no crossing), so that R_k^2 - b^2 needs
  // no range test
  float* RR = CR + 4 * (Ne + 2) + 2;
  RR[-2] = -std::numeric_limits<float>::infinity();
  RR[-1] = 0.0f;
  float* S2L = RR + 2 * (Nr + 1);  // low parts of sin^2 and cos^2
  float* K2L = S2L + (Ne + 1);
  float* PA = K2L + (Ne + 1);
  auto split = [](double v, float* hi, float* lo) {
    *hi = float(v);
    *lo = float(v - double(*hi));
  };
  for (int k = 0; k <= Nr; ++k) split(r_edges[k] * r_edges[k], &RR[2 * k], &RR[2 * k + 1]);
  for (int k = 0; k <= Ne; ++k) {
    const double t = std::min(kTablePi, std::max(0.0, theta_edges[k]));
    const double c = std::cos(t), sn = std::sin(t);
    CR[4 * k] = float(c);
    split(sn * sn, &CR[4 * k + 1], &S2L[k]);
    split(c * c, &CR[4 * k + 2], &K2L[k]);
  }
  for (int j = 0; j < M; ++j) PA[j] = float(planes[j] - planes[0]);
}

}  // namespace tsp
