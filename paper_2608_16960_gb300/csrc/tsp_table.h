// Host construction of a grid's boundary table (the layout tsp::TGrid reads
// from shared memory). A header of its own so that a host build of the
// traversal can use the same table.
#pragma once

#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "tsp_internal.h"

namespace tsp {

constexpr double kTablePi = 3.14159265358979323846;
constexpr double kTableTwoPi = 2.0 * kTablePi;

// Shared-memory table of a grid (layout R2 | R2L | C | S2 | S2L | K2 | K2L | PC |
// PS | PA | SEC | SEC'; the *L arrays hold the float32 rounding residue of the
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
  g->words = 2 * (Nr + 2) + 5 * (Ne + 1) + 5 * g->M;
  std::vector<float>& table = *table_out;
  table.assign(size_t(g->words), 0.0f);
  // R2 and R2L each start with an entry for k = -1 (the hole inside the
  // innermost sphere: no crossing), so that R_k^2 - b^2 needs no range test
  table[0] = -std::numeric_limits<float>::infinity();
  float* R2 = table.data() + 1;
  float* R2L = R2 + (Nr + 1) + 1;
  float* C = R2L + (Nr + 1);
  float* S2 = C + (Ne + 1);
  float* S2L = S2 + (Ne + 1);
  float* K2 = S2L + (Ne + 1);
  float* K2L = K2 + (Ne + 1);
  float* PC = K2L + (Ne + 1);
  float* PS = PC + g->M;
  float* PA = PS + g->M;
  int* SEC = reinterpret_cast<int*>(PA + g->M);
  auto split = [](double v, float* hi, float* lo) {
    *hi = float(v);
    *lo = float(v - double(*hi));
  };
  for (int k = 0; k <= Nr; ++k) split(r_edges[k] * r_edges[k], &R2[k], &R2L[k]);
  for (int k = 0; k <= Ne; ++k) {
    const double t = std::min(kTablePi, std::max(0.0, theta_edges[k]));
    const double c = std::cos(t), sn = std::sin(t);
    C[k] = float(c);
    split(sn * sn, &S2[k], &S2L[k]);
    split(c * c, &K2[k], &K2L[k]);
  }
  for (int j = 0; j < g->M; ++j) {
    PC[j] = float(std::cos(planes[j]));
    PS[j] = float(std::sin(planes[j]));
    PA[j] = float(planes[j] - planes[0]);
    SEC[j] = sec[j];
    SEC[g->M + j] = sec[j == 0 ? g->M - 1 : j - 1];  // the sector clockwise of plane j
  }
}

}  // namespace tsp
