// FP64-accumulating CPU oracle of the 3x3x3 spherical-grid convolution used by
// the learned warm start (test infrastructure only; shares nothing with the
// CUDA path).
//
// Layout: activations [B][Nr][Ne][Na][C] (float32 inputs), weights
// [27][Cout][Cin] with tap = (dr+1)*9 + (de+1)*3 + (da+1), offsets in {-1,0,1}.
// Boundaries: zero outside the grid in r and theta; periodic in phi when
// circular_phi != 0 (the azimuth wraps around the full circle), zero otherwise.
//   y[b,r,e,a,co] = bias[co] + sum_tap sum_ci w[tap,co,ci] x[b, r+dr, e+de, a+da, ci]
//   dgrad: gx[b,p,ci] = sum_tap sum_co w[tap,co,ci] gy[b, p - d_tap, co]   (adjoint of the above)
//   wgrad: gw[tap,co,ci] = sum_b,p gy[b,p,co] x[b, p + d_tap, ci];  gb[co] = sum gy[.,co]
//
// Threads split each loop nest so that every output element receives the same
// additions in the same order as a single thread would give it: the forward
// pass splits the output shells, dgrad the input channels, wgrad the
// (tap, output channel) pairs. Results do not depend on the thread count.
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

// Run f(lo, hi) over [0, n) split into contiguous parts, one per thread.
template <class F>
void parallel_for(int64_t n, F f) {
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(n, int64_t(std::thread::hardware_concurrency())));
  std::vector<std::thread> ts;
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
    ts.emplace_back([=] { f(lo, hi); });
  }
  for (auto& th : ts) th.join();
}

struct Shape {
  int B, Ci, Co, Nr, Ne, Na, circ;
};

// Flat voxel index of (r, e, a) + offset, or -1 outside.
inline int64_t neighbour(const Shape& s, int r, int e, int a, int dr, int de, int da) {
  const int rr = r + dr, ee = e + de;
  int aa = a + da;
  if (rr < 0 || rr >= s.Nr || ee < 0 || ee >= s.Ne) return -1;
  if (aa < 0 || aa >= s.Na) {
    if (!s.circ) return -1;
    aa = (aa + s.Na) % s.Na;
  }
  return (int64_t(rr) * s.Ne + ee) * s.Na + aa;
}

template <class T>
void conv_fwd(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const T* x, const T* w, const T* bias,
              double* y) {
  const Shape s{B, Ci, Co, Nr, Ne, Na, circ};
  const int64_t V = int64_t(Nr) * Ne * Na;
  parallel_for(int64_t(B) * Nr, [&](int64_t lo, int64_t hi) {
  for (int64_t br = lo; br < hi; ++br) {
    const int b = int(br / Nr), r = int(br % Nr);
      for (int e = 0; e < Ne; ++e)
        for (int a = 0; a < Na; ++a) {
          const int64_t p = (int64_t(r) * Ne + e) * Na + a;
          double* out = y + (b * V + p) * Co;
          for (int co = 0; co < Co; ++co) out[co] = bias ? bias[co] : 0.0;
          for (int tap = 0; tap < 27; ++tap) {
            const int64_t q = neighbour(s, r, e, a, tap / 9 - 1, (tap / 3) % 3 - 1, tap % 3 - 1);
            if (q < 0) continue;
            const T* xin = x + (b * V + q) * Ci;
            for (int co = 0; co < Co; ++co) {
              const T* wr = w + (int64_t(tap) * Co + co) * Ci;
              double acc = 0.0;
              for (int ci = 0; ci < Ci; ++ci) acc += double(wr[ci]) * double(xin[ci]);
              out[co] += acc;
            }
          }
        }
  }
  });
}

template <class T>
void conv_dgrad(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const T* gy, const T* w, double* gx) {
  const Shape s{B, Ci, Co, Nr, Ne, Na, circ};
  const int64_t V = int64_t(Nr) * Ne * Na;
  for (int64_t i = 0; i < B * V * Ci; ++i) gx[i] = 0.0;
  // scatter form of the adjoint: every (output p, tap) pair sends w^T gy to its input neighbour
  parallel_for(Ci, [&](int64_t c0, int64_t c1) {
  for (int b = 0; b < B; ++b)
    for (int r = 0; r < Nr; ++r)
      for (int e = 0; e < Ne; ++e)
        for (int a = 0; a < Na; ++a) {
          const int64_t p = (int64_t(r) * Ne + e) * Na + a;
          const T* g = gy + (b * V + p) * Co;
          for (int tap = 0; tap < 27; ++tap) {
            const int64_t q = neighbour(s, r, e, a, tap / 9 - 1, (tap / 3) % 3 - 1, tap % 3 - 1);
            if (q < 0) continue;
            double* dst = gx + (b * V + q) * Ci;
            for (int co = 0; co < Co; ++co) {
              const T* wr = w + (int64_t(tap) * Co + co) * Ci;
              for (int64_t ci = c0; ci < c1; ++ci) dst[ci] += double(wr[ci]) * double(g[co]);
            }
          }
        }
  });
}

template <class T>
void conv_wgrad(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const T* x, const T* gy, double* gw,
                double* gb) {
  const Shape s{B, Ci, Co, Nr, Ne, Na, circ};
  const int64_t V = int64_t(Nr) * Ne * Na;
  for (int i = 0; i < 27 * Co * Ci; ++i) gw[i] = 0.0;
  if (gb)
    for (int co = 0; co < Co; ++co) gb[co] = 0.0;
  // part k < 27 Co: the pair (tap, co) = (k / Co, k % Co); part 27 Co: the bias
  parallel_for(int64_t(27) * Co + 1, [&](int64_t k0, int64_t k1) {
  for (int64_t k = k0; k < k1; ++k) {
    if (k == int64_t(27) * Co) {
      if (gb)
        for (int b = 0; b < B; ++b)
          for (int64_t p = 0; p < V; ++p)
            for (int co = 0; co < Co; ++co) gb[co] += gy[(b * V + p) * Co + co];
      continue;
    }
    const int tap = int(k / Co), co = int(k % Co);
    double* dw = gw + (int64_t(tap) * Co + co) * Ci;
    for (int b = 0; b < B; ++b)
      for (int r = 0; r < Nr; ++r)
        for (int e = 0; e < Ne; ++e)
          for (int a = 0; a < Na; ++a) {
            const int64_t p = (int64_t(r) * Ne + e) * Na + a;
            const double g = double(gy[(b * V + p) * Co + co]);
            const int64_t q = neighbour(s, r, e, a, tap / 9 - 1, (tap / 3) % 3 - 1, tap % 3 - 1);
            if (q < 0) continue;
            const T* xin = x + (b * V + q) * Ci;
            for (int ci = 0; ci < Ci; ++ci) dw[ci] += g * double(xin[ci]);
          }
  }
  });
}

}  // namespace

extern "C" {

void oracle_conv3d_fwd(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const float* x, const float* w,
                       const float* bias, double* y) {
  conv_fwd(B, Ci, Co, Nr, Ne, Na, circ, x, w, bias, y);
}
void oracle_conv3d_dgrad(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const float* gy, const float* w,
                         double* gx) {
  conv_dgrad(B, Ci, Co, Nr, Ne, Na, circ, gy, w, gx);
}
void oracle_conv3d_wgrad(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const float* x, const float* gy,
                         double* gw, double* gb) {
  conv_wgrad(B, Ci, Co, Nr, Ne, Na, circ, x, gy, gw, gb);
}
void oracle_conv3d_fwd_f64(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const double* x, const double* w,
                           const double* bias, double* y) {
  conv_fwd(B, Ci, Co, Nr, Ne, Na, circ, x, w, bias, y);
}
void oracle_conv3d_dgrad_f64(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const double* gy,
                             const double* w, double* gx) {
  conv_dgrad(B, Ci, Co, Nr, Ne, Na, circ, gy, w, gx);
}
void oracle_conv3d_wgrad_f64(int B, int Ci, int Co, int Nr, int Ne, int Na, int circ, const double* x,
                             const double* gy, double* gw, double* gb) {
  conv_wgrad(B, Ci, Co, Nr, Ne, Na, circ, x, gy, gw, gb);
}

}  // extern "C"
