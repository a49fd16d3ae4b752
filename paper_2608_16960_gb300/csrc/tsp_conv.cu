// Learned warm start: a residual 3D convolutional network on the spherical grid
// (3x3x3 kernels, zero padding in r and theta, periodic in phi), bfloat16
// weights and activations, float32 accumulation, trained by its own kernels.
//
//   h1 = relu(conv(a; w1) + b1)                   1 -> 32   CUDA cores
//   h_k = h_{k-1} + relu(conv(h_{k-1}; wk) + bk)  32 -> 32  tensor cores (k = 2..5)
//   out = a + conv(h5; w6) + b6                   32 -> 1   tensor cores (forward; dgrad on CUDA cores)
//
// The 32 -> 32 layers are implicit GEMMs (M = voxels, N = 32, K = 27 taps x 32).
// Forward and dgrad run on the tcgen05 tensor cores with TMEM accumulators
// (conv32_tc_kernel): for each (r, theta) tap pair one 128-row window of a
// shared-memory slab of the neighbouring rows is the A operand and the three
// phi taps' weights side by side are B (N = 96), so one MMA computes all three
// phi taps of a window; the epilogue adds them with a one-row shift each.
// dgrad is the same kernel with the mirrored, transposed kernel. The weight
// gradient (wgrad32_tc_kernel) also runs on tcgen05: K = the voxels, M = four
// neighbouring (r, theta) rows x 32 input channels, N = 32 output channels,
// both operands MN-major, accumulated in TMEM over all of a CTA's rows.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <vector>

#include "tsp_internal.h"

struct tsp_net_s;

// Device error word of this translation unit: a tensor-core wait that gives up
// sets it (no trap); tsp_device_status reads and clears it.
static __device__ int g_conv_error_word;

namespace tsp {

static cudaError_t take_conv_error(int* out, cudaStream_t st) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_conv_error_word, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const int zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_conv_error_word, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *out |= v << 8;
  return e;
}

namespace {
struct ConvErrorRegistrar {
  ConvErrorRegistrar() { register_error_reader(&take_conv_error); }
};
ConvErrorRegistrar conv_error_registrar;

constexpr int CH = 32;

struct Dims {
  int B, Nr, Ne, Na;
  int64_t V;  // voxels per sample
};

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ int64_t nbr(const Dims& d, int r, int e, int a, int dr, int de, int da) {
  const int rr = r + dr, ee = e + de;
  if (rr < 0 || rr >= d.Nr || ee < 0 || ee >= d.Ne) return -1;
  int aa = a + da;
  aa = aa < 0 ? aa + d.Na : (aa >= d.Na ? aa - d.Na : aa);
  return (int64_t(rr) * d.Ne + ee) * d.Na + aa;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}
// 16-byte copy that reads `src_bytes` (16 or 0) bytes and zero-fills the rest
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, uint32_t src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}

// ---------------------------------------------------------------------------
// 32 -> 32 implicit GEMM on the 5th-generation tensor cores (tcgen05, TMEM).
// MODE 0 forward (bias, ReLU, residual, mask, bf16 out), MODE 1 dgrad
// (accumulate into float32 G), MODE 2 the 32 -> 1 output layer (weights in
// output channel 0, the others zero; out = a + z_0 + b into float32 G, with
// the one-channel input a passed as Y).
//
// Output positions of one shell are flattened with the two periodic halo
// columns of every theta-row, o = e * (N_a + 2) + p, p = 1..N_a the azimuth
// bins (p = 0 and N_a + 1 are computed and discarded); a "chunk" is T tiles of
// 128 consecutive positions. A shell buffer holds the theta-rows a chunk
// needs from one shell (halo columns included, zeros outside the grid),
// stored "chunk-major": the 16-byte chunk c (channels 8c..8c+7) of buffer row
// s at c * SBP * 16 + s * 16, row 0 a zero pad. In that layout the A operand
// of a tap is one 128-row window of a shell buffer, exactly the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices, 128 bytes apart
// along M, SBP * 16 apart along K), so one descriptor per (tap, K half)
// addresses it. The weights (B: N = 32 output channels x K = 27 taps x 32
// input channels) sit in the same layout, loaded once per CTA.
//
// Persistent CTAs take work items (sample, chunk, run of consecutive shells).
// Walking along r, a ring of three shell buffers holds shells r-1, r, r+1, so
// each step loads one new shell. One thread issues the step's 27 taps x T
// tiles x 2 K halves (M = 128, N = 32, K = 16, bf16 x bf16 -> f32) shell by
// shell, committing after the outgoing shell's taps so that its buffer is
// refilled with shell r+2 while the other MMAs run; accumulators alternate
// between two TMEM buffers so that every warp reads the previous step's
// (tcgen05.ld 32x32b) and runs its epilogue while the tensor cores work.
// ---------------------------------------------------------------------------
constexpr int WROWS = 27 * CH + 2;  // weight rows per chunk plane (+2: chunk planes 32 bytes off a bank period)
// Default bound of every mbarrier wait of the tensor-core kernels, in SM clock
// cycles (about one second): a kernel argument, so that a test can shorten it.
constexpr long long TC_WAIT_BUDGET = 2000000000LL;

// Tiles per chunk and shell-buffer geometry for an azimuth count (host and
// device agree). Slab columns per theta-row: the N_a bins plus the two halo
// columns, padded to a multiple of 8 so that every TMA box (8 channels x N_a
// bins of one theta-row, stored from column 1) starts on a 128-byte boundary
// of its chunk plane; the data start at buffer row TC_BASE. A 128-row tile
// yields TC_TOUT outputs (its first and last rows only feed their neighbours'
// azimuth taps), T tiles per chunk; a chunk's inputs span nrows theta-rows.
constexpr int TC_BASE = 7;
constexpr int TC_TOUT = 126;
// Epilogue: TC_ESPLIT warps per TMEM lane quarter, each with TC_ECH of the 32
// output channels; the CTA is an MMA warp, a loader warp, two idle warps and
// the epilogue warps (2 per quarter measured as fast as 4, fewer threads).
#ifndef TC_ESPLIT
#define TC_ESPLIT 2
#endif
constexpr int TC_ECH = 32 / TC_ESPLIT;
constexpr int TC_EPI_THREADS = 128 * TC_ESPLIT;
constexpr int TC_THREADS = 128 + TC_EPI_THREADS;
// Most tiles per step (2: two TMEM buffers of 192 columns, measured faster
// than 1 tile per step with five buffers of 96).
#ifndef TC_TILES
#define TC_TILES 2
#endif
struct TcPlan {
  int T, NB, colsP, nrows, SBP;  // NB: accumulator buffers of T x 96 TMEM columns (of 512)
  size_t smem;
};
__host__ __device__ inline TcPlan tc_plan(int Na) {
  TcPlan pl{1, 5, (Na + 2 + 7) / 8 * 8, 0, 0, 0};
  for (int T = TC_TILES; T >= 1; --T) {
    pl.T = T;
    pl.NB = 512 / (96 * T);
    pl.nrows = TC_TOUT * T / pl.colsP + 4;
    pl.SBP = (TC_BASE + pl.nrows * pl.colsP + 2 + 7) / 8 * 8;  // + the largest shift; planes 128-byte aligned
    pl.smem = 3 * size_t(pl.SBP) * 64 + size_t(WROWS) * 64;
    if (pl.smem <= 232448 - 1024) break;  // static shared memory: barriers, the epilogue's row exchange
  }
  return pl;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}
// Instruction descriptor, kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N = 96 (three azimuth taps x 32 output channels), M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((96u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// N consecutive accumulator columns (N = 8 or 16) of this thread's TMEM lane, no wait.
template <int N>
__device__ __forceinline__ void tmem_ld_nowait(uint32_t taddr, uint32_t (&r)[N]) {
  static_assert(N == 8 || N == 16, "8 or 16 columns");
  if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  }
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One 5-D tiled TMA box (coordinates innermost first) into shared memory,
// completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                           uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// Load shell rr of sample b, for the chunk whose first output theta-row is
// e_lo + 1, into a shell buffer (one warp): buffer row TC_BASE + j * colsP + p
// holds theta-row e_lo + j, column p (p = 1..N_a: azimuth p - 1; p = 0 and
// N_a + 1: the periodic halo, azimuths N_a - 1 and 0). Lane 0 registers the
// bytes and issues one TMA box per (theta-row, chunk plane) for columns
// 1..N_a (zeros outside the grid); all lanes copy the halo columns with
// 16-byte cp.async (zero-filled outside the grid), then arrive on `bar`.
__device__ __forceinline__ void tc_load_shell(const CUtensorMap* map, const Dims& d, const bf16* __restrict__ X, int b,
                                              int rr, int e_lo, const TcPlan& pl, unsigned char* buf, uint64_t* bar,
                                              int lane) {
  const int Na = d.Na;
  if (lane == 0) {
    mbar_expect_tx(bar, uint32_t(4 * pl.nrows * Na * 16));
    for (int j = 0; j < pl.nrows; ++j)
      for (int c = 0; c < 4; ++c)
        tma_load_5d(buf + size_t(c) * pl.SBP * 16 + size_t(TC_BASE + j * pl.colsP + 1) * 16, map, 8 * c, 0, e_lo + j,
                    rr, b, bar);
  }
  const bool shell_ok = rr >= 0 && rr < d.Nr;
  for (int i = lane; i < pl.nrows * 8; i += 32) {
    const int c = i & 3, side = (i >> 2) & 1, j = i >> 3;
    const int ee = e_lo + j;
    const bool ok = shell_ok && ee >= 0 && ee < d.Ne;
    const int aa = side == 0 ? Na - 1 : 0;
    const bf16* src = ok ? X + (((size_t(b) * d.Nr + rr) * d.Ne + ee) * Na + aa) * CH + c * 8 : X;
    cp_async16_zfill(buf + size_t(c) * pl.SBP * 16 + size_t(TC_BASE + j * pl.colsP + (side == 0 ? 0 : Na + 1)) * 16,
                     src, ok ? 16u : 0u);
  }
  cp_async_wait_all();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // halo copies -> tensor-core reads
  mbar_arrive(bar);
}

// Epilogue of one step (run by the four epilogue warps, warp w reading TMEM
// lane quarter w & 3). Tile t's accumulators sit in TMEM columns col0 + 96 t:
// row m holds, for position c_m = o0 + 126 t - 1 + m, the three azimuth-tap
// partial sums z_dai(c_m) (32 columns each). The output at c_m is
// z_0(c_m - 1) + z_1(c_m) + z_2(c_m + 1): rows m - 1 and m + 1 come from the
// neighbouring lanes by shuffle and, across a warp boundary, through `xch`.
// Rows m = 1..126 are outputs. Forward: y = x + relu(z + bias) with x the
// layer input (the residual), plus the ReLU mask; dgrad: G += z.
// TC_ESPLIT warps share each TMEM lane quarter: channel group `hf` handles
// output channels TC_ECH hf .. TC_ECH (hf + 1) - 1. The voxel of row m in tile t is vb[t] + roff
// (vb per work item, roff = r N_e N_a per radial step), if valid[t].
// Operands read back from memory (the residual x, or the gradient being
// accumulated) are fetched by tc_epilogue_fetch before the step's
// accumulators are ready, so their latency overlaps the wait.
template <int MODE>
struct EpiIn {
  uint4 x[2][TC_ECH / 8];   // forward: residual, this warp's channels of each tile's row
  float4 g[2][TC_ECH / 4];  // dgrad: G, this warp's channels of each tile's row
  float a[2];               // output layer: the network input a at each tile's row
};
template <int MODE, int T>
__device__ __forceinline__ void tc_epilogue_fetch(size_t roff, const size_t (&vb)[2], const bool (&valid)[2],
                                                  const bf16* __restrict__ Xres, const float* __restrict__ G, int hf,
                                                  EpiIn<MODE>& in) {
  const int c0 = TC_ECH * hf;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const size_t vox = valid[t] ? vb[t] + roff : 0;
    if (MODE == 0) {
      const uint4* xr = reinterpret_cast<const uint4*>(Xres + vox * CH + c0);
#pragma unroll
      for (int h = 0; h < TC_ECH / 8; ++h) in.x[t][h] = valid[t] ? xr[h] : make_uint4(0, 0, 0, 0);
    } else if (MODE == 2) {  // Xres: the one-channel input a
      in.a[t] = valid[t] && hf == 0 ? __bfloat162float(Xres[vox]) : 0.0f;
    } else {
      const float4* gp = reinterpret_cast<const float4*>(G + vox * CH + c0);
#pragma unroll
      for (int h = 0; h < TC_ECH / 4; ++h) in.g[t][h] = valid[t] ? gp[h] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}
// Empty asm through which a value passes: the compiler may not compute with
// it earlier (it would wait for the load there).
__device__ __forceinline__ void pin(uint4& v) { asm volatile("" : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)); }
__device__ __forceinline__ void pin(float4& v) { asm volatile("" : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w)); }

template <int MODE, int T>
__device__ __forceinline__ void tc_epilogue(size_t roff, const size_t (&vb)[2], const bool (&valid)[2],
                                            uint32_t tmem, uint32_t col0, EpiIn<MODE>& in, const float (&bz)[TC_ECH],
                                            bf16* __restrict__ Y, uint32_t* __restrict__ mask, float* __restrict__ G,
                                            int qd, int hf, int lane, float (*xch)[2][32]) {
  const int c0 = TC_ECH * hf;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    uint32_t r0[TC_ECH], r1[TC_ECH], r2[TC_ECH];
    const uint32_t ta = tmem + (uint32_t(32 * qd) << 16) + col0 + uint32_t(t) * 96 + uint32_t(c0);
    tmem_ld_nowait(ta, r0);
    tmem_ld_nowait(ta + 32, r1);
    tmem_ld_nowait(ta + 64, r2);
    tmem_wait();
    const size_t vox = valid[t] ? vb[t] + roff : 0;
    float (*xb)[2][32] = xch + 4 * (t & 1);  // exchange buffer of this tile (alternating)
    if (lane == 31)
#pragma unroll
      for (int j = 0; j < TC_ECH; ++j) xb[qd][0][c0 + j] = __uint_as_float(r0[j]);
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < TC_ECH; ++j) xb[qd][1][c0 + j] = __uint_as_float(r2[j]);
    asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI_THREADS) : "memory");
    // neighbours' taps: rows m-1 (columns 0..31) and m+1 (columns 64..95);
    // all shuffles first so that their latencies overlap
    float up[TC_ECH], dn[TC_ECH], acc[TC_ECH];
#pragma unroll
    for (int j = 0; j < TC_ECH; ++j) up[j] = __shfl_up_sync(0xffffffffu, __uint_as_float(r0[j]), 1);
#pragma unroll
    for (int j = 0; j < TC_ECH; ++j) dn[j] = __shfl_down_sync(0xffffffffu, __uint_as_float(r2[j]), 1);
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < TC_ECH; ++j) up[j] = qd > 0 ? xb[qd - 1][0][c0 + j] : 0.0f;
    if (lane == 31)
#pragma unroll
      for (int j = 0; j < TC_ECH; ++j) dn[j] = qd < 3 ? xb[qd + 1][1][c0 + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < TC_ECH; ++j) acc[j] = up[j] + __uint_as_float(r1[j]) + dn[j];
    if (!valid[t]) continue;
    if (MODE == 0) {
#pragma unroll
      for (int h = 0; h < TC_ECH / 8; ++h) pin(in.x[t][h]);
    } else if (MODE == 2) {
      asm volatile("" : "+f"(in.a[t]));
    } else {
#pragma unroll
      for (int h = 0; h < TC_ECH / 4; ++h) pin(in.g[t][h]);
    }
    if (MODE == 0) {
      uint32_t bits = 0;
      uint4* yo = reinterpret_cast<uint4*>(Y + vox * CH + c0);
#pragma unroll
      for (int h = 0; h < TC_ECH / 8; ++h) {
        const __nv_bfloat162* x2 = reinterpret_cast<const __nv_bfloat162*>(&in.x[t][h]);
        uint4 ov;
        __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(&ov);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int co = 8 * h + 2 * u;
          const float y0 = acc[co] + bz[co], y1 = acc[co + 1] + bz[co + 1];
          bits |= (y0 > 0.0f ? 1u : 0u) << co;
          bits |= (y1 > 0.0f ? 1u : 0u) << (co + 1);
          const float2 xf = __bfloat1622float2(x2[u]);
          o2[u] = __floats2bfloat162_rn(xf.x + fmaxf(y0, 0.0f), xf.y + fmaxf(y1, 0.0f));
        }
        yo[h] = ov;
      }
      // the mask word's 16-bit half for these channels (little-endian words)
      if (TC_ECH == 16) reinterpret_cast<uint16_t*>(mask)[2 * vox + hf] = uint16_t(bits);
      else reinterpret_cast<uint8_t*>(mask)[4 * vox + hf] = uint8_t(bits);
    } else if (MODE == 2) {  // output layer (32 -> 1, output channel 0): out = a + z_0 + b
      if (hf == 0) G[vox] = in.a[t] + (acc[0] + bz[0]);
    } else {
      float4* gp = reinterpret_cast<float4*>(G + vox * CH + c0);
#pragma unroll
      for (int h = 0; h < TC_ECH / 4; ++h) {
        float4 g = in.g[t][h];
        g.x += acc[4 * h];
        g.y += acc[4 * h + 1];
        g.z += acc[4 * h + 2];
        g.w += acc[4 * h + 3];
        gp[h] = g;
      }
    }
  }
}

// AND of `p` over the epilogue threads (named barrier 1): their decision to
// go on or give up is taken together, so none waits at the epilogue's named
// barriers for a warp that has left.
__device__ __forceinline__ bool epilogue_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, 1, %2, pi;\n selp.u32 %0, 1, 0, po;\n}"
      : "=r"(r)
      : "r"(uint32_t(p)), "n"(TC_EPI_THREADS)
      : "memory");
  return r != 0;
}

// Bounded wait on an mbarrier phase (at most `budget` SM cycles) that also
// gives up when another role of the CTA has already given up (s_abort); sets
// s_abort on its own timeout.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* s_abort, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*s_abort) return false;
    if (clock64() - t0 > budget) {
      *s_abort = 1;
      return false;
    }
  }
  return true;
}
// Warp-collective forms: the whole warp executes them (operands warp-uniform),
// one elected lane issues the MMA / the commit.
__device__ __forceinline__ void tc_mma_elect(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.u32 p, %4, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit_elect(uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(smem_u32(bar))
      : "memory");
}


template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) conv32_tc_kernel(const __grid_constant__ CUtensorMap xmap, Dims d, int rseg,
                                                           const bf16* __restrict__ X, const bf16* __restrict__ W,
                                                           const float* __restrict__ bias, bf16* __restrict__ Y,
                                                           uint32_t* __restrict__ mask, float* __restrict__ G,
                                                           long long budget, int stall_loader) {
  extern __shared__ __align__(128) unsigned char smem[];
  // full[s]: shell slot s loaded (32 loader arrivals + TMA bytes); empty[s]: its last MMA done (commit);
  // tfull[j]: TMEM buffer j holds a finished step (commit); tempty[j]: drained (one arrival per epilogue thread)
  __shared__ __align__(8) uint64_t full[3], empty[3], tfull[5], tempty[5];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ float xch[8][2][32];  // epilogue: accumulator rows that cross a warp boundary (two tiles)
  const TcPlan pl = tc_plan(d.Na);
  const int cols = pl.colsP, P = d.Ne * cols;
  const int T = pl.T, SBP = pl.SBP;
  const int NB = pl.NB;
  const uint32_t ncols = 512u;  // NB accumulator buffers of T x 96 columns
  unsigned char* s_w = smem + 3 * size_t(SBP) * 64;           // 4 chunk planes x WROWS rows x 16 B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nq = (P + TC_TOUT * T - 1) / (TC_TOUT * T), nseg = (d.Nr + rseg - 1) / rseg;
  const int items = d.B * nq * nseg;

  if (smem_u32(smem) & 127u) {  // TMA boxes need 128-byte aligned destinations: report, touch nothing
    if (tid == 0) atomicOr(&g_conv_error_word, 2);
    return;
  }
  // ---- set-up, all threads: zero the shell buffers (pad rows and padding columns stay zero), weights,
  // barriers, TMEM ----
  for (int i = tid; i < 3 * SBP * 4; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 27 * CH * 4; i += blockDim.x) {  // row = tap * 32 + output channel, K = input channel
    const int row = i >> 2, c = i & 3;
    cp_async16(s_w + size_t(c) * WROWS * 16 + row * 16, W + size_t(row) * CH + c * 8);
  }
  cp_async_wait_all();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < 3; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    for (int j = 0; j < NB; ++j) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[j])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty[j])), "n"(TC_EPI_THREADS)
                   : "memory");
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // Every role walks the same sequence: items, their steps r = r0..r1-1 (global
  // step K, TMEM buffer K mod NB) and their shell loads r0-1..r1 (global load G,
  // slot G % 3, the n-th use of a slot being phase n of its barriers).
  if (warp == 0) {  // ---- MMA issuer: the warp walks the schedule, one elected lane issues ----
    const uint32_t lbo_x = uint32_t(SBP) * 16, lbo_w = uint32_t(WROWS) * 16;
    const uint64_t wd0 = umma_desc(smem_u32(s_w), lbo_w, 128);
    int K = 0, G0 = 0, kb = 0;  // step, shell loads so far, TMEM buffer of step K
    uint32_t kph = 0;          // phase of buffer kb's barriers for step K
    bool go = true;
    for (int item = blockIdx.x; item < items && go; item += gridDim.x) {
      const int seg = item % nseg, q = (item / nseg) % nq;
      const int r0 = seg * rseg, n = min(rseg, d.Nr - r0);
      const int o0 = q * TC_TOUT * T, e_lo = (o0 - 1 + cols) / cols - 2;  // floor((o0 - 1) / cols) - 1
      for (int i = 0; i < n && go; ++i, ++K) {
        if (K >= NB && !__all_sync(0xffffffffu, tc_wait(&tempty[kb], kph ^ 1u, &s_abort, budget))) {
          go = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc0 = tmem + uint32_t(kb) * uint32_t(T) * 96;
        for (int dri = 0; dri < 3 && go; ++dri) {
          const int Gl = G0 + i + dri, slot = Gl % 3;
          if (!__all_sync(0xffffffffu, tc_wait(&full[slot], uint32_t(Gl / 3) & 1u, &s_abort, budget))) {
            go = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t xd0 = umma_desc(smem_u32(smem + size_t(slot) * SBP * 64), lbo_x, 128);
          for (int t = 0; t < T; ++t) {
            // tile rows m = 0..127 are the positions o0 + 126 t - 1 + m (input column p of each)
            const int orel = o0 + TC_TOUT * t - 1 - e_lo * cols;
#pragma unroll
            for (int dei = 0; dei < 3; ++dei) {
              const uint32_t srow = uint32_t(orel + (dei - 1) * cols + TC_BASE);
#pragma unroll
              for (int kk = 0; kk < 2; ++kk) {
                // B: the three azimuth taps (dri, dei, 0..2) x 32 output channels, contiguous rows
                const uint64_t ad = xd0 + ((srow * 16u + uint32_t(kk) * 2u * lbo_x) >> 4);
                const uint64_t bd = wd0 + ((uint32_t(dri * 9 + dei * 3) * CH * 16u + uint32_t(kk) * 2u * lbo_w) >> 4);
                tc_mma_elect(acc0 + uint32_t(t) * 96, ad, bd, (dri | dei | kk) != 0);
              }
            }
          }
          if (dri == 0 || i == n - 1) tc_commit_elect(&empty[slot]);  // this load's last use
          __syncwarp();
        }
        if (go) tc_commit_elect(&tfull[kb]);
        __syncwarp();
        if (++kb == NB) kb = 0, kph ^= 1u;
      }
      G0 += n + 2;
    }
    if (!go && lane == 0) {  // let issued MMAs land before TMEM is released
      const long long t0 = clock64();
      while (clock64() - t0 < budget / 8) {
      }
    }
    __syncwarp();
  } else if (warp == 1 && !stall_loader) {  // ---- shell loader (a test may stall it: no load at all) ----
    int G0 = 0;
    bool go = true;
    for (int item = blockIdx.x; item < items && go; item += gridDim.x) {
      const int seg = item % nseg, rest = item / nseg, q = rest % nq, b = rest / nq;
      const int r0 = seg * rseg, n = min(rseg, d.Nr - r0);
      const int e_lo = (q * TC_TOUT * T - 1 + cols) / cols - 2;
      for (int j = 0; j < n + 2; ++j) {
        const int Gl = G0 + j, slot = Gl % 3;
        if (Gl >= 3 && !__all_sync(0xffffffffu, tc_wait(&empty[slot], uint32_t(Gl / 3 - 1) & 1u, &s_abort, budget))) {
          go = false;
          break;
        }
        tc_load_shell(&xmap, d, X, b, r0 - 1 + j, e_lo, pl, smem + size_t(slot) * SBP * 64, &full[slot], lane);
      }
      G0 += n + 2;
    }
  } else if (warp >= 4) {  // ---- epilogue (TC_ESPLIT warps per TMEM lane quarter; warps 2-3 idle) ----
    const int qd = warp & 3;         // TMEM lane quarter this warp may read
    const int hf = (warp >> 2) - 1;  // channel group: TC_ECH channels from TC_ECH hf
    const int m = 32 * qd + lane;    // tile row of this thread
    const size_t plane = size_t(d.Ne) * d.Na;
    float bz[TC_ECH];
#pragma unroll
    for (int c = 0; c < TC_ECH; ++c)  // mode 2 has one bias value (output channel 0)
      bz[c] = MODE == 0 ? bias[TC_ECH * hf + c] : (MODE == 2 && hf == 0 && c == 0 ? bias[0] : 0.0f);
    int K = 0, kb = 0;
    uint32_t kph = 0;
    bool go = true;
    for (int item = blockIdx.x; item < items && go; item += gridDim.x) {
      const int seg = item % nseg, rest = item / nseg, q = rest % nq, b = rest / nq;
      const int r0 = seg * rseg, n = min(rseg, d.Nr - r0);
      // row m of tile t is position c = o0 + 126 t - 1 + m of the (theta, padded phi) plane
      size_t vb[2];
      bool vv[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int c = q * TC_TOUT * T + TC_TOUT * t - 1 + m;
        const int e = c >= 0 ? c / cols : -1, p = c - e * cols;
        vv[t] = t < T && m >= 1 && m <= TC_TOUT && c < P && p >= 1 && p <= d.Na;
        vb[t] = vv[t] ? (size_t(b) * d.Nr * d.Ne + e) * d.Na + (p - 1) : 0;
      }
      for (int i = 0; i < n; ++i, ++K) {
        const size_t roff = size_t(r0 + i) * plane;
        EpiIn<MODE> in;
        const bf16* xres = MODE == 2 ? Y : X;  // mode 2: Y carries the input a
        if (T == 2) tc_epilogue_fetch<MODE, 2>(roff, vb, vv, xres, G, hf, in);
        else tc_epilogue_fetch<MODE, 1>(roff, vb, vv, xres, G, hf, in);
        const bool ok = epilogue_and(tc_wait(&tfull[kb], kph, &s_abort, budget));
        if (!ok) {
          go = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t col0 = uint32_t(kb) * uint32_t(T) * 96;
        if (T == 2) tc_epilogue<MODE, 2>(roff, vb, vv, tmem, col0, in, bz, Y, mask, G, qd, hf, lane, xch);
        else tc_epilogue<MODE, 1>(roff, vb, vv, tmem, col0, in, bz, Y, mask, G, qd, hf, lane, xch);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&tempty[kb]);
        if (++kb == NB) kb = 0, kph ^= 1u;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && s_abort) atomicOr(&g_conv_error_word, 1);  // TSP_DEVERR_WAIT_TIMEOUT once shifted
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// 32 -> 32 weight gradient on the tcgen05 tensor cores:
//   dW[tap][co][ci] = sum_v Gz[v][co] H[v + d_tap][ci],  tap = (dr+1) 9 + (de+1) 3 + (da+1).
// One stage per output theta-row (b, r, e): the 9 neighbouring H rows
// (r + dr, e + de) as 36 chunk planes (row j = (dr+1) 3 + (de+1), chunk c:
// plane 4 j + c) of WG_PS bytes, position p at byte (WG_TB + p) 16 holding
// azimuth p - 1 (p = 0 and N_a + 1: the periodic halo), then the row's Gz as
// 4 chunk planes of N_a positions. A = H (M = 128: 4 consecutive rows x 32
// input channels, MN-major: core matrices along M one plane apart, along K
// 128 bytes apart; for MN-major the descriptor's leading offset is the K
// step and its stride offset the M / N step), B = Gz (N = 32 output channels, MN-major), K = 16
// positions per MMA; the azimuth tap shifts A's start by one position. Row
// groups start at rows 0, 4 and 5: the third covers row 8, and its blocks for
// rows 5-7 repeat the second group's and are not read back. Nine TMEM tiles
// of 32 columns (group x azimuth tap) accumulate over every row the CTA
// processes; at the end the epilogue writes the CTA's partial dW, which
// part_reduce_kernel sums in a fixed order.
// ---------------------------------------------------------------------------
constexpr int WG_TB = 7;  // position 1 of a plane starts 128-byte aligned (TMA destination)
__host__ __device__ inline int wg_ps(int Na) { return ((WG_TB + Na + 2) * 16 + 127) / 128 * 128; }
__host__ __device__ inline int wg_stage(int Na) { return 36 * wg_ps(Na) + 4 * Na * 16; }
// stages in flight (up to 3; each has its own loader warp, warps 1..3)
__host__ __device__ inline int wg_stages(int Na) {
  return 3 * wg_stage(Na) + 2048 <= 232448 ? 3 : (2 * wg_stage(Na) + 2048 <= 232448 ? 2 : 1);
}
__host__ __device__ inline int wg_gstart(int g) { return g == 0 ? 0 : (g == 1 ? 4 : 5); }
// Dynamic shared memory of a launch: the stages, at least 116 KB so that one
// CTA (which allocates all 512 TMEM columns) holds a multiprocessor.
inline int wg_smem(int Na) { return std::max(wg_stages(Na) * wg_stage(Na), 116 * 1024); }
// kind::f16: f32 accumulator, bf16 A and B, both MN-major, N = 32, M = 128.
constexpr uint32_t WG_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((32u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ void wg_mma_elect(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.u32 p, %4, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(WG_IDESC), "r"(accumulate)
      : "memory");
}

// Load the stage of output row (b, r, e) (one warp): lane 0 registers the
// bytes, the lanes issue the 40 TMA boxes (zeros outside the grid) and copy
// the 72 halo chunks with cp.async (zero-filled outside the grid), then arrive.
__device__ __forceinline__ void wg_load_stage(const CUtensorMap* hmap, const CUtensorMap* gmap, const Dims& d,
                                              const bf16* __restrict__ H, int b, int r, int e, unsigned char* buf,
                                              int PS, uint64_t* bar, int lane) {
  const int Na = d.Na;
  if (lane == 0) mbar_expect_tx(bar, uint32_t(40 * Na * 16));
  __syncwarp();
  for (int t = lane; t < 40; t += 32) {  // boxes issued from all lanes: 36 of H, 4 of Gz
    const int j = t >> 2, c = t & 3;
    if (j < 9)
      tma_load_5d(buf + size_t(t) * PS + (WG_TB + 1) * 16, hmap, 8 * c, 0, e + j % 3 - 1, r + j / 3 - 1, b, bar);
    else
      tma_load_5d(buf + size_t(36) * PS + size_t(c) * Na * 16, gmap, 8 * c, 0, e, r, b, bar);
  }
  for (int i = lane; i < 72; i += 32) {
    const int c = i & 3, side = (i >> 2) & 1, j = i >> 3;
    const int rr = r + j / 3 - 1, ee = e + j % 3 - 1;
    const bool ok = rr >= 0 && rr < d.Nr && ee >= 0 && ee < d.Ne;
    const int aa = side == 0 ? Na - 1 : 0;
    const bf16* src = ok ? H + (((size_t(b) * d.Nr + rr) * d.Ne + ee) * Na + aa) * CH + c * 8 : H;
    cp_async16_zfill(buf + size_t(4 * j + c) * PS + size_t(WG_TB + (side == 0 ? 0 : Na + 1)) * 16, src, ok ? 16u : 0u);
  }
  cp_async_wait_all();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // halo copies -> tensor-core reads
  mbar_arrive(bar);
}

// AND of p over the 128 epilogue threads of wgrad32_tc_kernel (named barrier 2).
__device__ __forceinline__ bool wg_epilogue_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, 2, 128, pi;\n selp.u32 %0, 1, 0, po;\n}"
      : "=r"(r)
      : "r"(uint32_t(p))
      : "memory");
  return r != 0;
}

// Warp 0 issues the MMAs, warps 1..NS each load one stage slot (their global
// halo copies wait in parallel), warps 4-7 read the accumulators back at the
// end. part: [gridDim.x][27][32][32].
__global__ void __launch_bounds__(256, 1) wgrad32_tc_kernel(const __grid_constant__ CUtensorMap hmap,
                                                            const __grid_constant__ CUtensorMap gmap, Dims d,
                                                            const bf16* __restrict__ H, float* __restrict__ part,
                                                            long long budget) {
  extern __shared__ __align__(128) unsigned char smem[];
  // full[s]: stage s loaded (32 loader arrivals + TMA bytes); empty[s]: its MMAs done (commit);
  // done: every MMA of the CTA done (commit)
  __shared__ __align__(8) uint64_t full[3], empty[3], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  const int Na = d.Na, PS = wg_ps(Na), ST = wg_stage(Na), NS = wg_stages(Na);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t rows = int64_t(d.B) * d.Nr * d.Ne;
  if (smem_u32(smem) & 127u) {  // TMA boxes need 128-byte aligned destinations: report, touch nothing
    if (tid == 0) atomicOr(&g_conv_error_word, 2);
    return;
  }
  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < 3; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(smem_u32(&full[k])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[k])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const bool any = int64_t(blockIdx.x) < rows;

  if (warp == 0) {  // ---- MMA issuer ----
    bool go = true;
    uint32_t started = 0;
    int i = 0;
    for (int64_t row = blockIdx.x; row < rows && go; row += gridDim.x, ++i) {
      const int slot = i % NS;
      if (!__all_sync(0xffffffffu, tc_wait(&full[slot], uint32_t(i / NS) & 1u, &s_abort, budget))) {
        go = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + size_t(slot) * ST), b0 = a0 + uint32_t(36 * PS);
      for (int g = 0; g < 3; ++g) {
        for (int dp = 0; dp < 3; ++dp) {
          const uint32_t dt = tmem + uint32_t(g * 3 + dp) * 32;
          for (int k = 0; k < Na / 16; ++k) {
            // MN-major, no swizzle: leading offset = between core matrices along K (128 bytes),
            // stride offset = between core matrices along M / N (one chunk plane)
            const uint64_t ad =
                umma_desc(a0 + uint32_t(4 * wg_gstart(g) * PS + (WG_TB + 16 * k + dp) * 16), 128, uint32_t(PS));
            const uint64_t bd = umma_desc(b0 + uint32_t(16 * k * 16), 128, uint32_t(Na * 16));
            wg_mma_elect(dt, ad, bd, started | uint32_t(k));
          }
        }
      }
      started = 1;
      tc_commit_elect(&empty[slot]);
      __syncwarp();
    }
    if (go) {
      tc_commit_elect(&done);
    } else if (lane == 0) {  // let issued MMAs land before TMEM is released
      const long long t0 = clock64();
      while (clock64() - t0 < budget / 8) {
      }
    }
    __syncwarp();
  } else if (warp >= 1 && warp <= NS) {  // ---- stage loaders: warp w fills slot w - 1 ----
    const int slot = warp - 1;
    int i = slot;
    for (int64_t row = blockIdx.x + int64_t(slot) * gridDim.x; row < rows; row += int64_t(NS) * gridDim.x, i += NS) {
      if (i >= NS && !__all_sync(0xffffffffu, tc_wait(&empty[slot], uint32_t(i / NS - 1) & 1u, &s_abort, budget))) break;
      const int e = int(row % d.Ne), r = int((row / d.Ne) % d.Nr), b = int(row / (int64_t(d.Ne) * d.Nr));
      wg_load_stage(&hmap, &gmap, d, H, b, r, e, smem + size_t(slot) * ST, PS, &full[slot], lane);
    }
  } else if (warp >= 4) {  // ---- epilogue: the CTA's partial dW ----
    const int q = warp & 3;
    float* out = part + size_t(blockIdx.x) * 27 * CH * CH;
    const bool ok = wg_epilogue_and(!any || tc_wait(&done, 0u, &s_abort, budget));
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int t = 0; t < 9; ++t) {
        const int g = t / 3, dp = t % 3;
        if (g == 2 && q < 3) continue;  // rows 5-7 again
        const int tap = 3 * (wg_gstart(g) + q) + dp;
        uint32_t v[16];
        for (int h = 0; h < 2; ++h) {  // output channels 16 h .. 16 h + 15 of input channel ci = lane
          if (any) {
            tmem_ld_nowait<16>(tmem + (uint32_t(32 * q) << 16) + uint32_t(t * 32 + 16 * h), v);
            tmem_wait();
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) out[(size_t(tap) * CH + 16 * h + j) * CH + lane] = any ? __uint_as_float(v[j]) : 0.0f;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && s_abort) atomicOr(&g_conv_error_word, 1);  // TSP_DEVERR_WAIT_TIMEOUT once shifted
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

// ---------------------------------------------------------------------------
// CUDA-core layers and element-wise pieces
// ---------------------------------------------------------------------------
__global__ void to_bf16_kernel(const float* __restrict__ x, bf16* __restrict__ y, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// Weight preparation from the float32 masters: bf16 tensors for the tensor-core
// layers (forward [tap][co][ci], dgrad [tap'][ci][co] with tap' the mirrored tap)
// and bf16-rounded float copies for the CUDA-core layers.
__global__ void prep_weights_kernel(const float* __restrict__ w, bf16* __restrict__ wf, bf16* __restrict__ wd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * CH * CH) return;
  const int tap = i / (CH * CH), co = (i / CH) % CH, ci = i % CH;
  const bf16 v = __float2bfloat16_rn(w[i]);
  wf[i] = v;
  wd[(size_t(26 - tap) * CH + ci) * CH + co] = v;
}

// Output layer weights w6 [27][32] in the 32 -> 32 layout [27][co][ci]:
// output channel 0 holds them, the other 31 are zero.
__global__ void pad_w6_kernel(const float* __restrict__ w6, bf16* __restrict__ wf6) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * CH * CH) return;
  const int tap = i / (CH * CH), co = (i / CH) % CH, ci = i % CH;
  wf6[i] = __float2bfloat16_rn(co == 0 ? w6[tap * CH + ci] : 0.0f);
}

__global__ void round_bf16_kernel(const float* __restrict__ w, float* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __bfloat162float(__float2bfloat16_rn(w[i]));
}

// h1 = relu(conv(a; w1) + b1), a has one channel.
__global__ void conv_in_fwd_kernel(Dims d, const bf16* __restrict__ a, const float* __restrict__ w1r,
                                   const float* __restrict__ b1, bf16* __restrict__ h1, uint32_t* __restrict__ mask) {
  __shared__ float sw[27 * CH];
  __shared__ float sb[CH];
  for (int i = threadIdx.x; i < 27 * CH; i += blockDim.x) sw[i] = w1r[i];
  if (threadIdx.x < CH) sb[threadIdx.x] = b1[threadIdx.x];
  __syncthreads();
  const int64_t gi = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gi >= int64_t(d.B) * d.V) return;
  const int b = int(gi / d.V);
  const int64_t v = gi - int64_t(b) * d.V;
  const int a_ = int(v % d.Na), e = int((v / d.Na) % d.Ne), r = int(v / (int64_t(d.Na) * d.Ne));
  float an[27];
#pragma unroll
  for (int tap = 0; tap < 27; ++tap) {
    const int64_t q = nbr(d, r, e, a_, tap / 9 - 1, (tap / 3) % 3 - 1, tap % 3 - 1);
    an[tap] = q < 0 ? 0.0f : __bfloat162float(a[int64_t(b) * d.V + q]);
  }
  uint32_t bits = 0;
  __nv_bfloat162 out[CH / 2];
#pragma unroll
  for (int co = 0; co < CH; co += 2) {
    float z0 = sb[co], z1 = sb[co + 1];
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) {
      z0 = fmaf(sw[tap * CH + co], an[tap], z0);
      z1 = fmaf(sw[tap * CH + co + 1], an[tap], z1);
    }
    bits |= (z0 > 0.0f ? 1u : 0u) << co;
    bits |= (z1 > 0.0f ? 1u : 0u) << (co + 1);
    out[co / 2] = __floats2bfloat162_rn(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f));
  }
  uint4* dst = reinterpret_cast<uint4*>(h1 + gi * CH);
  const uint4* src = reinterpret_cast<const uint4*>(out);
#pragma unroll
  for (int j = 0; j < 4; ++j) dst[j] = src[j];
  mask[gi] = bits;
}

// g_out = 2 (out - target) / n; shares[block] = the block's share of
// sum (out - target)^2 / n (double), summed by ordered_sum_kernel.
constexpr int MSE_BLOCKS = 152 * 8;
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ tgt, int64_t n,
                           float* __restrict__ g, double* __restrict__ shares) {
  double acc = 0.0;
  const double inv = 1.0 / double(n);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float diff = out[i] - tgt[i];
    g[i] = float(2.0 * inv * double(diff));
    acc += double(diff) * double(diff) * inv;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) shares[blockIdx.x] = v;
  }
}

// *out = sum of part[0 .. n) in a fixed order (one warp: strided lane sums,
// then a shuffle tree), so the loss repeats bit for bit.
__global__ void ordered_sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) v += part[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

// Output layer backward, input side: g_h[v][ci] = sum_tap w6[tap][ci] g_out[v - d_tap].
__global__ void conv_out_dgrad_kernel(Dims d, const float* __restrict__ gout, const float* __restrict__ w6r,
                                      float* __restrict__ gh) {
  __shared__ float sw[27 * CH];
  for (int i = threadIdx.x; i < 27 * CH; i += blockDim.x) sw[i] = w6r[i];
  __syncthreads();
  const int64_t gi = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gi >= int64_t(d.B) * d.V) return;
  const int b = int(gi / d.V);
  const int64_t v = gi - int64_t(b) * d.V;
  const int a_ = int(v % d.Na), e = int((v / d.Na) % d.Ne), r = int(v / (int64_t(d.Na) * d.Ne));
  float acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = 0.0f;
#pragma unroll 1
  for (int tap = 0; tap < 27; ++tap) {
    const int64_t q = nbr(d, r, e, a_, 1 - tap / 9, 1 - (tap / 3) % 3, 1 - tap % 3);
    if (q < 0) continue;
    const float gv = gout[int64_t(b) * d.V + q];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fmaf(sw[tap * CH + c], gv, acc[c]);
  }
  float4* dst = reinterpret_cast<float4*>(gh + gi * CH);
#pragma unroll
  for (int j = 0; j < 8; ++j) dst[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
}

// ---------------------------------------------------------------------------
// Weight gradients of the one-sided layers (one channel on one side, 32 on the
// other), in one pass over the voxels:
//   mode 0 (output layer 32 -> 1): dw[tap][c] = sum_v g1[v] X[v + d_tap][c]
//                                            = sum_u X[u][c] g1[u - d_tap],  db = sum g1
//   mode 1 (input layer 1 -> 32):  dw[tap][c] = sum_v gz[v][c] a1[v + d_tap],
//                                  gz = g_h where the pre-activation was positive, db[c] = sum gz
// Both read dw[tap][c] = sum_u P[u][c] s(u + sigma d_tap): P the 32-channel
// operand (X, or the gated g_h), s the scalar field (g1, or a1), sigma = -1 / +1.
// A CTA stages a tile of ET theta-rows of P (float) and the 3 x (ET + 2) rows
// of s around it in shared memory; 16 groups of 16 threads (one channel pair
// each) walk runs along phi with the 3 x 3 x 3 window of s in registers
// (27 taps x 2 channels of partial sums per thread). Each CTA writes its sums
// to its row of `part` (THIN_OUT floats: 27 x 32 weights, then 32 biases);
// part_reduce_kernel adds the rows in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int THIN_OUT = 27 * CH + CH;

// theta-rows per tile: the largest power of two <= 16 with ET N_a <= 384
inline int thin_et(int Na) {
  int et = 1;
  while (et < 16 && 2 * et * Na <= 384) et *= 2;
  return et;
}
inline size_t thin_smem(int Na) {
  const int et = thin_et(Na);
  return size_t(et) * Na * CH * sizeof(float) + size_t(3) * (et + 2) * Na * sizeof(float);
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) thin_wgrad_kernel(Dims d, int ET, const float* __restrict__ g1,
                                                            const bf16* __restrict__ X32, const float* __restrict__ gh,
                                                            const uint32_t* __restrict__ mask,
                                                            const bf16* __restrict__ a1, float* __restrict__ part) {
  extern __shared__ __align__(16) float thin_sm[];
  __shared__ float red[8][THIN_OUT];
  const int Na = d.Na, ETS = ET + 2;
  float* sP = thin_sm;                      // [ET * Na][32]
  float* sS = thin_sm + size_t(ET) * Na * CH;  // [3][ET + 2][Na]
  const int tid = threadIdx.x, g = tid >> 4, cp = tid & 15;
  const int runs = 16 / ET, el = g / runs, ri = g % runs;
  const int L = (Na + runs - 1) / runs, a_s = ri * L, a_e = min(Na, a_s + L);
  float acc[27][2], bacc[2] = {0.0f, 0.0f};
#pragma unroll
  for (int t = 0; t < 27; ++t) acc[t][0] = acc[t][1] = 0.0f;
  const int nET = (d.Ne + ET - 1) / ET;
  const int64_t tiles = int64_t(d.B) * d.Nr * nET;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int e0 = int(tile % nET) * ET, r = int((tile / nET) % d.Nr), b = int(tile / (int64_t(nET) * d.Nr));
    const int ETe = min(ET, d.Ne - e0);
    const int64_t v0 = ((int64_t(b) * d.Nr + r) * d.Ne + e0) * Na;  // first voxel of the tile (rows are contiguous)
    __syncthreads();  // the previous tile is no longer read
    for (int i = tid; i < ETe * Na * 8; i += 256) {
      const int vi = i >> 3, h = i & 7;
      float4 f;
      if (MODE == 1) {
        f = *reinterpret_cast<const float4*>(gh + (v0 + vi) * CH + 4 * h);
        const uint32_t m = mask[v0 + vi] >> (4 * h);
        f.x = (m & 1u) ? f.x : 0.0f;
        f.y = (m & 2u) ? f.y : 0.0f;
        f.z = (m & 4u) ? f.z : 0.0f;
        f.w = (m & 8u) ? f.w : 0.0f;
      } else {
        const uint2 u = *reinterpret_cast<const uint2*>(X32 + (v0 + vi) * CH + 4 * h);
        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        f = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
      reinterpret_cast<float4*>(sP)[i] = f;
    }
    for (int i = tid; i < 3 * ETS * Na; i += 256) {
      const int a_ = i % Na, ee = (i / Na) % ETS, rr = i / (Na * ETS);
      const int rg = r - 1 + rr, eg = e0 - 1 + ee;
      float v = 0.0f;
      if (rg >= 0 && rg < d.Nr && eg >= 0 && eg < d.Ne) {
        const int64_t q = int64_t(b) * d.V + (int64_t(rg) * d.Ne + eg) * Na + a_;
        v = MODE == 1 ? __bfloat162float(a1[q]) : g1[q];
      }
      sS[i] = v;
    }
    __syncthreads();
    if (el >= ETe || a_s >= a_e) continue;
    // window w[or][oe][k]: s at (r + or - 1, e + oe - 1, a + k - 1)
    float w[3][3][3];
    const float* srow = sS + size_t(el + 1) * Na;  // (rr, ee) row = srow + ((rr - 1) * ETS + ee - 1) * Na ...
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int ak = a_s - 1 + k;
      ak = ak < 0 ? ak + Na : (ak >= Na ? ak - Na : ak);
#pragma unroll
      for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int oe = 0; oe < 3; ++oe) w[o][oe][k] = srow[(o * ETS + oe - 1) * Na + ak];
    }
    const float* pp = sP + (size_t(el) * Na) * CH + 2 * cp;
    for (int a_ = a_s; a_ < a_e; ++a_) {
      const float2 p = *reinterpret_cast<const float2*>(pp + size_t(a_) * CH);
#pragma unroll
      for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int oe = 0; oe < 3; ++oe)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            // mode 1: the window offset is d_tap; mode 0: it is -d_tap
            const int tap = MODE == 1 ? o * 9 + oe * 3 + k : (2 - o) * 9 + (2 - oe) * 3 + (2 - k);
            acc[tap][0] = fmaf(p.x, w[o][oe][k], acc[tap][0]);
            acc[tap][1] = fmaf(p.y, w[o][oe][k], acc[tap][1]);
          }
      if (MODE == 1) {
        bacc[0] += p.x;
        bacc[1] += p.y;
      } else if (cp == 0) {
        bacc[0] += w[1][1][1];  // g1 of this voxel
      }
      int an = a_ + 2;
      an = an >= Na ? an - Na : an;
      an = an >= Na ? an - Na : an;
#pragma unroll
      for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int oe = 0; oe < 3; ++oe) {
          w[o][oe][0] = w[o][oe][1];
          w[o][oe][1] = w[o][oe][2];
          w[o][oe][2] = srow[(o * ETS + oe - 1) * Na + an];
        }
    }
  }
  // groups 2w and 2w + 1 share warp w: fold them, then the 8 warps in order
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int t = 0; t < 27; ++t)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float v = acc[t][j] + __shfl_xor_sync(0xffffffffu, acc[t][j], 16);
      if (lane < 16) red[warp][t * CH + 2 * cp + j] = v;
    }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float v = bacc[j] + __shfl_xor_sync(0xffffffffu, bacc[j], 16);
    if (lane < 16) red[warp][27 * CH + 2 * cp + j] = v;
  }
  __syncthreads();
  for (int i = tid; i < THIN_OUT; i += 256) {
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += red[k][i];
    part[size_t(blockIdx.x) * THIN_OUT + i] = sum;
  }
}

// out[i] += sum_k part[k][i] for i < n (rows of `stride` floats), k in order:
// 32 outputs per CTA, warp w takes rows w, w + 32, ...
__global__ void __launch_bounds__(1024) part_reduce_kernel(const float* __restrict__ part, int rows, int stride, int n,
                                                           float* __restrict__ out) {
  __shared__ float s[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float v = 0.0f;
  if (i < n)
    for (int k = warp; k < rows; k += 32) v += part[size_t(k) * stride + i];
  s[warp][lane] = v;
  __syncthreads();
  if (warp == 0 && i < n) {
    float t = 0.0f;
    for (int w = 0; w < 32; ++w) t += s[w][lane];
    out[i] += t;
  }
}

// g_z = bf16(g_h where the forward pre-activation was positive, else 0), 8
// channels per thread; each CTA also writes its column sums of g_z (the bias
// gradient, summed over the bf16 values) to its row of `part` (32 floats).
__global__ void __launch_bounds__(256) gate_kernel(const float* __restrict__ gh, const uint32_t* __restrict__ mask,
                                                   bf16* __restrict__ gz, int64_t nvox, float* __restrict__ part) {
  const int q = threadIdx.x & 3;  // channels 8q .. 8q + 7
  float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t v = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 2; v < nvox;
       v += (int64_t(gridDim.x) * blockDim.x) >> 2) {
    const float4 f0 = *reinterpret_cast<const float4*>(gh + v * CH + 8 * q);
    const float4 f1 = *reinterpret_cast<const float4*>(gh + v * CH + 8 * q + 4);
    const uint32_t m = mask[v] >> (8 * q);
    const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
    uint4 o;
    __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const __nv_bfloat162 z = __floats2bfloat162_rn((m >> (2 * u)) & 1u ? f[2 * u] : 0.0f,
                                                     (m >> (2 * u + 1)) & 1u ? f[2 * u + 1] : 0.0f);
      o2[u] = z;
      const float2 zf = __bfloat1622float2(z);
      cs[2 * u] += zf.x;
      cs[2 * u + 1] += zf.y;
    }
    *reinterpret_cast<uint4*>(gz + v * CH + 8 * q) = o;
  }
  // fold the 8 threads of each channel group in a warp, then the 8 warps in order
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float t = cs[c];
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 8);
    t += __shfl_xor_sync(0xffffffffu, t, 16);
    if (lane < 4) red[warp][8 * lane + c] = t;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[size_t(blockIdx.x) * CH + threadIdx.x] = t;
  }
}

int blocks_for(int64_t n, int threads) { return int(std::min<int64_t>((n + threads - 1) / threads, 1 << 30)); }

}  // namespace
}  // namespace tsp

using namespace tsp;

// Parameter layout (float32, flat): w1 [27][32][1], b1 [32], w2..w5 [27][32][32],
// b2..b5 [32], w6 [27][1][32], b6 [1].
struct tsp_net_s {
  Dims d{};
  int max_batch = 0;
  int device = 0;
  size_t n_params = 0;
  size_t off_w[6], off_b[6];
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wf[4] = {nullptr, nullptr, nullptr, nullptr}, *wd[4] = {nullptr, nullptr, nullptr, nullptr};
  float *w1r = nullptr, *w6r = nullptr;
  bf16* wf6 = nullptr;  // output layer weights in the 32 -> 32 layout (tensor-core forward)
  bf16* a16 = nullptr;
  bf16* h[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  uint32_t* mask[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  float *out = nullptr, *gout = nullptr, *gh = nullptr;
  bf16* gz = nullptr;
  double* loss = nullptr;
  double* loss_part = nullptr;  // per-block shares of the loss
  float* part = nullptr;  // per-CTA partial sums of the weight / bias gradient reductions
  int part_rows = 0;
  float* wpart = nullptr;  // per-CTA partial 32 -> 32 weight gradients [SMs][27][32][32]
  std::vector<void*> allocs;
  int adam_step = 0;
  bool prepared = false;  // wf / wd / w1r / w6r / wf6 hold the current parameters
  CUtensorMap map_h[5];  // TMA descriptors of the activations h1..h5 (inputs of the 32 -> 32 layers)
  CUtensorMap map_gz;    // and of the gated gradient (input of dgrad)
};

namespace {


// TMA descriptor of a bf16 activation tensor [B][N_r][N_e][N_a][32]: a 5-D
// tiled map (channels innermost) whose box is 8 channels x N_a azimuths, i.e.
// one 16-byte chunk of every voxel of a theta-row; out-of-range theta-rows and
// shells read as zeros.
tsp_status encode_act_map(CUtensorMap* m, const bf16* base, const Dims& d) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    TSP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(TSP_ECUDA, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[5] = {cuuint64_t(CH), cuuint64_t(d.Na), cuuint64_t(d.Ne), cuuint64_t(d.Nr), cuuint64_t(d.B)};
  const cuuint64_t strides[4] = {cuuint64_t(CH) * 2, cuuint64_t(CH) * 2 * d.Na, cuuint64_t(CH) * 2 * d.Na * d.Ne,
                                 cuuint64_t(CH) * 2 * d.Na * d.Ne * d.Nr};
  const cuuint32_t box[5] = {8u, cuuint32_t(d.Na), 1u, 1u, 1u};
  const cuuint32_t es[5] = {1u, 1u, 1u, 1u, 1u};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(base), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TSP_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
  return TSP_OK;
}

template <class T>
tsp_status net_alloc(tsp_net n, T** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
  if (e != cudaSuccess) return cuda_fail(e, "tsp_net_create: allocation");
  n->allocs.push_back(*p);
  return TSP_OK;
}

int g_sm_count = 152;  // multiprocessors of the device the network lives on (set at creation)

// Allow f the most dynamic shared memory a block may have on this device
// (the opt-in limit less f's static shared memory). The attribute belongs to
// the function, not to a net, so it is set to the largest value once instead
// of to one net's need (nets of several azimuth counts may coexist).
template <class F>
tsp_status allow_max_smem(F* f, int dev) {
  int optin = 0;
  TSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  TSP_CUDA(cudaFuncGetAttributes(&fa, f));
  TSP_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes)));
  return TSP_OK;
}

tsp_status set_attrs(int Na) {
  int dev = 0;
  TSP_CUDA(cudaGetDevice(&dev));
  TSP_CUDA(cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev));
  int optin = 0;
  TSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (int(tc_plan(Na).smem) + 4096 > optin || wg_smem(Na) + 4096 > optin || int(thin_smem(Na)) + 32768 > optin)
    return fail(TSP_ENOTSUP, "tsp_net_create: the azimuth count needs more shared memory than a block may have");
  tsp_status st = allow_max_smem(conv32_tc_kernel<0>, dev);
  if (st == TSP_OK) st = allow_max_smem(conv32_tc_kernel<1>, dev);
  if (st == TSP_OK) st = allow_max_smem(conv32_tc_kernel<2>, dev);
  if (st == TSP_OK) st = allow_max_smem(wgrad32_tc_kernel, dev);
  if (st == TSP_OK) st = allow_max_smem(thin_wgrad_kernel<0>, dev);
  if (st == TSP_OK) st = allow_max_smem(thin_wgrad_kernel<1>, dev);
  return st;
}

// Armed by tsp_debug_tc_stall: the wait budget (cycles) of the next
// tensor-core convolution launch, whose loader then stalls; 0 = not armed.
std::atomic<long long> g_tc_stall{0};

// Persistent launch: work items (sample, chunk, run of rseg shells), about
// four per multiprocessor, one CTA per multiprocessor (its shared memory).
void conv32(int mode, const Dims& d, int B, const CUtensorMap& xmap, const bf16* X, const bf16* W, const float* bias,
            bf16* Y, uint32_t* mask, float* G, cudaStream_t st) {
  Dims db = d;
  db.B = B;
  const TcPlan pl = tc_plan(d.Na);
  const int P = d.Ne * (d.Na + 2);
  const int nq = (P + TC_TOUT * pl.T - 1) / (TC_TOUT * pl.T);
  const int64_t steps = int64_t(B) * nq * d.Nr;
  const int rseg = int(std::max<int64_t>(2, std::min<int64_t>(d.Nr, steps / (4 * int64_t(g_sm_count)))));
  const int64_t items = int64_t(B) * nq * ((d.Nr + rseg - 1) / rseg);
  const unsigned grid = unsigned(std::min<int64_t>(items, g_sm_count));
  // the one-shot test hook of tsp_debug_tc_stall: this launch's loader issues
  // nothing and its waits give up after the armed number of cycles
  const long long armed = g_tc_stall.exchange(0);
  const long long budget = armed > 0 ? armed : TC_WAIT_BUDGET;
  const int stall = armed > 0 ? 1 : 0;
  if (mode == 0)
    conv32_tc_kernel<0><<<grid, TC_THREADS, pl.smem, st>>>(xmap, db, rseg, X, W, bias, Y, mask, G, budget, stall);
  else if (mode == 1)
    conv32_tc_kernel<1><<<grid, TC_THREADS, pl.smem, st>>>(xmap, db, rseg, X, W, bias, Y, mask, G, budget, stall);
  else conv32_tc_kernel<2><<<grid, TC_THREADS, pl.smem, st>>>(xmap, db, rseg, X, W, bias, Y, mask, G, budget, stall);
}

tsp_status prepare_weights(tsp_net n, cudaStream_t st) {
  for (int k = 0; k < 4; ++k)
    prep_weights_kernel<<<(27 * CH * CH + 255) / 256, 256, 0, st>>>(n->params + n->off_w[k + 1], n->wf[k], n->wd[k]);
  round_bf16_kernel<<<(27 * CH + 255) / 256, 256, 0, st>>>(n->params + n->off_w[0], n->w1r, 27 * CH);
  round_bf16_kernel<<<(27 * CH + 255) / 256, 256, 0, st>>>(n->params + n->off_w[5], n->w6r, 27 * CH);
  pad_w6_kernel<<<(27 * CH * CH + 255) / 256, 256, 0, st>>>(n->params + n->off_w[5], n->wf6);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

tsp_status net_forward(tsp_net n, const float* a, int B, cudaStream_t st) {
  const Dims& d = n->d;
  Dims db = d;
  db.B = B;
  const int64_t nv = int64_t(B) * d.V;
  if (!n->prepared) {  // the bf16 / rounded copies, refreshed only after the parameters change
    tsp_status s = prepare_weights(n, st);
    if (s != TSP_OK) return s;
    n->prepared = true;
  }
  to_bf16_kernel<<<blocks_for(nv, 256), 256, 0, st>>>(a, n->a16, nv);
  conv_in_fwd_kernel<<<blocks_for(nv, 128), 128, 0, st>>>(db, n->a16, n->w1r, n->params + n->off_b[0], n->h[0],
                                                          n->mask[0]);
  for (int k = 0; k < 4; ++k)
    conv32(0, d, B, n->map_h[k], n->h[k], n->wf[k], n->params + n->off_b[k + 1], n->h[k + 1], n->mask[k + 1], nullptr,
           st);
  conv32(2, d, B, n->map_h[4], n->h[4], n->wf6, n->params + n->off_b[5], n->a16, nullptr, n->out, st);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

}  // namespace

extern "C" tsp_status tsp_net_create(int n_r, int n_e, int n_a, int max_batch, tsp_net* out) {
  if (!out) return fail(TSP_EINVAL, "tsp_net_create: out is NULL");
  *out = nullptr;
  if (n_r <= 0 || n_e <= 0 || max_batch <= 0) return fail(TSP_EINVAL, "tsp_net_create: bad size");
  if (n_a % 32 != 0 || n_a < 32 || n_a > 192)
    return fail(TSP_ENOTSUP, "tsp_net_create: the azimuth count must be a multiple of 32 in [32, 192]");
  tsp_net n = new (std::nothrow) tsp_net_s();
  if (!n) return fail(TSP_ENOMEM, "tsp_net_create: host allocation");
  n->d = Dims{max_batch, n_r, n_e, n_a, int64_t(n_r) * n_e * n_a};
  n->max_batch = max_batch;
  cudaGetDevice(&n->device);
  size_t off = 0;
  const size_t wsz[6] = {27 * CH, 27 * CH * CH, 27 * CH * CH, 27 * CH * CH, 27 * CH * CH, 27 * CH};
  const size_t bsz[6] = {CH, CH, CH, CH, CH, 1};
  for (int k = 0; k < 6; ++k) {
    n->off_w[k] = off;
    off += wsz[k];
    n->off_b[k] = off;
    off += bsz[k];
  }
  n->n_params = off;
  const int64_t nv = int64_t(max_batch) * n->d.V;
  tsp_status st = TSP_OK;
  if (st == TSP_OK) st = net_alloc(n, &n->params, off);
  if (st == TSP_OK) st = net_alloc(n, &n->grads, off);
  if (st == TSP_OK) st = net_alloc(n, &n->m, off);
  if (st == TSP_OK) st = net_alloc(n, &n->v, off);
  for (int k = 0; k < 4 && st == TSP_OK; ++k) {
    st = net_alloc(n, &n->wf[k], 27 * CH * CH);
    if (st == TSP_OK) st = net_alloc(n, &n->wd[k], 27 * CH * CH);
  }
  if (st == TSP_OK) st = net_alloc(n, &n->w1r, 27 * CH);
  if (st == TSP_OK) st = net_alloc(n, &n->w6r, 27 * CH);
  if (st == TSP_OK) st = net_alloc(n, &n->wf6, 27 * CH * CH);
  if (st == TSP_OK) st = net_alloc(n, &n->a16, nv);
  for (int k = 0; k < 5 && st == TSP_OK; ++k) {
    st = net_alloc(n, &n->h[k], nv * CH);
    if (st == TSP_OK) st = net_alloc(n, &n->mask[k], nv);
  }
  if (st == TSP_OK) st = net_alloc(n, &n->out, nv);
  if (st == TSP_OK) st = net_alloc(n, &n->gout, nv);
  if (st == TSP_OK) st = net_alloc(n, &n->gh, nv * CH);
  if (st == TSP_OK) st = net_alloc(n, &n->gz, nv * CH);
  if (st == TSP_OK) st = net_alloc(n, &n->loss, 1);
  if (st == TSP_OK) st = net_alloc(n, &n->loss_part, MSE_BLOCKS);
  if (st == TSP_OK) st = set_attrs(n_a);
  if (st == TSP_OK) {  // one row per CTA of the reductions (2 per multiprocessor, THIN_OUT floats)
    n->part_rows = 2 * g_sm_count;
    st = net_alloc(n, &n->part, size_t(n->part_rows) * THIN_OUT);
    if (st == TSP_OK) st = net_alloc(n, &n->wpart, size_t(g_sm_count) * 27 * CH * CH);
  }
  for (int k = 0; k < 5 && st == TSP_OK; ++k) st = encode_act_map(&n->map_h[k], n->h[k], n->d);
  if (st == TSP_OK) st = encode_act_map(&n->map_gz, n->gz, n->d);
  if (st == TSP_OK) {
    cudaError_t e = cudaMemset(n->params, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * off);
    if (e != cudaSuccess) st = cuda_fail(e, "tsp_net_create: clear");
  }
  if (st != TSP_OK) {
    tsp_net_destroy(n);
    return st;
  }
  *out = n;
  return TSP_OK;
}

extern "C" void tsp_net_destroy(tsp_net n) {
  if (!n) return;
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

extern "C" tsp_status tsp_debug_tc_stall(int64_t wait_cycles) {
  if (wait_cycles <= 0 || wait_cycles > TC_WAIT_BUDGET)
    return fail(TSP_EINVAL, "tsp_debug_tc_stall: wait_cycles must be in 1 .. " + std::to_string(TC_WAIT_BUDGET));
  g_tc_stall.store((long long)wait_cycles);
  return TSP_OK;
}

extern "C" tsp_status tsp_net_num_params(tsp_net n, size_t* count) {
  if (!n || !count) return fail(TSP_EINVAL, "tsp_net_num_params: NULL argument");
  *count = n->n_params;
  return TSP_OK;
}

extern "C" tsp_status tsp_net_set_params(tsp_net n, const float* host, size_t count) {
  if (!n || !host || count != n->n_params) return fail(TSP_EINVAL, "tsp_net_set_params: bad argument");
  TSP_CUDA(cudaMemcpy(n->params, host, sizeof(float) * count, cudaMemcpyHostToDevice));
  TSP_CUDA(cudaMemset(n->m, 0, sizeof(float) * count));
  TSP_CUDA(cudaMemset(n->v, 0, sizeof(float) * count));
  n->adam_step = 0;
  n->prepared = false;
  return TSP_OK;
}

extern "C" tsp_status tsp_net_get_params(tsp_net n, float* host, size_t count) {
  if (!n || !host || count != n->n_params) return fail(TSP_EINVAL, "tsp_net_get_params: bad argument");
  TSP_CUDA(cudaMemcpy(host, n->params, sizeof(float) * count, cudaMemcpyDeviceToHost));
  return TSP_OK;
}

extern "C" tsp_status tsp_net_get_state(tsp_net n, float* params, float* m, float* v, size_t count,
                                        int* adam_step) {
  if (!n || !params || !m || !v || !adam_step || count != n->n_params)
    return fail(TSP_EINVAL, "tsp_net_get_state: bad argument");
  tsp_status st = check_device(n->device);
  if (st != TSP_OK) return st;
  TSP_CUDA(cudaDeviceSynchronize());  // Adam steps enqueued on any stream have landed
  TSP_CUDA(cudaMemcpy(params, n->params, sizeof(float) * count, cudaMemcpyDeviceToHost));
  TSP_CUDA(cudaMemcpy(m, n->m, sizeof(float) * count, cudaMemcpyDeviceToHost));
  TSP_CUDA(cudaMemcpy(v, n->v, sizeof(float) * count, cudaMemcpyDeviceToHost));
  *adam_step = n->adam_step;
  return TSP_OK;
}

extern "C" tsp_status tsp_net_set_state(tsp_net n, const float* params, const float* m, const float* v,
                                        size_t count, int adam_step) {
  if (!n || !params || !m || !v || count != n->n_params || adam_step < 0)
    return fail(TSP_EINVAL, "tsp_net_set_state: bad argument");
  tsp_status st = check_device(n->device);
  if (st != TSP_OK) return st;
  TSP_CUDA(cudaDeviceSynchronize());  // no kernel of an earlier call still reads the old state
  TSP_CUDA(cudaMemcpy(n->params, params, sizeof(float) * count, cudaMemcpyHostToDevice));
  TSP_CUDA(cudaMemcpy(n->m, m, sizeof(float) * count, cudaMemcpyHostToDevice));
  TSP_CUDA(cudaMemcpy(n->v, v, sizeof(float) * count, cudaMemcpyHostToDevice));
  n->adam_step = adam_step;
  n->prepared = false;
  return TSP_OK;
}

extern "C" tsp_status tsp_net_get_grads(tsp_net n, float* host, size_t count) {
  if (!n || !host || count != n->n_params) return fail(TSP_EINVAL, "tsp_net_get_grads: bad argument");
  TSP_CUDA(cudaMemcpy(host, n->grads, sizeof(float) * count, cudaMemcpyDeviceToHost));
  return TSP_OK;
}

extern "C" tsp_status tsp_net_forward(tsp_net n, const float* a, int batch, float* out, void* stream) {
  TSP_RANGE("tsp_net_forward");
  if (!n || !a || !out || batch <= 0 || batch > n->max_batch) return fail(TSP_EINVAL, "tsp_net_forward: bad argument");
  tsp_status st = check_device(n->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  st = net_forward(n, a, batch, cs);
  if (st != TSP_OK) return st;
  TSP_CUDA(cudaMemcpyAsync(out, n->out, sizeof(float) * size_t(batch) * n->d.V, cudaMemcpyDeviceToDevice, cs));
  return TSP_OK;
}

namespace {
// dW (27 x 32 x 32, added) of 32 -> 32 layer k + 1 from its input h[k] and
// the gated gradient gz: the tcgen05 kernel's per-CTA partials, then their
// fixed-order sum.
void wgrad32_tc(tsp_net n, int k, int batch, float* dW, cudaStream_t cs) {
  Dims db = n->d;
  db.B = batch;
  const int64_t rows = int64_t(batch) * db.Nr * db.Ne;
  const int grid = int(std::min<int64_t>(rows, g_sm_count));
  wgrad32_tc_kernel<<<grid, 256, wg_smem(db.Na), cs>>>(n->map_h[k], n->map_gz, db, n->h[k], n->wpart,
                                                       TC_WAIT_BUDGET);
  part_reduce_kernel<<<27 * CH * CH / 32, 1024, 0, cs>>>(n->wpart, grid, 27 * CH * CH, 27 * CH * CH, dW);
}

// Weight and bias gradient of a one-sided layer (mode 0: output layer from
// g_out and h5; mode 1: input layer from the gated g_h and a): per-CTA
// partial sums, then a fixed-order reduction added to dw (27 x 32) and db (nb).
void thin_wgrad(tsp_net n, int mode, const Dims& db, float* dw, float* dbias, int nb, cudaStream_t cs) {
  const int et = thin_et(db.Na);
  const int64_t tiles = int64_t(db.B) * db.Nr * ((db.Ne + et - 1) / et);
  const int grid = int(std::min<int64_t>(tiles, n->part_rows));
  const size_t sm = thin_smem(db.Na);
  if (mode == 0)
    thin_wgrad_kernel<0><<<grid, 256, sm, cs>>>(db, et, n->gout, n->h[4], nullptr, nullptr, nullptr, n->part);
  else
    thin_wgrad_kernel<1><<<grid, 256, sm, cs>>>(db, et, nullptr, nullptr, n->gh, n->mask[0], n->a16, n->part);
  part_reduce_kernel<<<(27 * CH + 31) / 32, 1024, 0, cs>>>(n->part, grid, THIN_OUT, 27 * CH, dw);
  part_reduce_kernel<<<1, 1024, 0, cs>>>(n->part + 27 * CH, grid, THIN_OUT, nb, dbias);
}
}  // namespace

extern "C" tsp_status tsp_net_loss_grad(tsp_net n, const float* a, const float* target, int batch, double* loss_host,
                                        void* stream) {
  TSP_RANGE("tsp_net_loss_grad");
  if (!n || !a || !target || batch <= 0 || batch > n->max_batch)
    return fail(TSP_EINVAL, "tsp_net_loss_grad: bad argument");
  tsp_status st = check_device(n->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  st = net_forward(n, a, batch, cs);
  if (st != TSP_OK) return st;
  const Dims& d = n->d;
  Dims db = d;
  db.B = batch;
  const int64_t nv = int64_t(batch) * d.V;
  TSP_CUDA(cudaMemsetAsync(n->grads, 0, sizeof(float) * n->n_params, cs));
  const int mse_blocks = int(std::min<int64_t>(blocks_for(nv, 256), MSE_BLOCKS));
  mse_kernel<<<mse_blocks, 256, 0, cs>>>(n->out, target, nv, n->gout, n->loss_part);
  ordered_sum_kernel<<<1, 32, 0, cs>>>(n->loss_part, mse_blocks, n->loss);
  // output layer
  thin_wgrad(n, 0, db, n->grads + n->off_w[5], n->grads + n->off_b[5], 1, cs);
  conv_out_dgrad_kernel<<<blocks_for(nv, 128), 128, 0, cs>>>(db, n->gout, n->w6r, n->gh);
  // residual 32 -> 32 layers, last to first
  const int ggrid = std::min(blocks_for(nv * 4, 256), n->part_rows);
  for (int k = 3; k >= 0; --k) {
    gate_kernel<<<ggrid, 256, 0, cs>>>(n->gh, n->mask[k + 1], n->gz, nv, n->part);
    part_reduce_kernel<<<1, 1024, 0, cs>>>(n->part, ggrid, CH, CH, n->grads + n->off_b[k + 1]);
    wgrad32_tc(n, k, batch, n->grads + n->off_w[k + 1], cs);
    if (st != TSP_OK) return st;
    conv32(1, d, batch, n->map_gz, n->gz, n->wd[k], nullptr, nullptr, nullptr, n->gh, cs);
  }
  // input layer (ReLU gate applied inside)
  thin_wgrad(n, 1, db, n->grads + n->off_w[0], n->grads + n->off_b[0], CH, cs);
  TSP_CUDA(cudaGetLastError());
  if (loss_host) {
    TSP_CUDA(cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, cs));
    TSP_CUDA(cudaStreamSynchronize(cs));
  }
  return TSP_OK;
}

extern "C" tsp_status tsp_net_adam(tsp_net n, float lr, float beta1, float beta2, float eps, float weight_decay,
                                   void* stream) {
  TSP_RANGE("tsp_net_adam");
  if (!n) return fail(TSP_EINVAL, "tsp_net_adam: NULL net");
  n->adam_step += 1;
  n->prepared = false;
  return tsp_adam(n->params, n->grads, n->m, n->v, int64_t(n->n_params), lr, beta1, beta2, eps, weight_decay,
                  n->adam_step, stream);
}

extern "C" tsp_status tsp_net_activation(tsp_net n, int layer, int batch, void* host) {
  if (!n || !host || layer < 0 || layer > 5 || batch <= 0 || batch > n->max_batch)
    return fail(TSP_EINVAL, "tsp_net_activation: bad argument");
  const size_t nv = size_t(batch) * n->d.V;
  if (layer < 5) TSP_CUDA(cudaMemcpy(host, n->h[layer], sizeof(bf16) * nv * CH, cudaMemcpyDeviceToHost));
  else TSP_CUDA(cudaMemcpy(host, n->out, sizeof(float) * nv, cudaMemcpyDeviceToHost));
  return TSP_OK;
}
