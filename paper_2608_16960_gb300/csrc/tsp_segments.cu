// Precomputed segment lists (the paper's steps 1-3 stored once, Sec. 3 and
// Sec. 4.4's stored region indices and lengths; step 4 repeated): per ray the
// (voxel, length) pairs of its valid segments in order along the ray,
// compressed (no padding slots: Eq. 8's padded arrays are not needed), and
// optionally their transpose per voxel (ray, length). Forward and adjoint on
// these lists are one streaming kernel over 8 bytes per segment: the lists
// are read once, coalesced, and multiply an input gathered from L2 (the
// volume, or the detector values), summed per output row in registers.
#include "tsp_kernels.cuh"

namespace tsp {
constexpr int SE = 8;             // entries per lane in the streaming kernel
constexpr int TILE = 32 * SE;     // entries per warp tile
constexpr uint32_t HEAD = 0x80000000u;  // bit 31 of a column: first entry of its row
constexpr uint32_t NO_ROW = 0xFFFFFFFFu;
}  // namespace tsp

// One direction of the lists: rows (rays or voxels) with their entries
// (column index with the row-head flag in bit 31, length), the ids of the
// non-empty rows in order, and per warp tile the number of row heads before
// it. carry / headless / open_row are per-call scratch of the streaming
// kernel (one value per tile).
struct SegList {
  int64_t n_rows = 0, n_cols = 0, S = 0, n_tiles = 0, n_nz = 0;
  int64_t* off = nullptr;        // [n_rows + 1] row offsets
  uint32_t* idx = nullptr;       // [S] column | HEAD on each row's first entry
  float* len = nullptr;          // [S]
  uint32_t* nz = nullptr;        // [n_nz] row id of the k-th non-empty row
  int64_t* tile_base = nullptr;  // [n_tiles + 1] heads before tile t
  float* carry = nullptr;        // [n_tiles]
  uint8_t* headless = nullptr;   // [n_tiles]
  uint32_t* open_row = nullptr;  // [n_tiles]
};

struct tsp_segments_s {
  int64_t n_rays = 0, n_segs = 0, V = 0;
  SegList fwd;  // ray-major: rows = rays, columns = voxels
  SegList adj;  // voxel-major (transposed): rows = voxels, columns = rays
  bool has_adj = false;
  size_t bytes = 0;
  int device = 0;
};

namespace tsp {
namespace {

struct CountOnlyOp {
  int* __restrict__ counts;
  int n;
  __device__ __forceinline__ bool begin(int64_t) {
    n = 0;
    return true;
  }
  __device__ __forceinline__ void operator()(int, float) { ++n; }
  __device__ __forceinline__ void end(int64_t ray) { counts[ray] = n; }
};

// The fill walk repeats the count walk bit for bit (same code, no FMA
// contraction), so each ray fills exactly its slots; the bound check only
// guards memory should that ever fail, and flags the error word.
struct FillOp {
  const int64_t* __restrict__ off;
  uint32_t* __restrict__ vox;
  float* __restrict__ len;
  int64_t pos, lim;
  __device__ __forceinline__ bool begin(int64_t ray) {
    pos = off[ray];
    first = pos;
    lim = off[ray + 1];
    return true;
  }
  int64_t first;
  __device__ __forceinline__ void operator()(int v, float dl) {
    if (pos < lim) {
      vox[pos] = uint32_t(v) | (pos == first ? HEAD : 0u);
      len[pos] = dl;
    }
    ++pos;
  }
  __device__ __forceinline__ void end(int64_t) {
    if (pos != lim) atomicOr(&g_tsp_error_word, 2);
  }
};

// ---- exclusive scan of int32 counts into int64 offsets (out[n] = total) ----
constexpr int SCAN_T = 1024, SCAN_E = 2;  // threads, elements per thread

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < int(blockDim.x >> 5) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    sh[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += sh[warp - 1];
  __syncthreads();
  return v;
}

__global__ void scan_blocks_kernel(const int* __restrict__ in, int64_t n, int64_t* __restrict__ block_sums) {
  __shared__ int64_t sh[32];
  const int64_t base = int64_t(blockIdx.x) * SCAN_T * SCAN_E + int64_t(threadIdx.x) * SCAN_E;
  int64_t s = 0;
  for (int k = 0; k < SCAN_E; ++k)
    if (base + k < n) s += in[base + k];
  const int64_t incl = block_incl_scan(s, sh);
  if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = incl;
}

// one block: exclusive scan of the block sums in place, total at [nb]
__global__ void scan_sums_kernel(int64_t* __restrict__ sums, int64_t nb) {
  __shared__ int64_t sh[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const int64_t v = i < nb ? sums[i] : 0;
    const int64_t incl = block_incl_scan(v, sh);
    const int64_t base = carry;
    if (i < nb) sums[i] = base + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = base + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_final_kernel(const int* __restrict__ in, int64_t n, const int64_t* __restrict__ sums,
                                  int64_t* __restrict__ out) {
  __shared__ int64_t sh[32];
  const int64_t base = int64_t(blockIdx.x) * SCAN_T * SCAN_E + int64_t(threadIdx.x) * SCAN_E;
  int64_t v[SCAN_E];
  int64_t s = 0;
  for (int k = 0; k < SCAN_E; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int64_t run = block_incl_scan(s, sh) - s + sums[blockIdx.x];
  for (int k = 0; k < SCAN_E; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    int64_t nb = gridDim.x;
    out[n] = sums[nb];
  }
}

tsp_status exclusive_scan(const int* in, int64_t n, int64_t* out, cudaStream_t st) {
  if (n == 0) {
    TSP_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return TSP_OK;
  }
  const int64_t per = int64_t(SCAN_T) * SCAN_E;
  const int64_t nb = (n + per - 1) / per;
  int64_t* sums = nullptr;
  TSP_CUDA(cudaMallocAsync(&sums, sizeof(int64_t) * size_t(nb + 1), st));
  scan_blocks_kernel<<<unsigned(nb), SCAN_T, 0, st>>>(in, n, sums);
  scan_sums_kernel<<<1, 1024, 0, st>>>(sums, nb);
  scan_final_kernel<<<unsigned(nb), SCAN_T, 0, st>>>(in, n, sums, out);
  TSP_CUDA(cudaGetLastError());
  TSP_CUDA(cudaFreeAsync(sums, st));
  return TSP_OK;
}

__global__ void voxel_hist_kernel(const uint32_t* __restrict__ vox, int64_t S, int64_t V, int* __restrict__ cnt) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < S; i += int64_t(gridDim.x) * blockDim.x)
    if ((vox[i] & ~HEAD) < V) atomicAdd(cnt + (vox[i] & ~HEAD), 1);
}

// ---- voxel-major transpose: stable LSD radix sort of the entries by voxel ----
// Keys are the voxel ids of the ray-major entries, carried with their ray id
// and length, RB bits of the key per pass. A pass counts each tile's digits,
// scans the counts digit-major (digit 0 of every tile, then digit 1, ...) and
// scatters: an entry goes to its digit's base in its tile plus the number of
// same-digit entries before it in the tile. Every pass keeps the order of
// equal digits, so after the last one each voxel's entries are in ray-major
// order (by ray, then along the ray): the same rows on every build.
constexpr int RB = 8, RD = 1 << RB;  // key bits per pass, digits
constexpr int RW = 8, RK = 8;        // warps per block, entries per lane
constexpr int RT = RW * 32 * RK;     // entries per tile

__device__ __forceinline__ uint32_t radix_key(const uint32_t* __restrict__ keys, bool first, int64_t i) {
  return first ? (keys[i] & ~HEAD) : keys[i];
}

__global__ void __launch_bounds__(RW * 32) radix_hist_kernel(const uint32_t* __restrict__ keys, bool first,
                                                             int64_t S, int shift, int64_t n_tiles,
                                                             int* __restrict__ hist) {
  __shared__ int h[RD];
  for (int d = threadIdx.x; d < RD; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t t = blockIdx.x, e0 = t * RT;
  for (int j = threadIdx.x; j < RT; j += blockDim.x) {
    const int64_t i = e0 + j;
    if (i < S) atomicAdd(&h[(radix_key(keys, first, i) >> shift) & (RD - 1)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RD; d += blockDim.x) hist[int64_t(d) * n_tiles + t] = h[d];
}

// One pass over a tile of RT entries (RD == threads per block). Ranking: a
// warp takes its 32 * RK consecutive entries in RK rounds of 32; lanes with
// equal digits find each other (match), take the warp's running count for the
// digit plus the number of such lanes below them, and the lowest of them
// advances the count. The warps' counts become offsets in warp order and the
// digits' totals offsets in digit order, which sorts the tile by digit in
// shared memory; the tile then leaves as one contiguous run per digit.
// FIRST reads the ray-major columns (keys with the head flag) and the ray ids
// and lengths beside them; FINAL writes only (ray, length).
template <bool FIRST, bool FINAL>
__global__ void __launch_bounds__(RW * 32) radix_scatter_kernel(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rays, const float* __restrict__ lens, int64_t S,
    int shift, int64_t n_tiles, const int64_t* __restrict__ base, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ rays_out, float* __restrict__ lens_out) {
  __shared__ int cnt[RW][RD];
  __shared__ int start[RD];
  __shared__ int64_t scan_sh[32];
  __shared__ uint32_t sk[RT], sr[RT];
  __shared__ float sl[RT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = lane; d < RD; d += 32) cnt[warp][d] = 0;
  __syncwarp();
  const int64_t t = blockIdx.x, w0 = t * RT + int64_t(warp) * (32 * RK);
  const unsigned below = (1u << lane) - 1u;
  uint32_t key[RK], ray[RK];
  float len[RK];
  int rank[RK];
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    const int64_t i = w0 + k * 32 + lane;
    const bool ok = i < S;
    key[k] = ok ? radix_key(keys, FIRST, i) : 0u;
    ray[k] = ok ? rays[i] : 0u;
    len[k] = ok ? lens[i] : 0.0f;
    const uint32_t d = ok ? (key[k] >> shift) & (RD - 1) : uint32_t(RD);  // past the end: a class of its own
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    rank[k] = ok ? cnt[warp][d] + __popc(peers & below) : 0;
    __syncwarp();
    if (ok && (peers & below) == 0) cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    int run = 0;
    for (int w = 0; w < RW; ++w) {
      const int c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
    const int64_t incl = block_incl_scan(run, scan_sh);
    start[d] = int(incl - run);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RK; ++k) {
    if (w0 + k * 32 + lane >= S) continue;
    const uint32_t d = (key[k] >> shift) & (RD - 1);
    const int lp = start[d] + cnt[warp][d] + rank[k];
    sk[lp] = key[k];
    sr[lp] = ray[k];
    sl[lp] = len[k];
  }
  __syncthreads();
  const int n = int(S - t * RT < RT ? S - t * RT : RT);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const uint32_t kk = sk[j];
    const uint32_t d = (kk >> shift) & (RD - 1);
    const int64_t g = base[int64_t(d) * n_tiles + t] + (j - start[d]);
    if (!FINAL) keys_out[g] = kk;
    rays_out[g] = sr[j];
    lens_out[g] = sl[j];
  }
}

// ray id of every ray-major entry (warp per ray)
__global__ void ray_ids_kernel(const int64_t* __restrict__ off, int64_t n_rays, uint32_t* __restrict__ rid) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_rays) return;
  for (int64_t s = off[w] + lane; s < off[w + 1]; s += 32) rid[s] = uint32_t(w);
}


// ---- streaming forward / adjoint ----
// The lists are read as one flat stream: warp t takes entries [t*TILE,
// (t+1)*TILE), SE consecutive ones per lane (two 16-byte loads of columns, two
// of lengths), gathers the input at the SE columns (L2-resident: the volume,
// or the detector values) and multiplies. Rows are runs of entries that start
// at a flagged head; a run's row id is nz[rank], its rank counted from the
// tile's head base plus the heads of earlier lanes. Each lane sums its runs
// in order; a shuffle scan of (pass-through, value) pairs carries an open run
// across lanes. Writes (no atomics, every row written by one thread per pass;
// "+=" when accumulating, a plain store otherwise):
//  - a run that starts and ends inside the tile: dst[row] (+)= sum;
//  - the run open at the tile's end (it starts at the tile's last head):
//    dst[row] (+)= partial, and open_row[t] = row when it continues;
//  - the piece before the tile's first head: carry[t] (the whole tile when it
//    has no head: headless[t] = 1).
// seg_fixup_kernel then adds, for each open row, the carries of the following
// tiles in order. Rows without entries are left alone (the caller zeroes dst
// when overwriting). All sums have a fixed order, so results are
// bit-reproducible.
template <bool FULL, bool ACC>
__device__ __forceinline__ void stream_tile(int64_t t, int lane, uint32_t* s_nz, const uint32_t* __restrict__ idx,
                                            const float* __restrict__ len, int64_t S, uint32_t col_max,
                                            const uint32_t* __restrict__ nz, int64_t n_nz, int64_t base,
                                            uint32_t nxt_first, const float* __restrict__ src,
                                            float* __restrict__ dst, float* __restrict__ carry,
                                            uint8_t* __restrict__ headless, uint32_t* __restrict__ open_row) {
  const int64_t T0 = t * TILE, e0 = T0 + int64_t(lane) * SE;
  uint32_t iv[SE];
  float lv[SE];
  if (FULL) {
    const uint4* pi = reinterpret_cast<const uint4*>(idx + e0);
    const float4* pl = reinterpret_cast<const float4*>(len + e0);
#pragma unroll
    for (int h = 0; h < SE / 4; ++h) {
      const uint4 a = __ldcs(pi + h);
      const float4 b = __ldcs(pl + h);
      iv[4 * h] = a.x, iv[4 * h + 1] = a.y, iv[4 * h + 2] = a.z, iv[4 * h + 3] = a.w;
      lv[4 * h] = b.x, lv[4 * h + 1] = b.y, lv[4 * h + 2] = b.z, lv[4 * h + 3] = b.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < SE; ++i) {
      const bool ok = e0 + i < S;
      iv[i] = ok ? __ldcs(idx + e0 + i) : 0u;
      lv[i] = ok ? __ldcs(len + e0 + i) : 0.0f;
    }
  }
  // row ids of the ranks this tile can touch (base-1 .. base+30), one coalesced load
  {
    const int64_t r = base - 1 + lane;
    s_nz[lane] = (r >= 0 && r < n_nz) ? nz[r] : NO_ROW;
  }
  unsigned heads = 0;
  float p[SE];
#pragma unroll
  for (int i = 0; i < SE; ++i) {
    heads |= (iv[i] >> 31) << i;
    p[i] = __ldg(src + min(iv[i] & ~HEAD, col_max));  // the clamp only guards memory: columns are valid
  }
#pragma unroll
  for (int i = 0; i < SE; ++i) p[i] = (FULL || e0 + i < S) ? p[i] * lv[i] : 0.0f;
  const int nh = __popc(heads);
  int hb = nh;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, hb, o);
    if (lane >= o) hb += v;
  }
  const int tile_heads = __shfl_sync(0xffffffffu, hb, 31);
  hb -= nh;
  __syncwarp();
  auto row_of = [&](int64_t rank) -> uint32_t {
    const int64_t i = rank - (base - 1);
    if (i >= 0 && i < 32) return s_nz[i];
    if (rank < 0 || rank >= n_nz) {  // inconsistent lists: reported, the write dropped
      atomicOr(&g_tsp_error_word, 8);
      return NO_ROW;
    }
    return nz[rank];
  };
  auto put = [&](uint32_t row, float v) {
    if (row == NO_ROW) return;
    if (ACC) dst[row] += v;
    else dst[row] = v;
  };
  // in-lane runs
  float run = 0.0f, lead = 0.0f;
  int64_t rk = base + hb - 1;
  bool seen = false;
#pragma unroll
  for (int i = 0; i < SE; ++i) {
    if ((heads >> i) & 1u) {
      if (!seen) {
        lead = run;
        seen = true;
      } else {
        put(row_of(rk), run);  // complete run inside this lane
      }
      run = 0.0f;
      ++rk;
    }
    run += p[i];
  }
  if (!seen) lead = run;
  // carry across lanes: lane function x -> seen ? tail : x + lead
  int c = seen ? 0 : 1;
  float d = seen ? run : lead;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int cp = __shfl_up_sync(0xffffffffu, c, o);
    const float dp = __shfl_up_sync(0xffffffffu, d, o);
    if (lane >= o) {
      d = c ? dp + d : d;
      c = cp & c;
    }
  }
  float cin = __shfl_up_sync(0xffffffffu, d, 1);
  if (lane == 0) cin = 0.0f;
  const float d_last = __shfl_sync(0xffffffffu, d, 31);
  if (seen) {
    const float tot = cin + lead;  // the run closed at this lane's first head
    if (hb > 0) put(row_of(base + hb - 1), tot);
    else carry[t] = tot;  // continues a row begun before this tile
  }
  if (lane == 31) {
    if (tile_heads == 0) {
      carry[t] = d_last;
      headless[t] = 1;
      open_row[t] = NO_ROW;
    } else {
      const uint32_t row = row_of(base + tile_heads - 1);
      put(row, d_last);
      headless[t] = 0;
      open_row[t] = (nxt_first & HEAD) ? NO_ROW : row;
    }
  }
}

template <bool ACC>
__global__ void __launch_bounds__(256, 6) seg_stream_kernel(const uint32_t* __restrict__ idx,
                                                         const float* __restrict__ len, int64_t S, uint32_t n_cols,
                                                         const uint32_t* __restrict__ nz, int64_t n_nz,
                                                         const int64_t* __restrict__ tile_base, int64_t n_tiles,
                                                         const float* __restrict__ src, float* __restrict__ dst,
                                                         float* __restrict__ carry, uint8_t* __restrict__ headless,
                                                         uint32_t* __restrict__ open_row) {
  __shared__ uint32_t s_nz[8][32];
  const int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_tiles) return;
  const int64_t base = tile_base[t];
  const int64_t nxt = (t + 1) * TILE;
  const uint32_t nxt_first = (lane == 31 && nxt < S) ? idx[nxt] : HEAD;  // does the next tile open a new row
  uint32_t* sn = s_nz[threadIdx.x >> 5];
  if (nxt <= S)
    stream_tile<true, ACC>(t, lane, sn, idx, len, S, n_cols - 1, nz, n_nz, base, nxt_first, src, dst, carry, headless,
                           open_row);
  else
    stream_tile<false, ACC>(t, lane, sn, idx, len, S, n_cols - 1, nz, n_nz, base, nxt_first, src, dst, carry,
                            headless, open_row);
}

// Long rows (voxel-major lists: hundreds of entries per voxel): a warp per row
// streams the row's entries, U per lane per pass (all U loads issued before
// the U gathers), and a shuffle tree sums the lanes. Fixed order, no atomics.
constexpr int RU = 4;

template <int NB>
__global__ void __launch_bounds__(256) row_gather_kernel(const int64_t* __restrict__ off,
                                                         const uint32_t* __restrict__ idx,
                                                         const float* __restrict__ len, int64_t n_rows,
                                                         uint32_t col_max, const float* __restrict__ src,
                                                         int64_t src_stride, float* __restrict__ dst,
                                                         int64_t dst_stride, int nb, int accumulate) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_rows) return;
  float acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = 0.0f;
  const int64_t s1 = off[w + 1];
  for (int64_t s = off[w] + lane; s < s1; s += 32 * RU) {
    uint32_t i[RU];
    float l[RU];
#pragma unroll
    for (int k = 0; k < RU; ++k) {
      const int64_t sk = s + 32 * k;
      i[k] = sk < s1 ? min(__ldcs(idx + sk) & ~HEAD, col_max) : 0u;
      l[k] = sk < s1 ? __ldcs(len + sk) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < RU; ++k)
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < nb) acc[b] = fmaf(__ldg(src + b * src_stride + i[k]), l[k], acc[b]);
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float v = acc[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0 && b < nb) {
      float* p = dst + b * dst_stride + w;
      *p = accumulate ? *p + v : v;
    }
  }
}

// dst[row] += the carries of the tiles after t that continue the row open at
// t's end, in tile order.
__global__ void seg_fixup_kernel(const float* __restrict__ carry, const uint8_t* __restrict__ headless,
                                 const uint32_t* __restrict__ open_row, int64_t n_tiles, float* __restrict__ dst) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const uint32_t row = open_row[t];
  if (row == NO_ROW) return;
  float v = 0.0f;
  for (int64_t k = t + 1; k < n_tiles; ++k) {
    v += carry[k];
    if (!headless[k]) break;
  }
  dst[row] += v;
}

// adjoint without the transposed lists: one atomic per segment
__global__ void seg_scatter_kernel(const int64_t* __restrict__ off, const uint32_t* __restrict__ vox,
                                   const float* __restrict__ len, const float* __restrict__ y, float* __restrict__ g,
                                   int64_t n_rays) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_rays) return;
  const float yv = y[w];
  if (yv == 0.0f) return;
  for (int64_t s = off[w] + lane; s < off[w + 1]; s += 32) atomicAdd(g + (vox[s] & ~HEAD), yv * len[s]);
}

// Rows at least this long on average take the warp-per-row kernel.
constexpr int64_t LONG_ROWS = 256;

// dst (+)= lists x src: long rows a warp each (up to 4 right-hand sides per
// pass over the lists), short rows by the flat stream (one per pass).
tsp_status rows_apply(const SegList& l, const float* src, int64_t src_stride, float* dst, int64_t dst_stride, int nb,
                      int accumulate, cudaStream_t st) {
  if (l.S >= LONG_ROWS * l.n_rows) {
    const unsigned blocks = unsigned((l.n_rows * 32 + 255) / 256);
    for (int b0 = 0; b0 < nb; b0 += 4) {
      const int k = std::min(4, nb - b0);
      const float* sp = src + b0 * src_stride;
      float* dp = dst + b0 * dst_stride;
      if (k == 1)
        row_gather_kernel<1><<<blocks, 256, 0, st>>>(l.off, l.idx, l.len, l.n_rows, uint32_t(l.n_cols - 1), sp,
                                                     src_stride, dp, dst_stride, 1, accumulate);
      else
        row_gather_kernel<4><<<blocks, 256, 0, st>>>(l.off, l.idx, l.len, l.n_rows, uint32_t(l.n_cols - 1), sp,
                                                     src_stride, dp, dst_stride, k, accumulate);
    }
    TSP_CUDA(cudaGetLastError());
    return TSP_OK;
  }
  if (!accumulate) {
    if (dst_stride == l.n_rows) {
      TSP_CUDA(cudaMemsetAsync(dst, 0, sizeof(float) * size_t(l.n_rows) * nb, st));
    } else {
      for (int b = 0; b < nb; ++b)
        TSP_CUDA(cudaMemsetAsync(dst + b * dst_stride, 0, sizeof(float) * size_t(l.n_rows), st));
    }
  }
  if (l.n_tiles == 0) return TSP_OK;
  const unsigned blocks = unsigned((l.n_tiles * 32 + 255) / 256);
  const unsigned fix_blocks = unsigned((l.n_tiles + 255) / 256);
  for (int b = 0; b < nb; ++b) {
    if (accumulate)
      seg_stream_kernel<true><<<blocks, 256, 0, st>>>(l.idx, l.len, l.S, uint32_t(l.n_cols), l.nz, l.n_nz,
                                                      l.tile_base, l.n_tiles, src + b * src_stride,
                                                      dst + b * dst_stride, l.carry, l.headless, l.open_row);
    else
      seg_stream_kernel<false><<<blocks, 256, 0, st>>>(l.idx, l.len, l.S, uint32_t(l.n_cols), l.nz, l.n_nz,
                                                       l.tile_base, l.n_tiles, src + b * src_stride,
                                                       dst + b * dst_stride, l.carry, l.headless, l.open_row);
    seg_fixup_kernel<<<fix_blocks, 256, 0, st>>>(l.carry, l.headless, l.open_row, l.n_tiles, dst + b * dst_stride);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

__global__ void nonempty_flags_kernel(const int64_t* __restrict__ off, int64_t n_rows, int* __restrict__ flag) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < n_rows) flag[r] = off[r + 1] > off[r] ? 1 : 0;
}

__global__ void nonempty_ids_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ pos, int64_t n_rows,
                                    uint32_t* __restrict__ nz) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < n_rows && off[r + 1] > off[r]) nz[pos[r]] = uint32_t(r);
}

__global__ void tile_heads_kernel(const uint32_t* __restrict__ idx, int64_t S, int64_t n_tiles, int* __restrict__ cnt) {
  const int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_tiles) return;
  int c = 0;
  for (int i = 0; i < SE; ++i) {
    const int64_t e = t * TILE + int64_t(lane) * SE + i;
    if (e < S) c += int(idx[e] >> 31);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[t] = c;
}

__global__ void mark_heads_kernel(const int64_t* __restrict__ off, int64_t n_rows, uint32_t* __restrict__ idx) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < n_rows && off[r + 1] > off[r]) idx[off[r]] |= HEAD;
}

// Non-empty row ids, tile head bases and the per-call scratch of one
// direction, once its offsets and (flagged) entries exist. `tmp` holds at
// least max(n_rows, n_tiles) ints, `pos` n_rows + 1 int64.
tsp_status finish_list(SegList& l, int* tmp, int64_t* pos, cudaStream_t st) {
  const unsigned rb = unsigned((l.n_rows + 255) / 256);
  nonempty_flags_kernel<<<rb, 256, 0, st>>>(l.off, l.n_rows, tmp);
  tsp_status r = exclusive_scan(tmp, l.n_rows, pos, st);
  if (r != TSP_OK) return r;
  TSP_CUDA(cudaMemcpyAsync(&l.n_nz, pos + l.n_rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TSP_CUDA(cudaStreamSynchronize(st));
  TSP_CUDA(dev_malloc(&l.nz, sizeof(uint32_t) * size_t(l.n_nz > 0 ? l.n_nz : 1)));
  nonempty_ids_kernel<<<rb, 256, 0, st>>>(l.off, pos, l.n_rows, l.nz);
  l.n_tiles = (l.S + TILE - 1) / TILE;
  const size_t nt = size_t(l.n_tiles > 0 ? l.n_tiles : 1);
  TSP_CUDA(dev_malloc(&l.tile_base, sizeof(int64_t) * (nt + 1)));
  TSP_CUDA(dev_malloc(&l.carry, sizeof(float) * nt));
  TSP_CUDA(dev_malloc(&l.headless, nt));
  TSP_CUDA(dev_malloc(&l.open_row, sizeof(uint32_t) * nt));
  if (l.n_tiles > 0) {
    tile_heads_kernel<<<unsigned((l.n_tiles * 32 + 255) / 256), 256, 0, st>>>(l.idx, l.S, l.n_tiles, tmp);
    r = exclusive_scan(tmp, l.n_tiles, l.tile_base, st);
    if (r != TSP_OK) return r;
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

// ---- SIRT on the stored lists (same update as tsp_sirt) ----
__global__ void fill_kernel(float* __restrict__ a, int64_t n, float v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    a[i] = v;
}

// a[i] = 1 / a[i], 0 where a[i] <= 0 (rays missing the grid, voxels no ray meets)
__global__ void recip_kernel(float* __restrict__ a, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float v = a[i];
    a[i] = v > 0.0f ? __frcp_rn(v) : 0.0f;
  }
}

// r = R * (y - f), in place over f
__global__ void residual_kernel(float* __restrict__ f, const float* __restrict__ y, const float* __restrict__ R,
                                int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    f[i] = __fmul_rn(R[i], __fsub_rn(y[i], f[i]));
}

// x += C * g, clamped at 0 if asked
__global__ void xupdate_kernel(float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ C,
                               int64_t n, int nonneg) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float v = fmaf(C[i], g[i], x[i]);
    if (nonneg) v = fmaxf(v, 0.0f);
    x[i] = v;
  }
}

unsigned ew_blocks(int64_t n) { return unsigned(std::min<int64_t>((n + 255) / 256, 152 * 16)); }
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t entries_alloc(int64_t S) { return size_t(S > 0 ? S : 1); }

void free_list(SegList& l) {
  cudaFree(l.off);
  cudaFree(l.idx);
  cudaFree(l.len);
  cudaFree(l.nz);
  cudaFree(l.tile_base);
  cudaFree(l.carry);
  cudaFree(l.headless);
  cudaFree(l.open_row);
  l = SegList();
}

size_t list_bytes(const SegList& l) {
  if (!l.off) return 0;
  const size_t nt = size_t(l.n_tiles > 0 ? l.n_tiles : 1);
  return sizeof(int64_t) * size_t(l.n_rows + 1) + 8 * entries_alloc(l.S) + 4 * size_t(l.n_nz > 0 ? l.n_nz : 1) +
         nt * (8 + 4 + 1 + 4) + 8;
}

}  // namespace
}  // namespace tsp

using namespace tsp;

extern "C" void tsp_segments_destroy(tsp_segments s) {
  if (!s) return;
  free_list(s->fwd);
  free_list(s->adj);
  delete s;
}

extern "C" tsp_status tsp_segments_build(tsp_grid grid, tsp_geom geom, int transpose, tsp_segments* out,
                                         void* stream) {
  TSP_RANGE("tsp_segments_build");
  if (!out) return fail(TSP_EINVAL, "tsp_segments_build: out is NULL");
  *out = nullptr;
  tsp_status st = check_trace_args(grid, geom, grid, geom, 1, nullptr, "tsp_segments_build");
  if (st != TSP_OK) return st;
  if (geom->n_rays >= (int64_t(1) << 31) || grid->voxels() >= (int64_t(1) << 31))
    return fail(TSP_ENOTSUP, "tsp_segments_build: 2^31 or more rays or voxels");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  tsp_segments s = new (std::nothrow) tsp_segments_s();
  if (!s) return fail(TSP_ENOMEM, "tsp_segments_build: host allocation");
  s->n_rays = geom->n_rays;
  s->V = grid->voxels();
  s->device = grid->device;
  int* counts = nullptr;
  int* vcount = nullptr;
  int* tmp = nullptr;
  int64_t* pos = nullptr;
  uint32_t *ka = nullptr, *kb = nullptr, *rb = nullptr;  // radix sort: keys of both buffers, B's ray ids
  float* lb = nullptr;                                    // and B's lengths
  int* rhist = nullptr;
  int64_t* rbase = nullptr;
  auto release = [&]() {
    cudaFree(counts);
    cudaFree(vcount);
    cudaFree(tmp);
    cudaFree(pos);
    cudaFree(ka);
    cudaFree(kb);
    cudaFree(rb);
    cudaFree(lb);
    cudaFree(rhist);
    cudaFree(rbase);
    counts = vcount = tmp = rhist = nullptr;
    pos = rbase = nullptr;
    ka = kb = rb = nullptr;
    lb = nullptr;
  };
  auto bail = [&](tsp_status r) {
    cudaStreamSynchronize(cs);
    release();
    tsp_segments_destroy(s);
    return r;
  };
#define SEG_TRY(call)                                                                        \
  do {                                                                                       \
    cudaError_t e__ = (call);                                                                \
    if (e__ == cudaErrorMemoryAllocation) {                                                  \
      cudaGetLastError(); /* not sticky: clear it */                                         \
      return bail(fail(TSP_ENOMEM, std::string("tsp_segments_build: out of device memory at ") + #call)); \
    }                                                                                        \
    if (e__ != cudaSuccess) return bail(cuda_fail(e__, #call));                              \
  } while (0)
  SegList& f = s->fwd;
  f.n_rows = s->n_rays;
  f.n_cols = s->V;
  SEG_TRY(dev_malloc(&counts, sizeof(int) * size_t(s->n_rays)));
  SEG_TRY(dev_malloc(&f.off, sizeof(int64_t) * size_t(s->n_rays + 1)));
  const tsp_launch l = preferred_launch(grid, geom, false);
  CountOnlyOp cop;
  cop.counts = counts;
  launch_trace(grid, geom, l, cop, cs);
  st = exclusive_scan(counts, s->n_rays, f.off, cs);
  if (st != TSP_OK) return bail(st);
  SEG_TRY(cudaMemcpyAsync(&s->n_segs, f.off + s->n_rays, sizeof(int64_t), cudaMemcpyDeviceToHost, cs));
  SEG_TRY(cudaStreamSynchronize(cs));
  if (s->n_segs >= (int64_t(1) << 32)) return bail(fail(TSP_ENOTSUP, "tsp_segments_build: 2^32 or more segments"));
  f.S = s->n_segs;
  const size_t P = entries_alloc(s->n_segs);
  SEG_TRY(dev_malloc(&f.idx, sizeof(uint32_t) * P));
  SEG_TRY(dev_malloc(&f.len, sizeof(float) * P));
  SEG_TRY(cudaMemsetAsync(f.idx, 0, sizeof(uint32_t) * P, cs));  // no stray head flags in unfilled slots
  FillOp fop;
  fop.off = f.off;
  fop.vox = f.idx;
  fop.len = f.len;
  launch_trace(grid, geom, l, fop, cs);
  SEG_TRY(cudaGetLastError());
  const int64_t rows_max = std::max<int64_t>(s->n_rays, s->V);
  SEG_TRY(dev_malloc(&tmp, sizeof(int) * size_t(std::max<int64_t>(rows_max, (s->n_segs + TILE - 1) / TILE + 1))));
  SEG_TRY(dev_malloc(&pos, sizeof(int64_t) * size_t(rows_max + 1)));
  st = finish_list(f, tmp, pos, cs);
  if (st != TSP_OK) return bail(st);
  if (transpose) {
    SegList& t = s->adj;
    t.n_rows = s->V;
    t.n_cols = s->n_rays;
    t.S = s->n_segs;
    SEG_TRY(dev_malloc(&vcount, sizeof(int) * size_t(s->V)));
    SEG_TRY(dev_malloc(&t.off, sizeof(int64_t) * size_t(s->V + 1)));
    SEG_TRY(dev_malloc(&t.idx, sizeof(uint32_t) * P));
    SEG_TRY(dev_malloc(&t.len, sizeof(float) * P));
    SEG_TRY(cudaMemsetAsync(vcount, 0, sizeof(int) * size_t(s->V), cs));
    SEG_TRY(cudaMemsetAsync(t.idx, 0, sizeof(uint32_t) * P, cs));
    voxel_hist_kernel<<<152 * 16, 256, 0, cs>>>(f.idx, s->n_segs, s->V, vcount);
    st = exclusive_scan(vcount, s->V, t.off, cs);
    if (st != TSP_OK) return bail(st);
    if (s->n_segs > 0) {
      // Stable radix sort by voxel. The last pass writes (ray, length) into t;
      // the passes before it alternate between the buffers A = (ka, t.idx,
      // t.len) and B = (kb, rb, lb) so that the last one reads B. The ray ids
      // of the ray-major entries start in the ray array that the first pass
      // does not write.
      int bits = 1;
      while (bits < 32 && (uint64_t(s->V - 1) >> bits) != 0) ++bits;
      const int passes = (bits + RB - 1) / RB;
      const int64_t n_rt = (s->n_segs + RT - 1) / RT;
      SEG_TRY(dev_malloc(&rhist, sizeof(int) * size_t(RD * n_rt)));
      SEG_TRY(dev_malloc(&rbase, sizeof(int64_t) * size_t(RD * n_rt + 1)));
      SEG_TRY(dev_malloc(&rb, sizeof(uint32_t) * P));
      if (passes > 1) {
        SEG_TRY(dev_malloc(&kb, sizeof(uint32_t) * P));
        SEG_TRY(dev_malloc(&lb, sizeof(float) * P));
      }
      if (passes > 2) SEG_TRY(dev_malloc(&ka, sizeof(uint32_t) * P));
      const bool first_to_a = (passes - 1) % 2 == 0;
      uint32_t* rid = first_to_a ? rb : t.idx;
      ray_ids_kernel<<<unsigned((s->n_rays * 32 + 255) / 256), 256, 0, cs>>>(f.off, s->n_rays, rid);
      const uint32_t *ik = f.idx, *ir = rid;
      const float* il = f.len;
      for (int p = 0; p < passes; ++p) {
        const bool first = p == 0, final_pass = p == passes - 1;
        const int shift = p * RB;
        radix_hist_kernel<<<unsigned(n_rt), RW * 32, 0, cs>>>(ik, first, s->n_segs, shift, n_rt, rhist);
        st = exclusive_scan(rhist, RD * n_rt, rbase, cs);
        if (st != TSP_OK) return bail(st);
        const bool to_a = final_pass || (passes - 1 - p) % 2 == 0;
        uint32_t* ok_ = to_a ? ka : kb;
        uint32_t* orr = to_a ? t.idx : rb;
        float* ol = to_a ? t.len : lb;
        const unsigned g = unsigned(n_rt);
        const int64_t S_ = s->n_segs;
        if (first && final_pass)
          radix_scatter_kernel<true, true><<<g, RW * 32, 0, cs>>>(ik, ir, il, S_, shift, n_rt, rbase, ok_, orr, ol);
        else if (first)
          radix_scatter_kernel<true, false><<<g, RW * 32, 0, cs>>>(ik, ir, il, S_, shift, n_rt, rbase, ok_, orr, ol);
        else if (final_pass)
          radix_scatter_kernel<false, true><<<g, RW * 32, 0, cs>>>(ik, ir, il, S_, shift, n_rt, rbase, ok_, orr, ol);
        else
          radix_scatter_kernel<false, false><<<g, RW * 32, 0, cs>>>(ik, ir, il, S_, shift, n_rt, rbase, ok_, orr, ol);
        SEG_TRY(cudaGetLastError());
        ik = ok_;
        ir = orr;
        il = ol;
      }
    }
    mark_heads_kernel<<<unsigned((s->V + 255) / 256), 256, 0, cs>>>(t.off, s->V, t.idx);
    SEG_TRY(cudaGetLastError());
    st = finish_list(t, tmp, pos, cs);
    if (st != TSP_OK) return bail(st);
    s->has_adj = true;
  }
  SEG_TRY(cudaStreamSynchronize(cs));
  release();
#undef SEG_TRY
  s->bytes = list_bytes(s->fwd) + list_bytes(s->adj);
  *out = s;
  return TSP_OK;
}

extern "C" tsp_status tsp_segments_info(tsp_segments s, int64_t* n_rays, int64_t* n_segments, size_t* bytes) {
  if (!s) return fail(TSP_EINVAL, "tsp_segments_info: NULL handle");
  if (n_rays) *n_rays = s->n_rays;
  if (n_segments) *n_segments = s->n_segs;
  if (bytes) *bytes = s->bytes;
  return TSP_OK;
}

extern "C" tsp_status tsp_segments_export(tsp_segments s, int64_t* ray_off, uint32_t* vox, float* len) {
  if (!s) return fail(TSP_EINVAL, "tsp_segments_export: NULL handle");
  tsp_status st = check_device(s->device);
  if (st != TSP_OK) return st;
  if (ray_off)
    TSP_CUDA(cudaMemcpy(ray_off, s->fwd.off, sizeof(int64_t) * size_t(s->n_rays + 1), cudaMemcpyDeviceToHost));
  if (vox && s->n_segs) {
    TSP_CUDA(cudaMemcpy(vox, s->fwd.idx, sizeof(uint32_t) * size_t(s->n_segs), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < s->n_segs; ++i) vox[i] &= ~HEAD;
  }
  if (len && s->n_segs) TSP_CUDA(cudaMemcpy(len, s->fwd.len, sizeof(float) * size_t(s->n_segs), cudaMemcpyDeviceToHost));
  return TSP_OK;
}

extern "C" tsp_status tsp_segments_export_transposed(tsp_segments s, int64_t* vox_off, uint32_t* ray, float* len) {
  if (!s) return fail(TSP_EINVAL, "tsp_segments_export_transposed: NULL handle");
  if (!s->has_adj) return fail(TSP_EINVAL, "tsp_segments_export_transposed: lists built without the transpose");
  tsp_status st = check_device(s->device);
  if (st != TSP_OK) return st;
  if (vox_off)
    TSP_CUDA(cudaMemcpy(vox_off, s->adj.off, sizeof(int64_t) * size_t(s->V + 1), cudaMemcpyDeviceToHost));
  if (ray && s->n_segs) {
    TSP_CUDA(cudaMemcpy(ray, s->adj.idx, sizeof(uint32_t) * size_t(s->n_segs), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < s->n_segs; ++i) ray[i] &= ~HEAD;
  }
  if (len && s->n_segs) TSP_CUDA(cudaMemcpy(len, s->adj.len, sizeof(float) * size_t(s->n_segs), cudaMemcpyDeviceToHost));
  return TSP_OK;
}

extern "C" tsp_status tsp_segments_forward(tsp_segments s, const float* rho, float* y, int batch, void* stream) {
  TSP_RANGE("tsp_segments_forward");
  if (!s || !rho || !y || batch <= 0) return fail(TSP_EINVAL, "tsp_segments_forward: bad argument");
  tsp_status st = check_device(s->device);
  if (st != TSP_OK) return st;
  return rows_apply(s->fwd, rho, s->V, y, s->n_rays, batch, 0, static_cast<cudaStream_t>(stream));
}

extern "C" tsp_status tsp_segments_adjoint(tsp_segments s, const float* y, float* rho, int batch, int accumulate,
                                           void* stream) {
  TSP_RANGE("tsp_segments_adjoint");
  if (!s || !y || !rho || batch <= 0) return fail(TSP_EINVAL, "tsp_segments_adjoint: bad argument");
  tsp_status st = check_device(s->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (s->has_adj) return rows_apply(s->adj, y, s->n_rays, rho, s->V, batch, accumulate, cs);
  if (!accumulate) TSP_CUDA(cudaMemsetAsync(rho, 0, sizeof(float) * size_t(s->V) * batch, cs));
  for (int b = 0; b < batch; ++b)
    seg_scatter_kernel<<<unsigned((s->n_rays * 32 + 255) / 256), 256, 0, cs>>>(s->fwd.off, s->fwd.idx, s->fwd.len,
                                                                              y + b * s->n_rays, rho + b * s->V,
                                                                              s->n_rays);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_segments_sirt_workspace_bytes(tsp_segments s, size_t* bytes) {
  if (!s || !bytes) return fail(TSP_EINVAL, "tsp_segments_sirt_workspace_bytes: NULL argument");
  *bytes = 2 * align256(sizeof(float) * size_t(s->n_rays)) + 2 * align256(sizeof(float) * size_t(s->V));
  return TSP_OK;
}

// R = 1 / (F 1), C = 1 / (F^T 1) from the lists (0 where a sum is 0); ones_v
// [V] and ones_r [n_rays] are scratch.
static tsp_status list_weights(tsp_segments s, float* R, float* C, float* ones_v, float* ones_r, cudaStream_t cs) {
  const int64_t nr = s->n_rays, V = s->V;
  fill_kernel<<<ew_blocks(V), 256, 0, cs>>>(ones_v, V, 1.0f);
  tsp_status st = rows_apply(s->fwd, ones_v, V, R, nr, 1, 0, cs);
  if (st != TSP_OK) return st;
  recip_kernel<<<ew_blocks(nr), 256, 0, cs>>>(R, nr);
  fill_kernel<<<ew_blocks(nr), 256, 0, cs>>>(ones_r, nr, 1.0f);
  st = s->has_adj ? rows_apply(s->adj, ones_r, nr, C, V, 1, 0, cs) : tsp_segments_adjoint(s, ones_r, C, 1, 0, cs);
  if (st != TSP_OK) return st;
  recip_kernel<<<ew_blocks(V), 256, 0, cs>>>(C, V);
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

extern "C" tsp_status tsp_segments_sirt_weights(tsp_segments s, float* R, float* C, void* stream) {
  if (!s || !R || !C) return fail(TSP_EINVAL, "tsp_segments_sirt_weights: NULL argument");
  tsp_status st = check_device(s->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  float* ones = nullptr;
  const int64_t n = std::max<int64_t>(std::max(s->n_rays, s->V), 1);
  TSP_CUDA(cudaMallocAsync(&ones, sizeof(float) * size_t(n) * 2, cs));
  st = list_weights(s, R, C, ones, ones + n, cs);
  cudaFreeAsync(ones, cs);
  return st;
}

extern "C" tsp_status tsp_segments_sirt(tsp_segments s, const float* y, float* x, int n_iter, int flags,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  TSP_RANGE("tsp_segments_sirt");
  if (!s || !y || !x || !workspace) return fail(TSP_EINVAL, "tsp_segments_sirt: NULL argument");
  if (n_iter < 0) return fail(TSP_EINVAL, "tsp_segments_sirt: n_iter < 0");
  if (flags & ~(TSP_SIRT_NONNEG | TSP_SIRT_REUSE_WEIGHTS)) return fail(TSP_EINVAL, "tsp_segments_sirt: unknown flags");
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return fail(TSP_EINVAL, "tsp_segments_sirt: workspace not 256-byte aligned");
  size_t need = 0;
  tsp_segments_sirt_workspace_bytes(s, &need);
  if (workspace_bytes < need)
    return fail(TSP_EINVAL, "tsp_segments_sirt: workspace of " + std::to_string(workspace_bytes) + " bytes, " +
                                std::to_string(need) + " needed");
  tsp_status st = check_device(s->device);
  if (st != TSP_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int64_t nr = s->n_rays, V = s->V;
  char* p = static_cast<char*>(workspace);
  float* R = reinterpret_cast<float*>(p);
  float* r = reinterpret_cast<float*>(p + align256(4 * size_t(nr)));
  float* C = reinterpret_cast<float*>(p + 2 * align256(4 * size_t(nr)));
  float* g = reinterpret_cast<float*>(p + 2 * align256(4 * size_t(nr)) + align256(4 * size_t(V)));
  if (!(flags & TSP_SIRT_REUSE_WEIGHTS)) {
    st = list_weights(s, R, C, g, r, cs);
    if (st != TSP_OK) return st;
  }
  for (int it = 0; it < n_iter; ++it) {
    st = rows_apply(s->fwd, x, V, r, nr, 1, 0, cs);  // r = F x
    if (st != TSP_OK) return st;
    residual_kernel<<<ew_blocks(nr), 256, 0, cs>>>(r, y, R, nr);
    st = tsp_segments_adjoint(s, r, g, 1, 0, stream);  // g = F^T r
    if (st != TSP_OK) return st;
    xupdate_kernel<<<ew_blocks(V), 256, 0, cs>>>(x, g, C, V, flags & TSP_SIRT_NONNEG);
  }
  TSP_CUDA(cudaGetLastError());
  return TSP_OK;
}

// ---------------------------------------------------------------------------
// Chunked segment lists: SIRT over many independent reconstructions whose
// stored lists together exceed device memory. Lists are built for one chunk
// of instances at a time (as many, in order, as fit the byte budget), every
// iteration of those instances runs from the lists, and the chunk's lists
// are freed before the next chunk is built. Each instance gets the same
// iterates as tsp_segments_sirt on its own lists.
// ---------------------------------------------------------------------------
extern "C" tsp_status tsp_sirt_chunked(const tsp_batch_item* items, int n_items, int n_iter, int flags,
                                       size_t budget_bytes, int* n_chunks, size_t* peak_bytes, void* stream) {
  TSP_RANGE("tsp_sirt_chunked");
  if (!items || n_items <= 0) return fail(TSP_EINVAL, "tsp_sirt_chunked: no items");
  if (n_iter < 0) return fail(TSP_EINVAL, "tsp_sirt_chunked: n_iter < 0");
  if (flags & ~TSP_SIRT_NONNEG) return fail(TSP_EINVAL, "tsp_sirt_chunked: unknown flags");
  for (int i = 0; i < n_items; ++i)
    if (!items[i].grid || !items[i].geom || !items[i].y || !items[i].x)
      return fail(TSP_EINVAL, "tsp_sirt_chunked: item " + std::to_string(i) + " has a NULL member");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (budget_bytes == 0) {  // default: 80% of what is free now
    size_t free_b = 0, total_b = 0;
    TSP_CUDA(cudaMemGetInfo(&free_b, &total_b));
    budget_bytes = free_b / 10 * 8;
  }
  std::vector<tsp_segments> chunk;
  size_t used = 0, peak = 0, ws_bytes = 0;
  void* ws = nullptr;
  int chunks = 0;
  auto release = [&]() {
    for (tsp_segments s : chunk) tsp_segments_destroy(s);
    chunk.clear();
    used = 0;
  };
  auto run_chunk = [&](int first) -> tsp_status {  // items first .. first + chunk.size() - 1
    for (size_t k = 0; k < chunk.size(); ++k) {
      size_t need = 0;
      tsp_segments_sirt_workspace_bytes(chunk[k], &need);
      if (need > ws_bytes) {
        if (ws) cudaFree(ws);
        ws = nullptr;
        ws_bytes = 0;
        cudaError_t e = dev_malloc(&ws, need);
        if (e != cudaSuccess) return cuda_fail(e, "tsp_sirt_chunked: workspace");
        ws_bytes = need;
      }
      const tsp_batch_item& it = items[first + int(k)];
      tsp_status st = tsp_segments_sirt(chunk[k], it.y, it.x, n_iter, flags, ws, ws_bytes, stream);
      if (st != TSP_OK) return st;
    }
    ++chunks;
    return TSP_OK;
  };
  tsp_status st = TSP_OK;
  int first = 0;
  for (int i = 0; i < n_items && st == TSP_OK; ++i) {
    tsp_segments s = nullptr;
    st = tsp_segments_build(items[i].grid, items[i].geom, 1, &s, stream);
    if (st == TSP_ENOMEM && !chunk.empty()) {  // no room next to the chunk: finish it, then retry alone
      st = run_chunk(first);
      if (st == TSP_OK) {
        cudaError_t e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "tsp_sirt_chunked: sync");
      }
      release();
      first = i;
      if (st == TSP_OK) st = tsp_segments_build(items[i].grid, items[i].geom, 1, &s, stream);
    }
    if (st != TSP_OK) break;
    size_t b = 0;
    tsp_segments_info(s, nullptr, nullptr, &b);
    if (!chunk.empty() && used + b > budget_bytes) {  // over budget: run the chunk built so far first
      st = run_chunk(first);
      if (st == TSP_OK) {
        cudaError_t e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "tsp_sirt_chunked: sync");
      }
      release();
      first = i;
    }
    chunk.push_back(s);
    used += b;
    peak = std::max(peak, used);
  }
  if (st == TSP_OK && !chunk.empty()) {
    st = run_chunk(first);
    if (st == TSP_OK) {
      cudaError_t e = cudaStreamSynchronize(cs);
      if (e != cudaSuccess) st = cuda_fail(e, "tsp_sirt_chunked: sync");
    }
  }
  release();
  if (ws) cudaFree(ws);
  if (n_chunks) *n_chunks = chunks;
  if (peak_bytes) *peak_bytes = peak;
  return st;
}
