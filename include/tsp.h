/*
 * tsp.h - C ABI of the GB300 spherical-grid tomographic projector.
 *
 * The projector F maps a density rho, piecewise constant on a spherical grid,
 * to line integrals y along rays (TomoSphero, Sec. 2.1, Eq. 3-5); its adjoint
 * F^T scatters y * (segment length) back onto the voxels (Sec. 4.4).
 *
 * Conventions shared by every entry point
 *  - Grid: radial shells r_0 < ... < r_Nr, polar cones theta_0 < ... < theta_Ne
 *    (polar angle from +Z, in [0, pi]), azimuthal half-planes phi_0 < ... < phi_Na
 *    (span <= 2 pi; a span of exactly 2 pi wraps, phi_Na being phi_0).
 *    Bins are half-open [edge_k, edge_{k+1}). Density is zero outside the grid.
 *  - rho: float32, C-order (batch, N_r, N_e, N_a); flat voxel = (ir*N_e + ie)*N_a + ia.
 *  - y:   float32, (batch, n_views, H, W) for cone/parallel detectors,
 *         (batch, n_rays) for free-form rays.
 *  - All array pointers passed to projection calls are DEVICE pointers owned by
 *    the caller (e.g. torch tensors). Handles own copies of the geometry.
 *  - Calls run asynchronously on the given CUDA stream (NULL = legacy default
 *    stream) on the current device, which must be the device the handles were
 *    created on. No call synchronises the host except where stated.
 *  - Errors are returned as tsp_status, never thrown. tsp_last_error() gives a
 *    thread-local message for the last failure. A kernel that detects an
 *    internal inconsistency sets a device error word instead of trapping;
 *    tsp_device_status() reads and clears it.
 */
#ifndef TSP_H_
#define TSP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsp_grid_s* tsp_grid;
typedef struct tsp_geom_s* tsp_geom;

typedef enum {
  TSP_OK = 0,
  TSP_EINVAL = 1,     /* null pointer, size <= 0, out-of-range argument */
  TSP_ENOTMONO = 2,   /* grid edges not strictly increasing */
  TSP_ENOMEM = 3,     /* device or host allocation failed */
  TSP_ECUDA = 4,      /* a CUDA runtime call failed (message has the CUDA error) */
  TSP_ETIMEOUT = 5,   /* a bounded device wait gave up */
  TSP_EDEVICE = 6,    /* a kernel set the device error word */
  TSP_ENOTSUP = 7     /* size beyond a documented limit */
} tsp_status;

/* Limits of one grid: N_r, N_e <= 1024, N_a <= 2048, voxels < 2^31. */

/*
 * tsp_grid_create - spherical grid from its boundary locations (Sec. 2.2, 4.1;
 * Fig. 2-4). Edges are host arrays of n_*_edges = N + 1 doubles, copied.
 * r_edges >= 0; theta_edges within [0, pi]; phi span <= 2 pi. Grids that cover
 * a wedge only (Fig. 3) are allowed. Returns TSP_ENOTMONO for non-increasing
 * edges, TSP_EINVAL for other bad input. Synchronous (uploads small tables).
 */
tsp_status tsp_grid_create(const double* r_edges, int n_r_edges, const double* theta_edges,
                           int n_theta_edges, const double* phi_edges, int n_phi_edges,
                           tsp_grid* out);
tsp_status tsp_grid_shape(tsp_grid grid, int* n_r, int* n_e, int* n_a);
void tsp_grid_destroy(tsp_grid grid);

/*
 * tsp_geom_cone - cone-beam views (Sec. 4.2 ConeRectGeom, Sec. 4.3 collections):
 * a pinhole detector at each pos (host, [n_views][3]) looking at look_at
 * (host [n_views][3], NULL = origin), with up hint (NULL = +Z, +Y if parallel
 * to the view axis). H x W pixel centres uniform in tangent space over the full
 * field of view fov_h_deg x fov_w_deg (degrees). Row 0 is at +up, column 0 at
 * -right (right = look x up). Ray i = (view*H + row)*W + col.
 */
tsp_status tsp_geom_cone(int n_views, const double* pos, const double* look_at, const double* up,
                         int H, int W, double fov_h_deg, double fov_w_deg, tsp_geom* out);

/*
 * tsp_geom_parallel - parallel-beam views (Sec. 4.2 ParallelGeom): a detector
 * plane through pos, perpendicular to the direction pos -> origin, of physical
 * size size_h x size_w, H x W pixels; every ray runs along that direction.
 */
tsp_status tsp_geom_parallel(int n_views, const double* pos, const double* up, int H, int W,
                             double size_h, double size_w, tsp_geom* out);

/*
 * tsp_geom_rays - free-form rays (Sec. 4.2 ViewGeom, Listing 4): DEVICE arrays
 * starts[3][n_rays] and dirs[3][n_rays] (structure of arrays, float32).
 * Directions need not be normalised; they are normalised in-kernel. A zero
 * direction yields y = 0 for that ray. copy != 0 copies the arrays (synchronous);
 * copy == 0 keeps the caller's pointers, which must outlive the handle.
 */
tsp_status tsp_geom_rays(int64_t n_rays, const float* starts, const float* dirs, int copy,
                         tsp_geom* out);
/*
 * tsp_geom_polar - polar-binned detectors (Sec. 6: images binned to n_rad
 * radial x n_az azimuthal polar pixels of an equivalent field of view): per
 * view a pinhole at pos looking at look_at (origin if NULL) with up hint up
 * (+Z if NULL; frame as tsp_geom_cone). Pixel (i, j) looks at the angle
 * (i + 1/2) / n_rad * fov_deg / 2 from the boresight, at azimuth
 * 2 pi (j + 1/2) / n_az from the right axis toward up. Rays are ordered
 * (view, i, j); the geometry has n_views views of n_rad x n_az rays, so the
 * dynamic projections see one volume per view. fov_deg in (0, 180).
 */
tsp_status tsp_geom_polar(int n_views, const double* pos, const double* look_at, const double* up, int n_rad,
                          int n_az, double fov_deg, tsp_geom* out);
tsp_status tsp_geom_num_rays(tsp_geom geom, int64_t* n_rays);
void tsp_geom_destroy(tsp_geom geom);

/* Launch knobs (chosen by tsp_autotune or set by hand). */
typedef struct {
  int block_threads;   /* threads per block: 64, 128, 256 or 512 */
  int warp_tile_w;     /* detector pixels per warp along a row: 4, 8, 16 or 32 */
  int scatter;         /* adjoint: 0 = one atomic add per segment, 1 = warp-aggregated: a lane
                          and its neighbour (lane ^ 1) on the same voxel in the same step add
                          their sum with one atomic */
} tsp_launch;

/*
 * tsp_forward - y = F rho (Eq. 5) for `batch` densities. rho: device float32
 * (batch, N_r, N_e, N_a); y: device float32 (batch, n_rays), overwritten.
 * Every segment of every ray is found in-kernel (Sec. 3.1-3.3) and gathered
 * (Sec. 3.4); nothing is precomputed. launch may be NULL (defaults).
 */
tsp_status tsp_forward(tsp_grid grid, tsp_geom geom, const float* rho, float* y, int batch,
                       void* stream);
tsp_status tsp_forward_ex(tsp_grid grid, tsp_geom geom, const float* rho, float* y, int batch,
                          const tsp_launch* launch, void* stream);

/*
 * tsp_adjoint - rho (+)= F^T y (adjoint of Eq. 5; Sec. 4.4). y: device float32
 * (batch, n_rays); rho: device float32 (batch, N_r, N_e, N_a). accumulate == 0
 * overwrites rho, otherwise adds to it. The traversal is bit-identical to
 * tsp_forward's, so <F x, y> = <x, F^T y> up to float32 summation order.
 */
tsp_status tsp_adjoint(tsp_grid grid, tsp_geom geom, const float* y, float* rho, int batch,
                       int accumulate, void* stream);
tsp_status tsp_adjoint_ex(tsp_grid grid, tsp_geom geom, const float* y, float* rho, int batch,
                          int accumulate, const tsp_launch* launch, void* stream);

/*
 * Dynamic objects (Sec. 4.4: an Operator called with a 4D object; Sec. 4.3,
 * 4.6: a collection of views taken in sequence while the grid stays fixed):
 * view k of geom (k = 0 .. n_views - 1, each H x W rays; free-form rays are
 * one view) sees volume k.
 * tsp_forward_dynamic - y[k] = F_k rho[k]. rho: device float32 (n_views, N_r,
 *   N_e, N_a); y: device float32 (n_views, H, W), overwritten.
 * tsp_adjoint_dynamic - rho[k] (+)= F_k^T y[k]; accumulate as tsp_adjoint.
 * Same traversal as tsp_forward / tsp_adjoint (bit-identical segments).
 */
tsp_status tsp_forward_dynamic(tsp_grid grid, tsp_geom geom, const float* rho, float* y, void* stream);
tsp_status tsp_adjoint_dynamic(tsp_grid grid, tsp_geom geom, const float* y, float* rho, int accumulate,
                               void* stream);

/*
 * tsp_count_segments - counts[i] = number of valid segments of ray i (pieces
 * of the ray inside the grid with an in-range voxel index: the non-zero rows
 * of Table 2c). counts: device int32 [n_rays], overwritten.
 */
tsp_status tsp_count_segments(tsp_grid grid, tsp_geom geom, int* counts, void* stream);

/*
 * Precomputed segment lists (Sec. 3: steps 1-3 done once and stored, step 4
 * repeated; Sec. 4.4's stored region indices and lengths). The lists are the
 * valid segments only (Table 2c's zeroed rows dropped), 8 bytes each: uint32
 * flat voxel index r*N_e*N_a + e*N_a + a and float32 length, ray-major in
 * order along each ray. With transpose != 0 the build also stores the same
 * segments voxel-major (uint32 ray index, float32 length), so that the
 * adjoint is a per-voxel gather instead of a per-segment scatter. The
 * transpose is a stable radix sort by voxel (8 key bits per pass), so each
 * voxel's list is in ray-major order and the lists, and every result computed
 * from them, are the same on every build; it takes about 18 bytes per segment of
 * temporary device memory during the build.
 *
 * The segments are those tsp_forward walks: lists and on-the-fly traversal
 * give the same F up to float32 rounding order. Forward and adjoint read the
 * lists once per call, coalesced, and sum each ray (voxel) in a fixed order
 * without atomics, so repeated calls on the same lists give identical
 * results. Memory: 8 bytes per segment (16 with transpose) plus at most 12
 * bytes per ray (and per voxel) and 17 bytes per 256 segments per direction;
 * tsp_segments_info reports it. A handle holds per-call scratch: calls on one
 * handle must not run concurrently on different streams. Limits: fewer than
 * 2^31 rays and voxels, fewer than 2^32 segments (TSP_ENOTSUP).
 */
typedef struct tsp_segments_s* tsp_segments;

/*
 * tsp_segments_build - traverses every ray of geom twice (count, then fill)
 * and builds the lists on grid's device. Synchronises `stream` (it reads the
 * total segment count back to size the lists). *out receives the handle, or
 * NULL on error. TSP_ENOMEM/TSP_ECUDA on allocation or launch failure.
 */
tsp_status tsp_segments_build(tsp_grid grid, tsp_geom geom, int transpose, tsp_segments* out,
                              void* stream);
/* n_rays, n_segments: counts; bytes: device memory held. Any may be NULL. */
tsp_status tsp_segments_info(tsp_segments s, int64_t* n_rays, int64_t* n_segments, size_t* bytes);
/*
 * tsp_segments_export - copies the ray-major lists to HOST buffers (any may be
 * NULL): ray_off int64 [n_rays + 1] (segments of ray i are [ray_off[i],
 * ray_off[i+1])), vox uint32 [n_segments], len float32 [n_segments].
 * Synchronous.
 */
tsp_status tsp_segments_export(tsp_segments s, int64_t* ray_off, uint32_t* vox, float* len);
/*
 * tsp_segments_export_transposed - copies the voxel-major lists (built with
 * transpose != 0) to HOST buffers (any may be NULL): vox_off int64 [V + 1]
 * (entries of voxel v are [vox_off[v], vox_off[v+1]), V = N_r N_e N_a), ray
 * uint32 [n_segments], len float32 [n_segments]. The transpose is a stable
 * radix sort of the ray-major entries by voxel, so each voxel's entries are
 * in ray-major order (by ray, then along the ray) and every build of the same
 * grid and geometry gives the same lists. Synchronous. TSP_EINVAL if the
 * handle has no voxel-major lists.
 */
tsp_status tsp_segments_export_transposed(tsp_segments s, int64_t* vox_off, uint32_t* ray, float* len);
/*
 * tsp_segments_forward - y = F rho (Eq. 5) from the stored lists, one pass
 * over the lists per density. Shapes as tsp_forward; y overwritten.
 */
tsp_status tsp_segments_forward(tsp_segments s, const float* rho, float* y, int batch, void* stream);
/*
 * tsp_segments_adjoint - rho (+)= F^T y from the stored lists: a gather over
 * the voxel-major lists when the handle has them, else one atomic add per
 * segment from the ray-major lists. Shapes and accumulate as tsp_adjoint.
 */
tsp_status tsp_segments_adjoint(tsp_segments s, const float* y, float* rho, int batch, int accumulate,
                                void* stream);
/*
 * tsp_segments_sirt - tsp_sirt (same update, weights and flags) with every
 * projection taken from the stored lists. The workspace needs
 * tsp_segments_sirt_workspace_bytes() bytes (the same as tsp_sirt's for the
 * grid and geometry the lists were built from), 256-byte aligned; with
 * TSP_SIRT_REUSE_WEIGHTS it must hold the weights of an earlier call on the
 * same lists. Per iteration: forward, residual, adjoint, update (plus the
 * lists' fixup and memset launches). No host synchronisation.
 */
tsp_status tsp_segments_sirt_workspace_bytes(tsp_segments s, size_t* bytes);
/*
 * tsp_segments_sirt_weights - the SIRT weights of tsp_sirt_weights from the
 * stored lists: R = 1/(F 1) per ray (device float32 [n_rays]) and
 * C = 1/(F^T 1) per voxel (device float32 [voxels]), 0 where the sum is 0,
 * as tsp_segments_sirt computes them. With the voxel-major lists every sum
 * runs in the lists' fixed order, so the weights are identical on every call
 * and every build (tsp_sirt_weights sums with atomics). Allocates and frees
 * 8 * max(n_rays, voxels) bytes of scratch in stream order.
 */
tsp_status tsp_segments_sirt_weights(tsp_segments s, float* R, float* C, void* stream);
/*
 * tsp_debug_fail_allocation - test hook: the device allocation `after`
 * allocations from now (0: the next one) made by the stored-list code
 * (tsp_segments_build, tsp_sirt_chunked) fails once as if the device were out
 * of memory; a negative value disarms it. Lets tests drive the out-of-memory
 * paths (TSP_ENOMEM, the chunked driver's finish-and-retry) without
 * exhausting a GPU. tsp_debug_allocation_count gives the number of such
 * allocations made so far (to aim the hook). Process-wide, not thread-safe
 * with respect to concurrent builds.
 */
tsp_status tsp_debug_fail_allocation(int64_t after);
tsp_status tsp_debug_allocation_count(int64_t* count);
tsp_status tsp_segments_sirt(tsp_segments s, const float* y, float* x, int n_iter, int flags,
                             void* workspace, size_t workspace_bytes, void* stream);
void tsp_segments_destroy(tsp_segments s);

/*
 * Attenuated projection (Sec. 9.3, Eq. 14-18): the optically thin model with
 * the first-order losses of photons from the sun to the scattering point
 * (optical depth tau_1, Eq. 14) and from there to the observer (tau_2, Eq. 15):
 *
 *   y = sum_i rho[v_i] e^{-tau_1[v_i]} e^{-tau_2,i} dl_i                 (Eq. 17)
 *   tau_2,i = sum_{j <= i} sigma[v_j] rho[v_j] dl_j  (inclusive cumsum, Eq. 18)
 *   tau_1 = F_1(sigma rho)                                                (Eq. 17)
 *
 * Segments i are the maximal runs of a ray in one voxel, in order from the
 * ray's start (consecutive pieces of one voxel are joined; pieces separated
 * by a stretch outside the grid stay apart). F_1 traces one ray per voxel
 * from its centroid toward the sun (Fig. 16b). sigma (the cross-section) and
 * rho are device float32 (batch, N_r, N_e, N_a); tau_1 has the same shape.
 *
 * tsp_sunward_rays - F_1's rays: for every voxel (flat order) its centroid
 *   (the point at the midpoints of its r, theta, phi edges) and the unit sun
 *   direction; sun is a host double[3] pointing toward the sun (non-zero).
 *   starts, dirs: device float32 [3][N_r N_e N_a], written. Pass them to
 *   tsp_geom_rays to get F_1's geometry.
 * tsp_atten_optical_depth - tau_1 = F_1(sigma rho) (one value per voxel);
 *   `sun` is a geometry with one ray per voxel (TSP_EINVAL otherwise).
 * tsp_atten_optical_depth_adjoint - g_rho (+)= sigma F_1^T g_tau1 and, if
 *   g_sigma != NULL, g_sigma (+)= rho F_1^T g_tau1; accumulate == 0
 *   overwrites the outputs, otherwise adds to them.
 * tsp_atten_forward - y (batch, n_rays) by Eq. 17-18, overwritten.
 * tsp_atten_backward - gradients of sum y gy with respect to rho, sigma and
 *   tau_1 (tau_1 taken as an independent input) into g_rho and, when not NULL,
 *   g_sigma and g_tau1; accumulate as above. y must be tsp_atten_forward's output for
 *   the same inputs (its running prefix is reused). Chain through tau_1 with
 *   tsp_atten_optical_depth_adjoint(g_tau1).
 * All of them traverse on the fly like tsp_forward and scatter with atomic
 * adds; errors as tsp_forward.
 */
tsp_status tsp_sunward_rays(tsp_grid grid, const double* sun, float* starts, float* dirs, void* stream);
tsp_status tsp_atten_optical_depth(tsp_grid grid, tsp_geom sun, const float* rho, const float* sigma, float* tau1,
                                   int batch, void* stream);
tsp_status tsp_atten_optical_depth_adjoint(tsp_grid grid, tsp_geom sun, const float* rho, const float* sigma,
                                           const float* g_tau1, float* g_rho, float* g_sigma, int batch,
                                           int accumulate, void* stream);
tsp_status tsp_atten_forward(tsp_grid grid, tsp_geom geom, const float* rho, const float* sigma, const float* tau1,
                             float* y, int batch, void* stream);
tsp_status tsp_atten_backward(tsp_grid grid, tsp_geom geom, const float* rho, const float* sigma,
                              const float* tau1, const float* y, const float* gy, float* g_rho, float* g_sigma,
                              float* g_tau1, int batch, int accumulate, void* stream);

/*
 * tsp_autotune - times candidate launch knobs (threads per block 64..512, warp
 * tiles 4..32 pixels wide, and for the adjoint the scatter strategy) for this
 * grid and geometry, and caches the fastest per size class (each grid and
 * detector dimension rounded up to a power of two). Calls made afterwards
 * without explicit knobs (launch == NULL) on a grid and geometry of the same
 * class use the cached choice. Synchronous: allocates and frees temporary
 * device buffers of one volume and one detector, launches each candidate
 * three times. fwd / adj receive the choices (may be NULL).
 */
tsp_status tsp_autotune(tsp_grid grid, tsp_geom geom, tsp_launch* fwd, tsp_launch* adj, void* stream);
/* Cached choice for this size class, or TSP_ENOTSUP if it was never tuned. */
tsp_status tsp_autotune_lookup(tsp_grid grid, tsp_geom geom, tsp_launch* fwd, tsp_launch* adj);
/*
 * Store fwd / adj as the cached choice for this size class, as if tuned (no
 * timing, nothing launched): pins the knobs of later calls without explicit
 * ones, for reproducible runs or to select a scatter strategy. Replaces an
 * earlier choice. TSP_EINVAL for NULL handles or knobs outside the ranges of
 * tsp_launch.
 */
tsp_status tsp_autotune_store(tsp_grid grid, tsp_geom geom, const tsp_launch* fwd, const tsp_launch* adj);
/* Forget every cached choice. */
void tsp_autotune_clear(void);

/*
 * SIRT - simultaneous iterative reconstruction (the paper cites it among the
 * algorithms its operator serves, Sec. 1 ref. [10]; standard definition):
 *   R = 1 / (F 1), C = 1 / (F^T 1)  (0 where the sum is 0)
 *   x <- x + C * F^T( R * (y - F x) )   repeated n_iter times.
 * y: device float32 (n_rays) measurements; x: device float32 (N_r, N_e, N_a),
 * the starting point on entry and the result on exit.
 * workspace: caller-owned DEVICE scratch of at least tsp_sirt_workspace_bytes()
 * bytes, 256-byte aligned; it holds R, C, the residual and the back-projection.
 * flags: TSP_SIRT_NONNEG clamps x at 0 after every update;
 * TSP_SIRT_REUSE_WEIGHTS skips recomputing R and C, which a previous call with
 * the same grid, geometry and workspace left in the workspace.
 * Enqueues 3 kernels per iteration (plus 3 for the weights and 2 memsets) on
 * `stream`; no host synchronisation.
 */
#define TSP_SIRT_NONNEG 1
#define TSP_SIRT_REUSE_WEIGHTS 2
tsp_status tsp_sirt_workspace_bytes(tsp_grid grid, tsp_geom geom, size_t* bytes);
tsp_status tsp_sirt(tsp_grid grid, tsp_geom geom, const float* y, float* x, int n_iter, int flags,
                    void* workspace, size_t workspace_bytes, const tsp_launch* launch, void* stream);

/*
 * tsp_sirt_noalloc - tsp_sirt without a caller workspace and without any
 * device allocation. (An addition of this library; the paper has no
 * counterpart.) It is for callers that cannot call cudaMalloc: onboard or
 * real-time reconstruction code bound to a memory budget fixed at start-up,
 * pipelines where an allocation's implicit synchronisation would stall
 * latency-critical work, and hosts whose own allocator owns the device pool.
 * The scratch lives in a static device array of TSP_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that every GPU loading this library holds until the process exits;
 * a grid and geometry needing more (about n_rays + voxels > 4.19 million)
 * return TSP_ENOTSUP with the size in the message, and allocate nothing.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any CUDA
 * stream capture. Every call on a device shares the array and leaves its
 * contents behind; each call clears what must start at zero and recomputes
 * the SIRT weights, so flags accepts TSP_SIRT_NONNEG only. Calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array.
 * Arguments and results are otherwise those of tsp_sirt.
 */
#define TSP_NOALLOC_SCRATCH_BYTES (32u << 20)
tsp_status tsp_sirt_noalloc(tsp_grid grid, tsp_geom geom, const float* y, float* x, int n_iter, int flags,
                            void* stream);

/*
 * Batched SIRT over many independent reconstructions of uneven sizes (each
 * item its own grid, geometry, measurements y and volume x; device pointers
 * owned by the caller, valid for the batch's lifetime). Each SIRT stage runs
 * as one persistent launch over all items: blocks take (item, detector tile)
 * work from an atomic counter. Per item, the warp tile and scatter strategy
 * come from tsp_autotune's cache for its size class (defaults otherwise); the
 * block size from the item with the most rays.
 *   tsp_batch_create         - host-side plan (synchronous; small upload).
 *   tsp_batch_workspace_bytes- device scratch for n_iter iterations: R and the
 *                              residual per ray, C and the back-projection per
 *                              voxel, stage counters; 256-byte aligned.
 *   tsp_batch_sirt           - enqueue weights + n_iter iterations on stream.
 *   tsp_batch_sirt_capture   - capture that schedule once into a CUDA graph
 *                              (on a private stream) bound to this workspace;
 *   tsp_batch_sirt_launch    - replay it with one graph launch on stream.
 * Each run starts from the items' current x. flags: TSP_SIRT_NONNEG only.
 */
typedef struct tsp_batch_s* tsp_batch;
typedef struct {
  tsp_grid grid;
  tsp_geom geom;
  const float* y;
  float* x;
} tsp_batch_item;
tsp_status tsp_batch_create(const tsp_batch_item* items, int n_items, tsp_batch* out);
tsp_status tsp_batch_workspace_bytes(tsp_batch batch, int n_iter, size_t* bytes);
tsp_status tsp_batch_sirt(tsp_batch batch, int n_iter, int flags, void* workspace, size_t workspace_bytes,
                          void* stream);
tsp_status tsp_batch_sirt_capture(tsp_batch batch, int n_iter, int flags, void* workspace, size_t workspace_bytes);
tsp_status tsp_batch_sirt_launch(tsp_batch batch, void* stream);
tsp_status tsp_batch_info(tsp_batch batch, int64_t* total_rays, int64_t* total_voxels, int* block_threads);
void tsp_batch_destroy(tsp_batch batch);

/*
 * tsp_sirt_chunked - SIRT (as tsp_segments_sirt, n_iter iterations from the
 * x given, flags 0 or TSP_SIRT_NONNEG) over n_items independent
 * reconstructions (grid, geom, y, x as in tsp_batch_item) from stored lists
 * whose total exceeds device memory: lists (with the transpose) are built
 * for a chunk of consecutive items that fits budget_bytes (0: 80% of the
 * free device memory), every iteration of those items runs from them, and
 * they are freed before the next chunk (an item whose lists do not fit next
 * to the chunk starts a new one). Synchronous (the builds read segment
 * counts back). n_chunks, peak_bytes (either may be NULL) receive the
 * number of chunks and the largest list memory held at once.
 * TSP_ENOMEM if one item's lists alone do not fit.
 */
tsp_status tsp_sirt_chunked(const tsp_batch_item* items, int n_items, int n_iter, int flags, size_t budget_bytes,
                            int* n_chunks, size_t* peak_bytes, void* stream);

/*
 * Parametric density model for reconstructions that differentiate through F
 * (Sec. 4.5 Eq. 7 and Listing 8; Sec. 6 Eq. 10 uses spherical harmonics per
 * shell): rho[ir][ie][ia] = sum_j sum_q B[ir][j] c[j][q] Y[ie,ia][q] with B the
 * n_basis_r clamped cubic B-splines on [r_min, r_max] (uniform interior knots)
 * and Y the real orthonormal spherical harmonics of degree <= L, q = l^2+l+m.
 * Bases are evaluated on the host (double) at the given voxel-centre
 * coordinates (host arrays) and kept on the device as float32 tables.
 * coeffs / grad_coeffs: device float32 [n_basis_r][(L+1)^2]; rho / grad_rho:
 * device float32 (N_r, N_e, N_a). The handle owns a small scratch buffer, so
 * render calls on one handle must not overlap on the GPU.
 * tsp_shbs_tables copies the float32 tables to host arrays (either may be
 * NULL): B [N_r][n_basis_r], Yt [(L+1)^2][N_e*N_a].
 */
typedef struct tsp_shbs_s* tsp_shbs;
tsp_status tsp_shbs_create(int n_basis_r, int L, const double* r_centres, int n_r, const double* theta_centres,
                           int n_e, const double* phi_centres, int n_a, double r_min, double r_max, tsp_shbs* out);
tsp_status tsp_shbs_tables(tsp_shbs model, float* B, float* Yt);
tsp_status tsp_shbs_render(tsp_shbs model, const float* coeffs, float* rho, void* stream);
tsp_status tsp_shbs_render_adjoint(tsp_shbs model, const float* grad_rho, float* grad_coeffs, void* stream);
/*
 * tsp_shbs_create_shells - the per-shell model of Eq. 10:
 * rho[ir, ie, ia] = sum_q coeffs[ir][q] Y_q(theta_ie, phi_ia), one harmonic
 * series per shell (the same handle type with the identity as radial basis:
 * coeffs is [N_r][(L+1)^2]; render / render_adjoint / tables as above).
 */
tsp_status tsp_shbs_create_shells(int L, int n_r, const double* theta_centres, int n_e, const double* phi_centres,
                                  int n_a, tsp_shbs* out);
void tsp_shbs_destroy(tsp_shbs model);

/*
 * tsp_adam - one Adam step (Kingma and Ba 2015) on n float32 device values:
 * g' = g + weight_decay * p; m = b1 m + (1-b1) g'; v = b2 v + (1-b2) g'^2;
 * p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). step >= 1.
 */
tsp_status tsp_adam(float* params, const float* grads, float* m, float* v, int64_t n, float lr, float beta1,
                    float beta2, float eps, float weight_decay, int step, void* stream);

/*
 * tsp_sq_residual - squared-error loss of Eq. 6: loss += sum (yhat - y)^2
 * (device double, accumulated: zero it first) and, if grad != NULL,
 * grad = 2 (yhat - y) (device float32, n values).
 */
tsp_status tsp_sq_residual(const float* yhat, const float* y, int64_t n, float* grad, double* loss, void* stream);

/*
 * tsp_tikhonov_radial - the regulariser of Eq. 10, lambda ||D_r c||^2 with
 * D_r the first difference between neighbouring shells of every
 * coefficient: coeffs device float32 [n_r][n_q]; loss += the value (device
 * double, accumulated; may be NULL); grad += its gradient (device float32
 * [n_r][n_q], accumulated; may be NULL). lambda >= 0.
 * tsp_sq_residual_weighted - the data term of Eq. 10 with Eq. 9's known
 * per-ray factor w = (g / 4 pi) phi(n): loss += sum (w yhat - y)^2 (device
 * double, accumulated) and, if grad != NULL, grad = 2 w (w yhat - y), where
 * yhat = F rho is the plain line integral.
 */
tsp_status tsp_tikhonov_radial(const float* coeffs, int n_r, int n_q, float lambda, float* grad, double* loss,
                               void* stream);
tsp_status tsp_sq_residual_weighted(const float* yhat, const float* w, const float* y, int64_t n, float* grad,
                                    double* loss, void* stream);

/*
 * Vector kernels of the iterative solvers (device float32 vectors of n
 * values): tsp_vec_dot - out += sum x y (device double, accumulated: zero it
 * first); tsp_vec_axpby - y = a x + b y; tsp_vec_mul - out = w x
 * (elementwise; out may alias x).
 */
tsp_status tsp_vec_dot(const float* x, const float* y, int64_t n, double* out, void* stream);
tsp_status tsp_vec_axpby(float a, const float* x, float b, float* y, int64_t n, void* stream);
tsp_status tsp_vec_mul(const float* w, const float* x, float* out, int64_t n, void* stream);

/*
 * Learned warm start: a residual 3D convolutional network on the spherical grid
 * (3x3x3 kernels; zero padding in r and theta, periodic in phi):
 *   h1 = relu(conv(a; w1) + b1)                  1 -> 32 channels
 *   h_k = h_{k-1} + relu(conv(h_{k-1}; wk) + bk)  32 -> 32, k = 2..5 (tensor cores)
 *   out = a + conv(h5; w6) + b6                  32 -> 1
 * bfloat16 weights and activations, float32 accumulation, float32 master
 * weights updated by Adam. (The paper has no network; it names learned and
 * physics-informed uses of the differentiable operator, Sec. 4.5.)
 * Parameters (float32, flat): w1 [27][32][1], b1 [32], w2..w5 [27][32][32],
 * b2..b5 [32], w6 [27][1][32], b6 [1]; tap = (dr+1)*9 + (de+1)*3 + (da+1).
 * Volumes a, target, out: device float32 [batch][N_r][N_e][N_a].
 * tsp_net_create allocates the parameters, Adam moments and the activations
 * of max_batch samples (about 224 bytes per voxel and sample); N_a must be a
 * multiple of 32 in [32, 192]. Calls on one net must not overlap on the GPU.
 *   tsp_net_forward   - out = net(a).
 *   tsp_net_loss_grad - mean squared error against target and its gradient
 *                       w.r.t. every parameter (kept in the net; synchronous if
 *                       loss != NULL, which receives the loss).
 *   tsp_net_adam      - one Adam step of the parameters with those gradients.
 *   tsp_net_activation- copy h_{layer+1} (bfloat16 [batch][V][32], layer 0..4)
 *                       or out (layer 5) to a host buffer (synchronous).
 */
typedef struct tsp_net_s* tsp_net;
tsp_status tsp_net_create(int n_r, int n_e, int n_a, int max_batch, tsp_net* out);
void tsp_net_destroy(tsp_net net);
tsp_status tsp_net_num_params(tsp_net net, size_t* count);
tsp_status tsp_net_set_params(tsp_net net, const float* host_params, size_t count);
tsp_status tsp_net_get_params(tsp_net net, float* host_params, size_t count);
tsp_status tsp_net_get_grads(tsp_net net, float* host_grads, size_t count);
/*
 * tsp_net_get_state / tsp_net_set_state - the whole training state, for
 * checkpoint and resume: parameters, Adam's first and second moments (HOST
 * float32 [count] each, count = tsp_net_num_params) and the Adam step
 * counter. Both synchronise the device. set_state replaces all of it, so the
 * next tsp_net_adam continues the optimiser exactly where get_state found it:
 * a resumed training run repeats an uninterrupted one bit for bit (given the
 * same data). TSP_EINVAL on a count mismatch or a negative step.
 */
tsp_status tsp_net_get_state(tsp_net net, float* params, float* m, float* v, size_t count, int* adam_step);
tsp_status tsp_net_set_state(tsp_net net, const float* params, const float* m, const float* v, size_t count,
                             int adam_step);
tsp_status tsp_net_forward(tsp_net net, const float* a, int batch, float* out, void* stream);
tsp_status tsp_net_loss_grad(tsp_net net, const float* a, const float* target, int batch, double* loss, void* stream);
tsp_status tsp_net_adam(tsp_net net, float lr, float beta1, float beta2, float eps, float weight_decay, void* stream);
tsp_status tsp_net_activation(tsp_net net, int layer, int batch, void* host);

/*
 * tsp_sirt_weights - the SIRT weights alone: R = 1/(F 1) per ray (device float32
 * [n_rays]) and C = 1/(F^T 1) per voxel (device float32 [voxels]), 0 where the
 * sum is 0. Used to form the warm start's input C * F^T(R * y) when it runs
 * without stored lists (with them, tsp_segments_sirt_weights). F^T 1 sums
 * with atomics, so C may differ in its last bits between calls.
 */
tsp_status tsp_sirt_weights(tsp_grid grid, tsp_geom geom, float* R, float* C, void* stream);

/*
 * Data pipeline of the learned warm start (synthetic training data).
 * tsp_phantoms  - rho[b] = exp(-r/H_b) + sum_j A_j exp(-|p - c_j|^2 / (2 s_j^2)) at
 *                 the voxel centres (arithmetic midpoints of the edges); params:
 *                 device float32 [batch][rows][5], row 0 = (H, 0, 0, 0, 0), each
 *                 further row a blob (c_x, c_y, c_z, A, s); rho [batch][voxels].
 * tsp_batch_max - out[b] = max_i x[b][i] (device float32 [batch]).
 * tsp_add_noise - y[b][i] += frac * max_i y[b][i] * z_i with z_i standard normal
 *                 from SplitMix64 on the counter seeds[b] + (i+1)*golden and
 *                 Box-Muller over the sample (z_i uses draws i and n+i);
 *                 seeds: device uint64 [batch]; ymax receives the per-sample max.
 * tsp_mul_bcast - x[b][i] *= s[i].
 * tsp_scale_batch - x[b][i] /= scale[b] (divide != 0) or *= scale[b]; scale 0
 *                 leaves the sample unchanged.
 * All device pointers; asynchronous on stream.
 */
tsp_status tsp_phantoms(tsp_grid grid, const float* params, int rows, int batch, float* rho, void* stream);
tsp_status tsp_batch_max(const float* x, int64_t n, int batch, float* out, void* stream);
tsp_status tsp_add_noise(float* y, int64_t n, int batch, const uint64_t* seeds, float frac, float* ymax,
                         void* stream);
tsp_status tsp_mul_bcast(float* x, const float* s, int64_t n, int batch, void* stream);
tsp_status tsp_scale_batch(float* x, const float* scale, int64_t n, int batch, int divide, void* stream);

/* Bits of the device error word (tsp_device_status). */
#define TSP_DEVERR_STEP_CAP 0x1        /* a traversal hit its step cap */
#define TSP_DEVERR_LIST_BOUND 0x2      /* a list fill wrote other than its counted entries */
#define TSP_DEVERR_LIST_ROWS 0x8       /* a list stream found a row rank outside the lists */
#define TSP_DEVERR_WAIT_TIMEOUT 0x100  /* a tensor-core kernel's bounded mbarrier wait gave up */
#define TSP_DEVERR_SMEM_ALIGN 0x200    /* a tensor-core kernel got misaligned shared memory */

/*
 * tsp_device_status - synchronises `stream`, then reads and clears the device
 * error word (0 = no kernel reported an inconsistency). Returns TSP_ETIMEOUT
 * if TSP_DEVERR_WAIT_TIMEOUT is set: the kernel gave up its waits, released
 * its tensor memory and returned, so the context stays usable but that
 * kernel's output is incomplete. Any other bit gives TSP_EDEVICE.
 */
tsp_status tsp_device_status(void* stream, int* code);

/*
 * tsp_debug_tc_stall - test hook (no counterpart in the paper): the next
 * launch of the tensor-core convolution (a tsp_net_* call) runs with its
 * shell loader stalled, issuing no copy at all, and with every bounded wait
 * limited to wait_cycles SM cycles (1 .. 2e9; the default bound is 2e9). Its
 * first wait for a shell therefore runs out: the kernel sets
 * TSP_DEVERR_WAIT_TIMEOUT, frees its tensor memory and returns with nothing
 * in flight, and tsp_device_status reports TSP_ETIMEOUT. One-shot and
 * process-wide; later launches run normally.
 */
tsp_status tsp_debug_tc_stall(int64_t wait_cycles);

/* Thread-local message describing the last non-OK status of this thread. */
const char* tsp_last_error(void);

/* Library version, for the binding's load check. */
int tsp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSP_H_ */
