/*
 * ohm_gb.h - C ABI of the GB300 (sm_103a) ray-integration library.
 *
 * The library integrates ray sets -- (sensor origin, sample) pairs -- into a
 * sparse voxel map, as in "OHM: GPU Based Occupancy Map Generation" (arxiv
 * 2206.06079).  Space is cut into regions of 32^3 voxels found through a hash
 * table (Sec. III-A); every ray is walked voxel by voxel (Sec. III-B, the
 * Amanatides & Woo traversal) applying a clamped log-odds "miss" to each voxel
 * it passes through and a "hit" to the voxel holding its sample (Eq. 2-3,
 * Sec. II-B), and the optional layers of Sec. II-D/F and III-C ride on the same
 * walk: per-voxel hit/miss counts, NDT-OM sample moments (mean/covariance), and
 * a TSDF weighted average.
 *
 * Conventions shared by every entry point:
 *  - Ownership: the caller owns every input and output buffer; the library owns
 *    the map's memory (allocated on the map's device at ohm_map_create).
 *  - Pointers: unless an entry point says otherwise, an array argument may be
 *    device memory or host memory; the library detects which and copies host
 *    data through its own device staging buffers.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is ordered on that stream.
 *  - Errors: every entry point returns an ohm_status; on failure the message is
 *    available from ohm_last_error() (thread-local, valid until the next call
 *    on that thread).  No failure traps or hangs a kernel: device loops are
 *    bounded and report through a status word in device memory.
 *  - Fixed point: world coordinates become integers with `frac_bits` fraction
 *    bits per voxel, q = rint((x - map_origin) * 2^frac_bits / voxel_size), in
 *    IEEE double with one rounding per operation.  The voxel of q is
 *    floor(q / 2^frac_bits); a point on a voxel face belongs to the upper voxel.
 */
#ifndef OHM_GB_H
#define OHM_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ohm_map ohm_map;

typedef enum {
  OHM_OK = 0,
  OHM_ERR_INVALID = 1,     /* bad argument; nothing was enqueued */
  OHM_ERR_CAPACITY = 2,    /* region / NDT pool or scratch too small; map unchanged */
  OHM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  OHM_ERR_PROBE_LIMIT = 4, /* hash probe bound exceeded; map unchanged */
  OHM_ERR_UNSUPPORTED = 5, /* the map lacks a layer the call needs */
  OHM_ERR_EVICTED = 6      /* an asynchronous call touched regions evicted to host memory; it changed
                              nothing: call ohm_map_restore_pending, then repeat it */
} ohm_status;

/* Layers (Sec. III-A "multiple contiguous layers for each voxel region"). */
enum {
  OHM_LAYER_OCCUPANCY = 1, /* float log-odds per voxel, NaN = unknown (Sec. II-B) */
  OHM_LAYER_NDT = 2,       /* int64 sample moments per voxel (Sec. II-D, III-C) */
  OHM_LAYER_TSDF = 4,      /* float signed distance + weight per voxel (Sec. II-F) */
  OHM_LAYER_COUNTS = 8,    /* uint32 hits H_i and misses M_i per voxel (Sec. II-D) */
  OHM_LAYER_DECAY = 16,    /* decay-rate map (Sec. II-E): per voxel the summed length of the rays'
                              paths through it, uint64 in units of 2^-20 m; with OHM_LAYER_COUNTS
                              the reflection rate is lambda = H / sum d */
  OHM_LAYER_MEAN = 32      /* voxel mean (Sec. III-C): per voxel a uint64 word, sample count n in
                              the high 32 bits, the mean sample position inside the voxel in the
                              low 30 (10 bits per axis, x lowest, in 1/1024 of the voxel) */
};

/* Per-ray flag bits. */
enum {
  OHM_FLAG_NO_RETURN = 1   /* the endpoint is not a sample: the ray only clears space */
};

typedef struct {
  double voxel_size;       /* voxel edge in metres (0.1 in Sec. IV-A) */
  double map_origin[3];    /* world position of the lower corner of voxel (0,0,0) */
  int32_t frac_bits;       /* fixed-point fraction bits per voxel, 8..20 (16 recommended) */
  uint32_t layers;         /* OR of OHM_LAYER_* */
  float hit;               /* log-odds increment for a sample, log(P(z|occ)/P(z|emp)) (Eq. 3) */
  float miss;              /* log-odds increment for a pass-through (Eq. 3) */
  float l_min, l_max;      /* clamp bounds (Sec. II-B) */
  float ndt_clear_below;   /* NDT layer: a miss that takes a voxel's log-odds from at or above this
                              value (or from unknown) to below it clears the voxel's samples
                              (Sec. II-D); -INFINITY never clears */
  double max_range;        /* rays are truncated to this length and lose their sample (Sec. IV-A) */
  double min_range;        /* TSDF only: samples at or below this range are ignored */
  double tsdf_trunc;       /* TSDF truncation distance tau in metres */
  double tsdf_wmax;        /* TSDF weight cap */
  int64_t max_regions;     /* capacity of the region pool, 1..65536 (8 GB of occupancy) */
  int64_t max_ndt_regions; /* capacity of the NDT layer pool (regions holding samples) */
  int64_t max_rays;        /* largest ray count accepted by one integrate call */
  int32_t segment_steps;   /* target voxels per ray segment (Sec. III-B ray segments): a ray
                              whose walk visits N voxels is cut into ceil(N / segment_steps)
                              segments (more where needed to keep each within 65535 steps of its
                              dominant axis), its dominant-axis steps dealt out to them as evenly
                              as possible, so segments of rays in any direction are about equally
                              long; 0 = 24 */
  int32_t device;          /* CUDA device ordinal */
  int32_t evict_when_full; /* nonzero: when ohm_integrate_rays finds the region or NDT pool full it
                              moves least recently used regions to host memory and repeats the call
                              (see the region cache below); 0: the call fails with OHM_ERR_CAPACITY */
  int32_t max_probe;       /* hash probe bound: a region key lookup or insertion gives up after this
                              many table entries (Sec. III-A region lookup) and the call fails with
                              OHM_ERR_PROBE_LIMIT, changing nothing; 0 = min(table capacity, 4096),
                              larger values are clamped to that */
} ohm_map_params;

/* Create a map (Sec. III-A: a map is a sparse set of regions of 32^3 voxels,
 * each region holding one contiguous block per layer, found from its region
 * key in O(1)).  Fills `*out` on success.  Allocates the region pool, the
 * region hash table (capacity: the next power of two >= 2 * max_regions, and
 * at least 2^18 entries with evict_when_full, since evicted regions keep their
 * keys), the
 * enabled layers and per-call scratch sized for max_rays, on `device`.
 * Errors: OHM_ERR_INVALID for out-of-range parameters (including
 * max_range * 2^frac_bits / voxel_size >= 2^30, which would overflow the exact
 * integer walk), OHM_ERR_CUDA if allocation fails. */
ohm_status ohm_map_create(const ohm_map_params* params, ohm_map** out);

/* Free the map and everything it owns (the region storage of Sec. III-A).
 * NULL is ignored.  Waits for the last work an entry point enqueued on the map
 * (and the map's own copy stream), not for the whole device; the caller must
 * not destroy a map while it still has other work on it pending. */
void ohm_map_destroy(ohm_map* map);

/* Integrate one ray set (Sec. III-B; one call is one "scan").
 * Decay layer: every voxel the walk visits gains the length of the ray inside
 * it, P(t_out) - P(t_in): t_in, t_out are the ray parameters where the walk
 * enters and leaves it (0 at the start, 1 at the end point; a crossing of axis
 * k at t = dist_k / A_k with dist_k the fixed-point distance from the start to
 * the crossed boundary along k and A_k = |b_k - a_k|), kept as
 * floor(2^32 t) / 2^32, and P(t) = rint(t L) with L = rint(|b - a| voxel_size
 * 2^(20 - F)) the walked length in 2^-20 m (double).  Each ray adds exactly L
 * over the voxels it visits.
 * Mean layer: a sample's position inside its voxel is quantised to 10 bits
 * per axis (p = floor(offset * 1024 / 2^F)); per call, with c samples of sum
 * S in a voxel holding count n and mean m, every axis takes
 * m <- floor((m n + S + floor((n + c) / 2)) / (n + c)) and n <- min(n + c,
 * 2^32 - 1), so the result does not depend on the order of the samples.
 * Requires max_rays <= 2^22.
 *   origins    n_origins x 3 float world positions, x y z interleaved;
 *              n_origins is 1 (a shared sensor origin) or n.
 *   endpoints  n x 3 float world positions of the samples.
 *   flags      n bytes of OHM_FLAG_* or NULL (all returns).
 * Semantics per voxel, per call: every ray passing through the voxel applies
 * l <- clamp(l + miss) and afterwards every sample in the voxel applies
 * l <- clamp(l + hit) (the two-phase order of Sec. III-C); an unknown voxel
 * starts at l = 0.  The voxel holding a ray's sample receives the hit, not a
 * miss, from that ray.  A ray longer than max_range is truncated to it and
 * carries no sample; a ray with a non-finite coordinate, or a point outside
 * +-2^24 voxels of the map origin, is skipped.  TSDF layer: each returned ray
 * whose length lies in (min_range, max_range] updates the voxels the walk
 * visits between ranges max(0, d - tau) and d + tau with the projective
 * distance s = clamp(d - (c - o).u, -tau, tau); per call
 * D <- (W D + sum s) / (W + count), W <- min(W + count, tsdf_wmax).
 * All-or-nothing: regions are allocated before any voxel changes; if a pool
 * or the hash probe bound runs out the map is left unchanged and the call
 * returns OHM_ERR_CAPACITY / OHM_ERR_PROBE_LIMIT.  Blocks until the work on
 * `stream` has finished and returns its status. */
ohm_status ohm_integrate_rays(ohm_map* map, const float* origins, int64_t n_origins, const float* endpoints,
                              const uint8_t* flags, int64_t n, void* stream);

/* As ohm_integrate_rays, but returns once the work is enqueued.  Device-side
 * failures are latched in the map and returned (and cleared) by the next
 * ohm_map_sync; a failed call still leaves the map unchanged.  Input buffers
 * must stay valid until the stream has passed the call.  Host inputs are
 * copied on a stream of the map's own into one of two staging slots (the
 * `stream` waits for the copy), so the copy of one call overlaps the kernels
 * of the previous one; pinned host memory keeps the copies asynchronous. */
ohm_status ohm_integrate_rays_async(ohm_map* map, const float* origins, int64_t n_origins, const float* endpoints,
                                    const uint8_t* flags, int64_t n, void* stream);

/* Wait for `stream` and return (then clear) the latched device status. */
ohm_status ohm_map_sync(ohm_map* map, void* stream);

/* Enqueue on `stream` a copy of the map's latched device status bits into
 * *status (host memory; pinned memory keeps the copy asynchronous) and return
 * at once.  After the stream has passed this point, *status == 0 means every
 * call enqueued before it succeeded so far; nonzero bits mean one failed (call
 * ohm_map_sync to get the error and clear it).  Lets a caller read each
 * call's result without waiting between calls.  The paper has no counterpart
 * (its API is synchronous). */
ohm_status ohm_map_status_async(ohm_map* map, int32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * Region cache (Sec. III-A: regions move between the GPU and host memory).
 * Every pool region carries the sequence number of the last integrate call
 * that touched it.  Eviction copies the least recently touched regions to
 * pinned host memory and frees their pool slots; the keys stay known.  A
 * later call that reaches an evicted region stops and changes nothing;
 * ohm_integrate_rays then restores the region and repeats the call by
 * itself, the asynchronous entry points report OHM_ERR_EVICTED through
 * ohm_map_sync.  Query and export see resident regions only.
 * ------------------------------------------------------------------------- */

/* Evict least recently used regions until at most keep_regions remain
 * resident; *evicted = how many left the device.  Synchronous. */
ohm_status ohm_map_evict(ohm_map* map, int64_t keep_regions, int64_t* evicted, void* stream);

/* Restore the evicted regions the last call asked for (after OHM_ERR_EVICTED);
 * evicts other least recently used regions first if the pool is full.  Call it
 * before the next integrate call on this map.  Synchronous. */
ohm_status ohm_map_restore_pending(ohm_map* map, int64_t* restored, void* stream);

/* Bring every evicted region back (fails with OHM_ERR_CAPACITY if they do not
 * all fit).  Synchronous. */
ohm_status ohm_map_restore_all(ohm_map* map, int64_t* restored, void* stream);

/* Regions resident on the device and regions held in host memory. */
ohm_status ohm_map_residency(ohm_map* map, int64_t* resident, int64_t* evicted, void* stream);

/* Look up n world points (Sec. III-A: region key then voxel index).  Outputs
 * (device memory only; any may be NULL):
 *   occupancy  n floats, log-odds or NaN when unknown
 *   known      n bytes, 1 if the voxel has been observed
 *   ndt        n x 10 floats: sample count, mean x y z (metres, world),
 *              population covariance xx xy xz yy yz zz (m^2); zeros if none
 *   tsdf       n x 2 floats: D, W (zeros if unobserved)
 *   counts     n x 2 uint32: hits H, misses M
 *   path_sum   n uint64: summed ray path length through the voxel, 2^-20 m units
 *   mean       n x 4 floats: voxel-mean position x y z (metres, world: the
 *              voxel's lower corner + (m + 0.5) / 1024 voxels) and the sample
 *              count; NaN position and count 0 without samples
 * A non-NULL buffer for a layer the map lacks is OHM_ERR_UNSUPPORTED
 * (path_sum, mean).  `points` may be host or device memory.  Returns once
 * enqueued. */
ohm_status ohm_query_voxels(ohm_map* map, const float* points, int64_t n, float* occupancy, uint8_t* known,
                            float* ndt, float* tsdf, uint32_t* counts, uint64_t* path_sum, float* mean,
                            void* stream);

/* Number of pool slots ever used by the map, resident or released by eviction
 * (synchronises `stream`).  Without evictions: the number of regions. */
ohm_status ohm_map_region_count(ohm_map* map, int64_t* out, void* stream);

/* Copy regions [first, first + count) in allocation order into device buffers
 * (any may be NULL): the map's regions and their layers (Sec. III-A), the way
 * the paper's GPU cache synchronises regions back to the CPU-side map.  Voxel
 * order inside a region: x fastest, then y, then z.
 *   keys       count x 3 int32 region coordinates (voxel index >> 5)
 *   occupancy  count x 32768 float
 *   counts     count x 32768 x 2 uint32 (hits, misses)
 *   ndt        count x 32768 x 10 int64 (n, Sx, Sy, Sz, Sxx, Sxy, Sxz, Syy,
 *              Syz, Szz), positions in fixed-point units relative to the
 *              voxel's lower corner
 *   tsdf       count x 32768 x 2 float (D, W)
 *   path_sum   count x 32768 uint64 summed path length, 2^-20 m units
 *   mean       count x 32768 uint64 voxel-mean words (see OHM_LAYER_MEAN)
 * A non-NULL buffer for a layer the map lacks is OHM_ERR_UNSUPPORTED.
 * Returns once enqueued. */
ohm_status ohm_map_export(ohm_map* map, int64_t first, int64_t count, int32_t* keys, float* occupancy,
                          uint32_t* counts, int64_t* ndt, float* tsdf, uint64_t* path_sum, uint64_t* mean,
                          void* stream);

typedef struct {
  int64_t rays;          /* rays passed to the last integrate call */
  int64_t segments;      /* ray segments walked by the last call */
  int64_t visits;        /* voxel visits of the last call (occupancy walk + TSDF band walks) */
  int64_t regions;       /* regions in the map after the call */
  int64_t ndt_regions;   /* regions holding an NDT layer */
  int64_t touched;       /* TSDF voxels updated by the last call */
  int64_t total_visits;  /* voxel visits of every call since the map was created */
  int64_t launches;      /* kernels this map has launched since it was created */
  int64_t atomics;       /* log-odds compare-and-swap operations the miss walk of the last
                            single-map call issued on first attempt (retries after a lost
                            race are not counted; 0 after a batched step) */
} ohm_call_stats;

/* Statistics of the last completed integrate call (synchronises `stream`). */
ohm_status ohm_map_stats(ohm_map* map, ohm_call_stats* out, void* stream);

/* Throughput of 32-bit compare-and-swap on random words of a `words`-word
 * device buffer (words a power of two, 2^10..2^32), the pattern of the miss
 * walk's log-odds updates: per operation a load of the word, then a CAS of it,
 * four operations in flight per thread, 4 blocks of 256 threads per SM.
 * Runs about `ops` operations on `device` (allocating and freeing the buffer)
 * and writes operations per second; the ceiling the walk's atomic rate is
 * reported against.  The paper has no counterpart.  Synchronous. */
ohm_status ohm_probe_cas_rate(int32_t device, int64_t words, int64_t ops, double* ops_per_second);

/* Measured ceilings for the miss walk's memory work (no counterpart in the
 * paper): throughput of the library's probe kernels on `device`, 8 blocks of
 * 256 threads per SM, 8 random locations in flight per thread, best of three
 * timed launches after a warm-up launch (which also fills L2).  Allocates
 * and frees its buffer.  Synchronous.
 *   OHM_PROBE_L2_ADD      fire-and-forget float atomic add of 1 to a random
 *                         word of a `units`-word buffer (the walk's miss
 *                         update): L2 atomic throughput when the buffer fits in
 *                         L2, over distinct words when it is large and over
 *                         few (contended) words when `units` is small
 *   OHM_PROBE_L2_CAS      load, then compare-and-swap of a random word
 *   OHM_PROBE_SECTOR_RMW  load of a word of a random 32-byte sector of a
 *                         `units`-sector buffer, then a store of it plus one:
 *                         with a buffer larger than L2 every operation reads a
 *                         sector from memory and writes it back
 * `units` is a power of two (at most 2^32 words, 2^29 sectors); `ops` the
 * operations per timed launch.  Writes operations per second. */
enum { OHM_PROBE_L2_ADD = 0, OHM_PROBE_L2_CAS = 1, OHM_PROBE_SECTOR_RMW = 2 };
ohm_status ohm_probe_rate(int32_t device, int32_t kind, int64_t units, int64_t ops, double* ops_per_second);

/* Kernel stages of an integrate call, for per-stage GPU timing. */
typedef enum {
  OHM_STAGE_BEGIN = 0,        /* rollback snapshot */
  OHM_STAGE_PREPARE = 1,      /* quantise, truncate, region allocation, segment table, NDT
                                 layer of each sample's region where the slot is known */
  OHM_STAGE_NDT_ALLOC = 2,    /* NDT layer allocation for the sample regions prepare left */
  OHM_STAGE_PREPARE_TSDF = 3, /* TSDF band end points and their regions */
  OHM_STAGE_WALK = 4,         /* voxel walk, miss updates (Sec. III-C phase one) */
  OHM_STAGE_HITS = 5,         /* sample updates and NDT moments (phase two) */
  OHM_STAGE_TSDF_WALK = 6,    /* TSDF band walk */
  OHM_STAGE_TSDF_APPLY = 7,   /* TSDF weighted average */
  OHM_STAGE_END = 8,          /* rollback of a failed call */
  OHM_STAGE_MEAN_APPLY = 9,   /* voxel-mean per-call update */
  OHM_STAGE_COUNT = 10
} ohm_stage;

/* Record CUDA events around the kernels of the stages whose bit (1 << stage)
 * is set in `stage_mask` in every later integrate call (0 turns recording
 * off).  Resets the accumulated times.  Events are recorded on the call's own
 * stream, so the times are device durations of those launches. */
ohm_status ohm_map_profile(ohm_map* map, uint32_t stage_mask);

/* As ohm_map_profile, but only every `every`-th later integrate call (the
 * 1st, the every+1-th, ...) records its events; the others run without any.
 * An event between two kernels ends the programmatic-launch overlap of the
 * call's kernel chain there, so sampling keeps the other calls unperturbed.
 * every >= 1, else OHM_ERR_INVALID. */
ohm_status ohm_map_profile_every(ohm_map* map, uint32_t stage_mask, int32_t every);

/* Wait for the recorded launches of `stage` and return their summed device
 * time in milliseconds and their number. */
ohm_status ohm_map_profile_read(ohm_map* map, int32_t stage, double* total_ms, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Depth images and the TSDF adjoint.
 * ------------------------------------------------------------------------- */

/* Integrate one z-depth image (width x height floats, device memory, row
 * major) seen from pose (3 x 4 row-major camera-to-world [R | t], host) with
 * intrinsics (fx, fy, cx, cy; host): pixel (u, v) with depth z becomes the ray
 * from t to e = R (z ((u - cx) / fx), z ((v - cy) / fy), z) + t, evaluated in
 * double with one rounding per operation in the order
 * e_k = ((R_k0 x + R_k1 y) + R_k2 z) + t_k and rounded to float.  A depth
 * outside (z_min, z_max] gives a NO_RETURN ray at depth z_max (it clears space
 * in occupancy layers and is skipped by the TSDF, Sec. II-F).  width * height
 * must not exceed max_rays.  Like ohm_integrate_rays_async: returns once
 * enqueued; failures are reported by ohm_map_sync. */
ohm_status ohm_integrate_depth(ohm_map* map, const float* depth, int32_t width, int32_t height,
                               const double* intrinsics, const double* pose, double z_min, double z_max,
                               void* stream);

/* Adjoint of the TSDF update of the depth frame just integrated (no counterpart
 * in the paper).  With D the TSDF distance after that frame, it computes the
 * gradient of L = sum_q grad_query[q] D(voxel of query_points[q]) with respect
 * to every pixel's depth (grad_depth, width x height floats) and to the pose as
 * a left twist xi = (rho, phi) that moves each world point p to
 * p + rho + phi x p (grad_twist, 6 doubles), holding fixed the voxels each
 * ray's band walk visits and the per-voxel counts (the update is piecewise
 * smooth in the geometry; this is its derivative inside a piece).  Each pixel's
 * walk is recomputed, nothing is stored by the forward pass.  Call it before
 * any other integration into the map, with the same frame arguments as the
 * forward call, and with TSDF weights below tsdf_wmax.  All arrays are device
 * memory except intrinsics and pose.  The first call allocates a per-voxel
 * weight layer (4 bytes per pool voxel).  Returns once enqueued. */
ohm_status ohm_tsdf_backward(ohm_map* map, const float* depth, int32_t width, int32_t height,
                             const double* intrinsics, const double* pose, double z_min, double z_max,
                             const float* query_points, const float* grad_query, int64_t n_query, float* grad_depth,
                             double* grad_twist, void* stream);

/* Integrate one ray set given in a sensor frame: origins (n_origins = 1 or
 * n) and endpoints are moved to the world by pose (3 x 4 row-major
 * camera-to-world [R | t], host), p_k = ((R_k0 x + R_k1 y) + R_k2 z) + t_k in
 * double with one rounding per operation, rounded to float, then integrated as
 * by ohm_integrate_rays_async (Sec. III-B).  All ray arrays are device memory;
 * n must not exceed max_rays.  Returns once enqueued; failures are reported by
 * ohm_map_sync. */
ohm_status ohm_integrate_posed(ohm_map* map, const double* pose, const float* origins, int64_t n_origins,
                               const float* endpoints, const uint8_t* flags, int64_t n, void* stream);

/* Adjoint of the NDT-OM statistics (Sec. II-D, III-C: per voxel the mean and
 * the population covariance of its samples) for the ray set just integrated by
 * ohm_integrate_posed with the same arguments.  With mean(v) and C(v) after
 * that call, it computes the gradient of
 *   L = sum_q grad_mean[q] . mean(v_q) + grad_cov[q] . C(v_q)
 * (query_points: n_query x 3 world points; grad_mean n_query x 3; grad_cov
 * n_query x 6, packed xx xy xz yy yz zz; queries of voxels without samples
 * contribute nothing) with respect to every ray's sensor-frame endpoint
 * (grad_endpoints, n x 3 floats; zero for rays without a sample) and to the
 * pose as a left twist xi = (rho, phi) moving each world point p to
 * p + rho + phi x p (grad_twist, 6 doubles), holding fixed which rays carry a
 * sample and the voxel of each sample: for sample j in a voxel with n samples
 * summing to S (positions relative to the voxel's corner),
 *   dL/dp_j = (1/n) [gm + (G + G^T)(p_j - S/n)],  G = upper-triangular(gc),
 * with p_j and S the stored (fixed-point) positions.  Each ray's quantisation
 * is recomputed, nothing is stored by the forward pass.  Call it before any
 * other integration into the map.  Needs the NDT layer and ndt_clear_below =
 * -INFINITY (OHM_ERR_UNSUPPORTED otherwise: sample clearing changes the
 * statistics discontinuously).  The first call allocates 36 bytes of weights
 * per voxel of the NDT pool.  All arrays are device memory except pose.
 * Returns once enqueued.  The paper has no counterpart. */
ohm_status ohm_ndt_backward(ohm_map* map, const double* pose, const float* origins, int64_t n_origins,
                            const float* endpoints, const uint8_t* flags, int64_t n, const float* query_points,
                            const float* grad_mean, const float* grad_cov, int64_t n_query, float* grad_endpoints,
                            double* grad_twist, void* stream);

/* The pose exp(xi) pose0 of the adjoint's pose parametrisation: the left
 * twist xi = (rho, phi) (6 doubles) as a rigid motion (rotation by Rodrigues'
 * formula, translation V rho with V the left Jacobian of SO(3); to first
 * order below |phi| = 1e-12) applied to the 3 x 4 row-major camera-to-world
 * pose0, written to pose (12 doubles).  Host memory, host arithmetic (double);
 * ohm_tsdf_backward's grad_twist is the gradient with respect to xi at 0 of
 * the frame seen from this pose.  The paper has no counterpart. */
ohm_status ohm_twist_pose(const double* xi, const double* pose0, double* pose);

/* ---------------------------------------------------------------------------
 * Batched integration of many maps (no counterpart in the paper, which
 * integrates one ray set into one map at a time).
 *
 * A batch groups up to OHM_BATCH_MAX_MAPS independent maps on one device.
 * ohm_batch_integrate integrates one ray set into each map with one kernel
 * launch per stage for all maps together, so small and uneven ray sets share
 * the GPU instead of running one after another.  Per map the result is exactly
 * that of ohm_integrate_rays_async on the same rays (same order semantics,
 * same all-or-nothing rule per map).  With use_graph != 0 the first call
 * captures the step into a CUDA graph and later calls replay it; the stream
 * must then be a created stream, not the legacy default stream.
 * ------------------------------------------------------------------------- */
#define OHM_BATCH_MAX_MAPS 32

typedef struct ohm_batch ohm_batch;

/* Group n_maps distinct maps (same device) into a batch.  The maps stay owned
 * by the caller and must outlive the batch. */
ohm_status ohm_batch_create(ohm_map* const* maps, int32_t n_maps, ohm_batch** out);

/* Free the batch (not its maps).  NULL is ignored. */
void ohm_batch_destroy(ohm_batch* batch);

/* Tile parameters of later steps: segment_steps (target voxel steps per ray
 * segment, as in ohm_map_params, applied to every map; 0 = unchanged) and the walk
 * kernel's blocks per SM (0 = unchanged).  Results do not depend on them.
 * Drops the captured graph.  Synchronises the device. */
ohm_status ohm_batch_tune(ohm_batch* batch, int32_t segment_steps, int32_t walk_blocks_per_sm);

/* One step: for map i, n[i] rays (0 = no rays this step) with n_origins[i]
 * origins (1 or n[i]) at origins[i], endpoints at endpoints[i] and flags at
 * flags[i] (flags or flags[i] may be NULL).  All ray arrays are device memory
 * and must stay valid until the stream has passed the step.  The small host
 * arrays are copied before the call returns.  Device-side failures are latched
 * per map and reported by ohm_batch_sync. */
ohm_status ohm_batch_integrate(ohm_batch* batch, const float* const* origins, const int64_t* n_origins,
                               const float* const* endpoints, const uint8_t* const* flags, const int64_t* n,
                               int32_t use_graph, void* stream);

/* Wait for `stream`; return (and clear) the first failure latched by any map. */
ohm_status ohm_batch_sync(ohm_batch* batch, void* stream);

/* Kernels launched through this batch (a graph replay counts its kernel
 * nodes), and the number of steps replayed from the captured graph. */
ohm_status ohm_batch_stats(ohm_batch* batch, int64_t* kernel_launches, int64_t* graph_launches);

/* ---------------------------------------------------------------------------
 * Allocation-free ray counting (the paper has no counterpart to this entry
 * point).
 *
 * For callers that cannot call cudaMalloc when they need to integrate rays:
 * code running while a stream is captured into a CUDA graph (allocation is not
 * allowed there), real-time loops that must not wait on the allocator or on
 * the synchronisation cudaFree implies, and plug-ins whose host application
 * owns all device memory.  ohm_count_rays_noalloc walks a ray set exactly like
 * ohm_integrate_rays (same quantisation, truncation and voxel walk) and adds
 * each ray's per-voxel counts to two uint32 arrays the caller owns: every voxel
 * a ray passes through gets misses += 1, the voxel holding its sample (if it
 * has one) gets hits += 1.  Voxels outside the grid are not counted.
 *
 * It allocates nothing: its working memory is one statically sized device
 * array inside the library (about 3 MB), which every GPU that loads the library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Every call uses the calling thread's current device and
 * shares the array: calls whose work may overlap on the GPU (unordered streams)
 * race on it and must not be issued.  Each call clears the part that must start
 * at zero.  All pointers must be device memory of the current device; hits and
 * misses must each hold dims[0] * dims[1] * dims[2] uint32 elements and flags
 * (if not NULL) n bytes -- the library cannot check the sizes of caller
 * buffers, and a short one is written or read out of bounds.
 * Errors: OHM_ERR_INVALID when n > OHM_NOALLOC_MAX_RAYS, when n times the
 * segments a ray can have (max_range / voxel_size + 2) / segment_steps + 1
 * exceeds 4 * OHM_NOALLOC_MAX_RAYS, for bad grid parameters or host pointers;
 * OHM_ERR_CUDA for a failed CUDA call.  Returns once the work is enqueued.
 * ------------------------------------------------------------------------- */
#define OHM_NOALLOC_MAX_RAYS 32768

typedef struct {
  double voxel_size;       /* voxel edge in metres */
  double map_origin[3];    /* world position of the lower corner of voxel (0,0,0) */
  int32_t frac_bits;       /* fixed-point fraction bits per voxel, 8..20 */
  int32_t segment_steps;   /* ray segment length in dominant-axis steps; 0 = 64 */
  double max_range;        /* truncation length in metres */
  int64_t corner[3];       /* voxel index of grid cell (0,0,0) */
  int64_t dims[3];         /* grid size in voxels; cell (x,y,z) is element x + dims[0] * (y + dims[1] * z) */
} ohm_count_grid;

ohm_status ohm_count_rays_noalloc(const ohm_count_grid* grid, const float* origins, int64_t n_origins,
                                  const float* endpoints, const uint8_t* flags, int64_t n, uint32_t* hits,
                                  uint32_t* misses, void* stream);

/* Thread-local message describing the last failure on this thread.  The
 * paper has no error interface; the failures reported are those of its steps:
 * the region allocation before the walk (Sec. III-B: a ray set's regions must
 * all be present before its voxels are updated), the hash probe bound of the
 * region lookup (Sec. III-A) and the argument checks of each entry point. */
const char* ohm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OHM_GB_H */
