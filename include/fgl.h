/*
 * fgl.h -- batched LiDAR ray casting on GB300 (sm_103a).
 *
 * The operation is the LiDAR measurement model of FGGS-LiDAR (arXiv
 * 2509.17390), Sec. IV-C:
 *   eq. r_j   : beam j of a sensor with pose T_s = [R_s | t_s] in SE(3) is
 *               the ray r_j(t) = x_s + t d_j, with origin x_s = t_s and unit
 *               direction d_j = R_s * (its sensor-frame direction);
 *   eq. t_j*  : its return is the nearest intersection parameter with the
 *               triangle mesh M, over (t_min, t_max] = (0, max_range];
 *   cost model: the mesh sits in a bounding-volume hierarchy and every ray
 *               walks it, pruned by its best-so-far t (Sec. IV-C,
 *               "GPU-accelerated ray-casting", eq. cost(r_j)).
 * Results are reported per ray as a float32 range (the ray parameter t;
 * directions are unit length up to float32 rounding, so t is metres) and
 * the int32 id of the hit triangle (its index in the input triangle array).
 * A miss reports (max_range, -1).  Ties in t go to the smaller triangle id,
 * so results never depend on traversal order, BVH width, packet shape,
 * stack depth, block size or batching.
 *
 * Conventions
 *   - Sensor frame: x forward, y left, z up.  Beam direction from elevation
 *     el and azimuth az (radians): (cos el cos az, cos el sin az, sin el),
 *     evaluated on the host in float64 and rounded once to float32.
 *   - Pose: float32 [3][4] row-major [R | t] (sensor -> world), 48 bytes per
 *     environment, environments contiguous.  The world direction is
 *     computed in float32 with every product and sum rounded separately, row
 *     i as ((R[i][0]*d0) + (R[i][1]*d1)) + (R[i][2]*d2).
 *   - Output layout: ray (env e, beam r) at index e * n_rays + r, where r is
 *     the beam's position in the table given to fgl_sensor_create.
 *   - Pointers marked "device" are CUDA device pointers owned by the caller;
 *     calls that take a stream are asynchronous on it.  Argument errors are
 *     reported synchronously; asynchronous CUDA errors and device-side
 *     traversal errors surface on fgl_sync() or the next call.
 *   - Every call returns an fgl_status; on failure fgl_last_error() gives a
 *     thread-local message.
 */
#ifndef FGL_H
#define FGL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* fgl_stream;

typedef enum {
  FGL_OK = 0,
  FGL_ERR_INVALID = 1,   /* bad argument (null pointer, size, NaN, id range) */
  FGL_ERR_OOM = 2,       /* device or host allocation failed */
  FGL_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  FGL_ERR_BUDGET = 4,    /* serving: request larger than the HBM budget */
  FGL_ERR_TIMEOUT = 5,   /* serving: wait timed out */
  FGL_ERR_CANCELLED = 6, /* serving: request cancelled */
  FGL_ERR_DEVICE = 7,    /* a kernel reported an error (traversal stack overflow; in the
                            checked library also an index out of range) */
  FGL_ERR_CAPACITY = 8,  /* output buffers too small; the needed counts are reported */
  FGL_ERR_INTERNAL = 9   /* serving: a host exception in the server's worker thread */
} fgl_status;

typedef struct fgl_scene_s* fgl_scene;
typedef struct fgl_sensor_s* fgl_sensor;

/* ------------------------------------------------------------------------ */
/* Scenes                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t width;      /* children per BVH node: 4 or 8 (0 = 8) */
  int32_t sah_bins;   /* binned-SAH bins per axis (0 = 128) */
  int32_t n_threads;  /* host build threads (0 = all cores) */
  int32_t upload;     /* 1 = upload to the current CUDA device (default when
                         opts is NULL); 0 = host-only build (tests, offline) */
} fgl_build_opts;

typedef struct {
  int64_t n_tris;       /* triangles in the scene */
  int64_t n_nodes;      /* wide BVH nodes */
  int64_t node_bytes;   /* bytes of the node array (node_stride * n_nodes) */
  int64_t tri_bytes;    /* bytes of the leaf triangle array (48 * n_tris) */
  int32_t width;        /* children per node */
  int32_t node_stride;  /* bytes per node record (256 for width 8, 144 for 4) */
  int32_t depth;        /* levels of the wide tree (root = 1) */
  int32_t resident;     /* 1 when the arrays are on the device */
  double sah_cost;      /* SAH cost of the wide tree (node visits + tri tests, area-weighted) */
  double build_ms;      /* host build time */
  float bounds_lo[3];   /* scene bounds */
  float bounds_hi[3];
  float margin;         /* outward margin added to every child box (metres) */
} fgl_scene_stats;

/* Build a scene from a triangle mesh (the mesh M of eq. t_j*).
 *   verts: host float32 [nv][3]; tris: host int32 [nt][3] vertex ids.
 *   Builds a binned-SAH binary BVH, collapses it to `width`-wide nodes with
 *   float32 child boxes stored as offsets from the node corner, rounded
 *   outward (plus a margin covering float32 rounding of the traversal's
 *   slab test), re-orders triangles into leaf
 *   order (48 bytes each) and, when opts->upload != 0, copies both arrays to
 *   the current device (synchronously).  The scene owns its device memory
 *   until fgl_scene_destroy and keeps its host copy for re-upload.
 *   Errors: FGL_ERR_INVALID for nv<1, nt<1, null pointers, non-finite
 *   vertices or ids outside [0,nv); FGL_ERR_OOM; FGL_ERR_CUDA. */
fgl_status fgl_scene_build(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                           const fgl_build_opts* opts, fgl_scene* out);
fgl_status fgl_scene_destroy(fgl_scene scene);
fgl_status fgl_scene_get_stats(fgl_scene scene, fgl_scene_stats* out);
/* Copy the host node / triangle arrays (sizes from the stats) -- for tests. */
fgl_status fgl_scene_export(fgl_scene scene, void* nodes, int64_t node_bytes, void* tris,
                            int64_t tri_bytes);
/* Check, in double arithmetic, that every child box (node corner plus the
 * stored float offsets) contains its subtree's triangles grown by the
 * margin, and the tree's structure (child indices, hit bits, every
 * triangle referenced once).
 * Writes the number of violations to *n_bad (0 for a correct build). */
fgl_status fgl_scene_verify(fgl_scene scene, int64_t* n_bad);
/* Upload (if evicted) / drop the device copy, keeping the host copy. */
fgl_status fgl_scene_upload(fgl_scene scene);
fgl_status fgl_scene_evict(fgl_scene scene);

/* ------------------------------------------------------------------------ */
/* Sensors (scan patterns, the d_j of eq. r_j)                               */
/* ------------------------------------------------------------------------ */

/* Create a sensor from per-beam elevation/azimuth (host float32 radians,
 * n_rays entries).  rows x cols describes the beam grid of a spinning sensor
 * (rows * cols == n_rays, beam r = row * cols + col); pass rows = 1,
 * cols = n_rays for a pattern with no grid.  tile_rows x tile_cols (0 = the
 * default 4 x 8) is the angular tile that consecutive rays of one warp are
 * drawn from; it changes speed only, never results.  Directions are computed
 * on the host in float64, rounded to float32 and uploaded (synchronously).
 * Errors: FGL_ERR_INVALID for n_rays<1, rows*cols != n_rays, non-finite
 * angles, tiles < 0. */
fgl_status fgl_sensor_create(const float* elev_rad, const float* azim_rad, int32_t n_rays,
                             int32_t rows, int32_t cols, int32_t tile_rows, int32_t tile_cols,
                             fgl_sensor* out);
fgl_status fgl_sensor_destroy(fgl_sensor sensor);
fgl_status fgl_sensor_n_rays(fgl_sensor sensor, int32_t* n_rays);
/* Host copy of the float32 sensor-frame directions [n_rays][3], beam order. */
fgl_status fgl_sensor_dirs(fgl_sensor sensor, float* out_dirs);

/* ------------------------------------------------------------------------ */
/* Casting                                                                   */
/* ------------------------------------------------------------------------ */

/* Plain form: one kernel launch, one thread per ray, over n_env poses of one
 * sensor against one scene, with t_min = 0 (a min_range needs the batched
 * form).
 *   poses:     device float32 [n_env][3][4]
 *   out_range: device float32 [n_env * n_rays]; out_tri: device int32, same.
 * n_env == 0 is a no-op.  Errors: FGL_ERR_INVALID (null handle/pointer,
 * n_env < 0, max_range not finite and > 0, scene not resident). */
fgl_status fgl_cast(fgl_scene scene, fgl_sensor sensor, const float* poses, int32_t n_env,
                    float max_range, float* out_range, int32_t* out_tri, fgl_stream stream);

/* One batched work item.  The return of each ray is its nearest mesh
 * intersection with t in [min_range, max_range] (eq. t_j*: intersections
 * outside the sensor's [t_min, t_max] are discarded), t > 0 always; a
 * surface nearer than min_range is passed through, so the ray may return a
 * farther surface behind it.  No intersection -> (max_range, -1).
 * With instances, the environment's mesh is the scene plus every instance
 * moved by its pose: each instance is cast in its own frame with the ray
 *   u = o - t_k;  o'_i = ((R_0i u_0 + R_1i u_1) + R_2i u_2),
 *   d'_i = ((R_0i d_0 + R_1i d_1) + R_2i d_2)   (float32, no FMA),
 * which keeps the ray parameter t of a rigid motion; the return is the
 * nearest over the scene and the instances, ties going to the scene, then to
 * the lower instance index. */
typedef struct {
  fgl_scene scene;
  fgl_sensor sensor;
  const float* poses;   /* device float32 [n_env][3][4] */
  int32_t n_env;
  float max_range;      /* t_max: finite, > 0 */
  float* out_range;     /* device float32 [n_env * n_rays] */
  int32_t* out_tri;     /* device int32  [n_env * n_rays] */
  float min_range;      /* t_min: finite, 0 <= min_range < max_range (0 = none) */
  /* Optional (zero-initialise to leave unused): */
  float* out_points;    /* device float32 [n_env * n_rays][3]: the world-frame return
                           point o + t d, each coordinate o_i + (t * d_i) rounded twice;
                           NaN for a miss */
  int32_t n_instances;  /* rigid instances per environment (0 = none) */
  const fgl_scene* instances;   /* host array [n_instances]: meshes in their own frames
                                   (any BVH width; resident on the device) */
  const float* instance_poses;  /* device float32 [n_env][n_instances][3][4]: world-from-local
                                   [R | t] of instance k in environment e, R orthonormal */
  int32_t* out_instance;        /* device int32 [n_env * n_rays]: k when the return lies on
                                   instance k (out_tri is then its triangle), -1 otherwise;
                                   may be NULL */
} fgl_cast_item;

typedef struct {
  int32_t packet_rays;    /* rays per work packet (0 = 32; multiple of 32) */
  int32_t block_threads;  /* threads per block (0 = 128; multiple of 32, <= 512) */
  int32_t stack_smem;     /* traversal stack entries kept in shared memory (0 = 6) */
  int32_t blocks_per_sm;  /* persistent blocks per SM (0 = as many as fit) */
  int32_t use_graph;      /* 1 = capture the launch sequence in a CUDA graph and
                             replay it while the item layout is unchanged */
  int32_t refill_min;     /* idle lanes before a warp pulls new rays (0 = 32:
                             refill once the whole warp is idle) */
  int32_t postpone_pct;   /* tri_mode 1 only: postpone leaf tests when fewer than
                             this % of the warp's tracing lanes want them
                             (0 = 20; -1 = never) */
  int32_t count_work;     /* 1 = count node visits and triangle tests (slower);
                             read with fgl_work_counters */
  int32_t tri_mode;       /* leaf triangle tests: 0 = pooled across the warp
                             (default), 1 = each lane tests its own, postponing
                             per postpone_pct */
} fgl_batch_opts;

/* fgl_cast with explicit launch options: block_threads, stack_smem,
 * tri_mode, postpone_pct and count_work apply; the other fields are ignored.  Results
 * are identical for every valid option set (only speed changes). */
fgl_status fgl_cast_opts(fgl_scene scene, fgl_sensor sensor, const float* poses, int32_t n_env,
                         float max_range, float* out_range, int32_t* out_tri,
                         const fgl_batch_opts* opts, fgl_stream stream);

/* Batched form: every item (scene, sensor, poses) goes into one device work
 * queue of ray packets drained by one persistent kernel (per BVH width
 * present in the batch).  Uneven ray counts, sensors and scenes mix freely.
 * Scratch (queue head, item table) is library-owned and cached per stream.
 * Errors: as fgl_cast for each item; FGL_ERR_INVALID for n_items < 0. */
fgl_status fgl_cast_batched(const fgl_cast_item* items, int32_t n_items,
                            const fgl_batch_opts* opts, fgl_stream stream);

/* End-to-end form of fgl_cast_batched for callers holding HOST buffers:
 * items[i].poses / out_range / out_tri -- and, when used, instance_poses,
 * out_instance and out_points -- are host pointers (page-locked for full
 * speed).  Copies the poses to library-owned device staging, runs the
 * batched kernels (instances and return points included) and synchronizes
 * the stream.  When every item's out_range and out_tri are page-locked and
 * it has no instances or points, the kernel stores the returns straight into
 * them over the host link as it runs; otherwise the results are cast into
 * device staging and copied back, large batches in up to 4 chunks of whole
 * environments whose copies back overlap the next chunk's cast. */
fgl_status fgl_cast_batched_host(const fgl_cast_item* items, int32_t n_items,
                                 const fgl_batch_opts* opts, fgl_stream stream);

/* fgl_cast_batched for callers that cannot allocate device memory (real-time
 * loops that must not trigger an allocator's device synchronisation, plugins
 * inside an application that owns every device allocation, processes whose
 * device memory belongs to a pool they do not own).  The paper has no counterpart: this is an
 * interface for such callers, not part of the method.
 *   Same arguments, layouts and results as fgl_cast_batched (use_graph is
 *   ignored); the caller still owns poses and outputs.  The work-queue scratch
 *   is a fixed array of ~25 KiB inside the library (held by every GPU that
 *   loads it until the process exits), so a call allocates nothing on the
 *   device, and nothing on the host when it succeeds.
 *   Limit: at most 256 items per call; more is rejected with FGL_ERR_INVALID.
 *   The first call on each device looks up the array's device address (with
 *   that device current); make that first call before any stream capture
 *   begins.
 *   All calls share the array and reset its queue head: calls whose work
 *   overlaps on the GPU race, so issue them on one stream or order them. */
fgl_status fgl_cast_batched_static(const fgl_cast_item* items, int32_t n_items,
                                   const fgl_batch_opts* opts, fgl_stream stream);

/* Autotuner for the batched form: picks the launch options (packet size,
 * block size, shared-memory stack depth, refill threshold, leaf-test mode)
 * that run `items` fastest, by coordinate descent from the defaults, timing
 * each candidate with CUDA events on `stream` (median of `reps` runs after one
 * warm-up).  The items are really cast (their outputs are overwritten).  BVH
 * width and sensor tile shape are properties of the scene and sensor objects;
 * tune them by building variants and calling this once per variant.  The
 * paper fixes none of these; they change speed only, never results.
 *   best: in = starting point and use_graph/count_work settings (NULL fields
 *         = defaults), out = the fastest options found.
 *   Errors: as fgl_cast_batched. */
typedef struct {
  int32_t reps;        /* timed runs per candidate (0 = 3) */
  int32_t passes;      /* coordinate-descent passes over the dimensions (0 = 2) */
} fgl_tune_opts;

typedef struct {
  double best_ms;      /* median time of the chosen options */
  double start_ms;     /* median time of the starting options */
  int32_t trials;      /* candidates timed */
} fgl_tune_result;

fgl_status fgl_autotune(const fgl_cast_item* items, int32_t n_items, const fgl_tune_opts* topts,
                        fgl_batch_opts* best, fgl_tune_result* result, fgl_stream stream);

/* Wait for the stream, then report any asynchronous CUDA error or
 * device-side traversal error (FGL_ERR_DEVICE) raised since the last check. */
fgl_status fgl_sync(fgl_stream stream);

/* Totals accumulated by count_work launches since the last call (then reset):
 * rays traced, wide-node visits, triangle tests (the N_nodes and K of the
 * paper's per-ray cost, eq. cost(r_j)). */
fgl_status fgl_work_counters(uint64_t* rays, uint64_t* node_visits, uint64_t* tri_tests);
/* The same counters plus the phases of the batched kernel, for attributing
 * its work (no counterpart in the paper), written to out[0..n-1] (n <= 8)
 * and then reset: [0] rays, [1] node visits, [2] triangle tests, [3] warp
 * iterations of the persistent kernel's main loop, [4] active lanes summed
 * over those iterations, [5] pooled leaf-test rounds (32 tests each at
 * most), [6] stack entries popped after the leaf tests, [7] ray packets
 * drawn by warps. */
fgl_status fgl_work_phase_counters(uint64_t* out, int32_t n);

/* Optional sensor effects on cast returns, applied in place after a cast
 * (the paper models the return as the nearest hit only, eq. t_j*, and leaves
 * richer sensor physics to future work, Sec. VI; these are an extension):
 *   random words  Philox-4x32-10 (Salmon et al., SC 2011), key (seed low 32
 *                 bits, seed high 32 bits), counter (ray j, env_offset + e,
 *                 step, 0) for ray j of environment e -> x0..x3;
 *   dropout       a hit is dropped, i.e. reported as the miss (max_range, -1),
 *                 when (x0 >> 8) * 2^-24 < drop_prob (exact in float32);
 *   range noise   a kept hit at range t becomes t + (sigma0 + sigma1 t) n,
 *                 n = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller) with
 *                 u1 = ((x1 >> 8) + 1) 2^-24, u2 = (x2 >> 8) 2^-24, in
 *                 float32, clamped to [0, max_range];
 *   misses are unchanged.  Dropout decisions are exact; noisy ranges carry
 *   float32 rounding (a few ulp of t plus ~1e-6 of the noise term).
 *   range, tri: device [n_env * n_rays] returns of one cast item (ray j of
 *   environment e at e * n_rays + j).  Errors: FGL_ERR_INVALID (null,
 *   drop_prob outside [0, 1], negative or non-finite sigma, max_range,
 *   env_offset), FGL_ERR_CUDA. */
typedef struct {
  uint64_t seed;
  uint32_t step;          /* frame counter: each step draws anew */
  int32_t env_offset;     /* counter id of the first environment (>= 0) */
  float drop_prob;        /* probability that a hit is dropped */
  float noise_sigma0;     /* range noise standard deviation at range 0 (m) */
  float noise_sigma1;     /* ... growing by this much per metre of range */
  float max_range;        /* the cast's max_range: dropped returns report it */
} fgl_sensor_effects;

fgl_status fgl_apply_sensor_effects(const fgl_sensor_effects* fx, float* range, int32_t* tri,
                                    int32_t n_env, int32_t n_rays, fgl_stream stream);

/* Bandwidth probe for the roofline (no counterpart in the paper): reads the
 * device buffer buf (16-byte aligned, `bytes` a multiple of 16) `reps` times
 * with 16-byte loads that bypass L1, on a grid of 4 blocks of 512 threads
 * per SM; time it with events on `stream` to get the L2 read bandwidth of a
 * buffer that stays resident in L2.  sink: device uint32 (written only with
 * a value no load can produce, i.e. in practice never).  Errors:
 * FGL_ERR_INVALID for null pointers, sizes or alignment. */
fgl_status fgl_probe_l2_read(const void* buf, int64_t bytes, int32_t reps, uint32_t* sink,
                             fgl_stream stream);

/* Debug export of the float32 world rays the kernels trace (eq. r_j):
 * out_o, out_d device float32 [n_env * n_rays][3]. */
fgl_status fgl_world_rays(fgl_sensor sensor, const float* poses, int32_t n_env, float* out_o,
                          float* out_d, fgl_stream stream);

/* ------------------------------------------------------------------------ */
/* Triangle LBVH built on the GPU (paper Sec. IV-C with the LBVH routine of  */
/* Sec. IV-A): for meshes that change every frame, and the paper's one-      */
/* thread-per-beam traversal                                                 */
/* ------------------------------------------------------------------------ */

typedef struct fgl_lbvh_s* fgl_lbvh;

typedef struct {
  int64_t n_tris;
  int64_t n_nodes;          /* internal nodes (n_tris - 1); leaves hold one triangle */
  int32_t depth;            /* levels of the binary tree (root = 1) */
  int32_t overflow;         /* bit 0: a cast's traversal stack overflowed (returns then wrong);
                               bit 1: a node or triangle index was out of range (checked
                               library only) */
  float build_ms;           /* host-observed build time of the last build, synchronised */
  float margin;             /* outward margin of every leaf box (metres) */
  float centroid_lo[3];     /* the box the Morton codes quantise (triangle centroids) */
  float centroid_hi[3];
} fgl_lbvh_stats;

/* Build (or, with *out already set, rebuild in place) a triangle LBVH on the
 * GPU from DEVICE arrays: verts float32 [nv][3], tris int32 [nt][3].
 * Morton codes (eqs. u_i, m_i: 10 bits per axis of the centroid in the box of
 * all centroids), a stable radix sort, the hierarchy from longest common
 * prefixes (eq. LCP; equal codes ordered by position), then node boxes bottom
 * up; leaf boxes are grown by 2^-17 max(1, max |coord|).  Synchronises
 * `stream` at the end.  Errors: FGL_ERR_INVALID (empty mesh, nt >= 2^30, a
 * vertex id out of range or a non-finite vertex), FGL_ERR_OOM, FGL_ERR_CUDA. */
fgl_status fgl_lbvh_build(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          fgl_stream stream, fgl_lbvh* out);
fgl_status fgl_lbvh_destroy(fgl_lbvh lbvh);
fgl_status fgl_lbvh_get_stats(fgl_lbvh lbvh, fgl_lbvh_stats* out);
/* Host copies of the nodes (64 B each: both child boxes as floats, then int32
 * left, right, parent, 0; a reference < 0 is ~leaf) and the triangles in
 * Morton order (48 B each, as the wide BVH's leaf records). */
fgl_status fgl_lbvh_export(fgl_lbvh lbvh, void* nodes, int64_t node_bytes, void* tris,
                           int64_t tri_bytes);
/* eq. t_j* over an LBVH, one thread per beam (the paper's form): the same
 * returns, bit for bit, as fgl_cast on a wide BVH of the same mesh (same
 * triangle test and (t, id) rule), t in [min_range, max_range]. */
fgl_status fgl_cast_lbvh(fgl_lbvh lbvh, fgl_sensor sensor, const float* poses, int32_t n_env,
                         float min_range, float max_range, float* out_range, int32_t* out_tri,
                         fgl_stream stream);

/* ------------------------------------------------------------------------ */
/* Gaussian-to-occupancy conversion (paper Sec. IV-A)                        */
/* ------------------------------------------------------------------------ */

/* 3D Gaussians (device pointers; the caller owns them). */
typedef struct {
  const float* mu;       /* [n][3] means */
  const float* scale;    /* [n][3] standard deviations along the Gaussian's own axes */
  const float* quat;     /* [n][4] rotation (w, x, y, z), any nonzero norm */
  const float* opacity;  /* [n] alpha */
  int64_t n;             /* < 2^32 */
} fgl_gaussians;

/* Isotropic voxel grid: voxel (i, j, k) has centre
 * origin + ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h) and linear index
 * (k * dims[1] + j) * dims[0] + i.  Tiles are tile^3 voxels, tile (a, b, c)
 * holding voxels [a*tile, a*tile + tile) x ... (partial at the far faces). */
typedef struct {
  float origin[3];
  float h;               /* voxel edge, finite and > 0 */
  int32_t dims[3];       /* >= 1 each */
  int32_t tile;          /* 4 or 8 (0 = 8) */
} fgl_grid;

typedef struct {
  int32_t timing;        /* in: 1 = time the call with CUDA events on `stream` (it then
                            synchronises the stream again before returning) */
  int64_t n_pairs;       /* out: (Gaussian, tile) candidate pairs */
  int64_t n_tiles;       /* out */
  int64_t n_voxels;      /* out */
  float ms_total;        /* out (timing): first to last launch of the call */
  float ms_density;      /* out (timing): the density kernel alone */
  int32_t n_launches;    /* out: kernels the call launched */
} fgl_density_stats;

/* Eq. D(v) on the grid, then eqs. V_occ, Int and Surf:
 *   D(v) = sum over the candidates G of v's tile of
 *          alpha_G^2 exp(-1/2 (v - mu_G)^T Sigma_G^-1 (v - mu_G)),
 *   Sigma = R diag(scale^2) R^T, R the rotation of the normalised quaternion;
 *   V_occ = D > theta; Int = V_occ at the voxel and its 6 face neighbours
 *   (outside the grid counts as empty); Surf = V_occ and not Int.
 * Candidates of a tile (eq. C_tile): the Gaussians whose axis-aligned box of
 * the 3-sigma ellipsoid meets the tile.  That integer decision is taken in
 * float32 with this exact operation sequence (round to nearest, no FMA):
 *   n = sqrt(((w*w + x*x) + y*y) + z*z); w, x, y, z /= n;
 *   R = [[1-2(yy+zz), 2(xy-wz), 2(xz+wy)], [2(xy+wz), 1-2(xx+zz), 2(yz-wx)],
 *        [2(xz-wy), 2(yz+wx), 1-2(xx+yy)]]   (xx = x*x, wz = w*z, ...);
 *   var_a = ((R_a0*s0)^2 + (R_a1*s1)^2) + (R_a2*s2)^2;  e_a = 3 * sqrt(var_a);
 *   cell = float(tile) * h;
 *   lo_a = floor(((mu_a - e_a) - origin_a) / cell), hi_a likewise with + e_a,
 *   both clamped to [-2^30, 2^30];
 * tile (a, b, c) is a candidate iff lo <= (a, b, c) <= hi per axis.  A
 * Gaussian with a non-finite mean or scale, a scale <= 0 or a zero quaternion
 * is nobody's candidate.  Each voxel sums its tile's candidates in increasing
 * Gaussian index (float32; the results are deterministic).
 *   out_density: device float32 [n_voxels] (required);
 *   out_occ / out_surf: device uint8 [n_voxels] (0/1), either may be NULL;
 *   stats: may be NULL (see fgl_density_stats for its one input field).
 * The call synchronises `stream` once (to size the pair buffers, cached per
 * stream); the rest is asynchronous.  Errors: FGL_ERR_INVALID (bad grid,
 * tile, null pointers, more than 2^31 - 1 pairs), FGL_ERR_CUDA. */
fgl_status fgl_gaussian_density(const fgl_gaussians* gaussians, const fgl_grid* grid, float theta,
                                float* out_density, uint8_t* out_occ, uint8_t* out_surf,
                                fgl_density_stats* stats, fgl_stream stream);

/* ------------------------------------------------------------------------ */
/* Mesh reconstruction (Sec. IV-B)                                           */
/* ------------------------------------------------------------------------ */
/* The steps between the surface-only occupancy (fgl_gaussian_density's
 * out_surf) and a triangle mesh: binary denoising and re-thresholding, the
 * narrow-band TSDF and its level set.  Grids are fgl_grid (tile ignored);
 * every voxel array is [dims[2]][dims[1]][dims[0]] contiguous device memory.
 * The voxel spacing is isotropic, so the paper's v_min is h.  Each call keeps
 * grow-only scratch per stream. */

/* Eq. V' then eq. rethresh:
 *   V'(x) = sum over k in [-R, R]^3 of w(k_x) w(k_y) w(k_z) V(x + k), V = 0
 *           outside the grid and 1 where the byte is nonzero,
 *   w(j)  = exp(-j^2 / (2 s^2)) / sum_{|i| <= R} exp(-i^2 / (2 s^2)),
 *   s = sigma / h voxels, R = ceil(3 s) (at most 32);
 *   mask  = V' >= tau (mode 0, value = tau), or V' >= the order statistic of
 *           V' of rank floor(q (N - 1)) in ascending order (mode 1, value =
 *           q in [0, 1]; exact, chosen among the float32 V' values).
 * V' is computed in float32 (weights rounded from FP64, three passes x, y,
 * z, taps summed in ascending order).
 *   surf: u8 voxels (in); out_blur: float V' (may be NULL); out_mask: u8 0/1;
 *   out_threshold: HOST float receiving the threshold used (may be NULL; in
 *   quantile mode this synchronises the stream).
 * Errors: FGL_ERR_INVALID (null pointers, bad grid, sigma <= 0 or too large,
 * mode, non-finite value, q outside [0, 1]), FGL_ERR_CUDA. */
fgl_status fgl_denoise(const uint8_t* surf, const fgl_grid* grid, float sigma, int32_t mode,
                       float value, float* out_blur, uint8_t* out_mask, float* out_threshold,
                       fgl_stream stream);

typedef struct {
  int32_t timing;        /* in: 1 = time the call with CUDA events (synchronises the stream) */
  int32_t n_layers;      /* out: shells grown, L = ceil(trunc / h) */
  int32_t n_launches;    /* out: kernels the call launched */
  float ms_total;        /* out (timing): first to last launch */
  int32_t delta_mode;    /* in: eq. delta as (p + 1/2) h (0, the default) or literally as
                            p h (1); see fgl_tsdf */
} fgl_tsdf_stats;

/* The narrow-band TSDF of a surface grid V (nonzero byte = surface voxel):
 *   sign   s = +1 on the free voxels (V = 0) reached from a one-voxel free
 *          frame around the grid through face neighbours over free voxels,
 *          s = -1 elsewhere (surface voxels and enclosed voids);
 *   shells S_0 = voxels with a face neighbour inside the grid whose V
 *          differs (eq. S_0); S_m adds the face neighbours of S_{m-1};
 *          p(x) = first m with x in S_m, for m <= L = ceil(trunc / h);
 *   phi    = s * min((p + 1/2) h, trunc), and s * trunc where p > L (eq. phi;
 *          the half voxel places the zero crossing between the two sides of
 *          S_0 instead of on grid points).  With stats->delta_mode = 1 the
 *          distance is eq. delta literally, p h: both sides of S_0 then sit
 *          at phi = +-0, and the iso = 0 level set passes through the
 *          centres of the occupied S_0 voxels, h/2 inside the default's.
 * phi is float32 and exact: (p + 1/2) h (or p h) rounds once.
 *   out_phi: float [N]; out_outside: u8 s > 0 (may be NULL); out_shell: u8
 *   p, 255 beyond L (may be NULL); stats may be NULL.
 * Asynchronous unless stats->timing.  Errors: FGL_ERR_INVALID (null pointers,
 * bad grid, more than 2^31 - 2 voxels, trunc <= 0, L > 254, delta_mode not 0
 * or 1), FGL_ERR_CUDA,
 * FGL_ERR_DEVICE (reported by the next call on the stream: a union-find
 * loop hit its N + 2 step bound, which correct input cannot cause). */
fgl_status fgl_tsdf(const uint8_t* surf, const fgl_grid* grid, float trunc, float* out_phi,
                    uint8_t* out_outside, uint8_t* out_shell, fgl_tsdf_stats* stats,
                    fgl_stream stream);

/* The level set phi = iso by marching tetrahedra on the samples of every
 * step-th voxel (paper's mc_step); sample (i, j, k) is voxel (i, j, k) * step
 * with centre origin + ((i step + 1/2) h, ...).  Each cube of eight samples
 * (corner c = dx + 2 dy + 4 dz) splits into the six tetrahedra (0,1,3,7),
 * (0,1,5,7), (0,2,3,7), (0,2,6,7), (0,4,5,7), (0,4,6,7); a sample is inside
 * when phi < iso (NaN counts as outside).  Output order (canonical, so the
 * mesh is reproducible bit for bit):
 *   vertices  one per sample edge a -> a + d (d of type t = dx + 2 dy + 4 dz,
 *             t = 1..7) whose ends disagree, by sample index then t, at
 *             P(a) + tau (P(a + d) - P(a)), tau = (iso - phi_a) / (phi_b - phi_a);
 *   triangles by cube (its lowest sample), tetrahedron, then: one corner on
 *             its own side -> the triangle on its three edges (the others in
 *             tetrahedron order); two inside (a, b) and two outside (c, d) ->
 *             (ac, ad, bd), (ac, bd, bc); a triangle whose normal through the
 *             edge midpoints points against (outside corners - inside corners)
 *             has its last two vertices swapped: normals face phi >= iso;
 *   normals   (optional) the central-difference gradient of phi on the sample
 *             grid (one-sided on the border), (1 - tau) g(a) + tau g(b),
 *             normalised.
 * The mesh is watertight wherever the level set stays inside the grid.
 *   out_verts: float [vert_capacity][3]; out_tris: int32 [tri_capacity][3];
 *   out_normals: float [vert_capacity][3] or NULL; n_verts, n_tris: HOST,
 *   receive the counts.  With out_verts, out_tris and out_normals all NULL the
 *   call only counts.
 * Synchronises the stream once (to read the counts).  Errors: FGL_ERR_INVALID
 * (null pointers, bad grid, step < 1, non-finite iso, more than 2^31 - 1
 * vertices or triangles), FGL_ERR_CAPACITY (counts set, nothing written),
 * FGL_ERR_CUDA. */
fgl_status fgl_marching_tets(const float* phi, const fgl_grid* grid, float iso, int32_t step,
                             float* out_verts, int64_t vert_capacity, int32_t* out_tris,
                             int64_t tri_capacity, float* out_normals, int64_t* n_verts,
                             int64_t* n_tris, fgl_stream stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of scan requests                             */
/* ------------------------------------------------------------------------ */
/* The paper batches thousands of environments on one GPU (Sec. IV-C; Table
 * I) but describes no request serving; this layer schedules the same casts.
 * Requests (scene, sensor, n_env environment poses, host output buffers)
 * arrive at any time.  The poses are either carried by the request or kept
 * on the device in the server's environment slots across requests (see
 * fgl_pose_source).  A worker admits requests in arrival order while their
 * device memory (own poses + results) plus any scene that must be uploaded
 * fits the HBM budget,
 * evicting least-recently-used idle scenes (the scene keeps its host copy, so
 * re-admission is an upload).  Every tick packs up to tick_rays rays from all
 * admitted requests into one batched launch, so large requests advance over
 * several ticks and requests that arrive meanwhile join the next tick.
 * The result copies of the requests a tick finishes are queued right behind
 * it; a request completes once its results are in the caller's host buffers,
 * and its latency is submission -> results in host memory.  mode 1 serves
 * the same requests the plain way (one fgl_cast per environment, one request
 * at a time) for comparison. */
typedef struct fgl_server_s* fgl_server;

typedef struct {
  int64_t hbm_budget_bytes;  /* device bytes for resident scenes + admitted
                                requests + the environment slot table (0 = 150 GiB) */
  int64_t tick_rays;         /* rays per tick (0 = 16 Mi) */
  int32_t max_active;        /* admitted requests at once (0 = 4096) */
  int32_t mode;              /* 0 = continuous batching, 1 = one launch per env */
  fgl_batch_opts opts;       /* launch options of a tick (use_graph ignored) */
  int32_t env_capacity;      /* resident environment slots (0 = 65536; at most 2^24):
                                48 B of device memory each, held from creation */
} fgl_server_opts;

/* Where a request's environment poses come from.  The server keeps a table
 * of environment slots whose poses live on the device across requests
 * (fgl_server_add_envs); a request either carries its own poses or names a
 * range of slots [env_first, env_first + n_env).  Slot updates are applied
 * when the request is admitted, in admission order; a request that updates
 * slots is admitted only once no admitted request uses any of them, and a
 * request that only scans slots waits for admitted requests updating them --
 * so each request scans exactly the poses the requests submitted before it
 * left there. */
typedef enum {
  FGL_POSES_REQUEST = 0,          /* poses: host [n_env][3][4], copied at submit, used by
                                     this request only (env_first ignored) */
  FGL_POSES_SLOTS = 1,            /* scan the slots' current poses (poses may be NULL):
                                     no pose bytes move */
  FGL_POSES_SLOTS_SET_HOST = 2,   /* overwrite the slots with host poses (copied at
                                     submit), then scan them */
  FGL_POSES_SLOTS_SET_DEVICE = 3  /* overwrite the slots with device poses (copied on the
                                     device at admission; keep them unchanged until the
                                     request completes), then scan them */
} fgl_pose_source;

typedef struct {
  int32_t scene_id;          /* from fgl_server_add_scene */
  int32_t sensor_id;         /* from fgl_server_add_sensor */
  int32_t n_env;             /* >= 1 */
  float max_range;
  const float* poses;        /* float32 [n_env][3][4], host or device per pose_source */
  float* out_range;          /* host float32 [n_env * n_rays]; page-locked is fastest
                                (pageable buffers are staged through page-locked memory) */
  int32_t* out_tri;          /* host int32  [n_env * n_rays] */
  float min_range;           /* t_min, as in fgl_cast_item (0 = none) */
  int32_t pose_source;       /* fgl_pose_source (0 = the request's own host poses) */
  int32_t env_first;         /* first environment slot (pose_source >= FGL_POSES_SLOTS) */
} fgl_request;

typedef struct {
  int32_t status;            /* the request's fgl_status */
  double queue_ms;           /* submission -> admission */
  double latency_ms;         /* submission -> results in host memory */
  int64_t rays;
} fgl_request_info;

typedef struct {
  int64_t submitted, completed, rejected, cancelled;
  int64_t evictions, uploads, ticks;
  int64_t rays;              /* rays of completed requests */
  double p50_ms, p99_ms, mean_ms;  /* latency of completed requests */
  double busy_s;             /* first submission -> last completion */
  double rays_per_s;         /* rays / busy_s */
  int64_t device_bytes;      /* held now (resident scenes + admitted requests) */
  int64_t pending, active;   /* requests waiting / admitted now */
} fgl_server_stats;

/* Create a server on the current device (worker + completion threads, two
 * streams, the environment slot table).  Errors: FGL_ERR_INVALID (mode,
 * env_capacity), FGL_ERR_BUDGET (slot table larger than the budget),
 * FGL_ERR_OOM, FGL_ERR_CUDA. */
fgl_status fgl_server_create(const fgl_server_opts* opts, fgl_server* out);
/* Register n_env environment slots holding the given initial poses (host
 * float32 [n_env][3][4], copied synchronously); their ids are
 * [*env_first, *env_first + n_env).  Slots live until fgl_server_destroy.
 * Errors: FGL_ERR_INVALID (null, n_env < 1, non-finite pose),
 * FGL_ERR_CAPACITY (more slots than env_capacity), FGL_ERR_CUDA. */
fgl_status fgl_server_add_envs(fgl_server server, int32_t n_env, const float* poses,
                               int32_t* env_first);
/* Copy the poses of slots [env_first, env_first + n_env) to host memory
 * (float32 [n_env][3][4]) as every request admitted so far left them; waits
 * for those updates.  Errors: FGL_ERR_INVALID (range), FGL_ERR_CUDA. */
fgl_status fgl_server_read_poses(fgl_server server, int32_t env_first, int32_t n_env, float* out);
/* Register a scene / sensor (the caller keeps ownership and must keep them
 * alive until fgl_server_destroy; the server uploads / evicts scenes). */
fgl_status fgl_server_add_scene(fgl_server server, fgl_scene scene, int32_t* scene_id);
fgl_status fgl_server_add_sensor(fgl_server server, fgl_sensor sensor, int32_t* sensor_id);
/* Queue a request.  Errors (synchronous): FGL_ERR_INVALID for unknown ids,
 * n_env < 1, a slot range outside the registered environments, null buffers,
 * non-finite host poses or max_range; FGL_ERR_BUDGET when the request and its
 * scene exceed the whole budget. */
fgl_status fgl_server_submit(fgl_server server, const fgl_request* req, int64_t* ticket);
/* Wait for a request (timeout_ms < 0: forever); on return the ticket is
 * released.  Returns the request's status (FGL_ERR_TIMEOUT if still running,
 * the ticket stays valid then; FGL_ERR_CANCELLED; FGL_ERR_OOM when its device
 * allocation failed). */
fgl_status fgl_server_wait(fgl_server server, int64_t ticket, int32_t timeout_ms,
                           fgl_request_info* info);
/* Cancel a request: pending ones finish at once, running ones stop taking
 * new ticks and finish when their in-flight chunks are done. */
fgl_status fgl_server_cancel(fgl_server server, int64_t ticket);
fgl_status fgl_server_get_stats(fgl_server server, fgl_server_stats* out);
fgl_status fgl_server_reset_stats(fgl_server server);
/* Fault injection for tests: the next n admissions fail their device
 * allocation (those requests complete with FGL_ERR_OOM). */
fgl_status fgl_server_inject_alloc_failures(fgl_server server, int32_t n);
/* Fault injection for tests: the next n ticks that have work throw a host
 * exception in the worker thread after they are packed and before their
 * launch.  The worker contains it: the requests with chunks in that tick
 * complete with FGL_ERR_INTERNAL (FGL_ERR_OOM for a failed host allocation),
 * no other request is affected, and the server keeps serving. */
fgl_status fgl_server_inject_worker_faults(fgl_server server, int32_t n);
/* Wait (up to 60 s) for in-flight ticks, stop the threads, free buffers. */
fgl_status fgl_server_destroy(fgl_server server);

/* Thread-local message for the last non-OK status of this thread. */
const char* fgl_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t fgl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FGL_H */
