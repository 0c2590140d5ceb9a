/*
 * vm.h -- C ABI of the GB300 voxel-map / multi-plane-segmentation library
 * (libvoxmps.so).  It implements the method of "Real-time Multi-Plane
 * Segmentation Based on GPU Accelerated High-Resolution 3D Voxel Mapping for
 * Legged Robot Locomotion" (arXiv 2510.01592): the voxel update of Sec. III.B
 * (Eq. 1) and the multi-plane segmentation of Sec. III.C (Eq. 3, Eq. 4,
 * Algorithm 1, cluster-parallel RANSAC, boundary polygons), every step as a
 * hand-written CUDA kernel for sm_103a.
 *
 * Conventions shared by every entry point:
 *  - Every call returns a vm_status.  Nothing aborts, traps or exits; on an
 *    error vm_last_error() returns a thread-local message.
 *  - Pointers are plain host or device pointers as stated per argument.  No
 *    call takes ownership of caller memory.
 *  - Work on one map is ordered on that map's CUDA stream.  Different maps may
 *    run concurrently on different streams.
 *  - Poses are row-major 3x4 [R | t] mapping sensor coordinates to map
 *    coordinates; the map frame has z up (gravity along -z).
 *  - Coordinates are metres, FP32.
 */
#ifndef VOXMPS_VM_H
#define VOXMPS_VM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VM_OK = 0,
    VM_ERR_INVALID_ARG = 1,    /* null pointer, zero/negative size, bad parameter        */
    VM_ERR_OUT_OF_MEMORY = 2,  /* a device or host allocation failed                     */
    VM_ERR_CAPACITY = 3,       /* the brick pool is full; points in new bricks dropped   */
    VM_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the CUDA error) */
    VM_ERR_TIMEOUT = 5,        /* a bounded device loop hit its iteration cap            */
    VM_ERR_EXTENT = 6          /* the grid is too large for 32-bit voxel ids             */
} vm_status;

typedef struct vm_map vm_map; /* opaque, library-owned */

/* Map geometry (Sec. III.B, 3D voxel map representation).  The grid has
 * dims[0] x dims[1] x dims[2] voxels of edge voxel_size whose lowest corner is
 * origin.  Storage is sparse: 8x8x8-voxel bricks are allocated on first touch
 * from a pool of brick_capacity bricks (0 = enough bricks for the whole grid). */
typedef struct {
    float origin[3];
    int32_t dims[3];
    float voxel_size;          /* metres; 1/voxel_size is formed in double, then rounded to FP32 */
    uint32_t brick_capacity;
    uint32_t flags;            /* VM_MAP_* bits */
} vm_map_params;

#define VM_MAP_STAGE_TIMING 1u /* record CUDA-event time per pipeline stage (vm_stage_times); implies VM_MAP_EAGER */
#define VM_MAP_EAGER 2u        /* launch the segmentation kernel by kernel instead of replaying a captured CUDA graph */

/* Segmentation parameters (Sec. III.C).  Defaults from the paper:
 * n_th = 3, theta 15 deg (cos_step = cos_ccl = 0.96592583f), d_th = 0.05 m,
 * n_hyp = I = 100, eps = 0.01 m. */
typedef struct {
    uint32_t n_th;             /* Eq. 4: minimum occupied neighbours N_th                 */
    float cos_step;            /* Eq. 4: steppable iff |n_z| >= cos_step                  */
    float d_th2;               /* Algorithm 1: edge iff |mu_i - mu_j|^2 < d_th2           */
    float cos_ccl;             /* Algorithm 1: edge iff |n_i . n_j| > cos_ccl             */
    uint32_t min_cluster;      /* clusters smaller than this are discarded                */
    uint32_t n_hyp;            /* RANSAC hypotheses per cluster (1..1024)                 */
    float eps;                 /* RANSAC inlier threshold: |n.p + d| <= eps               */
    uint64_t seed;             /* Philox4x64-10 key word 0                                */
    uint32_t classify;         /* 1: cluster steppable voxels only (paper); 0: all occupied */
    uint32_t planes_per_cluster; /* extraction rounds per cluster, 0 or 1: one plane (paper); up to 8.
                                  Round q + 1 fits the points of round q that are not its inliers
                                  (in order), Philox counter (label, h, q + 1, 0), when round q found
                                  a plane with >= min_cluster inliers and >= min_cluster points
                                  remain; it is output when it finds a plane.  vm_segment only.  */
} vm_segment_params;

/* One output plane: one per cluster (per extraction round when
 * planes_per_cluster > 1), in ascending label order, then round order. */
typedef struct {
    float normal[3];           /* refit normal (total least squares on the inliers), n_z >= 0 */
    float offset;              /* refit plane: normal . x + offset = 0                       */
    uint32_t inlier_count;     /* inliers of the selected RANSAC hypothesis                  */
    uint32_t label;            /* cluster label: smallest voxel id of the cluster / caller label */
    float ransac_normal[3];    /* selected hypothesis (bit-exact to the reference reading)   */
    float ransac_offset;
    float basis_u[3];          /* in-plane basis from the RANSAC normal                      */
    float basis_v[3];
    float hull_origin[3];      /* the cluster's first point                                  */
    uint32_t hull_offset;      /* first vertex in vm_planes.hull_xy / hull_xyz               */
    uint32_t hull_count;       /* vertices, counter-clockwise from the lexicographic minimum */
    uint32_t n_points;         /* points in the cluster                                      */
    int32_t best_h;            /* selected hypothesis index; -1: no valid hypothesis, no plane */
    uint32_t flags;            /* bit 0: refit ill-conditioned (lambda_mid < 10 lambda_min);
                                  bits 8-15: extraction round of the plane in its cluster     */
} vm_plane;

/* Result of vm_segment / vm_fit_planes; host memory owned by the library
 * until vm_planes_free. */
typedef struct {
    vm_plane* planes;
    uint32_t n_planes;
    int32_t* hull_xy;          /* [n_hull][2] in-plane coordinates, units of 2^-16 m */
    float* hull_xyz;           /* [n_hull][3] hull vertices lifted onto the refit plane, map frame */
    uint32_t n_hull;
} vm_planes;

typedef struct {
    uint64_t points_integrated;  /* points accumulated since creation / reset     */
    uint64_t points_dropped;     /* NaN, Inf or outside the grid                  */
    uint64_t points_no_capacity; /* dropped because the brick pool was full       */
    uint32_t bricks_allocated;
    uint32_t brick_capacity;
    uint32_t occupied_voxels;    /* at the last segmentation                      */
    uint32_t steppable_voxels;   /* at the last segmentation                      */
    uint32_t clusters;           /* kept clusters at the last segmentation        */
    uint32_t clustered_points;   /* points in kept clusters at the last segmentation */
    uint64_t device_bytes;       /* device memory held by the map                 */
    uint64_t voxels_cleared;     /* voxels cleared by ray casting since creation / reset */
    uint64_t voxels_evicted;     /* occupied voxels evicted by vm_scroll since creation / reset */
} vm_stats;

/* Create a map.  params: see vm_map_params.  cuda_stream: a cudaStream_t the
 * map's work is ordered on, or NULL to let the library create one.  On
 * success *out holds the map.  Errors: VM_ERR_INVALID_ARG (dims <= 0,
 * voxel_size <= 0, an extent beyond 16 m per axis), VM_ERR_EXTENT (more than
 * 2^32 voxel ids), VM_ERR_OUT_OF_MEMORY, VM_ERR_CUDA.  Sec. III.B. */
vm_status vm_create(const vm_map_params* params, void* cuda_stream, vm_map** out);

/* Voxel information update (Sec. III.B, Eq. 1), one thread per point.
 * xyz: n points, float32[n][3] (AoS), device memory if xyz_on_device != 0,
 * otherwise host memory (copied on the map's stream; pinned memory makes the
 * copy asynchronous).  pose3x4: host pointer to 12 floats, sensor->map.
 * Each point is transformed, keyed to its voxel, and accumulated as exact
 * fixed-point sums (2^-20 m units) plus a count; NaN/Inf points and points
 * outside the grid are dropped and counted.  Asynchronous on the map's stream
 * unless xyz is pageable host memory.  Errors: VM_ERR_INVALID_ARG,
 * VM_ERR_CUDA; a full brick pool is reported by the next vm_segment /
 * vm_get_stats as VM_ERR_CAPACITY. */
vm_status vm_integrate(vm_map* map, const float* xyz, uint32_t n, const float pose3x4[12], int xyz_on_device);

/* Voxel information clearing (Sec. III.B, Eq. 2) before the update.
 * flags: VM_INTEGRATE_CLEAR first clears every occupied voxel that the ray
 * from the sensor (the pose's translation) to one of the frame's points
 * passes through, the point's own voxel excepted, then integrates the frame
 * as vm_integrate does.  The ray is walked voxel by voxel from the sensor's
 * voxel to the point's (a monotone 6-connected grid traversal: each step on
 * the axis whose next voxel boundary comes first, ties to x, then y, then z,
 * among the axes not yet at the point's voxel coordinate; FP32, explicit
 * rounding), and stops where it leaves the grid.  A sensor outside the grid
 * casts no rays; points that are not finite cast none.  Other arguments and
 * errors as vm_integrate; cleared voxels are counted in vm_stats. */
#define VM_INTEGRATE_CLEAR 1u
vm_status vm_integrate_ex(vm_map* map, const float* xyz, uint32_t n, const float pose3x4[12], int xyz_on_device,
                          uint32_t flags);

/* Multi-plane segmentation of the accumulated map (Sec. III.C): mean
 * positions, normals and steppable classification (Eq. 3, Eq. 4), clustering
 * (Algorithm 1, as union-find over the same adjacency), clusters of at least
 * min_cluster voxels, per-cluster RANSAC (stages a-c), inlier refit and
 * convex hull.  Synchronises the map's stream.  *out receives library-owned
 * host arrays (free with vm_planes_free).  Errors: VM_ERR_INVALID_ARG,
 * VM_ERR_CAPACITY (the pool overflowed since the last call; the result covers
 * the points that fitted), VM_ERR_TIMEOUT, VM_ERR_OUT_OF_MEMORY, VM_ERR_CUDA. */
vm_status vm_segment(vm_map* map, const vm_segment_params* params, vm_planes* out);

/* Free the host arrays of a vm_planes and zero it.  NULL members are fine. */
vm_status vm_planes_free(vm_planes* planes);

/* Clear the map (every voxel free) without releasing memory; the window
 * (below) stays where it is. */
vm_status vm_reset(vm_map* map);

/* Robot-centric map (Sec. III.B: the map's centre follows the robot).  A
 * point's key is floor((p - origin) * inv_res) from the map's fixed base
 * origin (vm_map_params.origin); the grid of dims voxels is a window over
 * keys offset..offset + dims - 1, offset a multiple of 8 per axis (whole
 * bricks), 0 at creation.  vm_scroll moves the window by shift_bricks[3]
 * bricks: voxels whose brick leaves it are evicted (counted in vm_stats),
 * the bricks that enter are empty, and every kept voxel keeps its key, its
 * points and its exact sums.  Voxel ids (labels, exports) are window
 * coordinates, so they change with the window; planes and hulls stay in the
 * map frame.  The offset must stay within +-2^23 voxels (keys exact in
 * FP32): VM_ERR_INVALID_ARG otherwise, the window unchanged.  Sums exported
 * by vm_export_voxels are relative to the window's anchor, 2^-20 m units:
 * the mean position is position_origin + (sums / count) * 2^-20.  Precision
 * of keys and sums is that of FP32 offsets from the base origin (about 1 um
 * at 16 m, 8 um at 128 m).  Asynchronous on the map's stream; no graph is
 * re-captured.
 * vm_scroll_target: the shift that centres the window on center[3] (map
 * frame): the new offset is the centre's key minus dims / 2, rounded down to
 * a multiple of 8.  vm_scroll_to: vm_scroll_target then vm_scroll (shift may
 * be NULL).  vm_get_window: the offset (voxels) and position origin (map
 * frame); either may be NULL. */
vm_status vm_scroll(vm_map* map, const int32_t shift_bricks[3]);
vm_status vm_scroll_target(vm_map* map, const float center[3], int32_t shift_bricks[3]);
vm_status vm_scroll_to(vm_map* map, const float center[3], int32_t shift_bricks[3]);
vm_status vm_get_window(vm_map* map, int32_t offset_voxels[3], float position_origin[3]);

/* Destroy a map and release its device memory; waits for its stream.  A NULL
 * map is accepted and does nothing (VM_OK). */
vm_status vm_destroy(vm_map* map);

/* Counters of the map; synchronises its stream. */
vm_status vm_get_stats(vm_map* map, vm_stats* out);

/* Batched plane fitting on caller-formed clusters (Sec. III.C multi-plane
 * estimation and boundary polygons; the cluster-parallel form of Sec. IV-C):
 * one persistent RANSAC launch over all clusters, then refit and hull.
 * xyz: device float32[off[k]][3]; off: device uint32[k+1], cluster c holds
 * points off[c]..off[c+1]-1; labels: device uint32[k] keying each cluster's
 * Philox stream, or NULL for label = c.  stream: cudaStream_t or NULL (the
 * legacy default stream).  Synchronises the stream.  Errors:
 * VM_ERR_INVALID_ARG, VM_ERR_OUT_OF_MEMORY, VM_ERR_TIMEOUT, VM_ERR_CUDA. */
vm_status vm_fit_planes(const float* xyz, const uint32_t* off, const uint32_t* labels, uint32_t k,
                        const vm_segment_params* params, void* stream, vm_planes* out);

/* ---- Reusable batched fit ------------------------------------------------
 * The cluster-parallel plane fit of vm_fit_planes (Sec. III.C multi-plane
 * estimation stages a-c, refit, boundary polygons) as a reusable plan: the
 * plan owns every device buffer a batch needs, a result block in mapped
 * pinned host memory and one CUDA graph of the whole fit (hypotheses,
 * persistent scoring, selection, extraction, refit, hull, pack), so a run
 * with the same input pointers replays one graph and allocates nothing.
 * A batch larger than any seen so far (more clusters, points or hull
 * vertices) grows the buffers, captures again and re-runs.  Results are
 * identical to vm_fit_planes bit for bit under every tuning: the refit's
 * partial sums are formed per 256-point chunk of a cluster whatever the
 * work-item tile, and a cluster's result never depends on its batch. */
typedef struct vm_fit_plan vm_fit_plan; /* opaque, library-owned */

typedef struct {
    uint32_t tile;           /* points per work item, a multiple of 256 in 256..16384       */
    uint32_t hyp_per_thread; /* hypotheses each thread holds in registers: 1, 2, 4 or 8    */
    uint32_t ctas_per_sm;    /* persistent scoring CTAs per SM, 1..16                      */
    uint32_t schedule;       /* 0: a 256-thread CTA per work item; 1: a warp per work item  */
} vm_fit_tuning;

#define VM_FIT_STAGE_TIMING 1u /* CUDA-event time per stage (vm_fit_plan_stage_times); implies VM_FIT_EAGER */
#define VM_FIT_EAGER 2u        /* launch kernel by kernel instead of replaying the graph */

/* Creates a plan sized for k_cap clusters and n_cap points with params
 * (n_hyp, eps, seed are used).  stream: cudaStream_t or NULL (the library
 * creates one).  flags: 0, VM_FIT_EAGER or VM_FIT_STAGE_TIMING.  Errors: VM_ERR_INVALID_ARG,
 * VM_ERR_OUT_OF_MEMORY, VM_ERR_CUDA. */
vm_status vm_fit_plan_create(uint32_t k_cap, uint32_t n_cap, const vm_segment_params* params, void* stream,
                             uint32_t flags, vm_fit_plan** out);
/* Fits k clusters: xyz device float32[off[k]][3]; off device uint32[k+1];
 * labels device uint32[k] or NULL (label = index); the pointers must stay
 * valid until the call returns.  Synchronises the plan's stream; *out is
 * host memory owned by the library until vm_planes_free.  Errors as
 * vm_fit_planes. */
vm_status vm_fit_plan_run(vm_fit_plan* plan, const float* xyz, const uint32_t* off, const uint32_t* labels,
                          uint32_t k, vm_planes* out);
/* Asynchronous half of a run: enqueues the fit on the plan's stream and
 * returns; vm_fit_plan_wait synchronises and fills *out (NULL: only waits).
 * One launch at a time per plan. */
vm_status vm_fit_plan_launch(vm_fit_plan* plan, const float* xyz, const uint32_t* off, const uint32_t* labels,
                             uint32_t k);
vm_status vm_fit_plan_wait(vm_fit_plan* plan, vm_planes* out);
vm_status vm_fit_plan_set_tuning(vm_fit_plan* plan, const vm_fit_tuning* tuning);
vm_status vm_fit_plan_get_tuning(const vm_fit_plan* plan, vm_fit_tuning* tuning);
/* Autotuner (no counterpart in the paper): times the whole fit of this batch
 * (CUDA events around graph replays, reps timed runs after one warm-up run)
 * for each candidate tuning -- CTA-per-item tiles of 1024..8192 points and
 * warp-per-item tiles of 256..1024 points, 2..8 hypotheses per thread,
 * persistent CTAs per SM up to the occupancy limit -- and keeps the fastest.
 * *best and *best_ms (either may be NULL) receive it; *n_tried the number of
 * candidates timed.  Errors as vm_fit_plan_run. */
vm_status vm_fit_plan_autotune(vm_fit_plan* plan, const float* xyz, const uint32_t* off, const uint32_t* labels,
                               uint32_t k, uint32_t reps, vm_fit_tuning* best, float* best_ms, uint32_t* n_tried);
/* Device milliseconds and call counts per stage (names: vm_stage_name) since
 * the previous call, for a plan created with VM_FIT_STAGE_TIMING; then reset.
 * ms[cap], calls[cap] host arrays, either may be NULL. */
vm_status vm_fit_plan_stage_times(vm_fit_plan* plan, double* ms, uint64_t* calls, uint32_t cap, uint32_t* n_stages);
vm_status vm_fit_plan_destroy(vm_fit_plan* plan);

/* RANSAC without allocation.  The paper has no counterpart: this entry point
 * serves callers that must not allocate device memory while they run -- a
 * robot control loop with a hard deadline (cudaMalloc can stall on
 * device-wide synchronisation for an unbounded time) or a host program whose
 * device memory is owned up front by another allocator.  It runs the same
 * hypothesis, scoring and selection kernels as vm_fit_planes on
 * caller-formed clusters, with all scratch in one array compiled into the
 * library (about 11 MiB); it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 * Set-up: the array is placed on a GPU when the library's device code is
 * loaded there, which with lazy module loading (the CUDA default) happens at
 * the first call made on that device; that call also looks up the array's
 * device address (with the device current) and caches it.  Make that first
 * call during set-up, before any stream capture: a call with k == 0 does the
 * set-up and launches nothing.  From then on the array stays on that device
 * until the process exits.  The cached address does not survive
 * cudaDeviceReset (or any other teardown of the device's primary context):
 * do not call this entry point after one.
 * Limits: k <= 4096 clusters and k * n_hyp <= 524288; larger requests return
 * VM_ERR_CAPACITY with a message and launch nothing.
 * Inputs (device): xyz float32[off[k]][3]; off uint32[k+1]; labels uint32[k]
 * or NULL (label = cluster index).  Outputs (device, caller-owned):
 * planes_out float32[k][4] = (n_x, n_y, n_z, d) of the selected hypothesis,
 * best_h_out int32[k] (-1: no valid hypothesis), inliers_out uint32[k].
 * Results equal vm_fit_planes' ransac_normal / ransac_offset / best_h /
 * inlier_count bit for bit.  Asynchronous on stream (NULL: legacy default
 * stream); outputs are ready once the stream has synchronised.
 * Every call on a device shares the one scratch array, which keeps the last
 * call's contents (the work queue and counters are cleared at the start of
 * each call): calls whose work overlaps on the GPU race, so serialise them
 * (one stream, or events). */
vm_status vm_ransac_static(const float* xyz, const uint32_t* off, const uint32_t* labels, uint32_t k,
                           const vm_segment_params* params, void* stream, float* planes_out, int32_t* best_h_out,
                           uint32_t* inliers_out);

/* Debug / parity export of the occupied voxels, in voxel-id order.  Voxel ids
 * are brick-major: bricks of 8^3 voxels numbered x-fastest over the brick
 * grid, voxels inside a brick x-fastest.  Host output arrays of capacity cap:
 * vid[cap], sums[cap][3] (int64, 2^-20 m units relative to the origin),
 * counts[cap]; *n receives the number of occupied voxels (if > cap only cap
 * are written).  Any output pointer may be NULL.  Synchronises. */
vm_status vm_export_voxels(vm_map* map, uint32_t* vid, int64_t* sums, uint32_t* counts, uint32_t cap, uint32_t* n);

/* Debug / parity export of the last vm_segment's per-voxel state, in voxel-id
 * order over the occupied voxels: normal[cap][3], status[cap] (1 occupied,
 * 2 steppable), label[cap] (smallest voxel id of the voxel's component, or
 * 0xFFFFFFFF when the voxel is not clustered), nbr[cap] (occupied neighbours
 * N).  Host arrays; any may be NULL.  Synchronises. */
vm_status vm_export_labels(vm_map* map, uint32_t* vid, float* normal, uint8_t* status, uint32_t* label,
                           uint32_t* nbr, uint32_t cap, uint32_t* n);

/* Debug / parity export of the last vm_segment's cluster points: pts[cap][3]
 * (mean positions in cluster order), vid[cap] (their voxel ids) and
 * inlier[cap] (1 if an inlier of the cluster's selected hypothesis).  Host
 * arrays; any may be NULL; *n receives the point count.  Synchronises. */
vm_status vm_export_clusters(vm_map* map, float* pts, uint32_t* vid, uint8_t* inlier, uint32_t cap, uint32_t* n);

/* Fit schedule of a map's segmentations (work-item tile, hypotheses per
 * thread, persistent scoring CTAs per SM, CTA or warp per item; see
 * vm_fit_tuning).  Results never depend on it.  tuning NULL: the automatic
 * choice (the library default, 2048-point CTA items).  Errors:
 * VM_ERR_INVALID_ARG (out of range). */
vm_status vm_set_fit_tuning(vm_map* map, const vm_fit_tuning* tuning);
vm_status vm_get_fit_tuning(vm_map* map, vm_fit_tuning* tuning);
/* Autotuner for a map's segmentation (no counterpart in the paper): replays
 * the segmentation of the map as it stands (segmenting does not change the
 * map) under each candidate schedule -- CTA-per-item tiles of 512..4096
 * points, warp-per-item tiles of 256..1024 points, 2..8 hypotheses per
 * thread, 2..8 scoring CTAs per SM within the occupancy limit -- timing reps
 * runs of each with CUDA events after one warm-up run, and keeps the fastest.
 * *best, *best_ms, *n_tried may be NULL.  Synchronises the map's stream. */
vm_status vm_autotune_segment(vm_map* map, const vm_segment_params* params, uint32_t reps, vm_fit_tuning* best,
                              float* best_ms, uint32_t* n_tried);

/* ---- Serving ---------------------------------------------------------------
 * The paper runs one robot's map.  A server runs many sensor streams at once,
 * each with its own map kept resident on the device (no counterpart in the
 * paper; every request computes exactly the paper's integrate + segment for
 * its stream, and its result is the same as that stream's alone).
 * A request integrates one frame into its stream's map (Sec. III.B) and
 * segments the map (Sec. III.C).  Requests of one stream run in submission
 * order; requests of different streams overlap on the GPU.  A scheduler thread
 * owned by the server forms steps as requests arrive and GPU slots free up
 * (continuous batching): in VM_SERVE_BATCHED mode each request of a step
 * integrates and runs the front half of its segmentation (brick order ..
 * cluster points) on its map's stream, then the clusters of every map in the
 * step go through one batched fit (one persistent RANSAC launch, refit and
 * hull over all of them) on the server's stream, and each map's planes are
 * packed into its own result block; in VM_SERVE_STREAMS mode each request
 * replays its map's whole segmentation graph on its map's stream.
 * Admission by device memory: a stream is admitted when its worst-case
 * footprint (map pool at its brick capacity, segmentation scratch, result
 * block, input staging) fits in what is left of the budget; until then it
 * waits, its requests queued, and streams are admitted in the order they were
 * opened as closing streams free memory. */
typedef struct vm_server vm_server; /* opaque, library-owned */

#define VM_SERVE_BATCHED 0u
#define VM_SERVE_STREAMS 1u

typedef struct {
    uint32_t mode;             /* VM_SERVE_BATCHED or VM_SERVE_STREAMS                       */
    uint32_t max_batch;        /* requests per step at most, 1..64; VM_SERVE_BATCHED also
                                  caps a step at ceil(streams with work / max_inflight), so
                                  that with every stream busy the steps in flight share the
                                  streams and one step's front halves overlap another's fit */
    uint32_t max_inflight;     /* steps on the GPU at once, 1..4 (VM_SERVE_STREAMS: requests
                                  in flight at once is max_batch * max_inflight)              */
    uint32_t device;           /* CUDA device ordinal the server runs on                     */
    uint64_t hbm_budget;       /* bytes the streams may hold; 0: free device memory at
                                  creation minus hbm_reserve                                  */
    uint64_t hbm_reserve;      /* bytes kept free when hbm_budget is 0                        */
    vm_segment_params params;  /* segmentation parameters of every request                   */
    vm_fit_tuning tuning;      /* batched-fit schedule; tile 0 = the library default          */
} vm_server_params;

typedef struct {
    uint64_t ticket;           /* from vm_server_submit                                      */
    uint32_t stream;           /* stream id                                                  */
    vm_status status;          /* of this request (its planes are valid when VM_OK)          */
    vm_planes planes;          /* host memory owned by the caller: release with vm_planes_free */
    double t_arrival;          /* seconds on the server clock (vm_server_now)                */
    double t_start;            /* the request's step was launched                            */
    double t_done;             /* the result was ready on the host                           */
} vm_server_result;

typedef struct {
    uint32_t streams_open;     /* opened and not yet closed                                  */
    uint32_t streams_admitted; /* holding a map on the device                                */
    uint32_t streams_waiting;  /* opened, waiting for memory                                 */
    uint32_t reserved;
    uint64_t requests_submitted, requests_done, steps;
    uint64_t fallbacks;        /* requests re-run on their own map's path after a capacity miss */
    uint64_t hbm_budget, hbm_committed;
    double mean_step_requests; /* requests per step                                          */
    double launch_seconds;     /* scheduler-thread time spent launching steps                */
    double complete_seconds;   /* scheduler-thread time spent completing steps (result copies) */
    uint64_t graph_captures;   /* CUDA graphs captured by the library since the server started */
    uint64_t allocations;      /* device / pinned allocations by the library since then      */
} vm_server_stats;

/* Creates a server and starts its scheduler thread.  Errors:
 * VM_ERR_INVALID_ARG, VM_ERR_OUT_OF_MEMORY, VM_ERR_CUDA. */
vm_status vm_server_create(const vm_server_params* params, vm_server** out);
/* Opens a stream with its own map (params as vm_create); returns at once with
 * *stream_id.  The map is created when the stream is admitted.
 * VM_ERR_OUT_OF_MEMORY when its footprint exceeds the whole budget (it could
 * never be admitted); VM_ERR_INVALID_ARG / VM_ERR_EXTENT as vm_create. */
vm_status vm_server_open(vm_server* srv, const vm_map_params* map, uint32_t* stream_id);
/* Queues a request on a stream: xyz float32[n][3] in the sensor frame (device
 * memory if xyz_on_device, else host memory), pose3x4 copied.  xyz must stay
 * valid until the request's result has been polled.  t_arrival: the arrival
 * time on the server clock, or a negative value for now.  *ticket (may be
 * NULL) identifies the result.  Errors: VM_ERR_INVALID_ARG (unknown or closed
 * stream). */
vm_status vm_server_submit(vm_server* srv, uint32_t stream_id, const float* xyz, uint32_t n, const float pose3x4[12],
                           int xyz_on_device, double t_arrival, uint64_t* ticket);
/* Moves up to cap finished results into out[] (oldest first), waiting up to
 * timeout_ms (0: no wait, negative: until one is there) for the first; *n
 * receives the count. */
vm_status vm_server_poll(vm_server* srv, vm_server_result* out, uint32_t cap, uint32_t* n, int timeout_ms);
/* Waits until every submitted request has a result ready to poll (up to
 * timeout_ms; negative: no limit).  VM_ERR_TIMEOUT when the time ran out. */
vm_status vm_server_drain(vm_server* srv, int timeout_ms);
/* Closes a stream: its queued requests still run; then its map is destroyed
 * and its memory returns to the budget. */
vm_status vm_server_close(vm_server* srv, uint32_t stream_id);
vm_status vm_server_get_stats(vm_server* srv, vm_server_stats* out);
/* Device bytes vm_server_open would reserve for a map with these parameters. */
uint64_t vm_server_footprint(const vm_map_params* map, const vm_segment_params* params);
/* The server clock: seconds since the server was created (monotonic). */
double vm_server_now(vm_server* srv);
/* Stops the scheduler after the requests in flight, destroys every map.
 * Results not polled are released. */
vm_status vm_server_destroy(vm_server* srv);

/* Diagnostics (no counterpart in the paper).  Stage timing records CUDA
 * events around each pipeline stage on the stream it runs on: integrate,
 * order_bricks, finalize, moments, eigen, ccl_local, ccl_cross, clusters,
 * ransac_hyp, ransac_score, extract, refit_hull, pack, clear, rounds
 * (vm_stage_name gives the names; the RANSAC stages of every extraction round
 * add up under their own names, the work between rounds under rounds).
 * vm_stage_timing: enable (1) or disable (0) for a map, or for this thread's
 * vm_fit_planes calls when map is NULL.  vm_stage_times: device milliseconds
 * and call counts per stage accumulated since the previous call (then reset);
 * ms[cap], calls[cap] host arrays, either may be NULL; *n_stages receives the
 * stage count.  Synchronises the map's stream. */
vm_status vm_stage_timing(vm_map* map, int enable);
vm_status vm_stage_times(vm_map* map, double* ms, uint64_t* calls, uint32_t cap, uint32_t* n_stages);
const char* vm_stage_name(uint32_t stage);

/* Number of CUDA kernel launches the library has issued in this process
 * (kernels of a replayed graph count at each replay, not at capture). */
uint64_t vm_launch_count(void);
/* Number of CUDA graphs the library has captured, and of device or pinned
 * host allocations it has made, in this process (a map whose scratch grows
 * re-allocates and re-captures; both should stay flat in a steady state). */
uint64_t vm_capture_count(void);
uint64_t vm_allocation_count(void);
/* Shape of the map's captured segmentation graph (zeros before the first
 * graph segmentation, or for a map created with VM_MAP_EAGER): its kernel and
 * memcpy nodes, its dependency edges, and how many of those edges are
 * programmatic -- kernel-to-kernel dependencies that, like the programmatic
 * stream launches they were captured from, let the next kernel launch before
 * the one it depends on has finished.  Any pointer may be NULL. */
vm_status vm_graph_shape(vm_map* map, uint32_t* nodes, uint32_t* edges, uint32_t* programmatic);

/* Thread-local message describing the last error of this thread. */
const char* vm_last_error(void);

/* Library version string. */
const char* vm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VOXMPS_VM_H */
