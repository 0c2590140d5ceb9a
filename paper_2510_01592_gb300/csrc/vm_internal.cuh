// vm_internal.cuh -- internal declarations shared by the CUDA translation units
// of libvoxmps.so (not installed, not part of the C ABI).
//
// Numerics: every floating-point operation whose result decides an integer
// (a voxel index, a classification, an edge, an inlier) is written with an
// explicit IEEE round-to-nearest intrinsic (__fmaf_rn, __fmul_rn, __fadd_rn,
// __fsub_rn, __fdiv_rn, __fsqrt_rn) so the op sequence is fixed regardless of
// compiler contraction; the library is also built with --fmad=false.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/vm.h"

namespace vmx {

// Programmatic dependent launch (sm_90 and later).  Every kernel of the
// library opens with pdl_gate(): griddepcontrol.wait blocks until the kernel
// launched before it on the stream has completed and its memory is visible (a
// no-op for a launch that was not programmatic), then
// griddepcontrol.launch_dependents lets the next kernel on the stream start
// launching.  So each launch, and the rasterisation of its CTAs, overlaps the
// kernel before it instead of following it: in a chain of small kernels (a
// segmentation is ~40) that gap, not the work, is most of the time.  A kernel
// touches no global memory before the gate, so ordering is that of plain
// stream launches.  A long, issue-bound kernel that leaves room on its SMs
// (the persistent RANSAC scoring) waits without the early trigger
// (pdl_wait): its dependents then launch as it finishes instead of sitting
// resident beside it for its whole run.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_gate() {
    pdl_wait();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Whether launch_k marks launches programmatic (on unless the environment
// variable VOXMPS_PDL is "0"; read once).
bool pdl_enabled();
template <typename... K, typename... A>
cudaError_t launch_as(bool programmatic, void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      A&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = programmatic && pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}
// kernel<<<grid, block, smem, s>>>(args...) as a programmatic launch.
template <typename... K, typename... A>
cudaError_t launch_k(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    return launch_as(true, kernel, grid, block, smem, s, std::forward<A>(args)...);
}
// A plain launch, for a kernel whose grid is sized to fill the GPU and whose
// work is balanced by that placement (the persistent scoring, the chunked
// extraction passes): launched early beside the kernel before it, its CTAs
// would land unevenly on the SMs that kernel frees first.
template <typename... K, typename... A>
cudaError_t launch_full(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    return launch_as(false, kernel, grid, block, smem, s, std::forward<A>(args)...);
}

constexpr int kBrick = 8;
constexpr int kBrickVox = 512;
constexpr uint32_t kNone = 0xFFFFFFFFu;

// Device error word bits.
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrOverflow = 4u;
constexpr uint32_t kErrScratch = 8u;   // counts exceeded the scratch the work was launched with

// Iteration cap of every device retry loop (union-find, work queues).
constexpr int kLoopCap = 1 << 22;

struct Pose {
    float r[12];
};

// Grid geometry passed to kernels by value.
struct Grid {
    int nx, ny, nz;
    int nbx, nby, nbz;
    float ox, oy, oz;       // base origin: a point's key is floor((p - origin) * inv_res)
    float inv_res;
    int wx, wy, wz;         // window: the grid holds keys w .. w + n - 1 (multiples of 8)
    long long ax, ay, az;   // sums are rint((p - origin) * 2^20) - a, a = the window's anchor
    const float* po;        // device float[3]: origin of the mean positions (origin + a * 2^-20)
};

// Counters kept in device memory per map.
struct MapCounters {
    unsigned long long integrated;
    unsigned long long dropped;
    unsigned long long no_capacity;
    uint32_t n_bricks;   // bricks allocated (may exceed capacity on overflow)
    uint32_t err;        // error bits
    unsigned long long cleared;  // voxels cleared by ray casting (Eq. 2)
    unsigned long long evicted;  // occupied voxels evicted by scrolling the window
    uint32_t n_deferred;         // points of the frame waiting for their brick's claim (k_accum_deferred)
    uint32_t deferred_done;      // CTAs of k_accum_deferred finished
};

// Counters produced by one segmentation, read back by the host.
struct SegCounters {
    uint32_t n_sorted;   // bricks in key order
    uint32_t n_occ;      // occupied voxels
    uint32_t n_vert;     // clustered vertices (steppable or all occupied)
    uint32_t n_kept;     // clustered vertices in kept clusters
    uint32_t k;          // kept clusters
    uint32_t n_hull;     // hull vertices
    uint32_t err;        // error bits
    uint32_t tot;        // scan total scratch
    uint32_t n_bricks;   // bricks allocated in the pool (copied at the end)
    uint32_t map_err;    // map error bits (copied at the end)
    uint32_t fit_err;    // fit error bits (copied at the end)
    uint32_t n_list;     // occupied voxels listed for the eigen-solve
    uint32_t n_planes;   // output plane records (k, or more with several extraction rounds)
    uint32_t k_need;     // kept clusters before clamping to the scratch (sizes a re-run)
    uint32_t pad[2];
};

// Per-cluster fit state on the device.
struct FitCluster {
    float n[3];          // selected RANSAC plane
    float d;
    float u[3], v[3];    // in-plane basis
    float o[3];          // hull origin = first point of the cluster
    float c[3];          // inlier centroid
    int32_t best_h;
    uint32_t inliers;
    uint32_t n_surv;     // hull candidates after the octagon filter
    uint32_t hull_n;
    uint32_t hull_off;
    uint32_t flags;
    float refit_n[3];
    float refit_d;
    unsigned long long ext[16]; // filter extremes: (biased value << 32) | point index
};

// One cluster's output record: the refit plane, the selected hypothesis, the
// hull basis and origin; ho / hn: its first hull vertex and vertex count.
__device__ __forceinline__ vm_plane make_plane(const FitCluster& f, uint32_t label, uint32_t n_points, uint32_t ho,
                                               uint32_t hn) {
    vm_plane p;
    for (int a = 0; a < 3; ++a) {
        p.normal[a] = f.refit_n[a];
        p.ransac_normal[a] = f.n[a];
        p.basis_u[a] = f.u[a];
        p.basis_v[a] = f.v[a];
        p.hull_origin[a] = f.o[a];
    }
    p.offset = f.refit_d;
    p.ransac_offset = f.d;
    p.inlier_count = f.inliers;
    p.label = label;
    p.hull_offset = ho;
    p.hull_count = hn;
    p.n_points = n_points;
    p.best_h = f.best_h;
    p.flags = f.flags;
    return p;
}

// Writes hull vertex q (2^-16 m units in p's basis) at index at of the output
// arrays: the quantised pair and the point lifted onto p's refit plane.
__device__ __forceinline__ void write_vertex(const vm_plane& p, int2 q, uint32_t at, int32_t* __restrict__ hull_xy,
                                             float* __restrict__ hull_xyz) {
    hull_xy[2 * at] = q.x;
    hull_xy[2 * at + 1] = q.y;
    const float a = q.x * (1.0f / 65536.0f), b = q.y * (1.0f / 65536.0f);
    const float x = p.hull_origin[0] + a * p.basis_u[0] + b * p.basis_v[0];
    const float y = p.hull_origin[1] + a * p.basis_u[1] + b * p.basis_v[1];
    const float z = p.hull_origin[2] + a * p.basis_u[2] + b * p.basis_v[2];
    const float e = p.normal[0] * x + p.normal[1] * y + p.normal[2] * z + p.offset;
    hull_xyz[3 * at] = x - e * p.normal[0];
    hull_xyz[3 * at + 1] = y - e * p.normal[1];
    hull_xyz[3 * at + 2] = z - e * p.normal[2];
}

// Writes one cluster's output record and its hull vertices (called by a whole
// block; thread 0 writes the record).  ho is the cluster's first vertex in
// the output arrays, hn its vertex count; vertices at or beyond hull_cap are
// not written.
__device__ __forceinline__ void pack_cluster(const FitCluster& f, uint32_t label, uint32_t n_points,
                                             const int2* __restrict__ hull_src, uint32_t ho, uint32_t hn,
                                             vm_plane* __restrict__ plane, int32_t* __restrict__ hull_xy,
                                             float* __restrict__ hull_xyz, uint32_t hull_cap) {
    const vm_plane p = make_plane(f, label, n_points, ho, hn);
    if (threadIdx.x == 0) *plane = p;
    for (uint32_t i = threadIdx.x; i < hn && ho + i < hull_cap; i += blockDim.x)
        write_vertex(p, hull_src[i], ho + i, hull_xy, hull_xyz);
}

// ---------------------------------------------------------------- diagnostics
// Pipeline stages timed by the optional stage timer.
enum Stage {
    kStIntegrate = 0,  // claim + accumulate (and ray-cast clearing when asked)
    kStOrder,          // bricks in key order
    kStFinalize,       // integer means
    kStNormals,        // Eq. 3 window moments (k_moments)
    kStEigen,          // Eq. 3 eigen-solve + Eq. 4 (k_eigen)
    kStCclLocal,       // Algorithm 1 inside bricks (k_ccl_local)
    kStCcl,            // Algorithm 1 across bricks (k_ccl_cross, k_ccl_compress)
    kStClusters,       // sizes, numbering, compaction, sort, gather
    kStHyp,            // stage a
    kStScore,          // stage b
    kStExtract,        // stage c, inliers, centroid, filter
    kStHull,           // refit + hull
    kStPack,           // output records
    kStClear,          // Eq. 2 ray-cast clearing (before the frame's integration)
    kStRounds,         // further extraction rounds: staging, remaining points, final order
    kNumStages
};

// Records device time of stages on a stream (events); null = disabled.
struct StageHook {
    virtual void begin(int stage, cudaStream_t s) = 0;
    virtual void end(int stage, cudaStream_t s) = 0;
    virtual ~StageHook() {}
};
#define VM_STAGE_BEGIN(hk, st, s) \
    do {                          \
        if (hk) (hk)->begin((st), (s)); \
    } while (0)
#define VM_STAGE_END(hk, st, s) \
    do {                        \
        if (hk) (hk)->end((st), (s)); \
    } while (0)

// Kernel launches issued by the library in this process.
void count_launch(int n = 1);

// ---------------------------------------------------------------- scratch
// A device buffer that grows on demand (never shrinks).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Host-side helpers (api.cu).
void set_error(const std::string& msg);
vm_status cuda_status(cudaError_t e, const char* what);
vm_status ensure(DevBuf& b, size_t bytes);
#define VM_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::vmx::cuda_status(_e, #call);    \
    } while (0)
#define VM_TRY(expr)                                \
    do {                                            \
        vm_status _s = (expr);                      \
        if (_s != VM_OK) return _s;                 \
    } while (0)

// ---------------------------------------------------------------- scan.cu
// Exclusive prefix sum of n uint32 values: out[i] = sum(in[0..i-1]); *total
// (device) receives the sum.  in and out may alias.  tmp must hold
// scan_tmp_words(n) words and be zeroed once when it is allocated (it keeps
// the single-pass scan's look-back state, which every launch leaves ready
// for the next).  err (device, may be null): kErrTimeout when a bounded
// look-back wait ran out.
// Elements per tile of the single-pass scan; its look-back state is a
// ticket, a done count, an epoch, a pad word and one 64-bit word per tile.
constexpr size_t kScanTileElems = 2048;
constexpr size_t scan_tmp_words(size_t n) { return 4 + 2 * ((n + kScanTileElems - 1) / kScanTileElems) + 2; }
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint32_t* total, size_t n, uint32_t* tmp,
                               cudaStream_t s, uint32_t* err);
// Stable sort of (key, value) pairs by key, key < 2^bits (bits <= 32), LSD
// 8-bit digits.  keys/vals are sorted in place using the alt buffers; tmp
// (sort_tmp_words) zeroed once when allocated.
// Variants whose element count is read on the device from n_dev (clamped to
// the host bound n_cap, which sizes the grids): usable inside a CUDA graph.
// end: also write the sum at out[n] (n the device count clamped to n_cap; out
// then holds n_cap + 1 words), the closing offset of an offsets array.
cudaError_t exclusive_scan_dev(const uint32_t* in, uint32_t* out, uint32_t* total, const uint32_t* n_dev, size_t n_cap,
                               uint32_t* tmp, cudaStream_t s, uint32_t* err, bool end = false);
// Two arrays of the same length scanned as exclusive_scan_dev does (one
// launch when n_cap is small).
cudaError_t exclusive_scan2_dev(const uint32_t* in0, uint32_t* out0, uint32_t* total0, const uint32_t* in1,
                                uint32_t* out1, uint32_t* total1, const uint32_t* n_dev, size_t n_cap, uint32_t* tmp,
                                cudaStream_t s, uint32_t* err);
// key_bound (device, may be null): every key is below *key_bound; passes whose
// digit no key reaches are skipped on the device, and the result then lies in
// (keys, vals) after an even number of executed passes and in the alt buffers
// after an odd number (sort_result_alt tells which, on the device).  Without
// a bound the result is always in (keys, vals).
cudaError_t stable_sort_pairs_dev(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                  const uint32_t* n_dev, size_t n_cap, int bits, uint32_t* tmp, cudaStream_t s,
                                  uint32_t* err, const uint32_t* key_bound);
__device__ __forceinline__ bool sort_result_alt(uint32_t key_bound, int bits) {
    int executed = 1;
    for (int p = 1; p < (bits + 7) / 8; ++p) executed += (unsigned long long)key_bound > (1ull << (8 * p));
    return executed & 1;
}
size_t sort_tmp_words(size_t n);
// The allocated bricks of a brick table of nb entries in key order, in one
// kernel: rank_table[j] = the rank of brick key j (-1: unallocated),
// sorted_slot / sorted_key by rank; the count lands in clear[0] and the words
// clear[1 .. n_clear) and zero0 / zero1 (may be null) are cleared.  tmp: the
// look-back state of a scan of nb elements (scan_tmp_words(nb)), zeroed once.
cudaError_t order_bricks_dev(const int32_t* table, uint32_t nb, int32_t* rank_table, int32_t* sorted_slot,
                             int32_t* sorted_key, uint32_t* clear, int n_clear, uint32_t* zero0, uint32_t* zero1,
                             uint32_t* tmp, cudaStream_t s, uint32_t* err);
cudaError_t stable_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, size_t n,
                                  int bits, uint32_t* tmp, cudaStream_t s, uint32_t* err);

// ---------------------------------------------------------------- integrate.cu
// Robot-centric window (Sec. III.B): moves the window of g by shift whole
// bricks (g holds the old window; g2 the new one and its anchor; po2 its
// position origin).  Bricks that leave are evicted and their occupied voxels
// counted; the pool is compacted (kept bricks past the new count move into
// the holes), the kept sums are re-anchored (S -= C (a2 - a)), the table is
// rebuilt and po2 written to the device copy g2.po.  tmp: scratch of
// scroll_tmp_words(capacity) words, zeroed once when allocated.
size_t scroll_tmp_words(uint32_t capacity);
cudaError_t launch_scroll(const Grid& g, const Grid& g2, const int32_t shift[3], const float po2[3],
                          int32_t* brick_table, uint32_t nb_total, int32_t* slot_key, unsigned long long* S,
                          uint32_t* C, MapCounters* ctr, uint32_t capacity, uint32_t* tmp, cudaStream_t s);
// deferred: room for n point indices (the frame's points whose brick another
// thread was claiming); the map counters' deferred words are zero between calls.
cudaError_t launch_integrate(const float* xyz, uint32_t n, const Pose& pose, const Grid& g, int32_t* brick_table,
                             int32_t* slot_key, unsigned long long* S, uint32_t* C, uint32_t* deferred,
                             MapCounters* ctr, uint32_t capacity, cudaStream_t s);
// Voxel information clearing (Sec. III.B, Eq. 2): marks every occupied voxel
// that a point's ray from the sensor passes through before the point's own
// voxel (mark: one bit per voxel slot, capacity * 16 words, zero between
// calls), then clears the marked voxels and the marks.
cudaError_t launch_clear(const float* xyz, uint32_t n, const Pose& pose, const Grid& g,
                         const int32_t* brick_table, unsigned long long* S, uint32_t* C, uint32_t* mark,
                         MapCounters* ctr, uint32_t capacity, cudaStream_t s);

// ---------------------------------------------------------------- segment.cu
struct SegBuffers {
    // brick order
    uint32_t* flags;        // [nb_total + 1] scan scratch
    int32_t* rank_table;    // [nb_total]   brick key -> rank or -1
    int32_t* sorted_slot;   // [cap]        rank -> pool slot
    int32_t* sorted_key;    // [cap]        rank -> brick key
    // rank-dense voxel arrays, index = rank * 512 + local
    int32_t* M;             // [3][nv]  exact integer means (2^-20 m), INT32_MIN when empty
    float* nrm;             // [3][nv]
    uint8_t* status;        // [nv]     0 free, 1 occupied, 2 steppable
    uint8_t* nbr;           // [nv]     occupied neighbours N
    float4* rec;            // [2][nv]  packed (mu, status bits) and (normal, 0) per voxel
    uint32_t* list_idx;     // [nv]     occupied voxels (rank-dense index), in no particular order
    float* list_A;          // [6][nv]  their window covariances (FP32, rounded from exact integers)
    uint32_t* parent;       // [nv]     union-find parent, kNone when not a vertex
    uint32_t* count;        // [nv]     component sizes at roots
    uint32_t* cid;          // [nv + 1] kept-root flags -> cluster index (scan)
    uint32_t* vert_flag;    // [nv + 1] kept-vertex flags -> compact position (scan)
    // compact kept vertices
    uint32_t* keys;         // [nv] cluster index
    uint32_t* vals;         // [nv] rank-dense voxel index
    uint32_t* keys_alt;
    uint32_t* vals_alt;
    // clusters
    uint32_t* cl_size;      // [kcap + 1]
    uint32_t* cl_off;       // [kcap + 1]
    uint32_t* cl_label;     // [kcap]
    float* pts;             // [nv][3]  cluster points in cluster order
    uint32_t* pt_vid;       // [nv]
    uint32_t* scan_tmp;     // look-back state of the segmentation's scans
    uint32_t* sort_tmp;     // the radix sort's histograms and their scan state
    SegCounters* ctr;       // device
    size_t nv, kcap;
};

// Orders the allocated bricks by key (rank table, sorted slots/keys); the
// brick count lands in b.ctr->n_sorted.  Clears b.ctr first, and the device
// words zero0 / zero1 (either may be null).
cudaError_t seg_order_bricks(const int32_t* brick_table, uint32_t nb_total, SegBuffers& b, int sms, cudaStream_t s,
                             uint32_t* zero0 = nullptr, uint32_t* zero1 = nullptr);
// Means, normals, classification, clustering, cluster numbering, the cluster
// point lists in cluster order and their offsets, for the bricks ordered by
// seg_order_bricks.  Every count is read on the device (clamped to the
// scratch, with kErrScratch raised when it does not fit), so the launch
// sequence is fixed and can be captured in a CUDA graph.  kcap bounds the
// kept clusters.
cudaError_t seg_run(const Grid& g, const unsigned long long* S, const uint32_t* C, const vm_segment_params& p,
                    SegBuffers& b, uint32_t kcap, uint32_t* err, int sms, cudaStream_t s, StageHook* hk);

// ---------------------------------------------------------------- fit.cu
struct FitBuffers {
    float4* hyp;            // [kcap * H]
    uint8_t* hyp_valid;     // [kcap * H]
    uint32_t* counts;       // [kcap * H]
    FitCluster* cl;         // [kcap]
    uint32_t* item_off;     // [kcap + 1] work-item offsets (scan)
    uint32_t* item_cl;      // [items] the cluster of each work item
    uint32_t* queue;        // [4] work-queue heads
    uint8_t* inlier;        // [npts]
    float* part;            // [items][10] per-item partial sums
    float* cen;             // [kcap][3][2] inlier centroids, double-float (hi, lo)
    int2* surv;             // [npts] hull candidates (per-cluster segments at cluster offsets)
    int2* hull;             // [npts] hull vertices (per-cluster segments at cluster offsets)
    uint32_t* hull_cnt;     // [kcap + 1] -> hull offsets (scan)
    uint32_t* scan_tmp;
    uint32_t* err;          // device error word
    uint32_t* tot;          // [4] scan totals
    uint32_t* kdev;         // cluster count when the caller supplies it
    uint32_t* done;         // [kcap][3] per-cluster completion counters (scoring, extraction, filter)
    size_t kcap, npts_cap, items_cap;  // items_cap: 256-point partial-sum chunks
    int H;
};

struct FitTuning {
    int tile;               // points per work item, a multiple of 256 (the partial-sum chunk)
    int hyp_per_thread;     // hypotheses held in registers per thread
    int ctas_per_sm;        // persistent CTAs per SM
    int schedule;           // 0: a CTA per work item; 1: a warp per work item
};
FitTuning default_tuning();
// Resident scoring CTAs per SM for tuning t and H hypotheses (0 on error).
int score_max_ctas_per_sm(const FitTuning& t, int H);
size_t fit_hull_smem();

// Runs RANSAC, selection, extraction, refit and hull for the clusters whose
// points are pts[off[c]..off[c+1]) (device), labels (device, or nullptr for
// label = c).  The cluster count is read on the device from *kp (at most
// kcap, which sizes the grids), so the launch sequence is fixed and can be
// captured in a CUDA graph.  Per-cluster records land in fb.cl, hull vertices
// in fb.hull at each cluster's point offset and their offsets in fb.hull_cnt.
void fit_init_attributes();
cudaError_t fit_set_count(uint32_t* kdev, uint32_t k, cudaStream_t s);
// round: the extraction round (Philox counter word 2; 0 for the paper's
// single plane per cluster).
cudaError_t launch_fit(const float* pts, const uint32_t* off, const uint32_t* labels, const uint32_t* kp,
                       uint32_t kcap, const vm_segment_params& p, FitBuffers& fb, const FitTuning& t, int num_sms,
                       cudaStream_t s, StageHook* hk, uint32_t round = 0);

// A segmentation's result header: the segmentation counters, the hull-vertex
// and record totals (from the hull offsets' total, or, with several extraction
// rounds, from the rounds' words), the fit's and the map's error words and the
// map's brick count.
struct HeaderArgs {
    const SegCounters* ctr;
    const uint32_t* hull_off;  // [k + 1]: the total at [k]
    const uint32_t* rounds;    // null for one plane per cluster
    const uint32_t* fit_err;
    const MapCounters* mc;
    const uint32_t* seg_err;
    SegCounters* out;
};

// Packs vm_plane records and hull arrays (at most hull_cap vertices) for the
// *kp clusters; the destinations may be mapped host memory.  header (may be
// null): the kernel's first thread also writes this result header (its inputs
// all come from earlier kernels; the host reads it after the stream is done).
cudaError_t launch_pack(const FitBuffers& fb, const uint32_t* off, const uint32_t* labels, const uint32_t* kp,
                        uint32_t kcap, vm_plane* planes, int32_t* hull_xy, float* hull_xyz, uint32_t hull_cap,
                        cudaStream_t s, const HeaderArgs* header = nullptr);

// ---------------------------------------------------------------- rounds.cu
// Sequential multi-plane extraction (planes_per_cluster P > 1): round r + 1
// fits the points of round r that are not its inliers, for the clusters whose
// round r found a plane with >= min_cluster inliers and that keep >=
// min_cluster points.  Scratch for the remaining points of two rounds
// (ping-pong), the records of every round staged per cluster, and their hull
// vertices.
constexpr uint32_t kMaxRounds = 8;
struct RoundBuffers {
    float* pts[2];          // [nv][3]   remaining points, in cluster order
    uint32_t* off[2];       // [kcap + 1]
    uint32_t* lab[2];       // [kcap]    Philox labels
    uint32_t* orig[2];      // [kcap]    round-0 cluster index
    uint32_t* keep;         // [nv]      1: the point goes on to the next round
    uint32_t* kpos;         // [nv]      its position there (scan)
    uint32_t* act;          // [kcap]    1: the cluster goes on to the next round
    uint32_t* apos;         // [kcap]    its index there (scan)
    uint32_t* cnt;          // [kcap]    records per round-0 cluster
    uint32_t* cpos;         // [kcap]    first record (scan)
    uint32_t* hcnt;         // [kcap]    hull vertices per round-0 cluster
    uint32_t* hpos;         // [kcap]    first hull vertex (scan)
    uint32_t* word;         // [64] counts: k per round, staged hull bases, totals
    uint8_t* inl0;          // [nv]      round-0 inlier flags
    vm_plane* slot;         // [kcap][kMaxRounds] staged records
    int2* hull;             // [hcap]    staged hull vertices
    size_t nv, kcap, hcap;
};
// Word indices in RoundBuffers::word.
constexpr int kWordK = 0;                        // [kMaxRounds] clusters in round r (r >= 1)
constexpr int kWordHull = 8;                     // [kMaxRounds + 1] staged hull base of round r
constexpr int kWordNpts = 20, kWordKeep = 21;    // round points, kept points
constexpr int kWordRec = 22, kWordHullTot = 23;  // output records, output hull vertices

__device__ __forceinline__ void write_header(const HeaderArgs& a) {
    SegCounters h = *a.ctr;
    h.n_hull = a.rounds ? a.rounds[kWordHullTot] : a.hull_off[h.k];
    h.n_planes = a.rounds ? a.rounds[kWordRec] : h.k;
    h.fit_err = *a.fit_err;
    h.n_bricks = a.mc->n_bricks;
    h.map_err = a.mc->err;
    h.err |= *a.seg_err;
    *a.out = h;
}
size_t rounds_bytes(size_t nv, size_t kcap, size_t hcap);
void rounds_layout(char* base, RoundBuffers& rb, size_t nv, size_t kcap, size_t hcap);
// Runs every round on the clusters of b (count b.ctr->k) and writes the
// records in (cluster, round) order to planes (at most rec_cap) with their
// hull vertices (at most hull_cap); the totals land in rb.word[kWordRec] and
// rb.word[kWordHullTot].  scan_tmp: look-back state for scans of up to
// rb.nv + 1 elements.
cudaError_t launch_rounds(const SegBuffers& b, uint32_t kcap, const vm_segment_params& p, FitBuffers& fb,
                          RoundBuffers& rb, const FitTuning& t, int sms, uint32_t* scan_tmp, vm_plane* planes,
                          uint32_t rec_cap, int32_t* hull_xy, float* hull_xyz, uint32_t hull_cap, cudaStream_t s,
                          StageHook* hk);

}  // namespace vmx
