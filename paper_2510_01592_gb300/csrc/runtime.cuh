// runtime.cuh -- host-side internals shared by the C ABI translation units
// (api.cu: maps; fitplan.cu: reusable batched fits and the autotuner;
// serve.cu: the multi-stream server): scratch carving, stage timer, the map
// object and the pieces of one segmentation call.
#pragma once
#include <vector>

#include "vm_internal.cuh"

namespace vmx {

// CUDA-event stage timer: begin/end record events on the stream; elapsed times
// are folded in once the events have completed (at the next sync point).
struct Timer : StageHook {
    bool on = false;
    struct Rec {
        int st;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    cudaEvent_t open[kNumStages] = {};
    double ms[kNumStages] = {};
    unsigned long long calls[kNumStages] = {};
    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(int st, cudaStream_t s) override {
        if (!on) return;
        cudaEvent_t e = get();
        if (e) cudaEventRecord(e, s);
        open[st] = e;
    }
    void end(int st, cudaStream_t s) override {
        if (!on || !open[st]) return;
        cudaEvent_t e = get();
        if (!e) return;
        cudaEventRecord(e, s);
        recs.push_back({st, open[st], e});
        open[st] = nullptr;
    }
    void fold() {
        for (auto& r : recs) {
            float t = 0.0f;
            cudaEventSynchronize(r.b);
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                ms[r.st] += t;
                calls[r.st] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
    void release() {
        fold();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
    }
    StageHook* hook() { return on ? this : nullptr; }
};

// Carves aligned sub-buffers out of one allocation.
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += n * sizeof(T);
        return p;
    }
};

// Fit scratch owned by a map or by a calling thread.
struct FitContext {
    Timer timer;
    uint64_t gen = 0;      // bumps whenever the scratch moves
    DevBuf mem;
    FitBuffers fb{};
    size_t kcap = 0, npts = 0, items = 0;
    int H = 0;
    DevBuf out;          // device staging of planes / hull arrays
    void* host = nullptr;  // pinned host staging
    size_t host_bytes = 0;
};

void release(DevBuf& b);
size_t fit_bytes(size_t kcap, size_t npts, size_t chunks, int H);
// Sizes fit scratch (zeroing its scan state on s when it is re-allocated).
vm_status fit_prepare(FitContext& fc, size_t kcap, size_t npts, int H, int tile, cudaStream_t s);
void fit_release(FitContext& fc);
int device_sms();
vm_status check_params(const vm_segment_params* p);
// check_params, and one plane per cluster (the batched fits and vm_fit_planes
// run a single extraction round).
vm_status check_single_round(const vm_segment_params* p);
// Launch bookkeeping around graph capture: launches recorded while capturing
// are taken back and counted again at each replay.
unsigned long long launch_total();
void uncount_launch(unsigned long long n);
// Graph captures and device / pinned allocations made by the library in this
// process (diagnostics of the serving path).
void count_capture();
unsigned long long capture_total();
void count_alloc();
unsigned long long alloc_total();

// Result block in mapped pinned host memory: the counters, then kcap plane
// records, then hcap hull vertices (xy int32 pairs, then xyz floats).
size_t out_planes_off();
size_t out_xy_off(uint32_t kcap);
size_t out_xyz_off(uint32_t kcap, uint32_t hcap);

}  // namespace vmx

struct vm_map {
    vm_map_params prm{};
    vmx::Grid g{};
    uint32_t nb_total = 0;
    uint32_t capacity = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // pool
    int32_t* brick_table = nullptr;
    int32_t* slot_key = nullptr;
    unsigned long long* S = nullptr;
    uint32_t* C = nullptr;
    vmx::MapCounters* ctr = nullptr;
    uint32_t* err = nullptr;  // segmentation error word
    uint32_t* mark = nullptr; // ray-cast clearing marks, one bit per voxel slot
    uint32_t* scroll_tmp = nullptr;  // window-scroll scratch (flags, positions, holes, scan state)
    float* po_dev = nullptr;         // position origin of the window, read by the segmentation
    vmx::DevBuf pool;
    vmx::DevBuf stage;             // host points staged on the device
    vmx::DevBuf deferred;          // point indices deferred by the integration pass
    // segmentation
    vmx::DevBuf brick_mem;         // brick-level arrays (fixed size)
    vmx::DevBuf vox_mem;           // rank-dense voxel arrays (grow with the brick count)
    vmx::SegBuffers seg{};
    size_t seg_nv = 0;
    vmx::SegCounters* hctr = nullptr;  // pinned
    vmx::SegCounters last{};
    vmx::FitContext fit;
    vmx::FitTuning tune = vmx::default_tuning();
    bool segmented = false;
    // further extraction rounds (planes_per_cluster > 1)
    vmx::DevBuf round_mem;
    vmx::RoundBuffers rounds{};
    uint32_t seg_rounds = 1;      // rounds of the last segmentation launched
    uint32_t rec_hint = 0;        // output records of the last segmentation
    // results: mapped pinned host memory written by the kernels
    void* out_host = nullptr;
    char* out_dev = nullptr;
    size_t out_bytes = 0;
    uint32_t out_kcap = 0, out_hcap = 0;
    uint32_t kcap = 0;            // kept-cluster capacity of the scratch
    uint32_t brick_hint = 0, k_hint = 0, hull_hint = 0;
    uint64_t gen = 0;             // bumps whenever scratch or outputs move
    // captured segmentation (one CUDA graph, replayed per call)
    bool use_graph = true;
    cudaGraphExec_t gexec = nullptr;
    uint64_t ggen = ~0ull;
    vm_segment_params gprm{};
    unsigned long long glaunches = 0;
    uint32_t gnodes = 0, gedges = 0, gprog = 0;  // the captured graph's nodes, edges and programmatic edges
    // captured front half (brick order .. cluster points), for batched serving
    cudaGraphExec_t fexec = nullptr;
    uint64_t fgen = ~0ull;
    vm_segment_params fprm{};
    unsigned long long flaunches = 0;
};

namespace vmx {

vm_status check_map(vm_map* m);
vm_status alloc_vox(vm_map* m, uint32_t n_bricks);
vm_status ensure_out(vm_map* m, uint32_t kcap, uint32_t hcap);
// Sizes the map's scratch and result block for a segmentation with p (and
// its own fit scratch when with_fit).
vm_status plan_capacity(vm_map* m, const vm_segment_params& p, bool with_fit);
// Device bytes a map with these parameters can come to hold at its brick
// capacity: pool, segmentation scratch, result block and input staging (its
// own fit scratch, used only when a batched fit falls back, is not counted).
uint64_t map_footprint(const vm_map_params& p, const vm_segment_params& sp);
// Launches only the front half of a segmentation (graph replay when enabled):
// the map's cluster points, offsets, labels and counters are ready once the
// map's stream reaches this point.
vm_status launch_front(vm_map* m, const vm_segment_params& p);
// Updates the sizing hints from the map's result block; true when the last
// segmentation ran out of a capacity and must be re-run.
bool take_hints(vm_map* m);
// Front half of a segmentation (brick order .. cluster points), fit, pack +
// header into the map's result block; the whole call.
cudaError_t enqueue_front(vm_map* m, const vm_segment_params& p, StageHook* hk, uint32_t* also_zero = nullptr);
cudaError_t enqueue_segment(vm_map* m, const vm_segment_params& p, StageHook* hk);
// Launches the map's segmentation on its stream (graph replay when enabled)
// without waiting; finish_segment waits, re-runs with grown scratch when a
// capacity ran out, and copies the result out.
vm_status launch_segment(vm_map* m, const vm_segment_params& p);
vm_status finish_segment(vm_map* m, const vm_segment_params& p, vm_planes* out);
// Copies the result block of a completed segmentation into out and maps its
// status words to a vm_status.
vm_status read_result(vm_map* m, vm_planes* out);

}  // namespace vmx
