// fitplan.cu -- reusable batched plane fits (vm_fit_plan_*): the
// cluster-parallel fit of Sec. III.C (multi-plane estimation stages a-c,
// refit, boundary polygons) over caller-formed clusters, sized once and
// replayed as one CUDA graph, plus the autotuner that picks the scoring
// schedule (work-item tile, hypotheses per thread, persistent CTAs per SM,
// CTA or warp per item) for a batch by timing the whole fit.
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "runtime.cuh"

using namespace vmx;

namespace vmx {

// Result block header of a plan (the first 256 bytes of its mapped block).
struct FitHeader {
    uint32_t k;          // clusters fitted (0 when the batch did not fit the scratch)
    uint32_t n_points;   // off[k] as read on the device
    uint32_t n_hull;     // hull vertices written (may exceed the block's capacity)
    uint32_t err;        // kErr* bits
};

// Starts the fit's error word and rejects a batch whose point count exceeds
// the scratch: every later kernel then sees zero clusters, and the host grows
// the scratch and runs again.
__global__ void k_fit_guard(const uint32_t* __restrict__ off, uint32_t* __restrict__ kdev, uint32_t ncap,
                            uint32_t* __restrict__ err, uint32_t* __restrict__ n_out) {
    pdl_gate();
    const uint32_t k = *kdev;
    const uint32_t n = off[k];
    *n_out = n;
    *err = n > ncap ? kErrScratch : 0u;
    if (n > ncap) *kdev = 0;
}

__global__ void k_fit_header(const uint32_t* __restrict__ kdev, const uint32_t* __restrict__ n_pts,
                             const uint32_t* __restrict__ hull_off, const uint32_t* __restrict__ err,
                             FitHeader* __restrict__ out) {
    pdl_gate();
    FitHeader h;
    h.k = *kdev;
    h.n_points = *n_pts;
    h.n_hull = hull_off[h.k];
    h.err = *err;
    *out = h;
}

}  // namespace vmx

struct vm_fit_plan {
    cudaStream_t s = nullptr;
    bool own_stream = false;
    vm_segment_params prm{};
    uint32_t flags = 0;
    vmx::FitContext fc;
    vmx::FitTuning tune = vmx::default_tuning();
    // mapped result block
    void* out_host = nullptr;
    char* out_dev = nullptr;
    uint32_t out_kcap = 0, out_hcap = 0;
    uint32_t* k_host = nullptr;  // pinned: the cluster count the graph copies to the device
    uint64_t gen = 0;            // bumps when scratch, result block or tuning change
    // captured fit
    cudaGraphExec_t gexec = nullptr;
    uint64_t ggen = ~0ull;
    const float* gx = nullptr;
    const uint32_t* goff = nullptr;
    const uint32_t* glab = nullptr;
    unsigned long long glaunches = 0;
    // the launch in flight
    bool pending = false;
    const float* px = nullptr;
    const uint32_t* poff = nullptr;
    const uint32_t* plab = nullptr;
    uint32_t pk = 0;
};

namespace vmx {
namespace {

vm_status plan_out(vm_fit_plan* f, uint32_t kcap, uint32_t hcap) {
    if (f->out_host && kcap <= f->out_kcap && hcap <= f->out_hcap) return VM_OK;
    if (f->out_host) {
        cudaStreamSynchronize(f->s);
        cudaFreeHost(f->out_host);
    }
    f->out_host = nullptr;
    f->out_dev = nullptr;
    const size_t bytes = out_xyz_off(kcap, hcap) + (size_t)hcap * 12 + 256;
    count_alloc();
    cudaError_t e = cudaHostAlloc(&f->out_host, bytes, cudaHostAllocMapped);
    if (e != cudaSuccess) {
        f->out_host = nullptr;
        return cuda_status(e, "cudaHostAlloc(mapped)");
    }
    void* d = nullptr;
    VM_CUDA(cudaHostGetDevicePointer(&d, f->out_host, 0));
    memset(f->out_host, 0, 256);
    f->out_dev = static_cast<char*>(d);
    f->out_kcap = kcap;
    f->out_hcap = hcap;
    f->gen++;
    return VM_OK;
}

// Sizes scratch and result block for k clusters and n points (headroom on
// growth); never shrinks.
vm_status plan_size(vm_fit_plan* f, uint32_t k, uint32_t n, uint32_t hull) {
    const uint64_t g0 = f->fc.gen;
    const size_t kk = k > f->fc.kcap ? k : f->fc.kcap;
    const size_t nn = n > f->fc.npts ? n : f->fc.npts;
    VM_TRY(fit_prepare(f->fc, kk ? kk : 1, nn ? nn : 1, (int)f->prm.n_hyp, f->tune.tile, f->s));
    if (f->fc.gen != g0) f->gen++;
    uint32_t hcap = hull + hull / 2 + 4096;
    const uint32_t floor_h = (uint32_t)(f->fc.kcap * 64 < 65536 ? 65536 : f->fc.kcap * 64);
    if (hcap < floor_h) hcap = floor_h;
    if (hcap < f->out_hcap) hcap = f->out_hcap;
    return plan_out(f, (uint32_t)f->fc.kcap, hcap);
}

cudaError_t enqueue_fit(vm_fit_plan* f, const float* x, const uint32_t* off, const uint32_t* lab, StageHook* hk) {
    cudaStream_t s = f->s;
    FitBuffers& fb = f->fc.fb;
    const uint32_t kcap = (uint32_t)f->fc.kcap;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(fb.kdev, f->k_host, sizeof(uint32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    launch_k(k_fit_guard, dim3(1), dim3(1), 0, s, off, fb.kdev, (uint32_t)f->fc.npts, fb.err, fb.tot + 2);
    if ((e = launch_fit(x, off, lab, fb.kdev, kcap, f->prm, fb, f->tune, device_sms(), s, hk)) != cudaSuccess)
        return e;
    char* d = f->out_dev;
    VM_STAGE_BEGIN(hk, kStPack, s);
    e = launch_pack(fb, off, lab, fb.kdev, kcap, reinterpret_cast<vm_plane*>(d + out_planes_off()),
                    reinterpret_cast<int32_t*>(d + out_xy_off(f->out_kcap)),
                    reinterpret_cast<float*>(d + out_xyz_off(f->out_kcap, f->out_hcap)), f->out_hcap, s);
    if (e != cudaSuccess) return e;
    launch_k(k_fit_header, dim3(1), dim3(1), 0, s, fb.kdev, fb.tot + 2, fb.hull_cnt, fb.err,
             reinterpret_cast<FitHeader*>(d));
    VM_STAGE_END(hk, kStPack, s);
    count_launch(2);
    return cudaGetLastError();
}

vm_status capture_fit(vm_fit_plan* f, const float* x, const uint32_t* off, const uint32_t* lab) {
    if (f->gexec) {
        cudaGraphExecDestroy(f->gexec);
        f->gexec = nullptr;
    }
    fit_init_attributes();
    cudaGraph_t graph = nullptr;
    const unsigned long long l0 = launch_total();
    count_capture();
    VM_CUDA(cudaStreamBeginCapture(f->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_fit(f, x, off, lab, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(f->s, &graph);
    const unsigned long long n = launch_total() - l0;
    uncount_launch(n);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_status(e, "fit capture");
    }
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&f->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        f->gexec = nullptr;
        return cuda_status(e, "cudaGraphInstantiate");
    }
    f->glaunches = n;
    f->ggen = f->gen;
    f->gx = x;
    f->goff = off;
    f->glab = lab;
    return VM_OK;
}

vm_status plan_enqueue(vm_fit_plan* f, const float* x, const uint32_t* off, const uint32_t* lab, uint32_t k) {
    *f->k_host = k;
    StageHook* hk = f->fc.timer.hook();
    const bool graph = !(f->flags & VM_FIT_EAGER) && !hk;
    if (graph) {
        if (!f->gexec || f->ggen != f->gen || f->gx != x || f->goff != off || f->glab != lab)
            VM_TRY(capture_fit(f, x, off, lab));
        VM_CUDA(cudaGraphLaunch(f->gexec, f->s));
        count_launch((int)f->glaunches);
    } else {
        VM_CUDA(enqueue_fit(f, x, off, lab, hk));
    }
    return VM_OK;
}

vm_status plan_launch(vm_fit_plan* f, const float* x, const uint32_t* off, const uint32_t* lab, uint32_t k) {
    if (f->pending) {
        set_error("a launch is already in flight on this plan; wait for it first");
        return VM_ERR_INVALID_ARG;
    }
    if (k && (!x || !off)) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    if (k > f->fc.kcap) {  // more clusters than ever: learn the point count once
        uint32_t n = 0;
        VM_CUDA(cudaMemcpyAsync(&n, off + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, f->s));
        VM_CUDA(cudaStreamSynchronize(f->s));
        VM_TRY(plan_size(f, k, n, 0));
    }
    VM_TRY(plan_enqueue(f, x, off, lab, k));
    f->pending = true;
    f->px = x;
    f->poff = off;
    f->plab = lab;
    f->pk = k;
    return VM_OK;
}

vm_status plan_wait(vm_fit_plan* f, vm_planes* out) {
    if (out) memset(out, 0, sizeof(*out));
    if (!f->pending) {
        set_error("no launch in flight on this plan");
        return VM_ERR_INVALID_ARG;
    }
    f->pending = false;
    const FitHeader* h = nullptr;
    for (int attempt = 0;; ++attempt) {
        VM_CUDA(cudaStreamSynchronize(f->s));
        f->fc.timer.fold();
        h = static_cast<const FitHeader*>(f->out_host);
        const bool scratch = (h->err & kErrScratch) != 0;
        const bool hull = h->n_hull > f->out_hcap;
        if (!scratch && !hull) break;
        if (attempt == 3) {
            set_error("fit scratch could not be sized for this batch");
            return VM_ERR_OUT_OF_MEMORY;
        }
        VM_TRY(plan_size(f, f->pk, scratch ? h->n_points : 0, hull ? h->n_hull : 0));
        VM_TRY(plan_enqueue(f, f->px, f->poff, f->plab, f->pk));
    }
    if (out) {
        const uint32_t K = h->k, n_hull = h->n_hull;
        const size_t b_planes = (size_t)K * sizeof(vm_plane);
        out->planes = static_cast<vm_plane*>(malloc(b_planes ? b_planes : 1));
        out->hull_xy = static_cast<int32_t*>(malloc(n_hull ? (size_t)n_hull * 8 : 1));
        out->hull_xyz = static_cast<float*>(malloc(n_hull ? (size_t)n_hull * 12 : 1));
        if (!out->planes || !out->hull_xy || !out->hull_xyz) {
            vm_planes_free(out);
            set_error("host allocation of the result failed");
            return VM_ERR_OUT_OF_MEMORY;
        }
        const char* hb = static_cast<const char*>(f->out_host);
        memcpy(out->planes, hb + out_planes_off(), b_planes);
        memcpy(out->hull_xy, hb + out_xy_off(f->out_kcap), (size_t)n_hull * 8);
        memcpy(out->hull_xyz, hb + out_xyz_off(f->out_kcap, f->out_hcap), (size_t)n_hull * 12);
        out->n_planes = K;
        out->n_hull = n_hull;
    }
    if (h->err & kErrTimeout) {
        set_error("a bounded device loop reached its iteration cap during the plane fit");
        return VM_ERR_TIMEOUT;
    }
    if (h->err & kErrOverflow) {
        set_error("a cluster spans more than 2^28 hull quanta (4096 m) in its plane; its hull is not exact");
        return VM_ERR_EXTENT;
    }
    return VM_OK;
}

vm_status check_tuning(const vm_fit_tuning* t) {
    if (!t) {
        set_error("null tuning");
        return VM_ERR_INVALID_ARG;
    }
    const bool r_ok = t->hyp_per_thread == 1 || t->hyp_per_thread == 2 || t->hyp_per_thread == 4 ||
                      t->hyp_per_thread == 8;
    if (t->tile < 256 || t->tile > 16384 || t->tile % 256 || !r_ok || t->ctas_per_sm < 1 || t->ctas_per_sm > 16 ||
        t->schedule > 1) {
        set_error("tuning out of range (tile a multiple of 256 in 256..16384, hyp_per_thread 1/2/4/8, "
                  "ctas_per_sm 1..16, schedule 0/1)");
        return VM_ERR_INVALID_ARG;
    }
    return VM_OK;
}

vm_status apply_tuning(vm_fit_plan* f, const FitTuning& t) {
    f->tune = t;
    f->gen++;
    return plan_size(f, 0, 0, 0);  // the item count depends on the tile
}

}  // namespace
}  // namespace vmx

extern "C" {

vm_status vm_fit_plan_create(uint32_t k_cap, uint32_t n_cap, const vm_segment_params* params, void* stream,
                             uint32_t flags, vm_fit_plan** out) {
    VM_TRY(check_single_round(params));
    if (!out) {
        set_error("null output");
        return VM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    vm_fit_plan* f = new (std::nothrow) vm_fit_plan();
    if (!f) {
        set_error("host allocation failed");
        return VM_ERR_OUT_OF_MEMORY;
    }
    f->prm = *params;
    f->flags = flags;
    f->fc.timer.on = (flags & VM_FIT_STAGE_TIMING) != 0;
    cudaError_t e;
    if (stream) {
        f->s = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&f->s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete f;
            return cuda_status(e, "cudaStreamCreate");
        }
        f->own_stream = true;
    }
    void* kh = nullptr;
    e = cudaMallocHost(&kh, sizeof(uint32_t));
    if (e != cudaSuccess) {
        vm_fit_plan_destroy(f);
        return cuda_status(e, "cudaMallocHost");
    }
    f->k_host = static_cast<uint32_t*>(kh);
    const vm_status st = plan_size(f, k_cap, n_cap, 0);
    if (st != VM_OK) {
        vm_fit_plan_destroy(f);
        return st;
    }
    *out = f;
    return VM_OK;
}

vm_status vm_fit_plan_destroy(vm_fit_plan* f) {
    if (!f) return VM_OK;
    if (f->s) cudaStreamSynchronize(f->s);
    if (f->gexec) cudaGraphExecDestroy(f->gexec);
    fit_release(f->fc);
    if (f->out_host) cudaFreeHost(f->out_host);
    if (f->k_host) cudaFreeHost(f->k_host);
    if (f->own_stream && f->s) cudaStreamDestroy(f->s);
    delete f;
    return VM_OK;
}

vm_status vm_fit_plan_stage_times(vm_fit_plan* f, double* ms, uint64_t* calls, uint32_t cap, uint32_t* n_stages) {
    if (!f) {
        set_error("null plan");
        return VM_ERR_INVALID_ARG;
    }
    VM_CUDA(cudaStreamSynchronize(f->s));
    f->fc.timer.fold();
    for (uint32_t i = 0; i < (uint32_t)kNumStages && i < cap; ++i) {
        if (ms) ms[i] = f->fc.timer.ms[i];
        if (calls) calls[i] = f->fc.timer.calls[i];
        f->fc.timer.ms[i] = 0.0;
        f->fc.timer.calls[i] = 0;
    }
    if (n_stages) *n_stages = kNumStages;
    return VM_OK;
}

vm_status vm_fit_plan_launch(vm_fit_plan* f, const float* xyz, const uint32_t* off, const uint32_t* labels,
                             uint32_t k) {
    if (!f) {
        set_error("null plan");
        return VM_ERR_INVALID_ARG;
    }
    return plan_launch(f, xyz, off, labels, k);
}

vm_status vm_fit_plan_wait(vm_fit_plan* f, vm_planes* out) {
    if (!f) {
        set_error("null plan");
        return VM_ERR_INVALID_ARG;
    }
    return plan_wait(f, out);
}

vm_status vm_fit_plan_run(vm_fit_plan* f, const float* xyz, const uint32_t* off, const uint32_t* labels, uint32_t k,
                          vm_planes* out) {
    if (!f || !out) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    memset(out, 0, sizeof(*out));
    VM_TRY(plan_launch(f, xyz, off, labels, k));
    return plan_wait(f, out);
}

vm_status vm_fit_plan_set_tuning(vm_fit_plan* f, const vm_fit_tuning* t) {
    if (!f) {
        set_error("null plan");
        return VM_ERR_INVALID_ARG;
    }
    VM_TRY(check_tuning(t));
    if (f->pending) {
        set_error("a launch is in flight on this plan");
        return VM_ERR_INVALID_ARG;
    }
    return apply_tuning(f, FitTuning{(int)t->tile, (int)t->hyp_per_thread, (int)t->ctas_per_sm, (int)t->schedule});
}

vm_status vm_fit_plan_get_tuning(const vm_fit_plan* f, vm_fit_tuning* t) {
    if (!f || !t) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    t->tile = (uint32_t)f->tune.tile;
    t->hyp_per_thread = (uint32_t)f->tune.hyp_per_thread;
    t->ctas_per_sm = (uint32_t)f->tune.ctas_per_sm;
    t->schedule = (uint32_t)f->tune.schedule;
    return VM_OK;
}

vm_status vm_fit_plan_autotune(vm_fit_plan* f, const float* xyz, const uint32_t* off, const uint32_t* labels,
                               uint32_t k, uint32_t reps, vm_fit_tuning* best, float* best_ms, uint32_t* n_tried) {
    if (!f) {
        set_error("null plan");
        return VM_ERR_INVALID_ARG;
    }
    if (f->pending) {
        set_error("a launch is in flight on this plan");
        return VM_ERR_INVALID_ARG;
    }
    if (reps < 1) reps = 1;
    const int H = (int)f->prm.n_hyp;
    std::vector<FitTuning> cand;
    const int tiles_cta[] = {1024, 2048, 4096, 8192};
    const int tiles_warp[] = {256, 512, 768, 1024};
    const int rs[] = {2, 4, 8};
    const int ctas[] = {1, 2, 3, 4, 6, 8};
    for (int sched = 0; sched < 2; ++sched) {
        for (int ti = 0; ti < 4; ++ti) {
            for (int r : rs) {
                if (sched == 1 && (H + r - 1) / r > 32) continue;  // a warp holds every hypothesis
                if (sched == 0 && (H + r - 1) / r > 256) continue;
                const FitTuning base{sched ? tiles_warp[ti] : tiles_cta[ti], r, 1, sched};
                const int occ = score_max_ctas_per_sm(base, H);
                for (int c : ctas) {
                    if (c > occ) break;
                    FitTuning t = base;
                    t.ctas_per_sm = c;
                    cand.push_back(t);
                }
            }
        }
    }
    const FitTuning keep = f->tune;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    VM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_status(cudaErrorUnknown, "cudaEventCreate");
    }
    float best_t = -1.0f;
    FitTuning best_c = keep;
    uint32_t tried = 0;
    vm_status st = VM_OK;
    // Size for the smallest tile first so that no candidate re-allocates.
    f->tune.tile = tiles_warp[0];
    st = plan_size(f, 0, 0, 0);
    for (size_t i = 0; st == VM_OK && i < cand.size(); ++i) {
        st = apply_tuning(f, cand[i]);
        if (st != VM_OK) break;
        st = plan_launch(f, xyz, off, labels, k);  // warm-up; also sizes for this batch
        if (st == VM_OK) st = plan_wait(f, nullptr);
        if (st != VM_OK) break;
        cudaEventRecord(e0, f->s);
        for (uint32_t r = 0; r < reps && st == VM_OK; ++r) st = plan_enqueue(f, xyz, off, labels, k);
        cudaEventRecord(e1, f->s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_status(cudaGetLastError(), "autotune timing");
        if (st != VM_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        ++tried;
        if (best_t < 0.0f || ms < best_t) {
            best_t = ms;
            best_c = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    vm_status st2 = apply_tuning(f, st == VM_OK ? best_c : keep);
    if (st != VM_OK) return st;
    if (st2 != VM_OK) return st2;
    if (best) {
        best->tile = (uint32_t)best_c.tile;
        best->hyp_per_thread = (uint32_t)best_c.hyp_per_thread;
        best->ctas_per_sm = (uint32_t)best_c.ctas_per_sm;
        best->schedule = (uint32_t)best_c.schedule;
    }
    if (best_ms) *best_ms = best_t;
    if (n_tried) *n_tried = tried;
    return VM_OK;
}

}  // extern "C"
