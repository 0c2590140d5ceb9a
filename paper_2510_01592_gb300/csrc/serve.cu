// serve.cu -- the multi-stream server (vm_server_*): one device-resident map
// per sensor stream, admission by device memory, and a scheduler thread that
// forms steps from whatever requests are waiting whenever a GPU slot is free
// (continuous batching).  In batched mode a step runs each member's integrate
// (Sec. III.B) and the front half of its segmentation (Sec. III.C up to the
// cluster points) on the member's map stream, then ONE fit over the clusters
// of all members -- RANSAC (stages a-c), refit and hull -- on the server's
// stream, and packs each member's planes into its map's result block.
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "runtime.cuh"

using namespace vmx;

namespace vmx {
namespace {

constexpr int kMaxBatch = 64;
constexpr int kMaxSlots = 4;
constexpr int kGatherT = 256;

// One member of a batched fit: where its clusters are and where its planes go.
struct BatchEntry {
    const float* pts;            // cluster points, float[n][3] in cluster order
    const uint32_t* cl_off;      // [k + 1]
    const uint32_t* cl_label;    // [k]
    const SegCounters* ctr;      // k, tot (points), err of the member's front half
    const MapCounters* mc;
    const uint32_t* seg_err;
    vm_plane* planes;            // the member's result block (mapped host memory)
    int32_t* hull_xy;
    float* hull_xyz;
    SegCounters* header;
    uint32_t hull_cap;
    uint32_t base_k, base_n, k;  // written by k_batch_prefix
};

struct BatchTable {
    uint32_t n_maps;
    uint32_t K, N;               // clusters and points in the batch (0 when it overflowed)
    uint32_t K_need, N_need;
    uint32_t err;
    uint32_t pad[2];
    BatchEntry e[kMaxBatch];
};

struct BatchStatus {
    uint32_t K_need, N_need, err, fit_err;
};

// Batch offsets of every member; a member whose front half ran out of scratch
// contributes nothing (the host re-runs it alone).  A batch larger than the
// arena contributes nothing either and is re-run after the arena grows.
__global__ void k_batch_prefix(BatchTable* __restrict__ t, uint32_t kcap, uint32_t ncap, uint32_t* __restrict__ kdev,
                               uint32_t* __restrict__ fit_err) {
    pdl_gate();
    *fit_err = 0;  // the batch fit's error word starts clear
    uint32_t K = 0, N = 0;
    for (uint32_t m = 0; m < t->n_maps; ++m) {
        BatchEntry& e = t->e[m];
        const bool ok = !((*e.seg_err | e.ctr->err) & kErrScratch);
        const uint32_t k = ok ? e.ctr->k : 0u, n = ok ? e.ctr->tot : 0u;
        e.base_k = K;
        e.base_n = N;
        e.k = k;
        K += k;
        N += n;
    }
    t->K_need = K;
    t->N_need = N;
    t->err = 0;
    if (K > kcap || N > ncap) {
        t->err = kErrScratch;
        K = N = 0;
    }
    t->K = K;
    t->N = N;
    *kdev = K;
}

// Largest member m with base[m] <= i (members with nothing have equal bases
// and are skipped by taking the last one).
__device__ __forceinline__ uint32_t member_of(const uint32_t* base, uint32_t nm, uint32_t i) {
    uint32_t lo = 0, hi = nm - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (base[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Concatenates the members' cluster points, offsets and labels into the arena.
__global__ void __launch_bounds__(kGatherT) k_batch_gather(const BatchTable* __restrict__ t, float* __restrict__ apts,
                                                           uint32_t* __restrict__ aoff, uint32_t* __restrict__ alab) {
    pdl_gate();
    __shared__ uint32_t sbn[kMaxBatch], sbk[kMaxBatch];
    const uint32_t nm = t->n_maps, N = t->N, K = t->K;
    for (uint32_t m = threadIdx.x; m < nm; m += blockDim.x) {
        sbn[m] = t->e[m].base_n;
        sbk[m] = t->e[m].base_k;
    }
    __syncthreads();
    if (nm == 0) return;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const uint32_t m = member_of(sbn, nm, (uint32_t)i);
        const float* src = t->e[m].pts + 3 * (i - sbn[m]);
        apts[3 * i] = src[0];
        apts[3 * i + 1] = src[1];
        apts[3 * i + 2] = src[2];
    }
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < K; j += stride) {
        const uint32_t m = member_of(sbk, nm, (uint32_t)j);
        const uint32_t c = (uint32_t)j - sbk[m];
        aoff[j] = sbn[m] + t->e[m].cl_off[c];
        alab[j] = t->e[m].cl_label[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) aoff[K] = N;
}

// Each cluster's record and hull into its member's result block, with hull
// offsets relative to the member's first cluster.
__global__ void k_pack_batch(const BatchTable* __restrict__ t, const uint32_t* __restrict__ kdev,
                             const uint32_t* __restrict__ aoff, const uint32_t* __restrict__ alab,
                             const FitCluster* __restrict__ cl, const int2* __restrict__ hull,
                             const uint32_t* __restrict__ hull_off) {
    pdl_gate();
    __shared__ uint32_t sbk[kMaxBatch];
    const uint32_t nm = t->n_maps, K = *kdev;
    for (uint32_t m = threadIdx.x; m < nm; m += blockDim.x) sbk[m] = t->e[m].base_k;
    __syncthreads();
    if (nm == 0) return;
    for (uint32_t j = blockIdx.x; j < K; j += gridDim.x) {
        const uint32_t m = member_of(sbk, nm, j);
        const BatchEntry& E = t->e[m];
        const uint32_t hb = hull_off[E.base_k], ho = hull_off[j];
        pack_cluster(cl[j], alab[j], aoff[j + 1] - aoff[j], hull + aoff[j], ho - hb, hull_off[j + 1] - ho,
                     E.planes + (j - E.base_k), E.hull_xy, E.hull_xyz, E.hull_cap);
    }
}

// Each member's result header (the same record a single-map segmentation
// writes) and the batch status for the host.
__global__ void k_batch_header(const BatchTable* __restrict__ t, const uint32_t* __restrict__ hull_off,
                               const uint32_t* __restrict__ fit_err, BatchStatus* __restrict__ st) {
    pdl_gate();
    const uint32_t m = threadIdx.x;
    if (m < t->n_maps) {
        const BatchEntry& E = t->e[m];
        SegCounters h = *E.ctr;
        h.n_hull = t->err ? 0u : hull_off[E.base_k + E.k] - hull_off[E.base_k];
        h.n_planes = t->err ? 0u : h.k;
        h.fit_err = *fit_err;
        h.n_bricks = E.mc->n_bricks;
        h.map_err = E.mc->err;
        h.err |= *E.seg_err;
        *E.header = h;
    }
    if (m == 0) {
        BatchStatus s;
        s.K_need = t->K_need;
        s.N_need = t->N_need;
        s.err = t->err;
        s.fit_err = *fit_err;
        *st = s;
    }
}

// The batched fit of one server: the arena the members' clusters are gathered
// into, the fit scratch, and one captured graph per in-flight slot (each
// reads its slot's pinned copy of the batch table).
struct BatchFit {
    FitContext fc;
    FitTuning tune{};
    DevBuf arena;
    float* apts = nullptr;
    uint32_t* aoff = nullptr;
    uint32_t* alab = nullptr;
    uint32_t kcap = 0, ncap = 0;
    BatchTable* dtab = nullptr;
    BatchTable* htab[kMaxSlots] = {};
    BatchStatus* hstat[kMaxSlots] = {};
    BatchStatus* dstat[kMaxSlots] = {};
    cudaGraphExec_t gexec[kMaxSlots] = {};
    uint64_t ggen[kMaxSlots] = {};
    unsigned long long glaunches[kMaxSlots] = {};
    uint64_t gen = 1;
};

}  // namespace
}  // namespace vmx

struct vm_server {
    struct Req {
        uint64_t ticket;
        uint32_t stream;
        const float* xyz;
        uint32_t n;
        float pose[12];
        int on_dev;
        double t_arr;
    };
    struct Strm {
        vm_map_params mp{};
        uint64_t footprint = 0;
        int state = 0;  // 0 waiting, 1 admitted
        bool close_req = false;
        vm_map* map = nullptr;
        std::deque<Req> q;
        bool busy = false;
        cudaEvent_t ev = nullptr;
    };
    struct Step {
        int slot = -1;  // batched mode: the batch-table slot
        std::vector<uint32_t> ids;
        std::vector<Req> reqs;
        double t_start = 0.0;
        cudaEvent_t done = nullptr;
    };

    vm_server_params prm{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_result;
    std::map<uint32_t, Strm> streams;
    std::vector<uint32_t> open_order;
    uint32_t next_id = 0;
    uint64_t next_ticket = 1;
    std::deque<vm_server_result> results;
    uint64_t submitted = 0, finished = 0, steps = 0, step_reqs = 0, fallbacks = 0;
    double launch_s = 0.0, complete_s = 0.0;
    unsigned long long captures0 = 0, allocs0 = 0;
    uint64_t budget = 0, committed = 0;
    bool stop = false;
    std::thread th;
    // scheduler-thread state
    cudaStream_t fit_stream = nullptr;
    vmx::BatchFit bf;
    std::deque<Step> inflight;
    bool slot_busy[vmx::kMaxSlots] = {};
    std::vector<cudaEvent_t> free_events;
    uint32_t rr = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace vmx {
namespace {

using Server = vm_server;

// Grows the arena and the fit scratch for K clusters and N points.  The
// server's stream is drained first: steps already queued on it use the old
// buffers.
vm_status bf_size(Server* S, uint32_t K, uint32_t N) {
    BatchFit& b = S->bf;
    if (b.apts && K <= b.kcap && N <= b.ncap) return VM_OK;
    VM_CUDA(cudaStreamSynchronize(S->fit_stream));
    const uint32_t k2 = K > b.kcap ? (K > 2 * b.kcap ? K + K / 4 : 2 * b.kcap) : b.kcap;  // geometric growth
    const uint32_t n2 = N > b.ncap ? (N > 2 * b.ncap ? N + N / 4 : 2 * b.ncap) : b.ncap;
    VM_TRY(fit_prepare(b.fc, k2, n2, (int)S->prm.params.n_hyp, b.tune.tile, S->fit_stream));
    Carver dry{nullptr};
    dry.take<float>((size_t)n2 * 3);
    dry.take<uint32_t>((size_t)k2 + 1);
    dry.take<uint32_t>((size_t)k2 + 1);
    VM_TRY(ensure(b.arena, dry.off + 256));
    Carver c{static_cast<char*>(b.arena.p)};
    b.apts = c.take<float>((size_t)n2 * 3);
    b.aoff = c.take<uint32_t>((size_t)k2 + 1);
    b.alab = c.take<uint32_t>((size_t)k2 + 1);
    b.kcap = k2;
    b.ncap = n2;
    b.gen++;
    return VM_OK;
}

cudaError_t enqueue_batch(Server* S, int slot) {
    BatchFit& b = S->bf;
    cudaStream_t s = S->fit_stream;
    FitBuffers& fb = b.fc.fb;
    cudaError_t e;
    const int sms = device_sms();
    if ((e = cudaMemcpyAsync(b.dtab, b.htab[slot], sizeof(BatchTable), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    launch_k(k_batch_prefix, dim3(1), dim3(1), 0, s, b.dtab, b.kcap, b.ncap, fb.kdev, fb.err);
    const unsigned g = (unsigned)(sms * 8);
    launch_k(k_batch_gather, dim3(g), dim3(kGatherT), 0, s, b.dtab, b.apts, b.aoff, b.alab);
    count_launch(2);
    if ((e = launch_fit(b.apts, b.aoff, b.alab, fb.kdev, b.kcap, S->prm.params, fb, b.tune, sms, s, nullptr)) !=
        cudaSuccess)
        return e;
    launch_k(k_pack_batch, dim3(b.kcap < 4096 ? b.kcap : 4096), dim3(128), 0, s, b.dtab, fb.kdev, b.aoff, b.alab, fb.cl,
             fb.hull, fb.hull_cnt);
    launch_k(k_batch_header, dim3(1), dim3(kMaxBatch), 0, s, b.dtab, fb.hull_cnt, fb.err, b.dstat[slot]);
    count_launch(2);
    return cudaGetLastError();
}

vm_status launch_batch(Server* S, int slot) {
    BatchFit& b = S->bf;
    if (!b.gexec[slot] || b.ggen[slot] != b.gen) {
        if (b.gexec[slot]) cudaGraphExecDestroy(b.gexec[slot]);
        b.gexec[slot] = nullptr;
        fit_init_attributes();
        cudaGraph_t graph = nullptr;
        const unsigned long long l0 = launch_total();
        count_capture();
        VM_CUDA(cudaStreamBeginCapture(S->fit_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_batch(S, slot);
        cudaError_t e2 = cudaStreamEndCapture(S->fit_stream, &graph);
        b.glaunches[slot] = launch_total() - l0;
        uncount_launch(b.glaunches[slot]);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_status(e, "batched fit capture");
        }
        if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b.gexec[slot], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b.gexec[slot] = nullptr;
            return cuda_status(e, "cudaGraphInstantiate");
        }
        b.ggen[slot] = b.gen;
    }
    VM_CUDA(cudaGraphLaunch(b.gexec[slot], S->fit_stream));
    count_launch((int)b.glaunches[slot]);
    return VM_OK;
}

cudaEvent_t get_event(Server* S) {
    if (!S->free_events.empty()) {
        cudaEvent_t e = S->free_events.back();
        S->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

void push_result(Server* S, const Server::Req& r, vm_status st, const vm_planes& planes, double t_start) {
    vm_server_result res{};
    res.ticket = r.ticket;
    res.stream = r.stream;
    res.status = st;
    res.planes = planes;
    res.t_arrival = r.t_arr;
    res.t_start = t_start;
    res.t_done = S->now();
    std::lock_guard<std::mutex> lk(S->mu);
    S->results.push_back(res);
    S->finished++;
    auto it = S->streams.find(r.stream);
    if (it != S->streams.end()) it->second.busy = false;
    S->cv_result.notify_all();
}

// Runs a member on its own map's path (integrate already done): the whole
// single-map segmentation, with its own regrow-and-retry.
vm_status run_alone(Server* S, vm_map* m, vm_planes* out) {
    memset(out, 0, sizeof(*out));
    VM_TRY(launch_segment(m, S->prm.params));
    return finish_segment(m, S->prm.params, out);
}

void launch_step(Server* S, Server::Step& st) {
    const bool batched = S->prm.mode == VM_SERVE_BATCHED;
    st.t_start = S->now();
    std::vector<Server::Req> keep_r;
    std::vector<uint32_t> keep_i;
    BatchTable* tab = batched ? S->bf.htab[st.slot] : nullptr;
    uint32_t n_maps = 0, k_hint = 0, n_hint = 0;
    for (size_t i = 0; i < st.reqs.size(); ++i) {
        const Server::Req& r = st.reqs[i];
        Server::Strm* sp;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            sp = &S->streams[st.ids[i]];
        }
        vm_map* m = sp->map;
        vm_status s = vm_integrate(m, r.xyz, r.n, r.pose, r.on_dev);
        if (s == VM_OK) s = batched ? launch_front(m, S->prm.params) : launch_segment(m, S->prm.params);
        if (s == VM_OK && !sp->ev) sp->ev = get_event(S);
        if (s == VM_OK && cudaEventRecord(sp->ev, m->stream) != cudaSuccess)
            s = cuda_status(cudaGetLastError(), "event");
        if (s != VM_OK) {
            vm_planes none{};
            push_result(S, r, s, none, st.t_start);
            continue;
        }
        if (batched) {
            cudaStreamWaitEvent(S->fit_stream, sp->ev, 0);
            BatchEntry& E = tab->e[n_maps++];
            E.pts = m->seg.pts;
            E.cl_off = m->seg.cl_off;
            E.cl_label = m->seg.cl_label;
            E.ctr = m->seg.ctr;
            E.mc = m->ctr;
            E.seg_err = m->err;
            E.planes = reinterpret_cast<vm_plane*>(m->out_dev + out_planes_off());
            E.hull_xy = reinterpret_cast<int32_t*>(m->out_dev + out_xy_off(m->out_kcap));
            E.hull_xyz = reinterpret_cast<float*>(m->out_dev + out_xyz_off(m->out_kcap, m->out_hcap));
            E.header = reinterpret_cast<SegCounters*>(m->out_dev);
            E.hull_cap = m->out_hcap;
            k_hint += m->k_hint + m->k_hint / 4 + 64;
            n_hint += m->last.n_kept + m->last.n_kept / 4 + 4096;
        }
        keep_r.push_back(r);
        keep_i.push_back(st.ids[i]);
    }
    st.reqs.swap(keep_r);
    st.ids.swap(keep_i);
    if (!batched || st.reqs.empty()) return;
    tab->n_maps = n_maps;
    vm_status s = bf_size(S, k_hint, n_hint);
    if (s == VM_OK) s = launch_batch(S, st.slot);
    if (s == VM_OK) {
        st.done = get_event(S);
        if (!st.done || cudaEventRecord(st.done, S->fit_stream) != cudaSuccess)
            s = cuda_status(cudaGetLastError(), "event");
    }
    if (s != VM_OK) {  // the batch could not be launched: every member runs alone
        cudaStreamSynchronize(S->fit_stream);
        for (size_t i = 0; i < st.reqs.size(); ++i) {
            vm_map* m;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                m = S->streams[st.ids[i]].map;
            }
            vm_planes out{};
            const vm_status s2 = run_alone(S, m, &out);
            S->fallbacks++;
            push_result(S, st.reqs[i], s2, out, st.t_start);
        }
        st.reqs.clear();
        st.ids.clear();
    }
}

bool step_ready(Server* S, const Server::Step& st) {
    if (st.reqs.empty()) return true;
    if (S->prm.mode == VM_SERVE_BATCHED) return cudaEventQuery(st.done) != cudaErrorNotReady;
    for (uint32_t id : st.ids) {
        cudaEvent_t e;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            e = S->streams[id].ev;
        }
        if (cudaEventQuery(e) == cudaErrorNotReady) return false;
    }
    return true;
}

void complete_step(Server* S, Server::Step& st) {
    const bool batched = S->prm.mode == VM_SERVE_BATCHED;
    if (batched && !st.reqs.empty()) {
        BatchStatus* bs = S->bf.hstat[st.slot];  // written before st.done was recorded
        for (int attempt = 0; attempt < 3 && (bs->err & kErrScratch); ++attempt) {  // the arena was too small
            if (bf_size(S, bs->K_need, bs->N_need) != VM_OK) break;
            if (launch_batch(S, st.slot) != VM_OK) break;
            cudaStreamSynchronize(S->fit_stream);
        }
    }
    for (size_t i = 0; i < st.reqs.size(); ++i) {
        vm_map* m;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            m = S->streams[st.ids[i]].map;
        }
        vm_planes out{};
        vm_status s;
        if (batched) {
            cudaStreamSynchronize(m->stream);
            const bool batch_short = (S->bf.hstat[st.slot]->err & kErrScratch) != 0;
            if (take_hints(m) || batch_short) {
                S->fallbacks++;
                s = run_alone(S, m, &out);
            } else {
                s = read_result(m, &out);
            }
        } else {
            s = finish_segment(m, S->prm.params, &out);
        }
        push_result(S, st.reqs[i], s, out, st.t_start);
    }
    if (st.done) S->free_events.push_back(st.done);
    st.done = nullptr;
    if (st.slot >= 0) S->slot_busy[st.slot] = false;
}

void scheduler(Server* S) {
    cudaSetDevice((int)S->prm.device);
    const bool batched = S->prm.mode == VM_SERVE_BATCHED;
    const size_t max_steps = batched ? S->prm.max_inflight : (size_t)S->prm.max_inflight * S->prm.max_batch;
    const size_t per_step = batched ? S->prm.max_batch : 1;
    for (;;) {
        // 1. admissions and closes (map creation and destruction outside the lock)
        std::vector<uint32_t> admit, drop;
        bool stop;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            stop = S->stop;
            for (uint32_t id : S->open_order) {
                auto& s = S->streams[id];
                if (s.state == 0 && (!s.close_req || !s.q.empty())) {  // a closed stream's queue still runs
                    if (S->committed + s.footprint > S->budget) break;  // first come, first admitted
                    S->committed += s.footprint;
                    s.state = 1;  // reserved; the map follows below
                    admit.push_back(id);
                }
            }
            for (uint32_t id : S->open_order) {
                auto& s = S->streams[id];
                if (s.close_req && s.q.empty() && !s.busy) drop.push_back(id);
            }
        }
        for (uint32_t id : admit) {
            vm_map_params mp;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                mp = S->streams[id].mp;
            }
            vm_map* m = nullptr;
            const vm_status st = vm_create(&mp, nullptr, &m);
            std::lock_guard<std::mutex> lk(S->mu);
            auto& s = S->streams[id];
            if (st == VM_OK) {
                s.map = m;
            } else {  // the map could not be made: its requests fail
                s.state = 0;
                S->committed -= s.footprint;
                s.close_req = true;
                while (!s.q.empty()) {
                    Server::Req r = s.q.front();
                    s.q.pop_front();
                    vm_server_result res{};
                    res.ticket = r.ticket;
                    res.stream = id;
                    res.status = st;
                    res.t_arrival = r.t_arr;
                    res.t_start = res.t_done = S->now();
                    S->results.push_back(res);
                    S->finished++;
                }
                S->cv_result.notify_all();
            }
        }
        for (uint32_t id : drop) {
            vm_map* m;
            cudaEvent_t ev;
            uint64_t fp;
            int state;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                auto& s = S->streams[id];
                m = s.map;
                ev = s.ev;
                fp = s.footprint;
                state = s.state;
            }
            if (m) vm_destroy(m);
            if (ev) S->free_events.push_back(ev);
            std::lock_guard<std::mutex> lk(S->mu);
            if (state == 1) S->committed -= fp;
            S->streams.erase(id);
            for (size_t i = 0; i < S->open_order.size(); ++i)
                if (S->open_order[i] == id) {
                    S->open_order.erase(S->open_order.begin() + (long)i);
                    break;
                }
        }
        // 2. completions
        bool progressed = !admit.empty() || !drop.empty();
        for (auto it = S->inflight.begin(); it != S->inflight.end();) {
            if (!step_ready(S, *it)) {
                if (batched) break;  // batched steps finish in order on the server stream
                ++it;
                continue;
            }
            const double c0 = S->now();
            complete_step(S, *it);
            S->complete_s += S->now() - c0;
            it = S->inflight.erase(it);
            progressed = true;
        }
        if (stop && S->inflight.empty()) break;
        // 3. a new step from the streams that have a request waiting and none running
        if (!stop && S->inflight.size() < max_steps) {
            Server::Step st;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                const size_t n = S->open_order.size();
                // Batched: a step takes at most its share of the streams with work
                // (running or not) over the steps that may be in flight, so that
                // when every stream is busy the next step's integrate and front
                // halves overlap the previous step's fit instead of all streams
                // forming one step that nothing overlaps.
                size_t take = per_step;
                if (batched && max_steps > 1) {
                    size_t waiting = 0;
                    for (uint32_t id : S->open_order) {
                        const auto& s = S->streams[id];
                        waiting += s.state == 1 && s.map && (s.busy || !s.q.empty());
                    }
                    const size_t share = (waiting + max_steps - 1) / max_steps;
                    if (share >= 1 && share < take) take = share;
                }
                for (size_t j = 0; j < n && st.reqs.size() < take; ++j) {
                    const uint32_t id = S->open_order[(S->rr + j) % n];
                    auto& s = S->streams[id];
                    if (s.state != 1 || !s.map || s.busy || s.q.empty()) continue;
                    st.reqs.push_back(s.q.front());
                    st.ids.push_back(id);
                    s.q.pop_front();
                    s.busy = true;
                }
                if (n) S->rr = (S->rr + 1) % (uint32_t)n;
            }
            if (!st.reqs.empty()) {
                if (batched) {
                    for (int k = 0; k < kMaxSlots; ++k)
                        if (!S->slot_busy[k]) {
                            st.slot = k;
                            break;
                        }
                    S->slot_busy[st.slot] = true;
                }
                S->steps++;
                S->step_reqs += st.reqs.size();
                const double l0 = S->now();
                launch_step(S, st);
                S->launch_s += S->now() - l0;
                if (!st.reqs.empty()) {
                    S->inflight.push_back(std::move(st));
                } else if (st.slot >= 0) {
                    S->slot_busy[st.slot] = false;
                }
                continue;
            }
        }
        if (progressed) continue;
        if (!S->inflight.empty()) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            continue;
        }
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
}

vm_status check_map_params(const vm_map_params* p) {
    if (!p || p->dims[0] <= 0 || p->dims[1] <= 0 || p->dims[2] <= 0 || !(p->voxel_size > 0.0f)) {
        set_error("dims and voxel_size must be positive");
        return VM_ERR_INVALID_ARG;
    }
    uint64_t nb = 1;
    for (int a = 0; a < 3; ++a) {
        if ((double)p->dims[a] * (double)p->voxel_size > 16.0 + 1e-9) {
            set_error("map extent beyond 16 m on an axis");
            return VM_ERR_INVALID_ARG;
        }
        nb *= (uint64_t)((p->dims[a] + kBrick - 1) / kBrick);
    }
    if (nb * kBrickVox > 0xFFFFFFFFull) {
        set_error("more than 2^32 voxel ids");
        return VM_ERR_EXTENT;
    }
    return VM_OK;
}

void release_server(Server* S) {
    for (auto& kv : S->streams) {
        if (kv.second.map) vm_destroy(kv.second.map);
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    }
    S->streams.clear();
    for (auto& r : S->results) vm_planes_free(&r.planes);
    S->results.clear();
    for (auto e : S->free_events) cudaEventDestroy(e);
    S->free_events.clear();
    BatchFit& b = S->bf;
    for (int k = 0; k < kMaxSlots; ++k) {
        if (b.gexec[k]) cudaGraphExecDestroy(b.gexec[k]);
        if (b.htab[k]) cudaFreeHost(b.htab[k]);
        if (b.hstat[k]) cudaFreeHost(b.hstat[k]);
    }
    if (b.dtab) cudaFree(b.dtab);
    release(b.arena);
    fit_release(b.fc);
    if (S->fit_stream) cudaStreamDestroy(S->fit_stream);
}

}  // namespace
}  // namespace vmx

extern "C" {

uint64_t vm_server_footprint(const vm_map_params* map, const vm_segment_params* params) {
    if (!map || !params) return 0;
    return map_footprint(*map, *params);
}

vm_status vm_server_create(const vm_server_params* params, vm_server** out) {
    if (!params || !out) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    VM_TRY(check_single_round(&params->params));
    if (params->max_batch < 1 || params->max_batch > (uint32_t)kMaxBatch || params->max_inflight < 1 ||
        params->max_inflight > (uint32_t)kMaxSlots || params->mode > VM_SERVE_STREAMS) {
        set_error("max_batch must be 1..64, max_inflight 1..4, mode VM_SERVE_BATCHED or VM_SERVE_STREAMS");
        return VM_ERR_INVALID_ARG;
    }
    const vm_fit_tuning& t = params->tuning;
    if (t.tile && (t.tile < 256 || t.tile > 16384 || t.tile % 256 || !(t.hyp_per_thread == 1 || t.hyp_per_thread == 2 ||
                                                      t.hyp_per_thread == 4 || t.hyp_per_thread == 8) ||
                   t.ctas_per_sm < 1 || t.ctas_per_sm > 16 || t.schedule > 1)) {
        set_error("tuning out of range");
        return VM_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    VM_CUDA(cudaSetDevice((int)params->device));
    vm_server* S = new (std::nothrow) vm_server();
    if (!S) {
        cudaSetDevice(prev);
        set_error("host allocation failed");
        return VM_ERR_OUT_OF_MEMORY;
    }
    S->prm = *params;
    S->t0 = std::chrono::steady_clock::now();
    S->captures0 = capture_total();
    S->allocs0 = alloc_total();
    S->bf.tune = t.tile ? FitTuning{(int)t.tile, (int)t.hyp_per_thread, (int)t.ctas_per_sm, (int)t.schedule}
                        : default_tuning();
    vm_status st = VM_OK;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) st = cuda_status(e, "cudaMemGetInfo");
    if (st == VM_OK) {
        S->budget = params->hbm_budget ? params->hbm_budget
                                       : (free_b > params->hbm_reserve ? free_b - params->hbm_reserve : 0);
        e = cudaStreamCreateWithFlags(&S->fit_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_status(e, "cudaStreamCreate");
    }
    if (st == VM_OK) {
        e = cudaMalloc(&S->bf.dtab, sizeof(BatchTable));
        if (e != cudaSuccess) st = cuda_status(e, "cudaMalloc");
    }
    for (int k = 0; st == VM_OK && k < kMaxSlots; ++k) {
        void* h = nullptr;
        e = cudaMallocHost(&h, sizeof(BatchTable));
        if (e != cudaSuccess) {
            st = cuda_status(e, "cudaMallocHost");
            break;
        }
        memset(h, 0, sizeof(BatchTable));
        S->bf.htab[k] = static_cast<BatchTable*>(h);
        e = cudaHostAlloc(&h, sizeof(BatchStatus), cudaHostAllocMapped);
        if (e != cudaSuccess) {
            st = cuda_status(e, "cudaHostAlloc(mapped)");
            break;
        }
        memset(h, 0, sizeof(BatchStatus));
        S->bf.hstat[k] = static_cast<BatchStatus*>(h);
        void* d = nullptr;
        e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) {
            st = cuda_status(e, "cudaHostGetDevicePointer");
            break;
        }
        S->bf.dstat[k] = static_cast<BatchStatus*>(d);
    }
    if (st == VM_OK && params->mode == VM_SERVE_BATCHED) st = bf_size(S, 1024, 1u << 20);
    if (st != VM_OK) {
        release_server(S);
        delete S;
        cudaSetDevice(prev);
        return st;
    }
    S->th = std::thread(scheduler, S);
    cudaSetDevice(prev);
    *out = S;
    return VM_OK;
}

vm_status vm_server_open(vm_server* S, const vm_map_params* map, uint32_t* stream_id) {
    if (!S || !stream_id) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    VM_TRY(check_map_params(map));
    const uint64_t fp = map_footprint(*map, S->prm.params);
    std::lock_guard<std::mutex> lk(S->mu);
    if (fp > S->budget) {
        set_error("the stream's device-memory footprint exceeds the server's whole budget");
        return VM_ERR_OUT_OF_MEMORY;
    }
    const uint32_t id = S->next_id++;
    auto& s = S->streams[id];
    s.mp = *map;
    s.footprint = fp;
    S->open_order.push_back(id);
    *stream_id = id;
    S->cv_work.notify_one();
    return VM_OK;
}

vm_status vm_server_submit(vm_server* S, uint32_t stream_id, const float* xyz, uint32_t n, const float pose3x4[12],
                           int xyz_on_device, double t_arrival, uint64_t* ticket) {
    if (!S || !pose3x4 || (!xyz && n)) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    vm_server::Req r{};
    r.stream = stream_id;
    r.xyz = xyz;
    r.n = n;
    memcpy(r.pose, pose3x4, sizeof(r.pose));
    r.on_dev = xyz_on_device;
    r.t_arr = t_arrival >= 0.0 ? t_arrival : S->now();
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end() || it->second.close_req) {
        set_error("unknown or closed stream");
        return VM_ERR_INVALID_ARG;
    }
    r.ticket = S->next_ticket++;
    it->second.q.push_back(r);
    S->submitted++;
    if (ticket) *ticket = r.ticket;
    S->cv_work.notify_one();
    return VM_OK;
}

vm_status vm_server_poll(vm_server* S, vm_server_result* out, uint32_t cap, uint32_t* n, int timeout_ms) {
    if (!S || !n || (cap && !out)) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    *n = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->results.empty() && timeout_ms != 0) {
        auto pred = [&] { return !S->results.empty(); };
        if (timeout_ms < 0)
            S->cv_result.wait(lk, pred);
        else
            S->cv_result.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    uint32_t k = 0;
    while (k < cap && !S->results.empty()) {
        out[k++] = S->results.front();
        S->results.pop_front();
    }
    *n = k;
    return VM_OK;
}

vm_status vm_server_drain(vm_server* S, int timeout_ms) {
    if (!S) {
        set_error("null server");
        return VM_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto pred = [&] { return S->finished == S->submitted; };
    if (timeout_ms < 0) {
        S->cv_result.wait(lk, pred);
        return VM_OK;
    }
    if (!S->cv_result.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        set_error("requests still running when the drain timed out");
        return VM_ERR_TIMEOUT;
    }
    return VM_OK;
}

vm_status vm_server_close(vm_server* S, uint32_t stream_id) {
    if (!S) {
        set_error("null server");
        return VM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end()) {
        set_error("unknown stream");
        return VM_ERR_INVALID_ARG;
    }
    it->second.close_req = true;
    S->cv_work.notify_one();
    return VM_OK;
}

vm_status vm_server_get_stats(vm_server* S, vm_server_stats* out) {
    if (!S || !out) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    for (auto& kv : S->streams) {
        out->streams_open++;
        if (kv.second.state == 1) out->streams_admitted++; else out->streams_waiting++;
    }
    out->requests_submitted = S->submitted;
    out->requests_done = S->finished;
    out->steps = S->steps;
    out->fallbacks = S->fallbacks;
    out->hbm_budget = S->budget;
    out->hbm_committed = S->committed;
    out->mean_step_requests = S->steps ? (double)S->step_reqs / (double)S->steps : 0.0;
    out->launch_seconds = S->launch_s;
    out->complete_seconds = S->complete_s;
    out->graph_captures = capture_total() - S->captures0;
    out->allocations = alloc_total() - S->allocs0;
    return VM_OK;
}

double vm_server_now(vm_server* S) { return S ? S->now() : 0.0; }

vm_status vm_server_destroy(vm_server* S) {
    if (!S) return VM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice((int)S->prm.device);
    release_server(S);
    cudaSetDevice(prev);
    delete S;
    return VM_OK;
}

}  // extern "C"
