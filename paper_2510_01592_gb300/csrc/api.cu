// api.cu -- the C ABI of libvoxmps.so (include/vm.h): map lifecycle, device
// scratch management and the host-side ordering of the kernels of one call.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.cuh"

using namespace vmx;

namespace vmx {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launch_total() { return g_launches.load(); }
static std::atomic<unsigned long long> g_captures{0}, g_allocs{0};
void count_capture() { g_captures.fetch_add(1, std::memory_order_relaxed); }
unsigned long long capture_total() { return g_captures.load(); }
void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }
unsigned long long alloc_total() { return g_allocs.load(); }
void uncount_launch(unsigned long long n) { g_launches.fetch_sub(n); }

static const char* kStageNames[kNumStages] = {"integrate", "order_bricks", "finalize", "moments", "eigen",
                                              "ccl_local", "ccl_cross", "clusters", "ransac_hyp", "ransac_score",
                                              "extract", "refit_hull", "pack", "clear", "rounds"};


void set_error(const std::string& msg) { g_err = msg; }

bool pdl_enabled() {
    static const bool on = [] {
        const char* v = getenv("VOXMPS_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

vm_status cuda_status(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? VM_ERR_OUT_OF_MEMORY : VM_ERR_CUDA;
}

vm_status ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return VM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 4 + 256;
    count_alloc();
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e, "cudaMalloc");
    }
    b.bytes = want;
    return VM_OK;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}



// The fit scratch for kcap clusters, npts points, `chunks` 256-point partial
// sums and H hypotheses, carved in order.
static void fit_layout(Carver& c, FitBuffers& fb, size_t kcap, size_t npts, size_t chunks, int H) {
    fb.hyp = c.take<float4>(kcap * H);
    fb.hyp_valid = c.take<uint8_t>(kcap * H);
    fb.counts = c.take<uint32_t>(kcap * H);
    fb.cl = c.take<FitCluster>(kcap);
    fb.item_off = c.take<uint32_t>(kcap + 1);
    fb.item_cl = c.take<uint32_t>(chunks + 1);  // items never outnumber the chunk slots
    fb.queue = c.take<uint32_t>(4);
    fb.inlier = c.take<uint8_t>(npts + 1);
    fb.part = c.take<float>((chunks + 1) * 10);
    fb.cen = c.take<float>(kcap * 6);
    fb.surv = c.take<int2>(npts + 1);
    fb.hull = c.take<int2>(npts + 1);
    fb.hull_cnt = c.take<uint32_t>(kcap + 1);
    fb.scan_tmp = c.take<uint32_t>(scan_tmp_words(kcap + 1));
    fb.err = c.take<uint32_t>(4);
    fb.tot = c.take<uint32_t>(4);
    fb.kdev = c.take<uint32_t>(4);
    fb.done = c.take<uint32_t>(kcap * 3);
}

size_t fit_bytes(size_t kcap, size_t npts, size_t chunks, int H) {
    Carver dry{nullptr};
    FitBuffers fb{};
    fit_layout(dry, fb, kcap, npts, chunks, H);
    return dry.off + 256;
}

// Partial-sum chunks a batch can need with work items of `tile` points (a
// multiple of 256): every item holds tile / 256 chunk slots.
static size_t fit_chunks(size_t kcap, size_t npts, int tile) {
    return (npts / (size_t)tile + kcap + 1) * ((size_t)tile / 256);
}

vm_status fit_prepare(FitContext& fc, size_t kcap, size_t npts, int H, int tile, cudaStream_t s) {
    const size_t chunks = fit_chunks(kcap, npts, tile);
    if (fc.mem.p && kcap <= fc.kcap && npts <= fc.npts && chunks <= fc.items && H <= fc.H) return VM_OK;
    const size_t k2 = kcap + kcap / 4 + 16, n2 = npts + npts / 4 + 1024;
    const size_t c2 = fit_chunks(k2, n2, tile) > fc.items ? fit_chunks(k2, n2, tile) : fc.items;
    const int H2 = H > fc.H ? H : fc.H;
    VM_TRY(ensure(fc.mem, fit_bytes(k2, n2, c2, H2)));
    Carver c{static_cast<char*>(fc.mem.p)};
    FitBuffers fb{};
    fit_layout(c, fb, k2, n2, c2, H2);
    VM_CUDA(cudaMemsetAsync(fb.scan_tmp, 0, scan_tmp_words(k2 + 1) * sizeof(uint32_t), s));  // scan state
    fb.kcap = k2;
    fb.npts_cap = n2;
    fb.items_cap = c2;
    fb.H = H2;
    fc.fb = fb;
    fc.gen++;
    fc.kcap = k2;
    fc.npts = n2;
    fc.items = c2;
    fc.H = H2;
    return VM_OK;
}

void fit_release(FitContext& fc) {
    fc.timer.release();
    release(fc.mem);
    release(fc.out);
    if (fc.host) cudaFreeHost(fc.host);
    fc.host = nullptr;
    fc.host_bytes = 0;
    fc.kcap = fc.npts = fc.items = 0;
    fc.H = 0;
}

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

vm_status check_params(const vm_segment_params* p) {
    if (!p) {
        set_error("null segment params");
        return VM_ERR_INVALID_ARG;
    }
    if (p->n_hyp < 1 || p->n_hyp > 1024) {
        set_error("n_hyp must be in [1, 1024]");
        return VM_ERR_INVALID_ARG;
    }
    if (!(p->eps >= 0.0f) || !(p->d_th2 >= 0.0f)) {
        set_error("eps and d_th2 must be non-negative");
        return VM_ERR_INVALID_ARG;
    }
    if (p->planes_per_cluster > kMaxRounds) {
        set_error("planes_per_cluster must be at most 8");
        return VM_ERR_INVALID_ARG;
    }
    return VM_OK;
}

vm_status check_single_round(const vm_segment_params* p) {
    VM_TRY(check_params(p));
    if (p->planes_per_cluster > 1) {
        set_error("planes_per_cluster > 1 is supported by vm_segment only");
        return VM_ERR_INVALID_ARG;
    }
    return VM_OK;
}

// Runs the fit on k clusters and returns the packed result on the host.
static vm_status fit_and_pack(FitContext& fc, const float* pts, const uint32_t* off, const uint32_t* labels,
                              uint32_t k, uint32_t npts, const vm_segment_params& p, const FitTuning& tune,
                              cudaStream_t s, vm_planes* out) {
    memset(out, 0, sizeof(*out));
    if (k == 0) return VM_OK;
    VM_TRY(fit_prepare(fc, k, npts, (int)p.n_hyp, tune.tile, s));
    FitBuffers& fb = fc.fb;
    VM_CUDA(cudaMemsetAsync(fb.err, 0, sizeof(uint32_t), s));
    StageHook* hk = fc.timer.hook();
    VM_CUDA(fit_set_count(fb.kdev, k, s));
    VM_CUDA(launch_fit(pts, off, labels, fb.kdev, k, p, fb, tune, device_sms(), s, hk));
    uint32_t hdr[2];
    VM_CUDA(cudaMemcpyAsync(&hdr[0], fb.hull_cnt + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VM_CUDA(cudaMemcpyAsync(&hdr[1], fb.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VM_CUDA(cudaStreamSynchronize(s));
    const uint32_t n_hull = hdr[0];
    const size_t b_planes = (size_t)k * sizeof(vm_plane);
    const size_t b_xy = (size_t)n_hull * 2 * sizeof(int32_t);
    const size_t b_xyz = (size_t)n_hull * 3 * sizeof(float);
    const size_t o_xy = (b_planes + 255) & ~(size_t)255;
    const size_t o_xyz = (o_xy + b_xy + 255) & ~(size_t)255;
    const size_t total = o_xyz + b_xyz + 256;
    VM_TRY(ensure(fc.out, total));
    char* d = static_cast<char*>(fc.out.p);
    VM_STAGE_BEGIN(hk, kStPack, s);
    VM_CUDA(launch_pack(fb, off, labels, fb.kdev, k, reinterpret_cast<vm_plane*>(d),
                        reinterpret_cast<int32_t*>(d + o_xy), reinterpret_cast<float*>(d + o_xyz), n_hull, s));
    if (fc.host_bytes < total) {
        if (fc.host) cudaFreeHost(fc.host);
        fc.host = nullptr;
        fc.host_bytes = 0;
        VM_CUDA(cudaMallocHost(&fc.host, total + total / 4));
        fc.host_bytes = total + total / 4;
    }
    VM_CUDA(cudaMemcpyAsync(fc.host, d, total, cudaMemcpyDeviceToHost, s));
    VM_STAGE_END(hk, kStPack, s);
    VM_CUDA(cudaStreamSynchronize(s));
    fc.timer.fold();
    out->planes = static_cast<vm_plane*>(malloc(b_planes ? b_planes : 1));
    out->hull_xy = static_cast<int32_t*>(malloc(b_xy ? b_xy : 1));
    out->hull_xyz = static_cast<float*>(malloc(b_xyz ? b_xyz : 1));
    if (!out->planes || !out->hull_xy || !out->hull_xyz) {
        vm_planes_free(out);
        set_error("host allocation of the result failed");
        return VM_ERR_OUT_OF_MEMORY;
    }
    const char* h = static_cast<const char*>(fc.host);
    memcpy(out->planes, h, b_planes);
    memcpy(out->hull_xy, h + o_xy, b_xy);
    memcpy(out->hull_xyz, h + o_xyz, b_xyz);
    out->n_planes = k;
    out->n_hull = n_hull;
    if (hdr[1] & kErrTimeout) {
        set_error("a bounded device loop reached its iteration cap during the plane fit");
        return VM_ERR_TIMEOUT;
    }
    if (hdr[1] & kErrOverflow) {
        set_error("a cluster spans more than 2^28 hull quanta (4096 m) in its plane; its hull is not exact");
        return VM_ERR_EXTENT;
    }
    return VM_OK;
}



// Scan state for every scan of a segmentation (at most max(nv, bricks) + 1
// elements); the radix sort has its own region (histograms and their scan).
static size_t vox_tmp_words(size_t nv, uint32_t nb_total) {
    return scan_tmp_words((nv > (size_t)nb_total ? nv : (size_t)nb_total) + 1);
}

// The rank-dense voxel arrays of nv slots, carved in order.
static void vox_layout(Carver& c, SegBuffers& b, size_t nv, size_t tmp_words) {
    b.M = c.take<int32_t>(3 * nv);
    b.nrm = c.take<float>(3 * nv);
    b.status = c.take<uint8_t>(nv);
    b.nbr = c.take<uint8_t>(nv);
    b.rec = c.take<float4>(2 * nv);
    b.list_idx = c.take<uint32_t>(nv);
    b.list_A = c.take<float>(6 * nv);
    b.parent = c.take<uint32_t>(nv);
    b.count = c.take<uint32_t>(nv);
    b.cid = c.take<uint32_t>(nv + 1);
    b.vert_flag = c.take<uint32_t>(nv + 1);
    b.keys = c.take<uint32_t>(nv);
    b.vals = c.take<uint32_t>(nv);
    b.keys_alt = c.take<uint32_t>(nv);
    b.vals_alt = c.take<uint32_t>(nv);
    b.cl_size = c.take<uint32_t>(nv + 1);
    b.cl_off = c.take<uint32_t>(nv + 1);
    b.cl_label = c.take<uint32_t>(nv + 1);
    b.pts = c.take<float>(3 * nv);
    b.pt_vid = c.take<uint32_t>(nv);
    b.scan_tmp = c.take<uint32_t>(tmp_words);
    b.sort_tmp = c.take<uint32_t>(sort_tmp_words(nv));
}

vm_status alloc_vox(vm_map* m, uint32_t n_bricks) {
    const size_t need = (size_t)(n_bricks ? n_bricks : 1) * kBrickVox;
    if (m->vox_mem.p && need <= m->seg_nv) return VM_OK;
    size_t nv = need;
    const size_t cap_nv = (size_t)m->capacity * kBrickVox;
    if (nv > cap_nv) nv = cap_nv;
    m->gen++;
    const size_t tmp_words = vox_tmp_words(nv, m->nb_total);
    Carver dry{nullptr};
    SegBuffers tmp{};
    vox_layout(dry, tmp, nv, tmp_words);
    VM_TRY(ensure(m->vox_mem, dry.off + 256));
    Carver c{static_cast<char*>(m->vox_mem.p)};
    vox_layout(c, m->seg, nv, tmp_words);
    VM_CUDA(cudaMemsetAsync(m->seg.scan_tmp, 0, tmp_words * sizeof(uint32_t), m->stream));  // scan states
    VM_CUDA(cudaMemsetAsync(m->seg.sort_tmp, 0, sort_tmp_words(nv) * sizeof(uint32_t), m->stream));
    m->seg.nv = nv;
    m->seg.kcap = nv;
    m->seg_nv = nv;
    return VM_OK;
}

uint64_t map_footprint(const vm_map_params& p, const vm_segment_params& sp) {
    uint64_t nb = 1;
    for (int a = 0; a < 3; ++a) nb *= (uint64_t)((p.dims[a] + kBrick - 1) / kBrick);
    const uint64_t cap = p.brick_capacity && p.brick_capacity < nb ? p.brick_capacity : nb;
    const uint64_t pool = nb * 4 + cap * 4 + cap * kBrickVox * (3 * 8 + 4) + cap * (kBrickVox / 8) +
                          scroll_tmp_words((uint32_t)cap) * 4 + 4096;
    const uint64_t bricks = (nb + 1) * 4 + nb * 4 + cap * 8 + 4096;
    const size_t nv = (size_t)cap * kBrickVox;
    Carver dry{nullptr};
    SegBuffers tmp{};
    vox_layout(dry, tmp, nv, vox_tmp_words(nv, (uint32_t)nb));
    const uint32_t mc = sp.min_cluster > 16 ? sp.min_cluster : 16;
    const uint64_t kcap = nv / mc > 256 ? nv / mc : 256;
    const uint64_t hcap = 65536 + kcap * 16;
    const uint64_t out = 256 + kcap * sizeof(vm_plane) + hcap * 20 + 1024;
    const uint64_t stage = 22ull << 20;  // host-input staging and deferred indices for frames of up to ~1.4 M points
    return pool + bricks + (uint64_t)dry.off * 5 / 4 + out + stage;
}

size_t out_planes_off() { return 256; }
size_t out_xy_off(uint32_t kcap) { return (256 + (size_t)kcap * sizeof(vm_plane) + 255) & ~(size_t)255; }
size_t out_xyz_off(uint32_t kcap, uint32_t hcap) { return (out_xy_off(kcap) + (size_t)hcap * 8 + 255) & ~(size_t)255; }

vm_status ensure_out(vm_map* m, uint32_t kcap, uint32_t hcap) {
    if (m->out_host && kcap <= m->out_kcap && hcap <= m->out_hcap) return VM_OK;
    if (m->out_host) cudaFreeHost(m->out_host);
    m->out_host = nullptr;
    m->out_dev = nullptr;
    const size_t bytes = out_xyz_off(kcap, hcap) + (size_t)hcap * 12 + 256;
    count_alloc();
    cudaError_t e = cudaHostAlloc(&m->out_host, bytes, cudaHostAllocMapped);
    if (e != cudaSuccess) {
        m->out_host = nullptr;
        return cuda_status(e, "cudaHostAlloc(mapped)");
    }
    void* d = nullptr;
    e = cudaHostGetDevicePointer(&d, m->out_host, 0);
    if (e != cudaSuccess) return cuda_status(e, "cudaHostGetDevicePointer");
    memset(m->out_host, 0, 256);
    m->out_dev = static_cast<char*>(d);
    m->out_bytes = bytes;
    m->out_kcap = kcap;
    m->out_hcap = hcap;
    m->gen++;
    return VM_OK;
}

// Scratch of the further extraction rounds: remaining points of nv voxels,
// kcap clusters, hcap staged hull vertices (the result block's hull capacity).
static vm_status ensure_rounds(vm_map* m, size_t nv, size_t kcap, size_t hcap) {
    RoundBuffers& rb = m->rounds;
    if (m->round_mem.p && rb.nv >= nv && rb.kcap >= kcap && rb.hcap >= hcap) return VM_OK;
    VM_TRY(ensure(m->round_mem, rounds_bytes(nv, kcap, hcap)));
    rounds_layout(static_cast<char*>(m->round_mem.p), rb, nv, kcap, hcap);
    m->gen++;
    return VM_OK;
}

// Sizes the scratch from the last known counts with headroom; a launch whose
// counts still do not fit raises kErrScratch and the caller retries.
vm_status plan_capacity(vm_map* m, const vm_segment_params& p, bool with_fit) {
    const uint32_t want_b = m->brick_hint + m->brick_hint / 4 + 64;
    const uint32_t cap_b = want_b < m->capacity ? want_b : m->capacity;
    if (!m->vox_mem.p || (size_t)cap_b * kBrickVox > m->seg_nv) {
        // Geometric growth (at least 1024 bricks and 1.5x the hint, then
        // doubling): a map that grows every frame re-allocates, and its graph
        // is re-captured, only a few times.
        const size_t have_b = m->vox_mem.p ? m->seg_nv / kBrickVox : 0;
        size_t grow = have_b * 2 > 1024 ? have_b * 2 : 1024;
        if (grow < (size_t)cap_b + cap_b / 2) grow = (size_t)cap_b + cap_b / 2;
        if (grow > m->capacity) grow = m->capacity;
        VM_TRY(alloc_vox(m, (uint32_t)grow));
    }
    const size_t nv = m->seg_nv;
    // Cluster capacity from the last count with headroom (a segmentation with
    // more clusters flags itself and is re-run with the count it needed): the
    // fit's grids, the sort's digit passes and the fit scratch all scale with
    // it, so it tracks the map rather than the worst case nv / min_cluster.
    size_t kcap = (size_t)m->k_hint + m->k_hint / 4 + 64;
    if (kcap < 256) kcap = 256;
    if (kcap > nv) kcap = nv;
    if (kcap < m->kcap) kcap = m->kcap;  // never shrink: keeps the captured graph valid
    m->kcap = (uint32_t)kcap;
    if (with_fit) {
        const uint64_t g0 = m->fit.gen;
        VM_TRY(fit_prepare(m->fit, kcap, nv, (int)p.n_hyp, m->tune.tile, m->stream));
        if (m->fit.gen != g0) m->gen++;
    }
    uint32_t hcap = m->hull_hint + m->hull_hint / 2 + 4096;
    if (hcap < 65536) hcap = 65536;
    if (hcap < m->out_hcap) hcap = m->out_hcap;
    const uint32_t P = p.planes_per_cluster > 1 ? p.planes_per_cluster : 1;
    size_t rcap = kcap;  // output records: one per cluster, more with several rounds
    if (P > 1) {
        const size_t rh = (size_t)m->rec_hint + m->rec_hint / 4 + 64;
        if (rcap < rh) rcap = rh;
        if (rcap > kcap * P) rcap = kcap * P;
    }
    VM_TRY(ensure_out(m, (uint32_t)rcap, hcap));
    if (with_fit && P > 1) VM_TRY(ensure_rounds(m, nv, kcap, m->out_hcap));
    return VM_OK;
}

// The result header; rounds (null for one plane per cluster): the record and
// hull-vertex totals of the extraction rounds.
__global__ void k_header(HeaderArgs a) {
    pdl_gate();
    write_header(a);
}

// The whole segmentation as one fixed launch sequence (every count is read on
// the device): order bricks, means, normals, clustering, clusters, RANSAC,
// refit, hull, pack into the mapped result block, header.
cudaError_t enqueue_front(vm_map* m, const vm_segment_params& p, StageHook* hk, uint32_t* also_zero) {
    cudaStream_t s = m->stream;
    const int sms = device_sms();
    SegBuffers& b = m->seg;
    cudaError_t e;
    VM_STAGE_BEGIN(hk, kStOrder, s);
    if ((e = seg_order_bricks(m->brick_table, m->nb_total, b, sms, s, m->err, also_zero)) != cudaSuccess) return e;
    VM_STAGE_END(hk, kStOrder, s);
    return seg_run(m->g, m->S, m->C, p, b, m->kcap, m->err, sms, s, hk);
}

cudaError_t enqueue_segment(vm_map* m, const vm_segment_params& p, StageHook* hk) {
    cudaStream_t s = m->stream;
    const int sms = device_sms();
    SegBuffers& b = m->seg;
    FitBuffers& fb = m->fit.fb;
    cudaError_t e;
    if ((e = enqueue_front(m, p, hk, fb.err)) != cudaSuccess) return e;
    char* d = m->out_dev;
    vm_plane* planes = reinterpret_cast<vm_plane*>(d + out_planes_off());
    int32_t* hull_xy = reinterpret_cast<int32_t*>(d + out_xy_off(m->out_kcap));
    float* hull_xyz = reinterpret_cast<float*>(d + out_xyz_off(m->out_kcap, m->out_hcap));
    HeaderArgs ha{b.ctr, fb.hull_cnt, nullptr, fb.err, m->ctr, m->err, reinterpret_cast<SegCounters*>(d)};
    if (p.planes_per_cluster > 1) {
        e = launch_rounds(b, m->kcap, p, fb, m->rounds, m->tune, sms, b.scan_tmp, planes, m->out_kcap, hull_xy,
                          hull_xyz, m->out_hcap, s, hk);
        if (e != cudaSuccess) return e;
        ha.rounds = m->rounds.word;
        VM_STAGE_BEGIN(hk, kStPack, s);
        launch_k(k_header, dim3(1), dim3(1), 0, s, ha);
        count_launch(1);
    } else {
        if ((e = launch_fit(b.pts, b.cl_off, b.cl_label, &b.ctr->k, m->kcap, p, fb, m->tune, sms, s, hk)) !=
            cudaSuccess)
            return e;
        VM_STAGE_BEGIN(hk, kStPack, s);
        if (m->kcap) {  // the pack kernel writes the header too
            e = launch_pack(fb, b.cl_off, b.cl_label, &b.ctr->k, m->kcap, planes, hull_xy, hull_xyz, m->out_hcap, s,
                            &ha);
            if (e != cudaSuccess) return e;
        } else {
            launch_k(k_header, dim3(1), dim3(1), 0, s, ha);
            count_launch(1);
        }
    }
    VM_STAGE_END(hk, kStPack, s);
    return cudaGetLastError();
}

// Nodes, edges and programmatic edges (a kernel launched with programmatic
// stream serialization keeps that dependency type when captured) of a graph.
static void graph_shape(cudaGraph_t graph, uint32_t& nodes, uint32_t& edges, uint32_t& prog) {
    nodes = edges = prog = 0;
    size_t nn = 0, ne = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess ||
        cudaGraphGetEdges(graph, nullptr, nullptr, nullptr, &ne) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    nodes = (uint32_t)nn;
    edges = (uint32_t)ne;
    if (!ne) return;
    std::vector<cudaGraphNode_t> from(ne), to(ne);
    std::vector<cudaGraphEdgeData> data(ne);
    if (cudaGraphGetEdges(graph, from.data(), to.data(), data.data(), &ne) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    for (size_t i = 0; i < ne; ++i) prog += data[i].type == cudaGraphDependencyTypeProgrammatic;
}

vm_status capture_segment(vm_map* m, const vm_segment_params& p) {
    if (m->gexec) {
        cudaGraphExecDestroy(m->gexec);
        m->gexec = nullptr;
    }
    fit_init_attributes();
    cudaGraph_t graph = nullptr;
    const unsigned long long l0 = launch_total();
    count_capture();
    VM_CUDA(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_segment(m, p, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(m->stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_status(e, "segment capture");
    }
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
    graph_shape(graph, m->gnodes, m->gedges, m->gprog);
    e = cudaGraphInstantiate(&m->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        m->gexec = nullptr;
        return cuda_status(e, "cudaGraphInstantiate");
    }
    m->glaunches = launch_total() - l0;
    uncount_launch(m->glaunches);  // counted when replayed, not when captured
    m->ggen = m->gen;
    m->gprm = p;
    return VM_OK;
}

vm_status check_map(vm_map* m) {
    if (!m) {
        set_error("null map");
        return VM_ERR_INVALID_ARG;
    }
    return VM_OK;
}

vm_status launch_segment(vm_map* m, const vm_segment_params& p) {
    cudaStream_t s = m->stream;
    if (!m->vox_mem.p) {  // first call: size the scratch from the pool's brick count (one read)
        MapCounters c;
        VM_CUDA(cudaMemcpyAsync(&c, m->ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaStreamSynchronize(s));
        m->brick_hint = c.n_bricks < m->capacity ? c.n_bricks : m->capacity;
    }
    VM_TRY(plan_capacity(m, p, true));
    m->seg_rounds = p.planes_per_cluster > 1 ? p.planes_per_cluster : 1;
    StageHook* hk = m->fit.timer.hook();
    if (m->use_graph && !hk && (!m->gexec || m->ggen != m->gen || memcmp(&m->gprm, &p, sizeof(p)) != 0)) {
        if (capture_segment(m, p) != VM_OK) {  // e.g. a stream that cannot be captured: launch eagerly
            cudaGetLastError();
            m->use_graph = false;
        }
    }
    if (m->use_graph && !hk) {
        VM_CUDA(cudaGraphLaunch(m->gexec, s));
        count_launch((int)m->glaunches);
    } else {
        VM_CUDA(enqueue_segment(m, p, hk));
    }
    return VM_OK;
}

static vm_status capture_front(vm_map* m, const vm_segment_params& p) {
    if (m->fexec) {
        cudaGraphExecDestroy(m->fexec);
        m->fexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const unsigned long long l0 = launch_total();
    count_capture();
    VM_CUDA(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_front(m, p, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(m->stream, &graph);
    m->flaunches = launch_total() - l0;
    uncount_launch(m->flaunches);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_status(e, "front capture");
    }
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&m->fexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        m->fexec = nullptr;
        return cuda_status(e, "cudaGraphInstantiate");
    }
    m->fgen = m->gen;
    m->fprm = p;
    return VM_OK;
}

vm_status launch_front(vm_map* m, const vm_segment_params& p) {
    cudaStream_t s = m->stream;
    if (!m->vox_mem.p) {
        MapCounters c;
        VM_CUDA(cudaMemcpyAsync(&c, m->ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaStreamSynchronize(s));
        m->brick_hint = c.n_bricks < m->capacity ? c.n_bricks : m->capacity;
    }
    VM_TRY(plan_capacity(m, p, false));
    if (m->use_graph && (!m->fexec || m->fgen != m->gen || memcmp(&m->fprm, &p, sizeof(p)) != 0)) {
        if (capture_front(m, p) != VM_OK) {
            cudaGetLastError();
            m->use_graph = false;
        }
    }
    if (m->use_graph) {
        VM_CUDA(cudaGraphLaunch(m->fexec, s));
        count_launch((int)m->flaunches);
    } else {
        VM_CUDA(enqueue_front(m, p, nullptr));
    }
    return VM_OK;
}

// True when the completed segmentation in the result block ran out of a
// capacity (scratch or hull output) and must be re-run; updates the hints
// that size the next attempt.
bool take_hints(vm_map* m) {
    const SegCounters* hdr = static_cast<const SegCounters*>(m->out_host);
    m->brick_hint = hdr->n_bricks < m->capacity ? hdr->n_bricks : m->capacity;
    m->k_hint = hdr->k_need > hdr->k ? hdr->k_need : hdr->k;
    m->hull_hint = hdr->n_hull;
    m->rec_hint = hdr->n_planes;
    return (hdr->err & kErrScratch) || hdr->n_hull > m->out_hcap || hdr->n_planes > m->out_kcap;
}

vm_status finish_segment(vm_map* m, const vm_segment_params& p, vm_planes* out) {
    for (int attempt = 0;; ++attempt) {
        VM_CUDA(cudaStreamSynchronize(m->stream));
        m->fit.timer.fold();
        if (!take_hints(m)) break;
        if (attempt == 3) {
            set_error("segmentation scratch could not be sized for this map");
            return VM_ERR_OUT_OF_MEMORY;
        }
        VM_TRY(launch_segment(m, p));
    }
    return read_result(m, out);
}

vm_status read_result(vm_map* m, vm_planes* out) {
    const SegCounters* hdr = static_cast<const SegCounters*>(m->out_host);
    m->last = *hdr;
    m->segmented = true;
    const uint32_t K = hdr->n_planes, n_hull = hdr->n_hull;
    const size_t b_planes = (size_t)K * sizeof(vm_plane);
    out->planes = static_cast<vm_plane*>(malloc(b_planes ? b_planes : 1));
    out->hull_xy = static_cast<int32_t*>(malloc(n_hull ? (size_t)n_hull * 8 : 1));
    out->hull_xyz = static_cast<float*>(malloc(n_hull ? (size_t)n_hull * 12 : 1));
    if (!out->planes || !out->hull_xy || !out->hull_xyz) {
        vm_planes_free(out);
        set_error("host allocation of the result failed");
        return VM_ERR_OUT_OF_MEMORY;
    }
    const char* h = static_cast<const char*>(m->out_host);
    memcpy(out->planes, h + out_planes_off(), b_planes);
    memcpy(out->hull_xy, h + out_xy_off(m->out_kcap), (size_t)n_hull * 8);
    memcpy(out->hull_xyz, h + out_xyz_off(m->out_kcap, m->out_hcap), (size_t)n_hull * 12);
    out->n_planes = K;
    out->n_hull = n_hull;
    if ((hdr->err | hdr->fit_err) & kErrTimeout) {
        set_error("a bounded device loop reached its iteration cap");
        return VM_ERR_TIMEOUT;
    }
    if (hdr->fit_err & kErrOverflow) {
        set_error("a cluster spans more than 2^28 hull quanta (4096 m) in its plane; its hull is not exact");
        return VM_ERR_EXTENT;
    }
    if (hdr->map_err & kErrCapacity) {
        set_error("brick pool full: points in unallocated bricks were dropped");
        return VM_ERR_CAPACITY;
    }
    return VM_OK;
}

}  // namespace vmx

extern "C" {

const char* vm_last_error(void) { return g_err.c_str(); }

const char* vm_version(void) { return "voxmps 0.1 (sm_103a)"; }

vm_status vm_create(const vm_map_params* params, void* cuda_stream, vm_map** out) {
    if (!params || !out) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const vm_map_params& p = *params;
    if (p.dims[0] <= 0 || p.dims[1] <= 0 || p.dims[2] <= 0 || !(p.voxel_size > 0.0f)) {
        set_error("dims and voxel_size must be positive");
        return VM_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        if ((double)p.dims[a] * (double)p.voxel_size > 16.0 + 1e-9) {
            set_error("map extent beyond 16 m on an axis");
            return VM_ERR_INVALID_ARG;
        }
    }
    vm_map* m = new (std::nothrow) vm_map();
    if (!m) {
        set_error("host allocation failed");
        return VM_ERR_OUT_OF_MEMORY;
    }
    m->prm = p;
    m->fit.timer.on = (p.flags & VM_MAP_STAGE_TIMING) != 0;
    m->use_graph = (p.flags & VM_MAP_EAGER) == 0;
    Grid& g = m->g;
    g.nx = p.dims[0]; g.ny = p.dims[1]; g.nz = p.dims[2];
    g.nbx = (g.nx + kBrick - 1) / kBrick;
    g.nby = (g.ny + kBrick - 1) / kBrick;
    g.nbz = (g.nz + kBrick - 1) / kBrick;
    g.ox = p.origin[0]; g.oy = p.origin[1]; g.oz = p.origin[2];
    g.inv_res = (float)(1.0 / (double)p.voxel_size);
    g.wx = g.wy = g.wz = 0;  // the window starts at the base origin (anchor 0)
    g.ax = g.ay = g.az = 0;
    const unsigned long long nb = (unsigned long long)g.nbx * g.nby * g.nbz;
    if (nb * kBrickVox > 0xFFFFFFFFull) {
        delete m;
        set_error("more than 2^32 voxel ids");
        return VM_ERR_EXTENT;
    }
    m->nb_total = (uint32_t)nb;
    m->capacity = p.brick_capacity ? (p.brick_capacity < m->nb_total ? p.brick_capacity : m->nb_total) : m->nb_total;
    cudaError_t e;
    if (cuda_stream) {
        m->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete m;
            return cuda_status(e, "cudaStreamCreate");
        }
        m->own_stream = true;
    }
    // pool: table, slot keys, sums, counts, counters
    Carver dry{nullptr};
    dry.take<int32_t>(m->nb_total);
    dry.take<int32_t>(m->capacity);
    dry.take<unsigned long long>((size_t)m->capacity * 3 * kBrickVox);
    dry.take<uint32_t>((size_t)m->capacity * kBrickVox);
    dry.take<MapCounters>(1);
    dry.take<uint32_t>((size_t)m->capacity * (kBrickVox / 32));
    dry.take<uint32_t>(4);
    dry.take<uint32_t>(scroll_tmp_words(m->capacity));
    dry.take<float>(4);
    vm_status st = ensure(m->pool, dry.off + 256);
    if (st != VM_OK) {
        vm_destroy(m);
        return st;
    }
    Carver c{static_cast<char*>(m->pool.p)};
    m->brick_table = c.take<int32_t>(m->nb_total);
    m->slot_key = c.take<int32_t>(m->capacity);
    m->S = c.take<unsigned long long>((size_t)m->capacity * 3 * kBrickVox);
    m->C = c.take<uint32_t>((size_t)m->capacity * kBrickVox);
    m->ctr = c.take<MapCounters>(1);
    m->mark = c.take<uint32_t>((size_t)m->capacity * (kBrickVox / 32));
    m->err = c.take<uint32_t>(4);
    m->scroll_tmp = c.take<uint32_t>(scroll_tmp_words(m->capacity));
    m->po_dev = c.take<float>(4);
    g.po = m->po_dev;
    // brick-level segmentation arrays
    Carver bd{nullptr};
    bd.take<uint32_t>((size_t)m->nb_total + 1);
    bd.take<int32_t>(m->nb_total);
    bd.take<int32_t>(m->capacity);
    bd.take<int32_t>(m->capacity);
    bd.take<SegCounters>(1);
    st = ensure(m->brick_mem, bd.off + 256);
    if (st != VM_OK) {
        vm_destroy(m);
        return st;
    }
    Carver bc{static_cast<char*>(m->brick_mem.p)};
    m->seg.flags = bc.take<uint32_t>((size_t)m->nb_total + 1);
    m->seg.rank_table = bc.take<int32_t>(m->nb_total);
    m->seg.sorted_slot = bc.take<int32_t>(m->capacity);
    m->seg.sorted_key = bc.take<int32_t>(m->capacity);
    m->seg.ctr = bc.take<SegCounters>(1);
    e = cudaMallocHost(reinterpret_cast<void**>(&m->hctr), sizeof(SegCounters));
    if (e != cudaSuccess) {
        vm_destroy(m);
        return cuda_status(e, "cudaMallocHost");
    }
    st = vm_reset(m);
    if (st == VM_OK) {
        const float po[4] = {g.ox, g.oy, g.oz, 0.0f};
        e = cudaMemsetAsync(m->scroll_tmp, 0, scroll_tmp_words(m->capacity) * sizeof(uint32_t), m->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->po_dev, po, sizeof(po), cudaMemcpyHostToDevice, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = cuda_status(e, "map initialisation");
    }
    if (st != VM_OK) {
        vm_destroy(m);
        return st;
    }
    *out = m;
    return VM_OK;
}

vm_status vm_reset(vm_map* m) {
    VM_TRY(check_map(m));
    VM_CUDA(cudaMemsetAsync(m->brick_table, 0xFF, (size_t)m->nb_total * sizeof(int32_t), m->stream));
    VM_CUDA(cudaMemsetAsync(m->S, 0, (size_t)m->capacity * 3 * kBrickVox * sizeof(unsigned long long), m->stream));
    VM_CUDA(cudaMemsetAsync(m->C, 0, (size_t)m->capacity * kBrickVox * sizeof(uint32_t), m->stream));
    VM_CUDA(cudaMemsetAsync(m->ctr, 0, sizeof(MapCounters), m->stream));
    VM_CUDA(cudaMemsetAsync(m->mark, 0, (size_t)m->capacity * (kBrickVox / 32) * sizeof(uint32_t), m->stream));
    m->segmented = false;
    return VM_OK;
}

// The window's anchor in 2^-20 m units: at or below its corner, so the sums
// of the voxels inside stay small and non-negative.
static long long window_anchor(int w, float inv_res) {
    return (long long)floor((double)w * 1048576.0 / (double)inv_res);
}

vm_status vm_scroll(vm_map* m, const int32_t shift[3]) {
    VM_TRY(check_map(m));
    if (!shift) {
        set_error("null shift");
        return VM_ERR_INVALID_ARG;
    }
    if (!shift[0] && !shift[1] && !shift[2]) return VM_OK;
    Grid g2 = m->g;
    const int w[3] = {m->g.wx, m->g.wy, m->g.wz};
    int w2[3];
    for (int a = 0; a < 3; ++a) {
        const long long t = (long long)w[a] + 8ll * (long long)shift[a];
        if (t < -(1ll << 23) || t > (1ll << 23)) {
            set_error("window offset beyond 2^23 voxels (keys must stay exact in FP32)");
            return VM_ERR_INVALID_ARG;
        }
        w2[a] = (int)t;
    }
    g2.wx = w2[0]; g2.wy = w2[1]; g2.wz = w2[2];
    g2.ax = window_anchor(w2[0], g2.inv_res);
    g2.ay = window_anchor(w2[1], g2.inv_res);
    g2.az = window_anchor(w2[2], g2.inv_res);
    const float po2[3] = {(float)((double)g2.ox + (double)g2.ax / 1048576.0),
                          (float)((double)g2.oy + (double)g2.ay / 1048576.0),
                          (float)((double)g2.oz + (double)g2.az / 1048576.0)};
    VM_CUDA(launch_scroll(m->g, g2, shift, po2, m->brick_table, m->nb_total, m->slot_key, m->S, m->C, m->ctr,
                          m->capacity, m->scroll_tmp, m->stream));
    m->g = g2;
    return VM_OK;
}

vm_status vm_scroll_target(vm_map* m, const float center[3], int32_t shift[3]) {
    VM_TRY(check_map(m));
    if (!center || !shift) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    const float o[3] = {m->g.ox, m->g.oy, m->g.oz};
    const int n[3] = {m->g.nx, m->g.ny, m->g.nz}, w[3] = {m->g.wx, m->g.wy, m->g.wz};
    for (int a = 0; a < 3; ++a) {
        const float f = floorf((center[a] - o[a]) * m->g.inv_res);  // the centre's key, keyed as a point is
        if (!(fabsf(f) < 8388608.0f)) {
            set_error("window centre not finite or beyond 2^23 voxels");
            return VM_ERR_INVALID_ARG;
        }
        long long t = (long long)f - n[a] / 2;
        t = t >= 0 ? t / 8 : -((-t + 7) / 8);  // floor(t / 8): the new offset in bricks
        shift[a] = (int32_t)(t - w[a] / 8);
    }
    return VM_OK;
}

vm_status vm_scroll_to(vm_map* m, const float center[3], int32_t shift[3]) {
    int32_t sh[3];
    VM_TRY(vm_scroll_target(m, center, sh));
    if (shift) memcpy(shift, sh, sizeof(sh));
    return vm_scroll(m, sh);
}

vm_status vm_get_window(vm_map* m, int32_t offset[3], float position_origin[3]) {
    VM_TRY(check_map(m));
    const int w[3] = {m->g.wx, m->g.wy, m->g.wz};
    const long long A[3] = {m->g.ax, m->g.ay, m->g.az};
    const float o[3] = {m->g.ox, m->g.oy, m->g.oz};
    for (int a = 0; a < 3; ++a) {
        if (offset) offset[a] = w[a];
        if (position_origin) position_origin[a] = (float)((double)o[a] + (double)A[a] / 1048576.0);
    }
    return VM_OK;
}

vm_status vm_destroy(vm_map* m) {
    if (!m) return VM_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    release(m->pool);
    release(m->stage);
    release(m->deferred);
    release(m->brick_mem);
    release(m->vox_mem);
    release(m->round_mem);
    fit_release(m->fit);
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    if (m->fexec) cudaGraphExecDestroy(m->fexec);
    if (m->out_host) cudaFreeHost(m->out_host);
    if (m->hctr) cudaFreeHost(m->hctr);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return VM_OK;
}

vm_status vm_integrate(vm_map* m, const float* xyz, uint32_t n, const float pose3x4[12], int xyz_on_device) {
    return vm_integrate_ex(m, xyz, n, pose3x4, xyz_on_device, 0);
}

vm_status vm_integrate_ex(vm_map* m, const float* xyz, uint32_t n, const float pose3x4[12], int xyz_on_device,
                          uint32_t flags) {
    VM_TRY(check_map(m));
    if ((!xyz && n) || !pose3x4) {
        set_error("null points or pose");
        return VM_ERR_INVALID_ARG;
    }
    if (n == 0) return VM_OK;
    const float* d = xyz;
    if (!xyz_on_device) {
        VM_TRY(ensure(m->stage, (size_t)n * 3 * sizeof(float)));
        VM_CUDA(cudaMemcpyAsync(m->stage.p, xyz, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, m->stream));
        d = static_cast<const float*>(m->stage.p);
    }
    Pose P;
    memcpy(P.r, pose3x4, sizeof(P.r));
    StageHook* hk = m->fit.timer.hook();
    if (flags & VM_INTEGRATE_CLEAR) {
        VM_STAGE_BEGIN(hk, kStClear, m->stream);
        VM_CUDA(launch_clear(d, n, P, m->g, m->brick_table, m->S, m->C, m->mark, m->ctr, m->capacity, m->stream));
        VM_STAGE_END(hk, kStClear, m->stream);
    }
    VM_TRY(ensure(m->deferred, (size_t)n * sizeof(uint32_t)));
    VM_STAGE_BEGIN(hk, kStIntegrate, m->stream);
    VM_CUDA(launch_integrate(d, n, P, m->g, m->brick_table, m->slot_key, m->S, m->C,
                             static_cast<uint32_t*>(m->deferred.p), m->ctr, m->capacity, m->stream));
    VM_STAGE_END(hk, kStIntegrate, m->stream);
    return VM_OK;
}

vm_status vm_segment(vm_map* m, const vm_segment_params* params, vm_planes* out) {
    VM_TRY(check_map(m));
    VM_TRY(check_params(params));
    if (!out) {
        set_error("null output");
        return VM_ERR_INVALID_ARG;
    }
    memset(out, 0, sizeof(*out));
    VM_TRY(launch_segment(m, *params));
    return finish_segment(m, *params, out);
}

static bool tuning_ok(const vm_fit_tuning* t) {
    const bool r_ok = t->hyp_per_thread == 1 || t->hyp_per_thread == 2 || t->hyp_per_thread == 4 ||
                      t->hyp_per_thread == 8;
    return t->tile >= 256 && t->tile <= 16384 && t->tile % 256 == 0 && r_ok && t->ctas_per_sm >= 1 &&
           t->ctas_per_sm <= 16 && t->schedule <= 1;
}

vm_status vm_set_fit_tuning(vm_map* m, const vm_fit_tuning* t) {
    VM_TRY(check_map(m));
    if (t && !tuning_ok(t)) {
        set_error("tuning out of range (tile a multiple of 256 in 256..16384, hyp_per_thread 1/2/4/8, "
                  "ctas_per_sm 1..16, schedule 0/1)");
        return VM_ERR_INVALID_ARG;
    }
    m->tune = t ? FitTuning{(int)t->tile, (int)t->hyp_per_thread, (int)t->ctas_per_sm, (int)t->schedule}
                : default_tuning();
    m->gen++;  // the captured graph holds the old schedule
    return VM_OK;
}

vm_status vm_get_fit_tuning(vm_map* m, vm_fit_tuning* t) {
    VM_TRY(check_map(m));
    if (!t) {
        set_error("null output");
        return VM_ERR_INVALID_ARG;
    }
    t->tile = (uint32_t)m->tune.tile;
    t->hyp_per_thread = (uint32_t)m->tune.hyp_per_thread;
    t->ctas_per_sm = (uint32_t)m->tune.ctas_per_sm;
    t->schedule = (uint32_t)m->tune.schedule;
    return VM_OK;
}

vm_status vm_autotune_segment(vm_map* m, const vm_segment_params* params, uint32_t reps, vm_fit_tuning* best,
                              float* best_ms, uint32_t* n_tried) {
    VM_TRY(check_map(m));
    VM_TRY(check_params(params));
    if (reps < 1) reps = 1;
    const vm_segment_params& p = *params;
    const int H = (int)p.n_hyp;
    std::vector<FitTuning> cand;
    const int tiles_cta[] = {512, 1024, 2048, 4096};
    const int tiles_warp[] = {256, 512, 1024};
    const int rs[] = {2, 4, 8};
    const int ctas[] = {2, 3, 4, 6, 8};
    for (int sched = 0; sched < 2; ++sched) {
        const int* tiles = sched ? tiles_warp : tiles_cta;
        const int nt = sched ? 3 : 4;
        for (int ti = 0; ti < nt; ++ti)
            for (int r : rs) {
                if ((sched == 1 && (H + r - 1) / r > 32) || (sched == 0 && (H + r - 1) / r > 256)) continue;
                const FitTuning base{tiles[ti], r, 1, sched};
                const int occ = score_max_ctas_per_sm(base, H);
                for (int c : ctas) {
                    if (c > occ) break;
                    FitTuning t = base;
                    t.ctas_per_sm = c;
                    cand.push_back(t);
                }
            }
    }
    const FitTuning keep = m->tune;
    const bool timing = m->fit.timer.on;
    m->fit.timer.on = false;  // time graph replays
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    VM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        m->fit.timer.on = timing;
        return cuda_status(cudaErrorUnknown, "cudaEventCreate");
    }
    vm_status st = VM_OK;
    float best_t = -1.0f;
    FitTuning best_c = keep;
    uint32_t tried = 0;
    for (size_t i = 0; st == VM_OK && i < cand.size(); ++i) {
        m->tune = cand[i];
        m->gen++;
        st = launch_segment(m, p);  // warm-up: sizes and captures
        vm_planes tmp{};
        if (st == VM_OK) st = finish_segment(m, p, &tmp);
        vm_planes_free(&tmp);
        if (st != VM_OK) break;
        cudaEventRecord(e0, m->stream);
        for (uint32_t r = 0; r < reps && st == VM_OK; ++r) st = launch_segment(m, p);
        cudaEventRecord(e1, m->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_status(cudaGetLastError(), "autotune timing");
        if (st != VM_OK) break;
        if (take_hints(m)) continue;  // ran out of a capacity: not a valid timing
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
    m->fit.timer.on = timing;
    m->tune = st == VM_OK ? best_c : keep;
    m->gen++;
    if (st != VM_OK) return st;
    {  // leave the map ready: scratch sized and the graph captured for the chosen schedule
        vm_planes tmp{};
        st = launch_segment(m, p);
        if (st == VM_OK) st = finish_segment(m, p, &tmp);
        vm_planes_free(&tmp);
        if (st != VM_OK) return st;
    }
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

vm_status vm_planes_free(vm_planes* p) {
    if (!p) return VM_OK;
    free(p->planes);
    free(p->hull_xy);
    free(p->hull_xyz);
    memset(p, 0, sizeof(*p));
    return VM_OK;
}

vm_status vm_get_stats(vm_map* m, vm_stats* out) {
    VM_TRY(check_map(m));
    if (!out) {
        set_error("null output");
        return VM_ERR_INVALID_ARG;
    }
    MapCounters c;
    VM_CUDA(cudaMemcpyAsync(&c, m->ctr, sizeof(c), cudaMemcpyDeviceToHost, m->stream));
    VM_CUDA(cudaStreamSynchronize(m->stream));
    memset(out, 0, sizeof(*out));
    out->points_integrated = c.integrated;
    out->points_dropped = c.dropped;
    out->points_no_capacity = c.no_capacity;
    out->bricks_allocated = c.n_bricks < m->capacity ? c.n_bricks : m->capacity;
    out->brick_capacity = m->capacity;
    out->occupied_voxels = m->last.n_occ;
    out->steppable_voxels = m->last.n_vert;
    out->clusters = m->last.k;
    out->clustered_points = m->last.n_kept;
    out->voxels_cleared = c.cleared;
    out->voxels_evicted = c.evicted;
    out->device_bytes = m->pool.bytes + m->stage.bytes + m->brick_mem.bytes + m->vox_mem.bytes + m->fit.mem.bytes +
                        m->fit.out.bytes;
    (void)0;
    if (c.err & kErrCapacity) {
        set_error("brick pool full");
        return VM_ERR_CAPACITY;
    }
    return VM_OK;
}

vm_status vm_export_voxels(vm_map* m, uint32_t* vid, int64_t* sums, uint32_t* counts, uint32_t cap, uint32_t* n) {
    VM_TRY(check_map(m));
    if (!n) {
        set_error("null count output");
        return VM_ERR_INVALID_ARG;
    }
    cudaStream_t s = m->stream;
    if (!m->vox_mem.p) VM_TRY(alloc_vox(m, 1));  // scan scratch
    VM_CUDA(seg_order_bricks(m->brick_table, m->nb_total, m->seg, device_sms(), s));
    VM_CUDA(cudaMemcpyAsync(m->hctr, m->seg.ctr, sizeof(SegCounters), cudaMemcpyDeviceToHost, s));
    VM_CUDA(cudaStreamSynchronize(s));
    const uint32_t nb = m->hctr->n_sorted;
    std::vector<int32_t> slot(nb), key(nb);
    std::vector<unsigned long long> S((size_t)m->capacity * 3 * kBrickVox);
    std::vector<uint32_t> C((size_t)m->capacity * kBrickVox);
    if (nb) {
        VM_CUDA(cudaMemcpyAsync(slot.data(), m->seg.sorted_slot, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaMemcpyAsync(key.data(), m->seg.sorted_key, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaMemcpyAsync(S.data(), m->S, S.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaMemcpyAsync(C.data(), m->C, C.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    VM_CUDA(cudaStreamSynchronize(s));
    uint32_t k = 0;
    for (uint32_t r = 0; r < nb; ++r) {
        for (int l = 0; l < kBrickVox; ++l) {
            const size_t sv = (size_t)slot[r] * kBrickVox + l;
            if (!C[sv]) continue;
            if (k < cap) {
                if (vid) vid[k] = (uint32_t)key[r] * kBrickVox + l;
                if (counts) counts[k] = C[sv];
                if (sums)
                    for (int a = 0; a < 3; ++a)
                        sums[3 * (size_t)k + a] = (int64_t)S[((size_t)slot[r] * 3 + a) * kBrickVox + l];
            }
            ++k;
        }
    }
    *n = k;
    return VM_OK;
}

vm_status vm_export_labels(vm_map* m, uint32_t* vid, float* normal, uint8_t* status, uint32_t* label, uint32_t* nbr,
                           uint32_t cap, uint32_t* n) {
    VM_TRY(check_map(m));
    if (!n) {
        set_error("null count output");
        return VM_ERR_INVALID_ARG;
    }
    *n = 0;
    if (!m->segmented) return VM_OK;
    cudaStream_t s = m->stream;
    const uint32_t nb = m->last.n_sorted;
    const size_t nv = (size_t)nb * kBrickVox;
    std::vector<int32_t> key(nb);
    std::vector<uint8_t> st(nv), nb8(nv);
    std::vector<float> nrm(3 * nv);
    std::vector<uint32_t> par(nv);
    if (nb) {
        VM_CUDA(cudaMemcpyAsync(key.data(), m->seg.sorted_key, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaMemcpyAsync(st.data(), m->seg.status, nv, cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaMemcpyAsync(nb8.data(), m->seg.nbr, nv, cudaMemcpyDeviceToHost, s));
        VM_CUDA(cudaMemcpyAsync(par.data(), m->seg.parent, nv * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        for (int a = 0; a < 3; ++a)
            VM_CUDA(cudaMemcpyAsync(nrm.data() + a * nv, m->seg.nrm + a * m->seg.nv, nv * sizeof(float),
                                    cudaMemcpyDeviceToHost, s));
    }
    VM_CUDA(cudaStreamSynchronize(s));
    uint32_t k = 0;
    for (size_t i = 0; i < nv; ++i) {
        if (!st[i]) continue;
        if (k < cap) {
            const uint32_t v = (uint32_t)key[i / kBrickVox] * kBrickVox + (uint32_t)(i % kBrickVox);
            if (vid) vid[k] = v;
            if (normal)
                for (int a = 0; a < 3; ++a) normal[3 * (size_t)k + a] = nrm[a * nv + i];
            if (status) status[k] = st[i];
            if (nbr) nbr[k] = nb8[i];
            if (label) {
                const uint32_t p = par[i];
                label[k] = (p == kNone) ? kNone : (uint32_t)key[p / kBrickVox] * kBrickVox + p % kBrickVox;
            }
        }
        ++k;
    }
    *n = k;
    return VM_OK;
}

vm_status vm_export_clusters(vm_map* m, float* pts, uint32_t* vid, uint8_t* inlier, uint32_t cap, uint32_t* n) {
    VM_TRY(check_map(m));
    if (!n) {
        set_error("null count output");
        return VM_ERR_INVALID_ARG;
    }
    *n = 0;
    if (!m->segmented) return VM_OK;
    const uint32_t np = m->last.n_kept;
    const uint32_t w = np < cap ? np : cap;
    cudaStream_t s = m->stream;
    if (w) {
        if (pts) VM_CUDA(cudaMemcpyAsync(pts, m->seg.pts, (size_t)w * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (vid) VM_CUDA(cudaMemcpyAsync(vid, m->seg.pt_vid, (size_t)w * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        if (inlier && m->last.k)  // the first round's inliers (the paper's plane) when there were several
            VM_CUDA(cudaMemcpyAsync(inlier, m->seg_rounds > 1 ? m->rounds.inl0 : m->fit.fb.inlier, (size_t)w,
                                    cudaMemcpyDeviceToHost, s));
    }
    VM_CUDA(cudaStreamSynchronize(s));
    *n = np;
    return VM_OK;
}

static thread_local FitContext tl_fit;

vm_status vm_stage_timing(vm_map* map, int enable) {
    FitContext& fc = map ? map->fit : tl_fit;
    fc.timer.fold();
    fc.timer.on = enable != 0;
    return VM_OK;
}

vm_status vm_stage_times(vm_map* map, double* ms, uint64_t* calls, uint32_t cap, uint32_t* n_stages) {
    FitContext& fc = map ? map->fit : tl_fit;
    if (map && map->stream) VM_CUDA(cudaStreamSynchronize(map->stream));
    fc.timer.fold();
    for (uint32_t i = 0; i < (uint32_t)kNumStages && i < cap; ++i) {
        if (ms) ms[i] = fc.timer.ms[i];
        if (calls) calls[i] = fc.timer.calls[i];
        fc.timer.ms[i] = 0.0;
        fc.timer.calls[i] = 0;
    }
    if (n_stages) *n_stages = kNumStages;
    return VM_OK;
}

const char* vm_stage_name(uint32_t stage) { return stage < (uint32_t)kNumStages ? kStageNames[stage] : ""; }

uint64_t vm_launch_count(void) { return g_launches.load(); }

vm_status vm_graph_shape(vm_map* m, uint32_t* nodes, uint32_t* edges, uint32_t* programmatic) {
    VM_TRY(check_map(m));
    if (nodes) *nodes = m->gexec ? m->gnodes : 0;
    if (edges) *edges = m->gexec ? m->gedges : 0;
    if (programmatic) *programmatic = m->gexec ? m->gprog : 0;
    return VM_OK;
}
uint64_t vm_capture_count(void) { return capture_total(); }
uint64_t vm_allocation_count(void) { return alloc_total(); }

vm_status vm_fit_planes(const float* xyz, const uint32_t* off, const uint32_t* labels, uint32_t k,
                        const vm_segment_params* params, void* stream, vm_planes* out) {
    VM_TRY(check_single_round(params));
    if (!out || (k && (!xyz || !off))) {
        set_error("null argument");
        return VM_ERR_INVALID_ARG;
    }
    memset(out, 0, sizeof(*out));
    if (k == 0) return VM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t npts = 0;
    VM_CUDA(cudaMemcpyAsync(&npts, off + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VM_CUDA(cudaStreamSynchronize(s));
    return fit_and_pack(tl_fit, xyz, off, labels, k, npts, *params, default_tuning(), s, out);
}

}  // extern "C"
