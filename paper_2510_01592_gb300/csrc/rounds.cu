// rounds.cu -- sequential multi-plane extraction per cluster.
//
// The paper (Sec. III.C) fits one plane per cluster.  With planes_per_cluster
// P > 1 a cluster that holds more than one surface (a ramp joined to the floor
// under Algorithm 1's 15 deg normal test, a step whose riser is too short to
// split it) gives up further planes: round r + 1 fits, with the Philox counter
// (label, h, r + 1, 0), the points of round r that are not its inliers, in
// their order, when round r found a plane with at least min_cluster inliers
// and at least min_cluster points remain.  Round 0 is the paper's fit and is
// always output; a later round is output when it finds a plane.
//
// Every round is the same fixed launch sequence (launch_fit on the remaining
// points, whose cluster count is read on the device), so the whole loop is
// captured in the segmentation's CUDA graph.  Between rounds:
//   stage   records of round r into slot[orig][r], hull vertices into a
//           staging array at the round's base (the round's own hull offsets);
//   active  which clusters go on (flags, scanned into new cluster indices);
//   keep    which points go on (flags, scanned into new point positions: the
//           clusters are contiguous and in order, so one scan over all points
//           gives every remaining cluster its new offset);
//   scatter points, offsets, labels and round-0 indices of the next round.
// At the end, records are counted per round-0 cluster and scanned, and every
// record is written at (first record of its cluster) + round, with its hull
// vertices at offsets from a second scan: the output order is (label, round).
#include "vm_internal.cuh"

namespace vmx {
namespace {

constexpr int kRT = 256;

__global__ void __launch_bounds__(kRT) k_round_stage(const uint32_t* __restrict__ kp, const uint32_t* __restrict__ off,
                                                     const uint32_t* __restrict__ lab,
                                                     const uint32_t* __restrict__ orig,
                                                     const FitCluster* __restrict__ cl, const int2* __restrict__ hull,
                                                     const uint32_t* __restrict__ hull_off, uint32_t r,
                                                     uint32_t* __restrict__ hbase, vm_plane* __restrict__ slot,
                                                     uint32_t* __restrict__ cnt, int2* __restrict__ shull,
                                                     uint32_t hcap) {
    pdl_gate();
    const uint32_t k = *kp;
    const uint32_t base = r ? hbase[r] : 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) hbase[r + 1] = base + hull_off[k];
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) {
        const FitCluster& f = cl[c];
        if (r > 0 && f.best_h < 0) continue;  // a later round is output only when it finds a plane
        const uint32_t o = orig ? orig[c] : c;
        const uint32_t ho = hull_off[c], hn = hull_off[c + 1] - ho;
        if (threadIdx.x == 0) {
            vm_plane p = make_plane(f, lab[c], off[c + 1] - off[c], base + ho, hn);
            p.flags |= r << 8;
            slot[(size_t)o * kMaxRounds + r] = p;
            cnt[o] = r + 1;
        }
        const int2* src = hull + off[c];
        for (uint32_t i = threadIdx.x; i < hn; i += kRT)
            if (base + ho + i < hcap) shull[base + ho + i] = src[i];
    }
}

// act[c] = 1 when cluster c of this round goes on; *npts = the round's points.
__global__ void k_round_active(const uint32_t* __restrict__ kp, const uint32_t* __restrict__ off,
                               const FitCluster* __restrict__ cl, uint32_t minc, uint32_t* __restrict__ act,
                               uint32_t* __restrict__ npts) {
    pdl_gate();
    const uint32_t k = *kp;
    const uint32_t tid = blockIdx.x * kRT + threadIdx.x;
    if (tid == 0) *npts = off[k];
    for (uint32_t c = tid; c < k; c += gridDim.x * kRT) {
        const uint32_t n = off[c + 1] - off[c];
        const FitCluster& f = cl[c];
        const uint32_t ni = f.best_h >= 0 ? f.inliers : 0u;
        const uint32_t rest = n > ni ? n - ni : 0u;
        act[c] = (f.best_h >= 0 && ni >= minc && rest >= minc && rest > 0) ? 1u : 0u;
    }
}

// keep[i] = 1 for the points of active clusters that are not inliers; inl0
// (round 0 only, else null) keeps the round's inlier flags for export.  One
// thread per point; its cluster by binary search over the offsets (a few
// cached steps), so a large cluster does not serialise on one CTA.
__global__ void __launch_bounds__(kRT) k_round_keep(const uint32_t* __restrict__ kp, const uint32_t* __restrict__ off,
                                                    const uint32_t* __restrict__ act, const uint8_t* __restrict__ inl,
                                                    const uint32_t* __restrict__ npts, uint32_t* __restrict__ keep,
                                                    uint8_t* __restrict__ inl0) {
    pdl_gate();
    const uint32_t k = *kp, n = *npts;
    for (uint32_t i = blockIdx.x * kRT + threadIdx.x; i < n; i += gridDim.x * kRT) {
        uint32_t lo = 0, hi = k;  // the cluster c with off[c] <= i < off[c + 1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid;
        }
        const uint8_t v = inl[i];
        keep[i] = (act[lo] && !v) ? 1u : 0u;
        if (inl0) inl0[i] = v;
    }
}

__global__ void k_round_scatter(const uint32_t* __restrict__ kp, const uint32_t* __restrict__ off,
                                const uint32_t* __restrict__ lab, const uint32_t* __restrict__ orig,
                                const uint32_t* __restrict__ act, const uint32_t* __restrict__ apos,
                                const uint32_t* __restrict__ keep, const uint32_t* __restrict__ kpos,
                                const float* __restrict__ pts, const uint32_t* __restrict__ npts,
                                const uint32_t* __restrict__ knext, const uint32_t* __restrict__ keep_tot,
                                float* __restrict__ pts_n, uint32_t* __restrict__ off_n, uint32_t* __restrict__ lab_n,
                                uint32_t* __restrict__ orig_n) {
    pdl_gate();
    const uint32_t k = *kp, n = *npts;
    const uint32_t tid = blockIdx.x * kRT + threadIdx.x, stride = gridDim.x * kRT;
    for (uint32_t i = tid; i < n; i += stride) {
        if (!keep[i]) continue;
        const uint32_t j = kpos[i];
        pts_n[3 * (size_t)j] = pts[3 * (size_t)i];
        pts_n[3 * (size_t)j + 1] = pts[3 * (size_t)i + 1];
        pts_n[3 * (size_t)j + 2] = pts[3 * (size_t)i + 2];
    }
    for (uint32_t c = tid; c < k; c += stride) {
        if (!act[c]) continue;
        const uint32_t j = apos[c];
        off_n[j] = kpos[off[c]];
        lab_n[j] = lab[c];
        orig_n[j] = orig ? orig[c] : c;
    }
    if (tid == 0) off_n[*knext] = *keep_tot;
}

// Hull vertices per round-0 cluster, over its records.
__global__ void k_round_totals(const uint32_t* __restrict__ kp, const uint32_t* __restrict__ cnt,
                               const vm_plane* __restrict__ slot, uint32_t* __restrict__ hcnt) {
    pdl_gate();
    const uint32_t k = *kp;
    for (uint32_t c = blockIdx.x * kRT + threadIdx.x; c < k; c += gridDim.x * kRT) {
        uint32_t h = 0;
        for (uint32_t q = 0; q < cnt[c]; ++q) h += slot[(size_t)c * kMaxRounds + q].hull_count;
        hcnt[c] = h;
    }
}

// The records of round-0 cluster c at cpos[c] + round, their hull vertices
// from hpos[c] on, in round order.
__global__ void __launch_bounds__(kRT) k_round_pack(const uint32_t* __restrict__ kp, const uint32_t* __restrict__ cnt,
                                                    const uint32_t* __restrict__ cpos,
                                                    const uint32_t* __restrict__ hpos,
                                                    const vm_plane* __restrict__ slot, const int2* __restrict__ shull,
                                                    uint32_t hcap, vm_plane* __restrict__ planes, uint32_t rec_cap,
                                                    int32_t* __restrict__ hull_xy, float* __restrict__ hull_xyz,
                                                    uint32_t hull_cap) {
    pdl_gate();
    const uint32_t k = *kp;
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) {
        uint32_t ho = hpos[c];
        const uint32_t nq = cnt[c];
        for (uint32_t q = 0; q < nq; ++q) {
            vm_plane p = slot[(size_t)c * kMaxRounds + q];
            const uint32_t src = p.hull_offset, hn = p.hull_count;
            p.hull_offset = ho;
            const uint32_t at = cpos[c] + q;
            if (threadIdx.x == 0 && at < rec_cap) planes[at] = p;
            for (uint32_t i = threadIdx.x; i < hn; i += kRT)
                if (ho + i < hull_cap && src + i < hcap) write_vertex(p, shull[src + i], ho + i, hull_xy, hull_xyz);
            ho += hn;
        }
    }
}

inline unsigned clampg(size_t want, int sms, int per_sm) {
    const size_t cap = (size_t)sms * per_sm;
    if (want == 0) want = 1;
    return (unsigned)(want < cap ? want : cap);
}

}  // namespace

size_t rounds_bytes(size_t nv, size_t kcap, size_t hcap) {
    RoundBuffers rb{};
    rounds_layout(nullptr, rb, nv, kcap, hcap);
    return reinterpret_cast<size_t>(rb.hull) + hcap * sizeof(int2) + 256;
}

void rounds_layout(char* base, RoundBuffers& rb, size_t nv, size_t kcap, size_t hcap) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        char* p = base + off;
        off += bytes;
        return p;
    };
    for (int i = 0; i < 2; ++i) {
        rb.pts[i] = reinterpret_cast<float*>(take(nv * 3 * sizeof(float)));
        rb.off[i] = reinterpret_cast<uint32_t*>(take((kcap + 1) * sizeof(uint32_t)));
        rb.lab[i] = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
        rb.orig[i] = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    }
    rb.keep = reinterpret_cast<uint32_t*>(take(nv * sizeof(uint32_t)));
    rb.kpos = reinterpret_cast<uint32_t*>(take(nv * sizeof(uint32_t)));
    rb.act = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    rb.apos = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    rb.cnt = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    rb.cpos = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    rb.hcnt = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    rb.hpos = reinterpret_cast<uint32_t*>(take(kcap * sizeof(uint32_t)));
    rb.word = reinterpret_cast<uint32_t*>(take(64 * sizeof(uint32_t)));
    rb.inl0 = reinterpret_cast<uint8_t*>(take(nv));
    rb.slot = reinterpret_cast<vm_plane*>(take(kcap * kMaxRounds * sizeof(vm_plane)));
    rb.hull = reinterpret_cast<int2*>(take(0));
    rb.nv = nv;
    rb.kcap = kcap;
    rb.hcap = hcap;
}

cudaError_t launch_rounds(const SegBuffers& b, uint32_t kcap, const vm_segment_params& p, FitBuffers& fb,
                          RoundBuffers& rb, const FitTuning& t, int sms, uint32_t* scan_tmp, vm_plane* planes,
                          uint32_t rec_cap, int32_t* hull_xy, float* hull_xyz, uint32_t hull_cap, cudaStream_t s,
                          StageHook* hk) {
    const uint32_t P = p.planes_per_cluster < kMaxRounds ? (p.planes_per_cluster > 1 ? p.planes_per_cluster : 1)
                                                         : kMaxRounds;
    const uint32_t minc = p.min_cluster;
    const size_t nv = rb.nv;
    const uint32_t* k0 = &b.ctr->k;
    const unsigned gk = clampg((kcap + kRT - 1) / kRT, sms, 8);   // thread per cluster
    const unsigned gc = clampg(kcap, sms, 16);                     // CTA per cluster
    const unsigned gp = clampg((nv + kRT - 1) / kRT, sms, 16);     // thread per point
    cudaError_t e;
    const float* pts = b.pts;
    const uint32_t *off = b.cl_off, *lab = b.cl_label, *orig = nullptr, *kp = k0;
    for (uint32_t r = 0; r < P; ++r) {
        if ((e = launch_fit(pts, off, lab, kp, kcap, p, fb, t, sms, s, hk, r)) != cudaSuccess) return e;
        VM_STAGE_BEGIN(hk, kStRounds, s);
        launch_k(k_round_stage, dim3(gc), dim3(kRT), 0, s, kp, off, lab, orig, fb.cl, fb.hull, fb.hull_cnt, r,
                 rb.word + kWordHull, rb.slot, rb.cnt, rb.hull, (uint32_t)rb.hcap);
        count_launch(1);
        if (r + 1 < P) {
            const int nx = (r + 1) & 1;
            uint32_t* knext = rb.word + kWordK + r + 1;
            launch_k(k_round_active, dim3(gk), dim3(kRT), 0, s, kp, off, fb.cl, minc, rb.act, rb.word + kWordNpts);
            e = exclusive_scan_dev(rb.act, rb.apos, knext, kp, kcap, scan_tmp, s, fb.err);
            if (e != cudaSuccess) return e;
            launch_k(k_round_keep, dim3(gp), dim3(kRT), 0, s, kp, off, rb.act, fb.inlier, rb.word + kWordNpts, rb.keep,
                     r == 0 ? rb.inl0 : nullptr);
            e = exclusive_scan_dev(rb.keep, rb.kpos, rb.word + kWordKeep, rb.word + kWordNpts, nv, scan_tmp, s,
                                   fb.err);
            if (e != cudaSuccess) return e;
            launch_k(k_round_scatter, dim3(gp), dim3(kRT), 0, s, kp, off, lab, orig, rb.act, rb.apos, rb.keep, rb.kpos,
                     pts, rb.word + kWordNpts, knext, rb.word + kWordKeep, rb.pts[nx], rb.off[nx], rb.lab[nx],
                     rb.orig[nx]);
            count_launch(3);
            pts = rb.pts[nx];
            off = rb.off[nx];
            lab = rb.lab[nx];
            orig = rb.orig[nx];
            kp = knext;
        }
        VM_STAGE_END(hk, kStRounds, s);
    }
    VM_STAGE_BEGIN(hk, kStPack, s);
    launch_k(k_round_totals, dim3(gk), dim3(kRT), 0, s, k0, rb.cnt, rb.slot, rb.hcnt);
    count_launch(1);
    if ((e = exclusive_scan_dev(rb.cnt, rb.cpos, rb.word + kWordRec, k0, kcap, scan_tmp, s, fb.err)) != cudaSuccess)
        return e;
    if ((e = exclusive_scan_dev(rb.hcnt, rb.hpos, rb.word + kWordHullTot, k0, kcap, scan_tmp, s, fb.err)) !=
        cudaSuccess)
        return e;
    launch_k(k_round_pack, dim3(clampg(kcap, sms, 8)), dim3(kRT), 0, s, k0, rb.cnt, rb.cpos, rb.hpos, rb.slot, rb.hull,
                                                      (uint32_t)rb.hcap, planes, rec_cap, hull_xy, hull_xyz, hull_cap);
    count_launch(1);
    VM_STAGE_END(hk, kStPack, s);
    return cudaGetLastError();
}

}  // namespace vmx
