// fit.cu -- cluster-parallel plane estimation (Sec. III.C, multi-plane
// estimation stages a-c), inlier refit and boundary polygons (Sec. III.C,
// boundary polygon generation), for all clusters of a batch at once.
//
//  k_hyp     stage a: one thread per (cluster, hypothesis): three sample
//            indices from Philox4x64-10, plane through the samples.
//  k_score   stage b: a persistent kernel; CTAs pull (cluster, point tile)
//            work items from an atomic queue, stage the tile in shared memory
//            and test every point against every hypothesis held in registers;
//            integer counts are summed in shared memory and added to global
//            memory with integer atomics (order-free, hence exact).
//  k_select  stage c: max count, lowest hypothesis index on ties; in-plane
//            basis and hull origin.
//  k_extract inliers of the selected plane, centroid partial sums and the
//            extreme inliers along 16 integer directions (exact integer keys).
//  k_filter  covariance partial sums; points strictly inside the 16-gon of
//            extreme points cannot be hull vertices and are dropped (the GPU
//            filtering step of the cited convex-hull method), the rest are
//            appended.
//  k_refit   per cluster: TLS refit from the partial sums (double-float sums,
//            adjugate power iteration).
//  k_hull    per cluster: a second, 128-direction filter, then a bitonic sort
//            of the remaining quantised points in shared memory and Andrew's
//            monotone chain with exact int64 orientation tests; gift wrapping
//            over global memory when too many remain for shared memory.
#include <climits>
#include <mutex>
#include <string>

#include "vm_internal.cuh"

namespace vmx {
namespace {

constexpr int kT = 256;
constexpr int kHullCap = 2048;   // hull candidates sorted in shared memory
constexpr int kSurvCap = 12288;  // first-filter survivors staged in shared memory
constexpr size_t kFusedFitPoints = size_t(4) << 20;  // fits of at most this many points: per-cluster tails fused

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ void philox4x64_10(const unsigned long long ctr[4], const unsigned long long key[2],
                                              unsigned long long out[4]) {
    unsigned long long x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    unsigned long long k0 = key[0], k1 = key[1];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        const unsigned long long m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
        const unsigned long long hi0 = __umul64hi(m0, x0), lo0 = m0 * x0;
        const unsigned long long hi1 = __umul64hi(m1, x2), lo1 = m1 * x2;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

__device__ __forceinline__ float plane_dist(float nx, float ny, float nz, float d, float px, float py, float pz) {
    return fabsf(__fmaf_rn(nz, pz, __fmaf_rn(ny, py, __fmaf_rn(nx, px, d))));
}

// Stage b for one point against a thread's R hypotheses: acc[r] += 1 when
// |n_r . p + d_r| <= eps (the fma chain of plane_dist).  The comparison is a
// set to all-ones / zero subtracted from the count: two instructions a test
// after the three fused multiply-adds.
template <int R>
__device__ __forceinline__ void count_point(const float4 (&pl)[R], float4 p, float eps, uint32_t (&acc)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float dist = plane_dist(pl[r].x, pl[r].y, pl[r].z, pl[r].w, p.x, p.y, p.z);
        uint32_t t;
        asm("set.le.u32.f32 %0, %1, %2;" : "=r"(t) : "f"(dist), "f"(eps));
        acc[r] -= t;
    }
}

// The cluster of work item it: one load from the item -> cluster table k_hyp
// writes (item_cl), else a binary search over the item offsets.
__device__ __forceinline__ uint32_t find_cluster(const uint32_t* __restrict__ item_cl,
                                                 const uint32_t* __restrict__ item_off, uint32_t k, uint32_t it) {
    if (item_cl) return item_cl[it];
    uint32_t lo = 0, hi = k;  // largest c with item_off[c] <= it
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- stage a
// Also writes the item -> cluster table (item_cl, when not null): the thread
// of hypothesis 0 of each cluster fills its cluster's items.
__global__ void k_hyp(const float* __restrict__ pts, const uint32_t* __restrict__ off,
                      const uint32_t* __restrict__ labels, const uint32_t* __restrict__ kp, int H,
                      unsigned long long seed, uint32_t round, float4* __restrict__ hyp, uint8_t* __restrict__ valid,
                      uint32_t* __restrict__ counts, const uint32_t* __restrict__ item_off,
                      uint32_t* __restrict__ item_cl) {
    pdl_gate();
    const uint32_t k = *kp;
    const size_t total = (size_t)k * H;
    for (size_t t = (size_t)blockIdx.x * kT + threadIdx.x; t < total; t += (size_t)gridDim.x * kT) {
        const uint32_t c = (uint32_t)(t / H), h = (uint32_t)(t % H);
        if (h == 0 && item_cl)
            for (uint32_t it = item_off[c], e = item_off[c + 1]; it < e; ++it) item_cl[it] = c;
        const uint32_t base = off[c], n = off[c + 1] - base;
        const uint32_t label = labels ? labels[c] : c;
        const unsigned long long ctr[4] = {label, h, round, 0ull}, key[2] = {seed, 0ull};
        unsigned long long r[4];
        philox4x64_10(ctr, key, r);
        const uint32_t i0 = (uint32_t)__umul64hi(r[0], n), i1 = (uint32_t)__umul64hi(r[1], n),
                       i2 = (uint32_t)__umul64hi(r[2], n);
        counts[t] = 0;
        uint8_t ok = (i0 != i1) && (i0 != i2) && (i1 != i2);
        float4 pl = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0x7f800000));  // never an inlier
        if (ok) {
            const float* p0 = pts + 3 * ((size_t)base + i0);
            const float* p1 = pts + 3 * ((size_t)base + i1);
            const float* p2 = pts + 3 * ((size_t)base + i2);
            const float e1x = __fsub_rn(p1[0], p0[0]), e1y = __fsub_rn(p1[1], p0[1]), e1z = __fsub_rn(p1[2], p0[2]);
            const float e2x = __fsub_rn(p2[0], p0[0]), e2y = __fsub_rn(p2[1], p0[1]), e2z = __fsub_rn(p2[2], p0[2]);
            const float cx = __fmaf_rn(e1y, e2z, -__fmul_rn(e1z, e2y));
            const float cy = __fmaf_rn(e1z, e2x, -__fmul_rn(e1x, e2z));
            const float cz = __fmaf_rn(e1x, e2y, -__fmul_rn(e1y, e2x));
            const float nn = __fmaf_rn(cz, cz, __fmaf_rn(cy, cy, __fmul_rn(cx, cx)));
            if (nn > 0.0f) {
                const float inv = __fdiv_rn(1.0f, __fsqrt_rn(nn));
                const float nx = __fmul_rn(cx, inv), ny = __fmul_rn(cy, inv), nz = __fmul_rn(cz, inv);
                const float d = -__fmaf_rn(nz, p0[2], __fmaf_rn(ny, p0[1], __fmul_rn(nx, p0[0])));
                pl = make_float4(nx, ny, nz, d);
            } else {
                ok = 0;
            }
        }
        hyp[t] = pl;
        valid[t] = ok;
    }
}

// ---------------------------------------------------------------- stage c
// The record of cluster c from its best (count << 32 | ~h) key (0: no valid
// hypothesis): the selected plane, the in-plane basis and the hull origin.
__device__ __forceinline__ void select_record(uint32_t c, unsigned long long best, const float* __restrict__ pts,
                                              const uint32_t* __restrict__ off, int H,
                                              const float4* __restrict__ hyp, FitCluster* __restrict__ cl) {
    FitCluster f;
    memset(&f, 0, sizeof(f));
    const uint32_t n = off[c + 1] - off[c];
    if (best != 0) {
        const int h = (int)(~(uint32_t)(best & 0xffffffffu));
        const float4 pl = hyp[(size_t)c * H + h];
        f.best_h = h;
        f.n[0] = pl.x; f.n[1] = pl.y; f.n[2] = pl.z; f.d = pl.w;
        f.inliers = (uint32_t)(best >> 32);
        const float nx = pl.x, ny = pl.y, nz = pl.z;
        float ux, uy, uz;
        if (fabsf(nx) < 0.9f) { ux = 0.0f; uy = -nz; uz = ny; }  // e_x cross n
        else { ux = nz; uy = 0.0f; uz = -nx; }                   // e_y cross n
        const float ul = __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmul_rn(ux, ux)));
        const float ui = __fdiv_rn(1.0f, __fsqrt_rn(ul));
        ux = __fmul_rn(ux, ui); uy = __fmul_rn(uy, ui); uz = __fmul_rn(uz, ui);
        f.u[0] = ux; f.u[1] = uy; f.u[2] = uz;
        f.v[0] = __fmaf_rn(ny, uz, -__fmul_rn(nz, uy));
        f.v[1] = __fmaf_rn(nz, ux, -__fmul_rn(nx, uz));
        f.v[2] = __fmaf_rn(nx, uy, -__fmul_rn(ny, ux));
    } else {
        f.best_h = -1;
    }
    if (n) {
        const float* p = pts + 3 * (size_t)off[c];
        f.o[0] = p[0]; f.o[1] = p[1]; f.o[2] = p[2];
    }
    cl[c] = f;
}

// This thread's best (count << 32 | ~h) key over hypotheses h = i, i + step,
// ... of cluster c (counts read from L2: other CTAs added them).
__device__ __forceinline__ unsigned long long best_key(uint32_t c, int i, int step, int H,
                                                       const uint8_t* __restrict__ valid,
                                                       const uint32_t* __restrict__ counts) {
    unsigned long long best = 0;  // 0 = none
    for (int h = i; h < H; h += step) {
        const size_t t = (size_t)c * H + h;
        if (valid[t]) {
            const unsigned long long key = ((unsigned long long)__ldcg(counts + t) << 32) | (uint32_t)(~(uint32_t)h);
            best = key > best ? key : best;
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, s);
        best = o > best ? o : best;
    }
    return best;
}

// Stage c for cluster c by a whole CTA of kT threads (wbest: kT / 32 words
// of shared memory): maximum count, lowest hypothesis index on ties.
__device__ __forceinline__ void select_cta(uint32_t c, const float* __restrict__ pts, const uint32_t* __restrict__ off,
                                           int H, const float4* __restrict__ hyp, const uint8_t* __restrict__ valid,
                                           const uint32_t* __restrict__ counts, FitCluster* __restrict__ cl,
                                           unsigned long long* wbest) {
    unsigned long long best = best_key(c, threadIdx.x, kT, H, valid, counts);
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kT / 32; ++w) best = wbest[w] > best ? wbest[w] : best;
        select_record(c, best, pts, off, H, hyp, cl);
    }
    __syncthreads();
}

__global__ void k_select(const float* __restrict__ pts, const uint32_t* __restrict__ off,
                         const uint32_t* __restrict__ kp, int H, const float4* __restrict__ hyp,
                         const uint8_t* __restrict__ valid, const uint32_t* __restrict__ counts,
                         FitCluster* __restrict__ cl) {
    pdl_gate();
    const uint32_t k = *kp;
    __shared__ unsigned long long wbest[kT / 32];
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) select_cta(c, pts, off, H, hyp, valid, counts, cl, wbest);
}

// Per-cluster completion: every work item of a cluster, after its results
// are visible device-wide, counts itself done; the CTA (or warp) that
// completes the cluster's last item runs the cluster's next serial step
// (stage c after scoring, the centroid after extraction, the refit after the
// filter) in place of a kernel of its own.  done: three counters a cluster,
// cleared before the fit.
__device__ __forceinline__ bool cta_last_item(uint32_t* done, uint32_t n_items, uint32_t* flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *flag = atomicAdd(done, 1u) + 1u == n_items;
    __syncthreads();
    const bool last = *flag != 0u;
    if (last) __threadfence();
    return last;
}

// ---------------------------------------------------------------- stage b
template <int R>
__global__ void __launch_bounds__(kT) k_score(const float* __restrict__ pts, const uint32_t* __restrict__ off,
                                              const uint32_t* __restrict__ item_off,
                                              const uint32_t* __restrict__ item_cl, const uint32_t* __restrict__ kp,
                                              int H, int T, const float4* __restrict__ hyp,
                                              uint32_t* __restrict__ counts, uint32_t* __restrict__ queue, float eps) {
    pdl_wait();
    const uint32_t k = *kp;
    extern __shared__ float4 sp[];                // T staged points
    uint32_t* red = reinterpret_cast<uint32_t*>(sp + T);  // [P][G*R]
    __shared__ uint32_t s_item;
    const int G = (H + R - 1) / R;                // threads per point subset
    const int P = kT / G;                         // point subsets
    const int g = threadIdx.x / G, j = threadIdx.x % G;
    const bool active = g < P;
    const uint32_t n_items = item_off[k];
    for (int guard = 0; guard < kLoopCap; ++guard) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const uint32_t c = find_cluster(item_cl, item_off, k, it);
        const uint32_t start = off[c] + (it - item_off[c]) * (uint32_t)T;
        const uint32_t end = min(off[c + 1], start + (uint32_t)T);
        const int cnt = (int)(end - start);
        for (int q = threadIdx.x; q < cnt; q += kT) {
            const float* p = pts + 3 * ((size_t)start + q);
            sp[q] = make_float4(p[0], p[1], p[2], 0.0f);
        }
        float4 pl[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int h = j * R + r;
            pl[r] = (active && h < H) ? hyp[(size_t)c * H + h]
                                      : make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0x7f800000));
        }
        __syncthreads();
        uint32_t acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0;
        if (active) {
            for (int q = g; q < cnt; q += P) count_point<R>(pl, sp[q], eps, acc);
#pragma unroll
            for (int r = 0; r < R; ++r) red[g * (G * R) + j * R + r] = acc[r];
        }
        __syncthreads();
        for (int h = threadIdx.x; h < H; h += kT) {
            uint32_t s = 0;
            for (int q = 0; q < P; ++q) s += red[q * (G * R) + h];
            if (s) atomicAdd(&counts[(size_t)c * H + h], s);
        }
    }
}

// In-plane coordinates relative to the origin in units of 2^-16 m, before
// rounding: quantise() rounds exactly these values, so each lies within half
// a unit of its quantised coordinate.
__device__ __forceinline__ float2 plane_coords(const FitCluster& f, float px, float py, float pz) {
    const float qx = __fsub_rn(px, f.o[0]), qy = __fsub_rn(py, f.o[1]), qz = __fsub_rn(pz, f.o[2]);
    const float a = __fmaf_rn(qz, f.u[2], __fmaf_rn(qy, f.u[1], __fmul_rn(qx, f.u[0])));
    const float b = __fmaf_rn(qz, f.v[2], __fmaf_rn(qy, f.v[1], __fmul_rn(qx, f.v[0])));
    return make_float2(__fmul_rn(a, 65536.0f), __fmul_rn(b, 65536.0f));
}

// Quantised in-plane coordinates (units of 2^-16 m) relative to the origin.
__device__ __forceinline__ int2 quantise(const FitCluster& f, float px, float py, float pz) {
    const float2 w = plane_coords(f, px, py, pz);
    return make_int2(__float2int_rn(w.x), __float2int_rn(w.y));
}

// The 16 filter directions, counter-clockwise: (1,0) (2,1) (1,1) (1,2) (0,1)
// (-1,2) (-1,1) (-2,1) (-1,0) (-2,-1) (-1,-1) (-1,-2) (0,-1) (1,-2) (1,-1) (2,-1);
// direction d + 8 is direction d negated.  With |X|, |Y| < 2^28 every value
// fits in int32.
constexpr int kFiltDirs = 16;
__device__ __forceinline__ int32_t dir_value(int dir, int2 p) {
    const int a = (dir == 0 || dir == 2 || dir == 3 || dir == 14 || dir == 13) ? 1
                : (dir == 1 || dir == 15) ? 2
                : (dir == 4 || dir == 12) ? 0
                : (dir == 7 || dir == 9) ? -2 : -1;
    const int b = (dir == 0 || dir == 8) ? 0
                : (dir == 1 || dir == 2 || dir == 4 || dir == 6 || dir == 7) ? 1
                : (dir == 3 || dir == 5) ? 2
                : (dir == 11 || dir == 13) ? -2 : -1;
    return a * p.x + b * p.y;
}

__device__ __forceinline__ unsigned long long ext_key(int32_t v, uint32_t idx) {
    return ((unsigned long long)((uint32_t)v ^ 0x80000000u) << 32) | idx;
}

template <typename Tv>
__device__ __forceinline__ Tv block_sum(Tv v, Tv* sh) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    Tv t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
    return t;  // valid in thread 0
}

// Partial sums of the refit are formed per 256-point chunk of a cluster (one
// point per thread, a fixed reduction tree), whatever the work-item tile: the
// refit is then the same for every scoring schedule, and a cluster's result
// does not depend on the batch it is fitted in.
constexpr uint32_t kChunk = kT;

// Per-chunk sums in a fixed order without a barrier per chunk: each warp
// reduces its 32 values with a shuffle tree and parks the result in shared
// memory (wp[chunk][warp][value]); after the item's last chunk one barrier,
// then thread j adds chunk j's eight warp results in warp order.
constexpr int kMaxChunksPerItem = 16384 / (int)kChunk;

// The warp tree is the butterfly over lane offsets 16, 8, 4, 2, 1 for every
// value, transposed: at each of the first levels a lane keeps half of its
// values and sends the other half to its partner, which keeps the opposite
// half, so NV values (padded to P = 4 or 8) take 2 + 1 + 3 (P = 4) or
// 4 + 2 + 1 + 2 (P = 8) shuffles instead of 5 NV.  Each partial sum is
// the one the plain butterfly forms at that level (a + b = b + a exactly),
// so the totals are bit-identical to it.  Value e ends in the lanes whose top
// log2(P) lane bits equal e.
template <int NV>
__device__ __forceinline__ void warp_park(float (&v)[NV], float* wp, uint32_t j) {
    static_assert(NV == 4 || NV == 6, "4 or 6 values");
    constexpr int P = NV == 4 ? 4 : 8;
    constexpr int L = NV == 4 ? 2 : 3;  // log2(P): halving levels at offsets 16 .. 32 >> L
    const int lane = threadIdx.x & 31;
    float x[P];
#pragma unroll
    for (int e = 0; e < P; ++e) x[e] = e < NV ? v[e] : 0.0f;
#pragma unroll
    for (int lv = 0; lv < L; ++lv) {
        const int s = 16 >> lv, h = P >> (lv + 1);
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float keep = up ? x[h + i] : x[i];
            const float send = up ? x[i] : x[h + i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
#pragma unroll
    for (int s = 16 >> L; s > 0; s >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], s);
    const int e = (lane >> (5 - L)) & (P - 1);
    if ((lane & ((32 >> L) - 1)) == 0 && e < NV) wp[(j * (kT / 32) + (threadIdx.x >> 5)) * NV + e] = x[0];
}

template <int NV>
__device__ __forceinline__ void chunks_out(const float* wp, uint32_t n_chunks, float* dst /* [chunk][10] */,
                                           int first) {
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n_chunks; j += kT) {
        float t[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) t[e] = 0.0f;
        for (int w = 0; w < kT / 32; ++w)
#pragma unroll
            for (int e = 0; e < NV; ++e) t[e] += wp[(j * (kT / 32) + w) * NV + e];
#pragma unroll
        for (int e = 0; e < NV; ++e) dst[(size_t)j * 10 + first + e] = t[e];
    }
    __syncthreads();
}

// Double-float arithmetic: a value is hi + lo with |lo| at most half an ulp of
// hi, about 46 significant bits, on the FP32 pipes (FP64 is a slow path on
// this part).  Built from the error-free transformations TwoSum (Knuth) and
// TwoProduct (Dekker; exact here with an fma).
struct df2 {
    float hi, lo;
};
__device__ __forceinline__ df2 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df2 df_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df2 df_add(df2 x, df2 y) {
    df2 s = df_two_sum(x.hi, y.hi);
    const df2 t = df_two_sum(x.lo, y.lo);
    s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df2 df_neg(df2 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df2 df_sub(df2 x, df2 y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df2 df_mul(df2 x, df2 y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df2 df_mulf(df2 x, float y) { return df_mul(x, df2{y, 0.0f}); }
// x / n for a count n < 2^24 (exact in FP32): one quotient, its exact
// residual, one correction.
__device__ __forceinline__ df2 df_div_count(df2 x, uint32_t n) {
    const float fn = (float)n;
    const float q1 = __fdiv_rn(x.hi, fn);
    const df2 r = df_sub(x, df2{__fmul_rn(q1, fn), __fmaf_rn(q1, fn, -__fmul_rn(q1, fn))});
    return df_fast_two_sum(q1, __fdiv_rn(r.hi, fn));
}
__device__ __forceinline__ df2 df_shfl_xor(df2 x, int o) {
    return {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

// Sums NV double-float values over a CTA in a fixed order: a shuffle tree in
// each warp, then the warps' results in warp order.  The total is valid in
// thread 0.  sh: NV * (kT / 32) entries of shared memory.
template <int NV>
__device__ __forceinline__ void block_df_sum(df2 (&v)[NV], df2* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int e = 0; e < NV; ++e) v[e] = df_add(v[e], df_shfl_xor(v[e], o));
    if (lane == 0)
#pragma unroll
        for (int e = 0; e < NV; ++e) sh[e * (kT / 32) + w] = v[e];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            df2 t = sh[e * (kT / 32)];
            for (int q = 1; q < kT / 32; ++q) t = df_add(t, sh[e * (kT / 32) + q]);
            v[e] = t;
        }
}

// Inlier count and centroid of cluster c by a whole CTA: the per-chunk
// partial sums (read from L2: other CTAs wrote them) added in double-float in
// a fixed order (thread-strided, then block_df_sum), so the result does not
// depend on scheduling.  The centroid is kept as (hi, lo) per axis.
__device__ __forceinline__ void centroid_cta(uint32_t c, const uint32_t* __restrict__ off,
                                             const uint32_t* __restrict__ item_off, int T,
                                             const float* __restrict__ part, FitCluster* __restrict__ cl,
                                             float* __restrict__ cen, df2* sh, uint32_t* shn) {
    const uint32_t cpt = (uint32_t)T / kChunk;
    df2 v[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    uint32_t n = 0;
    const uint32_t base = item_off[c] * cpt, nch = (off[c + 1] - off[c] + kChunk - 1) / kChunk;
#pragma unroll 2
    for (uint32_t j = threadIdx.x; j < nch; j += kT) {
        const float* pp = part + (size_t)(base + j) * 10;
        n += (uint32_t)__ldcg(pp);
        v[0] = df_add(v[0], df2{__ldcg(pp + 1), 0.0f});
        v[1] = df_add(v[1], df2{__ldcg(pp + 2), 0.0f});
        v[2] = df_add(v[2], df2{__ldcg(pp + 3), 0.0f});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) shn[threadIdx.x >> 5] = n;
    block_df_sum<3>(v, sh);
    if (threadIdx.x == 0) {
        n = 0;
        for (int q = 0; q < kT / 32; ++q) n += shn[q];
        FitCluster& f = cl[c];
        f.inliers = n;
        df2 cx{f.o[0], 0.0f}, cy{f.o[1], 0.0f}, cz{f.o[2], 0.0f};
        if (n) {
            cx = df_add(cx, df_div_count(v[0], n));
            cy = df_add(cy, df_div_count(v[1], n));
            cz = df_add(cz, df_div_count(v[2], n));
        }
        float* ce = cen + 6 * (size_t)c;
        ce[0] = cx.hi; ce[1] = cx.lo; ce[2] = cy.hi; ce[3] = cy.lo; ce[4] = cz.hi; ce[5] = cz.lo;
        f.c[0] = cx.hi; f.c[1] = cy.hi; f.c[2] = cz.hi;
    }
    __syncthreads();  // shared partials reused next
}

// After an extraction item of cluster c: the CTA that completes the cluster's
// last item computes its centroid (out of line: the item loop keeps its
// registers).
__device__ __noinline__ void extract_tail(uint32_t c, const uint32_t* __restrict__ off,
                                          const uint32_t* __restrict__ item_off, int T,
                                          const float* __restrict__ part, FitCluster* __restrict__ cl,
                                          float* __restrict__ cen, uint32_t* __restrict__ done) {
    __shared__ df2 sh[3 * (kT / 32)];
    __shared__ uint32_t shn[kT / 32], s_last;
    if (cta_last_item(done + 3 * (size_t)c + 1, item_off[c + 1] - item_off[c], &s_last))
        centroid_cta(c, off, item_off, T, part, cl, cen, sh, shn);
}

// Inliers, centroid partials (relative to the origin) and the extreme inliers
// along the 16 filter directions (reduced per warp, then atomicMax).
// kTail: the CTA that completes a cluster's last item computes its centroid
// (done: the per-cluster completion counters).
template <bool kTail>
__global__ void __launch_bounds__(kT) k_extract(const float* __restrict__ pts, const uint32_t* __restrict__ off,
                                                const uint32_t* __restrict__ item_off,
                                                const uint32_t* __restrict__ item_cl, const uint32_t* __restrict__ kp,
                                                int T, FitCluster* __restrict__ cl, uint8_t* __restrict__ inlier,
                                                float* __restrict__ part, float eps, uint32_t* __restrict__ err,
                                                uint32_t* __restrict__ done, float* __restrict__ cen) {
    pdl_gate();
    const uint32_t k = *kp;
    __shared__ float wp[kMaxChunksPerItem * (kT / 32) * 4];
    const uint32_t n_items = item_off[k];
    const uint32_t cpt = (uint32_t)T / kChunk;  // chunks per work item
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint32_t c = find_cluster(item_cl, item_off, k, it);
        const FitCluster f = cl[c];
        const uint32_t start = off[c] + (it - item_off[c]) * (uint32_t)T;
        const uint32_t end = min(off[c + 1], start + (uint32_t)T);
        // per thread and direction d < 8: the largest value and its point (the
        // last one, i.e. the largest index, among equal values: points come in
        // index order), and the smallest value and its point; direction d + 8
        // is direction d negated, so its key is (-smallest, index)
        int vmax[kFiltDirs / 2], imax[kFiltDirs / 2], vmin[kFiltDirs / 2], imin[kFiltDirs / 2];
#pragma unroll
        for (int d = 0; d < kFiltDirs / 2; ++d) {
            vmax[d] = INT_MIN;
            vmin[d] = INT_MAX;
            imax[d] = imin[d] = 0;
        }
        bool big = false;
        // chunk within the item; its slot is it * cpt + j (item_off[c] * cpt + its chunk in the cluster)
        uint32_t j = 0;
#pragma unroll 4
        for (uint32_t q0 = start; q0 < end; q0 += kChunk, ++j) {  // unrolled: later chunks' loads go out early
            const uint32_t q = q0 + threadIdx.x;
            float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // count, sum (p - o)
            if (q < end) {
                const float px = pts[3 * (size_t)q], py = pts[3 * (size_t)q + 1], pz = pts[3 * (size_t)q + 2];
                const bool in = f.best_h >= 0 && plane_dist(f.n[0], f.n[1], f.n[2], f.d, px, py, pz) <= eps;
                inlier[q] = in;
                if (in) {
                    v[0] = 1.0f;
                    v[1] = __fsub_rn(px, f.o[0]);
                    v[2] = __fsub_rn(py, f.o[1]);
                    v[3] = __fsub_rn(pz, f.o[2]);
                    const int2 xy = quantise(f, px, py, pz);
                    big |= (abs(xy.x) >= (1 << 28)) | (abs(xy.y) >= (1 << 28));
                    const int idx = (int)(q - off[c]);
#pragma unroll
                    for (int d = 0; d < kFiltDirs / 2; ++d) {
                        const int val = dir_value(d, xy);
                        if (val >= vmax[d]) { vmax[d] = val; imax[d] = idx; }
                        if (val <= vmin[d]) { vmin[d] = val; imin[d] = idx; }
                    }
                }
            }
            warp_park<4>(v, wp, j);
        }
        chunks_out<4>(wp, j, part + (size_t)it * cpt * 10, 0);  // slot 0 holds the count (at most 256: exact)
        if (big) atomicOr(err, kErrOverflow);
        // the warp's largest key per direction: the extreme value, then the
        // largest index among the lanes that hold it
        const bool lane0 = (threadIdx.x & 31) == 0;
#pragma unroll
        for (int d = 0; d < kFiltDirs / 2; ++d) {
            const int wmax = __reduce_max_sync(0xffffffffu, vmax[d]);
            const int wimax = __reduce_max_sync(0xffffffffu, vmax[d] == wmax ? imax[d] : 0);
            const int wmin = __reduce_min_sync(0xffffffffu, vmin[d]);
            const int wimin = __reduce_max_sync(0xffffffffu, vmin[d] == wmin ? imin[d] : 0);
            if (lane0 && wmax != INT_MIN) atomicMax(&cl[c].ext[d], ext_key(wmax, (uint32_t)wimax));
            if (lane0 && wmin != INT_MAX) atomicMax(&cl[c].ext[d + 8], ext_key(-wmin, (uint32_t)wimin));
        }
        __syncthreads();
        if constexpr (kTail) extract_tail(c, off, item_off, T, part, cl, cen, done);
    }
}

__device__ __forceinline__ long long cross3(int2 o, int2 a, int2 b) {
    return (long long)(a.x - o.x) * (long long)(b.y - o.y) - (long long)(a.y - o.y) * (long long)(b.x - o.x);
}

__device__ __forceinline__ void refit_cta(uint32_t c, const uint32_t* __restrict__ off,
                                          const uint32_t* __restrict__ item_off, int T, const float* __restrict__ part,
                                          const float* __restrict__ cen, FitCluster* __restrict__ cl, df2* sh);

// After a filter item of cluster c: the CTA that completes the cluster's last
// item refits its plane (out of line).
__device__ __noinline__ void filter_tail(uint32_t c, const uint32_t* __restrict__ off,
                                         const uint32_t* __restrict__ item_off, int T, const float* __restrict__ part,
                                         const float* __restrict__ cen, FitCluster* __restrict__ cl,
                                         uint32_t* __restrict__ done) {
    __shared__ df2 sh[6 * (kT / 32)];
    __shared__ uint32_t s_last;
    if (cta_last_item(done + 3 * (size_t)c + 2, item_off[c + 1] - item_off[c], &s_last))
        refit_cta(c, off, item_off, T, part, cen, cl, sh);
}

// Covariance partials about the centroid, and the 16-gon filter: inliers
// strictly inside the polygon through the 16 extreme inliers cannot be hull
// vertices; the others are appended to the cluster's survivor list.  Each
// warp gathers its survivors in shared memory and reserves room in the list
// with one atomic per kSurvBuf survivors (usually one per work item) instead
// of one returned atomic per chunk on the loop's critical path.
//
// The polygon test runs in FP32 on the unrounded plane coordinates (af, bf)
// against each edge's line scaled by a bound E on the test's own error: with
// A -> B an edge (quantised ints, ex = B - A), c = ex A.y - ey A.x and the
// cluster's inliers within |X|, |Y| <= M - 1 (their extremes along +-x, +-y),
//   F = (ex bf - ey af - c) / E,  E = 2 (0.5 (|ex| + |ey|) + 2^-21 ((|ex| + |ey|) M + |c|) + 1),
// differs from the exact cross product (ex Y - ey X - c) / E by less than 0.5:
// af, bf lie within half a unit of X, Y, and the conversions, the divisions
// and the two fused multiply-adds add at most 2^-22 ((|ex| + |ey|) M + |c|).
// So min over the edges F > 1 means strictly inside every edge (the point is
// dropped) and F < -1 on some edge means outside it (a survivor); the few
// points in between take the exact integer test.  The edges' coefficients are
// read from shared memory once per kBatch chunks.
template <bool kTail>
__global__ void __launch_bounds__(kT) k_filter(const float* __restrict__ pts, const uint32_t* __restrict__ off,
                                               const uint32_t* __restrict__ item_off,
                                               const uint32_t* __restrict__ item_cl, const uint32_t* __restrict__ kp,
                                               int T, FitCluster* __restrict__ cl, const uint8_t* __restrict__ inlier,
                                               const float* __restrict__ cen, float* __restrict__ part,
                                               int2* __restrict__ surv, uint32_t* __restrict__ done) {
    pdl_gate();
    const uint32_t k = *kp;
    constexpr int kSurvBuf = 128;
    constexpr int kBatch = 4;  // chunks a thread tests against the edges together
    __shared__ float wp[kMaxChunksPerItem * (kT / 32) * 6];
    __shared__ int2 sxy[kFiltDirs];
    __shared__ int2 poly[kFiltDirs + 1];
    __shared__ float4 edge[kFiltDirs];  // (ex / E, -ey / E, -c / E): F = x bf + y af + z
    __shared__ int npoly;
    __shared__ float sM;
    __shared__ int2 sbuf[kT / 32][kSurvBuf];
    int2* sb = sbuf[threadIdx.x >> 5];
    const uint32_t n_items = item_off[k];
    const int lane = threadIdx.x & 31;
    const uint32_t cpt = (uint32_t)T / kChunk;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint32_t c = find_cluster(item_cl, item_off, k, it);
        const FitCluster f = cl[c];
        const uint32_t base = off[c];
        const uint32_t start = base + (it - item_off[c]) * (uint32_t)T;
        const uint32_t end = min(off[c + 1], start + (uint32_t)T);
        __syncthreads();
        if (threadIdx.x < kFiltDirs) {  // the extreme points, one direction a thread
            const int d = threadIdx.x;
            const unsigned long long key = cl[c].ext[d];  // not f.ext[d]: an indexed copy would live on the stack
            int2 xy = make_int2(INT_MIN, INT_MIN);  // none
            if (key) {
                const float* p = pts + 3 * ((size_t)base + (uint32_t)(key & 0xffffffffu));
                xy = quantise(f, p[0], p[1], p[2]);
            }
            sxy[d] = xy;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // polygon through the extreme points, counter-clockwise, duplicates removed
            int m = 0;
            for (int d = 0; d < kFiltDirs; ++d) {
                const int2 xy = sxy[d];
                if (xy.x == INT_MIN && xy.y == INT_MIN) continue;
                if (m && poly[m - 1].x == xy.x && poly[m - 1].y == xy.y) continue;
                poly[m++] = xy;
            }
            if (m > 1 && poly[m - 1].x == poly[0].x && poly[m - 1].y == poly[0].y) --m;
            // a degenerate (zero-area) polygon filters nothing
            long long area2 = 0;
            for (int i = 0; i < m; ++i) {
                const int2 a = poly[i], b = poly[(i + 1) % m];
                area2 += (long long)a.x * b.y - (long long)a.y * b.x;
            }
            npoly = (m >= 3 && area2 > 0) ? m : 0;
            // |X|, |Y| of every inlier: at most the extremes along +-x (directions 0, 8), +-y (4, 12)
            int mx = 0;
            for (int d = 0; d < kFiltDirs; d += 4)
                if (f.ext[d]) mx = max(mx, abs((int)((uint32_t)(f.ext[d] >> 32) ^ 0x80000000u)));
            sM = (float)mx + 1.0f;
        }
        __syncthreads();
        const int m = npoly;
        if (threadIdx.x < kFiltDirs) {  // the edges' scaled lines, one edge a thread; padding never decides
            const int i = threadIdx.x;
            float4 e = make_float4(0.0f, 0.0f, 2.0f, 0.0f);
            if (i < m) {
                const int2 A = poly[i], B = poly[(i + 1) % m];
                const long long ex = (long long)B.x - A.x, ey = (long long)B.y - A.y;
                const long long cc = (long long)((unsigned long long)ex * (unsigned long long)(long long)A.y -
                                                 (unsigned long long)ey * (unsigned long long)(long long)A.x);
                const float exf = (float)ex, eyf = (float)ey, cf = (float)cc;
                const float sum = fabsf(exf) + fabsf(eyf);
                const float E = 2.0f * (0.5f * sum + 4.76837158203125e-7f * (sum * sM + fabsf(cf)) + 1.0f);
                e = make_float4(__fdiv_rn(exf, E), -__fdiv_rn(eyf, E), -__fdiv_rn(cf, E), 0.0f);
            }
            edge[i] = e;
        }
        __syncthreads();
        const float cx = cen[6 * c], cy = cen[6 * c + 2], cz = cen[6 * c + 4];  // nearest floats of the centroid
        int cnt = 0;  // survivors in this warp's buffer (warp-uniform)
        auto flush = [&]() {
            uint32_t pos = 0;
            if (lane == 0) pos = atomicAdd(&cl[c].n_surv, (uint32_t)cnt);
            pos = __shfl_sync(0xffffffffu, pos, 0);
            for (int i = lane; i < cnt; i += 32) surv[base + pos + i] = sb[i];
            __syncwarp();
            cnt = 0;
        };
        uint32_t j = 0;
        for (uint32_t qb = start; qb < end; qb += kBatch * kChunk) {
            float px[kBatch], py[kBatch], pz[kBatch], af[kBatch], bf[kBatch], fmin[kBatch];
            bool live[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const uint32_t q = qb + u * kChunk + threadIdx.x;
                live[u] = q < end && inlier[q];
                px[u] = py[u] = pz[u] = af[u] = bf[u] = 0.0f;
                if (live[u]) {
                    px[u] = pts[3 * (size_t)q]; py[u] = pts[3 * (size_t)q + 1]; pz[u] = pts[3 * (size_t)q + 2];
                    const float2 w = plane_coords(f, px[u], py[u], pz[u]);
                    af[u] = w.x;
                    bf[u] = w.y;
                }
                fmin[u] = 2.0f;
            }
            if (m) {
#pragma unroll
                for (int i = 0; i < kFiltDirs; ++i) {
                    const float4 e = edge[i];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u)
                        fmin[u] = fminf(fmin[u], __fmaf_rn(e.x, bf[u], __fmaf_rn(e.y, af[u], e.z)));
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (qb + u * kChunk >= end) continue;  // uniform: past the item's last chunk
                bool keep = false;
                int2 xy = make_int2(0, 0);
                float v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // centred second moments
                if (live[u]) {
                    const float rx = __fsub_rn(px[u], cx), ry = __fsub_rn(py[u], cy), rz = __fsub_rn(pz[u], cz);
                    v[0] = __fmul_rn(rx, rx); v[1] = __fmul_rn(ry, ry); v[2] = __fmul_rn(rz, rz);
                    v[3] = __fmul_rn(rx, ry); v[4] = __fmul_rn(rx, rz); v[5] = __fmul_rn(ry, rz);
                    keep = !m || !(fmin[u] > 1.0f);
                    if (keep) {
                        xy = make_int2(__float2int_rn(af[u]), __float2int_rn(bf[u]));
                        if (m && !(fmin[u] < -1.0f)) {  // within the error band of an edge: the exact test
                            for (int i = 0; i < m; ++i) {  // strictly inside every edge -> not a hull vertex
                                if (cross3(poly[i], poly[(i + 1) % m], xy) <= 0) break;
                                if (i == m - 1) keep = false;
                            }
                        }
                    }
                }
                const uint32_t b = __ballot_sync(0xffffffffu, keep);
                if (cnt + __popc(b) > kSurvBuf) flush();
                if (keep) sb[cnt + __popc(b & ((1u << lane) - 1u))] = xy;
                cnt += __popc(b);
                __syncwarp();
                warp_park<6>(v, wp, j);
                ++j;
            }
        }
        if (cnt) flush();
        chunks_out<6>(wp, j, part + (size_t)it * cpt * 10, 4);
        if constexpr (kTail) filter_tail(c, off, item_off, T, part, cen, cl, done);
    }
}

// Refit of cluster c by a whole CTA: total least squares on the inliers.  The
// covariance A about the centroid is summed in double-float over the
// per-chunk partials and scaled by its trace.  Its smallest eigenvector is the
// dominant eigenvector of the adjugate adj(A) (eigenvalues lambda_j lambda_k);
// the adjugate's cofactors, where the cancellation is, are formed in
// double-float and rounded, then six steps of power iteration in FP32 from
// the selected RANSAC normal converge by lambda_min / lambda_mid per step.
// n_z >= 0, d = -n . centroid (double-float); lambda_mid < 10 lambda_min
// (from the trace, the Rayleigh quotient in double-float and
// x^T adj(A) x = lambda_1 lambda_2) flags the plane ill-conditioned.
__device__ __forceinline__ void refit_cta(uint32_t c, const uint32_t* __restrict__ off,
                                          const uint32_t* __restrict__ item_off, int T, const float* __restrict__ part,
                                          const float* __restrict__ cen, FitCluster* __restrict__ cl, df2* sh) {
    const uint32_t cpt = (uint32_t)T / kChunk;
    {
        df2 A[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) A[e] = df2{0.0f, 0.0f};
        const uint32_t base = item_off[c] * cpt, nch = (off[c + 1] - off[c] + kChunk - 1) / kChunk;
#pragma unroll 2
        for (uint32_t j = threadIdx.x; j < nch; j += kT)
#pragma unroll
            for (int e = 0; e < 6; ++e) A[e] = df_add(A[e], df2{__ldcg(part + (size_t)(base + j) * 10 + 4 + e), 0.0f});
        block_df_sum<6>(A, sh);
        if (threadIdx.x == 0) {
            FitCluster& f = cl[c];
            uint32_t flags = 0;
            float rn[3] = {0.0f, 0.0f, 0.0f}, rd = 0.0f;
            const float tr = __fadd_rn(__fadd_rn(A[0].hi, A[1].hi), A[2].hi);
            if (f.best_h >= 0 && f.inliers > 0 && tr > 0.0f) {
                // A / tr: entries of magnitude at most 1 (the diagonal is non-negative)
                const float itr = __fdiv_rn(1.0f, tr);
                df2 S[6];
    #pragma unroll
                for (int e = 0; e < 6; ++e) S[e] = df_mulf(A[e], itr);
                const df2 a = S[0], b = S[1], cc = S[2], d = S[3], e = S[4], g = S[5];
                // symmetric adjugate (cofactors) of [[a d e] [d b g] [e g cc]]
                const float m00 = df_sub(df_mul(b, cc), df_mul(g, g)).hi, m11 = df_sub(df_mul(a, cc), df_mul(e, e)).hi;
                const float m22 = df_sub(df_mul(a, b), df_mul(d, d)).hi, m01 = df_sub(df_mul(e, g), df_mul(d, cc)).hi;
                const float m02 = df_sub(df_mul(d, g), df_mul(e, b)).hi, m12 = df_sub(df_mul(d, e), df_mul(a, g)).hi;
                float x = f.n[0], y = f.n[1], z = f.n[2];
                bool ok = true;
                for (int it = 0; it < 6; ++it) {
                    const float nx = __fmaf_rn(m02, z, __fmaf_rn(m01, y, __fmul_rn(m00, x)));
                    const float ny = __fmaf_rn(m12, z, __fmaf_rn(m11, y, __fmul_rn(m01, x)));
                    const float nz = __fmaf_rn(m22, z, __fmaf_rn(m12, y, __fmul_rn(m02, x)));
                    const float q = __fmaf_rn(nz, nz, __fmaf_rn(ny, ny, __fmul_rn(nx, nx)));
                    if (!(q > 1e-30f) || !(q < 1e30f)) { ok = false; break; }  // rank <= 1: keep the RANSAC normal
                    const float sc = rsqrtf(q);
                    x = __fmul_rn(nx, sc); y = __fmul_rn(ny, sc); z = __fmul_rn(nz, sc);
                }
                if (!ok) {
                    x = f.n[0]; y = f.n[1]; z = f.n[2];
                    flags |= 1u;
                }
                // unit length to FP32 accuracy
                const float inv = __fdiv_rn(1.0f, __fsqrt_rn(__fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)))));
                x = __fmul_rn(x, inv); y = __fmul_rn(y, inv); z = __fmul_rn(z, inv);
                if (z < 0.0f || (z == 0.0f && (y < 0.0f || (y == 0.0f && x < 0.0f)))) { x = -x; y = -y; z = -z; }
                // eigenvalues (scaled by 1 / tr) for the conditioning flag
                const df2 ax = df_add(df_add(df_mulf(a, x), df_mulf(d, y)), df_mulf(e, z));
                const df2 ay = df_add(df_add(df_mulf(d, x), df_mulf(b, y)), df_mulf(g, z));
                const df2 az = df_add(df_add(df_mulf(e, x), df_mulf(g, y)), df_mulf(cc, z));
                const float lmin = df_add(df_add(df_mulf(ax, x), df_mulf(ay, y)), df_mulf(az, z)).hi;
                const float p12 = x * (m00 * x + m01 * y + m02 * z) + y * (m01 * x + m11 * y + m12 * z) +
                                  z * (m02 * x + m12 * y + m22 * z);
                const float Sx = 1.0f - lmin;
                const float disc = fmaxf(Sx * Sx - 4.0f * p12, 0.0f);
                const float lmax = 0.5f * (Sx + sqrtf(disc));
                const float lmid = lmax > 0.0f ? p12 / lmax : 0.0f;  // no cancellation
                if (!(lmid >= 10.0f * lmin)) flags |= 1u;
                rn[0] = x; rn[1] = y; rn[2] = z;
                const float* ce = cen + 6 * (size_t)c;
                const df2 dot = df_add(df_add(df_mulf(df2{ce[0], ce[1]}, x), df_mulf(df2{ce[2], ce[3]}, y)),
                                       df_mulf(df2{ce[4], ce[5]}, z));
                rd = -dot.hi;
            } else if (f.best_h >= 0 && f.inliers > 0) {
                flags |= 1u;  // zero spread: no plane to fit; the RANSAC normal through the centroid
                rn[0] = f.n[0]; rn[1] = f.n[1]; rn[2] = f.n[2];
                const float* ce = cen + 6 * (size_t)c;
                rd = -df_add(df_add(df_mulf(df2{ce[0], ce[1]}, rn[0]), df_mulf(df2{ce[2], ce[3]}, rn[1])),
                             df_mulf(df2{ce[4], ce[5]}, rn[2])).hi;
        }
        f.refit_n[0] = rn[0]; f.refit_n[1] = rn[1]; f.refit_n[2] = rn[2];
        f.refit_d = rd;
        f.flags = flags;
        }
    }
    __syncthreads();  // shared partials reused next
}

// The centroid and the refit of every cluster as kernels of their own (a CTA
// per cluster), for fits too large for the per-cluster completion counters
// to pay (launch_fit).
__global__ void __launch_bounds__(kT) k_centroid(const uint32_t* __restrict__ off,
                                                 const uint32_t* __restrict__ item_off, const uint32_t* __restrict__ kp,
                                                 int T, const float* __restrict__ part, FitCluster* __restrict__ cl,
                                                 float* __restrict__ cen) {
    pdl_gate();
    const uint32_t k = *kp;
    __shared__ df2 sh[3 * (kT / 32)];
    __shared__ uint32_t shn[kT / 32];
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) centroid_cta(c, off, item_off, T, part, cl, cen, sh, shn);
}

__global__ void __launch_bounds__(kT) k_refit(const uint32_t* __restrict__ off, const uint32_t* __restrict__ item_off,
                                              const uint32_t* __restrict__ kp, int T, const float* __restrict__ part,
                                              const float* __restrict__ cen, FitCluster* __restrict__ cl) {
    pdl_gate();
    const uint32_t k = *kp;
    __shared__ df2 sh[6 * (kT / 32)];
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) refit_cta(c, off, item_off, T, part, cen, cl, sh);
}

__device__ __forceinline__ unsigned long long xy_key(int2 p) {
    return ((unsigned long long)((uint32_t)p.x ^ 0x80000000u) << 32) | ((uint32_t)p.y ^ 0x80000000u);
}
__device__ __forceinline__ int2 key_xy(unsigned long long k) {
    return make_int2((int32_t)((uint32_t)(k >> 32) ^ 0x80000000u), (int32_t)((uint32_t)k ^ 0x80000000u));
}

// Monotone chain over sorted unique points; one thread builds a chain.  The
// two top entries stay in registers so a pop costs one shared-memory load.
__device__ int chain(const unsigned long long* P, int u, bool upper, uint32_t* st) {
    int kk = 0;
    int2 t1 = make_int2(0, 0), t0 = make_int2(0, 0);  // top, second
    for (int s = 0; s < u; ++s) {
        const int i = upper ? (u - 1 - s) : s;
        const int2 p = key_xy(P[i]);
        while (kk >= 2 && cross3(t0, t1, p) <= 0) {
            --kk;
            t1 = t0;
            if (kk >= 2) t0 = key_xy(P[st[kk - 2]]);
        }
        st[kk] = (uint32_t)i;
        t0 = t1;
        t1 = p;
        ++kk;
    }
    return kk;
}

// "Better next vertex" from cur: more clockwise, or collinear and farther.
__device__ __forceinline__ bool jarvis_better(int2 cur, int2 a, bool a_ok, int2 b, bool b_ok) {
    if (!b_ok) return false;
    if (!a_ok) return true;
    const long long cr = cross3(cur, a, b);
    if (cr < 0) return true;
    if (cr > 0) return false;
    const long long da = (long long)(a.x - cur.x) * (a.x - cur.x) + (long long)(a.y - cur.y) * (a.y - cur.y);
    const long long db = (long long)(b.x - cur.x) * (b.x - cur.x) + (long long)(b.y - cur.y) * (b.y - cur.y);
    return db > da;
}

// Directions of the second hull filter: kHullDirs integer vectors
// (rint(1024 cos), rint(1024 sin)) of multiples of 360/kHullDirs degrees, in
// counter-clockwise order.  Any closed polygon through input points serves
// the filter (a point strictly left of every edge has winding number >= 1, so
// it lies in the convex hull of the polygon's vertices and is not an extreme
// point); the directions only decide how much it removes.
constexpr int kHullDirs = 128;
constexpr int kSmallHull = kT;  // candidates ranked and tested in parallel, one a thread

// Per cluster hull of the first filter's survivors: (1) extreme survivors along
// kHullDirs directions; (2) survivors strictly inside the polygon they span
// are dropped (none of them can be a hull vertex), the rest gathered in shared
// memory;
// (3) bitonic sort by (X, Y), duplicates removed; (4) monotone chain, lower
// and upper halves built concurrently by two threads.  If more than
// kHullCap points remain, gift wrapping runs over the survivors instead.
// hull_ctr: a word that is zero at launch; the last CTA to finish turns
// hull_cnt into the hulls' offsets (exclusive scan, the total at [k]) and
// zeroes the word again.
__global__ void __launch_bounds__(kT) k_hull(const uint32_t* __restrict__ off, const uint32_t* __restrict__ kp,
                                             const FitCluster* __restrict__ cl, const int2* __restrict__ surv,
                                             int2* __restrict__ hull, uint32_t* __restrict__ hull_cnt,
                                             uint32_t* __restrict__ err, uint32_t* __restrict__ hull_ctr) {
    pdl_gate();
    const uint32_t k = *kp;
    extern __shared__ unsigned long long sk[];              // kHullCap keys, then kHullCap unique
    unsigned long long* uq = sk + kHullCap;
    uint32_t* st_lo = reinterpret_cast<uint32_t*>(uq + kHullCap);
    uint32_t* st_hi = st_lo + kHullCap;
    int2* ssv = reinterpret_cast<int2*>(st_hi + kHullCap);  // kSurvCap staged survivors
    __shared__ uint32_t wsum[kT / 32];
    __shared__ int s_klo, s_khi, s_m, s_cnt;
    __shared__ int2 poly[kHullDirs + 1];   // the extreme point of each direction
    __shared__ int2 hpoly[kHullDirs + 1];  // the filter polygon
    __shared__ long long warea[kT / 32];
    __shared__ int2 sdir[kHullDirs];
    __shared__ int2 jcand[kT];
    __shared__ int jok[kT];
    __shared__ unsigned long long wmin[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < kHullDirs; j += kT) {
        const float t = (float)j * (2.0f / kHullDirs);
        sdir[j] = make_int2(__float2int_rn(1024.0f * cospif(t)), __float2int_rn(1024.0f * sinpif(t)));
    }
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) {
        __syncthreads();
        const uint32_t base = off[c];
        const int s = (int)cl[c].n_surv;
        int2* out = hull + base;
        if (threadIdx.x == 0) s_cnt = 0;
        // stage the survivors (when they fit) so the scans below read shared memory
        const int2* sv = surv + base;
        if (s <= kSurvCap) {
            for (int i = threadIdx.x; i < s; i += kT) ssv[i] = sv[i];
            sv = ssv;
            __syncthreads();
        }
        // (1) extreme points along kHullDirs directions, warp w taking 16 of
        // them.  The projections are FP32: any closed polygon through input
        // points serves the filter below (which is exact), so an extreme point
        // only has to be an input point, not the exact maximiser.
        {
            constexpr int kPer = kHullDirs / (kT / 32);
            float dxq[kPer], dyq[kPer], bv[kPer];
            int bi[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                dxq[q] = (float)sdir[kPer * w + q].x;
                dyq[q] = (float)sdir[kPer * w + q].y;
                bv[q] = -INFINITY;
                bi[q] = -1;
            }
            for (int i = lane; i < s; i += 32) {
                const int2 p = sv[i];
                const float fx = (float)p.x, fy = (float)p.y;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const float v = fmaf(dxq[q], fx, dyq[q] * fy);
                    if (v > bv[q]) { bv[q] = v; bi[q] = i; }
                }
            }
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, bv[q], o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi[q], o);
                    if (ov > bv[q] || (ov == bv[q] && oi >= 0 && (bi[q] < 0 || oi < bi[q]))) { bv[q] = ov; bi[q] = oi; }
                }
                if (lane == 0) poly[kPer * w + q] = (bi[q] >= 0) ? sv[bi[q]] : make_int2(INT_MIN, INT_MIN);
            }
        }
        __syncthreads();
        // The polygon through the extremes, consecutive duplicates removed (and
        // the last vertex when it repeats the first), in parallel: a direction's
        // extreme is kept unless it repeats the previous direction's; a ballot
        // places the kept ones.  Every direction has an extreme when s > 0.
        {
            const bool valid = s > 0 && threadIdx.x < kHullDirs;
            int2 p = make_int2(0, 0);
            bool keep = false;
            if (valid) {
                p = poly[threadIdx.x];
                const int2 q = poly[threadIdx.x ? threadIdx.x - 1 : 0];
                keep = threadIdx.x == 0 || p.x != q.x || p.y != q.y;
            }
            const uint32_t b = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) wsum[w] = __popc(b);
            __syncthreads();
            uint32_t pos = __popc(b & ((1u << lane) - 1u)), m0 = 0;
            for (int q = 0; q < kT / 32; ++q) {
                pos += q < w ? wsum[q] : 0u;
                m0 += wsum[q];
            }
            if (keep) hpoly[pos] = p;
            __syncthreads();
            if (m0 > 1 && hpoly[m0 - 1].x == hpoly[0].x && hpoly[m0 - 1].y == hpoly[0].y) --m0;
            // twice the signed area: a degenerate (zero-area) polygon filters nothing
            long long a2 = 0;
            if (threadIdx.x < m0) {
                const int2 a = hpoly[threadIdx.x], bb = hpoly[threadIdx.x + 1 < m0 ? threadIdx.x + 1 : 0];
                a2 = (long long)a.x * bb.y - (long long)a.y * bb.x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            if (lane == 0) warea[w] = a2;
            __syncthreads();
            if (threadIdx.x == 0) {
                long long area2 = 0;
                for (int q = 0; q < kT / 32; ++q) area2 += warea[q];
                s_m = (m0 >= 3 && area2 > 0) ? (int)m0 : 0;
            }
        }
        __syncthreads();
        const int m = s_m;
        // (2) drop survivors strictly inside the polygon
        for (int i0 = 0; i0 < s; i0 += kT) {
            const int i = i0 + threadIdx.x;
            bool keep = false;
            int2 p = make_int2(0, 0);
            if (i < s) {
                p = sv[i];
                keep = (m == 0);
                for (int e = 0; e < m; ++e) {
                    if (cross3(hpoly[e], hpoly[e + 1 < m ? e + 1 : 0], p) <= 0) { keep = true; break; }
                }
            }
            const uint32_t b = __ballot_sync(0xffffffffu, keep);
            int pos = 0;
            if (lane == 0 && b) pos = atomicAdd(&s_cnt, __popc(b));
            pos = __shfl_sync(0xffffffffu, pos, 0) + __popc(b & ((1u << lane) - 1u));
            if (keep && pos < kHullCap) sk[pos] = xy_key(p);
        }
        __syncthreads();
        const int s2 = s_cnt;
        if (s2 <= kSmallHull) {
            // (3') at most kT candidates: rank sort with duplicates removed --
            // a candidate is kept if no earlier one has its key, and lands at
            // the number of kept keys below it
            const int i = threadIdx.x;
            unsigned long long key = 0;
            bool first = false;
            if (i < s2) {
                key = sk[i];
                first = true;
                for (int j = 0; j < i; ++j) first &= sk[j] != key;
            }
            st_lo[i] = first;  // kT flags
            __syncthreads();
            int rank = 0;
            if (first)
                for (int j = 0; j < s2; ++j) rank += (st_lo[j] != 0u) & (sk[j] < key);
            const uint32_t b = __ballot_sync(0xffffffffu, first);
            if (lane == 0) wsum[w] = __popc(b);
            __syncthreads();
            int u = 0;
            for (int q = 0; q < kT / 32; ++q) u += (int)wsum[q];
            if (first) uq[rank] = key;
            __syncthreads();
            if (u < 3) {
                if (i < u) out[i] = key_xy(uq[i]);
                if (i == 0) hull_cnt[c] = (uint32_t)u;
            } else {
                // (4') Andrew's chains by a test per candidate: in the sorted
                // order, P_i is a vertex of the lower chain iff it is an end or
                // cross(P_j, P_i, P_k) > 0 for every j < i < k -- the directions
                // P_i - P_j lie in a half-plane (x >= 0, x = 0 only upwards) where
                // cross orders them by angle, so it is enough that the most
                // counter-clockwise of them turns left into the most clockwise of
                // the P_k - P_i; the upper chain is the same over the reversed
                // order.  Collinear points fail (cross = 0), as in the chains.
                bool lo = false, hi = false;
                if (i < u) {
                    const int2 P = key_xy(uq[i]);
                    if (i == 0 || i == u - 1) {
                        lo = hi = true;
                    } else {
                        int2 D = make_int2(0, 0), E = make_int2(0, 0), D2 = make_int2(0, 0), E2 = make_int2(0, 0);
                        for (int j = 0; j < i; ++j) {  // lower: P - P_j (most ccw); upper: P_j - P (most cw)
                            const int2 Q = key_xy(uq[j]);
                            const int2 d = make_int2(P.x - Q.x, P.y - Q.y), e2 = make_int2(Q.x - P.x, Q.y - P.y);
                            if (j == 0 || cross3(make_int2(0, 0), D, d) > 0) D = d;
                            if (j == 0 || cross3(make_int2(0, 0), e2, E2) > 0) E2 = e2;
                        }
                        for (int k2 = i + 1; k2 < u; ++k2) {  // lower: P_k - P (most cw); upper: P - P_k (most ccw)
                            const int2 Q = key_xy(uq[k2]);
                            const int2 e = make_int2(Q.x - P.x, Q.y - P.y), d2 = make_int2(P.x - Q.x, P.y - Q.y);
                            if (k2 == i + 1 || cross3(make_int2(0, 0), e, E) > 0) E = e;
                            if (k2 == i + 1 || cross3(make_int2(0, 0), D2, d2) > 0) D2 = d2;
                        }
                        lo = cross3(make_int2(0, 0), D, E) > 0;
                        hi = cross3(make_int2(0, 0), D2, E2) > 0;
                    }
                    lo &= i < u - 1;  // the lower chain's last point opens the upper chain
                    hi &= i > 0;      // and the upper chain's last point is the first of the lower
                }
                // lower vertices in increasing order, then upper vertices in decreasing order
                const uint32_t bl = __ballot_sync(0xffffffffu, lo), bh = __ballot_sync(0xffffffffu, hi);
                if (lane == 0) {
                    wsum[w] = __popc(bl);
                    st_hi[w] = __popc(bh);
                }
                __syncthreads();
                int klo = 0, khi = 0, plo = __popc(bl & ((1u << lane) - 1u)), phi = __popc(bh >> lane) - (hi ? 1 : 0);
                for (int q = 0; q < kT / 32; ++q) {
                    klo += (int)wsum[q];
                    khi += (int)st_hi[q];
                    plo += q < w ? (int)wsum[q] : 0;
                    phi += q > w ? (int)st_hi[q] : 0;
                }
                if (lo) out[plo] = key_xy(uq[i]);
                if (hi) out[klo + phi] = key_xy(uq[i]);
                if (i == 0) hull_cnt[c] = (uint32_t)(klo + khi);
            }
        } else if (s2 <= kHullCap) {
            int n2 = 1;
            while (n2 < s2) n2 <<= 1;
            for (int i = s2 + threadIdx.x; i < n2; i += kT) sk[i] = ~0ull;
            __syncthreads();
            // (3) bitonic sort, ascending
            for (int size = 2; size <= n2; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = threadIdx.x; i < n2; i += kT) {
                        const int jdx = i ^ stride;
                        if (jdx > i) {
                            const bool up = (i & size) == 0;
                            const unsigned long long a = sk[i], b = sk[jdx];
                            if ((a > b) == up) { sk[i] = b; sk[jdx] = a; }
                        }
                    }
                    __syncthreads();
                }
            }
            // unique, order-preserving (block scan in chunks)
            int u = 0;
            for (int c0 = 0; c0 < s2; c0 += kT) {
                const int i = c0 + threadIdx.x;
                const uint32_t fl = (i < s2) && (i == 0 || sk[i] != sk[i - 1]);
                uint32_t inc = fl;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                if (lane == 31) wsum[w] = inc;
                __syncthreads();
                uint32_t wpre = 0, tot = 0;
                for (int q = 0; q < kT / 32; ++q) {
                    if (q < w) wpre += wsum[q];
                    tot += wsum[q];
                }
                if (fl) uq[u + wpre + inc - 1] = sk[i];
                u += (int)tot;
                __syncthreads();
            }
            // (4) monotone chain
            if (u < 3) {
                for (int i = threadIdx.x; i < u; i += kT) out[i] = key_xy(uq[i]);
                if (threadIdx.x == 0) hull_cnt[c] = (uint32_t)u;
            } else {
                if (threadIdx.x == 0) s_klo = chain(uq, u, false, st_lo);
                if (threadIdx.x == 32) s_khi = chain(uq, u, true, st_hi);
                __syncthreads();
                const int klo = s_klo - 1, khi = s_khi - 1;
                for (int i = threadIdx.x; i < klo + khi; i += kT)
                    out[i] = key_xy(uq[i < klo ? st_lo[i] : st_hi[i - klo]]);
                if (threadIdx.x == 0) hull_cnt[c] = (uint32_t)(klo + khi);
            }
        } else {
            // gift wrapping over all survivors in global memory
            unsigned long long bk = ~0ull;
            for (int i = threadIdx.x; i < s; i += kT) {
                const unsigned long long key = xy_key(sv[i]);
                bk = key < bk ? key : bk;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, bk, o);
                bk = t < bk ? t : bk;
            }
            if (lane == 0) wmin[w] = bk;
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int q = 1; q < kT / 32; ++q) bk = wmin[q] < bk ? wmin[q] : bk;
                wmin[0] = bk;
            }
            __syncthreads();
            const int2 start = key_xy(wmin[0]);
            int2 cur = start;
            int h = 0;
            if (threadIdx.x == 0) out[h] = cur;
            ++h;
            for (int guard = 0; guard <= s; ++guard) {
                int2 cand = make_int2(0, 0);
                bool ok = false;
                for (int i = threadIdx.x; i < s; i += kT) {
                    const int2 p = sv[i];
                    const bool pok = !(p.x == cur.x && p.y == cur.y);
                    if (jarvis_better(cur, cand, ok, p, pok)) { cand = p; ok = true; }
                }
                jcand[threadIdx.x] = cand;
                jok[threadIdx.x] = ok;
                __syncthreads();
                for (int r = kT / 2; r > 0; r >>= 1) {
                    if ((int)threadIdx.x < r) {
                        const int o = threadIdx.x + r;
                        if (jarvis_better(cur, jcand[threadIdx.x], jok[threadIdx.x], jcand[o], jok[o])) {
                            jcand[threadIdx.x] = jcand[o];
                            jok[threadIdx.x] = 1;
                        }
                    }
                    __syncthreads();
                }
                const int2 nxt = jcand[0];
                const bool nok = jok[0];
                __syncthreads();
                if (!nok || (nxt.x == start.x && nxt.y == start.y)) break;
                if (h >= s) {  // more vertices than points: only a broken invariant gets here
                    if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
                    break;
                }
                if (threadIdx.x == 0) out[h] = nxt;
                ++h;
                cur = nxt;
            }
            if (threadIdx.x == 0) hull_cnt[c] = (uint32_t)h;
        }
    }
    // hull offsets, by the last CTA to finish
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_cnt = atomicAdd(hull_ctr, 1u) + 1u == gridDim.x;
    __syncthreads();
    if (!s_cnt) return;
    __threadfence();
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < k; c0 += kT) {
        const uint32_t c = c0 + threadIdx.x;
        const uint32_t v = c < k ? __ldcg(hull_cnt + c) : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int q = 0; q < kT / 32; ++q) {
            if (q < w) wpre += wsum[q];
            tot += wsum[q];
        }
        if (c < k) hull_cnt[c] = carry + wpre + inc - v;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hull_cnt[k] = carry;
        *hull_ctr = 0;
    }
}

// Work items per cluster (scanned into the item offsets next) -- at least one,
// so that an empty cluster's per-cluster steps still run -- the work queue's
// heads and the per-cluster completion counters (done, may be null) cleared
// for the fit that follows.
__global__ void k_items(const uint32_t* __restrict__ off, const uint32_t* __restrict__ kp, int T,
                        uint32_t* __restrict__ item_cnt, uint32_t* __restrict__ queue, uint32_t* __restrict__ done) {
    pdl_gate();
    const uint32_t k = *kp;
    if (blockIdx.x == 0 && threadIdx.x < 4) queue[threadIdx.x] = 0;
    for (uint32_t c = blockIdx.x * kT + threadIdx.x; c < k; c += gridDim.x * kT) {
        const uint32_t n = off[c + 1] - off[c];
        item_cnt[c] = n ? (n + (uint32_t)T - 1) / (uint32_t)T : 1u;
        if (done) done[3 * (size_t)c] = done[3 * (size_t)c + 1] = done[3 * (size_t)c + 2] = 0u;
    }
}

// The work items of up to kItemsScanMax clusters and their offsets in one
// CTA: counts as in k_items, an exclusive scan with a carry across rounds,
// the total at item_off[k].
constexpr int kItemsScanT = 1024;
constexpr uint32_t kItemsScanMax = 16384;
__global__ void __launch_bounds__(kItemsScanT) k_items_scan(const uint32_t* __restrict__ off,
                                                             const uint32_t* __restrict__ kp, int T,
                                                             uint32_t* __restrict__ item_off,
                                                             uint32_t* __restrict__ queue,
                                                             uint32_t* __restrict__ done) {
    pdl_gate();
    __shared__ uint32_t ws[kItemsScanT / 32];
    const uint32_t k = *kp;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < 4) queue[threadIdx.x] = 0;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < k; c0 += kItemsScanT) {
        const uint32_t c = c0 + threadIdx.x;
        uint32_t v = 0;
        if (c < k) {
            const uint32_t n = off[c + 1] - off[c];
            v = n ? (n + (uint32_t)T - 1) / (uint32_t)T : 1u;
            if (done) done[3 * (size_t)c] = done[3 * (size_t)c + 1] = done[3 * (size_t)c + 2] = 0u;
        }
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) ws[w] = inc;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int q = 0; q < kItemsScanT / 32; ++q) {
            const uint32_t t = ws[q];
            wpre += q < w ? t : 0u;
            tot += t;
        }
        if (c < k) item_off[c] = carry + wpre + inc - v;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) item_off[k] = carry;
}

__global__ void k_pack(const uint32_t* __restrict__ off, const uint32_t* __restrict__ labels,
                       const uint32_t* __restrict__ kp, const FitCluster* __restrict__ cl,
                       const int2* __restrict__ hull, const uint32_t* __restrict__ hull_off,
                       vm_plane* __restrict__ planes, int32_t* __restrict__ hull_xy, float* __restrict__ hull_xyz,
                       uint32_t hull_cap, HeaderArgs ha) {
    pdl_gate();
    const uint32_t k = *kp;
    if (ha.out && blockIdx.x == 0 && threadIdx.x == 0) write_header(ha);
    for (uint32_t c = blockIdx.x; c < k; c += gridDim.x) {
        const uint32_t ho = hull_off[c];
        pack_cluster(cl[c], labels ? labels[c] : c, off[c + 1] - off[c], hull + off[c], ho, hull_off[c + 1] - ho,
                     planes + c, hull_xy, hull_xyz, hull_cap);
    }
}

// Stage b with one warp per work item (the schedule for many small
// clusters): each warp pulls its own items from the queue and stages the
// item's points in its own slice of shared memory; lanes hold R hypotheses
// each, 32 / ceil(H / R) lanes groups split the points, and the groups' counts
// are combined with shuffles before the integer atomics.  No CTA barrier.
template <int R>
__global__ void __launch_bounds__(kT) k_score_warp(const float* __restrict__ pts, const uint32_t* __restrict__ off,
                                                   const uint32_t* __restrict__ item_off,
                                                   const uint32_t* __restrict__ item_cl,
                                                   const uint32_t* __restrict__ kp, int H, int T,
                                                   const float4* __restrict__ hyp, uint32_t* __restrict__ counts,
                                                   uint32_t* __restrict__ queue, float eps) {
    pdl_wait();
    const uint32_t k = *kp;
    extern __shared__ float4 sp[];  // [kT / 32][T]
    const int lane = threadIdx.x & 31;
    float4* wp = sp + (size_t)(threadIdx.x >> 5) * T;
    const int G = (H + R - 1) / R;  // lanes per point group (<= 32, checked by the host)
    const int P = 32 / G;           // point groups per warp
    const int g = lane / G, j = lane % G;
    const bool active = g < P;
    const uint32_t n_items = item_off[k];
    for (int guard = 0; guard < kLoopCap; ++guard) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(queue, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const uint32_t c = find_cluster(item_cl, item_off, k, it);
        const uint32_t start = off[c] + (it - item_off[c]) * (uint32_t)T;
        const uint32_t end = min(off[c + 1], start + (uint32_t)T);
        const int cnt = (int)(end - start);
        __syncwarp();
        for (int q = lane; q < cnt; q += 32) {
            const float* p = pts + 3 * ((size_t)start + q);
            wp[q] = make_float4(p[0], p[1], p[2], 0.0f);
        }
        float4 pl[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int h = j * R + r;
            pl[r] = (active && h < H) ? hyp[(size_t)c * H + h]
                                      : make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0x7f800000));
        }
        __syncwarp();
        uint32_t acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0;
        if (active)
            for (int q = g; q < cnt; q += P) count_point<R>(pl, wp[q], eps, acc);
        for (int q = 1; q < P; ++q) {
            const int src = j + q * G;  // < 32 since P * G <= 32
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t v = __shfl_sync(0xffffffffu, acc[r], src);
                if (g == 0) acc[r] += v;
            }
        }
        if (g == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int h = j * R + r;
                if (h < H && acc[r]) atomicAdd(&counts[(size_t)c * H + h], acc[r]);
            }
        }
    }
}

// The scoring launch's arguments (stage b).
struct ScoreArgs {
    const float* pts;
    const uint32_t* off;
    const uint32_t* item_off;
    const uint32_t* item_cl;  // item -> cluster table, or null for a binary search
    const uint32_t* kp;
    int H, T;
    const float4* hyp;
    uint32_t* counts;
    uint32_t* queue;
    float eps;
    int grid;
};

template <int R>
cudaError_t launch_score(const ScoreArgs& a, cudaStream_t s) {
    const int G = (a.H + R - 1) / R;
    const int P = kT / G;
    const size_t smem = (size_t)a.T * sizeof(float4) + (size_t)P * G * R * sizeof(uint32_t);
    launch_full(k_score<R>, dim3(a.grid), dim3(kT), smem, s, a.pts, a.off, a.item_off, a.item_cl, a.kp, a.H, a.T,
                a.hyp, a.counts, a.queue, a.eps);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_score_warp(const ScoreArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)(kT / 32) * a.T * sizeof(float4);
    launch_full(k_score_warp<R>, dim3(a.grid), dim3(kT), smem, s, a.pts, a.off, a.item_off, a.item_cl, a.kp, a.H,
                a.T, a.hyp, a.counts, a.queue, a.eps);
    return cudaGetLastError();
}

__global__ void k_set_u32(uint32_t* __restrict__ p, uint32_t v) { pdl_gate(); *p = v; }

}  // namespace

FitTuning default_tuning() { return FitTuning{2048, 4, 4, 0}; }

// The scoring variant launch_fit picks for t and H: hypotheses per thread
// and whether the warp schedule applies.
static void score_variant(const FitTuning& t, int H, int& R, bool& warp) {
    R = t.hyp_per_thread;
    warp = t.schedule == 1 && H <= 256 && (size_t)(kT / 32) * t.tile * sizeof(float4) <= 200 * 1024;
    if (warp) {
        while (R < 8 && (H + R - 1) / R > 32) R <<= 1;
    } else {
        while (R < 8 && (H + R - 1) / R > kT) R <<= 1;
    }
}

int score_max_ctas_per_sm(const FitTuning& t, int H) {
    fit_init_attributes();
    int R;
    bool warp;
    score_variant(t, H, R, warp);
    const int G = (H + R - 1) / R;
    const size_t smem = warp ? (size_t)(kT / 32) * t.tile * sizeof(float4)
                             : (size_t)t.tile * sizeof(float4) + (size_t)(kT / G) * G * R * sizeof(uint32_t);
    int n = 0;
    cudaError_t e;
    if (warp) {
        switch (R) {
            case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score_warp<1>, kT, smem); break;
            case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score_warp<2>, kT, smem); break;
            case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score_warp<4>, kT, smem); break;
            default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score_warp<8>, kT, smem); break;
        }
    } else {
        switch (R) {
            case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score<1>, kT, smem); break;
            case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score<2>, kT, smem); break;
            case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score<8>, kT, smem); break;
            default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score<4>, kT, smem); break;
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

size_t fit_hull_smem() {
    return (size_t)kHullCap * (2 * sizeof(unsigned long long) + 2 * sizeof(uint32_t)) + (size_t)kSurvCap * sizeof(int2);
}

void fit_init_attributes() {
    static std::once_flag once;  // maps on several host threads may reach here together
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_hull, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fit_hull_smem());
        cudaFuncSetAttribute(k_score<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score_warp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score_warp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score_warp<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_score_warp<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
}

cudaError_t fit_set_count(uint32_t* kdev, uint32_t k, cudaStream_t s) {
    launch_k(k_set_u32, dim3(1), dim3(1), 0, s, kdev, k);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_fit(const float* pts, const uint32_t* off, const uint32_t* labels, const uint32_t* kp,
                       uint32_t kcap, const vm_segment_params& p, FitBuffers& fb, const FitTuning& t, int sms,
                       cudaStream_t s, StageHook* hk, uint32_t round) {
    if (kcap == 0) return cudaSuccess;
    fit_init_attributes();
    const int H = (int)p.n_hyp;
    const int T = (t.tile + (int)kChunk - 1) / (int)kChunk * (int)kChunk;  // callers validate; never below a chunk
    cudaError_t e;
    VM_STAGE_BEGIN(hk, kStHyp, s);
    if (kcap <= kItemsScanMax) {
        launch_k(k_items_scan, dim3(1), dim3(kItemsScanT), 0, s, off, kp, T, fb.item_off, fb.queue, fb.done);
        count_launch(1);
    } else {
        const unsigned kgrid = (kcap + kT - 1) / kT < (uint32_t)sms * 8 ? (kcap + kT - 1) / kT : (uint32_t)sms * 8;
        launch_k(k_items, dim3(kgrid), dim3(kT), 0, s, off, kp, T, fb.item_off, fb.queue, fb.done);
        e = exclusive_scan_dev(fb.item_off, fb.item_off, fb.tot, kp, kcap, fb.scan_tmp, s, fb.err, true);
        if (e != cudaSuccess) return e;
        count_launch(1);
    }
    const size_t kh = (size_t)kcap * H;
    const unsigned hgrid = (unsigned)((kh + kT - 1) / kT < (size_t)sms * 16 ? (kh + kT - 1) / kT : (size_t)sms * 16);
    launch_k(k_hyp, dim3(hgrid), dim3(kT), 0, s, pts, off, labels, kp, H, p.seed, round, fb.hyp, fb.hyp_valid,
             fb.counts, fb.item_off, fb.item_cl);
    VM_STAGE_END(hk, kStHyp, s);
    count_launch(1);
    const int grid = sms * t.ctas_per_sm;
    // The warp schedule needs ceil(H / R) <= 32 lanes with R <= 8 and its
    // per-warp tiles within the shared-memory limit; otherwise the CTA one
    // runs, with at most one subset row of kT threads.
    int R;
    bool warp;
    score_variant(t, H, R, warp);
    // Small fits (a map's segmentation) compute each cluster's centroid and
    // refit in the kernel before them, triggered by per-cluster completion
    // counters: that removes two dependent launches.  In large batches the
    // counters' fences wait, per work item, for the item's contended atomics,
    // which costs more than the launches; they take the separate kernels.
    // Results are the same.
    uint32_t* done = fb.npts_cap <= kFusedFitPoints ? fb.done : nullptr;
    VM_STAGE_BEGIN(hk, kStScore, s);
    const ScoreArgs sa{pts, off, fb.item_off, fb.item_cl, kp, H, T, fb.hyp, fb.counts, fb.queue, p.eps, grid};
    if (warp) {
        switch (R) {
            case 1: e = launch_score_warp<1>(sa, s); break;
            case 2: e = launch_score_warp<2>(sa, s); break;
            case 4: e = launch_score_warp<4>(sa, s); break;
            default: e = launch_score_warp<8>(sa, s); break;
        }
    } else {
        switch (R) {
            case 1: e = launch_score<1>(sa, s); break;
            case 2: e = launch_score<2>(sa, s); break;
            case 8: e = launch_score<8>(sa, s); break;
            default: e = launch_score<4>(sa, s); break;
        }
    }
    if (e != cudaSuccess) return e;
    VM_STAGE_END(hk, kStScore, s);
    count_launch(1);
    // stage c (k_select, a CTA per cluster), then the extraction; with the
    // completion counters the centroid runs in the extraction kernel and the
    // refit in the filter kernel, otherwise as kernels of their own
    const unsigned cgrid = kcap < (uint32_t)sms * 8 ? kcap : (uint32_t)sms * 8;
    VM_STAGE_BEGIN(hk, kStExtract, s);
    launch_k(k_select, dim3(cgrid), dim3(kT), 0, s, pts, off, kp, H, fb.hyp, fb.hyp_valid, fb.counts, fb.cl);
    count_launch(1);
    const unsigned igrid = (unsigned)sms * 8;
    launch_full(done ? k_extract<true> : k_extract<false>, dim3(igrid), dim3(kT), 0, s, pts, off, fb.item_off,
                fb.item_cl, kp, T, fb.cl, fb.inlier, fb.part, p.eps, fb.err, done, fb.cen);
    if (!done) {
        launch_k(k_centroid, dim3(cgrid), dim3(kT), 0, s, off, fb.item_off, kp, T, fb.part, fb.cl, fb.cen);
        count_launch(1);
    }
    launch_full(done ? k_filter<true> : k_filter<false>, dim3(igrid), dim3(kT), 0, s, pts, off, fb.item_off,
                fb.item_cl, kp, T, fb.cl, fb.inlier, fb.cen, fb.part, fb.surv, done);
    VM_STAGE_END(hk, kStExtract, s);
    count_launch(2);
    VM_STAGE_BEGIN(hk, kStHull, s);
    if (!done) {
        launch_k(k_refit, dim3(cgrid), dim3(kT), 0, s, off, fb.item_off, kp, T, fb.part, fb.cen, fb.cl);
        count_launch(1);
    }
    launch_k(k_hull, dim3(cgrid), dim3(kT), fit_hull_smem(), s, off, kp, fb.cl, fb.surv, fb.hull, fb.hull_cnt, fb.err,
             fb.queue + 3);
    VM_STAGE_END(hk, kStHull, s);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pack(const FitBuffers& fb, const uint32_t* off, const uint32_t* labels, const uint32_t* kp,
                        uint32_t kcap, vm_plane* planes, int32_t* hull_xy, float* hull_xyz, uint32_t hull_cap,
                        cudaStream_t s, const HeaderArgs* header) {
    if (kcap == 0) return cudaSuccess;
    const HeaderArgs ha = header ? *header : HeaderArgs{};
    launch_k(k_pack, dim3(kcap < 4096 ? kcap : 4096), dim3(128), 0, s, off, labels, kp, fb.cl, fb.hull, fb.hull_cnt,
             planes, hull_xy, hull_xyz, hull_cap, ha);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace vmx

// ---------------------------------------------------------------- no-allocation RANSAC
// vm_ransac_static runs the same hypothesis / scoring / selection kernels as
// vm_fit_planes, but every scratch buffer lives in one file-scope device array
// instead of memory obtained from cudaMalloc.  It exists for callers that may
// not allocate device memory once they are running -- a control loop with a
// hard deadline (cudaMalloc can block on device-wide synchronisation for an
// unbounded time), or a host program whose device memory is owned up front by
// another allocator.  The array is sized for at most kStaticMaxClusters
// clusters and kStaticMaxSlots (clusters x hypotheses); every GPU that loads
// the library holds it (about 11 MiB) until the process exits.
namespace vmx {
namespace {

constexpr uint32_t kStaticMaxClusters = 4096;
constexpr uint32_t kStaticMaxSlots = 524288;  // clusters x hypotheses

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffHyp = 0;
constexpr size_t kOffCounts = kOffHyp + align256((size_t)kStaticMaxSlots * sizeof(float4));
constexpr size_t kOffValid = kOffCounts + align256((size_t)kStaticMaxSlots * sizeof(uint32_t));
constexpr size_t kOffCl = kOffValid + align256((size_t)kStaticMaxSlots);
constexpr size_t kOffItems = kOffCl + align256((size_t)kStaticMaxClusters * sizeof(FitCluster));
constexpr size_t kOffQueue = kOffItems + align256((size_t)(kStaticMaxClusters + 1) * sizeof(uint32_t));
constexpr size_t kOffScan = kOffQueue + 256;  // the queue area also holds the count and a scan total
constexpr size_t kScanWords = 64;
static_assert(kScanWords >= scan_tmp_words(kStaticMaxClusters + 1), "static scan scratch too small");
constexpr size_t kStaticBytes = kOffScan + align256(kScanWords * sizeof(uint32_t));

// Copies the selected plane, hypothesis index and inlier count of each cluster
// to the caller's arrays.
__global__ void k_static_out(const FitCluster* __restrict__ cl, const uint32_t* __restrict__ kp,
                             float* __restrict__ planes, int32_t* __restrict__ best_h, uint32_t* __restrict__ inliers) {
    pdl_gate();
    const uint32_t k = *kp;
    for (uint32_t c = blockIdx.x * kT + threadIdx.x; c < k; c += gridDim.x * kT) {
        const FitCluster f = cl[c];
        planes[4 * c + 0] = f.n[0];
        planes[4 * c + 1] = f.n[1];
        planes[4 * c + 2] = f.n[2];
        planes[4 * c + 3] = f.d;
        best_h[c] = f.best_h;
        inliers[c] = f.best_h >= 0 ? f.inliers : 0u;
    }
}

}  // namespace
}  // namespace vmx

static __device__ __align__(256) unsigned char g_ransac_scratch[vmx::kStaticBytes];

namespace {
// Device address of g_ransac_scratch per device ordinal, looked up once per
// device (with that device current) by the first call made on it.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};
}  // namespace

extern "C" vm_status vm_ransac_static(const float* xyz, const uint32_t* off, const uint32_t* labels, uint32_t k,
                                      const vm_segment_params* params, void* stream, float* planes_out,
                                      int32_t* best_h_out, uint32_t* inliers_out) {
    using namespace vmx;
    if (!params || (k && (!xyz || !off || !planes_out || !best_h_out || !inliers_out))) {
        set_error("vm_ransac_static: null argument");
        return VM_ERR_INVALID_ARG;
    }
    if (params->n_hyp < 1 || params->n_hyp > 1024 || !(params->eps >= 0.0f) || params->planes_per_cluster > 1) {
        set_error("vm_ransac_static: n_hyp must be in [1, 1024], eps >= 0 and planes_per_cluster <= 1");
        return VM_ERR_INVALID_ARG;
    }
    if (k > kStaticMaxClusters || (uint64_t)k * params->n_hyp > kStaticMaxSlots) {
        set_error("vm_ransac_static: " + std::to_string(k) + " clusters x " + std::to_string(params->n_hyp) +
                  " hypotheses exceed the static scratch (at most " + std::to_string(kStaticMaxClusters) +
                  " clusters and " + std::to_string(kStaticMaxSlots) + " cluster-hypothesis pairs)");
        return VM_ERR_CAPACITY;
    }
    // The address lookup comes before the k == 0 return, so an empty call
    // serves as the set-up call that loads the array on this device.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("vm_ransac_static: device ordinal out of range");
        return VM_ERR_INVALID_ARG;
    }
    char* base;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_ransac_scratch);
            if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_ransac_scratch)");
            g_static_addr[dev] = p;
        }
        base = static_cast<char*>(g_static_addr[dev]);
    }
    if (k == 0) return VM_OK;
    const int H = (int)params->n_hyp;
    const FitTuning t = default_tuning();
    float4* hyp = reinterpret_cast<float4*>(base + kOffHyp);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
    uint8_t* valid = reinterpret_cast<uint8_t*>(base + kOffValid);
    FitCluster* cl = reinterpret_cast<FitCluster*>(base + kOffCl);
    uint32_t* item_off = reinterpret_cast<uint32_t*>(base + kOffItems);
    uint32_t* queue = reinterpret_cast<uint32_t*>(base + kOffQueue);
    uint32_t* kdev = queue + 8;
    uint32_t* total = queue + 9;
    uint32_t* scan_tmp = reinterpret_cast<uint32_t*>(base + kOffScan);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    fit_init_attributes();
    // the work queue starts at zero every call (k_items); counts are zeroed by k_hyp
    launch_k(k_set_u32, dim3(1), dim3(1), 0, s, kdev, k);
    launch_k(k_items, dim3((k + kT - 1) / kT), dim3(kT), 0, s, off, kdev, t.tile, item_off, queue,
             static_cast<uint32_t*>(nullptr));
    if ((e = exclusive_scan_dev(item_off, item_off, total, kdev, k, scan_tmp, s, nullptr, true)) != cudaSuccess)
        return cuda_status(e, "scan");
    const size_t kh = (size_t)k * H;
    const unsigned hgrid = (unsigned)((kh + kT - 1) / kT < (size_t)sms * 16 ? (kh + kT - 1) / kT : (size_t)sms * 16);
    launch_k(k_hyp, dim3(hgrid), dim3(kT), 0, s, xyz, off, labels, kdev, H, params->seed, 0u, hyp, valid, counts,
             item_off, static_cast<uint32_t*>(nullptr));
    // The CTA-per-item schedule whatever the tuning asks for: with no
    // item -> cluster table here, the clusters of work items come from a
    // binary search, which only that schedule does.
    FitTuning tc = t;
    tc.schedule = 0;
    int R;
    bool warp;
    score_variant(tc, H, R, warp);
    const int grid = sms * t.ctas_per_sm;
    const ScoreArgs sa{xyz, off, item_off, nullptr, kdev, H, t.tile, hyp, counts, queue, params->eps, grid};
    switch (R) {
        case 1: e = launch_score<1>(sa, s); break;
        case 2: e = launch_score<2>(sa, s); break;
        case 8: e = launch_score<8>(sa, s); break;
        default: e = launch_score<4>(sa, s); break;
    }
    if (e != cudaSuccess) return cuda_status(e, "k_score");
    const unsigned cgrid = k < (uint32_t)sms * 8 ? k : (uint32_t)sms * 8;
    launch_k(k_select, dim3(cgrid), dim3(kT), 0, s, xyz, off, kdev, H, hyp, valid, counts, cl);
    launch_k(k_static_out, dim3((k + kT - 1) / kT), dim3(kT), 0, s, cl, kdev, planes_out, best_h_out, inliers_out);
    count_launch(6);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "vm_ransac_static launch");
    return VM_OK;
}
