// scan.cu -- device-wide exclusive prefix sum and a stable LSD radix sort of
// (uint32 key, uint32 value) pairs.  These order the bricks and voxels by id,
// number the kept clusters and lay the cluster members out contiguously in
// voxel-id order (Sec. III.C: points sharing a label are grouped as clusters).
#include "vm_internal.cuh"

namespace vmx {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x == kScanThreads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_sums, uint32_t* block_total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = (lane < kScanThreads / 32) ? warp_sums[lane] : 0u;
        uint32_t si = warp_incl_scan(s);
        if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *block_total = si;
    }
    __syncthreads();
    return inc - v + warp_sums[w];
}

// n_dev (optional): the element count read on the device, clamped to n.
__device__ __forceinline__ size_t dev_count(size_t n, const uint32_t* n_dev) {
    if (!n_dev) return n;
    const size_t d = *n_dev;
    return d < n ? d : n;
}

// Single-pass scan with decoupled look-back (Merrill and Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016).  Each CTA takes the
// next tile from a ticket counter (so every earlier tile belongs to a CTA that
// has started), publishes its tile sum, then walks back over earlier tiles'
// published words until it meets an inclusive prefix, and publishes its own.
// A status word is (epoch << 34 | flag << 32 | value), a 30-bit epoch: words
// of an earlier launch (another epoch) read as not yet published, so no
// clearing pass is needed; the last CTA to finish resets the ticket and
// advances the epoch.
// The state (ticket, done, epoch, then one 64-bit word per tile) must start
// zeroed once, when its memory is allocated.  Every wait is bounded: a wait
// that runs out sets kErrTimeout in *err and counts the missing prefix as 0.
constexpr unsigned long long kFlagAgg = 1ull, kFlagInc = 2ull;
constexpr int kLookbackCap = 1 << 20;

constexpr uint32_t kEpochMask = (1u << 30) - 1u;
__device__ __forceinline__ unsigned long long lb_word(uint32_t epoch, unsigned long long flag, uint32_t v) {
    return ((unsigned long long)(epoch & kEpochMask) << 34) | (flag << 32) | (unsigned long long)v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_lookback(const uint32_t* in, uint32_t* out, size_t n_cap,
                                                                const uint32_t* __restrict__ n_dev,
                                                                uint32_t* __restrict__ total,
                                                                uint32_t* __restrict__ state, uint32_t* err, int end) {
    pdl_gate();
    __shared__ uint32_t buf[kScanTile];
    __shared__ uint32_t ws[kScanThreads / 32];
    __shared__ uint32_t tot, s_tile, s_prefix;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(state + 4);
    const size_t n = dev_count(n_cap, n_dev);
    const uint32_t nt_used = (uint32_t)((n + kScanTile - 1) / kScanTile);
    const uint32_t epoch = *(volatile uint32_t*)(state + 2);
    if (threadIdx.x == 0) s_tile = atomicAdd(state, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile < nt_used) {
        const size_t base = (size_t)tile * kScanTile;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int t = i * kScanThreads + threadIdx.x;
            const size_t j = base + t;
            buf[t] = (j < n) ? in[j] : 0u;
        }
        __syncthreads();
        uint32_t v[kScanItems];
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = buf[threadIdx.x * kScanItems + i];
            sum += v[i];
        }
        const uint32_t ex_local = block_excl_scan(sum, ws, &tot);
        if (threadIdx.x == 0) {
            const uint32_t agg = tot;
            uint32_t prefix = 0;
            if (tile == 0) {
                atomicExch(status, lb_word(epoch, kFlagInc, agg));
            } else {
                atomicExch(status + tile, lb_word(epoch, kFlagAgg, agg));
                for (int64_t p = (int64_t)tile - 1; p >= 0; --p) {
                    unsigned long long w = 0;
                    int it = 0;
                    for (; it < kLookbackCap; ++it) {
                        w = *(volatile unsigned long long*)(status + p);
                        if ((uint32_t)(w >> 34) == (epoch & kEpochMask) && ((w >> 32) & 3ull)) break;
                    }
                    if (it == kLookbackCap) {  // the predecessor never published: report, count it as 0
                        if (err) atomicOr(err, kErrTimeout);
                        break;
                    }
                    prefix += (uint32_t)(w & 0xffffffffull);
                    if (((w >> 32) & 3ull) == kFlagInc) break;
                }
                atomicExch(status + tile, lb_word(epoch, kFlagInc, prefix + agg));
            }
            s_prefix = prefix;
            if (tile == nt_used - 1) {
                if (total) *total = prefix + agg;
                if (end) out[n] = prefix + agg;  // no tile reads in[n]
            }
        }
        __syncthreads();
        uint32_t ex = ex_local + s_prefix;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            buf[threadIdx.x * kScanItems + i] = ex;
            ex += v[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int t = i * kScanThreads + threadIdx.x;
            const size_t j = base + t;
            if (j < n) out[j] = buf[t];
        }
    } else if (tile == 0 && threadIdx.x == 0) {  // nothing to scan
        if (total) *total = 0;
        if (end) out[0] = 0;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(state + 1, 1u) == gridDim.x - 1) {  // the last CTA: reset for the next launch
            state[0] = 0;
            state[1] = 0;
            state[2] = epoch + 1;
            __threadfence();
        }
    }
}

// The allocated bricks in key order in one pass (a stream compaction with the
// look-back scan above): tile t of the brick table flags its allocated
// entries (slot >= 0), ranks them within the tile, looks back for the count
// of allocated bricks before the tile, then writes every entry's rank (or -1)
// and, per allocated brick, its slot and key at its rank.  The last tile
// writes the count.  Block 0 also clears the words clear[1 .. n_clear) (a
// counter block whose word 0 is the count) and zero0 / zero1 (may be null).
__global__ void __launch_bounds__(kScanThreads) k_order_bricks(const int32_t* __restrict__ table, uint32_t nb,
                                                               int32_t* __restrict__ rank_table,
                                                               int32_t* __restrict__ sorted_slot,
                                                               int32_t* __restrict__ sorted_key,
                                                               uint32_t* __restrict__ clear, int n_clear,
                                                               uint32_t* __restrict__ zero0,
                                                               uint32_t* __restrict__ zero1,
                                                               uint32_t* __restrict__ state, uint32_t* err) {
    pdl_gate();
    __shared__ int32_t buf[kScanTile];
    __shared__ uint32_t ws[kScanThreads / 32];
    __shared__ uint32_t tot, s_tile, s_prefix;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(state + 4);
    if (blockIdx.x == 0) {
        for (int i = 1 + threadIdx.x; i < n_clear; i += kScanThreads) clear[i] = 0u;
        if (threadIdx.x == 0) {
            if (zero0) *zero0 = 0u;
            if (zero1) *zero1 = 0u;
        }
    }
    const uint32_t nt_used = (nb + kScanTile - 1) / kScanTile;
    const uint32_t epoch = *(volatile uint32_t*)(state + 2);
    if (threadIdx.x == 0) s_tile = atomicAdd(state, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile < nt_used) {
        const uint32_t base = tile * kScanTile;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const uint32_t j = base + i * kScanThreads + threadIdx.x;
            buf[i * kScanThreads + threadIdx.x] = j < nb ? table[j] : -1;
        }
        __syncthreads();
        int32_t v[kScanItems];
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = buf[threadIdx.x * kScanItems + i];
            sum += v[i] >= 0;
        }
        const uint32_t ex_local = block_excl_scan(sum, ws, &tot);
        if (threadIdx.x == 0) {
            const uint32_t agg = tot;
            uint32_t prefix = 0;
            if (tile == 0) {
                atomicExch(status, lb_word(epoch, kFlagInc, agg));
            } else {
                atomicExch(status + tile, lb_word(epoch, kFlagAgg, agg));
                for (int64_t p = (int64_t)tile - 1; p >= 0; --p) {
                    unsigned long long w = 0;
                    int it = 0;
                    for (; it < kLookbackCap; ++it) {
                        w = *(volatile unsigned long long*)(status + p);
                        if ((uint32_t)(w >> 34) == (epoch & kEpochMask) && ((w >> 32) & 3ull)) break;
                    }
                    if (it == kLookbackCap) {  // the predecessor never published: report, count it as 0
                        if (err) atomicOr(err, kErrTimeout);
                        break;
                    }
                    prefix += (uint32_t)(w & 0xffffffffull);
                    if (((w >> 32) & 3ull) == kFlagInc) break;
                }
                atomicExch(status + tile, lb_word(epoch, kFlagInc, prefix + agg));
            }
            s_prefix = prefix;
            if (tile == nt_used - 1) clear[0] = prefix + agg;
        }
        __syncthreads();
        uint32_t rank = ex_local + s_prefix;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const uint32_t j = base + threadIdx.x * kScanItems + i;
            if (j < nb) {
                if (v[i] >= 0) {
                    sorted_slot[rank] = v[i];
                    sorted_key[rank] = (int32_t)j;
                    rank_table[j] = (int32_t)rank;
                    ++rank;
                } else {
                    rank_table[j] = -1;
                }
            }
        }
    } else if (tile == 0 && threadIdx.x == 0) {  // an empty table
        clear[0] = 0u;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(state + 1, 1u) == gridDim.x - 1) {  // the last CTA: reset for the next launch
            state[0] = 0;
            state[1] = 0;
            state[2] = epoch + 1;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortIters = 8;                               // 32-item rounds per warp
constexpr int kSortTile = kSortThreads * kSortIters;        // 2048

// Pass `pass` of the sort runs only when some key reaches its digit: with a
// device bound kb on the keys (every key < kb), pass p > 0 runs iff
// kb > 2^(8p).  Tiles past the device count do nothing; the histograms are
// laid out digit-major over the used tiles only, and *cnt receives their
// count (the scan's length).
__device__ __forceinline__ bool rs_pass_active(const uint32_t* kb, int pass) {
    return pass == 0 || !kb || (unsigned long long)*kb > (1ull << (8 * pass));
}

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, size_t n_cap, const uint32_t* __restrict__ n_dev, int pass,
                          const uint32_t* __restrict__ kb, uint32_t* __restrict__ ghist, uint32_t* __restrict__ cnt) {
    pdl_gate();
    __shared__ uint32_t h[256];
    const bool active = rs_pass_active(kb, pass);
    const size_t n = active ? dev_count(n_cap, n_dev) : 0;
    const size_t ntu = (n + kSortTile - 1) / kSortTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = (uint32_t)(256 * ntu);
    if (blockIdx.x >= ntu) return;
    const int shift = 8 * pass;
    h[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortIters; ++i) {
        size_t j = base + (size_t)i * kSortThreads + threadIdx.x;
        if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    ghist[(size_t)threadIdx.x * ntu + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w owns items [w*256, w*256+256) of the tile, in order.
__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, size_t n_cap,
                             const uint32_t* __restrict__ n_dev, int pass, const uint32_t* __restrict__ kb,
                             const uint32_t* __restrict__ goff) {
    pdl_gate();
    __shared__ uint32_t wc[kSortWarps][256];
    if (!rs_pass_active(kb, pass)) return;
    const size_t n = dev_count(n_cap, n_dev);
    if ((size_t)blockIdx.x * kSortTile >= n) return;
    const size_t nt = (n + kSortTile - 1) / kSortTile;  // used tiles: the histogram stride
    const int shift = 8 * pass;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&wc[0][0])[d] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * kSortTile + (size_t)w * (32 * kSortIters);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t rank[kSortIters], dig[kSortIters];
#pragma unroll
    for (int i = 0; i < kSortIters; ++i) {
        size_t j = base + (size_t)i * 32 + lane;
        uint32_t d = (j < n) ? ((kin[j] >> shift) & 255u) : 256u;
        dig[i] = d;
        uint32_t m = __match_any_sync(0xffffffffu, d);
        uint32_t r = __popc(m & lt);
        uint32_t b = (d < 256u) ? wc[w][d] : 0u;
        __syncwarp();
        if (d < 256u && r == 0) wc[w][d] = b + __popc(m);
        __syncwarp();
        rank[i] = b + r;
    }
    __syncthreads();
    {   // exclusive offsets of each warp per digit
        const int d = threadIdx.x;  // kSortThreads == 256 digits
        uint32_t run = 0;
        for (int q = 0; q < kSortWarps; ++q) {
            uint32_t t = wc[q][d];
            wc[q][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortIters; ++i) {
        size_t j = base + (size_t)i * 32 + lane;
        if (j < n) {
            uint32_t d = dig[i];
            uint32_t pos = goff[(size_t)d * nt + blockIdx.x] + wc[w][d] + rank[i];
            kout[pos] = kin[j];
            vout[pos] = vin[j];
        }
    }
}

// Small inputs: one 1024-thread CTA scans everything, four items per thread
// per round, carrying the running total across rounds.
constexpr int kSmallThreads = 1024;
constexpr int kSmallItems = 4;
constexpr size_t kSmallMax = 16384;

__global__ void __launch_bounds__(kSmallThreads) k_scan_small(const uint32_t* in, uint32_t* out, size_t n_cap,
                                                              const uint32_t* __restrict__ n_dev, uint32_t* total,
                                                              int end) {
    pdl_gate();
    __shared__ uint32_t ws[kSmallThreads / 32];
    __shared__ uint32_t round_total;
    const size_t n = dev_count(n_cap, n_dev);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (size_t base = 0; base < n; base += (size_t)kSmallThreads * kSmallItems) {
        const size_t j0 = base + (size_t)threadIdx.x * kSmallItems;
        uint32_t v[kSmallItems], sum = 0;
#pragma unroll
        for (int i = 0; i < kSmallItems; ++i) {
            v[i] = (j0 + i < n) ? in[j0 + i] : 0u;
            sum += v[i];
        }
        const uint32_t inc = warp_incl_scan(sum);
        if (lane == 31) ws[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint32_t t = ws[lane];
            const uint32_t ti = warp_incl_scan(t);
            ws[lane] = ti - t;
            if (lane == 31) round_total = ti;
        }
        __syncthreads();
        uint32_t ex = carry + ws[w] + (inc - sum);
#pragma unroll
        for (int i = 0; i < kSmallItems; ++i) {
            if (j0 + i < n) out[j0 + i] = ex;
            ex += v[i];
        }
        carry += round_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (total) *total = carry;
        if (end) out[n] = carry;  // read by no thread: every load is below n
    }
}

// Two arrays of the same length scanned by one CTA (as k_scan_small, both at once).
__global__ void __launch_bounds__(kSmallThreads) k_scan2_small(const uint32_t* in0, uint32_t* out0, uint32_t* total0,
                                                               const uint32_t* in1, uint32_t* out1, uint32_t* total1,
                                                               size_t n_cap, const uint32_t* __restrict__ n_dev) {
    pdl_gate();
    __shared__ uint32_t ws[2][kSmallThreads / 32];
    __shared__ uint32_t round_total[2];
    const size_t n = dev_count(n_cap, n_dev);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry0 = 0, carry1 = 0;
    for (size_t base = 0; base < n; base += (size_t)kSmallThreads * kSmallItems) {
        const size_t j0 = base + (size_t)threadIdx.x * kSmallItems;
        uint32_t v0[kSmallItems], v1[kSmallItems], sum0 = 0, sum1 = 0;
#pragma unroll
        for (int i = 0; i < kSmallItems; ++i) {
            v0[i] = (j0 + i < n) ? in0[j0 + i] : 0u;
            v1[i] = (j0 + i < n) ? in1[j0 + i] : 0u;
            sum0 += v0[i];
            sum1 += v1[i];
        }
        const uint32_t inc0 = warp_incl_scan(sum0), inc1 = warp_incl_scan(sum1);
        if (lane == 31) {
            ws[0][w] = inc0;
            ws[1][w] = inc1;
        }
        __syncthreads();
        if (w < 2) {
            const uint32_t t = ws[w][lane];
            const uint32_t ti = warp_incl_scan(t);
            ws[w][lane] = ti - t;
            if (lane == 31) round_total[w] = ti;
        }
        __syncthreads();
        uint32_t ex0 = carry0 + ws[0][w] + (inc0 - sum0), ex1 = carry1 + ws[1][w] + (inc1 - sum1);
#pragma unroll
        for (int i = 0; i < kSmallItems; ++i) {
            if (j0 + i < n) {
                out0[j0 + i] = ex0;
                out1[j0 + i] = ex1;
            }
            ex0 += v0[i];
            ex1 += v1[i];
        }
        carry0 += round_total[0];
        carry1 += round_total[1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (total0) *total0 = carry0;
        if (total1) *total1 = carry1;
    }
}

}  // namespace

static_assert((size_t)kScanTile == kScanTileElems, "scan_tmp_words assumes the scan's tile size");

cudaError_t exclusive_scan2_dev(const uint32_t* in0, uint32_t* out0, uint32_t* total0, const uint32_t* in1,
                                uint32_t* out1, uint32_t* total1, const uint32_t* n_dev, size_t n_cap, uint32_t* tmp,
                                cudaStream_t s, uint32_t* err) {
    if (n_cap > 0 && n_cap <= kSmallMax) {
        launch_k(k_scan2_small, dim3(1), dim3(kSmallThreads), 0, s, in0, out0, total0, in1, out1, total1, n_cap,
                 n_dev);
        count_launch(1);
        return cudaGetLastError();
    }
    cudaError_t e = exclusive_scan_dev(in0, out0, total0, n_dev, n_cap, tmp, s, err);
    if (e != cudaSuccess) return e;
    return exclusive_scan_dev(in1, out1, total1, n_dev, n_cap, tmp, s, err);
}

cudaError_t exclusive_scan_dev(const uint32_t* in, uint32_t* out, uint32_t* total, const uint32_t* n_dev, size_t n_cap,
                               uint32_t* tmp, cudaStream_t s, uint32_t* err, bool end) {
    if (n_cap == 0) {
        cudaError_t e = cudaSuccess;
        if (total) e = cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        if (end && e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return e;
    }
    if (n_cap <= kSmallMax) {
        launch_k(k_scan_small, dim3(1), dim3(kSmallThreads), 0, s, in, out, n_cap, n_dev, total, (int)end);
        count_launch(1);
        return cudaGetLastError();
    }
    if (reinterpret_cast<uintptr_t>(tmp) & 7) return cudaErrorInvalidValue;  // 64-bit status words
    const size_t nt = (n_cap + kScanTile - 1) / kScanTile;
    launch_k(k_scan_lookback, dim3((unsigned)nt), dim3(kScanThreads), 0, s, in, out, n_cap, n_dev, total, tmp, err,
             (int)end);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t order_bricks_dev(const int32_t* table, uint32_t nb, int32_t* rank_table, int32_t* sorted_slot,
                             int32_t* sorted_key, uint32_t* clear, int n_clear, uint32_t* zero0, uint32_t* zero1,
                             uint32_t* tmp, cudaStream_t s, uint32_t* err) {
    if (reinterpret_cast<uintptr_t>(tmp) & 7) return cudaErrorInvalidValue;  // 64-bit status words
    const size_t nt = ((size_t)nb + kScanTile - 1) / kScanTile;
    launch_k(k_order_bricks, dim3((unsigned)(nt ? nt : 1)), dim3(kScanThreads), 0, s, table, nb, rank_table,
             sorted_slot, sorted_key, clear, n_clear, zero0, zero1, tmp, err);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint32_t* total, size_t n, uint32_t* tmp,
                               cudaStream_t s, uint32_t* err) {
    return exclusive_scan_dev(in, out, total, nullptr, n, tmp, s, err);
}

size_t sort_tmp_words(size_t n) {
    const size_t nt = (n + kSortTile - 1) / kSortTile;
    return 256 * nt + 64 + scan_tmp_words(256 * nt);
}

cudaError_t stable_sort_pairs_dev(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                  const uint32_t* n_dev, size_t n_cap, int bits, uint32_t* tmp, cudaStream_t s,
                                  uint32_t* err, const uint32_t* key_bound) {
    if (n_cap == 0 || bits <= 0) return cudaSuccess;
    const size_t nt = (n_cap + kSortTile - 1) / kSortTile;
    uint32_t* ghist = tmp;
    uint32_t* cnt = tmp + 256 * nt;          // the histogram scan's length (device)
    uint32_t* stmp = tmp + 256 * nt + 64;    // its look-back state
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        launch_k(k_rs_hist, dim3((unsigned)nt), dim3(kSortThreads), 0, s, ki, n_cap, n_dev, p, key_bound, ghist, cnt);
        cudaError_t e = exclusive_scan_dev(ghist, ghist, nullptr, cnt, 256 * nt, stmp, s, err);
        if (e != cudaSuccess) return e;
        launch_k(k_rs_scatter, dim3((unsigned)nt), dim3(kSortThreads), 0, s, ki, vi, ko, vo, n_cap, n_dev, p, key_bound,
                 ghist);
        count_launch(2);
        uint32_t* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (!key_bound && ki != keys) {  // odd number of passes: copy back (n_cap elements; the tail is scratch)
        cudaMemcpyAsync(keys, ki, n_cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vi, n_cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

cudaError_t stable_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, size_t n,
                                  int bits, uint32_t* tmp, cudaStream_t s, uint32_t* err) {
    return stable_sort_pairs_dev(keys, vals, keys_alt, vals_alt, nullptr, n, bits, tmp, s, err, nullptr);
}

}  // namespace vmx
