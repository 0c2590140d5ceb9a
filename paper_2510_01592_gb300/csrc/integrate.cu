// integrate.cu -- voxel information update (Sec. III.B, Eq. 1), one thread per
// sensor point.
//
// Storage: a direct-indexed brick table (one int32 per 8^3-voxel brick of the
// grid) maps a brick to a slot of a pool allocated on first touch.  A slot
// holds, per voxel, the exact fixed-point coordinate sums S (int64, 2^-20 m
// units relative to the window's anchor) and the point count C.  Eq. 1's
// running mean is the ratio S / C, independent of the order the points arrive
// in, so concurrent updates need only integer atomics.
//
// The grid is a window over voxel keys floor((p - origin) * inv_res) taken
// from the map's fixed base origin (Sec. III.B: the map's centre follows the
// robot): the window moves in whole bricks (launch_scroll), so a voxel keeps
// its key, its points and its exact sums for as long as it stays inside.
//
// One pass over a frame's points (k_accum): a point whose brick is
// unallocated claims it with a CAS on the table entry (the winner takes a
// pool slot); each warp groups its points by voxel (a match over the voxel
// key, wherever the points sit in the warp), reduces each group's integer
// sums, and the group's lowest lane issues one 64-bit atomic per axis plus
// one 32-bit count atomic.  The few points whose brick another thread was
// claiming at that moment are deferred to a second, small kernel
// (k_accum_deferred), so no thread ever waits on another.
#include "vm_internal.cuh"

namespace vmx {
namespace {

constexpr int kThreads = 256;

struct Keyed {
    int ok;
    uint32_t brick;   // linear brick key
    uint32_t local;   // voxel index inside the brick
    int32_t F[3];     // rint(d * 2^20), d = offset from the map origin
};

// Transform, key and quantise one point.  The op sequence is the reading of
// Sec. III.B: fma chain for R p + t, subtract the origin, floor(d * inv_res).
__device__ __forceinline__ Keyed key_point(const float* __restrict__ xyz, uint32_t i, const Pose& P, const Grid& g) {
    Keyed k;
    const float x = xyz[3 * (size_t)i + 0], y = xyz[3 * (size_t)i + 1], z = xyz[3 * (size_t)i + 2];
    const float wx = __fmaf_rn(P.r[2], z, __fmaf_rn(P.r[1], y, __fmaf_rn(P.r[0], x, P.r[3])));
    const float wy = __fmaf_rn(P.r[6], z, __fmaf_rn(P.r[5], y, __fmaf_rn(P.r[4], x, P.r[7])));
    const float wz = __fmaf_rn(P.r[10], z, __fmaf_rn(P.r[9], y, __fmaf_rn(P.r[8], x, P.r[11])));
    const float dx = __fsub_rn(wx, g.ox), dy = __fsub_rn(wy, g.oy), dz = __fsub_rn(wz, g.oz);
    const float fx = floorf(__fmul_rn(dx, g.inv_res));
    const float fy = floorf(__fmul_rn(dy, g.inv_res));
    const float fz = floorf(__fmul_rn(dz, g.inv_res));
    // window bounds: integers below 2^24, exact as floats
    k.ok = (fx >= (float)g.wx) & (fx < (float)(g.wx + g.nx)) & (fy >= (float)g.wy) & (fy < (float)(g.wy + g.ny)) &
           (fz >= (float)g.wz) & (fz < (float)(g.wz + g.nz));
    if (k.ok) {
        const int ix = (int)fx - g.wx, iy = (int)fy - g.wy, iz = (int)fz - g.wz;
        k.brick = ((uint32_t)(iz >> 3) * (uint32_t)g.nby + (uint32_t)(iy >> 3)) * (uint32_t)g.nbx + (uint32_t)(ix >> 3);
        k.local = (uint32_t)((((iz & 7) << 3) | (iy & 7)) << 3 | (ix & 7));
        k.F[0] = (int32_t)(__float2ll_rn(__fmul_rn(dx, 1048576.0f)) - g.ax);
        k.F[1] = (int32_t)(__float2ll_rn(__fmul_rn(dy, 1048576.0f)) - g.ay);
        k.F[2] = (int32_t)(__float2ll_rn(__fmul_rn(dz, 1048576.0f)) - g.az);
    } else {
        k.brick = kNone;
        k.local = 0;
        k.F[0] = k.F[1] = k.F[2] = 0;
    }
    return k;
}

// Adds a warp's points to their voxels: lanes with equal keys (kNone: no
// point) form a group wherever they sit in the warp (a raster camera gives
// runs of consecutive lanes, a spinning LiDAR's beams interleave); each
// group's integer sums are reduced and its lowest lane issues the group's
// atomics (64-bit sums sign-extended: a group's sum is negative when its
// points lie a quantum below the window's anchor).
__device__ __forceinline__ void accumulate_warp(uint32_t key, int32_t v0, int32_t v1, int32_t v2,
                                                unsigned long long* __restrict__ S, uint32_t* __restrict__ C) {
    if (!__any_sync(0xffffffffu, key != kNone)) return;  // nothing in this warp lands in the map
    const uint32_t grp = __match_any_sync(0xffffffffu, key);
    const int32_t s0 = __reduce_add_sync(grp, v0), s1 = __reduce_add_sync(grp, v1), s2 = __reduce_add_sync(grp, v2);
    if (key != kNone && (int)(threadIdx.x & 31) == __ffs(grp) - 1) {
        const uint32_t slot = key / kBrickVox, l = key % kBrickVox;
        unsigned long long* s = S + (size_t)slot * 3 * kBrickVox + l;
        atomicAdd(s, (unsigned long long)(long long)s0);
        atomicAdd(s + kBrickVox, (unsigned long long)(long long)s1);
        atomicAdd(s + 2 * kBrickVox, (unsigned long long)(long long)s2);
        atomicAdd(C + key, (uint32_t)__popc(grp));
    }
}

// Per-warp totals of accepted / dropped points into the map's counters.
__device__ __forceinline__ void count_points(uint32_t n_ok, uint32_t n_bad, uint32_t n_full,
                                             MapCounters* __restrict__ ctr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_ok += __shfl_xor_sync(0xffffffffu, n_ok, o);
        n_bad += __shfl_xor_sync(0xffffffffu, n_bad, o);
        n_full += __shfl_xor_sync(0xffffffffu, n_full, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_ok) atomicAdd(&ctr->integrated, (unsigned long long)n_ok);
        if (n_bad) atomicAdd(&ctr->dropped, (unsigned long long)n_bad);
        if (n_full) atomicAdd(&ctr->no_capacity, (unsigned long long)n_full);
    }
}

// One pass over the frame's points: a point whose brick is unallocated
// claims it (a CAS on the table entry from -1 to -2; the winner takes a pool
// slot and publishes it), a point whose brick has a slot is accumulated, and
// a point whose brick another thread is claiming right now is put on the
// deferred list (one atomic; no thread ever waits on another) for
// k_accum_deferred, after which every claim is published.
__global__ void __launch_bounds__(kThreads) k_accum(const float* __restrict__ xyz, uint32_t n, Pose P, Grid g,
                                                   int32_t* __restrict__ table, int32_t* __restrict__ slot_key,
                                                   unsigned long long* __restrict__ S, uint32_t* __restrict__ C,
                                                   uint32_t* __restrict__ deferred, MapCounters* __restrict__ ctr,
                                                   uint32_t capacity) {
    pdl_gate();
    const int lane = threadIdx.x & 31;
    const uint32_t warp_global = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * kThreads) >> 5;
    uint32_t n_ok = 0, n_bad = 0, n_full = 0;
    for (uint32_t base = warp_global * 32u; base < n; base += n_warps * 32u) {
        const uint32_t i = base + lane;
        uint32_t key = kNone;
        int32_t v0 = 0, v1 = 0, v2 = 0;
        if (i < n) {
            Keyed k = key_point(xyz, i, P, g);
            if (k.ok) {
                int32_t slot = table[k.brick];
                if (slot == -1) {  // unallocated: claim it, or find another thread claiming it
                    if (atomicCAS(&table[k.brick], -1, -2) == -1) {
                        const uint32_t sl = atomicAdd(&ctr->n_bricks, 1u);
                        if (sl < capacity) {
                            slot_key[sl] = (int32_t)k.brick;
                            table[k.brick] = (int32_t)sl;
                            slot = (int32_t)sl;
                        } else {
                            table[k.brick] = -3;  // pool full: the brick's points are dropped and counted
                            atomicOr(&ctr->err, kErrCapacity);
                            slot = -3;
                        }
                    } else {
                        slot = -2;
                    }
                }
                if (slot >= 0) {
                    key = (uint32_t)slot * kBrickVox + k.local;
                    v0 = k.F[0]; v1 = k.F[1]; v2 = k.F[2];
                    ++n_ok;
                } else if (slot == -2) {
                    deferred[atomicAdd(&ctr->n_deferred, 1u)] = i;
                } else {
                    ++n_full;
                }
            } else {
                ++n_bad;
            }
        }
        accumulate_warp(key, v0, v1, v2, S, C);
    }
    count_points(n_ok, n_bad, n_full, ctr);
}

// The deferred points, their bricks' claims now published; the last CTA to
// finish clears the list for the next frame.
__global__ void __launch_bounds__(kThreads) k_accum_deferred(const float* __restrict__ xyz, Pose P, Grid g,
                                                            const int32_t* __restrict__ table,
                                                            unsigned long long* __restrict__ S,
                                                            uint32_t* __restrict__ C,
                                                            const uint32_t* __restrict__ deferred,
                                                            MapCounters* __restrict__ ctr) {
    pdl_gate();
    __shared__ uint32_t s_last;
    const uint32_t nd = ctr->n_deferred;
    const uint32_t warp_global = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * kThreads) >> 5;
    uint32_t n_ok = 0, n_full = 0;
    for (uint32_t base = warp_global * 32u; base < nd; base += n_warps * 32u) {
        const uint32_t j = base + (threadIdx.x & 31);
        uint32_t key = kNone;
        int32_t v0 = 0, v1 = 0, v2 = 0;
        if (j < nd) {
            const Keyed k = key_point(xyz, deferred[j], P, g);
            const int32_t slot = table[k.brick];
            if (slot >= 0) {
                key = (uint32_t)slot * kBrickVox + k.local;
                v0 = k.F[0]; v1 = k.F[1]; v2 = k.F[2];
                ++n_ok;
            } else {
                ++n_full;
            }
        }
        accumulate_warp(key, v0, v1, v2, S, C);
    }
    count_points(n_ok, 0, n_full, ctr);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctr->deferred_done, 1u) + 1u == gridDim.x;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        ctr->n_deferred = 0;
        ctr->deferred_done = 0;
    }
}

// Eq. 2: one thread per point walks the point's ray from the sensor's voxel
// to the point's voxel (excluded): a monotone 6-connected walk, each step on
// the axis whose next voxel boundary comes first along the ray (ties to x,
// then y, then z) among the axes not yet at the end voxel's coordinate, all in
// FP32 with explicit round-to-nearest operations.  The walk stops when it
// leaves the grid (a monotone walk does not come back); the caller has
// checked that the sensor is inside the grid.  An occupied voxel on the walk
// gets its bit in the mark bitmap (a plain read skips the atomic when the bit
// is already set).
__global__ void __launch_bounds__(kThreads) k_clear_mark(const float* __restrict__ xyz, uint32_t n, Pose P, Grid g,
                                                        const int32_t* __restrict__ table,
                                                        const uint32_t* __restrict__ C, uint32_t* mark,
                                                        MapCounters* __restrict__ ctr) {
    pdl_gate();
    const float s[3] = {__fmul_rn(__fsub_rn(P.r[3], g.ox), g.inv_res), __fmul_rn(__fsub_rn(P.r[7], g.oy), g.inv_res),
                        __fmul_rn(__fsub_rn(P.r[11], g.oz), g.inv_res)};
    const int dims[3] = {g.nx, g.ny, g.nz};
    const int w0 = g.wx, w1 = g.wy, w2 = g.wz;
    const long long cap = (long long)g.nx + g.ny + g.nz + 3;  // a walk inside the grid is never longer
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const float x = xyz[3 * (size_t)i + 0], y = xyz[3 * (size_t)i + 1], z = xyz[3 * (size_t)i + 2];
        float e[3];
        e[0] = __fmul_rn(__fsub_rn(__fmaf_rn(P.r[2], z, __fmaf_rn(P.r[1], y, __fmaf_rn(P.r[0], x, P.r[3]))), g.ox),
                         g.inv_res);
        e[1] = __fmul_rn(__fsub_rn(__fmaf_rn(P.r[6], z, __fmaf_rn(P.r[5], y, __fmaf_rn(P.r[4], x, P.r[7]))), g.oy),
                         g.inv_res);
        e[2] = __fmul_rn(__fsub_rn(__fmaf_rn(P.r[10], z, __fmaf_rn(P.r[9], y, __fmaf_rn(P.r[8], x, P.r[11]))), g.oz),
                         g.inv_res);
        bool fin = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) fin &= isfinite(e[a]) && fabsf(e[a]) < 1073741824.0f;
        if (!fin) continue;
        // Per-axis state in scalars (an array indexed by the chosen axis would
        // live in local memory).  Keys fit in int32: the sensor is inside the
        // grid and |e| < 2^30.
        int v0, v1, v2, e0i, e1i, e2i, st0, st1, st2;
        float t0, t1, t2, dl0, dl1, dl2;
        auto axis = [](float sa, float ea, int& va, int& vea, int& sta, float& ta, float& dla) {
            va = (int)floorf(sa);
            vea = (int)floorf(ea);
            const float d = __fsub_rn(ea, sa);
            if (d > 0.0f) {
                sta = 1;
                ta = __fdiv_rn(__fsub_rn(__int2float_rn(va + 1), sa), d);
                dla = __fdiv_rn(1.0f, d);
            } else if (d < 0.0f) {
                sta = -1;
                ta = __fdiv_rn(__fsub_rn(__int2float_rn(va), sa), d);
                dla = __fdiv_rn(-1.0f, d);
            } else {
                sta = 0;
                ta = __int_as_float(0x7f800000);
                dla = __int_as_float(0x7f800000);
            }
        };
        axis(s[0], e[0], v0, e0i, st0, t0, dl0);
        axis(s[1], e[1], v1, e1i, st1, t1, dl1);
        axis(s[2], e[2], v2, e2i, st2, t2, dl2);
        const long long l64 = llabs((long long)e0i - v0) + llabs((long long)e1i - v1) + llabs((long long)e2i - v2);
        int left = (int)(l64 < cap ? l64 : cap);  // the walk leaves the grid first
        uint32_t cur_brick = kNone;  // the brick of the last step and its slot: one table read per brick crossed
        int32_t cur_slot = -1;
        for (; left > 0; --left) {
            const int q0 = v0 - w0, q1 = v1 - w1, q2 = v2 - w2;  // window coordinates
            const bool gone = (q0 < 0 && st0 <= 0) || (q0 >= dims[0] && st0 >= 0) || (q1 < 0 && st1 <= 0) ||
                              (q1 >= dims[1] && st1 >= 0) || (q2 < 0 && st2 <= 0) || (q2 >= dims[2] && st2 >= 0);
            if (gone) break;
            if (q0 >= 0 && q0 < dims[0] && q1 >= 0 && q1 < dims[1] && q2 >= 0 && q2 < dims[2]) {
                const uint32_t brick =
                    ((uint32_t)(q2 >> 3) * (uint32_t)g.nby + (uint32_t)(q1 >> 3)) * (uint32_t)g.nbx +
                    (uint32_t)(q0 >> 3);
                if (brick != cur_brick) {
                    cur_brick = brick;
                    cur_slot = table[brick];
                }
                if (cur_slot >= 0) {
                    const uint32_t idx =
                        (uint32_t)cur_slot * kBrickVox + (uint32_t)((((q2 & 7) << 3) | (q1 & 7)) << 3 | (q0 & 7));
                    const uint32_t bit = 1u << (idx & 31);
                    if (C[idx] && !(__ldcg(mark + (idx >> 5)) & bit)) atomicOr(mark + (idx >> 5), bit);
                }
            }
            // the axis whose next boundary comes first, ties to x, then y, then z, among those not at the end
            int best = -1;
            float bt = 0.0f;
            if (v0 != e0i) { best = 0; bt = t0; }
            if (v1 != e1i && (best < 0 || t1 < bt)) { best = 1; bt = t1; }
            if (v2 != e2i && (best < 0 || t2 < bt)) best = 2;
            if (best == 0) {
                v0 += st0;
                t0 = __fadd_rn(t0, dl0);
            } else if (best == 1) {
                v1 += st1;
                t1 = __fadd_rn(t1, dl1);
            } else {
                v2 += st2;
                t2 = __fadd_rn(t2, dl2);
            }
        }
    }
}

// Clears the marked voxels of the allocated slots (sums and count to zero)
// and their marks; counts the cleared voxels.
__global__ void __launch_bounds__(kThreads) k_clear_apply(unsigned long long* __restrict__ S, uint32_t* __restrict__ C,
                                                         uint32_t* __restrict__ mark, MapCounters* __restrict__ ctr,
                                                         uint32_t capacity) {
    pdl_gate();
    const uint32_t nb = min(ctr->n_bricks, capacity);
    const size_t words = (size_t)nb * (kBrickVox / 32);
    uint32_t cleared = 0;
    for (size_t w = (size_t)blockIdx.x * kThreads + threadIdx.x; w < words; w += (size_t)gridDim.x * kThreads) {
        uint32_t m = mark[w];
        if (!m) continue;
        mark[w] = 0;
        const uint32_t slot = (uint32_t)(w / (kBrickVox / 32));
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t l = (uint32_t)((w % (kBrickVox / 32)) * 32 + b);
            unsigned long long* sp = S + (size_t)slot * 3 * kBrickVox + l;
            sp[0] = 0;
            sp[kBrickVox] = 0;
            sp[2 * kBrickVox] = 0;
            C[(size_t)slot * kBrickVox + l] = 0;
            ++cleared;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cleared += __shfl_xor_sync(0xffffffffu, cleared, o);
    if ((threadIdx.x & 31) == 0 && cleared) atomicAdd(&ctr->cleared, (unsigned long long)cleared);
}

// ---------------------------------------------------------------- scrolling
// keep[s] = 1 when allocated slot s's brick lies in the window moved by
// (sx, sy, sz) bricks.
__global__ void k_scroll_keep(const int32_t* __restrict__ slot_key, const MapCounters* __restrict__ ctr,
                              uint32_t capacity, int sx, int sy, int sz, int nbx, int nby, int nbz,
                              uint32_t* __restrict__ keep) {
    pdl_gate();
    const uint32_t nb = min(ctr->n_bricks, capacity);
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < nb; s += gridDim.x * kThreads) {
        const int b = slot_key[s];
        const int bx = b % nbx - sx, by = (b / nbx) % nby - sy, bz = b / (nbx * nby) - sz;
        keep[s] = (bx >= 0 && bx < nbx && by >= 0 && by < nby && bz >= 0 && bz < nbz) ? 1u : 0u;
    }
}

// hole[r] = the r-th slot below the kept count that is not kept.
__global__ void k_scroll_holes(const MapCounters* __restrict__ ctr, uint32_t capacity,
                               const uint32_t* __restrict__ keep, const uint32_t* __restrict__ kpos,
                               const uint32_t* __restrict__ n_keep, uint32_t* __restrict__ hole) {
    pdl_gate();
    const uint32_t nk = *n_keep;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < nk; s += gridDim.x * kThreads)
        if (!keep[s]) hole[s - kpos[s]] = s;
}

// Occupied voxels of the evicted slots (one CTA per slot; before the move
// overwrites them).
__global__ void __launch_bounds__(kThreads) k_scroll_count(const uint32_t* __restrict__ keep, uint32_t capacity,
                                                          const uint32_t* __restrict__ C,
                                                          MapCounters* __restrict__ ctr) {
    pdl_gate();
    const uint32_t nb = min(ctr->n_bricks, capacity);
    uint32_t occ = 0;
    for (uint32_t s = blockIdx.x; s < nb; s += gridDim.x) {
        if (keep[s]) continue;
        for (int l = threadIdx.x; l < kBrickVox; l += kThreads) occ += C[(size_t)s * kBrickVox + l] != 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) occ += __shfl_xor_sync(0xffffffffu, occ, o);
    if ((threadIdx.x & 31) == 0 && occ) atomicAdd(&ctr->evicted, (unsigned long long)occ);
}

// One CTA per slot: a kept slot below the kept count stays and a kept slot
// above it moves into the hole of the same rank (holes are evicted slots, read
// by nothing here); either way its sums are re-anchored (S - C da) and its key
// shifted into the new window.
__global__ void __launch_bounds__(kThreads) k_scroll_move(const MapCounters* __restrict__ ctr, uint32_t capacity,
                                                         const uint32_t* __restrict__ keep,
                                                         const uint32_t* __restrict__ kpos,
                                                         const uint32_t* __restrict__ n_keep,
                                                         const uint32_t* __restrict__ hole, int32_t* slot_key,
                                                         int shift_key, long long dax, long long day, long long daz,
                                                         unsigned long long* S, uint32_t* C) {
    pdl_gate();
    const uint32_t nb = min(ctr->n_bricks, capacity), nk = *n_keep;
    const uint32_t below = nk < nb ? kpos[nk] : nk;  // kept slots below the kept count
    for (uint32_t s = blockIdx.x; s < nb; s += gridDim.x) {
        if (!keep[s]) continue;
        const uint32_t* cs = C + (size_t)s * kBrickVox;
        const uint32_t d = s < nk ? s : hole[kpos[s] - below];
        const unsigned long long* ss = S + (size_t)s * 3 * kBrickVox;
        unsigned long long* sd = S + (size_t)d * 3 * kBrickVox;
        uint32_t* cd = C + (size_t)d * kBrickVox;
        for (int l = threadIdx.x; l < kBrickVox; l += kThreads) {
            const uint32_t c = cs[l];
            const long long cc = (long long)c;
            sd[l] = (unsigned long long)((long long)ss[l] - cc * dax);
            sd[kBrickVox + l] = (unsigned long long)((long long)ss[kBrickVox + l] - cc * day);
            sd[2 * kBrickVox + l] = (unsigned long long)((long long)ss[2 * kBrickVox + l] - cc * daz);
            cd[l] = c;
        }
        if (threadIdx.x == 0) slot_key[d] = slot_key[s] - shift_key;
    }
}

// Zeroes the slots from the kept count to the old count (their bricks moved
// or were evicted) so they can be claimed again.
__global__ void k_scroll_zero(const uint32_t* __restrict__ n_keep, const MapCounters* __restrict__ ctr,
                              uint32_t capacity, unsigned long long* S, uint32_t* C) {
    pdl_gate();
    const size_t lo = (size_t)*n_keep * kBrickVox, hi = (size_t)min(ctr->n_bricks, capacity) * kBrickVox;
    for (size_t i = lo + (size_t)blockIdx.x * kThreads + threadIdx.x; i < hi; i += (size_t)gridDim.x * kThreads) {
        const size_t slot = i / kBrickVox, l = i % kBrickVox;
        S[slot * 3 * kBrickVox + l] = 0;
        S[slot * 3 * kBrickVox + kBrickVox + l] = 0;
        S[slot * 3 * kBrickVox + 2 * kBrickVox + l] = 0;
        C[i] = 0;
    }
}

// The brick table of the new window (cleared before), the new brick count
// and the new position origin.
__global__ void k_scroll_table(const uint32_t* __restrict__ n_keep, const int32_t* __restrict__ slot_key,
                               int32_t* __restrict__ table, MapCounters* __restrict__ ctr, float* __restrict__ po,
                               float px, float py, float pz) {
    pdl_gate();
    const uint32_t nk = *n_keep;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < nk; s += gridDim.x * kThreads)
        table[slot_key[s]] = (int32_t)s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->n_bricks = nk;
        po[0] = px;
        po[1] = py;
        po[2] = pz;
    }
}

}  // namespace

// Each array of the scratch starts on a 256-byte boundary (the scan's state
// holds 64-bit words).
static size_t scroll_stride(uint32_t capacity) { return ((size_t)capacity + 63) & ~(size_t)63; }

size_t scroll_tmp_words(uint32_t capacity) {
    return 3 * scroll_stride(capacity) + 64 + scan_tmp_words((size_t)capacity + 1);
}

cudaError_t launch_scroll(const Grid& g, const Grid& g2, const int32_t shift[3], const float po2[3],
                          int32_t* brick_table, uint32_t nb_total, int32_t* slot_key, unsigned long long* S,
                          uint32_t* C, MapCounters* ctr, uint32_t capacity, uint32_t* tmp, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t stride = scroll_stride(capacity);
    uint32_t* keep = tmp;
    uint32_t* kpos = keep + stride;
    uint32_t* hole = kpos + stride;
    uint32_t* word = hole + stride;  // [0] the kept count
    uint32_t* scan_state = word + 64;
    const unsigned gs = (unsigned)((capacity + kThreads - 1) / kThreads < (uint32_t)sms * 8
                                       ? (capacity + kThreads - 1) / kThreads
                                       : (uint32_t)sms * 8);
    const int shift_key = (shift[2] * g.nby + shift[1]) * g.nbx + shift[0];
    launch_k(k_scroll_keep, dim3(gs), dim3(kThreads), 0, s, slot_key, ctr, capacity, shift[0], shift[1], shift[2],
             g.nbx, g.nby, g.nbz, keep);
    cudaError_t e = exclusive_scan_dev(keep, kpos, word, &ctr->n_bricks, capacity, scan_state, s, nullptr);
    if (e != cudaSuccess) return e;
    launch_k(k_scroll_holes, dim3(gs), dim3(kThreads), 0, s, ctr, capacity, keep, kpos, word, hole);
    const unsigned gm = capacity < (uint32_t)sms * 8 ? capacity : (uint32_t)sms * 8;
    launch_k(k_scroll_count, dim3(gm), dim3(kThreads), 0, s, keep, capacity, C, ctr);
    launch_k(k_scroll_move, dim3(gm), dim3(kThreads), 0, s, ctr, capacity, keep, kpos, word, hole, slot_key, shift_key,
             g2.ax - g.ax, g2.ay - g.ay, g2.az - g.az, S, C);
    const size_t zw = ((size_t)capacity * kBrickVox + kThreads - 1) / kThreads;
    launch_k(k_scroll_zero, dim3((unsigned)(zw < (size_t)sms * 8 ? zw : (size_t)sms * 8)), dim3(kThreads), 0, s, word,
             ctr, capacity, S, C);
    if ((e = cudaMemsetAsync(brick_table, 0xFF, (size_t)nb_total * sizeof(int32_t), s)) != cudaSuccess) return e;
    launch_k(k_scroll_table, dim3(gs), dim3(kThreads), 0, s, word, slot_key, brick_table, ctr,
             const_cast<float*>(g2.po), po2[0], po2[1], po2[2]);
    count_launch(6);
    return cudaGetLastError();
}

cudaError_t launch_clear(const float* xyz, uint32_t n, const Pose& pose, const Grid& g, const int32_t* brick_table,
                         unsigned long long* S, uint32_t* C, uint32_t* mark, MapCounters* ctr, uint32_t capacity,
                         cudaStream_t s) {
    // A sensor outside the grid casts no rays (host check, same arithmetic as the walk's start).
    const float sx = (pose.r[3] - g.ox) * g.inv_res, sy = (pose.r[7] - g.oy) * g.inv_res,
                sz = (pose.r[11] - g.oz) * g.inv_res;
    if (!(sx >= (float)g.wx && sx < (float)(g.wx + g.nx) && sy >= (float)g.wy && sy < (float)(g.wy + g.ny) &&
          sz >= (float)g.wz && sz < (float)(g.wz + g.nz)) ||
        n == 0)
        return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t want = (n + kThreads - 1) / kThreads;
    const uint32_t grid = want < (uint32_t)(sms * 8) ? want : (uint32_t)(sms * 8);
    launch_k(k_clear_mark, dim3(grid), dim3(kThreads), 0, s, xyz, n, pose, g, brick_table, C, mark, ctr);
    const size_t words = (size_t)capacity * (kBrickVox / 32);
    const size_t wgrid = (words + kThreads - 1) / kThreads;
    launch_k(k_clear_apply, dim3((unsigned)(wgrid < (size_t)sms * 8 ? wgrid : (size_t)sms * 8)), dim3(kThreads), 0, s,
             S, C, mark, ctr, capacity);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const float* xyz, uint32_t n, const Pose& pose, const Grid& g, int32_t* brick_table,
                             int32_t* slot_key, unsigned long long* S, uint32_t* C, uint32_t* deferred,
                             MapCounters* ctr, uint32_t capacity, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t want = (n + kThreads - 1) / kThreads;
    const uint32_t grid = want < (uint32_t)(sms * 8) ? want : (uint32_t)(sms * 8);
    launch_k(k_accum, dim3(grid), dim3(kThreads), 0, s, xyz, n, pose, g, brick_table, slot_key, S, C, deferred, ctr,
             capacity);
    launch_k(k_accum_deferred, dim3(grid < (uint32_t)sms ? grid : (uint32_t)sms), dim3(kThreads), 0, s, xyz, pose, g,
             brick_table, S, C, deferred, ctr);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace vmx
