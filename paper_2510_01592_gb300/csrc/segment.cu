// segment.cu -- multi-plane segmentation up to the cluster point lists
// (Sec. III.C): mean positions from the exact sums, normals and steppable
// classification (Eq. 3, Eq. 4), clustering (Algorithm 1) and cluster
// formation.
//
// Layout.  After ordering the allocated bricks by brick key, every per-voxel
// array is "rank-dense": voxel (brick rank r, local index l) lives at
// r * 512 + l.  Because bricks are ranked by key and voxel ids are
// brick-major (key * 512 + l), index order equals voxel-id order, so the
// union-find root with the smallest index is the component's smallest voxel
// id -- the fixed point of Algorithm 1's min-label propagation.
//
// Normals and clustering run one CTA per brick (512 threads, a thread per
// voxel) with the brick and a one-voxel halo from its 26 neighbours staged in
// shared memory.
#include <climits>
#include <cstddef>
#include <mutex>

#include "vm_internal.cuh"

namespace vmx {
namespace {

constexpr int kT = 256;
constexpr float kInvQ = 9.5367431640625e-07f;  // 2^-20

__device__ __forceinline__ void brick_coords(int32_t key, const Grid& g, int& bx, int& by, int& bz) {
    bx = key % g.nbx;
    by = (key / g.nbx) % g.nby;
    bz = key / (g.nbx * g.nby);
}

// Mean of each voxel: M = floor((2 S + c) / (2 c)), the exact integer mean in
// 2^-20 m units rounded half up (Eq. 1's mu up to that quantum).
__global__ void __launch_bounds__(kT) k_finalize(const uint32_t* __restrict__ nsp, uint32_t cap_b,
                                                 const int32_t* __restrict__ sorted_slot,
                                                 const unsigned long long* __restrict__ S,
                                                 const uint32_t* __restrict__ C, int32_t* __restrict__ M,
                                                 uint8_t* __restrict__ status, size_t stride,
                                                 SegCounters* __restrict__ ctr) {
    pdl_gate();
    // more bricks than the scratch was sized for: the kernels clamp to it, the
    // host regrows and reruns
    if (blockIdx.x == 0 && threadIdx.x == 0 && *nsp > cap_b) atomicOr(&ctr->err, kErrScratch);
    const uint32_t n_sorted = min(*nsp, cap_b);
    uint32_t occ = 0;
    for (uint32_t r = blockIdx.x; r < n_sorted; r += gridDim.x) {
        const int32_t slot = sorted_slot[r];
        constexpr int kIt = kBrickVox / kT;
        uint32_t c[kIt];
        long long sv[kIt][3];
#pragma unroll
        for (int j = 0; j < kIt; ++j) c[j] = C[(size_t)slot * kBrickVox + threadIdx.x + j * kT];
#pragma unroll
        for (int j = 0; j < kIt; ++j)  // a thread's sums loaded together
            if (c[j])
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    sv[j][a] = (long long)S[((size_t)slot * 3 + a) * kBrickVox + threadIdx.x + j * kT];
#pragma unroll
        for (int j = 0; j < kIt; ++j) {
            const size_t o = (size_t)r * kBrickVox + threadIdx.x + j * kT;
            if (c[j]) {
                const long long c2 = 2ll * (long long)c[j];
#pragma unroll
                for (int a = 0; a < 3; ++a) M[a * stride + o] = (int32_t)((2ll * sv[j][a] + (long long)c[j]) / c2);
                status[o] = 1;
                ++occ;
            } else {
                M[o] = INT_MIN;
                M[stride + o] = INT_MIN;
                M[2 * stride + o] = INT_MIN;
                status[o] = 0;
            }
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) occ += __shfl_xor_sync(0xffffffffu, occ, s);
    if ((threadIdx.x & 31) == 0 && occ) atomicAdd(&ctr->n_occ, occ);
}

// ---------------------------------------------------------------- Jacobi (FP32)
// Cyclic Jacobi (Golub & Van Loan Sec. 8.5) on a symmetric 3x3 matrix, pairs
// (0,1), (0,2), (1,2), a fixed number of sweeps, pairs with a_pq == 0 skipped;
// tau = (a_qq - a_pp) / (2 a_pq), t = sgn(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1 / sqrt(1 + t^2), s = t c.  Every operation is an explicit IEEE
// round-to-nearest intrinsic.
__device__ __forceinline__ void jacobi3(float a00, float a11, float a22, float a01, float a02, float a12, int sweeps,
                                        float v[3][3], float d[3]) {
    float a[3][3] = {{a00, a01, a02}, {a01, a11, a12}, {a02, a12, a22}};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[r][c] = (r == c) ? 1.0f : 0.0f;
    for (int sw = 0; sw < sweeps; ++sw) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int p = (k == 2) ? 1 : 0, q = (k == 0) ? 1 : 2, r = 2 - k;
            const float apq = a[p][q];
            if (apq == 0.0f) continue;
            const float app = a[p][p], aqq = a[q][q];
            const float tau = __fdiv_rn(__fsub_rn(aqq, app), __fmul_rn(2.0f, apq));
            const float sg = (tau >= 0.0f) ? 1.0f : -1.0f;
            const float t = __fdiv_rn(sg, __fadd_rn(fabsf(tau), __fsqrt_rn(__fmaf_rn(tau, tau, 1.0f))));
            const float c = __fdiv_rn(1.0f, __fsqrt_rn(__fmaf_rn(t, t, 1.0f)));
            const float s = __fmul_rn(t, c);
            a[p][p] = __fmaf_rn(-t, apq, app);
            a[q][q] = __fmaf_rn(t, apq, aqq);
            a[p][q] = 0.0f;
            a[q][p] = 0.0f;
            const float arp = a[r][p], arq = a[r][q];
            const float nrp = __fmaf_rn(c, arp, -__fmul_rn(s, arq));
            const float nrq = __fmaf_rn(s, arp, __fmul_rn(c, arq));
            a[r][p] = nrp; a[p][r] = nrp;
            a[r][q] = nrq; a[q][r] = nrq;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float vip = v[i][p], viq = v[i][q];
                v[i][p] = __fmaf_rn(c, vip, -__fmul_rn(s, viq));
                v[i][q] = __fmaf_rn(s, vip, __fmul_rn(c, viq));
            }
        }
    }
    d[0] = a[0][0]; d[1] = a[1][1]; d[2] = a[2][2];
}

// Column of the smallest diagonal entry (lowest index on ties), scaled by
// 1/sqrt(n.n), oriented n_z >= 0 (then n_y, then n_x when zero).
__device__ __forceinline__ void pick_normal(float v[3][3], const float d[3], float n[3]) {
    int m = 0;
    if (d[1] < d[m]) m = 1;
    if (d[2] < d[m]) m = 2;
    float x = (m == 0) ? v[0][0] : (m == 1) ? v[0][1] : v[0][2];
    float y = (m == 0) ? v[1][0] : (m == 1) ? v[1][1] : v[1][2];
    float z = (m == 0) ? v[2][0] : (m == 1) ? v[2][1] : v[2][2];
    const float nn = __fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(nn));
    x = __fmul_rn(x, inv); y = __fmul_rn(y, inv); z = __fmul_rn(z, inv);
    const bool flip = (z < 0.0f) || (z == 0.0f && (y < 0.0f || (y == 0.0f && x < 0.0f)));
    if (flip) { x = -x; y = -y; z = -z; }
    n[0] = x; n[1] = y; n[2] = z;
}

// Rank of each of the 27 bricks around brick r (-1: none).
__device__ __forceinline__ void load_neighbour_ranks(int32_t key, const Grid& g, const int32_t* __restrict__ rank_table,
                                                     int32_t* nb) {
    if (threadIdx.x < 27) {
        int bx, by, bz;
        brick_coords(key, g, bx, by, bz);
        const int dz = (int)threadIdx.x / 9 - 1, dy = ((int)threadIdx.x / 3) % 3 - 1, dx = (int)threadIdx.x % 3 - 1;
        const int x = bx + dx, y = by + dy, z = bz + dz;
        nb[threadIdx.x] = (x >= 0 && y >= 0 && z >= 0 && x < g.nbx && y < g.nby && z < g.nbz)
                              ? rank_table[(z * g.nby + y) * g.nbx + x] : -1;
    }
}

// Rank-dense index of halo cell c of a 10^3 halo, or -1.
__device__ __forceinline__ int32_t halo_index(int c, const int32_t* nb) {
    const int hx = c % 10, hy = (c / 10) % 10, hz = c / 100;
    const int gx = hx - 1, gy = hy - 1, gz = hz - 1;
    const int bdx = gx < 0 ? -1 : (gx > 7 ? 1 : 0);
    const int bdy = gy < 0 ? -1 : (gy > 7 ? 1 : 0);
    const int bdz = gz < 0 ? -1 : (gz > 7 ? 1 : 0);
    const int32_t rk = nb[(bdz + 1) * 9 + (bdy + 1) * 3 + (bdx + 1)];
    if (rk < 0) return -1;
    const int lx = gx - 8 * bdx, ly = gy - 8 * bdy, lz = gz - 8 * bdz;
    return rk * kBrickVox + ((lz * 8 + ly) * 8 + lx);
}

// ---------------------------------------------------------------- union-find
// Global forest over rank-dense indices.  Hooking always puts the larger root
// under the smaller, so every root is the smallest index of its tree.
__device__ __forceinline__ uint32_t uf_find(uint32_t* P, uint32_t x, uint32_t* err) {
    for (int it = 0; it < kLoopCap; ++it) {
        const uint32_t p = __ldcg(P + x);
        if (p == x) return x;
        const uint32_t gp = __ldcg(P + p);
        if (gp != p) P[x] = gp;  // path halving: gp is an ancestor of x
        x = gp;
    }
    atomicOr(err, kErrTimeout);
    return x;
}

__device__ __forceinline__ void uf_union(uint32_t* P, uint32_t a, uint32_t b, uint32_t* err) {
    for (int it = 0; it < kLoopCap; ++it) {
        a = uf_find(P, a, err);
        b = uf_find(P, b, err);
        if (a == b) return;
        const uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
        const uint32_t old = atomicCAS(P + hi, hi, lo);
        if (old == hi) return;
        a = old;  // hi was hooked meanwhile: continue from its new parent
        b = lo;
    }
    atomicOr(err, kErrTimeout);
}

// The same forest in shared memory, over the 512 voxels of one brick.
__device__ __forceinline__ uint32_t lf_find(volatile uint32_t* P, uint32_t x) {
    for (int it = 0; it < 1024; ++it) {
        const uint32_t p = P[x];
        if (p == x) return x;
        const uint32_t gp = P[p];
        if (gp != p) P[x] = gp;
        x = gp;
    }
    return x;
}

__device__ __forceinline__ void lf_union(uint32_t* P, uint32_t a, uint32_t b, uint32_t* err) {
    for (int it = 0; it < 4096; ++it) {
        a = lf_find(P, a);
        b = lf_find(P, b);
        if (a == b) return;
        const uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
        const uint32_t old = atomicCAS(P + hi, hi, lo);
        if (old == hi) return;
        a = old;
        b = lo;
    }
    atomicOr(err, kErrTimeout);
}

// Algorithm 1's edge test: |mu_i - mu_j|^2 < d_th^2 and |n_i . n_j| > cos_ccl
// (symmetric in i and j).
__device__ __forceinline__ bool ccl_edge(float ax, float ay, float az, float anx, float any, float anz, float bx,
                                         float by, float bz, float bnx, float bny, float bnz, float d_th2,
                                         float cos_ccl) {
    const float ex = __fsub_rn(ax, bx), ey = __fsub_rn(ay, by), ez = __fsub_rn(az, bz);
    const float d2 = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
    const float cs = __fmaf_rn(anz, bnz, __fmaf_rn(any, bny, __fmul_rn(anx, bnx)));
    return d2 < d_th2 && fabsf(cs) > cos_ccl;
}

__device__ __forceinline__ float mean_pos(float o, int32_t m) {
    return __fadd_rn(o, __fmul_rn(__int2float_rn(m), kInvQ));
}

// Forward neighbour k of 13: (dz, dy, dx) lexicographically after (0, 0, 0).
__device__ __forceinline__ void fwd_offset(int k, int& dz, int& dy, int& dx) {
    dz = (k < 9) ? 1 : 0;
    dy = (k < 9) ? (k / 3 - 1) : ((k < 12) ? 1 : 0);
    dx = (k < 9) ? (k % 3 - 1) : ((k < 12) ? (k - 9 - 1) : 1);
}

// Eq. 3 / Eq. 4 in two kernels.
// k_moments, one 128-thread CTA per brick: the brick and a one-voxel halo of
// integer means are staged in shared memory; for every occupied voxel the
// window moments give the covariance of the 3x3x3 window of mean positions
// (self included) as the exact integer matrix N' sum(dd^T) - (sum d)(sum d)^T
// of offsets d = M_j - M_i, rounded to FP32.  Occupied voxels go to a flat
// list (A, N, voxel index) for k_eigen; every voxel's record gets its mean
// (status filled in by k_eigen; zero for free voxels).
constexpr int kNormT = 128;
__global__ void __launch_bounds__(kNormT) k_moments(const uint32_t* __restrict__ nsp, uint32_t cap_b, Grid g,
                                                    const int32_t* __restrict__ sorted_key,
                                                    const int32_t* __restrict__ rank_table,
                                                    const int32_t* __restrict__ M, float4* __restrict__ rec,
                                                    uint32_t* __restrict__ list_idx, float* __restrict__ list_A,
                                                    uint8_t* __restrict__ nbr, size_t stride,
                                                    SegCounters* __restrict__ ctr) {
    pdl_gate();
    const uint32_t n_sorted = min(*nsp, cap_b);
    const float pox = g.po[0], poy = g.po[1], poz = g.po[2];
    __shared__ int32_t sM[3][1000];
    __shared__ uint16_t list[512];
    __shared__ int32_t nb[27];
    __shared__ int n_list;
    __shared__ uint32_t gbase;
    for (uint32_t r = blockIdx.x; r < n_sorted; r += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) n_list = 0;
        load_neighbour_ranks(sorted_key[r], g, rank_table, nb);
        __syncthreads();
        // the 10^3 halo of means, each thread's loads issued four cells at a time
        constexpr int kIt = (1000 + kNormT - 1) / kNormT, kGroup = 4;
#pragma unroll 1
        for (int j0 = 0; j0 < kIt; j0 += kGroup) {
            int32_t idx[kGroup], m[kGroup][3];
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                const int c = threadIdx.x + (j0 + j) * kNormT;
                idx[j] = c < 1000 ? halo_index(c, nb) : -1;
                if (idx[j] >= 0) {
                    m[j][0] = M[idx[j]];
                    m[j][1] = M[stride + idx[j]];
                    m[j][2] = M[2 * stride + idx[j]];
                }
            }
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                const int c = threadIdx.x + (j0 + j) * kNormT;
                if (c >= 1000) continue;
                if (idx[j] >= 0) {
                    sM[0][c] = m[j][0];
                    sM[1][c] = m[j][1];
                    sM[2][c] = m[j][2];
                } else {
                    sM[0][c] = INT_MIN;
                }
            }
        }
        __syncthreads();
        for (int l = threadIdx.x; l < kBrickVox; l += kNormT) {
            const int c0 = (((l >> 6) + 1) * 10 + ((l >> 3) & 7) + 1) * 10 + (l & 7) + 1;
            const size_t o = (size_t)r * kBrickVox + l;
            if (sM[0][c0] != INT_MIN) {
                list[atomicAdd(&n_list, 1)] = (uint16_t)l;
                rec[o] = make_float4(mean_pos(pox, sM[0][c0]), mean_pos(poy, sM[1][c0]), mean_pos(poz, sM[2][c0]),
                                     __int_as_float(0));
            } else {
                rec[o] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0));
            }
        }
        __syncthreads();
        const int nl = n_list;
        if (threadIdx.x == 0) gbase = atomicAdd(&ctr->n_list, (uint32_t)nl);
        __syncthreads();
        for (int q = threadIdx.x; q < nl; q += kNormT) {
            const int l = list[q];
            const int c0 = (((l >> 6) + 1) * 10 + ((l >> 3) & 7) + 1) * 10 + (l & 7) + 1;
            const int32_t m0 = sM[0][c0], m1 = sM[1][c0], m2 = sM[2][c0];
            int32_t s1x = 0, s1y = 0, s1z = 0;
            long long sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
            int cnt = 0;
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int c = c0 + dz * 100 + dy * 10 + dx;
                        const int32_t a0 = sM[0][c];
                        if (a0 == INT_MIN) continue;
                        const int32_t ex = a0 - m0, ey = sM[1][c] - m1, ez = sM[2][c] - m2;
                        s1x += ex; s1y += ey; s1z += ez;
                        sxx += (long long)ex * ex; syy += (long long)ey * ey; szz += (long long)ez * ez;
                        sxy += (long long)ex * ey; sxz += (long long)ex * ez; syz += (long long)ey * ez;
                        ++cnt;
                    }
            const long long N = cnt;
            const size_t slot = gbase + q;
            const size_t o = (size_t)r * kBrickVox + l;
            list_idx[slot] = (uint32_t)o;
            list_A[slot] = __ll2float_rn(N * sxx - (long long)s1x * s1x);
            list_A[stride + slot] = __ll2float_rn(N * syy - (long long)s1y * s1y);
            list_A[2 * stride + slot] = __ll2float_rn(N * szz - (long long)s1z * s1z);
            list_A[3 * stride + slot] = __ll2float_rn(N * sxy - (long long)s1x * s1y);
            list_A[4 * stride + slot] = __ll2float_rn(N * sxz - (long long)s1x * s1z);
            list_A[5 * stride + slot] = __ll2float_rn(N * syz - (long long)s1y * s1z);
            nbr[o] = (uint8_t)(cnt - 1);
        }
    }
}

// k_eigen, one thread per occupied voxel: normal = eigenvector of the smallest
// eigenvalue by FP32 Jacobi (6 sweeps); steppable iff N >= n_th and
// |n_z| >= cos_step (status 2, else 1).
__global__ void __launch_bounds__(256) k_eigen(const SegCounters* __restrict__ ctr,
                                               const uint32_t* __restrict__ list_idx, const float* __restrict__ list_A,
                                               const uint8_t* __restrict__ nbr, float* __restrict__ nrm,
                                               uint8_t* __restrict__ status, float4* __restrict__ rec, size_t stride,
                                               uint32_t n_th, float cos_step) {
    pdl_gate();
    const uint32_t n = ctr->n_list;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        float v[3][3], d[3], nv[3];
        jacobi3(list_A[q], list_A[stride + q], list_A[2 * stride + q], list_A[3 * stride + q],
                list_A[4 * stride + q], list_A[5 * stride + q], 6, v, d);
        pick_normal(v, d, nv);
        const uint32_t o = list_idx[q];
        nrm[o] = nv[0];
        nrm[stride + o] = nv[1];
        nrm[2 * stride + o] = nv[2];
        const uint8_t st = (nbr[o] >= n_th && fabsf(nv[2]) >= cos_step) ? 2 : 1;
        status[o] = st;
        reinterpret_cast<int*>(rec + o)[3] = (int)st;
        rec[stride + o] = make_float4(nv[0], nv[1], nv[2], 0.0f);
    }
}

// The intra-brick half of Algorithm 1, one 128-thread CTA per brick: the
// brick's records staged in shared memory, its vertices joined over edges
// inside the brick with a union-find in shared memory; the global parent of
// each vertex is set to its local root (the smallest index of its in-brick
// component).  Edges that leave the brick follow in k_ccl_cross.
__global__ void __launch_bounds__(kNormT, 8) k_ccl_local(const uint32_t* __restrict__ nsp, uint32_t cap_b,
                                                      const float4* __restrict__ rec, uint32_t* __restrict__ parent,
                                                      uint32_t* __restrict__ count, size_t stride, uint8_t want,
                                                      float d_th2, float cos_ccl, uint32_t* err) {
    pdl_gate();
    const uint32_t n_sorted = min(*nsp, cap_b);
    __shared__ float4 sA[512];
    __shared__ float4 sB[512];
    __shared__ uint32_t lpar[512];
    for (uint32_t r = blockIdx.x; r < n_sorted; r += gridDim.x) {
        __syncthreads();
        {  // the brick's records, all of a thread's loads in flight together
            constexpr int kIt = kBrickVox / kNormT;
            float4 a[kIt], bn[kIt];
#pragma unroll
            for (int j = 0; j < kIt; ++j) a[j] = rec[(size_t)r * kBrickVox + threadIdx.x + j * kNormT];
#pragma unroll
            for (int j = 0; j < kIt; ++j)
                if (__float_as_int(a[j].w) >= want)
                    bn[j] = rec[stride + (size_t)r * kBrickVox + threadIdx.x + j * kNormT];
#pragma unroll
            for (int j = 0; j < kIt; ++j) {
                const int l = threadIdx.x + j * kNormT;
                const bool vert = __float_as_int(a[j].w) >= want;
                sA[l] = a[j];
                if (vert) sB[l] = bn[j];
                lpar[l] = vert ? (uint32_t)l : kNone;
            }
        }
        __syncthreads();
        // Runs along +x first, without atomics: each 8-voxel row lies in one
        // warp, whose ballot of +x edges gives every vertex the start (smallest
        // index) of its run as its parent.
        for (int l = threadIdx.x; l < kBrickVox; l += kNormT) {
            const bool vert = __float_as_int(sA[l].w) >= want;
            const int lx = l & 7;
            bool xe = false;
            if (vert && lx < 7 && __float_as_int(sA[l + 1].w) >= want) {
                const float4 a = sA[l], an = sB[l], b = sA[l + 1], bn = sB[l + 1];
                xe = ccl_edge(a.x, a.y, a.z, an.x, an.y, an.z, b.x, b.y, b.z, bn.x, bn.y, bn.z, d_th2, cos_ccl);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, xe);
            const uint32_t row = (bal >> ((threadIdx.x & 31) & ~7)) & 0xffu;
            const uint32_t gap = ~row & ((1u << lx) - 1u);  // missing +x edges below this voxel
            const int start = gap ? 32 - __clz(gap) : 0;
            if (vert) lpar[l] = (uint32_t)((l & ~7) + start);
        }
        __syncthreads();
        for (int l = threadIdx.x; l < kBrickVox; l += kNormT) {
            if (lpar[l] == kNone) continue;
            const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
            const float4 a = sA[l], an = sB[l];
#pragma unroll
            for (int k = 0; k < 12; ++k) {  // the +x offset (k = 12) was joined above
                int dz, dy, dx;
                fwd_offset(k, dz, dy, dx);
                const int x = lx + dx, y = ly + dy, z = lz + dz;
                if (x < 0 || x > 7 || y < 0 || y > 7 || z > 7) continue;
                const int j = (z * 8 + y) * 8 + x;
                if (__float_as_int(sA[j].w) < want) continue;
                const float4 b = sA[j], bn = sB[j];
                if (ccl_edge(a.x, a.y, a.z, an.x, an.y, an.z, b.x, b.y, b.z, bn.x, bn.y, bn.z, d_th2, cos_ccl))
                    lf_union(lpar, (uint32_t)l, (uint32_t)j, err);
            }
        }
        __syncthreads();
        for (int l = threadIdx.x; l < kBrickVox; l += kNormT) {
            const size_t o = (size_t)r * kBrickVox + l;
            uint32_t root = kNone;
            if (__float_as_int(sA[l].w) >= want) {  // read-only walk: entries are final once every union is done
                uint32_t x = (uint32_t)l;
                for (int it = 0; it < 1024; ++it) {
                    const uint32_t p = lpar[x];
                    if (p == x) break;
                    x = p;
                }
                root = (uint32_t)r * kBrickVox + x;
            }
            parent[o] = root;
            count[o] = 0;
        }
    }
}

// The inter-brick half of Algorithm 1, one 128-thread CTA per brick.  The
// brick's 10^3 halo of packed voxel records and current parents is staged in
// shared memory with independent loads; then every vertex whose forward
// neighbours can lie in another brick tests those neighbours from shared
// memory.  Forward offsets have dz in {0, 1}, dy in {-1, 0, 1} (-1 only with
// dz = 1) and dx in {-1, 0, 1}, so they leave the brick through the +z face,
// either y face or either x face.  An edge (i, j) that passes is recorded as
// the pair of their staged parents (ancestors of i and j, so joining them
// joins i and j) in a hash set in shared memory, and each distinct pair is
// joined once in the global forest: most of a brick's edges lead to the same
// few pairs.
constexpr int kCrossT = 128;
constexpr int kPairSlots = 256;
__global__ void __launch_bounds__(kCrossT) k_ccl_cross(const uint32_t* __restrict__ nsp, uint32_t cap_b, Grid g,
                                                       const int32_t* __restrict__ sorted_key,
                                                       const int32_t* __restrict__ rank_table,
                                                       const float4* __restrict__ rec, uint32_t* parent, size_t stride,
                                                       uint8_t want, float d_th2, float cos_ccl, uint32_t* err) {
    pdl_gate();
    const uint32_t n_sorted = min(*nsp, cap_b);
    // The halo at z 0..8 only (forward edges never reach z -1): 10 x 10 x 9
    // cells, cell c = halo cell c + 100.  Means without the status word (a
    // vertex is a cell whose parent is not kNone): 27 KB a CTA, 8 CTAs an SM.
    constexpr int kCells = 900;
    __shared__ float3 sA[kCells];
    __shared__ float4 sB[kCells];  // (normal, parent); parent kNone off the vertex set
    __shared__ unsigned long long set[kPairSlots];
    __shared__ int32_t nb[27];
    for (int q = threadIdx.x; q < kPairSlots; q += kCrossT) set[q] = ~0ull;
    for (uint32_t r = blockIdx.x; r < n_sorted; r += gridDim.x) {
        __syncthreads();
        load_neighbour_ranks(sorted_key[r], g, rank_table, nb);
        __syncthreads();
        // Load only the cells a cross-brick edge can touch: the brick's own
        // cells on the faces forward edges leave through (lx 0 or 7, ly 0 or
        // 7, lz 7) and the halo cells outside the brick at lz 0..8 (648 of the
        // 900); the others are staged as non-vertices.  A thread issues its
        // record loads four at a time before using them.
        constexpr int kIt = (kCells + kCrossT - 1) / kCrossT;  // cells per thread
        constexpr int kGroup = 4;                               // loads in flight per thread
#pragma unroll 1
        for (int j0 = 0; j0 < kIt; j0 += kGroup) {
            int32_t idx[kGroup];
            float4 a[kGroup];
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                const int c = threadIdx.x + (j0 + j) * kCrossT;
                idx[j] = -1;
                if (c < kCells) {
                    const int h = c + 100;  // the 10 x 10 x 10 halo index
                    const int gx = h % 10 - 1, gy = (h / 10) % 10 - 1, gz = h / 100 - 1;
                    const bool inside = gx >= 0 && gx <= 7 && gy >= 0 && gy <= 7 && gz <= 7;
                    const bool source = inside && (gx == 0 || gx == 7 || gy == 0 || gy == 7 || gz == 7);
                    if (source || !inside) idx[j] = halo_index(h, nb);
                }
                a[j] = idx[j] >= 0 ? rec[idx[j]] : make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0));
            }
            float4 bn[kGroup];
            uint32_t par[kGroup];
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                const bool v = idx[j] >= 0 && __float_as_int(a[j].w) >= want;
                bn[j] = v ? rec[stride + idx[j]] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                par[j] = v ? __ldcg(parent + idx[j]) : kNone;
            }
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                const int c = threadIdx.x + (j0 + j) * kCrossT;
                if (c < kCells) {
                    sA[c] = make_float3(a[j].x, a[j].y, a[j].z);
                    sB[c] = make_float4(bn[j].x, bn[j].y, bn[j].z, __uint_as_float(par[j]));
                }
            }
        }
        __syncthreads();
        unsigned long long last = ~0ull;
        for (int l = threadIdx.x; l < kBrickVox; l += kCrossT) {
            const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
            if (!((lx == 0) | (lx == 7) | (ly == 0) | (ly == 7) | (lz == 7))) continue;
            const int c0 = (lz * 10 + ly + 1) * 10 + lx + 1;
            const float3 a = sA[c0];
            const float4 an = sB[c0];
            const uint32_t pa = __float_as_uint(an.w);
            if (pa == kNone) continue;
            for (int k = 0; k < 13; ++k) {
                int dz, dy, dx;
                fwd_offset(k, dz, dy, dx);
                const int x = lx + dx, y = ly + dy, z = lz + dz;
                if (x >= 0 && x <= 7 && y >= 0 && y <= 7 && z <= 7) continue;  // inside the brick: done already
                const int c = c0 + dz * 100 + dy * 10 + dx;
                const float4 bn = sB[c];
                const uint32_t pb = __float_as_uint(bn.w);
                if (pb == kNone || pb == pa) continue;
                const float3 b = sA[c];
                if (!ccl_edge(a.x, a.y, a.z, an.x, an.y, an.z, b.x, b.y, b.z, bn.x, bn.y, bn.z, d_th2, cos_ccl))
                    continue;
                const uint32_t lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
                const unsigned long long key = ((unsigned long long)lo << 32) | hi;
                if (key == last) continue;
                last = key;
                uint32_t h = (lo * 2654435761u ^ hi * 40503u) & (kPairSlots - 1);
                bool placed = false;
                for (int probe = 0; probe < kPairSlots; ++probe) {
                    const unsigned long long prev = atomicCAS(&set[h], ~0ull, key);
                    if (prev == ~0ull || prev == key) { placed = true; break; }
                    h = (h + 1) & (kPairSlots - 1);
                }
                if (!placed) uf_union(parent, lo, hi, err);  // set full: join directly
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kPairSlots; q += kCrossT) {
            const unsigned long long key = set[q];
            if (key != ~0ull) {
                uf_union(parent, (uint32_t)(key >> 32), (uint32_t)key, err);
                set[q] = ~0ull;
            }
        }
    }
}

// Read-only walk to the root.  Used once linking is over: every thread writes
// only its own entry, so a finished entry is never overwritten by another
// thread's path shortcut (which could leave it on an intermediate node).
__device__ __forceinline__ uint32_t uf_root(const uint32_t* P, uint32_t x, uint32_t* err) {
    for (int it = 0; it < kLoopCap; ++it) {
        const uint32_t p = __ldcg(P + x);
        if (p == x) return x;
        x = p;
    }
    atomicOr(err, kErrTimeout);
    return x;
}



// Pointer jumping to the root and component sizes in one pass: each vertex
// walks to its root read-only, writes only its own entry (a walk through it
// then reads either its old parent or the root, both ancestors), and warps
// aggregate equal roots before the size atomics.  Afterwards parent[i] is the
// component's smallest index (its label) for every vertex.
__global__ void k_compress_count(const uint32_t* __restrict__ nsp, uint32_t cap_b, uint32_t* parent,
                                 uint32_t* __restrict__ count, SegCounters* __restrict__ ctr, uint32_t* err) {
    pdl_gate();
    const size_t nv = (size_t)min(*nsp, cap_b) * kBrickVox;
    uint32_t nvert = 0;
    for (size_t base = ((size_t)blockIdx.x * kT + threadIdx.x) & ~(size_t)31; base < nv;
         base += (size_t)gridDim.x * kT) {
        const size_t i = base + (threadIdx.x & 31);
        uint32_t root = kNone;
        if (i < nv && __ldcg(parent + i) != kNone) {
            root = uf_root(parent, (uint32_t)i, err);
            parent[i] = root;
        }
        const uint32_t m = __match_any_sync(0xffffffffu, root);
        if (root != kNone) {
            ++nvert;
            if ((threadIdx.x & 31) == (uint32_t)(__ffs(m) - 1)) atomicAdd(&count[root], (uint32_t)__popc(m));
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) nvert += __shfl_xor_sync(0xffffffffu, nvert, s);
    if ((threadIdx.x & 31) == 0 && nvert) atomicAdd(&ctr->n_vert, nvert);
}

__device__ __forceinline__ uint32_t vid_of(size_t idx, const int32_t* __restrict__ sorted_key) {
    return (uint32_t)sorted_key[idx / kBrickVox] * kBrickVox + (uint32_t)(idx % kBrickVox);
}

// Cluster formation, one 512-thread CTA per brick, one voxel per thread in
// index order.  A vertex is kept when its component has at least min_cluster
// vertices; its root is the component's smallest index.
// Block-wide exclusive count of a per-thread flag (thread order = index order).
__device__ __forceinline__ uint32_t brick_rank(bool f, uint32_t* wcnt, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    uint32_t pre = 0, tot = 0;
    for (int q = 0; q < kBrickVox / 32; ++q) {
        const uint32_t c = wcnt[q];
        pre += (q < w) ? c : 0u;
        tot += c;
    }
    __syncthreads();
    *total = tot;
    return pre + __popc(bal & ((1u << lane) - 1u));
}

// (1) per-brick counts of kept vertices and of kept roots, and the mask of the
// brick's kept roots;
__global__ void __launch_bounds__(kBrickVox) k_brick_tally(const uint32_t* __restrict__ nsp, uint32_t cap_b,
                                                           const uint32_t* __restrict__ parent,
                                                           const uint32_t* __restrict__ count, uint32_t min_cluster,
                                                           uint32_t* __restrict__ nvert, uint32_t* __restrict__ nroot,
                                                           uint32_t* __restrict__ rmask) {
    pdl_gate();
    const uint32_t n_sorted = min(*nsp, cap_b);
    __shared__ uint32_t wc[kBrickVox / 32];
    for (uint32_t r = blockIdx.x; r < n_sorted; r += gridDim.x) {
        const size_t i = (size_t)r * kBrickVox + threadIdx.x;
        const uint32_t p = parent[i];
        const bool kept = p != kNone && count[p] >= min_cluster;
        const bool root = kept && p == (uint32_t)i;
        const uint32_t bal = __ballot_sync(0xffffffffu, root);  // this brick's kept roots, 32 voxels a word
        if ((threadIdx.x & 31) == 0) rmask[(size_t)r * (kBrickVox / 32) + (threadIdx.x >> 5)] = bal;
        uint32_t tv, tr;
        brick_rank(kept, wc, &tv);
        brick_rank(root, wc, &tr);
        if (threadIdx.x == 0) { nvert[r] = tv; nroot[r] = tr; }
    }
}

// Cluster number of a kept root p: kept roots before its brick (rbase) plus
// kept roots before it in its brick (popcount of the brick's root mask).
__device__ __forceinline__ uint32_t cluster_of(uint32_t p, const uint32_t* __restrict__ rbase,
                                               const uint32_t* __restrict__ rmask) {
    const uint32_t r = p / kBrickVox, l = p % kBrickVox;
    const uint32_t* m = rmask + (size_t)r * (kBrickVox / 32);
    uint32_t c = rbase[r];
    for (uint32_t w = 0; w < (l >> 5); ++w) c += __popc(__ldg(m + w));
    return c + __popc(__ldg(m + (l >> 5)) & ((1u << (l & 31)) - 1u));
}

// (2) in one pass per brick: kept roots numbered in index order (= label
// order) with their sizes and labels, and kept vertices compacted in index
// order as (cluster, index) pairs.
__global__ void __launch_bounds__(kBrickVox) k_brick_clusters(const uint32_t* __restrict__ nsp, uint32_t cap_b,
                                                              const uint32_t* __restrict__ parent,
                                                              const uint32_t* __restrict__ count, uint32_t min_cluster,
                                                              const uint32_t* __restrict__ rbase,
                                                              const uint32_t* __restrict__ vbase,
                                                              const uint32_t* __restrict__ rmask,
                                                              const int32_t* __restrict__ sorted_key,
                                                              uint32_t* __restrict__ cl_size,
                                                              uint32_t* __restrict__ cl_label, uint32_t kcap,
                                                              uint32_t* __restrict__ keys,
                                                              uint32_t* __restrict__ vals,
                                                              SegCounters* __restrict__ ctr) {
    pdl_gate();
    const uint32_t n_sorted = min(*nsp, cap_b);
    __shared__ uint32_t wc[kBrickVox / 32];
    // Clusters beyond the scratch flag a re-run, and the count is clamped for
    // the kernels after this one (nothing here reads it).
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t k = ctr->k;
        ctr->k_need = k;
        if (k > kcap) {
            atomicOr(&ctr->err, kErrScratch);
            ctr->k = kcap;
        }
    }
    for (uint32_t r = blockIdx.x; r < n_sorted; r += gridDim.x) {
        const size_t i = (size_t)r * kBrickVox + threadIdx.x;
        const uint32_t p = parent[i];
        const bool kept = p != kNone && count[p] >= min_cluster;
        uint32_t t;
        const uint32_t vrank = brick_rank(kept, wc, &t);
        const uint32_t rrank = brick_rank(kept && p == (uint32_t)i, wc, &t);
        if (kept) {
            if (p == (uint32_t)i) {
                const uint32_t c = rbase[r] + rrank;
                if (c < kcap) {
                    cl_size[c] = count[i];
                    cl_label[c] = vid_of(i, sorted_key);
                }
            }
            const uint32_t pos = vbase[r] + vrank;
            keys[pos] = cluster_of(p, rbase, rmask);
            vals[pos] = (uint32_t)i;
        }
    }
}



// Cluster formation when every cluster number fits one byte (at most 256
// clusters): the kept (cluster, index) pairs, in index order, are counted per
// tile of 2048 and cluster; the counts are scanned cluster-major (each tile's
// first slot in each cluster, and at tile 0 each cluster's offset); each pair
// then goes, stably, straight to its slot with its mean position and voxel
// id.  This is one pass of a stable radix sort whose scatter writes the
// cluster point lists themselves, so the pairs are neither sorted first nor
// gathered after, and the cluster offsets come from the same scan.
constexpr int kClT = 256, kClWarps = kClT / 32, kClIt = 8, kClTile = kClT * kClIt;

__global__ void __launch_bounds__(kClT) k_cl_hist(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ np,
                                                  uint32_t* __restrict__ ghist, uint32_t* __restrict__ cnt) {
    pdl_gate();
    __shared__ uint32_t h[256];
    const uint32_t n = *np;
    const uint32_t ntu = (n + kClTile - 1) / kClTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = 256u * ntu;  // the scan's length
    if (blockIdx.x >= ntu) return;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kClTile;
    for (int i = 0; i < kClIt; ++i) {
        const uint32_t j = base + i * kClT + threadIdx.x;
        if (j < n) atomicAdd(&h[keys[j] & 255u], 1u);
    }
    __syncthreads();
    ghist[(size_t)threadIdx.x * ntu + blockIdx.x] = h[threadIdx.x];
}

// Stable within a tile: warp w owns pairs [w * 256, w * 256 + 256) of it, in order.
__global__ void __launch_bounds__(kClT) k_cl_scatter(const uint32_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ vals,
                                                     const uint32_t* __restrict__ np, const uint32_t* __restrict__ kp,
                                                     const uint32_t* __restrict__ goff,
                                                     const float4* __restrict__ rec,
                                                     const int32_t* __restrict__ sorted_key,
                                                     float* __restrict__ pts, uint32_t* __restrict__ pt_vid,
                                                     uint32_t* __restrict__ cl_off, SegCounters* __restrict__ ctr) {
    pdl_gate();
    __shared__ uint32_t wc[kClWarps][256];
    const uint32_t n = *np;
    const uint32_t ntu = (n + kClTile - 1) / kClTile;
    if (blockIdx.x == 0) {  // the cluster offsets, closed by the number of clustered points
        const uint32_t k = *kp;
        for (uint32_t c = threadIdx.x; c < k; c += kClT) cl_off[c] = ntu ? goff[(size_t)c * ntu] : 0u;
        if (threadIdx.x == 0) {
            cl_off[k] = n;
            ctr->tot = n;
        }
    }
    if (blockIdx.x >= ntu) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kClWarps * 256; d += kClT) (&wc[0][0])[d] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kClTile + (uint32_t)w * (32 * kClIt);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t rank[kClIt], dig[kClIt];
#pragma unroll
    for (int i = 0; i < kClIt; ++i) {
        const uint32_t j = base + i * 32 + lane;
        const uint32_t d = (j < n) ? (keys[j] & 255u) : 256u;
        dig[i] = d;
        const uint32_t m = __match_any_sync(0xffffffffu, d);
        const uint32_t r = __popc(m & lt);
        const uint32_t b = (d < 256u) ? wc[w][d] : 0u;
        __syncwarp();
        if (d < 256u && r == 0) wc[w][d] = b + __popc(m);
        __syncwarp();
        rank[i] = b + r;
    }
    __syncthreads();
    {   // exclusive offsets of each warp per cluster
        const int d = threadIdx.x;  // kClT == 256 clusters
        uint32_t run = 0;
        for (int q = 0; q < kClWarps; ++q) {
            const uint32_t t = wc[q][d];
            wc[q][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kClIt; ++i) {
        const uint32_t j = base + i * 32 + lane;
        if (j < n) {
            const uint32_t d = dig[i];
            const uint32_t pos = goff[(size_t)d * ntu + blockIdx.x] + wc[w][d] + rank[i];
            const uint32_t v = vals[j];
            const float4 a = rec[v];  // the mean position, as k_moments formed it
            pts[3 * (size_t)pos + 0] = a.x;
            pts[3 * (size_t)pos + 1] = a.y;
            pts[3 * (size_t)pos + 2] = a.z;
            pt_vid[pos] = vid_of(v, sorted_key);
        }
    }
}

// Cluster points in cluster order: mean positions and voxel ids.
__global__ void k_gather(const uint32_t* __restrict__ np, const uint32_t* __restrict__ vals_main,
                         const uint32_t* __restrict__ vals_alt, const uint32_t* __restrict__ kp, int bits,
                         const int32_t* __restrict__ M, size_t stride,
                         const int32_t* __restrict__ sorted_key, Grid g, float* __restrict__ pts,
                         uint32_t* __restrict__ pt_vid) {
    pdl_gate();
    const uint32_t n = *np;
    const uint32_t* __restrict__ vals = sort_result_alt(*kp, bits) ? vals_alt : vals_main;  // where the sort ended
    const float pox = g.po[0], poy = g.po[1], poz = g.po[2];
    for (uint32_t p = blockIdx.x * kT + threadIdx.x; p < n; p += gridDim.x * kT) {
        const uint32_t i = vals[p];
        pts[3 * (size_t)p + 0] = __fadd_rn(pox, __fmul_rn(__int2float_rn(M[i]), kInvQ));
        pts[3 * (size_t)p + 1] = __fadd_rn(poy, __fmul_rn(__int2float_rn(M[stride + i]), kInvQ));
        pts[3 * (size_t)p + 2] = __fadd_rn(poz, __fmul_rn(__int2float_rn(M[2 * stride + i]), kInvQ));
        pt_vid[p] = vid_of(i, sorted_key);
    }
}

inline unsigned grid_for(size_t n, int sms, int per_sm = 8) {
    size_t want = (n + kT - 1) / kT;
    size_t cap = (size_t)sms * per_sm;
    if (want < 1) want = 1;
    return (unsigned)(want < cap ? want : cap);
}

}  // namespace

cudaError_t seg_order_bricks(const int32_t* brick_table, uint32_t nb_total, SegBuffers& b, int sms, cudaStream_t s,
                             uint32_t* zero0, uint32_t* zero1) {
    (void)sms;
    // n_sorted is the counter block's word 0: the pass writes it and clears the others
    static_assert(offsetof(SegCounters, n_sorted) == 0, "the brick count leads the segmentation counters");
    return order_bricks_dev(brick_table, nb_total, b.rank_table, b.sorted_slot, b.sorted_key,
                            reinterpret_cast<uint32_t*>(b.ctr), (int)(sizeof(SegCounters) / 4), zero0, zero1,
                            b.scan_tmp, s, &b.ctr->err);
}

cudaError_t seg_run(const Grid& g, const unsigned long long* S, const uint32_t* C, const vm_segment_params& p,
                    SegBuffers& b, uint32_t kcap, uint32_t* err, int sms, cudaStream_t s, StageHook* hk) {
    // the cross-brick pass fits 8 CTAs an SM only with the largest shared-memory split
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_ccl_cross, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    });
    const uint32_t cap_b = (uint32_t)(b.nv / kBrickVox);
    const size_t stride = b.nv;
    const uint32_t* nsp = &b.ctr->n_sorted;
    const auto clampg = [&](uint32_t want, uint32_t mx) { return want < mx ? (want ? want : 1u) : mx; };
    VM_STAGE_BEGIN(hk, kStFinalize, s);
    launch_k(k_finalize, dim3(clampg(cap_b, sms * 16)), dim3(kT), 0, s, nsp, cap_b, b.sorted_slot, S, C, b.M, b.status,
             stride, b.ctr);
    VM_STAGE_END(hk, kStFinalize, s);
    const uint8_t want = p.classify ? 2 : 1;
    VM_STAGE_BEGIN(hk, kStNormals, s);
    launch_k(k_moments, dim3(clampg(cap_b, sms * 16)), dim3(kNormT), 0, s, nsp, cap_b, g, b.sorted_key, b.rank_table,
             b.M, b.rec, b.list_idx, b.list_A, b.nbr, stride, b.ctr);
    VM_STAGE_END(hk, kStNormals, s);
    VM_STAGE_BEGIN(hk, kStEigen, s);
    launch_k(k_eigen, dim3(clampg((uint32_t)((b.nv + 255) / 256), sms * 16)), dim3(256), 0, s, b.ctr, b.list_idx,
             b.list_A, b.nbr, b.nrm, b.status, b.rec, stride, p.n_th, p.cos_step);
    VM_STAGE_END(hk, kStEigen, s);
    VM_STAGE_BEGIN(hk, kStCclLocal, s);
    launch_k(k_ccl_local, dim3(clampg(cap_b, sms * 16)), dim3(kNormT), 0, s, nsp, cap_b, b.rec, b.parent, b.count,
             stride, want, p.d_th2, p.cos_ccl, err);
    VM_STAGE_END(hk, kStCclLocal, s);
    VM_STAGE_BEGIN(hk, kStCcl, s);
    launch_k(k_ccl_cross, dim3(clampg(cap_b, sms * 16)), dim3(kCrossT), 0, s, nsp, cap_b, g, b.sorted_key, b.rank_table,
             b.rec, b.parent, stride, want, p.d_th2, p.cos_ccl, err);
    VM_STAGE_END(hk, kStCcl, s);
    count_launch(5);
    VM_STAGE_BEGIN(hk, kStClusters, s);
    launch_k(k_compress_count, dim3(grid_for(b.nv, sms)), dim3(kT), 0, s, nsp, cap_b, b.parent, b.count, b.ctr, err);
    const uint32_t min_cl = p.min_cluster ? p.min_cluster : 1u;
    uint32_t* nvert = b.flags;      // per-brick tallies: flags reused for kept vertices,
    uint32_t* nroot = b.vert_flag;  // vert_flag for kept roots,
    uint32_t* rmask = b.cid;        // cid for the kept-root masks (16 words a brick)
    const unsigned bgrid = clampg(cap_b, sms * 4);
    launch_k(k_brick_tally, dim3(bgrid), dim3(kBrickVox), 0, s, nsp, cap_b, b.parent, b.count, min_cl, nvert, nroot,
             rmask);
    cudaError_t e = exclusive_scan2_dev(nroot, nroot, &b.ctr->k, nvert, nvert, &b.ctr->n_kept, nsp, cap_b, b.scan_tmp,
                                        s, err);
    if (e != cudaSuccess) return e;
    launch_k(k_brick_clusters, dim3(bgrid), dim3(kBrickVox), 0, s, nsp, cap_b, b.parent, b.count, min_cl, nroot, nvert,
             rmask, b.sorted_key, b.cl_size, b.cl_label, kcap, b.keys, b.vals, b.ctr);
    if (kcap <= 256) {  // one byte a cluster number: one scatter pass writes the cluster points
        const size_t nt = (b.nv + kClTile - 1) / kClTile;
        uint32_t* ghist = b.sort_tmp;
        uint32_t* cnt = b.sort_tmp + 256 * nt;
        uint32_t* stmp = b.sort_tmp + 256 * nt + 64;
        launch_k(k_cl_hist, dim3((unsigned)nt), dim3(kClT), 0, s, b.keys, &b.ctr->n_kept, ghist, cnt);
        e = exclusive_scan_dev(ghist, ghist, nullptr, cnt, 256 * nt, stmp, s, err);
        if (e != cudaSuccess) return e;
        launch_k(k_cl_scatter, dim3((unsigned)nt), dim3(kClT), 0, s, b.keys, b.vals, &b.ctr->n_kept, &b.ctr->k, ghist,
                 b.rec, b.sorted_key, b.pts, b.pt_vid, b.cl_off, b.ctr);
        VM_STAGE_END(hk, kStClusters, s);
        count_launch(5);
        return cudaGetLastError();
    }
    int bits = 1;
    while ((1ull << bits) < kcap && bits < 32) ++bits;
    e = stable_sort_pairs_dev(b.keys, b.vals, b.keys_alt, b.vals_alt, &b.ctr->n_kept, b.nv, bits, b.sort_tmp, s, err,
                              &b.ctr->k);
    if (e != cudaSuccess) return e;
    // cluster offsets, closed by the number of clustered points at cl_off[k]
    e = exclusive_scan_dev(b.cl_size, b.cl_off, &b.ctr->tot, &b.ctr->k, kcap, b.scan_tmp, s, err, true);
    if (e != cudaSuccess) return e;
    launch_k(k_gather, dim3(grid_for(b.nv, sms)), dim3(kT), 0, s, &b.ctr->n_kept, b.vals, b.vals_alt, &b.ctr->k, bits,
             b.M, b.nv, b.sorted_key, g, b.pts, b.pt_vid);
    VM_STAGE_END(hk, kStClusters, s);
    count_launch(4);
    return cudaGetLastError();
}

}  // namespace vmx
