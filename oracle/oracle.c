/*
 * oracle.c -- plain, slow CPU oracle for voxel integration and
 * multi-plane segmentation ("Real-time Multi-Plane Segmentation Based on GPU
 * Accelerated High-Resolution 3D Voxel Mapping for Legged Robot Locomotion",
 * arXiv 2510.01592).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline and reference legs of the benchmark may load this library.  It
 * shares no code, header, table or constant generator with the CUDA library;
 * the CUDA path never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.  Contraction
 * must stay off: every fused multiply-add below is an explicit fmaf()/fma().
 *
 * Where the paper is silent the readings are fixed here and listed in the
 * design notes; each function names the passage it follows.
 *
 * Parity pins (tests/test_oracle_*.py): every function below is pinned against
 * brute force, closed forms, numpy/scipy routines or invariants.  Nothing here
 * is "parity unpinned".
 *
 * orc_set_threads(n) (default 1) splits the stages whose items are
 * independent -- points of one integration (integer atomics), voxels of the
 * normal computation, clusters of the plane fit -- over n POSIX threads, for
 * the all-cores timing of the CPU baseline; results are identical to one
 * thread.  With one thread every loop below runs exactly as written.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : (n > 256 ? 256 : n); }
int orc_get_threads(void) { return g_threads; }

/* Runs fn(ctx, lo, hi) over contiguous ranges of [0, n) on g_threads threads
 * (the calling thread takes the first range). */
typedef void (*range_fn)(void *ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void *ctx; uint64_t lo, hi; } range_job;
static void *range_thread(void *p)
{
    range_job *j = (range_job *)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}
static void par_for(uint64_t n, range_fn fn, void *ctx)
{
    int t = g_threads;
    if (t <= 1 || n < 2) { fn(ctx, 0, n); return; }
    if ((uint64_t)t > n) t = (int)n;
    range_job jobs[256];
    pthread_t th[256];
    int started[256];
    for (int i = 0; i < t; ++i) {
        jobs[i].fn = fn; jobs[i].ctx = ctx;
        jobs[i].lo = n * (uint64_t)i / (uint64_t)t;
        jobs[i].hi = n * (uint64_t)(i + 1) / (uint64_t)t;
        started[i] = 0;
    }
    for (int i = 1; i < t; ++i) started[i] = pthread_create(&th[i], NULL, range_thread, &jobs[i]) == 0;
    for (int i = 1; i < t; ++i)
        if (!started[i]) range_thread(&jobs[i]);  /* no thread: run it here */
    range_thread(&jobs[0]);
    for (int i = 1; i < t; ++i)
        if (started[i]) pthread_join(th[i], NULL);
}

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_OUT_OF_MEMORY 2

#define BRICK 8
#define BRICK_VOX 512

/* ------------------------------------------------------------------------- */
/* Map: a dense array over every voxel of the grid, indexed by the voxel id.  */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t vid;        /* voxel id (brick-major, see vid_of)            */
    int32_t ijk[3];      /* grid coordinates                              */
    int64_t S[3];        /* quantised coordinate sums, 2^-20 m units      */
    uint32_t c;          /* point count                                   */
    int32_t M[3];        /* exact integer mean, 2^-20 m units             */
    float mu[3];         /* mean position, map frame                      */
    float n[3];          /* normal (Eq. 3)                                */
    uint32_t nbr;        /* N: occupied neighbours in the window          */
    uint32_t status;     /* 1 occupied, 2 steppable (Eq. 4)               */
    uint32_t label;      /* CCL label (min vid of the component), or ~0   */
} orc_voxel;

typedef struct {
    uint32_t label;
    uint32_t n_points;
    uint32_t inlier_count;
    int32_t best_h;          /* -1: every hypothesis degenerate, no plane    */
    int32_t ill_conditioned; /* refit: lambda_mid < 10 lambda_min             */
    float ransac_n[3];
    float ransac_d;
    double refit_n[3];
    double refit_d;
    float basis_u[3];
    float basis_v[3];
    float origin[3];
    uint32_t hull_off;
    uint32_t hull_n;
    uint32_t point_off;      /* offset of this cluster in the point arrays    */
    uint32_t round;          /* extraction round of this plane in its cluster */
    double cond;             /* refit: lambda_mid / lambda_min (inf when only lambda_min is 0, NaN when both are) */
} orc_plane;

typedef struct {
    int32_t nx, ny, nz;
    int32_t nbx, nby, nbz;
    float ox, oy, oz;    /* base origin: a point's key is floor((p - origin) * inv_res) */
    float inv_res;
    int32_t w[3];        /* window: the grid holds keys w .. w + dims - 1 (w a multiple of 8) */
    int64_t A[3];        /* sums are rint((p - origin) * 2^20) - A, A = anchor(w)          */
    float po[3];         /* origin of the mean positions: origin + A * 2^-20, rounded        */
    uint64_t nv;
    int64_t *S;      /* [nv][3] */
    uint32_t *C;     /* [nv]    */
    uint64_t n_in, n_dropped, n_evicted;
    /* last segmentation */
    orc_voxel *vox;  /* occupied voxels in vid order */
    uint32_t n_vox;
} orc_map;

typedef struct {
    uint32_t n_th;       /* Eq. 4 N_th */
    float cos_step;      /* cos(theta_th) of Eq. 4                      */
    float d_th2;         /* d_th^2 of Algorithm 1                       */
    float cos_ccl;       /* cos of Algorithm 1's normal-angle threshold */
    uint32_t min_cluster;
    uint32_t n_hyp;      /* RANSAC iterations I                         */
    float eps;           /* RANSAC inlier threshold epsilon             */
    uint64_t seed;
    uint32_t classify;   /* 1: cluster steppable voxels only (paper); 0: all occupied */
    uint32_t planes_per_cluster; /* extraction rounds per cluster; 0 or 1: one plane (paper) */
} orc_params;

/* Planes / hulls / per-point results of the last fit, owned by a result set. */
typedef struct {
    orc_plane *planes;
    uint32_t n_planes;
    int32_t *hull_xy;    /* [n_hull][2] */
    uint32_t n_hull, cap_hull;
    float *pts;          /* [n_pts][3] cluster points in cluster order */
    uint32_t *pt_vid;    /* [n_pts] voxel id of each cluster point (segment only) */
    uint8_t *inlier;     /* [n_pts] inlier flag under the selected hypothesis */
    uint32_t n_pts;
} orc_result;

/* Voxel id: brick-major linear index.  Bricks of 8^3 voxels are numbered
 * x-fastest over the brick grid, voxels inside a brick x-fastest.  The paper
 * fixes no voxel order; this one is a bijection with grid coordinates. */
static uint64_t vid_of(const orc_map *m, int i, int j, int k)
{
    uint64_t b = ((uint64_t)(k / BRICK) * (uint64_t)m->nby + (uint64_t)(j / BRICK)) * (uint64_t)m->nbx
                 + (uint64_t)(i / BRICK);
    uint64_t l = (uint64_t)(((k % BRICK) * BRICK + (j % BRICK)) * BRICK + (i % BRICK));
    return b * BRICK_VOX + l;
}

static void ijk_of(const orc_map *m, uint64_t vid, int32_t ijk[3])
{
    uint64_t b = vid / BRICK_VOX, l = vid % BRICK_VOX;
    int bx = (int)(b % (uint64_t)m->nbx);
    int by = (int)((b / (uint64_t)m->nbx) % (uint64_t)m->nby);
    int bz = (int)(b / ((uint64_t)m->nbx * (uint64_t)m->nby));
    ijk[0] = bx * BRICK + (int)(l % BRICK);
    ijk[1] = by * BRICK + (int)((l / BRICK) % BRICK);
    ijk[2] = bz * BRICK + (int)(l / (BRICK * BRICK));
}

void *orc_map_create(const int32_t dims[3], const float origin[3], float inv_res)
{
    if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0 || !(inv_res > 0.0f)) return NULL;
    orc_map *m = (orc_map *)calloc(1, sizeof(orc_map));
    if (!m) return NULL;
    m->nx = dims[0]; m->ny = dims[1]; m->nz = dims[2];
    m->nbx = (m->nx + BRICK - 1) / BRICK;
    m->nby = (m->ny + BRICK - 1) / BRICK;
    m->nbz = (m->nz + BRICK - 1) / BRICK;
    m->ox = origin[0]; m->oy = origin[1]; m->oz = origin[2];
    m->inv_res = inv_res;
    m->po[0] = origin[0]; m->po[1] = origin[1]; m->po[2] = origin[2];  /* w = 0: A = 0 */
    m->nv = (uint64_t)m->nbx * (uint64_t)m->nby * (uint64_t)m->nbz * BRICK_VOX;
    if (m->nv > 0xFFFFFFFFull) { free(m); return NULL; }
    m->S = (int64_t *)calloc(m->nv * 3, sizeof(int64_t));
    m->C = (uint32_t *)calloc(m->nv, sizeof(uint32_t));
    if (!m->S || !m->C) { free(m->S); free(m->C); free(m); return NULL; }
    return m;
}

void orc_map_destroy(void *h)
{
    orc_map *m = (orc_map *)h;
    if (!m) return;
    free(m->S); free(m->C); free(m->vox); free(m);
}

/* Section III.B, Eq. 1 and the thread-per-point update it describes.
 * Reading: the pose is sensor->map, row-major [R|t]; the transform is the
 * fma chain below; the voxel key is floor(d * inv_res) of the offset d from
 * the map's base origin, and the grid index is the key minus the window
 * offset w (0 until the map scrolls); points whose index falls outside the
 * grid (NaN included) are dropped and counted.  Eq. 1's running mean is kept
 * as exact integer sums of rint(d * 2^20) - A (2^-20 m ~ 0.95 um units, A
 * the window's anchor) plus a count: the mean it defines is recovered in
 * orc_segment up to that quantum, independent of point order. */
typedef struct { orc_map *m; const float *xyz; const float *pose; } integ_ctx;
static void integrate_range(void *vc, uint64_t lo, uint64_t hi)
{
    integ_ctx *cx = (integ_ctx *)vc;
    orc_map *m = cx->m;
    const float *xyz = cx->xyz, *pose = cx->pose;
    const int atomic = g_threads > 1;  /* integer sums: the same in any order */
    const float q = 1048576.0f; /* 2^20 */
    for (uint64_t p = lo; p < hi; ++p) {
        float x = xyz[3 * p + 0], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
        float wx = fmaf(pose[2], z, fmaf(pose[1], y, fmaf(pose[0], x, pose[3])));
        float wy = fmaf(pose[6], z, fmaf(pose[5], y, fmaf(pose[4], x, pose[7])));
        float wz = fmaf(pose[10], z, fmaf(pose[9], y, fmaf(pose[8], x, pose[11])));
        float dx = wx - m->ox, dy = wy - m->oy, dz = wz - m->oz;
        float fx = floorf(dx * m->inv_res), fy = floorf(dy * m->inv_res), fz = floorf(dz * m->inv_res);
        /* the window bounds are integers below 2^24: exact as floats */
        int ok = (fx >= (float)m->w[0]) && (fx < (float)(m->w[0] + m->nx)) && (fy >= (float)m->w[1]) &&
                 (fy < (float)(m->w[1] + m->ny)) && (fz >= (float)m->w[2]) && (fz < (float)(m->w[2] + m->nz));
        uint64_t v = ok ? vid_of(m, (int)fx - m->w[0], (int)fy - m->w[1], (int)fz - m->w[2]) : 0;
        int64_t F[3] = {0, 0, 0};
        if (ok) {
            F[0] = (int64_t)rintf(dx * q) - m->A[0];
            F[1] = (int64_t)rintf(dy * q) - m->A[1];
            F[2] = (int64_t)rintf(dz * q) - m->A[2];
        }
        if (!atomic) {
            if (!ok) { m->n_dropped++; continue; }
            m->S[3 * v + 0] += F[0];
            m->S[3 * v + 1] += F[1];
            m->S[3 * v + 2] += F[2];
            m->C[v] += 1u;
            m->n_in++;
        } else {
            if (!ok) { __atomic_fetch_add(&m->n_dropped, 1, __ATOMIC_RELAXED); continue; }
            __atomic_fetch_add(&m->S[3 * v + 0], F[0], __ATOMIC_RELAXED);
            __atomic_fetch_add(&m->S[3 * v + 1], F[1], __ATOMIC_RELAXED);
            __atomic_fetch_add(&m->S[3 * v + 2], F[2], __ATOMIC_RELAXED);
            __atomic_fetch_add(&m->C[v], 1u, __ATOMIC_RELAXED);
            __atomic_fetch_add(&m->n_in, 1, __ATOMIC_RELAXED);
        }
    }
}

int orc_integrate(void *h, const float *xyz, uint64_t n, const float pose[12])
{
    orc_map *m = (orc_map *)h;
    if (!m || (!xyz && n)) return ORC_ERR_INVALID_ARG;
    integ_ctx cx = {m, xyz, pose};
    par_for(n, integrate_range, &cx);
    return ORC_OK;
}

/* Section III.B, Eq. 2 (voxel information clearing): the voxels that the ray
 * from the sensor to a point passes through are free space; a voxel that at
 * least one ray of the frame passes through (n_i > 0) is cleared.  Reading:
 * the traversal is a monotone 6-connected walk in voxel units from the
 * sensor's voxel to the point's voxel (Amanatides and Woo's grid traversal,
 * 1987): s = (t - origin) * inv_res and e = (p' - origin) * inv_res in FP32
 * (p' is the point in the map frame, keyed exactly as orc_integrate keys it),
 * d = e - s; per axis the parameter of the next voxel boundary
 * tmax = (boundary - s) / d and its increment tdelta = 1 / |d|; each step
 * advances the axis with the smallest tmax (ties to x, then y, then z) among
 * the axes not yet at the end voxel's coordinate, so the walk reaches the
 * end voxel in exactly |ve - v0| (L1) steps.  Every voxel walked before the
 * end voxel is marked if it lies in the grid (its key minus the window
 * offset w in range); the end voxel (the point's own) is not.  The walk stops
 * once it leaves the grid (a monotone walk does not come back).  A sensor
 * outside the grid casts no rays (a robot-centric map holds its sensor);
 * points that are not finite, or more than 2^30 voxels away, cast no ray.
 * All marks of the frame are collected first, then the marked voxels are
 * cleared (sums and count to zero); integrating the frame's points follows. */
typedef struct { orc_map *m; const float *xyz; const float *pose; uint8_t *mark; } clear_ctx;
static void clear_range(void *vc, uint64_t lo, uint64_t hi)
{
    clear_ctx *cx = (clear_ctx *)vc;
    orc_map *m = cx->m;
    const float *xyz = cx->xyz, *pose = cx->pose;
    const int dims[3] = {m->nx, m->ny, m->nz};
    const float org[3] = {m->ox, m->oy, m->oz};
    const float tr[3] = {pose[3], pose[7], pose[11]};
    float s[3];
    for (int a = 0; a < 3; ++a) s[a] = (tr[a] - org[a]) * m->inv_res;
    for (uint64_t p = lo; p < hi; ++p) {
        float x = xyz[3 * p + 0], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
        float w[3];
        w[0] = fmaf(pose[2], z, fmaf(pose[1], y, fmaf(pose[0], x, pose[3])));
        w[1] = fmaf(pose[6], z, fmaf(pose[5], y, fmaf(pose[4], x, pose[7])));
        w[2] = fmaf(pose[10], z, fmaf(pose[9], y, fmaf(pose[8], x, pose[11])));
        float e[3];
        int fin = 1;
        for (int a = 0; a < 3; ++a) {
            e[a] = (w[a] - org[a]) * m->inv_res;
            fin &= isfinite(e[a]) && fabsf(e[a]) < 1073741824.0f;
        }
        if (!fin) continue;
        int64_t v[3], ve[3];
        int step[3];
        float tmax[3], tdel[3];
        int64_t left = 0;
        for (int a = 0; a < 3; ++a) {
            v[a] = (int64_t)floorf(s[a]);
            ve[a] = (int64_t)floorf(e[a]);
            const float d = e[a] - s[a];
            if (d > 0.0f) {
                step[a] = 1;
                tmax[a] = ((float)(v[a] + 1) - s[a]) / d;
                tdel[a] = 1.0f / d;
            } else if (d < 0.0f) {
                step[a] = -1;
                tmax[a] = ((float)v[a] - s[a]) / d;
                tdel[a] = -1.0f / d;
            } else {
                step[a] = 0;
                tmax[a] = INFINITY;
                tdel[a] = INFINITY;
            }
            left += ve[a] > v[a] ? ve[a] - v[a] : v[a] - ve[a];
        }
        for (; left > 0; --left) {
            int inside = 1, gone = 0;
            for (int a = 0; a < 3; ++a) {
                const int64_t g = v[a] - m->w[a];
                inside &= g >= 0 && g < dims[a];
                gone |= (g < 0 && step[a] <= 0) || (g >= dims[a] && step[a] >= 0);
            }
            if (gone) break;
            if (inside) {
                const uint64_t vid = vid_of(m, (int)(v[0] - m->w[0]), (int)(v[1] - m->w[1]), (int)(v[2] - m->w[2]));
                if (m->C[vid]) __atomic_store_n(&cx->mark[vid], (uint8_t)1, __ATOMIC_RELAXED);
            }
            int best = -1;
            for (int a = 0; a < 3; ++a) {
                if (v[a] == ve[a]) continue;
                if (best < 0 || tmax[a] < tmax[best]) best = a;
            }
            v[best] += step[best];
            tmax[best] += tdel[best];
        }
    }
}

int orc_clear_rays(void *h, const float *xyz, uint64_t n, const float pose[12], uint64_t *cleared)
{
    orc_map *m = (orc_map *)h;
    if (!m || (!xyz && n)) return ORC_ERR_INVALID_ARG;
    uint8_t *mark = (uint8_t *)calloc(m->nv ? m->nv : 1, 1);
    if (!mark) return ORC_ERR_OUT_OF_MEMORY;
    clear_ctx cx = {m, xyz, pose, mark};
    const float sv[3] = {(pose[3] - m->ox) * m->inv_res, (pose[7] - m->oy) * m->inv_res,
                         (pose[11] - m->oz) * m->inv_res};
    const int sensor_in = sv[0] >= (float)m->w[0] && sv[0] < (float)(m->w[0] + m->nx) &&
                          sv[1] >= (float)m->w[1] && sv[1] < (float)(m->w[1] + m->ny) &&
                          sv[2] >= (float)m->w[2] && sv[2] < (float)(m->w[2] + m->nz);
    if (sensor_in) par_for(n, clear_range, &cx);
    uint64_t k = 0;
    for (uint64_t v = 0; v < m->nv; ++v) {
        if (!mark[v]) continue;
        m->S[3 * v + 0] = m->S[3 * v + 1] = m->S[3 * v + 2] = 0;
        m->C[v] = 0;
        ++k;
    }
    free(mark);
    if (cleared) *cleared = k;
    return ORC_OK;
}

void orc_map_counts(void *h, uint64_t out[2])
{
    orc_map *m = (orc_map *)h;
    out[0] = m->n_in;
    out[1] = m->n_dropped;
}

/* Robot-centric map (Sec. III.B: the map's centre follows the robot).
 * Reading: the grid is a window over keys anchored at the base origin, moved
 * in whole bricks so that every kept voxel keeps its key, its points and its
 * exact sums; a voxel whose brick leaves the window is dropped (evicted) and
 * the bricks that enter are empty.  The sums are re-expressed against the
 * new window's anchor, an integer change: S -= C * (A' - A).  The anchor is
 * A = floor(w * 2^20 / inv_res) in double (at or below the window's corner
 * in 2^-20 m units, so sums stay small), and mean positions are
 * po + M * 2^-20 with po = (float)(origin + A * 2^-20) in double. */
static int64_t anchor_of(int32_t w, float inv_res)
{
    return (int64_t)floor((double)w * 1048576.0 / (double)inv_res);
}

int orc_map_scroll(void *h, const int32_t shift[3])
{
    orc_map *m = (orc_map *)h;
    if (!m || !shift) return ORC_ERR_INVALID_ARG;
    int32_t w2[3];
    for (int a = 0; a < 3; ++a) {
        const int64_t t = (int64_t)m->w[a] + 8 * (int64_t)shift[a];
        if (t < -(1 << 23) || t > (1 << 23)) return ORC_ERR_INVALID_ARG;  /* keys stay exact in FP32 */
        w2[a] = (int32_t)t;
    }
    int64_t A2[3], dA[3];
    for (int a = 0; a < 3; ++a) {
        A2[a] = anchor_of(w2[a], m->inv_res);
        dA[a] = A2[a] - m->A[a];
    }
    int64_t *S2 = (int64_t *)calloc(m->nv * 3, sizeof(int64_t));
    uint32_t *C2 = (uint32_t *)calloc(m->nv, sizeof(uint32_t));
    if (!S2 || !C2) { free(S2); free(C2); return ORC_ERR_OUT_OF_MEMORY; }
    /* every voxel of the old window: keep it if its key is in the new window */
    for (uint64_t v = 0; v < m->nv; ++v) {
        if (!m->C[v]) continue;
        int32_t ijk[3];
        ijk_of(m, v, ijk);
        int keep = 1;
        int32_t g[3];
        for (int a = 0; a < 3; ++a) {
            g[a] = ijk[a] + m->w[a] - w2[a];
            keep &= g[a] >= 0 && g[a] < (a == 0 ? m->nx : a == 1 ? m->ny : m->nz);
        }
        if (!keep) { m->n_evicted++; continue; }
        const uint64_t u = vid_of(m, g[0], g[1], g[2]);
        for (int a = 0; a < 3; ++a) S2[3 * u + a] = m->S[3 * v + a] - (int64_t)m->C[v] * dA[a];
        C2[u] = m->C[v];
    }
    free(m->S); free(m->C);
    m->S = S2; m->C = C2;
    const float o[3] = {m->ox, m->oy, m->oz};
    for (int a = 0; a < 3; ++a) {
        m->w[a] = w2[a];
        m->A[a] = A2[a];
        m->po[a] = (float)((double)o[a] + (double)A2[a] / 1048576.0);
    }
    return ORC_OK;
}

/* The brick shift that centres the window on c (map frame): the key of c,
 * floor((c - origin) * inv_res) in FP32 as a point is keyed, minus half the
 * grid, rounded down to a whole brick, is the new window offset. */
void orc_scroll_target(void *h, const float c[3], int32_t shift[3])
{
    orc_map *m = (orc_map *)h;
    const float o[3] = {m->ox, m->oy, m->oz};
    const int32_t n[3] = {m->nx, m->ny, m->nz};
    for (int a = 0; a < 3; ++a) {
        const int64_t key = (int64_t)floorf((c[a] - o[a]) * m->inv_res);
        int64_t t = key - n[a] / 2;
        t = (t >= 0 ? t / 8 : -((-t + 7) / 8));  /* floor(t / 8) */
        shift[a] = (int32_t)(t - m->w[a] / 8);
    }
}

void orc_map_window(void *h, int32_t w[3], int64_t A[3], float po[3], uint64_t *evicted)
{
    orc_map *m = (orc_map *)h;
    for (int a = 0; a < 3; ++a) {
        if (w) w[a] = m->w[a];
        if (A) A[a] = m->A[a];
        if (po) po[a] = m->po[a];
    }
    if (evicted) *evicted = m->n_evicted;
}

/* Occupied voxels in vid order with their sums and counts. */
uint32_t orc_count_occupied(void *h)
{
    orc_map *m = (orc_map *)h;
    uint32_t k = 0;
    for (uint64_t v = 0; v < m->nv; ++v) k += (m->C[v] > 0);
    return k;
}

void orc_export_sums(void *h, uint32_t *vid, int64_t *S, uint32_t *C)
{
    orc_map *m = (orc_map *)h;
    uint32_t k = 0;
    for (uint64_t v = 0; v < m->nv; ++v) {
        if (!m->C[v]) continue;
        vid[k] = (uint32_t)v;
        S[3 * k + 0] = m->S[3 * v + 0]; S[3 * k + 1] = m->S[3 * v + 1]; S[3 * k + 2] = m->S[3 * v + 2];
        C[k] = m->C[v];
        ++k;
    }
}

/* ------------------------------------------------------------------------- */
/* Symmetric 3x3 eigen-solver: cyclic Jacobi (Golub & Van Loan, Sec. 8.5).   */
/* ------------------------------------------------------------------------- */

/* FP32 cyclic Jacobi, pairs (0,1), (0,2), (1,2), a fixed number of sweeps.
 * a = {a00, a11, a22, a01, a02, a12}.  On return v holds the eigenvectors as
 * columns (v[r][c]) and d the diagonal.  A pair with a_pq == 0 is skipped.
 * Rotation: tau = (a_qq - a_pp) / (2 a_pq); t = sgn(tau)/(|tau| + sqrt(1+tau^2))
 * with sgn(0) = +1; c = 1/sqrt(1+t^2); s = t c. */
static void jacobi3_f32(const float a_in[6], int sweeps, float v[3][3], float d[3])
{
    float a[3][3] = {{a_in[0], a_in[3], a_in[4]}, {a_in[3], a_in[1], a_in[5]}, {a_in[4], a_in[5], a_in[2]}};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) v[r][c] = (r == c) ? 1.0f : 0.0f;
    static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2}, R[3] = {2, 1, 0};
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k], r = R[k];
            float apq = a[p][q];
            if (apq == 0.0f) continue;
            float app = a[p][p], aqq = a[q][q];
            float tau = (aqq - app) / (2.0f * apq);
            float sg = (tau >= 0.0f) ? 1.0f : -1.0f;
            float t = sg / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
            float c = 1.0f / sqrtf(fmaf(t, t, 1.0f));
            float s = t * c;
            a[p][p] = fmaf(-t, apq, app);
            a[q][q] = fmaf(t, apq, aqq);
            a[p][q] = 0.0f; a[q][p] = 0.0f;
            float arp = a[r][p], arq = a[r][q];
            float nrp = fmaf(c, arp, -(s * arq));
            float nrq = fmaf(s, arp, c * arq);
            a[r][p] = nrp; a[p][r] = nrp;
            a[r][q] = nrq; a[q][r] = nrq;
            for (int i = 0; i < 3; ++i) {
                float vip = v[i][p], viq = v[i][q];
                v[i][p] = fmaf(c, vip, -(s * viq));
                v[i][q] = fmaf(s, vip, c * viq);
            }
        }
    }
    d[0] = a[0][0]; d[1] = a[1][1]; d[2] = a[2][2];
}

/* Normal from a Jacobi result: the column of the smallest diagonal entry
 * (lowest index on ties), scaled by 1/sqrt(n.n), oriented n_z >= 0 (then
 * n_y >= 0, then n_x >= 0 when the earlier components are zero). */
static void pick_normal_f32(float v[3][3], const float d[3], float n[3])
{
    int m = 0;
    if (d[1] < d[m]) m = 1;
    if (d[2] < d[m]) m = 2;
    float x = v[0][m], y = v[1][m], z = v[2][m];
    float nn = fmaf(z, z, fmaf(y, y, x * x));
    float inv = 1.0f / sqrtf(nn);
    x = x * inv; y = y * inv; z = z * inv;
    int flip = (z < 0.0f) || (z == 0.0f && (y < 0.0f || (y == 0.0f && x < 0.0f)));
    if (flip) { x = -x; y = -y; z = -z; }
    n[0] = x; n[1] = y; n[2] = z;
}

/* Exposed for the pins: FP32 Jacobi on a given symmetric matrix. */
void orc_jacobi3_f32(const float a[6], int sweeps, float n_out[3], float d_out[3], float v_out[9])
{
    float v[3][3], d[3];
    jacobi3_f32(a, sweeps, v, d);
    pick_normal_f32(v, d, n_out);
    for (int i = 0; i < 3; ++i) d_out[i] = d[i];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) v_out[3 * r + c] = v[r][c];
}

/* Double-precision cyclic Jacobi (same rotation, no fused operations), used by
 * the refit. */
static void jacobi3_f64(const double a_in[6], int sweeps, double v[3][3], double d[3])
{
    double a[3][3] = {{a_in[0], a_in[3], a_in[4]}, {a_in[3], a_in[1], a_in[5]}, {a_in[4], a_in[5], a_in[2]}};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) v[r][c] = (r == c) ? 1.0 : 0.0;
    static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2}, R[3] = {2, 1, 0};
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k], r = R[k];
            double apq = a[p][q];
            if (apq == 0.0) continue;
            double app = a[p][p], aqq = a[q][q];
            double tau = (aqq - app) / (2.0 * apq);
            double sg = (tau >= 0.0) ? 1.0 : -1.0;
            double t = sg / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = 1.0 / sqrt(1.0 + t * t);
            double s = t * c;
            a[p][p] = app - t * apq;
            a[q][q] = aqq + t * apq;
            a[p][q] = 0.0; a[q][p] = 0.0;
            double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
            for (int i = 0; i < 3; ++i) {
                double vip = v[i][p], viq = v[i][q];
                v[i][p] = c * vip - s * viq;
                v[i][q] = s * vip + c * viq;
            }
        }
    }
    d[0] = a[0][0]; d[1] = a[1][1]; d[2] = a[2][2];
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.    */
/* ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ull; /* golden ratio Weyl increment */
            k1 += 0xBB67AE8584CAA73Bull; /* sqrt(3) - 1 Weyl increment  */
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, x0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ull, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* Per-cluster plane fit: RANSAC (Sec. III.C, stages a-c), refit, hull.       */
/* ------------------------------------------------------------------------- */

/* Hypothesis h of a cluster with the given label: three sample indices from
 * Philox4x64-10 with counter (label, h, 0, 0) and key (seed, 0); index
 * k = floor(r * n / 2^64).  Returns 0 for a degenerate sample (repeated index
 * or zero cross product). */
static int ransac_hypothesis(const float *pts, uint32_t n, uint32_t label, uint32_t h, uint32_t round,
                             uint64_t seed, float nrm[3], float *dd)
{
    uint64_t ctr[4] = {label, h, round, 0}, key[2] = {seed, 0}, r[4];
    orc_philox4x64(ctr, key, r);
    uint64_t k[3], lo;
    for (int i = 0; i < 3; ++i) mulhilo64(r[i], (uint64_t)n, &k[i], &lo);
    if (k[0] == k[1] || k[0] == k[2] || k[1] == k[2]) return 0;
    const float *p0 = pts + 3 * k[0], *p1 = pts + 3 * k[1], *p2 = pts + 3 * k[2];
    float e1x = p1[0] - p0[0], e1y = p1[1] - p0[1], e1z = p1[2] - p0[2];
    float e2x = p2[0] - p0[0], e2y = p2[1] - p0[1], e2z = p2[2] - p0[2];
    float cx = fmaf(e1y, e2z, -(e1z * e2y));
    float cy = fmaf(e1z, e2x, -(e1x * e2z));
    float cz = fmaf(e1x, e2y, -(e1y * e2x));
    float nn = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
    if (!(nn > 0.0f)) return 0;
    float inv = 1.0f / sqrtf(nn);
    nrm[0] = cx * inv; nrm[1] = cy * inv; nrm[2] = cz * inv;
    *dd = -fmaf(nrm[2], p0[2], fmaf(nrm[1], p0[1], nrm[0] * p0[0]));
    return 1;
}

/* Point-to-plane distance as the inlier test evaluates it (Sec. III.C b). */
static float plane_dist(const float nrm[3], float d, const float *p)
{
    return fabsf(fmaf(nrm[2], p[2], fmaf(nrm[1], p[1], fmaf(nrm[0], p[0], d))));
}

/* Exposed for the pins: the inlier count of every hypothesis of one cluster
 * (-1 for a degenerate sample), and the selected index under the rule "max
 * count, lowest h on ties". */
int32_t orc_ransac_counts(const float *pts, uint32_t n, uint32_t label, uint32_t n_hyp, uint64_t seed, float eps,
                          int64_t *counts, float *planes4)
{
    int32_t best_h = -1;
    int64_t best = -1;
    for (uint32_t h = 0; h < n_hyp; ++h) {
        float nrm[3], d;
        counts[h] = -1;
        planes4[4 * h] = planes4[4 * h + 1] = planes4[4 * h + 2] = planes4[4 * h + 3] = 0.0f;
        if (!ransac_hypothesis(pts, n, label, h, 0, seed, nrm, &d)) continue;
        int64_t cnt = 0;
        for (uint32_t k = 0; k < n; ++k) cnt += (plane_dist(nrm, d, pts + 3 * k) <= eps);
        counts[h] = cnt;
        planes4[4 * h] = nrm[0]; planes4[4 * h + 1] = nrm[1]; planes4[4 * h + 2] = nrm[2]; planes4[4 * h + 3] = d;
        if (cnt > best) { best = cnt; best_h = (int32_t)h; }
    }
    return best_h;
}

static int cmp_xy(const void *a, const void *b)
{
    const int32_t *u = (const int32_t *)a, *w = (const int32_t *)b;
    if (u[0] != w[0]) return u[0] < w[0] ? -1 : 1;
    if (u[1] != w[1]) return u[1] < w[1] ? -1 : 1;
    return 0;
}

static int64_t cross_i64(const int32_t *o, const int32_t *a, const int32_t *b)
{
    return ((int64_t)a[0] - o[0]) * ((int64_t)b[1] - o[1]) - ((int64_t)a[1] - o[1]) * ((int64_t)b[0] - o[0]);
}

/* Andrew's monotone chain on integer points: sort by (X, Y), drop duplicates,
 * keep strict left turns only.  Output counter-clockwise from the
 * lexicographically smallest point.  xy is sorted in place.  Returns the
 * vertex count written to hull (room for n + 1 points). */
uint32_t orc_hull_i32(int32_t *xy, uint32_t n, int32_t *hull)
{
    if (n == 0) return 0;
    qsort(xy, n, 2 * sizeof(int32_t), cmp_xy);
    uint32_t u = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (u && xy[2 * i] == xy[2 * (u - 1)] && xy[2 * i + 1] == xy[2 * (u - 1) + 1]) continue;
        xy[2 * u] = xy[2 * i]; xy[2 * u + 1] = xy[2 * i + 1]; ++u;
    }
    if (u < 3) {
        for (uint32_t i = 0; i < u; ++i) { hull[2 * i] = xy[2 * i]; hull[2 * i + 1] = xy[2 * i + 1]; }
        return u;
    }
    uint32_t k = 0;
    for (uint32_t i = 0; i < u; ++i) { /* lower chain */
        while (k >= 2 && cross_i64(hull + 2 * (k - 2), hull + 2 * (k - 1), xy + 2 * i) <= 0) --k;
        hull[2 * k] = xy[2 * i]; hull[2 * k + 1] = xy[2 * i + 1]; ++k;
    }
    uint32_t lower = k + 1;
    for (uint32_t i = u - 1; i-- > 0;) { /* upper chain */
        while (k >= lower && cross_i64(hull + 2 * (k - 2), hull + 2 * (k - 1), xy + 2 * i) <= 0) --k;
        hull[2 * k] = xy[2 * i]; hull[2 * k + 1] = xy[2 * i + 1]; ++k;
    }
    return k - 1; /* the last point repeats the first */
}

static int push_hull(orc_result *r, const int32_t *h, uint32_t k)
{
    if (r->n_hull + k > r->cap_hull) {
        uint32_t cap = r->cap_hull ? r->cap_hull : 1024;
        while (cap < r->n_hull + k) cap *= 2;
        int32_t *nh = (int32_t *)realloc(r->hull_xy, (size_t)cap * 2 * sizeof(int32_t));
        if (!nh) return ORC_ERR_OUT_OF_MEMORY;
        r->hull_xy = nh; r->cap_hull = cap;
    }
    memcpy(r->hull_xy + 2 * r->n_hull, h, (size_t)k * 2 * sizeof(int32_t));
    r->n_hull += k;
    return ORC_OK;
}

/* One cluster: RANSAC (Sec. III.C stages a-c), refit, boundary polygon
 * (Sec. III.C, boundary polygon generation).  pts are the cluster's points in
 * cluster order; inl receives the inlier flags. */
static int fit_cluster(const float *pts, uint32_t n, uint32_t label, uint32_t round, const orc_params *prm,
                       orc_plane *pl, uint8_t *inl, orc_result *res)
{
    memset(pl, 0, sizeof(*pl));
    pl->label = label;
    pl->n_points = n;
    pl->best_h = -1;
    pl->round = round;
    memset(inl, 0, n);
    /* a) hypotheses, b) inlier counting, c) selection: max count, lowest h on ties */
    int64_t best = -1;
    float bn[3] = {0, 0, 0}, bd = 0.0f;
    for (uint32_t h = 0; h < prm->n_hyp; ++h) {
        float nrm[3], d;
        if (!ransac_hypothesis(pts, n, label, h, round, prm->seed, nrm, &d)) continue;
        int64_t cnt = 0;
        for (uint32_t k = 0; k < n; ++k) cnt += (plane_dist(nrm, d, pts + 3 * k) <= prm->eps);
        if (cnt > best) { best = cnt; pl->best_h = (int32_t)h; bn[0] = nrm[0]; bn[1] = nrm[1]; bn[2] = nrm[2]; bd = d; }
    }
    if (pl->best_h < 0) return ORC_OK;
    pl->ransac_n[0] = bn[0]; pl->ransac_n[1] = bn[1]; pl->ransac_n[2] = bn[2]; pl->ransac_d = bd;
    /* c) inlier extraction under the selected hypothesis */
    uint32_t ni = 0;
    for (uint32_t k = 0; k < n; ++k) {
        inl[k] = (plane_dist(bn, bd, pts + 3 * k) <= prm->eps);
        ni += inl[k];
    }
    pl->inlier_count = ni;
    if (ni == 0) return ORC_OK;
    /* refit: total least squares on the inliers, in double, two passes */
    double c0 = 0, c1 = 0, c2 = 0;
    for (uint32_t k = 0; k < n; ++k)
        if (inl[k]) { c0 += pts[3 * k]; c1 += pts[3 * k + 1]; c2 += pts[3 * k + 2]; }
    c0 /= ni; c1 /= ni; c2 /= ni;
    double A[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t k = 0; k < n; ++k) {
        if (!inl[k]) continue;
        double x = pts[3 * k] - c0, y = pts[3 * k + 1] - c1, z = pts[3 * k + 2] - c2;
        A[0] += x * x; A[1] += y * y; A[2] += z * z; A[3] += x * y; A[4] += x * z; A[5] += y * z;
    }
    double V[3][3], D[3];
    jacobi3_f64(A, 10, V, D);
    int m = 0;
    if (D[1] < D[m]) m = 1;
    if (D[2] < D[m]) m = 2;
    double rx = V[0][m], ry = V[1][m], rz = V[2][m];
    double rl = sqrt(rx * rx + ry * ry + rz * rz);
    rx /= rl; ry /= rl; rz /= rl;
    if (rz < 0.0 || (rz == 0.0 && (ry < 0.0 || (ry == 0.0 && rx < 0.0)))) { rx = -rx; ry = -ry; rz = -rz; }
    pl->refit_n[0] = rx; pl->refit_n[1] = ry; pl->refit_n[2] = rz;
    pl->refit_d = -(rx * c0 + ry * c1 + rz * c2);
    double lo = D[m], mid;
    {
        double e[3] = {D[0], D[1], D[2]};
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j)
                if (e[j] < e[i]) { double t = e[i]; e[i] = e[j]; e[j] = t; }
        mid = e[1];
        lo = e[0];
    }
    pl->ill_conditioned = !(mid >= 10.0 * lo);
    pl->cond = lo > 0.0 ? mid / lo : (mid > 0.0 ? INFINITY : NAN);
    /* hull: in-plane basis from the RANSAC normal, origin = the cluster's first
     * point, coordinates quantised to 2^-16 m, exact integer monotone chain */
    float nx = bn[0], ny = bn[1], nz = bn[2];
    float ux, uy, uz;
    if (fabsf(nx) < 0.9f) { ux = 0.0f; uy = -nz; uz = ny; }   /* e_x x n */
    else { ux = nz; uy = 0.0f; uz = -nx; }                    /* e_y x n */
    float ul = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
    float ui = 1.0f / sqrtf(ul);
    ux = ux * ui; uy = uy * ui; uz = uz * ui;
    float vx = fmaf(ny, uz, -(nz * uy));
    float vy = fmaf(nz, ux, -(nx * uz));
    float vz = fmaf(nx, uy, -(ny * ux));
    pl->basis_u[0] = ux; pl->basis_u[1] = uy; pl->basis_u[2] = uz;
    pl->basis_v[0] = vx; pl->basis_v[1] = vy; pl->basis_v[2] = vz;
    pl->origin[0] = pts[0]; pl->origin[1] = pts[1]; pl->origin[2] = pts[2];
    int32_t *xy = (int32_t *)malloc((size_t)ni * 2 * sizeof(int32_t));
    int32_t *hh = (int32_t *)malloc(((size_t)ni + 1) * 2 * sizeof(int32_t));
    if (!xy || !hh) { free(xy); free(hh); return ORC_ERR_OUT_OF_MEMORY; }
    uint32_t j = 0;
    for (uint32_t k = 0; k < n; ++k) {
        if (!inl[k]) continue;
        float qx = pts[3 * k] - pts[0], qy = pts[3 * k + 1] - pts[1], qz = pts[3 * k + 2] - pts[2];
        float a = fmaf(qz, uz, fmaf(qy, uy, qx * ux));
        float b = fmaf(qz, vz, fmaf(qy, vy, qx * vx));
        xy[2 * j] = (int32_t)rintf(a * 65536.0f);
        xy[2 * j + 1] = (int32_t)rintf(b * 65536.0f);
        ++j;
    }
    uint32_t hn = orc_hull_i32(xy, ni, hh);
    pl->hull_off = res->n_hull;
    pl->hull_n = hn;
    int st = push_hull(res, hh, hn);
    free(xy); free(hh);
    return st;
}

/* The fit of clusters c = 0..k-1 (points pts + 3 off[c], n = off[c+1] -
 * off[c], Philox label lab[c]) into r->planes, in cluster order and, within a
 * cluster, in extraction round order, with their hulls appended to r in the
 * same order.  Round 0 is the paper's single plane (always recorded).  With
 * planes_per_cluster P > 1, round q + 1 runs on the points of round q that
 * are not its inliers (in their order) when round q found a plane with at
 * least min_cluster inliers and at least min_cluster points remain; its
 * Philox counter is (label, h, q + 1, 0); it is recorded when it finds a
 * plane.  With several threads each range of clusters keeps its planes and
 * hulls apart and they are appended in order afterwards. */
typedef struct {
    orc_result *r; const uint32_t *off; const uint32_t *lab; const orc_params *prm; uint32_t P;
    orc_plane *slots;  /* [k][P] */
    uint32_t *n_rec;   /* [k] records per cluster */
    int nt; orc_result part[256]; int st[256]; uint64_t lo[256];
} fit_ctx;
static void fit_range(void *vc, uint64_t lo, uint64_t hi)
{
    fit_ctx *cx = (fit_ctx *)vc;
    int t = 0;  /* this range's index: par_for splits [0, k) exactly as fit_all does */
    while (t + 1 < cx->nt && cx->lo[t] != lo) ++t;
    orc_result *hr = g_threads > 1 ? &cx->part[t] : cx->r;
    const uint32_t minc = cx->prm->min_cluster;
    for (uint64_t c = lo; c < hi && cx->st[t] == ORC_OK; ++c) {
        const uint32_t o = cx->off[c], n = cx->off[c + 1] - o;
        const uint32_t label = cx->lab ? cx->lab[c] : (uint32_t)c;
        orc_plane *pl = &cx->slots[c * cx->P];
        cx->st[t] = fit_cluster(cx->r->pts + 3 * (size_t)o, n, label, 0, cx->prm, pl, cx->r->inlier + o, hr);
        pl->point_off = o;
        cx->n_rec[c] = 1;
        if (cx->P <= 1 || cx->st[t] != ORC_OK) continue;
        /* further rounds on the points that are not inliers of the previous round */
        float *cur = (float *)malloc(((size_t)n + 1) * 3 * sizeof(float));
        float *nxt = (float *)malloc(((size_t)n + 1) * 3 * sizeof(float));
        uint8_t *inl = (uint8_t *)malloc((size_t)n + 1);
        if (!cur || !nxt || !inl) { free(cur); free(nxt); free(inl); cx->st[t] = ORC_ERR_OUT_OF_MEMORY; break; }
        memcpy(cur, cx->r->pts + 3 * (size_t)o, (size_t)n * 3 * sizeof(float));
        memcpy(inl, cx->r->inlier + o, n);
        uint32_t cn = n;
        orc_plane *prev = pl;
        for (uint32_t q = 1; q < cx->P; ++q) {
            if (prev->best_h < 0 || prev->inlier_count < minc) break;
            uint32_t m = 0;
            for (uint32_t i = 0; i < cn; ++i)
                if (!inl[i]) {
                    nxt[3 * m] = cur[3 * i]; nxt[3 * m + 1] = cur[3 * i + 1]; nxt[3 * m + 2] = cur[3 * i + 2];
                    ++m;
                }
            if (m < minc || m == 0) break;
            orc_plane *pq = &cx->slots[c * cx->P + q];
            cx->st[t] = fit_cluster(nxt, m, label, q, cx->prm, pq, inl, hr);
            if (cx->st[t] != ORC_OK) break;
            if (pq->best_h < 0) break;
            pq->point_off = o;
            cx->n_rec[c] = q + 1;
            float *sw = cur; cur = nxt; nxt = sw;
            cn = m;
            prev = pq;
        }
        free(cur); free(nxt); free(inl);
    }
}
static int fit_all(orc_result *r, const uint32_t *off, const uint32_t *lab, uint32_t k, const orc_params *prm)
{
    fit_ctx *cx = (fit_ctx *)calloc(1, sizeof(fit_ctx));
    if (!cx) return ORC_ERR_OUT_OF_MEMORY;
    const uint32_t P = prm->planes_per_cluster > 1 ? prm->planes_per_cluster : 1;
    cx->r = r; cx->off = off; cx->lab = lab; cx->prm = prm; cx->P = P;
    cx->slots = (orc_plane *)calloc((size_t)(k ? k : 1) * P, sizeof(orc_plane));
    cx->n_rec = (uint32_t *)calloc(k ? k : 1, sizeof(uint32_t));
    if (!cx->slots || !cx->n_rec) { free(cx->slots); free(cx->n_rec); free(cx); return ORC_ERR_OUT_OF_MEMORY; }
    int t = g_threads < (int)(k ? k : 1) ? g_threads : (int)(k ? k : 1);
    cx->nt = t;
    for (int i = 0; i < t; ++i) cx->lo[i] = (uint64_t)k * (uint64_t)i / (uint64_t)t;
    par_for(k, fit_range, cx);
    int st = ORC_OK;
    for (int i = 0; i < 256; ++i) if (cx->st[i] != ORC_OK) st = cx->st[i];
    if (g_threads > 1 && st == ORC_OK) {  /* hulls in order: shift each range's offsets */
        for (int i = 0; i < t && st == ORC_OK; ++i) {
            const uint64_t end = i + 1 < t ? cx->lo[i + 1] : k;
            for (uint64_t c = cx->lo[i]; c < end; ++c)
                for (uint32_t q = 0; q < cx->n_rec[c]; ++q) cx->slots[c * P + q].hull_off += r->n_hull;
            st = push_hull(r, cx->part[i].hull_xy, cx->part[i].n_hull);
        }
    }
    uint32_t np = 0;
    for (uint32_t c = 0; c < k; ++c) np += cx->n_rec[c];
    if (np > k) {
        orc_plane *grown = (orc_plane *)realloc(r->planes, (size_t)np * sizeof(orc_plane));
        if (!grown) st = ORC_ERR_OUT_OF_MEMORY; else r->planes = grown;
    }
    uint32_t j = 0;
    if (st == ORC_OK)
        for (uint32_t c = 0; c < k; ++c)
            for (uint32_t q = 0; q < cx->n_rec[c]; ++q) r->planes[j++] = cx->slots[c * P + q];
    for (int i = 0; i < 256; ++i) free(cx->part[i].hull_xy);
    free(cx->slots); free(cx->n_rec); free(cx);
    r->n_planes = j;
    return st;
}

void orc_result_free(void *h)
{
    orc_result *r = (orc_result *)h;
    if (!r) return;
    free(r->planes); free(r->hull_xy); free(r->pts); free(r->pt_vid); free(r->inlier); free(r);
}

/* Batched entry: caller-formed clusters (cluster k = points off[k]..off[k+1]),
 * label[k] keys its Philox stream (NULL: label = k). */
void *orc_fit_planes(const float *xyz, const uint32_t *off, const uint32_t *label, uint32_t k, const orc_params *prm)
{
    orc_result *r = (orc_result *)calloc(1, sizeof(orc_result));
    if (!r) return NULL;
    uint32_t npts = off[k];
    r->planes = (orc_plane *)calloc(k ? k : 1, sizeof(orc_plane));
    r->pts = (float *)malloc(((size_t)npts + 1) * 3 * sizeof(float));
    r->inlier = (uint8_t *)calloc((size_t)npts + 1, 1);
    if (!r->planes || !r->pts || !r->inlier) { orc_result_free(r); return NULL; }
    memcpy(r->pts, xyz, (size_t)npts * 3 * sizeof(float));
    r->n_pts = npts;
    if (fit_all(r, off, label, k, prm) != ORC_OK) {
        orc_result_free(r);
        return NULL;
    }
    return r;
}

/* ------------------------------------------------------------------------- */
/* Segmentation of the accumulated map (Sec. III.C).                         */
/* ------------------------------------------------------------------------- */

static int64_t idx_lookup(const orc_map *m, const int32_t *occ_index, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= m->nx || j >= m->ny || k >= m->nz) return -1;
    return occ_index[vid_of(m, i, j, k)];
}

/* Algorithm 1's edge test between two voxels: distance between mean
 * positions below d_th and normal angle below the threshold. */
static int ccl_edge(const orc_voxel *a, const orc_voxel *b, const orc_params *prm)
{
    float dx = a->mu[0] - b->mu[0], dy = a->mu[1] - b->mu[1], dz = a->mu[2] - b->mu[2];
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float c = fmaf(a->n[2], b->n[2], fmaf(a->n[1], b->n[1], a->n[0] * b->n[0]));
    return (d2 < prm->d_th2) && (fabsf(c) > prm->cos_ccl);
}

/* Eq. 3 / Eq. 4 for the occupied voxels lo..hi-1 (each reads the window's
 * means and writes only its own normal, N and status). */
typedef struct { orc_map *m; const int32_t *occ_index; const orc_params *prm; } normals_ctx;
static void normals_range(void *vc, uint64_t lo, uint64_t hi)
{
    normals_ctx *cx = (normals_ctx *)vc;
    orc_map *m = cx->m;
    const int32_t *occ_index = cx->occ_index;
    const orc_params *prm = cx->prm;
    for (uint64_t i = lo; i < hi; ++i) {
        orc_voxel *x = &m->vox[i];
        int64_t s1[3] = {0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0};
        int64_t cnt = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t j = idx_lookup(m, occ_index, x->ijk[0] + dx, x->ijk[1] + dy, x->ijk[2] + dz);
                    if (j < 0) continue;
                    const orc_voxel *y = &m->vox[j];
                    int64_t a = (int64_t)y->M[0] - x->M[0], b = (int64_t)y->M[1] - x->M[1],
                            c = (int64_t)y->M[2] - x->M[2];
                    s1[0] += a; s1[1] += b; s1[2] += c;
                    s2[0] += a * a; s2[1] += b * b; s2[2] += c * c;
                    s2[3] += a * b; s2[4] += a * c; s2[5] += b * c;
                    ++cnt;
                }
        x->nbr = (uint32_t)(cnt - 1);
        int64_t A[6];
        A[0] = cnt * s2[0] - s1[0] * s1[0];
        A[1] = cnt * s2[1] - s1[1] * s1[1];
        A[2] = cnt * s2[2] - s1[2] * s1[2];
        A[3] = cnt * s2[3] - s1[0] * s1[1];
        A[4] = cnt * s2[4] - s1[0] * s1[2];
        A[5] = cnt * s2[5] - s1[1] * s1[2];
        float Af[6];
        for (int a = 0; a < 6; ++a) Af[a] = (float)A[a];
        float V[3][3], D[3];
        jacobi3_f32(Af, 6, V, D);
        pick_normal_f32(V, D, x->n);
        x->status = (x->nbr >= prm->n_th && fabsf(x->n[2]) >= prm->cos_step) ? 2u : 1u;
    }
}

void *orc_segment(void *h, const orc_params *prm)
{
    orc_map *m = (orc_map *)h;
    if (!m || !prm) return NULL;
    free(m->vox);
    m->vox = NULL;
    m->n_vox = 0;
    /* occupied voxels in vid order: mean position from the exact sums */
    uint32_t nocc = orc_count_occupied(m);
    m->vox = (orc_voxel *)calloc(nocc ? nocc : 1, sizeof(orc_voxel));
    int32_t *occ_index = (int32_t *)malloc(m->nv * sizeof(int32_t));
    if (!m->vox || !occ_index) { free(occ_index); return NULL; }
    const float iq = 9.5367431640625e-07f; /* 2^-20 */
    const float o[3] = {m->po[0], m->po[1], m->po[2]};  /* the window's position origin */
    uint32_t k = 0;
    for (uint64_t v = 0; v < m->nv; ++v) {
        occ_index[v] = -1;
        if (!m->C[v]) continue;
        orc_voxel *x = &m->vox[k];
        x->vid = (uint32_t)v;
        ijk_of(m, v, x->ijk);
        x->c = m->C[v];
        for (int a = 0; a < 3; ++a) {
            x->S[a] = m->S[3 * v + a];
            /* Eq. 1's mean, exact in 2^-20 m units, rounded half up */
            x->M[a] = (int32_t)((2 * x->S[a] + (int64_t)x->c) / (2 * (int64_t)x->c));
            x->mu[a] = o[a] + (float)x->M[a] * iq;
        }
        x->label = 0xFFFFFFFFu;
        occ_index[v] = (int32_t)k;
        ++k;
    }
    m->n_vox = nocc;
    /* Eq. 3 / Eq. 4: covariance of the mean positions in the 3x3x3 window
     * (self included), normal = eigenvector of the smallest eigenvalue by FP32
     * Jacobi; steppable iff N >= N_th and |n_z| >= cos(theta_th). */
    normals_ctx ncx = {m, occ_index, prm};
    par_for(nocc, normals_range, &ncx);
    /* Algorithm 1: connected components of the steppable voxels under the
     * distance / normal-angle adjacency over the 26-neighbourhood.  The fixed
     * point of the min-label propagation labels every component by its
     * smallest voxel id; breadth-first search visits voxels in vid order, so
     * the first voxel of each component is that smallest id. */
    int32_t *queue = (int32_t *)malloc((size_t)(nocc ? nocc : 1) * sizeof(int32_t));
    if (!queue) { free(occ_index); return NULL; }
    for (uint32_t i = 0; i < nocc; ++i) {
        orc_voxel *x = &m->vox[i];
        uint32_t want = prm->classify ? 2u : 1u;
        if (x->status < want || x->label != 0xFFFFFFFFu) continue;
        uint32_t lab = x->vid;
        uint32_t qh = 0, qt = 0;
        queue[qt++] = (int32_t)i;
        x->label = lab;
        while (qh < qt) {
            orc_voxel *a = &m->vox[queue[qh++]];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy && !dz) continue;
                        int64_t j = idx_lookup(m, occ_index, a->ijk[0] + dx, a->ijk[1] + dy, a->ijk[2] + dz);
                        if (j < 0) continue;
                        orc_voxel *b = &m->vox[j];
                        if (b->status < want || b->label != 0xFFFFFFFFu) continue;
                        if (!ccl_edge(a, b, prm)) continue;
                        b->label = lab;
                        queue[qt++] = (int32_t)j;
                    }
        }
    }
    free(queue);
    free(occ_index);
    /* clusters: labels with at least min_cluster voxels, label ascending,
     * points in vid order */
    uint32_t n_lab = 0, n_pts = 0;
    uint32_t *lab_list = NULL, *lab_cnt = NULL;
    {
        /* labels are voxel ids of component roots: count through a scan of
         * the vid-ordered voxel list */
        uint32_t *cnt_by_idx = (uint32_t *)calloc(nocc ? nocc : 1, sizeof(uint32_t));
        int32_t *root_idx = (int32_t *)malloc((size_t)(nocc ? nocc : 1) * sizeof(int32_t));
        if (!cnt_by_idx || !root_idx) { free(cnt_by_idx); free(root_idx); return NULL; }
        /* map label (a vid) back to its voxel index by a binary search over the
         * sorted vid list */
        for (uint32_t i = 0; i < nocc; ++i) {
            root_idx[i] = -1;
            uint32_t L = m->vox[i].label;
            if (L == 0xFFFFFFFFu) continue;
            uint32_t lo = 0, hi = nocc;
            while (lo < hi) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (m->vox[mid].vid < L) lo = mid + 1; else hi = mid;
            }
            root_idx[i] = (int32_t)lo;
            cnt_by_idx[lo]++;
        }
        lab_list = (uint32_t *)malloc((size_t)(nocc ? nocc : 1) * sizeof(uint32_t));
        lab_cnt = (uint32_t *)malloc((size_t)(nocc ? nocc : 1) * sizeof(uint32_t));
        int32_t *cl_of_root = (int32_t *)malloc((size_t)(nocc ? nocc : 1) * sizeof(int32_t));
        if (!lab_list || !lab_cnt || !cl_of_root) {
            free(cnt_by_idx); free(root_idx); free(lab_list); free(lab_cnt); free(cl_of_root);
            return NULL;
        }
        for (uint32_t i = 0; i < nocc; ++i) {
            cl_of_root[i] = -1;
            if (cnt_by_idx[i] >= prm->min_cluster && cnt_by_idx[i] > 0) {
                cl_of_root[i] = (int32_t)n_lab;
                lab_list[n_lab] = m->vox[i].vid;
                lab_cnt[n_lab] = cnt_by_idx[i];
                n_pts += cnt_by_idx[i];
                n_lab++;
            }
        }
        orc_result *r = (orc_result *)calloc(1, sizeof(orc_result));
        uint32_t *off = (uint32_t *)calloc((size_t)n_lab + 1, sizeof(uint32_t));
        uint32_t *fill = (uint32_t *)calloc((size_t)n_lab + 1, sizeof(uint32_t));
        if (!r || !off || !fill) {
            free(r); free(off); free(fill); free(cnt_by_idx); free(root_idx); free(lab_list); free(lab_cnt);
            free(cl_of_root);
            return NULL;
        }
        for (uint32_t c = 0; c < n_lab; ++c) off[c + 1] = off[c] + lab_cnt[c];
        r->planes = (orc_plane *)calloc(n_lab ? n_lab : 1, sizeof(orc_plane));
        r->pts = (float *)malloc(((size_t)n_pts + 1) * 3 * sizeof(float));
        r->pt_vid = (uint32_t *)malloc(((size_t)n_pts + 1) * sizeof(uint32_t));
        r->inlier = (uint8_t *)calloc((size_t)n_pts + 1, 1);
        if (!r->planes || !r->pts || !r->pt_vid || !r->inlier) {
            orc_result_free(r); free(off); free(fill); free(cnt_by_idx); free(root_idx); free(lab_list);
            free(lab_cnt); free(cl_of_root);
            return NULL;
        }
        r->n_pts = n_pts;
        for (uint32_t i = 0; i < nocc; ++i) {
            if (root_idx[i] < 0) continue;
            int32_t c = cl_of_root[root_idx[i]];
            if (c < 0) continue;
            uint32_t pos = off[c] + fill[c]++;
            r->pts[3 * pos + 0] = m->vox[i].mu[0];
            r->pts[3 * pos + 1] = m->vox[i].mu[1];
            r->pts[3 * pos + 2] = m->vox[i].mu[2];
            r->pt_vid[pos] = m->vox[i].vid;
        }
        /* Sec. III.C: multi-plane estimation and boundary polygon per cluster */
        int st = fit_all(r, off, lab_list, n_lab, prm);
        free(off); free(fill); free(cnt_by_idx); free(root_idx); free(lab_list); free(lab_cnt); free(cl_of_root);
        if (st != ORC_OK) { orc_result_free(r); return NULL; }
        return r;
    }
}

/* ------------------------------------------------------------------------- */
/* Accessors for the Python binding.                                          */
/* ------------------------------------------------------------------------- */

uint32_t orc_map_n_vox(void *h) { return ((orc_map *)h)->n_vox; }
uint32_t orc_voxel_size(void) { return (uint32_t)sizeof(orc_voxel); }
uint32_t orc_plane_size(void) { return (uint32_t)sizeof(orc_plane); }
const orc_voxel *orc_map_voxels(void *h) { return ((orc_map *)h)->vox; }

void orc_result_sizes(void *h, uint32_t out[3])
{
    orc_result *r = (orc_result *)h;
    out[0] = r->n_planes; out[1] = r->n_hull; out[2] = r->n_pts;
}
const orc_plane *orc_result_planes(void *h) { return ((orc_result *)h)->planes; }
const int32_t *orc_result_hull(void *h) { return ((orc_result *)h)->hull_xy; }
const float *orc_result_pts(void *h) { return ((orc_result *)h)->pts; }
const uint32_t *orc_result_pt_vid(void *h) { return ((orc_result *)h)->pt_vid; }
const uint8_t *orc_result_inlier(void *h) { return ((orc_result *)h)->inlier; }
