// Scene upload (input arrays -> device records + FP64 copies + scene box) and
// the uniform-grid build: count -> exclusive scan -> scatter -> per-cell sort.
// The grid is the acceleration structure of the tracer; its build is the
// paper's preprocessing phase (Table 5). For animated scenes the geometry can
// be replaced in place (scene_update) and the grid rebuilt on the device with
// no host round trip (grid_rebuild: the geometry itself is computed by a
// one-thread kernel from the device-side scene box).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "gbrt_internal.h"

namespace gbrt {

// float <-> order-preserving uint32, so atomicMin/atomicMax reduce floats
__device__ __forceinline__ uint32_t ord_of(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
static float float_of_ord(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// One thread per object: device records, FP64 copies, padded-box inputs and a
// warp-reduced scene box. box[0..2] min, box[3..5] max (ordered), box[6] = 1
// when any object is invalid.
__global__ void __launch_bounds__(256) k_scene_prep(const float* sph_in, int64_t S, const float* cyl_in, int64_t C,
                                                     const uint32_t* color, int32_t K, float4* obj, double2* obj64,
                                                     float4* aabb, uint32_t* box, uint32_t* err) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float big = 3.0e38f;
    float lo[3] = {big, big, big}, hi[3] = {-big, -big, -big};
    bool bad = false;
    if (id < S) {
        const float* p = sph_in + 4 * id;
        float c[3] = {p[0], p[1], p[2]}, r = p[3];
        bad = !(isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]) && isfinite(r) && r > 0.0f);
        obj[2 * id] = make_float4(c[0], c[1], c[2], r);
        obj[2 * id + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        obj64[4 * id] = make_double2(c[0], c[1]);
        obj64[4 * id + 1] = make_double2(c[2], r);
        obj64[4 * id + 2] = make_double2(0.0, 0.0);
        obj64[4 * id + 3] = make_double2(0.0, 0.0);
        for (int k = 0; k < 3; ++k) {
            lo[k] = c[k] - r;
            hi[k] = c[k] + r;
        }
    } else if (id < S + C) {
        const int64_t j = id - S;
        const float* p = cyl_in + 7 * j;
        float p0[3] = {p[0], p[1], p[2]}, p1[3] = {p[3], p[4], p[5]}, r = p[6];
        float ax[3], a[3];
        double ax64[3], a64[3];
        bool fin = isfinite(r);
        for (int k = 0; k < 3; ++k) {
            fin = fin && isfinite(p0[k]) && isfinite(p1[k]);
            ax[k] = p1[k] - p0[k];
            ax64[k] = (double)p1[k] - (double)p0[k];
        }
        float L = sqrtf(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        double L64 = sqrt(ax64[0] * ax64[0] + ax64[1] * ax64[1] + ax64[2] * ax64[2]);
        bad = !(fin && r > 0.0f && L > 0.0f);
        for (int k = 0; k < 3; ++k) {
            a[k] = L > 0.0f ? ax[k] / L : 0.0f;
            a64[k] = L64 > 0.0 ? ax64[k] / L64 : 0.0;
        }
        obj[2 * id] = make_float4(p0[0], p0[1], p0[2], r);
        obj[2 * id + 1] = make_float4(a[0], a[1], a[2], L);
        obj64[4 * id] = make_double2(p0[0], p0[1]);
        obj64[4 * id + 1] = make_double2(p0[2], r);
        obj64[4 * id + 2] = make_double2(a64[0], a64[1]);
        obj64[4 * id + 3] = make_double2(a64[2], L64);
        for (int k = 0; k < 3; ++k) {
            float e = r * sqrtf(fmaxf(0.0f, 1.0f - a[k] * a[k]));
            lo[k] = fminf(p0[k], p1[k]) - e;
            hi[k] = fmaxf(p0[k], p1[k]) + e;
        }
    }
    if (id < S + C) {
        if (color[id] >= (uint32_t)K) bad = true;
        aabb[2 * id] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        aabb[2 * id + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
        if (bad) {
            box[6] = 1u;
            if (err) atomicOr(err, ERR_SCENE_DATA);
            for (int k = 0; k < 3; ++k) {
                lo[k] = big;
                hi[k] = -big;
            }
        }
    }
    // warp reduction, then one atomic per warp and component
    for (int k = 0; k < 3; ++k) {
        float l = lo[k], h = hi[k];
        for (int off = 16; off > 0; off >>= 1) {
            l = fminf(l, __shfl_xor_sync(0xffffffffu, l, off));
            h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, off));
        }
        if ((threadIdx.x & 31) == 0 && l <= h) {
            atomicMin(box + k, ord_of(l));
            atomicMax(box + 3 + k, ord_of(h));
        }
    }
}


__device__ __forceinline__ int build_cell(const BuildP& p, int k, float x) {
    int c = (int)floorf((x - p.lo[k]) * p.inv_h[k]);
    c = c < 0 ? 0 : c;
    return c > p.n[k] - 1 ? p.n[k] - 1 : c;
}

__device__ __forceinline__ void cell_range(const float4* aabb, int64_t id, const BuildP& p, int c0[3], int c1[3]) {
    float4 a = aabb[2 * id], b = aabb[2 * id + 1];
    c0[0] = build_cell(p, 0, a.x - p.pad);
    c0[1] = build_cell(p, 1, a.y - p.pad);
    c0[2] = build_cell(p, 2, a.z - p.pad);
    c1[0] = build_cell(p, 0, b.x + p.pad);
    c1[1] = build_cell(p, 1, b.y + p.pad);
    c1[2] = build_cell(p, 2, b.z + p.pad);
}

// Squared distance from point q to the box [lo, hi].
__device__ __forceinline__ float box_dist2(float qx, float qy, float qz, const float lo[3], const float hi[3]) {
    const float ex = fmaxf(fmaxf(lo[0] - qx, 0.0f), qx - hi[0]);
    const float ey = fmaxf(fmaxf(lo[1] - qy, 0.0f), qy - hi[1]);
    const float ez = fmaxf(fmaxf(lo[2] - qz, 0.0f), qz - hi[2]);
    return ex * ex + ey * ey + ez * ez;
}

// Does object `id` reach into cell (x, y, z)? A superset test on the cell box
// grown by pad: sphere -- distance from the centre to the box <= r; cylinder --
// distance from its axis segment to the box <= r (the capsule around the tube).
// Along the segment that distance is convex and 1-Lipschitz in the axial
// coordinate, so a ternary search leaves the minimiser inside an interval of
// width w and the midpoint's distance is at most the minimum + w/2: the test
// accepts at midpoint distance <= r + w/2 (+ a float rounding margin). Any
// point of an object lies in a cell this test accepts, so every hit is found.
__device__ __forceinline__ bool cell_reached(const float4* obj, int64_t id, const BuildP& p, int x, int y, int z) {
    const float4 A = obj[2 * id], B = obj[2 * id + 1];
    const int ci[3] = {x, y, z};
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = p.lo[k] + (float)ci[k] * p.h[k] - p.pad;
        hi[k] = p.lo[k] + (float)(ci[k] + 1) * p.h[k] + p.pad;
    }
    const float rr = A.w + p.pad;
    if (B.w == 0.0f) return box_dist2(A.x, A.y, A.z, lo, hi) <= rr * rr;
    float s0 = 0.0f, s1 = B.w;
    for (int it = 0; it < 14; ++it) {
        const float m1 = s0 + (s1 - s0) * (1.0f / 3.0f), m2 = s1 - (s1 - s0) * (1.0f / 3.0f);
        const float f1 = box_dist2(A.x + m1 * B.x, A.y + m1 * B.y, A.z + m1 * B.z, lo, hi);
        const float f2 = box_dist2(A.x + m2 * B.x, A.y + m2 * B.y, A.z + m2 * B.z, lo, hi);
        if (f1 < f2) s1 = m2;
        else s0 = m1;
    }
    const float sm = 0.5f * (s0 + s1);
    const float lim = rr + 0.5f * (s1 - s0) + 1e-5f * (B.w + 1.0f);
    return box_dist2(A.x + sm * B.x, A.y + sm * B.y, A.z + sm * B.z, lo, hi) <= lim * lim;
}

// Count and scatter run one warp per object (grid-stride over objects): the
// lanes take the cells of the object's box in turn, k = 0, 1, ... with x
// fastest, then y, then z, so an object's cells are tested in parallel.
__device__ __forceinline__ void span_cell(const int c0[3], int nx, int ny, int k, int& x, int& y, int& z) {
    x = c0[0] + k % nx;
    y = c0[1] + (k / nx) % ny;
    z = c0[2] + k / (nx * ny);
}

// Blocks of 256 threads for one warp per object over N objects.
inline int object_warp_blocks(int64_t N) {
    return (int)std::min<int64_t>((std::max<int64_t>(N, 1) + 7) / 8, 1 << 20);
}

// Count pass. When an object's box spans at most 64 cells, the cells its shape
// reaches are also recorded as bits k in reach[id], so the scatter pass need
// not repeat the test; wider objects get all-ones and are tested again there.
__global__ void __launch_bounds__(256) k_grid_count(const float4* aabb, const float4* obj, int64_t N,
                                                     const BuildP* bp, uint32_t* counts,
                                                     unsigned long long* reach) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const BuildP p = *bp;
    for (int64_t id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; id < N; id += warps) {
        int c0[3], c1[3];
        cell_range(aabb, id, p, c0, c1);
        const int nx = c1[0] - c0[0] + 1, ny = c1[1] - c0[1] + 1;
        const int span = nx * ny * (c1[2] - c0[2] + 1);
        unsigned long long bits = 0ull;
        for (int base = 0; base < span; base += 32) {
            const int k = base + lane;
            bool hit = false;
            if (k < span) {
                int x, y, z;
                span_cell(c0, nx, ny, k, x, y, z);
                hit = cell_reached(obj, id, p, x, y, z);
                if (hit) atomicAdd(counts + ((int64_t)z * p.n[1] + y) * p.n[0] + x, 1u);
            }
            const unsigned got = __ballot_sync(0xffffffffu, hit);
            if (base < 64) bits |= (unsigned long long)got << base;
        }
        if (lane == 0) reach[id] = span <= 64 ? bits : ~0ull;
    }
}

// Items past `items_cap` are dropped (a device-side rebuild that outgrew its
// buffer; its finish step then disables the grid and flags the error).
__global__ void __launch_bounds__(256) k_grid_scatter(const float4* aabb, const float4* obj, int64_t N,
                                                       const BuildP* bp, const unsigned long long* reach,
                                                       const uint2* cells, uint32_t* cursor, uint32_t* items,
                                                       uint64_t items_cap) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const BuildP p = *bp;
    for (int64_t id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; id < N; id += warps) {
        int c0[3], c1[3];
        cell_range(aabb, id, p, c0, c1);
        const int nx = c1[0] - c0[0] + 1, ny = c1[1] - c0[1] + 1;
        const int span = nx * ny * (c1[2] - c0[2] + 1);
        const unsigned long long bits = reach[id];
        const bool recorded = bits != ~0ull;  // then span <= 64
        for (int k = lane; k < span; k += 32) {
            int x, y, z;
            span_cell(c0, nx, ny, k, x, y, z);
            if (recorded ? !((bits >> k) & 1ull) : !cell_reached(obj, id, p, x, y, z)) continue;
            const int64_t c = ((int64_t)z * p.n[1] + y) * p.n[0] + x;
            const uint32_t slot = atomicAdd(cursor + c, 1u);
            const uint64_t at = (uint64_t)cells[c].x + slot;
            if (at < items_cap) items[at] = (uint32_t)id;
        }
    }
}

// Radius of the sphere about `ctr` that holds every object: sphere |c - ctr| + r,
// cylinder max over both ends of |p - ctr| + r (FP64, rounded up to float).
__global__ void __launch_bounds__(256) k_bound_radius(const double2* obj64, int64_t N, const double* ctr,
                                                       unsigned int* rbits) {
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float rr = 0.0f;
    if (id < N) {
        const double cx = ctr[0], cy = ctr[1], cz = ctr[2];
        const double2* q = obj64 + 4 * id;
        double2 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
        double px = q0.x - cx, py = q0.y - cy, pz = q1.x - cz;
        double r = q1.y, L = q3.y;
        double ex = px + L * q2.x, ey = py + L * q2.y, ez = pz + L * q3.x;
        double d = fmax(sqrt(px * px + py * py + pz * pz), sqrt(ex * ex + ey * ey + ez * ez)) + r;
        rr = __double2float_ru(d);
    }
    for (int off = 16; off > 0; off >>= 1) rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, off));
    if ((threadIdx.x & 31) == 0) atomicMax(rbits, __float_as_uint(rr));  // non-negative floats order as ints
}

// Atomic scatter order is arbitrary: sort each cell's ids ascending (spheres
// first, then cylinders; deterministic lists).
__global__ void __launch_bounds__(256) k_cell_sort(const uint2* cells, int64_t ncells, uint32_t* items,
                                                    uint64_t items_cap) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    uint2 cr = cells[c];
    if ((uint64_t)cr.x + cr.y > items_cap) return;  // overflowed rebuild: the grid is disabled
    uint32_t* it = items + cr.x;
    for (uint32_t a = 1; a < cr.y; ++a) {
        uint32_t v = it[a];
        uint32_t b = a;
        while (b > 0 && it[b - 1] > v) {
            it[b] = it[b - 1];
            --b;
        }
        it[b] = v;
    }
}

// ---- exclusive scan of the per-cell counts (three passes over 4096-wide tiles)

constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

// Exclusive block scan of one value per thread; returns the block total.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long& total) {
    __shared__ unsigned long long warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int off = 1; off < 32; off <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        unsigned long long w = lane < nw ? warp_tot[lane] : 0ull;
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    unsigned long long before = wid > 0 ? warp_tot[wid - 1] : 0ull;
    total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t* in, int64_t n, unsigned long long* sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    unsigned long long s = 0;
    for (int k = 0; k < SCAN_PER; ++k)
        if (base + k < n) s += in[base + k];
    unsigned long long tot;
    block_exclusive_scan(s, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(unsigned long long* sums, int64_t nb, unsigned long long* total) {
    int64_t per = (nb + SCAN_T - 1) / SCAN_T;
    int64_t b0 = (int64_t)threadIdx.x * per;
    unsigned long long s = 0;
    for (int64_t k = b0; k < b0 + per && k < nb; ++k) s += sums[k];
    unsigned long long tot;
    unsigned long long run = block_exclusive_scan(s, tot);
    for (int64_t k = b0; k < b0 + per && k < nb; ++k) {
        unsigned long long v = sums[k];
        sums[k] = run;
        run += v;
    }
    if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const uint32_t* in, int64_t n, const unsigned long long* offs,
                                                        uint2* cells) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    uint32_t v[SCAN_PER];
    unsigned long long s = 0;
    for (int k = 0; k < SCAN_PER; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    unsigned long long tot;
    unsigned long long run = offs[blockIdx.x] + block_exclusive_scan(s, tot);
    for (int k = 0; k < SCAN_PER; ++k) {
        if (base + k < n) cells[base + k] = make_uint2((uint32_t)run, v[k]);
        run += v[k];
    }
}

// ---------------------------------------------------------------- host side

#define GB_TRY(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) {               \
            rc = e_ == cudaErrorMemoryAllocation ? GBRT_ENOMEM : GBRT_EDEVICE; \
            goto fail;                         \
        }                                      \
    } while (0)

static bool host_scene_valid(const float* sph, int64_t S, const float* cyl, int64_t C, const uint32_t* color,
                             int32_t K) {
    for (int64_t i = 0; i < S; ++i) {
        const float* p = sph + 4 * i;
        if (!(std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]) && std::isfinite(p[3]) && p[3] > 0))
            return false;
    }
    for (int64_t j = 0; j < C; ++j) {
        const float* p = cyl + 7 * j;
        for (int k = 0; k < 7; ++k)
            if (!std::isfinite(p[k])) return false;
        if (!(p[6] > 0)) return false;
        if (p[0] == p[3] && p[1] == p[4] && p[2] == p[5]) return false;
    }
    for (int64_t i = 0; color && i < S + C; ++i)
        if (color[i] >= (uint32_t)K) return false;
    return true;
}

void scene_release(Scene* s) {
    cudaFree(s->obj);
    cudaFree(s->obj64);
    cudaFree(s->color);
    cudaFree(s->palette);
    cudaFree(s->aabb);
    cudaFree(s->d_box);
    cudaFree(s->d_in);
    *s = Scene();
}

int scene_upload(Ctx* ctx, const float* spheres, int64_t S, const float* cyl, int64_t C, const uint32_t* color,
                 const float* palette, int32_t K, int flags, Scene* s) {
    int rc = GBRT_OK;
    const bool host = (flags & GBRT_HOST_PTRS) != 0;
    const int64_t N = S + C;
    float* d_sph_in = nullptr;
    float* d_cyl_in = nullptr;
    uint32_t* d_box = nullptr;
    uint32_t h_box[8];
    if (host && N > 0 && !host_scene_valid(spheres, S, cyl, C, color, K)) return GBRT_EINVAL;
    *s = Scene();
    s->device = ctx->device;
    s->S = S;
    s->C = C;
    s->K = K;
    {
        const size_t nN = (size_t)std::max<int64_t>(N, 1);
        GB_TRY(cudaMalloc(&s->obj, 2 * nN * sizeof(float4)));
        GB_TRY(cudaMalloc(&s->obj64, 4 * nN * sizeof(double2)));
        GB_TRY(cudaMalloc(&s->color, nN * sizeof(uint32_t)));
        GB_TRY(cudaMalloc(&s->palette, (size_t)std::max(K, 1) * 3 * sizeof(float)));
        GB_TRY(cudaMalloc(&s->aabb, 2 * nN * sizeof(float4)));
        GB_TRY(cudaMalloc(&d_box, 8 * sizeof(uint32_t)));
        s->bytes = nN * (2 * sizeof(float4) + 4 * sizeof(double2) + sizeof(uint32_t) + 2 * sizeof(float4)) +
                   (size_t)std::max(K, 1) * 3 * sizeof(float);
        if (host) {
            if (S > 0) {
                GB_TRY(cudaMalloc(&d_sph_in, (size_t)S * 4 * sizeof(float)));
                GB_TRY(cudaMemcpyAsync(d_sph_in, spheres, (size_t)S * 4 * sizeof(float), cudaMemcpyHostToDevice,
                                       ctx->stream));
            }
            if (C > 0) {
                GB_TRY(cudaMalloc(&d_cyl_in, (size_t)C * 7 * sizeof(float)));
                GB_TRY(cudaMemcpyAsync(d_cyl_in, cyl, (size_t)C * 7 * sizeof(float), cudaMemcpyHostToDevice,
                                       ctx->stream));
            }
            if (N > 0) GB_TRY(cudaMemcpyAsync(s->color, color, (size_t)N * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                              ctx->stream));
            if (K > 0) GB_TRY(cudaMemcpyAsync(s->palette, palette, (size_t)K * 3 * sizeof(float),
                                              cudaMemcpyHostToDevice, ctx->stream));
        } else {
            d_sph_in = const_cast<float*>(spheres);
            d_cyl_in = const_cast<float*>(cyl);
            if (N > 0) GB_TRY(cudaMemcpyAsync(s->color, color, (size_t)N * sizeof(uint32_t),
                                              cudaMemcpyDeviceToDevice, ctx->stream));
            if (K > 0) GB_TRY(cudaMemcpyAsync(s->palette, palette, (size_t)K * 3 * sizeof(float),
                                              cudaMemcpyDeviceToDevice, ctx->stream));
        }
        // box init: min = ord(+big), max = ord(-big); flag 0
        uint32_t init[8];
        {
            float big = 3.0e38f, nbig = -3.0e38f;
            uint32_t ub, unb;
            memcpy(&ub, &big, 4);
            memcpy(&unb, &nbig, 4);
            uint32_t ob = ub | 0x80000000u, onb = ~unb;
            init[0] = init[1] = init[2] = ob;
            init[3] = init[4] = init[5] = onb;
            init[6] = init[7] = 0u;
        }
        GB_TRY(cudaMemcpyAsync(d_box, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
        if (N > 0) {
            int blocks = (int)((N + 255) / 256);
            k_scene_prep<<<blocks, 256, 0, ctx->stream>>>(d_sph_in, S, d_cyl_in, C, s->color, K, s->obj, s->obj64,
                                                          s->aabb, d_box, nullptr);
            ctx->launches++;
            GB_TRY(cudaGetLastError());
        }
        GB_TRY(cudaMemcpyAsync(h_box, d_box, sizeof(h_box), cudaMemcpyDeviceToHost, ctx->stream));
        GB_TRY(cudaStreamSynchronize(ctx->stream));
        if (h_box[6]) {
            rc = GBRT_EINVAL;
            goto fail;
        }
        for (int k = 0; k < 3; ++k) {
            s->lo[k] = N > 0 ? float_of_ord(h_box[k]) : 0.0f;
            s->hi[k] = N > 0 ? float_of_ord(h_box[3 + k]) : 0.0f;
        }
    }
    if (host) {
        cudaFree(d_sph_in);
        cudaFree(d_cyl_in);
    }
    s->d_box = d_box;  // kept: device-side rebuilds read the box from here
    return GBRT_OK;
fail:
    cudaStreamSynchronize(ctx->stream);
    if (host) {
        cudaFree(d_sph_in);
        cudaFree(d_cyl_in);
    }
    cudaFree(d_box);
    scene_release(s);
    return rc;
}

void grid_release(Grid* g) {
    cudaFree(g->cells);
    cudaFree(g->items);
    cudaFree(g->d_geom);
    cudaFree(g->d_aux);
    cudaFree(g->d_counts);
    cudaFree(g->d_sums);
    cudaFree(g->d_reach);
    cudaFree(g->d_stat);
    cudaFreeHost(g->h_stat);
    if (g->stat_ev) cudaEventDestroy(g->stat_ev);
    *g = Grid();
}

// a * b + c rounded twice, as on the host: the device must not fuse it, so a
// device-side rebuild gets the same geometry as a host build
__host__ __device__ inline double mul_add_rn(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(__dmul_rn(a, b), c);
#else
    return a * b + c;
#endif
}

// Cells per axis for a box of extents E[3] and a target of `target` cells
// (n_k = round(E_k (target / V)^(1/3)), clamped to [1, 1024]); host and device
// evaluate the same expression.
__host__ __device__ inline int64_t grid_dims(const double E[3], double kk, int32_t n[3]) {
    int64_t nc = 1;
    for (int k = 0; k < 3; ++k) {
        double nk = floor(mul_add_rn(E[k], kk, 0.5));
        nk = nk < 1.0 ? 1.0 : (nk > 1024.0 ? 1024.0 : nk);
        n[k] = (int32_t)nk;
        nc *= n[k];
    }
    return nc;
}

// Fill the grid geometry (GridDev fields, build parameters, bounding-sphere
// centre) from the padded scene box; `cells_cap` > 0 caps the cell count.
__host__ __device__ inline void grid_geometry(const float slo[3], const float shi[3], int64_t N, float lambda,
                                              int64_t cells_cap, GridDev& d, BuildAux& a) {
    float emax = fmaxf(shi[0] - slo[0], fmaxf(shi[1] - slo[1], shi[2] - slo[2]));
    float pad = 1e-5f * fmaxf(emax, 1.0f);
    double E[3], V = 1.0;
    for (int k = 0; k < 3; ++k) {
        d.lo[k] = slo[k] - pad;
        d.hi[k] = shi[k] + pad;
        E[k] = (double)d.hi[k] - (double)d.lo[k];
        V *= E[k];
    }
    double target = fmin(fmax((double)lambda * (double)N, 1.0), 67108864.0);
    double kk = cbrt(target / V);
    d.ncells = grid_dims(E, kk, d.n);
    for (int it = 0; cells_cap > 0 && d.ncells > cells_cap && it < 64; ++it) {
        kk *= 0.98 * cbrt((double)cells_cap / (double)d.ncells);
        d.ncells = grid_dims(E, kk, d.n);
    }
    if (cells_cap > 0 && d.ncells > cells_cap) {
        d.n[0] = d.n[1] = d.n[2] = 1;
        d.ncells = 1;
    }
    for (int k = 0; k < 3; ++k) {
        const double nk = (double)d.n[k];
        d.h64[k] = E[k] / nk;
        d.inv_h64[k] = nk / E[k];
        d.lo64[k] = (double)d.lo[k];
        d.hi64[k] = (double)d.hi[k];
        d.h[k] = (float)d.h64[k];
        d.inv_h[k] = (float)d.inv_h64[k];
        a.p.lo[k] = d.lo[k];
        a.p.inv_h[k] = d.inv_h[k];
        a.p.h[k] = d.h[k];
        a.p.n[k] = d.n[k];
        a.ctr[k] = 0.5 * ((double)d.lo[k] + d.hi[k]);
    }
    a.p.pad = pad;
    a.rbits = 0u;
    a.pad = 0u;
    d.empty = N == 0 ? 1 : 0;
}

// Bounding sphere from its centre and the reduced radius bits.
__host__ __device__ inline void grid_bound_sphere(const BuildAux& a, GridDev& d) {
    float rb;
    memcpy(&rb, &a.rbits, 4);
    const double rpad = mul_add_rn((double)rb, 1.0 + 1e-5, (double)a.p.pad);
    for (int k = 0; k < 3; ++k) {
        d.bs64[k] = a.ctr[k];
        d.bs[k] = (float)a.ctr[k];
    }
    d.bs64[3] = rpad;
    // the float copy: pad for the rounding of the float centre too
    d.bs[3] = (float)mul_add_rn(1e-6, fabs(a.ctr[0]) + fabs(a.ctr[1]) + fabs(a.ctr[2]) + 1.0, rpad);
}

__device__ __forceinline__ float float_of_ord_dev(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Device-side rebuild, step 1 (one thread): geometry from the current scene box.
__global__ void k_grid_geometry(const uint32_t* box, int64_t N, float lambda, int64_t cells_cap, const uint2* cells,
                                const uint32_t* items, int64_t items_cap, GridDev* geom, BuildAux* aux) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = N > 0 ? float_of_ord_dev(box[k]) : 0.0f;
        hi[k] = N > 0 ? float_of_ord_dev(box[3 + k]) : 0.0f;
    }
    GridDev d = *geom;
    BuildAux a;
    grid_geometry(lo, hi, N, lambda, cells_cap, d, a);
    d.cells = cells;
    d.items = items;
    d.nitems = items_cap;
    *geom = d;
    *aux = a;
}

// Device-side rebuild, last step (one thread): bounding sphere, reference
// count; a rebuild that outgrew its item buffer disables the grid (renders
// then see no objects) and flags the context's error word.
__global__ void k_grid_finish(GridDev* geom, const BuildAux* aux, const unsigned long long* total,
                              unsigned long long items_cap, GridStat* stat, uint32_t* err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GridDev d = *geom;
    grid_bound_sphere(*aux, d);
    const unsigned long long refs = *total;
    const unsigned int over = refs > items_cap ? 1u : 0u;
    if (over) {
        d.empty = 1;
        atomicOr(err, ERR_GRID_CAPACITY);
    }
    *geom = d;
    stat->refs = refs;
    stat->ncells = (unsigned long long)d.ncells;
    stat->overflow = over;
    stat->pad = 0u;
}

int grid_build(Ctx* ctx, const Scene* s, float lambda, Grid* g) {
    int rc = GBRT_OK;
    uint32_t* counts = nullptr;
    unsigned long long* reach = nullptr;
    uint32_t* cursor = nullptr;
    unsigned long long* sums = nullptr;
    unsigned long long h_total = 0;
    *g = Grid();
    if (!(lambda > 0.0f)) lambda = 2.0f;
    g->lambda = lambda;
    const int64_t N = s->S + s->C;
    g->N = N;
    g->device = s->device;
    GridDev& d = g->dev;
    if (s->box_stale) {
        rc = scene_refresh_host(const_cast<Scene*>(s), ctx->stream);
        if (rc != GBRT_OK) return rc;
    }
    {
        BuildAux a;
        grid_geometry(s->lo, s->hi, N, lambda, 0, d, a);
        const int64_t nc = d.ncells;
        GB_TRY(cudaMalloc(&g->cells, (size_t)nc * sizeof(uint2)));
        GB_TRY(cudaMalloc(&counts, (size_t)nc * sizeof(uint32_t)));
        GB_TRY(cudaMalloc(&reach, (size_t)std::max<int64_t>(N, 1) * sizeof(unsigned long long)));
        GB_TRY(cudaMemsetAsync(counts, 0, (size_t)nc * sizeof(uint32_t), ctx->stream));
        const int64_t nb = (nc + SCAN_TILE - 1) / SCAN_TILE;
        // sums: nb block sums, total, then the build parameters
        GB_TRY(cudaMalloc(&sums, (size_t)(nb + 2) * sizeof(unsigned long long) + sizeof(BuildAux)));
        BuildAux* d_aux = (BuildAux*)(sums + nb + 2);
        GB_TRY(cudaMemcpyAsync(d_aux, &a, sizeof(a), cudaMemcpyHostToDevice, ctx->stream));
        if (N > 0) {
            k_grid_count<<<object_warp_blocks(N), 256, 0, ctx->stream>>>(s->aabb, s->obj, N, &d_aux->p, counts,
                                                                          reach);
            k_bound_radius<<<(int)((N + 255) / 256), 256, 0, ctx->stream>>>(s->obj64, N, d_aux->ctr, &d_aux->rbits);
            ctx->launches += 2;
            GB_TRY(cudaGetLastError());
        }
        k_scan_reduce<<<(int)nb, SCAN_T, 0, ctx->stream>>>(counts, nc, sums);
        k_scan_sums<<<1, SCAN_T, 0, ctx->stream>>>(sums, nb, sums + nb);
        k_scan_apply<<<(int)nb, SCAN_T, 0, ctx->stream>>>(counts, nc, sums, g->cells);
        ctx->launches += 3;
        GB_TRY(cudaGetLastError());
        GB_TRY(cudaMemcpyAsync(&h_total, sums + nb, sizeof(h_total), cudaMemcpyDeviceToHost, ctx->stream));
        GB_TRY(cudaMemcpyAsync(&a.rbits, &d_aux->rbits, sizeof(a.rbits), cudaMemcpyDeviceToHost, ctx->stream));
        GB_TRY(cudaStreamSynchronize(ctx->stream));
        grid_bound_sphere(a, d);
        if (h_total >= 0xFFFFFFFFull) {
            rc = GBRT_ENOMEM;
            goto fail;
        }
        g->refs = (int64_t)h_total;
        GB_TRY(cudaMalloc(&g->items, (size_t)std::max<int64_t>(g->refs, 1) * sizeof(uint32_t)));
        if (N > 0) {
            cursor = counts;  // reuse as per-cell fill cursor
            GB_TRY(cudaMemsetAsync(cursor, 0, (size_t)nc * sizeof(uint32_t), ctx->stream));
            k_grid_scatter<<<object_warp_blocks(N), 256, 0, ctx->stream>>>(s->aabb, s->obj, N, &d_aux->p, reach,
                                                                            g->cells,
                                                                            cursor, g->items, (uint64_t)g->refs);
            k_cell_sort<<<(int)((nc + 255) / 256), 256, 0, ctx->stream>>>(g->cells, nc, g->items,
                                                                          (uint64_t)g->refs);
            ctx->launches += 2;
            GB_TRY(cudaGetLastError());
        }
        GB_TRY(cudaStreamSynchronize(ctx->stream));
        d.cells = g->cells;
        d.items = g->items;
        d.nitems = std::max<int64_t>(g->refs, 1);
        g->bytes = (size_t)nc * sizeof(uint2) + (size_t)std::max<int64_t>(g->refs, 1) * sizeof(uint32_t);
    }
    cudaFree(counts);
    cudaFree(reach);
    cudaFree(sums);
    return GBRT_OK;
fail:
    cudaStreamSynchronize(ctx->stream);
    cudaFree(counts);
    cudaFree(reach);
    cudaFree(sums);
    grid_release(g);
    return rc;
}

// ---------------------------------------------------------------- animation path

int scene_refresh_host(Scene* s, cudaStream_t stream) {
    if (!s->box_stale) return GBRT_OK;
    uint32_t h_box[8];
    if (cudaStreamSynchronize(stream) != cudaSuccess ||
        cudaMemcpy(h_box, s->d_box, sizeof(h_box), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GBRT_EDEVICE;
    const int64_t N = s->S + s->C;
    for (int k = 0; k < 3; ++k) {
        s->lo[k] = N > 0 ? float_of_ord(h_box[k]) : 0.0f;
        s->hi[k] = N > 0 ? float_of_ord(h_box[3 + k]) : 0.0f;
    }
    s->box_stale = false;
    return h_box[6] ? GBRT_EINVAL : GBRT_OK;
}

int scene_update(Ctx* ctx, Scene* s, const float* spheres, const float* cyl, int flags) {
    const bool host = (flags & GBRT_HOST_PTRS) != 0;
    const int64_t S = s->S, C = s->C, N = S + C;
    if (N == 0) return GBRT_OK;
    if (host && !host_scene_valid(spheres, S, cyl, C, nullptr, 0)) return GBRT_EINVAL;
    const float* sph_in = spheres;
    const float* cyl_in = cyl;
    if (host) {
        if (!s->d_in) {
            if (cudaMalloc(&s->d_in, (size_t)(4 * S + 7 * C) * sizeof(float)) != cudaSuccess) {
                s->d_in = nullptr;
                return GBRT_ENOMEM;
            }
        }
        float* dsph = s->d_in;
        float* dcyl = s->d_in + 4 * S;
        if (S > 0 && cudaMemcpyAsync(dsph, spheres, (size_t)S * 4 * sizeof(float), cudaMemcpyHostToDevice,
                                     ctx->stream) != cudaSuccess)
            return GBRT_EDEVICE;
        if (C > 0 && cudaMemcpyAsync(dcyl, cyl, (size_t)C * 7 * sizeof(float), cudaMemcpyHostToDevice,
                                     ctx->stream) != cudaSuccess)
            return GBRT_EDEVICE;
        sph_in = dsph;
        cyl_in = dcyl;
    }
    // box words: min <- all ones (above every ordered float), max <- 0, flag <- 0
    if (cudaMemsetAsync(s->d_box, 0xFF, 3 * sizeof(uint32_t), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(s->d_box + 3, 0, 5 * sizeof(uint32_t), ctx->stream) != cudaSuccess)
        return GBRT_EDEVICE;
    k_scene_prep<<<(int)((N + 255) / 256), 256, 0, ctx->stream>>>(sph_in, S, cyl_in, C, s->color, s->K, s->obj,
                                                                  s->obj64, s->aabb, s->d_box, ctx->d_err);
    ctx->launches++;
    s->box_stale = true;
    return cudaGetLastError() == cudaSuccess ? GBRT_OK : GBRT_EDEVICE;
}

// Buffers of a device-side rebuild: cells, counts and scan sums for cells_cap,
// items for items_cap. All or nothing: on failure the grid keeps its previous
// buffers (and stays usable); the caller has drained the stream.
static int dyn_alloc(Grid* g, int64_t cells_cap, int64_t items_cap) {
    const int64_t nb = (cells_cap + SCAN_TILE - 1) / SCAN_TILE;
    uint2* cells = nullptr;
    uint32_t* items = nullptr;
    uint32_t* counts = nullptr;
    unsigned long long* sums = nullptr;
    if (cudaMalloc(&cells, (size_t)cells_cap * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc(&items, (size_t)items_cap * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&counts, (size_t)cells_cap * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&sums, (size_t)(nb + 2) * sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(cells);
        cudaFree(items);
        cudaFree(counts);
        cudaFree(sums);
        return GBRT_ENOMEM;
    }
    cudaFree(g->cells);
    cudaFree(g->items);
    cudaFree(g->d_counts);
    cudaFree(g->d_sums);
    g->cells = cells;
    g->items = items;
    g->d_counts = counts;
    g->d_sums = sums;
    g->cells_cap = cells_cap;
    g->items_cap = items_cap;
    g->bytes = (size_t)cells_cap * (sizeof(uint2) + sizeof(uint32_t)) + (size_t)items_cap * sizeof(uint32_t);
    g->dev.cells = g->cells;
    g->dev.items = g->items;
    g->dev.nitems = items_cap;
    return GBRT_OK;
}

int grid_rebuild(Ctx* ctx, const Scene* s, Grid* g) {
    const int64_t N = s->S + s->C;
    if (N != g->N) return GBRT_EINVAL;
    int rc = GBRT_OK;
    if (!g->dynamic) {
        // first device-side rebuild: buffers with headroom for moving geometry
        // (a retry after a failure reuses what an earlier attempt allocated)
        if ((!g->d_geom && cudaMalloc(&g->d_geom, sizeof(GridDev)) != cudaSuccess) ||
            (!g->d_aux && cudaMalloc(&g->d_aux, sizeof(BuildAux)) != cudaSuccess) ||
            (!g->d_stat && cudaMalloc(&g->d_stat, sizeof(GridStat)) != cudaSuccess) ||
            (!g->d_reach &&
             cudaMalloc(&g->d_reach, (size_t)std::max<int64_t>(N, 1) * sizeof(unsigned long long)) != cudaSuccess) ||
            (!g->h_stat && cudaMallocHost(&g->h_stat, sizeof(GridStat)) != cudaSuccess) ||
            (!g->stat_ev && cudaEventCreateWithFlags(&g->stat_ev, cudaEventDisableTiming) != cudaSuccess))
            return GBRT_ENOMEM;
        cudaStreamSynchronize(ctx->stream);  // renders may still read the host-built arrays
        const int64_t target = (int64_t)std::min(std::max((double)g->lambda * (double)N, 1.0), 67108864.0);
        const int64_t cells_cap = std::max<int64_t>(g->dev.ncells, target + target / 2) + 4096;
        const int64_t items_cap = std::max<int64_t>(g->refs + g->refs / 2, 4096);
        if ((rc = dyn_alloc(g, cells_cap, items_cap)) != GBRT_OK) return rc;
        if (cudaMemcpy(g->d_geom, &g->dev, sizeof(GridDev), cudaMemcpyHostToDevice) != cudaSuccess) {
            // the new buffers hold no lists yet: leave the grid unusable (renders
            // reject it) until a rebuild succeeds
            g->dev.cells = nullptr;
            g->dev.items = nullptr;
            return GBRT_EDEVICE;
        }
        g->dynamic = true;
    } else if (g->stat_pending && cudaEventQuery(g->stat_ev) == cudaSuccess) {
        // the last finished rebuild's reference count: grow the item buffer
        // ahead of need, or after an overflow
        g->stat_pending = false;
        const GridStat st = *g->h_stat;
        g->refs = (int64_t)st.refs;
        if (st.overflow || (int64_t)st.refs > g->items_cap - g->items_cap / 8) {
            cudaStreamSynchronize(ctx->stream);
            const int64_t items_cap = (int64_t)st.refs + (int64_t)st.refs / 2 + 4096;
            if (items_cap >= (int64_t)0xFFFFFFFFll) return GBRT_ENOMEM;
            if ((rc = dyn_alloc(g, g->cells_cap, items_cap)) != GBRT_OK) return rc;
        }
    }
    g->stream = ctx->stream;
    cudaStream_t st = ctx->stream;
    const int64_t nc = g->cells_cap;
    const int64_t nb = (nc + SCAN_TILE - 1) / SCAN_TILE;
    const int blocksN = (int)((std::max<int64_t>(N, 1) + 255) / 256);
    if (cudaMemsetAsync(g->d_counts, 0, (size_t)nc * sizeof(uint32_t), st) != cudaSuccess) return GBRT_EDEVICE;
    k_grid_geometry<<<1, 32, 0, st>>>(s->d_box, N, g->lambda, nc, g->cells, g->items, g->items_cap, g->d_geom,
                                      g->d_aux);
    if (N > 0) {
        k_grid_count<<<object_warp_blocks(N), 256, 0, st>>>(s->aabb, s->obj, N, &g->d_aux->p, g->d_counts, g->d_reach);
        k_bound_radius<<<blocksN, 256, 0, st>>>(s->obj64, N, g->d_aux->ctr, &g->d_aux->rbits);
    }
    k_scan_reduce<<<(int)nb, SCAN_T, 0, st>>>(g->d_counts, nc, g->d_sums);
    k_scan_sums<<<1, SCAN_T, 0, st>>>(g->d_sums, nb, g->d_sums + nb);
    k_scan_apply<<<(int)nb, SCAN_T, 0, st>>>(g->d_counts, nc, g->d_sums, g->cells);
    if (N > 0) {
        if (cudaMemsetAsync(g->d_counts, 0, (size_t)nc * sizeof(uint32_t), st) != cudaSuccess) return GBRT_EDEVICE;
        k_grid_scatter<<<object_warp_blocks(N), 256, 0, st>>>(s->aabb, s->obj, N, &g->d_aux->p, g->d_reach, g->cells, g->d_counts,
                                                g->items,
                                                (uint64_t)g->items_cap);
        // no per-cell sort: no result depends on the order of a cell's ids
        // (nearest hits rank by (t, id), any-hit queries OR their tests)
    }
    k_grid_finish<<<1, 32, 0, st>>>(g->d_geom, g->d_aux, g->d_sums + nb, (unsigned long long)g->items_cap, g->d_stat,
                                    ctx->d_err);
    ctx->launches += N > 0 ? 8 : 5;
    if (cudaGetLastError() != cudaSuccess) return GBRT_EDEVICE;
    if (cudaMemcpyAsync(g->h_stat, g->d_stat, sizeof(GridStat), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(g->stat_ev, st) != cudaSuccess)
        return GBRT_EDEVICE;
    g->stat_pending = true;
    return GBRT_OK;
}

int grid_refresh_host(Grid* g) {
    if (!g->dynamic) return GBRT_OK;
    if (g->stream && cudaStreamSynchronize(g->stream) != cudaSuccess) return GBRT_EDEVICE;
    if (cudaMemcpy(&g->dev, g->d_geom, sizeof(GridDev), cudaMemcpyDeviceToHost) != cudaSuccess) return GBRT_EDEVICE;
    if (g->stat_pending) {
        g->stat_pending = false;
        g->refs = (int64_t)g->h_stat->refs;
    }
    return GBRT_OK;
}

}  // namespace gbrt
