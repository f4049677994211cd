// Render kernels, wavefront style, for one frame or a batch of frames:
//   k_patch_grids  (frames whose grid was rebuilt on the device) copies the
//              rebuilt geometry into the frame descriptors;
//   k_primary  persistent; each warp pulls a 32-pixel tile of some frame from
//              an atomic queue, walks the primary rays (nearest hit), refines
//              the winner in its object's frame and appends the hit (AO
//              origin, normal) to its frame's hit list; the last CTA to
//              finish lays out the AO pass (prefix sums of hits and AO rays
//              per frame);
//   k_ao_walk  persistent; each lane holds one AO (or direct-light shadow)
//              ray; a warp refills its idle lanes together from its ray pool
//              once fewer than `refill` lanes still hold a ray, walks all of
//              them in lockstep (several cells per iteration), expands the
//              (ray, object) pairs over the lanes and tests them 32 at a
//              time;
//   k_shade    one thread per hit: Phong + skylight with V = escaped / spp;
//   k_resolve  (supersampled frames) box-filters the finer raster.
// Plus the AO probe and the raw Philox kernel.
#include <string.h>

#include <algorithm>
#include <functional>
#include <type_traits>
#include <vector>

#include "gbrt_device.cuh"
#include "gbrt_internal.h"

namespace gbrt {

constexpr unsigned FULL = 0xffffffffu;

// A kernel launched as a programmatic dependent of the previous one in its
// stream (launch_dependent) starts while that kernel drains; it waits here,
// before reading anything the previous kernel wrote, until the previous grid
// has finished and its writes are visible. Without that launch attribute the
// wait returns at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Largest f with off[f] <= x (off nondecreasing, x < off[n]).
template <class T>
__device__ __forceinline__ int find_frame(const T* off, int n, T x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Primary ray of pixel (i, j), in FP64 (both paths derive their ray from it).
// 1/W, 1/H and the unit view direction come precomputed with the frame.
__device__ __forceinline__ void primary_ray64(const FrameDev& f, int i, int j, V3<double>& o, V3<double>& d) {
    double u = f.half_w * fma((double)(2 * i + 1), f.inv_w, -1.0);
    double v = f.half_h * fma(-(double)(2 * j + 1), f.inv_h, 1.0);
    V3<double> up = ld3(f.up), right = ld3(f.right);
    if (f.cam_kind == GBRT_CAMERA_ORTHO) {
        o = madd(madd(ld3(f.eye), u, right), v, up);
        d = ld3(f.dir_unit);
    } else {
        o = ld3(f.eye);
        V3<double> q = madd(madd(ld3(f.dir_unit), u, right), v, up);
        d = rsqrt(dot(q, q)) * q;
    }
}

// View direction of pixel q in FP32 (shading only).
__device__ __forceinline__ V3<float> view_dir_f(const FrameDev& f, uint32_t q) {
    V3<float> d = v3(f.dir_f[0], f.dir_f[1], f.dir_f[2]);
    if (f.cam_kind == GBRT_CAMERA_ORTHO) return d;
    const int i = (int)(q % (uint32_t)f.W), j = (int)(q / (uint32_t)f.W);
    float u = f.half_w_f * fmaf((float)(2 * i + 1), f.inv_w_f, -1.0f);
    float v = f.half_h_f * fmaf(-(float)(2 * j + 1), f.inv_h_f, 1.0f);
    d = madd(madd(d, u, v3(f.right_f[0], f.right_f[1], f.right_f[2])), v, v3(f.up_f[0], f.up_f[1], f.up_f[2]));
    return rsqrtf(dot(d, d)) * d;
}

// Float-float arithmetic (Dekker 1971, Knuth's TwoSum): a value held as an
// unevaluated sum hi + lo of two floats, about 48 bits. The float path forms
// its primary ray and the two points it rounds from that ray this way, on the
// FP32 pipe, instead of in FP64 (a GB300 SM runs FP64 at 1/64 of the FP32
// rate). Products and sums use the _rn intrinsics so that no step is fused.
struct Ff3 {
    V3<float> hi, lo;
};

// s + e = a + b exactly (s the rounded sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// round(x + t d - p), one component: x and d float pairs, t and p floats
__device__ __forceinline__ float ff_point(float xh, float xl, float t, float dh, float dl, float p) {
    float s1, e1, s2, e2;
    two_sum(xh, -p, s1, e1);
    const float pr = __fmul_rn(t, dh);
    const float ep = __fmaf_rn(t, dh, -pr);  // t dh - pr exactly
    two_sum(s1, pr, s2, e2);
    return __fadd_rn(s2, __fadd_rn(__fadd_rn(xl, e1), __fadd_rn(__fadd_rn(e2, ep), __fmul_rn(t, dl))));
}

// x + t d - p rounded to float, per component
__device__ __forceinline__ V3<float> ff_point3(const Ff3& x, float t, const Ff3& d, V3<float> p) {
    return v3(ff_point(x.hi.x, x.lo.x, t, d.hi.x, d.lo.x, p.x), ff_point(x.hi.y, x.lo.y, t, d.hi.y, d.lo.y, p.y),
              ff_point(x.hi.z, x.lo.z, t, d.hi.z, d.lo.z, p.z));
}

// round(x + t d) and what the rounding left out (x + t d = point + rest to
// about 2^-48 of the point), one component
__device__ __forceinline__ float ff_entry(float xh, float xl, float t, float dh, float dl, float& rest) {
    const float pr = __fmul_rn(t, dh);
    const float ep = __fmaf_rn(t, dh, -pr);
    float s, e;
    two_sum(xh, pr, s, e);
    const float l = __fadd_rn(__fadd_rn(xl, e), __fadd_rn(ep, __fmul_rn(t, dl)));
    const float pt = __fadd_rn(s, l);
    rest = __fsub_rn(l, __fsub_rn(pt, s));
    return pt;
}

// a0 + i ai + j aj as a float pair (i, j below 2^24, so i ai_hi and j aj_hi
// are split exactly by an FMA)
__device__ __forceinline__ void ff_affine(float a0h, float a0l, float fi, float aih, float ail, float fj, float ajh,
                                          float ajl, float& hi, float& lo) {
    const float p1 = __fmul_rn(fi, aih), e1 = __fmaf_rn(fi, aih, -p1);
    const float p2 = __fmul_rn(fj, ajh), e2 = __fmaf_rn(fj, ajh, -p2);
    float s1, r1, s2, r2;
    two_sum(a0h, p1, s1, r1);
    two_sum(s1, p2, s2, r2);
    const float l = __fadd_rn(__fadd_rn(__fadd_rn(a0l, __fmul_rn(fi, ail)), __fadd_rn(e1, e2)),
                              __fadd_rn(__fadd_rn(r1, r2), __fmul_rn(fj, ajl)));
    hi = __fadd_rn(s2, l);  // |l| is far below |s2|: a fast two-sum renormalises
    lo = __fsub_rn(l, __fsub_rn(hi, s2));
}

// a.hi + a.lo times b.hi + b.lo, as a pair (the lo * lo term dropped)
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& hi, float& lo) {
    const float p = __fmul_rn(ah, bh);
    const float e = __fadd_rn(__fmaf_rn(ah, bh, -p), __fadd_rn(__fmul_rn(ah, bl), __fmul_rn(al, bh)));
    hi = __fadd_rn(p, e);
    lo = __fsub_rn(e, __fsub_rn(hi, p));
}

// q / |q| as float pairs. 1/|q| starts from the hardware rsqrtf of |q|^2's
// high part and takes one Newton-Raphson step for the reciprocal square root,
// y1 = y0 + y0 (1 - n y0^2) / 2, with the residual 1 - n y0^2 formed from
// exact products; the step leaves about twice the seed's bits.
__device__ __forceinline__ void ff_normalise(Ff3& q) {
    float n, ne;  // |q|^2 = n + ne
    {
        float sq, se;
        ff_mul(q.hi.x, q.lo.x, q.hi.x, q.lo.x, n, ne);
        ff_mul(q.hi.y, q.lo.y, q.hi.y, q.lo.y, sq, se);
        float s, e;
        two_sum(n, sq, s, e);
        n = s;
        ne = __fadd_rn(__fadd_rn(ne, se), e);
        ff_mul(q.hi.z, q.lo.z, q.hi.z, q.lo.z, sq, se);
        two_sum(n, sq, s, e);
        n = s;
        ne = __fadd_rn(__fadd_rn(ne, se), e);
    }
    const float y0 = rsqrtf(n);
    float a, b;  // y0^2 = a + b exactly
    a = __fmul_rn(y0, y0);
    b = __fmaf_rn(y0, y0, -a);
    float c, cd;  // n a = c + cd exactly
    c = __fmul_rn(n, a);
    cd = __fmaf_rn(n, a, -c);
    // 1 - (n + ne)(a + b); 1 - c is exact (c is within a few ulp of 1)
    const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, c), cd), __fadd_rn(__fmul_rn(n, b), __fmul_rn(ne, a)));
    const float yl = __fmul_rn(__fmul_rn(0.5f, y0), r);
    ff_mul(q.hi.x, q.lo.x, y0, yl, q.hi.x, q.lo.x);
    ff_mul(q.hi.y, q.lo.y, y0, yl, q.hi.y, q.lo.y);
    ff_mul(q.hi.z, q.lo.z, y0, yl, q.hi.z, q.lo.z);
}

// The float path's primary ray of pixel (i, j) as float pairs, with no FP64:
// the orthographic origin, or the pinhole direction before normalisation, is
// affine in (i, j).
__device__ __forceinline__ void primary_ray_ff(const FrameDev& f, int i, int j, Ff3& o, Ff3& d) {
    const float fi = (float)i, fj = (float)j;
    Ff3 v;
    ff_affine(f.a0_hi[0], f.a0_lo[0], fi, f.ai_hi[0], f.ai_lo[0], fj, f.aj_hi[0], f.aj_lo[0], v.hi.x, v.lo.x);
    ff_affine(f.a0_hi[1], f.a0_lo[1], fi, f.ai_hi[1], f.ai_lo[1], fj, f.aj_hi[1], f.aj_lo[1], v.hi.y, v.lo.y);
    ff_affine(f.a0_hi[2], f.a0_lo[2], fi, f.ai_hi[2], f.ai_lo[2], fj, f.aj_hi[2], f.aj_lo[2], v.hi.z, v.lo.z);
    if (f.cam_kind == GBRT_CAMERA_ORTHO) {
        o = v;
        d.hi = v3(f.dir_hi[0], f.dir_hi[1], f.dir_hi[2]);
        d.lo = v3(f.dir_lo[0], f.dir_lo[1], f.dir_lo[2]);
    } else {
        o.hi = v3(f.eye_hi[0], f.eye_hi[1], f.eye_hi[2]);
        o.lo = v3(f.eye_lo[0], f.eye_lo[1], f.eye_lo[2]);
        ff_normalise(v);
        d = v;
    }
}

// Refinement of an FP32 root in the object's own frame. The FP32 walk's root t
// (along the ray x + t d, x its grid-entry point) is turned into the hit's
// offset from the object's base point p0 -- the point x + t d - p0 formed from
// float pairs (p0 is a float: the scene's coordinates are) and rounded to
// FP32; it has the size of the object (|w| <= r + L), so FP32 holds it to
// ~1e-7 of that -- and Newton steps in FP32 then move it along the ray by s to
// the surface: F(s) = |w_p + s d_p|^2 - r^2 (w_p, d_p: the parts perpendicular
// to the axis a; all of w and d for a sphere). The result is the offset w + s d
// (the re-projection then needs no more precision than FP32) and the root
// t + s, exactly, as a float pair for ranking near-ties. False when the steps
// do not settle (a grazing ray): the offset then stays at the FP32 root's
// point.
struct LocalHit {
    V3<float> w;     // hit point - p0
    float t, t_lo;   // root along the ray from its grid entry: t + t_lo exactly
};

// x = (oe, rest): the ray's grid-entry point and what its rounding left out;
// t: the FP32 root measured from oe along d (d.hi: the walk's direction)
__device__ __forceinline__ bool local_root(const SceneDev& sc, uint32_t id, const Ff3& x, const Ff3& d, float t,
                                           LocalHit& lh) {
    const V3<float> df = d.hi;
    V3<float> p0f, a;
    float L, r;
    Obj<float>::load(sc.obj, id, p0f, a, L, r);
    const V3<float> w = ff_point3(x, t, d, p0f);
    const float wa = dot(w, a), da = dot(df, a);
    const V3<float> wp = madd(w, -wa, a), dp = madd(df, -da, a);
    const float A = dot(dp, dp), B = dot(wp, dp), C = fmaf(-r, r, dot(wp, wp));
    float s = 0.0f, corr = 0.0f;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const float As = A * s;
        corr = __fdividef(fmaf(As + 2.0f * B, s, C), 2.0f * (As + B));
        s -= corr;
    }
    const bool ok = fabsf(corr) <= 1e-4f * (fabsf(s) + r) && isfinite(s);
    if (!ok) s = 0.0f;
    lh.w = madd(w, s, df);
    two_sum(t, s, lh.t, lh.t_lo);
    return ok;
}

// The ray's grid-entry point at te0, rounded once (x.hi), and what the
// rounding left out (x.lo).
__device__ __forceinline__ void entry_point(const Ff3& o, const Ff3& d, float te0, Ff3& x) {
    x.hi.x = ff_entry(o.hi.x, o.lo.x, te0, d.hi.x, d.lo.x, x.lo.x);
    x.hi.y = ff_entry(o.hi.y, o.lo.y, te0, d.hi.y, d.lo.y, x.lo.y);
    x.hi.z = ff_entry(o.hi.z, o.lo.z, te0, d.hi.z, d.lo.z, x.lo.z);
}

// FP32 path: nearest hit in FP32 from the float-float ray re-based at its
// grid entry (one rounding, so coordinates stay small relative to the scene),
// then the winner -- and a runner-up within a relative 1e-4 band -- refined in
// its object's frame (local_root); the nearer refined root wins.
__device__ __forceinline__ bool nearest_fp32_refined(const FrameDev& f, int i, int j, uint32_t& id, LocalHit& lh,
                                                     bool& overflow) {
    const float inf = Num<float>::inf();
    Ff3 o, d, x;
    primary_ray_ff(f, i, j, o, d);
    float te0, te1;
    if (!clip_grid<float>(f.grid, o.hi, d.hi, 0.0f, inf, te0, te1)) return false;
    // the walk starts at the entry point rounded once
    entry_point(o, d, te0, x);
    Nearest<float> h;
    if (!trace_nearest<float>(f.grid, f.scene, x.hi, d.hi, 0.0f, inf, h, overflow)) return false;
    // the refinement needs what the rounding left out: the ray and its entry
    // point are formed again (the same steps give the same floats), which is
    // cheaper than holding their low parts in registers through the walk
    // (the copies of i and j keep the compiler from reusing the first ones)
    int i2, j2;
    asm volatile("mov.b32 %0, %1;" : "=r"(i2) : "r"(i));
    asm volatile("mov.b32 %0, %1;" : "=r"(j2) : "r"(j));
    primary_ray_ff(f, i2, j2, o, d);
    entry_point(o, d, te0, x);
    local_root(f.scene, h.id1, x, d, h.t1, lh);
    id = h.id1;
    if (h.id2 != GBRT_MISS && (h.t2 - h.t1) <= 1e-4f * (h.t1 + te0)) {
        LocalHit l2;
        local_root(f.scene, h.id2, x, d, h.t2, l2);
        // t + t_lo pairs are normalised, so comparing them in order compares
        // the exact roots
        const bool nearer = l2.t < lh.t || (l2.t == lh.t && l2.t_lo < lh.t_lo);
        const bool same = l2.t == lh.t && l2.t_lo == lh.t_lo;
        if (nearer || (same && h.id2 < h.id1)) {
            id = h.id2;
            lh = l2;
        }
    }
    return true;
}

// Hit records: (AO origin xyz, pixel) and (normal xyz, object id). Bit 31 of
// the pixel word marks a hit from inside the surface (its normal turned
// toward the axis or centre); pixel indices stay below 2^31.
constexpr uint32_t HIT_INSIDE = 0x80000000u;
template <class R>
struct HitIO;

template <>
struct HitIO<float> {
    static __device__ __forceinline__ void store(void* hits, int64_t slot, V3<double> o, V3<double> n, uint32_t q,
                                                 uint32_t id) {
        store_f(hits, slot, to_f(o), to_f(n), q, id);
    }
    static __device__ __forceinline__ void store_f(void* hits, int64_t slot, V3<float> o, V3<float> n, uint32_t q,
                                                   uint32_t id) {
        float4* H = (float4*)hits + 2 * slot;
        H[0] = make_float4(o.x, o.y, o.z, __uint_as_float(q));
        H[1] = make_float4(n.x, n.y, n.z, __uint_as_float(id));
    }
    static __device__ __forceinline__ void load(const void* hits, int64_t slot, V3<float>& o, V3<float>& n,
                                                uint32_t& q, uint32_t& id) {
        const float4* H = (const float4*)hits + 2 * slot;
        float4 a = H[0], b = H[1];
        o = v3(a.x, a.y, a.z);
        q = __float_as_uint(a.w);
        n = v3(b.x, b.y, b.z);
        id = __float_as_uint(b.w);
    }
};

template <>
struct HitIO<double> {
    static __device__ __forceinline__ void store(void* hits, int64_t slot, V3<double> o, V3<double> n, uint32_t q,
                                                 uint32_t id) {
        double2* H = (double2*)hits + 4 * slot;
        H[0] = make_double2(o.x, o.y);
        H[1] = make_double2(o.z, __longlong_as_double((long long)q));
        H[2] = make_double2(n.x, n.y);
        H[3] = make_double2(n.z, __longlong_as_double((long long)id));
    }
    static __device__ __forceinline__ void load(const void* hits, int64_t slot, V3<double>& o, V3<double>& n,
                                                uint32_t& q, uint32_t& id) {
        const double2* H = (const double2*)hits + 4 * slot;
        double2 a = H[0], b = H[1], c = H[2], e = H[3];
        o = v3(a.x, a.y, b.x);
        q = (uint32_t)__double_as_longlong(b.y);
        n = v3(c.x, c.y, e.x);
        id = (uint32_t)__double_as_longlong(e.y);
    }
};

template <class R>
__device__ __forceinline__ R ao_maxdist(const FrameDev& f);
template <>
__device__ __forceinline__ float ao_maxdist<float>(const FrameDev& f) { return f.ao_maxdist_f; }
template <>
__device__ __forceinline__ double ao_maxdist<double>(const FrameDev& f) { return f.ao_maxdist; }

// ---------------------------------------------------------------- primary pass

// Prefix sums of hits and AO rays per frame; resets the AO and shading queues.
// Run by one thread of the primary pass's last CTA once every CTA's hits are
// counted (the counts are read through L2: other CTAs added them atomically).
__device__ __forceinline__ void ao_plan(const BatchDev& b) {
    unsigned long long jobs = 0, hits = 0;
    b.job_off[0] = 0;
    b.hit_off[0] = 0;
    for (int f = 0; f < b.nframes; ++f) {
        unsigned long long h = __ldcg(b.hit_count + f);
        hits += h;
        jobs += h * (unsigned long long)b.frames[f].jobs_per_hit;
        b.hit_off[f + 1] = hits;
        b.job_off[f + 1] = jobs;
    }
    b.queue[1] = 0;
    b.queue[2] = 0;
}


template <int MODE>
__global__ void __launch_bounds__(256) k_primary(const __grid_constant__ BatchDev b) {
    typedef typename std::conditional<MODE == GBRT_FP32, float, double>::type R;
    const int lane = threadIdx.x & 31;
    const long long total = b.tile_off[b.nframes];
    bool overflow = false;
    while (true) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(b.queue, 1ull);
        item = __shfl_sync(FULL, item, 0);
        if (item >= total) break;
        const int f = find_frame(b.tile_off, b.nframes, item);
        const FrameDev& F = b.frames[f];
        const long long t = item - b.tile_off[f];
        const int tx = (int)(t % F.tiles_x), ty = (int)(t / F.tiles_x);
        const int i = tx * b.tile_w + lane % b.tile_w;
        const int j = F.row0 + ty * b.tile_h + lane / b.tile_w;
        const bool inside = i < F.W && j < F.row0 + F.rows;
        V3<double> o64, d64;
        uint32_t id = GBRT_MISS;
        double t64 = 0.0;
        LocalHit lh;
        bool hit = false;
        if (inside) {
            if (MODE == GBRT_FP32) {
                hit = nearest_fp32_refined(F, i, j, id, lh, overflow);
            } else {
                primary_ray64(F, i, j, o64, d64);
                Nearest<double> h;
                hit = trace_nearest<double>(F.grid, F.scene, o64, d64, 0.0, Num<double>::inf(), h, overflow);
                id = h.id1;
                t64 = h.t1;
            }
        }
        // warp-aggregated append to this frame's hit list
        const unsigned hm = __ballot_sync(FULL, hit);
        unsigned base = 0;
        if (hm) {
            const int leader = __ffs(hm) - 1;
            if (lane == leader) base = atomicAdd(b.hit_count + f, (unsigned)__popc(hm));
            base = __shfl_sync(FULL, base, leader);
        }
        if (!inside) continue;
        const uint32_t q = (uint32_t)j * (uint32_t)F.W + (uint32_t)i;
        if (hit) {
            const int64_t slot = GBRT_INDEX(F.hit_base + base + __popc(hm & ((1u << lane) - 1u)), b.hit_cap);
            if (MODE == GBRT_FP32) {
                // the refined offset w from p0 splits into its foot on the
                // generator (centre or axis), p0 + (w.a) a, and w_p, the
                // radial part (length r at the refined root); the re-projected
                // surface point plus eps along the normal facing the ray is
                // p0 + (w.a) a + (r +- eps) w_p/|w_p|, formed in FP32 relative
                // to p0 and rounded once when p0 is added
                V3<float> p0, a;
                float L, r;
                Obj<float>::load(F.scene.obj, id, p0, a, L, r);
                const float wa = dot(lh.w, a);
                const V3<float> wp = madd(lh.w, -wa, a);
                const float inv = rsqrtf(dot(wp, wp));
                V3<float> nf = inv * wp;
                const bool flip = dot(view_dir_f(F, q), nf) > 0.0f;
                const V3<float> off = madd(wa * a, flip ? r - F.eps_f : r + F.eps_f, nf);
                const V3<float> ao_o = p0 + off;
                if (flip) nf = v3(-nf.x, -nf.y, -nf.z);
                HitIO<float>::store_f(b.hits, slot, ao_o, nf, q | (flip ? HIT_INSIDE : 0u), id);
            } else {
                V3<double> p, n;
                const bool inside_hit = reproject64(F.scene, id, o64, d64, t64, p, n);
                HitIO<R>::store(b.hits, slot, madd(p, F.eps, n), n, q | (inside_hit ? HIT_INSIDE : 0u), id);
            }
            b.vis[slot] = 0u;
            b.lmask[slot] = 0u;
            if (F.out_ids) F.out_ids[q] = id;
        } else {
            if (MODE == GBRT_FP32) {
                float* out = (float*)F.out_rgb + 3 * (size_t)(q - F.rgb_q0);
                out[0] = F.bg_f[0];
                out[1] = F.bg_f[1];
                out[2] = F.bg_f[2];
            } else {
                double* out = (double*)F.out_rgb + 3 * (size_t)(q - F.rgb_q0);
                out[0] = F.bg[0];
                out[1] = F.bg[1];
                out[2] = F.bg[2];
            }
            if (F.out_ids) F.out_ids[q] = GBRT_MISS;
            if (F.out_vis) F.out_vis[q] = 0u;
        }
    }
    if (overflow) atomicOr(b.err, ERR_DDA_STEPS);
    // the last CTA to finish lays out the AO pass (queue[3] counts finished
    // CTAs; it starts at zero with the batch's counters)
    __shared__ bool last_cta;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_cta = atomicAdd(b.queue + 3, 1ull) == (unsigned long long)gridDim.x - 1ull;
    }
    __syncthreads();
    if (last_cta && threadIdx.x == 0) {
        __threadfence();
        ao_plan(b);
    }
}

// ---------------------------------------------------------------- AO pass

// One AO job -- AO sample or direct-light shadow ray -- of the batch's
// global job index jj (hits of all frames x jobs per hit): the hit slot whose
// count or light bit it settles, its ray, and the hit's own object when that
// object cannot be met again (a hit on a convex outer side), else GBRT_MISS.
template <class R>
struct AoJob {
    V3<R> o, d;
    R tmax;
    uint32_t lbit;  // 0: an AO sample; 1 << l: the shadow ray toward light l
    uint32_t self;
    int64_t vslot;
    const FrameDev* F;
};

// False when no ray is cast: the surface faces away from the light (its bit
// stays clear).
template <class R>
__device__ __forceinline__ bool ao_job(const BatchDev& b, unsigned long long jj, AoJob<R>& J) {
    const int f = b.nframes == 1 ? 0 : find_frame(b.job_off, b.nframes, jj);
    const FrameDev& F = b.frames[f];
    J.F = &F;
    const unsigned long long jl = jj - b.job_off[f];
    const uint32_t jph = (uint32_t)F.jobs_per_hit;
    uint32_t h;
    if (jl >= 0xFFFFFFFFull) {
        h = (uint32_t)(jl / jph);
    } else if (jph > 1u) {
        // jl / jph by the multiplier ceil(2^32 / jph): the product's high word
        // is the quotient or one more
        h = __umulhi((uint32_t)jl, F.jph_magic);
        if ((unsigned long long)h * jph > jl) --h;
    } else {
        h = (uint32_t)jl;
    }
    const uint32_t smp = (uint32_t)(jl - (unsigned long long)h * jph);
    J.vslot = GBRT_INDEX(F.hit_base + (int64_t)h, b.hit_cap);
    V3<R> n;
    uint32_t q;
    HitIO<R>::load(b.hits, J.vslot, J.o, n, q, J.self);
    // the own object can be skipped only behind a convex outer side
    if (q & HIT_INSIDE) J.self = GBRT_MISS;
    q &= ~HIT_INSIDE;
    if (smp < (uint32_t)F.spp) {
        uint32_t b1, b2;
        ao_uniforms(q, smp, F.frame, F.seed_lo, F.seed_hi, b1, b2);
        J.d = cosine_dir(n, b1, b2);
        J.tmax = ao_maxdist<R>(F);
        J.lbit = 0u;
        return true;
    }
    // shadow ray toward light l (none where the surface faces away)
    const int l = (int)(smp - (uint32_t)F.spp);
    J.d = ShadeP<R>::ldir(F, l);
    J.tmax = Num<R>::inf();
    J.lbit = 1u << l;
    return dot(n, J.d) > R(0);
}

// A ray that leaves the objects' bounds unoccluded: one more escaped AO
// sample, or its light's bit.
__device__ __forceinline__ void ao_escape(const BatchDev& b, int64_t vslot, uint32_t lbit) {
    if (lbit) atomicOr(b.lmask + vslot, lbit);
    else atomicAdd(b.vis + vslot, 1u);
}

// Ray record in shared memory: (origin, tmax) and (direction, -) -- two
// 128-bit loads per test in the FP32 path.
template <class R>
struct __align__(16) AoRay {
    V3<R> o;
    R tmax;
    V3<R> d;
    R pad;
};

// Per-warp shared state of the cooperative AO walk.
//   ray[lane]      the lane's ray (origin, tmax, direction)
//   sd             where each ray's pairs of the current iteration find their
//                  items (one range per cell taken)
//   owner          the ray whose pairs start at a position of the current chunk
//   mbox[lane]     direct-mapped ids this ray already tested (rows padded by
//                  one word so distinct rays and slots fall in distinct
//                  banks); a re-test of a missed object cannot hit, so
//                  skipping it is exact
//   obj, items     the ray's scene records and grid item list (batches mix
//                  scenes)
//   fifo[lane]     cells the ray has stepped to and loaded but not yet taken
//   q              (FP64 path) surviving (ray, object) pairs waiting for a
//                  full test batch
// cells each active ray takes per lockstep iteration: further cells while it
// holds fewer than AoCfg<R>::min_pairs candidates, at most AO_CELLS
constexpr int AO_CELLS = 4;
// AO rays a warp claims from the global queue at once (its local pool)
constexpr unsigned AO_CLAIM = 64;

// Per-precision choices. FP32: pairs are tested where they were mapped, one
// per lane, so a lane whose pair is a re-test would compute and discard it
// anyway -- no mailbox (a re-test of a missed object misses again, and the
// hit's own object cannot be met behind a convex outer side, so testing
// either is exact). FP64: the test occupies the FP64 pipe, so lanes left idle
// cost more than shared memory -- an 8-slot mailbox drops re-tests, and the
// surviving pairs are queued and tested in full batches of 32 (in-place tests
// measured 13% slower there).
template <class R>
struct AoCfg;
template <>
struct AoCfg<float> {
    static constexpr int mbox = 0;
    static constexpr bool queue = false;
    static constexpr unsigned min_pairs = 8;  // 6: 0.5% slower, 12: 1.5% slower
};
template <>
struct AoCfg<double> {
    static constexpr int mbox = 8;
    static constexpr bool queue = true;
    static constexpr unsigned min_pairs = 4;  // 3: 0.4% slower, 6: 2.1%, 8: 5.0%
};

template <class R, bool Q = AoCfg<R>::queue>
struct AoQueue {};
template <class R>
struct AoQueue<R, true> {
    uint2 q[64];  // queued pairs (ray lane, object id)
};

// per ray: direct-mapped ids it already tested (rows padded by one word so
// distinct rays and slots fall in distinct banks)
template <class R, int M = AoCfg<R>::mbox>
struct AoMbox {
    uint32_t mbox[32][M + 1];
};
template <class R>
struct AoMbox<R, 0> {};

// per ray: its scene records and grid item list, when a batch mixes scenes
// (UNI: every frame of the batch has the same scene and grid -- the pointers
// are then kernel-wide)
template <class R, bool UNI>
struct AoPtrs {
    ObjPtr<R> obj[32];
    const uint32_t* items[32];
#ifdef GBRT_CHECKED
    int64_t nitems[32];  // the lengths the checked build tests indices against
    int64_t nobj[32];
#endif
};
template <class R>
struct AoPtrs<R, true> {};

// 4 KB a warp at most in the FP32 path: four resident CTAs of 8 warps fit the
// 132 KB shared-memory configuration, leaving 124 KB of the SM's 256 KB to the
// L1 that caches the walk's cell, item and object loads. Measured: 5.25 KB a
// warp (60 KB of L1) 2.5% slower, 5 KB (92 KB of L1, with an 8-slot mailbox
// and a test queue) 1% slower.
static_assert(AO_CELLS == 4, "the pair segments of a ray are kept as one uint4 of starts and one of offsets");
template <class R, bool UNI>
struct AoWarp : AoQueue<R>, AoMbox<R>, AoPtrs<R, UNI> {
    AoRay<R> ray[32];
    // item index of pair p of ray r: p + sdo[r][g] for the last cell g whose
    // pairs start at or before p (sds[r][g])
    uint4 sds[32];
    uint4 sdo[32];
    uint32_t owner[32];  // ray whose pairs start at this position of the current chunk
    // cells a ray has loaded but not yet taken, oldest first: an iteration takes
    // at least one of its at most AO_CELLS cells, so AO_CELLS - 1 wait at most
    uint2 fifo[32][AO_CELLS - 1];
};
static_assert(sizeof(AoWarp<float, false>) <= 4096, "the FP32 AO walk's per-warp state outgrew its 4 KB");

template <class R, bool UNI>
__device__ __forceinline__ ObjPtr<R> ao_obj(const AoWarp<R, UNI>& S, unsigned r, ObjPtr<R> uni) {
    if constexpr (UNI) return uni;
    else return S.obj[r];
}
template <class R, bool UNI>
__device__ __forceinline__ const uint32_t* ao_items(const AoWarp<R, UNI>& S, unsigned r, const uint32_t* uni) {
    if constexpr (UNI) return uni;
    else return S.items[r];
}
#ifdef GBRT_CHECKED
// ray r's item-buffer length and object count (the checked build's bounds)
template <class R, bool UNI>
__device__ __forceinline__ int64_t ao_nitems(const AoWarp<R, UNI>& S, unsigned r, int64_t uni) {
    if constexpr (UNI) return uni;
    else return S.nitems[r];
}
template <class R, bool UNI>
__device__ __forceinline__ int64_t ao_nobj(const AoWarp<R, UNI>& S, unsigned r, int64_t uni) {
    if constexpr (UNI) return uni;
    else return S.nobj[r];
}
#define GBRT_AO_ITEM(idx, r) GBRT_INDEX(idx, ao_nitems(S, r, unitems))
#define GBRT_AO_OBJ(id, r) GBRT_INDEX(id, ao_nobj(S, r, unobj))
#else
#define GBRT_AO_ITEM(idx, r) (idx)
#define GBRT_AO_OBJ(id, r) (id)
#endif

// FP64 path: test queued pairs [0, n) (1 <= n <= 32), one per lane (lanes
// past n redo pair 0 and discard it, so the batch runs without branches);
// returns the rays hit, as bits.
template <class R, bool UNI>
__device__ __forceinline__ unsigned ao_test_batch(AoWarp<R, UNI>& S, int lane, unsigned n, ObjPtr<R> uobj) {
    const unsigned idx = (unsigned)lane < n ? (unsigned)lane : 0u;
    const uint2 e = S.q[idx];
    const unsigned r = e.x;
    const uint32_t id = e.y;
    const AoRay<R> ray = S.ray[r];
    const bool hit = any_hit_object<R>(ao_obj(S, r, uobj), id, ray.o, ray.d, ray.tmax) && (unsigned)lane < n;
    return __reduce_or_sync(FULL, hit ? (1u << r) : 0u);
}

// Lockstep cooperative walk: every iteration each active ray takes its next
// one to AO_CELLS cells (all lanes run the same step code); the warp lays the
// (ray, item) pairs of those cells out densely with a scan and tests them 32
// at a time, one pair per lane (the FP64 path skipping the ray's own object
// and re-tests). UNI: every frame of the batch has the same scene and grid.
template <class R, bool UNI>
__global__ void __launch_bounds__(256) k_ao_walk(const __grid_constant__ BatchDev b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AoWarp<R, UNI>& S = reinterpret_cast<AoWarp<R, UNI>*>(smem_raw)[threadIdx.x >> 5];
    grid_dependency_wait();
    ObjPtr<R> uobj = nullptr;
    const uint32_t* uitems = nullptr;
    const uint2* ucells = nullptr;
    if constexpr (UNI) {
        uobj = Obj<R>::base(b.frames[0].scene);
        uitems = b.frames[0].grid.items;
        ucells = b.frames[0].grid.cells;
    }
#ifdef GBRT_CHECKED
    const int64_t unitems = b.frames[0].grid.nitems;
    const int64_t unobj = (int64_t)b.frames[0].scene.S + b.frames[0].scene.C;
#endif
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned long long total = b.job_off[b.nframes];
    const int refill = b.refill;
    bool has = false, exhausted = false, overflow = false;
    Walk<R> w;
    unsigned nf = 0;      // cells waiting in this lane's fifo
    bool wend = false;    // the walk has no further cells
    uint32_t lbit = 0;  // 0: an AO sample; 1 << l: the shadow ray toward light l
    int64_t vslot = 0;
    const uint2* cells = nullptr;
    // the warp's pool of claimed rays [pool, pool_end) (warp-uniform)
    unsigned long long pool = 0, pool_end = 0;
    while (true) {
        // 1. compaction of rays: idle lanes take the next rays together, from
        //    the warp's pool, which claims AO_CLAIM more rays from the global
        //    queue when it runs short (one atomic per AO_CLAIM rays)
        const unsigned act = __ballot_sync(FULL, has);
        if (!exhausted && __popc(act) < refill) {
            const unsigned idle = ~act;
            const unsigned need = __popc(idle);
            const unsigned long long rem = pool_end - pool;
            unsigned long long fresh_base = 0;
            if (rem < need) {
                if (lane == 0) fresh_base = atomicAdd(b.queue + 1, (unsigned long long)AO_CLAIM);
                fresh_base = __shfl_sync(FULL, fresh_base, 0);
                if (fresh_base >= total) exhausted = true;
            }
            if (!has) {
                const unsigned i = __popc(idle & lt);
                const unsigned long long jj = i < rem ? pool + i : fresh_base + (i - rem);
                if (jj < total) {
                    AoJob<R> J;
                    const bool cast = ao_job<R>(b, jj, J);
                    vslot = J.vslot;
                    lbit = J.lbit;
                    if (!cast) {
                        // the light cannot reach this side: its bit stays clear
                    } else if (walk_start(J.F->grid, J.o, J.d, R(0), J.tmax, w)) {
                        if constexpr (UNI) {
                            cells = ucells;
                        } else {
                            cells = J.F->grid.cells;
                            S.obj[lane] = Obj<R>::base(J.F->scene);
                            S.items[lane] = J.F->grid.items;
#ifdef GBRT_CHECKED
                            S.nitems[lane] = J.F->grid.nitems;
                            S.nobj[lane] = (int64_t)J.F->scene.S + J.F->scene.C;
#endif
                        }
                        AoRay<R> ray;
                        ray.o = J.o;
                        ray.tmax = J.tmax;
                        ray.d = J.d;
                        ray.pad = R(0);
                        S.ray[lane] = ray;
                        if constexpr (AoCfg<R>::mbox > 0) {
#pragma unroll
                            for (int m = 0; m < AoCfg<R>::mbox; ++m) S.mbox[lane][m] = GBRT_MISS;
                            // the own object starts in the mailbox: it is skipped like a
                            // re-test while it stays there (testing it is harmless too --
                            // behind a convex outer side the ray cannot meet it again)
                            if (J.self != GBRT_MISS) S.mbox[lane][J.self & (AoCfg<R>::mbox - 1)] = J.self;
                        }
                        // the walk stands on its first cell: its record waits in
                        // the fifo, so every later cell comes from a step
                        S.fifo[lane][0] = __ldg(cells + GBRT_INDEX(w.cell, w.ncells));
                        nf = 1;
                        wend = false;
                        has = true;
                    } else {
                        ao_escape(b, vslot, lbit);  // misses the objects' bounds: escapes
                    }
                }
            }
            if (rem >= need) {
                pool += need;
            } else {
                pool = fresh_base + (need - rem);
                pool_end = fresh_base + AO_CLAIM;
            }
        }
        if (exhausted && __ballot_sync(FULL, has) == 0) break;
        // 2. every active ray takes its next cells: its first, and further ones
        //    while it holds fewer than min_pairs candidates (an any-hit
        //    query may test objects past its first hit, so taking several at
        //    once is exact). The ray's fifo is first topped up to AO_CELLS
        //    loaded cells -- the new cells' loads are independent and overlap
        //    -- and the cells it does not take wait there for the next iteration
        // the walk's bound, counted per iteration rather than per step (every
        // iteration takes at least one cell or ends the ray, so a walk of the
        // grid's nx + ny + nz + 1 cells never reaches it; one whose crossing
        // times are not numbers ends here)
        if (has && --w.left <= 0) {
            overflow = true;
            wend = true;
            nf = 0;
        }
        bool ending = false;
        unsigned kg[AO_CELLS], ng[AO_CELLS];
        unsigned avail = 0u;
#pragma unroll
        for (int g = 0; g < AO_CELLS; ++g) {
            uint2 cr = make_uint2(0u, 0u);
            const bool queued = has && g < AO_CELLS - 1 && (unsigned)g < nf;
            if (queued) cr = S.fifo[lane][g];
            if (has && !queued && !wend) {
                if (walk_step(w)) cr = __ldg(cells + GBRT_INDEX(w.cell, w.ncells));
                else wend = true;
            }
            if (has && (queued || !wend)) avail = (unsigned)g + 1u;
            kg[g] = cr.x;
            ng[g] = cr.y;
        }
        if (has) {
            // take cells 0..m-1; the rest go back to the fifo
            // m = 1 + the number of prefixes (cells 0..g-1, g < avail) still
            // below min_pairs candidates: both conditions only turn false
            // (m = 0 when the walk has no cell left: the ray escapes below)
            const unsigned c1 = ng[0], c2 = c1 + ng[1], c3 = c2 + ng[2];
            constexpr unsigned MP = AoCfg<R>::min_pairs;
            const unsigned m = (avail > 0u) + (avail > 1u && c1 < MP) + (avail > 2u && c2 < MP) + (avail > 3u && c3 < MP);
#pragma unroll
            for (int g = 1; g < AO_CELLS; ++g) {
                if ((unsigned)g >= m && (unsigned)g < avail) S.fifo[lane][g - m] = make_uint2(kg[g], ng[g]);
                ng[g] = (unsigned)g >= m ? 0u : ng[g];
            }
            nf = avail - m;
            ending = wend && nf == 0u;  // escapes unless this iteration's tests hit
        }
        // 3. lay the warp's (ray, item) pairs out densely
        unsigned cnt = 0u;
#pragma unroll
        for (int g = 0; g < AO_CELLS; ++g) cnt += ng[g];
        unsigned incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        const unsigned T = __shfl_sync(FULL, incl, 31);
        unsigned hitbits = 0;
        if (T > 0) {
            const unsigned ex = incl - cnt;
            const unsigned s1 = ex + ng[0], s2 = s1 + ng[1], s3 = s2 + ng[2];
            S.sds[lane] = make_uint4(ex, s1, s2, s3);
            S.sdo[lane] = make_uint4(kg[0] - ex, kg[1] - s1, kg[2] - s2, kg[3] - s3);
            // 4. map pairs to (ray, object) 32 at a time and test them: in
            //    place in the FP32 path (lanes past the last pair redo it, so
            //    the test runs without branches), through the queue in full
            //    batches of 32 after the mailbox in the FP64 path
            unsigned qn = 0;
            for (unsigned base = 0; base < T; base += 32) {
                // rays mark where their pairs start inside this chunk; a pair's
                // ray is the last start at or before it. A ray takes part when its
                // pairs [ex, incl) are not empty and meet [base, base + 32).
                const unsigned u = ex > base ? ex : base;
                const unsigned pos = u - base;
                const bool mine = pos < 32u && incl > u;
                if (mine) S.owner[pos] = (uint32_t)lane;
                const unsigned starts = __reduce_or_sync(FULL, mine ? (1u << pos) : 0u);
                __syncwarp();
                const unsigned p = base + lane < T ? base + lane : T - 1u;
                const unsigned r = S.owner[31 - __clz(starts & (0xFFFFFFFFu >> (31 - lane)))];
                const uint4 st = S.sds[r], so = S.sdo[r];
                unsigned di = so.x;
                di = p >= st.y ? so.y : di;
                di = p >= st.z ? so.z : di;
                di = p >= st.w ? so.w : di;
                const uint32_t id = GBRT_AO_OBJ(__ldg(ao_items(S, r, uitems) + GBRT_AO_ITEM(p + di, r)), r);
                if constexpr (AoCfg<R>::queue) {
                    uint32_t* slot = &S.mbox[r][id & (AoCfg<R>::mbox - 1)];
                    const bool keep = base + lane < T && *slot != id;
                    const unsigned bal = __ballot_sync(FULL, keep);
                    if (keep) {
                        *slot = id;
                        S.q[qn + __popc(bal & lt)] = make_uint2(r, id);
                    }
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn >= 32) {
                        hitbits |= ao_test_batch(S, lane, 32u, uobj);
                        __syncwarp();
                        if ((unsigned)lane < qn - 32) S.q[lane] = S.q[32 + lane];
                        qn -= 32;
                        __syncwarp();
                    }
                } else {
                    const AoRay<R> ray = S.ray[r];
                    R t;
                    const bool hit = hit_object<R>(ao_obj(S, r, uobj), id, ray.o, ray.d, R(0), ray.tmax, t);
                    hitbits |= hit ? (1u << r) : 0u;  // OR-ed over the warp after the last chunk
                    __syncwarp();
                }
            }
            if constexpr (AoCfg<R>::queue) {
                if (qn > 0) hitbits |= ao_test_batch(S, lane, qn, uobj);
            } else {
                hitbits = __reduce_or_sync(FULL, hitbits);
            }
        }
        // 5. any hit occludes the ray; a ray whose walk ended escapes
        const bool occluded = (hitbits >> lane) & 1u;
        if (has && (occluded || ending)) {
            if (!occluded) ao_escape(b, vslot, lbit);
            has = false;
        }
        __syncwarp();
    }
    if (overflow) atomicOr(b.err, ERR_DDA_STEPS);
}

// ---------------------------------------------------------------- shading

template <class R>
__global__ void __launch_bounds__(256) k_shade(const __grid_constant__ BatchDev b) {
    grid_dependency_wait();
    const unsigned long long total = b.hit_off[b.nframes];
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        const int f = find_frame(b.hit_off, b.nframes, g);
        const FrameDev& F = b.frames[f];
        const int64_t slot = GBRT_INDEX(F.hit_base + (int64_t)(g - b.hit_off[f]), b.hit_cap);
        V3<R> o, n;
        uint32_t q, id;
        HitIO<R>::load(b.hits, slot, o, n, q, id);
        q = GBRT_INDEX(q & ~HIT_INSIDE, (uint32_t)F.W * (uint32_t)F.H);
        id = GBRT_INDEX(id, F.scene.S + F.scene.C);
        const uint32_t vis = b.vis[slot];
        V3<R> d;
        if (std::is_same<R, float>::value) {
            V3<float> df = view_dir_f(F, q);
            d = v3((R)df.x, (R)df.y, (R)df.z);
        } else {
            V3<double> o64, d64;
            primary_ray64(F, (int)(q % (uint32_t)F.W), (int)(q / (uint32_t)F.W), o64, d64);
            d = v3((R)d64.x, (R)d64.y, (R)d64.z);
        }
        R V = F.spp > 0 ? (R)vis / (R)F.spp : R(1);
        const uint32_t lit = F.shadows ? b.lmask[slot] : 0xFFFFFFFFu;
        R rgb[3];
        shade<R>(F, id, n, d, V, lit, rgb);
        // the colour buffer holds pixels [rgb_q0, ...): the whole image (rgb_q0 = 0)
        // or, for a supersampled frame, the finer raster's band (rgb_q0 = row0 W);
        // either way the band's pixels end at (row0 + rows) W
        R* out = (R*)F.out_rgb +
                 3 * (size_t)GBRT_INDEX((int64_t)q - F.rgb_q0, (int64_t)(F.row0 + F.rows) * F.W - F.rgb_q0);
        out[0] = rgb[0];
        out[1] = rgb[1];
        out[2] = rgb[2];
        if (F.out_vis) F.out_vis[q] = vis;
    }
}

// ---------------------------------------------------------------- grids rebuilt on the device

// Frames whose grid was rebuilt on the device take its current geometry
// before the frame's kernels run (their descriptors were written on the host).
__global__ void k_patch_grids(const __grid_constant__ BatchDev b) {
    FrameDev* frames = const_cast<FrameDev*>(b.frames);
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < b.nframes; f += gridDim.x * blockDim.x)
        if (frames[f].grid_src) frames[f].grid = *frames[f].grid_src;
}

// ---------------------------------------------------------------- supersampling

// Box filter of supersampled frames: output pixel (i, j) is the mean of the
// m x m finer-raster colours (m i + a, m j + b), summed sub-row by sub-row.
// Frames are strided over blockIdx.y; frames without supersampling are skipped.
template <class R>
__global__ void __launch_bounds__(256) k_resolve(const __grid_constant__ BatchDev b) {
    grid_dependency_wait();
    for (int f = blockIdx.y; f < b.nframes; f += gridDim.y) {
        const FrameDev& F = b.frames[f];
        const int m = F.aa;
        if (m <= 1) continue;
        const int w = F.W / m;
        const int j0 = F.row0 / m;
        const long long n = (long long)w * (F.rows / m);
        const R mm = (R)(m * m);
        const R* fine = (const R*)F.out_rgb;
        R* out = (R*)F.out_final;
        for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
             k += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(k % w), j = j0 + (int)(k / w);
            R acc[3] = {R(0), R(0), R(0)};
            for (int sb = 0; sb < m; ++sb) {
                const R* row = fine + 3 * ((long long)(m * j + sb) * F.W + (long long)m * i - F.rgb_q0);
                for (int sa = 0; sa < m; ++sa) {
                    acc[0] += row[3 * sa];
                    acc[1] += row[3 * sa + 1];
                    acc[2] += row[3 * sa + 2];
                }
            }
            R* o = out + 3 * ((long long)j * w + i);
            o[0] = acc[0] / mm;
            o[1] = acc[1] / mm;
            o[2] = acc[2] / mm;
        }
    }
}

// ---------------------------------------------------------------- probe, Philox

template <int MODE>
__global__ void __launch_bounds__(128) k_ao_probe(const __grid_constant__ FrameDev f, const double* pts,
                                                  const double* nrm, int64_t n, float* out, uint32_t* err) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    V3<double> p = ld3(pts + 3 * k), nn = ld3(nrm + 3 * k);
    V3<double> o = madd(p, f.eps, nn);
    bool overflow = false;
    int vis;
    if (MODE == GBRT_FP32)
        vis = ao_visible<float>(f, (uint32_t)k, to_f(o), to_f(nn), f.ao_maxdist_f, overflow);
    else
        vis = ao_visible<double>(f, (uint32_t)k, o, nn, f.ao_maxdist, overflow);
    out[k] = f.spp > 0 ? (float)vis / (float)f.spp : 1.0f;
    if (overflow) atomicOr(err, ERR_DDA_STEPS);
}

__global__ void k_philox(const uint4* ctr, const uint2* key, int64_t n, uint4* out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = philox4x32_10(ctr[k], key[k]);
}

// ---------------------------------------------------------------- host side

namespace {

int err_of(cudaError_t e) {
    if (e == cudaSuccess) return GBRT_OK;
    return e == cudaErrorMemoryAllocation ? GBRT_ENOMEM : GBRT_EDEVICE;
}

// Grow a device buffer (the stream is drained first: old work may still read it).
int grow(Ctx* ctx, void** p, size_t* cap, size_t need) {
    if (*cap >= need) return GBRT_OK;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = std::max(need, (size_t)4096);
    int rc = err_of(cudaMalloc(p, want));
    if (rc == GBRT_OK) *cap = want;
    ctx->graph_valid = false;
    return rc;
}

template <class K>
int persistent_grid(Ctx* ctx, K kernel, int block, size_t smem = 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (ctx->tuning.ctas_per_sm > 0) per_sm = std::min(per_sm, ctx->tuning.ctas_per_sm);
    return per_sm * ctx->num_sms;
}

}  // namespace

// Lay out one batch (all frames of one precision), upload its descriptors and
// enqueue memsets + the four kernels on `stream`.
struct Grids {
    int primary, ao, shade, resolve;
};

// Launch `kernel` as a programmatic dependent of the kernel before it in
// `stream`: its CTAs may be scheduled while that kernel drains, and they wait
// (grid_dependency_wait) for its results before reading them.
static cudaError_t launch_dependent(void (*kernel)(BatchDev), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t stream, const BatchDev& bd) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, bd);
}

// The AO walk of one precision and scene layout (UNI: one scene and grid for
// the whole batch) with its dynamic shared memory; launched with an explicit
// grid, or with one sized for the current device (grid <= 0).
template <class R, bool UNI>
static size_t ao_smem(int block) {
    return (size_t)(block / 32) * sizeof(AoWarp<R, UNI>);
}

// Shared-memory share of the SM asked for the FP32 walk: just enough for four
// resident CTAs of 256 threads (and the driver's per-CTA reservation), so the
// rest of the SM's 256 KB serves as L1 for the walk's cell, item and object
// loads (the 100 KB configuration instead of the 132 KB one the driver picks
// by default: AO walk 1.185 -> 1.176 ms on the paper frame).
template <bool UNI>
static cudaError_t prefer_small_carveout() {
    int dev = 0, per_sm = 0, reserved = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess || per_sm <= 0) return e;
    const long long need = 4ll * ((long long)ao_smem<float, UNI>(256) + reserved);
    const int pct = (int)std::min<long long>(100, (need * 100 + per_sm - 1) / per_sm);
    return cudaFuncSetAttribute(k_ao_walk<float, UNI>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

static cudaError_t set_ao_smem_limits() {
    // a refused preference leaves the driver's choice (and its error is
    // cleared here, so it is not taken for a later launch's)
    if (prefer_small_carveout<true>() != cudaSuccess || prefer_small_carveout<false>() != cudaSuccess)
        (void)cudaGetLastError();
    // the AO kernels' per-warp staging can exceed the 48 KB default
    cudaError_t e = cudaFuncSetAttribute(k_ao_walk<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ao_smem<float, false>(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ao_walk<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ao_smem<float, true>(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ao_walk<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ao_smem<double, false>(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ao_walk<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ao_smem<double, true>(256));
    return e;
}

template <class R, bool UNI>
static int ao_grid(Ctx* ctx, int block) {
    return persistent_grid(ctx, k_ao_walk<R, UNI>, block, ao_smem<R, UNI>(block));
}

template <class R>
static void launch_ao(const BatchDev& bd, bool uni, int grid, int block, cudaStream_t stream) {
    if (uni) launch_dependent(k_ao_walk<R, true>, grid, block, ao_smem<R, true>(block), stream, bd);
    else launch_dependent(k_ao_walk<R, false>, grid, block, ao_smem<R, false>(block), stream, bd);
}

// The passes after the primary one: AO walk, shading, and the box filter of
// supersampled frames (the AO plan runs in the primary kernel's last CTA).
template <class R>
static void launch_after_primary(const BatchDev& bd, bool uni, int ao_grid, int block, int shade_grid,
                                 int resolve_grid, bool resolve, cudaStream_t stream,
                                 const std::function<void(int)>& mark) {
    launch_ao<R>(bd, uni, ao_grid, block, stream);
    mark(3);
    launch_dependent(k_shade<R>, shade_grid, 256, 0, stream, bd);
    if (resolve) launch_dependent(k_resolve<R>, dim3(resolve_grid, std::min(bd.nframes, 65535)), 256, 0, stream, bd);
}

static Grids grids_for(Ctx* ctx, int precision, bool uni) {
    const int block = ctx->tuning.block;
    if (!ctx->smem_configured) {
        set_ao_smem_limits();
        ctx->smem_configured = true;
    }
    Grids g;
    if (precision == GBRT_FP32) {
        g.primary = persistent_grid(ctx, k_primary<GBRT_FP32>, block);
        g.ao = uni ? ao_grid<float, true>(ctx, block) : ao_grid<float, false>(ctx, block);
    } else {
        g.primary = persistent_grid(ctx, k_primary<GBRT_FP64>, block);
        g.ao = uni ? ao_grid<double, true>(ctx, block) : ao_grid<double, false>(ctx, block);
    }
    g.shade = ctx->num_sms * 8;
    g.resolve = ctx->num_sms * 4;
    return g;
}

// Every frame of the batch reads the same scene and grid (device-side rebuilt
// grids: the same rebuilt grid).
static bool one_scene(const FrameDev* frames, int n) {
    for (int f = 1; f < n; ++f) {
        const FrameDev& a = frames[0];
        const FrameDev& c = frames[f];
        if (c.scene.obj != a.scene.obj || c.scene.obj64 != a.scene.obj64 || c.grid.items != a.grid.items ||
            c.grid.cells != a.grid.cells || c.grid_src != a.grid_src)
            return false;
    }
    return true;
}

// optional passes of a batch, and its scene layout
enum : int { EXTRA_RESOLVE = 1, EXTRA_PATCH = 2, EXTRA_UNI = 4 };

static int enqueue_batch(Ctx* ctx, cudaStream_t stream, int precision, const BatchDev& bd, size_t desc_bytes,
                         const Grids& gr, int extra) {
    const bool resolve = (extra & EXTRA_RESOLVE) != 0;
    cudaError_t e = cudaMemcpyAsync(ctx->d_desc, ctx->h_desc, desc_bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_counters, 0, ctx->counters_bytes_used, stream);
    if (e != cudaSuccess) return err_of(e);
    const int block = ctx->tuning.block;
    if (extra & EXTRA_PATCH) {
        k_patch_grids<<<1, 128, 0, stream>>>(bd);
        ctx->launches++;
    }
    // events between the kernels when timing (never inside a graph capture);
    // the AO-walk mode records only events 2 and 3, around the AO walk
    const int tm = stream == ctx->stream ? ctx->profiling : 0;
    auto mark = [&](int k) {
        if (tm == GBRT_PROFILE_ALL || (tm == GBRT_PROFILE_AO_WALK && (k == 2 || k == 3)))
            cudaEventRecord(ctx->ev[k], stream);
    };
    mark(0);
    const bool uni = (extra & EXTRA_UNI) != 0;
    if (precision == GBRT_FP32) {
        k_primary<GBRT_FP32><<<gr.primary, block, 0, stream>>>(bd);
        mark(1);
        mark(2);
        launch_after_primary<float>(bd, uni, gr.ao, block, gr.shade, gr.resolve, resolve, stream, mark);
    } else {
        k_primary<GBRT_FP64><<<gr.primary, block, 0, stream>>>(bd);
        mark(1);
        mark(2);
        launch_after_primary<double>(bd, uni, gr.ao, block, gr.shade, gr.resolve, resolve, stream, mark);
    }
    mark(4);
    if (tm) ctx->timed = tm;
    ctx->launches += resolve ? 4 : 3;
    return err_of(cudaGetLastError());
}

int render_frames(Ctx* ctx, FrameDev* frames, int n, bool use_graph) {
    if (n == 0) return GBRT_OK;
    const int precision = frames[0].precision;
    for (int f = 1; f < n; ++f)
        if (frames[f].precision != precision) return GBRT_EINVAL;
    const int tw = ctx->tuning.tile_w, th = ctx->tuning.tile_h;
    const size_t rec = precision == GBRT_FP32 ? 2 * sizeof(float4) : 4 * sizeof(double2);
    // descriptors: frames, then tile_off (n + 1)
    const size_t frames_bytes = ((size_t)n * sizeof(FrameDev) + 255) & ~(size_t)255;
    const size_t desc_bytes = frames_bytes + (size_t)(n + 1) * sizeof(long long);
    // counters: queue [4], hit_count [n], job_off [n + 1], hit_off [n + 1]
    const size_t counters_bytes = 4 * sizeof(unsigned long long) + (size_t)n * sizeof(unsigned) +
                                  2 * (size_t)(n + 1) * sizeof(unsigned long long) + 64;
    int64_t px = 0;
    long long tiles = 0;
    size_t fine_bytes = 0;  // finer-raster colours of the supersampled frames' bands
    bool resolve = false;
    int extra = 0;
    const size_t rgb_px = 3 * (precision == GBRT_FP32 ? sizeof(float) : sizeof(double));
    for (int f = 0; f < n; ++f) {
        frames[f].tiles_x = (frames[f].W + tw - 1) / tw;
        frames[f].tiles_y = (frames[f].rows + th - 1) / th;
        frames[f].hit_base = px;
        px += (int64_t)frames[f].W * frames[f].rows;
        tiles += (long long)frames[f].tiles_x * frames[f].tiles_y;
        if (frames[f].grid_src) extra |= EXTRA_PATCH;
        if (frames[f].aa > 1) {
            resolve = true;
            extra |= EXTRA_RESOLVE;
            fine_bytes += ((size_t)frames[f].W * frames[f].rows * rgb_px + 255) & ~(size_t)255;
        }
    }
    int rc;
    if (resolve) {
        if ((rc = grow(ctx, &ctx->d_fine, &ctx->fine_cap, fine_bytes)) != GBRT_OK) return rc;
        size_t off = 0;
        for (int f = 0; f < n; ++f) {
            if (frames[f].aa <= 1) continue;
            frames[f].out_rgb = (char*)ctx->d_fine + off;
            frames[f].rgb_q0 = (int64_t)frames[f].row0 * frames[f].W;
            off += ((size_t)frames[f].W * frames[f].rows * rgb_px + 255) & ~(size_t)255;
        }
    }
    if ((rc = grow(ctx, &ctx->d_hits, &ctx->hits_cap, (size_t)px * rec)) != GBRT_OK) return rc;
    if ((rc = grow(ctx, (void**)&ctx->d_vis, &ctx->vis_cap, (size_t)px * sizeof(unsigned))) != GBRT_OK) return rc;
    if ((rc = grow(ctx, (void**)&ctx->d_lmask, &ctx->lmask_cap, (size_t)px * sizeof(unsigned))) != GBRT_OK)
        return rc;
    if ((rc = grow(ctx, &ctx->d_desc, &ctx->desc_cap, desc_bytes)) != GBRT_OK) return rc;
    if ((rc = grow(ctx, &ctx->d_counters, &ctx->counters_cap, counters_bytes)) != GBRT_OK) return rc;
    if (ctx->h_desc_cap < desc_bytes) {
        if (ctx->staging_pending) cudaEventSynchronize(ctx->staging_done);
        cudaFreeHost(ctx->h_desc);
        ctx->h_desc = nullptr;
        ctx->h_desc_cap = 0;
        if (cudaMallocHost(&ctx->h_desc, desc_bytes) != cudaSuccess) return GBRT_ENOMEM;
        ctx->h_desc_cap = desc_bytes;
        ctx->graph_valid = false;
    }
    // the pinned staging buffer is read by the previous batch's copy: wait for it
    if (ctx->staging_pending) cudaEventSynchronize(ctx->staging_done);
    memcpy(ctx->h_desc, frames, (size_t)n * sizeof(FrameDev));
    long long* toff = (long long*)((char*)ctx->h_desc + frames_bytes);
    toff[0] = 0;
    for (int f = 0; f < n; ++f) toff[f + 1] = toff[f] + (long long)frames[f].tiles_x * frames[f].tiles_y;

    BatchDev bd;
    bd.frames = (const FrameDev*)ctx->d_desc;
    bd.tile_off = (const long long*)((char*)ctx->d_desc + frames_bytes);
    char* cb = (char*)ctx->d_counters;
    bd.queue = (unsigned long long*)cb;
    bd.job_off = (unsigned long long*)(cb + 4 * sizeof(unsigned long long));
    bd.hit_off = bd.job_off + (n + 1);
    bd.hit_count = (unsigned*)(bd.hit_off + (n + 1));
    bd.hits = ctx->d_hits;
    bd.vis = ctx->d_vis;
    bd.lmask = ctx->d_lmask;
    bd.err = ctx->d_err;
    bd.hit_cap = (int64_t)px;
    bd.nframes = n;
    bd.tile_w = tw;
    bd.tile_h = th;
    bd.refill = ctx->tuning.refill;
    ctx->counters_bytes_used = counters_bytes;

    const bool uni = one_scene(frames, n);
    if (uni) extra |= EXTRA_UNI;
    const Grids gr = grids_for(ctx, precision, uni);
    if (!use_graph) {
        rc = enqueue_batch(ctx, ctx->stream, precision, bd, desc_bytes, gr, extra);
    } else {
        // replay a captured graph of {copy, memset, 4 kernels} when the batch
        // layout (buffers, counts, launch shape) is unchanged
        const long long key = ((long long)n << 40) ^ ((long long)precision << 36) ^ ((long long)gr.primary << 18) ^
                              (long long)gr.ao ^ ((long long)desc_bytes << 1);
        if (!ctx->graph_valid || ctx->graph_key != key || ctx->graph_extra != extra ||
            memcmp(&ctx->graph_bd, &bd, sizeof(bd)) != 0) {
            if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
            ctx->graph_valid = false;
            if (!ctx->capture_stream &&
                cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
                return GBRT_EDEVICE;
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return GBRT_EDEVICE;
            int64_t launches0 = ctx->launches;
            int crc = enqueue_batch(ctx, ctx->capture_stream, precision, bd, desc_bytes, gr, extra);
            ctx->launches = launches0;
            cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
            if (crc != GBRT_OK || ce != cudaSuccess) return crc != GBRT_OK ? crc : GBRT_EDEVICE;
            ce = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return GBRT_EDEVICE;
            ctx->graph_valid = true;
            ctx->graph_key = key;
            ctx->graph_extra = extra;
            ctx->graph_bd = bd;
        }
        rc = err_of(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
        ctx->launches += 3 + (resolve ? 1 : 0) + ((extra & EXTRA_PATCH) ? 1 : 0);
    }
    if (rc != GBRT_OK) return rc;
    cudaEventRecord(ctx->staging_done, ctx->stream);
    ctx->staging_pending = true;
    return GBRT_OK;
}

int configure_render_kernels() { return err_of(set_ao_smem_limits()); }

int enqueue_prepared(const BatchDev& bd, int precision, cudaStream_t stream, int block, int num_sms, bool patch) {
    auto grid_of = [&](auto kernel, size_t smem) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return per_sm * num_sms;
    };
    // one frame: one scene and grid
    if (patch) k_patch_grids<<<1, 128, 0, stream>>>(bd);
    const auto none = [](int) {};
    if (precision == GBRT_FP32) {
        k_primary<GBRT_FP32><<<grid_of(k_primary<GBRT_FP32>, 0), block, 0, stream>>>(bd);
        launch_after_primary<float>(bd, true, grid_of(k_ao_walk<float, true>, ao_smem<float, true>(block)), block,
                                    num_sms * 8, 0, false, stream, none);
    } else {
        k_primary<GBRT_FP64><<<grid_of(k_primary<GBRT_FP64>, 0), block, 0, stream>>>(bd);
        launch_after_primary<double>(bd, true, grid_of(k_ao_walk<double, true>, ao_smem<double, true>(block)), block,
                                     num_sms * 8, 0, false, stream, none);
    }
    return err_of(cudaGetLastError());
}

int launch_ao_probe(Ctx* ctx, const FrameDev& f, const double* pts, const double* nrm, int64_t n, float* out) {
    if (n == 0) return GBRT_OK;
    int blocks = (int)((n + 127) / 128);
    if (f.precision == GBRT_FP32)
        k_ao_probe<GBRT_FP32><<<blocks, 128, 0, ctx->stream>>>(f, pts, nrm, n, out, ctx->d_err);
    else
        k_ao_probe<GBRT_FP64><<<blocks, 128, 0, ctx->stream>>>(f, pts, nrm, n, out, ctx->d_err);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GBRT_OK : GBRT_EDEVICE;
}

int launch_philox(Ctx* ctx, const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out) {
    if (n == 0) return GBRT_OK;
    int blocks = (int)((n + 255) / 256);
    k_philox<<<blocks, 256, 0, ctx->stream>>>((const uint4*)ctr, (const uint2*)key, n, (uint4*)out);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GBRT_OK : GBRT_EDEVICE;
}

#ifdef GBRT_CHECKED
// Indices the checked build found outside their buffers since the last call
// (the render kernels' counter), cleared as it is read.
unsigned long long checked_violations_render() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_oob, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_oob, &z, sizeof(z));
    return v;
}
#endif

}  // namespace gbrt
