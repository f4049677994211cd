// Device math of the ray tracer: vectors, ray-sphere and ray-cylinder roots,
// the Amanatides-Woo grid walk, Philox4x32-10, cosine-weighted AO directions,
// hit refinement and Phong + skylight shading. Templated on the arithmetic
// type R: float for the FP32 path, double for the plain FP64 path.
#pragma once

#include <stdint.h>

#include <type_traits>

#include "gbrt_types.h"

namespace gbrt {

// ---------------------------------------------------------------- checked build

// GBRT_INDEX(i, n): an index that comes from data (a cell, an item, an object
// id, a hit slot, a pixel) into a buffer of n elements. In the normal build it
// is i itself. In the checked build (-DGBRT_CHECKED, libgbrt_checked.so) an
// index outside [0, n) is counted in this translation unit's g_oob and
// replaced by 0, so the access stays inside the buffer; gbrt_sync then
// reports GBRT_EBOUNDS.
#ifdef GBRT_CHECKED
static __device__ unsigned long long g_oob;
__device__ __forceinline__ unsigned long long checked_index(unsigned long long i, unsigned long long n) {
    if (i < n) return i;
    atomicAdd(&g_oob, 1ull);
    return 0ull;
}
#define GBRT_INDEX(i, n) ((decltype(i))::gbrt::checked_index((unsigned long long)(i), (unsigned long long)(n)))
#else
#define GBRT_INDEX(i, n) (i)
#endif

// ---------------------------------------------------------------- scalars

template <class R>
struct Num;

template <>
struct Num<float> {
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    // a ray is treated as parallel to a cylinder axis below this |d_perp|^2
    static __device__ __forceinline__ float parallel_eps() { return 1e-12f; }
};

template <>
struct Num<double> {
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double parallel_eps() { return 1e-24; }
};

template <class R>
struct V3 {
    R x, y, z;
};

template <class R>
__device__ __forceinline__ V3<R> v3(R x, R y, R z) { return V3<R>{x, y, z}; }
template <class R>
__device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class R>
__device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class R>
__device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return v3(s * a.x, s * a.y, s * a.z); }
template <class R>
__device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// a + s b
template <class R>
__device__ __forceinline__ V3<R> madd(V3<R> a, R s, V3<R> b) { return v3(a.x + s * b.x, a.y + s * b.y, a.z + s * b.z); }

template <class R>
__device__ __forceinline__ V3<R> normalized(V3<R> a) {
    R l = Num<R>::sqrt_(dot(a, a));
    return l > R(0) ? v3(a.x / l, a.y / l, a.z / l) : a;
}

__device__ __forceinline__ V3<float> to_f(V3<double> a) { return v3((float)a.x, (float)a.y, (float)a.z); }
__device__ __forceinline__ V3<double> to_d(V3<float> a) { return v3((double)a.x, (double)a.y, (double)a.z); }
__device__ __forceinline__ V3<double> ld3(const double* p) { return v3(p[0], p[1], p[2]); }

// ---------------------------------------------------------------- objects

// Reciprocal and square root used inside the primitive test: the FP32 path
// takes the hardware approximations (about 2 ulp), the FP64 path IEEE ones.
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_pos(float x) {
    x = fmaxf(x, 1e-30f);
    return x * rsqrtf(x);
}
__device__ __forceinline__ double sqrt_pos(double x) { return sqrt(fmax(x, 0.0)); }

template <class R>
struct Obj;

template <>
struct Obj<float> {
    static __device__ __forceinline__ void load(const float4* obj, uint32_t id, V3<float>& p0, V3<float>& a, float& L,
                                                float& r) {
        float4 A = __ldg(obj + 2 * (size_t)id);
        float4 B = __ldg(obj + 2 * (size_t)id + 1);
        p0 = v3(A.x, A.y, A.z);
        r = A.w;
        a = v3(B.x, B.y, B.z);
        L = B.w;
    }
    static __device__ __forceinline__ const float4* base(const SceneDev& s) { return s.obj; }
};

template <>
struct Obj<double> {
    static __device__ __forceinline__ void load(const double2* obj, uint32_t id, V3<double>& p0, V3<double>& a,
                                                double& L, double& r) {
        const double2* q = obj + 4 * (size_t)id;
        double2 q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2), q3 = __ldg(q + 3);
        p0 = v3(q0.x, q0.y, q1.x);
        r = q1.y;
        a = v3(q2.x, q2.y, q3.x);
        L = q3.y;
    }
    static __device__ __forceinline__ const double2* base(const SceneDev& s) { return s.obj64; }
};

template <class R>
using ObjPtr = typename std::conditional<std::is_same<R, float>::value, const float4*, const double2*>::type;

// One branch-free test for both primitives. An open cylinder of radius r about
// p0 + s a, 0 <= s <= L (|a| = 1): in the plane perpendicular to a the ray is
// w_p + t d_p (w = o - p0); the closest approach is at t_c = -(w_p.d_p)/|d_p|^2
// with squared distance h^2, the roots are t_c -/+ sqrt((r^2 - h^2)/|d_p|^2),
// and a root counts when its axial coordinate s = (w + t d).a is in [0, L].
// With a = 0 and L = 0 the same arithmetic is the ray-sphere test about
// p0: d_p = d, w_p = o - p0, t_c = -(o - p0).d, h = distance of the line to
// p0, and s = 0 for both roots. Nearest root in (tmin, tmax].
template <class R>
__device__ __forceinline__ bool hit_prim(V3<R> o, V3<R> d, V3<R> p0, V3<R> a, R L, R r, R tmin, R tmax, R& t) {
    V3<R> w = o - p0;
    R wa = dot(w, a), da = dot(d, a);
    V3<R> wp = madd(w, -wa, a);
    V3<R> dp = madd(d, -da, a);
    R A = dot(dp, dp);
    R inv = rcp_(A);
    R tc = -dot(wp, dp) * inv;
    V3<R> m = madd(wp, tc, dp);
    R disc = r * r - dot(m, m);
    R half = sqrt_pos(disc * inv);
    R t0 = tc - half, t1 = tc + half;
    R s0 = wa + t0 * da, s1 = wa + t1 * da;
    bool ok = disc >= R(0) && A > Num<R>::parallel_eps();
    bool h0 = ok && t0 > tmin && t0 <= tmax && s0 >= R(0) && s0 <= L;
    bool h1 = ok && t1 > tmin && t1 <= tmax && s1 >= R(0) && s1 <= L;
    t = h0 ? t0 : t1;
    return h0 || h1;
}

template <class R>
__device__ __forceinline__ bool hit_object(ObjPtr<R> obj, uint32_t id, V3<R> o, V3<R> d, R tmin, R tmax, R& t) {
    V3<R> p0, a;
    R L, r;
    Obj<R>::load(obj, id, p0, a, L, r);
    return hit_prim(o, d, p0, a, L, r, tmin, tmax, t);
}

template <class R>
__device__ __forceinline__ bool hit_object(const SceneDev& s, uint32_t id, V3<R> o, V3<R> d, R tmin, R tmax, R& t) {
    return hit_object<R>(Obj<R>::base(s), id, o, d, tmin, tmax, t);
}

// Whether the same primitive has a root in (0, tmax], without the root itself
// (shadow and AO rays). The FP64 path multiplies the root conditions through
// by A = |d_p|^2 > 0: the roots are t = (-B -/+ sqrt(D)) / A with B = w_p.d_p
// and D = B^2 - A (|w_p|^2 - r^2) (= A times hit_prim's disc), so A t and
// A s = A (w.a) + (A t)(d.a) are tested against (0, A tmax] and [0, A L],
// which leaves one square root and no division (FP64 division and square
// root are instruction sequences on the FP64 pipe). The FP32 path keeps
// hit_prim, whose reciprocal and square root are single instructions.
template <class R>
__device__ __forceinline__ bool any_hit_prim(V3<R> o, V3<R> d, V3<R> p0, V3<R> a, R L, R r, R tmax) {
    R t;
    return hit_prim(o, d, p0, a, L, r, R(0), tmax, t);
}

template <>
__device__ __forceinline__ bool any_hit_prim<double>(V3<double> o, V3<double> d, V3<double> p0, V3<double> a,
                                                     double L, double r, double tmax) {
    const V3<double> w = o - p0;
    const double wa = dot(w, a), da = dot(d, a);
    const V3<double> wp = madd(w, -wa, a), dp = madd(d, -da, a);
    const double A = dot(dp, dp), B = dot(wp, dp);
    const double D = fma(B, B, -A * fma(-r, r, dot(wp, wp)));
    const double sq = sqrt(fmax(D, 0.0));
    const double n0 = -B - sq, n1 = -B + sq;  // A t at the two roots
    const double tA = tmax * A, LA = L * A, waA = wa * A;
    const double s0 = fma(n0, da, waA), s1 = fma(n1, da, waA);  // A s at the two roots
    const bool ok = D >= 0.0 && A > Num<double>::parallel_eps();
    const bool h0 = n0 > 0.0 && n0 <= tA && s0 >= 0.0 && s0 <= LA;
    const bool h1 = n1 > 0.0 && n1 <= tA && s1 >= 0.0 && s1 <= LA;
    return ok && (h0 || h1);
}

template <class R>
__device__ __forceinline__ bool any_hit_object(ObjPtr<R> obj, uint32_t id, V3<R> o, V3<R> d, R tmax) {
    V3<R> p0, a;
    R L, r;
    Obj<R>::load(obj, id, p0, a, L, r);
    return any_hit_prim<R>(o, d, p0, a, L, r, tmax);
}

// ---------------------------------------------------------------- grid walk

template <class R>
struct GridP;

template <>
struct GridP<float> {
    static __device__ __forceinline__ float bs(const GridDev& g, int k) { return g.bs[k]; }
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ float lo(const GridDev& g, int k) { return g.lo[k]; }
    static __device__ __forceinline__ float hi(const GridDev& g, int k) { return g.hi[k]; }
    static __device__ __forceinline__ float h(const GridDev& g, int k) { return g.h[k]; }
    static __device__ __forceinline__ float inv_h(const GridDev& g, int k) { return g.inv_h[k]; }
};

template <>
struct GridP<double> {
    static __device__ __forceinline__ double bs(const GridDev& g, int k) { return g.bs64[k]; }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double lo(const GridDev& g, int k) { return g.lo64[k]; }
    static __device__ __forceinline__ double hi(const GridDev& g, int k) { return g.hi64[k]; }
    static __device__ __forceinline__ double h(const GridDev& g, int k) { return g.h64[k]; }
    static __device__ __forceinline__ double inv_h(const GridDev& g, int k) { return g.inv_h64[k]; }
};

// Clip o + t d, t in [tmin, tmax], to the grid box and to the bounding sphere
// of the objects (nothing can be hit outside either). inv = 1/d per axis
// (unused where d is 0).
template <class R>
__device__ __forceinline__ bool clip_grid(const GridDev& g, V3<R> o, V3<R> d, V3<R> inv, R tmin, R tmax, R& t0,
                                          R& t1) {
    R a = tmin, b = tmax;
    const R oo[3] = {o.x, o.y, o.z};
    const R dd[3] = {d.x, d.y, d.z};
    const R ii[3] = {inv.x, inv.y, inv.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R lo = GridP<R>::lo(g, k), hi = GridP<R>::hi(g, k);
        if (dd[k] == R(0)) {
            if (oo[k] < lo || oo[k] > hi) return false;
        } else {
            R ta = (lo - oo[k]) * ii[k], tb = (hi - oo[k]) * ii[k];
            R mn = ta < tb ? ta : tb, mx = ta < tb ? tb : ta;
            a = mn > a ? mn : a;
            b = mx < b ? mx : b;
        }
    }
    // bounding sphere: |o + t d - c| <= rb (|d| = 1)
    V3<R> f = v3(o.x - GridP<R>::bs(g, 0), o.y - GridP<R>::bs(g, 1), o.z - GridP<R>::bs(g, 2));
    R bb = dot(f, d);
    V3<R> v = madd(f, -bb, d);
    R rb = GridP<R>::bs(g, 3);
    R disc = rb * rb - dot(v, v);
    if (disc < R(0)) return false;
    R sq = Num<R>::sqrt_(disc);
    a = (-bb - sq) > a ? (-bb - sq) : a;
    b = (-bb + sq) < b ? (-bb + sq) : b;
    t0 = a;
    t1 = b;
    return a <= b;
}

template <class R>
__device__ __forceinline__ V3<R> inv_dir(V3<R> d) {
    return v3(GridP<R>::rcp(d.x), GridP<R>::rcp(d.y), GridP<R>::rcp(d.z));
}

template <class R>
__device__ __forceinline__ bool clip_grid(const GridDev& g, V3<R> o, V3<R> d, R tmin, R tmax, R& t0, R& t1) {
    return clip_grid(g, o, d, inv_dir(d), tmin, tmax, t0, t1);
}

// Amanatides & Woo (1987) traversal state: the current cell's index, per
// axis the index change of one step, the t of the next boundary crossing and
// the t between crossings; the end of the clipped interval and the number of
// cells (the walk's bounds); `left` counts down the steps (or, in the AO walk,
// the lockstep iterations) a walk may take: nx + ny + nz + 3.
template <class R>
struct Walk {
    int stx, sty, stz;
    R tnx, tny, tnz;
    R tdx, tdy, tdz;
    R t1;
    int cell;
    int left;
    unsigned ncells;
};

// One axis of the walk's set-up (selects, not branches: lanes differ in the
// signs of their directions). Moving up the axis the next boundary is the
// cell's upper face, moving down its lower face; a zero component never steps.
template <class R>
__device__ __forceinline__ void axis_setup(const GridDev& g, int k, R o, R d, R inv, int c, int stride, int& st,
                                           R& tn, R& td) {
    const bool up = d > R(0), down = d < R(0);
    const R h = GridP<R>::h(g, k);
    st = up ? stride : (down ? -stride : 0);
    const R face = GridP<R>::lo(g, k) + R(up ? c + 1 : c) * h;
    tn = (up || down) ? (face - o) * inv : Num<R>::inf();
    td = (up || down) ? (up ? h : -h) * inv : Num<R>::inf();
}

template <class R>
__device__ __forceinline__ int cell_of(const GridDev& g, int k, R x) {
    R f = floor((x - GridP<R>::lo(g, k)) * GridP<R>::inv_h(g, k));
    int c = (int)f;
    c = c < 0 ? 0 : c;
    return c > g.n[k] - 1 ? g.n[k] - 1 : c;
}

template <class R>
__device__ __forceinline__ bool walk_start(const GridDev& g, V3<R> o, V3<R> d, R tmin, R tmax, Walk<R>& w) {
    R t0, t1;
    const V3<R> inv = inv_dir(d);
    if (g.empty || !clip_grid(g, o, d, inv, tmin, tmax, t0, t1)) return false;
    V3<R> p = madd(o, t0, d);
    const int cx = cell_of(g, 0, p.x), cy = cell_of(g, 1, p.y), cz = cell_of(g, 2, p.z);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    axis_setup(g, 0, o.x, d.x, inv.x, cx, 1, w.stx, w.tnx, w.tdx);
    axis_setup(g, 1, o.y, d.y, inv.y, cy, nx, w.sty, w.tny, w.tdy);
    axis_setup(g, 2, o.z, d.z, inv.z, cz, nx * ny, w.stz, w.tnz, w.tdz);
    w.ncells = (unsigned)g.ncells;
    w.t1 = t1;
    w.cell = (cz * ny + cy) * nx + cx;
    w.left = nx + ny + nz + 3;
    return true;
}

template <class R>
__device__ __forceinline__ R walk_cell_exit(const Walk<R>& w) {
    R m = w.tnx < w.tny ? w.tnx : w.tny;
    return m < w.tnz ? m : w.tnz;
}

// Step to the next cell (ties: x, then y, then z). False when the walk leaves
// the clipped interval or the grid's index range. Written with selects rather
// than a branch per axis: the lanes of a warp step along different axes.
//
// The clipped interval ends inside the grid, so in exact arithmetic no step
// leaves it. Rounding in the accumulated crossings can carry the last one or
// few steps just past the grid's edge, into a cell of another row or out of
// the index range; the range check ends the walk, and the cells of another row
// cost tests but change no result: every object the ray meets has its hit
// point inside the grid, in a cell the walk visits before, and a test of any
// other object finds only true intersections.
template <class R>
__device__ __forceinline__ bool walk_step(Walk<R>& w) {
    const bool bx = w.tnx <= w.tny && w.tnx <= w.tnz;
    const bool by = !bx && w.tny <= w.tnz;
    const bool bz = !bx && !by;
    const R tn = bx ? w.tnx : (by ? w.tny : w.tnz);
    if (tn > w.t1) return false;
    w.tnx = bx ? w.tnx + w.tdx : w.tnx;
    w.tny = by ? w.tny + w.tdy : w.tny;
    w.tnz = bz ? w.tnz + w.tdz : w.tnz;
    w.cell += bx ? w.stx : (by ? w.sty : w.stz);
    return (unsigned)w.cell < w.ncells;
}

// walk_step within the walk's step bound: past it (only a walk whose crossing
// times are not numbers can get there) the walk ends and *overflow is set.
template <class R>
__device__ __forceinline__ bool walk_next(Walk<R>& w, bool& overflow) {
    if (--w.left <= 0) {
        overflow = true;
        return false;
    }
    return walk_step(w);
}

// ---------------------------------------------------------------- traversal

template <class R>
struct Nearest {
    R t1, t2;
    uint32_t id1, id2;
};

template <class R>
__device__ __forceinline__ void nearest_consider(Nearest<R>& h, uint32_t id, R t) {
    if (id == h.id1) return;  // the same object listed in another cell
    if (t < h.t1 || (t == h.t1 && id < h.id1)) {
        h.t2 = h.t1;
        h.id2 = h.id1;
        h.t1 = t;
        h.id1 = id;
    } else if (id != h.id2 && (t < h.t2 || (t == h.t2 && id < h.id2))) {
        h.t2 = t;
        h.id2 = id;
    }
}

// Nearest hit in (tmin, tmax]: walk cells in ray order and stop after the
// first cell whose exit t is at or beyond the best hit (every object whose hit
// point lies in a visited cell is listed there).
template <class R>
__device__ bool trace_nearest(const GridDev& g, const SceneDev& s, V3<R> o, V3<R> d, R tmin, R tmax, Nearest<R>& h,
                              bool& overflow) {
    h.t1 = h.t2 = Num<R>::inf();
    h.id1 = h.id2 = GBRT_MISS;
    Walk<R> w;
    if (!walk_start(g, o, d, tmin, tmax, w)) return false;
    do {
        uint2 cr = __ldg(g.cells + GBRT_INDEX(w.cell, g.ncells));
        for (uint32_t k = cr.x, e = cr.x + cr.y; k < e; ++k) {
            uint32_t id = GBRT_INDEX(__ldg(g.items + GBRT_INDEX(k, g.nitems)), s.S + s.C);
            R t;
            if (hit_object(s, id, o, d, tmin, tmax, t)) nearest_consider(h, id, t);
        }
        if (h.id1 != GBRT_MISS && h.t1 <= walk_cell_exit(w)) break;
    } while (walk_next(w, overflow));
    return h.id1 != GBRT_MISS;
}

// Any hit with 0 < t <= tmax (AO shadow ray): the first hit ends the walk.
template <class R>
__device__ bool trace_any(const GridDev& g, const SceneDev& s, V3<R> o, V3<R> d, R tmax, bool& overflow) {
    Walk<R> w;
    if (!walk_start(g, o, d, R(0), tmax, w)) return false;
    do {
        uint2 cr = __ldg(g.cells + GBRT_INDEX(w.cell, g.ncells));
        for (uint32_t k = cr.x, e = cr.x + cr.y; k < e; ++k) {
            uint32_t id = GBRT_INDEX(__ldg(g.items + GBRT_INDEX(k, g.nitems)), s.S + s.C);
            if (any_hit_object<R>(Obj<R>::base(s), id, o, d, tmax)) return true;
        }
    } while (walk_next(w, overflow));
    return false;
}

// ---------------------------------------------------------------- sampling

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw; SC'11): 10 rounds of two 32x32
// multiplies with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Two AO uniforms of sample s of point/pixel q: counter (q, s, frame, 0xA0),
// key (seed_lo, seed_hi); the top 24 bits of words 0 and 1 times 2^-24.
__device__ __forceinline__ void ao_uniforms(uint32_t q, uint32_t s, uint32_t frame, uint32_t seed_lo,
                                            uint32_t seed_hi, uint32_t& b1, uint32_t& b2) {
    uint4 x = philox4x32_10(make_uint4(q, s, frame, 0xA0u), make_uint2(seed_lo, seed_hi));
    b1 = x.x >> 8;
    b2 = x.y >> 8;
}

template <class R>
__device__ __forceinline__ void sincos_2pi(R u, R& s, R& c);
template <>
__device__ __forceinline__ void sincos_2pi<float>(float u, float& s, float& c) { sincospif(2.0f * u, &s, &c); }
template <>
__device__ __forceinline__ void sincos_2pi<double>(double u, double& s, double& c) { sincospi(2.0 * u, &s, &c); }

// Cosine-weighted direction about n (Malley: a uniform disk point r = sqrt(u1),
// phi = 2 pi u2 lifted to z = sqrt(1 - u1)), in the basis of Duff et al. 2017.
template <class R>
__device__ __forceinline__ V3<R> cosine_dir(V3<R> n, uint32_t b1, uint32_t b2) {
    const R scale = R(1) / R(16777216);
    R u1 = R(b1) * scale, u2 = R(b2) * scale;
    R sign = copysign(R(1), n.z);
    R a = R(-1) / (sign + n.z);
    R b = n.x * n.y * a;
    V3<R> e1 = v3(R(1) + sign * n.x * n.x * a, sign * b, -sign * n.x);
    V3<R> e2 = v3(b, sign + n.y * n.y * a, -n.y);
    R r = sqrt_pos(u1);
    R sp, cp;
    sincos_2pi<R>(u2, sp, cp);
    R x = r * cp, y = r * sp, z = sqrt_pos(R(1) - u1);
    return v3(x * e1.x + y * e2.x + z * n.x, x * e1.y + y * e2.y + z * n.y, x * e1.z + y * e2.z + z * n.z);
}

// Number of AO samples of (index q) that escape, from origin o about normal n.
template <class R>
__device__ __forceinline__ int ao_visible(const FrameDev& f, uint32_t q, V3<R> o, V3<R> n, R maxdist, bool& overflow) {
    int vis = 0;
    for (int s = 0; s < f.spp; ++s) {
        uint32_t b1, b2;
        ao_uniforms(q, (uint32_t)s, f.frame, f.seed_lo, f.seed_hi, b1, b2);
        V3<R> d = cosine_dir(n, b1, b2);
        if (!trace_any(f.grid, f.scene, o, d, maxdist, overflow)) ++vis;
    }
    return vis;
}

// ---------------------------------------------------------------- refinement

// FP64 hit point re-projected onto the surface of object id, and the geometric
// normal turned to face the incoming ray.
__device__ __forceinline__ bool reproject64(const SceneDev& s, uint32_t id, V3<double> o, V3<double> d, double t,
                                            V3<double>& p, V3<double>& n) {
    V3<double> p0, a;
    double L, r;
    Obj<double>::load(s.obj64, id, p0, a, L, r);
    p = madd(o, t, d);
    // closest point of the generator (centre, or axis point) to the hit point
    double sa = dot(p - p0, a);
    V3<double> q = madd(p0, sa, a);
    V3<double> v = p - q;
    n = (1.0 / sqrt(dot(v, v))) * v;
    p = madd(q, r, n);
    // true when the ray met the surface from inside (the normal is turned)
    if (dot(n, d) > 0.0) {
        n = v3(-n.x, -n.y, -n.z);
        return true;
    }
    return false;
}

// ---------------------------------------------------------------- shading

template <class R>
struct ShadeP;

template <>
struct ShadeP<float> {
    static __device__ __forceinline__ V3<float> ldir(const FrameDev& f, int l) {
        return v3(f.ldir_f[l][0], f.ldir_f[l][1], f.ldir_f[l][2]);
    }
    static __device__ __forceinline__ float lI(const FrameDev& f, int l) { return f.lI_f[l]; }
    static __device__ __forceinline__ float sky_kao(const FrameDev& f) { return f.sky_kao_f; }
    static __device__ __forceinline__ float k_d(const FrameDev& f) { return f.k_d_f; }
    static __device__ __forceinline__ float k_s(const FrameDev& f) { return f.k_s_f; }
    static __device__ __forceinline__ float phong(const FrameDev& f) { return f.phong_f; }
    static __device__ __forceinline__ float pow_(float x, float e) { return powf(x, e); }
};

template <>
struct ShadeP<double> {
    static __device__ __forceinline__ V3<double> ldir(const FrameDev& f, int l) { return ld3(f.ldir[l]); }
    static __device__ __forceinline__ double lI(const FrameDev& f, int l) { return f.lI[l]; }
    static __device__ __forceinline__ double sky_kao(const FrameDev& f) { return f.sky_kao; }
    static __device__ __forceinline__ double k_d(const FrameDev& f) { return f.k_d; }
    static __device__ __forceinline__ double k_s(const FrameDev& f) { return f.k_s; }
    static __device__ __forceinline__ double phong(const FrameDev& f) { return f.phong; }
    static __device__ __forceinline__ double pow_(double x, double e) { return pow(x, e); }
};

// colour = clamp01(albedo (skylight k_ao V + sum_l s I_l k_d max(0, n.l))
//                  + sum_{n.l > 0} s I_l k_s max(0, r_l.v)^p), r_l = 2 (n.l) n - l
// lit: bit l clear drops light l (its shadow ray was blocked).
template <class R>
__device__ __forceinline__ void shade(const FrameDev& f, uint32_t id, V3<R> n, V3<R> d, R V, uint32_t lit, R rgb[3]) {
    R diff = R(0), spec = R(0);
    V3<R> v = v3(-d.x, -d.y, -d.z);
    for (int l = 0; l < f.nl; ++l) {
        V3<R> L = ShadeP<R>::ldir(f, l);
        R ndl = dot(n, L);
        if (ndl <= R(0) || !((lit >> l) & 1u)) continue;
        R I = ShadeP<R>::lI(f, l);
        diff += I * ShadeP<R>::k_d(f) * ndl;
        V3<R> r = madd(v3(-L.x, -L.y, -L.z), R(2) * ndl, n);
        R rv = dot(r, v);
        if (rv > R(0)) spec += I * ShadeP<R>::k_s(f) * ShadeP<R>::pow_(rv, ShadeP<R>::phong(f));
    }
    uint32_t ci = __ldg(f.scene.color + id);
    R amb = ShadeP<R>::sky_kao(f) * V + diff;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R c = R(__ldg(f.scene.palette + 3 * ci + k)) * amb + spec;
        rgb[k] = c < R(0) ? R(0) : (c > R(1) ? R(1) : c);
    }
}

}  // namespace gbrt
