/*
 * oracle.c -- plain FP64 CPU oracle of the molecular ambient-occlusion ray
 * tracer (primary rays, AO shadow rays, Phong + skylight shading).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or helper with the CUDA library: both read the same seeded input
 * arrays and parameter values, nothing else.
 *
 * What it computes, and where each step comes from:
 *  - The paper (Sec. 2) renders with a Tachyon build whose arithmetic is all
 *    double precision, at -res W H, with ambient occlusion computed by random
 *    sampling of the incoming light, -rescale_lights 0.3 and -add_skylight 1.0.
 *    Everything here is in double precision with libm.
 *  - The paper does not spell out the tracer's algorithms. The readings used
 *    (camera, materials, epsilon, sampling map) come in as parameters; this
 *    file implements:
 *      * nearest hit = the smallest t over ALL objects (brute force is the
 *        definition); equal t -> smaller global id (spheres 0..S-1, then
 *        cylinders S..S+C-1);
 *      * a uniform grid + 3D-DDA (Amanatides & Woo, Eurographics 1987) as an
 *        accelerated mode, which must return the same hits;
 *      * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by seed,
 *        counter (pixel, sample, frame, 0xA0);
 *      * cosine-weighted hemisphere sampling (Malley's method: uniform disk
 *        lifted to the hemisphere) in the orthonormal basis of Duff et al.,
 *        JCGT 6(1), 2017;
 *      * Phong shading with an AO-weighted skylight term.
 *
 * Parity pins live in the test suite: closed-form ray-sphere/ray-cylinder
 * hits, a bisection root of each implicit surface, the analytic AO of a sphere
 * resting on a plane and of a point facing a sphere, AO = 1 for a lone convex
 * object, brute force == grid on tiny scenes, Philox known-answer vectors,
 * sampling moments and hand-derived shading values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MISS 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3.2 / Table 2 constants)         */
/* ------------------------------------------------------------------------ */

static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The two AO uniforms of (index, sample): 24-bit fractions of words 0 and 1. */
void oracle_ao_uniforms(uint32_t index, uint32_t sample, uint32_t frame, uint64_t seed,
                        double* u1, double* u2)
{
    uint32_t ctr[4] = {index, sample, frame, 0xA0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    oracle_philox4x32_10(ctr, key, x);
    *u1 = (double)(x[0] >> 8) * (1.0 / 16777216.0);
    *u2 = (double)(x[1] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* Orthonormal basis (Duff et al. 2017, Listing 3 reading) and cosine sample  */
/* ------------------------------------------------------------------------ */

void oracle_onb(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a;
    b1[1] = sign * b;
    b1[2] = -sign * n[0];
    b2[0] = b;
    b2[1] = sign + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/* Malley's method: a uniform point (r, phi) of the unit disk, r = sqrt(u1),
 * phi = 2 pi u2, lifted to z = sqrt(1 - r^2) gives density cos(theta)/pi. */
void oracle_cosine_dir(const double n[3], double u1, double u2, double d[3])
{
    double b1[3], b2[3];
    oracle_onb(n, b1, b2);
    double r = sqrt(u1);
    double phi = 2.0 * M_PI * u2;
    double x = r * cos(phi), y = r * sin(phi), z = sqrt(1.0 - u1);
    for (int k = 0; k < 3; ++k) d[k] = x * b1[k] + y * b2[k] + z * n[k];
}

/* ------------------------------------------------------------------------ */
/* Vector helpers                                                            */
/* ------------------------------------------------------------------------ */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void normalize3(double v[3])
{
    double l = sqrt(dot3(v, v));
    if (l > 0) { v[0] /= l; v[1] /= l; v[2] /= l; }
}

/* ------------------------------------------------------------------------ */
/* Ray-object intersection. Each returns the nearest root t with             */
/* tmin < t <= tmax (1 = hit, 0 = miss) plus a grazing record:               */
/*   disc_rel : (r^2 - h^2)/r^2, h = closest distance of ray to the surface's */
/*              generator (sphere centre / cylinder axis); < 0 means miss.   */
/*   t_close  : ray parameter of that closest approach.                      */
/*   t_near   : where a flip of the silhouette decision acts: the nearer     */
/*              root when the ray meets the surface (disc >= 0), else t_close */
/*   s_out    : cylinders only, how far the closest approach lies outside the */
/*              segment along the axis (0 within it; 0 for spheres)          */
/*   end_mrg[k], t_end[k] : cylinders only, for root k (0 near, 1 far) in   */
/*              (tmin, tmax]: the axial distance of its point to the nearer  */
/*              clip plane (scene units) and its t; +inf otherwise.          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double disc_rel, t_close, t_near, s_out, end_mrg[2], t_end[2];
} graze_t;

/* Sphere |p - c| = r, ray p = o + t d with |d| = 1. With f = o - c and
 * b = f.d the closest approach vector is f - b d, of squared length h^2; the
 * roots are t = -b -/+ sqrt(r^2 - h^2) (Haines et al., Ray Tracing Gems ch. 7:
 * the discriminant taken from the perpendicular vector, not from |f|^2 - b^2). */
int oracle_hit_sphere(const double o[3], const double d[3], const double c[3], double r,
                      double tmin, double tmax, double* t_out, graze_t* g)
{
    double f[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    double b = dot3(f, d);
    double v[3] = {f[0] - b * d[0], f[1] - b * d[1], f[2] - b * d[2]};
    double h2 = dot3(v, v);
    double disc = r * r - h2;
    if (g) {
        g->disc_rel = disc / (r * r);
        g->t_close = -b;
        g->t_near = -b;
        g->s_out = 0.0;
        g->end_mrg[0] = g->end_mrg[1] = INFINITY;
        g->t_end[0] = g->t_end[1] = INFINITY;
    }
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double t0 = -b - sq, t1 = -b + sq;
    if (g) g->t_near = t0;
    if (t0 > tmin && t0 <= tmax) { *t_out = t0; return 1; }
    if (t1 > tmin && t1 <= tmax) { *t_out = t1; return 1; }
    return 0;
}

/* Open (uncapped) finite cylinder: points at distance r from the segment axis
 * p0 + s a (|a| = 1, 0 <= s <= L). With w = o - p0 and the components of w and
 * d perpendicular to a (w_p, d_p), the wall is |w_p + t d_p| = r. The closest
 * approach in the perpendicular plane is at t_c = -(w_p.d_p)/(d_p.d_p), at
 * squared distance h^2, and the roots are t_c -/+ sqrt((r^2 - h^2)/(d_p.d_p)).
 * A root counts when its axial coordinate s = (w + t d).a is in [0, L]. */
int oracle_hit_cylinder(const double o[3], const double d[3], const double p0[3], const double p1[3],
                        double r, double tmin, double tmax, double* t_out, graze_t* g)
{
    double ax[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double L = sqrt(dot3(ax, ax));
    if (g) {
        g->disc_rel = -INFINITY; g->t_close = 0.0; g->t_near = 0.0; g->s_out = INFINITY;
        g->end_mrg[0] = g->end_mrg[1] = INFINITY;
        g->t_end[0] = g->t_end[1] = INFINITY;
    }
    if (!(L > 0.0)) return 0;
    double a[3] = {ax[0] / L, ax[1] / L, ax[2] / L};
    double w[3] = {o[0] - p0[0], o[1] - p0[1], o[2] - p0[2]};
    double wa = dot3(w, a), da = dot3(d, a);
    double wp[3] = {w[0] - wa * a[0], w[1] - wa * a[1], w[2] - wa * a[2]};
    double dp[3] = {d[0] - da * a[0], d[1] - da * a[1], d[2] - da * a[2]};
    double A = dot3(dp, dp);
    if (!(A > 1e-24)) return 0; /* parallel to the axis: an open tube is never crossed */
    double tc = -dot3(wp, dp) / A;
    double m[3] = {wp[0] + tc * dp[0], wp[1] + tc * dp[1], wp[2] + tc * dp[2]};
    double h2 = dot3(m, m);
    double disc = r * r - h2;
    if (g) {
        double sc = wa + tc * da;
        g->disc_rel = disc / (r * r);
        g->t_close = tc;
        g->t_near = tc;
        g->s_out = fmax(0.0, fmax(-sc, sc - L));
    }
    if (disc < 0.0) return 0;
    double half = sqrt(disc / A);
    double roots[2] = {tc - half, tc + half};
    if (g) g->t_near = roots[0];
    int hit = 0;
    for (int k = 0; k < 2; ++k) {
        double t = roots[k];
        if (!(t > tmin && t <= tmax)) continue;
        double s = wa + t * da;
        if (g) { g->end_mrg[k] = fmin(fabs(s), fabs(L - s)); g->t_end[k] = t; }
        if (!hit && s >= 0.0 && s <= L) { *t_out = t; hit = 1; }
    }
    return hit;
}

/* ------------------------------------------------------------------------ */
/* Scene (double copies of the float input arrays)                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t S, C;
    const double* sph; /* S x 4 : cx cy cz r */
    const double* cyl; /* C x 7 : p0 p1 r */
    const uint32_t* color;
    const double* palette;
    int32_t K;
} oscene;

static void object_aabb(const oscene* sc, int64_t id, double lo[3], double hi[3])
{
    if (id < sc->S) {
        const double* s = sc->sph + 4 * id;
        for (int k = 0; k < 3; ++k) { lo[k] = s[k] - s[3]; hi[k] = s[k] + s[3]; }
    } else {
        const double* c = sc->cyl + 7 * (id - sc->S);
        double ax[3] = {c[3] - c[0], c[4] - c[1], c[5] - c[2]};
        double L = sqrt(dot3(ax, ax));
        for (int k = 0; k < 3; ++k) {
            double ak = L > 0 ? ax[k] / L : 0.0;
            double e = c[6] * sqrt(fmax(0.0, 1.0 - ak * ak));
            lo[k] = fmin(c[k], c[3 + k]) - e;
            hi[k] = fmax(c[k], c[3 + k]) + e;
        }
    }
}

/* Test one object; returns 1 on a hit in (tmin, tmax]. */
static int hit_object(const oscene* sc, int64_t id, const double o[3], const double d[3],
                      double tmin, double tmax, double* t, graze_t* g)
{
    if (id < sc->S) {
        const double* s = sc->sph + 4 * id;
        return oracle_hit_sphere(o, d, s, s[3], tmin, tmax, t, g);
    }
    const double* c = sc->cyl + 7 * (id - sc->S);
    return oracle_hit_cylinder(o, d, c, c + 3, c[6], tmin, tmax, t, g);
}

/* ------------------------------------------------------------------------ */
/* Uniform grid (the acceleration structure of the method)                   */
/*  - object box: sphere c -/+ r; cylinder per axis min/max of the end        */
/*    points -/+ r sqrt(1 - a_k^2); all boxes padded by pad;                   */
/*  - scene box: union of object boxes, padded by pad = 1e-5 max(extent, 1);  */
/*  - cells: n_k = clamp(round(E_k cbrt(lambda N / V)), 1, 1024), with the   */
/*    product capped through lambda N <= 2^26;                                */
/*  - an object is listed in every cell its padded box overlaps, in id order. */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lo[3], hi[3], h[3];
    int n[3];
    int64_t ncells;
    int64_t* start; /* ncells + 1 */
    uint32_t* items;
    int empty;
} ogrid;

static int cell_coord(const ogrid* gr, int k, double x)
{
    double f = floor((x - gr->lo[k]) / gr->h[k]);
    if (f < 0) f = 0;
    if (f > gr->n[k] - 1) f = gr->n[k] - 1;
    return (int)f;
}

static void grid_free(ogrid* gr)
{
    free(gr->start);
    free(gr->items);
    gr->start = NULL;
    gr->items = NULL;
}

static int grid_build(const oscene* sc, double lambda, ogrid* gr)
{
    memset(gr, 0, sizeof(*gr));
    int64_t N = sc->S + sc->C;
    if (N == 0) {
        gr->empty = 1;
        return 0;
    }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t id = 0; id < N; ++id) {
        double a[3], b[3];
        object_aabb(sc, id, a, b);
        for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], a[k]); hi[k] = fmax(hi[k], b[k]); }
    }
    double emax = fmax(hi[0] - lo[0], fmax(hi[1] - lo[1], hi[2] - lo[2]));
    double pad = 1e-5 * fmax(emax, 1.0);
    double E[3], V = 1.0;
    for (int k = 0; k < 3; ++k) {
        gr->lo[k] = lo[k] - pad;
        gr->hi[k] = hi[k] + pad;
        E[k] = gr->hi[k] - gr->lo[k];
        V *= E[k];
    }
    double target = lambda * (double)N;
    if (target > 67108864.0) target = 67108864.0;
    if (target < 1.0) target = 1.0;
    double kk = cbrt(target / V);
    gr->ncells = 1;
    for (int k = 0; k < 3; ++k) {
        double nk = floor(E[k] * kk + 0.5);
        if (nk < 1) nk = 1;
        if (nk > 1024) nk = 1024;
        gr->n[k] = (int)nk;
        gr->h[k] = E[k] / nk;
        gr->ncells *= gr->n[k];
    }
    gr->start = (int64_t*)calloc((size_t)gr->ncells + 1, sizeof(int64_t));
    if (!gr->start) return -1;
    /* count */
    for (int64_t id = 0; id < N; ++id) {
        double a[3], b[3];
        int c0[3], c1[3];
        object_aabb(sc, id, a, b);
        for (int k = 0; k < 3; ++k) { c0[k] = cell_coord(gr, k, a[k] - pad); c1[k] = cell_coord(gr, k, b[k] + pad); }
        for (int z = c0[2]; z <= c1[2]; ++z)
            for (int y = c0[1]; y <= c1[1]; ++y)
                for (int x = c0[0]; x <= c1[0]; ++x)
                    gr->start[((int64_t)z * gr->n[1] + y) * gr->n[0] + x + 1] += 1;
    }
    for (int64_t c = 0; c < gr->ncells; ++c) gr->start[c + 1] += gr->start[c];
    gr->items = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(gr->start[gr->ncells] + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)gr->ncells);
    if (!gr->items || !fill) { free(fill); grid_free(gr); return -1; }
    memcpy(fill, gr->start, sizeof(int64_t) * (size_t)gr->ncells);
    /* fill in id order: every cell's list ends up sorted by id */
    for (int64_t id = 0; id < N; ++id) {
        double a[3], b[3];
        int c0[3], c1[3];
        object_aabb(sc, id, a, b);
        for (int k = 0; k < 3; ++k) { c0[k] = cell_coord(gr, k, a[k] - pad); c1[k] = cell_coord(gr, k, b[k] + pad); }
        for (int z = c0[2]; z <= c1[2]; ++z)
            for (int y = c0[1]; y <= c1[1]; ++y)
                for (int x = c0[0]; x <= c1[0]; ++x) {
                    int64_t c = ((int64_t)z * gr->n[1] + y) * gr->n[0] + x;
                    gr->items[fill[c]++] = (uint32_t)id;
                }
    }
    free(fill);
    return 0;
}

/* Clip the ray to the grid box: [t0, t1] within [tmin, tmax]. Returns 0 when
 * the ray misses the box. */
static int clip_box(const ogrid* gr, const double o[3], const double d[3], double tmin, double tmax,
                    double* t0, double* t1)
{
    double a = tmin, b = tmax;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < gr->lo[k] || o[k] > gr->hi[k]) return 0;
            continue;
        }
        double ta = (gr->lo[k] - o[k]) / d[k];
        double tb = (gr->hi[k] - o[k]) / d[k];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > a) a = ta;
        if (tb < b) b = tb;
    }
    if (a > b) return 0;
    *t0 = a;
    *t1 = b;
    return 1;
}

/* Amanatides-Woo walk state. */
typedef struct {
    int c[3], step[3];
    double tnext[3], tdelta[3];
    double t1;
    int left;
} dda_t;

static int dda_start(const ogrid* gr, const double o[3], const double d[3], double tmin, double tmax,
                     dda_t* w)
{
    double t0, t1;
    if (!clip_box(gr, o, d, tmin, tmax, &t0, &t1)) return 0;
    w->t1 = t1;
    w->left = gr->n[0] + gr->n[1] + gr->n[2] + 3;
    for (int k = 0; k < 3; ++k) {
        double p = o[k] + t0 * d[k];
        w->c[k] = cell_coord(gr, k, p);
        if (d[k] > 0.0) {
            w->step[k] = 1;
            w->tnext[k] = (gr->lo[k] + (w->c[k] + 1) * gr->h[k] - o[k]) / d[k];
            w->tdelta[k] = gr->h[k] / d[k];
        } else if (d[k] < 0.0) {
            w->step[k] = -1;
            w->tnext[k] = (gr->lo[k] + w->c[k] * gr->h[k] - o[k]) / d[k];
            w->tdelta[k] = -gr->h[k] / d[k];
        } else {
            w->step[k] = 0;
            w->tnext[k] = INFINITY;
            w->tdelta[k] = INFINITY;
        }
    }
    return 1;
}

static double dda_cell_exit(const dda_t* w)
{
    return fmin(w->tnext[0], fmin(w->tnext[1], w->tnext[2]));
}

/* Advance to the next cell; returns 0 when the walk leaves the grid or the
 * clipped interval. Ties between axes step x, then y, then z. */
static int dda_next(const ogrid* gr, dda_t* w)
{
    double te = dda_cell_exit(w);
    if (te > w->t1) return 0;
    if (--w->left <= 0) return 0;
    int k = 0;
    if (w->tnext[1] < w->tnext[k]) k = 1;
    if (w->tnext[2] < w->tnext[k]) k = 2;
    w->c[k] += w->step[k];
    if (w->c[k] < 0 || w->c[k] >= gr->n[k]) return 0;
    w->tnext[k] += w->tdelta[k];
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Nearest hit and any hit                                                   */
/* ------------------------------------------------------------------------ */

#define GRAZE_DISC 1e-4   /* |disc_rel| below this: the ray grazes a silhouette */
#define GRAZE_TIE 1e-5    /* (t2 - t1)/t1 below this: two objects nearly tie */
#define GRAZE_END 1e-4    /* axial margin to a cylinder clip plane, x (L + 1) */

typedef struct {
    int64_t cells, sph, cyl;
} ocount;

typedef struct {
    double t1, t2;      /* nearest and second-nearest distinct hits */
    uint32_t id1, id2;
    double t_graze;     /* smallest t of a grazing encounter */
    uint32_t id_graze;  /* the object of that encounter */
} nearest_t;

static void nearest_reset(nearest_t* nr)
{
    nr->t1 = nr->t2 = INFINITY;
    nr->id1 = nr->id2 = OR_MISS;
    nr->t_graze = INFINITY;
    nr->id_graze = OR_MISS;
}

static void consider(const oscene* sc, int64_t id, const double o[3], const double d[3],
                     double tmin, double tmax, nearest_t* nr, ocount* cnt)
{
    double t;
    graze_t g;
    if (id < sc->S) cnt->sph++; else cnt->cyl++;
    int hit = hit_object(sc, id, o, d, tmin, tmax, &t, &g);
    double L = 0.0; /* a tube's length (clip-plane margin GRAZE_END (L + 1)) */
    if (id >= sc->S) {
        const double* c = sc->cyl + 7 * (id - sc->S);
        double ax[3] = {c[3] - c[0], c[4] - c[1], c[5] - c[2]};
        L = sqrt(dot3(ax, ax));
    }
    /* a silhouette decision within rounding of flipping, in front of the origin
     * (for a tube: with the closest approach within the clip margin of the
     * segment; elsewhere no root can count): it acts at the nearer root (at
     * the closest approach when the ray misses) */
    if (fabs(g.disc_rel) < GRAZE_DISC && g.t_close > tmin && g.s_out <= GRAZE_END * (L + 1.0) &&
        g.t_near < nr->t_graze) {
        nr->t_graze = g.t_near;
        nr->id_graze = (uint32_t)id;
    }
    if (id >= sc->S) {
        for (int k = 0; k < 2; ++k) {
            if (g.end_mrg[k] < GRAZE_END * (L + 1.0) && g.t_end[k] < nr->t_graze) {
                nr->t_graze = g.t_end[k];
                nr->id_graze = (uint32_t)id;
            }
        }
    }
    if (!hit) return;
    uint32_t uid = (uint32_t)id;
    if (uid == nr->id1) return; /* same object seen again from another cell */
    if (t < nr->t1 || (t == nr->t1 && uid < nr->id1)) {
        if (nr->id1 != OR_MISS) { nr->t2 = nr->t1; nr->id2 = nr->id1; }
        nr->t1 = t;
        nr->id1 = uid;
    } else if (uid != nr->id2 && (t < nr->t2 || (t == nr->t2 && uid < nr->id2))) {
        nr->t2 = t;
        nr->id2 = uid;
    }
}

static void nearest_brute(const oscene* sc, const double o[3], const double d[3], double tmin, double tmax,
                          nearest_t* nr, ocount* cnt)
{
    int64_t N = sc->S + sc->C;
    for (int64_t id = 0; id < N; ++id) consider(sc, id, o, d, tmin, tmax, nr, cnt);
}

static void nearest_grid(const oscene* sc, const ogrid* gr, const double o[3], const double d[3],
                         double tmin, double tmax, nearest_t* nr, ocount* cnt)
{
    if (gr->empty) return;
    dda_t w;
    if (!dda_start(gr, o, d, tmin, tmax, &w)) return;
    do {
        cnt->cells++;
        int64_t c = ((int64_t)w.c[2] * gr->n[1] + w.c[1]) * gr->n[0] + w.c[0];
        for (int64_t i = gr->start[c]; i < gr->start[c + 1]; ++i)
            consider(sc, gr->items[i], o, d, tmin, tmax, nr, cnt);
        /* every object whose hit point lies in a visited cell has been tested */
        if (nr->id1 != OR_MISS && nr->t1 <= dda_cell_exit(&w)) break;
    } while (dda_next(gr, &w));
    if (nr->id1 == OR_MISS) return;
    /* Not part of the method's work (no counts): the cells entered before
     * t1 (1 + GRAZE_TIE), so that a near-tie or grazing encounter just past
     * the cell of the hit is seen as brute force sees it. */
    ocount extra = {0, 0, 0};
    const double t_lim = nr->t1 * (1.0 + GRAZE_TIE) + 1e-9;
    while (dda_cell_exit(&w) <= t_lim && dda_next(gr, &w)) {
        int64_t c = ((int64_t)w.c[2] * gr->n[1] + w.c[1]) * gr->n[0] + w.c[0];
        for (int64_t i = gr->start[c]; i < gr->start[c + 1]; ++i)
            consider(sc, gr->items[i], o, d, tmin, tmax, nr, &extra);
    }
}

static int anyhit_brute(const oscene* sc, const double o[3], const double d[3], double tmax, ocount* cnt)
{
    int64_t N = sc->S + sc->C;
    double t;
    for (int64_t id = 0; id < N; ++id) {
        if (id < sc->S) cnt->sph++; else cnt->cyl++;
        if (hit_object(sc, id, o, d, 0.0, tmax, &t, NULL)) return 1;
    }
    return 0;
}

static int anyhit_grid(const oscene* sc, const ogrid* gr, const double o[3], const double d[3], double tmax,
                       ocount* cnt)
{
    if (gr->empty) return 0;
    dda_t w;
    double t;
    if (!dda_start(gr, o, d, 0.0, tmax, &w)) return 0;
    do {
        cnt->cells++;
        int64_t c = ((int64_t)w.c[2] * gr->n[1] + w.c[1]) * gr->n[0] + w.c[0];
        for (int64_t i = gr->start[c]; i < gr->start[c + 1]; ++i) {
            uint32_t id = gr->items[i];
            if (id < sc->S) cnt->sph++; else cnt->cyl++;
            if (hit_object(sc, id, o, d, 0.0, tmax, &t, NULL)) return 1;
        }
    } while (dda_next(gr, &w));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Hit refinement: hit point re-projected onto the surface, geometric normal */
/* facing the ray.                                                           */
/* ------------------------------------------------------------------------ */

static void refine(const oscene* sc, uint32_t id, const double o[3], const double d[3], double t,
                   double p[3], double n[3])
{
    for (int k = 0; k < 3; ++k) p[k] = o[k] + t * d[k];
    if (id < sc->S) {
        const double* s = sc->sph + 4 * id;
        double v[3] = {p[0] - s[0], p[1] - s[1], p[2] - s[2]};
        normalize3(v);
        for (int k = 0; k < 3; ++k) { p[k] = s[k] + s[3] * v[k]; n[k] = v[k]; }
    } else {
        const double* c = sc->cyl + 7 * (id - sc->S);
        double a[3] = {c[3] - c[0], c[4] - c[1], c[5] - c[2]};
        normalize3(a);
        double w[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
        double s = dot3(w, a);
        double q[3] = {c[0] + s * a[0], c[1] + s * a[1], c[2] + s * a[2]};
        double v[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
        normalize3(v);
        for (int k = 0; k < 3; ++k) { p[k] = q[k] + c[6] * v[k]; n[k] = v[k]; }
    }
    if (dot3(n, d) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
}

/* ------------------------------------------------------------------------ */
/* Camera                                                                    */
/*  cam[0] kind (0 ortho, 1 pinhole), cam[1..3] eye, [4..6] dir, [7..9] up,  */
/*  [10..12] right, [13] half_w, [14] half_h, [15] m: sub-pixel grid side     */
/*  (supersampling; 0 or 1 = one ray through the pixel centre)                */
/* The ray passes through the image-plane point (x, y) in pixel units,       */
/* x across from the left edge, y down from the top edge.                     */
/* ------------------------------------------------------------------------ */

static void primary_ray(const double* cam, int W, int H, double x, double y, double o[3], double d[3])
{
    double u = cam[13] * (2.0 * x / W - 1.0);
    double v = cam[14] * (1.0 - 2.0 * y / H);
    if (cam[0] == 0.0) {
        for (int k = 0; k < 3; ++k) { o[k] = cam[1 + k] + u * cam[10 + k] + v * cam[7 + k]; d[k] = cam[4 + k]; }
    } else {
        for (int k = 0; k < 3; ++k) { o[k] = cam[1 + k]; d[k] = cam[4 + k] + u * cam[10 + k] + v * cam[7 + k]; }
    }
    normalize3(d);
}

/* ------------------------------------------------------------------------ */
/* Shading: Phong with directional lights scaled by light_scale plus an AO   */
/* skylight term (paper Sec. 2: -rescale_lights, -add_skylight, AO).          */
/*  sp: [0] light_scale [1] skylight [2] k_ao [3] k_d [4] k_s [5] phong_exp  */
/*      [6] eps [7] ao_maxdist [8..10] background rgb [11] shadows (0/1)     */
/* lit[l] = 0 drops light l (its shadow ray was blocked).                     */
/* ------------------------------------------------------------------------ */

static void shade(const double albedo[3], const double n[3], const double d[3], double V,
                  const double* ldir, const double* lI, int nl, const double* sp, const int* lit, double rgb[3])
{
    double diff = 0.0, spec = 0.0;
    double v[3] = {-d[0], -d[1], -d[2]};
    for (int l = 0; l < nl; ++l) {
        const double* L = ldir + 3 * l;
        double ndl = dot3(n, L);
        if (ndl <= 0.0 || !lit[l]) continue;
        diff += sp[0] * lI[l] * sp[3] * ndl;
        double r[3] = {2.0 * ndl * n[0] - L[0], 2.0 * ndl * n[1] - L[1], 2.0 * ndl * n[2] - L[2]};
        double rv = dot3(r, v);
        if (rv > 0.0) spec += sp[0] * lI[l] * sp[4] * pow(rv, sp[5]);
    }
    for (int k = 0; k < 3; ++k) {
        double c = albedo[k] * (sp[1] * sp[2] * V + diff) + spec;
        rgb[k] = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
    }
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    oscene sc;
    ogrid gr;
    int mode; /* 0 brute force, 1 grid */
} oworld;

static int world_init(oworld* w, int64_t S, const double* sph, int64_t C, const double* cyl,
                      const uint32_t* color, const double* palette, int32_t K, int mode, double lambda)
{
    memset(w, 0, sizeof(*w));
    w->sc.S = S; w->sc.C = C; w->sc.sph = sph; w->sc.cyl = cyl;
    w->sc.color = color; w->sc.palette = palette; w->sc.K = K;
    w->mode = mode;
    if (mode == 1) return grid_build(&w->sc, lambda, &w->gr);
    w->gr.empty = 1;
    return 0;
}

static void world_nearest(const oworld* w, const double o[3], const double d[3], double tmin, double tmax,
                          nearest_t* nr, ocount* cnt)
{
    nearest_reset(nr);
    if (w->mode == 1) nearest_grid(&w->sc, &w->gr, o, d, tmin, tmax, nr, cnt);
    else nearest_brute(&w->sc, o, d, tmin, tmax, nr, cnt);
}

static int world_anyhit(const oworld* w, const double o[3], const double d[3], double tmax, ocount* cnt)
{
    if (w->mode == 1) return anyhit_grid(&w->sc, &w->gr, o, d, tmax, cnt);
    return anyhit_brute(&w->sc, o, d, tmax, cnt);
}

/* Grazing ray (parity of hit ids is not asserted on it): a silhouette or
 * clip-plane decision within rounding of flipping at or before the winning t
 * (relative GRAZE_TIE), or a miss with such an encounter anywhere in front,
 * or the two nearest distinct hits within a relative GRAZE_TIE. */
static int is_grazing(const nearest_t* nr)
{
    if (nr->id1 == OR_MISS) return nr->t_graze < INFINITY;
    if (nr->t_graze <= nr->t1 * (1.0 + GRAZE_TIE) + 1e-9) return 1;
    if (nr->id2 != OR_MISS && (nr->t2 - nr->t1) <= GRAZE_TIE * fabs(nr->t1)) return 1;
    return 0;
}

/* The other outcomes a grazing ray may legitimately give -- its runner-up
 * (the second-nearest distinct hit) and the object of its nearest grazing
 * encounter -- from the brute-force definition (the grid walk stops before
 * the runner-up of a hit far ahead of it). Not counted as the method's work. */
static void grazing_alternatives(const oworld* w, const double o[3], const double d[3], double tmin,
                                 double tmax, nearest_t* nr)
{
    if (w->mode != 1) return;  /* brute force considered every object already */
    nearest_t b;
    ocount c = {0, 0, 0};
    nearest_reset(&b);
    nearest_brute(&w->sc, o, d, tmin, tmax, &b, &c);
    nr->t2 = b.t2;
    nr->id2 = b.id2;
    nr->id_graze = b.id_graze;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Nearest hits of explicit rays (o, d unit). out_grazing, out_id2 and
 * out_idg may be NULL; out_id2 / out_idg receive, for grazing rays, the
 * runner-up and the object of the nearest grazing encounter (OR_MISS when
 * there is none; OR_MISS on every other ray). */
int oracle_nearest(int64_t S, const double* sph, int64_t C, const double* cyl, int32_t mode, double lambda,
                   int64_t nrays, const double* orig, const double* dirs, double tmin, double tmax,
                   uint32_t* out_id, double* out_t, uint8_t* out_grazing, uint32_t* out_id2, uint32_t* out_idg,
                   int64_t* counters)
{
    oworld w;
    if (world_init(&w, S, sph, C, cyl, NULL, NULL, 0, mode, lambda)) return -1;
    ocount tot = {0, 0, 0};
    for (int64_t r = 0; r < nrays; ++r) {
        nearest_t nr;
        ocount cnt = {0, 0, 0};
        world_nearest(&w, orig + 3 * r, dirs + 3 * r, tmin, tmax, &nr, &cnt);
        out_id[r] = nr.id1;
        out_t[r] = nr.id1 == OR_MISS ? INFINITY : nr.t1;
        const int gz = is_grazing(&nr);
        if (gz) grazing_alternatives(&w, orig + 3 * r, dirs + 3 * r, tmin, tmax, &nr);
        if (out_grazing) out_grazing[r] = (uint8_t)gz;
        if (out_id2) out_id2[r] = gz ? nr.id2 : OR_MISS;
        if (out_idg) out_idg[r] = gz ? nr.id_graze : OR_MISS;
        tot.cells += cnt.cells; tot.sph += cnt.sph; tot.cyl += cnt.cyl;
    }
    if (counters) { counters[0] = tot.cells; counters[1] = tot.sph; counters[2] = tot.cyl; }
    grid_free(&w.gr);
    return 0;
}

/* Any hit in (0, tmax] of explicit rays (o, d unit), the query of an AO or
 * shadow ray: out_hit[r] = 1 when ray r meets an object; counters = cells
 * walked, sphere tests and cylinder tests over all rays (the AO rays' work
 * counts of the roofline come from this walk). */
int oracle_anyhit(int64_t S, const double* sph, int64_t C, const double* cyl, int32_t mode, double lambda,
                  int64_t nrays, const double* orig, const double* dirs, double tmax, uint8_t* out_hit,
                  int64_t* counters)
{
    oworld w;
    if (world_init(&w, S, sph, C, cyl, NULL, NULL, 0, mode, lambda)) return -1;
    ocount tot = {0, 0, 0};
    for (int64_t r = 0; r < nrays; ++r) {
        ocount cnt = {0, 0, 0};
        out_hit[r] = (uint8_t)world_anyhit(&w, orig + 3 * r, dirs + 3 * r, tmax, &cnt);
        tot.cells += cnt.cells; tot.sph += cnt.sph; tot.cyl += cnt.cyl;
    }
    if (counters) { counters[0] = tot.cells; counters[1] = tot.sph; counters[2] = tot.cyl; }
    grid_free(&w.gr);
    return 0;
}

/* Visited cells (flattened indices) of one ray walking the whole grid. */
int oracle_grid_walk(int64_t S, const double* sph, int64_t C, const double* cyl, double lambda,
                     const double o[3], const double d[3], double tmin, double tmax,
                     int64_t max_out, int64_t* out_cells, int32_t* out_dims)
{
    oworld w;
    if (world_init(&w, S, sph, C, cyl, NULL, NULL, 0, 1, lambda)) return -1;
    int64_t n = 0;
    if (out_dims) { out_dims[0] = w.gr.n[0]; out_dims[1] = w.gr.n[1]; out_dims[2] = w.gr.n[2]; }
    dda_t it;
    if (!w.gr.empty && dda_start(&w.gr, o, d, tmin, tmax, &it)) {
        do {
            if (n < max_out) out_cells[n] = ((int64_t)it.c[2] * w.gr.n[1] + it.c[1]) * w.gr.n[0] + it.c[0];
            n++;
        } while (dda_next(&w.gr, &it));
    }
    grid_free(&w.gr);
    return (int)n;
}

/* Grid geometry: lo[3], hi[3], n[3], total references. */
int oracle_grid_info(int64_t S, const double* sph, int64_t C, const double* cyl, double lambda,
                     double* out_lo_hi, int32_t* out_dims, int64_t* out_refs)
{
    oworld w;
    if (world_init(&w, S, sph, C, cyl, NULL, NULL, 0, 1, lambda)) return -1;
    for (int k = 0; k < 3; ++k) {
        out_lo_hi[k] = w.gr.lo[k];
        out_lo_hi[3 + k] = w.gr.hi[k];
        out_dims[k] = w.gr.n[k];
    }
    *out_refs = w.gr.empty ? 0 : w.gr.start[w.gr.ncells];
    grid_free(&w.gr);
    return 0;
}

/* AO visibility fraction of points with normals: origin p + eps n, `spp`
 * cosine-weighted directions, counter (index, sample, frame, 0xA0). */
int oracle_ao_probe(int64_t S, const double* sph, int64_t C, const double* cyl, int32_t mode, double lambda,
                    int64_t npts, const double* pts, const double* nrm, int32_t spp, uint64_t seed,
                    uint32_t frame, double eps, double maxdist, double* out_vis, int32_t nthreads)
{
    oworld w;
    if (world_init(&w, S, sph, C, cyl, NULL, NULL, 0, mode, lambda)) return -1;
#ifdef _OPENMP
    /* the thread count applies to this call only (0: all cores) */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
    for (int64_t i = 0; i < npts; ++i) {
        const double* p = pts + 3 * i;
        const double* n = nrm + 3 * i;
        double o[3] = {p[0] + eps * n[0], p[1] + eps * n[1], p[2] + eps * n[2]};
        int64_t vis = 0;
        ocount cnt = {0, 0, 0};
        for (int s = 0; s < spp; ++s) {
            double u1, u2, dir[3];
            oracle_ao_uniforms((uint32_t)i, (uint32_t)s, frame, seed, &u1, &u2);
            oracle_cosine_dir(n, u1, u2, dir);
            if (!world_anyhit(&w, o, dir, maxdist, &cnt)) vis++;
        }
        out_vis[i] = spp > 0 ? (double)vis / spp : 1.0;
    }
    grid_free(&w.gr);
    return 0;
}

/*
 * Render the listed pixels (pix[k] = j*W + i; pix == NULL -> all W*H in order).
 * Per pixel and per sub-sample (a, b) of its m x m regular sub-pixel grid
 * (m = cam[15]; m = 1: the pixel centre only): primary ray through the point
 * (i + (a + 0.5)/m, j + (b + 0.5)/m) -> nearest hit -> refined hit point and
 * normal -> `spp` AO rays from p + eps n -> shade -> clamp. The pixel's colour
 * is the mean of its m^2 sub-sample colours (a box filter). The AO samples of
 * sub-sample (a, b) use Philox counter word 0 = its index in the m-times finer
 * raster, (m j + b) (m W) + (m i + a), which is the pixel index when m = 1.
 * Outputs (any may be NULL): rgb (3 doubles) per listed pixel; hit id
 * (0xFFFFFFFF = miss), hit t, number of unoccluded AO samples and grazing flag
 * per sub-sample, at [k m^2 + b m + a]; for grazing sub-samples the runner-up
 * id and the id of the nearest grazing encounter (0xFFFFFFFF: none, and on
 * every non-grazing sub-sample).
 * counters[16] (may be NULL): 0 primary rays, 1 AO rays, 2 hit pixels,
 *   3 primary cells, 4 primary sphere tests, 5 primary cylinder tests,
 *   6 AO cells, 7 AO sphere tests, 8 AO cylinder tests, 9 unoccluded AO rays.
 */
int oracle_render(int64_t S, const double* sph, int64_t C, const double* cyl,
                  const uint32_t* color, const double* palette, int32_t K,
                  const double* cam, int32_t W, int32_t H,
                  const double* ldir, const double* lI, int32_t nl, const double* sp,
                  int32_t spp, uint64_t seed, uint32_t frame,
                  int32_t mode, double lambda,
                  int64_t npix, const int64_t* pix,
                  double* out_rgb, uint32_t* out_id, double* out_t, int32_t* out_vis, uint8_t* out_grazing,
                  uint32_t* out_id2, uint32_t* out_idg, int64_t* counters, int32_t nthreads)
{
    if (W <= 0 || H <= 0) return -2;
    const int m = cam[15] >= 1.0 ? (int)cam[15] : 1;
    if (m > 16) return -2;
    oworld w;
    if (world_init(&w, S, sph, C, cyl, color, palette, K, mode, lambda)) return -1;
    if (!pix) npix = (int64_t)W * H;
    int64_t tot[16];
    memset(tot, 0, sizeof(tot));
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        int64_t loc[16];
        memset(loc, 0, sizeof(loc));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < npix; ++k) {
            int64_t q = pix ? pix[k] : k;
            int64_t i = q % W, j = q / W;
            double acc[3] = {0.0, 0.0, 0.0};
            for (int b = 0; b < m; ++b) {
                for (int a = 0; a < m; ++a) {
                    const int64_t sub = k * m * m + b * m + a;
                    /* counter word 0: the sub-sample's index in the finer raster */
                    const uint32_t qf = (uint32_t)(((int64_t)m * j + b) * ((int64_t)m * W) + ((int64_t)m * i + a));
                    double o[3], d[3];
                    primary_ray(cam, W, H, (double)i + (a + 0.5) / m, (double)j + (b + 0.5) / m, o, d);
                    nearest_t nr;
                    ocount pc = {0, 0, 0}, ac = {0, 0, 0};
                    world_nearest(&w, o, d, 0.0, INFINITY, &nr, &pc);
                    loc[0]++;
                    loc[3] += pc.cells; loc[4] += pc.sph; loc[5] += pc.cyl;
                    double rgb[3] = {sp[8], sp[9], sp[10]};
                    int32_t vis = 0;
                    if (nr.id1 != OR_MISS) {
                        loc[2]++;
                        double p[3], n[3];
                        refine(&w.sc, nr.id1, o, d, nr.t1, p, n);
                        double ao_o[3] = {p[0] + sp[6] * n[0], p[1] + sp[6] * n[1], p[2] + sp[6] * n[2]};
                        for (int s = 0; s < spp; ++s) {
                            double u1, u2, dir[3];
                            oracle_ao_uniforms(qf, (uint32_t)s, frame, seed, &u1, &u2);
                            oracle_cosine_dir(n, u1, u2, dir);
                            if (!world_anyhit(&w, ao_o, dir, sp[7], &ac)) vis++;
                        }
                        loc[1] += spp;
                        loc[6] += ac.cells; loc[7] += ac.sph; loc[8] += ac.cyl; loc[9] += vis;
                        double V = spp > 0 ? (double)vis / spp : 1.0;
                        /* direct-light shadow rays: from the AO origin toward each light
                         * the surface faces; any hit (0 < t) blocks that light */
                        int lit[64];
                        for (int l = 0; l < nl && l < 64; ++l) {
                            lit[l] = 1;
                            if (sp[11] != 0.0 && dot3(n, ldir + 3 * l) > 0.0) {
                                ocount sc_ = {0, 0, 0};
                                lit[l] = !world_anyhit(&w, ao_o, ldir + 3 * l, INFINITY, &sc_);
                            }
                        }
                        uint32_t ci = w.sc.color[nr.id1];
                        double albedo[3] = {palette[3 * ci], palette[3 * ci + 1], palette[3 * ci + 2]};
                        shade(albedo, n, d, V, ldir, lI, nl, sp, lit, rgb);
                    }
                    acc[0] += rgb[0]; acc[1] += rgb[1]; acc[2] += rgb[2];
                    if (out_id) out_id[sub] = nr.id1;
                    if (out_t) out_t[sub] = nr.id1 == OR_MISS ? INFINITY : nr.t1;
                    if (out_vis) out_vis[sub] = vis;
                    const int gz = is_grazing(&nr);
                    if (gz) grazing_alternatives(&w, o, d, 0.0, INFINITY, &nr);
                    if (out_grazing) out_grazing[sub] = (uint8_t)gz;
                    if (out_id2) out_id2[sub] = gz ? nr.id2 : OR_MISS;
                    if (out_idg) out_idg[sub] = gz ? nr.id_graze : OR_MISS;
                }
            }
            if (out_rgb) {
                const double mm = (double)m * m;
                out_rgb[3 * k] = acc[0] / mm; out_rgb[3 * k + 1] = acc[1] / mm; out_rgb[3 * k + 2] = acc[2] / mm;
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int c = 0; c < 16; ++c) tot[c] += loc[c];
    }
    if (counters) memcpy(counters, tot, sizeof(tot));
    grid_free(&w.gr);
    return 0;
}
