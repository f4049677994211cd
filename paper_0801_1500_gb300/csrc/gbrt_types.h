// Internal device-side views of scenes, grids and frames, shared by the host
// orchestration code and the kernels of libgbrt (never exposed in the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbrt.h"

namespace gbrt {

// Error bits of the context's device error word.
enum : uint32_t {
    ERR_DDA_STEPS = 1u,      // a grid walk exceeded nx + ny + nz + 3 steps
    ERR_SCENE_DATA = 2u,     // non-finite / non-positive scene values (device upload path)
    ERR_QUEUE_TIMEOUT = 4u,  // reserved: a bounded wait ran out (no kernel of this version waits)
    ERR_GRID_CAPACITY = 8u,  // a device-side grid rebuild outgrew its item buffer
};

// Scene in the device layout: one record per object, indexed by global id
// (spheres 0..S-1, then cylinders S..S+C-1), the same shape for both kinds so
// a single branch-free test serves both (a sphere is a cylinder record with a
// zero axis and zero length):
//   obj    float4 [2 (S+C)]  (p0 xyz, radius), (unit axis xyz, length)
//   obj64  double2[4 (S+C)]  (p0x, p0y), (p0z, radius), (ax, ay), (az, length)
//   color  uint32 [S+C] palette index; palette float [K*3]
struct SceneDev {
    int32_t S, C, K, pad;
    const float4* obj;
    const double2* obj64;
    const uint32_t* color;
    const float* palette;
};

// Uniform grid. cells[c] = (first item, item count) of cell
// c = (z * ny + y) * nx + x; items are global object ids, ascending per cell
// after a host build, in scatter order after a device-side rebuild (no result
// depends on the order).
struct GridDev {
    float lo[3], hi[3], h[3], inv_h[3];
    double lo64[3], hi64[3], h64[3], inv_h64[3];
    // bounding sphere of all objects (centre xyz, radius): walks are clipped to
    // it, so rays skip the empty corners of the grid box
    float bs[4];
    double bs64[4];
    int32_t n[3];
    int32_t empty;
    int64_t ncells;
    int64_t nitems;  // length of the item buffer
    const uint2* cells;
    const uint32_t* items;
};

// Everything one frame needs, in the precision each path reads.
struct FrameDev {
    SceneDev scene;
    GridDev grid;
    // camera (double) -- the float path rounds the primary ray from these
    double eye[3], dir[3], up[3], right[3];
    double half_w, half_h;
    double inv_w, inv_h;  // 1/W, 1/H
    double dir_unit[3];   // dir / |dir|
    float dir_f[3], up_f[3], right_f[3];
    float half_w_f, half_h_f, inv_w_f, inv_h_f;
    // the float path's primary rays as float-float pairs (value = hi + lo,
    // |lo| <= half an ulp of hi). The part that varies with pixel (i, j) is
    // affine in it, a0 + i ai + j aj: the orthographic origin (direction
    // dir_unit), or the pinhole direction before normalisation (origin eye)
    float a0_hi[3], a0_lo[3], ai_hi[3], ai_lo[3], aj_hi[3], aj_lo[3];
    float dir_hi[3], dir_lo[3], eye_hi[3], eye_lo[3];
    int32_t cam_kind;
    int32_t W, H, spp;
    int32_t shadows;       // 1: one shadow ray per light the surface faces
    int32_t jobs_per_hit;  // AO samples + shadow rays of one hit
    uint32_t jph_magic;    // ceil(2^32 / jobs_per_hit) when jobs_per_hit > 1 (division by multiply)
    uint32_t frame;
    uint32_t seed_lo, seed_hi;
    int32_t precision;
    // shading
    int32_t nl;
    double ldir[GBRT_MAX_LIGHTS][3];
    double lI[GBRT_MAX_LIGHTS];  // intensity * scale
    float ldir_f[GBRT_MAX_LIGHTS][3];
    float lI_f[GBRT_MAX_LIGHTS];
    double sky_kao, k_d, k_s, phong;
    float sky_kao_f, k_d_f, k_s_f, phong_f;
    double eps, ao_maxdist;
    float eps_f;
    float ao_maxdist_f;
    double bg[3];
    float bg_f[3];
    // outputs (device). Pixel q of the rendered raster writes its colour at
    // out_rgb + 3 (q - rgb_q0). With supersampling (aa = m > 1) the rendered
    // raster is the m-times finer one (W, H, row0, rows count its pixels),
    // out_rgb is the library's buffer for the band's finer rows, and the
    // resolve pass box-filters it into out_final ((W/m) x (H/m) pixels).
    void* out_rgb;
    uint32_t* out_ids;
    uint32_t* out_vis;
    void* out_final;
    int64_t rgb_q0;
    int32_t aa;
    // grid rebuilt on the device: its current geometry, copied over `grid`
    // before the frame's kernels run (null for grids built on the host)
    const GridDev* grid_src;
    // rows [row0, row0 + rows) of the image are rendered (a band, or all rows);
    // their tiling into primary-ray work items (tile_w x tile_h = 32)
    int32_t row0, rows;
    int32_t tiles_x, tiles_y;
    int64_t hit_base;  // first slot of this frame's region of the hit buffers
};

// One batch of frames as the render kernels see it (a kernel parameter).
//   frames    [n] descriptors (device)
//   tile_off  [n + 1] prefix sums of primary work items (device)
//   hit_count [n] hits appended by the primary pass, per frame
//   job_off   [n + 1] prefix sums of AO rays (hits x samples) per frame
//   hit_off   [n + 1] prefix sums of hits per frame
//   hits      2 records per hit (FP32: float4 pairs; FP64: 4 double2), at
//             frames[f].hit_base + h:  (origin xyz, pixel)  (normal xyz, object id)
//   vis       escaped AO samples per hit slot
//   lmask     per hit slot, bit l set when the shadow ray toward light l escaped
//   queue     [0] next primary work item, [1] next AO ray, [2] next shading item
struct BatchDev {
    const FrameDev* frames;
    const long long* tile_off;
    unsigned int* hit_count;
    unsigned long long* job_off;
    unsigned long long* hit_off;
    void* hits;
    unsigned int* vis;
    unsigned int* lmask;
    unsigned long long* queue;
    unsigned int* err;
    int64_t hit_cap;  // hit slots (records, vis, lmask) of the batch
    int32_t nframes;
    int32_t tile_w, tile_h;
    int32_t refill;
};

}  // namespace gbrt
