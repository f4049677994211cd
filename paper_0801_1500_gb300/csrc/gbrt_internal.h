// Host-side objects behind the C ABI handles, and the launch functions each
// translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbrt.h"
#include "gbrt_types.h"

namespace gbrt {

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t* d_err = nullptr;   // device error word (ERR_* bits)
    uint32_t* h_err = nullptr;   // pinned mirror
    int64_t launches = 0;
    gbrt_tuning tuning{};
    // device buffers for renders whose outputs are host memory
    void* d_out = nullptr;
    size_t d_out_bytes = 0;
    // batch descriptors / work queue
    FrameDev* d_frames = nullptr;
    FrameDev* h_frames = nullptr;  // pinned staging
    int32_t frames_cap = 0;
    unsigned long long* d_queue = nullptr;  // [0] next work item, [1] spare
    // CUDA graph of the last batch shape
    cudaGraphExec_t graph_exec = nullptr;
    int32_t graph_n = -1;
    int64_t graph_items = -1;
};

struct Scene {
    int device = 0;
    int64_t S = 0, C = 0;
    int32_t K = 0;
    float4* sph = nullptr;
    float4* cyl_a = nullptr;
    float4* cyl_b = nullptr;
    double2* sph64 = nullptr;
    double2* cyl64 = nullptr;
    uint32_t* color = nullptr;
    float* palette = nullptr;
    float4* aabb = nullptr;  // [2 (S + C)]: lo (xyz), hi (xyz) per object
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    size_t bytes = 0;

    SceneDev view() const {
        SceneDev v;
        v.S = (int32_t)S;
        v.C = (int32_t)C;
        v.K = K;
        v.pad = 0;
        v.sph = sph;
        v.cyl_a = cyl_a;
        v.cyl_b = cyl_b;
        v.sph64 = sph64;
        v.cyl64 = cyl64;
        v.color = color;
        v.palette = palette;
        return v;
    }
};

struct Grid {
    GridDev dev{};
    uint2* cells = nullptr;
    uint32_t* items = nullptr;
    int64_t refs = 0;
    size_t bytes = 0;
    float lambda = 0.f;
};

// scene_grid.cu: fill a caller-allocated object; on failure it frees what it
// allocated and leaves the object empty.
int scene_upload(Ctx* ctx, const float* spheres, int64_t S, const float* cyl, int64_t C, const uint32_t* color,
                 const float* palette, int32_t K, int flags, Scene* out);
void scene_release(Scene* s);
int grid_build(Ctx* ctx, const Scene* s, float lambda, Grid* out);
void grid_release(Grid* g);

// render.cu
int launch_render(Ctx* ctx, const FrameDev& f);
int launch_ao_probe(Ctx* ctx, const FrameDev& f, const double* pts, const double* nrm, int64_t n, float* out);
int launch_philox(Ctx* ctx, const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out);

}  // namespace gbrt

struct gbrt_ctx : public gbrt::Ctx {};
struct gbrt_scene : public gbrt::Scene {};
struct gbrt_grid : public gbrt::Grid {};
