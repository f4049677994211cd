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
    int num_sms = 1;
    bool smem_configured = false;
    cudaStream_t stream = nullptr;
    uint32_t* d_err = nullptr;   // device error word (ERR_* bits)
    uint32_t* h_err = nullptr;   // pinned mirror
    int64_t launches = 0;
    gbrt_tuning tuning{};
    // renders whose outputs are host memory: two device staging buffers used
    // in turn, copied back on copy_stream, so one frame's copy overlaps the
    // next frame's kernels
    void* d_out[2] = {nullptr, nullptr};
    size_t d_out_bytes[2] = {0, 0};
    int out_slot = 0;                               // the buffer the next render uses
    cudaStream_t copy_stream = nullptr;             // created at the first host-output render
    cudaEvent_t out_ready[2] = {nullptr, nullptr};  // the render into buffer k finished
    cudaEvent_t out_free[2] = {nullptr, nullptr};   // the copy out of buffer k finished
    bool out_used[2] = {false, false};              // out_free[k] has been recorded
    // wavefront buffers: hit records, escaped-sample counts, descriptors, counters
    void* d_hits = nullptr;
    size_t hits_cap = 0;
    unsigned int* d_vis = nullptr;
    size_t vis_cap = 0;
    unsigned int* d_lmask = nullptr;
    size_t lmask_cap = 0;
    void* d_fine = nullptr;  // finer-raster colours of supersampled frames
    size_t fine_cap = 0;
    void* d_desc = nullptr;
    size_t desc_cap = 0;
    void* h_desc = nullptr;  // pinned staging of the descriptors
    size_t h_desc_cap = 0;
    void* d_counters = nullptr;
    size_t counters_cap = 0;
    size_t counters_bytes_used = 0;
    cudaEvent_t staging_done = nullptr;  // the last descriptor copy has been consumed
    bool staging_pending = false;
    // CUDA graph of the last batch layout
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_valid = false;
    long long graph_key = 0;
    int graph_extra = 0;  // optional passes in the captured graph (EXTRA_* bits)
    BatchDev graph_bd{};
    // per-kernel timing: 0 off, GBRT_PROFILE_ALL, GBRT_PROFILE_AO_WALK; the
    // mode the last timed render ran under (0: none timed)
    int profiling = 0;
    int timed = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

struct Scene {
    int device = 0;
    int64_t S = 0, C = 0;
    int32_t K = 0;
    float4* obj = nullptr;
    double2* obj64 = nullptr;
    uint32_t* color = nullptr;
    float* palette = nullptr;
    float4* aabb = nullptr;  // [2 (S + C)]: lo (xyz), hi (xyz) per object
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    size_t bytes = 0;
    // scene box on the device (order-preserving words: min xyz, max xyz,
    // invalid flag); kept so device-side rebuilds read the current box
    uint32_t* d_box = nullptr;
    float* d_in = nullptr;  // staging of host geometry for gbrt_scene_update
    bool box_stale = false;  // lo/hi above predate a device-side update

    SceneDev view() const {
        SceneDev v;
        v.S = (int32_t)S;
        v.C = (int32_t)C;
        v.K = K;
        v.pad = 0;
        v.obj = obj;
        v.obj64 = obj64;
        v.color = color;
        v.palette = palette;
        return v;
    }
};

// Counts a device-side rebuild reports back (page-locked host copy).
struct GridStat {
    unsigned long long refs;
    unsigned long long ncells;
    unsigned int overflow;
    unsigned int pad;
};

// Geometry handed to the build kernels through device memory, so a rebuild
// can compute it on the device.
struct BuildP {
    float lo[3], inv_h[3], h[3];
    int32_t n[3];
    float pad;
};
struct BuildAux {
    BuildP p;
    double ctr[3];        // centre of the bounding sphere
    unsigned int rbits;   // its radius (float bits, atomicMax)
    unsigned int pad;
};

struct Grid {
    GridDev dev{};
    uint2* cells = nullptr;
    uint32_t* items = nullptr;
    int64_t refs = 0;
    size_t bytes = 0;
    float lambda = 0.f;
    int64_t N = 0;  // objects of the scene it was built for
    int device = 0;  // the scene's device
    // device-side rebuilds (gbrt_grid_rebuild): the authoritative geometry is
    // d_geom on the device; renders copy it into their frame descriptors
    bool dynamic = false;
    GridDev* d_geom = nullptr;
    BuildAux* d_aux = nullptr;
    uint32_t* d_counts = nullptr;
    unsigned long long* d_sums = nullptr;
    unsigned long long* d_reach = nullptr;  // per object: cells reached, from the count pass
    GridStat* d_stat = nullptr;
    GridStat* h_stat = nullptr;
    cudaEvent_t stat_ev = nullptr;
    bool stat_pending = false;
    int64_t cells_cap = 0, items_cap = 0;
    cudaStream_t stream = nullptr;  // stream of the last rebuild
};

// scene_grid.cu: fill a caller-allocated object; on failure it frees what it
// allocated and leaves the object empty.
int scene_upload(Ctx* ctx, const float* spheres, int64_t S, const float* cyl, int64_t C, const uint32_t* color,
                 const float* palette, int32_t K, int flags, Scene* out);
void scene_release(Scene* s);
int grid_build(Ctx* ctx, const Scene* s, float lambda, Grid* out);
void grid_release(Grid* g);
// device-side animation path: new geometry for a resident scene, and a grid
// rebuild that neither allocates (after its first call) nor waits for the GPU
int scene_update(Ctx* ctx, Scene* s, const float* spheres, const float* cyl, int flags);
int grid_rebuild(Ctx* ctx, const Scene* s, Grid* g);
// wait for a grid's last device-side rebuild and refresh the host copies
int grid_refresh_host(Grid* g);
// refresh a scene's host box after device-side updates (waits for `stream`)
int scene_refresh_host(Scene* s, cudaStream_t stream);
// microbench.cu: FMA rates (TFLOP/s) and L2 read bandwidth (GB/s) of the device
int run_microbench(Ctx* ctx, int kind, double* value);

// capi.cu: argument checks and the frame descriptor of one render
int check_frame_args(const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* cam, int32_t W, int32_t H,
                     int32_t spp, const gbrt_lights* lights, const gbrt_params* params, const void* out_rgb);
FrameDev make_frame(const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* cam, int32_t W, int32_t H,
                    int32_t spp, const gbrt_lights* lights, const gbrt_params* p, void* out_rgb, uint32_t* out_ids,
                    uint32_t* out_vis);

// render.cu: render n frames of one precision (descriptors filled by the
// caller; tiling and hit-buffer fields are set here).
int render_frames(Ctx* ctx, FrameDev* frames, int n, bool use_graph);
// render.cu: for a batch whose descriptors and buffers the caller laid out:
// opt the AO kernels into their shared memory (once per device), then launch
// the four wavefront kernels with grids sized for the current device.
int configure_render_kernels();
int enqueue_prepared(const BatchDev& bd, int precision, cudaStream_t stream, int block, int num_sms, bool patch);

#ifdef GBRT_CHECKED
// checked build: indices the render kernels found outside their buffers since
// the last call (cleared as read)
unsigned long long checked_violations_render();
#endif
int launch_ao_probe(Ctx* ctx, const FrameDev& f, const double* pts, const double* nrm, int64_t n, float* out);
int launch_philox(Ctx* ctx, const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out);

}  // namespace gbrt

struct gbrt_ctx : public gbrt::Ctx {};
struct gbrt_scene : public gbrt::Scene {};
struct gbrt_grid : public gbrt::Grid {};
