// gbrt_render_noalloc: the render path for callers that cannot allocate device
// memory while they render. Everything the render needs beyond the caller's
// inputs and outputs -- hit records, escaped-sample counts, the frame
// descriptor, work-queue counters -- lives in one file-scope device array of
// fixed size, so the call makes no cudaMalloc/cudaFree and no allocating
// library call.
#include <mutex>

#include "gbrt_internal.h"

namespace gbrt {
namespace {

// Scratch layout (bytes, each region 256-aligned):
//   counters   queue[4] (u64), job_off[2], hit_off[2] (u64), hit_count[1] (u32), err (u32)
//   desc       one FrameDev, then tile_off[2] (i64)
//   vis        GBRT_NOALLOC_MAX_PIXELS x u32
//   lmask      GBRT_NOALLOC_MAX_PIXELS x u32 (shadow-ray light bits)
//   hits       GBRT_NOALLOC_MAX_PIXELS x 64 B (large enough for FP64 records)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_COUNTERS = 0;
constexpr size_t OFF_DESC = 256;
constexpr size_t OFF_TILES = OFF_DESC + align256(sizeof(FrameDev));
constexpr size_t OFF_VIS = OFF_TILES + 256;
constexpr size_t OFF_LMASK = OFF_VIS + align256((size_t)GBRT_NOALLOC_MAX_PIXELS * sizeof(uint32_t));
constexpr size_t OFF_HITS = OFF_LMASK + align256((size_t)GBRT_NOALLOC_MAX_PIXELS * sizeof(uint32_t));
constexpr size_t SCRATCH_BYTES = OFF_HITS + (size_t)GBRT_NOALLOC_MAX_PIXELS * 64;

// Every GPU that loads the library holds this array until the process exits.
// In host code `g_scratch` is only a host-side stand-in for the symbol; the
// device address comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};

// Once per device, with that device current: the array's device address and
// the render kernels' shared-memory opt-in.
int setup_device(int dev, unsigned char** base, int* sms) {
    if (dev < 0 || dev >= MAX_DEVICES) return GBRT_EDEVICE;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GBRT_EDEVICE;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return GBRT_EDEVICE;
        int rc = configure_render_kernels();
        if (rc != GBRT_OK) return rc;
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *base = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return GBRT_OK;
}

// Writes the frame descriptor and tile prefix into the scratch and clears the
// counters that must start at zero (the array keeps the previous call's data).
__global__ void k_noalloc_prepare(const __grid_constant__ FrameDev f, unsigned char* base, long long tiles) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long* q = (unsigned long long*)(base + OFF_COUNTERS);
    for (int k = 0; k < 8; ++k) q[k] = 0ull;
    unsigned int* c32 = (unsigned int*)(q + 8);
    c32[0] = 0u;  // hit_count
    c32[1] = 0u;  // error word
    *(FrameDev*)(base + OFF_DESC) = f;
    long long* toff = (long long*)(base + OFF_TILES);
    toff[0] = 0;
    toff[1] = tiles;
}

}  // namespace
}  // namespace gbrt

using namespace gbrt;

extern "C" GBRT_API int gbrt_render_noalloc(const gbrt_scene* scene, const gbrt_grid* grid,
                                            const gbrt_camera* camera, int32_t width, int32_t height,
                                            int32_t ao_samples, const gbrt_lights* lights,
                                            const gbrt_params* params, void* out_rgb, uint32_t* out_hit_ids,
                                            uint32_t* out_ao_visible, void* cuda_stream) {
    int rc = check_frame_args(scene, grid, camera, width, height, ao_samples, lights, params, out_rgb);
    if (rc != GBRT_OK) return rc;
    if (params->out_flags != 0) return GBRT_EINVAL;  // outputs must be device memory
    if ((int64_t)width * height > GBRT_NOALLOC_MAX_PIXELS) return GBRT_EINVAL;
    if (camera->aa > 1) return GBRT_EINVAL;  // supersampling needs a finer-raster buffer
    // an error left pending by the caller's earlier work is the caller's:
    // report it without enqueueing anything and leave it pending, so the
    // error read after this call's own launch below is this call's
    if (cudaPeekAtLastError() != cudaSuccess) return GBRT_EDEVICE;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return GBRT_EDEVICE;
    if (prev != scene->device && cudaSetDevice(scene->device) != cudaSuccess) return GBRT_EDEVICE;
    unsigned char* base = nullptr;
    int sms = 0;
    rc = setup_device(scene->device, &base, &sms);
    if (rc == GBRT_OK) {
        const int tw = 8, th = 4, block = 256, refill = 16;
        FrameDev f = make_frame(scene, grid, camera, width, height, ao_samples, lights, params, out_rgb,
                                out_hit_ids, out_ao_visible);
        f.tiles_x = (width + tw - 1) / tw;
        f.tiles_y = (height + th - 1) / th;
        f.hit_base = 0;
        const long long tiles = (long long)f.tiles_x * f.tiles_y;
        cudaStream_t stream = (cudaStream_t)cuda_stream;
        k_noalloc_prepare<<<1, 32, 0, stream>>>(f, base, tiles);
        BatchDev bd;
        unsigned long long* q = (unsigned long long*)(base + OFF_COUNTERS);
        bd.frames = (const FrameDev*)(base + OFF_DESC);
        bd.tile_off = (const long long*)(base + OFF_TILES);
        bd.queue = q;
        bd.job_off = q + 4;
        bd.hit_off = q + 6;
        bd.hit_count = (unsigned int*)(q + 8);
        bd.err = (unsigned int*)(q + 8) + 1;
        bd.hits = base + OFF_HITS;
        bd.vis = (unsigned int*)(base + OFF_VIS);
        bd.lmask = (unsigned int*)(base + OFF_LMASK);
        bd.hit_cap = (int64_t)width * height;
        bd.nframes = 1;
        bd.tile_w = tw;
        bd.tile_h = th;
        bd.refill = refill;
        rc = cudaGetLastError() == cudaSuccess ? GBRT_OK : GBRT_EDEVICE;
        if (rc == GBRT_OK) rc = enqueue_prepared(bd, params->precision, stream, block, sms, f.grid_src != nullptr);
    }
    if (prev != scene->device) cudaSetDevice(prev);
    return rc;
}
