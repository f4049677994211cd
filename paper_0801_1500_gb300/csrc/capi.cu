// The C ABI (include/gbrt.h): argument validation, handles, streams, error
// word, and the frame descriptors handed to the kernels. No C++ exception
// crosses this boundary.
#include <math.h>
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "gbrt_internal.h"

using namespace gbrt;

namespace gbrt {

static bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int check_frame_args(const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* cam, int32_t W, int32_t H,
                     int32_t spp, const gbrt_lights* lights, const gbrt_params* params, const void* out_rgb) {
    if (!scene || !grid || !cam || !lights || !params || !out_rgb) return GBRT_EINVAL;
    if (W <= 0 || H <= 0 || W > GBRT_MAX_DIM || H > GBRT_MAX_DIM || (int64_t)W * H >= (1ll << 31)) return GBRT_EINVAL;
    if (spp < 0 || spp > GBRT_MAX_SAMPLES) return GBRT_EINVAL;
    if (cam->kind != GBRT_CAMERA_ORTHO && cam->kind != GBRT_CAMERA_PINHOLE) return GBRT_EINVAL;
    if (cam->aa < 0 || cam->aa > GBRT_MAX_AA) return GBRT_EINVAL;
    {
        const int64_t m = cam->aa > 1 ? cam->aa : 1;
        if (m * W * m * H >= (1ll << 31)) return GBRT_EINVAL;
    }
    if (!finite3(cam->eye) || !finite3(cam->dir) || !finite3(cam->up) || !finite3(cam->right)) return GBRT_EINVAL;
    if (!(cam->half_w > 0) || !(cam->half_h > 0) || !std::isfinite(cam->half_w) || !std::isfinite(cam->half_h))
        return GBRT_EINVAL;
    double dl = cam->dir[0] * cam->dir[0] + cam->dir[1] * cam->dir[1] + cam->dir[2] * cam->dir[2];
    if (!(dl > 0)) return GBRT_EINVAL;
    if (lights->n < 0 || lights->n > GBRT_MAX_LIGHTS) return GBRT_EINVAL;
    for (int l = 0; l < lights->n; ++l)
        if (!finite3(lights->dir[l]) || !std::isfinite(lights->intensity[l])) return GBRT_EINVAL;
    if (!std::isfinite(lights->scale) || !std::isfinite(lights->skylight)) return GBRT_EINVAL;
    if (params->precision != GBRT_FP32 && params->precision != GBRT_FP64) return GBRT_EINVAL;
    if (!(params->eps >= 0) || !std::isfinite(params->eps)) return GBRT_EINVAL;
    if (!(params->ao_maxdist > 0)) return GBRT_EINVAL;  // +inf allowed
    if (!std::isfinite(params->k_ao) || !std::isfinite(params->k_d) || !std::isfinite(params->k_s) ||
        !std::isfinite(params->phong_exp) || !finite3(params->background))
        return GBRT_EINVAL;
    if (grid->dev.cells == nullptr) return GBRT_EINVAL;
    // a grid lists ids of the scene it was built for, on that scene's device
    if (grid->N != scene->S + scene->C || grid->device != scene->device) return GBRT_EINVAL;
    return GBRT_OK;
}

FrameDev make_frame(const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* cam, int32_t W, int32_t H,
                    int32_t spp, const gbrt_lights* lights, const gbrt_params* p, void* out_rgb, uint32_t* out_ids,
                    uint32_t* out_vis) {
    FrameDev f;
    memset(&f, 0, sizeof(f));
    // supersampling renders the m-times finer raster (its pixel centres are
    // the sub-sample points) and box-filters it afterwards
    const int32_t m = cam->aa > 1 ? cam->aa : 1;
    W *= m;
    H *= m;
    f.aa = m;
    f.scene = scene->view();
    f.grid = grid->dev;
    for (int k = 0; k < 3; ++k) {
        f.eye[k] = cam->eye[k];
        f.dir[k] = cam->dir[k];
        f.up[k] = cam->up[k];
        f.right[k] = cam->right[k];
    }
    f.half_w = cam->half_w;
    f.half_h = cam->half_h;
    f.inv_w = 1.0 / (double)W;
    f.inv_h = 1.0 / (double)H;
    {
        double l = sqrt(cam->dir[0] * cam->dir[0] + cam->dir[1] * cam->dir[1] + cam->dir[2] * cam->dir[2]);
        for (int k = 0; k < 3; ++k) {
            f.dir_unit[k] = cam->dir[k] / l;
            f.dir_f[k] = (float)f.dir_unit[k];
            f.up_f[k] = (float)cam->up[k];
            f.right_f[k] = (float)cam->right[k];
        }
    }
    f.half_w_f = (float)cam->half_w;
    f.half_h_f = (float)cam->half_h;
    f.inv_w_f = (float)f.inv_w;
    f.inv_h_f = (float)f.inv_h;
    {
        // pixel (i, j) sits at u right + v up from the view axis with
        // u = half_w ((2i + 1)/W - 1) = a_u i + b_u and v = half_h (1 - (2j + 1)/H)
        // = a_v j + b_v: the orthographic origin eye + u right + v up and the
        // pinhole direction dir_unit + u right + v up (before normalisation)
        // are a0 + i ai + j aj; each vector split into float pairs
        const double a_u = 2.0 * f.half_w * f.inv_w, b_u = f.half_w * (f.inv_w - 1.0);
        const double a_v = -2.0 * f.half_h * f.inv_h, b_v = f.half_h * (1.0 - f.inv_h);
        auto split = [](double x, float& hi, float& lo) {
            hi = (float)x;
            lo = (float)(x - (double)hi);
        };
        const double* base = cam->kind == GBRT_CAMERA_ORTHO ? f.eye : f.dir_unit;
        for (int k = 0; k < 3; ++k) {
            split(base[k] + b_u * f.right[k] + b_v * f.up[k], f.a0_hi[k], f.a0_lo[k]);
            split(a_u * f.right[k], f.ai_hi[k], f.ai_lo[k]);
            split(a_v * f.up[k], f.aj_hi[k], f.aj_lo[k]);
            split(f.dir_unit[k], f.dir_hi[k], f.dir_lo[k]);
            split(f.eye[k], f.eye_hi[k], f.eye_lo[k]);
        }
    }
    f.cam_kind = cam->kind;
    f.W = W;
    f.H = H;
    f.row0 = 0;
    f.rows = H;
    f.spp = spp;
    f.shadows = p->shadows ? 1 : 0;
    f.jobs_per_hit = spp + (f.shadows ? lights->n : 0);
    f.jph_magic = f.jobs_per_hit > 1
                      ? (uint32_t)(((1ull << 32) + (uint64_t)f.jobs_per_hit - 1) / (uint64_t)f.jobs_per_hit)
                      : 0u;
    f.frame = p->frame;
    f.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFull);
    f.seed_hi = (uint32_t)(p->seed >> 32);
    f.precision = p->precision;
    f.nl = lights->n;
    for (int l = 0; l < lights->n; ++l) {
        for (int k = 0; k < 3; ++k) {
            f.ldir[l][k] = lights->dir[l][k];
            f.ldir_f[l][k] = (float)lights->dir[l][k];
        }
        f.lI[l] = lights->intensity[l] * lights->scale;
        f.lI_f[l] = (float)f.lI[l];
    }
    f.sky_kao = lights->skylight * p->k_ao;
    f.k_d = p->k_d;
    f.k_s = p->k_s;
    f.phong = p->phong_exp;
    f.sky_kao_f = (float)f.sky_kao;
    f.k_d_f = (float)f.k_d;
    f.k_s_f = (float)f.k_s;
    f.phong_f = (float)f.phong;
    f.eps = p->eps;
    f.eps_f = (float)p->eps;
    f.ao_maxdist = p->ao_maxdist;
    f.ao_maxdist_f = (float)p->ao_maxdist;
    for (int k = 0; k < 3; ++k) {
        f.bg[k] = p->background[k];
        f.bg_f[k] = (float)p->background[k];
    }
    f.grid_src = grid->dynamic ? grid->d_geom : nullptr;
    f.out_rgb = out_rgb;
    f.out_final = out_rgb;
    f.rgb_q0 = 0;
    f.out_ids = out_ids;
    f.out_vis = out_vis;
    return f;
}

}  // namespace gbrt

namespace {

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int err_of(cudaError_t e) {
    if (e == cudaSuccess) return GBRT_OK;
    return e == cudaErrorMemoryAllocation ? GBRT_ENOMEM : GBRT_EDEVICE;
}

// Staging buffer `slot` of host-output renders, at least `bytes` long; the
// copy stream and its events are created on first use.
int ensure_out(Ctx* c, int slot, size_t bytes) {
    if (!c->copy_stream) {
        if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            c->copy_stream = nullptr;
            return GBRT_EDEVICE;
        }
    }
    for (int k = 0; k < 2; ++k) {
        if ((!c->out_ready[k] && cudaEventCreateWithFlags(&c->out_ready[k], cudaEventDisableTiming) != cudaSuccess) ||
            (!c->out_free[k] && cudaEventCreateWithFlags(&c->out_free[k], cudaEventDisableTiming) != cudaSuccess))
            return GBRT_EDEVICE;
    }
    if (c->d_out_bytes[slot] >= bytes) return GBRT_OK;
    if (c->d_out[slot]) {
        // a render or a copy in flight may still use it
        cudaStreamSynchronize(c->stream);
        cudaStreamSynchronize(c->copy_stream);
        cudaFree(c->d_out[slot]);
        c->d_out[slot] = nullptr;
        c->d_out_bytes[slot] = 0;
    }
    int rc = err_of(cudaMalloc(&c->d_out[slot], bytes));
    if (rc == GBRT_OK) c->d_out_bytes[slot] = bytes;
    return rc;
}

int read_error_word(Ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return err_of(e);
    uint32_t w = *c->h_err;
    if (w) {
        cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), c->stream);
        cudaStreamSynchronize(c->stream);
    }
#ifdef GBRT_CHECKED
    if (checked_violations_render() != 0) return GBRT_EBOUNDS;
#endif
    if (w & ERR_QUEUE_TIMEOUT) return GBRT_ETIMEDOUT;
    if (w & ERR_DDA_STEPS) return GBRT_ETRAVERSAL;
    if (w & ERR_GRID_CAPACITY) return GBRT_ECAPACITY;
    if (w) return GBRT_EINVAL;
    return GBRT_OK;
}

// Wait for the host-output copies, then read the error word.
int sync_all(Ctx* c) {
    if (c->copy_stream && cudaStreamSynchronize(c->copy_stream) != cudaSuccess) {
        read_error_word(c);
        return GBRT_EDEVICE;
    }
    return read_error_word(c);
}

}  // namespace

extern "C" {

GBRT_API int gbrt_version(void) { return GBRT_VERSION; }

GBRT_API const char* gbrt_strerror(int code) {
    switch (code) {
        case GBRT_OK: return "ok";
        case GBRT_EINVAL: return "invalid argument or scene data";
        case GBRT_ENOMEM: return "out of device or pinned memory";
        case GBRT_EDEVICE: return "CUDA device or runtime error";
        case GBRT_ETIMEDOUT: return "a bounded device wait ran out";
        case GBRT_EBOUNDS: return "an index fell outside its buffer (checked build)";
        case GBRT_ETRAVERSAL: return "a grid walk exceeded its step bound";
        case GBRT_ECAPACITY: return "a device-side grid rebuild outgrew its buffer";
        default: return "unknown error";
    }
}

GBRT_API int gbrt_create(gbrt_ctx** out, int device, void* cuda_stream) {
    if (!out) return GBRT_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return GBRT_EDEVICE;
    }
    if (device < 0 || device >= n) return GBRT_EINVAL;
    DeviceGuard g(device);
    if (!g.ok) return GBRT_EDEVICE;
    gbrt_ctx* c = new (std::nothrow) gbrt_ctx();
    if (!c) return GBRT_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->tuning.tile_w = 8;
    c->tuning.tile_h = 4;
    c->tuning.block = 256;
    c->tuning.ctas_per_sm = 0;
    c->tuning.refill = 16;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        c->num_sms < 1)
        c->num_sms = 1;
    if (cudaEventCreateWithFlags(&c->staging_done, cudaEventDisableTiming) != cudaSuccess) {
        delete c;
        return GBRT_EDEVICE;
    }
    if (cudaMalloc(&c->d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&c->h_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(uint32_t)) != cudaSuccess) {
        cudaFree(c->d_err);
        cudaFreeHost(c->h_err);
        cudaEventDestroy(c->staging_done);
        delete c;
        return GBRT_ENOMEM;
    }
    *out = c;
    return GBRT_OK;
}

GBRT_API int gbrt_set_stream(gbrt_ctx* ctx, void* cuda_stream) {
    if (!ctx) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    // work already enqueued reads the context's buffers: drain the old stream
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    ctx->stream = (cudaStream_t)cuda_stream;
    return GBRT_OK;
}

GBRT_API int gbrt_sync(gbrt_ctx* ctx) {
    if (!ctx) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    return sync_all(ctx);
}

GBRT_API int gbrt_destroy(gbrt_ctx* ctx) {
    if (!ctx) return GBRT_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (int k = 0; k < 2; ++k) {
        if (ctx->out_ready[k]) cudaEventDestroy(ctx->out_ready[k]);
        if (ctx->out_free[k]) cudaEventDestroy(ctx->out_free[k]);
        cudaFree(ctx->d_out[k]);
    }
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (int k = 0; k < 5; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    cudaEventDestroy(ctx->staging_done);
    cudaFree(ctx->d_err);
    cudaFreeHost(ctx->h_err);
    cudaFree(ctx->d_hits);
    cudaFree(ctx->d_vis);
    cudaFree(ctx->d_lmask);
    cudaFree(ctx->d_fine);
    cudaFree(ctx->d_desc);
    cudaFreeHost(ctx->h_desc);
    cudaFree(ctx->d_counters);
    delete ctx;
    return GBRT_OK;
}

GBRT_API int gbrt_scene_upload(gbrt_ctx* ctx, const float* spheres, int64_t n_spheres, const float* cylinders,
                               int64_t n_cylinders, const uint32_t* color_idx, const float* palette,
                               int32_t n_palette, int flags, gbrt_scene** out) {
    if (!ctx || !out) return GBRT_EINVAL;
    *out = nullptr;
    if (n_spheres < 0 || n_cylinders < 0 || n_spheres + n_cylinders >= (int64_t)GBRT_MISS) return GBRT_EINVAL;
    if (flags & ~GBRT_HOST_PTRS) return GBRT_EINVAL;
    const int64_t N = n_spheres + n_cylinders;
    if ((n_spheres > 0 && !spheres) || (n_cylinders > 0 && !cylinders)) return GBRT_EINVAL;
    if (N > 0 && (!color_idx || !palette || n_palette <= 0)) return GBRT_EINVAL;
    if (n_palette < 0) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    gbrt_scene* s = new (std::nothrow) gbrt_scene();
    if (!s) return GBRT_ENOMEM;
    int rc = scene_upload(ctx, spheres, n_spheres, cylinders, n_cylinders, color_idx, palette, n_palette, flags, s);
    if (rc != GBRT_OK) {
        delete s;
        return rc;
    }
    *out = s;
    return GBRT_OK;
}

GBRT_API int gbrt_scene_info(const gbrt_scene* scene, int64_t* n_spheres, int64_t* n_cylinders,
                             int64_t* device_bytes) {
    if (!scene) return GBRT_EINVAL;
    if (n_spheres) *n_spheres = scene->S;
    if (n_cylinders) *n_cylinders = scene->C;
    if (device_bytes) *device_bytes = (int64_t)scene->bytes;
    return GBRT_OK;
}

GBRT_API int gbrt_scene_free(gbrt_ctx* ctx, gbrt_scene* scene) {
    if (!scene) return GBRT_OK;
    if (!ctx) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    scene_release(scene);
    delete scene;
    return GBRT_OK;
}

GBRT_API int gbrt_grid_build(gbrt_ctx* ctx, const gbrt_scene* scene, float lambda, gbrt_grid** out) {
    if (!ctx || !scene || !out) return GBRT_EINVAL;
    *out = nullptr;
    if (!std::isfinite(lambda) || lambda > 1.0e6f) return GBRT_EINVAL;
    if (scene->device != ctx->device) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    gbrt_grid* gr = new (std::nothrow) gbrt_grid();
    if (!gr) return GBRT_ENOMEM;
    int rc = grid_build(ctx, scene, lambda, gr);
    if (rc != GBRT_OK) {
        delete gr;
        return rc;
    }
    *out = gr;
    return GBRT_OK;
}

GBRT_API int gbrt_grid_info(const gbrt_grid* grid, int32_t dims[3], float lo[3], float hi[3], int64_t* refs,
                            int64_t* device_bytes) {
    if (!grid) return GBRT_EINVAL;
    if (grid->dynamic) {
        int rc = grid_refresh_host(const_cast<gbrt_grid*>(grid));
        if (rc != GBRT_OK) return rc;
    }
    for (int k = 0; k < 3; ++k) {
        if (dims) dims[k] = grid->dev.n[k];
        if (lo) lo[k] = grid->dev.lo[k];
        if (hi) hi[k] = grid->dev.hi[k];
    }
    if (refs) *refs = grid->refs;
    if (device_bytes) *device_bytes = (int64_t)grid->bytes;
    return GBRT_OK;
}

GBRT_API int gbrt_microbench(gbrt_ctx* ctx, int kind, double* value) {
    if (!ctx || !value) return GBRT_EINVAL;
    if (kind != GBRT_MB_FP32_FMA && kind != GBRT_MB_FP64_FMA && kind != GBRT_MB_L2_READ) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    return run_microbench(ctx, kind, value);
}

GBRT_API int gbrt_scene_update(gbrt_ctx* ctx, gbrt_scene* scene, const float* spheres, const float* cylinders,
                               int flags) {
    if (!ctx || !scene) return GBRT_EINVAL;
    if (flags & ~GBRT_HOST_PTRS) return GBRT_EINVAL;
    if ((scene->S > 0 && !spheres) || (scene->C > 0 && !cylinders)) return GBRT_EINVAL;
    if (scene->device != ctx->device) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    return scene_update(ctx, scene, spheres, cylinders, flags);
}

GBRT_API int gbrt_grid_rebuild(gbrt_ctx* ctx, gbrt_grid* grid, const gbrt_scene* scene) {
    if (!ctx || !grid || !scene) return GBRT_EINVAL;
    if (scene->device != ctx->device) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    return grid_rebuild(ctx, scene, grid);
}

GBRT_API int gbrt_grid_free(gbrt_ctx* ctx, gbrt_grid* grid) {
    if (!grid) return GBRT_OK;
    if (!ctx) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    grid_release(grid);
    delete grid;
    return GBRT_OK;
}

GBRT_API int gbrt_render(gbrt_ctx* ctx, const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* camera,
                         int32_t width, int32_t height, int32_t ao_samples, const gbrt_lights* lights,
                         const gbrt_params* params, void* out_rgb, uint32_t* out_hit_ids,
                         uint32_t* out_ao_visible) {
    if (!ctx) return GBRT_EINVAL;
    int rc = check_frame_args(scene, grid, camera, width, height, ao_samples, lights, params, out_rgb);
    if (rc != GBRT_OK) return rc;
    if (scene->device != ctx->device) return GBRT_EINVAL;
    if (params->out_flags & ~(GBRT_HOST_PTRS | GBRT_HOST_ASYNC)) return GBRT_EINVAL;
    if ((params->out_flags & GBRT_HOST_ASYNC) && !(params->out_flags & GBRT_HOST_PTRS)) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    const bool host = (params->out_flags & GBRT_HOST_PTRS) != 0;
    const bool async = (params->out_flags & GBRT_HOST_ASYNC) != 0;
    const size_t aa = camera->aa > 1 ? (size_t)camera->aa : 1;
    const size_t rgb_bytes =
        (size_t)width * height * 3 * (params->precision == GBRT_FP64 ? sizeof(double) : sizeof(float));
    const size_t npx = (size_t)width * height * aa * aa;  // hit ids and AO counts: one per sub-sample
    void* d_rgb = out_rgb;
    uint32_t* d_ids = out_hit_ids;
    uint32_t* d_vis = out_ao_visible;
    const int slot = ctx->out_slot;
    if (host) {
        size_t need = rgb_bytes + (out_hit_ids ? npx * 4 : 0) + (out_ao_visible ? npx * 4 : 0);
        rc = ensure_out(ctx, slot, (need + 255) & ~(size_t)255);
        if (rc != GBRT_OK) return rc;
        // the copy out of this buffer two renders ago must end before the
        // render writes it
        if (ctx->out_used[slot] && cudaStreamWaitEvent(ctx->stream, ctx->out_free[slot], 0) != cudaSuccess)
            return GBRT_EDEVICE;
        char* base = (char*)ctx->d_out[slot];
        d_rgb = base;
        size_t off = (rgb_bytes + 15) & ~(size_t)15;
        if (out_hit_ids) {
            d_ids = (uint32_t*)(base + off);
            off += npx * 4;
        }
        if (out_ao_visible) d_vis = (uint32_t*)(base + off);
    }
    FrameDev f = make_frame(scene, grid, camera, width, height, ao_samples, lights, params, d_rgb, d_ids, d_vis);
    rc = render_frames(ctx, &f, 1, false);
    if (rc != GBRT_OK) return rc;
    if (host) {
        // the copies run on the copy stream once the render's kernels are done,
        // overlapping whatever the context's stream does next
        cudaStream_t cs = ctx->copy_stream;
        cudaError_t e = cudaEventRecord(ctx->out_ready[slot], ctx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->out_ready[slot], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_rgb, d_rgb, rgb_bytes, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && out_hit_ids)
            e = cudaMemcpyAsync(out_hit_ids, d_ids, npx * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && out_ao_visible)
            e = cudaMemcpyAsync(out_ao_visible, d_vis, npx * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->out_free[slot], cs);
        if (e != cudaSuccess) return err_of(e);
        ctx->out_used[slot] = true;
        ctx->out_slot = slot ^ 1;
        return async ? GBRT_OK : sync_all(ctx);
    }
    return GBRT_OK;
}

GBRT_API int gbrt_render_batch(gbrt_ctx* ctx, const gbrt_render_item* items, int32_t n, int flags) {
    if (!ctx || n < 0 || (n > 0 && !items)) return GBRT_EINVAL;
    if (flags & ~GBRT_BATCH_GRAPH) return GBRT_EINVAL;
    for (int32_t k = 0; k < n; ++k) {
        const gbrt_render_item& it = items[k];
        int rc = check_frame_args(it.scene, it.grid, &it.camera, it.width, it.height, it.ao_samples, &it.lights,
                                  &it.params, it.out_rgb);
        if (rc != GBRT_OK) return rc;
        if (it.scene->device != ctx->device) return GBRT_EINVAL;
        if (it.params.out_flags != 0) return GBRT_EINVAL;
        if (!(it.row_begin == 0 && it.row_end == 0) &&
            !(0 <= it.row_begin && it.row_begin < it.row_end && it.row_end <= it.height))
            return GBRT_EINVAL;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    // one wavefront launch sequence per precision present in the batch
    for (int prec = GBRT_FP32; prec <= GBRT_FP64; ++prec) {
        std::vector<FrameDev> frames;
        for (int32_t k = 0; k < n; ++k) {
            const gbrt_render_item& it = items[k];
            if (it.params.precision != prec) continue;
            frames.push_back(make_frame(it.scene, it.grid, &it.camera, it.width, it.height, it.ao_samples,
                                        &it.lights, &it.params, it.out_rgb, it.out_hit_ids, it.out_ao_visible));
            if (it.row_end > 0) {
                const int32_t m = frames.back().aa;
                frames.back().row0 = m * it.row_begin;
                frames.back().rows = m * (it.row_end - it.row_begin);
            }
        }
        if (frames.empty()) continue;
        int rc = render_frames(ctx, frames.data(), (int)frames.size(), (flags & GBRT_BATCH_GRAPH) != 0);
        if (rc != GBRT_OK) return rc;
    }
    return GBRT_OK;
}

GBRT_API int gbrt_ao_probe(gbrt_ctx* ctx, const gbrt_scene* scene, const gbrt_grid* grid, const double* pts,
                           const double* nrm, int64_t n, int32_t ao_samples, const gbrt_params* params,
                           float* out_visibility) {
    if (!ctx || !scene || !grid || !params || n < 0 || (n > 0 && (!pts || !nrm || !out_visibility)))
        return GBRT_EINVAL;
    if (n >= (1ll << 32)) return GBRT_EINVAL;
    if (ao_samples < 0 || ao_samples > GBRT_MAX_PROBE_SAMPLES) return GBRT_EINVAL;
    if (params->precision != GBRT_FP32 && params->precision != GBRT_FP64) return GBRT_EINVAL;
    if (!(params->eps >= 0) || !(params->ao_maxdist > 0)) return GBRT_EINVAL;
    if (grid->N != scene->S + scene->C || grid->device != scene->device || scene->device != ctx->device)
        return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    gbrt_camera cam;
    memset(&cam, 0, sizeof(cam));
    gbrt_lights lights;
    memset(&lights, 0, sizeof(lights));
    if (grid->dynamic) {
        // the probe takes the geometry by value: wait for the device-side rebuild
        int rc = grid_refresh_host(const_cast<gbrt_grid*>(grid));
        if (rc != GBRT_OK) return rc;
    }
    if (grid->dev.cells == nullptr) return GBRT_EINVAL;  // a grid left unusable by a failed rebuild
    FrameDev f = make_frame(scene, grid, &cam, 1, 1, ao_samples, &lights, params, nullptr, nullptr, nullptr);
    return launch_ao_probe(ctx, f, pts, nrm, n, out_visibility);
}

GBRT_API int gbrt_philox4x32_10(gbrt_ctx* ctx, const uint32_t* ctr, const uint32_t* key, int64_t n,
                                uint32_t* out) {
    if (!ctx || n < 0 || (n > 0 && (!ctr || !key || !out))) return GBRT_EINVAL;
    if (((uintptr_t)ctr & 15) || ((uintptr_t)out & 15) || ((uintptr_t)key & 7)) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GBRT_EDEVICE;
    return launch_philox(ctx, ctr, key, n, out);
}

GBRT_API int gbrt_set_tuning(gbrt_ctx* ctx, const gbrt_tuning* t) {
    if (!ctx || !t) return GBRT_EINVAL;
    if (t->tile_w <= 0 || t->tile_h <= 0 || t->tile_w * t->tile_h != 32) return GBRT_EINVAL;
    if (t->block < 32 || t->block > 256 || t->block % 32 != 0) return GBRT_EINVAL;
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32) return GBRT_EINVAL;
    if (t->refill < 1 || t->refill > 32) return GBRT_EINVAL;
    ctx->tuning = *t;
    return GBRT_OK;
}

GBRT_API int gbrt_get_tuning(const gbrt_ctx* ctx, gbrt_tuning* t) {
    if (!ctx || !t) return GBRT_EINVAL;
    *t = ctx->tuning;
    return GBRT_OK;
}

GBRT_API int gbrt_set_profiling(gbrt_ctx* ctx, int mode) {
    if (!ctx) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (mode && !ctx->ev[0]) {
        for (int k = 0; k < 5; ++k)
            if (cudaEventCreate(&ctx->ev[k]) != cudaSuccess) return GBRT_EDEVICE;
    }
    ctx->profiling = mode == 0 ? 0 : (mode == GBRT_PROFILE_AO_WALK ? GBRT_PROFILE_AO_WALK : GBRT_PROFILE_ALL);
    return GBRT_OK;
}

GBRT_API int gbrt_phase_times(gbrt_ctx* ctx, float ms[4]) {
    if (!ctx || !ms || !ctx->timed) return GBRT_EINVAL;
    DeviceGuard g(ctx->device);
    if (ctx->timed == GBRT_PROFILE_AO_WALK) {
        if (cudaEventSynchronize(ctx->ev[3]) != cudaSuccess) return GBRT_EDEVICE;
        ms[0] = ms[1] = ms[3] = -1.0f;
        return cudaEventElapsedTime(ms + 2, ctx->ev[2], ctx->ev[3]) == cudaSuccess ? GBRT_OK : GBRT_EDEVICE;
    }
    if (cudaEventSynchronize(ctx->ev[4]) != cudaSuccess) return GBRT_EDEVICE;
    for (int k = 0; k < 4; ++k)
        if (cudaEventElapsedTime(ms + k, ctx->ev[k], ctx->ev[k + 1]) != cudaSuccess) return GBRT_EDEVICE;
    return GBRT_OK;
}

GBRT_API int64_t gbrt_launch_count(const gbrt_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
