// Render kernels: primary ray -> nearest hit -> FP64 refinement -> AO shadow
// rays -> shading, one pixel per thread; plus the AO probe and raw Philox.
#include "gbrt_device.cuh"
#include "gbrt_internal.h"

namespace gbrt {

// Primary ray of pixel (i, j), in FP64 (both paths derive their ray from it).
__device__ __forceinline__ void primary_ray64(const FrameDev& f, int i, int j, V3<double>& o, V3<double>& d) {
    double u = f.half_w * (2.0 * ((double)i + 0.5) / (double)f.W - 1.0);
    double v = f.half_h * (1.0 - 2.0 * ((double)j + 0.5) / (double)f.H);
    V3<double> eye = ld3(f.eye), dir = ld3(f.dir), up = ld3(f.up), right = ld3(f.right);
    if (f.cam_kind == GBRT_CAMERA_ORTHO) {
        o = madd(madd(eye, u, right), v, up);
        d = normalized(dir);
    } else {
        o = eye;
        d = normalized(madd(madd(dir, u, right), v, up));
    }
}

// FP32 path: nearest hit in FP32 from the FP32 ray re-based at the grid entry
// (one FP64 point rounded once, so coordinates stay small relative to the
// scene), then the winner -- and a runner-up within a relative 1e-4 band --
// re-solved as an FP64 quadratic from the FP64 ray.
__device__ __forceinline__ bool nearest_fp32_refined(const FrameDev& f, V3<double> o64, V3<double> d64,
                                                     uint32_t& id, double& t64, bool& overflow) {
    const float inf = Num<float>::inf();
    V3<float> of = to_f(o64), df = to_f(d64);
    float te0, te1;
    if (!clip_grid<float>(f.grid, of, df, 0.0f, inf, te0, te1)) return false;
    V3<float> oe = to_f(madd(o64, (double)te0, d64));
    Nearest<float> h;
    if (!trace_nearest<float>(f.grid, f.scene, oe, df, 0.0f, inf, h, overflow)) return false;
    double ta = 0.0, tb = 0.0;
    bool ok1 = hit_object<double>(f.scene, h.id1, o64, d64, 0.0, Num<double>::inf(), ta);
    id = h.id1;
    t64 = ok1 ? ta : (double)te0 + (double)h.t1;  // FP64 disagrees only on grazing rays
    if (h.id2 != GBRT_MISS && (h.t2 - h.t1) <= 1e-4f * (h.t1 + te0)) {
        bool ok2 = hit_object<double>(f.scene, h.id2, o64, d64, 0.0, Num<double>::inf(), tb);
        if (ok2 && (!ok1 || tb < ta || (tb == ta && h.id2 < h.id1))) {
            id = h.id2;
            t64 = tb;
        }
    }
    return true;
}

template <int MODE>
__device__ __forceinline__ void render_pixel(const FrameDev& f, int i, int j, bool& overflow) {
    const uint32_t q = (uint32_t)j * (uint32_t)f.W + (uint32_t)i;
    V3<double> o64, d64;
    primary_ray64(f, i, j, o64, d64);
    uint32_t id = GBRT_MISS;
    double t64 = 0.0;
    bool hit;
    if (MODE == GBRT_FP32) {
        hit = nearest_fp32_refined(f, o64, d64, id, t64, overflow);
    } else {
        Nearest<double> h;
        hit = trace_nearest<double>(f.grid, f.scene, o64, d64, 0.0, Num<double>::inf(), h, overflow);
        id = h.id1;
        t64 = h.t1;
    }
    uint32_t vis = 0;
    if (MODE == GBRT_FP32) {
        float rgb[3] = {f.bg_f[0], f.bg_f[1], f.bg_f[2]};
        if (hit) {
            V3<double> p, n;
            reproject64(f.scene, id, o64, d64, t64, p, n);
            V3<float> nf = to_f(n);
            vis = ao_visible<float>(f, q, to_f(madd(p, f.eps, n)), nf, f.ao_maxdist_f, overflow);
            float V = f.spp > 0 ? (float)vis / (float)f.spp : 1.0f;
            shade<float>(f, id, nf, to_f(d64), V, rgb);
        }
        float* out = (float*)f.out_rgb + 3 * (size_t)q;
        out[0] = rgb[0];
        out[1] = rgb[1];
        out[2] = rgb[2];
    } else {
        double rgb[3] = {f.bg[0], f.bg[1], f.bg[2]};
        if (hit) {
            V3<double> p, n;
            reproject64(f.scene, id, o64, d64, t64, p, n);
            vis = ao_visible<double>(f, q, madd(p, f.eps, n), n, f.ao_maxdist, overflow);
            double V = f.spp > 0 ? (double)vis / (double)f.spp : 1.0;
            shade<double>(f, id, n, d64, V, rgb);
        }
        double* out = (double*)f.out_rgb + 3 * (size_t)q;
        out[0] = rgb[0];
        out[1] = rgb[1];
        out[2] = rgb[2];
    }
    if (f.out_ids) f.out_ids[q] = hit ? id : GBRT_MISS;
    if (f.out_vis) f.out_vis[q] = vis;
}

constexpr int TILE_W = 16, TILE_H = 8;

template <int MODE>
__global__ void __launch_bounds__(TILE_W* TILE_H) k_render_tiled(const __grid_constant__ FrameDev f, uint32_t* err) {
    int i = blockIdx.x * TILE_W + (threadIdx.x % TILE_W);
    int j = blockIdx.y * TILE_H + (threadIdx.x / TILE_W);
    if (i >= f.W || j >= f.H) return;
    bool overflow = false;
    render_pixel<MODE>(f, i, j, overflow);
    if (overflow) atomicOr(err, ERR_DDA_STEPS);
}

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

// ---------------------------------------------------------------- launchers

int launch_render(Ctx* ctx, const FrameDev& f) {
    dim3 grid((f.W + TILE_W - 1) / TILE_W, (f.H + TILE_H - 1) / TILE_H);
    if (f.precision == GBRT_FP32)
        k_render_tiled<GBRT_FP32><<<grid, TILE_W * TILE_H, 0, ctx->stream>>>(f, ctx->d_err);
    else
        k_render_tiled<GBRT_FP64><<<grid, TILE_W * TILE_H, 0, ctx->stream>>>(f, ctx->d_err);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GBRT_OK : GBRT_EDEVICE;
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

}  // namespace gbrt
