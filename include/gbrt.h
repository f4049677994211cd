/*
 * gbrt.h -- C ABI of the GB300 molecular ambient-occlusion ray tracer.
 *
 * The library renders molecular scenes of spheres (atoms) and open cylinders
 * (bonds) the way the paper's Tachyon runs do (Sec. 2: a given image size,
 * ambient occlusion on, lights rescaled by 0.3, a skylight of 1.0): one primary
 * ray per pixel, its nearest hit, Monte-Carlo ambient-occlusion shadow rays
 * from the hit point, then Phong shading under rescaled directional lights plus
 * an AO-weighted skylight. Rays walk a uniform grid built on the device (the
 * preprocessing phase of Table 5). Every step runs in CUDA kernels compiled for
 * sm_103a.
 *
 * Conventions for every entry point:
 *  - Return value: GBRT_OK (0) or a negative GBRT_E* code; nothing throws.
 *    gbrt_strerror() names a code. Invalid arguments are rejected with
 *    GBRT_EINVAL before any work is enqueued.
 *  - Pointers are device pointers unless the call's flags say
 *    GBRT_HOST_PTRS. Device pointers must be valid on the context's device.
 *  - Calls enqueue work on the context's stream (the caller's stream, e.g.
 *    the current PyTorch stream) and return without waiting, except where a
 *    call says it synchronises. Output buffers are owned by the caller and
 *    must stay alive until the stream reaches the work.
 *  - Scenes and grids are owned by the library until gbrt_scene_free /
 *    gbrt_grid_free. A context is used by one host thread at a time.
 *  - Kernel-side failures (a grid walk that exceeds its step bound, a
 *    device-side grid rebuild that outgrows its buffer) set a device error
 *    word; gbrt_sync() reports it (GBRT_ETRAVERSAL / GBRT_ECAPACITY) and
 *    clears it. No kernel waits on another: every work queue is a counter
 *    that only grows, so every kernel ends. The checked build of the
 *    library (libgbrt_checked.so) also tests every index that comes from
 *    data against its buffer and reports a stray one as GBRT_EBOUNDS.
 */
#ifndef GBRT_H
#define GBRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GBRT_API __attribute__((visibility("default")))
#else
#define GBRT_API
#endif

/* 4: host-output copies run on a stream of the context's own (complete at
 *    gbrt_sync); a grid must belong to the rendered scene. */
#define GBRT_VERSION 4

/* ---- error codes ---- */
#define GBRT_OK 0
#define GBRT_EINVAL (-1)      /* invalid argument or scene data */
#define GBRT_ENOMEM (-2)      /* device or pinned allocation failed */
#define GBRT_EDEVICE (-3)     /* CUDA runtime error / no device */
#define GBRT_ETIMEDOUT (-4)   /* reserved: a bounded device wait ran out (no kernel of this version waits) */
#define GBRT_ETRAVERSAL (-5)  /* a grid walk exceeded its step bound */
#define GBRT_ECAPACITY (-6)   /* a device-side grid rebuild outgrew its buffer */
#define GBRT_EBOUNDS (-7)     /* an index outside its buffer (reported by the checked build only) */

/* ---- flags ---- */
#define GBRT_DEVICE_PTRS 0
#define GBRT_HOST_PTRS 1      /* array arguments are host memory */
#define GBRT_HOST_ASYNC 4     /* with GBRT_HOST_PTRS: host outputs are filled asynchronously */
#define GBRT_BATCH_GRAPH 2    /* gbrt_render_batch: replay through a CUDA graph */

/* ---- precision ---- */
#define GBRT_FP32 0  /* FP32 traversal, intersection and shading; float-float ray, hit refined in its object's frame */
#define GBRT_FP64 1  /* FP64 throughout (the paper's all-double-precision build, Sec. 2) */

#define GBRT_CAMERA_ORTHO 0
#define GBRT_CAMERA_PINHOLE 1
#define GBRT_MAX_LIGHTS 8
#define GBRT_MISS 0xFFFFFFFFu    /* hit id of a pixel whose ray hits nothing */
#define GBRT_MAX_SAMPLES 4096    /* ao_samples bound of a render */
#define GBRT_MAX_PROBE_SAMPLES (1 << 20) /* ao_samples bound of gbrt_ao_probe */
#define GBRT_MAX_DIM 65536       /* width/height bound; width*height < 2^31 */
#define GBRT_MAX_AA 4            /* largest sub-pixel grid side (camera.aa) */

typedef struct gbrt_ctx gbrt_ctx;
typedef struct gbrt_scene gbrt_scene;
typedef struct gbrt_grid gbrt_grid;

/* Camera. Pixel (i, j) -- column i, row j, row 0 at the top -- uses
 *   u = half_w (2 (i + 0.5)/W - 1),  v = half_h (1 - 2 (j + 0.5)/H).
 * Ortho: ray origin eye + u right + v up, direction dir.
 * Pinhole: origin eye, direction normalize(dir + u right + v up).
 * dir, up, right: unit and mutually orthogonal.
 * aa: supersampling, an addition to the paper's one ray per pixel. 0 or 1:
 *   one ray through the pixel centre. m = 2..GBRT_MAX_AA: m x m rays through
 *   (i + (a + 0.5)/m, j + (b + 0.5)/m), a, b = 0..m-1 -- the pixel centres of
 *   the m-times finer raster of (m W) x (m H) pixels -- and the pixel's colour
 *   is the mean of their (clamped) colours. Sub-sample (a, b) draws its AO
 *   samples with counter word 0 = its finer-raster index
 *   (m j + b) (m W) + (m i + a); hit ids and AO counts are reported per
 *   sub-sample in that finer raster. (m W) (m H) must stay below 2^31. */
typedef struct gbrt_camera {
    int32_t kind;
    int32_t aa;
    double eye[3];
    double dir[3];
    double up[3];
    double right[3];
    double half_w;
    double half_h;
} gbrt_camera;

/* Directional lights: dir[l] is the unit vector toward light l. Every light's
 * intensity is multiplied by `scale` (tachyon -rescale_lights, Sec. 2); the
 * skylight (tachyon -add_skylight, Sec. 2) weights the AO term. */
typedef struct gbrt_lights {
    int32_t n;
    int32_t reserved;
    double dir[GBRT_MAX_LIGHTS][3];
    double intensity[GBRT_MAX_LIGHTS];
    double scale;
    double skylight;
} gbrt_lights;

/* Per-frame parameters.
 *  precision   GBRT_FP32 | GBRT_FP64
 *  seed, frame Philox4x32-10 key = (seed low word, seed high word); the AO
 *              sample s of pixel q uses counter (q, s, frame, 0xA0) and the
 *              24-bit fractions of output words 0 and 1
 *  eps         AO rays start at the re-projected hit point + eps * normal
 *  ao_maxdist  AO rays count hits with 0 < t <= ao_maxdist (may be +inf)
 *  k_ao, k_d, k_s, phong_exp  material: colour =
 *      clamp01(albedo (skylight k_ao V + sum_l scale I_l k_d max(0, n.l))
 *              + sum_{l: n.l > 0} scale I_l k_s max(0, r_l.v)^phong_exp)
 *      with V the fraction of AO samples that escape (V = 1 when
 *      ao_samples = 0), r_l the mirror of l about n, v = -ray direction
 *  background  colour of pixels whose primary ray hits nothing
 *  shadows     1: direct-light shadow rays -- from the AO origin, one ray per
 *              light the surface faces; any hit (0 < t) drops that light's
 *              diffuse and specular terms. 0: lights are never blocked
 *  out_flags   GBRT_HOST_PTRS: the render's output pointers are host memory
 *              (the call then synchronises). GBRT_HOST_PTRS | GBRT_HOST_ASYNC:
 *              host outputs too, but the call returns once the copies are
 *              enqueued; the outputs are complete, and device-side errors
 *              reported, at the next gbrt_sync (a synchronisation of the
 *              caller's stream alone does not cover the copies). The render
 *              goes into one of two device staging buffers of the context,
 *              used in turn, and the copies run on a stream of the context's
 *              own once its kernels are done, so one frame's copy overlaps the
 *              next frame's work; page-locked host memory makes them truly
 *              asynchronous. A stream of frames thus runs without a host round
 *              trip per frame. */
typedef struct gbrt_params {
    int32_t precision;
    int32_t out_flags;
    uint64_t seed;
    uint32_t frame;
    int32_t shadows;
    double eps;
    double ao_maxdist;
    double k_ao;
    double k_d;
    double k_s;
    double phong_exp;
    double background[3];
} gbrt_params;

/* One frame -- or a band of rows of one frame -- in a batch
 * (gbrt_render_batch). Fields as for gbrt_render, plus:
 *  row_begin, row_end  render only rows [row_begin, row_end) of the
 *              width x height image (0, 0 = all rows). Pixels keep their
 *              whole-image coordinates and sample counters, so the band's
 *              pixels are exactly those of the whole-frame render; outputs
 *              are the whole-image buffers and only the band's rows are
 *              written. */
typedef struct gbrt_render_item {
    const gbrt_scene* scene;
    const gbrt_grid* grid;
    gbrt_camera camera;
    int32_t width;
    int32_t height;
    int32_t ao_samples;
    int32_t reserved;
    int32_t row_begin;
    int32_t row_end;
    gbrt_lights lights;
    gbrt_params params;
    void* out_rgb;
    uint32_t* out_hit_ids;
    uint32_t* out_ao_visible;
} gbrt_render_item;

/* Launch shape of the render kernels, chosen by the autotuner.
 *  tile_w x tile_h  pixels of one primary-ray work item (a warp); the product
 *                   must be 32
 *  block            threads per CTA of the persistent kernels (multiple of
 *                   32, <= 256)
 *  ctas_per_sm      resident CTAs per SM of the persistent launches (0 = as
 *                   many as fit)
 *  refill           AO lanes: a warp refills its idle lanes with new shadow
 *                   rays (ballot + popc compaction) once fewer than `refill`
 *                   of its 32 lanes still hold a ray (1..32) */
typedef struct gbrt_tuning {
    int32_t tile_w;
    int32_t tile_h;
    int32_t block;
    int32_t ctas_per_sm;
    int32_t refill;
    int32_t reserved[3];
} gbrt_tuning;

/* Library version (GBRT_VERSION). Host only; needs no device. */
GBRT_API int gbrt_version(void);

/* Static string naming an error code. Host only; needs no device. */
GBRT_API const char* gbrt_strerror(int code);

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream; owned by the caller).
 * Allocates the context's device error word. GBRT_EDEVICE without a device. */
GBRT_API int gbrt_create(gbrt_ctx** out, int device, void* cuda_stream);

/* Change the stream later calls enqueue on. */
GBRT_API int gbrt_set_stream(gbrt_ctx* ctx, void* cuda_stream);

/* Wait for the context's stream, then read and clear the device error word. */
GBRT_API int gbrt_sync(gbrt_ctx* ctx);

/* Destroy a context (synchronises its stream first). Scenes and grids must be
 * freed before. NULL is accepted. */
GBRT_API int gbrt_destroy(gbrt_ctx* ctx);

/* Upload a scene (Sec. 2: the molecular model of spheres and cylinders).
 *  spheres    float32 [S][4]  centre x y z, radius > 0
 *  cylinders  float32 [C][7]  end p0 x y z, end p1 x y z, radius > 0, p0 != p1
 *             (open tubes: no end caps)
 *  color_idx  uint32 [S + C]  palette entry of each object, < K; objects are
 *             numbered spheres 0..S-1 then cylinders S..S+C-1 (global ids)
 *  palette    float32 [K][3]  linear RGB albedo
 *  flags      GBRT_HOST_PTRS if the four arrays are host memory
 * The library copies the data into its own device layout (float4 sphere and
 * cylinder records, FP64 copies for the hit refinement) and computes the scene
 * box. S or C may be 0 (an empty scene renders background). Synchronises.
 * GBRT_EINVAL on non-finite values, radius <= 0, zero-length cylinders or a
 * colour index >= K. */
GBRT_API int gbrt_scene_upload(gbrt_ctx* ctx, const float* spheres, int64_t n_spheres, const float* cylinders,
                               int64_t n_cylinders, const uint32_t* color_idx, const float* palette,
                               int32_t n_palette, int flags, gbrt_scene** out);

/* Scene size in bytes on the device, and object counts (host only). */
GBRT_API int gbrt_scene_info(const gbrt_scene* scene, int64_t* n_spheres, int64_t* n_cylinders,
                             int64_t* device_bytes);

GBRT_API int gbrt_scene_free(gbrt_ctx* ctx, gbrt_scene* scene);

/* Build the uniform grid (Table 5 "Preprocess"): about lambda * (S + C) cells
 * over the scene box (lambda <= 0 selects 2.0); each object is listed in every
 * cell its padded bounding box overlaps, ids ascending within a cell
 * (counting sort: count, exclusive scan, scatter, per-cell sort). Synchronises
 * (the reference count sizes the item array). */
GBRT_API int gbrt_grid_build(gbrt_ctx* ctx, const gbrt_scene* scene, float lambda, gbrt_grid** out);

/* Grid geometry: cells per axis, padded box, total references. Host only for
 * a grid built by gbrt_grid_build; for a grid rebuilt on the device it first
 * waits for the last rebuild's stream. */
GBRT_API int gbrt_grid_info(const gbrt_grid* grid, int32_t dims[3], float lo[3], float hi[3], int64_t* refs,
                            int64_t* device_bytes);

GBRT_API int gbrt_grid_free(gbrt_ctx* ctx, gbrt_grid* grid);

/* Animated scenes (molecular-dynamics frames) -- an addition to the paper,
 * which renders one static scene (its grid build is the "Preprocess" phase
 * of Table 5). The two calls below replace that preprocess per frame without
 * a host round trip, so the GPU can run a frame's rebuild right after the
 * previous frame's render.
 *
 * gbrt_scene_update: new geometry for a resident scene -- sphere and
 * cylinder arrays of the scene's own S and C, layouts as for
 * gbrt_scene_upload; colours and palette stay. Asynchronous on the context's
 * stream. Host arrays (flags GBRT_HOST_PTRS) are checked before any launch
 * (GBRT_EINVAL) and copied through a staging buffer the scene allocates on
 * its first update; page-locked host arrays are read asynchronously, so keep
 * them unchanged until the stream has passed the copy. Device arrays are
 * checked on the device: a bad value makes the next gbrt_sync return
 * GBRT_EINVAL, and the scene's geometry is then unspecified until the next
 * good update. Grids built on the scene keep their contents until
 * gbrt_grid_rebuild. */
GBRT_API int gbrt_scene_update(gbrt_ctx* ctx, gbrt_scene* scene, const float* spheres, const float* cylinders,
                               int flags);

/* gbrt_grid_rebuild: rebuild `grid` on the device for `scene`'s current
 * geometry (the scene it was built for: same object count, else
 * GBRT_EINVAL) with the grid's own cells-per-object density: scene box ->
 * cells per axis -> count -> exclusive scan -> scatter -> bounding sphere,
 * all on the context's stream; renders enqueued after it use the new grid.
 * The ids of a cell stay in scatter order (a host build sorts them; no
 * render result depends on the order). The first call allocates buffers with headroom (cells
 * for 1.5x the target count, items for 1.5x the current references) and
 * waits for the stream once; later calls neither allocate nor wait, except
 * that a call which finds, from an earlier finished rebuild, that the items
 * came within 1/8 of the buffer grows it (and waits). A rebuild whose
 * references exceed the item buffer leaves the grid empty (renders then see
 * no objects) and makes the next gbrt_sync return GBRT_ECAPACITY; the next
 * rebuild after that sync grows the buffer. */
GBRT_API int gbrt_grid_rebuild(gbrt_ctx* ctx, gbrt_grid* grid, const gbrt_scene* scene);

/* Render one frame (Sec. 2's tachyon run: -res width height, AO with
 * ao_samples Monte-Carlo samples per pixel, lights, skylight).
 *  out_rgb         [height][width][3], float32 for GBRT_FP32, float64 for GBRT_FP64
 *  out_hit_ids     optional uint32 [height][width]: nearest object id, GBRT_MISS
 *  out_ao_visible  optional uint32 [height][width]: AO samples that escaped
 * With supersampling (camera->aa = m > 1) out_hit_ids and out_ao_visible hold
 * one entry per sub-sample, [m height][m width] (the finer raster), and the
 * library keeps the finer raster's colours in a context buffer
 * (m^2 width height x 3 values) that it box-filters into out_rgb.
 * Output pointers are device memory unless params->out_flags has
 * GBRT_HOST_PTRS, in which case the library renders into one of its two
 * device staging buffers and copies back (then synchronises unless
 * GBRT_HOST_ASYNC is set). Asynchronous otherwise. The grid must have been
 * built for this scene (same object count) and both must live on the
 * context's device: GBRT_EINVAL otherwise, before any work is enqueued. */
GBRT_API int gbrt_render(gbrt_ctx* ctx, const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* camera,
                         int32_t width, int32_t height, int32_t ao_samples, const gbrt_lights* lights,
                         const gbrt_params* params, void* out_rgb, uint32_t* out_hit_ids,
                         uint32_t* out_ao_visible);

/* Render n frames of uneven size through one persistent launch that drains a
 * device queue of (frame, tile) work items. Each item is rendered exactly as
 * gbrt_render would render it alone. Items' output pointers are device memory.
 * flags: GBRT_BATCH_GRAPH replays the upload + launch through a CUDA graph
 * captured on first use for this batch size. Asynchronous. */
GBRT_API int gbrt_render_batch(gbrt_ctx* ctx, const gbrt_render_item* items, int32_t n, int flags);

/* AO visibility of explicit points (Sec. 2's Monte-Carlo sampling of
 * illumination, as a probe): for point k, `ao_samples` cosine-weighted rays
 * from pts[k] + eps * nrm[k] with Philox counter (k, s, frame, 0xA0);
 * out_visibility[k] = escaped / ao_samples. pts, nrm: float64 [n][3] device,
 * nrm unit; ao_samples <= GBRT_MAX_PROBE_SAMPLES. Uses params precision,
 * seed, frame, eps and ao_maxdist. Async. */
GBRT_API int gbrt_ao_probe(gbrt_ctx* ctx, const gbrt_scene* scene, const gbrt_grid* grid, const double* pts,
                           const double* nrm, int64_t n, int32_t ao_samples, const gbrt_params* params,
                           float* out_visibility);

/* Raw Philox4x32-10 blocks (the AO sampler's generator): out[k] =
 * Philox(counter ctr[k] (4 words), key key[k] (2 words)). Device arrays,
 * uint32 [n][4], [n][2], [n][4]. Async. */
GBRT_API int gbrt_philox4x32_10(gbrt_ctx* ctx, const uint32_t* ctr, const uint32_t* key, int64_t n,
                                uint32_t* out);

/* Render one frame without allocating anything (no counterpart in the paper:
 * this entry point exists for the library's users).
 *
 * Some callers cannot allocate device memory at render time: a host
 * application whose own allocator has reserved all free device memory (a
 * cudaMalloc here would fail or fragment it), or a latency-critical loop that
 * must not call cudaMalloc/cudaFree (cudaFree synchronises the device).
 * gbrt_render allocates its working buffers in the context on first use;
 * this variant instead keeps them in one fixed device array of about 4.5 MB
 * inside the library, which every GPU that loads the library holds until the
 * process exits. It needs no context: the caller passes the scene and grid
 * (prepared earlier), the outputs (device memory) and the stream to use.
 *
 *  - width * height must not exceed GBRT_NOALLOC_MAX_PIXELS (256 x 256);
 *    larger frames are rejected with GBRT_EINVAL, as are host output
 *    pointers (params->out_flags must be 0) and supersampling
 *    (camera->aa > 1).
 *  - The first call on a device does that device's set-up: it looks up the
 *    array's device address and configures the kernels, both synchronous
 *    runtime calls.
 *  - All calls share the one array and it keeps the last call's contents;
 *    the call clears what must start at zero. Calls whose work overlaps on
 *    the GPU (different streams, or different host threads) race on it:
 *    order them on one stream.
 *  - The scene and grid are read on `cuda_stream`, not on the stream of the
 *    context that made them. After gbrt_scene_update or gbrt_grid_rebuild
 *    (asynchronous on the context's stream) the caller must order
 *    `cuda_stream` after that stream -- gbrt_sync on the context, or an event
 *    recorded there that `cuda_stream` waits on -- before this call, else it
 *    may read half-written geometry or cells.
 *  - The set-up is kept for the life of the process: after a reset of the
 *    device (cudaDeviceReset) the library must not be used again.
 *  - A CUDA error already pending in the calling thread (from the caller's
 *    earlier work) makes the call return GBRT_EDEVICE with nothing enqueued;
 *    the error stays pending for the caller.
 *  - Arguments as for gbrt_render; output buffers are caller-owned.
 *    Asynchronous on `cuda_stream`. Device-side walk-bound errors are not
 *    reported by this entry point. */
#define GBRT_NOALLOC_MAX_PIXELS 65536
GBRT_API int gbrt_render_noalloc(const gbrt_scene* scene, const gbrt_grid* grid, const gbrt_camera* camera,
                                 int32_t width, int32_t height, int32_t ao_samples, const gbrt_lights* lights,
                                 const gbrt_params* params, void* out_rgb, uint32_t* out_hit_ids,
                                 uint32_t* out_ao_visible, void* cuda_stream);

/* Kernel launch shape used by later renders (see gbrt_tuning). */
GBRT_API int gbrt_set_tuning(gbrt_ctx* ctx, const gbrt_tuning* tuning);
GBRT_API int gbrt_get_tuning(const gbrt_ctx* ctx, gbrt_tuning* tuning);

/* Per-kernel timing (phase timers). mode 0: off. GBRT_PROFILE_ALL (or any
 * other non-zero value): renders record CUDA events between all their kernels
 * on the context's stream. GBRT_PROFILE_AO_WALK: events only just before and
 * after the AO shadow-ray walk -- each event between two kernels costs a few
 * microseconds and the overlap of the dependent launch, so this mode times
 * the dominant kernel with the least disturbance. Renders replayed from a
 * CUDA graph are not timed. */
#define GBRT_PROFILE_ALL 1
#define GBRT_PROFILE_AO_WALK 2
GBRT_API int gbrt_set_profiling(gbrt_ctx* ctx, int mode);

/* Device time in ms of the last timed render's kernels: [0] primary walk and
 * refinement (its last CTA also lays out the AO pass), [1] 0 (the AO plan has
 * no kernel of its own), [2] AO shadow-ray walk, [3] shading; under
 * GBRT_PROFILE_AO_WALK only [2] is measured and the others are -1. Waits for
 * that render. GBRT_EINVAL if no render was timed. */
GBRT_API int gbrt_phase_times(gbrt_ctx* ctx, float ms[4]);

/* Micro-benchmarks of the GPU the context runs on (not part of the paper's
 * method: they calibrate the roofline the render kernels are compared with),
 * timed with CUDA events on the context's stream at whatever clock the GPU
 * runs; synchronises. *value receives
 *   GBRT_MB_FP32_FMA  FP32 fused multiply-add rate, TFLOP/s (2 flop per FMA)
 *   GBRT_MB_FP64_FMA  FP64 fused multiply-add rate, TFLOP/s
 *   GBRT_MB_L2_READ   read bandwidth of a buffer of half the L2's size, GB/s
 * GBRT_EINVAL for another kind; allocates (and frees) its own buffer. */
#define GBRT_MB_FP32_FMA 0
#define GBRT_MB_FP64_FMA 1
#define GBRT_MB_L2_READ 2
GBRT_API int gbrt_microbench(gbrt_ctx* ctx, int kind, double* value);

/* Number of kernels this context has launched so far (host counter). */
GBRT_API int64_t gbrt_launch_count(const gbrt_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GBRT_H */
