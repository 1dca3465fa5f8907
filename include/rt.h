/*
 * rt.h -- C ABI of the B300 (sm_103a) per-pixel Whitted ray tracer of
 * "Accelerating Java Ray Tracing Applications on Heterogeneous Hardware"
 * (arXiv 2305.07450, Section 3).
 *
 * The paper's accelerated method is one call, Renderer::render(pixels, dimensions,
 * camera, rayTracingProperties, bodyPositions, bodySizes, bodyColors,
 * bodyReflectivities, skybox, skyboxDimensions) (Section 3.9, render signature
 * listing), fed by a task schedule that streams the camera, the properties and the
 * body positions in every frame and streams the pixels out (Section 3.9, task
 * schedule listing).  Here that split becomes: upload the scene once
 * (rt_scene_upload / rt_scene_update), then render as often as wanted (rt_render);
 * the framebuffer stays on the device.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers; every other pointer is a host
 *    pointer that the call reads before it returns (the caller keeps ownership).
 *  - The caller owns every output, hit-record, gradient and workspace buffer; the
 *    library owns the memory behind an rt_scene handle.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously on it; the call returns once it is enqueued.
 *  - Arguments are validated on the host before any launch; an invalid argument
 *    returns RT_ERR_INVALID_ARG and enqueues nothing.  Launch failures are mapped
 *    from cudaGetLastError to RT_ERR_CUDA.  Nothing aborts, throws or traps.
 *  - Waits inside kernels are bounded; a wait that gives up sets a device error
 *    word instead of hanging, which rt_device_errors() reports.
 *  - FP32 arithmetic on the device; all records are FP32.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,   /* a null pointer, size, format or record out of range */
    RT_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed                 */
    RT_ERR_OOM = 3,           /* device or pinned host allocation failed              */
    RT_ERR_UNSUPPORTED = 4,   /* valid input outside what the library handles         */
    RT_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (see rt_device_errors) */
    RT_ERR_EXCEEDS_SCRATCH = 6 /* the work does not fit the fixed scratch of
                                  rt_render_batch_noalloc                             */
} rt_status;

enum { RT_PHONG = 0, RT_BLINN_PHONG = 1 };          /* Section 3.5.1 / 3.5.2           */
enum { RT_OUT_RGBA8 = 0, RT_OUT_F32 = 1 };          /* toInt of Section 3.9 / linear   */

#define RT_SPHERE_FIELDS 10
#define RT_PLANE_FIELDS 10
#define RT_LIGHT_FIELDS 8
#define RT_MAX_LIGHTS 16
#define RT_MAX_SAMPLES 1024
#define RT_MAX_DEPTH 16

/* Scene records (Section 3.4 object table: position, size, colour, reflectivity;
 * widened by the material fields the shading of Section 3.5 needs).
 *   sphere [10]: cx, cy, cz, radius, albedo r, g, b, k_s, spec_exp, reflectivity
 *   plane  [10]: nx, ny, nz, d (n.x + d = 0, |n| = 1), albedo r, g, b, k_s,
 *                spec_exp, reflectivity
 *   light  [8] : x, y, z, intensity, area_side (> 0: horizontal square light of
 *                that side, sampled on a stratified grid), sphere_radius (> 0:
 *                spherical light sampled with sunflower points, Section 3.6.1),
 *                0, 0.  Both zero = point light.
 * Reflectivity is the reflection ratio of Section 3.7 in [0, 1].  The ground plane
 * is optional (has_plane), infinite and two-sided.  Pointers are host pointers for
 * rt_scene_upload; for rt_scene_update they are host or device pointers as the
 * caller states.  Lights must lie outside every sphere (RT_ERR_UNSUPPORTED
 * otherwise): the device's shadow test relies on it. */
typedef struct {
    int32_t n_spheres;
    const float *spheres;     /* [n_spheres][10] */
    int32_t has_plane;
    const float *plane;       /* [10], may be NULL when has_plane == 0 */
    int32_t n_lights;         /* 0 .. RT_MAX_LIGHTS */
    const float *lights;      /* [n_lights][8] */
} rt_scene_desc;

/* The paper's camera float[6] (Section 3.1, Section 3.9): position, yaw and pitch
 * in degrees (pitch about x first, positive looks up; then yaw about y, positive
 * turns toward +x), field of view in degrees spanning the shorter image side. */
typedef struct {
    float pos[3];
    float yaw_deg, pitch_deg, fov_deg;
} rt_camera;

/* The paper's dimensions int[2] and rayTracingProperties int[2] (Section 3.9:
 * shadow sample size, reflection bounce limit), plus the choices the paper leaves
 * open. */
typedef struct {
    int32_t width, height;    /* 1 .. 32768 each                                      */
    int32_t max_depth;        /* reflection bounce limit D, 0 .. RT_MAX_DEPTH          */
    int32_t shadow_samples;   /* samples per sampled light, 1 .. RT_MAX_SAMPLES; a
                                 perfect square when a square area light is present   */
    int32_t shading_model;    /* RT_PHONG or RT_BLINN_PHONG                            */
    int32_t out_format;       /* RT_OUT_RGBA8 (uint32 0xAABBGGRR) or RT_OUT_F32
                                 (float RGBA, A = 1, linear, not clamped)             */
    float ambient;            /* ambient strength k_a in [0, 1] (Section 3.5.1)        */
    float eps;                /* offset of secondary ray origins along the normal     */
    int32_t refl_coupled;     /* 0: reflection ratio = the reflectivity field;  1: the
                                 paper's coupling (Section 3.7): ratio = spec_exp /
                                 max_reflectivity, clamped to 1 (forward only)        */
    float max_reflectivity;   /* MAX_REFLECTIVITY of the coupling (> 0 when coupled)   */
    uint64_t seed;            /* Philox4x32-10 key of the area-light samples           */
} rt_render_params;

/* Launch shape of the render kernels.  A zeroed struct (or NULL) means "library
 * default".  Threads of a CTA form block_x * block_y pixels; each warp covers an
 * 8 x 4 pixel patch.  staging: 0 = default, 1 = one TMA bulk copy of the scene
 * table into shared memory, 2 = cooperative copy by all threads, 3 = the tiled
 * loop (each warp streams the sphere table through its own shared-memory slot;
 * taken anyway when the table does not fit).  accel: 0 = brute force over the
 * spheres (the paper's method), 1 = the scene's bounding-volume hierarchy
 * (rt_scene_build_bvh; rt_render and rt_render_region only, staging 1 or 2).
 * Every choice gives the same results bit for bit. */
typedef struct {
    int32_t block_x, block_y; /* multiples of 8 and 4, block_x * block_y in 32..256 */
    int32_t staging;
    int32_t min_blocks_per_sm;/* occupancy hint for the batch kernel's grid size     */
    int32_t accel;            /* 0 brute force, 1 bounding-volume hierarchy          */
} rt_launch_config;

typedef struct rt_scene rt_scene;   /* opaque, device-resident */

/* Copy a scene to the device (Section 3.9: the body arrays streamed in).  Validates
 * every record; enqueues one host-to-device copy on `stream` from a pinned staging
 * buffer owned by the handle.  *out receives a new handle (free with rt_scene_free).
 * Errors: RT_ERR_INVALID_ARG (null pointers, counts, non-finite or out-of-range
 * fields), RT_ERR_UNSUPPORTED (a light inside a sphere), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_scene_upload(const rt_scene_desc *desc, void *stream, rt_scene **out);

/* Overwrite the contents of a scene in place with a description of the same
 * counts (the paper's per-frame streamIn of the body positions; also the
 * parameter update of inverse rendering).  desc_on_device != 0: the three record
 * pointers are device pointers, copied device-to-device without host validation.
 * Counts must match the handle's (RT_ERR_INVALID_ARG otherwise). */
rt_status rt_scene_update(rt_scene *scene, const rt_scene_desc *desc, int32_t desc_on_device,
                          void *stream);

/* Release a scene's device and pinned memory (synchronises the device first).
 * NULL is accepted. */
rt_status rt_scene_free(rt_scene *scene);

/* ---------------------------------------------------------------- sky and physics
 * The paper's additional components (Section 3.8): an HDR sky panorama shown by
 * rays that leave the scene, and a Verlet physics system that moves the bodies
 * between frames (their positions are streamed in every frame, Section 3.9).  The
 * paper's sky image is not available; any panorama can be given. */

/* Give the scene a sky panorama, or remove it (texels NULL: misses are black).
 *   texels: host array of height rows (the first row is straight up) of width RGBA
 *           FP32 texels (A ignored), copied to the device before the call returns
 *           (width, height in 1..16384; every value finite).
 * A ray that leaves the scene at bounce k adds T_k sky(d) with the equirectangular
 * UV mapping u = 1/2 + atan2(d_z, d_x) / (2 pi), v = 1/2 - asin(d_y) / pi and
 * bilinear interpolation between texel centres, wrapping in u, clamped in v.
 * Removing or resizing a sky synchronises the device.  rt_render_backward refuses
 * scenes with a sky (RT_ERR_UNSUPPORTED). */
rt_status rt_scene_set_sky(rt_scene *scene, const float *texels, int32_t width, int32_t height, void *stream);

/* Advance n bodies by `steps` steps of position Verlet integration under gravity
 * (0, -gravity, 0) with time step dt (one kernel launch on `stream`):
 *   x' = x + (x - x_prev) + a dt^2;
 * with a ground plane (plane: host [4] = nx, ny, nz, d of n.x + d = 0, |n| = 1; or
 * NULL for none) a sphere that crosses it is moved back along n until it touches
 * it, and the step's velocity component into the plane is dropped when it is at
 * most 2 gravity dt^2 (resting contact), else reversed and scaled by restitution
 * (0..1).
 *   spheres_dev: device sphere records [n][10] (the rt_scene_desc layout); centres
 *                (fields 0..2) are read and updated in place, radii (field 3) read.
 *   prev_dev:    device [n][3] previous centres, updated in place.
 * Feed the records to rt_scene_update(desc_on_device = 1) to render the new frame.
 * Errors: RT_ERR_INVALID_ARG (counts, pointers, dt <= 0, restitution outside
 * [0, 1], a non-unit plane normal). */
rt_status rt_verlet_step(float *spheres_dev, float *prev_dev, int32_t n, const float *plane, float dt,
                         float gravity, float restitution, int32_t steps, void *stream);

/* ---------------------------------------------------------------- hierarchy
 * Bounding-volume hierarchy over the spheres: the spatial acceleration structure
 * the paper names as future work (Section 6); the paper's own kernel tests every
 * sphere (Section 3.4.1).  Rendering with it (rt_launch_config.accel = 1) gives
 * the brute-force images bit for bit: the same per-sphere arithmetic, ties to the
 * lower index, and boxes widened per ray beyond the FP32 error of both tests.
 * Built on the host by binned surface-area splits (leaves of at most 8 spheres,
 * depth at most 44), from the sphere table as the device holds it. */
typedef struct {
    int32_t n_nodes;          /* interior nodes (64 bytes each); 0 for no spheres   */
    int32_t depth;            /* deepest leaf (root = 0)                           */
    int32_t max_leaf;         /* most spheres in one leaf                          */
    float r_scene;            /* max over spheres of max(|cx|, |cy|, |cz|) + r     */
} rt_bvh_info;

/* Build (or rebuild) the scene's hierarchy from the contents last given on the
 * host (rt_scene_upload or a host-side rt_scene_update) and enqueue its copy to
 * the device on `stream`.  A host-side rt_scene_update of a scene that has a
 * hierarchy rebuilds it; a device-side update (desc_on_device) leaves it stale,
 * and accel renders then return RT_ERR_UNSUPPORTED until a host-side update.
 * Scenes whose coordinates reach 1e15 are refused (RT_ERR_UNSUPPORTED).
 * info (nullable) receives the hierarchy's figures. */
rt_status rt_scene_build_bvh(rt_scene *scene, void *stream, rt_bvh_info *info);

/* Host-only build of the same hierarchy for inspection (no device, no CUDA call):
 * the records of `desc` as rt_scene_upload takes them (validated the same way).
 *   nodes:    NULL, or room for nodes_cap 64-byte nodes: for each node the two
 *             children's boxes as floats (a.lo xyz, a.hi xyz, b.lo xyz, b.hi xyz)
 *             then int32 references a, b and two zero words; a reference r >= 0
 *             is node r, r < 0 a leaf of the (((-1 - r) & 15) + 1) spheres listed
 *             at prim_idx[(-1 - r) >> 4 ...]; an empty child has lo > hi.
 *   prim_idx: NULL, or room for n_spheres int32 sphere indices.
 * RT_ERR_INVALID_ARG when nodes_cap is below the node count (reported in info). */
rt_status rt_bvh_build_host(const rt_scene_desc *desc, void *nodes, int32_t nodes_cap, int32_t *prim_idx,
                            rt_bvh_info *info);

/* Render one frame: for every pixel (x, y) a primary ray through its NDC point
 * (Section 3.2, 3.3), the closest of all primitives by brute force (Section
 * 3.4.1; or through the hierarchy when cfg->accel = 1, same result), ambient + per-light diffuse and specular shading with hard or sampled
 * shadows (Sections 3.5, 3.6), reflection bounces to depth D (Section 3.7) and the
 * colour written to the framebuffer (Section 3.9 render listing).
 *   out_dev: device buffer of `height` rows, `out_pitch_bytes` apart (a multiple
 *            of 16, >= width * 4 for RGBA8 or width * 16 for F32); row y holds
 *            pixel x at byte offset x * 4 (RGBA8) or x * 16 (F32 RGBA).
 *   hitrec_dev: NULL, or a device buffer of rt_hitrec_bytes() bytes that receives
 *            the per-pixel hit record used by rt_render_backward.
 *   cfg:     launch shape (NULL = default).
 * One kernel launch on `stream`. */
rt_status rt_render(const rt_scene *scene, const rt_camera *cam, const rt_render_params *params,
                    void *out_dev, size_t out_pitch_bytes, void *hitrec_dev,
                    const rt_launch_config *cfg, void *stream);

/* Device workspace bytes rt_render_ws suggests for this frame (256-byte aligned
 * buffer): a 256-byte control block and two path queues of ceil(W*H/4) entries of
 * 64 bytes each (about 133 bytes per 4 pixels; 265 MB at 3840x2160).  0 on
 * invalid arguments. */
size_t rt_render_workspace_bytes(const rt_scene *scene, const rt_render_params *params);

/* Render one frame as rt_render does -- the same arguments, and every pixel and
 * hit-record entry bit for bit the same -- in passes over compacted paths, using
 * the caller's workspace (no allocation).  A warp of the one-pass kernel runs the
 * bounce loop until its slowest lane is done, so a few pixels whose reflections
 * keep hitting idle the rest of their warp; here persistent warps trace every
 * pixel's primary ray, its shading and its bounce-1 ray, and hand the paths whose
 * bounce-1 ray hits to a queue; pass k (k = 1..D) then shades the queued bounce-k
 * hits 32 per warp and queues those whose next ray hits again.  Not in the paper
 * (an execution strategy of its Section 3.7 recursion).
 *   workspace_dev, workspace_bytes: a device buffer, 256-byte aligned, of at least
 *            256 bytes; queue capacity = (workspace_bytes - 256) / 128 paths.  A
 *            smaller workspace is correct: paths that find their queue full are
 *            finished by the lane that holds them.
 * Enqueued on `stream`: one 256-byte memset, then D + 1 kernel launches (a pass
 * whose queue is empty returns at once).  The workspace must not be reused by
 * another call before this one completes (stream order or events).  The staged
 * brute-force path uses the queues; the hierarchy (cfg->accel = 1) and scenes too
 * large for shared memory render exactly as rt_render (the workspace unused). */
rt_status rt_render_ws(const rt_scene *scene, const rt_camera *cam, const rt_render_params *params,
                       void *out_dev, size_t out_pitch_bytes, void *hitrec_dev, const rt_launch_config *cfg,
                       void *workspace_dev, size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------- batches
 * Many frames (scenes of uneven sphere counts and resolutions) rendered by
 * persistent kernels over a work queue: the (frame, tile) work items are ordered
 * longest first (estimated tile cost) and each CTA claims the next item with an
 * atomic add on a work counter until none is left, restaging the scene table in
 * shared memory when its frame changes.  The items are split by shading path (the
 * line filter from 128 spheres on, the segment test below), one persistent
 * instance per class; the line-filter class's frames hand bounce-1 hits to bounce
 * queues that one persistent pass per bounce works through (rt_render_ws's
 * scheme).  Each pixel is computed exactly as rt_render computes it
 * (bit-identical output).  Not in the paper (which renders one frame
 * per call, Section 3.9); it serves many small scenes at once.
 *   scenes[n], cams[n], params[n], outs_dev[n], pitches[n]: one entry per frame,
 *   with the same meaning and rules as for rt_render (hit records are not
 *   written).  Scenes must stay alive while the batch is in flight.  The batch
 *   kernel takes CTAs of at most 128 threads (block_x * block_y <= 128). */

/* Device workspace bytes rt_render_batch needs (256-byte aligned buffer): the work
 * counters, the frame table and the item list, then the bounce queues of the
 * frames rendered with the line filter (scenes of 128 spheres or more) whose
 * bounce limit is at least 1 -- a control block and two queues of a quarter of the
 * frame's pixels, 64 bytes per entry (the queued render of rt_render_ws, inside the
 * batch).  0 on invalid arguments. */
size_t rt_batch_workspace_bytes(int32_t n, const rt_scene *const *scenes, const rt_render_params *params,
                                const rt_launch_config *cfg);

/* Enqueue one batched render on `stream` using the caller's workspace (no device
 * allocation): one host-to-device copy of the work tables (pageable source,
 * staged by the runtime before the call returns), a reset of the bounce queues'
 * counters, then the persistent kernels in stream order: the line-filter class's
 * instance, one queue pass per bounce of its deferring frames, the segment-test
 * class's instance (empty classes launch nothing).  The caller must not reuse the
 * workspace before the launches complete. */
rt_status rt_render_batch(int32_t n, const rt_scene *const *scenes, const rt_camera *cams,
                          const rt_render_params *params, void *const *outs_dev, const size_t *pitches,
                          void *workspace_dev, size_t workspace_bytes, const rt_launch_config *cfg,
                          void *stream);

typedef struct rt_batch rt_batch;   /* a planned batch captured in a CUDA graph */

/* Plan a batch: validate, build the work tables, copy them to a library-owned
 * workspace (enqueued on `stream`), and capture a CUDA graph of {reset the work
 * counters and the bounce queues' counters, the persistent kernels and queue
 * passes of rt_render_batch}.  Cameras and parameters are fixed at creation;
 * scene contents may change between launches (rt_scene_update). */
rt_status rt_batch_create(int32_t n, const rt_scene *const *scenes, const rt_camera *cams,
                          const rt_render_params *params, void *const *outs_dev, const size_t *pitches,
                          const rt_launch_config *cfg, void *stream, rt_batch **out);

/* Replay the batch's graph on `stream` (ordered after the creation's copy).
 * Launches of one batch must not overlap (they share the work counter). */
rt_status rt_batch_launch(rt_batch *batch, void *stream);

/* Release a batch (synchronises the device first).  NULL is accepted. */
rt_status rt_batch_free(rt_batch *batch);

/* Batched render that allocates nothing.  The paper has no counterpart: it is
 * here for callers that must not allocate device memory while they render --
 * code embedded in a host application or framework that owns every device
 * allocation, or a latency-bound frame loop in which cudaMalloc/cudaFree would
 * synchronise the device and could fail mid-run.  Same arguments and results as
 * rt_render_batch minus the workspace: the work counter, frame table and item
 * list live in one fixed scratch array of RT_NOALLOC_SCRATCH_BYTES in the
 * library's device image (every GPU that loads the library holds it until the
 * process exits), filled by one host-to-device copy from a static host buffer.
 *   - At most RT_NOALLOC_MAX_FRAMES frames, and the work tables (work counters,
 *     frame table, item list: rt_batch_workspace_bytes of a batch without bounce
 *     queues) at most RT_NOALLOC_SCRATCH_BYTES: otherwise RT_ERR_EXCEEDS_SCRATCH
 *     and nothing is enqueued.  No frame defers its bounces here (the queues would
 *     not fit): the images are the same bits either way.
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress, with that device current).
 *   - It must not be captured into a CUDA graph: a captured copy would read the
 *     shared static host image when the graph replays, after later calls have
 *     rewritten it.  A call on a stream that is capturing returns
 *     RT_ERR_UNSUPPORTED and enqueues nothing (checked before any set-up).
 *   - Every call reuses the same array (the copy rewrites it, including the work
 *     counter, which it resets to zero): calls whose work overlaps on the GPU,
 *     on any stream, race.  Order them (same stream or events). */
#define RT_NOALLOC_SCRATCH_BYTES (4u << 20)
#define RT_NOALLOC_MAX_FRAMES 256
rt_status rt_render_batch_noalloc(int32_t n, const rt_scene *const *scenes, const rt_camera *cams,
                                  const rt_render_params *params, void *const *outs_dev, const size_t *pitches,
                                  const rt_launch_config *cfg, void *stream);

/* Render only the rectangle [x0, x0 + width) x [y0, y0 + height) of the frame that
 * `params` describes, into out_dev (row 0 = frame row y0, column 0 = frame column
 * x0; same formats and pitch rules as rt_render, for `width` pixels per row).
 * Every pixel is computed exactly as in the full frame (NDC, Philox counters and
 * all arithmetic use frame coordinates), so bands rendered separately -- e.g. one
 * per GPU -- stitch into the full frame bit for bit.  x0 must be a multiple of 8;
 * no hit record. */
rt_status rt_render_region(const rt_scene *scene, const rt_camera *cam, const rt_render_params *params,
                           int32_t x0, int32_t y0, int32_t width, int32_t height, void *out_dev,
                           size_t out_pitch_bytes, const rt_launch_config *cfg, void *stream);

/* Bytes of the hit record of one frame: for each bounce k in 0..D and each pixel,
 * the primitive id (int32, -1 = miss), the hit distance t (float) and the visible
 * fraction of every light (float), stored plane by plane:
 *   element (k, f, y, x) at 4 * (((k * (2 + L) + f) * H + y) * W + x),
 *   f = 0 id, 1 t, 2 + l visibility of light l. */
size_t rt_hitrec_bytes(const rt_scene *scene, const rt_render_params *params);

/* Bytes of the scene's device table: what rt_scene_upload and a host-side
 * rt_scene_update copy to the device.  0 for NULL. */
size_t rt_scene_bytes(const rt_scene *scene);

/* ---------------------------------------------------------------- adjoint
 * Reverse-mode derivative of the forward render with visibility held fixed (no
 * silhouette or shadow-edge terms), for inverse rendering.  Not in the paper.
 * Gradient layout (floats): sphere i at 8i + {albedo r, g, b, k_s, reflectivity,
 * centre x, y, z}; the plane at 8N + {albedo r, g, b, k_s, reflectivity, 0, 0,
 * 0}; light l at 8(N + 1) + 4l + {position x, y, z, intensity}.  The
 * "reflectivity" entry is the derivative with respect to the field that sets the
 * reflection ratio: the reflectivity record field, or, with refl_coupled (the
 * paper's ratio = exponent / MAX_REFLECTIVITY capped at 1, Section 3.7), the
 * specular exponent field, including the exponent's effect on the specular terms.
 * Scenes with a sky panorama are refused (RT_ERR_UNSUPPORTED). */

/* Number of floats of the packed gradient: 8 (N + 1) + 4 L. */
size_t rt_grad_count(const rt_scene *scene);

/* Device workspace bytes rt_render_backward needs (one partial gradient per CTA). */
size_t rt_backward_workspace_bytes(const rt_scene *scene, const rt_render_params *params,
                                   const rt_launch_config *cfg);

/* grad_dev (rt_grad_count floats, overwritten) = sum over pixels and RGB channels
 * of dL/dpixel * dpixel/dtheta for L = sum dL_dimg * image.
 *   dl_dimg_dev: device buffer laid out like the F32 framebuffer (rows of width
 *                float RGBA, dl_pitch_bytes apart, multiple of 16; A ignored).
 *   hitrec_dev:  the hit record of rt_render for the same scene contents, camera
 *                and params (replay), or NULL to recompute the paths (trace again,
 *                no hit-record memory).
 *   workspace_dev: rt_backward_workspace_bytes bytes, 16-byte aligned.
 * Two launches (adjoint, then a fixed-order sum of the per-CTA partials): the
 * result is reproducible bit for bit.  On return the workspace holds the partials,
 * partial b (CTA b = blockIdx.y * grid_x + blockIdx.x) at floats [b G, b G + G);
 * grad[e] = sum over w = 0..31 (in order) of s_w[e], s_w[e] = sum over b = w,
 * w + 32, w + 64, ... (in order) of partial b's entry e, in FP32. */
rt_status rt_render_backward(const rt_scene *scene, const rt_camera *cam, const rt_render_params *params,
                             const float *dl_dimg_dev, size_t dl_pitch_bytes, const void *hitrec_dev,
                             float *grad_dev, void *workspace_dev, size_t workspace_bytes,
                             const rt_launch_config *cfg, void *stream);

/* Read and clear the device error word (bit 0: a shared-memory staging wait gave
 * up; bit 1: a batch work-queue wait gave up; bit 2: a hierarchy traversal stack
 * would have overflowed).  Synchronises `stream`.  Returns
 * RT_ERR_TIMEOUT when a bit was set, RT_OK otherwise; *bits (nullable) receives
 * the word. */
rt_status rt_device_errors(void *stream, uint32_t *bits);

/* Failure-detection self-test: launches one small kernel whose bounded wait can
 * never be satisfied (an mbarrier expecting bytes no copy delivers, with no copy
 * issued); after `polls` polls (1 .. 2^20) it sets bit 0 of the device error
 * word and returns.  rt_device_errors then reports RT_ERR_TIMEOUT, and the
 * context stays usable.  The same give-up path guards every staging wait. */
rt_status rt_selftest_wait_timeout(uint32_t polls, void *stream);

/* Number of this library's kernel launches enqueued since the process started
 * (host-side count; used to report launches in benchmarks). */
uint64_t rt_launch_count(void);

/* Human-readable name of a status. */
const char *rt_status_string(rt_status s);

#ifdef __cplusplus
}
#endif

#endif /* RT_H */
