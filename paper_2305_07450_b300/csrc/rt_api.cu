// rt_api.cu -- the C ABI of include/rt.h and the kernels behind it, for sm_103a.
// One translation unit: the device error word and the kernels live here.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/rt.h"
#include "rt_batch.cuh"
#include "rt_bvh.cuh"
#include "rt_bvh_build.h"
#include "rt_bwd.cuh"
#include "rt_device.cuh"
#include "rt_errword.cuh"
#include "rt_stage.cuh"
#include "rt_trace.cuh"

using namespace rtd;

static std::atomic<uint64_t> g_launches{0};

struct rt_scene {
    int ns = 0, ns_pad = 0, has_plane = 0, nl = 0;
    int any_area = 0, any_sphere_light = 0;
    // the light kinds above describe the device contents (false after a device-side
    // update, which may change them; the lean kernels are then not chosen)
    bool kinds_known = true;
    size_t bytes = 0;
    void* dev = nullptr;     // device blob: header, geo, mat, mat2
    void* pinned = nullptr;  // host staging of the blob
    cudaEvent_t copy_done = nullptr;
    int device = 0;
    // the pinned blob holds the device contents (false after a device-side update)
    bool host_current = true;
    // hierarchy: 0 none, 1 current, 2 stale (device-side update since the build)
    int bvh_state = 0;
    void* bvh_dev = nullptr;     // [nodes][prim_idx], room for the most nodes ns can need
    void* bvh_pinned = nullptr;
    size_t bvh_cap = 0;
    cudaEvent_t bvh_copy_done = nullptr;
    rt_bvh_info bvh_info{};

    // sky panorama (Section 3.8): sky_h rows of sky_w RGBA texels, or none
    void* sky_dev = nullptr;
    int sky_w = 0, sky_h = 0;
};

// Which kinds of light a host description holds (area squares, spherical lights).
static void set_light_kinds(rt_scene* s, const rt_scene_desc* desc) {
    s->any_area = 0;
    s->any_sphere_light = 0;
    for (int l = 0; l < desc->n_lights; ++l) {
        if (desc->lights[8 * l + 4] > 0.f) s->any_area = 1;
        if (desc->lights[8 * l + 5] > 0.f) s->any_sphere_light = 1;
    }
    s->kinds_known = true;
}

static SceneView view_of(const rt_scene* s) {
    const char* b = static_cast<const char*>(s->dev);
    SceneView v;
    v.hdr = reinterpret_cast<const SceneHdr*>(b);
    v.geo = reinterpret_cast<const float4*>(b + sizeof(SceneHdr));
    v.mat = v.geo + s->ns_pad;
    v.mat2 = v.mat + s->ns_pad;
    v.sky.tex = static_cast<const float4*>(s->sky_dev);
    v.sky.w = s->sky_w;
    v.sky.h = s->sky_h;
    return v;
}

// ============================================================ forward kernel
// Register budget of the forward kernels per shading path: 80 for the segment test
// alone (6 CTAs of 128 threads per SM), 128 for the line filter, whose out-of-line
// group loop saves the caller's state per call and whose groups of 7 segments hold
// 42 registers of unit vectors (4 CTAs per SM; 4K queued frame with groups of 4:
// 9.97 ms against 10.22 at 80, 10.11 at 96, 10.48 at 104, 10.25 at 112, 10.46 at
// 144, 10.39 at 168; with groups of 7 the one-pass kernel too: 11.73 ms at 128
// against 12.05 ms for groups of 4 at 80).
constexpr int fwd_regs(int fm) { return fm_path(fm) == 1 ? 128 : 80; }


// One thread per pixel.  The CTA covers block_x x block_y pixels; warp w covers an
// 8 x 4 patch (lanes 0..7 = one row), so that a warp's primary and shadow rays
// are coherent.  The scene header and geometry table are staged in shared memory
// once per CTA.  Register budget 80 (6 CTAs of 128 threads per SM): measured on
// B300 at 4K as 16.05 ms against 16.25 (96), 16.01 (72), 16.02 (64) and slower
// at 104 / 112 / 128; the spills it causes sit outside the sphere loops.
template <bool HITREC, bool CH, int FM>
__global__ void __maxnreg__(fwd_regs(FM)) rt_fwd_kernel(const SceneView sv, const Frame fr, void* __restrict__ out,
                                                     size_t pitch, float* __restrict__ hr, size_t hr_plane,
                                                     int staging, int block_x, int block_y, uint32_t flower_off,
                                                     int flower_n) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    // whole table: header + geometry; tiled loop: header only (geometry per warp chunk)
    const uint32_t stage_bytes =
        CH ? (uint32_t)sizeof(SceneHdr) : (uint32_t)(sizeof(SceneHdr) + 16u * (uint32_t)__ldg(&sv.hdr->ns_pad));
    if (!stage_to_smem(smem, sv.hdr, stage_bytes, staging, &bar, phase, &g_err_word)) return;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const SceneHdr* hdr = reinterpret_cast<const SceneHdr*>(smem);
    float4* tab = reinterpret_cast<float4*>(smem + sizeof(SceneHdr));
    StagedScene sc{hdr, CH ? nullptr : tab, sv.geo, CH ? tab + (size_t)warp * kChunk : nullptr, sv.mat, sv.mat2};
    sc.sky = sv.sky;
    sc.flower = sunflower_table(reinterpret_cast<float4*>(smem + flower_off), flower_n, fr.nsamp);
    if constexpr (!CH && (fm_path(FM) == 1 || fm_skip(FM))) staged_cone(tab, hdr->ns_pad, sc);

    const int wpr = block_x >> 3;
    const int x = fr.rx0 + blockIdx.x * block_x + (warp % wpr) * 8 + (lane & 7);
    const int y = fr.ry0 + blockIdx.y * block_y + (warp / wpr) * 4 + (lane >> 3);
    const bool valid = x < fr.rx1 && y < fr.ry1;
    render_pixel<HITREC, CH, false, FM>(sc, fr, x, y, valid, out, pitch, hr, hr_plane);
}

// ============================================================ queued render (rt_render_ws)
// Workspace: a control block of counters, then two path queues of `cap` entries
// (64 bytes each) used in turn: queue k (the paths whose bounce-k ray hit) lives in
// the first when k is odd, in the second when k is even.
struct WsCtl {
    unsigned claim0;                    // warp patches claimed by the first pass
    unsigned count[RT_MAX_DEPTH + 2];   // entries appended to queue k
    unsigned head[RT_MAX_DEPTH + 2];    // entries claimed from queue k
};
constexpr size_t kWsCtlBytes = 256;
// Queue passes of at most this many paths per resident warp run in wide mode.
constexpr unsigned kWidePathsPerWarp = 8;
constexpr size_t kWsEntryBytes = 64;
static_assert(sizeof(WsCtl) <= kWsCtlBytes, "workspace control block");

__host__ __device__ inline unsigned ws_cap(size_t bytes) {
    const size_t n = bytes <= kWsCtlBytes ? 0 : (bytes - kWsCtlBytes) / (2 * kWsEntryBytes);
    return (unsigned)(n < (size_t(1) << 30) ? n : (size_t(1) << 30));
}
__device__ __forceinline__ PathQueue ws_queue(unsigned char* ws, unsigned cap, int k) {
    WsCtl* c = reinterpret_cast<WsCtl*>(ws);
    float4* q = reinterpret_cast<float4*>(ws + kWsCtlBytes + ((k & 1) ? 0 : (size_t)cap * kWsEntryBytes));
    return PathQueue{q, &c->count[k], cap};
}

// First pass: persistent CTAs (one per resident slot) stage the scene once; each
// warp claims 8 x 4 pixel patches (in the order of block_x x block_y tiles) and
// traces them, pushing paths whose bounce-1 ray hits to queue 1.
template <bool HITREC, int FM>
__global__ void __maxnreg__(fwd_regs(FM)) rt_fwd_p0_kernel(const SceneView sv, const Frame fr, void* __restrict__ out,
                                                 size_t pitch, float* __restrict__ hr, size_t hr_plane, int staging,
                                                 int block_x, int block_y, int tiles_x, unsigned n_items,
                                                 unsigned char* __restrict__ ws, unsigned cap, uint32_t flower_off,
                                                 int flower_n) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t stage_bytes = (uint32_t)(sizeof(SceneHdr) + 16u * (uint32_t)__ldg(&sv.hdr->ns_pad));
    if (!stage_to_smem(smem, sv.hdr, stage_bytes, staging, &bar, phase, &g_err_word)) return;
    const int lane = threadIdx.x;
    const SceneHdr* hdr = reinterpret_cast<const SceneHdr*>(smem);
    StagedScene sc{hdr, reinterpret_cast<const float4*>(smem + sizeof(SceneHdr)), sv.geo, nullptr, sv.mat, sv.mat2};
    sc.sky = sv.sky;
    sc.flower = sunflower_table(reinterpret_cast<float4*>(smem + flower_off), flower_n, fr.nsamp);
    if constexpr (fm_path(FM) == 1 || fm_skip(FM)) staged_cone(sc.geo, hdr->ns_pad, sc);
    WsCtl* ctl = reinterpret_cast<WsCtl*>(ws);
    const PathQueue q1 = ws_queue(ws, cap, 1);
    const int wpr = block_x >> 3, wpt = (block_x * block_y) >> 5;
#pragma unroll 1
    while (true) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(&ctl->claim0, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const int tile = (int)(it / (unsigned)wpt), wi = (int)(it % (unsigned)wpt);
        const int x = fr.rx0 + (tile % tiles_x) * block_x + (wi % wpr) * 8 + (lane & 7);
        const int y = fr.ry0 + (tile / tiles_x) * block_y + (wi / wpr) * 4 + (lane >> 3);
        const bool valid = x < fr.rx1 && y < fr.ry1;
        render_pixel<HITREC, false, false, FM>(sc, fr, x, y, valid, out, pitch, hr, hr_plane,
                                              fr.D >= 1 ? &q1 : nullptr);
    }
}

// Pass k >= 1: persistent CTAs; each warp claims 32 entries of queue k at a time.
// CTAs beyond the ones the queue's length needs return before staging.
// A queue of at most wide_max paths (line-filter instances only) is taken one path
// per warp (trace_queued_wide), each carried to its end: such passes are bound by
// one warp's latency for one hit, which spreading the hit's segments over the lanes
// cuts; the passes after a wide one find their queues empty.
template <bool HITREC, int FM>
__global__ void __maxnreg__(fwd_regs(FM)) rt_fwd_queue_kernel(const SceneView sv, const Frame fr, void* __restrict__ out,
                                                    size_t pitch, float* __restrict__ hr, size_t hr_plane,
                                                    int staging, unsigned char* __restrict__ ws, unsigned cap, int k,
                                                    unsigned wide_max, uint32_t flower_off, int flower_n) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    WsCtl* ctl = reinterpret_cast<WsCtl*>(ws);
    const unsigned n = min(*reinterpret_cast<volatile unsigned*>(&ctl->count[k]), cap);
    const bool wide = fm_path(FM) == 1 && n <= wide_max;
    const unsigned per_cta = wide ? blockDim.y : 32u * blockDim.y;
    if ((unsigned)blockIdx.x * per_cta >= n) return;  // the whole CTA, before any barrier
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t stage_bytes = (uint32_t)(sizeof(SceneHdr) + 16u * (uint32_t)__ldg(&sv.hdr->ns_pad));
    if (!stage_to_smem(smem, sv.hdr, stage_bytes, staging, &bar, phase, &g_err_word)) return;
    const int lane = threadIdx.x;
    const SceneHdr* hdr = reinterpret_cast<const SceneHdr*>(smem);
    StagedScene sc{hdr, reinterpret_cast<const float4*>(smem + sizeof(SceneHdr)), sv.geo, nullptr, sv.mat, sv.mat2};
    sc.sky = sv.sky;
    sc.flower = sunflower_table(reinterpret_cast<float4*>(smem + flower_off), flower_n, fr.nsamp);
    if constexpr (fm_path(FM) == 1 || fm_skip(FM)) staged_cone(sc.geo, hdr->ns_pad, sc);
    const PathQueue cur = ws_queue(ws, cap, k);
    const PathQueue nxt = ws_queue(ws, cap, k + 1);
    if constexpr (fm_path(FM) == 1) {
        if (wide) {
#pragma unroll 1
            while (true) {
                unsigned i = 0;
                if (lane == 0) i = atomicAdd(&ctl->head[k], 1u);
                i = __shfl_sync(0xffffffffu, i, 0);
                if (i >= n) break;
                trace_queued_wide<HITREC, fm_lean(FM)>(sc, fr, cur.ent + (size_t)i * 4, k, out, pitch, hr, hr_plane);
                __syncwarp();
            }
            return;
        }
    }
#pragma unroll 1
    while (true) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&ctl->head[k], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const unsigned i = base + (unsigned)lane;
        if (i < n) trace_queued<HITREC, FM>(sc, fr, cur.ent + (size_t)i * 4, k, nxt, out, pitch, hr, hr_plane);
        __syncwarp();
    }
}

// Forward kernel over the sphere hierarchy: the same pixels as rt_fwd_kernel, the
// closest hit and the shadow segments taken through the hierarchy.  When
// bvh_stage_bytes != 0 the geometry table and the hierarchy are staged in shared
// memory after the header (two copies on the same barrier); otherwise both are
// read from global memory through the caches.
template <bool HITREC>
__global__ void __launch_bounds__(256) rt_fwd_bvh_kernel(const SceneView sv, const BvhView bv,
                                                         uint32_t bvh_stage_bytes, const Frame fr,
                                                         void* __restrict__ out, size_t pitch, float* __restrict__ hr,
                                                         size_t hr_plane, int staging, int block_x, int block_y) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const bool staged = bvh_stage_bytes != 0;
    const uint32_t geo_bytes = staged ? 16u * (uint32_t)__ldg(&sv.hdr->ns_pad) : 0u;
    if (!stage_to_smem(smem, sv.hdr, (uint32_t)sizeof(SceneHdr) + geo_bytes, staging, &bar, phase, &g_err_word))
        return;
    unsigned char* bvh_s = smem + sizeof(SceneHdr) + geo_bytes;
    if (staged && !stage_to_smem(bvh_s, bv.nodes, bvh_stage_bytes, staging, &bar, phase, &g_err_word)) return;
    const SceneHdr* hdr = reinterpret_cast<const SceneHdr*>(smem);
    StagedScene sc{hdr, staged ? reinterpret_cast<const float4*>(smem + sizeof(SceneHdr)) : sv.geo, sv.geo, nullptr,
                   sv.mat, sv.mat2};
    sc.bvh = bv;
    sc.sky = sv.sky;
    if (staged) {
        sc.bvh.nodes = reinterpret_cast<const BvhNode*>(bvh_s);
        sc.bvh.prim = reinterpret_cast<const int32_t*>(bvh_s + (size_t)bv.n_nodes * sizeof(BvhNode));
    }
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int wpr = block_x >> 3;
    const int x = fr.rx0 + blockIdx.x * block_x + (warp % wpr) * 8 + (lane & 7);
    const int y = fr.ry0 + blockIdx.y * block_y + (warp / wpr) * 4 + (lane >> 3);
    const bool valid = x < fr.rx1 && y < fr.ry1;
    render_pixel<HITREC, false, true>(sc, fr, x, y, valid, out, pitch, hr, hr_plane);
}

// Failure-detection self-test: the barrier expects bytes that no copy will ever
// deliver (none is issued), so the bounded wait must give up after `polls` polls,
// flag the error word and return -- the path a stalled staging copy takes.
__global__ void rt_selftest_wait_kernel(uint32_t polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, 16);
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, polls);
    if (!ok && threadIdx.x == 0) atomicOr(&g_err_word, kErrStageTimeout);
}

// Device-side packing of scene records (rt_scene_update with device pointers):
// thread i < ns packs sphere i; thread ns packs the header's plane and lights.
__global__ void rt_pack_kernel(SceneView sv, int ns, const float* __restrict__ sph, int has_plane,
                               const float* __restrict__ plane, int nl, const float* __restrict__ lights) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float4* geo = const_cast<float4*>(sv.geo);
    float4* mat = const_cast<float4*>(sv.mat);
    float4* mat2 = const_cast<float4*>(sv.mat2);
    if (i < ns) {
        const float* f = sph + 10 * (size_t)i;
        sphere_put(geo, i, make_float4(f[0], f[1], f[2], -(f[3] * f[3])));
        mat[i] = make_float4(f[4], f[5], f[6], f[7]);
        mat2[i] = make_float4(f[8], f[9], f[3], __frcp_rn(f[3]));
    } else if (i == ns) {
        SceneHdr* h = const_cast<SceneHdr*>(sv.hdr);
        if (has_plane) {
            h->plane_g = make_float4(plane[0], plane[1], plane[2], plane[3]);
            h->plane_m = make_float4(plane[4], plane[5], plane[6], plane[7]);
            h->plane_m2 = make_float4(plane[8], plane[9], 0.f, 0.f);
        }
        for (int l = 0; l < nl; ++l) {
            const float* f = lights + 8 * l;
            h->light_p[l] = make_float4(f[0], f[1], f[2], f[3]);
            h->light_s[l] = make_float4(f[4], f[5], 0.f, 0.f);
        }
    }
}

// Physics step of the animated loop (Section 3.8: the bodies move by Verlet
// integration; their positions are streamed in every frame, Section 3.9).  One
// thread per sphere, `steps` steps of position Verlet under gravity (0, -g, 0):
// x' = x + (x - x_prev) + a dt^2; a sphere that crosses the ground plane
// n.x + pd = 0 is moved back along n until it touches it, and the step velocity's
// normal component into the plane is dropped when it is at most two steps of
// gravity (resting contact has one), else reversed and scaled by the restitution e; the
// previous position is set so that the next step carries that velocity.  The
// centre is updated in place in the sphere record; prev holds x_prev [n][3].
__global__ void rt_verlet_kernel(float* __restrict__ sph, float* __restrict__ prev, int n, float4 plane,
                                 int has_plane, float dt, float g, float e, int steps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* rec = sph + 10 * (size_t)i;
    float* pv = prev + 3 * (size_t)i;
    const float r = rec[3];
    f3 x = mk3(rec[0], rec[1], rec[2]), xp = mk3(pv[0], pv[1], pv[2]);
    const f3 nn = mk3(plane.x, plane.y, plane.z);
    const float gdt2 = g * dt * dt;
#pragma unroll 1
    for (int s = 0; s < steps; ++s) {
        f3 xn = add(x, sub(x, xp));
        xn.y -= gdt2;
        f3 xq = x;
        if (has_plane) {
            const float sd = dot(nn, xn) + plane.w - r;
            if (sd < 0.0f) {
                f3 v = sub(xn, x);
                xn = sub(xn, scl(nn, sd));
                const float vn = dot(v, nn);
                if (vn < 0.0f) v = sub(v, scl(nn, -vn <= 2.0f * gdt2 ? vn : (1.0f + e) * vn));
                xq = sub(xn, v);
            }
        }
        xp = xq;
        x = xn;
    }
    rec[0] = x.x;
    rec[1] = x.y;
    rec[2] = x.z;
    pv[0] = xp.x;
    pv[1] = xp.y;
    pv[2] = xp.z;
}

// ============================================================ host helpers
namespace {

bool finite_all(const float* f, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(f[i])) return false;
    return true;
}

// Distance from point c to the axis-aligned horizontal square of side a centred
// at L (y = L.y).
double dist_point_square(const double* c, const float* L, double a) {
    const double h = a / 2;
    const double dx = std::fmax(std::fabs(c[0] - L[0]) - h, 0.0);
    const double dz = std::fmax(std::fabs(c[2] - L[2]) - h, 0.0);
    const double dy = c[1] - L[1];
    return std::sqrt(dx * dx + dy * dy + dz * dz);
}

rt_status validate_desc(const rt_scene_desc* d) {
    if (!d || d->n_spheres < 0 || d->n_spheres > (1 << 20) || d->n_lights < 0 || d->n_lights > RT_MAX_LIGHTS)
        return RT_ERR_INVALID_ARG;
    if ((d->n_spheres && !d->spheres) || (d->n_lights && !d->lights) || (d->has_plane && !d->plane))
        return RT_ERR_INVALID_ARG;
    for (int i = 0; i < d->n_spheres; ++i) {
        const float* f = d->spheres + 10 * (size_t)i;
        if (!finite_all(f, 10) || !(f[3] > 0.f) || f[7] < 0.f || f[8] < 0.f || f[9] < 0.f || f[9] > 1.f)
            return RT_ERR_INVALID_ARG;
    }
    if (d->has_plane) {
        const float* f = d->plane;
        if (!finite_all(f, 10) || f[7] < 0.f || f[8] < 0.f || f[9] < 0.f || f[9] > 1.f) return RT_ERR_INVALID_ARG;
        const double nn = (double)f[0] * f[0] + (double)f[1] * f[1] + (double)f[2] * f[2];
        if (std::fabs(nn - 1.0) > 1e-5) return RT_ERR_INVALID_ARG;
    }
    for (int l = 0; l < d->n_lights; ++l) {
        const float* f = d->lights + 8 * l;
        if (!finite_all(f, 8) || f[3] < 0.f || f[4] < 0.f || f[5] < 0.f || (f[4] > 0.f && f[5] > 0.f))
            return RT_ERR_INVALID_ARG;
        // the shadow test needs every light (its whole sampled extent) outside every sphere
        for (int i = 0; i < d->n_spheres; ++i) {
            const float* s = d->spheres + 10 * (size_t)i;
            const double c[3] = {s[0], s[1], s[2]};
            double dist;
            if (f[4] > 0.f) {
                dist = dist_point_square(c, f, f[4]);
            } else {
                const double dx = c[0] - f[0], dy = c[1] - f[1], dz = c[2] - f[2];
                dist = std::sqrt(dx * dx + dy * dy + dz * dz) - f[5];
            }
            if (!(dist > (double)s[3])) return RT_ERR_UNSUPPORTED;
        }
    }
    return RT_OK;
}

void pack_host(const rt_scene_desc* d, int ns_pad, unsigned char* blob) {
    std::memset(blob, 0, scene_bytes(ns_pad));
    SceneHdr* h = reinterpret_cast<SceneHdr*>(blob);
    h->ns = d->n_spheres;
    h->ns_pad = ns_pad;
    h->has_plane = d->has_plane ? 1 : 0;
    h->nl = d->n_lights;
    if (d->has_plane) {
        const float* f = d->plane;
        h->plane_g = make_float4(f[0], f[1], f[2], f[3]);
        h->plane_m = make_float4(f[4], f[5], f[6], f[7]);
        h->plane_m2 = make_float4(f[8], f[9], 0.f, 0.f);
    }
    for (int l = 0; l < d->n_lights; ++l) {
        const float* f = d->lights + 8 * l;
        h->light_p[l] = make_float4(f[0], f[1], f[2], f[3]);
        h->light_s[l] = make_float4(f[4], f[5], 0.f, 0.f);
    }
    float4* geo = reinterpret_cast<float4*>(blob + sizeof(SceneHdr));
    float4* mat = geo + ns_pad;
    float4* mat2 = mat + ns_pad;
    for (int i = 0; i < ns_pad; ++i) {
        if (i < d->n_spheres) {
            const float* f = d->spheres + 10 * (size_t)i;
            sphere_put(geo, i, make_float4(f[0], f[1], f[2], -(float)((double)f[3] * f[3])));
            mat[i] = make_float4(f[4], f[5], f[6], f[7]);
            mat2[i] = make_float4(f[8], f[9], f[3], (float)(1.0 / (double)f[3]));
        } else {
            sphere_put(geo, i, make_float4(0.f, 0.f, 0.f, 1.f));  // never hit, never blocks
            mat[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            mat2[i] = make_float4(0.f, 0.f, 1.f, 1.f);
        }
    }
}

rt_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RT_OK;
    if (e == cudaErrorMemoryAllocation) return RT_ERR_OOM;
    return RT_ERR_CUDA;
}

rt_status validate_params(const rt_scene* s, const rt_render_params* p) {
    if (!s || !p) return RT_ERR_INVALID_ARG;
    if (p->width < 1 || p->height < 1 || p->width > 32768 || p->height > 32768) return RT_ERR_INVALID_ARG;
    if (p->max_depth < 0 || p->max_depth > RT_MAX_DEPTH) return RT_ERR_INVALID_ARG;
    if (p->shadow_samples < 1 || p->shadow_samples > RT_MAX_SAMPLES) return RT_ERR_INVALID_ARG;
    if (p->shading_model != RT_PHONG && p->shading_model != RT_BLINN_PHONG) return RT_ERR_INVALID_ARG;
    if (p->out_format != RT_OUT_RGBA8 && p->out_format != RT_OUT_F32) return RT_ERR_INVALID_ARG;
    if (!std::isfinite(p->ambient) || !std::isfinite(p->eps) || p->eps < 0.f) return RT_ERR_INVALID_ARG;
    if (p->refl_coupled != 0 && p->refl_coupled != 1) return RT_ERR_INVALID_ARG;
    if (p->refl_coupled && !(p->max_reflectivity > 0.f && std::isfinite(p->max_reflectivity))) return RT_ERR_INVALID_ARG;
    if (s->any_area) {
        const int g = (int)std::lround(std::sqrt((double)p->shadow_samples));
        if (g * g != p->shadow_samples) return RT_ERR_INVALID_ARG;
    }
    return RT_OK;
}

rt_status validate_camera(const rt_camera* c) {
    if (!c) return RT_ERR_INVALID_ARG;
    const float f[6] = {c->pos[0], c->pos[1], c->pos[2], c->yaw_deg, c->pitch_deg, c->fov_deg};
    if (!finite_all(f, 6) || !(c->fov_deg > 0.f) || !(c->fov_deg < 180.f)) return RT_ERR_INVALID_ARG;
    return RT_OK;
}

// Camera basis rotated by pitch (about x) then yaw (about y), computed in double.
Frame make_frame(const rt_scene* s, const rt_camera* c, const rt_render_params* p) {
    Frame fr;
    std::memset(&fr, 0, sizeof(fr));
    fr.W = p->width;
    fr.H = p->height;
    fr.D = p->max_depth;
    fr.nsamp = p->shadow_samples;
    fr.model = p->shading_model;
    fr.fmt = p->out_format;
    fr.ka = p->ambient;
    fr.eps = p->eps;
    fr.m = p->width < p->height ? p->width : p->height;
    const double deg = M_PI / 180.0;
    const double yw = c->yaw_deg * deg, pt = c->pitch_deg * deg, fov = c->fov_deg * deg;
    const double cy = std::cos(yw), sy = std::sin(yw), cp = std::cos(pt), sp = std::sin(pt);
    const double b = 1.0 / std::tan(fov / 2.0);
    fr.cam = make_float3(c->pos[0], c->pos[1], c->pos[2]);
    fr.right = make_float3((float)cy, 0.f, (float)-sy);
    fr.up = make_float3((float)(-sp * sy), (float)cp, (float)(-sp * cy));
    fr.fwd = make_float3((float)(b * cp * sy), (float)(b * sp), (float)(b * cp * cy));
    fr.key0 = (uint32_t)(p->seed & 0xffffffffu);
    fr.key1 = (uint32_t)(p->seed >> 32);
    fr.refl_inv_max = p->refl_coupled ? (float)(1.0 / (double)p->max_reflectivity) : 0.0f;
    fr.rx0 = 0;
    fr.ry0 = 0;
    fr.rx1 = p->width;
    fr.ry1 = p->height;
    const int g = (int)std::lround(std::sqrt((double)p->shadow_samples));
    fr.sample_g = g > 0 ? g : 1;
    fr.sample_g_inv = (float)(1.0 / (double)fr.sample_g);
    fr.sample_g_magic = (uint32_t)(((1u << 22) + (uint32_t)fr.sample_g - 1u) / (uint32_t)fr.sample_g);
    (void)s;
    return fr;
}

// Coordinates at or above this are refused by the hierarchy (its per-ray box
// widening and the slab products stay far from FP32 overflow below it).
constexpr double kBvhCoordLimit = 1e15;

struct Launch {
    int bx, by, staging, min_blocks, accel;
};

rt_status resolve_launch(const rt_launch_config* cfg, Launch* L) {
    L->bx = 16;
    L->by = 8;
    L->staging = 1;
    L->min_blocks = 0;
    L->accel = 0;
    if (cfg) {
        if (cfg->block_x) L->bx = cfg->block_x;
        if (cfg->block_y) L->by = cfg->block_y;
        if (cfg->staging) L->staging = cfg->staging;
        if (cfg->min_blocks_per_sm < 0 || cfg->min_blocks_per_sm > 32) return RT_ERR_INVALID_ARG;
        L->min_blocks = cfg->min_blocks_per_sm;
        if (cfg->accel < 0 || cfg->accel > 1) return RT_ERR_INVALID_ARG;
        L->accel = cfg->accel;
    }
    if (L->bx % 8 || L->by % 4 || L->bx < 8 || L->by < 4 || L->bx * L->by < 32 || L->bx * L->by > 256)
        return RT_ERR_INVALID_ARG;
    if (L->staging < 1 || L->staging > 3) return RT_ERR_INVALID_ARG;
    if (L->accel && L->staging == 3) return RT_ERR_INVALID_ARG;
    return RT_OK;
}

int max_smem_optin() {
    static int v = -1;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    if (v < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
    }
    return v;
}

// The whole geometry table is staged unless it does not fit (or the tiled loop is
// forced with staging = 3).
constexpr size_t kStaticSmemReserve = 12 * 1024 + 9 * 4 * kSegStride * kFiltGroup;
size_t stage_smem_bytes(bool chunked, int ns_pad, int nwarps) {
    return chunked ? sizeof(SceneHdr) + (size_t)nwarps * kChunk * 16 : sizeof(SceneHdr) + (size_t)ns_pad * 16;
}

bool use_tiled_loop(const Launch& L, int ns_pad, size_t extra = 0) {
    if (L.staging == 3) return true;
    // room left for the kernels' static shared memory (the shadow test's segment
    // vectors, 42 KB, and the barriers)
    return stage_smem_bytes(false, ns_pad, 0) + 16 + extra + kStaticSmemReserve > (size_t)max_smem_optin();
}

// Resident CTAs of `kernel` on the current device (threads per CTA, dynamic shared
// memory), cached per (device, kernel, threads, bytes).
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::vector<std::tuple<int, const void*, int, size_t, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    for (const auto& e : cache)
        if (std::get<0>(e) == dev && std::get<1>(e) == (const void*)kernel && std::get<2>(e) == threads &&
            std::get<3>(e) == smem)
            return std::get<4>(e);
    int per_sm = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) per_sm = 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 1;
    const int n = std::max(1, per_sm) * std::max(1, nsm);
    cache.emplace_back(dev, (const void*)kernel, threads, smem, n);
    return n;
}

template <typename K>
rt_status ensure_smem(K kernel, size_t bytes) {
    // the kernel's static shared memory, looked up once per kernel (the query costs
    // tens of microseconds, as much as a small frame)
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> known;
    size_t stat = 0;
    bool found = false;
    {
        std::lock_guard<std::mutex> g(mu);
        for (const auto& e : known)
            if (e.first == (const void*)kernel) {
                stat = e.second;
                found = true;
                break;
            }
    }
    if (!found) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return RT_ERR_CUDA;
        stat = fa.sharedSizeBytes;
        std::lock_guard<std::mutex> g(mu);
        known.emplace_back((const void*)kernel, stat);
    }
    if (bytes + stat <= 48 * 1024) return RT_OK;
    const int cap = max_smem_optin() - (int)stat;  // what the kernel's static shared memory leaves
    if ((long long)bytes > cap) return RT_ERR_UNSUPPORTED;
    return cuda_status(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
}

// ------------------------------------------------------------ batch packing
struct BatchPlanHost {
    std::vector<unsigned char> table;  // workspace image: head, frames, items, deferring frames
    int n_items = 0;
    int n_filt = 0;  // the first n_filt items: frames rendered with the line filter
    int n_defer = 0, dmax = 0;  // frames with bounce queues, their largest bounce limit
    size_t ctl_off = 0, ctl_bytes = 0;  // their control blocks (reset before every launch)
    size_t ws_bytes = 0;                // the whole workspace (the queues follow the table)
    size_t smem = 0;
    bool chunked = false;
};

// The shading path a frame of a batch takes: the line filter (with the cone
// passes) from kFilterMinPad spheres on, as rt_render does, unless the batch stages
// its tables chunk by chunk.
bool batch_filtered(const rt_scene* s, bool chunked) { return !chunked && s->ns_pad >= kFilterMinPad; }

// The batch's bounce queues (rt_render_ws's scheme inside the batch): every frame of
// the line-filter class with a bounce limit of at least 1 defers its bounce-1 paths,
// with a quarter of its pixels per queue (a full queue is not an error: the lane
// finishes the path itself).  Layout after the items (ending at items_end): the
// deferring frames' indices (int), then their 256-byte control blocks, then each
// frame's two queues.  Fills the frames' queue fields when `frames` is given and
// returns the workspace's total size.
size_t batch_defer_layout(int n, const rt_scene* const* scenes, const rt_render_params* params, bool chunked,
                          size_t items_end, BatchFrame* frames, std::vector<int>* list, int* n_defer, int* dmax,
                          size_t* ctl_off, size_t* ctl_bytes) {
    int nd = 0, dm = 0;
    for (int i = 0; i < n; ++i)
        if (batch_filtered(scenes[i], chunked) && params[i].max_depth >= 1) {
            ++nd;
            dm = std::max(dm, params[i].max_depth);
        }
    const size_t c0 = (items_end + (size_t)nd * sizeof(int) + 255) / 256 * 256;
    size_t off = c0 + (size_t)nd * kBatchQCtl;
    int j = 0;
    for (int i = 0; i < n; ++i) {
        if (!(batch_filtered(scenes[i], chunked) && params[i].max_depth >= 1)) continue;
        const unsigned cap = (unsigned)std::min<size_t>(((size_t)params[i].width * params[i].height + 3) / 4,
                                                        (size_t)1 << 30);
        if (frames) {
            frames[i].q_ctl = c0 + (size_t)j * kBatchQCtl;
            frames[i].q_ent = off;
            frames[i].q_cap = cap;
        }
        if (list) list->push_back(i);
        off += 2 * (size_t)cap * kWsEntryBytes;
        ++j;
    }
    *n_defer = nd;
    *dmax = dm;
    *ctl_off = c0;
    *ctl_bytes = (size_t)nd * kBatchQCtl;
    return nd ? off : items_end;  // no deferring frame: the work tables alone
}

// Relative cost of one tile of a frame, for the longest-first item order.
double tile_cost(const rt_scene* s, const rt_render_params* p) {
    double rays = 1.0;
    // every light needs at least one shadow ray; sampled lights need shadow_samples
    rays += (double)s->nl + (double)(s->any_area + s->any_sphere_light) * (p->shadow_samples - 1);
    return (double)(s->ns_pad + 2) * (1.0 + p->max_depth) * rays;
}

rt_status batch_pack(int n, const rt_scene* const* scenes, const rt_camera* cams, const rt_render_params* params,
                     void* const* outs, const size_t* pitches, const Launch& L, BatchPlanHost* plan) {
    if (n < 1 || n > (1 << (32 - kItemTileBits)) || !scenes || !cams || !params || !outs || !pitches)
        return RT_ERR_INVALID_ARG;
    if (L.bx * L.by > kBatchMaxThreads) return RT_ERR_INVALID_ARG;
    if (L.accel) return RT_ERR_UNSUPPORTED;
    std::vector<BatchFrame> frames((size_t)n);
    std::vector<int> tiles((size_t)n);
    long long n_items = 0;
    int max_pad = 0;
    for (int i = 0; i < n; ++i)
        if (scenes[i]) max_pad = std::max(max_pad, scenes[i]->ns_pad);
    const bool chunked = use_tiled_loop(L, max_pad);
    const size_t smem = stage_smem_bytes(chunked, max_pad, (L.bx * L.by) / 32);
    for (int i = 0; i < n; ++i) {
        const rt_scene* s = scenes[i];
        const rt_render_params* p = &params[i];
        rt_status st = validate_params(s, p);
        if (st != RT_OK) return st;
        if ((st = validate_camera(&cams[i])) != RT_OK) return st;
        const size_t row = (size_t)p->width * (p->out_format == RT_OUT_F32 ? 16 : 4);
        if (!outs[i] || (reinterpret_cast<uintptr_t>(outs[i]) & 15) || pitches[i] < row || (pitches[i] & 15))
            return RT_ERR_INVALID_ARG;
        BatchFrame& B = frames[(size_t)i];
        std::memset(&B, 0, sizeof(B));
        B.sv = view_of(s);
        B.fr = make_frame(s, &cams[i], p);
        B.out = outs[i];
        B.pitch = pitches[i];
        B.stage_bytes = (uint32_t)(chunked ? sizeof(SceneHdr) : sizeof(SceneHdr) + (size_t)s->ns_pad * 16);
        B.tiles_x = (p->width + L.bx - 1) / L.bx;
        const long long t = (long long)B.tiles_x * ((p->height + L.by - 1) / L.by);
        if (t >= (1ll << kItemTileBits)) return RT_ERR_UNSUPPORTED;
        tiles[(size_t)i] = (int)t;
        n_items += t;
    }
    if (n_items >= (1ll << 31)) return RT_ERR_UNSUPPORTED;
    // the line-filter frames first, then the others; each class longest-first (frames
    // by estimated tile cost, tiles of a frame in raster order)
    std::vector<int> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const bool fa = batch_filtered(scenes[a], chunked), fb = batch_filtered(scenes[b], chunked);
        if (fa != fb) return fa;
        return tile_cost(scenes[a], &params[a]) > tile_cost(scenes[b], &params[b]);
    });
    long long n_filt = 0;
    for (int i = 0; i < n; ++i)
        if (batch_filtered(scenes[i], chunked)) n_filt += tiles[(size_t)i];
    const size_t items_off = batch_items_offset(n);
    const size_t items_end = items_off + (size_t)n_items * 4;
    std::vector<int> defer;
    plan->ws_bytes = batch_defer_layout(n, scenes, params, chunked, items_end, frames.data(), &defer, &plan->n_defer,
                                        &plan->dmax, &plan->ctl_off, &plan->ctl_bytes);
    plan->table.assign(items_end + defer.size() * sizeof(int), 0);
    std::memcpy(plan->table.data() + batch_frames_offset(), frames.data(), (size_t)n * sizeof(BatchFrame));
    if (!defer.empty()) std::memcpy(plan->table.data() + items_end, defer.data(), defer.size() * sizeof(int));
    uint32_t* items = reinterpret_cast<uint32_t*>(plan->table.data() + items_off);
    size_t k = 0;
    for (int f : order)
        for (int t = 0; t < tiles[(size_t)f]; ++t) items[k++] = ((uint32_t)f << kItemTileBits) | (uint32_t)t;
    plan->n_items = (int)n_items;
    plan->n_filt = (int)n_filt;
    plan->smem = smem;
    plan->chunked = chunked;
    return RT_OK;
}

// Resident CTAs of the batch kernels: grid[0] for the segment-test instance,
// grid[1] for the line-filter one, grid[2] for the queue passes.
rt_status batch_grid(const Launch& L, size_t smem, bool chunked, int grid[3]) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    for (int fm = 0; fm < 3; ++fm) {
        int per_sm = 0;
        if (L.min_blocks > 0) {
            per_sm = L.min_blocks;
        } else if (fm == 2) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt_batch_queue_kernel<1>, L.bx * L.by, smem);
        } else if (chunked) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt_batch_kernel<true, 0>, L.bx * L.by, smem);
        } else {
            e = fm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt_batch_kernel<false, 1>, L.bx * L.by, smem)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt_batch_kernel<false, 0>, L.bx * L.by, smem);
        }
        if (e != cudaSuccess) return cuda_status(e);
        grid[fm] = sms * std::max(per_sm, 1);
    }
    return RT_OK;
}

}  // namespace

rt_status batch_smem(bool chunked, size_t smem) {
    if (chunked) return ensure_smem(rt_batch_kernel<true, 0>, smem);
    rt_status st = ensure_smem(rt_batch_kernel<false, 0>, smem);
    if (st == RT_OK) st = ensure_smem(rt_batch_kernel<false, 1>, smem);
    return st != RT_OK ? st : ensure_smem(rt_batch_queue_kernel<1>, smem);
}

// The line-filter instance over items [0, n_filt), the queue passes k = 1..dmax of
// its deferring frames, then the segment-test instance over [n_filt, n_items), in
// stream order; an empty class launches nothing.  Returns the number of launches.
int batch_launch(bool chunked, const int grid[3], const Launch& L, size_t smem, cudaStream_t st, unsigned char* ws,
                 int n, int n_items, int n_filt, int n_defer, int dmax) {
    const dim3 block(32, (L.bx * L.by) / 32);
    const int hstage = L.staging == 2 ? 2 : 1;
    int launches = 0;
    if (n_filt > 0) {
        rt_batch_kernel<false, 1><<<grid[1], block, smem, st>>>(ws, n, 0, n_filt, hstage, L.bx, L.by);
        ++launches;
        for (int k = 1; n_defer > 0 && k <= dmax; ++k, ++launches)
            rt_batch_queue_kernel<1><<<grid[2], block, smem, st>>>(ws, n, n_items, n_defer, k, hstage);
    }
    if (n_items > n_filt) {
        ++launches;
        if (chunked)
            rt_batch_kernel<true, 0><<<grid[0], block, smem, st>>>(ws, n, n_filt, n_items - n_filt, hstage, L.bx,
                                                                   L.by);
        else
            rt_batch_kernel<false, 0><<<grid[0], block, smem, st>>>(ws, n, n_filt, n_items - n_filt, hstage, L.bx,
                                                                    L.by);
    }
    return launches;
}

struct rt_batch {
    bool chunked = false;
    int n = 0, n_items = 0, n_filt = 0, n_defer = 0, dmax = 0, launches = 0;
    size_t table_bytes = 0, ctl_off = 0, ctl_bytes = 0;
    int grid[3] = {0, 0, 0};
    Launch L{};
    size_t smem = 0, ws_bytes = 0;
    void* ws = nullptr;
    void* pinned = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ready = nullptr;
};

// ============================================================ C ABI
extern "C" {

const char* rt_status_string(rt_status s) {
    switch (s) {
        case RT_OK: return "RT_OK";
        case RT_ERR_INVALID_ARG: return "RT_ERR_INVALID_ARG";
        case RT_ERR_CUDA: return "RT_ERR_CUDA";
        case RT_ERR_OOM: return "RT_ERR_OOM";
        case RT_ERR_UNSUPPORTED: return "RT_ERR_UNSUPPORTED";
        case RT_ERR_TIMEOUT: return "RT_ERR_TIMEOUT";
        case RT_ERR_EXCEEDS_SCRATCH: return "RT_ERR_EXCEEDS_SCRATCH";
    }
    return "RT_ERR_UNKNOWN";
}

uint64_t rt_launch_count(void) { return g_launches.load(); }

}  // extern "C"

namespace {

// (Re)build the hierarchy from the pinned host copy of the scene table and enqueue
// its copy to the device.  Device room is sized once for the most nodes the sphere
// count can need (n - 1 interior nodes of a binary tree over n leaves at most).
rt_status bvh_refresh(rt_scene* s, cudaStream_t st_) {
    if (!s->host_current) return RT_ERR_UNSUPPORTED;
    const float4* geo = reinterpret_cast<const float4*>(static_cast<const char*>(s->pinned) + sizeof(SceneHdr));
    rtbvh::Result R;
    rtbvh::build(geo, s->ns, &R);
    if (!((double)R.r_scene < kBvhCoordLimit)) return RT_ERR_UNSUPPORTED;
    const int n_nodes = (int)R.nodes.size();
    const size_t bytes = bvh_bytes(n_nodes, s->ns);
    cudaError_t e = cudaSuccess;
    if (bytes > 0) {
        if (!s->bvh_dev) {
            const size_t cap = bvh_bytes(std::max(s->ns - 1, 1), s->ns);
            e = cudaMalloc(&s->bvh_dev, cap);
            if (e == cudaSuccess) e = cudaMallocHost(&s->bvh_pinned, cap);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->bvh_copy_done, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_status(e);
            s->bvh_cap = cap;
        } else {
            e = cudaEventSynchronize(s->bvh_copy_done);  // the previous copy has left the staging buffer
            if (e != cudaSuccess) return cuda_status(e);
        }
        if (bytes > s->bvh_cap) return RT_ERR_UNSUPPORTED;
        unsigned char* h = static_cast<unsigned char*>(s->bvh_pinned);
        std::memset(h, 0, bytes);
        std::memcpy(h, R.nodes.data(), (size_t)n_nodes * sizeof(BvhNode));
        std::memcpy(h + (size_t)n_nodes * sizeof(BvhNode), R.prim.data(), R.prim.size() * 4);
        e = cudaMemcpyAsync(s->bvh_dev, h, bytes, cudaMemcpyHostToDevice, st_);
        if (e == cudaSuccess) e = cudaEventRecord(s->bvh_copy_done, st_);
        if (e != cudaSuccess) return cuda_status(e);
    }
    s->bvh_info.n_nodes = n_nodes;
    s->bvh_info.depth = R.depth;
    s->bvh_info.max_leaf = R.max_leaf;
    s->bvh_info.r_scene = R.r_scene;
    s->bvh_state = 1;
    return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_scene_build_bvh(rt_scene* s, void* stream, rt_bvh_info* info) {
    if (!s) return RT_ERR_INVALID_ARG;
    const rt_status st = bvh_refresh(s, static_cast<cudaStream_t>(stream));
    if (st == RT_OK && info) *info = s->bvh_info;
    return st;
}

rt_status rt_bvh_build_host(const rt_scene_desc* desc, void* nodes, int32_t nodes_cap, int32_t* prim_idx,
                            rt_bvh_info* info) {
    rt_status st = validate_desc(desc);
    if (st != RT_OK) return st;
    std::vector<float4> geo((size_t)pad_spheres(desc->n_spheres));  // the paired table, as packed for the device
    for (int i = 0; i < desc->n_spheres; ++i) {
        const float* f = desc->spheres + 10 * (size_t)i;
        sphere_put(geo.data(), i, make_float4(f[0], f[1], f[2], -(float)((double)f[3] * f[3])));
    }
    rtbvh::Result R;
    rtbvh::build(geo.data(), desc->n_spheres, &R);
    if (!((double)R.r_scene < kBvhCoordLimit)) return RT_ERR_UNSUPPORTED;
    if (info) {
        info->n_nodes = (int32_t)R.nodes.size();
        info->depth = R.depth;
        info->max_leaf = R.max_leaf;
        info->r_scene = R.r_scene;
    }
    if (nodes) {
        if (nodes_cap < (int32_t)R.nodes.size()) return RT_ERR_INVALID_ARG;
        std::memcpy(nodes, R.nodes.data(), R.nodes.size() * sizeof(BvhNode));
    }
    if (prim_idx) std::memcpy(prim_idx, R.prim.data(), R.prim.size() * 4);
    return RT_OK;
}

rt_status rt_scene_upload(const rt_scene_desc* desc, void* stream, rt_scene** out) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    rt_status st = validate_desc(desc);
    if (st != RT_OK) return st;
    rt_scene* s = new (std::nothrow) rt_scene();
    if (!s) return RT_ERR_OOM;
    s->ns = desc->n_spheres;
    s->ns_pad = pad_spheres(desc->n_spheres);
    s->has_plane = desc->has_plane ? 1 : 0;
    s->nl = desc->n_lights;
    set_light_kinds(s, desc);
    s->bytes = scene_bytes(s->ns_pad);
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->dev, s->bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->pinned, s->bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->copy_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        rt_scene_free(s);
        return cuda_status(e);
    }
    pack_host(desc, s->ns_pad, static_cast<unsigned char*>(s->pinned));
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(s->dev, s->pinned, s->bytes, cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess) e = cudaEventRecord(s->copy_done, st_);
    if (e != cudaSuccess) {
        rt_scene_free(s);
        return cuda_status(e);
    }
    *out = s;
    return RT_OK;
}

rt_status rt_scene_update(rt_scene* s, const rt_scene_desc* desc, int32_t desc_on_device, void* stream) {
    if (!s || !desc) return RT_ERR_INVALID_ARG;
    if (desc->n_spheres != s->ns || (desc->has_plane ? 1 : 0) != s->has_plane || desc->n_lights != s->nl)
        return RT_ERR_INVALID_ARG;
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    if (desc_on_device) {
        if ((s->ns && !desc->spheres) || (s->nl && !desc->lights) || (s->has_plane && !desc->plane))
            return RT_ERR_INVALID_ARG;
        const int n = s->ns + 1;
        rt_pack_kernel<<<(n + 255) / 256, 256, 0, st_>>>(view_of(s), s->ns, desc->spheres, s->has_plane,
                                                         desc->plane, s->nl, desc->lights);
        g_launches++;
        s->host_current = false;
        s->kinds_known = false;
        if (s->bvh_state) s->bvh_state = 2;
        return cuda_status(cudaGetLastError());
    }
    rt_status st = validate_desc(desc);
    if (st != RT_OK) return st;
    set_light_kinds(s, desc);
    cudaError_t e = cudaEventSynchronize(s->copy_done);  // the previous copy has left the staging buffer
    if (e != cudaSuccess) return cuda_status(e);
    pack_host(desc, s->ns_pad, static_cast<unsigned char*>(s->pinned));
    e = cudaMemcpyAsync(s->dev, s->pinned, s->bytes, cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess) e = cudaEventRecord(s->copy_done, st_);
    if (e != cudaSuccess) return cuda_status(e);
    s->host_current = true;
    return s->bvh_state ? bvh_refresh(s, st_) : RT_OK;
}

rt_status rt_scene_free(rt_scene* s) {
    if (!s) return RT_OK;
    cudaDeviceSynchronize();
    if (s->dev) cudaFree(s->dev);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->copy_done) cudaEventDestroy(s->copy_done);
    if (s->bvh_dev) cudaFree(s->bvh_dev);
    if (s->bvh_pinned) cudaFreeHost(s->bvh_pinned);
    if (s->bvh_copy_done) cudaEventDestroy(s->bvh_copy_done);
    if (s->sky_dev) cudaFree(s->sky_dev);
    delete s;
    return RT_OK;
}

size_t rt_scene_bytes(const rt_scene* s) { return s ? s->bytes : 0; }

rt_status rt_scene_set_sky(rt_scene* s, const float* texels, int32_t width, int32_t height, void* stream) {
    if (!s) return RT_ERR_INVALID_ARG;
    if (!texels) {
        if (s->sky_dev) {
            cudaDeviceSynchronize();  // renders in flight may still read it
            cudaFree(s->sky_dev);
        }
        s->sky_dev = nullptr;
        s->sky_w = s->sky_h = 0;
        return RT_OK;
    }
    if (width < 1 || height < 1 || width > 16384 || height > 16384) return RT_ERR_INVALID_ARG;
    const size_t n = (size_t)width * (size_t)height * 4;
    if (!finite_all(texels, (int)n)) return RT_ERR_INVALID_ARG;  // n <= 2^30
    if (s->sky_dev && (s->sky_w != width || s->sky_h != height)) {
        cudaDeviceSynchronize();
        cudaFree(s->sky_dev);
        s->sky_dev = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!s->sky_dev) e = cudaMalloc(&s->sky_dev, n * 4);
    // pageable source: the runtime stages it before returning
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sky_dev, texels, n * 4, cudaMemcpyHostToDevice,
                                              static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status(e);
    s->sky_w = width;
    s->sky_h = height;
    return RT_OK;
}

rt_status rt_verlet_step(float* spheres_dev, float* prev_dev, int32_t n, const float* plane, float dt, float gravity,
                         float restitution, int32_t steps, void* stream) {
    if (n < 0 || steps < 0 || steps > (1 << 20) || (n && (!spheres_dev || !prev_dev)) ||
        (reinterpret_cast<uintptr_t>(spheres_dev) & 3) || (reinterpret_cast<uintptr_t>(prev_dev) & 3))
        return RT_ERR_INVALID_ARG;
    if (!(dt > 0.0f) || !std::isfinite(dt) || !std::isfinite(gravity) || !(restitution >= 0.0f) ||
        !(restitution <= 1.0f))
        return RT_ERR_INVALID_ARG;
    float4 pl = make_float4(0.f, 1.f, 0.f, 0.f);
    if (plane) {
        if (!finite_all(plane, 4)) return RT_ERR_INVALID_ARG;
        const double nn = (double)plane[0] * plane[0] + (double)plane[1] * plane[1] + (double)plane[2] * plane[2];
        if (std::fabs(nn - 1.0) > 1e-5) return RT_ERR_INVALID_ARG;
        pl = make_float4(plane[0], plane[1], plane[2], plane[3]);
    }
    if (n == 0 || steps == 0) return RT_OK;
    rt_verlet_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        spheres_dev, prev_dev, n, pl, plane ? 1 : 0, dt, gravity, restitution, steps);
    g_launches++;
    return cuda_status(cudaGetLastError());
}

size_t rt_hitrec_bytes(const rt_scene* s, const rt_render_params* p) {
    if (!s || !p || p->width < 1 || p->height < 1 || p->max_depth < 0) return 0;
    return (size_t)(p->max_depth + 1) * (size_t)(2 + s->nl) * (size_t)p->width * (size_t)p->height * 4u;
}

static rt_status render_region(const rt_scene* s, const rt_camera* cam, const rt_render_params* p, int32_t x0,
                               int32_t y0, int32_t rw, int32_t rh, void* out_dev, size_t out_pitch_bytes,
                               void* hitrec_dev, const rt_launch_config* cfg, void* stream, void* ws = nullptr,
                               size_t ws_bytes = 0) {
    rt_status st = validate_params(s, p);
    if (st != RT_OK) return st;
    if ((st = validate_camera(cam)) != RT_OK) return st;
    if (x0 < 0 || y0 < 0 || (x0 & 7) || rw < 1 || rh < 1 || x0 + rw > p->width || y0 + rh > p->height)
        return RT_ERR_INVALID_ARG;
    const size_t row = (size_t)rw * (p->out_format == RT_OUT_F32 ? 16 : 4);
    if (!out_dev || (reinterpret_cast<uintptr_t>(out_dev) & 15) || out_pitch_bytes < row || (out_pitch_bytes & 15))
        return RT_ERR_INVALID_ARG;
    if (hitrec_dev && ((reinterpret_cast<uintptr_t>(hitrec_dev) & 3) || rw != p->width || rh != p->height))
        return RT_ERR_INVALID_ARG;
    Launch L;
    if ((st = resolve_launch(cfg, &L)) != RT_OK) return st;
    Frame fr = make_frame(s, cam, p);
    fr.rx0 = x0;
    fr.ry0 = y0;
    fr.rx1 = x0 + rw;
    fr.ry1 = y0 + rh;
    const int nwarps = (L.bx * L.by) / 32;
    const int hstage = L.staging == 2 ? 2 : 1;  // how the header (and the whole table) is staged
    const dim3 block(32, nwarps);
    const dim3 grid((rw + L.bx - 1) / L.bx, (rh + L.by - 1) / L.by);
    const size_t plane = (size_t)p->width * (size_t)p->height;
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    float* hr = static_cast<float*>(hitrec_dev);
    if (L.accel) {
        if (s->bvh_state != 1) return RT_ERR_UNSUPPORTED;
        for (int k = 0; k < 3; ++k)
            if (!(std::fabs(cam->pos[k]) < kBvhCoordLimit)) return RT_ERR_UNSUPPORTED;
        BvhView bv;
        bv.nodes = static_cast<const BvhNode*>(s->bvh_dev);
        bv.n_nodes = s->bvh_info.n_nodes;
        bv.prim = reinterpret_cast<const int32_t*>(static_cast<const char*>(s->bvh_dev) +
                                                   (size_t)bv.n_nodes * sizeof(BvhNode));
        bv.r_scene = s->bvh_info.r_scene;
        const size_t bb = bvh_bytes(bv.n_nodes, s->ns);
        const size_t full = sizeof(SceneHdr) + (size_t)s->ns_pad * 16 + bb;
        const bool staged = bv.n_nodes > 0 && full + 4096 <= (size_t)(max_smem_optin() - 1024);
        const size_t smem = staged ? full : sizeof(SceneHdr);
        const uint32_t stage_b = staged ? (uint32_t)bb : 0u;
#define RT_BVH_LAUNCH(HR)                                                                                       \
    do {                                                                                                        \
        if ((st = ensure_smem(rt_fwd_bvh_kernel<HR>, smem)) != RT_OK) return st;                               \
        rt_fwd_bvh_kernel<HR><<<grid, block, smem, st_>>>(view_of(s), bv, stage_b, fr, out_dev, out_pitch_bytes, \
                                                         hr, plane, hstage, L.bx, L.by);                       \
    } while (0)
        if (hr) RT_BVH_LAUNCH(true);
        else RT_BVH_LAUNCH(false);
#undef RT_BVH_LAUNCH
        g_launches++;
        return cuda_status(cudaGetLastError());
    }
    // the sunflower table of a spherical light's samples follows the staged data (from
    // 16 samples on: with fewer, its set-up per CTA costs more than it saves)
    const int flower_n = s->any_sphere_light && p->shadow_samples >= 16 ? p->shadow_samples : 0;
    // no sky and, as far as the host knows, no spherical light: the lean kernels
    const bool lean = !s->sky_dev && s->kinds_known && !s->any_sphere_light;
    // sampled lights of several rays possible: the segment-test kernels with light_clear
    const bool sampled = p->shadow_samples > 1 && (!s->kinds_known || s->any_area || s->any_sphere_light);
    const bool chunked = use_tiled_loop(L, s->ns_pad, (size_t)flower_n * 16);
    const uint32_t flower_off = (uint32_t)((stage_smem_bytes(chunked, s->ns_pad, nwarps) + 15) / 16 * 16);
    const size_t smem = flower_off + (size_t)flower_n * 16;
    if (ws && !chunked) {
        // queued render: reset the counters, first pass, then one pass per bounce
        unsigned char* w = static_cast<unsigned char*>(ws);
        const unsigned cap = ws_cap(ws_bytes);
        if ((st = cuda_status(cudaMemsetAsync(ws, 0, kWsCtlBytes, st_))) != RT_OK) return st;
        const unsigned n_items = grid.x * grid.y * (unsigned)nwarps;
        // the shading path compiled in: the line filter from kFilterMinPad spheres on
        const bool filt = s->ns_pad >= kFilterMinPad;
#define RT_WS_LAUNCH(HR, FM)                                                                                      \
    do {                                                                                                          \
        if ((st = ensure_smem(rt_fwd_p0_kernel<HR, FM>, smem)) != RT_OK) return st;                              \
        if ((st = ensure_smem(rt_fwd_queue_kernel<HR, FM>, smem)) != RT_OK) return st;                           \
        const int threads = (int)(block.x * block.y);                                                             \
        const unsigned g0 = std::min<unsigned>((unsigned)resident_ctas(rt_fwd_p0_kernel<HR, FM>, threads, smem), \
                                               (n_items + nwarps - 1) / nwarps);                                  \
        rt_fwd_p0_kernel<HR, FM><<<g0, block, smem, st_>>>(view_of(s), fr, out_dev, out_pitch_bytes, hr, plane,   \
                                                           hstage, L.bx, L.by, (int)grid.x, n_items, w, cap,      \
                                                           flower_off, flower_n);                                 \
        g_launches++;                                                                                             \
        const unsigned gq =                                                                                       \
            std::min<unsigned>((unsigned)resident_ctas(rt_fwd_queue_kernel<HR, FM>, threads, smem),               \
                               std::max(1u, (cap + 32u * nwarps - 1) / (32u * nwarps)));                          \
        const unsigned wide_max = gq * (unsigned)nwarps * kWidePathsPerWarp;                                     \
        for (int k = 1; k <= p->max_depth && cap > 0; ++k) {                                                      \
            rt_fwd_queue_kernel<HR, FM><<<gq, block, smem, st_>>>(view_of(s), fr, out_dev, out_pitch_bytes, hr,   \
                                                                  plane, hstage, w, cap, k, wide_max, flower_off, \
                                                                  flower_n);                                      \
            g_launches++;                                                                                         \
        }                                                                                                         \
    } while (0)
        if (hr) {
            if (filt && lean) RT_WS_LAUNCH(true, 1 | kFmLean);
            else if (filt) RT_WS_LAUNCH(true, 1);
            else if (sampled) RT_WS_LAUNCH(true, kFmSkip);
            else RT_WS_LAUNCH(true, 0);
        } else {
            if (filt && lean) RT_WS_LAUNCH(false, 1 | kFmLean);
            else if (filt) RT_WS_LAUNCH(false, 1);
            else if (sampled) RT_WS_LAUNCH(false, kFmSkip);
            else RT_WS_LAUNCH(false, 0);
        }
#undef RT_WS_LAUNCH
        return cuda_status(cudaGetLastError());
    }
#define RT_FWD_LAUNCH(HR, CHK, FM)                                                                               \
    do {                                                                                                         \
        if ((st = ensure_smem(rt_fwd_kernel<HR, CHK, FM>, smem)) != RT_OK) return st;                           \
        rt_fwd_kernel<HR, CHK, FM><<<grid, block, smem, st_>>>(view_of(s), fr, out_dev, out_pitch_bytes, hr,    \
                                                              plane, hstage, L.bx, L.by, flower_off, flower_n); \
    } while (0)
    // the shading path compiled in: the line filter from kFilterMinPad spheres on
    // (the tiled loop keeps the segment test)
    const bool filt = !chunked && s->ns_pad >= kFilterMinPad;
    if (hr) {
        if (chunked) RT_FWD_LAUNCH(true, true, 0);
        else if (filt && lean) RT_FWD_LAUNCH(true, false, 1 | kFmLean);
        else if (filt) RT_FWD_LAUNCH(true, false, 1);
        else if (sampled) RT_FWD_LAUNCH(true, false, kFmSkip);
        else RT_FWD_LAUNCH(true, false, 0);
    } else {
        if (chunked) RT_FWD_LAUNCH(false, true, 0);
        else if (filt && lean) RT_FWD_LAUNCH(false, false, 1 | kFmLean);
        else if (filt) RT_FWD_LAUNCH(false, false, 1);
        else if (sampled) RT_FWD_LAUNCH(false, false, kFmSkip);
        else RT_FWD_LAUNCH(false, false, 0);
    }
#undef RT_FWD_LAUNCH
    g_launches++;
    return cuda_status(cudaGetLastError());
}

extern "C" rt_status rt_render(const rt_scene* s, const rt_camera* cam, const rt_render_params* p, void* out_dev,
                               size_t out_pitch_bytes, void* hitrec_dev, const rt_launch_config* cfg, void* stream) {
    if (!p) return RT_ERR_INVALID_ARG;
    return render_region(s, cam, p, 0, 0, p->width, p->height, out_dev, out_pitch_bytes, hitrec_dev, cfg, stream);
}

extern "C" rt_status rt_render_region(const rt_scene* s, const rt_camera* cam, const rt_render_params* p,
                                      int32_t x0, int32_t y0, int32_t width, int32_t height, void* out_dev,
                                      size_t out_pitch_bytes, const rt_launch_config* cfg, void* stream) {
    return render_region(s, cam, p, x0, y0, width, height, out_dev, out_pitch_bytes, nullptr, cfg, stream);
}

extern "C" size_t rt_render_workspace_bytes(const rt_scene* s, const rt_render_params* p) {
    if (!s || !p || p->width < 1 || p->height < 1) return 0;
    const size_t px = (size_t)p->width * (size_t)p->height;
    return kWsCtlBytes + 2 * kWsEntryBytes * ((px + 3) / 4);
}

extern "C" rt_status rt_render_ws(const rt_scene* s, const rt_camera* cam, const rt_render_params* p, void* out_dev,
                                  size_t out_pitch_bytes, void* hitrec_dev, const rt_launch_config* cfg,
                                  void* workspace_dev, size_t workspace_bytes, void* stream) {
    if (!p || !workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) & 255) || workspace_bytes < kWsCtlBytes)
        return RT_ERR_INVALID_ARG;
    return render_region(s, cam, p, 0, 0, p->width, p->height, out_dev, out_pitch_bytes, hitrec_dev, cfg, stream,
                         workspace_dev, workspace_bytes);
}

size_t rt_batch_workspace_bytes(int32_t n, const rt_scene* const* scenes, const rt_render_params* params,
                                const rt_launch_config* cfg) {
    Launch L;
    if (n < 1 || !scenes || !params || resolve_launch(cfg, &L) != RT_OK) return 0;
    size_t items = 0;
    int max_pad = 0;
    for (int i = 0; i < n; ++i) {
        const rt_render_params* p = &params[i];
        if (p->width < 1 || p->height < 1 || !scenes[i]) return 0;
        items += (size_t)((p->width + L.bx - 1) / L.bx) * (size_t)((p->height + L.by - 1) / L.by);
        max_pad = std::max(max_pad, scenes[i]->ns_pad);
    }
    int nd = 0, dm = 0;
    size_t co = 0, cb = 0;
    return batch_defer_layout(n, scenes, params, use_tiled_loop(L, max_pad), batch_items_offset(n) + items * 4, nullptr,
                              nullptr, &nd, &dm, &co, &cb);
}

rt_status rt_render_batch(int32_t n, const rt_scene* const* scenes, const rt_camera* cams,
                          const rt_render_params* params, void* const* outs_dev, const size_t* pitches,
                          void* workspace_dev, size_t workspace_bytes, const rt_launch_config* cfg, void* stream) {
    Launch L;
    rt_status st = resolve_launch(cfg, &L);
    if (st != RT_OK) return st;
    BatchPlanHost plan;
    if ((st = batch_pack(n, scenes, cams, params, outs_dev, pitches, L, &plan)) != RT_OK) return st;
    if (!workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) & 255) || workspace_bytes < plan.ws_bytes)
        return RT_ERR_INVALID_ARG;
    if ((st = batch_smem(plan.chunked, plan.smem)) != RT_OK) return st;
    int grid[3] = {0, 0, 0};
    if ((st = batch_grid(L, plan.smem, plan.chunked, grid)) != RT_OK) return st;
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    // pageable source: the runtime stages it before returning, so the vector may go
    cudaError_t e = cudaMemcpyAsync(workspace_dev, plan.table.data(), plan.table.size(), cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess && plan.ctl_bytes)
        e = cudaMemsetAsync(static_cast<unsigned char*>(workspace_dev) + plan.ctl_off, 0, plan.ctl_bytes, st_);
    if (e != cudaSuccess) return cuda_status(e);
    g_launches += batch_launch(plan.chunked, grid, L, plan.smem, st_, static_cast<unsigned char*>(workspace_dev), n,
                               plan.n_items, plan.n_filt, plan.n_defer, plan.dmax);
    return cuda_status(cudaGetLastError());
}

rt_status rt_batch_free(rt_batch* b) {
    if (!b) return RT_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->ws) cudaFree(b->ws);
    if (b->pinned) cudaFreeHost(b->pinned);
    delete b;
    return RT_OK;
}

rt_status rt_batch_create(int32_t n, const rt_scene* const* scenes, const rt_camera* cams,
                          const rt_render_params* params, void* const* outs_dev, const size_t* pitches,
                          const rt_launch_config* cfg, void* stream, rt_batch** out) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    Launch L;
    rt_status st = resolve_launch(cfg, &L);
    if (st != RT_OK) return st;
    BatchPlanHost plan;
    if ((st = batch_pack(n, scenes, cams, params, outs_dev, pitches, L, &plan)) != RT_OK) return st;
    if ((st = batch_smem(plan.chunked, plan.smem)) != RT_OK) return st;
    rt_batch* b = new (std::nothrow) rt_batch();
    if (!b) return RT_ERR_OOM;
    b->chunked = plan.chunked;
    b->n = n;
    b->n_items = plan.n_items;
    b->n_filt = plan.n_filt;
    b->n_defer = plan.n_defer;
    b->dmax = plan.dmax;
    b->ctl_off = plan.ctl_off;
    b->ctl_bytes = plan.ctl_bytes;
    b->L = L;
    b->smem = plan.smem;
    b->ws_bytes = plan.ws_bytes;
    b->table_bytes = plan.table.size();
    if ((st = batch_grid(L, plan.smem, plan.chunked, b->grid)) != RT_OK) {
        rt_batch_free(b);
        return st;
    }
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&b->ws, b->ws_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->pinned, b->table_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        std::memcpy(b->pinned, plan.table.data(), b->table_bytes);
        e = cudaMemcpyAsync(b->ws, b->pinned, b->table_bytes, cudaMemcpyHostToDevice, st_);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ready, st_);
    // graph: reset the two work counters and the bounce queues' counters, then the
    // persistent kernel instances and the queue passes
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(b->ws, 0, 2 * sizeof(unsigned), b->cap);
        if (b->ctl_bytes) cudaMemsetAsync(static_cast<unsigned char*>(b->ws) + b->ctl_off, 0, b->ctl_bytes, b->cap);
        b->launches = batch_launch(b->chunked, b->grid, L, b->smem, b->cap, static_cast<unsigned char*>(b->ws), n,
                                   b->n_items, b->n_filt, b->n_defer, b->dmax);
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &b->graph);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        rt_batch_free(b);
        return cuda_status(e);
    }
    *out = b;
    return RT_OK;
}

rt_status rt_batch_launch(rt_batch* b, void* stream) {
    if (!b || !b->exec) return RT_ERR_INVALID_ARG;
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamWaitEvent(st_, b->ready, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st_);
    if (e == cudaSuccess) g_launches += b->launches;
    return cuda_status(e);
}

size_t rt_grad_count(const rt_scene* s) { return s ? (size_t)grad_count(s->ns, s->nl) : 0; }

size_t rt_backward_workspace_bytes(const rt_scene* s, const rt_render_params* p, const rt_launch_config* cfg) {
    Launch L;
    if (!s || !p || p->width < 1 || p->height < 1 || resolve_launch(cfg, &L) != RT_OK) return 0;
    const size_t ctas = (size_t)((p->width + L.bx - 1) / L.bx) * (size_t)((p->height + L.by - 1) / L.by);
    return ctas * (size_t)grad_count(s->ns, s->nl) * 4;
}

rt_status rt_render_backward(const rt_scene* s, const rt_camera* cam, const rt_render_params* p,
                             const float* dl_dimg_dev, size_t dl_pitch_bytes, const void* hitrec_dev,
                             float* grad_dev, void* workspace_dev, size_t workspace_bytes,
                             const rt_launch_config* cfg, void* stream) {
    rt_status st = validate_params(s, p);
    if (st != RT_OK) return st;
    if ((st = validate_camera(cam)) != RT_OK) return st;
    if (s->sky_dev) return RT_ERR_UNSUPPORTED;
    if (!dl_dimg_dev || (reinterpret_cast<uintptr_t>(dl_dimg_dev) & 15) || dl_pitch_bytes < (size_t)p->width * 16 ||
        (dl_pitch_bytes & 15) || !grad_dev || (hitrec_dev && (reinterpret_cast<uintptr_t>(hitrec_dev) & 3)))
        return RT_ERR_INVALID_ARG;
    Launch L;
    if ((st = resolve_launch(cfg, &L)) != RT_OK) return st;
    if (L.accel) return RT_ERR_UNSUPPORTED;
    const size_t need = rt_backward_workspace_bytes(s, p, cfg);
    if (!workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) & 15) || workspace_bytes < need)
        return RT_ERR_INVALID_ARG;
    const int G = grad_count(s->ns, s->nl);
    const int nwarps = (L.bx * L.by) / 32;
    const size_t tabs = (size_t)nwarps * G * 4;
    const bool chunked = L.staging == 3 || stage_smem_bytes(false, s->ns_pad, nwarps) + tabs + kStaticSmemReserve >
                                               (size_t)max_smem_optin();
    const size_t smem = stage_smem_bytes(chunked, s->ns_pad, nwarps) + tabs;
    const int hstage = L.staging == 2 ? 2 : 1;
    const Frame fr = make_frame(s, cam, p);
    const dim3 block(32, nwarps);
    const dim3 grid((p->width + L.bx - 1) / L.bx, (p->height + L.by - 1) / L.by);
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    float* parts = static_cast<float*>(workspace_dev);
    const float* hr = static_cast<const float*>(hitrec_dev);
#define RT_BWD_LAUNCH(HR, CHK)                                                                                   \
    do {                                                                                                         \
        if ((st = ensure_smem(rt_bwd_kernel<HR, CHK>, smem)) != RT_OK) return st;                               \
        rt_bwd_kernel<HR, CHK><<<grid, block, smem, st_>>>(view_of(s), fr, dl_dimg_dev, dl_pitch_bytes, hr, parts, \
                                                          G, hstage, L.bx, L.by);                               \
    } while (0)
    if (hr) {
        if (chunked) RT_BWD_LAUNCH(true, true);
        else RT_BWD_LAUNCH(true, false);
    } else {
        if (chunked) RT_BWD_LAUNCH(false, true);
        else RT_BWD_LAUNCH(false, false);
    }
#undef RT_BWD_LAUNCH
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    rt_grad_reduce_kernel<<<(G + 31) / 32, 32 * kReduceWarps, 0, st_>>>(parts, (int)(grid.x * grid.y), G,
                                                                   grad_dev);
    g_launches++;
    return cuda_status(cudaGetLastError());
}

rt_status rt_selftest_wait_timeout(uint32_t polls, void* stream) {
    if (polls == 0 || polls > (1u << 20)) return RT_ERR_INVALID_ARG;
    rt_selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(polls);
    g_launches++;
    return cuda_status(cudaGetLastError());
}

rt_status rt_device_errors(void* stream, uint32_t* bits) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status(e);
    uint32_t v = 0;
    e = cudaMemcpyFromSymbol(&v, g_err_word, sizeof(v));
    if (e != cudaSuccess) return cuda_status(e);
    if (bits) *bits = v;
    if (v) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_err_word, &z, sizeof(z));
        return RT_ERR_TIMEOUT;
    }
    return RT_OK;
}

}  // extern "C"

// ============================================================ batch without allocation
// Scratch of rt_render_batch_noalloc: work counter, frame table and item list (the
// workspace layout of rt_render_batch) in a fixed array of the device image.  In
// host code `g_noalloc_scratch` only stands for the symbol; its device address
// comes from cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_dev_ptr[kMaxDevices] = {};
// host image of the tables, static so that no call touches the heap
alignas(256) unsigned char g_noalloc_host[RT_NOALLOC_SCRATCH_BYTES];

// The workspace image of rt_render_batch, written into a fixed buffer without any
// heap use (line-filter frames first, each class in longest-first order by tile
// cost, tiles in raster order).
rt_status batch_pack_fixed(int n, const rt_scene* const* scenes, const rt_camera* cams,
                           const rt_render_params* params, void* const* outs, const size_t* pitches,
                           const Launch& L, unsigned char* buf, size_t cap, size_t* bytes, int* n_items_out,
                           int* n_filt_out, size_t* smem_out, bool* chunked_out) {
    if (n < 1 || !scenes || !cams || !params || !outs || !pitches) return RT_ERR_INVALID_ARG;
    if (L.bx * L.by > kBatchMaxThreads) return RT_ERR_INVALID_ARG;
    if (L.accel) return RT_ERR_UNSUPPORTED;
    if (n > RT_NOALLOC_MAX_FRAMES) return RT_ERR_EXCEEDS_SCRATCH;
    int order[RT_NOALLOC_MAX_FRAMES];
    int tiles[RT_NOALLOC_MAX_FRAMES];
    long long n_items = 0, n_filt = 0;
    const size_t items_off = batch_items_offset(n);
    if (items_off > cap) return RT_ERR_EXCEEDS_SCRATCH;
    std::memset(buf, 0, items_off);  // the work counter starts at zero
    BatchFrame* frames = reinterpret_cast<BatchFrame*>(buf + batch_frames_offset());
    int max_pad = 0;
    for (int i = 0; i < n; ++i)
        if (scenes[i]) max_pad = std::max(max_pad, scenes[i]->ns_pad);
    const bool chunked = use_tiled_loop(L, max_pad);
    for (int i = 0; i < n; ++i) {
        const rt_scene* s = scenes[i];
        const rt_render_params* p = &params[i];
        rt_status st = validate_params(s, p);
        if (st != RT_OK) return st;
        if ((st = validate_camera(&cams[i])) != RT_OK) return st;
        const size_t row = (size_t)p->width * (p->out_format == RT_OUT_F32 ? 16 : 4);
        if (!outs[i] || (reinterpret_cast<uintptr_t>(outs[i]) & 15) || pitches[i] < row || (pitches[i] & 15))
            return RT_ERR_INVALID_ARG;
        BatchFrame& B = frames[i];
        B.sv = view_of(s);
        B.fr = make_frame(s, &cams[i], p);
        B.out = outs[i];
        B.pitch = pitches[i];
        B.stage_bytes = (uint32_t)(chunked ? sizeof(SceneHdr) : sizeof(SceneHdr) + (size_t)s->ns_pad * 16);
        B.tiles_x = (p->width + L.bx - 1) / L.bx;
        const long long t = (long long)B.tiles_x * ((p->height + L.by - 1) / L.by);
        if (t >= (1ll << kItemTileBits)) return RT_ERR_UNSUPPORTED;
        tiles[i] = (int)t;
        n_items += t;
        const bool filt = batch_filtered(s, chunked);
        if (filt) n_filt += t;
        // insertion into the order of rt_render_batch: line-filter frames first, each
        // class longest-first (stable: ties keep input order)
        const double c = tile_cost(s, p);
        int j = i;
        while (j > 0) {
            const int q = order[j - 1];
            const bool fq = batch_filtered(scenes[q], chunked);
            if (!(filt && !fq) && !(filt == fq && tile_cost(scenes[q], &params[q]) < c)) break;
            order[j] = order[j - 1];
            --j;
        }
        order[j] = i;
    }
    const size_t total = items_off + (size_t)n_items * 4;
    if (total > cap) return RT_ERR_EXCEEDS_SCRATCH;
    uint32_t* items = reinterpret_cast<uint32_t*>(buf + items_off);
    size_t k = 0;
    for (int oi = 0; oi < n; ++oi) {
        const int f = order[oi];
        for (int t = 0; t < tiles[f]; ++t) items[k++] = ((uint32_t)f << kItemTileBits) | (uint32_t)t;
    }
    *bytes = total;
    *n_items_out = (int)n_items;
    *n_filt_out = (int)n_filt;
    *smem_out = stage_smem_bytes(chunked, max_pad, (L.bx * L.by) / 32);
    *chunked_out = chunked;
    return RT_OK;
}

}  // namespace

extern "C" rt_status rt_render_batch_noalloc(int32_t n, const rt_scene* const* scenes, const rt_camera* cams,
                                             const rt_render_params* params, void* const* outs_dev,
                                             const size_t* pitches, const rt_launch_config* cfg, void* stream) {
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    // A captured call would record a copy from the shared static host image, which a
    // later call overwrites before the graph replays: refuse capture, before any set-up.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st_, &cap);
    if (e != cudaSuccess) return cuda_status(e);
    if (cap != cudaStreamCaptureStatusNone) return RT_ERR_UNSUPPORTED;
    Launch L;
    rt_status st = resolve_launch(cfg, &L);
    if (st != RT_OK) return st;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return RT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_noalloc_mu);
    // set-up, once per device, with that device current
    if (!g_noalloc_dev_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        g_noalloc_dev_ptr[dev] = ptr;
    }
    size_t bytes = 0, smem = 0;
    int n_items = 0, n_filt = 0;
    bool chunked = false;
    st = batch_pack_fixed(n, scenes, cams, params, outs_dev, pitches, L, g_noalloc_host, sizeof(g_noalloc_host),
                          &bytes, &n_items, &n_filt, &smem, &chunked);
    if (st != RT_OK) return st;
    if ((st = batch_smem(chunked, smem)) != RT_OK) return st;
    int grid[3] = {0, 0, 0};
    if ((st = batch_grid(L, smem, chunked, grid)) != RT_OK) return st;
    // pageable source: staged by the runtime before the call returns, so the static
    // host image is free for the next call
    e = cudaMemcpyAsync(g_noalloc_dev_ptr[dev], g_noalloc_host, bytes, cudaMemcpyHostToDevice, st_);
    if (e != cudaSuccess) return cuda_status(e);
    // no bounce queues: the scratch holds the work tables only
    g_launches += batch_launch(chunked, grid, L, smem, st_, static_cast<unsigned char*>(g_noalloc_dev_ptr[dev]), n,
                               n_items, n_filt, 0, 0);
    return cuda_status(cudaGetLastError());
}
