// rt_batch.cuh -- batched persistent render: many scenes of uneven sphere counts
// and resolutions in one launch.  Work items are (scene, tile) pairs in a list
// ordered by estimated tile cost (longest first); each CTA claims the next item
// with one atomicAdd on a work counter until the list is exhausted, restaging the
// scene table in shared memory whenever its scene changes.  The counter only ever
// advances, so no CTA waits on another.
#pragma once

#include "rt_errword.cuh"
#include "rt_stage.cuh"
#include "rt_trace.cuh"

namespace rtd {

// One frame of the batch (device-resident descriptor).
struct __align__(16) BatchFrame {
    SceneView sv;
    Frame fr;
    void* out;
    size_t pitch;
    uint32_t stage_bytes;  // header + geometry bytes staged in shared memory
    int tiles_x;
    // bounce queues of a deferring frame (workspace offsets), q_cap = 0: none
    uint64_t q_ctl, q_ent;
    uint32_t q_cap;
};

// Bounce queues of a deferring frame -- the queued render of rt_render_ws inside the
// batch: the line-filter instance hands a path whose bounce-1 ray hits to the
// frame's queue 1, and pass k (rt_batch_queue_kernel) shades bounce k of the
// frame's queue-k paths and hands those whose next ray hits to queue k + 1.  Per
// frame: a control block of append and claim counters per bounce, then two queues
// of q_cap entries (64 bytes each: the path state, as rt_render_ws stores it) used
// in turn, queue k in the first when k is odd.  A path's arithmetic is the same
// wherever it runs, so the images equal the one-pass render's bit for bit.
struct BatchQueueCtl {
    unsigned count[RT_MAX_DEPTH + 2];  // entries appended to queue k (may pass q_cap)
    unsigned head[RT_MAX_DEPTH + 2];   // entries claimed from queue k
};
constexpr size_t kBatchQCtl = 256;
static_assert(sizeof(BatchQueueCtl) <= kBatchQCtl, "batch queue control block");
__device__ __forceinline__ PathQueue batch_queue(unsigned char* ws, const BatchFrame& B, int k) {
    BatchQueueCtl* c = reinterpret_cast<BatchQueueCtl*>(ws + B.q_ctl);
    float4* q = reinterpret_cast<float4*>(ws + B.q_ent + ((k & 1) ? 0 : (size_t)B.q_cap * 64));
    return PathQueue{q, &c->count[k], B.q_cap};
}

// Workspace layout (device): [two work counters, padded to 256 B][BatchFrame x n]
// [item x n_items] with item = (frame index << 20) | tile index.  The items of the
// frames rendered with the line filter come first, then the others; each class is
// in longest-first order and is worked through by its own instance of the kernel
// (FM = 1 / 0), which claims items with counter FM.
constexpr int kItemTileBits = 20;
constexpr int kBatchMaxThreads = 128;  // launch bounds of the batch kernel (segment test: 6 CTAs per SM, 13.20 ms
                                        // for the 64-scene batch on B300 against 13.50 at 5 and 13.60 at 7)
constexpr size_t kWsHead = 256;

__host__ __device__ inline size_t batch_frames_offset() { return kWsHead; }
__host__ __device__ inline size_t batch_items_offset(int n) {
    return (kWsHead + (size_t)n * sizeof(BatchFrame) + 255) / 256 * 256;
}

// FM: the shading path of every frame of this instance's class -- 0 the segment test
// alone (80 registers, 6 CTAs per SM), 1 the line filter with the cone passes, for
// frames of kFilterMinPad spheres or more (128 registers, 4 CTAs per SM, as the
// per-frame kernels).  Both give the same bits (the filter's and the cones' bounds).
// item0 / n_items: this class's items in the list.
template <bool CH, int FM>
__global__ void __launch_bounds__(128, FM == 1 ? 4 : 6) rt_batch_kernel(unsigned char* __restrict__ ws, int n_frames,
                                                                         int item0, int n_items, int staging,
                                                                         int block_x, int block_y) {
    static_assert(!(CH && FM == 1), "the line filter reads the staged table");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int s_item[2];
    __shared__ Frame s_fr;
    __shared__ void* s_out;
    __shared__ size_t s_pitch;
    __shared__ int s_tiles_x;
    __shared__ const float4* s_geo;
    __shared__ const float4* s_mat;
    __shared__ const float4* s_mat2;
    __shared__ SkyView s_sky;
    __shared__ PathQueue s_q1;  // the frame's queue 1, or ent = null: no deferral
    unsigned* counter = reinterpret_cast<unsigned*>(ws) + FM;
    const BatchFrame* frames = reinterpret_cast<const BatchFrame*>(ws + batch_frames_offset());
    const uint32_t* items = reinterpret_cast<const uint32_t*>(ws + batch_items_offset(n_frames)) + item0;
    float cone_r2 = 0.0f, cone_cmax = 0.0f;  // of the staged scene (line-filter instance)
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    int cur = -1;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int wpr = block_x >> 3;
    // the next item is claimed while the current one renders: two slots, swapped
    // after the barrier that ends each tile
    if (tid == 0) s_item[0] = (int)atomicAdd(counter, 1u);
    __syncthreads();
    int buf = 0;
#pragma unroll 1
    while (true) {
        const int it = s_item[buf];
        if (it >= n_items) break;  // the same value in every thread
        if (tid == 0) s_item[buf ^ 1] = (int)atomicAdd(counter, 1u);
        const uint32_t code = __ldg(items + it);
        const int fi = (int)(code >> kItemTileBits);
        const int tile = (int)(code & ((1u << kItemTileBits) - 1u));
        if (fi != cur) {
            const BatchFrame* B = frames + fi;
            if (tid == 0) {
                s_fr = B->fr;
                s_out = B->out;
                s_pitch = B->pitch;
                s_tiles_x = B->tiles_x;
                s_geo = B->sv.geo;
                s_mat = B->sv.mat;
                s_mat2 = B->sv.mat2;
                s_sky = B->sv.sky;
                s_q1 = (FM == 1 && B->q_cap > 0 && B->fr.D >= 1) ? batch_queue(ws, *B, 1)
                                                                 : PathQueue{nullptr, nullptr, 0u};
                // shared memory was last read by the generic proxy; order those reads
                // before the bulk copy's writes
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            if (!stage_to_smem(smem, B->sv.hdr, B->stage_bytes, staging, &bar, phase, &g_err_word)) return;
            if constexpr (FM == 1) {
                StagedScene cs{};
                staged_cone(reinterpret_cast<const float4*>(smem + sizeof(SceneHdr)),
                            reinterpret_cast<const SceneHdr*>(smem)->ns_pad, cs);
                cone_r2 = cs.cone_r2;
                cone_cmax = cs.cone_cmax;
            }
            cur = fi;
        }
        float4* tab = reinterpret_cast<float4*>(smem + sizeof(SceneHdr));
        StagedScene sc{reinterpret_cast<const SceneHdr*>(smem), CH ? nullptr : tab, s_geo,
                       CH ? tab + (size_t)warp * kChunk : nullptr, s_mat, s_mat2};
        sc.sky = s_sky;
        sc.cone_r2 = cone_r2;
        sc.cone_cmax = cone_cmax;
        const int tx = tile % s_tiles_x, ty = tile / s_tiles_x;
        const int x = tx * block_x + (warp % wpr) * 8 + (lane & 7);
        const int y = ty * block_y + (warp / wpr) * 4 + (lane >> 3);
        const bool valid = x < s_fr.W && y < s_fr.H;
        if constexpr (FM == 1) {
            const PathQueue q1 = s_q1;
            render_pixel<false, CH, false, FM>(sc, s_fr, x, y, valid, s_out, s_pitch, nullptr, 0,
                                               q1.ent ? &q1 : nullptr);
        } else {
            render_pixel<false, CH, false, FM>(sc, s_fr, x, y, valid, s_out, s_pitch, nullptr, 0);
        }
        __syncthreads();  // every thread is done with this tile, its slot and the staged scene
        buf ^= 1;
    }
}

// Pass k >= 1 of the batch's bounce queues: persistent CTAs walk the deferring
// frames (the list after the items) in order; for each frame whose queue k still
// holds unclaimed paths, a CTA stages its scene and its warps claim 32 paths at a
// time (trace_queued: shade bounce k, trace the next ray, hand a hit on to queue
// k + 1); then the CTA moves on.  Each queue only ever advances its claim counter,
// so no CTA waits on another.
template <int FM>
__global__ void __launch_bounds__(128, FM == 1 ? 4 : 6) rt_batch_queue_kernel(unsigned char* __restrict__ ws,
                                                                               int n_frames, int n_items, int n_defer,
                                                                               int k, int staging) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int s_go;
    __shared__ Frame s_fr;
    __shared__ void* s_out;
    __shared__ size_t s_pitch;
    __shared__ const float4* s_geo;
    __shared__ const float4* s_mat;
    __shared__ const float4* s_mat2;
    __shared__ SkyView s_sky;
    const BatchFrame* frames = reinterpret_cast<const BatchFrame*>(ws + batch_frames_offset());
    const int* defer =
        reinterpret_cast<const int*>(ws + batch_items_offset(n_frames) + (size_t)n_items * sizeof(uint32_t));
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = threadIdx.x;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    int cur = -1;
    float cone_r2 = 0.0f, cone_cmax = 0.0f;
#pragma unroll 1
    for (int j = 0; j < n_defer; ++j) {
        const int fi = defer[j];
        const BatchFrame* B = frames + fi;
        BatchQueueCtl* ctl = reinterpret_cast<BatchQueueCtl*>(ws + B->q_ctl);
        const unsigned n = k <= B->fr.D ? min(*reinterpret_cast<volatile unsigned*>(&ctl->count[k]), B->q_cap) : 0u;
        if (tid == 0) s_go = n > 0 && *reinterpret_cast<volatile unsigned*>(&ctl->head[k]) < n;
        __syncthreads();
        const bool go = s_go != 0;
        __syncthreads();  // every thread has read s_go
        if (!go) continue;
        if (fi != cur) {
            if (tid == 0) {
                s_fr = B->fr;
                s_out = B->out;
                s_pitch = B->pitch;
                s_geo = B->sv.geo;
                s_mat = B->sv.mat;
                s_mat2 = B->sv.mat2;
                s_sky = B->sv.sky;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            if (!stage_to_smem(smem, B->sv.hdr, B->stage_bytes, staging, &bar, phase, &g_err_word)) return;
            if constexpr (FM == 1) {
                StagedScene cs{};
                staged_cone(reinterpret_cast<const float4*>(smem + sizeof(SceneHdr)),
                            reinterpret_cast<const SceneHdr*>(smem)->ns_pad, cs);
                cone_r2 = cs.cone_r2;
                cone_cmax = cs.cone_cmax;
            }
            cur = fi;
        }
        StagedScene sc{reinterpret_cast<const SceneHdr*>(smem), reinterpret_cast<const float4*>(smem + sizeof(SceneHdr)),
                       s_geo, nullptr, s_mat, s_mat2};
        sc.sky = s_sky;
        sc.cone_r2 = cone_r2;
        sc.cone_cmax = cone_cmax;
        const PathQueue cq = batch_queue(ws, *B, k), nq = batch_queue(ws, *B, k + 1);
#pragma unroll 1
        while (true) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&ctl->head[k], 32u);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= n) break;
            const unsigned i = base + (unsigned)lane;
            if (i < n) trace_queued<false, FM>(sc, s_fr, cq.ent + (size_t)i * 4, k, nq, s_out, s_pitch, nullptr, 0);
            __syncwarp();
        }
        __syncthreads();  // every warp is done with this frame's staged scene
    }
}

}  // namespace rtd
