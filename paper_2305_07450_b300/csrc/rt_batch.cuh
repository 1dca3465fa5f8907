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
};

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
        render_pixel<false, CH, false, FM>(sc, s_fr, x, y, valid, s_out, s_pitch, nullptr, 0);
        __syncthreads();  // every thread is done with this tile, its slot and the staged scene
        buf ^= 1;
    }
}

}  // namespace rtd
