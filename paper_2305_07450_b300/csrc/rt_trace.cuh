// rt_trace.cuh -- per-pixel path of the Whitted ray tracer (arXiv 2305.07450,
// Section 3) in FP32: primary ray, brute-force closest hit, shading with hard or
// sampled shadows (the segment test, and in front of it for large scenes a line
// filter that decides most sphere-segment pairs in fewer operations with the same
// verdict, and cone tests -- a sampled light's cone per lane, warp cones for point
// lights and for each batch of rays -- that skip blocks of spheres no segment or ray
// can reach), register-resident reflection loop, and the bounce queues of the queued
// render with their one-path-per-warp ("wide") form.  Every skip is proved by an
// error bound stated beside it, so each result is the brute-force method's, bit for
// bit.  Shared by the per-frame and queued kernels, the batched persistent kernel and
// the adjoint's recompute mode.
#pragma once

#include "rt_bvh.cuh"
#include "rt_device.cuh"

namespace rtd {

// Staged scene as one CTA sees it: header in shared memory; the geometry table
// either whole in shared memory (geo), or -- when it does not fit -- read chunk by
// chunk into the warp's own slot of kChunk entries (chunk), the tiled loop; the
// global table (geo_g) and the materials are read through the read-only cache.
constexpr int kChunk = 64;

struct StagedScene {
    const SceneHdr* hdr;   // shared
    const float4* geo;     // shared, hdr->ns_pad entries (whole-table staging)
    const float4* geo_g;   // global, hdr->ns_pad entries
    float4* chunk;         // shared, this warp's kChunk entries (tiled loop)
    const float4* mat;     // global
    const float4* mat2;    // global
    BvhView bvh;           // hierarchy over the spheres (ACC kernels only)
    SkyView sky;           // panorama of the misses (null: black)
    const float4* flower;  // shared sunflower table (sunflower_table), or null: computed per sample
    float cone_r2 = 0.0f;  // rho^2 of the cone pre-pass (staged_cone), or 0: no pre-pass
    float cone_cmax = 0.0f;  // bound on the centres' |c| (staged_cone)
};

// The sunflower points of a spherical light that do not depend on the hit: for
// sample s of n, (sqrt(s / n), cos 2 pi f_s, sin 2 pi f_s) with f_s = frac(s (3 -
// sqrt 5) / 2) -- the values sample_point otherwise computes per sample, by the same
// operations.  Written into shared memory at `tab` by all threads of the CTA (which
// must all call), for s < n_tab; returns the table (null when n_tab is 0).
__device__ __forceinline__ const float4* sunflower_table(float4* tab, int n_tab, int nsamp) {
    if (n_tab <= 0) return nullptr;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nth = blockDim.x * blockDim.y;
    for (int s = tid; s < n_tab; s += nth) {
        const float q = sqrtf((float)s / (float)nsamp);
        const uint32_t frac = (uint32_t)s * 0x61C88647u;  // 2^32 (3 - sqrt 5) / 2
        float sn, cs;
        sincospif((float)(frac >> 8) * (1.0f / 8388608.0f), &sn, &cs);  // 2 frac
        tab[s] = make_float4(q, cs, sn, 0.0f);
    }
    __syncthreads();
    return tab;
}

// Tiled loop: entries [c0, c0 + m) of the global table into the warp's slot, copied
// by the lanes in `mask` (the lanes that run the loop), 16 bytes per lane per step.
__device__ __forceinline__ void stage_chunk(const StagedScene& sc, unsigned mask, int c0, int m) {
    const int lane = threadIdx.x & 31;
    const int rank = __popc(mask & ((1u << lane) - 1u)), cnt = __popc(mask);
    __syncwarp(mask);
    for (int k = rank; k < m; k += cnt) sc.chunk[k] = __ldg(sc.geo_g + c0 + k);
    __syncwarp(mask);
}

// ---------------------------------------------------------------- Section 3.2-3.3
// NDC of pixel (x, y): the shorter side spans [-1, 1] (NDC listing of Section 3.2,
// integer pixel coordinates): u = (2x - W) / m, v = (H - 2y) / m, m = min(W, H).
// The direction is normalize(u R + v U + b F): the paper's normalize(P - C) with
// P = (u, v, 0), C = (0, 0, -b), rotated by pitch then yaw (Section 3.3.1), with
// the rotation folded into the camera basis on the host.
__device__ __forceinline__ f3 primary_dir(const Frame& fr, int x, int y) {
    const float u = __fdiv_rn((float)(2 * x - fr.W), (float)fr.m);
    const float v = __fdiv_rn((float)(fr.H - 2 * y), (float)fr.m);
    f3 d = mk3(fr.fwd.x, fr.fwd.y, fr.fwd.z);
    d = fma3(mk3(fr.up.x, fr.up.y, fr.up.z), v, d);
    d = fma3(mk3(fr.right.x, fr.right.y, fr.right.z), u, d);
    return normalize(d);
}

// ---------------------------------------------------------------- Section 3.4.1
// Closest of all primitives by brute force; spheres 0..N-1 then the plane N; a
// strictly smaller distance wins, so ties keep the lower index.  Sphere test: the
// vector from the ray's line to the centre has length |(c - o) x d| (d is a unit
// vector), so m = |c x d - o x d|^2 - r^2 is the negated discriminant; with
// -(o x d) formed once per ray, a pair of spheres costs three packed FMAs per
// component and three for the square (9 packed instructions; the projection form
// oc - (oc.d) d needs 12).  Both forms round the same long terms (|c|, |o| of tens
// of units) once each and neither subtracts squares of them, so m keeps an
// absolute error of a few ulps of those terms.  A hit needs m < 0; its distance
// tca -+ sqrt(-m), tca = c.d - o.d, is formed only for those spheres: the near
// root if it is > 0, else the far one.  The two spheres of a pair are tested by
// the same packed instructions; a block of kPad spheres computes its m branch-free
// and takes the roots only when one of them is negative (one branch per block).
struct RayPair {  // -o in both halves of a pair (shadow segments)
    float2 nox, noy, noz;
};
__device__ __forceinline__ RayPair ray_pair(f3 o) { return RayPair{dup2(-o.x), dup2(-o.y), dup2(-o.z)}; }

struct RayCross {  // d, -d and -(o x d) in both halves of a pair; -(o.d)
    float2 dx, dy, dz, ndx, ndy, ndz, nwx, nwy, nwz;
    float nod;
};
__device__ __forceinline__ RayCross ray_cross(f3 o, f3 d) {
    const RayX x = ray_x(o, d);
    return RayCross{dup2(d.x),    dup2(d.y),    dup2(d.z),    dup2(-d.x), dup2(-d.y),
                    dup2(-d.z),   dup2(x.nw.x), dup2(x.nw.y), dup2(x.nw.z), x.nod};
}

// m of sphere hf of pair q: the packed operations of the pair, one half.
__device__ __forceinline__ float sphere_m(const float4 A, const float4 B, int hf, const RayCross& r) {
    const float cx = hf ? A.y : A.x, cy = hf ? A.w : A.z, cz = hf ? B.y : B.x, nr = hf ? B.w : B.z;
    const float px = fmaf(cy, r.dz.x, fmaf(cz, r.ndy.x, r.nwx.x));
    const float py = fmaf(cz, r.dx.x, fmaf(cx, r.ndz.x, r.nwy.x));
    const float pz = fmaf(cx, r.dy.x, fmaf(cy, r.ndx.x, r.nwz.x));
    return fmaf(px, px, fmaf(py, py, fmaf(pz, pz, nr)));
}
// closest_block with the roots of the flagged spheres in one copy of the code.
__device__ __forceinline__ void closest_block_compact(const float4* __restrict__ geo, int base, const RayCross& r,
                                                      float& tb, int& best) {
    uint32_t neg = 0;  // bit i: sphere i's m has its sign bit set
#pragma unroll
    for (int q = 0; q < kPad / 2; ++q) {
        const float4 A = geo[2 * q], B = geo[2 * q + 1];
        const float2 cx = make_float2(A.x, A.y), cy = make_float2(A.z, A.w), cz = make_float2(B.x, B.y);
        const float2 px = fma2(cy, r.dz, fma2(cz, r.ndy, r.nwx));
        const float2 py = fma2(cz, r.dx, fma2(cx, r.ndz, r.nwy));
        const float2 pz = fma2(cx, r.dy, fma2(cy, r.ndx, r.nwz));
        const float2 m = fma2(px, px, fma2(py, py, fma2(pz, pz, make_float2(B.z, B.w))));
        neg |= ((__float_as_uint(m.x) >> 31) | ((__float_as_uint(m.y) >> 31) << 1)) << (2 * q);
    }
    // the roots of the flagged spheres in index order, one copy of the code: m is
    // formed again by the same operations (a fused multiply-add per lane, so the
    // scalar form gives the packed one's bits)
#pragma unroll 1
    while (neg) {
        const int i = __ffs(neg) - 1;
        neg &= neg - 1u;
        const float4 A = geo[2 * (i >> 1)], B = geo[2 * (i >> 1) + 1];
        const int hf = i & 1;
        const float mm = sphere_m(A, B, hf, r);
        if (mm < 0.0f) {
            const float cx = hf ? A.y : A.x, cy = hf ? A.w : A.z, cz = hf ? B.y : B.x;
            const float tc = fmaf(cx, r.dx.x, fmaf(cy, r.dy.x, fmaf(cz, r.dz.x, r.nod)));
            const float s = __fsqrt_rn(-mm);
            float t = tc - s;
            if (t <= 0.0f) t = tc + s;
            if (t > 0.0f && t < tb) {
                tb = t;
                best = base + i;
            }
        }
    }
}

// One block of kPad spheres (kPad / 2 pairs at geo[0..kPad)); base = index of its first sphere.
// COMPACT: the roots of the flagged spheres through one copy of the code (the
// line-filter kernels, whose code outgrows the instruction cache: 4K frame 3.80 ->
// 3.61 ms); otherwise unrolled per sphere (the segment-test kernels: 1080p 0.267 ms
// against 0.272 with the compact form).  Both give the same bits.
template <bool COMPACT>
__device__ __forceinline__ void closest_block(const float4* __restrict__ geo, int base, const RayCross& r, float& tb,
                                              int& best) {
    if constexpr (COMPACT) {
        closest_block_compact(geo, base, r, tb, best);
        return;
    }
    float2 m[kPad / 2];
    uint32_t neg = 0;
#pragma unroll
    for (int q = 0; q < kPad / 2; ++q) {
        const float4 A = geo[2 * q], B = geo[2 * q + 1];
        const float2 cx = make_float2(A.x, A.y), cy = make_float2(A.z, A.w), cz = make_float2(B.x, B.y);
        const float2 px = fma2(cy, r.dz, fma2(cz, r.ndy, r.nwx));
        const float2 py = fma2(cz, r.dx, fma2(cx, r.ndz, r.nwy));
        const float2 pz = fma2(cx, r.dy, fma2(cy, r.ndx, r.nwz));
        m[q] = fma2(px, px, fma2(py, py, fma2(pz, pz, make_float2(B.z, B.w))));
        neg |= __float_as_uint(m[q].x) | __float_as_uint(m[q].y);
    }
    if (neg >> 31) {
#pragma unroll
        for (int q = 0; q < kPad / 2; ++q) {
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const float mm = hf ? m[q].y : m[q].x;
                if (mm < 0.0f) {
                    const float4 A = geo[2 * q], B = geo[2 * q + 1];
                    const float cx = hf ? A.y : A.x, cy = hf ? A.w : A.z, cz = hf ? B.y : B.x;
                    const float tc = fmaf(cx, r.dx.x, fmaf(cy, r.dy.x, fmaf(cz, r.dz.x, r.nod)));
                    const float s = __fsqrt_rn(-mm);
                    float t = tc - s;
                    if (t <= 0.0f) t = tc + s;
                    if (t > 0.0f && t < tb) {
                        tb = t;
                        best = base + 2 * q + hf;
                    }
                }
            }
        }
    }
}

// blocks: the blocks of kPad spheres to test (bits, ray_cull), or null: every
// block (the staged table only; visited in index order either way).
template <bool CH, bool ACC = false, bool COMPACT = false>
__device__ __forceinline__ int closest_hit(const StagedScene& sc, f3 o, f3 d, float& t_out,
                                           const uint32_t* blocks = nullptr) {
    float tb = __int_as_float(0x7f800000);  // +inf
    int best = -1;
    const int n = sc.hdr->ns_pad;
    if constexpr (ACC) {
        closest_bvh(sc.geo, sc.bvh, o, d, tb, best);
    } else {
        const RayCross rp = ray_cross(o, d);
        if constexpr (CH) {
            const unsigned mask = __activemask();
#pragma unroll 1
            for (int c0 = 0; c0 < n; c0 += kChunk) {
                const int m = min(kChunk, n - c0);
                stage_chunk(sc, mask, c0, m);
#pragma unroll 1
                for (int i0 = 0; i0 < m; i0 += kPad) closest_block<COMPACT>(sc.chunk + i0, c0 + i0, rp, tb, best);
            }
        } else {
            const int nb = n / kPad;
#pragma unroll 1
            for (int w0 = 0; w0 < nb; w0 += 32) {
                uint32_t m = blocks ? blocks[w0 >> 5] : (nb - w0 >= 32 ? 0xffffffffu : (1u << (nb - w0)) - 1u);
#pragma unroll 1
                while (m) {
                    const int i0 = (w0 + __ffs(m) - 1) * kPad;
                    m &= m - 1u;
                    closest_block<COMPACT>(sc.geo + i0, i0, rp, tb, best);
                }
            }
        }
    }
    const SceneHdr& h = *sc.hdr;
    if (h.has_plane) {
        const f3 n = xyz(h.plane_g);
        const float den = dot(d, n);
        if (den != 0.0f) {
            const float t = __fdiv_rn(-(dot(o, n) + h.plane_g.w), den);
            if (t > 0.0f && t < tb) {
                tb = t;
                best = h.ns;
            }
        }
    }
    t_out = tb;
    return best;
}

// ---------------------------------------------------------------- Section 3.6
// Any-hit of R shadow segments that leave the same origin o (one shading point).
// Segment r is o + u V_r, u in [0, 1], V_r = the light point minus the hit point
// (so it ends at the light point displaced by the origin's offset); it is blocked by a sphere
// iff its point closest to the centre lies inside the ball: u* = clamp(oc.W_r, 0,
// 1) with W_r = V_r / |V_r|^2 (the clamp is the saturation of the last FMA), and
// |oc - u* V_r|^2 - r^2 < 0.  That is the paper's "a root in (0, dist)" whenever
// the light is outside the sphere (checked at upload), including origins inside a
// sphere.  The sign bits of the pair's two results are OR-ed into a per-segment
// word; oc = c - o and the sphere loads are shared by the R segments.  The loop
// runs in blocks of kPad spheres and leaves once every segment of every active lane
// is blocked: the method's early break (Section 3.6 cast-shadows listing), taken
// warp-wide.
// Shadow segments traced together from one shading point (shared sphere loads).
constexpr int kShadowGroup = 4;

struct SegPair {  // segment r: W in both halves (x also scalar), -V in both halves
    float wx;
    float2 wy, wz, nvx, nvy, nvz;
};
__device__ __forceinline__ SegPair seg_pair(f3 w, f3 nv) {
    return SegPair{w.x, dup2(w.y), dup2(w.z), dup2(nv.x), dup2(nv.y), dup2(nv.z)};
}

// One block of kPad spheres (kPad / 2 pairs at geo[0..kPad)) against R segments;
// returns true when every segment of every lane in `mask` is blocked.
template <int R>
__device__ __forceinline__ bool occluded_block(const float4* __restrict__ geo, unsigned mask, const RayPair& o2,
                                               const SegPair (&sg)[kShadowGroup], uint32_t (&acc)[kShadowGroup]) {
#pragma unroll
    for (int q = 0; q < kPad / 2; ++q) {
        const float4 A = geo[2 * q], B = geo[2 * q + 1];
        const float2 ocx = add2(make_float2(A.x, A.y), o2.nox);
        const float2 ocy = add2(make_float2(A.z, A.w), o2.noy);
        const float2 ocz = add2(make_float2(B.x, B.y), o2.noz);
        const float2 nr = make_float2(B.z, B.w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 t = fma2(ocy, sg[r].wy, mul2(ocz, sg[r].wz));
            const float2 u = make_float2(fma_sat(ocx.x, sg[r].wx, t.x), fma_sat(ocx.y, sg[r].wx, t.y));
            const float2 qx = fma2(u, sg[r].nvx, ocx), qy = fma2(u, sg[r].nvy, ocy), qz = fma2(u, sg[r].nvz, ocz);
            const float2 e = fma2(qx, qx, fma2(qy, qy, fma2(qz, qz, nr)));
            acc[r] |= __float_as_uint(e.x) | __float_as_uint(e.y);
        }
    }
    bool done = true;
#pragma unroll
    for (int r = 0; r < R; ++r) done = done && (acc[r] >> 31);
    return __all_sync(mask, done);
}

// Line filter in front of the segment test.  The segment o + u V (u in [0, 1]) can
// only be blocked by a sphere that the infinite line through it passes within r
// of: D^2 = |oc|^2 - (oc.V^)^2 < r^2 with V^ the unit vector along V.  Per sphere
// pair the filter forms |oc|^2 (3 packed FMAs, shared by the group's segments),
// and per segment t' = oc.V^ (3) and g = t'^2 + K2 r^2 - K1 |oc|^2 (1): 4 packed
// instructions instead of the segment test's 8 packed plus 2 scalar.  Where g > 0
// or is NaN ("maybe"), the segment test runs as before and decides; elsewhere it
// would have said "not blocked", so every verdict is the segment test's, bit for
// bit.  Why g <= 0 implies that (u = 2^-24; oc, V, r^2 the FP32 values both tests
// use): the segment test's e is negative only if D^2 < r^2 (1 + 9u) (q = oc - u V
// carries one rounding per component, e three).  V^ = V rsqrtf(S), S = fl(V.V), is
// within 7u of the unit vector componentwise (S's rounding halved by the root, at
// most 2 ulp for rsqrtf -- CUDA's documented bound -- and the product), so the FP32
// t' is within 10u |oc| of oc.V^ and t'^2 >= |oc|^2 - D^2 - 20u |oc|^2; the filter's
// roundings cost at most 5u |oc|^2 + 3u r^2.  With K1 = 1 - 64u and K2 = 1 + 64u,
// e < 0 gives g > 39u |oc|^2 + 54u r^2 > 0.  The bound needs finite arithmetic: a pair whose
// |oc|^2 exceeds 2^100 is flagged too, and a group whose S leaves [2^-60, 2^100]
// for some lane takes the segment test throughout.  The flags are kept as the AND
// of sign bits ("certainly clear" = every value negative), so NaN and +inf count
// as "maybe".  W, -V and V^ of each segment wait in shared memory (9 floats per
// segment and thread, written once per group): V^ for the filter, W and -V for the
// pairs that need the segment test.
constexpr int kFilterMinPad = 128;  // smaller sphere tables keep the segment test alone
// Segments traced together by the filtered path.  Without the cone pre-pass larger
// groups paid |oc|^2 and the pair's flags fewer times per hit (4K queued frame:
// 9.99 / 9.79 / 9.64 / 9.48 / 9.64 ms for groups of 4 / 5 / 6 / 7 / 8); with the
// pre-pass and the warp cones a group visits a few blocks, and groups of 4 let each
// slot keep its unit vector in shared memory beside W and -V (9 floats per slot and
// thread, 36 KB per CTA): 4K frame 5.36 -> 5.07 ms against groups of 7 with the unit
// vectors in a local array.
constexpr int kFiltGroup = 4;
constexpr float kFiltK1 = 1.0f - 64.0f / 16777216.0f;
constexpr float kFiltK2 = 1.0f + 64.0f / 16777216.0f;
constexpr int kSegStride = 256;  // threads per CTA at most (the launch shapes allow 256)

// One array per kernel (namespace scope): every instantiation of the shadow test
// shares it.
__shared__ float s_seg[9 * kFiltGroup * kSegStride];

struct SegFilt {  // V^ of a segment in both halves
    float2 vx, vy, vz;
};

// Cone pre-pass of a sampled light (square area light or spherical light).  All the
// light's segments start at the shadow origin o and run along V_j = X_j - p towards
// sample points X_j of a small region, so their unit vectors lie within an angle
// alpha = arccos(kappa) of one axis a: every segment's line lies in the double cone
// {o + x : |x.a| >= |x| cos alpha}.  A sphere whose centre is farther than rho from
// that cone is farther than rho from every one of the lines, and the segment test
// reports a block only at a line distance D with D^2 < r^2 (1 + 9u) (the line
// filter's bound), so rho^2 >= r_max^2 (1 + 9u) over the table suffices.  With t =
// oc.a (a of unit length) and d^2 = |oc|^2 - t^2, the distance to the double cone is
// d kappa - |t| sin alpha where positive; "d kappa - |t| sin alpha < rho", squared
// (both sides non-negative) and with sin alpha replaced by sigma >= sin alpha, gives
// the necessary condition kappa^2 |oc|^2 - t^2 < rho^2 + 2 rho sigma |t|.  The pass
// evaluates h = t^2 + 2 rho sigma |t| + rho^2 - (kappa^2 - 2^-16) |oc|^2 per sphere
// pair (t: 3 packed FMAs, h: 3) and calls a pair clear when h < 0 in both halves and
// |oc|^2 < 2^100.  Error budget (u = 2^-24): the FP32 axis is within 8u per component
// of a unit vector (cone_unit), so the computed t is within 17u |oc| of the exact
// projection; t^2, the |t| term, |oc|^2 and the three roundings of h add at most
// 75u |oc|^2 + 25u rho^2, below the 2^-16 |oc|^2 (256u) taken off kappa^2 and the
// 2^-14 rho^2 added to r_max^2.
// NaN (canonical, positive) and +inf never clear.  A warp keeps one bit per block of
// kPad spheres, set when some lane's cone is not clear of some pair of the block.  A
// group whose every segment belongs to the cone's light, each V^ checked to satisfy
// V^.a >= kappa + 2^-18 (the check's roundings stay below 25u = 2^-18 / 2.5), visits
// only the blocks whose bit is set: a skipped block could block none of its segments,
// so every verdict is the segment test's, bit for bit.  The warp's coarse pass uses
// one cone for all lanes (apex p0 = one lane's shadow origin): a lane's blocking
// sphere lies within rho of its segment (the segment test's u is in [0, 1]), the
// segment lies in the lane's cone at its apex po, that cone in the warp's cone moved
// to po, hence the sphere within rho + |po - p0| of the warp's cone, up to the
// roundings of c - po and c - p0 (2u |oc|, inside the same |oc|^2 slack).
constexpr int kConeWords = 16;                        // bits per warp: 32 * kConeWords blocks
// The cone light's segments go in groups of kConeGroup, and every group of at most
// kConeGroup segments (the point lights' too, unused slots counting as blocked) runs
// through the one instance occluded_filtered<kConeGroup>: with the pre-pass a group
// visits few blocks, and a hit whose groups ran three instances (3, 7 and 2 segments
// for the 4K scene's 3 + 16) stalled on instruction fetch (ncu: no_instruction 2.69
// stalls per issue against 0.29).  Measured on B300, 4K queued frame, groups of 7 /
// 4 with their own instances / 3, 4, 5, 6 through one instance: 8.03 / 7.60 / 6.97,
// 6.91, 7.32, 7.51 ms.
constexpr int kConeGroup = 4;
constexpr int kConeMaxPad = 32 * kConeWords * kPad;   // larger tables take no pre-pass
__shared__ uint32_t s_cone[(kSegStride / 32) * 2 * kConeWords];  // per warp: sampled light, point lights
__shared__ unsigned s_r2max;

// rho^2 of the pre-pass: the largest r^2 of the staged table times (1 + 2^-14) (pad
// entries, -r^2 = +1, fall out), or 0 (no pre-pass) for tables of more than
// kConeMaxPad entries or when it leaves (0, 2^60]; and a bound on the centres' |c|
// (for the primary rays' cull).  Every thread of the CTA calls.
__shared__ unsigned s_c2max;
__device__ __forceinline__ void staged_cone(const float4* geo, int ns_pad, StagedScene& sc) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nth = blockDim.x * blockDim.y;
    if (tid == 0) {
        s_r2max = 0u;
        s_c2max = 0u;
    }
    __syncthreads();
    float m = 0.0f, c2 = 0.0f;
    for (int q = tid; q < ns_pad / 2; q += nth) {
        const float4 A = geo[2 * q], B = geo[2 * q + 1];
        m = fmaxf(m, fmaxf(-B.z, -B.w));
        c2 = fmaxf(c2, fmaxf(fmaf(A.x, A.x, fmaf(A.z, A.z, B.x * B.x)), fmaf(A.y, A.y, fmaf(A.w, A.w, B.y * B.y))));
    }
    if (m > 0.0f) atomicMax(&s_r2max, __float_as_uint(m));  // non-negative floats order as their bits
    if (c2 > 0.0f) atomicMax(&s_c2max, __float_as_uint(c2));
    __syncthreads();
    const float r2 = __uint_as_float(s_r2max) * (1.0f + 0x1p-14f);
    sc.cone_r2 = (ns_pad <= kConeMaxPad && r2 > 0.0f && r2 <= 0x1p60f) ? r2 : 0.0f;
    sc.cone_cmax = sqrtf(__uint_as_float(s_c2max)) * (1.0f + 0x1p-20f);  // +inf when |c|^2 overflows
}

// Unit vector for the cones' axes: rsqrtf (within 2 ulp) instead of the correctly
// rounded root; every bound below allows 8u per component for it.
__device__ __forceinline__ f3 cone_unit(f3 a) { return scl(a, rsqrtf(dot(a, a))); }

// True when the cone (apex o via o2, axis ax, c0 = kappa^2 - 2^-16, tw = 2 rho sigma,
// r2 = rho^2) is clear of every pair of the block of kPad spheres at g.
__device__ __forceinline__ bool cone_block_clear(const float4* __restrict__ g, const RayPair& o2, float2 axx,
                                                 float2 axy, float2 axz, float2 nc0, float2 tw, float2 r2) {
    uint32_t clr = 0xffffffffu;
    // each lane starts at pair (lane mod 4): lanes testing different blocks (128 bytes
    // apart) would otherwise load from the same shared-memory banks
    static_assert(((kPad / 2) & (kPad / 2 - 1)) == 0, "pairs per block: a power of two");
    const int rot = threadIdx.x & (kPad / 2 - 1);
#pragma unroll
    for (int qq = 0; qq < kPad / 2; ++qq) {
        const int q = (qq + rot) & (kPad / 2 - 1);
        const float4 A = g[2 * q], B = g[2 * q + 1];
        const float2 ocx = add2(make_float2(A.x, A.y), o2.nox);
        const float2 ocy = add2(make_float2(A.z, A.w), o2.noy);
        const float2 ocz = add2(make_float2(B.x, B.y), o2.noz);
        const float2 oc2 = fma2(ocx, ocx, fma2(ocy, ocy, mul2(ocz, ocz)));
        const float2 big = add2(oc2, dup2(-0x1p100f));
        const float2 t = fma2(ocx, axx, fma2(ocy, axy, mul2(ocz, axz)));
        const float2 at = make_float2(fabsf(t.x), fabsf(t.y));
        const float2 h = fma2(oc2, nc0, fma2(t, t, fma2(at, tw, r2)));
        clr &= __float_as_uint(h.x) & __float_as_uint(h.y) & __float_as_uint(big.x) & __float_as_uint(big.y);
    }
    return (clr >> 31) != 0;
}

// The blocks of the table split over the lanes (this lane's share: rank, rank +
// cnt, ...), each tested once against one cone (apex, unit axis, c0 = kappa^2 -
// 2^-16, tw = 2 rho sigma, r2 = rho^2 with its slack); bit b of cw is set for every
// block the cone does not clear.  One copy of the loop for every warp-cone pass.
__device__ __noinline__ void cone_blocks_split(const float4* __restrict__ geo, int nb, int rank, int cnt, f3 apex,
                                               f3 axis, float c0, float tw, float r2, uint32_t* cw) {
    const RayPair o2 = ray_pair(apex);
    const float2 ax = dup2(axis.x), ay = dup2(axis.y), az = dup2(axis.z);
    const float2 nc0 = dup2(-c0), tw2 = dup2(tw), r22 = dup2(r2);
#pragma unroll 1
    for (int b = rank; b < nb; b += cnt)
        if (!cone_block_clear(geo + (size_t)b * kPad, o2, ax, ay, az, nc0, tw2, r22)) atomicOr(&cw[b >> 5], 1u << (b & 31));
}

// The warp's block bits for the cones of the lanes in `mask` whose `use` is set (this
// lane's cone: apex o, axis ax, c0, twors, rho2), written to cw[0 .. n / kPad / 32].
// With `coarse`, a first pass splits the blocks over the lanes and tests each once
// against the warp's cone (apex p0, axis aw, wc0, wtw, wr2), which holds every
// lane's cone moved to p0 (its width covers each lane's axis offset plus its width,
// its radius rho plus the farthest lane apex): only the blocks it does not clear
// are tested against the lanes' own cones.  Out of line: the shading code keeps its
// registers.
// Returns this lane's own bits of blocks 0..31 (its cone alone; for item_groups).
__device__ __noinline__ uint32_t cone_pass(const float4* __restrict__ geo, int n, unsigned mask, f3 o, f3 ax,
                                           float c0, float twors, float rho2, bool use, uint32_t* cw, f3 p0, f3 aw,
                                           float wc0, float wtw, float wr2, bool coarse) {
    const int lane = threadIdx.x & 31;
    const int nb = n / kPad;
    const bool leader = lane == __ffs(mask) - 1;
    if (coarse) {
        const int rank = __popc(mask & ((1u << lane) - 1u)), cnt = __popc(mask);
        for (int w = rank; w < (nb + 31) / 32; w += cnt) cw[w] = 0u;
        __syncwarp(mask);
        cone_blocks_split(geo, nb, rank, cnt, p0, aw, wc0, wtw, wr2, cw);
        __syncwarp(mask);
    }
    const RayPair o2 = ray_pair(o);
    const float2 axx = dup2(ax.x), axy = dup2(ax.y), axz = dup2(ax.z);
    const float2 nc0 = dup2(-c0), tw = dup2(twors), r2 = dup2(rho2);
    uint32_t own = 0;
#pragma unroll 1
    for (int w0 = 0; w0 < nb; w0 += 32) {
        uint32_t m = coarse ? cw[w0 >> 5] : (nb - w0 >= 32 ? 0xffffffffu : (1u << (nb - w0)) - 1u);
        uint32_t word = 0;
#pragma unroll 1
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            const bool need = use && !cone_block_clear(geo + (size_t)(w0 + b) * kPad, o2, axx, axy, axz, nc0, tw, r2);
            if (w0 == 0 && need) own |= 1u << b;
            word |= (__any_sync(mask, need) ? 1u : 0u) << b;
        }
        __syncwarp(mask);  // every lane has read the coarse word
        if (leader) cw[w0 >> 5] = word;
    }
    __syncwarp(mask);
    return own;
}

// Closest-hit cull for the rays of the lanes in `mask` (origin o, direction d each).
// The closest-hit test finds a root only where its computed m = |c x d - o x d|^2 -
// r^2 is negative: with -(o x d) rounded once per component and two FMAs per
// component, the computed vector is within 7u (|c| + |o|) of the exact one, so m < 0
// needs a line distance below r (1 + 7u) + 9u (|c| + |o|) <= r_max + 2^-16 (c_max +
// |o|).  One cone holds every lane's line: apex p0 = the first lane's origin, axis a
// along the sum of the first and last lane's directions (cone_unit), kappa the
// warp's minimum of a.d less 2^-18 (the roundings of a.d stay below 25u); a lane's
// line lies within |o - p0| of it, so rho = (r_max + 2^-16 (c_max + max |o|) + max |o
// - p0|) (1 + 2^-16) bounds the distance of every sphere with a root.  The blocks
// are split over the lanes and tested once against that cone (cone_block_clear,
// whose slack covers the rounding of c - p0); bit b of cw is set for every block the
// cone does not clear.  A skipped block holds no sphere with a root, so the closest
// hit (strict <, index order over the rest) is unchanged.  For a warp of primary
// rays p0 is every lane's origin (the camera) and the cone is the patch's view
// frustum.  Returns false, writing nothing, when the rays do not fit a cone of
// half-angle below 60 degrees.
__device__ __noinline__ bool ray_cull(const float4* __restrict__ geo, int n, unsigned mask, f3 o, f3 d,
                                      float r_max, float c_max, uint32_t* cw) {
    const int lane = threadIdx.x & 31;
    const int lo = __ffs(mask) - 1, hi = 31 - __clz(mask);
    const f3 dl = mk3(__shfl_sync(mask, d.x, lo), __shfl_sync(mask, d.y, lo), __shfl_sync(mask, d.z, lo));
    const f3 dh = mk3(__shfl_sync(mask, d.x, hi), __shfl_sync(mask, d.y, hi), __shfl_sync(mask, d.z, hi));
    const f3 p0 = mk3(__shfl_sync(mask, o.x, lo), __shfl_sync(mask, o.y, lo), __shfl_sync(mask, o.z, lo));
    const f3 a = cone_unit(add(dl, dh));
    const float k = dot(a, d);
    const f3 dp = sub(o, p0);
    // warp minimum / maxima (non-negative floats order as their bits)
    const float kw = __uint_as_float(__reduce_min_sync(mask, __float_as_uint(k >= 0.5f ? k : 0.0f))) - 0x1p-18f;
    const float om = __uint_as_float(__reduce_max_sync(mask, __float_as_uint(sqrt_bound(dot(o, o)))));
    const float dm = __uint_as_float(__reduce_max_sync(mask, __float_as_uint(sqrt_bound(dot(dp, dp)))));
    const float rho = (r_max + 0x1p-16f * (c_max + om) + dm) * (1.0f + 0x1p-16f);
    if (!(kw >= 0.5f && rho <= 0x1p30f)) return false;
    const float sw = sqrt_bound(fmaxf(fmaf(-kw, kw, 1.0f), 0.0f)) * (1.0f + 0x1p-18f);
    const int nb = n / kPad;
    const int rank = __popc(mask & ((1u << lane) - 1u)), cnt = __popc(mask);
    for (int w = rank; w < (nb + 31) / 32; w += cnt) cw[w] = 0u;
    __syncwarp(mask);
    cone_blocks_split(geo, nb, rank, cnt, p0, a, fmaf(kw, kw, -0x1p-16f), 2.0f * rho * sw,
                      rho * rho * (1.0f + 0x1p-15f), cw);
    __syncwarp(mask);
    return true;
}

// Point lights.  A segment of point light L starts at its lane's shadow origin po and
// ends at po + V = L + E (E: the origin's offset eps n, plus roundings), so it lies
// within |E| of the segment from po to L, which lies in any cone with apex L that
// holds the direction to po.  For each light l of `lights` the lanes whose group
// holds l (bit l of gl) form one cone: axis from L to the first such lane's po, kappa
// the lanes' minimum cosine less 2^-18, rho_l = (rho + max |E| + 2^-16 (|L| + max |po
// - L|)) (1 + 2^-15), the 2^-16 term covering the roundings of E and of c - L.  The
// blocks are split over the lanes and tested once per light (cone_block_clear); cw
// receives the union of the blocks no cone clears.  Returns false (visit every
// block) when some light's lanes do not fit a cone below 60 degrees.
__device__ __noinline__ bool point_pass(const float4* __restrict__ geo, int n, unsigned mask, const SceneHdr& h, f3 p,
                                        f3 p_lo, f3 po, uint32_t gl, unsigned lights, float rho, uint32_t* cw) {
    const int lane = threadIdx.x & 31;
    const int nb = n / kPad;
    const int rank = __popc(mask & ((1u << lane) - 1u)), cnt = __popc(mask);
    for (int w = rank; w < (nb + 31) / 32; w += cnt) cw[w] = 0u;
    __syncwarp(mask);
    bool ok = true;
    unsigned rest = lights;
#pragma unroll 1
    while (rest) {
        const int l = __ffs(rest) - 1;
        rest &= rest - 1u;
        const f3 L = xyz(h.light_p[l]);
        const bool has = (gl >> l) & 1u;
        const int ld = __ffs(__ballot_sync(mask, has)) - 1;
        const f3 dir = has ? cone_unit(sub(po, L)) : mk3(0.f, 0.f, 0.f);
        const f3 a = mk3(__shfl_sync(mask, dir.x, ld), __shfl_sync(mask, dir.y, ld), __shfl_sync(mask, dir.z, ld));
        float k = 1.0f, e = 0.0f, dd = 0.0f;
        if (has) {
            k = dot(a, dir);
            k = k >= 0.5f ? k : 0.0f;  // NaN: 0
            const f3 E = sub(add(po, sub(sub(L, p), p_lo)), L);  // po + V - L, V as the set-up forms it
            e = sqrt_bound(dot(E, E));
            const f3 D = sub(po, L);
            dd = sqrt_bound(dot(D, D));
        }
        // warp minimum / maxima (non-negative floats order as their bits)
        const float kw = __uint_as_float(__reduce_min_sync(mask, __float_as_uint(k))) - 0x1p-18f;
        const float em = __uint_as_float(__reduce_max_sync(mask, __float_as_uint(e)));
        const float dm = __uint_as_float(__reduce_max_sync(mask, __float_as_uint(dd)));
        const float rl = (rho + em + 0x1p-16f * (sqrt_bound(dot(L, L)) + dm)) * (1.0f + 0x1p-15f);
        if (!(kw >= 0.5f && rl <= 0x1p30f)) {
            ok = false;
            break;
        }
        const float sw = sqrt_bound(fmaxf(fmaf(-kw, kw, 1.0f), 0.0f)) * (1.0f + 0x1p-18f);
        cone_blocks_split(geo, nb, rank, cnt, L, a, fmaf(kw, kw, -0x1p-16f), 2.0f * rl * sw,
                          rl * rl * (1.0f + 0x1p-15f), cw);
    }
    __syncwarp(mask);
    return ok;
}

// Segment test of pair q (spheres 2q, 2q + 1 of geo) against the R segments, the
// operations of occluded_block; W and -V from shared memory (seg[k * kSegStride],
// k = 9 r + (0..2: W, 3..5: -V); 6..8 hold V^).
template <int R>
__device__ __forceinline__ void pair_exact(const float4* __restrict__ geo, int q, const RayPair& o2,
                                           const float* seg, uint32_t (&acc)[kFiltGroup]) {
    const float4 A = geo[2 * q], B = geo[2 * q + 1];
    const float2 ocx = add2(make_float2(A.x, A.y), o2.nox);
    const float2 ocy = add2(make_float2(A.z, A.w), o2.noy);
    const float2 ocz = add2(make_float2(B.x, B.y), o2.noz);
    const float2 nr = make_float2(B.z, B.w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float* g = seg + 9 * r * kSegStride;
        const float wx = g[0], wy = g[kSegStride], wz = g[2 * kSegStride];
        const float2 t = fma2(ocy, dup2(wy), mul2(ocz, dup2(wz)));
        const float2 u = make_float2(fma_sat(ocx.x, wx, t.x), fma_sat(ocx.y, wx, t.y));
        const float2 qx = fma2(u, dup2(g[3 * kSegStride]), ocx), qy = fma2(u, dup2(g[4 * kSegStride]), ocy),
                     qz = fma2(u, dup2(g[5 * kSegStride]), ocz);
        const float2 e = fma2(qx, qx, fma2(qy, qy, fma2(qz, qz, nr)));
        acc[r] |= __float_as_uint(e.x) | __float_as_uint(e.y);
    }
}

// One block of kPad spheres through the filter; the segment test for the pairs
// some lane flags (every pair with `force`, warp-uniform: the filter skipped).
// Returns true when every segment of every lane in `mask` is blocked (checked only
// after a segment test ran: the filter alone blocks nothing).
template <int R>
__device__ __forceinline__ bool occluded_block_filtered(const float4* __restrict__ geo, unsigned mask,
                                                        const RayPair& o2, const SegFilt (&sf)[kFiltGroup],
                                                        const float* seg, uint32_t (&acc)[kFiltGroup], bool force) {
    // pairs some lane flags, one warp-uniform bit each; one copy of the segment test
    uint32_t need = (1u << (kPad / 2)) - 1u;
    if (!force) {
        uint32_t clear[kPad / 2];
#pragma unroll
        for (int q = 0; q < kPad / 2; ++q) {
            const float4 A = geo[2 * q], B = geo[2 * q + 1];
            const float2 ocx = add2(make_float2(A.x, A.y), o2.nox);
            const float2 ocy = add2(make_float2(A.z, A.w), o2.noy);
            const float2 ocz = add2(make_float2(B.x, B.y), o2.noz);
            const float2 oc2 = fma2(ocx, ocx, fma2(ocy, ocy, mul2(ocz, ocz)));
            // K2 r^2 - K1 |oc|^2 (B.zw = -r^2), and |oc|^2 - 2^100 (positive: too large)
            const float2 c = fma2(oc2, dup2(-kFiltK1), mul2(make_float2(B.z, B.w), dup2(-kFiltK2)));
            const float2 big = add2(oc2, dup2(-0x1p100f));
            clear[q] = __float_as_uint(big.x) & __float_as_uint(big.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 t = fma2(ocx, sf[r].vx, fma2(ocy, sf[r].vy, mul2(ocz, sf[r].vz)));
                const float2 g = fma2(t, t, c);
                clear[q] &= __float_as_uint(g.x) & __float_as_uint(g.y);
            }
        }
        if (__all_sync(mask, ((clear[0] & clear[1] & clear[2] & clear[3]) >> 31) != 0)) return false;
        need = 0;
#pragma unroll
        for (int q = 0; q < kPad / 2; ++q) need |= __all_sync(mask, (clear[q] >> 31) != 0) ? 0u : (1u << q);
    }
#pragma unroll 1
    while (need) {
        const int q = __ffs(need) - 1;
        need &= need - 1u;
        pair_exact<R>(geo, q, o2, seg, acc);
    }
    bool done = true;
#pragma unroll
    for (int r = 0; r < R; ++r) done = done && (acc[r] >> 31);
    return __all_sync(mask, done);
}

// Item mode of a group (occluded_filtered with items): where the lanes' hits lie far
// apart (queue passes), the blocks some lane's cone reaches are needed by a few lanes
// each (ncu-side count at 4K: 5 of 32 lanes per visited block), so iterating the
// warp's union idles most of each step.  Instead the (lane, block) pairs of the lanes'
// own bits are numbered (warp scan of the counts) and the 32 lanes take them 32 at a
// time: lane j tests block b for lane L's segments -- L's origin and slots read from
// shared memory, the filter and, for the pairs it flags, the segment test, the
// operations of occluded_block_filtered -- and ORs the blocked segments into L's
// result word.  Every pair of every own block is tested (no early exit), and a
// verdict is an OR over blocks, so the result equals the union loop's bit for bit.
// Lanes whose segments are all blocked already contribute no pairs.  A full warp calls.
__shared__ float s_it_o[3 * kSegStride];
__shared__ int s_it_start[kSegStride];
__shared__ uint32_t s_it_own[kSegStride], s_it_res[kSegStride];
template <int R>
__device__ __forceinline__ uint32_t item_groups(const float4* __restrict__ geo, f3 o, uint32_t blocked_in,
                                                const float* seg, uint32_t own) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wb = tid - lane;
    const uint32_t rmask = (1u << R) - 1u;
    const uint32_t mine = (blocked_in & rmask) == rmask ? 0u : own;
    const int cnt = __popc(mine);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    s_it_start[tid] = incl - cnt;
    s_it_own[tid] = mine;
    s_it_o[tid] = o.x;
    s_it_o[kSegStride + tid] = o.y;
    s_it_o[2 * kSegStride + tid] = o.z;
    s_it_res[tid] = blocked_in & rmask;
    __syncwarp();
    const float* seg0 = seg - lane;  // slot base of the warp's first lane
#pragma unroll 1
    for (int i = lane; i < total; i += 32) {
        // owner: the last lane whose first item is at most i (counts of zero share a start)
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (s_it_start[wb + L + step] <= i) L += step;
        uint32_t x = s_it_own[wb + L];
        for (int k = i - s_it_start[wb + L]; k > 0; --k) x &= x - 1u;
        const float4* g = geo + (size_t)(__ffs(x) - 1) * kPad;
        const float* segL = seg0 + L;
        const RayPair o2 = ray_pair(mk3(s_it_o[wb + L], s_it_o[kSegStride + wb + L], s_it_o[2 * kSegStride + wb + L]));
        SegFilt sf[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            sf[r] = SegFilt{dup2(segL[(9 * r + 6) * kSegStride]), dup2(segL[(9 * r + 7) * kSegStride]),
                            dup2(segL[(9 * r + 8) * kSegStride])};
        uint32_t acc[kFiltGroup];
#pragma unroll
        for (int r = 0; r < kFiltGroup; ++r) acc[r] = 0u;
#pragma unroll 1
        for (int q = 0; q < kPad / 2; ++q) {
            const float4 A = g[2 * q], B = g[2 * q + 1];
            const float2 ocx = add2(make_float2(A.x, A.y), o2.nox);
            const float2 ocy = add2(make_float2(A.z, A.w), o2.noy);
            const float2 ocz = add2(make_float2(B.x, B.y), o2.noz);
            const float2 oc2 = fma2(ocx, ocx, fma2(ocy, ocy, mul2(ocz, ocz)));
            const float2 c = fma2(oc2, dup2(-kFiltK1), mul2(make_float2(B.z, B.w), dup2(-kFiltK2)));
            const float2 big = add2(oc2, dup2(-0x1p100f));
            uint32_t clear = __float_as_uint(big.x) & __float_as_uint(big.y);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 t = fma2(ocx, sf[r].vx, fma2(ocy, sf[r].vy, mul2(ocz, sf[r].vz)));
                const float2 gg = fma2(t, t, c);
                clear &= __float_as_uint(gg.x) & __float_as_uint(gg.y);
            }
            if (!(clear >> 31)) pair_exact<R>(g, q, o2, segL, acc);
        }
        uint32_t bits = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) bits |= (acc[r] >> 31) << r;
        if (bits) atomicOr(&s_it_res[wb + L], bits);
    }
    __syncwarp();
    return s_it_res[tid];
}

// The filtered sphere loop of one group, out of line: inlined into the shading
// code its registers and the caller's live state spilled inside the sphere loop
// (ncu: 2e8 local loads and stores per 1080p launch); called, the caller's state is
// saved once per group.  The caller has written W, -V and V^ of segment r to slot r
// of seg (shared memory; V^ zero for segments already blocked); blocked_in / the
// result: bit r = segment r blocked.  exact_only: the segment
// test for every pair (a group for which the filter's bound is not established).
// cone: the warp's block bits of the cone pre-pass (only the blocks whose bit is set
// are visited), or null (every block).  items (a full warp, blocks 0..31 only): each
// lane's own bits `own` instead of the warp's union -- see item_groups.
// IT: the item mode compiled in (the queue passes' kernel; in the first pass, whose
// warps are mostly coherent, its code cost more instruction fetch than it saved).
template <int R, bool IT>
__device__ __noinline__ uint32_t occluded_filtered(const float4* __restrict__ geo, int n, unsigned mask, f3 o,
                                                   uint32_t blocked_in, const float* seg, bool exact_only,
                                                   const uint32_t* cone, uint32_t own, bool items) {
    if constexpr (IT) {
        if (items && !exact_only) return item_groups<R>(geo, o, blocked_in, seg, own);
    }
    const RayPair o2 = ray_pair(o);
    SegFilt sf[kFiltGroup];
    uint32_t acc[kFiltGroup];
#pragma unroll
    for (int r = 0; r < kFiltGroup; ++r) {
        acc[r] = (blocked_in >> r) & 1u ? 0x80000000u : 0u;
        sf[r] = r < R ? SegFilt{dup2(seg[(9 * r + 6) * kSegStride]), dup2(seg[(9 * r + 7) * kSegStride]),
                                dup2(seg[(9 * r + 8) * kSegStride])}
                      : SegFilt{dup2(0.f), dup2(0.f), dup2(0.f)};
    }
    // exact_only (the filter's bound does not hold for some lane): the segment test
    // for every pair of every block
    if (exact_only) cone = nullptr;
    const int nb = n / kPad;
    bool stop = false;
#pragma unroll 1
    for (int w0 = 0; w0 < nb && !stop; w0 += 32) {
        uint32_t m = cone ? cone[w0 >> 5] : (nb - w0 >= 32 ? 0xffffffffu : (1u << (nb - w0)) - 1u);
#pragma unroll 1
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            if (occluded_block_filtered<R>(geo + (size_t)(w0 + b) * kPad, mask, o2, sf, seg, acc, exact_only)) {
                stop = true;
                break;
            }
        }
    }
    uint32_t out = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) out |= (acc[r] >> 31) << r;
    return out;
}

// Segment r is o + u V_r (u in [0, 1]) with -V_r = nv[r] and W_r = w[r].  occ[r]
// enters true for unused slots (and leaves true for blocked segments).  The plane is
// tested first: a segment it blocks enters the sphere loop as blocked (the verdict
// is an OR, so the order does not matter).
template <int R, bool CH, bool ACC = false>
__device__ __forceinline__ void occluded_group(const StagedScene& sc, f3 o, const f3 (&w)[kShadowGroup],
                                               const f3 (&nv)[kShadowGroup], bool (&occ)[kShadowGroup]) {
    const SceneHdr& h = *sc.hdr;
    if (h.has_plane) {
        const f3 pn = xyz(h.plane_g);
        const float num = -(dot(o, pn) + h.plane_g.w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            // root u = num / (V.n) in (0, 1)  <=>  same signs and |num| < |V.n|
            const float den = -dot(nv[r], pn);
            if (!occ[r] && den != 0.0f && num != 0.0f && ((num > 0.0f) == (den > 0.0f)) && fabsf(num) < fabsf(den))
                occ[r] = true;
        }
    }
    const int n = h.ns_pad;
    if constexpr (ACC) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (!occ[r]) occ[r] = occluded_bvh(sc.geo, sc.bvh, o, w[r], nv[r]);
    } else {
        const unsigned mask = __activemask();
        const RayPair o2 = ray_pair(o);
        uint32_t acc[kShadowGroup];
#pragma unroll
        for (int r = 0; r < kShadowGroup; ++r) acc[r] = occ[r] ? 0x80000000u : 0u;
        if constexpr (CH) {
            SegPair sg[kShadowGroup];
#pragma unroll
            for (int r = 0; r < kShadowGroup; ++r) sg[r] = seg_pair(w[r], nv[r]);
            bool stop = false;
#pragma unroll 1
            for (int c0 = 0; c0 < n && !stop; c0 += kChunk) {
                const int m = min(kChunk, n - c0);
                stage_chunk(sc, mask, c0, m);
#pragma unroll 1
                for (int i0 = 0; i0 < m; i0 += kPad) {
                    if (occluded_block<R>(sc.chunk + i0, mask, o2, sg, acc)) {
                        stop = true;
                        break;
                    }
                }
            }
        } else {
            SegPair sg[kShadowGroup];
#pragma unroll
            for (int r = 0; r < kShadowGroup; ++r) sg[r] = seg_pair(w[r], nv[r]);
#pragma unroll 1
            for (int i0 = 0; i0 < n; i0 += kPad)
                if (occluded_block<R>(sc.geo + i0, mask, o2, sg, acc)) break;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) occ[r] = (acc[r] >> 31) != 0;
    }
}

// ---------------------------------------------------------------- Section 3.6.1
// The in-plane axes of a spherical light seen from p: w = normalize(p - L), u =
// normalize(w x up), v = u x w (up = +y, or +x when w is nearly vertical).  They
// depend on the hit and the light only, so a hit computes them once per light.
struct LightFrame {
    f3 u, v;
};
__device__ __forceinline__ LightFrame light_frame(f3 p, float4 Lp) {
    const f3 wv = normalize(sub(p, xyz(Lp)));
    const f3 up = fabsf(wv.y) < 0.999f ? mk3(0.f, 1.f, 0.f) : mk3(1.f, 0.f, 0.f);
    const f3 u = normalize(mk3(wv.y * up.z - wv.z * up.y, wv.z * up.x - wv.x * up.z, wv.x * up.y - wv.y * up.x));
    const f3 v = mk3(u.y * wv.z - u.z * wv.y, u.z * wv.x - u.x * wv.z, u.x * wv.y - u.y * wv.x);
    return LightFrame{u, v};
}

// Target point of shadow ray s of sampled light (Lp, Ls) seen from p.
// Square area light of side a: n = g*g strata, sample s in stratum
// (s mod g, s div g) at ((i + xi1)/g - 1/2, (j + xi2)/g - 1/2) * a in x and z,
// xi from Philox call s div 2 with counter (pixel, bounce, light, call), words
// 2(s mod 2), 2(s mod 2) + 1 (`w` holds the call's words; refreshed on even s).
// Spherical light of radius R: sunflower point s of n on the great circle facing p,
// radius R sqrt(s/n) at angle s * phi, phi = pi (3 - sqrt 5) (the angle is reduced
// exactly as 2 pi frac(s (3 - sqrt 5) / 2) in 32-bit fixed point).
// lf: light_frame(p, Lp) for a spherical light (unused otherwise); flower: the
// sunflower table of this frame's sample count, or null.
template <bool LEAN = false>
__device__ __forceinline__ f3 sample_point(const Frame& fr, uint32_t pix, int k, int l, int s, float4 Lp, float4 Ls,
                                           uint4& w, const LightFrame& lf, const float4* flower) {
    if (Ls.x > 0.0f) {
        if ((s & 1) == 0)
            w = philox10(make_uint4(pix, (uint32_t)k, (uint32_t)l, (uint32_t)(s >> 1)), fr.key0, fr.key1);
        const float xi1 = u24((s & 1) ? w.z : w.x);
        const float xi2 = u24((s & 1) ? w.w : w.y);
        const int g = fr.sample_g;
        // j = s div g by a multiply-high: with M = ceil(2^22 / g) the product s 2^10 M /
        // 2^32 exceeds s / g by less than 2^-12 < 1 / g (s < 2^10, g <= 32), so its floor
        // is s div g (checked for every such s and g)
        const int j = (int)__umulhi((uint32_t)s << 10, fr.sample_g_magic);
        const int i = s - j * g;
        const float a = Ls.x, ginv = fr.sample_g_inv;
        return mk3(Lp.x + (((float)i + xi1) * ginv - 0.5f) * a, Lp.y, Lp.z + (((float)j + xi2) * ginv - 0.5f) * a);
    }
    if constexpr (LEAN) return xyz(Lp);  // no spherical light in the scene: never reached
    float q, sn, cs;
    if (flower) {
        const float4 f = flower[s];
        q = f.x;
        cs = f.y;
        sn = f.z;
    } else {
        q = sqrtf((float)s / (float)fr.nsamp);
        const uint32_t frac = (uint32_t)s * 0x61C88647u;  // 2^32 (3 - sqrt 5) / 2
        sincospif((float)(frac >> 8) * (1.0f / 8388608.0f), &sn, &cs);  // 2 frac
    }
    const float r = Ls.y * q;
    return add(xyz(Lp), add(scl(lf.u, r * cs), scl(lf.v, r * sn)));
}

// ---------------------------------------------------------------- Sections 3.5-3.6
// Shading of one hit: A = k_a + sum_l I_l vis_l max(n.l, 0), S = sum_l I_l vis_l k_s
// spec_l; a light is skipped when n.l <= 0.  Phong spec = max(v.r, 0)^exp with r
// the light direction mirrored about n and v = -d; Blinn spec = max(n.h, 0)^exp.
// The shadow rays of the hit (one per lit point light, n per lit sampled light,
// in light order) are traced in groups from the common origin po -- up to
// kShadowGroup (4) with the segment test alone, kFiltGroup (7) through the line
// filter; a group's size is the warp's maximum of the lanes' remaining rays.
struct HitShade {
    float A, S;
};

__device__ __forceinline__ float light_spec(const Frame& fr, f3 n, f3 d, f3 lh, float ndl, float e) {
    if (fr.model == RT_PHONG) {
        const f3 r = sub(scl(n, 2.0f * ndl), lh);
        const float vr = -dot(d, r);
        return vr > 0.0f ? spec_pow(vr, e) : 0.0f;
    }
    const f3 hv = normalize(sub(lh, d));
    const float nh = dot(n, hv);
    return nh > 0.0f ? spec_pow(nh, e) : 0.0f;
}

__device__ __forceinline__ int rays_of_light(const Frame& fr, float4 Ls) {
    return (Ls.x > 0.0f || Ls.y > 0.0f) ? fr.nsamp : 1;
}

// A sampled light (nr > 1 rays) whose every segment from this shading point is
// certainly unblocked: the cone of its sample region seen from p (the one-lane path's
// cone pre-pass: axis to the centre, kappa below the cosine to the square's corners or
// the sphere's tangent cone, less 2^-17) clears every block of the staged table, by
// cone_block_clear with apex po, and the plane cannot block either (the one-lane
// path's skip, same bounds).  Each segment would test unblocked, so vis = n / n = 1.
// Needs the cone bound of the staged table (sc.cone_r2 > 0).
__device__ __forceinline__ bool light_clear(const StagedScene& sc, const SceneHdr& h, int l, f3 p, f3 p_lo, f3 po) {
    const float4 Lp = h.light_p[l], Ls = h.light_s[l];
    const f3 Lv = sub(sub(xyz(Lp), p), p_lo);
    const float ri = rsqrtf(dot(Lv, Lv));
    const f3 ax = scl(Lv, ri);
    float kap;
    if (Ls.x > 0.0f) {
        const float hs = 0.5f * Ls.x;
        kap = 1.0f;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            const f3 cv = add(Lv, mk3((c & 1) ? hs : -hs, 0.0f, (c & 2) ? hs : -hs));
            kap = fminf(kap, dot(ax, cv) * rsqrtf(dot(cv, cv)));
        }
    } else {
        const float sr = Ls.y * ri * (1.0f + 0x1p-20f);  // >= R / dist
        kap = sqrt_bound(fmaxf(fmaf(-sr, sr, 1.0f), 0.0f));
    }
    kap -= 0x1p-17f;
    if (!(kap >= 0.5f)) return false;  // NaN: not clear
    const float sg = sqrt_bound(fmaxf(fmaf(-kap, kap, 1.0f), 0.0f)) * (1.0f + 0x1p-18f);  // >= sin alpha
    const float2 nc0 = dup2(-fmaf(kap, kap, -0x1p-16f)), tw = dup2(2.0f * sqrt_bound(sc.cone_r2) * sg);
    const float2 r2 = dup2(sc.cone_r2);
    const RayPair o2 = ray_pair(po);
    const float2 axx = dup2(ax.x), axy = dup2(ax.y), axz = dup2(ax.z);
#pragma unroll 1
    for (int i0 = 0; i0 < h.ns_pad; i0 += kPad)
        if (!cone_block_clear(sc.geo + i0, o2, axx, axy, axz, nc0, tw, r2)) return false;
    if (!h.has_plane) return true;
    const f3 pn = xyz(h.plane_g);
    const float num = -(dot(po, pn) + h.plane_g.w);
    if (num == 0.0f) return true;
    if (num > 0.0f) return false;
    const float an = fabsf(pn.x) + fabsf(pn.y) + fabsf(pn.z);
    const float ext = Ls.x > 0.0f ? 0.5f * Ls.x * (fabsf(pn.x) + fabsf(pn.z)) : Ls.y * an;
    const float lo = dot(xyz(Lp), pn) - ext - (dot(p, pn) + dot(p_lo, pn));
    const float sc_ = (fmaxf(fabsf(Lp.x), fmaxf(fabsf(Lp.y), fabsf(Lp.z))) + Ls.x + Ls.y +
                       fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))) + 1.0f) * an;
    return lo > 0x1p-14f * sc_;  // NaN: false
}

template <bool HITREC, bool CH, bool ACC = false, bool SKIP = false>
__device__ __forceinline__ HitShade shade_hit(const StagedScene& sc, const Frame& fr, uint32_t pix, int k, f3 p,
                                              f3 p_lo, f3 n, f3 po, f3 d, float ks, float e, float* __restrict__ hr,
                                              size_t hr_k, size_t hr_plane) {
    const SceneHdr& h = *sc.hdr;
    HitShade out{fr.ka, 0.0f};
    // lights on the lit side and the number of shadow rays they need; sampled lights
    // that light_clear proves unblocked take no rays (vis = 1)
    uint32_t lit = 0, clear = 0;
    int total = 0;
#pragma unroll 1
    for (int li = 0; li < h.nl; ++li) {
        const f3 lh = normalize(sub(sub(xyz(h.light_p[li]), p), p_lo));
        if (dot(n, lh) > 0.0f) {
            lit |= 1u << li;
            const int nr = rays_of_light(fr, h.light_s[li]);
            bool skip = false;
            if constexpr (!CH && !ACC && SKIP) skip = nr > 1 && sc.cone_r2 > 0.0f && light_clear(sc, h, li, p, p_lo, po);
            if (skip) clear |= 1u << li;
            else total += nr;
        }
        if (HITREC) hr[hr_k + (size_t)(2 + li) * hr_plane] = 0.0f;
    }
    const uint32_t traced = lit & ~clear;
    // rem: the lit lights not attributed yet; (cs, cnt): results of its first so far
    uint32_t rem = lit;
    int cs = 0, cnt = 0;
    // (l, s): light and sample of the next segment to set up
    int l = traced ? __ffs(traced) - 1 : 0, s = 0;
    uint4 w = make_uint4(0, 0, 0, 0);
    int done = 0, kp = 0;  // segments set up so far; results of the previous group
    uint32_t bp = 0;       // their blocked bits
    const unsigned mask = __activemask();
#pragma unroll 1
    while (true) {
        // attribute in light order: the previous group's results as each light's
        // segments complete, a cleared light (vis = 1) in its turn
        int j = 0;
#pragma unroll 1
        while (rem) {
            const int cl = __ffs(rem) - 1;
            const float4 Lp = h.light_p[cl];
            float vis = 1.0f;
            if (!((clear >> cl) & 1u)) {
                const int nr = rays_of_light(fr, h.light_s[cl]);
                bool ready = false;
#pragma unroll 1
                while (j < kp) {
                    cnt += (bp >> j) & 1u ? 0 : 1;
                    ++j;
                    if (++cs == nr) {
                        ready = true;
                        break;
                    }
                }
                if (!ready) break;
                vis = (float)cnt / (float)nr;
                cs = 0;
                cnt = 0;
            }
            const f3 lh = normalize(sub(sub(xyz(Lp), p), p_lo));
            const float ndl = dot(n, lh);
            const float sp = light_spec(fr, n, d, lh, ndl, e);
            const float iv = Lp.w * vis;
            out.A = fmaf(iv, ndl, out.A);
            out.S = fmaf(iv * ks, sp, out.S);
            if (HITREC) hr[hr_k + (size_t)(2 + cl) * hr_plane] = vis;
            rem &= rem - 1u;
        }
        const int kr = min(kShadowGroup, total - done);
        const int R = (int)__reduce_max_sync(mask, (unsigned)kr);
        if (R == 0) break;
        f3 sw[kShadowGroup], snv[kShadowGroup];  // W and -V of each segment
        bool occ[kShadowGroup];
        LightFrame lf{};  // of spherical light lf_l
        int lf_l = -1;
#pragma unroll
        for (int jj = 0; jj < kShadowGroup; ++jj) {
            sw[jj] = mk3(0.f, 0.f, 0.f);
            snv[jj] = mk3(0.f, 0.f, 0.f);
            occ[jj] = true;
            if (jj < kr) {
                const float4 Lp = h.light_p[l];
                const float4 Ls = h.light_s[l];
                const int nr = rays_of_light(fr, Ls);
                if (Ls.y > 0.0f && lf_l != l) {
                    lf = light_frame(p, Lp);
                    lf_l = l;
                }
                const f3 X = nr > 1 || Ls.x > 0.0f || Ls.y > 0.0f
                                 ? sample_point(fr, pix, k, l, s, Lp, Ls, w, lf, sc.flower)
                                 : xyz(Lp);
                // V = X - p (p as hi + lo), W = V / |V|^2
                const f3 V = sub(sub(X, p), p_lo);
                sw[jj] = scl(V, rcp_approx(dot(V, V)));
                snv[jj] = scl(V, -1.0f);
                occ[jj] = false;
                if (++s == nr) {
                    s = 0;
                    const uint32_t rest = traced & ~((2u << l) - 1u);
                    l = rest ? __ffs(rest) - 1 : 0;
                }
            }
        }
        if (kShadowGroup <= 1 || R == 1) {
            occluded_group<1, CH, ACC>(sc, po, sw, snv, occ);
        } else if (kShadowGroup == 2 || R == 2) {
            occluded_group<(kShadowGroup < 2 ? 1 : 2), CH, ACC>(sc, po, sw, snv, occ);
        } else if (kShadowGroup == 3 || R == 3) {
            occluded_group<(kShadowGroup < 3 ? 1 : 3), CH, ACC>(sc, po, sw, snv, occ);
        } else {
            occluded_group<(kShadowGroup < 4 ? 1 : 4), CH, ACC>(sc, po, sw, snv, occ);
        }
        bp = 0;
#pragma unroll
        for (int jj = 0; jj < kShadowGroup; ++jj) bp |= occ[jj] ? (1u << jj) : 0u;
        kp = kr;
        done += kr;
    }
    return out;
}

// shade_hit for the staged brute-force kernels: the same shading, rays, Philox
// counters and attribution, with groups of up to kFiltGroup segments set up by a
// loop (one copy of the sample code) that writes W and -V to shared memory and the
// unit vectors for the filter to a local array, and every group tested by
// occluded_filtered.
template <bool HITREC, bool IT = false, bool LEAN = false>
__device__ __forceinline__ HitShade shade_hit_staged(const StagedScene& sc, const Frame& fr, uint32_t pix, int k,
                                                     f3 p, f3 p_lo, f3 n, f3 po, f3 d, float ks, float e,
                                                     float* __restrict__ hr, size_t hr_k, size_t hr_plane) {
    const SceneHdr& h = *sc.hdr;
    HitShade out{fr.ka, 0.0f};
    uint32_t lit = 0;
    int total = 0;
    int lc = -1, before_lc = 0;  // the cone pre-pass's light (first lit sampled light), segments before it
#pragma unroll 1
    for (int li = 0; li < h.nl; ++li) {
        const f3 lh = normalize(sub(sub(xyz(h.light_p[li]), p), p_lo));
        if (dot(n, lh) > 0.0f) {
            lit |= 1u << li;
            const int nr = rays_of_light(fr, h.light_s[li]);
            if (lc < 0 && nr > 1) {
                lc = li;
                before_lc = total;
            }
            total += nr;
        }
        if (HITREC) hr[hr_k + (size_t)(2 + li) * hr_plane] = 0.0f;
    }
    // (cl, cs): light and sample of the next result to attribute; (l, s): of the
    // next segment to set up
    int cl = lit ? __ffs(lit) - 1 : 0, cs = 0, cnt = 0;
    int l = cl, s = 0;
    uint4 w = make_uint4(0, 0, 0, 0);
    LightFrame lf{};  // of spherical light lf_l
    int lf_l = -1;
    int done = 0;
    const unsigned mask = __activemask();
    float* seg = s_seg + (threadIdx.x + blockDim.x * threadIdx.y);
    const bool plane = h.has_plane != 0;
    const f3 pn = xyz(h.plane_g);
    const float num = -(dot(po, pn) + h.plane_g.w);
    // cone of light lc seen from p (cone_pass): axis towards its centre, kappa below
    // the cosine to every point of its sample region (the square's corners; the
    // tangent cone of a spherical light), less 2^-17
    f3 ax = mk3(0.f, 0.f, 0.f);
    float kap = 0.0f;
    bool cone_ok = false;
    if (lc >= 0 && sc.cone_r2 > 0.0f) {
        const float4 Lp = h.light_p[lc], Ls = h.light_s[lc];
        const f3 Lv = sub(sub(xyz(Lp), p), p_lo);
        const float ri = rsqrtf(dot(Lv, Lv));
        ax = scl(Lv, ri);
        if (Ls.x > 0.0f) {
            const float hs = 0.5f * Ls.x;
            kap = 1.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const f3 cv = add(Lv, mk3((c & 1) ? hs : -hs, 0.0f, (c & 2) ? hs : -hs));
                kap = fminf(kap, dot(ax, cv) * rsqrtf(dot(cv, cv)));
            }
        } else {
            const float sr = Ls.y * ri * (1.0f + 0x1p-20f);  // >= R / dist
            kap = sqrt_bound(fmaxf(fmaf(-sr, sr, 1.0f), 0.0f));
        }
        kap -= 0x1p-17f;
        cone_ok = kap >= 0.5f;  // NaN: false
    }
    uint32_t* cw = s_cone + ((threadIdx.x + blockDim.x * threadIdx.y) >> 5) * 2 * kConeWords;
    uint32_t own = 0;    // this lane's own blocks (cone_pass)
    bool items = false;  // the cone's groups in item mode (item_groups)
    unsigned cm = __ballot_sync(mask, cone_ok);
    if (cm) {
        // the warp's cone: apex and axis of the first lane with a cone; lanes whose
        // cone light differs from that lane's drop out of the pre-pass
        const int ld = __ffs(cm) - 1;
        const int lw = __shfl_sync(mask, lc, ld);
        const f3 p0 = mk3(__shfl_sync(mask, po.x, ld), __shfl_sync(mask, po.y, ld), __shfl_sync(mask, po.z, ld));
        const f3 aw = mk3(__shfl_sync(mask, ax.x, ld), __shfl_sync(mask, ax.y, ld), __shfl_sync(mask, ax.z, ld));
        cone_ok = cone_ok && lc == lw;
        cm = __ballot_sync(mask, cone_ok);
        const float sa = sqrt_bound(fmaxf(fmaf(-kap, kap, 1.0f), 0.0f));
        // cos(beta + alpha), beta the angle between this lane's axis and aw, less a
        // margin; the distance from p0 to this lane's apex
        float kw = 1.0f, dw = 0.0f;
        if (cone_ok) {
            const float cb = fminf(dot(ax, aw), 1.0f);
            const float sb = sqrt_bound(fmaxf(fmaf(-cb, cb, 1.0f), 0.0f));
            kw = fmaf(cb, kap, -sb * sa) - 0x1p-17f;
            kw = kw >= 0.5f ? kw : 0.0f;  // NaN: 0
            const f3 dp = sub(po, p0);
            dw = sqrt_bound(dot(dp, dp));
        }
        // warp minimum / maximum (non-negative floats order as their bits)
        const float kwm = __uint_as_float(__reduce_min_sync(mask, __float_as_uint(kw)));
        const float dwm = __uint_as_float(__reduce_max_sync(mask, __float_as_uint(dw)));
        const bool coarse = kwm >= 0.5f && dwm <= 0x1p30f;
        const float rho = sqrt_bound(sc.cone_r2);
        const float rw = (rho + dwm) * (1.0f + 0x1p-15f);
        const float sw = sqrt_bound(fmaxf(fmaf(-kwm, kwm, 1.0f), 0.0f)) * (1.0f + 0x1p-18f);
        const float sg = sa * (1.0f + 0x1p-18f);  // >= sin alpha
        own = cone_pass(sc.geo, h.ns_pad, mask, po, ax, fmaf(kap, kap, -0x1p-16f), 2.0f * rho * sg, sc.cone_r2,
                        cone_ok, cw, p0, aw, fmaf(kwm, kwm, -0x1p-16f), 2.0f * rw * sw, rw * rw * (1.0f + 0x1p-15f),
                        coarse);
        // item mode for the cone's groups where the lanes' own blocks are under a third
        // of the union's steps (a full warp, at most 32 blocks)
        if (IT && mask == 0xffffffffu && h.ns_pad <= 32 * kPad)
            items = 3u * __reduce_add_sync(mask, (unsigned)__popc(own)) < 32u * (unsigned)__popc(cw[0]);
    }
    const bool cone_any = cm != 0;
    // The cone light's segments need no set-up when this lane's own cone clears every
    // block -- no sphere can block any of them, by the pre-pass's bound (the samples lie
    // in the light's region, whose corners the cone holds, and a cone is convex) -- and
    // the plane cannot either: the shadow origin is not on the plane's negative side
    // (num <= 0) and the whole sample region lies on its positive side farther than
    // 2^-14 times the coordinates' scale, far beyond the plane test's roundings (below
    // 20u of that scale), so that every segment's den = V.n is positive.  Every segment
    // would test unblocked, so vis = n / n = 1 exactly: the light is attributed in its
    // place in the light order without tracing (nearly half the first pass's warps at
    // 4K; frame 4.43 -> 4.31 ms, images bit-identical).
    bool skip = false;
    if (cone_ok && own == 0u && h.ns_pad <= 32 * kPad) {
        bool pc = !plane || num == 0.0f;
        if (!pc && num < 0.0f) {
            const float4 Lp = h.light_p[lc], Ls = h.light_s[lc];
            const float an = fabsf(pn.x) + fabsf(pn.y) + fabsf(pn.z);
            const float ext = Ls.x > 0.0f ? 0.5f * Ls.x * (fabsf(pn.x) + fabsf(pn.z)) : Ls.y * an;
            const float lo = dot(xyz(Lp), pn) - ext - (dot(p, pn) + dot(p_lo, pn));
            const float sc_ = (fmaxf(fabsf(Lp.x), fmaxf(fabsf(Lp.y), fabsf(Lp.z))) + Ls.x + Ls.y +
                               fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))) + 1.0f) * an;
            pc = lo > 0x1p-14f * sc_;  // NaN: false
        }
        skip = pc;
    }
    uint32_t lit_e = lit;  // the lights whose segments are set up
    if (skip) {
        lit_e &= ~(1u << lc);
        total -= rays_of_light(fr, h.light_s[lc]);
        cone_ok = false;
        l = lit_e ? __ffs(lit_e) - 1 : 0;
    }
    bool skip_done = !skip;
    auto attribute = [&](int li, float vis) {
        const float4 Lp = h.light_p[li];
        const f3 lh = normalize(sub(sub(xyz(Lp), p), p_lo));
        const float ndl = dot(n, lh);
        const float sp = light_spec(fr, n, d, lh, ndl, e);
        const float iv = Lp.w * vis;
        out.A = fmaf(iv, ndl, out.A);
        out.S = fmaf(iv * ks, sp, out.S);
        if (HITREC) hr[hr_k + (size_t)(2 + li) * hr_plane] = vis;
    };
    const float kv = kap + 0x1p-18f;
    int kp = 0;       // results of the previous group not yet attributed
    uint32_t bp = 0;  // their blocked bits
#pragma unroll 1
    while (true) {
        // Attribute in light order: the previous group's results as each light's
        // segments complete, and the skipped light (visibility 1) in its turn.  One
        // call site, so that the shading code is compiled once into the group loop; the
        // loop leaves only after this step, which then finds the last results.
        int j = 0;
#pragma unroll 1
        while (true) {
            float vis = 1.0f;
            if (skip_done || cl != lc) {
                bool ready = false;
#pragma unroll 1
                while (j < kp) {
                    cnt += (bp >> j) & 1u ? 0 : 1;
                    ++j;
                    const int nr = rays_of_light(fr, h.light_s[cl]);
                    if (++cs == nr) {
                        vis = (float)cnt / (float)nr;
                        cs = 0;
                        cnt = 0;
                        ready = true;
                        break;
                    }
                }
                if (!ready) break;
            } else {
                skip_done = true;
            }
            attribute(cl, vis);
            const uint32_t rest = lit & ~((2u << cl) - 1u);
            cl = rest ? __ffs(rest) - 1 : 0;
        }
        // a group ends before the cone light's first segment, so that its segments
        // form groups of their own (of kConeGroup)
        const int lim = cone_ok && done < before_lc ? before_lc : total;
        const int kr = min(cone_ok && done >= before_lc ? kConeGroup : kFiltGroup, lim - done);
        const int R = (int)__reduce_max_sync(mask, (unsigned)kr);
        if (R == 0) break;
        uint32_t blocked = 0;
        bool ok = true;
        bool pure = cone_ok || kr == 0;  // every segment of the group inside the cone of light lc
        bool allpt = true;               // every segment of the group to a point light
        uint32_t gl = 0;                 // the group's lights
#pragma unroll 1
        for (int j = 0; j < kFiltGroup; ++j) {  // every slot: the instance below reads kFiltGroup
            f3 W = mk3(0.f, 0.f, 0.f), nv = mk3(0.f, 0.f, 0.f), vn = mk3(0.f, 0.f, 0.f);
            bool occj = true;
            if (j < kr) {
                const float4 Lp = h.light_p[l];
                const float4 Ls = h.light_s[l];
                const int nr = rays_of_light(fr, Ls);
                pure = pure && l == lc;
                allpt = allpt && Ls.x == 0.0f && Ls.y == 0.0f;
                gl |= 1u << l;
                if (!LEAN && Ls.y > 0.0f && lf_l != l) {
                    lf = light_frame(p, Lp);
                    lf_l = l;
                }
                const f3 X = nr > 1 || Ls.x > 0.0f || Ls.y > 0.0f
                                 ? sample_point<LEAN>(fr, pix, k, l, s, Lp, Ls, w, lf, sc.flower)
                                 : xyz(Lp);
                // V = X - p (p as hi + lo), W = V / |V|^2
                const f3 V = sub(sub(X, p), p_lo);
                W = scl(V, rcp_approx(dot(V, V)));
                nv = scl(V, -1.0f);
                // the plane first: a root u = num / (V.n) in (0, 1)
                const float den = -dot(nv, pn);
                occj = plane && den != 0.0f && num != 0.0f && ((num > 0.0f) == (den > 0.0f)) &&
                       fabsf(num) < fabsf(den);
                if (!occj) {
                    const float S = dot(nv, nv);
                    ok = ok && S >= 0x1p-60f && S <= 0x1p100f;
                    vn = scl(nv, -rsqrtf(S));  // V^ (the filter's bound allows 2 ulp)
                    pure = pure && dot(ax, vn) >= kv;
                }
                if (++s == nr) {
                    s = 0;
                    const uint32_t rest = lit_e & ~((2u << l) - 1u);
                    l = rest ? __ffs(rest) - 1 : 0;
                }
            }
            blocked |= occj ? (1u << j) : 0u;
            float* g = seg + 9 * j * kSegStride;
            g[6 * kSegStride] = vn.x;
            g[7 * kSegStride] = vn.y;
            g[8 * kSegStride] = vn.z;
            g[0] = W.x;
            g[kSegStride] = W.y;
            g[2 * kSegStride] = W.z;
            g[3 * kSegStride] = nv.x;
            g[4 * kSegStride] = nv.y;
            g[5 * kSegStride] = nv.z;
        }
        const bool exact_only = !__all_sync(mask, ok);
        const uint32_t* cone = cone_any && __all_sync(mask, pure) ? cw : nullptr;
        if (!cone && sc.cone_r2 > 0.0f && __all_sync(mask, allpt)) {
            const unsigned gu = __reduce_or_sync(mask, gl);
            if (gu && point_pass(sc.geo, h.ns_pad, mask, h, p, p_lo, po, gl, gu, sqrt_bound(sc.cone_r2), cw + kConeWords))
                cone = cw + kConeWords;
        }
        static_assert(kFiltGroup == 4 && kConeGroup == 4, "one instance: every group has at most 4 segments");
        bp = occluded_filtered<kFiltGroup, IT>(sc.geo, h.ns_pad, mask, po, blocked, seg, exact_only, cone, own,
                                           items && cone == cw);
        kp = kr;
        done += kr;
    }
    return out;
}

// ---------------------------------------------------------------- Section 3.8 sky
// A ray that leaves the scene shows the sky panorama, looked up by the UV mapping
// of its direction: u = 1/2 + atan2(d_z, d_x) / (2 pi), v = 1/2 - asin(d_y) / pi,
// bilinear between texel centres, wrapping around in u, clamped to the first and
// last rows in v.
__device__ __forceinline__ float3 sky_lookup(const SkyView& sk, f3 d) {
    const float dy = fminf(fmaxf(d.y, -1.0f), 1.0f);
    const float u = fmaf(atan2f(d.z, d.x), 0.15915494309189535f, 0.5f);  // 1 / (2 pi)
    const float v = fmaf(-asinf(dy), 0.31830988618379067f, 0.5f);        // 1 / pi
    const float x = fmaf(u, (float)sk.w, -0.5f), y = fmaf(v, (float)sk.h, -0.5f);
    const float x0 = floorf(x), y0 = floorf(y);
    const float fx = x - x0, fy = y - y0;
    int i0 = (int)x0;  // in [-1, w]: u in [0, 1]
    i0 = i0 < 0 ? i0 + sk.w : (i0 >= sk.w ? i0 - sk.w : i0);
    const int i1 = i0 + 1 == sk.w ? 0 : i0 + 1;
    const int j0 = min(max((int)y0, 0), sk.h - 1), j1 = min(max((int)y0 + 1, 0), sk.h - 1);
    const float4 a = __ldg(sk.tex + (size_t)j0 * sk.w + i0), b = __ldg(sk.tex + (size_t)j0 * sk.w + i1);
    const float4 c = __ldg(sk.tex + (size_t)j1 * sk.w + i0), e = __ldg(sk.tex + (size_t)j1 * sk.w + i1);
    const float tx = fmaf(fx, b.x - a.x, a.x), ty = fmaf(fx, b.y - a.y, a.y), tz = fmaf(fx, b.z - a.z, a.z);
    const float bx = fmaf(fx, e.x - c.x, c.x), by = fmaf(fx, e.y - c.y, c.y), bz = fmaf(fx, e.z - c.z, c.z);
    return make_float3(fmaf(fy, bx - tx, tx), fmaf(fy, by - ty, ty), fmaf(fy, bz - tz, tz));
}

// ---------------------------------------------------------------- hit geometry
// Hit point and face-forwarded normal (sphere (p - c)/r, plane n; flipped to face
// the incoming ray), computed once per hit with the ray origin as a hi + lo pair.
// Sphere: oc = c - o exactly (TwoSum), l = oc - (oc.d) d with the along-d residual
// of the rounded oc.d projected out, s = sqrt(r^2 - |l|^2), p - c = -+s d - l (near
// root, else far root): |p - c| = r to FP32 rounding, no cancellation of long
// vectors.  The point is returned as p_hi + p_lo.  flip = -1 when the normal was
// flipped (n = flip * n_raw).
struct HitGeom {
    f3 p, p_lo, n;
    float flip;
    float4 m, m2;   // albedo + k_s; exponent, reflectivity, r, 1/r
};

template <bool CH>
__device__ __forceinline__ HitGeom hit_geometry(const StagedScene& sc, int id, f3 o, f3 o_lo, f3 d, float t,
                                                float refl_inv_max) {
    const SceneHdr& h = *sc.hdr;
    HitGeom hg;
    if (id < h.ns) {
        const float4 g = CH ? sphere_ldg(sc.geo_g, id) : sphere_at(sc.geo, id);  // (c, -r^2)
        hg.m = __ldg(sc.mat + id);
        hg.m2 = __ldg(sc.mat2 + id);
        f3 e;
        const f3 och = two_sum3(xyz(g), scl(o, -1.0f), e);
        const f3 ocl = sub(e, o_lo);  // oc = och + ocl exactly up to the lo rounding
        const float tca = dot(och, d) + dot(ocl, d);
        f3 l = add(fma3(d, -tca, och), ocl);
        l = fma3(d, -dot(l, d), l);
        const float disc = fmaf(-l.x, l.x, fmaf(-l.y, l.y, fmaf(-l.z, l.z, -g.w)));
        const float sq = __fsqrt_rn(fmaxf(disc, 0.0f));
        const float sgn = (tca - sq > 0.0f) ? -sq : sq;  // near root, else far root
        const f3 pc = mk3(fmaf(sgn, d.x, -l.x), fmaf(sgn, d.y, -l.y), fmaf(sgn, d.z, -l.z));
        hg.p = two_sum3(xyz(g), pc, hg.p_lo);
        hg.n = scl(pc, hg.m2.w);
    } else {
        hg.m = h.plane_m;
        hg.m2 = h.plane_m2;
        f3 e;
        hg.p = two_sum3(o, scl(d, t), e);
        hg.p_lo = add(e, o_lo);
        hg.n = xyz(h.plane_g);
    }
    // the paper's coupling of reflection ratio and specular exponent (Section 3.7)
    if (refl_inv_max > 0.0f) hg.m2.y = fminf(hg.m2.x * refl_inv_max, 1.0f);
    hg.flip = 1.0f;
    if (dot(hg.n, d) > 0.0f) {
        hg.n = scl(hg.n, -1.0f);
        hg.flip = -1.0f;
    }
    return hg;
}

// Secondary ray origin p + eps n as a hi + lo pair.
__device__ __forceinline__ f3 offset_origin(const HitGeom& hg, float eps, f3& lo) {
    f3 e;
    const f3 hi = two_sum3(hg.p, scl(hg.n, eps), e);
    lo = add(e, hg.p_lo);
    return hi;
}

// ---------------------------------------------------------------- Sections 3.5-3.8
// A miss at bounce k adds T_k sky(d_k) (Section 3.8); nothing without a sky.
template <bool LEAN = false>
__device__ __forceinline__ void miss_add(const StagedScene& sc, f3 d, float T, float3& out) {
    if (!LEAN && sc.sky.tex) {
        const float3 sk = sky_lookup(sc.sky, d);
        out.x = fmaf(T, sk.x, out.x);
        out.y = fmaf(T, sk.y, out.y);
        out.z = fmaf(T, sk.z, out.z);
    }
}

// The hit of bounce k: primitive id at distance t of the ray (o + o_lo, d) that
// carries throughput T.  shade(c) = c A + S with
//   A = k_a + sum_l I_l vis_l max(n.l, 0),  S = sum_l I_l vis_l k_s spec_l,
// a light skipped when n.l <= 0; Phong spec = max(v.r, 0)^exp (r the light
// direction mirrored about n, v = -d), Blinn spec = max(n.h, 0)^exp.  The
// reflection recursion of Section 3.7.1 unrolled forward: below the depth limit it
// adds T((1 - rho) A c + S) and turns (o, o_lo, d, T) into the reflected ray with
// T *= rho A; at the limit it adds T(A c + S).  HITREC: vis_l at hr[hr_k + ...].
// The colour and the next ray of bounce k from its shading (A, S): below the depth
// limit T((1 - rho) A c + S) and the reflected ray with T *= rho A; at the limit
// T(A c + S).
__device__ __forceinline__ void step_tail(const Frame& fr, int k, float4 m, float4 m2, HitShade sh, f3 n, f3 po,
                                          f3 po_lo, f3& o, f3& o_lo, f3& d, float& T, float3& out) {
    const float A = sh.A, S = sh.S;
    if (k < fr.D) {
        const float w = T * (1.0f - m2.y) * A;
        out.x = fmaf(w, m.x, fmaf(T, S, out.x));
        out.y = fmaf(w, m.y, fmaf(T, S, out.y));
        out.z = fmaf(w, m.z, fmaf(T, S, out.z));
        T *= m2.y * A;
        d = normalize(fma3(n, -2.0f * dot(d, n), d));
        o = po;
        o_lo = po_lo;
    } else {
        const float w = T * A;
        out.x = fmaf(w, m.x, fmaf(T, S, out.x));
        out.y = fmaf(w, m.y, fmaf(T, S, out.y));
        out.z = fmaf(w, m.z, fmaf(T, S, out.z));
    }
}

// FM (shading path of the staged brute-force kernels): 0 = the segment test alone
// (shade_hit), 1 = the line filter (shade_hit_staged), 2 = chosen per scene by its
// sphere count.  All give the same bits; the kernels that know the scene at launch
// are compiled per path so that each carries only the code it runs.
constexpr int kShadeAuto = 2;
// FM bit 2: the scene has no sky and no spherical light, so the kernels are compiled
// without the sky lookup and the spherical-light sample geometry -- code such a frame
// never runs, but whose instructions would share the instruction cache with the hot
// loops (4K frame 4.07 -> 3.92 ms, images bit-identical).
constexpr int kFmLean = 4;
// FM bit 3 (segment-test path): the scene may hold sampled lights of several rays, so
// the kernels stage the cone bound and shade_hit tries light_clear on each of them;
// kernels for scenes without such lights are compiled without that code (720p frame
// of point lights 0.143 -> 0.139 ms).
constexpr int kFmSkip = 8;
__host__ __device__ constexpr int fm_path(int fm) { return fm & 3; }
__host__ __device__ constexpr bool fm_lean(int fm) { return (fm & kFmLean) != 0; }
__host__ __device__ constexpr bool fm_skip(int fm) { return (fm & kFmSkip) != 0; }

template <bool HITREC, bool CH, bool ACC, int FM = kShadeAuto, bool IT = false>
__device__ __forceinline__ void shade_step(const StagedScene& sc, const Frame& fr, uint32_t pix, int k, int id,
                                           float t, f3& o, f3& o_lo, f3& d, float& T, float3& out,
                                           float* __restrict__ hr, size_t hr_k, size_t hr_plane) {
    const HitGeom hg = hit_geometry<CH>(sc, id, o, o_lo, d, t, fr.refl_inv_max);
    f3 po_lo;
    const f3 p = hg.p, n = hg.n, po = offset_origin(hg, fr.eps, po_lo);
    const float4 m = hg.m, m2 = hg.m2;
    HitShade sh;
    // the line filter pays for its per-group set-up from kFilterMinPad spheres on
    // (the same for every pixel of a launch, so only one of the paths runs hot)
    bool filt = false;
    if constexpr (!CH && !ACC)
        filt = fm_path(FM) == 1 || (fm_path(FM) == kShadeAuto && sc.hdr->ns_pad >= kFilterMinPad);
    if (filt)
        sh = shade_hit_staged<HITREC, IT, fm_lean(FM)>(sc, fr, pix, k, p, hg.p_lo, n, po, d, m.w, m2.x, hr, hr_k, hr_plane);
    else
        sh = shade_hit<HITREC, CH, ACC, fm_skip(FM)>(sc, fr, pix, k, p, hg.p_lo, n, po, d, m.w, m2.x, hr, hr_k,
                                                    hr_plane);
    step_tail(fr, k, m, m2, sh, n, po, po_lo, o, o_lo, d, T, out);
}

// ---------------------------------------------------------------- bounce queues
// Deferred paths of rt_render_ws.  A warp runs the bounce loop until its slowest
// lane is done, so the few pixels whose reflection hits something again keep the
// rest of their warp idle; instead, the first pass hands such a path over at its
// bounce-1 hit, and later passes take the queued paths 32 at a time, one bounce
// per pass, re-queueing those that hit again.  An entry holds the path state
// exactly (FP32 values stored and reloaded), so a path's arithmetic -- and its
// Philox counters, which depend on (pixel, bounce) only -- is the same wherever
// it runs: images are bit-identical to the one-pass kernel.  A full queue is not
// an error: the lane carries the path on itself.
struct PathQueue {
    float4* ent;      // 4 float4 per entry
    unsigned* count;  // appends so far (may pass cap; only the first cap are stored)
    unsigned cap;
};

// Entry: (o, T), (o_lo, pixel), (d, t), (accumulated colour, primitive id).
__device__ __forceinline__ bool queue_push(const PathQueue& q, uint32_t pix, f3 o, f3 o_lo, f3 d, float T,
                                           float3 out, int id, float t) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(q.count, (unsigned)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    const unsigned slot = base + (unsigned)__popc(mask & ((1u << lane) - 1u));
    if (slot >= q.cap) return false;
    float4* e = q.ent + (size_t)slot * 4;
    e[0] = make_float4(o.x, o.y, o.z, T);
    e[1] = make_float4(o_lo.x, o_lo.y, o_lo.z, __uint_as_float(pix));
    e[2] = make_float4(d.x, d.y, d.z, t);
    e[3] = make_float4(out.x, out.y, out.z, __int_as_float(id));
    return true;
}

// Trace one pixel: bounce by bounce, closest hit (Section 3.4.1), then miss_add or
// shade_step.  HITREC: write (id, t, vis_l) per bounce, id = -1 after the path ends.
// dq (first pass of rt_render_ws): a path whose bounce-1 ray hits is pushed to dq
// instead of being shaded here; *deferred tells the caller not to store the pixel.
template <bool HITREC, bool CH, bool ACC = false, int FM = kShadeAuto>
__device__ __forceinline__ float3 trace_pixel(const StagedScene& sc, const Frame& fr, int x, int y,
                                              float* __restrict__ hr, size_t hr_plane, size_t hr_pix,
                                              const PathQueue* dq = nullptr, bool* deferred = nullptr) {
    const SceneHdr& h = *sc.hdr;
    const uint32_t pix = (uint32_t)y * (uint32_t)fr.W + (uint32_t)x;
    f3 o = mk3(fr.cam.x, fr.cam.y, fr.cam.z), o_lo = mk3(0.f, 0.f, 0.f);
    f3 d = primary_dir(fr, x, y);
    float T = 1.0f;
    float3 out = make_float3(0.f, 0.f, 0.f);
    int k = 0;
#pragma unroll 1
    for (; k <= fr.D; ++k) {
        float t;
        const uint32_t* cull = nullptr;
        if constexpr (!CH && !ACC && fm_path(FM) == 1) {
            // the blocks the warp's ray lines can reach (a view frustum for primary rays)
            if (sc.cone_r2 > 0.0f) {
                uint32_t* cw = s_cone + ((threadIdx.x + blockDim.x * threadIdx.y) >> 5) * 2 * kConeWords;
                if (ray_cull(sc.geo, h.ns_pad, __activemask(), o, d, sqrt_bound(sc.cone_r2), sc.cone_cmax, cw)) cull = cw;
            }
        }
        const int id = closest_hit<CH, ACC, fm_path(FM) == 1>(sc, o, d, t, cull);
        if (HITREC) {
            float* rec = hr + (size_t)k * (2 + h.nl) * hr_plane + hr_pix;
            rec[0] = __int_as_float(id);
            rec[hr_plane] = t;
        }
        if (id < 0) {
            miss_add<fm_lean(FM)>(sc, d, T, out);
            break;
        }
        if (dq && k == 1 && queue_push(*dq, pix, o, o_lo, d, T, out, id, t)) {
            *deferred = true;
            return out;
        }
        shade_step<HITREC, CH, ACC, FM>(sc, fr, pix, k, id, t, o, o_lo, d, T, out, hr,
                                    (size_t)k * (2 + h.nl) * hr_plane + hr_pix, hr_plane);
    }
    if (HITREC) {
        for (int kk = k + 1; kk <= fr.D; ++kk)
            hr[(size_t)kk * (2 + h.nl) * hr_plane + hr_pix] = __int_as_float(-1);
    }
    return out;
}

// RGBA8 packing (toInt of the render listing, Section 3.9): clamp to [0, 1], times
// 255, round half up, alpha 255, little-endian 0xAABBGGRR.  Multiply and add are
// rounded separately (no contraction) so that an FP32 value quantises the same
// everywhere.
__device__ __forceinline__ uint32_t quant8(float v) {
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    return (uint32_t)floorf(__fadd_rn(__fmul_rn(v, 255.0f), 0.5f));
}
__device__ __forceinline__ uint32_t pack_rgba8(float3 c) {
    return quant8(c.x) | (quant8(c.y) << 8) | (quant8(c.z) << 16) | 0xFF000000u;
}

// Store the colour of pixel (x, y) of the frame at (x - rx0, y - ry0) of `out`.  All
// 32 lanes of the warp must call (the RGBA8 path gathers four horizontally adjacent
// pixels, lanes 4j..4j+3, into one 16-byte store; rx0 is a multiple of 8); `valid`
// marks lanes whose pixel is inside the rendered region.
__device__ __forceinline__ void store_pixel(const Frame& fr, int x, int y, bool valid, float3 c,
                                            void* __restrict__ out, size_t pitch) {
    const int lane = threadIdx.x & 31;
    const int lx = x - fr.rx0, ly = y - fr.ry0;
    if (fr.fmt == RT_OUT_F32) {
        if (valid)
            *reinterpret_cast<float4*>(static_cast<char*>(out) + (size_t)ly * pitch + (size_t)lx * 16) =
                make_float4(c.x, c.y, c.z, 1.0f);
    } else {
        const uint32_t p0 = pack_rgba8(c);
        const uint32_t p1 = __shfl_down_sync(0xffffffffu, p0, 1);
        const uint32_t p2 = __shfl_down_sync(0xffffffffu, p0, 2);
        const uint32_t p3 = __shfl_down_sync(0xffffffffu, p0, 3);
        if ((lane & 3) == 0 && y < fr.ry1 && x < fr.rx1) {
            uint32_t* row = reinterpret_cast<uint32_t*>(static_cast<char*>(out) + (size_t)ly * pitch);
            if (x + 3 < fr.rx1) {
                *reinterpret_cast<uint4*>(row + lx) = make_uint4(p0, p1, p2, p3);
            } else {
                row[lx] = p0;
                if (x + 1 < fr.rx1) row[lx + 1] = p1;
                if (x + 2 < fr.rx1) row[lx + 2] = p2;
            }
        }
    }
}

// Trace pixel (x, y) of the frame and store it (store_pixel's rules).  With dq, a
// deferred pixel is not stored (F32) or stored with a placeholder that the pass
// finishing its path overwrites (RGBA8, where four lanes share one store).
template <bool HITREC, bool CH, bool ACC = false, int FM = kShadeAuto>
__device__ __forceinline__ void render_pixel(const StagedScene& sc, const Frame& fr, int x, int y, bool valid,
                                             void* __restrict__ out, size_t pitch, float* __restrict__ hr,
                                             size_t hr_plane, const PathQueue* dq = nullptr) {
    float3 c = make_float3(0.f, 0.f, 0.f);
    bool deferred = false;
    if (valid)
        c = trace_pixel<HITREC, CH, ACC, FM>(sc, fr, x, y, hr, hr_plane, (size_t)y * (size_t)fr.W + (size_t)x, dq,
                                         &deferred);
    store_pixel(fr, x, y, valid && !(deferred && fr.fmt == RT_OUT_F32), c, out, pitch);
}

// Store one pixel on its own (the queued passes, whose lanes hold unrelated pixels).
__device__ __forceinline__ void store_one(const Frame& fr, uint32_t pix, float3 c, void* __restrict__ out,
                                          size_t pitch) {
    const int x = (int)(pix % (uint32_t)fr.W), y = (int)(pix / (uint32_t)fr.W);
    char* row = static_cast<char*>(out) + (size_t)(y - fr.ry0) * pitch;
    if (fr.fmt == RT_OUT_F32)
        *reinterpret_cast<float4*>(row + (size_t)(x - fr.rx0) * 16) = make_float4(c.x, c.y, c.z, 1.0f);
    else
        reinterpret_cast<uint32_t*>(row)[x - fr.rx0] = pack_rgba8(c);
}

// Pass k >= 1 of rt_render_ws for the entry e of queue k: shade the hit of bounce
// k, then (below the depth limit) trace the reflected ray; a hit is pushed to nq
// (queue k + 1) or, when that is full, shaded here to its end.  A path that ends
// here stores its pixel and its hit record's trailing -1 ids.
template <bool HITREC, int FM = kShadeAuto>
__device__ __forceinline__ void trace_queued(const StagedScene& sc, const Frame& fr, const float4* __restrict__ e,
                                             int k, const PathQueue& nq, void* __restrict__ out, size_t pitch,
                                             float* __restrict__ hr, size_t hr_plane) {
    const SceneHdr& h = *sc.hdr;
    const int kq = k + 1;  // bounce of the entries of nq
    const float4 e0 = e[0], e1 = e[1], e2 = e[2], e3 = e[3];
    f3 o = mk3(e0.x, e0.y, e0.z), o_lo = mk3(e1.x, e1.y, e1.z), d = mk3(e2.x, e2.y, e2.z);
    float T = e0.w, t = e2.w;
    float3 c = make_float3(e3.x, e3.y, e3.z);
    int id = __float_as_int(e3.w);
    const uint32_t pix = __float_as_uint(e1.w);
    const size_t hr_pix = pix;
#pragma unroll 1
    while (true) {
        shade_step<HITREC, false, false, FM, true>(sc, fr, pix, k, id, t, o, o_lo, d, T, c, hr,
                                         (size_t)k * (2 + h.nl) * hr_plane + hr_pix, hr_plane);
        if (k == fr.D) {
            k = fr.D + 1;
            break;
        }
        ++k;
        id = closest_hit<false, false, fm_path(FM) == 1>(sc, o, d, t);
        if (HITREC) {
            float* rec = hr + (size_t)k * (2 + h.nl) * hr_plane + hr_pix;
            rec[0] = __int_as_float(id);
            rec[hr_plane] = t;
        }
        if (id < 0) {
            miss_add<fm_lean(FM)>(sc, d, T, c);
            break;
        }
        if (k == kq && queue_push(nq, pix, o, o_lo, d, T, c, id, t)) return;
    }
    if (HITREC) {
        for (int kk = k + 1; kk <= fr.D; ++kk)
            hr[(size_t)kk * (2 + h.nl) * hr_plane + hr_pix] = __int_as_float(-1);
    }
    store_one(fr, pix, c, out, pitch);
}

// ---------------------------------------------------------------- wide queue passes
// When a queue pass holds few paths it is bound by the latency of one warp shading
// one hit (a lane traces the hit's 19 shadow segments against every sphere, in
// groups), not by work.  In wide mode a warp takes ONE path: lane j sets up and
// tests segment j of the hit (the filtered loop with one segment per lane), the
// visible counts per light come from warp votes, and the next ray's closest hit is
// split by blocks of spheres across the lanes and reduced to the lowest (t, index).
// Every per-segment and per-sphere value is computed by the same operations as in
// the one-lane path, and the shading sums run over the lights in the same order,
// so the results are bit-identical; only the latency changes.

// Closest hit with the spheres split across the warp (all 32 lanes call): lane j
// tests blocks j, j + 32, ...; the lexicographic minimum of (t, index) over the
// lanes equals the strict-< scan in index order.  Then the plane, as closest_hit.
__device__ __forceinline__ int closest_hit_wide(const StagedScene& sc, f3 o, f3 d, float& t_out) {
    const int lane = threadIdx.x & 31;
    float tb = __int_as_float(0x7f800000);
    int best = -1;
    const int n = sc.hdr->ns_pad;
    const RayCross rp = ray_cross(o, d);
#pragma unroll 1
    for (int i0 = lane * kPad; i0 < n; i0 += 32 * kPad) closest_block<true>(sc.geo + i0, i0, rp, tb, best);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float t2 = __shfl_xor_sync(0xffffffffu, tb, off);
        const int b2 = __shfl_xor_sync(0xffffffffu, best, off);
        if (b2 >= 0 && (best < 0 || t2 < tb || (t2 == tb && b2 < best))) {
            tb = t2;
            best = b2;
        }
    }
    const SceneHdr& h = *sc.hdr;
    if (h.has_plane) {
        const f3 pn = xyz(h.plane_g);
        const float den = dot(d, pn);
        if (den != 0.0f) {
            const float t = __fdiv_rn(-(dot(o, pn) + h.plane_g.w), den);
            if (t > 0.0f && t < tb) {
                tb = t;
                best = h.ns;
            }
        }
    }
    t_out = tb;
    return best;
}

// shade_hit_staged with the hit's segments spread over the warp (all 32 lanes call
// with the same hit; the result is the same in every lane).
template <bool HITREC, bool LEAN = false>
__device__ __forceinline__ HitShade shade_hit_wide(const StagedScene& sc, const Frame& fr, uint32_t pix, int k,
                                                   f3 p, f3 p_lo, f3 n, f3 po, f3 d, float ks, float e,
                                                   float* __restrict__ hr, size_t hr_k, size_t hr_plane) {
    const SceneHdr& h = *sc.hdr;
    const int lane = threadIdx.x & 31;
    HitShade out{fr.ka, 0.0f};
    uint32_t lit = 0;
    int total = 0;
#pragma unroll 1
    for (int li = 0; li < h.nl; ++li) {
        const f3 lh = normalize(sub(sub(xyz(h.light_p[li]), p), p_lo));
        if (dot(n, lh) > 0.0f) {
            lit |= 1u << li;
            total += rays_of_light(fr, h.light_s[li]);
        }
        if (HITREC && lane == 0) hr[hr_k + (size_t)(2 + li) * hr_plane] = 0.0f;
    }
    int cnt[RT_MAX_LIGHTS];
#pragma unroll
    for (int li = 0; li < RT_MAX_LIGHTS; ++li) cnt[li] = 0;
    float* seg = s_seg + (threadIdx.x + blockDim.x * threadIdx.y);
    const bool plane = h.has_plane != 0;
    const f3 pn = xyz(h.plane_g);
    const float num = -(dot(po, pn) + h.plane_g.w);
#pragma unroll 1
    for (int c0 = 0; c0 < total; c0 += 32) {
        // segment c0 + lane: its light l and sample s, in the one-lane path's order
        int rem = c0 + lane, l = -1;
        const bool valid = rem < total;
        if (valid) {
            uint32_t rest = lit;
            while (true) {
                l = __ffs(rest) - 1;
                const int nr = rays_of_light(fr, h.light_s[l]);
                if (rem < nr) break;
                rem -= nr;
                rest &= rest - 1u;
            }
        }
        f3 W = mk3(0.f, 0.f, 0.f), nv = mk3(0.f, 0.f, 0.f), vn = mk3(0.f, 0.f, 0.f);
        bool occj = true, ok = true;
        if (valid) {
            const int s = rem;
            const float4 Lp = h.light_p[l];
            const float4 Ls = h.light_s[l];
            const int nr = rays_of_light(fr, Ls);
            // sample s of an area light uses the words of Philox call s / 2
            uint4 w = make_uint4(0, 0, 0, 0);
            if (Ls.x > 0.0f && (s & 1))
                w = philox10(make_uint4(pix, (uint32_t)k, (uint32_t)l, (uint32_t)(s >> 1)), fr.key0, fr.key1);
            const LightFrame lf = !LEAN && Ls.y > 0.0f ? light_frame(p, Lp) : LightFrame{};
            const f3 X = nr > 1 || Ls.x > 0.0f || Ls.y > 0.0f
                             ? sample_point<LEAN>(fr, pix, k, l, s, Lp, Ls, w, lf, sc.flower)
                             : xyz(Lp);
            const f3 V = sub(sub(X, p), p_lo);
            W = scl(V, rcp_approx(dot(V, V)));
            nv = scl(V, -1.0f);
            const float den = -dot(nv, pn);
            occj = plane && den != 0.0f && num != 0.0f && ((num > 0.0f) == (den > 0.0f)) && fabsf(num) < fabsf(den);
            if (!occj) {
                const float S = dot(nv, nv);
                ok = S >= 0x1p-60f && S <= 0x1p100f;
                vn = scl(nv, -rsqrtf(S));
            }
        }
        seg[6 * kSegStride] = vn.x;
        seg[7 * kSegStride] = vn.y;
        seg[8 * kSegStride] = vn.z;
        seg[0] = W.x;
        seg[kSegStride] = W.y;
        seg[2 * kSegStride] = W.z;
        seg[3 * kSegStride] = nv.x;
        seg[4 * kSegStride] = nv.y;
        seg[5 * kSegStride] = nv.z;
        const bool exact_only = !__all_sync(0xffffffffu, ok);
        const uint32_t blocked = occluded_filtered<1, false>(sc.geo, h.ns_pad, 0xffffffffu, po, occj ? 1u : 0u, seg,
                                                      exact_only, nullptr, 0u, false);
        const bool vis = valid && !(blocked & 1u);
#pragma unroll
        for (int li = 0; li < RT_MAX_LIGHTS; ++li)
            if ((lit >> li) & 1u) cnt[li] += __popc(__ballot_sync(0xffffffffu, vis && l == li));
    }
    // the shading sums in light order, as the one-lane attribution
#pragma unroll
    for (int li = 0; li < RT_MAX_LIGHTS; ++li) {
        if ((lit >> li) & 1u) {
            const float4 Lp = h.light_p[li];
            const int nr = rays_of_light(fr, h.light_s[li]);
            const float vis = (float)cnt[li] / (float)nr;
            const f3 lh = normalize(sub(sub(xyz(Lp), p), p_lo));
            const float ndl = dot(n, lh);
            const float sp = light_spec(fr, n, d, lh, ndl, e);
            const float iv = Lp.w * vis;
            out.A = fmaf(iv, ndl, out.A);
            out.S = fmaf(iv * ks, sp, out.S);
            if (HITREC && lane == 0) hr[hr_k + (size_t)(2 + li) * hr_plane] = vis;
        }
    }
    return out;
}

// trace_queued in wide mode: the whole warp carries the path of entry e (all 32
// lanes call with the same entry) to its end -- the queues after a wide pass are
// shorter still, so re-queueing would only add passes (4K frame 9.60 -> 9.57 ms,
// 1080p 2.76 -> 2.73 ms); lane 0 stores the pixel and writes the record.
template <bool HITREC, bool LEAN = false>
__device__ __forceinline__ void trace_queued_wide(const StagedScene& sc, const Frame& fr,
                                                  const float4* __restrict__ e, int k, void* __restrict__ out,
                                                  size_t pitch, float* __restrict__ hr, size_t hr_plane) {
    const SceneHdr& h = *sc.hdr;
    const int lane = threadIdx.x & 31;
    const float4 e0 = e[0], e1 = e[1], e2 = e[2], e3 = e[3];
    f3 o = mk3(e0.x, e0.y, e0.z), o_lo = mk3(e1.x, e1.y, e1.z), d = mk3(e2.x, e2.y, e2.z);
    float T = e0.w, t = e2.w;
    float3 c = make_float3(e3.x, e3.y, e3.z);
    int id = __float_as_int(e3.w);
    const uint32_t pix = __float_as_uint(e1.w);
    const size_t hr_pix = pix;
#pragma unroll 1
    while (true) {
        const size_t hr_k = (size_t)k * (2 + h.nl) * hr_plane + hr_pix;
        const HitGeom hg = hit_geometry<false>(sc, id, o, o_lo, d, t, fr.refl_inv_max);
        f3 po_lo;
        const f3 po = offset_origin(hg, fr.eps, po_lo);
        const HitShade sh =
            shade_hit_wide<HITREC, LEAN>(sc, fr, pix, k, hg.p, hg.p_lo, hg.n, po, d, hg.m.w, hg.m2.x, hr, hr_k, hr_plane);
        step_tail(fr, k, hg.m, hg.m2, sh, hg.n, po, po_lo, o, o_lo, d, T, c);
        if (k == fr.D) {
            k = fr.D + 1;
            break;
        }
        ++k;
        id = closest_hit_wide(sc, o, d, t);
        if (HITREC && lane == 0) {
            float* rec = hr + (size_t)k * (2 + h.nl) * hr_plane + hr_pix;
            rec[0] = __int_as_float(id);
            rec[hr_plane] = t;
        }
        if (id < 0) {
            miss_add<LEAN>(sc, d, T, c);
            break;
        }
    }
    if (lane == 0) {
        if (HITREC) {
            for (int kk = k + 1; kk <= fr.D; ++kk)
                hr[(size_t)kk * (2 + h.nl) * hr_plane + hr_pix] = __int_as_float(-1);
        }
        store_one(fr, pix, c, out, pitch);
    }
}

}  // namespace rtd
