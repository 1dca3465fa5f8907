// rt_bwd.cuh -- adjoint of the per-pixel render (reverse mode), for inverse
// rendering.  Not in the paper: it differentiates the forward path of Sections
// 3.2-3.7 with visibility held fixed (no silhouette or shadow-edge terms).
//
// Forward recurrence of one pixel (k = 0..K-1 hits, D the bounce limit):
//   R_k = beta_k A_k c_k + S_k + [k < D] rho_k A_k R_{k+1},  beta_k = 1 - rho_k (k < D), 1 (k = D)
//   A_k = k_a + sum_l I_l vis_kl max(n_k.l_kl, 0),  S_k = sum_l I_l vis_kl k_s spec_kl
//   pixel = R_0, R_K = 0 when the path ends in a miss.
// With the loss gradient g = dL/dpixel, the adjoint of R_k is T_k g,
// T_0 = 1, T_{k+1} = T_k rho_k A_k.  The kernel replays the path forward (rays,
// throughputs), then walks it backward, carrying R_{k+1} and the adjoint of the
// ray that left hit k (origin p + eps n, direction reflect(d, n)), and pushes the
// adjoints through shading, the next ray and the hit point (p = o + t d with t
// fixed implicitly by |p - c| = r, or by the plane equation).
//
// Gradient layout (floats): sphere i at 8i + {albedo r, g, b, k_s, reflectivity,
// centre x, y, z}; the plane at 8N + {albedo r, g, b, k_s, reflectivity, 0, 0, 0};
// light l at 8(N + 1) + 4l + {position x, y, z, intensity}.  "Reflectivity" is the
// field that sets the reflection ratio: rho itself, or -- with the paper's coupling
// of Section 3.7, rho = min(e / MAX_REFLECTIVITY, 1) -- the specular exponent e,
// whose gradient then also carries its effect on the specular terms
// (d(x^e)/de = x^e ln x).
//
// Reduction (deterministic): within a warp, lanes that hit the same primitive are
// summed by a fixed butterfly and the group's first lane adds the sum to the
// warp's own table in shared memory; the CTA then sums its warps' tables in warp
// order into one partial per CTA, and a second kernel sums the partials in a fixed
// order (rt_grad_reduce_kernel).  No floating-point atomics, so the result is
// reproducible bit for bit.
#pragma once

#include "rt_errword.cuh"
#include "rt_stage.cuh"
#include "rt_trace.cuh"

namespace rtd {

constexpr int kMaxBounce = RT_MAX_DEPTH + 1;
constexpr int kRecStride = 2 + RT_MAX_LIGHTS;

__host__ __device__ inline int grad_count(int ns, int nl) { return 8 * (ns + 1) + 4 * nl; }

// Add v[0..7] of every lane to entry `key` (-1: nothing) of the warp's table.
__device__ __forceinline__ void warp_group_add(float* __restrict__ wtab, int key, const float (&v)[8]) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(full, key >= 0);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int gid = __shfl_sync(full, key, leader);
        const bool in = key == gid;
        float s[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            s[j] = in ? v[j] : 0.0f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s[j] += __shfl_xor_sync(full, s[j], off);
        }
        if (lane == leader) {
#pragma unroll
            for (int j = 0; j < 8; ++j) wtab[8 * gid + j] += s[j];
        }
        __syncwarp(full);
        todo &= ~__ballot_sync(full, in);
    }
}

template <bool FROM_HITREC, bool CH>
__global__ void __launch_bounds__(256) rt_bwd_kernel(const SceneView sv, const Frame fr,
                                                     const float* __restrict__ dl, size_t dl_pitch,
                                                     const float* __restrict__ hr, float* __restrict__ partials,
                                                     int G, int staging, int block_x, int block_y) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    const int lane = threadIdx.x, warp = threadIdx.y;
    if (staging == 1 && tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t ns_pad = (uint32_t)__ldg(&sv.hdr->ns_pad);
    const uint32_t stage_bytes = CH ? (uint32_t)sizeof(SceneHdr) : (uint32_t)(sizeof(SceneHdr) + 16u * ns_pad);
    if (!stage_to_smem(smem, sv.hdr, stage_bytes, staging, &bar, phase, &g_err_word)) return;
    const SceneHdr& h = *reinterpret_cast<const SceneHdr*>(smem);
    float4* tab = reinterpret_cast<float4*>(smem + sizeof(SceneHdr));
    const uint32_t table_bytes = CH ? (uint32_t)(blockDim.y * kChunk * 16) : 16u * ns_pad;
    const StagedScene sc{&h, CH ? nullptr : tab, sv.geo, CH ? tab + (size_t)threadIdx.y * kChunk : nullptr, sv.mat,
                         sv.mat2};
    float* wtabs = reinterpret_cast<float*>(smem + sizeof(SceneHdr) + table_bytes);
    float* wtab = wtabs + (size_t)warp * G;
    for (int e = lane; e < G; e += 32) wtab[e] = 0.0f;
    __syncwarp();

    const int wpr = block_x >> 3;
    const int x = blockIdx.x * block_x + (warp % wpr) * 8 + (lane & 7);
    const int y = blockIdx.y * block_y + (warp / wpr) * 4 + (lane >> 3);
    const bool valid = x < fr.W && y < fr.H;
    const int nl = h.nl;
    const size_t plane = (size_t)fr.W * (size_t)fr.H;

    // ---- the path: (id, t, vis_l) per bounce
    float rec[kMaxBounce * kRecStride];
    int K = 0;
    f3 g = mk3(0.f, 0.f, 0.f);
    if (valid) {
        const size_t pix = (size_t)y * fr.W + x;
        if (FROM_HITREC) {
            for (int k = 0; k <= fr.D; ++k) {
                const float* src = hr + (size_t)k * (2 + nl) * plane + pix;
                for (int f = 0; f < 2 + nl; ++f) rec[k * kRecStride + f] = __ldg(src + (size_t)f * plane);
            }
        } else {
            // recompute: the forward trace itself, recording into registers/local memory
            float loc[kMaxBounce * (2 + RT_MAX_LIGHTS)];
            trace_pixel<true, CH, false, 0>(sc, fr, x, y, loc, 1, 0);  // recompute: the segment test alone
            for (int k = 0; k <= fr.D; ++k)
                for (int f = 0; f < 2 + nl; ++f) rec[k * kRecStride + f] = loc[k * (2 + nl) + f];
        }
        for (int k = 0; k <= fr.D; ++k) {
            if (__float_as_int(rec[k * kRecStride]) < 0) break;
            K = k + 1;
        }
        const float4 gv = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(dl) + (size_t)y * dl_pitch +
                                                           (size_t)x * 16);
        g = mk3(gv.x, gv.y, gv.z);
    }

    // ---- forward replay: ray origin (hi + lo), direction and throughput per bounce
    f3 Oh[kMaxBounce], Ol[kMaxBounce], Dd[kMaxBounce];
    float Tt[kMaxBounce];
    {
        f3 o = mk3(fr.cam.x, fr.cam.y, fr.cam.z), o_lo = mk3(0.f, 0.f, 0.f);
        f3 d = valid ? primary_dir(fr, x, y) : mk3(0.f, 0.f, 1.f);
        float T = 1.0f;
        for (int k = 0; k < K; ++k) {
            Oh[k] = o;
            Ol[k] = o_lo;
            Dd[k] = d;
            Tt[k] = T;
            const int id = __float_as_int(rec[k * kRecStride]);
            const float t = rec[k * kRecStride + 1];
            const HitGeom hg = hit_geometry<CH>(sc, id, o, o_lo, d, t, fr.refl_inv_max);
            float A = fr.ka;
            for (int li = 0; li < nl; ++li) {
                const float4 Lp = h.light_p[li];
                const f3 lh = normalize(sub(sub(xyz(Lp), hg.p), hg.p_lo));
                const float ndl = dot(hg.n, lh);
                if (ndl > 0.0f) A = fmaf(Lp.w * rec[k * kRecStride + 2 + li], ndl, A);
            }
            if (k < fr.D) {
                T *= hg.m2.y * A;
                f3 po_lo;
                const f3 po = offset_origin(hg, fr.eps, po_lo);
                d = normalize(fma3(hg.n, -2.0f * dot(d, hg.n), d));
                o = po;
                o_lo = po_lo;
            }
        }
    }

    // ---- reverse walk
    float lg[RT_MAX_LIGHTS][4];
    for (int li = 0; li < RT_MAX_LIGHTS; ++li) lg[li][0] = lg[li][1] = lg[li][2] = lg[li][3] = 0.0f;
    f3 Rn = mk3(0.f, 0.f, 0.f);                     // R_{k+1}
    f3 Ob = mk3(0.f, 0.f, 0.f), Db = mk3(0.f, 0.f, 0.f);  // adjoint of ray k+1
    const int Kw = (int)__reduce_max_sync(0xffffffffu, (unsigned)K);
    const bool coupled = fr.refl_inv_max > 0.0f;
    for (int k = Kw - 1; k >= 0; --k) {
        float pg[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int pid = -1;
        if (k < K) {
            const int id = __float_as_int(rec[k * kRecStride]);
            const float t = rec[k * kRecStride + 1];
            const f3 d = Dd[k];
            const HitGeom hg = hit_geometry<CH>(sc, id, Oh[k], Ol[k], d, t, fr.refl_inv_max);
            const f3 n = hg.n;
            const f3 alb = mk3(hg.m.x, hg.m.y, hg.m.z);
            const float ks = hg.m.w, ex = hg.m2.x, rho = hg.m2.y;
            const bool last = (k == fr.D);
            const float beta = last ? 1.0f : 1.0f - rho;
            const f3 Rb = scl(g, Tt[k]);
            // the adjoints of A and S do not depend on A and S themselves
            const float Ab = dot(Rb, last ? scl(alb, beta) : add(scl(alb, beta), scl(Rn, rho)));
            const float Sb = Rb.x + Rb.y + Rb.z;
            f3 pb = mk3(0.f, 0.f, 0.f), nb = mk3(0.f, 0.f, 0.f), db = mk3(0.f, 0.f, 0.f);
            float exb = 0.0f;  // adjoint of the exponent through the specular terms (coupled mode)
            // lights, one pass: the forward sums A and S (light order, as the forward
            // pass forms them) and their adjoints
            float A = fr.ka, S = 0.0f;
            for (int li = 0; li < nl; ++li) {
                const float4 Lp = h.light_p[li];
                float dist;
                const f3 Lv = sub(sub(xyz(Lp), hg.p), hg.p_lo);
                const f3 lh = normalize(Lv, &dist);
                const float ndl = dot(n, lh);
                if (ndl <= 0.0f) continue;
                const float v = rec[k * kRecStride + 2 + li];
                const float sp = light_spec(fr, n, d, lh, ndl, ex);
                A = fmaf(Lp.w * v, ndl, A);
                S = fmaf(Lp.w * v * ks, sp, S);
                if (v == 0.0f) continue;
                const float I = Lp.w;
                lg[li][3] += Ab * v * ndl + Sb * v * ks * sp;
                pg[3] += Sb * I * v * sp;
                float ndlb = Ab * I * v;
                const float spb = Sb * I * v * ks;
                f3 lhb = mk3(0.f, 0.f, 0.f);
                if (fr.model == RT_PHONG) {
                    const f3 r = sub(scl(n, 2.0f * ndl), lh);
                    const float vr = -dot(d, r);
                    if (vr > 0.0f && sp > 0.0f) {
                        if (coupled) exb = fmaf(spb * sp, logf(vr), exb);
                        const float vrb = spb * ex * sp / vr;
                        db = fma3(r, -vrb, db);
                        const f3 rb = scl(d, -vrb);
                        ndlb += 2.0f * dot(rb, n);
                        nb = fma3(rb, 2.0f * ndl, nb);
                        lhb = sub(lhb, rb);
                    }
                } else {
                    float ulen;
                    const f3 hv = normalize(sub(lh, d), &ulen);
                    const float nh = dot(n, hv);
                    if (nh > 0.0f && sp > 0.0f) {
                        if (coupled) exb = fmaf(spb * sp, logf(nh), exb);
                        const float nhb = spb * ex * sp / nh;
                        nb = fma3(hv, nhb, nb);
                        const f3 hb = scl(n, nhb);
                        const f3 ub = scl(fma3(hv, -dot(hb, hv), hb), 1.0f / ulen);
                        lhb = add(lhb, ub);
                        db = sub(db, ub);
                    }
                }
                nb = fma3(lh, ndlb, nb);
                lhb = fma3(n, ndlb, lhb);
                const f3 Lvb = scl(fma3(lh, -dot(lhb, lh), lhb), 1.0f / dist);
                lg[li][0] += Lvb.x;
                lg[li][1] += Lvb.y;
                lg[li][2] += Lvb.z;
                pb = sub(pb, Lvb);
            }
            const f3 R = add(add(scl(alb, beta * A), mk3(S, S, S)), last ? mk3(0.f, 0.f, 0.f) : scl(Rn, rho * A));
            // colour terms
            pg[0] = beta * A * Rb.x;
            pg[1] = beta * A * Rb.y;
            pg[2] = beta * A * Rb.z;
            const float rhob = last ? 0.0f : dot(Rb, sub(scl(Rn, A), scl(alb, A)));
            // coupled: rho = min(e / MAX_REFLECTIVITY, 1) has slope 1 / MAX_REFLECTIVITY
            // below the cap and 0 at it
            pg[4] = coupled ? fmaf(ex * fr.refl_inv_max < 1.0f ? fr.refl_inv_max : 0.0f, rhob, exb) : rhob;
            // the ray that left this hit: origin p + eps n, direction d - 2 (d.n) n
            if (!last) {
                pb = add(pb, Ob);
                nb = fma3(Ob, fr.eps, nb);
                const float dn = dot(d, n), Dbn = dot(Db, n);
                db = add(db, fma3(n, -2.0f * Dbn, Db));
                nb = fma3(Db, -2.0f * dn, nb);
                nb = fma3(d, -2.0f * Dbn, nb);
            }
            // hit point p = o + t d, t fixed by the surface; normal n = flip (p - c) / r
            f3 ob, cb = mk3(0.f, 0.f, 0.f);
            if (id < h.ns) {
                const float ir = hg.m2.w;
                const f3 nraw = scl(n, hg.flip);
                pb = fma3(nb, hg.flip * ir, pb);
                cb = scl(nb, -hg.flip * ir);
                const float tb = dot(pb, d);
                const float nd = dot(nraw, d);
                ob = pb;
                db = fma3(pb, t, db);
                const float q = tb / nd;
                ob = fma3(nraw, -q, ob);
                db = fma3(nraw, -q * t, db);
                cb = fma3(nraw, q, cb);
            } else {
                const f3 N = xyz(h.plane_g);
                const float tb = dot(pb, d);
                const float dN = dot(d, N);
                ob = pb;
                db = fma3(pb, t, db);
                const float q = tb / dN;
                ob = fma3(N, -q, ob);
                db = fma3(N, -q * t, db);
            }
            pg[5] = cb.x;
            pg[6] = cb.y;
            pg[7] = cb.z;
            Ob = ob;
            Db = db;
            Rn = R;
            pid = id;
        }
        warp_group_add(wtab, pid, pg);
    }
    // lights: whole-warp sums, lane 0 adds them to the warp's table
    const int lbase = 8 * (h.ns + 1);
    for (int li = 0; li < nl; ++li) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float s = lg[li][c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) wtab[lbase + 4 * li + c] += s;
        }
    }
    __syncthreads();
    // CTA partial: the warps' tables summed in warp order
    const int nwarps = blockDim.y;
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int e = tid; e < G; e += nthreads) {
        float s = 0.0f;
        for (int w = 0; w < nwarps; ++w) s += wtabs[(size_t)w * G + e];
        partials[cta * G + e] = s;
    }
}

// grad[e] = sum over CTAs b of partials[b][e], in a fixed order: a block owns 32
// entries (one per lane) and its warp w sums the partials b = w, w + 32, w + 64, ...
// in increasing b (8 loads in flight per lane); the 32 warp sums are then added in
// warp order.  One thread per entry summing every partial in turn was bound by
// load latency (thousands of dependent steps).
constexpr int kReduceWarps = 32;
__global__ void __launch_bounds__(32 * kReduceWarps) rt_grad_reduce_kernel(const float* __restrict__ partials,
                                                                          int n_parts, int G,
                                                                          float* __restrict__ grad) {
    __shared__ float s[kReduceWarps][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (e < G) {
        int b = w;
        for (; b + 7 * kReduceWarps < n_parts; b += 8 * kReduceWarps) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __ldg(partials + (size_t)(b + j * kReduceWarps) * G + e);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += v[j];
        }
        for (; b < n_parts; b += kReduceWarps) acc += __ldg(partials + (size_t)b * G + e);
    }
    s[w][lane] = acc;
    __syncthreads();
    if (w == 0 && e < G) {
        float t = 0.0f;
        for (int j = 0; j < kReduceWarps; ++j) t += s[j][lane];
        grad[e] = t;
    }
}

}  // namespace rtd
