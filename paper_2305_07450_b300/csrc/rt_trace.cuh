// rt_trace.cuh -- per-pixel path of the Whitted ray tracer (arXiv 2305.07450,
// Section 3) in FP32: primary ray, brute-force closest hit, shading with hard or
// sampled shadows, register-resident reflection loop.  Shared by the per-frame
// kernel, the batched persistent kernel and the adjoint's recompute mode.
#pragma once

#include "rt_device.cuh"

namespace rtd {

// Staged scene as one CTA sees it: header and geometry in shared memory,
// materials in global memory (read at hits only).
struct StagedScene {
    const SceneHdr* hdr;   // shared
    const float4* geo;     // shared, hdr->ns_pad entries
    const float4* mat;     // global
    const float4* mat2;    // global
};

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
    return normalize_rn(d);
}

// ---------------------------------------------------------------- Section 3.4.1
// Closest of all primitives by brute force; spheres 0..N-1 then the plane N; a
// strictly smaller distance wins, so ties keep the lower index.  Sphere test in the
// well-conditioned form: with oc = c - o and tca = oc.d, the squared distance of
// the centre from the ray's line is |oc - tca d|^2, so disc = r^2 - |oc - tca d|^2
// avoids the cancellation of tca^2 - |oc|^2 for distant spheres.  Roots tca -+
// sqrt(disc); the near one if it is > 0, else the far one.
__device__ __forceinline__ int closest_hit(const StagedScene& sc, f3 o, f3 d, float& t_out) {
    float tb = __int_as_float(0x7f800000);  // +inf
    int best = -1;
    const float4* __restrict__ geo = sc.geo;
    const int n = sc.hdr->ns_pad;
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
        const float4 g = geo[i];
        const float ocx = g.x - o.x, ocy = g.y - o.y, ocz = g.z - o.z;
        const float tca = fmaf(ocx, d.x, fmaf(ocy, d.y, ocz * d.z));
        const float lx = fmaf(-tca, d.x, ocx), ly = fmaf(-tca, d.y, ocy), lz = fmaf(-tca, d.z, ocz);
        const float disc = fmaf(-lx, lx, fmaf(-ly, ly, fmaf(-lz, lz, g.w)));
        if (disc >= 0.0f) {
            const float s = __fsqrt_rn(disc);
            float t = tca - s;
            if (t <= 0.0f) t = tca + s;
            if (t > 0.0f && t < tb) {
                tb = t;
                best = i;
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
// Any-hit of the shadow segment from o along unit dir for length dist.  For a
// sphere the segment is blocked iff its closest point to the centre is inside the
// ball: tc = clamp(oc.dir, 0, dist), |oc - tc dir|^2 < r^2.  With every light
// outside every sphere (checked at upload) this is the same predicate as "a root
// of the ray-sphere quadratic lies in (0, dist)".  The loop runs in blocks of
// kPad spheres and leaves once every active lane of the warp is blocked (the
// method's early break, Section 3.6 cast-shadows listing, taken warp-wide).
__device__ __forceinline__ bool occluded(const StagedScene& sc, f3 o, f3 dir, float dist) {
    const float4* __restrict__ geo = sc.geo;
    const int n = sc.hdr->ns_pad;
    bool occ = false;
    const unsigned mask = __activemask();
#pragma unroll 1
    for (int i0 = 0; i0 < n; i0 += kPad) {
#pragma unroll
        for (int j = 0; j < kPad; ++j) {
            const float4 g = geo[i0 + j];
            const float ocx = g.x - o.x, ocy = g.y - o.y, ocz = g.z - o.z;
            const float tca = fmaf(ocx, dir.x, fmaf(ocy, dir.y, ocz * dir.z));
            const float tc = fminf(fmaxf(tca, 0.0f), dist);
            const float qx = fmaf(-tc, dir.x, ocx), qy = fmaf(-tc, dir.y, ocy), qz = fmaf(-tc, dir.z, ocz);
            const float e = fmaf(qx, qx, fmaf(qy, qy, fmaf(qz, qz, -g.w)));
            occ |= (e < 0.0f);
        }
        if (__all_sync(mask, occ)) break;
    }
    const SceneHdr& h = *sc.hdr;
    if (!occ && h.has_plane) {
        const f3 n = xyz(h.plane_g);
        const float den = dot(dir, n);
        const float num = -(dot(o, n) + h.plane_g.w);
        // t = num / den in (0, dist)  <=>  same signs and |num| < dist |den|
        if (den != 0.0f && ((num > 0.0f) == (den > 0.0f)) && num != 0.0f &&
            fabsf(num) < dist * fabsf(den))
            occ = true;
    }
    return occ;
}

// ---------------------------------------------------------------- Section 3.6.1
// Visible fraction of a sampled light seen from p (shadow rays leave from po).
// Square area light of side a: n = g*g strata, sample s in stratum
// (s mod g, s div g) at ((i + xi1)/g - 1/2, (j + xi2)/g - 1/2) * a in x and z,
// xi from Philox call s div 2 with counter (pixel, bounce, light, call), words
// 2(s mod 2), 2(s mod 2) + 1.  Spherical light of radius R: sunflower points on the
// great circle facing p, radius R sqrt(i/n) at angle i * phi, phi = pi (3 - sqrt 5)
// (the angle is reduced exactly as 2 pi frac(i (3 - sqrt 5) / 2) in 32-bit fixed
// point).
__device__ __forceinline__ float sampled_visibility(const StagedScene& sc, const Frame& fr, uint32_t pix,
                                                    int k, int l, f3 p, f3 po, float4 Lp, float4 Ls) {
    int unblocked = 0;
    const int n = fr.nsamp;
    if (Ls.x > 0.0f) {
        const int g = fr.sample_g;
        const float ginv = fr.sample_g_inv;
        const float a = Ls.x;
        uint4 w = make_uint4(0, 0, 0, 0);
#pragma unroll 1
        for (int s = 0; s < n; ++s) {
            if ((s & 1) == 0) w = philox10(make_uint4(pix, (uint32_t)k, (uint32_t)l, (uint32_t)(s >> 1)), fr.key0, fr.key1);
            const float xi1 = u24((s & 1) ? w.z : w.x);
            const float xi2 = u24((s & 1) ? w.w : w.y);
            const int i = s % g, j = s / g;
            const f3 X = mk3(Lp.x + (((float)i + xi1) * ginv - 0.5f) * a, Lp.y,
                             Lp.z + (((float)j + xi2) * ginv - 0.5f) * a);
            float dist;
            const f3 dir = normalize_rn(sub(X, p), &dist);
            unblocked += occluded(sc, po, dir, dist) ? 0 : 1;
        }
    } else {
        const float R = Ls.y;
        f3 w = normalize_rn(sub(p, xyz(Lp)));
        const f3 up = fabsf(w.y) < 0.999f ? mk3(0.f, 1.f, 0.f) : mk3(1.f, 0.f, 0.f);
        const f3 u = normalize_rn(mk3(w.y * up.z - w.z * up.y, w.z * up.x - w.x * up.z, w.x * up.y - w.y * up.x));
        const f3 v = mk3(u.y * w.z - u.z * w.y, u.z * w.x - u.x * w.z, u.x * w.y - u.y * w.x);
        const float inv_n = 1.0f / (float)n;
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            const float r = R * sqrtf((float)i * inv_n);
            const uint32_t frac = (uint32_t)i * 0x61C88647u;  // 2^32 (3 - sqrt 5) / 2
            float sn, cs;
            sincospif((float)(frac >> 8) * (1.0f / 8388608.0f), &sn, &cs);  // 2 frac
            const f3 X = add(xyz(Lp), add(scl(u, r * cs), scl(v, r * sn)));
            float dist;
            const f3 dir = normalize_rn(sub(X, p), &dist);
            unblocked += occluded(sc, po, dir, dist) ? 0 : 1;
        }
    }
    return (float)unblocked / (float)n;
}

// ---------------------------------------------------------------- Sections 3.5-3.7
// Trace one pixel.  shade(c) = c A + S with
//   A = k_a + sum_l I_l vis_l max(n.l, 0),  S = sum_l I_l vis_l k_s spec_l,
// a light skipped when n.l <= 0; Phong spec = max(v.r, 0)^exp (r the light
// direction mirrored about n, v = -d), Blinn spec = max(n.h, 0)^exp.  The
// reflection recursion of Section 3.7.1 is unrolled forward with a scalar
// throughput: k < D adds T((1 - rho) A c + S) and sets T *= rho A; k = D adds
// T(A c + S); a miss ends the path.  HITREC: write (id, t, vis_l) per bounce.
template <bool HITREC>
__device__ __forceinline__ float3 trace_pixel(const StagedScene& sc, const Frame& fr, int x, int y,
                                              float* __restrict__ hr, size_t hr_plane) {
    const SceneHdr& h = *sc.hdr;
    const uint32_t pix = (uint32_t)y * (uint32_t)fr.W + (uint32_t)x;
    const size_t hr_pix = (size_t)y * (size_t)fr.W + (size_t)x;
    f3 o = mk3(fr.cam.x, fr.cam.y, fr.cam.z);
    f3 d = primary_dir(fr, x, y);
    float T = 1.0f;
    float3 out = make_float3(0.f, 0.f, 0.f);
    int k = 0;
#pragma unroll 1
    for (; k <= fr.D; ++k) {
        float t;
        const int id = closest_hit(sc, o, d, t);
        if (HITREC) {
            float* rec = hr + (size_t)k * (2 + h.nl) * hr_plane + hr_pix;
            rec[0] = __int_as_float(id);
            rec[hr_plane] = t;
        }
        if (id < 0) break;
        // hit point and face-forwarded normal
        f3 p, n;
        float4 m, m2;
        if (id < h.ns) {
            const float4 g = sc.geo[id];
            m = __ldg(sc.mat + id);
            m2 = __ldg(sc.mat2 + id);
            const f3 oc = sub(xyz(g), o);
            const float tca = dot(oc, d);
            const f3 l = fma3(d, -tca, oc);
            const f3 pc = fma3(d, t - tca, scl(l, -1.0f));  // p - c = (t - tca) d - l
            p = add(xyz(g), pc);
            n = scl(pc, m2.w);
        } else {
            m = h.plane_m;
            m2 = h.plane_m2;
            p = fma3(d, t, o);
            n = xyz(h.plane_g);
        }
        if (dot(n, d) > 0.0f) n = scl(n, -1.0f);
        const f3 po = fma3(n, fr.eps, p);
        // shading with shadows
        float A = fr.ka, S = 0.0f;
#pragma unroll 1
        for (int li = 0; li < h.nl; ++li) {
            const float4 Lp = h.light_p[li];
            const float4 Ls = h.light_s[li];
            float dist;
            const f3 lh = normalize_rn(sub(xyz(Lp), p), &dist);
            const float ndl = dot(n, lh);
            float vis = 0.0f;
            if (ndl > 0.0f) {
                if (Ls.x > 0.0f || Ls.y > 0.0f)
                    vis = sampled_visibility(sc, fr, pix, k, li, p, po, Lp, Ls);
                else
                    vis = occluded(sc, po, lh, dist) ? 0.0f : 1.0f;
                float sp;
                if (fr.model == RT_PHONG) {
                    const f3 r = sub(scl(n, 2.0f * ndl), lh);
                    const float vr = -dot(d, r);
                    sp = vr > 0.0f ? spec_pow(vr, m2.x) : 0.0f;
                } else {
                    const f3 hv = normalize_rn(sub(lh, d));
                    const float nh = dot(n, hv);
                    sp = nh > 0.0f ? spec_pow(nh, m2.x) : 0.0f;
                }
                const float iv = Lp.w * vis;
                A = fmaf(iv, ndl, A);
                S = fmaf(iv * m.w, sp, S);
            }
            if (HITREC) hr[((size_t)k * (2 + h.nl) + 2 + li) * hr_plane + hr_pix] = vis;
        }
        if (k < fr.D) {
            const float w = T * (1.0f - m2.y) * A;
            out.x = fmaf(w, m.x, fmaf(T, S, out.x));
            out.y = fmaf(w, m.y, fmaf(T, S, out.y));
            out.z = fmaf(w, m.z, fmaf(T, S, out.z));
            T *= m2.y * A;
            d = normalize_rn(fma3(n, -2.0f * dot(d, n), d));
            o = po;
        } else {
            const float w = T * A;
            out.x = fmaf(w, m.x, fmaf(T, S, out.x));
            out.y = fmaf(w, m.y, fmaf(T, S, out.y));
            out.z = fmaf(w, m.z, fmaf(T, S, out.z));
        }
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

}  // namespace rtd
