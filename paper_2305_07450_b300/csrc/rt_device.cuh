// rt_device.cuh -- device-side arithmetic of the per-pixel Whitted ray tracer of
// arXiv 2305.07450 (Section 3), FP32, for sm_103a.  Included by the one CUDA
// translation unit of the library (rt_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rt.h"

namespace rtd {

// ------------------------------------------------------------------ vectors
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 add(f3 a, f3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ f3 sub(f3 a, f3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ f3 scl(f3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ f3 fma3(f3 a, float s, f3 b) {  // a * s + b
    return mk3(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y), fmaf(a.z, s, b.z));
}
__device__ __forceinline__ float dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ f3 xyz(float4 v) { return mk3(v.x, v.y, v.z); }
// Unit vector by the hardware reciprocal square root (rsqrtf, within 2 ulp by CUDA's
// documented bound): every path -- one-pass, queued, batch, hierarchy, adjoint --
// forms ray and light directions through this one function, so they agree bit for
// bit; against the FP64 definition the 2 ulp are far inside the 1e-4 colour
// tolerance.  The correctly rounded root (__frsqrt_rn) cost the 4K frame 2.5 %.
__device__ __forceinline__ f3 normalize(f3 a, float* len_out = nullptr) {
    float l2 = dot(a, a);
    float inv = rsqrtf(l2);
    if (len_out) *len_out = __fsqrt_rn(l2);
    return scl(a, inv);
}

// Square root for the culling passes' bounds: x * rsqrtf(x), within 3 ulp (every
// bound it enters carries at least 2^-18 of relative slack); 0 for x = 0; NaN for
// NaN and +inf, which the callers' range checks take as "no bound".
__device__ __forceinline__ float sqrt_bound(float x) { return x == 0.0f ? 0.0f : x * rsqrtf(x); }

// Approximate reciprocal (rcp.approx.f32: within 1 ulp, subnormals kept), for the
// segment parameter's W = V / |V|^2: u = clamp(oc.W, 0, 1) only picks the point of
// the segment where the distance to the centre is evaluated, and every bound on the
// segment test (the line filter's, the cones') holds for any u in [0, 1].
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (sm_100 family): one instruction performs two FP32 operations,
// each rounded exactly as its scalar counterpart, so a pair of sphere tests costs
// one issue slot per step instead of two.
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a * b + c rounded once, then clamped to [0, 1] (NaN to 0): the parameter of the
// point of a segment closest to a centre.
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Error-free sum (Knuth's TwoSum): s + err == a + b exactly.  Used only per hit, to
// carry ray origins as unevaluated hi + lo pairs: positions of tens of units lose
// ~1e-6 to FP32 rounding, which a small sphere turns into ~1e-6 rad of normal.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
__device__ __forceinline__ f3 two_sum3(f3 a, f3 b, f3& err) {
    return mk3(two_sum(a.x, b.x, err.x), two_sum(a.y, b.y, err.y), two_sum(a.z, b.z, err.z));
}

// ------------------------------------------------------------------ scene
// Device scene blob: header, then the padded sphere tables.  The header and the
// geometry table are staged into shared memory by every CTA; materials are read
// through the read-only cache only at hits.
constexpr int kPad = 8;  // sphere tables are padded to a multiple of this

struct __align__(16) SceneHdr {
    int ns;          // spheres
    int ns_pad;      // padded count (multiple of kPad); pad entries never hit
    int has_plane;
    int nl;          // lights
    float4 plane_g;  // nx, ny, nz, d
    float4 plane_m;  // albedo r, g, b, k_s
    float4 plane_m2; // spec_exp, reflectivity, 0, 0
    float4 light_p[RT_MAX_LIGHTS];  // x, y, z, intensity
    float4 light_s[RT_MAX_LIGHTS];  // area_side, sphere_radius, 0, 0
};
static_assert(sizeof(SceneHdr) % 16 == 0, "header must keep 16-byte alignment");

// geo: spheres in pairs (2q, 2q + 1), two float4 per pair, so that one packed
// instruction tests both:  geo[2q] = (cx0, cx1, cy0, cy1), geo[2q + 1] = (cz0, cz1,
// -r0^2, -r1^2).  Pad entries: centre 0, -r^2 = +1 (never hit, never block).
// mat[i]  = (albedo r, g, b, k_s)
// mat2[i] = (spec_exp, reflectivity, r, 1/r)
// Sky panorama of the misses (Section 3.8): h rows of w RGBA texels from the top
// row, or tex == nullptr (black).
struct SkyView {
    const float4* tex;
    int w, h;
};

struct SceneView {
    const SceneHdr* hdr;
    const float4* geo;
    const float4* mat;
    const float4* mat2;
    SkyView sky;
};

__host__ __device__ inline size_t scene_geo_offset() { return sizeof(SceneHdr); }

// Sphere i of the paired geometry table as (cx, cy, cz, -r^2).
__host__ __device__ inline float4 sphere_at(const float4* geo, int i) {
    const float4 a = geo[i & ~1], b = geo[(i & ~1) + 1];
    return (i & 1) ? make_float4(a.y, a.w, b.y, b.w) : make_float4(a.x, a.z, b.x, b.z);
}
#ifdef __CUDACC__
__device__ __forceinline__ float4 sphere_ldg(const float4* geo, int i) {
    const float4 a = __ldg(geo + (i & ~1)), b = __ldg(geo + (i & ~1) + 1);
    return (i & 1) ? make_float4(a.y, a.w, b.y, b.w) : make_float4(a.x, a.z, b.x, b.z);
}
#endif
// Write sphere i (cx, cy, cz, -r^2) into the paired table.
__host__ __device__ inline void sphere_put(float4* geo, int i, float4 s) {
    float4& a = geo[i & ~1];
    float4& b = geo[(i & ~1) + 1];
    if (i & 1) {
        a.y = s.x; a.w = s.y; b.y = s.z; b.w = s.w;
    } else {
        a.x = s.x; a.z = s.y; b.x = s.z; b.z = s.w;
    }
}
__host__ __device__ inline size_t scene_bytes(int ns_pad) { return sizeof(SceneHdr) + (size_t)ns_pad * 48; }
__host__ __device__ inline int pad_spheres(int ns) { return (ns + kPad - 1) / kPad * kPad; }

// Per-frame constants computed on the host (in double, rounded once to float).
struct Frame {
    int W, H, D, nsamp, model, fmt;
    float ka, eps;
    int m;                   // min(W, H): the side the NDC square spans (Section 3.2)
    int rx0, ry0, rx1, ry1;  // rendered region [rx0, rx1) x [ry0, ry1) of the frame
    float3 cam;              // ray origin
    float3 right, up, fwd;   // rotated camera basis; fwd already scaled by b
    uint32_t key0, key1;     // Philox key = seed
    float sample_g_inv;      // 1 / g for the g x g stratified grid
    int sample_g;
    uint32_t sample_g_magic; // ceil(2^22 / g): s div g = umulhi(s * 2^10, it) for s < 2^10, g <= 32
    float refl_inv_max;      // > 0: reflection ratio = min(spec_exp * refl_inv_max, 1)
};

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds;
// each multiplies two counter words by the round constants, xors the high halves
// into the other two words with the round key, and permutes; the key advances by
// the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
// 24 high bits as a float in [0, 1): exact.
__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// ------------------------------------------------------------------ specular power
// x^e for x in (0, 1]: exact repeated squaring for small integer exponents (the
// usual 32), exp2(e log2 x) otherwise.
__device__ __forceinline__ float spec_pow(float x, float e) {
    const int ei = (int)e;
    if ((float)ei == e && ei >= 0 && ei <= 256) {
        float r = 1.0f, b = x;
        int k = ei;
#pragma unroll 1
        while (k) {
            if (k & 1) r *= b;
            b *= b;
            k >>= 1;
        }
        return r;
    }
    return exp2f(e * __log2f(x));
}

}  // namespace rtd
