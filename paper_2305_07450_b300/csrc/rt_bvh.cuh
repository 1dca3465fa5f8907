// rt_bvh.cuh -- bounding-volume hierarchy over the spheres: the spatial
// acceleration structure the paper leaves to future work (Section 6).  It changes
// the work, not the result: each sphere is tested with the same FP32 operations as
// the brute-force loop, ties keep the lower index, shadow segments OR the same
// per-sphere predicate, and no box that could hold an accepted sphere is culled --
// so images are bit for bit those of the brute-force kernels.
//
// Why nothing is culled.  Boxes hold their spheres' exact extents (rounded outward
// on the host).  A sphere the FP32 test accepts at parameter t has its point o + t d
// within r + 31u M of the centre (u = 2^-24, M = |o|_inf + R, R the largest
// |c|_inf + r of the scene: each component of c x d - o x d is off by at most 7u M,
// so the line passes within r + 17u M of the centre, and tca = c.d - o.d with the
// root's rounding moves t by at most 14u M along d), and the FP32 slab parameters
// are within 5u M / |d_axis| of the exact ones (d the ray direction, or the vector
// V of a shadow segment o + u V, u in [0, 1]; the segment test's point is within
// r + 26u M).  Every box is therefore widened, per ray, by delta = 2^-16 M = 256u M
// per side, seven times what the two bounds need; the box then starts before t
// and ends after it, in FP32 too.
#pragma once

#include "rt_device.cuh"
#include "rt_errword.cuh"

namespace rtd {

constexpr int kBvhStack = 48;        // traversal stack; the builder keeps depth <= 44
constexpr int kBvhLeafMax = 8;       // spheres per leaf
constexpr uint32_t kErrBvhStack = 4u;  // device error word: stack overflow or a walk past its bound

// Node (64 bytes) = the two children's boxes and references.  ref >= 0: interior
// node index; ref < 0: leaf, v = -1 - ref, spheres prim[v >> 4 .. (v >> 4) + (v & 15)].
// An empty child has an inverted box (never entered).
struct __align__(16) BvhNode {
    float4 q0;  // a.lo.x, a.lo.y, a.lo.z, a.hi.x
    float4 q1;  // a.hi.y, a.hi.z, b.lo.x, b.lo.y
    float4 q2;  // b.lo.z, b.hi.x, b.hi.y, b.hi.z
    int4 q3;    // ref a, ref b, 0, 0
};
static_assert(sizeof(BvhNode) == 64, "node size");

__host__ __device__ inline int32_t bvh_leaf_ref(int first, int count) { return -1 - ((first << 4) | (count - 1)); }

struct BvhView {
    const BvhNode* nodes;
    const int32_t* prim;
    int n_nodes;
    float r_scene;  // max over spheres of |c|_inf + r, rounded up
};

__host__ __device__ inline size_t bvh_bytes(int n_nodes, int ns) {
    return (size_t)n_nodes * sizeof(BvhNode) + ((size_t)ns * 4 + 15) / 16 * 16;
}

// ---------------------------------------------------------------- per sphere
// The brute-force block tests of Sections 3.4.1 and 3.6 for one sphere g = (c, -r^2),
// element for element the operations of the packed pair tests, in the same order
// (closest root from m = |c x d - o x d|^2 - r^2 and tca = c.d - o.d; blocked
// segment o + u V, u = clamp(oc.W, 0, 1), -V = nv).
struct RayX {  // -(o x d) and -(o.d) of a ray, formed once per ray
    f3 nw;
    float nod;
};
__device__ __forceinline__ RayX ray_x(f3 o, f3 d) {
    RayX x;
    x.nw = mk3(fmaf(o.z, d.y, -(o.y * d.z)), fmaf(o.x, d.z, -(o.z * d.x)), fmaf(o.y, d.x, -(o.x * d.y)));
    x.nod = -dot(o, d);
    return x;
}

__device__ __forceinline__ bool sphere_root_t(float4 g, const RayX& x, f3 d, float& t) {
    const float px = fmaf(g.y, d.z, fmaf(g.z, -d.y, x.nw.x));
    const float py = fmaf(g.z, d.x, fmaf(g.x, -d.z, x.nw.y));
    const float pz = fmaf(g.x, d.y, fmaf(g.y, -d.x, x.nw.z));
    const float m = fmaf(px, px, fmaf(py, py, fmaf(pz, pz, g.w)));
    if (!(m < 0.0f)) return false;
    const float tc = fmaf(g.x, d.x, fmaf(g.y, d.y, fmaf(g.z, d.z, x.nod)));
    const float s = __fsqrt_rn(-m);
    t = tc - s;
    if (t <= 0.0f) t = tc + s;
    return t > 0.0f;
}

__device__ __forceinline__ bool segment_blocked(float4 g, f3 o, f3 w, f3 nv) {
    const float ocx = g.x + (-o.x), ocy = g.y + (-o.y), ocz = g.z + (-o.z);
    const float u = fma_sat(ocx, w.x, fmaf(ocy, w.y, ocz * w.z));
    const float qx = fmaf(u, nv.x, ocx), qy = fmaf(u, nv.y, ocy), qz = fmaf(u, nv.z, ocz);
    const float e = fmaf(qx, qx, fmaf(qy, qy, fmaf(qz, qz, g.w)));
    return e < 0.0f;
}

// ---------------------------------------------------------------- slab test
// Per ray: 1/d (components below 1e-20 in magnitude taken as +-1e-20; the host
// keeps coordinates below 1e15, so no product overflows), and the offsets of the
// near and far planes of the widened box: t = plane * inv + (-o inv -+ delta |inv|).
struct RayInv {
    f3 inv, on, of;
};

__device__ __forceinline__ RayInv ray_inv(f3 o, f3 d, float r_scene) {
    const float tiny = 1e-20f;
    RayInv q;
    q.inv = mk3(1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    const float delta = (fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fabsf(o.z)) + r_scene) * (1.0f / 65536.0f);
    const float px = delta * fabsf(q.inv.x), py = delta * fabsf(q.inv.y), pz = delta * fabsf(q.inv.z);
    q.on = mk3(fmaf(-o.x, q.inv.x, -px), fmaf(-o.y, q.inv.y, -py), fmaf(-o.z, q.inv.z, -pz));
    q.of = mk3(fmaf(-o.x, q.inv.x, px), fmaf(-o.y, q.inv.y, py), fmaf(-o.z, q.inv.z, pz));
    return q;
}

// Widened box [l, h] against the ray on [0, tmax]: entry distance in tn.
__device__ __forceinline__ bool box_hit(const RayInv& q, float lx, float ly, float lz, float hx, float hy, float hz,
                                        float tmax, float& tn) {
    const bool px = q.inv.x >= 0.0f, py = q.inv.y >= 0.0f, pz = q.inv.z >= 0.0f;
    const float nx = fmaf(px ? lx : hx, q.inv.x, q.on.x), fx = fmaf(px ? hx : lx, q.inv.x, q.of.x);
    const float ny = fmaf(py ? ly : hy, q.inv.y, q.on.y), fy = fmaf(py ? hy : ly, q.inv.y, q.of.y);
    const float nz = fmaf(pz ? lz : hz, q.inv.z, q.on.z), fz = fmaf(pz ? hz : lz, q.inv.z, q.of.z);
    tn = fmaxf(fmaxf(nx, ny), fmaxf(nz, 0.0f));
    const float tf = fminf(fminf(fx, fy), fminf(fz, tmax));
    return tn <= tf;
}

__device__ __forceinline__ void node_boxes(const BvhNode& nd, const RayInv& q, float tmax, bool& ha, float& ta,
                                           bool& hb, float& tb) {
    ha = box_hit(q, nd.q0.x, nd.q0.y, nd.q0.z, nd.q0.w, nd.q1.x, nd.q1.y, tmax, ta);
    hb = box_hit(q, nd.q1.z, nd.q1.w, nd.q2.x, nd.q2.y, nd.q2.z, nd.q2.w, tmax, tb);
}

__device__ __forceinline__ BvhNode load_node(const BvhNode* nodes, int i) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    BvhNode nd;
    nd.q0 = p[0];
    nd.q1 = p[1];
    nd.q2 = p[2];
    nd.q3 = reinterpret_cast<const int4*>(p)[3];
    return nd;
}

// ---------------------------------------------------------------- traversals
// Both walks are out-of-line functions: inlined into every shading site they made
// the kernel's code large enough that instruction fetch dominated its stalls
// (4K frame 23.1 ms inlined, 9.6 ms called, on B300).
// Closest sphere hit: updates (tb, best) with (t < tb) || (t == tb && i < best),
// the brute-force order's result in any visiting order.  Nearer child first; the
// farther one is pushed with its entry distance and skipped when that exceeds the
// best hit found meanwhile.
__device__ __noinline__ void closest_bvh(const float4* __restrict__ geo, const BvhView& bv, f3 o, f3 d, float& tb,
                                            int& best) {
    if (bv.n_nodes <= 0) return;
    const RayInv q = ray_inv(o, d, bv.r_scene);
    const RayX rx = ray_x(o, d);
    int stack[kBvhStack];
    float stack_t[kBvhStack];
    int sp = 0;
    int ref = 0;
    // a tree of n nodes has 2n + 1 references: a walk never takes more steps
    const int max_steps = 2 * bv.n_nodes + 1;
#pragma unroll 1
    for (int step = 0;; ++step) {
        if (step > max_steps) {
            atomicOr(&g_err_word, kErrBvhStack);
            break;
        }
        if (ref >= 0) {
            const BvhNode nd = load_node(bv.nodes, ref);
            bool ha, hb;
            float ta, tbb;
            node_boxes(nd, q, tb, ha, ta, hb, tbb);
            if (ha && hb) {
                const bool a_first = ta <= tbb;
                ref = a_first ? nd.q3.x : nd.q3.y;
                if (sp < kBvhStack) {
                    stack[sp] = a_first ? nd.q3.y : nd.q3.x;
                    stack_t[sp] = a_first ? tbb : ta;
                    ++sp;
                } else {
                    atomicOr(&g_err_word, kErrBvhStack);
                }
                continue;
            }
            if (ha || hb) {
                ref = ha ? nd.q3.x : nd.q3.y;
                continue;
            }
        } else {
            const int v = -1 - ref;
            const int first = v >> 4, cnt = (v & 15) + 1;
#pragma unroll 1
            for (int k = 0; k < cnt; ++k) {
                const int i = bv.prim[first + k];
                float t;
                if (sphere_root_t(sphere_at(geo, i), rx, d, t) && (t < tb || (t == tb && i < best))) {
                    tb = t;
                    best = i;
                }
            }
        }
        // pop the next subtree that can still hold a hit no farther than tb
        bool found = false;
#pragma unroll 1
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= tb) {
                ref = stack[sp];
                found = true;
                break;
            }
        }
        if (!found) break;
    }
}

// Any sphere blocking the segment o + u V, u in [0, 1] (-V = nv, W = V / |V|^2):
// the OR of the brute-force predicate over the spheres of the entered leaves (boxes
// taken along V on [0, 1]); the first blocker ends the walk.
__device__ __noinline__ bool occluded_bvh(const float4* __restrict__ geo, const BvhView& bv, f3 o, f3 w, f3 nv) {
    if (bv.n_nodes <= 0) return false;
    const float dist = 1.0f;
    const RayInv q = ray_inv(o, scl(nv, -1.0f), bv.r_scene);
    int stack[kBvhStack];
    int sp = 0;
    int ref = 0;
    const int max_steps = 2 * bv.n_nodes + 1;
#pragma unroll 1
    for (int step = 0;; ++step) {
        if (step > max_steps) {
            atomicOr(&g_err_word, kErrBvhStack);
            break;
        }
        if (ref >= 0) {
            const BvhNode nd = load_node(bv.nodes, ref);
            bool ha, hb;
            float ta, tbb;
            node_boxes(nd, q, dist, ha, ta, hb, tbb);
            if (ha && hb) {
                ref = nd.q3.x;
                if (sp < kBvhStack) stack[sp++] = nd.q3.y;
                else atomicOr(&g_err_word, kErrBvhStack);
                continue;
            }
            if (ha || hb) {
                ref = ha ? nd.q3.x : nd.q3.y;
                continue;
            }
        } else {
            const int v = -1 - ref;
            const int first = v >> 4, cnt = (v & 15) + 1;
#pragma unroll 1
            for (int k = 0; k < cnt; ++k)
                if (segment_blocked(sphere_at(geo, bv.prim[first + k]), o, w, nv)) return true;
        }
        if (sp == 0) break;
        ref = stack[--sp];
    }
    return false;
}

}  // namespace rtd
