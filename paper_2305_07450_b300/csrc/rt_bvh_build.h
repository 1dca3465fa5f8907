// rt_bvh_build.h -- host builder of the sphere hierarchy traversed by rt_bvh.cuh.
// Binned surface-area-heuristic splits (16 bins per axis over the centroids);
// below depth 24, or when the centroids of a range do not separate, an object
// median split along the widest centroid axis, so depth stays <= 24 + 20 for up
// to 2^20 spheres (the traversal stack holds 48).  Boxes are the spheres' exact
// extents, from the same FP32 centre and r^2 the kernels read, computed in double
// and rounded outward.  Deterministic: no randomness, ties broken by index.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "rt_bvh.cuh"

namespace rtbvh {

struct Box {
    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL};
    double hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    void grow_pt(const double* p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    bool empty() const { return !(lo[0] <= hi[0]); }
    double area() const {
        if (empty()) return 0.0;
        const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct Prim {
    Box box;
    double c[3];
    int idx;
};

struct Result {
    std::vector<rtd::BvhNode> nodes;
    std::vector<int32_t> prim;
    int depth = 0;
    int max_leaf = 0;
    float r_scene = 0.f;
};

constexpr int kBins = 16;
constexpr int kSahDepth = 24;
constexpr double kCostNode = 1.0;    // visiting a node: two box tests
constexpr double kCostSphere = 1.0;  // one sphere test

inline float down(double v) {
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}
inline float up(double v) {
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

class Builder {
  public:
    Builder(std::vector<Prim>& p, Result& r) : P(p), R(r) {}

    // Reference for the range [b, e) at depth `depth` (a leaf or a new node).
    int32_t child(int b, int e, int depth) {
        const int n = e - b;
        R.depth = std::max(R.depth, depth);
        if (n <= 1 || (n <= rtd::kBvhLeafMax && leaf_cheaper(b, e))) return leaf(b, e);
        return node(b, e, depth);
    }

    // New interior node over [b, e) (n >= 2); returns its index.
    int32_t node(int b, int e, int depth) {
        const int id = (int)R.nodes.size();
        R.nodes.emplace_back();
        const int mid = split(b, e, depth);
        Box ba, bb;
        for (int i = b; i < mid; ++i) ba.grow(P[(size_t)i].box);
        for (int i = mid; i < e; ++i) bb.grow(P[(size_t)i].box);
        const int32_t ra = child(b, mid, depth + 1);
        const int32_t rb = child(mid, e, depth + 1);
        set(R.nodes[(size_t)id], ba, bb, ra, rb);
        return id;
    }

    static void set(rtd::BvhNode& nd, const Box& a, const Box& b, int32_t ra, int32_t rb) {
        float al[3], ah[3], bl[3], bh[3];
        for (int k = 0; k < 3; ++k) {
            al[k] = a.empty() ? 1e30f : down(a.lo[k]);
            ah[k] = a.empty() ? -1e30f : up(a.hi[k]);
            bl[k] = b.empty() ? 1e30f : down(b.lo[k]);
            bh[k] = b.empty() ? -1e30f : up(b.hi[k]);
        }
        nd.q0 = make_float4(al[0], al[1], al[2], ah[0]);
        nd.q1 = make_float4(ah[1], ah[2], bl[0], bl[1]);
        nd.q2 = make_float4(bl[2], bh[0], bh[1], bh[2]);
        nd.q3 = make_int4(ra, rb, 0, 0);
    }

    int32_t leaf(int b, int e) {
        const int first = (int)R.prim.size();
        for (int i = b; i < e; ++i) R.prim.push_back(P[(size_t)i].idx);
        R.max_leaf = std::max(R.max_leaf, e - b);
        return rtd::bvh_leaf_ref(first, e - b);
    }

  private:
    std::vector<Prim>& P;
    Result& R;

    Box bounds(int b, int e) const {
        Box bx;
        for (int i = b; i < e; ++i) bx.grow(P[(size_t)i].box);
        return bx;
    }

    bool leaf_cheaper(int b, int e) {
        double cost;
        int axis;
        int cut;
        if (!best_sah(b, e, cost, axis, cut)) return true;
        return (double)(e - b) * kCostSphere <= cost;
    }

    // Cheapest binned SAH split of [b, e): cost relative to the parent's area.
    bool best_sah(int b, int e, double& best_cost, int& best_axis, int& best_cut) const {
        Box cb;
        for (int i = b; i < e; ++i) cb.grow_pt(P[(size_t)i].c);
        const double pa = bounds(b, e).area();
        best_cost = HUGE_VAL;
        best_axis = -1;
        best_cut = -1;
        if (!(pa > 0.0)) return false;
        for (int k = 0; k < 3; ++k) {
            const double ext = cb.hi[k] - cb.lo[k];
            if (!(ext > 0.0)) continue;
            Box bin[kBins];
            int cnt[kBins] = {0};
            for (int i = b; i < e; ++i) {
                const int j = bin_of(P[(size_t)i].c[k], cb.lo[k], ext);
                bin[j].grow(P[(size_t)i].box);
                ++cnt[j];
            }
            double ra[kBins];
            int na[kBins];
            Box acc;
            int n = 0;
            for (int j = kBins - 1; j > 0; --j) {
                acc.grow(bin[j]);
                n += cnt[j];
                ra[j] = acc.area();
                na[j] = n;
            }
            acc = Box();
            n = 0;
            for (int j = 0; j < kBins - 1; ++j) {
                acc.grow(bin[j]);
                n += cnt[j];
                if (n == 0 || na[j + 1] == 0) continue;
                const double c = kCostNode + (acc.area() * n + ra[j + 1] * na[j + 1]) / pa * kCostSphere;
                if (c < best_cost) {
                    best_cost = c;
                    best_axis = k;
                    best_cut = j;
                }
            }
        }
        return best_axis >= 0;
    }

    static int bin_of(double c, double lo, double ext) {
        int j = (int)((c - lo) / ext * kBins);
        return std::min(std::max(j, 0), kBins - 1);
    }

    // Partition [b, e) and return the first index of the right part (b < mid < e).
    int split(int b, int e, int depth) {
        Box cb;
        for (int i = b; i < e; ++i) cb.grow_pt(P[(size_t)i].c);
        double cost;
        int axis, cut;
        if (depth < kSahDepth && best_sah(b, e, cost, axis, cut)) {
            const double lo = cb.lo[axis], ext = cb.hi[axis] - cb.lo[axis];
            auto it = std::stable_partition(P.begin() + b, P.begin() + e,
                                            [&](const Prim& p) { return bin_of(p.c[axis], lo, ext) <= cut; });
            const int mid = (int)(it - P.begin());
            if (mid > b && mid < e) return mid;
        }
        // object median along the widest centroid axis (ties by sphere index)
        int k = 0;
        for (int a = 1; a < 3; ++a)
            if (cb.hi[a] - cb.lo[a] > cb.hi[k] - cb.lo[k]) k = a;
        const int mid = b + (e - b) / 2;
        std::nth_element(P.begin() + b, P.begin() + mid, P.begin() + e, [k](const Prim& x, const Prim& y) {
            return x.c[k] < y.c[k] || (x.c[k] == y.c[k] && x.idx < y.idx);
        });
        return mid;
    }
};

// geo: the paired sphere table as the kernels hold it (sphere_at gives (cx, cy, cz, -r^2)).
inline void build(const float4* geo, int ns, Result* out) {
    out->nodes.clear();
    out->prim.clear();
    out->depth = 0;
    out->max_leaf = 0;
    out->r_scene = 0.f;
    if (ns <= 0) return;
    std::vector<Prim> P((size_t)ns);
    double rs = 0.0;
    for (int i = 0; i < ns; ++i) {
        const float4 g = rtd::sphere_at(geo, i);
        const double r = std::sqrt(-(double)g.w);
        Prim& p = P[(size_t)i];
        p.c[0] = g.x;
        p.c[1] = g.y;
        p.c[2] = g.z;
        for (int k = 0; k < 3; ++k) {
            p.box.lo[k] = p.c[k] - r;
            p.box.hi[k] = p.c[k] + r;
        }
        p.idx = i;
        rs = std::max(rs, std::max(std::max(std::fabs(p.c[0]), std::fabs(p.c[1])), std::fabs(p.c[2])) + r);
    }
    out->r_scene = up(rs * (1.0 + 1e-7));
    out->nodes.reserve((size_t)std::max(ns - 1, 1));
    out->prim.reserve((size_t)ns);
    Builder B(P, *out);
    if (ns == 1) {
        out->nodes.emplace_back();
        const int32_t ra = B.leaf(0, 1);
        Builder::set(out->nodes[0], P[0].box, Box(), ra, ra);
        out->depth = 1;
        return;
    }
    B.node(0, ns, 0);
}

}  // namespace rtbvh
