"""The sphere hierarchy's host builder (rt_bvh_build_host, no GPU): every sphere in
exactly one leaf, every box holding what lies under it (the spheres' exact
extents from the FP32 centre and r^2 the kernels read), the depth bound the
device stack relies on, determinism, and the degenerate inputs."""
import numpy as np
import pytest

from oracle_pins import light, mk, sphere
from paper_2305_07450_b300 import rt, scenes as S

DEPTH_BOUND = 44  # the device traversal stack holds 48 entries
LEAF_MAX = 8


def leaf_of(ref):
    v = -1 - int(ref)
    return v >> 4, (v & 15) + 1


def sphere_boxes(scene):
    sph = scene.spheres.astype(np.float64)
    r2 = (sph[:, 3] * sph[:, 3]).astype(np.float32).astype(np.float64)  # as packed for the device
    r = np.sqrt(r2)
    return sph[:, :3] - r[:, None], sph[:, :3] + r[:, None]


def check_hierarchy(scene):
    nodes, prim, info = rt.bvh_build_host(scene)
    n = scene.n_spheres
    if n == 0:
        assert info["n_nodes"] == 0 and len(prim) == 0
        return info
    assert 1 <= info["n_nodes"] <= max(n - 1, 1)
    assert info["depth"] <= DEPTH_BOUND and 1 <= info["max_leaf"] <= LEAF_MAX
    lo, hi = sphere_boxes(scene)
    seen = np.zeros(n, np.int64)

    def contains(blo, bhi, qlo, qhi):
        return np.all(blo.astype(np.float64) <= qlo) and np.all(bhi.astype(np.float64) >= qhi)

    def walk(ref, blo, bhi, depth):
        """Check the subtree under child box [blo, bhi]; returns its max depth."""
        if ref < 0:
            first, cnt = leaf_of(ref)
            assert cnt <= LEAF_MAX and first + cnt <= n
            for i in prim[first:first + cnt]:
                seen[i] += 1
                assert contains(blo, bhi, lo[i], hi[i]), (i, blo, bhi, lo[i], hi[i])
            return depth
        assert 0 < ref < len(nodes)
        nd = nodes[ref]
        for k in ("a", "b"):
            assert contains(blo, bhi, nd[k + "_lo"].astype(np.float64), nd[k + "_hi"].astype(np.float64))
        return max(walk(int(nd["ref"][0]), nd["a_lo"], nd["a_hi"], depth + 1),
                   walk(int(nd["ref"][1]), nd["b_lo"], nd["b_hi"], depth + 1))

    root = nodes[0]
    if n == 1:
        first, cnt = leaf_of(root["ref"][0])
        assert (first, cnt) == (0, 1) and np.all(root["b_lo"] > root["b_hi"])  # empty second child
        assert contains(root["a_lo"], root["a_hi"], lo[0], hi[0])
        return info
    deepest = max(walk(int(root["ref"][0]), root["a_lo"], root["a_hi"], 1),
                  walk(int(root["ref"][1]), root["b_lo"], root["b_hi"], 1))
    assert np.all(seen == 1), "every sphere in exactly one leaf"
    assert sorted(prim.tolist()) == list(range(n))
    assert deepest == info["depth"]
    # r_scene bounds every centre coordinate plus radius
    sph = scene.spheres.astype(np.float64)
    assert info["r_scene"] >= np.max(np.max(np.abs(sph[:, :3]), 1) + np.sqrt((sph[:, 3] ** 2).astype(np.float32)))
    return info


@pytest.mark.parametrize("name", ["whitted_256", "whitted_720p", "area_4k", "paper_scene"])
def test_workload_hierarchies(name):
    w = getattr(S, name)()
    info = check_hierarchy(w.scene)
    print(name, info)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 9, 100])
def test_small_counts(n):
    sc = S.random_scene(5, n, 1, 1.0)
    check_hierarchy(sc)


def test_large_random_scene():
    sc = S.random_scene(77, 20000, 2, 35.0)
    info = check_hierarchy(sc)
    assert info["depth"] <= DEPTH_BOUND


def test_coincident_centres_split_by_median():
    """300 concentric spheres: no split separates their centroids, so the builder
    falls back to object-median splits; depth stays logarithmic."""
    sph = [sphere((1.0, 2.0, 3.0), 0.1 + 0.01 * i) for i in range(300)]
    sc, _, _ = mk(spheres=sph, lights=[light((0, 50, 0))])
    info = check_hierarchy(sc)
    assert info["depth"] <= 8


def test_duplicate_spheres_and_a_line():
    sph = [sphere((0.0, 1.0, 0.0), 0.5)] * 20 + [sphere((0.25 * i, 1.0, 0.0), 0.2) for i in range(200)]
    sc, _, _ = mk(spheres=sph, lights=[light((0, 50, 0))])
    check_hierarchy(sc)


def test_deterministic():
    w = S.area_4k()
    a = rt.bvh_build_host(w.scene)
    b = rt.bvh_build_host(w.scene)
    assert a[0].tobytes() == b[0].tobytes() and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_refuses_huge_coordinates_and_bad_records():
    sc, _, _ = mk(spheres=[sphere((2e15, 0, 0), 1.0)], lights=[light((0, 50, 0))])
    with pytest.raises(rt.RtError) as e:
        rt.bvh_build_host(sc)
    assert e.value.status == 4  # RT_ERR_UNSUPPORTED
    bad, _, _ = mk(spheres=[sphere((0, 0, 0), -1.0)], lights=[light((0, 50, 0))])
    with pytest.raises(rt.RtError) as e:
        rt.bvh_build_host(bad)
    assert e.value.status == 1  # RT_ERR_INVALID_ARG
