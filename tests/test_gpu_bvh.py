"""The binary hierarchy rt_load_scene builds, read back with rt_get_bvh:
a tree over every hierarchy leaf with the root first and children after
their parents, node boxes that contain their children's boxes, and a
surface-area cost that puts the PLOC clustering below the Karras radix tree
(the reason PLOC is the default)."""
import numpy as np
import pytest

from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _structure(nodes):
    ref = nodes[:, 12:14].copy().view(np.int32)
    m = nodes.shape[0]
    seen_int = np.zeros(m, np.int32)
    leaves = []
    for k in range(m):
        for c in ref[k]:
            if c >= 0:
                assert k < c < m, (k, c)
                seen_int[c] += 1
            else:
                leaves.append(~c)
    assert seen_int[0] == 0 and np.all(seen_int[1:] == 1)
    leaves = np.sort(np.array(leaves))
    assert np.array_equal(leaves, np.arange(m + 1))   # m internal nodes over m + 1 leaves
    return ref


def _node_boxes(nodes):
    b0, b1 = nodes[:, 0:6].astype(np.float64), nodes[:, 6:12].astype(np.float64)
    lo = np.minimum(b0[:, :3], b1[:, :3])
    hi = np.maximum(b0[:, 3:], b1[:, 3:])
    return lo, hi


def _area_cost(nodes):
    lo, hi = _node_boxes(nodes)
    d = hi - lo
    a = d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0]
    return float(a.sum() / a[0])


@pytest.mark.parametrize("builder", [rt.BVH_PLOC, rt.BVH_KARRAS])
def test_tree_structure_and_boxes(builder):
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    tr = rt.Tracer(0, 3.5e9)
    tr.set_bvh_builder(builder)
    tr.load_scene(sc)
    nodes = rt.rt_get_bvh(tr.ctx)
    assert nodes.shape[0] >= 1
    ref = _structure(nodes)
    lo, hi = _node_boxes(nodes)
    # the box stored for an internal child in its parent contains the child's own children
    for k in range(nodes.shape[0]):
        for s, c in enumerate(ref[k]):
            if c >= 0:
                stored = nodes[k, 6 * s:6 * s + 6].astype(np.float64)
                assert np.all(stored[:3] <= lo[c] + 1e-6) and np.all(stored[3:] >= hi[c] - 1e-6)
    tr.close()


def test_ploc_area_cost_below_karras():
    sc = S.city_scene(20)
    costs = {}
    for builder in (rt.BVH_PLOC, rt.BVH_KARRAS):
        tr = rt.Tracer(0, 3.5e9)
        tr.set_bvh_builder(builder)
        tr.load_scene(sc)
        nodes = rt.rt_get_bvh(tr.ctx)
        _structure(nodes)
        costs[builder] = _area_cost(nodes)
        tr.close()
    print("area cost PLOC / Karras:", costs[rt.BVH_PLOC], costs[rt.BVH_KARRAS])
    assert costs[rt.BVH_PLOC] < 0.8 * costs[rt.BVH_KARRAS]


def test_get_bvh_small_scenes():
    tr = rt.Tracer(0, 3.5e9)
    # one triangle in the hierarchy: a single node whose children are both that leaf
    tiny = S.tiny_scene()
    tr.load_scene(tiny)
    n = rt.rt_get_bvh(tr.ctx).shape[0]
    assert n >= 1
    tr.close()
