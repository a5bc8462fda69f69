"""Pins of the oracle's R*-tree agglomeration (Section 4.1, Algorithms 1, 2):
the tree's structural invariants, small cases with a unique answer, and the
properties the multigrid hierarchy needs (a nested partition of the mesh)."""
import numpy as np
import pytest

from oracle import rtree
from paper_2602_16312_gb300 import workloads as W


def _walk(node, depth, out):
    out.append((node, depth))
    if node.level > 0:
        for e in node.entries:
            _walk(e[1], depth + 1, out)


def _check_tree(tree, boxes):
    nodes = []
    _walk(tree.root, 0, nodes)
    seen = []
    for node, depth in nodes:
        # every leaf at the same depth: the root's height
        if node.level == 0:
            assert depth == tree.root.level
            seen.extend(e[1] for e in node.entries)
            for e in node.entries:
                assert e[0][0] == list(boxes[e[1]][0]) and e[0][1] == list(boxes[e[1]][1])
        else:
            for e in node.entries:
                child = e[1]
                assert child.parent is node and child.level == node.level - 1
                lo = [min(f[0][0][k] for f in child.entries) for k in range(tree.dim)]
                hi = [max(f[0][1][k] for f in child.entries) for k in range(tree.dim)]
                assert e[0][0] == lo and e[0][1] == hi
        n = len(node.entries)
        if node is tree.root:
            assert n >= (2 if node.level > 0 else 1) and n <= tree.M
        else:
            assert tree.m <= n <= tree.M
    assert sorted(seen) == list(range(len(boxes)))


MESHES = {
    "jsquare2d_20": lambda: W.jittered_square_2d(n=20, n_levels=2),
    "jcube3d_6": lambda: W.jittered_cube_3d(n=6, degree=1, n_levels=2, group=2),
    "shell_q1": lambda: W.ventricle_shell(16, 8, 4, degree=1, n_levels=2),
}


@pytest.mark.parametrize("M", [4, 7, 12])
@pytest.mark.parametrize("name", list(MESHES))
def test_tree_invariants_and_nested_partition(name, M):
    wl = MESHES[name]()
    boxes = rtree.element_boxes(wl.mesh.vertices.tolist(), wl.mesh.elements.tolist())
    tree = rtree.build(wl.mesh.vertices, wl.mesh.elements, M)
    _check_tree(tree, boxes)
    lv = tree.levels()
    maps = rtree.agglomeration_maps(tree, wl.mesh.n_elements, len(lv))
    sizes = [wl.mesh.n_elements] + [len(x) for x in lv]
    for k, mp in enumerate(maps):
        assert len(mp) == sizes[k]
        assert np.array_equal(np.unique(mp), np.arange(sizes[k + 1]))      # onto the next level
    # Algorithm 2: the elements below a node are those the composed maps send to it
    comp = maps[0].copy()
    for k in range(1, len(maps)):
        for i, node in enumerate(lv[k - 1]):
            assert sorted(rtree.extract_leaves(node)) == sorted(np.flatnonzero(comp == i).tolist())
        comp = maps[k][comp]
    assert np.all(comp == 0)                                                # the root holds everything


def test_small_cases():
    # up to M elements: one leaf, the root
    boxes = [([float(i), 0.0], [i + 1.0, 1.0]) for i in range(5)]
    tree = rtree.RStarTree(2, 5)
    for i, b in enumerate(boxes):
        tree.insert_element(b, i)
    assert tree.root.level == 0 and [e[1] for e in tree.root.entries] == list(range(5))
    # two clusters far apart: the first split separates them
    pts = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (50.0, 50.0), (51.0, 50.0)]
    tree = rtree.RStarTree(2, 4)
    for i, (x, y) in enumerate(pts):
        tree.insert_element(([x, y], [x + 0.5, y + 0.5]), i)
    assert tree.root.level == 1
    groups = sorted(sorted(e[1] for e in child.entries) for _, child in tree.root.entries)
    assert groups == [[0, 1, 2], [3, 4]]


def test_leaves_are_compact_on_a_uniform_grid():
    """On a uniform grid the R* heuristics (least enlargement, least
    overlap, least-margin splits) make most leaf agglomerates exact
    rectangles: bounding-box area over element area is 1 for most leaves and
    close to 1 on average."""
    wl = W.square_2d_fhn(32, 1)
    tree = rtree.build(wl.mesh.vertices, wl.mesh.elements, 8)
    h = 1.0 / 32
    ratio = []
    for node in tree.levels()[0]:
        lo = [min(e[0][0][k] for e in node.entries) for k in range(2)]
        hi = [max(e[0][1][k] for e in node.entries) for k in range(2)]
        ratio.append((hi[0] - lo[0]) * (hi[1] - lo[1]) / (len(node.entries) * h * h))
    ratio = np.array(ratio)
    assert np.mean(np.abs(ratio - 1.0) < 1e-9) >= 0.85 and ratio.mean() <= 1.15
