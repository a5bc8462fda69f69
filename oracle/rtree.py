"""R*-tree agglomeration (Section 4.1, Algorithms 1 and 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The elements' bounding boxes are inserted one by one, in element order, into
an R*-tree of order (m, M) (the insertion algorithm of Beckmann et al. 1990,
which the paper adopts); the nodes of tree level l then agglomerate the
elements below them (Algorithm 2 descends from a node to its leaves), and
successive levels give nested agglomerates, i.e. the maps of a multigrid
hierarchy: level 0 = elements, level k >= 1 = tree nodes of height k - 1.

Determinism (readings where the published algorithm leaves a choice):
  m = max(2, floor(0.4 M)), p = max(1, floor(0.3 M)) entries reinserted;
  ChooseSubtree at a node whose children are leaves: least overlap
    enlargement, then least area enlargement, then least area, then the
    first entry; elsewhere least area enlargement, then least area, then
    the first entry;
  overflow: one forced reinsert per tree level and inserted element (not at
    the root), else a split; reinsert: entries sorted by decreasing squared
    distance of their centre from the node's centre (ties: entry order), the
    first p removed and inserted again closest first;
  split: per axis the entries sorted by (lower, upper, entry order) and by
    (upper, lower, entry order); the axis with the least sum of margins
    over all distributions (first axis on ties); on it the distribution
    with the least overlap, then the least area sum, lower-value sort
    before upper-value sort and fewer entries in the first group first;
  numbering: nodes of each level in depth-first order from the root,
    entries in their stored order.
Every quantity is computed with scalar float64 operations in a fixed order
(area: product of extents over the axes; margin: their sum; overlap:
product of the clipped extents).
"""


def _area(lo, hi):
    a = 1.0
    for k in range(len(lo)):
        a *= hi[k] - lo[k]
    return a


def _margin(lo, hi):
    s = 0.0
    for k in range(len(lo)):
        s += hi[k] - lo[k]
    return s


def _union(a, b):
    return ([min(x, y) for x, y in zip(a[0], b[0])], [max(x, y) for x, y in zip(a[1], b[1])])


def _overlap(a, b):
    v = 1.0
    for k in range(len(a[0])):
        e = min(a[1][k], b[1][k]) - max(a[0][k], b[0][k])
        if e <= 0.0:
            return 0.0
        v *= e
    return v


def _mbr(boxes):
    lo = list(boxes[0][0])
    hi = list(boxes[0][1])
    for b in boxes[1:]:
        for k in range(len(lo)):
            lo[k] = min(lo[k], b[0][k])
            hi[k] = max(hi[k], b[1][k])
    return (lo, hi)


class _Node:
    __slots__ = ("level", "entries", "parent")

    def __init__(self, level):
        self.level = level
        self.entries = []        # [box, child]: child is an element id (level 0) or a _Node
        self.parent = None


class RStarTree:
    def __init__(self, dim, M):
        self.dim = dim
        self.M = M
        self.m = max(2, (2 * M) // 5)
        self.p = max(1, (3 * M) // 10)
        self.root = _Node(0)

    # ------------------------------------------------------------ helpers
    def _box(self, node):
        return _mbr([e[0] for e in node.entries])

    def _adjust_up(self, node):
        while node.parent is not None:
            par = node.parent
            for e in par.entries:
                if e[1] is node:
                    e[0] = self._box(node)
                    break
            node = par

    # ------------------------------------------------------------ insertion
    def insert_element(self, box, eid):
        self._reinserted = set()
        self._insert([box, eid], 0)

    def _choose_subtree(self, box, level):
        node = self.root
        while node.level > level:
            best, best_key = None, None
            if node.level == 1:
                for i, e in enumerate(node.entries):
                    u = _union(e[0], box)
                    ov = 0.0
                    for j, f in enumerate(node.entries):
                        if j != i:
                            ov += _overlap(u, f[0]) - _overlap(e[0], f[0])
                    a = _area(*e[0])
                    key = (ov, _area(*u) - a, a)
                    if best_key is None or key < best_key:
                        best, best_key = e, key
            else:
                for e in node.entries:
                    a = _area(*e[0])
                    key = (_area(*_union(e[0], box)) - a, a)
                    if best_key is None or key < best_key:
                        best, best_key = e, key
            node = best[1]
        return node

    def _insert(self, entry, level):
        node = self._choose_subtree(entry[0], level)
        node.entries.append(entry)
        if level > 0:
            entry[1].parent = node
        if len(node.entries) > self.M:
            self._overflow(node)
        else:
            self._adjust_up(node)

    def _overflow(self, node):
        if node is not self.root and node.level not in self._reinserted:
            self._reinserted.add(node.level)
            self._reinsert(node)
        else:
            self._split(node)

    def _reinsert(self, node):
        lo, hi = self._box(node)
        c = [0.5 * (lo[k] + hi[k]) for k in range(self.dim)]

        def dist(e):
            d = 0.0
            for k in range(self.dim):
                t = 0.5 * (e[0][0][k] + e[0][1][k]) - c[k]
                d += t * t
            return d
        order = sorted(range(len(node.entries)), key=lambda i: (-dist(node.entries[i]), i))
        removed = [node.entries[i] for i in order[:self.p]]
        keep = sorted(order[self.p:])
        node.entries = [node.entries[i] for i in keep]
        self._adjust_up(node)
        for e in reversed(removed):          # closest of the removed first
            self._insert(e, node.level)

    def _distributions(self, entries, axis):
        lo_sort = sorted(range(len(entries)), key=lambda i: (entries[i][0][0][axis], entries[i][0][1][axis], i))
        hi_sort = sorted(range(len(entries)), key=lambda i: (entries[i][0][1][axis], entries[i][0][0][axis], i))
        out = []
        for srt in (lo_sort, hi_sort):
            for k in range(1, self.M - 2 * self.m + 3):
                n1 = self.m - 1 + k
                out.append((srt[:n1], srt[n1:]))
        return out

    def _split(self, node):
        entries = node.entries
        best_axis, best_s = 0, None
        for axis in range(self.dim):
            s = 0.0
            for g1, g2 in self._distributions(entries, axis):
                b1 = _mbr([entries[i][0] for i in g1])
                b2 = _mbr([entries[i][0] for i in g2])
                s += _margin(*b1) + _margin(*b2)
            if best_s is None or s < best_s:
                best_axis, best_s = axis, s
        best, best_key = None, None
        for g1, g2 in self._distributions(entries, best_axis):
            b1 = _mbr([entries[i][0] for i in g1])
            b2 = _mbr([entries[i][0] for i in g2])
            key = (_overlap(b1, b2), _area(*b1) + _area(*b2))
            if best_key is None or key < best_key:
                best, best_key = (g1, g2), key
        g1, g2 = best
        sib = _Node(node.level)
        node.entries = [entries[i] for i in g1]
        sib.entries = [entries[i] for i in g2]
        if node.level > 0:
            for e in sib.entries:
                e[1].parent = sib
        if node is self.root:
            root = _Node(node.level + 1)
            root.entries = [[self._box(node), node], [self._box(sib), sib]]
            node.parent = sib.parent = root
            self.root = root
            return
        par = node.parent
        for e in par.entries:
            if e[1] is node:
                e[0] = self._box(node)
                break
        par.entries.append([self._box(sib), sib])
        sib.parent = par
        if len(par.entries) > self.M:
            self._overflow(par)
        else:
            self._adjust_up(par)

    # ------------------------------------------------------------ Algorithms 1 and 2
    def levels(self):
        """Nodes of each height (0 = leaf nodes) in depth-first order."""
        out = [[] for _ in range(self.root.level + 1)]

        def visit(node):
            out[node.level].append(node)
            if node.level > 0:
                for e in node.entries:
                    visit(e[1])
        visit(self.root)
        return out


def element_boxes(vertices, elements):
    """Axis-aligned bounding box of each element's corner vertices."""
    boxes = []
    for cell in elements:
        pts = [vertices[v] for v in cell]
        lo = [min(p[k] for p in pts) for k in range(len(pts[0]))]
        hi = [max(p[k] for p in pts) for k in range(len(pts[0]))]
        boxes.append((lo, hi))
    return boxes


def build(vertices, elements, M):
    import numpy as np
    vertices = np.asarray(vertices, dtype=float).tolist()
    tree = RStarTree(len(vertices[0]), M)
    for e, b in enumerate(element_boxes(vertices, np.asarray(elements).tolist())):
        tree.insert_element(b, e)
    return tree


def agglomeration_maps(tree, n_elements, n_maps):
    """Maps of the multigrid hierarchy from the tree (Algorithm 1 applied at
    every height; Algorithm 2 is the descent from a node to its elements):
    map 0: element -> its leaf node; map k: node of height k-1 -> its parent."""
    import numpy as np
    lv = tree.levels()
    if n_maps > len(lv):
        raise ValueError("the tree has only %d levels" % len(lv))
    ids = [{id(nd): i for i, nd in enumerate(level)} for level in lv]
    maps = []
    m0 = np.full(n_elements, -1, dtype=np.int32)
    for i, nd in enumerate(lv[0]):
        for e in nd.entries:
            m0[e[1]] = i
    maps.append(m0)
    for k in range(1, n_maps):
        mk = np.full(len(lv[k - 1]), -1, dtype=np.int32)
        for i, nd in enumerate(lv[k]):
            for e in nd.entries:
                mk[ids[k - 1][id(e[1])]] = i
        maps.append(mk)
    return maps


def extract_leaves(node):
    """Algorithm 2: the elements below `node` (depth-first)."""
    if node.level == 0:
        return [e[1] for e in node.entries]
    out = []
    for e in node.entries:
        out.extend(extract_leaves(e[1]))
    return out
