// R*-tree agglomeration (Section 4.1, Algorithms 1 and 2) on the host.
//
// The elements' bounding boxes go one by one, in element order, into an
// R*-tree of order (m, M) built with the insertion algorithm of Beckmann et
// al. (1990), the variant the paper adopts: choose-subtree by least overlap
// enlargement above the leaves and least area enlargement higher up, one
// forced reinsert per tree level and inserted element, and the margin /
// overlap split. The nodes of height h then agglomerate the elements below
// them (Algorithm 2 is the descent from a node to its leaves), and the
// heights 0, 1, ... give nested agglomerates: the maps of a multigrid
// hierarchy. Every choice the published algorithm leaves open is fixed:
//   m = max(2, floor(2M/5)), p = max(1, floor(3M/10)) entries reinserted;
//   ties: least area enlargement, then least area, then the first entry;
//   reinsert order: decreasing squared centre distance (ties: entry order),
//   the p farthest removed and inserted again closest first;
//   split sorts: (lower, upper, entry order) and (upper, lower, entry
//   order) per axis; the least margin sum picks the axis (first on ties),
//   the least overlap, then the least area sum, picks the distribution
//   (lower-value sort first, smaller first group first);
//   node numbering: depth-first from the root, entries in stored order.
// Areas, margins and overlaps are scalar float64 products and sums over the
// axes in increasing order.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/aggmg.h"
#include "setup.h"

namespace aggmg {
namespace {

struct Box {
  double lo[3], hi[3];
};

struct RTree {
  struct Entry {
    Box box;
    int64_t child;   // element id (height-0 node) or node index
  };
  struct Node {
    int height = 0;
    int64_t parent = -1;
    std::vector<Entry> entries;
  };

  int dim, M, m, p;
  std::vector<Node> nodes;
  int64_t root = 0;
  std::vector<char> reinserted;

  RTree(int d, int max_entries) : dim(d), M(max_entries) {
    m = std::max(2, (2 * M) / 5);
    p = std::max(1, (3 * M) / 10);
    nodes.emplace_back();
  }

  double area(const Box& b) const {
    double a = 1.0;
    for (int k = 0; k < dim; ++k) a *= b.hi[k] - b.lo[k];
    return a;
  }
  double margin(const Box& b) const {
    double s = 0.0;
    for (int k = 0; k < dim; ++k) s += b.hi[k] - b.lo[k];
    return s;
  }
  Box join(const Box& a, const Box& b) const {
    Box u;
    for (int k = 0; k < dim; ++k) {
      u.lo[k] = std::min(a.lo[k], b.lo[k]);
      u.hi[k] = std::max(a.hi[k], b.hi[k]);
    }
    return u;
  }
  double overlap(const Box& a, const Box& b) const {
    double v = 1.0;
    for (int k = 0; k < dim; ++k) {
      const double e = std::min(a.hi[k], b.hi[k]) - std::max(a.lo[k], b.lo[k]);
      if (e <= 0.0) return 0.0;
      v *= e;
    }
    return v;
  }
  Box bound(const std::vector<Entry>& es, const std::vector<int>& idx) const {
    Box b = es[idx[0]].box;
    for (size_t i = 1; i < idx.size(); ++i) b = join(b, es[idx[i]].box);
    return b;
  }
  Box bound(const Node& nd) const {
    Box b = nd.entries[0].box;
    for (size_t i = 1; i < nd.entries.size(); ++i) b = join(b, nd.entries[i].box);
    return b;
  }
  void refresh_entry(int64_t parent, int64_t child) {
    for (Entry& e : nodes[parent].entries)
      if (e.child == child) {
        e.box = bound(nodes[child]);
        return;
      }
  }
  void adjust_up(int64_t n) {
    while (nodes[n].parent >= 0) {
      refresh_entry(nodes[n].parent, n);
      n = nodes[n].parent;
    }
  }

  void insert_element(const Box& b, int64_t e) {
    reinserted.assign(nodes[root].height + 2, 0);
    insert(Entry{b, e}, 0);
  }

  int64_t choose_subtree(const Box& b, int height) const {
    int64_t n = root;
    while (nodes[n].height > height) {
      const Node& nd = nodes[n];
      int best = -1;
      double k0 = 0, k1 = 0, k2 = 0;
      for (int i = 0; i < (int)nd.entries.size(); ++i) {
        const Box& eb = nd.entries[i].box;
        const Box u = join(eb, b);
        const double a = area(eb);
        const double enl = area(u) - a;
        if (nd.height == 1) {
          double ov = 0.0;
          for (int j = 0; j < (int)nd.entries.size(); ++j)
            if (j != i) ov += overlap(u, nd.entries[j].box) - overlap(eb, nd.entries[j].box);
          if (best < 0 || ov < k0 || (ov == k0 && (enl < k1 || (enl == k1 && a < k2)))) {
            best = i;
            k0 = ov;
            k1 = enl;
            k2 = a;
          }
        } else if (best < 0 || enl < k1 || (enl == k1 && a < k2)) {
          best = i;
          k1 = enl;
          k2 = a;
        }
      }
      n = nd.entries[best].child;
    }
    return n;
  }

  void insert(const Entry& en, int height) {
    const int64_t n = choose_subtree(en.box, height);
    nodes[n].entries.push_back(en);
    if (height > 0) nodes[en.child].parent = n;
    if ((int)nodes[n].entries.size() > M) overflow(n);
    else adjust_up(n);
  }

  void overflow(int64_t n) {
    const int h = nodes[n].height;
    if ((int)reinserted.size() <= h) reinserted.resize(h + 1, 0);
    if (n != root && !reinserted[h]) {
      reinserted[h] = 1;
      reinsert(n);
    } else {
      split(n);
    }
  }

  void reinsert(int64_t n) {
    const Box nb = bound(nodes[n]);
    double c[3];
    for (int k = 0; k < dim; ++k) c[k] = 0.5 * (nb.lo[k] + nb.hi[k]);
    const std::vector<Entry> es = nodes[n].entries;
    std::vector<double> d(es.size(), 0.0);
    for (size_t i = 0; i < es.size(); ++i)
      for (int k = 0; k < dim; ++k) {
        const double t = 0.5 * (es[i].box.lo[k] + es[i].box.hi[k]) - c[k];
        d[i] += t * t;
      }
    std::vector<int> order(es.size());
    for (size_t i = 0; i < es.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return d[a] > d[b] || (d[a] == d[b] && a < b); });
    std::vector<int> keep(order.begin() + p, order.end());
    std::sort(keep.begin(), keep.end());
    nodes[n].entries.clear();
    for (int i : keep) nodes[n].entries.push_back(es[i]);
    adjust_up(n);
    const int h = nodes[n].height;
    for (int t = p - 1; t >= 0; --t) insert(es[order[t]], h);
  }

  // distributions of one axis: (lower sort, then upper sort) x k
  void distributions(const std::vector<Entry>& es, int axis, std::vector<std::vector<int>>& sorts) const {
    sorts.assign(2, std::vector<int>(es.size()));
    for (int s = 0; s < 2; ++s) {
      for (size_t i = 0; i < es.size(); ++i) sorts[s][i] = (int)i;
      std::sort(sorts[s].begin(), sorts[s].end(), [&](int a, int b) {
        const double a0 = s ? es[a].box.hi[axis] : es[a].box.lo[axis];
        const double b0 = s ? es[b].box.hi[axis] : es[b].box.lo[axis];
        if (a0 != b0) return a0 < b0;
        const double a1 = s ? es[a].box.lo[axis] : es[a].box.hi[axis];
        const double b1 = s ? es[b].box.lo[axis] : es[b].box.hi[axis];
        if (a1 != b1) return a1 < b1;
        return a < b;
      });
    }
  }

  void split(int64_t n) {
    const std::vector<Entry> es = nodes[n].entries;
    const int kmax = M - 2 * m + 2;
    std::vector<std::vector<int>> sorts;
    int best_axis = 0;
    double best_s = 0.0;
    for (int axis = 0; axis < dim; ++axis) {
      distributions(es, axis, sorts);
      double s = 0.0;
      for (int so = 0; so < 2; ++so)
        for (int k = 1; k <= kmax; ++k) {
          const int n1 = m - 1 + k;
          std::vector<int> g1(sorts[so].begin(), sorts[so].begin() + n1), g2(sorts[so].begin() + n1, sorts[so].end());
          s += margin(bound(es, g1)) + margin(bound(es, g2));
        }
      if (axis == 0 || s < best_s) {
        best_axis = axis;
        best_s = s;
      }
    }
    distributions(es, best_axis, sorts);
    std::vector<int> b1, b2;
    double o_best = 0.0, a_best = 0.0;
    bool have = false;
    for (int so = 0; so < 2; ++so)
      for (int k = 1; k <= kmax; ++k) {
        const int n1 = m - 1 + k;
        std::vector<int> g1(sorts[so].begin(), sorts[so].begin() + n1), g2(sorts[so].begin() + n1, sorts[so].end());
        const Box x1 = bound(es, g1), x2 = bound(es, g2);
        const double o = overlap(x1, x2), a = area(x1) + area(x2);
        if (!have || o < o_best || (o == o_best && a < a_best)) {
          have = true;
          o_best = o;
          a_best = a;
          b1 = g1;
          b2 = g2;
        }
      }
    const int64_t sib = (int64_t)nodes.size();
    nodes.emplace_back();
    nodes[sib].height = nodes[n].height;
    nodes[n].entries.clear();
    for (int i : b1) nodes[n].entries.push_back(es[i]);
    for (int i : b2) nodes[sib].entries.push_back(es[i]);
    if (nodes[n].height > 0)
      for (const Entry& e : nodes[sib].entries) nodes[e.child].parent = sib;
    if (n == root) {
      const int64_t r = (int64_t)nodes.size();
      nodes.emplace_back();
      nodes[r].height = nodes[n].height + 1;
      nodes[r].entries.push_back(Entry{bound(nodes[n]), n});
      nodes[r].entries.push_back(Entry{bound(nodes[sib]), sib});
      nodes[n].parent = nodes[sib].parent = r;
      root = r;
      return;
    }
    const int64_t par = nodes[n].parent;
    refresh_entry(par, n);
    nodes[par].entries.push_back(Entry{bound(nodes[sib]), sib});
    nodes[sib].parent = par;
    if ((int)nodes[par].entries.size() > M) overflow(par);
    else adjust_up(par);
  }

  // node ids per height, depth first from the root
  void number(std::vector<std::vector<int64_t>>& per_height) const {
    per_height.assign(nodes[root].height + 1, {});
    std::vector<int64_t> stack{root};
    while (!stack.empty()) {
      const int64_t n = stack.back();
      stack.pop_back();
      per_height[nodes[n].height].push_back(n);
      if (nodes[n].height > 0)
        for (auto it = nodes[n].entries.rbegin(); it != nodes[n].entries.rend(); ++it) stack.push_back(it->child);
    }
  }
};

}  // namespace

int rtree_agglomerate(const Mesh& m, int max_entries, int n_maps, int32_t* const* maps, int64_t* n_units,
                      int* height, std::string& err) {
  if (max_entries < 4) {
    err = "max_entries must be >= 4";
    return AGG_EINVAL;
  }
  const int dim = m.dim, V = 1 << dim;
  RTree t(dim, max_entries);
  for (int64_t e = 0; e < m.ne; ++e) {
    Box b;
    for (int k = 0; k < dim; ++k) {
      b.lo[k] = m.X[m.cells[e * V] * dim + k];
      b.hi[k] = b.lo[k];
    }
    for (int c = 1; c < V; ++c)
      for (int k = 0; k < dim; ++k) {
        const double x = m.X[m.cells[e * V + c] * dim + k];
        b.lo[k] = std::min(b.lo[k], x);
        b.hi[k] = std::max(b.hi[k], x);
      }
    t.insert_element(b, e);
  }
  std::vector<std::vector<int64_t>> ph;
  t.number(ph);
  if (height) *height = (int)ph.size();
  if (n_maps > (int)ph.size()) {
    err = "n_maps exceeds the number of tree levels";
    return AGG_EINVAL;
  }
  if (n_maps > 0 && (!maps || !n_units)) {
    err = "NULL maps or n_units";
    return AGG_EINVAL;
  }
  std::vector<int64_t> local(t.nodes.size(), -1);
  for (auto& lv : ph)
    for (size_t i = 0; i < lv.size(); ++i) local[lv[i]] = (int64_t)i;
  for (int k = 0; k < n_maps; ++k) {
    if (!maps[k]) {
      err = "NULL map array";
      return AGG_EINVAL;
    }
    n_units[k] = (int64_t)ph[k].size();
    for (int64_t n : ph[k])
      for (const auto& e : t.nodes[n].entries) {
        const int64_t src = (k == 0) ? e.child : local[e.child];
        maps[k][src] = (int32_t)local[n];
      }
  }
  return AGG_OK;
}

}  // namespace aggmg
