// Lit-panel search of Sec. 3.3 on the host: a binary cluster tree over the
// panels (Def. bct) with a bounding ball per cluster, and the recursive
// search ApproximateLitLeaves (Algorithm lit_leaves), which keeps the leaves
// whose ball the backward light cone of a point may meet (the ball test of
// Theorem phi_xi_sphere). Host arrays in, host arrays out: no device.
//
// The GPU kernels do not use it: they find the candidate trial panels of a
// test column by binary searches on the time-sorted panels of each trial
// column, then apply the same ball test per panel (the sparsity contract).
// This implementation serves the cardinality study of Sec. 4.1 (experiment
// 1): |X_N(x)| against |Sigma_N^Xi(x)| as N grows.
//
// Tree: clusters split at the median of the panel centroids along the
// coordinate (t, x, y, z) of largest extent, down to n_min panels per leaf
// (a balanced geometric bisection; O(N log N)). Balls: the approximate
// bounding sphere of Ritter (1990) carried over to R^4 - a first ball on the
// two mutually far vertices found from an arbitrary one, then grown to take
// in every vertex outside it - over the vertices of the cluster's panels.
#include <algorithm>
#include <cmath>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "stbem_internal.h"

struct bem_cluster_tree {
  struct Node {
    int32_t begin, end;     // panels perm[begin, end)
    int32_t left, right;    // children (-1: leaf)
    double c[4], r;         // bounding ball (t, x, y, z)
  };
  std::vector<Node> nodes;
  std::vector<int32_t> perm;
  int32_t depth = 0;
};

namespace {

using stbem::set_error;

// Ritter's approximate bounding sphere in R^4 of the points p[0..n)
void ritter4(const std::vector<const double*>& p, double c[4], double* r) {
  auto d2 = [](const double* a, const double* b) {
    double s = 0.0;
    for (int k = 0; k < 4; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
    return s;
  };
  auto farthest = [&](const double* from) {
    const double* best = p[0];
    double bd = -1.0;
    for (const double* q : p) {
      const double d = d2(from, q);
      if (d > bd) { bd = d; best = q; }
    }
    return best;
  };
  const double* a = farthest(p[0]);
  const double* b = farthest(a);
  for (int k = 0; k < 4; ++k) c[k] = 0.5 * (a[k] + b[k]);
  double rad = 0.5 * std::sqrt(d2(a, b));
  for (const double* q : p) {
    const double d = std::sqrt(d2(c, q));
    if (d > rad) {   // grow: the new ball touches q and the far side of the old one
      const double nr = 0.5 * (rad + d);
      const double shift = (nr - rad) / d;
      for (int k = 0; k < 4; ++k) c[k] += shift * (q[k] - c[k]);
      rad = nr;
    }
  }
  // rounding of the updates: enlarge to contain every point exactly
  for (const double* q : p) rad = std::max(rad, std::sqrt(d2(c, q)));
  *r = rad;
}

}  // namespace

extern "C" bem_status bem_cluster_tree_create(int64_t n_vert, const double* vert_txyz, int64_t n_tet,
                                              const int32_t* tets, int32_t n_min, bem_cluster_tree** out) {
  if (!out || !vert_txyz || !tets || n_vert <= 0 || n_tet <= 0 || n_min < 1 || n_tet > INT32_MAX) {
    set_error("bem_cluster_tree_create: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int64_t j = 0; j < 4 * n_tet; ++j)
    if (tets[j] < 0 || tets[j] >= n_vert) {
      set_error("bem_cluster_tree_create: vertex index out of range");
      return BEM_ERR_INVALID_ARG;
    }
  std::unique_ptr<bem_cluster_tree> T(new (std::nothrow) bem_cluster_tree());
  if (!T) {
    set_error("out of host memory");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  const int32_t n = (int32_t)n_tet;
  std::vector<double> cen(4 * (size_t)n);
  for (int32_t j = 0; j < n; ++j)
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int v = 0; v < 4; ++v) s += vert_txyz[4 * (size_t)tets[4 * (size_t)j + v] + k];
      cen[4 * (size_t)j + k] = 0.25 * s;
    }
  T->perm.resize(n);
  std::iota(T->perm.begin(), T->perm.end(), 0);
  // breadth of the recursion by an explicit stack: (node index, depth)
  T->nodes.push_back({0, n, -1, -1, {0, 0, 0, 0}, 0.0});
  std::vector<std::pair<int32_t, int32_t>> stack{{0, 0}};
  std::vector<const double*> pts;
  while (!stack.empty()) {
    const int32_t id = stack.back().first, dep = stack.back().second;
    stack.pop_back();
    T->depth = std::max(T->depth, dep);
    const int32_t b = T->nodes[id].begin, e = T->nodes[id].end;
    pts.clear();
    for (int32_t q = b; q < e; ++q)
      for (int v = 0; v < 4; ++v) pts.push_back(vert_txyz + 4 * (size_t)tets[4 * (size_t)T->perm[q] + v]);
    ritter4(pts, T->nodes[id].c, &T->nodes[id].r);
    if (e - b <= n_min) continue;
    // split at the median of the centroids along the coordinate of largest extent
    double lo[4], hi[4];
    for (int k = 0; k < 4; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int32_t q = b; q < e; ++q)
      for (int k = 0; k < 4; ++k) {
        lo[k] = std::min(lo[k], cen[4 * (size_t)T->perm[q] + k]);
        hi[k] = std::max(hi[k], cen[4 * (size_t)T->perm[q] + k]);
      }
    int ax = 0;
    for (int k = 1; k < 4; ++k)
      if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
    const int32_t mid = b + (e - b) / 2;
    std::nth_element(T->perm.begin() + b, T->perm.begin() + mid, T->perm.begin() + e, [&](int32_t u, int32_t v) {
      const double cu = cen[4 * (size_t)u + ax], cv = cen[4 * (size_t)v + ax];
      return cu < cv || (cu == cv && u < v);
    });
    const int32_t l = (int32_t)T->nodes.size();
    T->nodes.push_back({b, mid, -1, -1, {0, 0, 0, 0}, 0.0});
    T->nodes.push_back({mid, e, -1, -1, {0, 0, 0, 0}, 0.0});
    T->nodes[id].left = l;
    T->nodes[id].right = l + 1;
    stack.push_back({l + 1, dep + 1});
    stack.push_back({l, dep + 1});
  }
  *out = T.release();
  return BEM_OK;
}

extern "C" bem_status bem_cluster_tree_info(const bem_cluster_tree* T, int64_t* n_nodes, int64_t* n_leaves,
                                            int32_t* depth) {
  if (!T) {
    set_error("bem_cluster_tree_info: null tree");
    return BEM_ERR_INVALID_ARG;
  }
  int64_t leaves = 0;
  for (const auto& nd : T->nodes) leaves += nd.left < 0;
  if (n_nodes) *n_nodes = (int64_t)T->nodes.size();
  if (n_leaves) *n_leaves = leaves;
  if (depth) *depth = T->depth;
  return BEM_OK;
}

extern "C" bem_status bem_cluster_tree_query(const bem_cluster_tree* T, const double* x_txyz, int64_t cap,
                                             int32_t* panels, int64_t* n_panels, int64_t* n_visited) {
  if (!T || !x_txyz || !n_panels || cap < 0 || (cap > 0 && !panels)) {
    set_error("bem_cluster_tree_query: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  const double t = x_txyz[0];
  int64_t found = 0, visited = 0;
  std::vector<int32_t> stack{0};
  while (!stack.empty()) {
    const bem_cluster_tree::Node& nd = T->nodes[stack.back()];
    stack.pop_back();
    ++visited;
    // Theorem phi_xi_sphere: phi(x - z) = |x - z| - (t - s) over the ball
    // B_r(y) ranges over [phi(x - y) - d_r(|x - y|), phi(x - y) + r sqrt 2];
    // the cone misses the ball iff that range lies on one side of 0
    const double dx = x_txyz[1] - nd.c[1], dy = x_txyz[2] - nd.c[2], dz = x_txyz[3] - nd.c[3];
    const double al = std::sqrt(dx * dx + dy * dy + dz * dz);
    const double phi = al - (t - nd.c[0]);
    const double r = nd.r;
    const double dr = al < r / std::sqrt(2.0) ? al + std::sqrt(r * r - al * al) : r * std::sqrt(2.0);
    if (phi < -r * std::sqrt(2.0) || phi > dr) continue;
    if (nd.left < 0) {
      for (int32_t q = nd.begin; q < nd.end; ++q) {
        if (found < cap) panels[found] = T->perm[q];
        ++found;
      }
    } else {
      stack.push_back(nd.right);
      stack.push_back(nd.left);
    }
  }
  *n_panels = found;
  if (n_visited) *n_visited = visited;
  if (found > cap) {
    set_error("bem_cluster_tree_query: more panels than cap (n_panels holds the count)");
    return BEM_ERR_INVALID_ARG;
  }
  return BEM_OK;
}

extern "C" void bem_cluster_tree_destroy(bem_cluster_tree* T) { delete T; }
