// Domain decomposition of a mesh (Section 3.3, "Mixed Elements and Domain
// Decomposition"): elements are split into parts by recursive coordinate
// bisection of their centroids, either with per-type weights (one
// partitioning of all elements) or balanced (every type split on its own so
// each part holds the same number of elements of each type).
#include <algorithm>
#include <numeric>

#include "fr_mesh.hpp"

namespace frgb {

namespace {

struct Item {
  double x[3];
  double w;
  int64_t id;
};

// Assign parts [p0, p0 + np) to items[lo, hi): split along the widest
// centroid extent at the weighted fraction floor(np/2)/np.
void bisect(std::vector<Item>& it, size_t lo, size_t hi, int p0, int np,
            std::vector<int32_t>& part) {
  if (hi <= lo) return;
  if (np == 1) {
    for (size_t i = lo; i < hi; ++i) part[it[i].id] = p0;
    return;
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  double wt = 0.0;
  for (size_t i = lo; i < hi; ++i) {
    for (int k = 0; k < 3; ++k) {
      mn[k] = std::min(mn[k], it[i].x[k]);
      mx[k] = std::max(mx[k], it[i].x[k]);
    }
    wt += it[i].w;
  }
  int ax = 0;
  for (int k = 1; k < 3; ++k)
    if (mx[k] - mn[k] > mx[ax] - mn[ax]) ax = k;
  std::sort(it.begin() + lo, it.begin() + hi, [ax](const Item& a, const Item& b) {
    if (a.x[ax] != b.x[ax]) return a.x[ax] < b.x[ax];
    return a.id < b.id;
  });
  const int nl = np / 2;
  const double target = wt * double(nl) / double(np);
  double acc = 0.0;
  size_t cut = lo;
  while (cut < hi && acc + 0.5 * it[cut].w <= target) acc += it[cut++].w;
  // every side keeps at least as many items as it has parts, when possible
  const size_t n = hi - lo;
  if (n >= size_t(np)) {
    cut = std::max(cut, lo + size_t(nl));
    cut = std::min(cut, hi - size_t(np - nl));
  }
  bisect(it, lo, cut, p0, nl, part);
  bisect(it, cut, hi, p0 + nl, np - nl, part);
}

}  // namespace

std::string partition_elements(const std::vector<HostType>& types, int nparts,
                               int mode, const double w[3],
                               std::vector<int32_t>& part) {
  if (nparts < 1) return "number of parts must be positive";
  if (mode != 0 && mode != 1) return "partition mode must be 0 (weighted) or 1 (balanced)";
  if (mode == 0)
    for (int k = 0; k < 3; ++k)
      if (!(w[k] > 0.0)) return "element weights must be positive";
  int64_t total = 0;
  for (auto& T : types) total += T.ne;
  part.assign(size_t(total), 0);
  std::vector<Item> all;
  int64_t off = 0;
  for (auto& T : types) {
    const int nv = T.ref.nverts;
    const double wk = mode == 0 ? w[T.kind] : 1.0;
    if (!(wk > 0.0)) return "element weights must be positive";
    std::vector<Item> own;
    for (int64_t e = 0; e < T.ne; ++e) {
      Item it{{0, 0, 0}, wk, off + e};
      for (int v = 0; v < nv; ++v)
        for (int k = 0; k < 3; ++k) it.x[k] += T.verts[(size_t(e) * nv + v) * 3 + k] / nv;
      (mode == 0 ? all : own).push_back(it);
    }
    if (mode == 1) bisect(own, 0, own.size(), 0, nparts, part);
    off += T.ne;
  }
  if (mode == 0) bisect(all, 0, all.size(), 0, nparts, part);
  return "";
}

}  // namespace frgb
