// tree.cpp -- the leaves of a tree-refined 2D grid and their face neighbours.
//
// The tree-based AMR meshes of Sec. 4.2-4.4 are read as a root grid of equal
// cells, each leaf a square of level l (edge h / 2^l) given by its integer
// coordinates at that level, with face neighbours at most one level apart.
// The builder checks that the leaves tile the domain and keep the 2:1 rule,
// and lists for every leaf and side 2a + (s > 0) its one neighbour (same or
// coarser level), its two finer neighbours in increasing transverse order, or
// none at the domain edge.
#include <string>
#include <vector>

#include "ctx.h"

namespace ibdvm {

bool build_tree_mesh(const ibdvm_grid_desc &root, const ibdvm_tree_desc &t, std::vector<int> &lev,
                     std::vector<int> &nb, std::string &err) {
  if (root.dim != 2) {
    err = "create_tree: tree-refined grids are 2D";
    return false;
  }
  const int L = t.maxlevel;
  if (L < 0 || L > 12 || t.nleaf <= 0 || !t.level || !t.ix || !t.iy) {
    err = "create_tree: need 0 <= maxlevel <= 12, nleaf > 0 and the level, ix and iy arrays";
    return false;
  }
  for (int a = 0; a < 2; ++a)
    if (root.n[a] <= 0 || ((long long)root.n[a] << L) > (1LL << 20)) {
      err = "create_tree: the root grid or the finest level is too large";
      return false;
    }
  const long long nfx = (long long)root.n[0] << L, nfy = (long long)root.n[1] << L;
  if (nfx * nfy > (1LL << 28)) {
    err = "create_tree: the finest grid would exceed 2^28 cells";
    return false;
  }
  std::vector<int> own(static_cast<size_t>(nfx * nfy), -1);
  const int n = t.nleaf;
  for (int c = 0; c < n; ++c) {
    const int l = t.level[c];
    if (l < 0 || l > L || t.ix[c] < 0 || t.iy[c] < 0 || t.ix[c] >= (root.n[0] << l) || t.iy[c] >= (root.n[1] << l)) {
      err = "create_tree: leaf " + std::to_string(c) + " lies outside its level's grid";
      return false;
    }
    const long long s = 1LL << (L - l);
    for (long long i = t.ix[c] * s; i < (t.ix[c] + 1) * s; ++i)
      for (long long j = t.iy[c] * s; j < (t.iy[c] + 1) * s; ++j) {
        int &o = own[static_cast<size_t>(i + nfx * j)];
        if (o >= 0) {
          err = "create_tree: leaves " + std::to_string(o) + " and " + std::to_string(c) + " overlap";
          return false;
        }
        o = c;
      }
  }
  for (size_t q = 0; q < own.size(); ++q)
    if (own[q] < 0) {
      err = "create_tree: the leaves leave a hole";
      return false;
    }
  lev.assign(t.level, t.level + n);
  nb.assign(static_cast<size_t>(n) * 8, -1);
  for (int c = 0; c < n; ++c) {
    const int l = t.level[c];
    const long long s = 1LL << (L - l);
    const long long i0 = t.ix[c] * s, j0 = t.iy[c] * s;
    for (int a = 0; a < 2; ++a)
      for (int side = 0; side < 2; ++side) {
        int *out = &nb[static_cast<size_t>(c) * 8 + (2 * a + side) * 2];
        // the finest cells just beyond the face, in increasing transverse order
        const long long fa = (a == 0) ? (side ? i0 + s : i0 - 1) : (side ? j0 + s : j0 - 1);
        if (fa < 0 || fa >= (a == 0 ? nfx : nfy)) continue; // the domain edge
        int cnt = 0;
        for (long long q = 0; q < s; ++q) {
          const long long cell = (a == 0) ? fa + nfx * (j0 + q) : (i0 + q) + nfx * fa;
          const int o = own[static_cast<size_t>(cell)];
          if (cnt > 0 && out[cnt - 1] == o) continue;
          if (cnt == 2) {
            err = "create_tree: leaf " + std::to_string(c) + " has more than two neighbours on a side";
            return false;
          }
          out[cnt++] = o;
        }
        const bool one = cnt == 1 && (t.level[out[0]] == l || t.level[out[0]] == l - 1);
        const bool two = cnt == 2 && t.level[out[0]] == l + 1 && t.level[out[1]] == l + 1;
        if (!one && !two) {
          err = "create_tree: leaf " + std::to_string(c) + " has a neighbour more than one level apart";
          return false;
        }
      }
  }
  return true;
}

} // namespace ibdvm
