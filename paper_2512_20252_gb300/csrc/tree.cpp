// tree.cpp -- the leaves of a tree-refined 2D grid and their face neighbours.
//
// The tree-based AMR meshes of Sec. 4.2-4.4 are read as a root grid of equal
// cells, each leaf a square of level l (edge h / 2^l) given by its integer
// coordinates at that level, with face neighbours at most one level apart.
// The builder checks that the leaves tile the domain and keep the 2:1 rule,
// and lists for every leaf and side 2a + (s > 0) its one neighbour (same or
// coarser level), its two finer neighbours in increasing transverse order, or
// none at the domain edge.  The stencil tables of the tree sweep come from
// these lists; a body placed on the finest grid is moved onto the leaves
// when its ghost band lies in the finest level.
#include <string>
#include <vector>

#include "ctx.h"

namespace ibdvm {

bool build_tree_mesh(const ibdvm_grid_desc &root, const ibdvm_tree_desc &t, std::vector<int> &lev,
                     std::vector<int> &nb, std::vector<int> &own, std::string &err) {
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
  own.assign(static_cast<size_t>(nfx * nfy), -1);
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

// The stencil tables of the tree sweep, one record per leaf so that a block
// reads its leaves' stencils in one pass.  Entry t of leaf c: t < 2 the leaf
// itself along axis t; t >= 2 the upwind neighbour j = (t - 2) & 1 on side
// sd = ((t - 2) >> 1) & 1 of axis a = (t - 2) >> 2.  Ints per entry: the cell,
// its - side (one or two leaves), its + side, the mutual flag (the entry is
// c's only neighbour on that side and has c as its only neighbour on the
// other), then padding; rows -1 none, -2 the freestream halo, -3 - l the
// ghost value of link l (a ghost neighbour, C29; an upwind neighbour that is
// a ghost is its link's row alone).  Doubles per entry: the reciprocal
// centre distances to the - and + sides (the neighbour's centre, or h to the
// halo), h, and 1 / h for t < 2.  Ints per leaf: the number of leaves on
// side 2a + sd (0 at the domain edge, 1, 2, or 3 for a ghost), the regular
// flag (one fluid leaf of c's level on every side, each with one leaf or the
// domain edge beyond it), the fluid flag.
void build_tree_stencils(const std::vector<int> &lev, const std::vector<int> &nb, const double h0[2],
                         const std::vector<uint8_t> &type, const std::vector<int> &glink,
                         std::vector<int> &sti, std::vector<double> &stg, std::vector<int> &lrec) {
  const size_t n = lev.size();
  sti.assign(n * 10 * 8, -1);
  stg.assign(n * 10 * 4, 0.0);
  lrec.assign(n * 8, 0);
  auto edge = [&](int leaf, int a) { return h0[a] / static_cast<double>(1 << lev[leaf]); };
  auto side = [&](size_t c, int s, int j) { return nb[c * 8 + s * 2 + j]; };
  auto fluid = [&](int leaf) { return type.empty() || type[leaf] == IBDVM_CELL_FLUID; };
  // the row c sees across its side s: a leaf (two for two finer leaves), the
  // halo, or the ghost value of the link from a ghost neighbour
  auto rows = [&](int c, int s, int *r0, int *r1) {
    const int n0 = side(c, s, 0), n1 = side(c, s, 1);
    *r1 = -1;
    if (n0 < 0) *r0 = -2;
    else if (!fluid(n0)) *r0 = -3 - glink[static_cast<size_t>(c) * 4 + s];
    else {
      *r0 = n0;
      if (n1 >= 0) *r1 = n1;
    }
  };
  for (size_t c = 0; c < n; ++c) {
    const int ci = static_cast<int>(c);
    if (!fluid(ci)) continue; // no update: no stencils
    for (int t = 0; t < 10; ++t) {
      int a, u, sd = 0;
      if (t < 2) {
        a = t;
        u = ci;
      } else {
        a = (t - 2) >> 2;
        sd = ((t - 2) >> 1) & 1;
        u = side(c, 2 * a + sd, (t - 2) & 1);
      }
      if (u < 0) continue;
      int *I = &sti[(c * 10 + t) * 8];
      double *D = &stg[(c * 10 + t) * 4];
      if (!fluid(u)) { // an upwind ghost: its link's value
        I[0] = -3 - glink[c * 4 + 2 * a + sd];
        continue;
      }
      I[0] = u;
      rows(u, 2 * a, &I[1], &I[2]);
      rows(u, 2 * a + 1, &I[3], &I[4]);
      if (t >= 2)
        I[5] = (side(c, 2 * a + sd, 1) < 0 && side(u, 2 * a + 1 - sd, 0) == ci && side(u, 2 * a + 1 - sd, 1) < 0)
                   ? 1
                   : 0;
      const double h = edge(u, a);
      for (int q = 0; q < 2; ++q) {
        const int n0 = side(u, 2 * a + q, 0);
        D[q] = 1.0 / ((n0 < 0) ? h : 0.5 * (h + edge(n0, a)));
      }
      D[2] = h;
      D[3] = (t < 2) ? 1.0 / h : 0.0;
    }
    bool regular = true;
    for (int s = 0; s < 4; ++s) {
      const int n0 = side(c, s, 0), n1 = side(c, s, 1);
      lrec[c * 8 + s] = (n0 < 0) ? 0 : (!fluid(n0) ? 3 : (n1 < 0 ? 1 : 2));
      regular = regular && n0 >= 0 && fluid(n0) && n1 < 0 && side(n0, s ^ 1, 0) == ci && side(n0, s ^ 1, 1) < 0 &&
                side(n0, s, 1) < 0;
    }
    lrec[c * 8 + 4] = regular ? 1 : 0;
    lrec[c * 8 + 5] = 1;
  }
}

// A body on a tree (C29): placed on the finest grid Gv by the uniform grid's
// geometry, then moved onto the leaves.  The ghost band must lie in the
// finest level, where the tree's arithmetic is the uniform grid's.
bool map_tree_body(const Geom &Gv, const std::vector<int> &own, const std::vector<int> &lev, int L, Geom &Gt,
                   std::vector<int> &glink, std::vector<int> &far, std::string &err) {
  const long long nx = Gv.n[0], ny = Gv.n[1];
  const size_t nleaf = lev.size();
  auto finest = [&](long long v) { return lev[own[static_cast<size_t>(v)]] == L; };
  auto nbr = [&](long long v, int a, int s) -> long long { // -1 beyond the domain edge
    long long i = v % nx, j = v / nx;
    (a == 0 ? i : j) += s;
    if (i < 0 || i >= nx || j < 0 || j >= ny) return -1;
    return i + nx * j;
  };
  std::vector<uint8_t> type(nleaf, 255);
  for (long long v = 0; v < Gv.ncell; ++v) {
    const int c = own[static_cast<size_t>(v)];
    const uint8_t t = Gv.type[static_cast<size_t>(v)];
    if (type[c] == 255) type[c] = t;
    if (type[c] != t || (t == IBDVM_CELL_GHOST && lev[c] != L)) {
      err = "set_body: the body must lie in the finest level of the tree (it cuts leaf " + std::to_string(c) + ")";
      return false;
    }
  }
  for (const Link &K : Gv.links) {
    bool ok = finest(K.ghost) && finest(K.donor) && (K.aux < 0 || finest(K.aux));
    const long long fv = nbr(K.donor, K.axis, K.side);
    if (fv >= 0 && Gv.type[static_cast<size_t>(fv)] == IBDVM_CELL_FLUID && !finest(fv)) ok = false;
    if (!ok) {
      err = "set_body: the body must lie in the finest level of the tree (a donor, an auxiliary cell or the "
            "cell beyond a donor is a coarser leaf)";
      return false;
    }
  }
  for (int sc : Gv.surf_cell) {
    bool ok = finest(sc);
    for (int a = 0; a < 2 && ok; ++a)
      for (int s = -1; s <= 1; s += 2) {
        const long long q = nbr(sc, a, s);
        if (q >= 0 && Gv.type[static_cast<size_t>(q)] == IBDVM_CELL_FLUID && !finest(q)) ok = false;
      }
    if (!ok) {
      err = "set_body: the body must lie in the finest level of the tree (a surface cell or its neighbour is a "
            "coarser leaf)";
      return false;
    }
  }
  // the ghost band in leaf indices
  Gt.body = Gv.body;
  Gt.verts = Gv.verts;
  Gt.type = type;
  Gt.nfluid = 0;
  for (uint8_t t : type) Gt.nfluid += (t == IBDVM_CELL_FLUID);
  Gt.ghosts.resize(Gv.ghosts.size());
  for (size_t i = 0; i < Gv.ghosts.size(); ++i) Gt.ghosts[i] = own[static_cast<size_t>(Gv.ghosts[i])];
  Gt.ghost_first = Gv.ghost_first;
  Gt.ghost_nlinks = Gv.ghost_nlinks;
  Gt.links = Gv.links;
  for (Link &K : Gt.links) {
    K.ghost = own[static_cast<size_t>(K.ghost)];
    K.donor = own[static_cast<size_t>(K.donor)];
    K.aux = (K.aux >= 0) ? own[static_cast<size_t>(K.aux)] : -1;
  }
  Gt.surf_off = Gv.surf_off;
  Gt.surf_cell.resize(Gv.surf_cell.size());
  for (size_t e = 0; e < Gv.surf_cell.size(); ++e) Gt.surf_cell[e] = own[static_cast<size_t>(Gv.surf_cell[e])];
  Gt.wg = Gv.wg;
  // a fluid leaf's ghost neighbours: the link of each, by side 2a + (s > 0)
  const size_t nl = Gv.links.size();
  glink.assign(nleaf * 4, -1);
  for (size_t l = 0; l < nl; ++l) {
    const Link &K = Gt.links[l];
    glink[static_cast<size_t>(K.donor) * 4 + 2 * K.axis + ((-K.side) > 0 ? 1 : 0)] = static_cast<int>(l);
  }
  // beyond each donor along its link axis: a leaf, the halo or another ghost
  far.assign(nl, -2);
  for (size_t l = 0; l < nl; ++l) {
    const Link &K = Gv.links[l];
    const long long fv = nbr(K.donor, K.axis, K.side);
    if (fv < 0) continue;
    if (Gv.type[static_cast<size_t>(fv)] == IBDVM_CELL_FLUID)
      far[l] = own[static_cast<size_t>(fv)];
    else
      far[l] = -3 - glink[static_cast<size_t>(Gt.links[l].donor) * 4 + 2 * K.axis + (K.side > 0 ? 1 : 0)];
  }
  return true;
}

} // namespace ibdvm
