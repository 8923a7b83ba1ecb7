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
#include <algorithm>
#include <string>
#include <vector>

#include "ctx.h"

namespace ibdvm {

bool build_tree_mesh(const ibdvm_grid_desc &root, const ibdvm_tree_desc &t, std::vector<int> &lev,
                     std::vector<int> &nb, std::vector<int> &own, std::string &err) {
  const int D = root.dim;
  if (D != 2 && D != 3) {
    err = "create_tree: tree-refined grids are 2D (quadtrees) or 3D (octrees)";
    return false;
  }
  const int L = t.maxlevel;
  if (L < 0 || L > 12 || t.nleaf <= 0 || !t.level || !t.ix || !t.iy || (D == 3 && !t.iz)) {
    err = "create_tree: need 0 <= maxlevel <= 12, nleaf > 0 and the level, ix, iy (and in 3D iz) arrays";
    return false;
  }
  long long nf[3] = {1, 1, 1};
  for (int a = 0; a < D; ++a) {
    if (root.n[a] <= 0 || ((long long)root.n[a] << L) > (1LL << 20)) {
      err = "create_tree: the root grid or the finest level is too large";
      return false;
    }
    nf[a] = (long long)root.n[a] << L;
  }
  if (nf[0] * nf[1] * nf[2] > (1LL << 28)) {
    err = "create_tree: the finest grid would exceed 2^28 cells";
    return false;
  }
  own.assign(static_cast<size_t>(nf[0] * nf[1] * nf[2]), -1);
  const int n = t.nleaf;
  auto origin = [&](int c, long long *q0, long long &s) {
    s = 1LL << (L - t.level[c]);
    q0[0] = t.ix[c] * s;
    q0[1] = t.iy[c] * s;
    q0[2] = (D == 3) ? t.iz[c] * s : 0;
  };
  for (int c = 0; c < n; ++c) {
    const int l = t.level[c];
    const int co[3] = {t.ix[c], t.iy[c], (D == 3) ? t.iz[c] : 0};
    bool in = l >= 0 && l <= L;
    for (int a = 0; a < D && in; ++a) in = co[a] >= 0 && co[a] < (root.n[a] << l);
    if (!in) {
      err = "create_tree: leaf " + std::to_string(c) + " lies outside its level's grid";
      return false;
    }
    long long q0[3], s;
    origin(c, q0, s);
    const long long sz = (D == 3) ? s : 1;
    for (long long k = q0[2]; k < q0[2] + sz; ++k)
      for (long long j = q0[1]; j < q0[1] + s; ++j)
        for (long long i = q0[0]; i < q0[0] + s; ++i) {
          int &o = own[static_cast<size_t>(i + nf[0] * (j + nf[1] * k))];
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
  const int NF = 1 << (D - 1);
  lev.assign(t.level, t.level + n);
  nb.assign(static_cast<size_t>(n) * 2 * D * NF, -1);
  for (int c = 0; c < n; ++c) {
    const int l = t.level[c];
    long long q0[3], s;
    origin(c, q0, s);
    for (int a = 0; a < D; ++a)
      for (int side = 0; side < 2; ++side) {
        int *out = &nb[(static_cast<size_t>(c) * 2 * D + 2 * a + side) * NF];
        // the finest cells just beyond the face, the first transverse axis
        // fastest: their distinct owners in the order met
        const long long fa = side ? q0[a] + s : q0[a] - 1;
        if (fa < 0 || fa >= nf[a]) continue; // the domain edge
        const int u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2;
        const long long sv = (D == 3) ? s : 1;
        int cnt = 0;
        for (long long tv = 0; tv < sv; ++tv)
          for (long long tu = 0; tu < s; ++tu) {
            long long q[3];
            q[a] = fa;
            q[u] = q0[u] + tu;
            q[v] = (D == 3) ? q0[v] + tv : 0;
            const int o = own[static_cast<size_t>(q[0] + nf[0] * (q[1] + nf[1] * q[2]))];
            bool seen = false;
            for (int m = 0; m < cnt; ++m) seen = seen || out[m] == o;
            if (seen) continue;
            if (cnt == NF) {
              err = "create_tree: leaf " + std::to_string(c) + " has too many neighbours on a side";
              return false;
            }
            out[cnt++] = o;
          }
        bool ok = cnt == 1 && (t.level[out[0]] == l || t.level[out[0]] == l - 1);
        if (cnt == NF && cnt > 1) {
          ok = true;
          for (int m = 0; m < cnt; ++m) ok = ok && t.level[out[m]] == l + 1;
        }
        if (!ok) {
          err = "create_tree: leaf " + std::to_string(c) + " has a neighbour more than one level apart";
          return false;
        }
      }
  }
  return true;
}

// The stencil tables of the tree sweep, one record per leaf so that a block
// reads its leaves' stencils in one pass (dimension D, NF = 2^(D-1) leaves
// at most beyond a face).  Entry t of leaf c: t < D the leaf itself along
// axis t; t >= D the upwind neighbour j = u % NF on side sd = (u / NF) % 2 of
// axis a = u / (2 NF), u = t - D.  Ints per entry (8 in 2D, 12 in 3D): the
// cell, the NF rows of its - side (one leaf, the finer leaves, or the halo),
// the NF rows of its + side, the mutual flag (the entry is c's only
// neighbour on that side and has c as its only neighbour on the other),
// padding; rows -1 none, -2 the freestream halo, -3 - l the ghost value of
// link l (a ghost neighbour, C29; an upwind neighbour that is a ghost is its
// link's row alone).  Doubles per entry: the reciprocal centre distances to
// the - and + sides (the neighbour's centre, or h to the halo), h, and 1 / h
// for t < D.  Eight ints per leaf: the number of leaves on each side 2a + sd
// (0 at the domain edge, 1, NF, or 3 for a ghost), then the regular flag
// (one fluid leaf of c's level on every side, each with one leaf or the
// domain edge beyond it) and the fluid flag.
void build_tree_stencils(int D, const std::vector<int> &lev, const std::vector<int> &nb, const double h0[3],
                         const std::vector<uint8_t> &type, const std::vector<int> &glink,
                         std::vector<int> &sti, std::vector<double> &stg, std::vector<int> &lrec) {
  const size_t n = lev.size();
  const int NF = 1 << (D - 1), NS = 2 * D, E = tree_entries(D), EI = tree_entry_ints(D);
  sti.assign(n * E * EI, -1);
  stg.assign(n * E * 4, 0.0);
  lrec.assign(n * 8, 0);
  auto edge = [&](int leaf, int a) { return h0[a] / static_cast<double>(1 << lev[leaf]); };
  auto side = [&](size_t c, int s, int j) { return nb[(c * NS + s) * NF + j]; };
  auto fluid = [&](int leaf) { return type.empty() || type[leaf] == IBDVM_CELL_FLUID; };
  // the rows c sees across its side s: a leaf, the finer leaves, the halo,
  // or the ghost value of the link from a ghost neighbour
  auto rows = [&](int c, int s, int *r) {
    for (int j = 0; j < NF; ++j) r[j] = -1;
    const int n0 = side(c, s, 0);
    if (n0 < 0) r[0] = -2;
    else if (!fluid(n0)) r[0] = -3 - glink[static_cast<size_t>(c) * NS + s];
    else
      for (int j = 0; j < NF; ++j) r[j] = side(c, s, j);
  };
  for (size_t c = 0; c < n; ++c) {
    const int ci = static_cast<int>(c);
    if (!fluid(ci)) continue; // no update: no stencils
    for (int t = 0; t < E; ++t) {
      int a, u, sd = 0;
      if (t < D) {
        a = t;
        u = ci;
      } else {
        const int v = t - D;
        a = v / (2 * NF);
        sd = (v / NF) % 2;
        u = side(c, 2 * a + sd, v % NF);
      }
      if (u < 0) continue;
      int *I = &sti[(c * E + t) * EI];
      double *Dd = &stg[(c * E + t) * 4];
      if (!fluid(u)) { // an upwind ghost: its link's value
        I[0] = -3 - glink[c * NS + 2 * a + sd];
        continue;
      }
      I[0] = u;
      rows(u, 2 * a, &I[1]);
      rows(u, 2 * a + 1, &I[1 + NF]);
      if (t >= D)
        I[1 + 2 * NF] = (side(c, 2 * a + sd, 1) < 0 && side(u, 2 * a + 1 - sd, 0) == ci &&
                         (NF < 2 || side(u, 2 * a + 1 - sd, 1) < 0))
                            ? 1
                            : 0;
      const double h = edge(u, a);
      for (int q = 0; q < 2; ++q) {
        const int n0 = side(u, 2 * a + q, 0);
        Dd[q] = 1.0 / ((n0 < 0) ? h : 0.5 * (h + edge(n0, a)));
      }
      Dd[2] = h;
      Dd[3] = (t < D) ? 1.0 / h : 0.0;
    }
    bool regular = true;
    for (int s = 0; s < NS; ++s) {
      const int n0 = side(c, s, 0), n1 = side(c, s, 1);
      lrec[c * 8 + s] = (n0 < 0) ? 0 : (!fluid(n0) ? 3 : (n1 < 0 ? 1 : NF));
      regular = regular && n0 >= 0 && fluid(n0) && n1 < 0 && side(n0, s ^ 1, 0) == ci && side(n0, s ^ 1, 1) < 0 &&
                side(n0, s, 1) < 0;
    }
    lrec[c * 8 + NS] = regular ? 1 : 0;
    lrec[c * 8 + NS + 1] = 1;
  }
}

// The order in which the sweep's blocks take the leaves: within each window
// of 256 consecutive leaves (the caller's order, near in space for leaves in
// Z order), the regular leaves (the gather-first path), then the other fluid
// leaves (the general path), then the solid ones, so that the four leaves of
// a block take paths of about the same length while the blocks of a window
// share the rows they read.
std::vector<int> tree_schedule(int D, const std::vector<int> &lrec) {
  constexpr size_t kWindow = 256;
  const size_t n = lrec.size() / 8;
  std::vector<int> sched;
  sched.reserve(n);
  for (size_t w0 = 0; w0 < n; w0 += kWindow)
    for (int cls = 0; cls < 3; ++cls)
      for (size_t c = w0; c < std::min(n, w0 + kWindow); ++c) {
        const bool fluid = lrec[c * 8 + 2 * D + 1] != 0, regular = lrec[c * 8 + 2 * D] != 0;
        if ((fluid && regular ? 0 : fluid ? 1 : 2) == cls) sched.push_back(static_cast<int>(c));
      }
  return sched;
}

// A body on a tree (C29): placed on the finest grid Gv by the uniform grid's
// geometry, then moved onto the leaves.  The ghost band must lie in the
// finest level, where the tree's arithmetic is the uniform grid's.
bool map_tree_body(const Geom &Gv, const std::vector<int> &own, const std::vector<int> &lev, int L, Geom &Gt,
                   std::vector<int> &glink, std::vector<int> &far, std::string &err) {
  const int D = Gv.dim, NS = 2 * D;
  const long long nx = Gv.n[0], ny = Gv.n[1], nz = Gv.n[2];
  const size_t nleaf = lev.size();
  auto finest = [&](long long v) { return lev[own[static_cast<size_t>(v)]] == L; };
  auto nbr = [&](long long v, int a, int s) -> long long { // -1 beyond the domain edge
    long long q[3] = {v % nx, (v / nx) % ny, v / (nx * ny)};
    q[a] += s;
    if (q[a] < 0 || q[a] >= Gv.n[a]) return -1;
    return q[0] + nx * (q[1] + ny * q[2]);
  };
  (void)nz;
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
    for (int a = 0; a < D && ok; ++a)
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
  glink.assign(nleaf * NS, -1);
  for (size_t l = 0; l < nl; ++l) {
    const Link &K = Gt.links[l];
    glink[static_cast<size_t>(K.donor) * NS + 2 * K.axis + ((-K.side) > 0 ? 1 : 0)] = static_cast<int>(l);
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
      far[l] = -3 - glink[static_cast<size_t>(Gt.links[l].donor) * NS + 2 * K.axis + (K.side > 0 ? 1 : 0)];
  }
  return true;
}

} // namespace ibdvm
