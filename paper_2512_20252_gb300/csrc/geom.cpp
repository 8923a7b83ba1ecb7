// geom.cpp -- host-side geometry for the immersed-boundary DVM solver.
//
// Cell and point classes follow arXiv 2512.20252 Sec. 3.2.1; the incident
// measures of cut velocity boxes follow Sec. 3.2.3 (Eqs. fwc, cc_np).  The
// readings taken where the paper is silent (a centre on the surface is solid;
// one link per ghost/fluid face pair; the crossing nearest the donor; the mean
// normal at a polygon vertex; a zero donor slope without a fluid auxiliary
// cell) are stated where they are used.
#include "geom.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace ibdvm {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Coordinate c + m * (hw / M) for an integer m: exactly antisymmetric about the
// interval centre, so mirrored nodes (and cells) are exact negatives and the
// exact-zero decisions of the method (upwind-weight fallback, node sign on the
// wall plane) are mirror-symmetric.
inline double centred(double lo, double hi, long m, long M) {
  return 0.5 * (lo + hi) + static_cast<double>(m) * ((0.5 * (hi - lo)) / static_cast<double>(M));
}

struct Body {
  const Geom &G;
  explicit Body(const Geom &g) : G(g) {}

  // <= 0 inside or on the surface
  double level(const double *x) const {
    const ibdvm_body_desc &b = G.body;
    switch (b.kind) {
    case IBDVM_BODY_CIRCLE:
    case IBDVM_BODY_SPHERE: {
      double s = 0.0;
      for (int a = 0; a < G.dim; ++a) s += (x[a] - b.center[a]) * (x[a] - b.center[a]);
      return s - b.radii[0] * b.radii[0];
    }
    case IBDVM_BODY_ELLIPSE: {
      double dx = x[0] - b.center[0], dy = x[1] - b.center[1];
      double ca = std::cos(b.angle), sa = std::sin(b.angle);
      double u = ca * dx + sa * dy, v = -sa * dx + ca * dy;
      return (u / b.radii[0]) * (u / b.radii[0]) + (v / b.radii[1]) * (v / b.radii[1]) - 1.0;
    }
    case IBDVM_BODY_POLYGON:
      return inside_polygon(x) ? -1.0 : 1.0;
    case IBDVM_BODY_HALFSPACE: {
      double s = 0.0;
      for (int a = 0; a < G.dim; ++a) s += (x[a] - b.center[a]) * b.radii[a];
      return s;
    }
    default:
      return 1.0;
    }
  }

  // even-odd crossing rule along +x
  bool inside_polygon(const double *x) const {
    const std::vector<double> &v = G.verts;
    int m = static_cast<int>(v.size() / 2);
    bool in = false;
    for (int i = 0, j = m - 1; i < m; j = i++) {
      double yi = v[2 * i + 1], yj = v[2 * j + 1];
      if ((yi > x[1]) != (yj > x[1])) {
        double xc = v[2 * j] + (x[1] - yj) * (v[2 * i] - v[2 * j]) / (yi - yj);
        if (x[0] < xc) in = !in;
      }
    }
    return in;
  }

  // Intersect point on the axis-aligned segment from the ghost centre xg to the
  // donor centre xd (closed forms), and the unit normal into the gas there.
  void intersect(const double *xg, const double *xd, int axis, int side, double *xw,
                 double *nw) const {
    const ibdvm_body_desc &b = G.body;
    for (int a = 0; a < 3; ++a) xw[a] = xg[a];
    double nrm[3] = {0, 0, 0};
    switch (b.kind) {
    case IBDVM_BODY_CIRCLE:
    case IBDVM_BODY_SPHERE: {
      // along the axis: (y - c)^2 = r^2 - (distance in the other coordinates)^2;
      // leaving the ball in direction `side` exits at c + side * sqrt(.)
      double q = b.radii[0] * b.radii[0];
      for (int a = 0; a < G.dim; ++a)
        if (a != axis) q -= (xg[a] - b.center[a]) * (xg[a] - b.center[a]);
      double y = b.center[axis] + side * std::sqrt(std::max(q, 0.0));
      xw[axis] = clamp_on_segment(y, xg[axis], xd[axis]);
      for (int a = 0; a < G.dim; ++a) nrm[a] = xw[a] - b.center[a];
      break;
    }
    case IBDVM_BODY_ELLIPSE: {
      double ca = std::cos(b.angle), sa = std::sin(b.angle);
      double dx = xg[0] - b.center[0], dy = xg[1] - b.center[1];
      double u0 = ca * dx + sa * dy, v0 = -sa * dx + ca * dy;
      double ex = xd[0] - xg[0], ey = xd[1] - xg[1];
      double eu = ca * ex + sa * ey, ev = -sa * ex + ca * ey;
      double ia = 1.0 / (b.radii[0] * b.radii[0]), ib = 1.0 / (b.radii[1] * b.radii[1]);
      double A = eu * eu * ia + ev * ev * ib;
      double B = 2.0 * (u0 * eu * ia + v0 * ev * ib);
      double C = u0 * u0 * ia + v0 * v0 * ib - 1.0;
      double disc = std::sqrt(std::max(B * B - 4.0 * A * C, 0.0));
      // larger root of A t^2 + B t + C (C <= 0), cancellation-free form
      double t = (B > 0.0) ? (-2.0 * C) / (B + disc) : (-B + disc) / (2.0 * A);
      t = std::min(std::max(t, 0.0), 1.0);
      xw[0] = xg[0] + t * ex;
      xw[1] = xg[1] + t * ey;
      double px = xw[0] - b.center[0], py = xw[1] - b.center[1];
      double u = ca * px + sa * py, v = -sa * px + ca * py;
      nrm[0] = ca * (u * ia) - sa * (v * ib);
      nrm[1] = sa * (u * ia) + ca * (v * ib);
      break;
    }
    case IBDVM_BODY_HALFSPACE: {
      double phg = 0.0, den = 0.0;
      for (int a = 0; a < G.dim; ++a) {
        phg += (xg[a] - b.center[a]) * b.radii[a];
        den += (xd[a] - xg[a]) * b.radii[a];
      }
      double t = (den != 0.0) ? -phg / den : 0.0;
      t = std::min(std::max(t, 0.0), 1.0);
      xw[axis] = xg[axis] + t * (xd[axis] - xg[axis]);
      for (int a = 0; a < G.dim; ++a) nrm[a] = b.radii[a];
      break;
    }
    case IBDVM_BODY_POLYGON:
      polygon_crossing(xg, xd, xw, nrm);
      break;
    default:
      break;
    }
    double len = 0.0;
    for (int a = 0; a < G.dim; ++a) len += nrm[a] * nrm[a];
    len = std::sqrt(len);
    for (int a = 0; a < 3; ++a) nw[a] = (a < G.dim && len > 0.0) ? nrm[a] / len : 0.0;
  }

  static double clamp_on_segment(double y, double yg, double yd) {
    double lo = std::min(yg, yd), hi = std::max(yg, yd);
    return std::min(std::max(y, lo), hi);
  }

  // every edge crossed by the segment; the crossing nearest the donor wins;
  // at a vertex the two adjacent edge normals are averaged
  void polygon_crossing(const double *xg, const double *xd, double *xw, double *nrm) const {
    const std::vector<double> &v = G.verts;
    int m = static_cast<int>(v.size() / 2);
    double dx = xd[0] - xg[0], dy = xd[1] - xg[1];
    double best_t = -1.0, best_u = 0.5;
    int best = -1;
    for (int e = 0; e < m; ++e) {
      double ax = v[2 * e], ay = v[2 * e + 1];
      double bx = v[2 * ((e + 1) % m)], by = v[2 * ((e + 1) % m) + 1];
      double ex = bx - ax, ey = by - ay;
      double cross = dx * ey - dy * ex;
      if (cross == 0.0) continue;
      double wx = ax - xg[0], wy = ay - xg[1];
      double t = (wx * ey - wy * ex) / cross;
      double u = (wx * dy - wy * dx) / cross;
      if (t < 0.0 || t > 1.0 || u < 0.0 || u > 1.0) continue;
      if (t > best_t) {
        best_t = t;
        best_u = u;
        best = e;
      }
    }
    if (best < 0) {
      best = 0;
      best_t = 0.0;
      best_u = 0.5;
    }
    xw[0] = xg[0] + best_t * dx;
    xw[1] = xg[1] + best_t * dy;
    int edges[2] = {best, best};
    if (best_u < 1e-9) edges[0] = (best + m - 1) % m;
    if (best_u > 1.0 - 1e-9) edges[1] = (best + 1) % m;
    int cnt = (edges[0] == edges[1]) ? 1 : 2;
    nrm[0] = nrm[1] = 0.0;
    for (int q = 0; q < cnt; ++q) {
      int e = edges[q];
      double ex = v[2 * ((e + 1) % m)] - v[2 * e], ey = v[2 * ((e + 1) % m) + 1] - v[2 * e + 1];
      double l = std::sqrt(ex * ex + ey * ey);
      // counter-clockwise: the outward normal is the edge direction turned clockwise
      nrm[0] += ey / l;
      nrm[1] += -ex / l;
    }
  }
};

// Length of {y in [y0, y1] : nx * x + ny * y <= d} at abscissa x.
inline double clipped_length(double x, double y0, double y1, double nx, double ny, double d) {
  double full = y1 - y0;
  if (ny == 0.0) return (nx * x <= d) ? full : 0.0;
  double ys = (d - nx * x) / ny;
  double len = (ny > 0.0) ? ys - y0 : y1 - ys;
  return std::min(std::max(len, 0.0), full);
}

// Area of {p in [x0,x1]x[y0,y1] : nx px + ny py <= d}: the clipped length is
// piecewise linear in x with breaks where the line meets y = y0 or y = y1
// (a step at x = d/nx when ny = 0); the midpoint rule is exact on every
// linear piece and never samples a break.
double area_below(double x0, double x1, double y0, double y1, double nx, double ny, double d) {
  if (x1 <= x0 || y1 <= y0) return 0.0;
  double br[4];
  int nb = 0;
  br[nb++] = x0;
  if (nx != 0.0) {
    double xa = (d - ny * y0) / nx, xb = (d - ny * y1) / nx;
    if (xa > x0 && xa < x1) br[nb++] = xa;
    if (xb > x0 && xb < x1) br[nb++] = xb;
  }
  br[nb++] = x1;
  std::sort(br, br + nb);
  double A = 0.0;
  for (int i = 0; i + 1 < nb; ++i) {
    double a = br[i], b = br[i + 1];
    if (b <= a) continue;
    A += (b - a) * clipped_length(0.5 * (a + b), y0, y1, nx, ny, d);
  }
  return A;
}

} // namespace

double incident_area_2d(const double *lo, const double *hi, const double *n) {
  return area_below(lo[0], hi[0], lo[1], hi[1], n[0], n[1], 0.0);
}

// Volume of {p in box : n.p <= 0}: the slice area at height z is piecewise
// quadratic with breaks where the plane meets a vertical box edge (a step
// when n is along z); the two-point Gauss rule is exact on every quadratic
// piece and samples only its interior.
double incident_volume_3d(const double *lo, const double *hi, const double *n) {
  double br[6];
  int nb = 0;
  br[nb++] = lo[2];
  if (n[2] != 0.0) {
    for (int cx = 0; cx < 2; ++cx)
      for (int cy = 0; cy < 2; ++cy) {
        double z = -(n[0] * (cx ? hi[0] : lo[0]) + n[1] * (cy ? hi[1] : lo[1])) / n[2];
        if (z > lo[2] && z < hi[2]) br[nb++] = z;
      }
  }
  br[nb++] = hi[2];
  std::sort(br, br + nb);
  auto slice = [&](double z) {
    return area_below(lo[0], hi[0], lo[1], hi[1], n[0], n[1], -n[2] * z);
  };
  double V = 0.0;
  for (int i = 0; i + 1 < nb; ++i) {
    double a = br[i], b = br[i + 1];
    if (b <= a) continue;
    const double h = 0.5 * (b - a), m = 0.5 * (a + b), g = h / std::sqrt(3.0);
    V += h * (slice(m - g) + slice(m + g));
  }
  return V;
}

double cell_coord(const Geom &G, int a, int i) {
  return centred(G.lo[a], G.hi[a], 2L * i + 1 - G.n[a], G.n[a]);
}

bool build_grid(const ibdvm_grid_desc &g, const ibdvm_vgrid_desc &v, const ibdvm_gas_desc &gas,
                Geom &G, std::string &err) {
  if (g.dim != 2 && g.dim != 3) {
    err = "grid.dim must be 2 or 3";
    return false;
  }
  G = Geom();
  G.dim = g.dim;
  G.ncomp = (g.dim == 2) ? 2 : 1;
  G.ncell = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < g.dim) {
      if (g.n[a] < 4 || g.n[a] > (1 << 20)) {
        err = "grid.n[a] must be in [4, 2^20]";
        return false;
      }
      if (!(g.hi[a] > g.lo[a]) || !std::isfinite(g.lo[a]) || !std::isfinite(g.hi[a])) {
        err = "grid.lo < grid.hi required";
        return false;
      }
      G.n[a] = g.n[a];
      G.lo[a] = g.lo[a];
      G.hi[a] = g.hi[a];
      G.dx[a] = (g.hi[a] - g.lo[a]) / g.n[a];
      if (v.n[a] < 2 || v.n[a] > 4096) {
        err = "vgrid.n[a] must be in [2, 4096]";
        return false;
      }
      if (v.rule == IBDVM_RULE_NODES) {
        if (!v.nodes[a]) {
          err = "vgrid.nodes[a] is required for IBDVM_RULE_NODES";
          return false;
        }
        for (int i = 0; i < v.n[a]; ++i)
          if (!std::isfinite(v.nodes[a][i]) || (i > 0 && !(v.nodes[a][i] > v.nodes[a][i - 1]))) {
            err = "vgrid.nodes[a] must be finite and strictly increasing";
            return false;
          }
      } else if (!(v.hi[a] > v.lo[a])) {
        err = "vgrid.lo < vgrid.hi required";
        return false;
      }
      G.nvx[a] = v.n[a];
    } else {
      G.n[a] = 1;
      G.lo[a] = 0.0;
      G.hi[a] = 1.0;
      G.dx[a] = 1.0;
      G.nvx[a] = 1;
    }
    G.ncell *= G.n[a];
  }
  if (v.rule != IBDVM_RULE_TRAPEZOID && v.rule != IBDVM_RULE_MIDPOINT && v.rule != IBDVM_RULE_NODES) {
    err = "vgrid.rule must be trapezoid (0), midpoint (1) or nodes (2)";
    return false;
  }
  long long nv = 1;
  for (int a = 0; a < 3; ++a) nv *= G.nvx[a];
  if (nv > (1LL << 24)) {
    err = "too many velocity nodes";
    return false;
  }
  G.rule = v.rule;
  G.nv = static_cast<int>(nv);
  // padding of the velocity count: 64, or 128 for the FP32 sweeps' chunks of
  // 128 velocities (the padded velocities carry zero weight and no flux)
  const int pad = (gas.precision == IBDVM_MIXED) ? 2 * kVelPad : kVelPad;
  G.nvp = (G.nv + pad - 1) / pad * pad;
  // per-axis nodes, weights and dual boxes (Eq. quadrature)
  std::vector<double> ax[3], al[3], ah[3];
  for (int a = 0; a < 3; ++a) {
    int m = G.nvx[a];
    ax[a].resize(m);
    al[a].resize(m);
    ah[a].resize(m);
    if (a >= g.dim) {
      ax[a][0] = 0.0;
      al[a][0] = 0.0;
      ah[a][0] = 1.0; // unit measure along the absent axis
      continue;
    }
    double lo = v.lo[a], hi = v.hi[a];
    if (v.rule == IBDVM_RULE_NODES) {
      // given nodes: each owns the box between the midpoints to its neighbours
      for (int i = 0; i < m; ++i) ax[a][i] = v.nodes[a][i];
      for (int i = 0; i < m; ++i) {
        al[a][i] = (i == 0) ? ax[a][0] : 0.5 * (ax[a][i - 1] + ax[a][i]);
        ah[a][i] = (i == m - 1) ? ax[a][m - 1] : 0.5 * (ax[a][i] + ax[a][i + 1]);
      }
    } else if (v.rule == IBDVM_RULE_TRAPEZOID) {
      double h = (hi - lo) / (m - 1);
      for (int i = 0; i < m; ++i) {
        ax[a][i] = centred(lo, hi, 2L * i - (m - 1), m - 1);
        al[a][i] = (i == 0) ? lo : ax[a][i] - 0.5 * h;
        ah[a][i] = (i == m - 1) ? hi : ax[a][i] + 0.5 * h;
      }
    } else {
      double h = (hi - lo) / m;
      for (int i = 0; i < m; ++i) {
        ax[a][i] = centred(lo, hi, 2L * i + 1 - m, m);
        al[a][i] = ax[a][i] - 0.5 * h;
        ah[a][i] = ax[a][i] + 0.5 * h;
      }
    }
  }
  G.xi.assign(3 * G.nv, 0.0);
  G.w.assign(G.nv, 0.0);
  G.blo.assign(3 * G.nv, 0.0);
  G.bhi.assign(3 * G.nv, 0.0);
  for (int k = 0; k < G.nv; ++k) {
    int id[3] = {k % G.nvx[0], (k / G.nvx[0]) % G.nvx[1], k / (G.nvx[0] * G.nvx[1])};
    double wk = 1.0;
    for (int a = 0; a < 3; ++a) {
      G.xi[3 * k + a] = (a < g.dim) ? ax[a][id[a]] : 0.0;
      G.blo[3 * k + a] = al[a][id[a]];
      G.bhi[3 * k + a] = ah[a][id[a]];
      wk *= ah[a][id[a]] - al[a][id[a]];
    }
    G.w[k] = wk;
  }
  // gas (Sec. 4)
  if (!(gas.Kn > 0.0) || !(gas.Pr > 0.0) || !(gas.gamma > 0.0) || !(gas.rho_inf > 0.0) ||
      !(gas.T_inf > 0.0) || !(gas.alpha_vhs > 0.0) || !(gas.Ma >= 0.0) ||
      !(gas.omega_vhs > 0.0 && gas.omega_vhs < 2.5)) {
    err = "gas parameters out of range (Kn, Pr, gamma, rho_inf, T_inf, alpha_vhs > 0; Ma >= 0)";
    return false;
  }
  if (!(gas.dt > 0.0) && !(gas.cfl > 0.0)) {
    err = "either gas.dt > 0 or gas.cfl > 0 is required";
    return false;
  }
  if (gas.precision != IBDVM_FP64 && gas.precision != IBDVM_MIXED) {
    err = "gas.precision must be IBDVM_FP64 or IBDVM_MIXED";
    return false;
  }
  G.gas = gas;
  G.mu0 = 5.0 * (gas.alpha_vhs + 1.0) * (gas.alpha_vhs + 2.0) * std::sqrt(kPi) /
          (4.0 * gas.alpha_vhs * (5.0 - 2.0 * gas.omega_vhs) * (7.0 - 2.0 * gas.omega_vhs)) * gas.Kn;
  double dn = 0.0;
  for (int a = 0; a < g.dim; ++a) dn += gas.dir[a] * gas.dir[a];
  dn = std::sqrt(dn);
  double U = gas.Ma * std::sqrt(gas.gamma * gas.T_inf / 2.0);
  for (int a = 0; a < 3; ++a) G.Uinf[a] = (a < g.dim && dn > 0.0) ? U * gas.dir[a] / dn : 0.0;
  if (gas.dt > 0.0) {
    G.dt = gas.dt;
  } else {
    double rate = 0.0; // sum over axes of the largest |xi_a| per cell width
    for (int a = 0; a < g.dim; ++a) {
      double mx = std::max(std::fabs(ax[a].front()), std::fabs(ax[a].back()));
      for (double x : ax[a]) mx = std::max(mx, std::fabs(x));
      rate += mx / G.dx[a];
    }
    G.dt = gas.cfl / rate;
  }
  G.type.assign(G.ncell, IBDVM_CELL_FLUID);
  G.nfluid = G.ncell;
  G.body = ibdvm_body_desc{};
  G.body.kind = IBDVM_BODY_NONE;
  return true;
}

bool place_body(const ibdvm_body_desc &bd, Geom &G, std::string &err) {
  // validate
  switch (bd.kind) {
  case IBDVM_BODY_NONE:
    break;
  case IBDVM_BODY_CIRCLE:
  case IBDVM_BODY_ELLIPSE:
  case IBDVM_BODY_POLYGON:
    if (G.dim != 2) {
      err = "circle, ellipse and polygon bodies are 2D";
      return false;
    }
    break;
  case IBDVM_BODY_SPHERE:
    if (G.dim != 3) {
      err = "a sphere body is 3D";
      return false;
    }
    break;
  case IBDVM_BODY_HALFSPACE:
    break;
  default:
    err = "unknown body kind";
    return false;
  }
  if ((bd.kind == IBDVM_BODY_CIRCLE || bd.kind == IBDVM_BODY_SPHERE) && !(bd.radii[0] > 0.0)) {
    err = "radius must be positive";
    return false;
  }
  if (bd.kind == IBDVM_BODY_ELLIPSE && !(bd.radii[0] > 0.0 && bd.radii[1] > 0.0)) {
    err = "ellipse semi-axes must be positive";
    return false;
  }
  if (bd.kind == IBDVM_BODY_POLYGON && (bd.nverts < 3 || bd.verts == nullptr)) {
    err = "a polygon needs at least 3 vertices";
    return false;
  }
  if (bd.kind == IBDVM_BODY_HALFSPACE) {
    double l = 0.0;
    for (int a = 0; a < G.dim; ++a) l += bd.radii[a] * bd.radii[a];
    if (!(l > 0.0)) {
      err = "half-space normal must be non-zero";
      return false;
    }
  }
  if (bd.kind != IBDVM_BODY_NONE && (!(bd.accom_alpha >= 0.0 && bd.accom_alpha <= 1.0) ||
                                     !(bd.T_w > 0.0))) {
    err = "accom_alpha must be in [0,1] and T_w > 0";
    return false;
  }
  G.body = bd;
  G.body.verts = nullptr;
  G.verts.clear();
  if (bd.kind == IBDVM_BODY_POLYGON) G.verts.assign(bd.verts, bd.verts + 2 * bd.nverts);
  if (bd.kind == IBDVM_BODY_HALFSPACE) { // keep a unit normal
    double l = 0.0;
    for (int a = 0; a < G.dim; ++a) l += bd.radii[a] * bd.radii[a];
    l = std::sqrt(l);
    for (int a = 0; a < G.dim; ++a) G.body.radii[a] = bd.radii[a] / l;
  }
  Body body(G);
  const int D = G.dim;
  auto centre = [&](long long c, double *x) {
    long long i = c % G.n[0], j = (c / G.n[0]) % G.n[1], k = c / (static_cast<long long>(G.n[0]) * G.n[1]);
    long long ijk[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) x[a] = (a < D) ? cell_coord(G, a, static_cast<int>(ijk[a])) : 0.0;
  };
  auto index = [&](long long i, long long j, long long k) -> long long {
    if (i < 0 || j < 0 || k < 0 || i >= G.n[0] || j >= G.n[1] || k >= G.n[2]) return -1;
    return i + G.n[0] * (j + static_cast<long long>(G.n[1]) * k);
  };
  auto coords = [&](long long c, long long *ijk) {
    ijk[0] = c % G.n[0];
    ijk[1] = (c / G.n[0]) % G.n[1];
    ijk[2] = c / (static_cast<long long>(G.n[0]) * G.n[1]);
  };
  // 1. solid cells: centre inside or on the body (a surface point counts as solid)
  G.type.assign(G.ncell, IBDVM_CELL_FLUID);
  if (bd.kind != IBDVM_BODY_NONE) {
    for (long long c = 0; c < G.ncell; ++c) {
      double x[3];
      centre(c, x);
      if (body.level(x) <= 0.0) G.type[c] = IBDVM_CELL_SOLID;
    }
  }
  // 2. ghost cells: solid with a fluid face neighbour
  std::vector<uint8_t> t0 = G.type;
  for (long long c = 0; c < G.ncell; ++c) {
    if (t0[c] != IBDVM_CELL_SOLID) continue;
    long long ijk[3];
    coords(c, ijk);
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        long long q[3] = {ijk[0], ijk[1], ijk[2]};
        q[a] += s;
        long long nb = index(q[0], q[1], q[2]);
        if (nb >= 0 && t0[nb] == IBDVM_CELL_FLUID) G.type[c] = IBDVM_CELL_GHOST;
      }
  }
  G.nfluid = 0;
  for (long long c = 0; c < G.ncell; ++c) G.nfluid += (G.type[c] == IBDVM_CELL_FLUID);
  // 3. links and surface cells, ghosts in ascending order
  G.ghosts.clear();
  G.ghost_first.clear();
  G.ghost_nlinks.clear();
  G.links.clear();
  G.surf_off.assign(1, 0);
  G.surf_cell.clear();
  for (long long c = 0; c < G.ncell; ++c) {
    if (G.type[c] != IBDVM_CELL_GHOST) continue;
    int gidx = static_cast<int>(G.ghosts.size());
    G.ghosts.push_back(static_cast<int>(c));
    G.ghost_first.push_back(static_cast<int>(G.links.size()));
    long long ijk[3];
    coords(c, ijk);
    double xg[3];
    centre(c, xg);
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        long long q[3] = {ijk[0], ijk[1], ijk[2]};
        q[a] += s;
        long long d = index(q[0], q[1], q[2]);
        if (d < 0 || G.type[d] != IBDVM_CELL_FLUID) continue;
        Link L{};
        L.ghost = static_cast<int>(c);
        L.gidx = gidx;
        L.donor = static_cast<int>(d);
        L.axis = a;
        L.side = s;
        double xd[3];
        centre(d, xd);
        body.intersect(xg, xd, a, s, L.xw, L.nw);
        q[a] += s;
        long long ac = index(q[0], q[1], q[2]);
        L.aux = (ac >= 0 && G.type[ac] == IBDVM_CELL_FLUID) ? static_cast<int>(ac) : -1;
        double yg = xg[a], yd = xd[a], yw = L.xw[a];
        double ysp = yw + 0.5 * (yd - yg);   // Eq. sp
        double yac = yd + s * G.dx[a];
        L.c_sp = (L.aux >= 0) ? (ysp - yd) / (yac - yd) : 0.0;
        L.c_iw = (yw - ysp) / (yg - ysp);
        L.c_gc = (yg - ysp) / (yw - ysp);
        G.links.push_back(L);
      }
    G.ghost_nlinks.push_back(static_cast<int>(G.links.size()) - G.ghost_first.back());
    // surface cells: fluid cells among the 3^D - 1 neighbours
    int zr = (D == 3) ? 1 : 0;
    for (int oz = -zr; oz <= zr; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (ox == 0 && oy == 0 && oz == 0) continue;
          long long j = index(ijk[0] + ox, ijk[1] + oy, ijk[2] + oz);
          if (j >= 0 && G.type[j] == IBDVM_CELL_FLUID) G.surf_cell.push_back(static_cast<int>(j));
        }
    G.surf_off.push_back(static_cast<int>(G.surf_cell.size()));
  }
  // 4. incident-side measure of every velocity box at every link (Sec. 3.2.3)
  const bool cut = !(G.gas.flags & IBDVM_NO_CUTCELL);
  const size_t nl = G.links.size();
  G.wg.assign(nl * G.nv, 0.0);
  for (size_t l = 0; l < nl; ++l) {
    const double *n = G.links[l].nw;
    for (int k = 0; k < G.nv; ++k) {
      const double *bl = &G.blo[3 * k], *bh = &G.bhi[3 * k];
      double xn = 0.0;
      for (int a = 0; a < D; ++a) xn += G.xi[3 * k + a] * n[a];
      double m = 0.0;
      bool straddles = false;
      if (cut) {
        double mn = 0.0, mx = 0.0; // extreme values of n.p over the box corners
        for (int a = 0; a < D; ++a) {
          double p = n[a] * bl[a], q = n[a] * bh[a];
          mn += std::min(p, q);
          mx += std::max(p, q);
        }
        straddles = (mn < 0.0 && mx > 0.0);
      }
      if (straddles) {
        m = (D == 2) ? incident_area_2d(bl, bh, n) : incident_volume_3d(bl, bh, n);
      } else {
        m = (xn <= 0.0) ? G.w[k] : 0.0; // Eq. general bc at the node
      }
      G.wg[l * G.nv + k] = m;
    }
  }
  return true;
}

} // namespace ibdvm
