/*
 * ibdvm_oracle.c -- plain, slow, FP64 CPU oracle of one explicit time step of
 * the ghost-cell immersed-boundary discrete velocity method for the Shakhov
 * model (Ge, Cai, Zhang, Xiao, arXiv 2512.20252).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline of the benchmark may load it. The solver product never links it
 * and shares no code with it.
 *
 * Everything here is double precision and written as loops over cells,
 * velocities and components in the order in which the paper states the
 * method (Sec. 2.2, Sec. 3.2, Sec. 4).  There is no blocking, fusion or
 * reordering beyond what the definitions state.
 *
 * Readings where the paper is silent or ambiguous (each one is a named
 * choice here and in the design notes):
 *   C1  reduced-distribution temperature and heat flux follow from the
 *       moment definitions (Eqs. moments1-3) with h, b carrying the third
 *       translational degree of freedom.
 *   C2  quadrature: trapezoid or composite midpoint; each node owns the dual
 *       box [xi_k - dxi/2, xi_k + dxi/2] clipped to the truncated domain.
 *   C3  a cell centre on the body surface counts as solid.
 *   C4  one link per (ghost cell, fluid face neighbour); each link has its
 *       own intersect point, shifted point and ghost value.
 *   C5  with several crossings on a ghost-donor segment, the crossing
 *       nearest the donor is taken.
 *   C6  on a polygon vertex the normal is the normalised mean of the two
 *       edge normals.
 *   C7  the donor slope is zero when the auxiliary cell is not a fluid cell
 *       of the domain.
 *   C8  the moments of the bulk update use plain quadrature; the cut-cell
 *       correction applies at wall points only (Sec. 3.2.3).
 *   C9  pre-ghost slopes of surface cells use fluid and domain-halo
 *       neighbours only (van Leer with both, one-sided with one, zero with
 *       none).
 *   C10 the unit vector of the upwind weights points from the surface cell
 *       to the ghost cell, so that a zero weight sum marks velocities that
 *       leave the wall (Eq. upwind and the text after it).
 *   C11 the wall balance uses the incident set xi.n <= 0 of Eq. general bc,
 *       a single factor xi_n, and the unit-density wall Maxwellian
 *       (2D reduced: 1/(pi T_w) exp(-|xi-U_w|^2/T_w), B_w = T_w/2 H_w).
 *   C12 the incident/reflected split is the plane xi.n = 0 for any U_w.
 *   C13 accommodation alpha < 1: the specular part is f^i at the mirrored
 *       velocity by multilinear interpolation on the velocity grid (zero
 *       outside it), and the wall density balances the total mass flux.
 *   C14 the ghost cell's slope along the link axis is the one-sided
 *       difference toward the donor.
 *   C15 forward Euler for transport and relaxation alike.
 *   C16 dt = CFL / sum_a (max_k |xi_a| / dx_a) unless given.
 *   C17 two halo layers outside the domain hold the freestream Maxwellian.
 *   C18 residual components whose sum of |W| is zero are skipped.
 *   C19 surface force and heat flux: momentum and energy carried through the
 *       donor-ghost faces by the face fluxes the update applies.
 *   C25 a non-uniform velocity grid is the tensor product of per-axis node
 *       lists (a stretched Cartesian grid, standing in for the locally
 *       refined mesh of Sec. 4.4): the interval of an axis is [x_0, x_n-1],
 *       each node owns the box between the midpoints to its neighbours (the
 *       trapezoid rule on non-uniform nodes), and the specular interpolation
 *       (C13) brackets a velocity by bisection on each axis.
 *   C27 optional ablation (default off): without the upwind-weighted
 *       strategy (Sec. 3.3.4), the intermediate ghost value of a link is the
 *       linear extrapolation 2 f_d - f_ac from its donor and auxiliary cell
 *       along the link axis, in place of Eq. extrapolation 1; the rest of the
 *       construction is unchanged.
 *   C26 optional (default off): a ghost value of Eq. extrapolation 2 below
 *       zero is set to zero.  The extrapolation from the shifted point
 *       through the wall value (up to threefold) can turn negative where the
 *       wall distribution is small, and a nearly empty donor cell in a
 *       strong expansion then loses positivity; a distribution function is
 *       nonnegative, and with nonnegative ghost values the limited upwind
 *       transport keeps it so.
 *   C24 a domain face may instead be a diffuse wall (Sec. 2.3 with alpha = 1
 *       on the plane of the face, normal into the domain): its two halo
 *       layers hold, for velocities entering the domain through the face,
 *       rho_w times the unit-density wall Maxwellian, and for the others the
 *       boundary cell's own value (so the outgoing face value is the cell
 *       value: the limiter sees a zero difference); rho_w makes the mass flux
 *       through the face zero with those face values.
 *
 *   C28 tree-refined physical grids (Sec. 4.2-4.4 use a tree-based AMR mesh
 *       and give no scheme for it): a root grid of equal cells, each leaf a
 *       square (2D, a quadtree) or cube (3D, an octree) of level l (edge
 *       h / 2^l), face neighbours at most one level apart (2:1).  Finite
 *       volumes on the leaves with the uniform grid's arithmetic: the van
 *       Leer slope of a cell along an axis from the value on each side (the
 *       neighbour's, the mean of the 2^(dim-1) finer neighbours', or the
 *       freestream halo) over the distance between centres along the axis
 *       ((h_c + h_n) / 2; h_c across the domain edge); the face value of the
 *       upwind cell f + s sigma h / 2; the inflow of a side with finer
 *       neighbours the mean of their face values (each covers an equal share
 *       of the side), so the flux through every interface is the same for
 *       both cells; one time step for all cells,
 *       C16 with the finest cell size.  On a tree of one level it is the
 *       uniform grid's step.
 *   C29 a body on a tree (Sec. 4.2-4.4 refine the mesh towards the wall):
 *       the body lies in the finest level, so its ghost band (ghost cells,
 *       donors, auxiliary cells and the cells beyond the donors, surface
 *       cells and their fluid neighbours) is the uniform grid's on the
 *       finest grid, and a fluid leaf next to a ghost sees the link's ghost
 *       value as that side's value (slope) and, when the ghost is upwind,
 *       the mean of the link value and its own value as the inflow (C14);
 *       a coarser leaf is all fluid or all solid; solid leaves keep their
 *       values and the residual runs over the fluid leaves.
 *
 * Parity unpinned: C4-C7, C9, C10, C14, C16-C19 and the first-order
 * outgoing face of C24 are choices the paper does not fix; they are pinned
 * only by agreement with an independent implementation, not by the paper.
 */
#include "ibdvm_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int g, d, ac;      /* ghost, donor and auxiliary cell (ac = -1 when unusable) */
  int axis, side;    /* side = sign of (x_d - x_g) along axis */
  double xw[3];      /* intersect point */
  double nw[3];      /* outward unit normal at the intersect point (into the gas) */
  double yg, yd, yw, ysp, yac; /* coordinates along the link axis */
} or_link;

typedef struct {
  int cell;
  int first_link, nlinks;
  int ns;        /* number of surface cells */
  int *surf;     /* surface cells */
} or_ghost;

struct or_case {
  or_params p;
  double *verts;
  int dim, ncomp;
  int n[3];
  double dx[3];
  long nc;
  int nvx[3];
  int nv;
  double *xi, *w, *blo, *bhi;
  double *f, *fnew;
  double *finf;
  unsigned char *type;
  int *ghost_of;
  int nlink, nghost;
  or_link *links;
  or_ghost *ghosts;
  double *wg;   /* incident-side measure per link and velocity */
  double *lval; /* ghost value f*_gc per link, velocity, component */
  double *wrho; /* rho_w of the diffuse domain faces of the state last given (C24), [cell][6] */
  int nthreads; /* host threads of the per-ghost and per-cell loops (1 by default) */
  int any_wall;
  double dt, mu0, Uinf[3];
};

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t s)
{
  void *q = calloc(n ? n : 1, s);
  if (!q) {
    fprintf(stderr, "oracle: out of memory\n");
    abort();
  }
  return q;
}

static void cell_ijk(const or_case *C, long c, int ijk[3])
{
  ijk[0] = (int)(c % C->n[0]);
  ijk[1] = (int)((c / C->n[0]) % C->n[1]);
  ijk[2] = (int)(c / ((long)C->n[0] * C->n[1]));
}

static long cell_index(const or_case *C, const int ijk[3])
{
  for (int a = 0; a < 3; ++a)
    if (ijk[a] < 0 || ijk[a] >= C->n[a]) return -1;
  return ijk[0] + (long)C->n[0] * (ijk[1] + (long)C->n[1] * ijk[2]);
}

/* cell centres about the domain centre, exactly mirror-symmetric (see axis_nodes) */
static void cell_centre(const or_case *C, long c, double x[3])
{
  int ijk[3];
  cell_ijk(C, c, ijk);
  for (int a = 0; a < 3; ++a) {
    if (a >= C->dim) {
      x[a] = 0.0;
      continue;
    }
    double ctr = 0.5 * (C->p.lo[a] + C->p.hi[a]), hw = 0.5 * (C->p.hi[a] - C->p.lo[a]);
    x[a] = ctr + (2 * ijk[a] + 1 - C->n[a]) * (hw / C->n[a]);
  }
}

/* neighbour across the face (axis a, side s); -1 outside the domain */
static long neighbour(const or_case *C, long c, int a, int s)
{
  int ijk[3];
  cell_ijk(C, c, ijk);
  ijk[a] += s;
  return cell_index(C, ijk);
}

static double *F(const or_case *C, double *f, long c, int k)
{
  return f + ((size_t)c * C->nv + k) * C->ncomp;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: VHS reference viscosity                                           */
/* ------------------------------------------------------------------------ */

double or_mu0(double Kn, double alpha, double omega)
{
  return 5.0 * (alpha + 1.0) * (alpha + 2.0) * sqrt(M_PI) /
         (4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega)) * Kn;
}

/* ------------------------------------------------------------------------ */
/* Eq. limiter: van Leer slope from the two one-sided slopes                 */
/* ------------------------------------------------------------------------ */

static double sgn(double v) { return (v > 0.0) - (v < 0.0); }

double or_vanleer(double s1, double s2)
{
  double a1 = fabs(s1), a2 = fabs(s2);
  if (a1 + a2 == 0.0) return 0.0;
  return (sgn(s1) + sgn(s2)) * a1 * a2 / (a1 + a2);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1 / Sec. 4: Maxwellian, Shakhov equilibrium, moments               */
/* ------------------------------------------------------------------------ */

/* Reduced (2D: H, B) or full (3D: g) Maxwellian at every velocity node. */
void or_maxwellian(const or_case *C, double rho, const double *U, double T, double *g)
{
  for (int k = 0; k < C->nv; ++k) {
    double c2 = 0.0;
    for (int a = 0; a < C->dim; ++a) {
      double c = C->xi[3 * k + a] - U[a];
      c2 += c * c;
    }
    if (C->dim == 2) {
      double H = rho / (M_PI * T) * exp(-c2 / T);
      g[2 * k + 0] = H;
      g[2 * k + 1] = 0.5 * T * H;
    } else {
      g[k] = rho / pow(M_PI * T, 1.5) * exp(-c2 / T);
    }
  }
}

/* Shakhov equilibrium: 2D reduced forms H^S, B^S of Sec. 4; in 3D the
   non-dimensional form of g^S of Sec. 2.1, bracket (2c^2/T - 5). */
void or_shakhov(const or_case *C, double rho, const double *U, double T, const double *q,
                double *gS)
{
  double Pr = C->p.Pr;
  or_maxwellian(C, rho, U, T, gS);
  for (int k = 0; k < C->nv; ++k) {
    double c2 = 0.0, cq = 0.0;
    for (int a = 0; a < C->dim; ++a) {
      double c = C->xi[3 * k + a] - U[a];
      c2 += c * c;
      cq += c * q[a];
    }
    double coef = 4.0 * (1.0 - Pr) / (5.0 * rho * T * T) * cq;
    if (C->dim == 2) {
      gS[2 * k + 0] *= 1.0 + coef * (2.0 * c2 / T - 4.0);
      gS[2 * k + 1] *= 1.0 + coef * (2.0 * c2 / T - 2.0);
    } else {
      gS[k] *= 1.0 + coef * (2.0 * c2 / T - 5.0);
    }
  }
}

/* Moments of one cell's distribution (Eqs. moments1-3 with the quadrature,
   2D reduced forms by integrating over xi_z).
   out = [rho, rhoU_0..rhoU_{D-1}, rhoE, T, p, q_0..q_{D-1}] */
void or_cell_moments(const or_case *C, const double *fc, double *out)
{
  int D = C->dim;
  double rho = 0.0, mom[3] = {0, 0, 0}, rhoE = 0.0;
  for (int k = 0; k < C->nv; ++k) {
    double w = C->w[k];
    double x2 = 0.0;
    for (int a = 0; a < D; ++a) x2 += C->xi[3 * k + a] * C->xi[3 * k + a];
    double h = fc[k * C->ncomp];
    rho += w * h;
    for (int a = 0; a < D; ++a) mom[a] += w * C->xi[3 * k + a] * h;
    if (D == 2)
      rhoE += 0.5 * w * (x2 * h + fc[k * 2 + 1]);
    else
      rhoE += 0.5 * w * x2 * h;
  }
  double U[3] = {0, 0, 0}, U2 = 0.0;
  for (int a = 0; a < D; ++a) {
    U[a] = mom[a] / rho;
    U2 += U[a] * U[a];
  }
  /* three translational degrees of freedom: rho e = 3/2 p, p = rho T / 2 */
  double T = 4.0 / 3.0 * (rhoE - 0.5 * rho * U2) / rho;
  double pr = 0.5 * rho * T;
  double q[3] = {0, 0, 0};
  for (int k = 0; k < C->nv; ++k) {
    double w = C->w[k];
    double c[3] = {0, 0, 0}, c2 = 0.0;
    for (int a = 0; a < D; ++a) {
      c[a] = C->xi[3 * k + a] - U[a];
      c2 += c[a] * c[a];
    }
    double h = fc[k * C->ncomp];
    double e = (D == 2) ? (c2 * h + fc[k * 2 + 1]) : c2 * h;
    for (int a = 0; a < D; ++a) q[a] += 0.5 * w * c[a] * e;
  }
  int i = 0;
  out[i++] = rho;
  for (int a = 0; a < D; ++a) out[i++] = mom[a];
  out[i++] = rhoE;
  out[i++] = T;
  out[i++] = pr;
  for (int a = 0; a < D; ++a) out[i++] = q[a];
}

/* ------------------------------------------------------------------------ */
/* Velocity grid (Eq. quadrature; dual boxes for the cut cells)              */
/* ------------------------------------------------------------------------ */

/* Nodes are written about the interval centre, c + m * (half width / M) with an
   integer m, so that a grid symmetric about zero is exactly antisymmetric in
   floating point (xi_{n-1-i} = -xi_i); the upwind-weight fallback and the
   incident/reflected split are decided by exact zeros that need this. */
static void axis_nodes(int n, double lo, double hi, int rule, const double *given, double *x, double *w,
                       double *bl, double *bh)
{
  double c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
  if (rule == 2) {
    /* given nodes: each owns the box between the midpoints to its neighbours */
    for (int i = 0; i < n; ++i) x[i] = given[i];
    for (int i = 0; i < n; ++i) {
      bl[i] = (i == 0) ? x[0] : 0.5 * (x[i - 1] + x[i]);
      bh[i] = (i == n - 1) ? x[n - 1] : 0.5 * (x[i] + x[i + 1]);
      w[i] = bh[i] - bl[i];
    }
  } else if (rule == 0) {
    double d = (hi - lo) / (n - 1);
    for (int i = 0; i < n; ++i) {
      x[i] = c + (2 * i - (n - 1)) * (hw / (n - 1));
      bl[i] = (i == 0) ? lo : x[i] - 0.5 * d;
      bh[i] = (i == n - 1) ? hi : x[i] + 0.5 * d;
      w[i] = bh[i] - bl[i];
    }
  } else {
    double d = (hi - lo) / n;
    for (int i = 0; i < n; ++i) {
      x[i] = c + (2 * i + 1 - n) * (hw / n);
      bl[i] = x[i] - 0.5 * d;
      bh[i] = x[i] + 0.5 * d;
      w[i] = d;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Body geometry: level set, intersect point, normal                         */
/* ------------------------------------------------------------------------ */

/* point-in-polygon by the crossing number (even-odd) */
static int polygon_inside(const or_case *C, const double *x)
{
  int nv = C->p.nverts, inside = 0;
  const double *v = C->verts;
  for (int i = 0, j = nv - 1; i < nv; j = i++) {
    double xi = v[2 * i], yi = v[2 * i + 1], xj = v[2 * j], yj = v[2 * j + 1];
    if ((yi > x[1]) != (yj > x[1])) {
      double xc = xj + (x[1] - yj) * (xi - xj) / (yi - yj);
      if (x[0] < xc) inside = !inside;
    }
  }
  return inside;
}

/* level-set value: <= 0 inside the body or on its surface */
static double level(const or_case *C, const double *x)
{
  const or_params *p = &C->p;
  switch (p->kind) {
  case OR_BODY_CIRCLE:
  case OR_BODY_SPHERE: {
    double s = 0.0;
    for (int a = 0; a < C->dim; ++a) s += (x[a] - p->center[a]) * (x[a] - p->center[a]);
    return s - p->radii[0] * p->radii[0];
  }
  case OR_BODY_ELLIPSE: {
    double dx = x[0] - p->center[0], dy = x[1] - p->center[1];
    double ca = cos(p->angle), sa = sin(p->angle);
    double u = ca * dx + sa * dy, v = -sa * dx + ca * dy;
    return (u / p->radii[0]) * (u / p->radii[0]) + (v / p->radii[1]) * (v / p->radii[1]) - 1.0;
  }
  case OR_BODY_POLYGON:
    return polygon_inside(C, x) ? -1.0 : 1.0;
  case OR_BODY_HALFSPACE: {
    double s = 0.0;
    for (int a = 0; a < C->dim; ++a) s += (x[a] - p->center[a]) * p->radii[a];
    return s;
  }
  default:
    return 1.0;
  }
}

/* intersect point on the segment from xg (solid) to xd (gas), and the normal */
static void intersect(const or_case *C, const double *xg, const double *xd, double *xw,
                      double *nw)
{
  const or_params *p = &C->p;
  int D = C->dim;
  if (p->kind == OR_BODY_POLYGON) {
    /* every polygon edge crossed by the segment; keep the crossing nearest the donor (C5) */
    double best_t = -1.0, best_u = 0.0;
    int best_e = -1;
    int nv = p->nverts;
    for (int e = 0; e < nv; ++e) {
      const double *A = C->verts + 2 * e, *B = C->verts + 2 * ((e + 1) % nv);
      double rx = xd[0] - xg[0], ry = xd[1] - xg[1];
      double sx = B[0] - A[0], sy = B[1] - A[1];
      double den = rx * sy - ry * sx;
      if (den == 0.0) continue;
      double qx = A[0] - xg[0], qy = A[1] - xg[1];
      double t = (qx * sy - qy * sx) / den; /* along the segment */
      double u = (qx * ry - qy * rx) / den; /* along the edge */
      if (t < 0.0 || t > 1.0 || u < 0.0 || u > 1.0) continue;
      if (t > best_t) {
        best_t = t;
        best_u = u;
        best_e = e;
      }
    }
    if (best_e < 0) { /* numerically grazing: fall back to the ghost centre */
      best_t = 0.0;
      best_e = 0;
      best_u = 0.5;
    }
    for (int a = 0; a < 3; ++a) xw[a] = xg[a] + best_t * (xd[a] - xg[a]);
    /* outward normal of a counter-clockwise polygon edge A->B is (dy, -dx) */
    int e0 = best_e, e1 = best_e;
    if (best_u < 1e-9) e0 = (best_e + nv - 1) % nv;     /* vertex at A: with previous edge */
    if (best_u > 1.0 - 1e-9) e1 = (best_e + 1) % nv;    /* vertex at B: with next edge */
    double nx = 0.0, ny = 0.0;
    int es[2] = {e0, e1};
    int ne = (e0 == e1) ? 1 : 2;
    for (int q = 0; q < ne; ++q) {
      const double *A = C->verts + 2 * es[q], *B = C->verts + 2 * ((es[q] + 1) % nv);
      double dx = B[0] - A[0], dy = B[1] - A[1], len = sqrt(dx * dx + dy * dy);
      nx += dy / len;
      ny += -dx / len;
    }
    double len = sqrt(nx * nx + ny * ny);
    nw[0] = nx / len;
    nw[1] = ny / len;
    nw[2] = 0.0;
    return;
  }
  /* smooth bodies: bisection of the level set to machine precision */
  double tl = 0.0, th = 1.0;
  for (int it = 0; it < 200; ++it) {
    double tm = 0.5 * (tl + th);
    if (tm <= tl || tm >= th) break;
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = xg[a] + tm * (xd[a] - xg[a]);
    if (level(C, x) <= 0.0)
      tl = tm;
    else
      th = tm;
  }
  double t = 0.5 * (tl + th);
  for (int a = 0; a < 3; ++a) xw[a] = xg[a] + t * (xd[a] - xg[a]);
  double n[3] = {0, 0, 0};
  if (p->kind == OR_BODY_CIRCLE || p->kind == OR_BODY_SPHERE) {
    for (int a = 0; a < D; ++a) n[a] = xw[a] - p->center[a];
  } else if (p->kind == OR_BODY_ELLIPSE) {
    double dx = xw[0] - p->center[0], dy = xw[1] - p->center[1];
    double ca = cos(p->angle), sa = sin(p->angle);
    double u = ca * dx + sa * dy, v = -sa * dx + ca * dy;
    double gu = u / (p->radii[0] * p->radii[0]), gv = v / (p->radii[1] * p->radii[1]);
    n[0] = ca * gu - sa * gv;
    n[1] = sa * gu + ca * gv;
  } else {
    for (int a = 0; a < D; ++a) n[a] = p->radii[a];
  }
  double len = 0.0;
  for (int a = 0; a < D; ++a) len += n[a] * n[a];
  len = sqrt(len);
  for (int a = 0; a < 3; ++a) nw[a] = (a < D) ? n[a] / len : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Velocity-space cut cells (Sec. 3.2.3): measure of box ∩ {xi.n <= 0}       */
/* ------------------------------------------------------------------------ */

/* 2D: clip the rectangle by the half plane (Sutherland-Hodgman) and take the
   polygon area by the shoelace formula. */
double or_cut_fraction_2d(const double *blo, const double *bhi, const double *n)
{
  double px[8], py[8], qx[8], qy[8];
  int np = 4, nq = 0;
  px[0] = blo[0]; py[0] = blo[1];
  px[1] = bhi[0]; py[1] = blo[1];
  px[2] = bhi[0]; py[2] = bhi[1];
  px[3] = blo[0]; py[3] = bhi[1];
  for (int i = 0; i < np; ++i) {
    int j = (i + 1) % np;
    double si = n[0] * px[i] + n[1] * py[i];
    double sj = n[0] * px[j] + n[1] * py[j];
    if (si <= 0.0) {
      qx[nq] = px[i];
      qy[nq] = py[i];
      ++nq;
    }
    if ((si <= 0.0) != (sj <= 0.0)) {
      double t = si / (si - sj);
      qx[nq] = px[i] + t * (px[j] - px[i]);
      qy[nq] = py[i] + t * (py[j] - py[i]);
      ++nq;
    }
  }
  double A = 0.0;
  for (int i = 0; i < nq; ++i) {
    int j = (i + 1) % nq;
    A += qx[i] * qy[j] - qx[j] * qy[i];
  }
  return 0.5 * fabs(A);
}

/* 3D: the area of the slice at height z is piecewise quadratic in z with
   breaks where the plane passes a box corner; integrate each piece with the
   three-point Gauss-Legendre rule (exact for quadratics). */
double or_cut_fraction_3d(const double *blo, const double *bhi, const double *n)
{
  double br[10];
  int nb = 0;
  br[nb++] = blo[2];
  br[nb++] = bhi[2];
  if (n[2] != 0.0) {
    for (int ix = 0; ix < 2; ++ix)
      for (int iy = 0; iy < 2; ++iy) {
        double x = ix ? bhi[0] : blo[0], y = iy ? bhi[1] : blo[1];
        double z = -(n[0] * x + n[1] * y) / n[2];
        if (z > blo[2] && z < bhi[2]) br[nb++] = z;
      }
  }
  /* sort the break points */
  for (int i = 1; i < nb; ++i)
    for (int j = i; j > 0 && br[j - 1] > br[j]; --j) {
      double t = br[j];
      br[j] = br[j - 1];
      br[j - 1] = t;
    }
  static const double gx[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};
  static const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  double V = 0.0;
  for (int s = 0; s + 1 < nb; ++s) {
    double z0 = br[s], z1 = br[s + 1];
    if (z1 <= z0) continue;
    for (int g = 0; g < 3; ++g) {
      double z = 0.5 * (z0 + z1) + 0.5 * (z1 - z0) * gx[g];
      /* slice: {(x,y) in rect : n0 x + n1 y + n2 z <= 0}; shift the plane */
      double lo2[2] = {blo[0], blo[1]}, hi2[2] = {bhi[0], bhi[1]};
      double area;
      /* half plane n0 x + n1 y <= -n2 z: translate so it passes the origin */
      double nn = n[0] * n[0] + n[1] * n[1];
      if (nn == 0.0) {
        area = (n[2] * z <= 0.0) ? (bhi[0] - blo[0]) * (bhi[1] - blo[1]) : 0.0;
      } else {
        double sh = -n[2] * z / nn; /* point sh*(n0,n1) lies on the line */
        double l2[2] = {lo2[0] - sh * n[0], lo2[1] - sh * n[1]};
        double h2[2] = {hi2[0] - sh * n[0], hi2[1] - sh * n[1]};
        double n2[2] = {n[0], n[1]};
        area = or_cut_fraction_2d(l2, h2, n2);
      }
      V += 0.5 * (z1 - z0) * gw[g] * area;
    }
  }
  return V;
}

static double cut_measure(const or_case *C, int k, const double *nw)
{
  if (C->dim == 2) return or_cut_fraction_2d(C->blo + 3 * k, C->bhi + 3 * k, nw);
  return or_cut_fraction_3d(C->blo + 3 * k, C->bhi + 3 * k, nw);
}

/* ------------------------------------------------------------------------ */
/* Case construction: grids, classification (Sec. 3.2.1), links, cut table   */
/* ------------------------------------------------------------------------ */

or_case *or_create(const or_params *p)
{
  or_case *C = (or_case *)xcalloc(1, sizeof(or_case));
  C->p = *p;
  C->nthreads = 1;
  if (p->kind == OR_BODY_POLYGON && p->nverts > 0) {
    C->verts = (double *)xcalloc(2 * p->nverts, sizeof(double));
    memcpy(C->verts, p->verts, sizeof(double) * 2 * p->nverts);
  }
  C->p.verts = C->verts;
  int D = C->dim = p->dim;
  C->ncomp = (D == 2) ? 2 : 1;
  C->nc = 1;
  C->nv = 1;
  for (int a = 0; a < 3; ++a) {
    C->n[a] = (a < D) ? p->n[a] : 1;
    C->dx[a] = (a < D) ? (p->hi[a] - p->lo[a]) / p->n[a] : 1.0;
    C->nvx[a] = (a < D) ? p->nv[a] : 1;
    C->nc *= C->n[a];
    C->nv *= C->nvx[a];
  }
  /* velocity nodes and weights: tensor product of the per-axis rule */
  double *ax[3], *aw[3], *al[3], *ah[3];
  for (int a = 0; a < 3; ++a) {
    int m = C->nvx[a];
    ax[a] = (double *)xcalloc(m, sizeof(double));
    aw[a] = (double *)xcalloc(m, sizeof(double));
    al[a] = (double *)xcalloc(m, sizeof(double));
    ah[a] = (double *)xcalloc(m, sizeof(double));
    if (a < D)
      axis_nodes(m, p->vlo[a], p->vhi[a], p->rule, p->vnodes[a], ax[a], aw[a], al[a], ah[a]);
    else {
      ax[a][0] = 0.0;
      aw[a][0] = 1.0;
      al[a][0] = 0.0;
      ah[a][0] = 0.0;
    }
  }
  C->xi = (double *)xcalloc(3 * C->nv, sizeof(double));
  C->w = (double *)xcalloc(C->nv, sizeof(double));
  C->blo = (double *)xcalloc(3 * C->nv, sizeof(double));
  C->bhi = (double *)xcalloc(3 * C->nv, sizeof(double));
  for (int iz = 0; iz < C->nvx[2]; ++iz)
    for (int iy = 0; iy < C->nvx[1]; ++iy)
      for (int ix = 0; ix < C->nvx[0]; ++ix) {
        int k = ix + C->nvx[0] * (iy + C->nvx[1] * iz);
        int id[3] = {ix, iy, iz};
        C->w[k] = 1.0;
        for (int a = 0; a < 3; ++a) {
          C->xi[3 * k + a] = ax[a][id[a]];
          C->blo[3 * k + a] = al[a][id[a]];
          C->bhi[3 * k + a] = ah[a][id[a]];
          C->w[k] *= aw[a][id[a]];
        }
      }
  for (int a = 0; a < 3; ++a) {
    free(ax[a]);
    free(aw[a]);
    free(al[a]);
    free(ah[a]);
  }

  /* gas constants (Sec. 4) */
  C->mu0 = or_mu0(p->Kn, p->alpha_vhs, p->omega_vhs);
  double dn = 0.0;
  for (int a = 0; a < D; ++a) dn += p->dir[a] * p->dir[a];
  dn = sqrt(dn);
  double Uinf = p->Ma * sqrt(p->gamma * p->T_inf / 2.0);
  for (int a = 0; a < 3; ++a) C->Uinf[a] = (a < D && dn > 0.0) ? Uinf * p->dir[a] / dn : 0.0;
  if (p->dt > 0.0) {
    C->dt = p->dt;
  } else {
    double s = 0.0;
    for (int a = 0; a < D; ++a) {
      double m = 0.0;
      for (int k = 0; k < C->nv; ++k) m = fmax(m, fabs(C->xi[3 * k + a]));
      s += m / C->dx[a];
    }
    C->dt = p->cfl / s;
  }

  /* freestream and initial condition */
  C->finf = (double *)xcalloc((size_t)C->nv * C->ncomp, sizeof(double));
  or_maxwellian(C, p->rho_inf, C->Uinf, p->T_inf, C->finf);
  size_t nf = (size_t)C->nc * C->nv * C->ncomp;
  C->f = (double *)xcalloc(nf, sizeof(double));
  C->fnew = (double *)xcalloc(nf, sizeof(double));
  for (long c = 0; c < C->nc; ++c)
    memcpy(C->f + (size_t)c * C->nv * C->ncomp, C->finf, sizeof(double) * C->nv * C->ncomp);

  /* classification: solid iff the centre is inside or on the body (C3) */
  C->type = (unsigned char *)xcalloc(C->nc, 1);
  for (long c = 0; c < C->nc; ++c) {
    double x[3];
    cell_centre(C, c, x);
    C->type[c] = (p->kind != OR_BODY_NONE && level(C, x) <= 0.0) ? OR_SOLID : OR_FLUID;
  }
  /* ghost: solid with a fluid face neighbour */
  for (long c = 0; c < C->nc; ++c) {
    if (C->type[c] != OR_SOLID) continue;
    int is_ghost = 0;
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        long nb = neighbour(C, c, a, s);
        if (nb >= 0 && C->type[nb] == OR_FLUID) is_ghost = 1;
      }
    if (is_ghost) C->type[c] = OR_GHOST;
  }
  C->ghost_of = (int *)xcalloc(C->nc, sizeof(int));
  int ng = 0, nl = 0;
  for (long c = 0; c < C->nc; ++c) {
    C->ghost_of[c] = -1;
    if (C->type[c] != OR_GHOST) continue;
    C->ghost_of[c] = ng++;
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        long nb = neighbour(C, c, a, s);
        if (nb >= 0 && C->type[nb] == OR_FLUID) ++nl;
      }
  }
  C->nghost = ng;
  C->nlink = nl;
  C->ghosts = (or_ghost *)xcalloc(ng, sizeof(or_ghost));
  C->links = (or_link *)xcalloc(nl, sizeof(or_link));
  int gi = 0, li = 0;
  for (long c = 0; c < C->nc; ++c) {
    if (C->type[c] != OR_GHOST) continue;
    or_ghost *G = &C->ghosts[gi++];
    G->cell = (int)c;
    G->first_link = li;
    double xg[3];
    cell_centre(C, c, xg);
    /* links, canonical order: direction 2*axis + (side > 0) */
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        long d = neighbour(C, c, a, s);
        if (d < 0 || C->type[d] != OR_FLUID) continue;
        or_link *L = &C->links[li++];
        L->g = (int)c;
        L->d = (int)d;
        L->axis = a;
        L->side = s;
        double xd[3];
        cell_centre(C, d, xd);
        intersect(C, xg, xd, L->xw, L->nw);
        long ac = neighbour(C, d, a, s);
        L->ac = (ac >= 0 && C->type[ac] == OR_FLUID) ? (int)ac : -1; /* C7 */
        L->yg = xg[a];
        L->yd = xd[a];
        L->yw = L->xw[a];
        L->ysp = L->yw + 0.5 * (L->yd - L->yg); /* Eq. sp */
        L->yac = L->yd + s * C->dx[a];
      }
    G->nlinks = li - G->first_link;
    /* surface cells: fluid cells among the 3^D - 1 face/edge/corner neighbours */
    int ijk[3];
    cell_ijk(C, c, ijk);
    int tmp[27], ns = 0;
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (!ox && !oy && !oz) continue;
          int q[3] = {ijk[0] + ox, ijk[1] + oy, ijk[2] + oz};
          long j = cell_index(C, q);
          if (j >= 0 && C->type[j] == OR_FLUID) tmp[ns++] = (int)j;
        }
    G->ns = ns;
    G->surf = (int *)xcalloc(ns, sizeof(int));
    memcpy(G->surf, tmp, sizeof(int) * ns);
  }

  /* incident-side measure per link and velocity (Sec. 3.2.3) */
  C->wg = (double *)xcalloc((size_t)nl * C->nv, sizeof(double));
  for (int l = 0; l < nl; ++l) {
    const double *nw = C->links[l].nw;
    for (int k = 0; k < C->nv; ++k) {
      double xn = 0.0;
      for (int a = 0; a < D; ++a) xn += C->xi[3 * k + a] * nw[a];
      double wg;
      if (C->p.cutcell) {
        /* corner test: the plane cuts the box iff the corners lie on both sides */
        int below = 0, above = 0;
        for (int corner = 0; corner < (1 << D); ++corner) {
          double s = 0.0;
          for (int a = 0; a < D; ++a)
            s += ((corner >> a) & 1 ? C->bhi[3 * k + a] : C->blo[3 * k + a]) * nw[a];
          if (s < 0.0) below = 1;
          if (s > 0.0) above = 1;
        }
        if (below && above)
          wg = cut_measure(C, k, nw);
        else
          wg = (xn <= 0.0) ? C->w[k] : 0.0;
      } else {
        wg = (xn <= 0.0) ? C->w[k] : 0.0;
      }
      C->wg[(size_t)l * C->nv + k] = wg;
    }
  }
  C->lval = (double *)xcalloc((size_t)nl * C->nv * C->ncomp, sizeof(double));
  C->wrho = (double *)xcalloc((size_t)C->nc * 6, sizeof(double));
  for (int i = 0; i < 2 * C->dim; ++i) C->any_wall |= (p->wall[i] != 0);
  return C;
}

void or_set_threads(or_case *C, int nthreads) { C->nthreads = nthreads > 0 ? nthreads : 1; }

void or_destroy(or_case *C)
{
  if (!C) return;
  for (int g = 0; g < C->nghost; ++g) free(C->ghosts[g].surf);
  free(C->ghosts);
  free(C->links);
  free(C->verts);
  free(C->xi);
  free(C->w);
  free(C->blo);
  free(C->bhi);
  free(C->f);
  free(C->fnew);
  free(C->finf);
  free(C->type);
  free(C->ghost_of);
  free(C->wg);
  free(C->lval);
  free(C->wrho);
  free(C);
}

/* ------------------------------------------------------------------------ */
/* the domain halo: freestream (C17) or diffuse walls (C24)                  */
/* ------------------------------------------------------------------------ */

/* unit-density Maxwellian of domain face i at velocity node k, component m */
static double wall_maxwellian(const or_case *C, int i, int k, int m)
{
  double T = C->p.wall_T[i], c2 = 0.0;
  for (int a = 0; a < C->dim; ++a) {
    double c = C->xi[3 * k + a] - C->p.wall_U[i][a];
    c2 += c * c;
  }
  if (C->dim == 2) {
    double H = exp(-c2 / T) / (M_PI * T);
    return (m == 0) ? H : 0.5 * T * H;
  }
  return exp(-c2 / T) / pow(M_PI * T, 1.5);
}

/* rho_w of every diffuse domain face of fluid cells for the state f: the
   mass flux out of the domain through the face, carried by the cell's own
   value, is returned by rho_w times the wall Maxwellian (Eq. dnpc on the
   face, incident set s xi_a > 0) */
static void domain_walls(const or_case *C, const double *f)
{
  if (!C->any_wall) return;
  for (long c = 0; c < C->nc; ++c) {
    for (int i = 0; i < 6; ++i) C->wrho[c * 6 + i] = 0.0;
    if (C->type[c] != OR_FLUID) continue;
    for (int a = 0; a < C->dim; ++a)
      for (int s = -1; s <= 1; s += 2) {
        int i = 2 * a + (s > 0);
        if (!C->p.wall[i] || neighbour(C, c, a, s) >= 0) continue;
        double out = 0.0, in = 0.0;
        for (int k = 0; k < C->nv; ++k) {
          double xs = s * C->xi[3 * k + a];
          if (xs > 0.0)
            out += C->w[k] * xs * F(C, (double *)f, c, k)[0];
          else if (xs < 0.0)
            in += C->w[k] * xs * wall_maxwellian(C, i, k, 0);
        }
        C->wrho[c * 6 + i] = -out / in;
      }
  }
}

void or_domain_wall_density(const or_case *C, const double *f, double *out)
{
  domain_walls(C, f);
  for (long i = 0; i < C->nc * 6; ++i) out[i] = C->any_wall ? C->wrho[i] : 0.0;
}

/* value of the halo cells across domain face (a, s) of cell c (both layers
   hold the same value); domain_walls has been run on f */
static double halo_value(const or_case *C, const double *f, long c, int a, int s, int k, int m)
{
  int i = 2 * a + (s > 0);
  if (!C->p.wall[i]) return C->finf[k * C->ncomp + m];
  if (s * C->xi[3 * k + a] < 0.0) return C->wrho[c * 6 + i] * wall_maxwellian(C, i, k, m);
  return F(C, (double *)f, c, k)[m];
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.1-3.2.3: the ghost band                                          */
/* ------------------------------------------------------------------------ */

/* pre-ghost slope of a surface cell along axis a (C9): fluid and halo
   neighbours only */
static double preghost_slope(const or_case *C, const double *f, long j, int a, int k, int m)
{
  double fj = F(C, (double *)f, j, k)[m];
  long jm = neighbour(C, j, a, -1), jp = neighbour(C, j, a, +1);
  int have_m = (jm < 0) || C->type[jm] == OR_FLUID;
  int have_p = (jp < 0) || C->type[jp] == OR_FLUID;
  double fm = (jm < 0) ? halo_value(C, f, j, a, -1, k, m) : (have_m ? F(C, (double *)f, jm, k)[m] : 0.0);
  double fp = (jp < 0) ? halo_value(C, f, j, a, +1, k, m) : (have_p ? F(C, (double *)f, jp, k)[m] : 0.0);
  double h = C->dx[a];
  if (have_m && have_p) return or_vanleer((fj - fm) / h, (fp - fj) / h);
  if (have_m) return (fj - fm) / h;
  if (have_p) return (fp - fj) / h;
  return 0.0;
}

/* the weights of Eq. upwind for velocity k over the surface cells of ghost
   G: max(0, xi_k . r_j / |r_j|)^2 normalised to a unit sum, or 1 / N_S when
   they all vanish (the text after Eq. upwind); 1 / N_S for every velocity
   without upwind weighting */
static void upwind_weights(const or_case *C, const or_ghost *G, int k, double *wt)
{
  int ig[3];
  cell_ijk(C, G->cell, ig);
  double wsum = 0.0;
  for (int j = 0; j < G->ns; ++j) {
    /* r from the integer cell offset times the spacing, so that velocities
       tangent to r give an exact zero */
    int ij[3];
    cell_ijk(C, G->surf[j], ij);
    double r[3], rl = 0.0;
    for (int a = 0; a < C->dim; ++a) {
      int o = (C->p.upwind == 2) ? (ij[a] - ig[a]) : (ig[a] - ij[a]);
      r[a] = o * C->dx[a];
      rl += r[a] * r[a];
    }
    rl = sqrt(rl);
    double dot = 0.0;
    for (int a = 0; a < C->dim; ++a) dot += C->xi[3 * k + a] * r[a] / rl;
    double mx = dot > 0.0 ? dot : 0.0;
    wt[j] = (C->p.upwind == 0) ? 0.0 : mx * mx;
    wsum += wt[j];
  }
  for (int j = 0; j < G->ns; ++j) wt[j] = (wsum != 0.0) ? wt[j] / wsum : 1.0 / G->ns;
}

void or_upwind_weights(const or_case *C, int gi, double *out)
{
  const or_ghost *G = &C->ghosts[gi];
  double wt[27];
  for (int k = 0; k < C->nv; ++k) {
    upwind_weights(C, G, k, wt);
    for (int j = 0; j < G->ns; ++j) out[(size_t)j * C->nv + k] = wt[j];
  }
}

/* f_gc of Eq. extrapolation 1 with the weights of Eq. upwind */
static double ghost_interp(const or_case *C, const double *f, const or_ghost *G, int k, int m)
{
  int ig[3];
  cell_ijk(C, G->cell, ig);
  double wt[27];
  upwind_weights(C, G, k, wt);
  double fgc = 0.0;
  for (int j = 0; j < G->ns; ++j) {
    long jc = G->surf[j];
    int ij[3];
    cell_ijk(C, jc, ij);
    /* f_j - sigma_j . r_j with r_j = x_j - x_g */
    double v = F(C, (double *)f, jc, k)[m];
    for (int a = 0; a < C->dim; ++a) {
      double ra = (ij[a] - ig[a]) * C->dx[a];
      if (ra != 0.0) v -= preghost_slope(C, f, jc, a, k, m) * ra;
    }
    fgc += wt[j] * v;
  }
  return fgc;
}

/* value of f^i_w at an arbitrary velocity by multilinear interpolation on the
   node grid, zero outside it (C13) */
static double interp_velocity(const or_case *C, const double *fi, const double *xq, int m)
{
  int D = C->dim;
  int i0[3] = {0, 0, 0};
  double t[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    int na = C->nvx[a];
    int stride = (a == 0) ? 1 : (a == 1 ? C->nvx[0] : C->nvx[0] * C->nvx[1]);
    double x0 = C->xi[3 * 0 + a];
    double x1 = C->xi[3 * ((na - 1) * stride) + a];
    if (xq[a] < x0 || xq[a] > x1) return 0.0;
    if (C->p.rule == 2) {
      /* non-uniform nodes (C25): the bracketing interval by bisection */
      int lo = 0, hi = na - 1;
      while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (C->xi[3 * (mid * stride) + a] <= xq[a])
          lo = mid;
        else
          hi = mid;
      }
      double xl = C->xi[3 * (lo * stride) + a], xh = C->xi[3 * (hi * stride) + a];
      i0[a] = lo;
      t[a] = (xq[a] - xl) / (xh - xl);
      continue;
    }
    double d = (na > 1) ? (x1 - x0) / (na - 1) : 1.0;
    double u = (xq[a] - x0) / d;
    int i = (int)floor(u);
    if (i >= na - 1) i = na - 2;
    if (i < 0) i = 0;
    i0[a] = i;
    t[a] = u - i;
  }
  double v = 0.0;
  for (int corner = 0; corner < (1 << D); ++corner) {
    double wt = 1.0;
    int id[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      int b = (corner >> a) & 1;
      id[a] = i0[a] + b;
      wt *= b ? t[a] : 1.0 - t[a];
    }
    int k = id[0] + C->nvx[0] * (id[1] + C->nvx[1] * id[2]);
    v += wt * fi[k * C->ncomp + m];
  }
  return v;
}

void or_ghost_band(const or_case *C, const double *f, double *fgc_out, double *fsp_out,
                   double *fiw_out, double *fstarw_out, double *fstargc_out, double *rhow_out)
{
  int D = C->dim, nv = C->nv, nc = C->ncomp;
  double alpha = C->p.accom;
  domain_walls(C, f); /* the halo values the pre-ghost slopes see */
  /* ghosts are independent of each other: every ghost writes only its own
     links, so the result does not depend on the number of threads */
#pragma omp parallel num_threads(C->nthreads)
  {
  double *fgc = (double *)xcalloc((size_t)nv * nc, sizeof(double));
  double *fsp = (double *)xcalloc((size_t)nv * nc, sizeof(double));
  double *fi = (double *)xcalloc((size_t)nv * nc, sizeof(double));
  double *fs = (double *)xcalloc((size_t)nv * nc, sizeof(double));
  double *Gw = (double *)xcalloc((size_t)nv * nc, sizeof(double));
#pragma omp for schedule(dynamic)
  for (int gi = 0; gi < C->nghost; ++gi) {
    const or_ghost *G = &C->ghosts[gi];
    /* step 2: intermediate ghost value f_gc (shared by the ghost's links) */
    if (C->p.upwind != 3)
      for (int k = 0; k < nv; ++k)
        for (int m = 0; m < nc; ++m) fgc[k * nc + m] = ghost_interp(C, f, G, k, m);
    for (int l = G->first_link; l < G->first_link + G->nlinks; ++l) {
      const or_link *L = &C->links[l];
      if (C->p.upwind == 3)
        /* the construction without upwind weighting (Sec. 3.3.4): the ghost
           value extrapolated linearly from the donor and the auxiliary cell
           along the link axis, f_g = 2 f_d - f_ac (f_d without an auxiliary
           cell, as C7) */
        for (int k = 0; k < nv; ++k)
          for (int m = 0; m < nc; ++m) {
            double fd = F(C, (double *)f, L->d, k)[m];
            fgc[k * nc + m] = (L->ac >= 0) ? 2.0 * fd - F(C, (double *)f, L->ac, k)[m] : fd;
          }
      /* step 1: shifted point, Eq. fsp with the auxiliary-cell slope */
      for (int k = 0; k < nv; ++k)
        for (int m = 0; m < nc; ++m) {
          double fd = F(C, (double *)f, L->d, k)[m];
          double sig = 0.0;
          if (L->ac >= 0) sig = (F(C, (double *)f, L->ac, k)[m] - fd) / (L->yac - L->yd);
          fsp[k * nc + m] = fd + sig * (L->ysp - L->yd);
        }
      /* step 3: incident distribution at the intersect point, Eq. fw */
      for (int k = 0; k < nv * nc; ++k)
        fi[k] = fsp[k] + (fgc[k] - fsp[k]) / (L->yg - L->ysp) * (L->yw - L->ysp);
      /* wall Maxwellian of unit density, Eq. boundary maxwell (reduced in 2D) */
      double Uw[3] = {C->p.Uw[0], C->p.Uw[1], C->p.Uw[2]};
      or_maxwellian(C, 1.0, Uw, C->p.Tw, Gw);
      /* specular part: f^i at the mirrored velocity (C13) */
      for (int k = 0; k < nv; ++k) {
        double xn = 0.0;
        for (int a = 0; a < D; ++a) xn += C->xi[3 * k + a] * L->nw[a];
        double xm[3];
        for (int a = 0; a < D; ++a) xm[a] = C->xi[3 * k + a] - 2.0 * xn * L->nw[a];
        for (int m = 0; m < nc; ++m) fs[k * nc + m] = (alpha < 1.0) ? interp_velocity(C, fi, xm, m) : 0.0;
      }
      /* wall density from zero net normal mass flux with the cut-cell split, Eq. rhowc */
      double Nsum = 0.0, Dsum = 0.0, Ssum = 0.0;
      for (int k = 0; k < nv; ++k) {
        double xn = 0.0;
        for (int a = 0; a < D; ++a) xn += C->xi[3 * k + a] * L->nw[a];
        double wg = C->wg[(size_t)l * nv + k];
        double ws = C->w[k] - wg;
        Nsum += wg * xn * fi[k * nc];
        Dsum += ws * xn * Gw[k * nc];
        Ssum += ws * xn * fs[k * nc];
      }
      double rhow = (alpha > 0.0) ? -(Nsum + (1.0 - alpha) * Ssum) / (alpha * Dsum) : 0.0;
      /* wall distribution (Eqs. general bc, Maxwell BC, fwc) and ghost value (Eq. extrapolation 2) */
      for (int k = 0; k < nv; ++k) {
        double wg = C->wg[(size_t)l * nv + k];
        double ws = C->w[k] - wg;
        for (int m = 0; m < nc; ++m) {
          int i = k * nc + m;
          double fr = alpha * rhow * Gw[i] + (1.0 - alpha) * fs[i];
          double fstar = (C->w[k] > 0.0) ? (wg * fi[i] + ws * fr) / C->w[k] : fi[i];
          double fgs = fsp[i] + (fstar - fsp[i]) / (L->yw - L->ysp) * (L->yg - L->ysp);
          if (C->p.ghost_nonneg && fgs < 0.0) fgs = 0.0; /* C26 */
          size_t o = ((size_t)l * nv + k) * nc + m;
          if (fgc_out) fgc_out[o] = fgc[i];
          if (fsp_out) fsp_out[o] = fsp[i];
          if (fiw_out) fiw_out[o] = fi[i];
          if (fstarw_out) fstarw_out[o] = fstar;
          if (fstargc_out) fstargc_out[o] = fgs;
        }
      }
      if (rhow_out) rhow_out[l] = rhow;
    }
  }
  free(fgc);
  free(fsp);
  free(fi);
  free(fs);
  free(Gw);
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: slopes, face values and the forward-Euler update                */
/* ------------------------------------------------------------------------ */

static int find_link(const or_case *C, long g, long d)
{
  const or_ghost *G = &C->ghosts[C->ghost_of[g]];
  for (int l = G->first_link; l < G->first_link + G->nlinks; ++l)
    if (C->links[l].d == d) return l;
  return -1;
}

/* value of the cell across face (a, s) of fluid cell c as this cell sees it:
   halo -> freestream (C17) or diffuse wall (C24); ghost -> the link's ghost
   value (C4) */
static double seen_value(const or_case *C, const double *f, long c, int a, int s, int k, int m)
{
  long nb = neighbour(C, c, a, s);
  if (nb < 0) return halo_value(C, f, c, a, s, k, m);
  if (C->type[nb] == OR_FLUID) return F(C, (double *)f, nb, k)[m];
  int l = find_link(C, nb, c);
  return C->lval[((size_t)l * C->nv + k) * C->ncomp + m];
}

/* van Leer slope of a fluid cell along axis a (Eq. limiter) */
static double fluid_slope(const or_case *C, const double *f, long c, int a, int k, int m)
{
  double h = C->dx[a];
  double fc = F(C, (double *)f, c, k)[m];
  double fm = seen_value(C, f, c, a, -1, k, m);
  double fp = seen_value(C, f, c, a, +1, k, m);
  return or_vanleer((fc - fm) / h, (fp - fc) / h);
}

/* reconstructed value on face (a, s) of fluid cell c, Eq. reconstruction */
static double face_value(const or_case *C, const double *f, long c, int a, int s, int k, int m)
{
  double xia = C->xi[3 * k + a];
  double h = C->dx[a];
  double fc = F(C, (double *)f, c, k)[m];
  if (xia * s > 0.0) /* the particle leaves c through this face: c is upwind */
    return fc + fluid_slope(C, f, c, a, k, m) * (s * 0.5 * h);
  long nb = neighbour(C, c, a, s);
  if (nb < 0) {
    /* halo cell: its neighbours are the next halo cell and c */
    double fh = halo_value(C, f, c, a, s, k, m);
    double sig;
    if (s > 0) /* left neighbour c, right neighbour the next halo cell */
      sig = or_vanleer((fh - fc) / h, (fh - fh) / h);
    else /* left neighbour the next halo cell, right neighbour c */
      sig = or_vanleer((fh - fh) / h, (fc - fh) / h);
    return fh + sig * (-s * 0.5 * h);
  }
  if (C->type[nb] == OR_FLUID) return F(C, (double *)f, nb, k)[m] + fluid_slope(C, f, nb, a, k, m) * (-s * 0.5 * h);
  /* ghost neighbour: link value with the one-sided slope toward the donor (C14) */
  int l = find_link(C, nb, c);
  double fg = C->lval[((size_t)l * C->nv + k) * C->ncomp + m];
  double sig = (fc - fg) / (-s * h); /* (f_d - f*_gc) / (x_d - x_g) with x_g = x_d + s h */
  return fg + sig * (-s * 0.5 * h);
}

static void cell_macros(const or_case *C, const double *f, long c, double *rho, double *U,
                        double *T, double *q, double *tau)
{
  double out[16];
  or_cell_moments(C, f + (size_t)c * C->nv * C->ncomp, out);
  int D = C->dim;
  *rho = out[0];
  for (int a = 0; a < D; ++a) U[a] = out[1 + a] / out[0];
  for (int a = D; a < 3; ++a) U[a] = 0.0;
  *T = out[D + 2];
  double pr = out[D + 3];
  for (int a = 0; a < D; ++a) q[a] = out[D + 4 + a];
  for (int a = D; a < 3; ++a) q[a] = 0.0;
  double mu = C->mu0 * pow(*T, C->p.omega_vhs); /* Eq. viscosity with T_0 = 1 */
  *tau = mu / pr;
}

static void conservative(const or_case *C, const double *f, long c, double *W)
{
  double out[16];
  or_cell_moments(C, f + (size_t)c * C->nv * C->ncomp, out);
  for (int i = 0; i < C->dim + 2; ++i) W[i] = out[i];
}

double or_residual(const or_case *C, const double *Wold, const double *Wnew)
{
  int nw = C->dim + 2;
  double res = 0.0;
  for (int i = 0; i < nw; ++i) {
    double num = 0.0, den = 0.0;
    for (long c = 0; c < C->nc; ++c) {
      if (C->type[c] != OR_FLUID) continue;
      double d = Wnew[c * nw + i] - Wold[c * nw + i];
      num += d * d;
      den += fabs(Wnew[c * nw + i]);
    }
    if (den == 0.0) continue; /* C18 */
    double r = sqrt(num) / den;
    if (r > res) res = r;
  }
  return res;
}

int or_step(or_case *C, int nsteps, double *residual)
{
  int D = C->dim, nv = C->nv, nc = C->ncomp;
  int nw = D + 2;
  double *Wold = (double *)xcalloc((size_t)C->nc * nw, sizeof(double));
  double *Wnew = (double *)xcalloc((size_t)C->nc * nw, sizeof(double));
  double res = 0.0;
  for (int it = 0; it < nsteps; ++it) {
    /* ghost band on f^n: link values f*_gc */
    or_ghost_band(C, C->f, NULL, NULL, NULL, NULL, C->lval, NULL);
    /* fluid cells: transport and relaxation (every cell writes only its own
       values, so the result does not depend on the number of threads) */
    memcpy(C->fnew, C->f, sizeof(double) * (size_t)C->nc * nv * nc);
#pragma omp parallel num_threads(C->nthreads)
    {
    double *gS = (double *)xcalloc((size_t)nv * nc, sizeof(double));
#pragma omp for schedule(dynamic, 16)
    for (long c = 0; c < C->nc; ++c) {
      if (C->type[c] != OR_FLUID) continue;
      double rho, U[3], T, q[3], tau;
      cell_macros(C, C->f, c, &rho, U, &T, q, &tau);
      conservative(C, C->f, c, Wold + c * nw);
      or_shakhov(C, rho, U, T, q, gS);
      for (int k = 0; k < nv; ++k)
        for (int m = 0; m < nc; ++m) {
          double fc = F(C, C->f, c, k)[m];
          double div = 0.0;
          for (int a = 0; a < D; ++a) {
            double xia = C->xi[3 * k + a];
            double fR = face_value(C, C->f, c, a, +1, k, m);
            double fL = face_value(C, C->f, c, a, -1, k, m);
            div += (xia * fR - xia * fL) / C->dx[a];
          }
          F(C, C->fnew, c, k)[m] = fc - C->dt * div + C->dt / tau * (gS[k * nc + m] - fc);
        }
    }
    free(gS);
    }
    double *t = C->f;
    C->f = C->fnew;
    C->fnew = t;
    for (long c = 0; c < C->nc; ++c)
      if (C->type[c] == OR_FLUID) conservative(C, C->f, c, Wnew + c * nw);
    res = or_residual(C, Wold, Wnew);
  }
  free(Wold);
  free(Wnew);
  if (residual) *residual = res;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Surface force and heat flux through the donor-ghost faces (C19)           */
/* ------------------------------------------------------------------------ */

void or_forces(const or_case *C, double *F3, double *Q, double *CD, double *CL)
{
  int D = C->dim, nv = C->nv;
  /* link values of the current state */
  or_ghost_band(C, C->f, NULL, NULL, NULL, NULL, C->lval, NULL);
  double Fx[3] = {0, 0, 0}, Qs = 0.0;
  for (int l = 0; l < C->nlink; ++l) {
    const or_link *L = &C->links[l];
    int a = L->axis;
    int s = -L->side; /* face of the donor toward the ghost */
    double S = 1.0;
    for (int b = 0; b < D; ++b)
      if (b != a) S *= C->dx[b];
    for (int k = 0; k < nv; ++k) {
      double xn_in = C->xi[3 * k + a] * s; /* velocity into the solid */
      double fh = face_value(C, C->f, L->d, a, s, k, 0);
      double x2 = 0.0;
      for (int b = 0; b < D; ++b) x2 += C->xi[3 * k + b] * C->xi[3 * k + b];
      for (int b = 0; b < D; ++b) Fx[b] += S * C->w[k] * C->xi[3 * k + b] * xn_in * fh;
      double e = 0.5 * x2 * fh;
      if (D == 2) e += 0.5 * face_value(C, C->f, L->d, a, s, k, 1);
      Qs += S * C->w[k] * e * xn_in;
    }
  }
  for (int b = 0; b < 3; ++b) F3[b] = Fx[b];
  *Q = Qs;
  double U2 = 0.0;
  for (int b = 0; b < 3; ++b) U2 += C->Uinf[b] * C->Uinf[b];
  double Uinf = sqrt(U2);
  double Lref = C->p.Lref;
  if (Lref <= 0.0) {
    switch (C->p.kind) {
    case OR_BODY_CIRCLE: Lref = 2.0 * C->p.radii[0]; break;
    case OR_BODY_ELLIPSE: Lref = 2.0 * fmax(C->p.radii[0], C->p.radii[1]); break;
    case OR_BODY_SPHERE: Lref = M_PI * C->p.radii[0] * C->p.radii[0]; break;
    case OR_BODY_POLYGON: {
      double mn = 1e300, mx = -1e300;
      for (int i = 0; i < C->p.nverts; ++i) {
        mn = fmin(mn, C->verts[2 * i]);
        mx = fmax(mx, C->verts[2 * i]);
      }
      Lref = mx - mn;
      break;
    }
    default: Lref = 1.0;
    }
  }
  double qdyn = 0.5 * C->p.rho_inf * U2 * Lref;
  if (Uinf > 0.0 && qdyn > 0.0) {
    double e[3] = {C->Uinf[0] / Uinf, C->Uinf[1] / Uinf, C->Uinf[2] / Uinf};
    double lift[3] = {-e[1], e[0], 0.0};
    *CD = (Fx[0] * e[0] + Fx[1] * e[1] + Fx[2] * e[2]) / qdyn;
    *CL = (Fx[0] * lift[0] + Fx[1] * lift[1]) / qdyn;
  } else {
    *CD = 0.0;
    *CL = 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* accessors                                                                 */
/* ------------------------------------------------------------------------ */

void or_sizes(const or_case *C, long long *o)
{
  long nf = 0;
  for (long c = 0; c < C->nc; ++c) nf += C->type[c] == OR_FLUID;
  o[0] = C->nc;
  o[1] = C->nv;
  o[2] = C->ncomp;
  o[3] = C->nlink;
  o[4] = C->nghost;
  o[5] = nf;
}

double or_dt(const or_case *C) { return C->dt; }

void or_velocities(const or_case *C, double *xi, double *w)
{
  memcpy(xi, C->xi, sizeof(double) * 3 * C->nv);
  memcpy(w, C->w, sizeof(double) * C->nv);
}

void or_cell_types(const or_case *C, unsigned char *types) { memcpy(types, C->type, C->nc); }

void or_links(const or_case *C, int *ghost, int *donor, int *aux, int *axis, int *side,
              double *xw, double *nw)
{
  for (int l = 0; l < C->nlink; ++l) {
    const or_link *L = &C->links[l];
    ghost[l] = L->g;
    donor[l] = L->d;
    aux[l] = L->ac;
    axis[l] = L->axis;
    side[l] = L->side;
    for (int a = 0; a < 3; ++a) {
      xw[3 * l + a] = L->xw[a];
      nw[3 * l + a] = L->nw[a];
    }
  }
}

void or_cut_table(const or_case *C, double *wg)
{
  memcpy(wg, C->wg, sizeof(double) * (size_t)C->nlink * C->nv);
}

int or_surface_count(const or_case *C)
{
  int n = 0;
  for (int g = 0; g < C->nghost; ++g) n += C->ghosts[g].ns;
  return n;
}

void or_surface_cells(const or_case *C, int *ghost_cell, int *offsets, int *cells)
{
  int o = 0;
  for (int g = 0; g < C->nghost; ++g) {
    ghost_cell[g] = C->ghosts[g].cell;
    offsets[g] = o;
    for (int j = 0; j < C->ghosts[g].ns; ++j) cells[o++] = C->ghosts[g].surf[j];
  }
  offsets[C->nghost] = o;
}

void or_get_f(const or_case *C, double *f)
{
  memcpy(f, C->f, sizeof(double) * (size_t)C->nc * C->nv * C->ncomp);
}

void or_set_f(or_case *C, const double *f)
{
  memcpy(C->f, f, sizeof(double) * (size_t)C->nc * C->nv * C->ncomp);
}

void or_freestream(const or_case *C, double *finf)
{
  memcpy(finf, C->finf, sizeof(double) * C->nv * C->ncomp);
}

void or_moments(const or_case *C, double *W, double *q)
{
  int D = C->dim;
  double out[16];
  for (long c = 0; c < C->nc; ++c) {
    or_cell_moments(C, C->f + (size_t)c * C->nv * C->ncomp, out);
    for (int i = 0; i < D + 2; ++i) W[c * (D + 2) + i] = out[i];
    for (int a = 0; a < D; ++a) q[c * D + a] = out[D + 4 + a];
  }
}

/* ------------------------------------------------------------------------ */
/* Tree-refined 2D grids (reading C28)                                       */
/* ------------------------------------------------------------------------ */

struct or_tree {
  or_case *V;   /* velocity grid, gas, time step and body: a case on the finest uniform grid */
  long n;       /* leaves */
  int L;        /* finest level */
  int D, NF;    /* dimension; leaves beyond a face at most (2^(D-1) finer ones) */
  int *lev;
  double *h;    /* [n][D] edge lengths */
  long *nb;     /* [n][2D][NF] face neighbours, sides 2a + (s > 0) */
  double *f, *fnew, *sl; /* [n][nv][nc]; slopes [n][D][nv][nc] */
  unsigned char *type;   /* [n] OR_FLUID, OR_GHOST, OR_SOLID (C29) */
  long *leafv;  /* [n] the finest-grid cell of a finest leaf, -1 for coarser leaves */
  int body;
  int nthreads;
};

/* the leaf owning finest-grid cell q is of the finest level */
static int finest_owned(const long *own, const int *level, int L, long q) { return q >= 0 && level[own[q]] == L; }

/* C29: every cell the immersed boundary reads or writes lies in the finest
   level: the ghost cells, the donors, the auxiliary cells and the cells
   beyond the donors along the link axes (their slopes and face values), the
   surface cells and their fluid face neighbours (the pre-ghost slopes).  A
   coarser leaf is all fluid or all solid. */
static int tree_body_fits(const or_case *V, const long *own, const int *level, int L)
{
  for (int l = 0; l < V->nlink; ++l) {
    const or_link *K = &V->links[l];
    if (!finest_owned(own, level, L, K->g) || !finest_owned(own, level, L, K->d)) return 0;
    if (K->ac >= 0 && !finest_owned(own, level, L, K->ac)) return 0;
    const long far = neighbour(V, K->d, K->axis, K->side);
    if (far >= 0 && V->type[far] == OR_FLUID && !finest_owned(own, level, L, far)) return 0;
  }
  for (int gi = 0; gi < V->nghost; ++gi) {
    const or_ghost *G = &V->ghosts[gi];
    for (int j = 0; j < G->ns; ++j) {
      if (!finest_owned(own, level, L, G->surf[j])) return 0;
      for (int a = 0; a < V->dim; ++a)
        for (int s = -1; s <= 1; s += 2) {
          const long q = neighbour(V, G->surf[j], a, s);
          if (q >= 0 && V->type[q] == OR_FLUID && !finest_owned(own, level, L, q)) return 0;
        }
    }
  }
  return 1;
}

/* the finest-grid cells of a leaf: origin q0 and edge s (in finest cells) */
static void leaf_block(const int *ix, const int *iy, const int *iz, int D, int L, int l, long c, long q0[3],
                       long *s)
{
  *s = 1L << (L - l);
  q0[0] = ix[c] * *s;
  q0[1] = iy[c] * *s;
  q0[2] = (D == 3) ? iz[c] * *s : 0;
}

or_tree *or_tree_create(const or_params *p, long nleaf, int maxlevel, const int *level, const int *ix,
                        const int *iy, const int *iz, int *why)
{
  if (why) *why = 1;
  const int D = p->dim;
  if ((D != 2 && D != 3) || maxlevel < 0 || maxlevel > 12 || nleaf <= 0 || (D == 3 && !iz)) return NULL;
  for (int i = 0; i < 6; ++i)
    if (p->wall[i]) return NULL;
  long nf[3] = {1, 1, 1};
  for (int a = 0; a < D; ++a) nf[a] = (long)p->n[a] << maxlevel;
  const long nfc = nf[0] * nf[1] * nf[2];
  /* owner of every cell of the finest grid */
  long *own = (long *)xcalloc((size_t)nfc, sizeof(long));
  for (long q = 0; q < nfc; ++q) own[q] = -1;
  int ok = 1;
  for (long c = 0; c < nleaf && ok; ++c) {
    const int l = level[c];
    const int co[3] = {ix[c], iy[c], (D == 3) ? iz[c] : 0};
    if (l < 0 || l > maxlevel) ok = 0;
    for (int a = 0; a < D && ok; ++a)
      if (co[a] < 0 || co[a] >= (p->n[a] << l)) ok = 0;
    if (!ok) break;
    long q0[3], s;
    leaf_block(ix, iy, iz, D, maxlevel, l, c, q0, &s);
    const long sz = (D == 3) ? s : 1;
    for (long k = q0[2]; k < q0[2] + sz; ++k)
      for (long j = q0[1]; j < q0[1] + s; ++j)
        for (long i = q0[0]; i < q0[0] + s; ++i) {
          const long q = i + nf[0] * (j + nf[1] * k);
          if (own[q] >= 0) ok = 0; /* overlapping leaves */
          own[q] = c;
        }
  }
  for (long q = 0; ok && q < nfc; ++q)
    if (own[q] < 0) ok = 0; /* a hole */
  or_tree *T = NULL;
  if (ok) {
    T = (or_tree *)xcalloc(1, sizeof(or_tree));
    or_params pf = *p;
    for (int a = 0; a < D; ++a) pf.n[a] = (int)nf[a];
    T->V = or_create(&pf);
    /* the helper case never steps: only its state buffer is used (the
       scatter target of the body's ghost band) */
    free(T->V->fnew);
    T->V->fnew = NULL;
    T->n = nleaf;
    T->L = maxlevel;
    T->D = D;
    T->NF = 1 << (D - 1);
    const int NF = T->NF;
    T->lev = (int *)xcalloc((size_t)nleaf, sizeof(int));
    T->h = (double *)xcalloc((size_t)nleaf * D, sizeof(double));
    T->nb = (long *)xcalloc((size_t)nleaf * 2 * D * NF, sizeof(long));
    T->nthreads = 1;
    double H[3];
    for (int a = 0; a < D; ++a) H[a] = (p->hi[a] - p->lo[a]) / p->n[a];
    for (long c = 0; c < nleaf && ok; ++c) {
      const int l = level[c];
      T->lev[c] = l;
      for (int a = 0; a < D; ++a) T->h[(size_t)D * c + a] = H[a] / (double)(1L << l);
      long q0[3], s;
      leaf_block(ix, iy, iz, D, maxlevel, l, c, q0, &s);
      for (int a = 0; a < D && ok; ++a)
        for (int side = 0; side < 2 && ok; ++side) {
          long *out = T->nb + ((size_t)c * 2 * D + 2 * a + side) * NF;
          for (int j = 0; j < NF; ++j) out[j] = -1;
          /* the finest cells just beyond the face, the first transverse axis
             fastest: their distinct owners in the order met */
          const long fa = side ? q0[a] + s : q0[a] - 1;
          if (fa < 0 || fa >= nf[a]) continue; /* the domain edge */
          const int u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2; /* the transverse axes */
          const long sv = (D == 3) ? s : 1;
          int cnt = 0;
          for (long tv = 0; tv < sv && ok; ++tv)
            for (long tu = 0; tu < s && ok; ++tu) {
              long q[3];
              q[a] = fa;
              q[u] = q0[u] + tu;
              q[v] = (D == 3) ? q0[v] + tv : 0;
              const long o = own[q[0] + nf[0] * (q[1] + nf[1] * q[2])];
              int seen = 0;
              for (int j = 0; j < cnt; ++j) seen |= out[j] == o;
              if (seen) continue;
              if (cnt == NF) {
                ok = 0;
                break;
              }
              out[cnt++] = o;
            }
          /* 2:1: one neighbour of the same or the coarser level, or NF of the finer one */
          if (cnt == 1 && !(level[out[0]] == l || level[out[0]] == l - 1)) ok = 0;
          if (cnt > 1) {
            if (cnt != NF) ok = 0;
            for (int j = 0; j < cnt; ++j)
              if (level[out[j]] != l + 1) ok = 0;
          }
        }
    }
    if (ok) {
      /* leaf classes from the finest grid (C29) */
      or_case *V = T->V;
      T->body = p->kind != OR_BODY_NONE;
      T->type = (unsigned char *)xcalloc((size_t)nleaf, 1);
      T->leafv = (long *)xcalloc((size_t)nleaf, sizeof(long));
      int fits = tree_body_fits(V, own, level, maxlevel);
      for (long c = 0; c < nleaf && fits; ++c) {
        const int l = level[c];
        long q0[3], s;
        leaf_block(ix, iy, iz, D, maxlevel, l, c, q0, &s);
        const long q00 = q0[0] + nf[0] * (q0[1] + nf[1] * q0[2]);
        T->leafv[c] = (l == maxlevel) ? q00 : -1;
        const unsigned char t0 = V->type[q00];
        const long sz = (D == 3) ? s : 1;
        for (long k = q0[2]; k < q0[2] + sz && fits; ++k)
          for (long j = q0[1]; j < q0[1] + s && fits; ++j)
            for (long i = q0[0]; i < q0[0] + s; ++i)
              if (V->type[i + nf[0] * (j + nf[1] * k)] != t0 || (l < maxlevel && t0 == OR_GHOST)) fits = 0;
        T->type[c] = t0;
      }
      if (!fits) {
        ok = 0;
        if (why) *why = 2;
      }
    }
    if (ok) {
      const size_t sz = (size_t)nleaf * T->V->nv * T->V->ncomp;
      T->f = (double *)xcalloc(sz, sizeof(double));
      T->fnew = (double *)xcalloc(sz, sizeof(double));
      T->sl = (double *)xcalloc(sz * D, sizeof(double));
      for (long c = 0; c < nleaf; ++c)
        memcpy(T->f + (size_t)c * T->V->nv * T->V->ncomp, T->V->finf, sizeof(double) * T->V->nv * T->V->ncomp);
    }
  }
  free(own);
  if (T && !ok) {
    or_tree_destroy(T);
    T = NULL;
  }
  if (T && why) *why = 0;
  return T;
}

void or_tree_destroy(or_tree *T)
{
  if (!T) return;
  if (T->V) or_destroy(T->V);
  free(T->lev);
  free(T->h);
  free(T->nb);
  free(T->f);
  free(T->fnew);
  free(T->sl);
  free(T->type);
  free(T->leafv);
  free(T);
}

void or_tree_set_threads(or_tree *T, int nthreads) { T->nthreads = nthreads > 0 ? nthreads : 1; }

void or_tree_sizes(const or_tree *T, long long *o)
{
  o[0] = T->n;
  o[1] = T->V->nv;
  o[2] = T->V->ncomp;
}

double or_tree_dt(const or_tree *T) { return T->V->dt; }

void or_tree_neighbours(const or_tree *T, long long *nb)
{
  for (long i = 0; i < T->n * 2 * T->D * T->NF; ++i) nb[i] = T->nb[i];
}

void or_tree_get_f(const or_tree *T, double *f)
{
  memcpy(f, T->f, sizeof(double) * (size_t)T->n * T->V->nv * T->V->ncomp);
}

void or_tree_set_f(or_tree *T, const double *f)
{
  memcpy(T->f, f, sizeof(double) * (size_t)T->n * T->V->nv * T->V->ncomp);
}

/* the ghost value of the link from ghost leaf g to its fluid face neighbour
   c (both of the finest level, C29): the value c sees across that face */
static double tree_link_value(const or_tree *T, long g, long c, int k, int m)
{
  const int l = find_link(T->V, T->leafv[g], T->leafv[c]);
  return T->V->lval[((size_t)l * T->V->nv + k) * T->V->ncomp + m];
}

/* the finest leaves' values into the finest grid of the helper case (the
   cells the immersed boundary reads, C29) */
static void tree_scatter(or_tree *T)
{
  const size_t row = (size_t)T->V->nv * T->V->ncomp;
  for (long c = 0; c < T->n; ++c)
    if (T->leafv[c] >= 0) memcpy(T->V->f + (size_t)T->leafv[c] * row, T->f + (size_t)c * row, sizeof(double) * row);
}

/* the leaves beyond side (a, s) of leaf c */
static const long *tree_nbrs(const or_tree *T, long c, int a, int s)
{
  return T->nb + ((size_t)c * 2 * T->D + 2 * a + (s > 0)) * T->NF;
}

/* the value on side (a, s) of fluid leaf c as its slope sees it (the
   neighbour's, the mean of the finer neighbours', the freestream halo; a
   ghost neighbour's link value, C29), and the distance to it along a (C28) */
static double tree_side(const or_tree *T, const double *f, long c, int a, int s, int k, int m, double *dist)
{
  const long *nb = tree_nbrs(T, c, a, s);
  const int nv = T->V->nv, nc = T->V->ncomp, D = T->D;
  const double hc = T->h[(size_t)D * c + a];
  if (nb[0] < 0) {
    *dist = hc;
    return T->V->finf[k * nc + m]; /* the freestream halo */
  }
  *dist = 0.5 * (hc + T->h[(size_t)D * nb[0] + a]);
  if (T->type[nb[0]] != OR_FLUID) return tree_link_value(T, nb[0], c, k, m);
  double v = f[((size_t)nb[0] * nv + k) * nc + m];
  int cnt = 1;
  while (cnt < T->NF && nb[cnt] >= 0) v += f[((size_t)nb[cnt++] * nv + k) * nc + m];
  return (cnt == 1) ? v : v * (1.0 / cnt);
}

/* face value on side (a, s) of leaf c (Eq. reconstruction with the slope of C28) */
static double tree_face(const or_tree *T, const double *f, long c, int a, int s, int k, int m)
{
  const int nv = T->V->nv, nc = T->V->ncomp, D = T->D;
  const double fc = f[((size_t)c * nv + k) * nc + m];
  const double sig = T->sl[(((size_t)c * D + a) * nv + k) * nc + m];
  return fc + sig * (s * 0.5 * T->h[(size_t)D * c + a]);
}

int or_tree_step(or_tree *T, int nsteps, double *residual)
{
  or_case *V = T->V;
  const int nv = V->nv, nc = V->ncomp, D = T->D, nw = D + 2;
  const long n = T->n;
  double *Wold = (double *)xcalloc((size_t)n * nw, sizeof(double));
  double *Wnew = (double *)xcalloc((size_t)n * nw, sizeof(double));
  double res = 0.0;
  for (int it = 0; it < nsteps; ++it) {
    /* the ghost band on the finest grid around the body: link values f*_gc */
    if (T->body) {
      tree_scatter(T);
      or_ghost_band(V, V->f, NULL, NULL, NULL, NULL, V->lval, NULL);
    }
    /* slopes of every fluid leaf along each axis (Eq. limiter over the centre distances) */
#pragma omp parallel for num_threads(T->nthreads) schedule(dynamic, 16)
    for (long c = 0; c < n; ++c) {
      if (T->type[c] != OR_FLUID) continue;
      for (int a = 0; a < D; ++a)
        for (int k = 0; k < nv; ++k)
          for (int m = 0; m < nc; ++m) {
            const double fc = T->f[((size_t)c * nv + k) * nc + m];
            double dm, dp;
            const double fm = tree_side(T, T->f, c, a, -1, k, m, &dm);
            const double fp = tree_side(T, T->f, c, a, +1, k, m, &dp);
            T->sl[(((size_t)c * D + a) * nv + k) * nc + m] = or_vanleer((fc - fm) / dm, (fp - fc) / dp);
          }
    }
    /* transport and relaxation of every leaf */
#pragma omp parallel num_threads(T->nthreads)
    {
      double *gS = (double *)xcalloc((size_t)nv * nc, sizeof(double));
#pragma omp for schedule(dynamic, 16)
      for (long c = 0; c < n; ++c) {
        const size_t row = (size_t)nv * nc;
        if (T->type[c] != OR_FLUID) { /* solid leaves keep their values */
          memcpy(T->fnew + c * row, T->f + c * row, sizeof(double) * row);
          conservative(V, T->f, c, Wold + c * nw);
          continue;
        }
        double rho, U[3], Tm, q[3], tau;
        cell_macros(V, T->f, c, &rho, U, &Tm, q, &tau);
        conservative(V, T->f, c, Wold + c * nw);
        or_shakhov(V, rho, U, Tm, q, gS);
        for (int k = 0; k < nv; ++k)
          for (int m = 0; m < nc; ++m) {
            const double fc = T->f[((size_t)c * nv + k) * nc + m];
            double div = 0.0;
            for (int a = 0; a < D; ++a) {
              const double xia = V->xi[3 * k + a];
              if (xia == 0.0) continue;
              const int s = (xia > 0.0) ? 1 : -1; /* the downwind side */
              const double fout = tree_face(T, T->f, c, a, s, k, m);
              /* inflow through the upwind side: the upwind cells' face values,
                 each over the share of the side it covers */
              const long *nb = tree_nbrs(T, c, a, -s);
              double fin;
              if (nb[0] < 0) {
                fin = V->finf[k * nc + m]; /* halo: its value, zero slope */
              } else if (T->type[nb[0]] != OR_FLUID) {
                /* a ghost: its link value with the one-sided slope (C14) */
                fin = 0.5 * (tree_link_value(T, nb[0], c, k, m) + fc);
              } else {
                fin = tree_face(T, T->f, nb[0], a, s, k, m);
                int cnt = 1;
                while (cnt < T->NF && nb[cnt] >= 0) fin += tree_face(T, T->f, nb[cnt++], a, s, k, m);
                if (cnt > 1) fin *= 1.0 / cnt;
              }
              div += fabs(xia) * (fout - fin) / T->h[(size_t)D * c + a];
            }
            T->fnew[((size_t)c * nv + k) * nc + m] = fc - V->dt * div + V->dt / tau * (gS[k * nc + m] - fc);
          }
      }
      free(gS);
    }
    double *t = T->f;
    T->f = T->fnew;
    T->fnew = t;
    for (long c = 0; c < n; ++c) conservative(V, T->f, c, Wnew + c * nw);
    /* residual over the fluid leaves (the formula of the uniform grid, C18) */
    res = 0.0;
    for (int i = 0; i < nw; ++i) {
      double num = 0.0, den = 0.0;
      for (long c = 0; c < n; ++c) {
        if (T->type[c] != OR_FLUID) continue;
        const double d = Wnew[c * nw + i] - Wold[c * nw + i];
        num += d * d;
        den += fabs(Wnew[c * nw + i]);
      }
      if (den == 0.0) continue;
      const double r = sqrt(num) / den;
      if (r > res) res = r;
    }
  }
  free(Wold);
  free(Wnew);
  if (residual) *residual = res;
  return 0;
}

void or_tree_cell_types(const or_tree *T, unsigned char *types) { memcpy(types, T->type, (size_t)T->n); }

/* the helper case on the finest grid, holding the finest leaves' current
   values (the cells the body's ghost band reads, C29); owned by the tree */
or_case *or_tree_finest(or_tree *T)
{
  tree_scatter(T);
  return T->V;
}

/* surface force and heat flux of the current state through the donor-ghost
   faces (C19), on the finest grid around the body (C29) */
void or_tree_forces(or_tree *T, double *F3, double *Q, double *CD, double *CL)
{
  tree_scatter(T);
  or_forces(T->V, F3, Q, CD, CL);
}

void or_tree_moments(const or_tree *T, double *W, double *q)
{
  const int D = T->D, nv = T->V->nv, nc = T->V->ncomp;
  double out[16];
  for (long c = 0; c < T->n; ++c) {
    or_cell_moments(T->V, T->f + (size_t)c * nv * nc, out);
    for (int i = 0; i < D + 2; ++i) W[c * (D + 2) + i] = out[i];
    for (int a = 0; a < D; ++a) q[c * D + a] = out[D + 4 + a];
  }
}
