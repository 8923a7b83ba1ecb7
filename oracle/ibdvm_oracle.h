/*
 * ibdvm_oracle.h -- interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check of the entry
 * module and the CPU-baseline leg of the benchmark load this library. The
 * solver product never includes this header, never links the oracle and
 * shares no code with it.
 *
 * The oracle follows the ghost-cell immersed-boundary discrete velocity
 * method of Ge, Cai, Zhang and Xiao (arXiv 2512.20252) step by step:
 *   Sec. 2.1  Shakhov model, moments (Eqs. moments1-3)
 *   Sec. 2.2  discrete velocity equation, quadrature, finite volume,
 *             upwind reconstruction with the van Leer limiter
 *   Sec. 2.3  Maxwell gas-surface interaction, no-penetration density
 *   Sec. 3.2  ghost, fluid, surface, donor and auxiliary cells; shifted
 *             point; upwind-weighted compact interpolation; intersect-point
 *             construction; ghost-cell construction; velocity-space cut cells
 *   Sec. 4    reduced distributions h, b (2D), non-dimensional Maxwellians,
 *             VHS viscosity, residual, forward Euler.
 */
#ifndef IBDVM_ORACLE_H
#define IBDVM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Body kinds understood by the oracle. */
enum {
  OR_BODY_NONE = 0,
  OR_BODY_CIRCLE = 1,    /* 2D: centre, radii[0] */
  OR_BODY_ELLIPSE = 2,   /* 2D: centre, semi-axes radii[0] (along the rotated x) and radii[1], angle */
  OR_BODY_SPHERE = 3,    /* 3D: centre, radii[0] */
  OR_BODY_POLYGON = 4,   /* 2D: counter-clockwise vertices verts[2*nverts] */
  OR_BODY_HALFSPACE = 5  /* 2D/3D: solid where (x - centre).radii <= 0; radii = unit normal into the gas */
};

/* Cell classes, Sec. 3.2.1. */
enum { OR_FLUID = 0, OR_GHOST = 1, OR_SOLID = 2 };

typedef struct {
  /* physical grid: uniform Cartesian, n[a] cells on [lo[a], hi[a]] */
  int dim;
  int n[3];
  double lo[3], hi[3];
  /* velocity grid: nv[a] nodes on [vlo[a], vhi[a]], rule 0 = trapezoid, 1 = composite midpoint,
     2 = the nodes vnodes[a][0 .. nv[a]-1] (strictly increasing; C25) */
  int nv[3];
  double vlo[3], vhi[3];
  int rule;
  /* gas (non-dimensional, Sec. 4) */
  double Kn, Ma, Pr, gamma, omega_vhs, alpha_vhs;
  double rho_inf, T_inf;
  double dir[3];
  double cfl, dt; /* dt <= 0: dt from the CFL number */
  /* body and wall (Sec. 2.3) */
  int kind;
  double center[3], radii[3], angle;
  const double *verts;
  int nverts;
  double accom; /* Maxwell accommodation coefficient alpha */
  double Tw, Uw[3];
  double Lref; /* reference length (2D) or area (3D) for force coefficients; <= 0: from the body */
  /* method switches */
  int cutcell; /* 1: velocity-space cut-cell correction (Sec. 3.2.3); 0: node classification only */
  int upwind;  /* 1: upwind weights with r pointing from the fluid cell to the ghost cell,
                  2: upwind weights with r pointing from the ghost cell to the fluid cell,
                  0: plain average 1/N_S,
                  3: no interpolation: the linear extrapolation 2 f_d - f_ac along the
                     link axis (the construction without upwind weighting, Sec. 3.3.4) */
  /* domain faces 2a + (s > 0) (x-, x+, y-, y+, z-, z+): 0 = two freestream
     halo layers (C17), 1 = diffuse wall at wall_T with velocity wall_U (C24) */
  int wall[6];
  double wall_T[6];
  double wall_U[6][3];
  /* rule 2: the nodes of each axis */
  const double *vnodes[3];
  /* 1: ghost values below zero are set to zero (C26) */
  int ghost_nonneg;
} or_params;

typedef struct or_case or_case;

or_case *or_create(const or_params *p);
void or_destroy(or_case *C);
/* host threads of the per-ghost and per-cell loops (OpenMP when the library is
   built with it; default 1).  Ghosts and cells are computed independently and
   the reductions (residual, forces) stay serial, so the results are bitwise
   the same for any thread count. */
void or_set_threads(or_case *C, int nthreads);

/* sizes: ncell, nvel, ncomp, nlink, nghost, nfluid */
void or_sizes(const or_case *C, long long *out6);
double or_dt(const or_case *C);
/* per-velocity node and weight: xi[k*3+a], w[k] */
void or_velocities(const or_case *C, double *xi, double *w);
/* cell classes */
void or_cell_types(const or_case *C, unsigned char *types);
/* link table in canonical order (ghost cell ascending, then direction 2*axis + (side > 0)) */
void or_links(const or_case *C, int *ghost, int *donor, int *aux, int *axis, int *side,
              double *xw, double *nw);
/* incident-side velocity measure omega^g per link and velocity: wg[L*nvel + k] */
void or_cut_table(const or_case *C, double *wg);
/* surface cells of every ghost (CSR): offsets[nghost+1], cells[...] */
int or_surface_count(const or_case *C);
void or_surface_cells(const or_case *C, int *ghost_cell, int *offsets, int *cells);

/* state: f[cell][k][comp] */
void or_get_f(const or_case *C, double *f);
void or_set_f(or_case *C, const double *f);
void or_freestream(const or_case *C, double *finf);

/* one forward-Euler step per iteration; residual of the last step */
int or_step(or_case *C, int nsteps, double *residual);
/* conservative variables W[cell][dim+2] and heat flux q[cell][dim] of the current state */
void or_moments(const or_case *C, double *W, double *q);
/* surface force and heat flux, Eq. moments applied to the face fluxes on the link faces */
void or_forces(const or_case *C, double *F3, double *Q, double *CD, double *CL);

/* wall density rho_w of every diffuse domain face of the given state,
   out[cell * 6 + 2a + (s > 0)] (0 where the face is not a diffuse wall of a
   fluid cell) */
void or_domain_wall_density(const or_case *C, const double *f, double *out);

/* the ghost band on the given state (Sec. 3.2.1 steps 1-4) */
void or_ghost_band(const or_case *C, const double *f, double *fgc, double *fsp, double *fiw,
                   double *fstarw, double *fstargc, double *rhow);

/* building blocks, exposed for the pins */
/* weights of Eq. upwind of ghost gi (index in the ghost list): out[j * nvel + k]
   for its surface cells j (the order of or_surface_cells) and velocities k */
void or_upwind_weights(const or_case *C, int gi, double *out);
double or_mu0(double Kn, double alpha, double omega);
double or_vanleer(double s1, double s2);
void or_cell_moments(const or_case *C, const double *fcell, double *out);
void or_shakhov(const or_case *C, double rho, const double *U, double T, const double *q,
                double *gS);
void or_maxwellian(const or_case *C, double rho, const double *U, double T, double *g);
double or_cut_fraction_2d(const double *blo, const double *bhi, const double *n);
double or_cut_fraction_3d(const double *blo, const double *bhi, const double *n);
double or_residual(const or_case *C, const double *Wold, const double *Wnew);

/* Tree-refined grids (reading C28), quadtrees in 2D and octrees in 3D:
   leaves (level, ix, iy, iz) over the root grid p->n on [lo, hi], integer
   coordinates of the leaf's level (0 <= ix < n[0] 2^level; iz NULL in 2D);
   the leaves must tile the domain and face neighbours differ by at most one
   level (a face borders one leaf or 2^(dim-1) finer ones).  The domain
   faces are freestream.
   A body (reading C29) must lie in the finest level: every cell its ghost
   band reads or writes is a leaf of the finest level, a coarser leaf is all
   fluid or all solid.  NULL when refused; *why (if given) = 1 for an invalid
   tree, 2 for a body outside the finest level, 0 on success. */
typedef struct or_tree or_tree;
or_tree *or_tree_create(const or_params *p, long nleaf, int maxlevel, const int *level, const int *ix,
                        const int *iy, const int *iz, int *why);
void or_tree_destroy(or_tree *T);
void or_tree_set_threads(or_tree *T, int nthreads);
/* sizes: nleaf, nvel, ncomp */
void or_tree_sizes(const or_tree *T, long long *out3);
double or_tree_dt(const or_tree *T);
/* face neighbours nb[leaf][side 2a + (s > 0)][2^(dim-1)] (-1: none; the first
   is -1 at the domain edge, the others unless finer neighbours share the
   side, in the order met with the first transverse axis fastest) */
void or_tree_neighbours(const or_tree *T, long long *nb);
void or_tree_get_f(const or_tree *T, double *f);
void or_tree_set_f(or_tree *T, const double *f);
int or_tree_step(or_tree *T, int nsteps, double *residual);
void or_tree_moments(const or_tree *T, double *W, double *q);
void or_tree_cell_types(const or_tree *T, unsigned char *types);
void or_tree_forces(or_tree *T, double *F3, double *Q, double *CD, double *CL);
/* the helper case on the finest grid with the finest leaves' current values
   (the body's links and ghost band in the order of the tree's links); owned
   by the tree, valid until it is destroyed */
or_case *or_tree_finest(or_tree *T);

#ifdef __cplusplus
}
#endif
#endif
