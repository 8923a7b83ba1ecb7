/*
 * ibdvm.h -- C-ABI of the GB300-native immersed-boundary discrete velocity
 * solver (libibdvm.so).
 *
 * The library advances the discrete velocity model of the Shakhov-Boltzmann
 * equation on a uniform Cartesian grid with an immersed rigid body, following
 * the ghost-cell immersed boundary method of Ge, Cai, Zhang and Xiao,
 * "An immersed boundary method for the discrete velocity model of the
 * Boltzmann equation" (arXiv 2512.20252):
 *   - Sec. 2.2: finite-volume upwind fluxes with van Leer-limited linear
 *     reconstruction (Eqs. half-discrete, reconstruction, limiter), velocity
 *     quadrature (Eq. quadrature), Shakhov relaxation (Eq. shakhov);
 *   - Sec. 2.3: Maxwell gas-surface interaction (Eqs. general bc, Maxwell BC,
 *     boundary maxwell) with the wall density from zero normal mass flux
 *     (Eqs. npc, dnpc);
 *   - Sec. 3.2: ghost, fluid, surface, donor and auxiliary cells, shifted
 *     point (Eqs. sp, fsp), upwind-weighted compact interpolation
 *     (Eqs. extrapolation 1, upwind), intersect point (Eq. fw), ghost-cell
 *     construction (Eq. extrapolation 2) and the velocity-space cut-cell
 *     correction (Eqs. fwc, cc_np, rhowc);
 *   - Sec. 4: reduced distributions h, b in 2D, non-dimensional equilibria,
 *     VHS viscosity (Eq. viscosity), residual and forward Euler time marching.
 *
 * Conventions for every call:
 *   - Status codes: every call returns an ibdvm_status and never aborts or
 *     traps.  On an error the context state is unchanged unless the call says
 *     otherwise, and ibdvm_last_error() returns a one-line reason.
 *   - Host arrays are caller-owned, row-major, FP64 unless stated; the library
 *     copies inputs and never keeps caller pointers.
 *   - Cell index c = i + n0*(j + n1*k) (x fastest); velocity index
 *     k = kx + nv0*(ky + nv1*kz) (xi_x fastest); distribution arrays are
 *     f[cell][k][comp] with comp = {h, b} in 2D (Sec. 4 reduced distributions)
 *     and comp = {f} in 3D.
 *   - A context owns all its device memory and is bound to one CUDA stream;
 *     it is not thread-safe; distinct contexts are independent.
 *   - Quantities are non-dimensional as in Sec. 4 (xi / sqrt(2 R T0), ...).
 */
#ifndef IBDVM_H
#define IBDVM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibdvm_ctx ibdvm_ctx;
typedef struct ibdvm_geom ibdvm_geom;

typedef enum {
  IBDVM_OK = 0,
  IBDVM_E_INVAL = 1,        /* an argument is out of range or inconsistent */
  IBDVM_E_NOMEM = 2,        /* host or device allocation failed */
  IBDVM_E_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  IBDVM_E_UNSTABLE = 4,     /* dt / tau > 1 somewhere: forward Euler relaxation would overshoot */
  IBDVM_E_NONFINITE = 5,    /* a non-finite moment or residual appeared */
  IBDVM_E_NOTCONVERGED = 6, /* reserved for callers that iterate to a residual */
  IBDVM_E_TIMEOUT = 7,      /* a bounded device wait gave up */
  IBDVM_E_STATE = 8         /* the call is not valid in the current state */
} ibdvm_status;

enum { IBDVM_RULE_TRAPEZOID = 0, IBDVM_RULE_MIDPOINT = 1, IBDVM_RULE_NODES = 2 };
enum { IBDVM_FP64 = 0, IBDVM_MIXED = 1 };
enum {
  IBDVM_BODY_NONE = 0,
  IBDVM_BODY_CIRCLE = 1,   /* 2D: center, radii[0] */
  IBDVM_BODY_ELLIPSE = 2,  /* 2D: center, semi-axes radii[0] (rotated x) and radii[1], angle (rad) */
  IBDVM_BODY_SPHERE = 3,   /* 3D: center, radii[0] */
  IBDVM_BODY_POLYGON = 4,  /* 2D: counter-clockwise verts[2*nverts] */
  IBDVM_BODY_HALFSPACE = 5 /* 2D/3D: solid where (x - center).radii <= 0, radii = unit normal into the gas */
};
enum { IBDVM_CELL_FLUID = 0, IBDVM_CELL_GHOST = 1, IBDVM_CELL_SOLID = 2 };
/* method switches (ibdvm_gas_desc.flags) */
enum {
  IBDVM_NO_CUTCELL = 1,        /* incident/reflected by the node sign of xi.n only (no Sec. 3.2.3) */
  IBDVM_PLAIN_AVERAGE = 2,     /* weights 1/N_S instead of Eq. upwind (ablation) */
  IBDVM_RHAT_GHOST_TO_FLUID = 4, /* Eq. upwind with r pointing from the ghost to the fluid cell */
  IBDVM_GHOST_NONNEG = 8,        /* ghost values of Eq. extrapolation 2 below zero are set to zero
                                    (off by default: keeps the supersonic cases of Sec. 4.4 positive) */
  IBDVM_NAIVE_EXTRAPOLATION = 16 /* ablation: no upwind-weighted interpolation; the intermediate ghost
                                    value of a link is the linear extrapolation 2 f_d - f_ac from its
                                    donor and auxiliary cell (Sec. 3.3.4; f_d without an auxiliary cell) */
};

/* Uniform Cartesian grid: dim = 2 or 3, n[a] cells on [lo[a], hi[a]]. */
typedef struct {
  int dim;
  int n[3];
  double lo[3], hi[3];
} ibdvm_grid_desc;

/* Velocity grid (Eq. quadrature): n[a] nodes per axis on [lo[a], hi[a]],
   rule = IBDVM_RULE_TRAPEZOID (nodes at both ends) or IBDVM_RULE_MIDPOINT
   (composite midpoint, Sec. 3.2.3).  Each node owns the dual box
   [xi - dxi/2, xi + dxi/2] clipped to the interval; its measure is the weight.
   rule = IBDVM_RULE_NODES: a non-uniform (stretched) grid standing in for the
   locally refined velocity mesh of Sec. 4.4, the tensor product of the n[a]
   strictly increasing finite nodes nodes[a][0 .. n[a]-1] of each axis (lo
   and hi are ignored: the interval is [nodes[a][0], nodes[a][n[a]-1]]);
   each node owns the box between the midpoints to its neighbours (the
   trapezoid rule on non-uniform nodes).  The library copies the nodes. */
typedef struct {
  int n[3];
  double lo[3], hi[3];
  int rule;
  const double *nodes[3]; /* IBDVM_RULE_NODES only (else ignored) */
} ibdvm_vgrid_desc;

/* Gas and run parameters (Sec. 4): Knudsen and Mach numbers, Prandtl number,
   specific-heat ratio, VHS omega and alpha (Eq. viscosity: mu0 from Kn),
   freestream density, temperature and flow direction (U = Ma sqrt(gamma T/2)),
   CFL number or a fixed dt (> 0 overrides the CFL), precision (IBDVM_FP64 or
   IBDVM_MIXED: FP32 storage of f and FP32 transport/relaxation, FP64 wall
   balance, forces and residual), method flags. */
typedef struct {
  double Kn, Ma, Pr, gamma, omega_vhs, alpha_vhs;
  double rho_inf, T_inf;
  double dir[3];
  double cfl, dt;
  int precision;
  int flags;
} ibdvm_gas_desc;

/* Tree-refined grid (the tree-based AMR meshes of Sec. 4.2-4.4, which the
   paper states but does not specify): nleaf leaves of a quadtree (2D) or an
   octree (3D) over the root grid of ibdvm_create_tree, leaf c of level
   level[c] (0 = a root cell, edge halved per level, at most maxlevel <= 12)
   at integer coordinates (ix[c], iy[c], iz[c]) of its level (0 <= ix < n[0]
   2^level; iz NULL in 2D).  The leaves must tile the domain and face
   neighbours differ by at most one level (2:1: a face borders one leaf or
   2^(dim-1) finer ones).  The arrays are read during the call only. */
typedef struct {
  int nleaf;
  int maxlevel;
  const int *level, *ix, *iy;
  const int *iz;
} ibdvm_tree_desc;

/* Immersed body and its wall (Sec. 2.3): Maxwell accommodation coefficient
   accom_alpha in [0,1] (1 = fully diffuse), wall temperature T_w and velocity
   U_w; L_ref is the reference length (2D, per unit span) or area (3D) of the
   force coefficients (<= 0: diameter, major axis, chord or pi r^2). */
typedef struct {
  int kind;
  double center[3], radii[3], angle;
  const double *verts;
  int nverts;
  double accom_alpha, T_w, U_w[3], L_ref;
} ibdvm_body_desc;

typedef struct {
  int dim, ncomp;
  long long ncell, nfluid;
  int nvel, nvel_padded;
  int nlink, nghost;
  double dt;
  int precision;
  long long steps_done;
  size_t device_bytes;
  int sweep_variant; /* 0: plain sweep (kernels.cu), 1: TMA-staged 2D FP32 sweep (sweep_tma.cu),
                        2: TMA-staged 3D FP32 sweep (sweep3d_tma.cu), 3: the sweep of a
                        tree-refined grid (kernels.cu) */
} ibdvm_info;

/* Creates a context: the uniform Cartesian grid and the discrete velocity
   grid with its quadrature weights (Sec. 2.2, Eq. quadrature), the gas in the
   non-dimensional form of Sec. 4 (rho_inf = T_inf = 1, |U_inf| = Ma sqrt(gamma
   / 2), the VHS viscosity mu = mu0 T^omega with mu0 from Kn, tau = mu / p),
   dt from the CFL number when gas->dt <= 0 (dt = CFL / sum_a max|xi_a| / dx_a,
   a reading: the paper gives none), the freestream Maxwellian in every cell,
   no body.  cuda_stream is a cudaStream_t (NULL = the legacy default stream);
   the context keeps it for every launch.  The context owns all device memory
   it allocates (ibdvm_destroy frees it); descriptors are copied, not kept.
   Errors: IBDVM_E_INVAL (bad descriptor), IBDVM_E_NOMEM (device memory short:
   checked against cudaMemGetInfo before allocating), IBDVM_E_CUDA. */
ibdvm_status ibdvm_create_grid(const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid,
                               const ibdvm_gas_desc *gas, void *cuda_stream, ibdvm_ctx **out);

/* Creates a context on a tree-refined grid: root is the grid of level-0
   cells (dim 2 or 3), tree its leaves (ibdvm_tree_desc), which are the cells of
   the context in the order given (ncell = nleaf; ibdvm_moments, ibdvm_get_f
   and ibdvm_set_f index them so).  Finite volumes on the leaves: the van Leer
   slope of a leaf along an axis from the value on each side (the neighbour,
   the mean of the finer neighbours, or the freestream halo) over the distance
   between centres; the upwind leaf's face value; a side shared with finer
   leaves takes the mean of their face values, so every interface conserves;
   dt from the CFL number with the finest edge.  FP64 or mixed precision (the
   mixed path keeps FP32 f and runs the same kernel in FP32).  A body may be
   placed with ibdvm_set_body (below); no domain walls: ibdvm_set_domain
   returns IBDVM_E_STATE on such a context, which cannot join a batch.  The
   context keeps the geometry of the finest uniform grid (root.n 2^maxlevel
   cells per axis) on the host for the body.  Errors as ibdvm_create_grid;
   IBDVM_E_INVAL (with a message) for leaves that do not tile the domain or
   face neighbours more than one level apart. */
ibdvm_status ibdvm_create_tree(const ibdvm_grid_desc *root, const ibdvm_tree_desc *tree,
                               const ibdvm_vgrid_desc *vgrid, const ibdvm_gas_desc *gas, void *cuda_stream,
                               ibdvm_ctx **out);

/* The face neighbours of every leaf of a tree context: nb[leaf][side][m]
   with side = 2a + (s > 0) and m < 2^(dim-1) (-1: none; the first is -1 at
   the domain edge, the others unless finer leaves share the side, in the
   order met with the first transverse axis fastest).  IBDVM_E_STATE on a
   context that is not a tree. */
ibdvm_status ibdvm_tree_neighbours(const ibdvm_ctx *ctx, long long *nb);

/* Places the body (Sec. 3.2.1): classifies the cells, builds one link per
   (ghost cell, fluid face neighbour) with its intersect point, normal, donor,
   auxiliary cell and shifted point, the surface-cell lists, and the
   incident-side velocity measures of the cut cells (Sec. 3.2.3).  Resets
   nothing else: f is kept.  On a tree context (reading C29 of the tree
   meshes of Sec. 4.2-4.4) the body is placed on the finest uniform grid and
   its ghost band moved onto the leaves; every cell the band reads or writes
   (ghosts, donors, auxiliary cells and the cells beyond the donors, surface
   cells and their fluid neighbours) must be a leaf of the finest level and
   every coarser leaf all fluid or all solid, else IBDVM_E_INVAL with a
   message and the context unchanged.  Errors: IBDVM_E_INVAL, IBDVM_E_NOMEM,
   IBDVM_E_CUDA. */
ibdvm_status ibdvm_set_body(ibdvm_ctx *ctx, const ibdvm_body_desc *body);

/* Domain faces, index 2a + (s > 0): x-, x+, y-, y+, z-, z+.  A freestream face
   has two halo layers holding the freestream Maxwellian (the default).  A
   diffuse wall face is the Maxwell wall of Sec. 2.3 with alpha = 1 on the
   plane of the face (normal into the domain): for velocities entering the
   domain through it, both halo layers hold rho_w times the unit-density wall
   Maxwellian at (T_w, U_w) (2D reduced: H_w = exp(-|xi - U_w|^2 / T_w) /
   (pi T_w), B_w = T_w / 2 H_w); for the other velocities they hold the
   boundary cell's own value, so the outgoing face value is the cell value;
   rho_w (FP64, per boundary cell, from f^n each step) makes the mass flux
   through the face zero, the velocities split by the plane xi_a = 0 (the
   lid-driven cavity of Sec. 4.1). */
enum { IBDVM_FACE_FREESTREAM = 0, IBDVM_FACE_DIFFUSE_WALL = 1 };
typedef struct {
  int kind[6];       /* IBDVM_FACE_*; the z faces of a 2D grid must be freestream */
  double T_w[6];     /* wall temperature (> 0) of a diffuse wall face */
  double U_w[6][3];  /* wall velocity; its normal component does not move the split plane */
} ibdvm_domain_desc;

/* Sets the domain faces.  FP32 cases keep their TMA sweep, which reads the
   wall halo at the domain faces; FP64 cases run the generic sweep kernel.
   Cases with a wall cannot be batch members.  The state is kept.  With any wall the library allocates
   (2 ncell / n[a] summed over the D axes) * nvel_padded * ncomp elements of
   the storage type for the halo values, and frees them with the context or
   on the next call.
   Errors: IBDVM_E_INVAL (a bad kind, a z wall in 2D, T_w <= 0 or a
   non-finite U_w; nothing changes), IBDVM_E_STATE (the context is a batch
   member), IBDVM_E_NOMEM. */
ibdvm_status ibdvm_set_domain(ibdvm_ctx *ctx, const ibdvm_domain_desc *d);

/* Advances nsteps forward-Euler steps (Sec. 4): ghost band, then transport
   and relaxation of every fluid cell, then the moments.  residual_out
   (nullable) receives the residual of the last step (Sec. 4 convergence
   criterion).  Errors: IBDVM_E_INVAL (nsteps < 0), IBDVM_E_UNSTABLE,
   IBDVM_E_NONFINITE (the state is then the one after the failing step),
   IBDVM_E_CUDA. */
ibdvm_status ibdvm_step(ibdvm_ctx *ctx, int nsteps, double *residual_out);

/* Conservative variables W[cell][dim+2] = (rho, rho U, rho E) and heat flux
   q[cell][dim] of the current state (Eqs. moments1-3; plain quadrature), and
   the cell classes (nullable outputs).  Values of non-fluid cells are not
   meaningful. */
ibdvm_status ibdvm_moments(ibdvm_ctx *ctx, double *W, double *q, unsigned char *celltype);

/* Surface force F[3] (per unit span in 2D) and heat flux Q into the body:
   momentum and energy carried into the solid through the donor-ghost faces by
   the face fluxes of the update, on the current state; CD, CL normalised by
   rho_inf U^2 L_ref / 2 along and normal to the flow (normalisation of the
   pressure coefficient, Sec. 4.3).  Any output may be NULL. */
ibdvm_status ibdvm_forces(ibdvm_ctx *ctx, double F[3], double *Q, double *CD, double *CL);

/* The surface force and heat flux of the face fluxes that the last
   ibdvm_step applied (computed on the device every step, FP64), normalised as
   in ibdvm_forces.  Any output may be NULL.  Before the first step: zeros. */
ibdvm_status ibdvm_step_forces(ibdvm_ctx *ctx, double F[3], double *Q, double *CD, double *CL);

/* State transfer in FP64: f[cell][k][comp] with k < nvel (padding excluded). */
ibdvm_status ibdvm_get_f(ibdvm_ctx *ctx, double *f);
ibdvm_status ibdvm_set_f(ibdvm_ctx *ctx, const double *f);

/* State transfer in the storage precision and layout: f[cell][k_padded][comp]
   of double (FP64) or float (mixed); bytes must equal
   ncell * nvel_padded * ncomp * sizeof(element).  Velocity k (natural order,
   x index fastest) sits at position pos[k] of ibdvm_velocity_positions; the
   other positions are padding, zero in every state the library writes.
   Pinned host memory makes these copies asynchronous-capable; they complete
   before returning. */
ibdvm_status ibdvm_get_f_native(ibdvm_ctx *ctx, void *host, size_t bytes);
ibdvm_status ibdvm_set_f_native(ibdvm_ctx *ctx, const void *host, size_t bytes);

/* The native position of every velocity: pos[nvel] (caller-owned) receives,
   for velocity k in the natural order of the velocity grid, its index in
   [0, nvel_padded) along the velocity axis of the native layout.  It is k
   itself, except for 3D cases in FP32 storage with the TMA sweep, which store
   the velocities grouped by the signs of their components (octants, each
   padded to whole sweep chunks) so that every chunk has one upwind direction
   per axis.  A layout choice of this library; the paper prescribes none. */
ibdvm_status ibdvm_velocity_positions(const ibdvm_ctx *ctx, int *pos);

/* The ghost band of the current state (Sec. 3.2.1 steps 1-4) for every link:
   incident distribution at the intersect point fiw, wall distribution fstarw,
   ghost value fstargc ([link][k][comp], nullable) and wall density rhow[link]. */
ibdvm_status ibdvm_ghost_band(ibdvm_ctx *ctx, double *fiw, double *fstarw, double *fstargc,
                              double *rhow);

/* Wall-point quantities of the current state, one row of IBDVM_WALL_COLS
   doubles per link (links in the order of ibdvm_geom_links, whose xw and nw
   give each row's intersect point and unit normal into the gas).  Each row
   holds moments (Sec. 2.1, Eqs. moments1-3) of the wall distribution f*_w of
   Sec. 2.3 (Eqs. general bc, Maxwell BC, fwc) at the intersect point: the
   surface pressure, shear stress, heat flux, slip and temperature jump the
   paper reports along walls (Sec. 4.2-4.4), and C_p of Sec. 4.3.  With h the
   mass-carrying component (f in 3D), b the second reduced one (0 in 3D) and
   the velocity-box weights w (the cut boxes of f*_w already hold the blend of
   their incident and reflected parts):
     IBDVM_WALL_RHO     rho = sum w h
     IBDVM_WALL_SLIP    3 values: U - U_w, U = sum w xi h / rho
     IBDVM_WALL_T       T with 3/2 rho T = sum w (|c|^2 h + b), c = xi - U
     IBDVM_WALL_TJUMP   T - T_w
     IBDVM_WALL_P       p = n.P.n, P_ab = sum w c_a c_b h (normal stress)
     IBDVM_WALL_TAU     3 values: P.n - p n (tangential stress)
     IBDVM_WALL_QN      n.q, q = 1/2 sum w c (|c|^2 h + b) (Eq. moments3)
     IBDVM_WALL_CP      2 (p - p_0) / (rho_0 |U_0|^2), p_0 = rho_0 T_0 / 2;
                        NaN without a free-stream velocity
   Computed on the device (the ghost band writes f*_w in FP64 into a scratch
   buffer of nlink * nvel_padded * ncomp doubles, allocated for the call, and
   one block per link reduces it in FP64); the state is not changed.  out is
   caller-owned host memory of nlink * IBDVM_WALL_COLS doubles; nothing is
   written when the body has no links.  E_INVAL for a NULL out, E_NOMEM when
   the scratch buffer cannot be allocated. */
enum {
  IBDVM_WALL_RHO = 0,
  IBDVM_WALL_SLIP = 1,
  IBDVM_WALL_T = 4,
  IBDVM_WALL_TJUMP = 5,
  IBDVM_WALL_P = 6,
  IBDVM_WALL_TAU = 7,
  IBDVM_WALL_QN = 10,
  IBDVM_WALL_CP = 11,
  IBDVM_WALL_COLS = 12
};
ibdvm_status ibdvm_wall(ibdvm_ctx *ctx, double *out);

/* Kernel timing.  With profiling on, every kernel launch class is bracketed
   by CUDA events on the context's stream; ms[8] receives the accumulated
   device time and launches[8] the number of kernel launches per class
   (0 ghost band, 1 transport/relaxation sweep, 2 moments and residual,
   3 forces, 4-7 reserved).  Launch counts are kept with profiling off too. */
ibdvm_status ibdvm_set_profiling(ibdvm_ctx *ctx, int on);
ibdvm_status ibdvm_get_kernel_times(ibdvm_ctx *ctx, double *ms, long long *launches);
ibdvm_status ibdvm_reset_kernel_times(ibdvm_ctx *ctx);

/* Residual without any device allocation.  The paper has no counterpart:
   this is a service for callers that cannot allocate device memory when they
   need the residual -- code running while another runtime owns the device
   memory pool and forbids cudaMalloc, hosts that must keep a fixed footprint
   after start-up, and work enqueued between other launches where an
   allocation would synchronise the device.  It returns, on the device, the
   same residual that ibdvm_step reports (max over components of
   sqrt(sum_j dW_ij^2) / sum_j |W_ij|, cells with celltype != fluid skipped,
   components whose sum of |W| is zero skipped).
     W_old, W_new  device arrays [ncell][dim+2], FP64, caller-owned (the
                   layout ibdvm_moments writes on the host);
     celltype      device array [ncell] of IBDVM_CELL_* or NULL (all cells count);
     residual      device pointer to one double, caller-owned; written on the stream;
     cuda_stream   cudaStream_t (NULL = legacy default stream); the call is
                   asynchronous and does not synchronise.
   Partial sums live in a built-in device array of 8192 x 10 doubles (640 KiB,
   held by every GPU that loads the library until exit), so ncell is limited
   to 2,097,152; larger sizes return IBDVM_E_INVAL with the limit in
   ibdvm_last_error(NULL).  The first call in each CUDA context (the one
   current at the call: the device's primary context for runtime-API callers,
   made current if none is; or a context the caller made current with the
   driver API) looks up the array's device address in that context
   (cudaGetSymbolAddress) and caches it under the context's handle: make that
   first call before any stream capture.  A context destroyed and replaced by
   one with the same handle (cudaDeviceReset) is not detected: make the first
   call again outside any capture.  All calls share the array and it keeps the
   last call's contents; calls that overlap on the GPU race on it and must be
   serialised by the caller. */
ibdvm_status ibdvm_residual_noalloc(const double *W_old, const double *W_new,
                                    const unsigned char *celltype, long long ncell, int dim,
                                    double *residual, void *cuda_stream);

/* Check of the bounded device waits (the paper has no counterpart).  The
   TMA-staged sweeps wait on mbarriers for their tile copies with a bound and
   report IBDVM_E_TIMEOUT instead of hanging when a copy never arrives; this
   runs that same bounded wait in a one-block kernel on a barrier that expects
   16 bytes, delivered by a bulk copy (deliver != 0: returns IBDVM_OK) or never
   delivered (deliver == 0: the wait gives up after spin_limit polls and the
   call returns IBDVM_E_TIMEOUT, the context of the device still usable).
   seconds (nullable) receives the wall time of the call.  spin_limit in
   [0, 2^18] (a poll suspends a few microseconds on GB300, so 2^18 polls are about
   one second, the bound of the sweeps); errors: IBDVM_E_INVAL, IBDVM_E_CUDA. */
ibdvm_status ibdvm_selftest_bounded_wait(int deliver, int spin_limit, double *seconds, void *cuda_stream);

/* This GPU's FP64 arithmetic rate, the roof of the FP64 path (whose sweep is
   bound by the FP64 pipe, not by HBM): eight independent FMA chains per
   thread, iters x 4 FMAs per chain, on eight blocks of 256 threads per SM,
   timed with CUDA events on cuda_stream (NULL = default) after one untimed
   launch.  *tflops receives the rate in TFLOP/s (an FMA counts as two
   flops), *ms (nullable) the time of the timed launch.  Allocates and frees a
   small device buffer; IBDVM_E_INVAL for iters <= 0 or tflops NULL,
   IBDVM_E_CUDA on a CUDA failure.  A measurement of the device, not of the
   paper's method. */
ibdvm_status ibdvm_fp64_fma_rate(int iters, double *tflops, double *ms, void *cuda_stream);

ibdvm_status ibdvm_get_info(const ibdvm_ctx *ctx, ibdvm_info *info);
ibdvm_status ibdvm_set_stream(ibdvm_ctx *ctx, void *cuda_stream);
/* Geometry of the context (host copy); see ibdvm_geom_* for the layouts. */
const ibdvm_geom *ibdvm_get_geom(const ibdvm_ctx *ctx);
void ibdvm_destroy(ibdvm_ctx *ctx);
const char *ibdvm_last_error(const ibdvm_ctx *ctx);
const char *ibdvm_status_string(ibdvm_status s);

/* ------------------------------------------------------------------------
 * Batched form: many cases of uneven size advanced together.  The paper
 * solves one case at a time; batching changes no arithmetic.  A member's
 * step is the one ibdvm_step takes (the same kernel bodies), launched for all
 * members at once:
 *   - one grouped ghost-band launch over every member's links (Sec. 3.2);
 *   - one grouped force launch, plus one block per member for the totals;
 *   - one persistent transport / relaxation / moment sweep (Sec. 2.2, Sec. 4)
 *     over a packed work list of items, largest first, which the blocks take
 *     from a device counter: (member, 8-column strip, velocity chunk, row
 *     range) in 2D, (member, 4 x 4 column tile, 128-velocity chunk, plane
 *     range) in 3D;
 *   - one grouped finalize launch, plus one block per member for its residual.
 * Pairs of steps replay captured CUDA graphs.
 *
 * Members are contexts in FP32 storage (IBDVM_MIXED) with the TMA sweep
 * (ibdvm_info.sweep_variant 1 in 2D, 2 in 3D), all of one dimension, bound to
 * the batch's stream.  A batch references its members and does not own them;
 * a context belongs to at most one batch, and ibdvm_destroy takes a member
 * out of its batch.  Members can be added and removed between steps
 * (continuous batching): a change of membership, of a member's body or of the
 * tiling rebuilds the batch's device tables (small uploads, synchronous) and
 * drops its graphs.  Not thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct ibdvm_batch ibdvm_batch;

/* Errors: IBDVM_E_INVAL (out is NULL), IBDVM_E_NOMEM. */
ibdvm_status ibdvm_batch_create(void *cuda_stream, ibdvm_batch **out);
/* Appends ctx.  Errors: IBDVM_E_INVAL (NULL, not FP32 with the TMA sweep,
   another dimension than the members, or bound to another stream),
   IBDVM_E_STATE (already a member of a batch). */
ibdvm_status ibdvm_batch_add(ibdvm_batch *b, ibdvm_ctx *ctx);
/* Removes ctx; later members move up one place.  Errors: IBDVM_E_INVAL (not a
   member of b). */
ibdvm_status ibdvm_batch_remove(ibdvm_batch *b, ibdvm_ctx *ctx);
/* Number of members (-1 for NULL) and member i in order of addition (NULL if
   out of range). */
int ibdvm_batch_size(const ibdvm_batch *b);
ibdvm_ctx *ibdvm_batch_member(const ibdvm_batch *b, int i);

/* Advances every member nsteps steps.  residuals[m] (nullable) receives the
   residual of member m's last step, statuses[m] (nullable) its status
   (IBDVM_OK, IBDVM_E_UNSTABLE, IBDVM_E_NONFINITE, IBDVM_E_TIMEOUT).  Returns
   IBDVM_OK when every member is OK, else the status of the first member that
   is not (its index is in the message); the members' states are then the ones
   after the last step, as with ibdvm_step.  IBDVM_E_CUDA on a failed launch;
   IBDVM_E_INVAL for nsteps < 0. */
ibdvm_status ibdvm_batch_step(ibdvm_batch *b, int nsteps, double *residuals, int *statuses);

/* Surface force and heat flux of the face fluxes that the last batched step
   applied, per member: F[m][3], Q[m], CD[m], CL[m] (each nullable), normalised
   as in ibdvm_forces.  Zeros for a member that has not stepped since the
   batch last rebuilt its tables (a change of membership, body or tiling). */
ibdvm_status ibdvm_batch_forces(ibdvm_batch *b, double *F, double *Q, double *CD, double *CL);

/* Tiling of the sweep's work items.  rows: target rows (3D: planes) per item
   (0 = whole columns).  kpt (0, 2 or 4) is accepted and has no effect: every
   member's sweep takes the velocity chunks of its orthant layout (2D: 192,
   128 or 64 velocities; 3D: 256 or 128), and get_tiling reports the
   velocities per lane of the first member's chunk (chunk / 32; 0 without
   members), the number of work items, the persistent grid and whether graphs
   are in use. */
typedef struct {
  int rows, kpt, nitems, grid, graphs;
} ibdvm_batch_tiling;
ibdvm_status ibdvm_batch_set_tiling(ibdvm_batch *b, int rows, int kpt);
ibdvm_status ibdvm_batch_get_tiling(const ibdvm_batch *b, ibdvm_batch_tiling *out);

/* Autotuner: for each candidate tiling (rows in {16, 32, 64, 128, whole
   columns}) times steps_per_trial batched steps (even, >= 2) with CUDA
   events on the batch's stream, after one untimed pair of steps, and keeps
   the fastest.  The trials are real steps: every member advances
   5 x (steps_per_trial + 2) steps.  best_ms (nullable) receives
   the kept tiling's time per step.  Errors: as ibdvm_batch_step;
   IBDVM_E_INVAL for a bad steps_per_trial; IBDVM_E_STATE with no members. */
ibdvm_status ibdvm_batch_tune(ibdvm_batch *b, int steps_per_trial, double *best_ms);

/* Kernel timing of the batched launches, classes as ibdvm_get_kernel_times;
   steps are not captured in graphs while profiling is on. */
ibdvm_status ibdvm_batch_set_profiling(ibdvm_batch *b, int on);
ibdvm_status ibdvm_batch_get_kernel_times(ibdvm_batch *b, double *ms, long long *launches);
ibdvm_status ibdvm_batch_reset_kernel_times(ibdvm_batch *b);

/* Releases the batch's tables and graphs; the members stay valid. */
void ibdvm_batch_destroy(ibdvm_batch *b);
const char *ibdvm_batch_last_error(const ibdvm_batch *b);

/* ------------------------------------------------------------------------
 * Serving: a request loop over many solves.  Requests (a case: grid,
 * velocity grid, gas, body) are queued on submission and admitted first come
 * first served while the device bytes of the admitted cases stay within an
 * HBM budget; each admitted request is a context in FP32 storage that joins a
 * batch (one for 2D, one for 3D cases, on two streams, so their launches
 * overlap on the device); every poll advances all admitted requests by a
 * round of steps, then retires those whose residual (Sec. 4 criterion) is
 * below the tolerance, those that failed and those that reached the step cap,
 * with the surface force and heat flux of their last state (ibdvm_forces),
 * and frees their memory for the queue.  A request's result does not depend on
 * the other requests (a member of a batch steps as it would alone).
 * sequential_fp64 = 1 gives the plain form for comparison: one request at a
 * time, in the FP64 path, without batching.  Not thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct ibdvm_server ibdvm_server;

typedef struct {
  double tol;            /* residual below which a request is done (e.g. 1e-6) */
  long long max_steps;   /* a request still above tol after max_steps ends with IBDVM_E_NOTCONVERGED */
  int steps_per_round;   /* steps per poll between convergence checks (even, >= 2) */
  size_t hbm_budget;     /* device bytes the admitted cases may hold; 0 = 90% of the free memory at creation */
  int max_active;        /* requests on the device at once; 0 = no cap */
  int sequential_fp64;   /* 1: one request at a time in the FP64 path (the plain form) */
} ibdvm_server_desc;

typedef struct {
  long long id;
  int done;              /* 1 when the request has left the device */
  int status;            /* IBDVM_OK (converged), IBDVM_E_NOTCONVERGED (step cap), IBDVM_E_STATE
                            (cancelled), or the error */
  long long steps;       /* steps taken */
  double residual;       /* residual of the last step */
  double F[3], Q, CD, CL; /* as ibdvm_forces, on the final state */
  double t_submit, t_admit, t_done; /* seconds since the server was created (-1: not yet) */
  size_t device_bytes;   /* device bytes of the request's context */
} ibdvm_result;

/* Errors: IBDVM_E_INVAL (bad descriptor: tol < 0, max_steps < 1, odd or
   small steps_per_round), IBDVM_E_NOMEM, IBDVM_E_CUDA. */
ibdvm_status ibdvm_server_create(const ibdvm_server_desc *desc, ibdvm_server **out);
/* Queues a request; the descriptors are copied (gas->precision is replaced by
   the server's).  id receives the request's id (consecutive from 0).
   Errors: IBDVM_E_INVAL (NULL or invalid descriptor: the grid and velocity
   grid are checked here, the body when the request is admitted). */
ibdvm_status ibdvm_server_submit(ibdvm_server *s, const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid,
                                 const ibdvm_gas_desc *gas, const ibdvm_body_desc *body, long long *id);
/* One scheduling round: admits queued requests, advances the admitted ones by
   steps_per_round steps and retires the finished ones.  Outputs (nullable):
   requests on the device, in the queue, and finished in this round.  A
   request that fails is retired with its status; the call itself fails only
   on a CUDA error of the loop. */
ibdvm_status ibdvm_server_poll(ibdvm_server *s, int *nactive, int *nqueued, int *nfinished);
/* Cancels request id between polls: a queued request leaves the queue, an
   admitted one leaves the device (its memory is freed) with the force and
   heat flux of its current state; either is done with status IBDVM_E_STATE.
   Cancelling a finished request does nothing.  The other requests are not
   affected.  Errors: IBDVM_E_INVAL (unknown id). */
ibdvm_status ibdvm_server_cancel(ibdvm_server *s, long long id);
/* The state of request id (done = 0 while queued or on the device).
   Errors: IBDVM_E_INVAL (unknown id). */
ibdvm_status ibdvm_server_result(ibdvm_server *s, long long id, ibdvm_result *out);
/* Seconds since the server was created (the clock of the result times). */
double ibdvm_server_clock(const ibdvm_server *s);
/* Destroys the server and every context it still holds. */
void ibdvm_server_destroy(ibdvm_server *s);
const char *ibdvm_server_last_error(const ibdvm_server *s);

/* ------------------------------------------------------------------------
 * Host-only geometry (no GPU needed): the classification, links, surface
 * cells and cut-cell table that ibdvm_set_body builds.
 * ------------------------------------------------------------------------ */
ibdvm_status ibdvm_geom_build(const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid,
                              const ibdvm_gas_desc *gas, const ibdvm_body_desc *body,
                              ibdvm_geom **out);
/* sizes[8] = ncell, nvel, ncomp, nlink, nghost, nfluid, nsurf, nvel_padded */
ibdvm_status ibdvm_geom_sizes(const ibdvm_geom *g, long long *sizes);
ibdvm_status ibdvm_geom_cells(const ibdvm_geom *g, unsigned char *types);
/* links in canonical order: ghost cell ascending, then direction 2*axis + (side > 0);
   side = sign of (x_donor - x_ghost) along axis; aux = -1 when unusable;
   xw[link][3] intersect point, nw[link][3] unit normal into the gas */
ibdvm_status ibdvm_geom_links(const ibdvm_geom *g, int *ghost, int *donor, int *aux, int *axis,
                              int *side, double *xw, double *nw);
/* incident-side measure omega^g[link][k] of every velocity box */
ibdvm_status ibdvm_geom_cut_table(const ibdvm_geom *g, double *wg);
ibdvm_status ibdvm_geom_velocities(const ibdvm_geom *g, double *xi, double *w);
/* surface cells: ghost_cell[nghost], offsets[nghost+1], cells[nsurf] */
ibdvm_status ibdvm_geom_surface(const ibdvm_geom *g, int *ghost_cell, int *offsets, int *cells);
double ibdvm_geom_dt(const ibdvm_geom *g);
void ibdvm_geom_destroy(ibdvm_geom *g);
const char *ibdvm_geom_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
