// ctx.h -- the solver context behind the C-ABI handle and the kernel launch
// interface shared by capi.cpp and the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "geom.h"

namespace ibdvm {

// Per-cell macroscopic slots (array of [ncell][kMac] in the storage type, so a
// cell's parameters are three aligned 16-byte vectors in FP32): the Shakhov
// equilibrium parameters of the current state (Sec. 2.1, Sec. 4).
enum MacSlot {
  kPre = 0,    // rho / (pi T)      (2D reduced)  or rho / (pi T)^{3/2}  (3D)
  kU0 = 1,     // U_x, U_y, U_z
  kInvT = 4,   // 1 / T
  kHalfT = 5,  // T / 2              (B = T/2 H, Sec. 4)
  kShA = 6,    // 4 (1 - Pr) / (5 rho T^2)
  kQ0 = 7,     // q_x, q_y, q_z
  kDtTau = 10, // dt / tau, tau = mu / p, mu = mu0 T^omega
  kMac = 12
};

// kernel classes of the timing counters
enum KernelClass { kKGhost = 0, kKSweep = 1, kKMoments = 2, kKForces = 3, kKOther = 4 };

// columns of the wall-point quantities (ibdvm_wall)
constexpr int kWallCols = 12;

// cell ranges of a pipelined host upload of the state (ibdvm_set_f_native)
constexpr int kUploadParts = 8;

// flags written by the moment kernel
enum : int { kFlagNonFinite = 1, kFlagUnstable = 2, kFlagTimeout = 4 };

} // namespace ibdvm

struct ibdvm_batch; // batch.cpp

struct ibdvm_ctx {
  ibdvm::Geom geom;
  cudaStream_t stream = nullptr;
  int precision = 0, dim = 2, ncomp = 2, nv = 0, nvp = 0;
  long long ncell = 0;
  size_t esize = 8;
  // state and per-cell data
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  void *mac = nullptr;       // [ncell][kMac]
  double *W[2] = {nullptr, nullptr}; // [dim+2][ncell]
  int wcur = 0;
  double *part = nullptr;    // moment partial sums [nchunk][NM][ncell]
  int nchunk = 1, kloop = 1;
  double *resblk = nullptr;  // residual partial sums per block
  int nresblk = 0;
  double *d_res = nullptr;   // residual scalar
  int *d_flags = nullptr;
  // velocity tables, indexed by the stored position of a velocity
  void *xiT = nullptr, *wT = nullptr, *finf = nullptr;
  double *xiD = nullptr, *wD = nullptr; // wD: [2][nvp], the weights then their reciprocals (0 at padding)
  // stored position of every velocity in its natural order (x index fastest):
  // the identity, or, for the orthant layout of the FP32 TMA sweeps,
  // velocities grouped by the signs of their components with each group
  // padded to a whole number of sweep chunks (padding positions hold zero
  // weight and zero f)
  int *kst = nullptr;          // [nv] device
  std::vector<int> kst_h;      // [nv] host copy
  int oct_kc = 0;              // orthant layout: velocities per sweep chunk (0: natural order)
  float *oct_const = nullptr;  // orthant layout: per stored velocity |a_x|, |a_y|, |a_z| or w, w or 0 (FP32)
  uint8_t *oct_sign = nullptr; // orthant layout: per chunk, bit a set when component a is negative
  // cell tables
  uint8_t *ctype = nullptr;
  uint8_t *cmask = nullptr;  // per cell: ghost neighbour per face (bit 2a + (s > 0)), 64 = not fluid
  int *dslot = nullptr, *dlinks = nullptr;
  // TMA sweep of 2D FP32 cases (sweep_tma.cu)
  bool use_tma = false;
  float *partf = nullptr;    // FP32 moment partial sums [nchunk][9][ncell]
  int tma_nchunk = 0;
  alignas(64) unsigned char tmap[2][128];
  alignas(64) unsigned char tmap3[2][3][128]; // 3D: tile, x halo strip, y halo strip per buffer
  // ghost band
  int nlink = 0, nghost = 0, nsurf = 0;
  int *l_int = nullptr;      // [nlink][8]
  double *l_dbl = nullptr;   // [nlink][8]
  double *l_wg = nullptr;    // [nlink][nvp]
  int *g_int = nullptr;      // [nghost][4]
  int *s_int = nullptr;      // [nsurf][8]
  double *s_dbl = nullptr;   // [nsurf][8]
  void *lval = nullptr;      // [nlink][nvp][ncomp] ghost values f*_gc
  void *fi_scr = nullptr;    // [nlink][nvp][ncomp] incident distribution at the wall
  void *fsp_scr = nullptr;   // [nlink][nvp][ncomp] shifted-point value
  double *rhow = nullptr;    // [nlink]
  double *fpart = nullptr;   // [nlink][4] force partial sums
  double *gw_unit = nullptr; // [nvp] unit-density wall Maxwellian H_w / g_w of the body's wall
  double *d_forces = nullptr; // [4]
  double *d_step_forces = nullptr; // [4] forces of the fluxes the last step applied
  // kernel timing (CUDA events around each launch class, when enabled)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks; // (kernel class, index of the start event)
  double kernel_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long kernel_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // CUDA graphs of two consecutive steps, keyed by the parities of the state
  // and moment buffers at their start; replayed by ibdvm_step
  bool graphs_enabled = true;
  cudaGraphExec_t graph2[4] = {nullptr, nullptr, nullptr, nullptr};
  long long graph2_launches[4][8] = {};
  // the batch this context is a member of, and a counter of body changes
  // (a batch rebuilds its tables when it changes)
  ibdvm_batch *batch = nullptr;
  unsigned body_gen = 0;
  // diffuse domain walls: faces 2a + (s > 0) in wall_mask, their wall state,
  // the first halo slot of each face (wall_off[6] = all slots) and the halo
  // values [slots][nvp][ncomp] in the storage type
  int wall_mask = 0;
  double wall_T[6] = {1, 1, 1, 1, 1, 1};
  double wall_U[6][3] = {};
  long long wall_off[7] = {};
  void *whalo = nullptr;
  bool tma_ok = false; // the TMA sweep was set up (it serves cases with and without domain walls)
  // a tree-refined 2D grid: the cells are the leaves of a quadtree
  bool tree = false;
  int *tree_sti = nullptr;    // [leaf][10][8] stencil rows and flags (build_tree_stencils)
  double *tree_stg = nullptr; // [leaf][10][4] stencil geometry
  int *tree_lrec = nullptr;   // [leaf][8] side counts, regular flag
  int *tree_sched = nullptr;  // [leaf] the order of the leaves in the sweep's blocks
  double tree_h0[3] = {0, 0, 0};
  int tree_L = 0;
  std::vector<int> tree_lev_h, tree_own; // leaf levels; the leaf of every finest-grid cell
  ibdvm::Geom tree_vgeom;                // the finest grid (a body is placed there)
  int *tree_far = nullptr;               // [link] row beyond the donor (map_tree_body)
  int tree_qb[3] = {0, 0, 0}; // first stored velocity of the quadrants 1, 2, 3 (bit 0: x < 0, bit 1: y < 0)
  std::vector<int> tree_nb_h;
  // host uploads of the state in cell ranges (a copy stream, one event per range)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[ibdvm::kUploadParts + 1] = {};
  // bookkeeping
  long long steps = 0;
  size_t dev_bytes = 0;
  std::string err;
};

namespace ibdvm {

// Kernel launchers (kernels.cu).  All enqueue on ctx->stream and return the
// launch status.
cudaError_t launch_init_state(ibdvm_ctx *ctx);
// moments of f^n, W^n and the Shakhov parameters of the cells [c0, c1),
// without transport (two passes: about zero, then about the bulk velocity)
cudaError_t launch_refresh_range(ibdvm_ctx *ctx, long long c0, long long c1);
// W^n and q^n as rows per cell ([ncell][D + 2] and [ncell][D], device)
cudaError_t launch_interleave(ibdvm_ctx *ctx, double *Wo, double *qo);
// wall-point quantities per link ([nlink][kWallCols], device) from the wall
// distribution f*_w written by the ghost band ([nlink][nvp][ncomp], FP64)
cudaError_t launch_wall(ibdvm_ctx *ctx, const double *fstar, double *out);
cudaError_t launch_ghost_band(ibdvm_ctx *ctx, double *dbg_fstarw);
cudaError_t launch_sweep(ibdvm_ctx *ctx);
cudaError_t launch_forces(ibdvm_ctx *ctx, double *dst);
// TMA sweep (sweep_tma.cu)
bool tma_sweep_applicable(const ibdvm_ctx *ctx);
int tma_sweep_nchunk(const ibdvm_ctx *ctx);
cudaError_t tma_sweep_prepare(ibdvm_ctx *ctx);
cudaError_t tma_sweep_launch(ibdvm_ctx *ctx);
// The orthant layout of the velocities for the FP32 TMA sweeps (layout.cpp):
// chunks whose components have one sign each (quadrants in 2D, octants in
// 3D).  orthant_layout gives the stored position of every velocity of G
// (natural order), the padded count and the chunk size; orthant_tables fills
// the per-velocity constants (|a_x|, |a_y|, |a_z| or w, w or 0; a_a = dt xi_a /
// dx_a) and the per-chunk signs (bit a: component a negative).
int orthant_layout(const Geom &G, std::vector<int> &kst, int &nvp);
void orthant_tables(const Geom &G, const std::vector<int> &kst, int nvp, int kc, std::vector<float> &vconst,
                    std::vector<uint8_t> &sign);
// the driver's tensor-map encoder can be reached (the TMA sweeps can run)
bool tma_encoder_available();
// tree.cpp: the face neighbour tables of a tree-refined 2D grid; false with a
// message when the leaves do not tile the domain or break the 2:1 rule
// (own: the leaf of every cell of the finest grid, x fastest)
bool build_tree_mesh(const ibdvm_grid_desc &root, const ibdvm_tree_desc &t, std::vector<int> &lev,
                     std::vector<int> &nb, std::vector<int> &own, std::string &err);
// the sweep's stencil tables; type (leaf classes) and glink (the link from
// the ghost across side 2a + sd of a fluid leaf, [leaf][2 dim]) may be empty
// without a body
void build_tree_stencils(int D, const std::vector<int> &lev, const std::vector<int> &nb, const double h0[3],
                         const std::vector<uint8_t> &type, const std::vector<int> &glink,
                         std::vector<int> &sti, std::vector<double> &stg, std::vector<int> &lrec);
// the leaves in the order the sweep's blocks take them (regular, other fluid, solid)
std::vector<int> tree_schedule(int D, const std::vector<int> &lrec);
// the stencil entries of a leaf (D own + 2 D 2^(D-1) upwind) and the ints of an entry
__host__ __device__ constexpr int tree_entries(int D) { return D + 2 * D * (1 << (D - 1)); }
__host__ __device__ constexpr int tree_entry_ints(int D) { return D == 2 ? 8 : 12; }
// a body placed on the finest grid Gv of a tree, moved onto its leaves: false
// with a message unless every cell the ghost band reads or writes is a leaf
// of the finest level and every coarser leaf is all fluid or all solid.
// Gt receives the leaf classes and the ghost band in leaf indices; glink
// [leaf][2 dim] the link of a ghost face neighbour; far [link] the row the
// donor's slope sees beyond it along the link axis (a leaf, -2 the halo,
// -3 - l the ghost value of link l)
bool map_tree_body(const Geom &Gv, const std::vector<int> &own, const std::vector<int> &lev, int L, Geom &Gt,
                   std::vector<int> &glink, std::vector<int> &far, std::string &err);
// TMA sweep of 3D FP32 cases (sweep3d_tma.cu)
bool tma3_sweep_applicable(const ibdvm_ctx *ctx);
int tma3_sweep_nchunk(const ibdvm_ctx *ctx);
cudaError_t tma3_sweep_prepare(ibdvm_ctx *ctx);
cudaError_t tma3_sweep_launch(ibdvm_ctx *ctx);

// Grouped launches over the members of a batch (kernels.cu; FP32 storage, one
// dimension per batch).  Each member has two argument blocks, for the buffer
// parities after an even and an odd number of batched steps; the launch names
// the parity.  Member m writes its residual to res[m], ORs its flags into
// flags[m] and its step forces go to forces[4 m .. 4 m + 3].
struct GroupTables {
  int dim = 2, ncase = 0;
  void *ghost = nullptr, *force = nullptr, *fin = nullptr; // [ncase][2] argument blocks
  int *link_start = nullptr, *fin_start = nullptr;         // [ncase + 1] block prefix sums
  int link_blocks = 0, fin_blocks = 0;
};
cudaError_t group_build(const std::vector<ibdvm_ctx *> &cases, const std::vector<int> &nchunk, double *res,
                        int *flags, double *forces, GroupTables &t, cudaStream_t s);
void group_free(GroupTables &t);
cudaError_t group_ghost(const GroupTables &t, int par, cudaStream_t s);
cudaError_t group_forces(const GroupTables &t, int par, cudaStream_t s);
cudaError_t group_finalize(const GroupTables &t, int par, cudaStream_t s);

// The batched TMA sweep of 2D FP32 members (sweep_tma.cu): persistent
// launches over a packed work list of (member, column strip, velocity chunk,
// row range) items, one per chunk width of the members' layouts.  kpt is not
// used (the chunk is that of each member's layout); rows = target rows per
// item (0: whole columns).
struct SweepTables {
  void *args = nullptr, *tmaps = nullptr, *items = nullptr; // [ncase][2], [ncase][2], [nitems]
  int *next = nullptr; // work counters (2D: one per class)
  int nitems = 0, grid = 0, dim = 2;
  int ksel = 0;        // 3D: velocities per lane of every item (8 or 4), 0 for a mix
  // 2D: the items grouped by velocities per lane (6, 4, 2), one persistent
  // launch per class: items [cls_off[c], cls_off[c + 1]) on cls_grid[c] blocks
  int cls_off[4] = {0, 0, 0, 0}, cls_grid[3] = {0, 0, 0};
};
bool tma_batch_member_ok(const ibdvm_ctx *ctx);
int tma_batch_kpt_max(const ibdvm_ctx *ctx);
cudaError_t tma_batch_build(const std::vector<ibdvm_ctx *> &cases, const std::vector<int> &kpt, int rows,
                            int *flags, SweepTables &t, cudaStream_t s);
void tma_batch_free(SweepTables &t);
cudaError_t tma_batch_launch(const SweepTables &t, int par, cudaStream_t s);
// 3D members (sweep3d_tma.cu): 128-velocity chunks; zrows = target planes per
// item (0: whole columns)
cudaError_t tma3_batch_build(const std::vector<ibdvm_ctx *> &cases, int zrows, int *flags, SweepTables &t,
                             cudaStream_t s);
cudaError_t tma3_batch_launch(const SweepTables &t, int par, cudaStream_t s);

// batch.cpp: takes a context that is being destroyed out of its batch
void batch_detach(ibdvm_ctx *ctx);
// batch.cpp: enqueues nsteps batched steps without waiting for them, and
// waits for them and reads every member's residual and status
ibdvm_status batch_enqueue(ibdvm_batch *b, int nsteps);
ibdvm_status batch_collect(ibdvm_batch *b, double *residuals, int *statuses);
// capi.cpp: an upper estimate of the device bytes of a context (before its body is placed)
size_t estimate_ctx_bytes(const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid, const ibdvm_gas_desc *gas);
// capi.cpp: F[3], Q, CD, CL (each nullable) from the force sums h[4] of ctx
void force_outputs(const ibdvm_ctx *ctx, const double *h, double *F, double *Q, double *CD, double *CL);

// dense FP64 [ncells][nv][ncomp] (device) <-> cells [c0, c0 + ncells) of the current state
cudaError_t launch_convert(ibdvm_ctx *ctx, double *dense, long long c0, long long ncells, bool to_state);

} // namespace ibdvm
