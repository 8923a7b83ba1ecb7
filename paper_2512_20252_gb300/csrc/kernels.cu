// kernels.cu -- CUDA kernels (sm_103a) of one forward-Euler step of the
// ghost-cell immersed-boundary discrete velocity method (arXiv 2512.20252).
//
//   ghost_band_kernel   Sec. 3.2.1-3.2.3: per link, the upwind-weighted compact
//                       interpolation f_gc (Eqs. extrapolation 1, upwind), the
//                       shifted point (Eqs. sp, fsp), the incident distribution
//                       at the intersect point (Eq. fw), the wall density from
//                       zero normal mass flux with the cut-cell split (Eq. rhowc,
//                       FP64 block reduction), the cut-cell blend (Eq. fwc) and
//                       the ghost value (Eq. extrapolation 2).
//   sweep_kernel        Sec. 2.2 and Sec. 4: per (cell, velocity), van Leer
//                       limited upwind face values (Eqs. reconstruction,
//                       limiter), flux divergence, Shakhov relaxation with the
//                       reduced equilibria, forward Euler, and the velocity
//                       moments of the new state reduced per cell.
//   finalize_kernel     moments -> W, T, q, tau per cell; residual partial sums
//                       (Sec. 4, FP64).
//   forces kernels      momentum and energy through the donor-ghost faces (FP64).
//
// Storage type T is double (FP64 path) or float (mixed path: FP32 f, FP32
// transport and relaxation with compensated FP32 moment sums; FP64 wall
// balance, forces and residual).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "ctx.h"
#include "tma_sync.cuh"

namespace ibdvm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kThreadsPerCell = 64; // threads over velocities for one cell
constexpr int kCellsPerBlock = 4;   // cells of one sweep block
constexpr int kBlock = kThreadsPerCell * kCellsPerBlock;
constexpr int kGhostThreads = 512; // threads over the velocities of one link
// The ghost band's tiling: U velocities a thread takes at a time, and blocks
// of 512 threads per SM.  FP32 storage: two velocities at a time, two blocks
// per SM (64 registers); FP64 storage and the grouped launches of a batch
// (their arguments come from shared memory) need more registers: one block.
template <typename T, bool GROUPED> struct GhostTiling {
  static constexpr bool two = std::is_same<T, float>::value && !GROUPED;
  static constexpr int U = 2;
  static constexpr int blocks = two ? 2 : 1;
};

template <int D> struct Dims {
  static constexpr int NC = (D == 2) ? 2 : 1;   // components: (h, b) or f
  static constexpr int NM = (D == 2) ? 9 : 14;  // moment sums per cell
  static constexpr int NW = D + 2;              // conservative variables
};

// ---------------------------------------------------------------------------
// small numerics
// ---------------------------------------------------------------------------

// van Leer limited difference, Eq. limiter: (sgn a + sgn b)|a||b|/(|a|+|b|)
// written as 2ab/(a+b) when a and b have the same sign, 0 otherwise.
template <typename T> __device__ __forceinline__ T vanleer(T a, T b) {
  T p = a * b;
  return (p > T(0)) ? (T(2) * p) / (a + b) : T(0);
}

__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }

// round-to-nearest products and sums without contraction: the upwind-weight
// fallback is decided by an exact zero of xi.r, which fused multiply-adds
// would perturb
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

// Accumulator: plain sum in FP64, Neumaier-compensated sum in FP32.
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void merge(double os, double) { s += os; }
  __device__ __forceinline__ double hi() const { return s; }
  __device__ __forceinline__ double lo() const { return 0.0; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = __fadd_rn(s, x);
    c = __fadd_rn(c, (fabsf(s) >= fabsf(x)) ? __fadd_rn(__fsub_rn(s, t), x)
                                             : __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  __device__ __forceinline__ void merge(float os, float oc) {
    add(os);
    c = __fadd_rn(c, oc);
  }
  __device__ __forceinline__ float hi() const { return s; }
  __device__ __forceinline__ float lo() const { return c; }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------------------------
// the sweep: transport, relaxation and moments
// ---------------------------------------------------------------------------

// The domain halo (two layers across every domain face, Sec. 2.2): the
// freestream Maxwellian, or, across a diffuse domain wall, the values the wall
// gives both layers (rho_w M_w for velocities entering the domain, the
// boundary cell's own value for the others), one slot of nvp x NC values per
// boundary cell, refreshed from f^n by domain_wall_kernel.
template <typename T> struct HaloArgs {
  const T *__restrict__ whalo; // [slots][nvp][NC]; null without diffuse walls
  long long off[6];            // first slot of face 2a + (s > 0)
  int mask;                    // bit 2a + (s > 0): that face is a diffuse wall
};

// slot offset of cell ijk within the slots of a face normal to axis a
__device__ __forceinline__ long long face_slot(const int *n, const int *ijk, int a) {
  return (a == 0) ? ijk[1] + (long long)n[1] * ijk[2]
                  : (a == 1) ? ijk[0] + (long long)n[0] * ijk[2] : ijk[0] + (long long)n[0] * ijk[1];
}

// the halo value across face (a, s) of the boundary cell ijk, velocity k, component m
template <typename T>
__device__ __forceinline__ T halo_value(const HaloArgs<T> &H, const T *finf, const int *n, const int *ijk, int a,
                                        int s, int nvp, int nc, int k, int m) {
  const int i = 2 * a + (s > 0);
  if (!((H.mask >> i) & 1)) return finf[(size_t)k * nc + m];
  return H.whalo[((size_t)(H.off[i] + face_slot(n, ijk, a)) * nvp + k) * nc + m];
}

template <typename T> struct SweepArgs {
  const T *__restrict__ f;
  T *__restrict__ fn;
  const T *__restrict__ mac;
  const T *__restrict__ xi;   // [3][nvp]
  const T *__restrict__ w;    // [nvp]
  const T *__restrict__ finf; // [nvp][NC]
  const uint8_t *__restrict__ ctype;
  const int *__restrict__ dslot;
  const int *__restrict__ dlinks;
  const T *__restrict__ lval; // [nlink][nvp][NC]
  const int *__restrict__ kst; // [nv] stored position of each velocity (natural order)
  double *__restrict__ part;  // [nchunk][NM][ncell]
  long long ncell;
  int n[3];
  int nv, nvp, kloop;
  T dt;
  T rdx[3];
  int update; // 1: step f -> fn and take the moments of fn; 0: moments of f
  int shift;  // 1: moments about the stored bulk velocity U^n; 0: about zero
  HaloArgs<T> H;
};

// the NC components of one (cell, velocity): a vector access for (h, b) pairs
template <typename T, int NC>
__device__ __forceinline__ void load_nc(const T *p, T *o) {
  if constexpr (NC == 2 && sizeof(T) == 8) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    o[0] = v.x;
    o[1] = v.y;
  } else if constexpr (NC == 2 && sizeof(T) == 4) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    o[0] = v.x;
    o[1] = v.y;
  } else {
#pragma unroll
    for (int m = 0; m < NC; ++m) o[m] = p[m];
  }
}
template <typename T, int NC>
__device__ __forceinline__ void store_nc(T *p, const T *o) {
  if constexpr (NC == 2 && sizeof(T) == 8) {
    *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
  } else if constexpr (NC == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
  } else {
#pragma unroll
    for (int m = 0; m < NC; ++m) p[m] = o[m];
  }
}

// value of the cell across face (a, s) of fluid cell c, as c sees it: the
// freestream outside the domain (two halo layers), the link's ghost value for
// a ghost neighbour (one ghost value per link), else the neighbour's f
template <typename T, int NC>
__device__ __forceinline__ void seen(const SweepArgs<T> &A, long long c, const int *ijk, int a,
                                     int s, int k, T *out) {
  int q = ijk[a] + s;
  if (q < 0 || q >= A.n[a]) {
#pragma unroll
    for (int m = 0; m < NC; ++m) out[m] = halo_value(A.H, A.finf, A.n, ijk, a, s, A.nvp, NC, k, m);
    return;
  }
  long long stride = (a == 0) ? 1LL : (a == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1]);
  long long nb = c + s * stride;
  if (A.ctype[nb] == IBDVM_CELL_GHOST) {
    // every fluid face neighbour of a ghost is a donor with a link in this
    // direction; the guards only keep a corrupted table from reading out of bounds
    const int slot = A.dslot[c];
    const int l = (slot >= 0) ? A.dlinks[slot * 6 + 2 * a + (s > 0)] : -1;
    load_nc<T, NC>((l >= 0) ? A.lval + ((size_t)l * A.nvp + k) * NC : A.finf + (size_t)k * NC, out);
  } else {
    load_nc<T, NC>(A.f + ((size_t)nb * A.nvp + k) * NC, out);
  }
}

template <typename T> __device__ __forceinline__ T shfl_down(T v, int o) {
  return __shfl_down_sync(0xffffffffu, v, o);
}

template <typename T, int D>
__global__ void __launch_bounds__(kBlock) sweep_kernel(SweepArgs<T> A) {
  constexpr int NC = Dims<D>::NC;
  constexpr int NM = Dims<D>::NM;
  __shared__ double red[kCellsPerBlock][2][NM];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long c = (long long)blockIdx.x * kCellsPerBlock + ty;
  const int chunk = blockIdx.y;
  const bool active = (c < A.ncell) && (A.ctype[c] == IBDVM_CELL_FLUID);
  Acc<T> acc[NM];
  if (active) {
    int ijk[3];
    ijk[0] = (int)(c % A.n[0]);
    ijk[1] = (int)((c / A.n[0]) % A.n[1]);
    ijk[2] = (int)(c / ((long long)A.n[0] * A.n[1]));
    const T *M = A.mac;
    const long long nc = A.ncell;
    T U[3], q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      U[a] = A.shift ? M[c * kMac + kU0 + a] : T(0);
      q[a] = M[c * kMac + kQ0 + a];
    }
    const T pre = M[c * kMac + kPre], invT = M[c * kMac + kInvT], halfT = M[c * kMac + kHalfT];
    const T shA = M[c * kMac + kShA], dtau = M[c * kMac + kDtTau];
    for (int j = 0; j < A.kloop; ++j) {
      const int iv = (chunk * A.kloop + j) * kThreadsPerCell + tx;
      if (iv >= A.nv) break;
      const int k = A.kst[iv];
      T fc[NC];
      load_nc<T, NC>(A.f + ((size_t)c * A.nvp + k) * NC, fc);
      T cv[3] = {T(0), T(0), T(0)};
      T c2 = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        cv[a] = A.xi[a * A.nvp + k] - U[a];
        c2 += cv[a] * cv[a];
      }
      T fo[NC];
      if (A.update) {
        T div[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) div[m] = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const T xa = A.xi[a * A.nvp + k];
          if (xa == T(0)) continue;
          const int s = (xa > T(0)) ? 1 : -1;
          T fb[NC], ff[NC], fin[NC];
          seen<T, NC>(A, c, ijk, a, -s, k, fb);
          seen<T, NC>(A, c, ijk, a, s, k, ff);
          // upwind neighbour u = c - s e_a supplies the incoming face value
          const int qa = ijk[a] - s;
          if (qa < 0 || qa >= A.n[a]) {
            // halo: both layers hold the same value, zero slope
#pragma unroll
            for (int m = 0; m < NC; ++m) fin[m] = halo_value(A.H, A.finf, A.n, ijk, a, -s, A.nvp, NC, k, m);
          } else {
            long long stride = (a == 0) ? 1LL : (a == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1]);
            long long u = c - s * stride;
            if (A.ctype[u] == IBDVM_CELL_GHOST) {
              // ghost cell: link value with the one-sided slope toward the donor
#pragma unroll
              for (int m = 0; m < NC; ++m) fin[m] = T(0.5) * (fb[m] + fc[m]);
            } else {
              int iu[3] = {ijk[0], ijk[1], ijk[2]};
              iu[a] = qa;
              T fuu[NC];
              seen<T, NC>(A, u, iu, a, -s, k, fuu);
#pragma unroll
              for (int m = 0; m < NC; ++m)
                fin[m] = fb[m] + T(0.5) * vanleer(fb[m] - fuu[m], fc[m] - fb[m]);
            }
          }
          const T coef = fabs(xa) * A.rdx[a];
#pragma unroll
          for (int m = 0; m < NC; ++m) {
            T fout = fc[m] + T(0.5) * vanleer(fc[m] - fb[m], ff[m] - fc[m]);
            div[m] += coef * (fout - fin[m]);
          }
        }
        // Shakhov equilibrium (Sec. 4 reduced forms in 2D, Sec. 2.1 in 3D)
        T cq = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) cq += cv[a] * q[a];
        const T e = pre * exp_t(-c2 * invT);
        const T corr = shA * cq;
        const T tc = T(2) * c2 * invT;
        if (D == 2) {
          const T H = e * (T(1) + corr * (tc - T(4)));
          const T B = halfT * e * (T(1) + corr * (tc - T(2)));
          fo[0] = fc[0] - A.dt * div[0] + dtau * (H - fc[0]);
          fo[NC - 1] = fc[NC - 1] - A.dt * div[NC - 1] + dtau * (B - fc[NC - 1]);
        } else {
          const T g = e * (T(1) + corr * (tc - T(5)));
          fo[0] = fc[0] - A.dt * div[0] + dtau * (g - fc[0]);
        }
        T *dst = A.fn + ((size_t)c * A.nvp + k) * NC;
#pragma unroll
        for (int m = 0; m < NC; ++m) dst[m] = fo[m];
      } else {
#pragma unroll
        for (int m = 0; m < NC; ++m) fo[m] = fc[m];
      }
      // moments about the current bulk velocity: c' = xi - U^n
      const T wk = A.w[k];
      const T wh = wk * fo[0];
      const T wb = (D == 2) ? wk * fo[NC - 1] : T(0);
      const T e2 = c2 * wh + wb;
      acc[0].add(wh);
      if (D == 2) {
        acc[1].add(cv[0] * wh);
        acc[2].add(cv[1] * wh);
        acc[3].add(e2);
        acc[4].add(cv[0] * cv[0] * wh);
        acc[5].add(cv[0] * cv[1] * wh);
        acc[6].add(cv[1] * cv[1] * wh);
        acc[7].add(cv[0] * e2);
        acc[8].add(cv[1] * e2);
      } else {
        acc[1].add(cv[0] * wh);
        acc[2].add(cv[1] * wh);
        acc[3].add(cv[2] * wh);
        acc[4].add(e2);
        acc[5].add(cv[0] * cv[0] * wh);
        acc[6].add(cv[0] * cv[1] * wh);
        acc[7].add(cv[0] * cv[2] * wh);
        acc[8].add(cv[1] * cv[1] * wh);
        acc[9].add(cv[1] * cv[2] * wh);
        acc[10].add(cv[2] * cv[2] * wh);
        acc[11].add(cv[0] * e2);
        acc[12].add(cv[1] * e2);
        acc[13].add(cv[2] * e2);
      }
    }
  }
  // reduce the moment sums of each cell over its 64 threads (two warps)
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    T h = acc[m].hi(), l = acc[m].lo();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T oh = shfl_down(h, o), ol = shfl_down(l, o);
      Acc<T> t;
      t.s = h;
      if constexpr (sizeof(T) == 4) t.c = l;
      t.merge(oh, ol);
      h = t.hi();
      l = t.lo();
    }
    if ((tx & 31) == 0) red[ty][tx >> 5][m] = (double)h + (double)l;
  }
  __syncthreads();
  if (c < A.ncell && tx < NM) {
    double v = active ? red[ty][0][tx] + red[ty][1][tx] : 0.0;
    A.part[((size_t)chunk * NM + tx) * A.ncell + c] = v;
  }
}

// ---------------------------------------------------------------------------
// tree-refined grids (the tree-based AMR meshes of Sec. 4.2-4.4; the paper
// gives no scheme for them): finite volumes on the leaves of a 2:1-balanced
// quadtree (2D) or octree (3D).  The slope of a cell along an axis is the van
// Leer limited slope of the values on each side (the neighbour's, the mean of
// the 2^(D-1) finer neighbours', or the freestream halo) over the distances
// between centres along the axis; the upwind cell supplies the face value
// f + s sigma h / 2; a side with finer neighbours takes the mean of their
// face values as its inflow, so both cells of an interface see the same
// flux.  One time step for all leaves (the CFL of the finest cell).
//
// The geometry is static: the host lists for every leaf and axis the
// reciprocal centre distances to both sides, half the edge and its
// reciprocal.  A block takes four leaves; before its velocity loop it builds
// in shared memory, per leaf and axis, the stencil of the leaf itself and of
// each upwind neighbour on either side, so that the loop holds no division
// of the geometry and no lookup of levels.  The velocities of tree cases are
// stored grouped by orthant, so the threads of a warp share their upwind
// sides and take the same branches.
// ---------------------------------------------------------------------------

template <typename T> struct TreeArgs {
  SweepArgs<T> S;
  const int4 *__restrict__ sti;     // [leaf][entries][ints / 4]: stencil rows (-1 none, -2 the halo, -3 - l a ghost value) and the mutual flag
  const double2 *__restrict__ stg;  // [leaf][entries][2]: 1/d-, 1/d+, h, 1/h (own entries)
  const int4 *__restrict__ lrec;    // [leaf][2]: leaves on the sides, regular flag, fluid flag
  const int *__restrict__ sched;    // [leaf]: the leaf of each block slot (regular, other fluid, solid)
  int qb[3];                        // 2D: first stored position of the quadrants 1, 2, 3 (bit 0: x < 0, bit 1: y < 0)
};

// the stencil of one cell along one axis: the rows [nvp][NC] of the cell and
// of the NF leaves at most on its - and + sides (null beyond the first for a
// single neighbour; the freestream's row alone at the domain edge; a ghost's
// link row alone, C29), the reciprocal centre distances to both sides and
// the edge.  `mut` marks an upwind neighbour u of leaf c that is c's only
// neighbour on that side and has c as its only neighbour on the other: u's
// value and the value on its side towards c are then c's side value and
// c's own value.
template <typename T, int NF> struct __align__(16) TreeStencil {
  const T *c, *m[NF], *p[NF];
  T rdm, rdp, h;
  int mut;
};

// the value on one side of a cell as its slope sees it: the neighbour's, or
// the mean of the finer neighbours'
template <typename T, int NC, int NF>
__device__ __forceinline__ void tree_side_value(const T *const *r, int k, T *v) {
  load_nc<T, NC>(r[0] + (size_t)k * NC, v);
  int cnt = 1;
#pragma unroll
  for (int j = 1; j < NF; ++j)
    if (r[j]) {
      T w[NC];
      load_nc<T, NC>(r[j] + (size_t)k * NC, w);
#pragma unroll
      for (int m = 0; m < NC; ++m) v[m] += w[m];
      ++cnt;
    }
  if (cnt > 1) {
    const T rc = T(1) / T(cnt);
#pragma unroll
    for (int m = 0; m < NC; ++m) v[m] *= rc;
  }
}

// the van Leer limiter of the tree sweep: FP64 divides; FP32 takes the
// hardware reciprocal (as the packed quadtree path does)
__device__ __forceinline__ double tree_vanleer(double a, double b) { return vanleer(a, b); }
__device__ __forceinline__ float tree_vanleer(float a, float b) {
  const float p = a * b;
  return (p > 0.f) ? 2.f * p * dev::rcp_approx(a + b) : 0.f;
}

// the face value on side s of a cell of value fc with side values fm, fp:
// the limited slope over the centre distances times s h / 2
template <typename T, int NC, int NF>
__device__ __forceinline__ void tree_face_value(const TreeStencil<T, NF> &S, const T *fc, const T *fm, const T *fp, T s,
                                                T *out) {
  const T sh = s * (T(0.5) * S.h);
#pragma unroll
  for (int m = 0; m < NC; ++m) out[m] = fc[m] + tree_vanleer((fc[m] - fm[m]) * S.rdm, (fp[m] - fc[m]) * S.rdp) * sh;
}

// the face value of the upwind stencil S on side s (its own value and sides loaded)
template <typename T, int NC, int NF>
__device__ __forceinline__ void tree_upwind_face(const TreeStencil<T, NF> &S, T s, int k, T *out) {
  T fu[NC], um[NC], up[NC];
  load_nc<T, NC>(S.c + (size_t)k * NC, fu);
  tree_side_value<T, NC, NF>(S.m, k, um);
  tree_side_value<T, NC, NF>(S.p, k, up);
  tree_face_value<T, NC, NF>(S, fu, um, up, s, out);
}

// FP32 (h, b) pairs of quadtrees: packed arithmetic, the limiter through the
// hardware reciprocal (half the van Leer slope times the edge: h ab / (a + b))
__device__ __forceinline__ float2 tree_side2(const float *r0, const float *r1, int k) {
  const float2 v = reinterpret_cast<const float2 *>(r0)[k];
  if (!r1) return v;
  const float2 w = reinterpret_cast<const float2 *>(r1)[k];
  return __fmul2_rn(__fadd2_rn(v, w), dev::dup(0.5f));
}
__device__ __forceinline__ float2 tree_face2(const TreeStencil<float, 2> &S, float2 fc, float2 fm, float2 fp, float s) {
  const float2 a = __fmul2_rn(dev::sub2(fc, fm), dev::dup(S.rdm));
  const float2 b = __fmul2_rn(dev::sub2(fp, fc), dev::dup(S.rdp));
  return __ffma2_rn(dev::dup(s * S.h), dev::vl_half2(a, b), fc);
}
// 2^x (the hardware base-2 exponential)
__device__ __forceinline__ float tree_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
constexpr float kTreeLog2e = 1.442695040888963407f;

// FP32: four blocks of 256 threads per SM (the loop waits on gathers from L2
// and HBM: resident warps hide it, a few spilled registers cost less); FP64,
// bound by its arithmetic: two
template <typename T, int D>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4) ? 4 : 2) tree_sweep_kernel(TreeArgs<T> TA) {
  constexpr int NC = Dims<D>::NC;
  constexpr int NM = Dims<D>::NM;
  constexpr int NF = 1 << (D - 1); // leaves at most beyond a face
  constexpr int NS = 2 * D;        // sides
  constexpr int E = tree_entries(D), EI = tree_entry_ints(D);
  constexpr bool kF32 = std::is_same<T, float>::value && D == 2; // the packed quadtree paths
  static_assert(E <= kThreadsPerCell, "one thread per stencil entry");
  const SweepArgs<T> &A = TA.S;
  __shared__ double red[kCellsPerBlock][2][NM];
  // per leaf: its own stencil along each axis, then the upwind neighbours'
  // along axis a, side sd (0: -, 1: +), neighbour j at D + (2a + sd) NF + j
  __shared__ TreeStencil<T, NF> st[kCellsPerBlock][E];
  __shared__ int nup[kCellsPerBlock][NS]; // leaves on side 2a + sd: 0 (domain edge), 1, NF, 3 (a ghost)
  __shared__ T rh[kCellsPerBlock][D];     // 1 / h
  __shared__ int fast[kCellsPerBlock];    // one neighbour of the leaf's own level on every side (2D)
  __shared__ int fluid[kCellsPerBlock];   // the leaf is updated (not a solid leaf of a body, C29)
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long slot = (long long)blockIdx.x * kCellsPerBlock + ty;
  const bool active = slot < A.ncell;
  const long long c = active ? TA.sched[slot] : slot;
  const int chunk = blockIdx.y;
  if (active && tx < E) {
    // the stencil tables built on the host (one pass, no chain of lookups)
    const size_t e = (size_t)c * E + tx;
    int I[EI];
#pragma unroll
    for (int q = 0; q < EI / 4; ++q) {
      const int4 v = TA.sti[e * (EI / 4) + q];
      I[4 * q] = v.x;
      I[4 * q + 1] = v.y;
      I[4 * q + 2] = v.z;
      I[4 * q + 3] = v.w;
    }
    const double2 g0 = TA.stg[2 * e], g1 = TA.stg[2 * e + 1];
    auto row = [&](int i) -> const T * {
      return (i >= 0) ? A.f + (size_t)i * A.nvp * NC
             : (i == -2) ? A.finf
             : (i <= -3) ? A.lval + (size_t)(-3 - i) * A.nvp * NC // a ghost's value for this leaf (C29)
                         : nullptr;
    };
    TreeStencil<T, NF> S;
    S.c = row(I[0]);
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      S.m[j] = row(I[1 + j]);
      S.p[j] = row(I[1 + NF + j]);
    }
    S.mut = I[1 + 2 * NF];
    S.rdm = (T)g0.x;
    S.rdp = (T)g0.y;
    S.h = (T)g1.x;
    st[ty][tx] = S;
    if (tx < D) rh[ty][tx] = (T)g1.y;
  } else if (active && tx == E) {
    const int4 r0 = TA.lrec[(size_t)c * 2], r1 = TA.lrec[(size_t)c * 2 + 1];
    const int r[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
    for (int s = 0; s < NS; ++s) nup[ty][s] = r[s];
    fast[ty] = r[NS];
    fluid[ty] = r[NS + 1];
  }
  __syncthreads();
  T acc[NM];
#pragma unroll
  for (int m = 0; m < NM; ++m) acc[m] = T(0);
  // the moment sums of one velocity of value fo about the current bulk
  // velocity (c' = xi - U^n), in the order of the finalize kernel
  auto moments = [&](const T *cv, T c2, T wk, const T *fo) {
    const T wh = wk * fo[0];
    const T e2 = c2 * wh + ((D == 2) ? wk * fo[NC - 1] : T(0));
    acc[0] += wh;
    if constexpr (D == 2) {
      acc[1] += cv[0] * wh;
      acc[2] += cv[1] * wh;
      acc[3] += e2;
      acc[4] += cv[0] * cv[0] * wh;
      acc[5] += cv[0] * cv[1] * wh;
      acc[6] += cv[1] * cv[1] * wh;
      acc[7] += cv[0] * e2;
      acc[8] += cv[1] * e2;
    } else {
      acc[1] += cv[0] * wh;
      acc[2] += cv[1] * wh;
      acc[3] += cv[2] * wh;
      acc[4] += e2;
      acc[5] += cv[0] * cv[0] * wh;
      acc[6] += cv[0] * cv[1] * wh;
      acc[7] += cv[0] * cv[2] * wh;
      acc[8] += cv[1] * cv[1] * wh;
      acc[9] += cv[1] * cv[2] * wh;
      acc[10] += cv[2] * cv[2] * wh;
      acc[11] += cv[0] * e2;
      acc[12] += cv[1] * e2;
      acc[13] += cv[2] * e2;
    }
  };
  if (active) {
    const T *M = A.mac;
    T U[3], q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      U[a] = M[c * kMac + kU0 + a];
      q[a] = M[c * kMac + kQ0 + a];
    }
    const T pre = M[c * kMac + kPre], invT = M[c * kMac + kInvT], halfT = M[c * kMac + kHalfT];
    const T shA = M[c * kMac + kShA], dtau = M[c * kMac + kDtTau];
    const T *own = st[ty][0].c;
    // the stored velocities of a tree case come first, padding after
    const int kbeg = chunk * A.kloop * kThreadsPerCell;
    const int kend = min(A.nv, kbeg + A.kloop * kThreadsPerCell);
    // the general path: any leaf (levels apart, finer or ghost neighbours, the domain edge)
    auto general = [&]() {
        for (int k = kbeg + tx; k < kend; k += kThreadsPerCell) {
          T fc[NC], div[NC];
          T cv[3] = {T(0), T(0), T(0)};
          T c2 = T(0);
          load_nc<T, NC>(own + (size_t)k * NC, fc);
#pragma unroll
          for (int m = 0; m < NC; ++m) div[m] = T(0);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const T xa = A.xi[a * A.nvp + k];
            cv[a] = xa - U[a];
            c2 += cv[a] * cv[a];
            if (xa == T(0)) continue;
            const T s = (xa > T(0)) ? T(1) : T(-1);
            const int sd = (xa > T(0)) ? 0 : 1;
            const TreeStencil<T, NF> &So = st[ty][a];
            T fm[NC], fp[NC], fout[NC], fin[NC];
            tree_side_value<T, NC, NF>(So.m, k, fm);
            tree_side_value<T, NC, NF>(So.p, k, fp);
            tree_face_value<T, NC, NF>(So, fc, fm, fp, s, fout);
            const int n = nup[ty][2 * a + sd];
            const TreeStencil<T, NF> *Su = &st[ty][D + (2 * a + sd) * NF];
            if (n == 0) {
              load_nc<T, NC>(A.finf + (size_t)k * NC, fin); // the halo: its value, zero slope
            } else if (n == 3) {
              // a ghost upwind (C29): its link value with the one-sided slope
              load_nc<T, NC>(Su[0].c + (size_t)k * NC, fin);
#pragma unroll
              for (int m = 0; m < NC; ++m) fin[m] = T(0.5) * (fin[m] + fc[m]);
            } else if (n == 1 && Su[0].mut) {
              // one upwind leaf of c's level: its value and its side towards c
              // are c's side value and c's own value
              T far[NC];
              tree_side_value<T, NC, NF>(sd ? Su[0].p : Su[0].m, k, far);
              tree_face_value<T, NC, NF>(Su[0], sd ? fp : fm, sd ? fc : far, sd ? far : fc, s, fin);
            } else {
              // the upwind leaves' face values, each over its share of the side
              tree_upwind_face<T, NC, NF>(Su[0], s, k, fin);
              if (n > 1) {
                for (int j = 1; j < n; ++j) {
                  T g[NC];
                  tree_upwind_face<T, NC, NF>(Su[j], s, k, g);
#pragma unroll
                  for (int m = 0; m < NC; ++m) fin[m] += g[m];
                }
                const T rn = T(1) / T(n);
#pragma unroll
                for (int m = 0; m < NC; ++m) fin[m] *= rn;
              }
            }
            const T wa = fabs(xa) * rh[ty][a];
#pragma unroll
            for (int m = 0; m < NC; ++m) div[m] += wa * (fout[m] - fin[m]);
          }
          // Shakhov equilibrium (Sec. 4 reduced forms in 2D, g^S in 3D)
          T cq = T(0);
#pragma unroll
          for (int a = 0; a < D; ++a) cq += cv[a] * q[a];
          const T e = pre * exp_t(-c2 * invT);
          const T corr = shA * cq;
          const T tc = T(2) * c2 * invT;
          T fo[NC];
          if constexpr (D == 2) {
            const T H = e * (T(1) + corr * (tc - T(4)));
            const T B = halfT * e * (T(1) + corr * (tc - T(2)));
            fo[0] = fc[0] - A.dt * div[0] + dtau * (H - fc[0]);
            fo[NC - 1] = fc[NC - 1] - A.dt * div[NC - 1] + dtau * (B - fc[NC - 1]);
          } else {
            const T g = e * (T(1) + corr * (tc - T(5)));
            fo[0] = fc[0] - A.dt * div[0] + dtau * (g - fc[0]);
          }
          store_nc<T, NC>(A.fn + ((size_t)c * A.nvp + k) * NC, fo);
          moments(cv, c2, A.w[k], fo);
        }
    };
    if (!fluid[ty]) {
      // a solid leaf (C29): not updated; the moments of its stored values
      for (int k = kbeg + tx; k < kend; k += kThreadsPerCell) {
        T fc[NC], cv[3] = {T(0), T(0), T(0)}, c2 = T(0);
        load_nc<T, NC>(A.f + ((size_t)c * A.nvp + k) * NC, fc);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          cv[a] = A.xi[a * A.nvp + k] - U[a];
          c2 += cv[a] * cv[a];
        }
        moments(cv, c2, A.w[k], fc);
      }
    } else if constexpr (kF32) {
      const float nl2 = -invT * kTreeLog2e;
      const float2 *finf2 = reinterpret_cast<const float2 *>(A.finf);
      // relaxation, the store of f^{n+1} and the moment sums of one velocity
      auto finish = [&](int k, float2 f2, float2 dv, const float *cv, float c2, float wk) {
        // Shakhov equilibrium (Sec. 4 reduced forms)
        const float cq = fmaf(cv[1], q[1], cv[0] * q[0]);
        const float e = pre * tree_ex2(c2 * nl2);
        const float corr = shA * cq;
        const float tc = 2.f * c2 * invT;
        const float H = e * fmaf(corr, tc - 4.f, 1.f);
        const float B = halfT * e * fmaf(corr, tc - 2.f, 1.f);
        float fo[2];
        fo[0] = f2.x - A.dt * dv.x + dtau * (H - f2.x);
        fo[1] = f2.y - A.dt * dv.y + dtau * (B - f2.y);
        reinterpret_cast<float2 *>(A.fn)[(size_t)c * A.nvp + k] = make_float2(fo[0], fo[1]);
        // moments about the current bulk velocity: c' = xi - U^n
        const float wh = wk * fo[0];
        const float e2 = fmaf(c2, wh, wk * fo[1]);
        acc[0] += wh;
        acc[1] = fmaf(cv[0], wh, acc[1]);
        acc[2] = fmaf(cv[1], wh, acc[2]);
        acc[3] += e2;
        acc[4] = fmaf(cv[0] * cv[0], wh, acc[4]);
        acc[5] = fmaf(cv[0] * cv[1], wh, acc[5]);
        acc[6] = fmaf(cv[1] * cv[1], wh, acc[6]);
        acc[7] = fmaf(cv[0], e2, acc[7]);
        acc[8] = fmaf(cv[1], e2, acc[8]);
      };
      if (fast[ty]) {
        // a leaf with one neighbour of its own level on every side: the
        // upwind neighbour's value and its side towards the leaf are the
        // leaf's side value and own value, so one velocity reads the leaf,
        // its four neighbours and the two far neighbours upwind; every load
        // is issued before any arithmetic, the upwind sides taken from the
        // quadrant of the stored position (a zero component moves nothing)
        const TreeStencil<float, 2> &Sx = st[ty][0], &Sy = st[ty][1];
        const float2 *xm = reinterpret_cast<const float2 *>(Sx.m[0]), *xp = reinterpret_cast<const float2 *>(Sx.p[0]);
        const float2 *ym = reinterpret_cast<const float2 *>(Sy.m[0]), *yp = reinterpret_cast<const float2 *>(Sy.p[0]);
        const float2 *xf0 = reinterpret_cast<const float2 *>(st[ty][2].m[0]);
        const float2 *xf1 = reinterpret_cast<const float2 *>(st[ty][4].p[0]);
        const float2 *yf0 = reinterpret_cast<const float2 *>(st[ty][6].m[0]);
        const float2 *yf1 = reinterpret_cast<const float2 *>(st[ty][8].p[0]);
        const float2 *own2 = reinterpret_cast<const float2 *>(own);
        for (int k = kbeg + tx; k < kend; k += kThreadsPerCell) {
          const int o = (k >= TA.qb[0]) + (k >= TA.qb[1]) + (k >= TA.qb[2]); // bit 0: x < 0, bit 1: y < 0
          const int bx = o & 1, by = o >> 1;
          const float2 f2 = own2[k], vxm = xm[k], vxp = xp[k], vym = ym[k], vyp = yp[k];
          const float2 vxf = (bx ? xf1 : xf0)[k], vyf = (by ? yf1 : yf0)[k];
          const float xix = A.xi[k], xiy = A.xi[A.nvp + k], wk = A.w[k];
          const float sx = bx ? -1.f : 1.f, sy = by ? -1.f : 1.f;
          const float2 foutx = tree_face2(Sx, f2, vxm, vxp, sx);
          const float2 fouty = tree_face2(Sy, f2, vym, vyp, sy);
          const float2 finx = tree_face2(st[ty][bx ? 4 : 2], bx ? vxp : vxm, bx ? f2 : vxf, bx ? vxf : f2, sx);
          const float2 finy = tree_face2(st[ty][by ? 8 : 6], by ? vyp : vym, by ? f2 : vyf, by ? vyf : f2, sy);
          float2 dv = __fmul2_rn(dev::dup(fabsf(xix) * rh[ty][0]), dev::sub2(foutx, finx));
          dv = __ffma2_rn(dev::dup(fabsf(xiy) * rh[ty][1]), dev::sub2(fouty, finy), dv);
          const float cv[2] = {xix - U[0], xiy - U[1]};
          finish(k, f2, dv, cv, fmaf(cv[1], cv[1], cv[0] * cv[0]), wk);
        }
      } else {
      for (int k = kbeg + tx; k < kend; k += kThreadsPerCell) {
        const float2 f2 = reinterpret_cast<const float2 *>(own)[k];
        float2 dv = make_float2(0.f, 0.f);
        float cv[2], c2 = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const float xa = A.xi[a * A.nvp + k];
          cv[a] = xa - U[a];
          c2 = fmaf(cv[a], cv[a], c2);
          if (xa == 0.f) continue;
          const float s = (xa > 0.f) ? 1.f : -1.f; // the downwind side
          const int sd = (xa > 0.f) ? 0 : 1;       // the upwind side
          const TreeStencil<float, 2> &So = st[ty][a];
          const float2 fm = tree_side2(So.m[0], So.m[1], k), fp = tree_side2(So.p[0], So.p[1], k);
          const float2 fout = tree_face2(So, f2, fm, fp, s);
          const int n = nup[ty][2 * a + sd];
          float2 fin;
          if (n == 0) {
            fin = finf2[k]; // the halo: its value, zero slope
          } else if (n == 3) {
            // a ghost upwind (C29): its link value with the one-sided slope
            const float2 g = reinterpret_cast<const float2 *>(st[ty][2 + 4 * a + 2 * sd].c)[k];
            fin = __fmul2_rn(__fadd2_rn(g, f2), dev::dup(0.5f));
          } else {
            const TreeStencil<float, 2> &S0 = st[ty][2 + 4 * a + 2 * sd];
            if (S0.mut) {
              const float2 fu = sd ? fp : fm;
              const float2 far = sd ? tree_side2(S0.p[0], S0.p[1], k) : tree_side2(S0.m[0], S0.m[1], k);
              fin = tree_face2(S0, fu, sd ? f2 : far, sd ? far : f2, s);
            } else {
              fin = tree_face2(S0, reinterpret_cast<const float2 *>(S0.c)[k], tree_side2(S0.m[0], S0.m[1], k),
                               tree_side2(S0.p[0], S0.p[1], k), s);
              if (n == 2) {
                const TreeStencil<float, 2> &S1 = st[ty][3 + 4 * a + 2 * sd];
                const float2 g1 = tree_face2(S1, reinterpret_cast<const float2 *>(S1.c)[k],
                                             tree_side2(S1.m[0], S1.m[1], k), tree_side2(S1.p[0], S1.p[1], k), s);
                fin = __fmul2_rn(__fadd2_rn(fin, g1), dev::dup(0.5f));
              }
            }
          }
          dv = __ffma2_rn(dev::dup(fabsf(xa) * rh[ty][a]), dev::sub2(fout, fin), dv);
        }
        finish(k, f2, dv, cv, c2, A.w[k]);
      }
      }
    } else if constexpr (D == 3 && std::is_same<T, float>::value) {
      if (fast[ty]) {
        // an octree leaf with one fluid neighbour of its own level on every
        // side: one velocity reads the leaf, its six neighbours and the three
        // far neighbours upwind (the mutual shortcut), every load before any
        // arithmetic
        const T *nm[3], *np[3], *fm0[3], *fp1[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          nm[a] = st[ty][a].m[0];
          np[a] = st[ty][a].p[0];
          fm0[a] = st[ty][D + (2 * a) * NF].m[0];     // beyond the - neighbour
          fp1[a] = st[ty][D + (2 * a + 1) * NF].p[0]; // beyond the + neighbour
        }
        for (int k = kbeg + tx; k < kend; k += kThreadsPerCell) {
          T xa[3], vm[3], vp[3], vf[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) xa[a] = A.xi[a * A.nvp + k];
          const T fc = own[k];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            vm[a] = nm[a][k];
            vp[a] = np[a][k];
            vf[a] = (xa[a] > T(0)) ? fm0[a][k] : fp1[a][k];
          }
          T cv[3], c2 = T(0), div = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            cv[a] = xa[a] - U[a];
            c2 += cv[a] * cv[a];
            const bool pos = xa[a] > T(0);
            const T s = pos ? T(1) : T(-1);
            const TreeStencil<T, NF> &So = st[ty][a];
            const TreeStencil<T, NF> &Su = st[ty][D + (2 * a + (pos ? 0 : 1)) * NF];
            const T fout = fc + tree_vanleer((fc - vm[a]) * So.rdm, (vp[a] - fc) * So.rdp) * (s * (T(0.5) * So.h));
            const T fu = pos ? vm[a] : vp[a];
            const T um = pos ? vf[a] : fc, up = pos ? fc : vf[a];
            const T fin = fu + tree_vanleer((fu - um) * Su.rdm, (up - fu) * Su.rdp) * (s * (T(0.5) * Su.h));
            div += fabs(xa[a]) * rh[ty][a] * (fout - fin); // zero for a zero component
          }
          T cq = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) cq += cv[a] * q[a];
          const T e = pre * exp_t(-c2 * invT);
          const T g = e * (T(1) + shA * cq * (T(2) * c2 * invT - T(5)));
          T fo[NC];
          fo[0] = fc - A.dt * div + dtau * (g - fc);
          A.fn[(size_t)c * A.nvp + k] = fo[0];
          moments(cv, c2, A.w[k], fo);
        }
      } else {
        general();
      }
    } else {
      general();
    }
  }
  // reduce the moment sums of each leaf over its 64 threads (two warps)
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    T v = acc[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_down(v, o);
    if ((tx & 31) == 0) red[ty][tx >> 5][m] = (double)v;
  }
  __syncthreads();
  if (active && tx < NM) {
    double v = red[ty][0][tx] + red[ty][1][tx];
    A.part[((size_t)chunk * NM + tx) * A.ncell + c] = v;
  }
}

// ---------------------------------------------------------------------------
// moments of a stored state, without transport (after a state is loaded or a
// body is set): one warp per cell reads the cell's row of velocities with
// 16-byte loads, several in flight per lane; plain sums over the velocities of
// one group of loads, compensated (FP32) sums over the groups, and a
// compensated butterfly over the lanes. The moment sums are those of the
// sweep, written as one velocity chunk.
// ---------------------------------------------------------------------------

template <typename T> struct MomArgs {
  const T *__restrict__ f;   // [ncell][nvp][NC]
  const T *__restrict__ mac; // [ncell][kMac]
  const T *__restrict__ xi;  // [3][nvp]
  const T *__restrict__ w;   // [nvp]
  const uint8_t *__restrict__ ctype;
  double *__restrict__ part; // [NM][ncell]
  long long ncell;
  long long c0, c1; // the cells [c0, c1) of this launch
  int nv, nvp;
  int shift; // 1: moments about the stored bulk velocity U^n; 0: about zero
};

constexpr int kMomWarps = 8;  // cells of one moments block
constexpr int kMomUnroll = 4; // 16-byte loads in flight per lane

template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static __device__ __forceinline__ void unpack(const float4 &q, float *e) {
    e[0] = q.x;
    e[1] = q.y;
    e[2] = q.z;
    e[3] = q.w;
  }
};
template <> struct Vec16<double> {
  using type = double2;
  static __device__ __forceinline__ void unpack(const double2 &q, double *e) {
    e[0] = q.x;
    e[1] = q.y;
  }
};

template <typename T, int D>
__global__ void __launch_bounds__(32 * kMomWarps, (D == 2 && sizeof(T) == 4) ? 4 : 2) moments_kernel(MomArgs<T> A) {
  constexpr int NC = Dims<D>::NC;
  constexpr int NM = Dims<D>::NM;
  constexpr int V = 16 / (int)sizeof(T); // elements of one load
  constexpr int VPL = V / NC;            // velocities of one load
  using Q = typename Vec16<T>::type;
  const int lane = threadIdx.x & 31;
  const long long c = A.c0 + (long long)blockIdx.x * kMomWarps + (threadIdx.x >> 5);
  if (c >= A.c1) return; // the whole warp
  double out = 0.0;
  if (A.ctype[c] == IBDVM_CELL_FLUID) {
    T U[3] = {T(0), T(0), T(0)};
    if (A.shift)
#pragma unroll
      for (int a = 0; a < D; ++a) U[a] = A.mac[c * kMac + kU0 + a];
    const Q *row = reinterpret_cast<const Q *>(A.f + (size_t)c * A.nvp * NC);
    const int nvec = A.nvp * NC / V; // loads in the row (the padding makes it whole)
    Acc<T> acc[NM];
    for (int v0 = 0; v0 < nvec; v0 += 32 * kMomUnroll) {
      Q buf[kMomUnroll];
#pragma unroll
      for (int u = 0; u < kMomUnroll; ++u) {
        const int v = v0 + u * 32 + lane;
        if (v < nvec) buf[u] = row[v];
      }
      T s[NM];
#pragma unroll
      for (int m = 0; m < NM; ++m) s[m] = T(0);
#pragma unroll
      for (int u = 0; u < kMomUnroll; ++u) {
        const int v = v0 + u * 32 + lane;
        if (v >= nvec) continue;
        T e[V];
        Vec16<T>::unpack(buf[u], e);
#pragma unroll
        for (int j = 0; j < VPL; ++j) {
          const int k = v * VPL + j;
          const T wk = A.w[k];
          const bool live = wk != T(0); // padding positions hold no mass
          const T wh = live ? wk * e[j * NC] : T(0);
          const T wb = (D == 2 && live) ? wk * e[j * NC + NC - 1] : T(0);
          T cv[3] = {T(0), T(0), T(0)};
          T c2 = T(0);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            cv[a] = A.xi[a * A.nvp + k] - U[a];
            c2 += cv[a] * cv[a];
          }
          const T e2 = c2 * wh + wb;
          s[0] += wh;
#pragma unroll
          for (int a = 0; a < D; ++a) s[1 + a] += cv[a] * wh;
          s[1 + D] += e2;
          int m = 2 + D;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) s[m++] += cv[a] * cv[b] * wh;
#pragma unroll
          for (int a = 0; a < D; ++a) s[m + a] += cv[a] * e2;
        }
      }
#pragma unroll
      for (int m = 0; m < NM; ++m) acc[m].add(s[m]);
    }
    // butterfly over the lanes; every lane ends with the cell's sums
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      T h = acc[m].hi(), l = acc[m].lo();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        Acc<T> t;
        t.s = h;
        if constexpr (sizeof(T) == 4) t.c = l;
        t.merge(oh, ol);
        h = t.hi();
        l = t.lo();
      }
      if (lane == m) out = (double)h + (double)l;
    }
  }
  if (lane < NM) A.part[(size_t)lane * A.ncell + c] = out;
}

// ---------------------------------------------------------------------------
// moments -> macroscopic state, Shakhov parameters, residual partial sums
// ---------------------------------------------------------------------------

template <typename T, typename P = double> struct FinalArgs {
  const P *__restrict__ part;
  T *__restrict__ mac;
  const double *__restrict__ Wold; // [NW][ncell], may be null
  double *__restrict__ Wnew;
  const uint8_t *__restrict__ ctype;
  double *__restrict__ resblk; // [nblock][2 NW]
  int *__restrict__ flags;
  long long ncell;
  int nchunk;
  int shift;
  double mu0, omega, Pr, dt;
  int nblk;         // blocks of the finalize launch (residual partial sums)
  double *res_out;  // residual of the step
  long long c0, c1; // the cells [c0, c1) of this launch
};

template <typename T, int D, typename P>
__device__ __forceinline__ void finalize_body(const FinalArgs<T, P> &A, const int blk) {
  constexpr int NM = Dims<D>::NM;
  constexpr int NW = Dims<D>::NW;
  __shared__ double red[2 * NW][8];
  const long long c = A.c0 + (long long)blk * blockDim.x + threadIdx.x;
  double rnum[NW], rden[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) rnum[i] = rden[i] = 0.0;
  if (c < A.c1 && A.ctype[c] == IBDVM_CELL_FLUID) {
    double M[NM];
    if constexpr (std::is_same<P, float>::value) {
      // FP32 partial sums of the velocity chunks: added in order by a
      // Neumaier-compensated FP32 sum and widened once (GB300's FP64 rate is a
      // small fraction of its FP32 rate)
      Acc<float> acc[NM];
      for (int ch = 0; ch < A.nchunk; ++ch)
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m].add(A.part[((size_t)ch * NM + m) * A.ncell + c]);
#pragma unroll
      for (int m = 0; m < NM; ++m) M[m] = acc[m].value();
    } else {
#pragma unroll
      for (int m = 0; m < NM; ++m) M[m] = 0.0;
      for (int ch = 0; ch < A.nchunk; ++ch)
#pragma unroll
        for (int m = 0; m < NM; ++m) M[m] += (double)A.part[((size_t)ch * NM + m) * A.ncell + c];
    }
    const long long nc = A.ncell;
    double V[3] = {0.0, 0.0, 0.0};
    if (A.shift)
      for (int a = 0; a < D; ++a) V[a] = (double)A.mac[c * kMac + kU0 + a];
    const double rho = M[0];
    double M1[3] = {0, 0, 0}, d[3] = {0, 0, 0}, d2 = 0.0, VM1 = 0.0, V2 = 0.0;
    for (int a = 0; a < D; ++a) {
      M1[a] = M[1 + a];
      d[a] = M1[a] / rho;
      d2 += d[a] * d[a];
      VM1 += V[a] * M1[a];
      V2 += V[a] * V[a];
    }
    const double M2 = M[D + 1];
    // second moments M_ab about V (symmetric, packed row-wise)
    double Mab[3][3];
    {
      int p = D + 2;
      for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b) {
          Mab[a][b] = Mab[b][a] = M[p++];
        }
    }
    const double *M3 = &M[D + 2 + D * (D + 1) / 2];
    // conservative variables (Eq. moments1) and temperature (Eq. moments2) with
    // three translational degrees of freedom: rho E = rho |U|^2 / 2 + 3/4 rho T
    const double rhoE = 0.5 * (M2 + 2.0 * VM1 + V2 * rho);
    const double T_ = (2.0 / 3.0) * (M2 - rho * d2) / rho;
    double q[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      double s = 0.0;
      for (int b = 0; b < D; ++b) s += d[b] * Mab[a][b];
      // heat flux (Eq. moments3) about U = V + d from the sums about V
      q[a] = 0.5 * (M3[a] - d[a] * M2 - 2.0 * s + 2.0 * rho * d2 * d[a]);
    }
    double Wn[NW];
    Wn[0] = rho;
    for (int a = 0; a < D; ++a) Wn[1 + a] = rho * V[a] + M1[a];
    Wn[D + 1] = rhoE;
    T *Mc = A.mac;
    double dtau;
    if constexpr (std::is_same<T, float>::value) {
      // the mixed path stores the Shakhov parameters in FP32: take them in
      // FP32 (W, q and the residual above stay FP64)
      const float Tf = (float)T_, rf = (float)rho;
      const float mu = (float)A.mu0 * powf(Tf, (float)A.omega); // Eq. viscosity, T0 = 1
      const float dtf = (float)A.dt * (0.5f * rf * Tf) / mu;     // tau = mu / p
      dtau = dtf;
      const float piT = (float)kPi * Tf;
      Mc[c * kMac + kPre] = (D == 2) ? rf / piT : rf / (piT * sqrtf(piT));
      Mc[c * kMac + kInvT] = 1.f / Tf;
      Mc[c * kMac + kHalfT] = 0.5f * Tf;
      Mc[c * kMac + kShA] = 4.f * (1.f - (float)A.Pr) / (5.f * rf * Tf * Tf);
      Mc[c * kMac + kDtTau] = dtf;
    } else {
      const double p = 0.5 * rho * T_;
      const double mu = A.mu0 * pow(T_, A.omega); // Eq. viscosity, T0 = 1
      dtau = A.dt * p / mu;                         // tau = mu / p
      Mc[c * kMac + kPre] = (T)((D == 2) ? rho / (kPi * T_) : rho / pow(kPi * T_, 1.5));
      Mc[c * kMac + kInvT] = (T)(1.0 / T_);
      Mc[c * kMac + kHalfT] = (T)(0.5 * T_);
      Mc[c * kMac + kShA] = (T)(4.0 * (1.0 - A.Pr) / (5.0 * rho * T_ * T_));
      Mc[c * kMac + kDtTau] = (T)dtau;
    }
    const bool bad = !(rho > 0.0) || !(T_ > 0.0) || !isfinite(rhoE) || !isfinite(dtau);
    if (bad) atomicOr(A.flags, kFlagNonFinite);
    if (dtau > 1.0) atomicOr(A.flags, kFlagUnstable);
    for (int a = 0; a < 3; ++a) {
      Mc[c * kMac + kU0 + a] = (T)((a < D) ? V[a] + d[a] : 0.0);
      Mc[c * kMac + kQ0 + a] = (T)((a < D) ? q[a] : 0.0);
    }
    for (int a = 0; a < D; ++a) A.Wnew[(NW + a) * nc + c] = q[a];
    for (int i = 0; i < NW; ++i) {
      A.Wnew[i * nc + c] = Wn[i];
      if (A.Wold) {
        double dd = Wn[i] - A.Wold[i * nc + c];
        rnum[i] = dd * dd;
        rden[i] = fabs(Wn[i]);
      }
    }
  }
  if (A.resblk) {
    // fixed-order block reduction of the residual sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      double a = rnum[i], b = rden[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        red[i][wid] = a;
        red[NW + i][wid] = b;
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * NW) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
      A.resblk[(size_t)blk * 2 * NW + threadIdx.x] = s;
    }
  }
}

template <typename T, int D, typename P>
__global__ void __launch_bounds__(256) finalize_kernel(FinalArgs<T, P> A) {
  finalize_body<T, D, P>(A, blockIdx.x);
}

// res = max_i sqrt(sum_j dW_ij^2) / sum_j |W_ij| (Sec. 4), components with a
// zero denominator skipped; one block, fixed summation order
template <int NW>
__device__ __forceinline__ void residual_body(const double *__restrict__ resblk, int nblk, double *__restrict__ out) {
  __shared__ double sh[256];
  __shared__ double tot[2 * NW];
  for (int i = 0; i < 2 * NW; ++i) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += resblk[(size_t)b * 2 * NW + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) tot[i] = sh[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < NW; ++i) {
      if (tot[NW + i] == 0.0) continue;
      double v = sqrt(tot[i]) / tot[NW + i];
      r = (v > r) ? v : r;
    }
    *out = r;
  }
}

template <int NW>
__global__ void residual_kernel(const double *__restrict__ resblk, int nblk, double *__restrict__ out) {
  residual_body<NW>(resblk, nblk, out);
}

// ---------------------------------------------------------------------------
// the ghost band
// ---------------------------------------------------------------------------

template <typename T> struct GhostArgs {
  const T *__restrict__ f;
  const T *__restrict__ finf;
  const double *__restrict__ xiD; // [3][nvp]
  const double *__restrict__ wD;  // [nvp]
  const double *__restrict__ rwD; // [nvp]: 1 / w (0 at padding positions)
  const T *__restrict__ xiT;
  const int *__restrict__ l_int;  // [nlink][8]: gidx, donor, aux, axis, side, ghost, s0, s1
  const double *__restrict__ l_dbl; // [nlink][8]: c_sp, c_iw, c_gc, n0, n1, n2, S, -
  const double *__restrict__ l_wg;  // [nlink][nvp]
  const int *__restrict__ s_int;    // [nsurf][8]: cell, codes of the 6 face neighbours
  const double *__restrict__ s_dbl; // [nsurf][8]: r (weights), |r|, x_j - x_g, 1 / |r|
  const double *__restrict__ gwu;   // [nvp] unit-density wall Maxwellian
  const int *__restrict__ kst;      // [nv] stored position of each velocity (natural order)
  T *__restrict__ lval;
  T *__restrict__ fi;
  T *__restrict__ fsp;
  double *__restrict__ rhow;
  double *__restrict__ dbg_fstar; // optional [nlink][nvp][NC] (FP64)
  int nv, nvp;
  int nvx[3];
  double vx0[3], vh[3]; // first node and node spacing per axis (mirror interpolation)
  double dx[3];
  double Tw, Uw[3], accom;
  int plain_average;
  int naive; // the linear extrapolation 2 f_d - f_ac in place of Eq. extrapolation 1 (Sec. 3.3.4)
  HaloArgs<T> H; // the domain halo the pre-ghost slopes see
  int n[3];
  int nodes_rule; // non-uniform velocity nodes (the specular interpolation bisects)
  int ghost_nonneg; // ghost values below zero are set to zero
};

template <int NT> __device__ __forceinline__ double block_sum(double v, double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) s += sh[w];
    sh[NT / 32] = s;
  }
  __syncthreads();
  return sh[NT / 32];
}

// pre-ghost slope of surface cell j along axis a: van Leer with two fluid or
// halo neighbours, one-sided with one, zero with none
template <typename T, int NC>
__device__ __forceinline__ T preghost_slope(const GhostArgs<T> &G, int code_m, int code_p, T fj,
                                            int k, int m, T rh, int jc, int a) {
  const bool hm = code_m != -2, hp = code_p != -2;
  T fm = T(0), fp = T(0);
  int ijk[3] = {0, 0, 0};
  if (code_m == -1 || code_p == -1) { // a domain halo neighbour
    ijk[0] = jc % G.n[0];
    ijk[1] = (jc / G.n[0]) % G.n[1];
    ijk[2] = jc / (G.n[0] * G.n[1]);
  }
  if (hm)
    fm = (code_m >= 0) ? G.f[((size_t)code_m * G.nvp + k) * NC + m]
                       : halo_value(G.H, G.finf, G.n, ijk, a, -1, G.nvp, NC, k, m);
  if (hp)
    fp = (code_p >= 0) ? G.f[((size_t)code_p * G.nvp + k) * NC + m]
                       : halo_value(G.H, G.finf, G.n, ijk, a, +1, G.nvp, NC, k, m);
  if (hm && hp) return vanleer((fj - fm) * rh, (fp - fj) * rh);
  if (hm) return (fj - fm) * rh;
  if (hp) return (fp - fj) * rh;
  return T(0);
}

// the node interval of the velocity grid holding coordinate x along axis a:
// the lower node i and the fraction t of the multilinear interpolation
// (C13); false when x lies outside the grid.  Uniform axes by division,
// non-uniform ones (given nodes) by bisection on the node coordinates.
template <typename T>
__device__ __forceinline__ bool mirror_bracket(const GhostArgs<T> &G, int a, double x, int &i0, double &t) {
  const int n = G.nvx[a];
  if (G.nodes_rule) {
    const int stride = (a == 0) ? 1 : (a == 1 ? G.nvx[0] : G.nvx[0] * G.nvx[1]);
    const double *xa = G.xiD + (size_t)a * G.nvp;
    // node i of the axis is the velocity of natural index i * stride
    auto node = [&](int i) { return xa[G.kst[i * stride]]; };
    if (x < node(0) || x > node(n - 1)) return false;
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (node(mid) <= x)
        lo = mid;
      else
        hi = mid;
    }
    const double xl = node(lo), xh = node(hi);
    i0 = lo;
    t = (x - xl) / (xh - xl);
    return true;
  }
  const double xl = G.vx0[a], xh = G.vx0[a] + G.vh[a] * (n - 1);
  const double u = (x - xl) / G.vh[a];
  int i = (int)floor(u);
  i = min(max(i, 0), n - 2);
  i0 = i;
  t = u - i;
  return !(x < xl || x > xh);
}

// The ghost band of link l, one block: every thread takes U velocities at a
// time (strided by the block), so that U independent chains of loads are in
// flight per thread and the link's surface-cell entries are read once per U
// velocities.
template <typename T, int D, int U>
__device__ __forceinline__ void ghost_band_body(const GhostArgs<T> &G, const int l) {
  constexpr int NC = Dims<D>::NC;
  __shared__ double sh[kGhostThreads / 32 + 1];
  const int *li = G.l_int + 8 * l;
  const double *ld = G.l_dbl + 8 * l;
  const int donor = li[1], aux = li[2], s0 = li[6], s1 = li[7];
  const int ns = s1 - s0;
  const double c_sp = ld[0], c_iw = ld[1], c_gc = ld[2];
  const double nw[3] = {ld[3], ld[4], ld[5]};
  const double alpha = G.accom;
  const double *wgl = G.l_wg + (size_t)l * G.nvp;
  // per-link constants in the storage type, converted once (FP64 divisions
  // and conversions run on GB300's narrow FP64 pipe)
  T rdx[3];
  for (int a = 0; a < 3; ++a) rdx[a] = (a < D) ? (T)(1.0 / G.dx[a]) : T(0);
  const T csp = (T)c_sp, ciw = (T)c_iw, wfall = T(1) / T(ns > 0 ? ns : 1);
  double Nsum = 0.0, Dsum = 0.0;
  for (int iv0 = threadIdx.x; iv0 < G.nv; iv0 += U * blockDim.x) {
    int k[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int iv = iv0 + u * blockDim.x;
      ok[u] = iv < G.nv;
      k[u] = G.kst[ok[u] ? iv : iv0];
    }
    // upwind weights, Eq. upwind (FP64 for the exact-zero decision in the FP64 path)
    T xiT[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u)
      for (int a = 0; a < 3; ++a) xiT[u][a] = (a < D) ? G.xiT[a * G.nvp + k[u]] : T(0);
    T wsum[U];
#pragma unroll
    for (int u = 0; u < U; ++u) wsum[u] = T(0);
    for (int j = 0; j < (G.naive ? 0 : ns); ++j) {
      const double *sd = G.s_dbl + 8 * (s0 + j);
      T r[3];
      for (int a = 0; a < 3; ++a) r[a] = (a < D) ? (T)sd[a] : T(0);
      const T rinv = (T)sd[7];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        // xi.r without contraction: tangential velocities give an exact zero
        T xr = T(0);
        for (int a = 0; a < D; ++a) xr = add_rn(xr, mul_rn(xiT[u][a], r[a]));
        const T dot = mul_rn(xr, rinv);
        const T mx = dot > T(0) ? dot : T(0);
        wsum[u] = add_rn(wsum[u], mul_rn(mx, mx));
      }
    }
    T fgc[U][NC];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int m = 0; m < NC; ++m) fgc[u][m] = T(0);
    if (G.naive) { // the construction without upwind weighting, Sec. 3.3.4
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          const T fd = G.f[((size_t)donor * G.nvp + k[u]) * NC + m];
          fgc[u][m] = (aux >= 0) ? T(2) * fd - G.f[((size_t)aux * G.nvp + k[u]) * NC + m] : fd;
        }
    }
    for (int j = 0; j < (G.naive ? 0 : ns); ++j) {
      const int *si = G.s_int + 8 * (s0 + j);
      const double *sd = G.s_dbl + 8 * (s0 + j);
      const int jc = si[0];
      T r[3], dxg[3];
      bool has[3];
      for (int a = 0; a < 3; ++a) {
        r[a] = (a < D) ? (T)sd[a] : T(0);
        has[a] = (a < D) && sd[4 + a] != 0.0;
        dxg[a] = (a < D) ? (T)sd[4 + a] : T(0);
      }
      const T rinv = (T)sd[7];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool fallback = G.plain_average || !(wsum[u] != T(0));
        T wt;
        if (fallback) {
          wt = wfall;
        } else {
          T xr = T(0);
          for (int a = 0; a < D; ++a) xr = add_rn(xr, mul_rn(xiT[u][a], r[a]));
          const T dot = mul_rn(xr, rinv);
          const T mx = dot > T(0) ? dot : T(0);
          wt = mul_rn(mx, mx) / wsum[u];
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
          const T fj = G.f[((size_t)jc * G.nvp + k[u]) * NC + m];
          T v = fj; // f_j - sigma_j . (x_j - x_g)
          for (int a = 0; a < D; ++a) {
            if (has[a]) {
              T sig = preghost_slope<T, NC>(G, si[1 + 2 * a], si[2 + 2 * a], fj, k[u], m, rdx[a], jc, a);
              v -= sig * dxg[a];
            }
          }
          fgc[u][m] += wt * v;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int ku = k[u];
      // shifted point (Eq. fsp) and incident distribution at the wall (Eq. fw)
      T fiv0 = T(0);
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        const T fd = G.f[((size_t)donor * G.nvp + ku) * NC + m];
        T sp = fd;
        if (aux >= 0) sp = fd + csp * (G.f[((size_t)aux * G.nvp + ku) * NC + m] - fd);
        const T fiv = sp + ciw * (fgc[u][m] - sp);
        if (m == 0) fiv0 = fiv;
        G.fsp[((size_t)l * G.nvp + ku) * NC + m] = sp;
        G.fi[((size_t)l * G.nvp + ku) * NC + m] = fiv;
      }
      // zero-net-mass-flux balance with the cut-cell split (Eq. rhowc), FP64
      double xn = 0.0;
      for (int a = 0; a < D; ++a) xn += G.xiD[a * G.nvp + ku] * nw[a];
      const double Gw = G.gwu[ku];
      const double wg = wgl[ku], ws = G.wD[ku] - wg;
      Nsum += wg * xn * (double)fiv0;
      Dsum += ws * xn * Gw;
    }
  }
  __syncthreads(); // scratch writes of this block are visible to the block
  const double N = block_sum<kGhostThreads>(Nsum, sh);
  const double Dd = block_sum<kGhostThreads>(Dsum, sh);
  double Ssum = 0.0;
  if (alpha < 1.0) {
    // specular part: f^i at the mirrored velocity by multilinear interpolation
    for (int iv = threadIdx.x; iv < G.nv; iv += blockDim.x) {
      const int k = G.kst[iv];
      double xn = 0.0;
      for (int a = 0; a < D; ++a) xn += G.xiD[a * G.nvp + k] * nw[a];
      double xm[3];
      for (int a = 0; a < D; ++a) xm[a] = G.xiD[a * G.nvp + k] - 2.0 * xn * nw[a];
      bool inside = true;
      int i0[3] = {0, 0, 0};
      double t[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a)
        if (!mirror_bracket(G, a, xm[a], i0[a], t[a])) inside = false;
      double v = 0.0;
      if (inside)
        for (int corner = 0; corner < (1 << D); ++corner) {
          double wt = 1.0;
          int id[3] = {0, 0, 0};
          for (int a = 0; a < D; ++a) {
            int b = (corner >> a) & 1;
            id[a] = i0[a] + b;
            wt *= b ? t[a] : 1.0 - t[a];
          }
          const int kk = G.kst[id[0] + G.nvx[0] * (id[1] + G.nvx[1] * id[2])];
          v += wt * (double)G.fi[((size_t)l * G.nvp + kk) * NC];
        }
      Ssum += (G.wD[k] - wgl[k]) * xn * v;
    }
  }
  const double S = (alpha < 1.0) ? block_sum<kGhostThreads>(Ssum, sh) : 0.0;
  const double rho_w = (alpha > 0.0) ? -(N + (1.0 - alpha) * S) / (alpha * Dd) : 0.0;
  if (threadIdx.x == 0) G.rhow[l] = rho_w;
  // wall distribution (Eqs. general bc, Maxwell BC, fwc) and ghost value (Eq. extrapolation 2)
#pragma unroll U
  for (int iv = threadIdx.x; iv < G.nv; iv += blockDim.x) {
    const int k = G.kst[iv];
    double xn = 0.0;
    for (int a = 0; a < D; ++a) xn += G.xiD[a * G.nvp + k] * nw[a];
    const double Gw = G.gwu[k];
    double fsv[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) fsv[m] = 0.0;
    if (alpha < 1.0) {
      double xm[3];
      for (int a = 0; a < D; ++a) xm[a] = G.xiD[a * G.nvp + k] - 2.0 * xn * nw[a];
      bool inside = true;
      int i0[3] = {0, 0, 0};
      double t[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a)
        if (!mirror_bracket(G, a, xm[a], i0[a], t[a])) inside = false;
      if (inside)
        for (int corner = 0; corner < (1 << D); ++corner) {
          double wt = 1.0;
          int id[3] = {0, 0, 0};
          for (int a = 0; a < D; ++a) {
            int b = (corner >> a) & 1;
            id[a] = i0[a] + b;
            wt *= b ? t[a] : 1.0 - t[a];
          }
          const int kk = G.kst[id[0] + G.nvx[0] * (id[1] + G.nvx[1] * id[2])];
#pragma unroll
          for (int m = 0; m < NC; ++m) fsv[m] += wt * (double)G.fi[((size_t)l * G.nvp + kk) * NC + m];
        }
    }
    const double wk = G.wD[k], wg = wgl[k], ws = wk - wg;
    if (std::is_same<T, float>::value && !G.dbg_fstar) {
      // FP32 storage: the wall distribution and the ghost value of the step
      // in FP32 (the wall density above stays FP64; a launch that reports
      // f*_w for the wall quantities takes the FP64 branch below, so that
      // the normal mass flux of f*_w vanishes to FP64 rounding)
      const float wkf = (float)wk, wgf = (float)wg, wsf = wkf - wgf, rw = (float)G.rwD[k];
      const float arw = (float)(alpha * rho_w), oma = (float)(1.0 - alpha), cgc = (float)c_gc, Gwf = (float)Gw;
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        const size_t o = ((size_t)l * G.nvp + k) * NC + m;
        const float gw = (m == 0) ? Gwf : (float)(0.5 * G.Tw) * Gwf;
        const float fr = arw * gw + oma * (float)fsv[m];
        const float fiv = (float)G.fi[o];
        const float fstar = (wkf > 0.f) ? (wgf * fiv + wsf * fr) * rw : fiv;
        const float spv = (float)G.fsp[o];
        float gv = spv + cgc * (fstar - spv);
        if (G.ghost_nonneg && gv < 0.f) gv = 0.f;
        G.lval[o] = (T)gv;
      }
      continue;
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const size_t o = ((size_t)l * G.nvp + k) * NC + m;
      const double gw = (m == 0) ? Gw : 0.5 * G.Tw * Gw; // B_w = T_w / 2 H_w
      const double fr = alpha * rho_w * gw + (1.0 - alpha) * fsv[m];
      const double fiv = (double)G.fi[o];
      const double fstar = (wk > 0.0) ? (wg * fiv + ws * fr) * G.rwD[k] : fiv;
      const double spv = (double)G.fsp[o];
      double gv = spv + c_gc * (fstar - spv);
      if (G.ghost_nonneg && gv < 0.0) gv = 0.0; // optional nonnegative ghost values
      G.lval[o] = (T)gv;
      if (G.dbg_fstar) G.dbg_fstar[o] = fstar;
    }
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kGhostThreads, (GhostTiling<T, false>::blocks)) ghost_band_kernel(GhostArgs<T> G) {
  ghost_band_body<T, D, GhostTiling<T, false>::U>(G, blockIdx.x);
}

// ---------------------------------------------------------------------------
// diffuse domain walls: the halo values of every boundary cell of a wall face
// ---------------------------------------------------------------------------

template <typename T> struct DomainArgs {
  const T *__restrict__ f;
  const uint8_t *__restrict__ ctype;
  const double *__restrict__ xiD; // [3][nvp]
  const double *__restrict__ wD;  // [nvp]
  T *__restrict__ whalo;          // [slots][nvp][NC]
  const int *__restrict__ kst;    // [nv] stored position of each velocity (natural order)
  long long off[7];               // first slot of each face; off[6] = all slots
  int mask;
  int n[3];
  int nv, nvp;
  double Tw[6], Uw[6][3];
};

constexpr int kDomainThreads = 256;

// One block per slot of a wall face: the boundary cell's mass flux out of the
// domain through the face, carried by its own value (sum over s xi_a > 0), is
// returned by rho_w times the face's unit-density wall Maxwellian (the plane
// xi_a = 0 splits the velocities; FP64 sums); the halo then holds rho_w M_w
// for the entering velocities and the cell's own value for the others.
template <typename T, int D> __global__ void __launch_bounds__(kDomainThreads) domain_wall_kernel(DomainArgs<T> A) {
  constexpr int NC = Dims<D>::NC;
  __shared__ double sh[kDomainThreads / 32 + 1];
  const long long slot = blockIdx.x;
  int i = 0;
  while (i < 5 && slot >= A.off[i + 1]) ++i;
  if (!((A.mask >> i) & 1)) return; // a freestream face: no slots in use
  const int a = i >> 1, s = (i & 1) ? 1 : -1;
  const long long t = slot - A.off[i];
  int ijk[3];
  const int u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2; // the transverse axes, in order
  ijk[a] = (s > 0) ? A.n[a] - 1 : 0;
  ijk[u] = (int)(t % A.n[u]);
  ijk[v] = (int)(t / A.n[u]);
  const long long c = ijk[0] + (long long)A.n[0] * (ijk[1] + (long long)A.n[1] * ijk[2]);
  T *dst = A.whalo + (size_t)slot * A.nvp * NC;
  const T *fc = A.f + (size_t)c * A.nvp * NC;
  if (A.ctype[c] != IBDVM_CELL_FLUID) { // never read: the cell has no faces of its own
    for (int k = threadIdx.x; k < A.nvp * NC; k += blockDim.x) dst[k] = T(0);
    return;
  }
  const double Tw = A.Tw[i];
  const double norm = (D == 2) ? 1.0 / (kPi * Tw) : 1.0 / pow(kPi * Tw, 1.5);
  double so = 0.0, si = 0.0;
  for (int iv = threadIdx.x; iv < A.nv; iv += blockDim.x) {
    const int k = A.kst[iv];
    const double xs = s * A.xiD[a * A.nvp + k];
    if (xs > 0.0) {
      so += A.wD[k] * xs * (double)fc[(size_t)k * NC];
    } else if (xs < 0.0) {
      double c2 = 0.0;
      for (int b = 0; b < D; ++b) {
        const double cb = A.xiD[b * A.nvp + k] - A.Uw[i][b];
        c2 += cb * cb;
      }
      si += A.wD[k] * xs * norm * exp(-c2 / Tw);
    }
  }
  const double out = block_sum<kDomainThreads>(so, sh);
  const double in = block_sum<kDomainThreads>(si, sh);
  const double rho_w = -out / in;
  for (int k = threadIdx.x; k < A.nvp; k += blockDim.x) {
    const double xs = s * A.xiD[a * A.nvp + k]; // zero at padding positions
    if (xs < 0.0) {
      double c2 = 0.0;
      for (int b = 0; b < D; ++b) {
        const double cb = A.xiD[b * A.nvp + k] - A.Uw[i][b];
        c2 += cb * cb;
      }
      const double H = rho_w * norm * exp(-c2 / Tw);
      dst[(size_t)k * NC] = (T)H;
      if (NC == 2) dst[(size_t)k * NC + NC - 1] = (T)(0.5 * Tw * H); // B_w = T_w / 2 H_w
    } else {
#pragma unroll
      for (int m = 0; m < NC; ++m) dst[(size_t)k * NC + m] = fc[(size_t)k * NC + m];
    }
  }
}

// ---------------------------------------------------------------------------
// wall points: moments of the wall distribution f*_w (FP64)
// ---------------------------------------------------------------------------

struct WallArgs {
  const double *__restrict__ fstar; // [nlink][nvp][NC], f*_w of the ghost band
  const double *__restrict__ xiD;   // [3][nvp]
  const double *__restrict__ wD;    // [nvp]
  const double *__restrict__ l_dbl; // [nlink][8]; the wall normal at 3..5
  const int *__restrict__ kst;      // [nv] stored position of each velocity (natural order)
  double *__restrict__ out;         // [nlink][kWallCols]
  int nv, nvp;
  double Tw, Uw[3];
  double p0, dyn0; // free-stream pressure rho_0 T_0 / 2 and rho_0 |U_0|^2
};

constexpr int kWallThreads = 256;

// One block per link: rho and U from the first pass, then the central
// moments about U (temperature, stress tensor, heat flux of Eq. moments3) and
// the wall-point quantities from them.  The cut boxes of f*_w already hold the
// blend of the incident and reflected parts, so the plain weights give the
// cut-corrected moments.
template <int D> __global__ void __launch_bounds__(kWallThreads) wall_kernel(WallArgs A) {
  constexpr int NC = Dims<D>::NC;
  constexpr int NP = D * (D + 1) / 2; // independent stress components
  __shared__ double sh[kWallThreads / 32 + 1];
  const int l = blockIdx.x;
  const double *fs = A.fstar + (size_t)l * A.nvp * NC;
  double s0 = 0.0, s1[3] = {0.0, 0.0, 0.0};
  for (int iv = threadIdx.x; iv < A.nv; iv += blockDim.x) {
    const int k = A.kst[iv];
    const double wh = A.wD[k] * fs[(size_t)k * NC];
    s0 += wh;
#pragma unroll
    for (int a = 0; a < D; ++a) s1[a] += A.xiD[a * A.nvp + k] * wh;
  }
  const double rho = block_sum<kWallThreads>(s0, sh);
  double U[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < D; ++a) U[a] = block_sum<kWallThreads>(s1[a], sh) / rho;
  double se = 0.0, sp[NP], sq[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < NP; ++i) sp[i] = 0.0;
  for (int iv = threadIdx.x; iv < A.nv; iv += blockDim.x) {
    const int k = A.kst[iv];
    const double h = fs[(size_t)k * NC], b = (NC == 2) ? fs[(size_t)k * NC + 1] : 0.0;
    double c[3], c2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      c[a] = A.xiD[a * A.nvp + k] - U[a];
      c2 += c[a] * c[a];
    }
    const double wk = A.wD[k], wh = wk * h, we = wk * (c2 * h + b);
    se += we;
    int i = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = a; bb < D; ++bb) sp[i++] += c[a] * c[bb] * wh;
#pragma unroll
    for (int a = 0; a < D; ++a) sq[a] += c[a] * we;
  }
  const double E = block_sum<kWallThreads>(se, sh);
  double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  {
    int i = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = a; bb < D; ++bb) {
        const double v = block_sum<kWallThreads>(sp[i++], sh);
        P[a][bb] = P[bb][a] = v;
      }
  }
  double q[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < D; ++a) q[a] = 0.5 * block_sum<kWallThreads>(sq[a], sh);
  if (threadIdx.x == 0) {
    const double *n = A.l_dbl + 8 * (size_t)l + 3;
    double Pn[3], p = 0.0, qn = 0.0;
    for (int a = 0; a < 3; ++a) Pn[a] = P[a][0] * n[0] + P[a][1] * n[1] + P[a][2] * n[2];
    for (int a = 0; a < 3; ++a) {
      p += n[a] * Pn[a];
      qn += n[a] * q[a];
    }
    const double T = 2.0 * E / (3.0 * rho);
    double *o = A.out + (size_t)l * kWallCols;
    o[0] = rho;
    for (int a = 0; a < 3; ++a) o[1 + a] = U[a] - A.Uw[a];
    o[4] = T;
    o[5] = T - A.Tw;
    o[6] = p;
    for (int a = 0; a < 3; ++a) o[7 + a] = Pn[a] - p * n[a];
    o[10] = qn;
    o[11] = (A.dyn0 > 0.0) ? 2.0 * (p - A.p0) / A.dyn0 : CUDART_NAN;
  }
}

// ---------------------------------------------------------------------------
// forces: momentum and energy through the donor-ghost faces (FP64 sums)
// ---------------------------------------------------------------------------

template <typename T> struct ForceArgs {
  SweepArgs<T> S;
  const int *__restrict__ l_int;
  const double *__restrict__ l_dbl;
  const double *__restrict__ xiD;
  const double *__restrict__ wD;
  double *__restrict__ fpart; // [nlink][4]
  int nlink;
  double *__restrict__ dst;   // [4]: F_x, F_y, F_z, Q
  // a tree (C29): per link the row beyond the donor along the link axis (a
  // leaf, -2 the halo, -3 - l the ghost value of link l); null on uniform grids
  const int *__restrict__ tree_far;
};

template <typename T, int D>
__device__ __forceinline__ void forces_body(const ForceArgs<T> &A, const int l) {
  constexpr int NC = Dims<D>::NC;
  __shared__ double sh[16];
  const int *li = A.l_int + 8 * l;
  const int d = li[1], a = li[3], side = li[4];
  const int sf = -side; // face of the donor toward the ghost
  const double Sface = A.l_dbl[8 * l + 6];
  const SweepArgs<T> &S = A.S;
  int ijk[3];
  ijk[0] = d % S.n[0];
  ijk[1] = (d / S.n[0]) % S.n[1];
  ijk[2] = d / (S.n[0] * S.n[1]);
  double acc[4] = {0, 0, 0, 0};
  for (int iv = threadIdx.x; iv < S.nv; iv += blockDim.x) {
    const int k = S.kst[iv];
    const double xin = A.xiD[a * S.nvp + k] * sf; // velocity into the solid
    if (xin == 0.0) continue;
    T fd[NC], fg[NC], face[NC];
    load_nc<T, NC>(S.f + ((size_t)d * S.nvp + k) * NC, fd);
    if (A.tree_far) load_nc<T, NC>(S.lval + ((size_t)l * S.nvp + k) * NC, fg);
    else seen<T, NC>(S, d, ijk, a, sf, k, fg); // the link's ghost value
    if (xin > 0.0) {
      T fb[NC];
      if (A.tree_far) {
        const int r = A.tree_far[l];
        load_nc<T, NC>((r >= 0) ? S.f + ((size_t)r * S.nvp + k) * NC
                       : (r == -2) ? S.finf + (size_t)k * NC : S.lval + ((size_t)(-3 - r) * S.nvp + k) * NC, fb);
      } else {
        seen<T, NC>(S, d, ijk, a, -sf, k, fb);
      }
#pragma unroll
      for (int m = 0; m < NC; ++m) face[m] = fd[m] + T(0.5) * vanleer(fd[m] - fb[m], fg[m] - fd[m]);
    } else {
#pragma unroll
      for (int m = 0; m < NC; ++m) face[m] = T(0.5) * (fg[m] + fd[m]);
    }
    const double wk = A.wD[k];
    double x2 = 0.0;
    for (int b = 0; b < D; ++b) {
      const double x = A.xiD[b * S.nvp + k];
      x2 += x * x;
      acc[b] += Sface * wk * x * xin * (double)face[0];
    }
    double e = 0.5 * x2 * (double)face[0];
    if (D == 2) e += 0.5 * (double)face[NC - 1];
    acc[3] += Sface * wk * e * xin;
  }
  for (int i = 0; i < 4; ++i) {
    double s = block_sum<256>(acc[i], sh);
    if (threadIdx.x == 0) A.fpart[4 * l + i] = s;
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(256) forces_kernel(ForceArgs<T> A) {
  forces_body<T, D>(A, blockIdx.x);
}

__device__ __forceinline__ void forces_total_body(const double *__restrict__ fpart, int nlink,
                                                  double *__restrict__ out) {
  __shared__ double sh[256];
  for (int i = 0; i < 4; ++i) {
    double s = 0.0;
    for (int l = threadIdx.x; l < nlink; l += blockDim.x) s += fpart[4 * l + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
    __syncthreads();
  }
}

__global__ void forces_total_kernel(const double *__restrict__ fpart, int nlink, double *__restrict__ out) {
  forces_total_body(fpart, nlink, out);
}

// ---------------------------------------------------------------------------
// grouped launches: one launch over the members of a batch.  Virtual block b
// belongs to case c with start[c] <= b < start[c + 1]; every case has two
// argument blocks, for the buffer parities after an even and an odd number of
// steps, and the launch names the parity.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int group_case(const int *__restrict__ start, int ncase, int b) {
  int lo = 0, hi = ncase - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, int D>
__global__ void __launch_bounds__(kGhostThreads, (GhostTiling<T, true>::blocks)) ghost_band_grouped(const GhostArgs<T> *__restrict__ tab,
                                                          const int *__restrict__ start, int ncase, int par) {
  __shared__ GhostArgs<T> sG;
  const int c = group_case(start, ncase, blockIdx.x);
  if (threadIdx.x == 0) sG = tab[2 * c + par];
  __syncthreads();
  ghost_band_body<T, D, GhostTiling<T, true>::U>(sG, blockIdx.x - __ldg(start + c));
}

template <typename T, int D>
__global__ void __launch_bounds__(256) forces_grouped(const ForceArgs<T> *__restrict__ tab,
                                                      const int *__restrict__ start, int ncase, int par) {
  __shared__ ForceArgs<T> sA;
  const int c = group_case(start, ncase, blockIdx.x);
  if (threadIdx.x == 0) sA = tab[2 * c + par];
  __syncthreads();
  forces_body<T, D>(sA, blockIdx.x - __ldg(start + c));
}

template <typename T>
__global__ void __launch_bounds__(256) forces_total_grouped(const ForceArgs<T> *__restrict__ tab, int par) {
  const ForceArgs<T> &A = tab[2 * blockIdx.x + par];
  forces_total_body(A.fpart, A.nlink, A.dst);
}

template <typename T, int D, typename P>
__global__ void __launch_bounds__(256) finalize_grouped(const FinalArgs<T, P> *__restrict__ tab,
                                                        const int *__restrict__ start, int ncase, int par) {
  __shared__ FinalArgs<T, P> sA;
  const int c = group_case(start, ncase, blockIdx.x);
  if (threadIdx.x == 0) sA = tab[2 * c + par];
  __syncthreads();
  finalize_body<T, D, P>(sA, blockIdx.x - __ldg(start + c));
}

template <typename T, int D, typename P>
__global__ void __launch_bounds__(256) residual_grouped(const FinalArgs<T, P> *__restrict__ tab, int par) {
  const FinalArgs<T, P> &A = tab[2 * blockIdx.x + par];
  residual_body<Dims<D>::NW>(A.resblk, A.nblk, A.res_out);
}

// ---------------------------------------------------------------------------
// initial state and format conversion
// ---------------------------------------------------------------------------

template <typename T>
__global__ void init_state_kernel(T *__restrict__ f0, T *__restrict__ f1, const T *__restrict__ finf,
                                  long long ncell, int per_cell) {
  const long long total = ncell * per_cell;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = finf[i % per_cell];
    f0[i] = v;
    f1[i] = v;
  }
}

// dense FP64 [cells][nv][NC] in the natural velocity order <-> the state
// [cells][nvp][NC] at the stored positions, for a range of cells
template <typename T>
__global__ void convert_kernel(T *__restrict__ state, double *__restrict__ dense, const int *__restrict__ kst,
                               long long c0, long long ncells, int nv, int nvp, int NC, int to_state) {
  const long long total = ncells * (long long)nv * NC;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long cell = i / ((long long)nv * NC);
    const long long r = i % ((long long)nv * NC);
    const int iv = (int)(r / NC), m = (int)(r % NC);
    const size_t si = ((size_t)(c0 + cell) * nvp + kst[iv]) * NC + m;
    if (to_state)
      state[si] = (T)dense[i];
    else
      dense[i] = (double)state[si];
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

// the domain halo of a context (the freestream, or its diffuse walls)
template <typename T> HaloArgs<T> halo_args(const ibdvm_ctx *ctx) {
  HaloArgs<T> H{};
  H.whalo = static_cast<const T *>(ctx->whalo);
  H.mask = ctx->wall_mask;
  for (int i = 0; i < 6; ++i) H.off[i] = ctx->wall_off[i];
  return H;
}

template <typename T> SweepArgs<T> sweep_args(const ibdvm_ctx *ctx, int update, int shift = 1, int cur = -1) {
  if (cur < 0) cur = ctx->cur;
  SweepArgs<T> A{};
  A.f = static_cast<const T *>(ctx->f[cur]);
  A.fn = static_cast<T *>(ctx->f[1 - cur]);
  A.mac = static_cast<const T *>(ctx->mac);
  A.xi = static_cast<const T *>(ctx->xiT);
  A.w = static_cast<const T *>(ctx->wT);
  A.finf = static_cast<const T *>(ctx->finf);
  A.ctype = ctx->ctype;
  A.dslot = ctx->dslot;
  A.dlinks = ctx->dlinks;
  A.lval = static_cast<const T *>(ctx->lval);
  A.kst = ctx->kst;
  A.part = ctx->part;
  A.ncell = ctx->ncell;
  for (int a = 0; a < 3; ++a) {
    A.n[a] = ctx->geom.n[a];
    A.rdx[a] = (T)(1.0 / ctx->geom.dx[a]);
  }
  A.nv = ctx->nv;
  A.nvp = ctx->nvp;
  A.kloop = ctx->kloop;
  A.dt = (T)ctx->geom.dt;
  A.update = update;
  A.shift = shift;
  A.H = halo_args<T>(ctx);
  return A;
}

template <typename T, int D> cudaError_t sweep_t(ibdvm_ctx *ctx, int update, int shift) {
  SweepArgs<T> A = sweep_args<T>(ctx, update, shift);
  dim3 block(kThreadsPerCell, kCellsPerBlock);
  dim3 grid((unsigned)((ctx->ncell + kCellsPerBlock - 1) / kCellsPerBlock), (unsigned)ctx->nchunk);
  sweep_kernel<T, D><<<grid, block, 0, ctx->stream>>>(A);
  return cudaGetLastError();
}

template <typename T, int D> cudaError_t tree_sweep_t(ibdvm_ctx *ctx) {
  {
    TreeArgs<T> A{};
    A.S = sweep_args<T>(ctx, 1, 1);
    A.sti = reinterpret_cast<const int4 *>(ctx->tree_sti);
    A.stg = reinterpret_cast<const double2 *>(ctx->tree_stg);
    A.lrec = reinterpret_cast<const int4 *>(ctx->tree_lrec);
    A.sched = ctx->tree_sched;
    for (int i = 0; i < 3; ++i) A.qb[i] = ctx->tree_qb[i];
    dim3 block(kThreadsPerCell, kCellsPerBlock);
    dim3 grid((unsigned)((ctx->ncell + kCellsPerBlock - 1) / kCellsPerBlock), (unsigned)ctx->nchunk);
    tree_sweep_kernel<T, D><<<grid, block, 0, ctx->stream>>>(A);
    return cudaGetLastError();
  }
}

// arguments of the finalize kernel for moment buffer parity wcur
template <typename T, typename P>
FinalArgs<T, P> final_args(const ibdvm_ctx *ctx, int wcur, bool shift, bool residual, const P *part, int nchunk) {
  FinalArgs<T, P> A{};
  A.part = part;
  A.mac = static_cast<T *>(ctx->mac);
  A.Wold = residual ? ctx->W[wcur] : nullptr;
  A.Wnew = ctx->W[1 - wcur];
  A.ctype = ctx->ctype;
  A.resblk = residual ? ctx->resblk : nullptr;
  A.flags = ctx->d_flags;
  A.ncell = ctx->ncell;
  A.nchunk = nchunk;
  A.shift = shift ? 1 : 0;
  A.mu0 = ctx->geom.mu0;
  A.omega = ctx->geom.gas.omega_vhs;
  A.Pr = ctx->geom.gas.Pr;
  A.dt = ctx->geom.dt;
  A.nblk = (int)((ctx->ncell + 255) / 256);
  A.res_out = ctx->d_res;
  A.c0 = 0;
  A.c1 = ctx->ncell;
  return A;
}

template <typename T, int D, typename P = double>
cudaError_t finalize_t(ibdvm_ctx *ctx, bool shift, bool residual, const P *part = nullptr, int nchunk = 0) {
  const P *pp;
  if constexpr (std::is_same<P, double>::value)
    pp = part ? part : ctx->part;
  else
    pp = part;
  const FinalArgs<T, P> A = final_args<T, P>(ctx, ctx->wcur, shift, residual, pp, nchunk ? nchunk : ctx->nchunk);
  finalize_kernel<T, D, P><<<A.nblk, 256, 0, ctx->stream>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (residual) {
    residual_kernel<Dims<D>::NW><<<1, 256, 0, ctx->stream>>>(ctx->resblk, A.nblk, ctx->d_res);
    e = cudaGetLastError();
  }
  ctx->wcur = 1 - ctx->wcur;
  return e;
}

// arguments of the ghost-band kernel for state buffer parity cur
template <typename T> GhostArgs<T> ghost_args(const ibdvm_ctx *ctx, int cur, double *dbg) {
  const Geom &g = ctx->geom;
  GhostArgs<T> G{};
  G.f = static_cast<const T *>(ctx->f[cur]);
  G.finf = static_cast<const T *>(ctx->finf);
  G.xiD = ctx->xiD;
  G.wD = ctx->wD;
  G.rwD = ctx->wD + ctx->nvp;
  G.xiT = static_cast<const T *>(ctx->xiT);
  G.l_int = ctx->l_int;
  G.l_dbl = ctx->l_dbl;
  G.l_wg = ctx->l_wg;
  G.s_int = ctx->s_int;
  G.s_dbl = ctx->s_dbl;
  G.gwu = ctx->gw_unit;
  G.kst = ctx->kst;
  G.lval = static_cast<T *>(ctx->lval);
  G.fi = static_cast<T *>(ctx->fi_scr);
  G.fsp = static_cast<T *>(ctx->fsp_scr);
  G.rhow = ctx->rhow;
  G.dbg_fstar = dbg;
  G.nv = ctx->nv;
  G.nvp = ctx->nvp;
  for (int a = 0; a < 3; ++a) {
    G.nvx[a] = g.nvx[a];
    G.dx[a] = g.dx[a];
    G.Uw[a] = g.body.U_w[a];
    // first node and spacing per axis of the node grid
    const int stride = (a == 0) ? 1 : (a == 1 ? g.nvx[0] : g.nvx[0] * g.nvx[1]);
    const double x0 = g.xi[3 * 0 + a];
    const double x1 = g.xi[3 * ((g.nvx[a] - 1) * stride) + a];
    G.vx0[a] = x0;
    G.vh[a] = (g.nvx[a] > 1) ? (x1 - x0) / (g.nvx[a] - 1) : 1.0;
  }
  G.Tw = g.body.T_w;
  G.accom = g.body.accom_alpha;
  G.plain_average = (g.gas.flags & IBDVM_PLAIN_AVERAGE) ? 1 : 0;
  G.naive = (g.gas.flags & IBDVM_NAIVE_EXTRAPOLATION) ? 1 : 0;
  G.H = halo_args<T>(ctx);
  for (int a = 0; a < 3; ++a) G.n[a] = g.n[a];
  G.nodes_rule = (g.rule == IBDVM_RULE_NODES) ? 1 : 0;
  G.ghost_nonneg = (g.gas.flags & IBDVM_GHOST_NONNEG) ? 1 : 0;
  return G;
}

template <typename T, int D> cudaError_t domain_t(ibdvm_ctx *ctx) {
  const Geom &g = ctx->geom;
  DomainArgs<T> A{};
  A.f = static_cast<const T *>(ctx->f[ctx->cur]);
  A.ctype = ctx->ctype;
  A.xiD = ctx->xiD;
  A.wD = ctx->wD;
  A.whalo = static_cast<T *>(ctx->whalo);
  A.kst = ctx->kst;
  for (int i = 0; i < 7; ++i) A.off[i] = ctx->wall_off[i];
  A.mask = ctx->wall_mask;
  for (int a = 0; a < 3; ++a) A.n[a] = g.n[a];
  A.nv = ctx->nv;
  A.nvp = ctx->nvp;
  for (int i = 0; i < 6; ++i) {
    A.Tw[i] = ctx->wall_T[i];
    for (int a = 0; a < 3; ++a) A.Uw[i][a] = ctx->wall_U[i][a];
  }
  domain_wall_kernel<T, D><<<(unsigned)ctx->wall_off[6], kDomainThreads, 0, ctx->stream>>>(A);
  return cudaGetLastError();
}

template <typename T, int D> cudaError_t ghost_t(ibdvm_ctx *ctx, double *dbg) {
  if (ctx->nlink == 0) return cudaSuccess;
  ghost_band_kernel<T, D><<<ctx->nlink, kGhostThreads, 0, ctx->stream>>>(ghost_args<T>(ctx, ctx->cur, dbg));
  return cudaGetLastError();
}

// arguments of the force kernels for state buffer parity cur
template <typename T> ForceArgs<T> force_args(const ibdvm_ctx *ctx, int cur, double *dst) {
  ForceArgs<T> A{};
  A.S = sweep_args<T>(ctx, 0, 1, cur);
  A.l_int = ctx->l_int;
  A.l_dbl = ctx->l_dbl;
  A.xiD = ctx->xiD;
  A.wD = ctx->wD;
  A.fpart = ctx->fpart;
  A.nlink = ctx->nlink;
  A.dst = dst;
  A.tree_far = ctx->tree ? ctx->tree_far : nullptr;
  return A;
}

template <typename T, int D> cudaError_t forces_t(ibdvm_ctx *ctx, double *dst) {
  if (ctx->nlink == 0) return cudaMemsetAsync(dst, 0, 4 * sizeof(double), ctx->stream);
  forces_kernel<T, D><<<ctx->nlink, 256, 0, ctx->stream>>>(force_args<T>(ctx, ctx->cur, dst));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  forces_total_kernel<<<1, 256, 0, ctx->stream>>>(ctx->fpart, ctx->nlink, dst);
  return cudaGetLastError();
}

// CUDA events around a launch class when the context profiles its kernels
struct Timed {
  ibdvm_ctx *ctx;
  int cls;
  size_t start = 0;
  bool on;
  Timed(ibdvm_ctx *c, int k) : ctx(c), cls(k), on(c->profiling) {
    if (!on) return;
    if (ctx->ev_used + 2 > ctx->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          on = false;
          return;
        }
        ctx->ev_pool.push_back(e);
      }
    }
    start = ctx->ev_used;
    ctx->ev_used += 2;
    cudaEventRecord(ctx->ev_pool[start], ctx->stream);
  }
  ~Timed() {
    if (!on) return;
    cudaEventRecord(ctx->ev_pool[start + 1], ctx->stream);
    ctx->ev_marks.emplace_back(cls, start);
  }
};

template <typename F> cudaError_t dispatch(ibdvm_ctx *ctx, F &&fn) {
  if (ctx->precision == IBDVM_FP64) {
    if (ctx->dim == 2) return fn(double(), std::integral_constant<int, 2>());
    return fn(double(), std::integral_constant<int, 3>());
  }
  if (ctx->dim == 2) return fn(float(), std::integral_constant<int, 2>());
  return fn(float(), std::integral_constant<int, 3>());
}

} // namespace

cudaError_t launch_init_state(ibdvm_ctx *ctx) {
  const int per_cell = ctx->nvp * ctx->ncomp;
  const long long total = ctx->ncell * per_cell;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 64);
  if (ctx->precision == IBDVM_FP64)
    init_state_kernel<double><<<grid, 256, 0, ctx->stream>>>(
        static_cast<double *>(ctx->f[0]), static_cast<double *>(ctx->f[1]),
        static_cast<const double *>(ctx->finf), ctx->ncell, per_cell);
  else
    init_state_kernel<float><<<grid, 256, 0, ctx->stream>>>(
        static_cast<float *>(ctx->f[0]), static_cast<float *>(ctx->f[1]),
        static_cast<const float *>(ctx->finf), ctx->ncell, per_cell);
  return cudaGetLastError();
}

cudaError_t launch_refresh_range(ibdvm_ctx *ctx, long long c0, long long c1) {
  if (c1 <= c0) return cudaSuccess;
  Timed t(ctx, kKMoments);
  ctx->kernel_launches[kKMoments] += 4;
  return dispatch(ctx, [&](auto t, auto d) -> cudaError_t {
    using T = decltype(t);
    constexpr int D = decltype(d)::value;
    // first pass about zero (W into W[1 - wcur]), second about the bulk
    // velocity that pass stored (W into W[wcur])
    for (int pass = 0; pass < 2; ++pass) {
      MomArgs<T> M{};
      M.f = static_cast<const T *>(ctx->f[ctx->cur]);
      M.mac = static_cast<const T *>(ctx->mac);
      M.xi = static_cast<const T *>(ctx->xiT);
      M.w = static_cast<const T *>(ctx->wT);
      M.ctype = ctx->ctype;
      M.part = ctx->part;
      M.ncell = ctx->ncell;
      M.c0 = c0;
      M.c1 = c1;
      M.nv = ctx->nv;
      M.nvp = ctx->nvp;
      M.shift = pass;
      const unsigned grid = (unsigned)((c1 - c0 + kMomWarps - 1) / kMomWarps);
      moments_kernel<T, D><<<grid, 32 * kMomWarps, 0, ctx->stream>>>(M);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      FinalArgs<T, double> A =
          final_args<T, double>(ctx, pass == 0 ? ctx->wcur : 1 - ctx->wcur, pass == 1, false, ctx->part, 1);
      A.c0 = c0;
      A.c1 = c1;
      A.nblk = (int)((c1 - c0 + 255) / 256);
      finalize_kernel<T, D, double><<<A.nblk, 256, 0, ctx->stream>>>(A);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  });
}

// rows of W^n and q^n per cell, [ncell][D + 2] and [ncell][D], from the
// per-quantity layout [D + 2 + D][ncell]
__global__ void __launch_bounds__(256) interleave_kernel(const double *__restrict__ W, double *__restrict__ Wo,
                                                         double *__restrict__ qo, long long nc, int NW, int D) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  if (Wo)
    for (int i = 0; i < NW; ++i) Wo[c * NW + i] = W[i * nc + c];
  if (qo)
    for (int a = 0; a < D; ++a) qo[c * D + a] = W[(NW + a) * nc + c];
}

cudaError_t launch_interleave(ibdvm_ctx *ctx, double *Wo, double *qo) {
  const long long nc = ctx->ncell;
  interleave_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, ctx->stream>>>(ctx->W[ctx->wcur], Wo, qo, nc,
                                                                          ctx->dim + 2, ctx->dim);
  return cudaGetLastError();
}

cudaError_t launch_ghost_band(ibdvm_ctx *ctx, double *dbg) {
  if (ctx->nlink == 0 && ctx->wall_mask == 0) return cudaSuccess;
  Timed t(ctx, kKGhost);
  // the halo values of diffuse domain walls first: the pre-ghost slopes and
  // the sweep read them
  ctx->kernel_launches[kKGhost] += (ctx->wall_mask ? 1 : 0) + (ctx->nlink ? 1 : 0);
  return dispatch(ctx, [&](auto t, auto d) -> cudaError_t {
    using T = decltype(t);
    constexpr int D = decltype(d)::value;
    if (ctx->wall_mask) {
      cudaError_t e = domain_t<T, D>(ctx);
      if (e != cudaSuccess) return e;
    }
    return ghost_t<T, D>(ctx, dbg);
  });
}

cudaError_t launch_wall(ibdvm_ctx *ctx, const double *fstar, double *out) {
  if (ctx->nlink == 0) return cudaSuccess;
  const Geom &g = ctx->geom;
  WallArgs A{};
  A.fstar = fstar;
  A.xiD = ctx->xiD;
  A.wD = ctx->wD;
  A.l_dbl = ctx->l_dbl;
  A.kst = ctx->kst;
  A.out = out;
  A.nv = ctx->nv;
  A.nvp = ctx->nvp;
  A.Tw = g.body.T_w;
  for (int a = 0; a < 3; ++a) A.Uw[a] = g.body.U_w[a];
  A.p0 = 0.5 * g.gas.rho_inf * g.gas.T_inf;
  A.dyn0 = g.gas.rho_inf * (g.Uinf[0] * g.Uinf[0] + g.Uinf[1] * g.Uinf[1] + g.Uinf[2] * g.Uinf[2]);
  ctx->kernel_launches[kKOther] += 1;
  if (ctx->dim == 2)
    wall_kernel<2><<<ctx->nlink, kWallThreads, 0, ctx->stream>>>(A);
  else
    wall_kernel<3><<<ctx->nlink, kWallThreads, 0, ctx->stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_sweep(ibdvm_ctx *ctx) {
  return dispatch(ctx, [&](auto t, auto d) -> cudaError_t {
    using T = decltype(t);
    constexpr int D = decltype(d)::value;
    cudaError_t e;
    const bool tma = std::is_same<T, float>::value && ctx->use_tma;
    {
      Timed tm(ctx, kKSweep);
      ctx->kernel_launches[kKSweep] += 1;
      e = ctx->tree ? tree_sweep_t<T, D>(ctx)
          : tma     ? (D == 2 ? tma_sweep_launch(ctx) : tma3_sweep_launch(ctx))
                    : sweep_t<T, D>(ctx, 1, 1);
    }
    if (e != cudaSuccess) return e;
    ctx->cur = 1 - ctx->cur;
    Timed tm(ctx, kKMoments);
    ctx->kernel_launches[kKMoments] += 2;
    if (tma) return finalize_t<T, D, float>(ctx, true, true, ctx->partf, ctx->tma_nchunk);
    return finalize_t<T, D>(ctx, true, true);
  });
}

cudaError_t launch_forces(ibdvm_ctx *ctx, double *dst) {
  Timed t(ctx, kKForces);
  ctx->kernel_launches[kKForces] += ctx->nlink ? 2 : 0;
  return dispatch(ctx, [&](auto t, auto d) -> cudaError_t {
    using T = decltype(t);
    constexpr int D = decltype(d)::value;
    return forces_t<T, D>(ctx, dst);
  });
}

cudaError_t launch_convert(ibdvm_ctx *ctx, double *dense, long long c0, long long ncells, bool to_state) {
  const long long total = ncells * (long long)ctx->nv * ctx->ncomp;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 64);
  if (total == 0) return cudaSuccess;
  if (ctx->precision == IBDVM_FP64)
    convert_kernel<double><<<grid, 256, 0, ctx->stream>>>(static_cast<double *>(ctx->f[ctx->cur]), dense, ctx->kst, c0,
                                                          ncells, ctx->nv, ctx->nvp, ctx->ncomp, to_state);
  else
    convert_kernel<float><<<grid, 256, 0, ctx->stream>>>(static_cast<float *>(ctx->f[ctx->cur]), dense, ctx->kst, c0,
                                                         ncells, ctx->nv, ctx->nvp, ctx->ncomp, to_state);
  return cudaGetLastError();
}

} // namespace ibdvm

// ---------------------------------------------------------------------------
// grouped launches over the members of a batch
// ---------------------------------------------------------------------------

namespace ibdvm {

namespace {
template <typename T> cudaError_t upload_table(const std::vector<T> &h, void *&d, cudaStream_t s) {
  cudaError_t e = cudaMalloc(&d, std::max<size_t>(h.size(), 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (h.empty()) return cudaSuccess;
  return cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}
} // namespace

void group_free(GroupTables &t) {
  void *ps[] = {t.ghost, t.force, t.fin, t.link_start, t.fin_start};
  for (void *p : ps)
    if (p) cudaFree(p);
  t = GroupTables{};
}

cudaError_t group_build(const std::vector<ibdvm_ctx *> &cases, const std::vector<int> &nchunk, double *res,
                        int *flags, double *forces, GroupTables &t, cudaStream_t s) {
  group_free(t);
  const int n = static_cast<int>(cases.size());
  t.ncase = n;
  t.dim = n ? cases[0]->dim : 2;
  std::vector<int> ls(n + 1, 0), fs(n + 1, 0);
  std::vector<GhostArgs<float>> g(2 * n);
  std::vector<ForceArgs<float>> fa(2 * n);
  std::vector<FinalArgs<float, float>> fi(2 * n);
  for (int i = 0; i < n; ++i) {
    const ibdvm_ctx *ctx = cases[i];
    ls[i + 1] = ls[i] + ctx->nlink;
    fs[i + 1] = fs[i] + static_cast<int>((ctx->ncell + 255) / 256);
    for (int p = 0; p < 2; ++p) {
      g[2 * i + p] = ghost_args<float>(ctx, ctx->cur ^ p, nullptr);
      fa[2 * i + p] = force_args<float>(ctx, ctx->cur ^ p, forces + 4 * i);
      FinalArgs<float, float> A = final_args<float, float>(ctx, ctx->wcur ^ p, true, true, ctx->partf, nchunk[i]);
      A.flags = flags + i;
      A.res_out = res + i;
      fi[2 * i + p] = A;
    }
  }
  t.link_blocks = ls[n];
  t.fin_blocks = fs[n];
  cudaError_t e;
  if ((e = upload_table(g, t.ghost, s)) != cudaSuccess) return e;
  if ((e = upload_table(fa, t.force, s)) != cudaSuccess) return e;
  if ((e = upload_table(fi, t.fin, s)) != cudaSuccess) return e;
  void *p0 = nullptr, *p1 = nullptr;
  if ((e = upload_table(ls, p0, s)) != cudaSuccess) return e;
  t.link_start = static_cast<int *>(p0);
  if ((e = upload_table(fs, p1, s)) != cudaSuccess) return e;
  t.fin_start = static_cast<int *>(p1);
  return cudaStreamSynchronize(s); // the host tables go out of scope
}

cudaError_t group_ghost(const GroupTables &t, int par, cudaStream_t s) {
  if (t.link_blocks == 0) return cudaSuccess;
  const auto *tab = static_cast<const GhostArgs<float> *>(t.ghost);
  if (t.dim == 2)
    ghost_band_grouped<float, 2><<<t.link_blocks, kGhostThreads, 0, s>>>(tab, t.link_start, t.ncase, par);
  else
    ghost_band_grouped<float, 3><<<t.link_blocks, kGhostThreads, 0, s>>>(tab, t.link_start, t.ncase, par);
  return cudaGetLastError();
}

cudaError_t group_forces(const GroupTables &t, int par, cudaStream_t s) {
  if (t.ncase == 0) return cudaSuccess;
  const auto *tab = static_cast<const ForceArgs<float> *>(t.force);
  if (t.link_blocks > 0) {
    if (t.dim == 2)
      forces_grouped<float, 2><<<t.link_blocks, 256, 0, s>>>(tab, t.link_start, t.ncase, par);
    else
      forces_grouped<float, 3><<<t.link_blocks, 256, 0, s>>>(tab, t.link_start, t.ncase, par);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  forces_total_grouped<float><<<t.ncase, 256, 0, s>>>(tab, par);
  return cudaGetLastError();
}

cudaError_t group_finalize(const GroupTables &t, int par, cudaStream_t s) {
  if (t.ncase == 0) return cudaSuccess;
  const auto *tab = static_cast<const FinalArgs<float, float> *>(t.fin);
  if (t.dim == 2)
    finalize_grouped<float, 2, float><<<t.fin_blocks, 256, 0, s>>>(tab, t.fin_start, t.ncase, par);
  else
    finalize_grouped<float, 3, float><<<t.fin_blocks, 256, 0, s>>>(tab, t.fin_start, t.ncase, par);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (t.dim == 2)
    residual_grouped<float, 2, float><<<t.ncase, 256, 0, s>>>(tab, par);
  else
    residual_grouped<float, 3, float><<<t.ncase, 256, 0, s>>>(tab, par);
  return cudaGetLastError();
}

} // namespace ibdvm
