// sweep_tma.cu -- the transport / relaxation / moments sweep of 2D cases in
// FP32 storage (the mixed path), staged through shared memory by TMA.
//
// Same arithmetic as sweep_kernel in kernels.cu (Sec. 2.2 Eqs. reconstruction
// and limiter, Sec. 4 reduced Shakhov equilibria, forward Euler, Eqs.
// moments1-3 by quadrature), organised for GB300:
//
//   * a block owns TX = 8 columns of cells (one warp per column), a chunk of
//     KC = 32 * KPT velocities (lane l owns velocities l, l + 32, ..., so every
//     shared-memory access of a warp is 256 contiguous bytes), and marches up
//     a range of rows;
//   * every row of the block (its TX columns plus two halo columns on each
//     side, all KC velocities) arrives in shared memory by one TMA tensor copy
//     (cp.async.bulk.tensor.3d) into a ring of NST stages guarded by
//     mbarriers, issued NST - 3 rows ahead, so HBM is read once per row and
//     the x stencil comes from shared memory;
//   * each lane keeps its column's y stencil in registers (f at rows y..y+2
//     and the reconstructed faces of rows y-1..y+1), rotated by moves (one copy
//     of the row body keeps the instruction cache warm);
//   * x faces are exchanged through shared memory: every warp publishes the
//     face value of its own cell on the downwind side and reads its upwind
//     neighbour's as the inflow face; the faces of the two halo columns are
//     spread over all threads of the block (one velocity each);
//   * the nine moment sums of the new state (about the stored bulk velocity)
//     are reduced over the 32 lanes by a butterfly (each shuffle round halves
//     the values a lane holds) and written as FP32 partial sums per velocity
//     chunk; the finalize kernel adds the chunks in FP64.
//
// Conditions that are the same for a whole warp (a ghost neighbour, the
// domain edge, a cell that is not fluid) select between a fast path and a
// general path per warp, never per velocity.  Every mbarrier wait is bounded:
// on timeout the block sets an error flag, drains its copies (bounded) and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "ctx.h"
#include "tma_sync.cuh"

namespace ibdvm {
namespace {

using namespace dev;

constexpr int TX = 8;       // interior columns per block, one warp each
constexpr int NST = 6;      // TMA row stages
constexpr int COLS = TX + 4;
constexpr int NTHREADS = TX * 32;
constexpr int NM = 9;       // moment sums (2D)

template <int KPT> struct Cfg {
  static constexpr int KC = 32 * KPT;
  static constexpr int KC2 = 2 * KC; // floats of one column in a staged row
  static constexpr int STAGE_FLOATS = COLS * KC2;
  static constexpr int STAGE_BYTES = STAGE_FLOATS * 4;
  static constexpr int PHI_FLOATS = (TX + 2) * KC2;
  static constexpr size_t SMEM = (size_t)(NST * STAGE_FLOATS + 2 * PHI_FLOATS + KC2 + KC + 2 * TX * kMac) * 4 + NST * 8;
};

struct TmaArgs {
  float *__restrict__ fn;
  const float *__restrict__ f;
  const float *__restrict__ mac;  // [ncell][kMac]
  const float *__restrict__ xi;   // [3][nvp]
  const float *__restrict__ w;    // [nvp]
  const float *__restrict__ finf; // [nvp][2]
  const uint8_t *__restrict__ cmask;
  const int *__restrict__ dslot;
  const int *__restrict__ dlinks;
  const float *__restrict__ lval; // [nlink][nvp][2]
  float *__restrict__ part;       // [nchunk][NM][ncell]
  int *__restrict__ err;
  long long ncell;
  int nx, ny, nvp, nv, rows;
  float dt, rdx, rdy;
  // diffuse domain walls: faces 2a + (s > 0) in wmask, the halo values of
  // their boundary cells [slot][nvp][2] from the first slot woff[face]
  const float *__restrict__ whalo;
  long long woff[4];
  int wmask;
};

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tma_row(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}



__device__ __forceinline__ float2 link_value(const TmaArgs &A, long long c, int dir, int k) {
  const int slot = A.dslot[c];
  const int l = (slot >= 0) ? A.dlinks[slot * 6 + dir] : -1;
  const float *p = (l >= 0) ? A.lval + ((size_t)l * A.nvp + k) * 2 : A.finf + (size_t)k * 2;
  return make_float2(p[0], p[1]);
}

enum : uint8_t { kXm = 1, kXp = 2, kYm = 4, kYp = 8, kNotFluid = 64, kGhostAny = 15 };

template <int KPT> using Ring = float2[KPT];

// Shared state of one block's march, passed to the per-row body.
template <int KPT> struct March {
  const TmaArgs &A;
  const CUtensorMap *tm;
  float *stage, *phix, *sfinf, *sxi;
  uint64_t *full;
  int warp, lane, x0, x, k0, y0, y1, ylast;
  int st;       // stage of row y
  unsigned pb;  // parity of that stage's current use
  bool col_in;
  long long nc;
  float xix[KPT], xiy[KPT], wk[KPT];
  float ax[KPT], ay[KPT];    // dt |xi_a| / dx_a
  float sy[KPT];             // sign of xi_y
  float *smac;               // [2][TX][kMac]: cell parameters of rows y and y + 1
  float pre_mac;             // lanes 0..kMac-1: one parameter of the next row's cell
  uint8_t mask_next2;        // flags of (x, y + 2)
  bool abort_local;
  bool inner_x;              // the column is inside the domain, away from its x edges
  // the halo column face this thread owns (threads below KC): chunk velocity,
  // column, its slot in a staged row, its face slot
  int h_kk, h_col, h_scol, h_out;
  bool h_in, h_fast;         // the column lies in the domain; and away from its x edges
  float2 h_s2;               // sign of that velocity's xi_x, packed
  // running pointers of row y, advanced by one row per step
  const uint8_t *cm_row;     // flags of row y
  const float *mac_next;     // this lane's parameter of the cell at row y + 1
  float *fn_cell;            // f^{n+1} of the own cell, first chunk velocity
  float *part_cell;          // moment partial sums of the own cell (sum index of the lane)
};

// velocity q of a lane: k = k0 + lane + 32 q, so a warp touches 32 consecutive
// (h, b) pairs per access (256 contiguous bytes, no bank conflicts)
template <int KPT> __device__ __forceinline__ int klo(const March<KPT> &M, int q) { return M.lane + 32 * q; }
template <int KPT> __device__ __forceinline__ int kof(const March<KPT> &M, int q) { return M.k0 + klo(M, q); }

template <int KPT> __device__ __forceinline__ float2 sm2(const float *base, int kk) {
  return *reinterpret_cast<const float2 *>(base + 2 * kk);
}

// the values of the halo cells across face i = 2a + (s > 0) of the boundary
// cell at transverse index t (the row for x faces, the column for y faces),
// from the chunk's first velocity: the slot a diffuse wall wrote this step,
// or the freestream (both halo layers hold the same values)
// (W: the case has diffuse domain walls; without, the code is that of the
// freestream halo alone)
template <int KPT, bool W> __device__ __forceinline__ const float *halo_ptr(const March<KPT> &M, int i, int t) {
  if constexpr (!W) {
    return M.sfinf;
  } else {
    if (!((M.A.wmask >> i) & 1)) return M.sfinf;
    return M.A.whalo + ((size_t)(M.A.woff[i] + t) * M.A.nvp + M.k0) * 2;
  }
}

template <int KPT> __device__ __forceinline__ void issue_row(March<KPT> &M, int r, int st) {
  using C = Cfg<KPT>;
  mbar_expect_tx(&M.full[st], C::STAGE_BYTES);
  tma_row(M.stage + st * C::STAGE_FLOATS, M.tm, 2 * M.k0, M.x0 - 2, r, &M.full[st]);
}

template <int KPT> __device__ __forceinline__ uint8_t cmask_of(const March<KPT> &M, int cx, int r) {
  if (cx < 0 || cx >= M.A.nx || r < 0 || r >= M.A.ny) return 0;
  return M.A.cmask[cx + (long long)M.A.nx * r];
}

// downwind x face of column cx at row y for chunk velocity kk, with the
// domain edge, ghost neighbours and cells that are not fluid
template <int KPT, bool W>
__device__ __forceinline__ float2 phi_x_one(const March<KPT> &M, const float *srow, int cx, int scol, int y,
                                            uint8_t m, int kk, float xi) {
  using C = Cfg<KPT>;
  // halo column: its value, zero slope
  if (cx < 0 || cx >= M.A.nx) return sm2<KPT>(halo_ptr<KPT, W>(M, cx < 0 ? 0 : 1, y), kk);
  if (m & kNotFluid) return make_float2(0.f, 0.f);
  const float *pc = srow + scol * C::KC2;
  const float2 f = sm2<KPT>(pc, kk);
  float2 lo = (cx - 1 < 0) ? sm2<KPT>(halo_ptr<KPT, W>(M, 0, y), kk) : sm2<KPT>(pc - C::KC2, kk);
  float2 hi = (cx + 1 >= M.A.nx) ? sm2<KPT>(halo_ptr<KPT, W>(M, 1, y), kk) : sm2<KPT>(pc + C::KC2, kk);
  if (m & (kXm | kXp)) {
    const long long c = cx + (long long)M.A.nx * y;
    if (m & kXm) lo = link_value(M.A, c, 0, M.k0 + kk);
    if (m & kXp) hi = link_value(M.A, c, 1, M.k0 + kk);
  }
  return face2(f, lo, hi, dup(copysignf(1.f, xi)));
}

// downwind y face of row r, cell (x, r): fr = f(r), lo = f(r-1), hi = f(r+1)
template <int KPT, bool W>
__device__ __forceinline__ void phi_y(const March<KPT> &M, int r, uint8_t m, const Ring<KPT> &fr,
                                      const Ring<KPT> &lo, const Ring<KPT> &hi, Ring<KPT> &out) {
  if (r < 0 || r >= M.A.ny || !M.col_in) { // halo row: its value, zero slope
    const float *h = M.col_in ? halo_ptr<KPT, W>(M, r < 0 ? 2 : 3, M.x) : M.sfinf;
#pragma unroll
    for (int q = 0; q < KPT; ++q) out[q] = sm2<KPT>(h, klo(M, q));
    return;
  }
  if (m & kNotFluid) {
#pragma unroll
    for (int q = 0; q < KPT; ++q) out[q] = make_float2(0.f, 0.f);
    return;
  }
  // the last row under a top wall: the ring holds the freestream past the
  // edge; the wall's halo slot holds the value across it
  const bool top = W && (r == M.A.ny - 1) && (M.A.wmask & 8);
  if (!(m & (kYm | kYp)) && !top) { // fast path
#pragma unroll
    for (int q = 0; q < KPT; ++q) out[q] = face2(fr[q], lo[q], hi[q], dup(M.sy[q]));
    return;
  }
  const long long c = M.x + (long long)M.A.nx * r;
  const float *th = top ? halo_ptr<KPT, W>(M, 3, M.x) : M.sfinf;
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    const float2 l = (m & kYm) ? link_value(M.A, c, 2, kof(M, q)) : lo[q];
    const float2 h = (m & kYp) ? link_value(M.A, c, 3, kof(M, q)) : (top ? sm2<KPT>(th, klo(M, q)) : hi[q]);
    out[q] = face2(fr[q], l, h, dup(M.sy[q]));
  }
}

// One row y of the march.  Ring arguments: Ra = f(y), Rb = f(y+1), Rc <- f(y+2);
// Pa = phi(y-1), Pb = phi(y), Pc <- phi(y+1); mc = flags of (x, y), carried to
// the next row as the flags of (x, y+1).  Returns false when the block aborts.
template <int KPT, bool W>
__device__ __forceinline__ bool row(March<KPT> &M, int y, int par, uint8_t &mc, Ring<KPT> &Ra, Ring<KPT> &Rb,
                                    Ring<KPT> &Rc, Ring<KPT> &Pa, Ring<KPT> &Pb, Ring<KPT> &Pc) {
  using C = Cfg<KPT>;
  const TmaArgs &A = M.A;
  const long long cell = M.x + (long long)A.nx * y;
  const uint8_t m0 = mc;
  const bool fluid = !(m0 & kNotFluid);
  // prefetch for the next row: one cell parameter per lane, the flags of (x, y + 3);
  // this row's parameters were staged in shared memory by the previous row
  const float pre_next = (M.lane < kMac && M.col_in && y + 1 < A.ny) ? __ldg(M.mac_next) : 0.f;
  const uint8_t mn = M.mask_next2; // flags of (x, y + 1), loaded a row ahead
  const uint8_t mn3 = M.col_in ? ((y + 2 < A.ny) ? M.cm_row[2 * A.nx + M.x] : 0) : kNotFluid;
  // stages of rows y and y + 2
  const int st = M.st;
  int st2 = st + 2;
  unsigned pb2 = M.pb;
  if (st2 >= NST) {
    st2 -= NST;
    pb2 ^= 1u;
  }
  // (1) own column of row y + 2 (the y stencil)
  if (y + 2 < A.ny && !mbar_wait(&M.full[st2], pb2)) M.abort_local = true;
  {
    // the own column of row y + 2, or the freestream past the domain edge
    // (where the top face is a wall, phi_y reads its halo for the last row)
    const float *src = (y + 2 < A.ny && M.col_in) ? M.stage + st2 * C::STAGE_FLOATS + (M.warp + 2) * C::KC2
                                                  : M.sfinf;
#pragma unroll
    for (int q = 0; q < KPT; ++q) Rc[q] = sm2<KPT>(src, klo(M, q));
  }
  const float *srow = M.stage + st * C::STAGE_FLOATS; // row y, [COLS][KC][2]
  float *ph = M.phix + par * C::PHI_FLOATS;            // [TX + 2][KC][2]
  // (2) downwind x face of the own cell
  Ring<KPT> PX;
  if (M.inner_x && fluid && !(m0 & (kXm | kXp))) {
    const float *pc = srow + (M.warp + 2) * C::KC2;
#pragma unroll
    for (int q = 0; q < KPT; ++q)
      PX[q] = face2(Ra[q], sm2<KPT>(pc - C::KC2, klo(M, q)), sm2<KPT>(pc + C::KC2, klo(M, q)),
                    dup(copysignf(1.f, M.xix[q])));
  } else {
#pragma unroll
    for (int q = 0; q < KPT; ++q)
      PX[q] = phi_x_one<KPT, W>(M, srow, M.x, M.warp + 2, y, M.col_in ? m0 : 0, klo(M, q), M.xix[q]);
  }
#pragma unroll
  for (int q = 0; q < KPT; ++q) *reinterpret_cast<float2 *>(ph + (M.warp + 1) * C::KC2 + 2 * klo(M, q)) = PX[q];
  // the halo column that is upwind of the block for each velocity: x0 - 1
  // for xi_x >= 0, x0 + TX otherwise; one velocity per thread
  static_assert(Cfg<KPT>::KC <= NTHREADS, "one halo face per thread at most");
  if (threadIdx.x < C::KC) {
    const uint8_t hm = M.h_in ? M.cm_row[M.h_col] : 0;
    float2 o;
    if (M.h_fast && !(hm & (kNotFluid | kXm | kXp))) {
      // interior halo column, fluid, no ghost along x: f and its neighbours
      // from the staged row, the sign of the velocity decides the side
      const float *pc = srow + M.h_scol * C::KC2;
      o = face2(sm2<KPT>(pc, M.h_kk), sm2<KPT>(pc - C::KC2, M.h_kk), sm2<KPT>(pc + C::KC2, M.h_kk), M.h_s2);
    } else {
      o = phi_x_one<KPT, W>(M, srow, M.h_col, M.h_scol, y, hm, M.h_kk, M.sxi[M.h_kk]);
    }
    *reinterpret_cast<float2 *>(ph + M.h_out) = o;
  }
  // (3) downwind y face of row y + 1
  phi_y<KPT, W>(M, y + 1, mn, Rb, Ra, Rc, Pc);
  // (4) barrier: x faces published, the stage of row y - 1 released; all
  //     threads agree on an abort
  if (__syncthreads_or(M.abort_local ? 1 : 0)) return false;
  if (threadIdx.x == 0 && y + NST - 1 < M.ylast) {
    fence_proxy_async();
    issue_row(M, y + NST - 1, st == 0 ? NST - 1 : st - 1);
  }
  // (5) update of the own cell and its moment sums
  float2 a03 = make_float2(0.f, 0.f), a17 = a03, a28 = a03, a45 = a03;
  float a6 = 0.f;
  if (fluid) {
    const float4 *pm = reinterpret_cast<const float4 *>(M.smac + (par * TX + M.warp) * kMac);
    const float4 p0 = pm[0], p1 = pm[1], p2 = pm[2];
    const float pre = p0.x, U0 = p0.y, U1 = p0.z;
    const float invT = p1.x, halfT = p1.y, shA = p1.z, q0 = p1.w;
    const float q1 = p2.x, dtau = p2.z;
    const float Tc = 2.f * halfT;
    const float2 omd = dup(1.f - dtau), dt2 = dup(dtau);
    const bool ghosty = (m0 & kGhostAny) != 0;
    Ring<KPT> out;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      // inflow faces: the upwind neighbour's downwind face
      const bool posx = M.xix[q] >= 0.f, posy = M.xiy[q] >= 0.f;
      float2 ix = sm2<KPT>(ph + (M.warp + (posx ? 0 : 2)) * C::KC2, klo(M, q));
      float2 iy = posy ? Pa[q] : Pc[q];
      if (ghosty) { // a ghost upwind neighbour: mean of its link value and this cell
        if (posx ? (m0 & kXm) : (m0 & kXp)) {
          const float2 g = link_value(A, cell, posx ? 0 : 1, kof(M, q));
          ix = __fmul2_rn(dup(0.5f), __fadd2_rn(g, Ra[q]));
        }
        if (posy ? (m0 & kYm) : (m0 & kYp)) {
          const float2 g = link_value(A, cell, posy ? 2 : 3, kof(M, q));
          iy = __fmul2_rn(dup(0.5f), __fadd2_rn(g, Ra[q]));
        }
      }
      // Shakhov equilibrium (Sec. 4 reduced forms) from the stored state:
      // (H, B) = (e, T/2 e) + m (2t - 4, T t - T), t = c^2 / T
      const float cx = M.xix[q] - U0, cy = M.xiy[q] - U1;
      const float c2 = fmaf(cx, cx, cy * cy);
      const float t = c2 * invT;
      const float e = pre * __expf(-t);
      const float mm = e * shA * fmaf(cx, q0, cy * q1);
      const float2 G = make_float2(fmaf(mm, fmaf(2.f, t, -4.f), e), fmaf(mm, fmaf(Tc, t, -Tc), halfT * e));
      // forward Euler: relaxation and the flux divergence of both axes,
      // |xi_a| dt / dx_a (inflow face - outflow face)
      float2 n = __ffma2_rn(Ra[q], omd, __fmul2_rn(dt2, G));
      n = __ffma2_rn(dup(M.ax[q]), sub2(ix, PX[q]), n);
      n = __ffma2_rn(dup(M.ay[q]), sub2(iy, Pb[q]), n);
      out[q] = n;
      // moments of the new state about the stored bulk velocity
      const float wh = M.wk[q] * n.x;
      const float e2 = fmaf(c2, wh, M.wk[q] * n.y); // w (c^2 h + b)
      a03.x += wh;
      a03.y += e2;
      a17.x = fmaf(cx, wh, a17.x);
      a17.y = fmaf(cx, e2, a17.y);
      a28.x = fmaf(cy, wh, a28.x);
      a28.y = fmaf(cy, e2, a28.y);
      const float cxwh = cx * wh;
      a45.x = fmaf(cx, cxwh, a45.x);
      a45.y = fmaf(cy, cxwh, a45.y);
      a6 = fmaf(cy * cy, wh, a6);
    }
#pragma unroll
    for (int q = 0; q < KPT; ++q) *reinterpret_cast<float2 *>(M.fn_cell + 2 * klo(M, q)) = out[q];
  }
  // (6) butterfly reduction of the sums over the 32 lanes: three rounds halve
  //     the eight values a lane holds, two more finish the one it keeps; the
  //     ninth sum is a plain xor tree
  {
    const float acc[NM] = {a03.x, a17.x, a28.x, a03.y, a45.x, a45.y, a6, a17.y, a28.y};
    const int lane = M.lane;
    float v4[4];
    const bool b16 = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float keep = b16 ? acc[4 + i] : acc[i];
      const float send = b16 ? acc[i] : acc[4 + i];
      v4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float v2[2];
    const bool b8 = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float keep = b8 ? v4[2 + i] : v4[i];
      const float send = b8 ? v4[i] : v4[2 + i];
      v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const bool b4 = lane & 4;
    float v1 = (b4 ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, b4 ? v2[0] : v2[1], 4);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
    float s8 = acc[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s8 += __shfl_xor_sync(0xffffffffu, s8, o);
    if (M.col_in) {
      if ((lane & 3) == 0) *M.part_cell = v1;
      if (lane == 1) *M.part_cell = s8;
    }
  }
  if (M.lane < kMac) M.smac[((par ^ 1) * TX + M.warp) * kMac + M.lane] = pre_next;
  M.mask_next2 = mn3;
  mc = mn;
  M.cm_row += A.nx;
  M.mac_next += (size_t)A.nx * kMac;
  M.fn_cell += (size_t)A.nx * A.nvp * 2;
  M.part_cell += A.nx;
  if (++M.st == NST) {
    M.st = 0;
    M.pb ^= 1u;
  }
  return true;
}

// The march of one block over columns [x0, x0 + TX), chunk velocities
// [k0, k0 + KC) and rows [y0, y1).  reinit: the block's mbarriers hold an
// earlier march (all of whose copies have landed) and are invalidated first.
// Returns false when the block aborted on a timed-out wait.
template <int KPT, bool W>
__device__ __forceinline__ bool march2d(const TmaArgs &A, const CUtensorMap *tmf, int x0, int k0, int y0, int y1,
                                        unsigned char *smem_raw, bool reinit) {
  using C = Cfg<KPT>;
  March<KPT> M{A, tmf};
  M.stage = reinterpret_cast<float *>(smem_raw);
  M.phix = M.stage + NST * C::STAGE_FLOATS;
  M.sfinf = M.phix + 2 * C::PHI_FLOATS;
  M.sxi = M.sfinf + C::KC2;
  M.smac = M.sxi + C::KC;
  M.full = reinterpret_cast<uint64_t *>(M.smac + 2 * TX * kMac);
  M.warp = threadIdx.x >> 5;
  M.lane = threadIdx.x & 31;
  M.x0 = x0;
  M.k0 = k0;
  M.y0 = y0;
  M.y1 = y1;
  M.ylast = min(A.ny, M.y1 + 2); // rows this block reads: [y0, ylast)
  M.x = M.x0 + M.warp;
  M.col_in = M.x < A.nx;
  M.nc = A.ncell;
  M.inner_x = M.col_in && M.x > 0 && M.x + 1 < A.nx;
  M.cm_row = A.cmask + (long long)A.nx * M.y0;
  M.mac_next = A.mac + (M.x + (long long)A.nx * (M.y0 + 1)) * kMac + (M.lane < kMac ? M.lane : 0);
  M.fn_cell = A.fn + ((size_t)(M.x + (long long)A.nx * M.y0) * A.nvp + M.k0) * 2;
  {
    // lanes 4 i write sum i (i < 8); lane 1 writes the ninth sum
    const int sidx = ((M.lane & 3) == 0) ? (M.lane >> 2) : 8;
    M.part_cell = A.part + ((size_t)(M.k0 / C::KC) * NM + sidx) * M.nc + M.x + (long long)A.nx * M.y0;
  }
  if (threadIdx.x < C::KC) {
    M.h_kk = threadIdx.x;
    const bool left = A.xi[M.k0 + M.h_kk] >= 0.f; // the halo column upwind of the block
    M.h_col = left ? M.x0 - 1 : M.x0 + TX;
    M.h_scol = left ? 1 : TX + 2;
    M.h_out = (left ? 0 : TX + 1) * C::KC2 + 2 * M.h_kk;
    M.h_in = M.h_col >= 0 && M.h_col < A.nx;
    M.h_fast = M.h_col >= 1 && M.h_col + 1 < A.nx;
    M.h_s2 = dup(left ? 1.f : -1.f);
  }
  M.st = 0;
  M.pb = 0;
  M.abort_local = false;
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    const int k = kof(M, q);
    const bool valid = k < A.nv;
    // padding velocities: an enormous speed makes the equilibrium vanish,
    // zero flux coefficients and zero weight keep them out of everything
    M.xix[q] = valid ? A.xi[k] : 1e18f;
    M.xiy[q] = valid ? A.xi[A.nvp + k] : 1e18f;
    M.wk[q] = valid ? A.w[k] : 0.f;
    M.ax[q] = valid ? A.dt * fabsf(M.xix[q]) * A.rdx : 0.f;
    M.ay[q] = valid ? A.dt * fabsf(M.xiy[q]) * A.rdy : 0.f;
    M.sy[q] = copysignf(1.f, M.xiy[q]);
  }
  // parameters of the first row's cells, and the flags of row y0 + 1
  if (M.lane < kMac)
    M.smac[M.warp * kMac + M.lane] = M.col_in ? A.mac[(M.x + (long long)A.nx * M.y0) * kMac + M.lane] : 0.f;
  M.mask_next2 = M.col_in ? ((M.y0 + 1 < A.ny) ? cmask_of(M, M.x, M.y0 + 1) : 0) : kNotFluid;
  for (int i = threadIdx.x; i < C::KC2; i += NTHREADS) M.sfinf[i] = A.finf[2 * M.k0 + i];
  for (int i = threadIdx.x; i < C::KC; i += NTHREADS) M.sxi[i] = A.xi[M.k0 + i];
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      if (reinit) mbar_inval(&M.full[s]);
      mbar_init(&M.full[s], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int r = M.y0; r < min(M.ylast, M.y0 + NST - 1); ++r) issue_row(M, r, r - M.y0);

  // own-column ring for rows y0-2 .. y0+1, straight from global memory
  auto own = [&](int r, Ring<KPT> &v) {
    if (r < 0 || r >= A.ny || !M.col_in) {
      const float *h = M.col_in ? halo_ptr<KPT, W>(M, r < 0 ? 2 : 3, M.x) : M.sfinf;
#pragma unroll
      for (int q = 0; q < KPT; ++q) v[q] = sm2<KPT>(h, klo(M, q));
    } else {
      const float *src = A.f + ((size_t)(M.x + (long long)A.nx * r) * A.nvp + M.k0) * 2;
#pragma unroll
      for (int q = 0; q < KPT; ++q) v[q] = *reinterpret_cast<const float2 *>(src + 2 * klo(M, q));
    }
  };
  Ring<KPT> R0, R1, R2, P0, P1, P2;
  {
    Ring<KPT> Rm2;
    own(M.y0 - 2, Rm2);
    own(M.y0 - 1, R2);
    own(M.y0, R0);
    own(M.y0 + 1, R1);
    phi_y<KPT, W>(M, M.y0 - 1, M.col_in ? cmask_of(M, M.x, M.y0 - 1) : kNotFluid, R2, Rm2, R0, P0);
    phi_y<KPT, W>(M, M.y0, M.col_in ? cmask_of(M, M.x, M.y0) : kNotFluid, R0, R2, R1, P1);
  }
  // rows y0 and y0+1 are read from shared memory by the x stencil
  for (int r = M.y0; r < min(M.ylast, M.y0 + 2); ++r)
    if (!mbar_wait(&M.full[r - M.y0], 0)) M.abort_local = true;
  uint8_t mc = M.col_in ? cmask_of(M, M.x, M.y0) : kNotFluid;
  int y = M.y0;
  int par = 0;
  bool ok = true;
  for (; y < M.y1; ++y) {
    ok = row<KPT, W>(M, y, par, mc, R0, R1, R2, P0, P1, P2);
    if (!ok) break;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      R0[q] = R1[q];
      R1[q] = R2[q];
      P0[q] = P1[q];
      P1[q] = P2[q];
    }
    par ^= 1;
  }
  if (!ok && threadIdx.x == 0) {
    atomicOr(A.err, kFlagTimeout);
    // drain: rows issued but not yet waited for must land (or time out
    // again) before the block's shared memory is released
    const int issued_end = min(M.ylast, y + NST - 1);
    for (int r = max(M.y0 + 2, y + 2); r < issued_end; ++r) {
      const int j = r - M.y0;
      mbar_wait(&M.full[j % NST], (j / NST) & 1);
    }
  }
  return ok;
}

template <int KPT, bool W>
__global__ void __launch_bounds__(NTHREADS, 2) sweep2d_tma_kernel(const __grid_constant__ CUtensorMap tmf,
                                                                  TmaArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int y0 = blockIdx.z * A.rows;
  march2d<KPT, W>(A, &tmf, blockIdx.x * TX, blockIdx.y * Cfg<KPT>::KC, y0, min(A.ny, y0 + A.rows), smem_raw, false);
}

// One item of the batched sweep: a march of one member case.
struct WorkItem {
  int cas;    // member index
  int x0, k0; // first column and first chunk velocity
  int y0, y1; // rows
  int kpt;    // velocities per lane (2 or 4)
  int pad[2];
};

// The batched sweep: a persistent grid whose blocks take work items in order
// from a shared counter (items sorted by decreasing size).  Member c at step
// parity par uses args[2 c + par] and tmaps[2 c + par].  KSEL = 4 or 2 when
// every item takes that many velocities per lane, 0 for a mix.
template <int KSEL>
__global__ void __launch_bounds__(NTHREADS, 2)
    sweep2d_tma_batch_kernel(const TmaArgs *__restrict__ args, const CUtensorMap *__restrict__ tmaps,
                             const WorkItem *__restrict__ items, int nitems, int *__restrict__ next, int par) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ TmaArgs sA;
  __shared__ int s_item;
  bool reinit = false;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int i = s_item;
    if (i >= nitems) break;
    const WorkItem it = items[i];
    if (threadIdx.x == 0) sA = args[2 * it.cas + par];
    __syncthreads();
    const CUtensorMap *tm = tmaps + 2 * it.cas + par;
    bool ok;
    if constexpr (KSEL == 4)
      ok = march2d<4, false>(sA, tm, it.x0, it.k0, it.y0, it.y1, smem_raw, reinit);
    else if constexpr (KSEL == 2)
      ok = march2d<2, false>(sA, tm, it.x0, it.k0, it.y0, it.y1, smem_raw, reinit);
    else
      ok = (it.kpt == 4) ? march2d<4, false>(sA, tm, it.x0, it.k0, it.y0, it.y1, smem_raw, reinit)
                         : march2d<2, false>(sA, tm, it.x0, it.k0, it.y0, it.y1, smem_raw, reinit);
    if (!ok) break; // uniform: the abort vote is block-wide
    reinit = true;
    __syncthreads(); // the item's shared memory and arguments are released
  }
}

// driver entry point for the tensor-map encoder, looked up once
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

} // namespace

// The TMA sweep applies to 2D cases in FP32 storage with the velocity count
// padded to a multiple of 64.
bool tma_sweep_applicable(const ibdvm_ctx *ctx) {
  return ctx->dim == 2 && ctx->precision == IBDVM_MIXED && (ctx->nvp % 64) == 0 && encoder() != nullptr;
}

int tma_sweep_kpt(const ibdvm_ctx *ctx) { return (ctx->nvp % 128 == 0) ? 4 : 2; }
int tma_sweep_nchunk(const ibdvm_ctx *ctx) { return ctx->nvp / (32 * tma_sweep_kpt(ctx)); }

cudaError_t tma_sweep_prepare(ibdvm_ctx *ctx) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const int kpt = tma_sweep_kpt(ctx);
  const int kc = 32 * kpt;
  for (int b = 0; b < 2; ++b) {
    CUtensorMap *tm = reinterpret_cast<CUtensorMap *>(ctx->tmap[b]);
    cuuint64_t dims[3] = {(cuuint64_t)ctx->nvp * 2, (cuuint64_t)ctx->geom.n[0], (cuuint64_t)ctx->geom.n[1]};
    cuuint64_t strides[2] = {(cuuint64_t)ctx->nvp * 2 * 4, (cuuint64_t)ctx->geom.n[0] * ctx->nvp * 2 * 4};
    cuuint32_t box[3] = {(cuuint32_t)(2 * kc), (cuuint32_t)COLS, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ctx->f[b], dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  const int s4 = (int)Cfg<4>::SMEM, s2 = (int)Cfg<2>::SMEM;
  cudaError_t e = (kpt == 4) ? cudaFuncSetAttribute(sweep2d_tma_kernel<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4)
                             : cudaFuncSetAttribute(sweep2d_tma_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
  if (e != cudaSuccess) return e;
  return (kpt == 4) ? cudaFuncSetAttribute(sweep2d_tma_kernel<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4)
                    : cudaFuncSetAttribute(sweep2d_tma_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
}

cudaError_t tma_sweep_launch(ibdvm_ctx *ctx) {
  TmaArgs A{};
  A.f = static_cast<const float *>(ctx->f[ctx->cur]);
  A.fn = static_cast<float *>(ctx->f[1 - ctx->cur]);
  A.mac = static_cast<const float *>(ctx->mac);
  A.xi = static_cast<const float *>(ctx->xiT);
  A.w = static_cast<const float *>(ctx->wT);
  A.finf = static_cast<const float *>(ctx->finf);
  A.cmask = ctx->cmask;
  A.dslot = ctx->dslot;
  A.dlinks = ctx->dlinks;
  A.lval = static_cast<const float *>(ctx->lval);
  A.part = ctx->partf;
  A.err = ctx->d_flags;
  A.ncell = ctx->ncell;
  A.nx = ctx->geom.n[0];
  A.ny = ctx->geom.n[1];
  A.nvp = ctx->nvp;
  A.nv = ctx->nv;
  A.dt = (float)ctx->geom.dt;
  A.rdx = (float)(1.0 / ctx->geom.dx[0]);
  A.rdy = (float)(1.0 / ctx->geom.dx[1]);
  A.whalo = static_cast<const float *>(ctx->whalo);
  A.wmask = ctx->wall_mask;
  for (int i = 0; i < 4; ++i) A.woff[i] = ctx->wall_off[i];
  const int kpt = tma_sweep_kpt(ctx);
  const int nstrip = (A.nx + TX - 1) / TX;
  const int nchunk = ctx->nvp / (32 * kpt);
  // rows per block: about 64 (many short marches leave a short tail: on
  // 512^2 x 48^2, 64 rows per block beat 128, 256 and 32), and enough blocks
  // for several waves of two blocks per SM
  int nrb = (A.ny + 63) / 64;
  while ((long long)nstrip * nchunk * nrb < 8LL * 152 && A.ny / (nrb * 2) >= 16) nrb *= 2;
  A.rows = (A.ny + nrb - 1) / nrb;
  dim3 grid(nstrip, nchunk, (A.ny + A.rows - 1) / A.rows);
  const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(ctx->tmap[ctx->cur]);
  // cases with diffuse domain walls read their halo at the domain edges
  if (A.wmask) {
    if (kpt == 4)
      sweep2d_tma_kernel<4, true><<<grid, NTHREADS, Cfg<4>::SMEM, ctx->stream>>>(*tm, A);
    else
      sweep2d_tma_kernel<2, true><<<grid, NTHREADS, Cfg<2>::SMEM, ctx->stream>>>(*tm, A);
  } else if (kpt == 4) {
    sweep2d_tma_kernel<4, false><<<grid, NTHREADS, Cfg<4>::SMEM, ctx->stream>>>(*tm, A);
  } else {
    sweep2d_tma_kernel<2, false><<<grid, NTHREADS, Cfg<2>::SMEM, ctx->stream>>>(*tm, A);
  }
  return cudaGetLastError();
}

bool tma_batch_member_ok(const ibdvm_ctx *ctx) {
  if (ctx->precision != IBDVM_MIXED || ctx->partf == nullptr || encoder() == nullptr) return false;
  if (ctx->dim == 2) return (ctx->nvp % 64) == 0;
  return tma3_sweep_applicable(ctx);
}

int tma_batch_kpt_max(const ibdvm_ctx *ctx) { return (ctx->dim == 3 || ctx->nvp % 128 == 0) ? 4 : 2; }

void tma_batch_free(SweepTables &t) {
  void *ps[] = {t.args, t.tmaps, t.items, t.next};
  for (void *p : ps)
    if (p) cudaFree(p);
  t = SweepTables{};
}

cudaError_t tma_batch_build(const std::vector<ibdvm_ctx *> &cases, const std::vector<int> &kpt, int rows,
                            int *flags, SweepTables &t, cudaStream_t s) {
  tma_batch_free(t);
  if (!cases.empty() && cases[0]->dim == 3) return tma3_batch_build(cases, rows, flags, t, s);
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const int n = static_cast<int>(cases.size());
  std::vector<TmaArgs> args(2 * n);
  std::vector<CUtensorMap> maps(2 * n);
  std::vector<WorkItem> items;
  for (int i = 0; i < n; ++i) {
    const ibdvm_ctx *ctx = cases[i];
    const int kc = 32 * kpt[i];
    for (int p = 0; p < 2; ++p) {
      const int cur = ctx->cur ^ p;
      TmaArgs &A = args[2 * i + p];
      A = TmaArgs{};
      A.f = static_cast<const float *>(ctx->f[cur]);
      A.fn = static_cast<float *>(ctx->f[1 - cur]);
      A.mac = static_cast<const float *>(ctx->mac);
      A.xi = static_cast<const float *>(ctx->xiT);
      A.w = static_cast<const float *>(ctx->wT);
      A.finf = static_cast<const float *>(ctx->finf);
      A.cmask = ctx->cmask;
      A.dslot = ctx->dslot;
      A.dlinks = ctx->dlinks;
      A.lval = static_cast<const float *>(ctx->lval);
      A.part = ctx->partf;
      A.err = flags + i;
      A.ncell = ctx->ncell;
      A.nx = ctx->geom.n[0];
      A.ny = ctx->geom.n[1];
      A.nvp = ctx->nvp;
      A.nv = ctx->nv;
      A.rows = 0;
      A.dt = (float)ctx->geom.dt;
      A.rdx = (float)(1.0 / ctx->geom.dx[0]);
      A.rdy = (float)(1.0 / ctx->geom.dx[1]);
      cuuint64_t dims[3] = {(cuuint64_t)ctx->nvp * 2, (cuuint64_t)A.nx, (cuuint64_t)A.ny};
      cuuint64_t strides[2] = {(cuuint64_t)ctx->nvp * 2 * 4, (cuuint64_t)A.nx * ctx->nvp * 2 * 4};
      cuuint32_t box[3] = {(cuuint32_t)(2 * kc), (cuuint32_t)COLS, 1};
      cuuint32_t estr[3] = {1, 1, 1};
      CUresult r = enc(&maps[2 * i + p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ctx->f[cur], dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    // items: column strips x velocity chunks x row ranges of about `rows` rows
    const int nx = ctx->geom.n[0], ny = ctx->geom.n[1];
    const int nrb = (rows <= 0 || rows >= ny) ? 1 : (ny + rows - 1) / rows;
    const int per = (ny + nrb - 1) / nrb;
    for (int x0 = 0; x0 < nx; x0 += TX)
      for (int k0 = 0; k0 < ctx->nvp; k0 += kc)
        for (int y0 = 0; y0 < ny; y0 += per) {
          WorkItem it{};
          it.cas = i;
          it.x0 = x0;
          it.k0 = k0;
          it.y0 = y0;
          it.y1 = std::min(ny, y0 + per);
          it.kpt = kpt[i];
          items.push_back(it);
        }
  }
  // largest items first, so the last items to start are the short ones
  std::stable_sort(items.begin(), items.end(), [](const WorkItem &a, const WorkItem &b) {
    return (long long)(a.y1 - a.y0) * a.kpt > (long long)(b.y1 - b.y0) * b.kpt;
  });
  cudaError_t e;
  auto up = [&](const void *h, size_t bytes, void *&d) -> cudaError_t {
    cudaError_t r = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (r != cudaSuccess || bytes == 0) return r;
    return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
  };
  if ((e = up(args.data(), args.size() * sizeof(TmaArgs), t.args)) != cudaSuccess) return e;
  if ((e = up(maps.data(), maps.size() * sizeof(CUtensorMap), t.tmaps)) != cudaSuccess) return e;
  if ((e = up(items.data(), items.size() * sizeof(WorkItem), t.items)) != cudaSuccess) return e;
  void *nx = nullptr;
  if ((e = cudaMalloc(&nx, sizeof(int))) != cudaSuccess) return e;
  t.next = static_cast<int *>(nx);
  t.nitems = static_cast<int>(items.size());
  {
    bool all4 = true, all2 = true;
    for (int k : kpt) {
      all4 = all4 && k == 4;
      all2 = all2 && k == 2;
    }
    t.ksel = all4 ? 4 : (all2 ? 2 : 0);
  }
  const int smem = (int)std::max(Cfg<4>::SMEM, Cfg<2>::SMEM);
  const void *fn = (t.ksel == 4) ? (const void *)sweep2d_tma_batch_kernel<4>
                   : (t.ksel == 2) ? (const void *)sweep2d_tma_batch_kernel<2>
                                   : (const void *)sweep2d_tma_batch_kernel<0>;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTHREADS, smem)) != cudaSuccess) return e;
  t.grid = std::max(1, std::min(t.nitems, nsm * std::max(per_sm, 1)));
  return cudaStreamSynchronize(s); // the host tables go out of scope
}

cudaError_t tma_batch_launch(const SweepTables &t, int par, cudaStream_t s) {
  if (t.dim == 3) return tma3_batch_launch(t, par, s);
  if (t.nitems == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.next, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int smem = (int)std::max(Cfg<4>::SMEM, Cfg<2>::SMEM);
  const TmaArgs *a = static_cast<const TmaArgs *>(t.args);
  const CUtensorMap *m = static_cast<const CUtensorMap *>(t.tmaps);
  const WorkItem *it = static_cast<const WorkItem *>(t.items);
  if (t.ksel == 4)
    sweep2d_tma_batch_kernel<4><<<t.grid, NTHREADS, smem, s>>>(a, m, it, t.nitems, t.next, par);
  else if (t.ksel == 2)
    sweep2d_tma_batch_kernel<2><<<t.grid, NTHREADS, smem, s>>>(a, m, it, t.nitems, t.next, par);
  else
    sweep2d_tma_batch_kernel<0><<<t.grid, NTHREADS, smem, s>>>(a, m, it, t.nitems, t.next, par);
  return cudaGetLastError();
}

} // namespace ibdvm
