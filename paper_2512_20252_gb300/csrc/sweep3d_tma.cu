// sweep3d_tma.cu -- the transport / relaxation / moments sweep of 3D cases in
// FP32 storage (the mixed path), staged through shared memory by TMA.
//
// Same arithmetic as sweep_kernel in kernels.cu (Sec. 2.2 Eqs. reconstruction
// and limiter, the Shakhov equilibrium of Sec. 2.1 in the non-dimensional
// form of Sec. 4, forward Euler, Eqs. moments1-3 by quadrature), organised for
// GB300:
//
//   * a block owns a 4 x 4 tile of (x, y) columns of cells (16 warps, one per
//     column) and a chunk of KC = 32 * KPT velocities (lane l owns the pairs of
//     neighbouring velocities 2 l + 64 j, 2 l + 64 j + 1), and marches along z;
//     every per-velocity operation works on such a pair with Blackwell's packed
//     FP32 instructions (__ffma2_rn and friends) and 64-bit loads and stores;
//   * every z plane of the block arrives in shared memory as a cross-shaped
//     slab: the 4 x 4 tile and two halo strips of two cells on each side in x
//     and in y (48 cells x KC velocities), five TMA tensor copies
//     (cp.async.bulk.tensor.4d) on one mbarrier per stage of a 5-stage ring;
//   * each lane keeps its column's z stencil in registers (f at planes z..z+2
//     and the reconstructed faces of planes z-1..z+1);
//   * a face is f + s vl(f - f_lo, f_hi - f) with s the sign of the velocity
//     (the van Leer half slope is symmetric and odd), so no face is selected;
//   * x and y faces are exchanged through shared memory: every warp publishes
//     the downwind faces of its cell; the faces of the halo cells on the
//     upwind side of the tile are spread over all threads;
//   * the fourteen moment sums (about the stored bulk velocity) are reduced
//     over the 32 lanes by a butterfly and written as FP32 partial sums per
//     velocity chunk; the finalize kernel adds the chunks in FP64.
//
// Conditions that hold for a whole warp (ghost neighbours, the domain edge, a
// cell that is not fluid) select a general path per warp.  Every mbarrier
// wait is bounded: on timeout the block sets an error flag, drains its copies
// (bounded) and returns.
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

constexpr int TX = 4, TY = 4;   // tile of columns, one warp each
constexpr int NW = TX * TY;     // warps per block
constexpr int NTHREADS = NW * 32;
constexpr int NST = 5;          // TMA plane stages
constexpr int NCELL = TX * TY + 2 * (2 * TY) + 2 * (2 * TX); // cells of the cross-shaped slab (48)
constexpr int NM = 14;          // moment sums (3D)

// slot of slab cell (i, j), i in [-2, TX+2), j in [-2, TY+2), cross-shaped
__device__ __forceinline__ int slot(int i, int j) {
  if (i >= 0 && i < TX && j >= 0 && j < TY) return j * TX + i;              // centre [y][x]
  if (i < 0) return TX * TY + j * 2 + (i + 2);                              // x halo low  [y][2]
  if (i >= TX) return TX * TY + 2 * TY + j * 2 + (i - TX);                  // x halo high [y][2]
  if (j < 0) return TX * TY + 4 * TY + (j + 2) * TX + i;                    // y halo low  [2][x]
  return TX * TY + 4 * TY + 2 * TX + (j - TY) * TX + i;                      // y halo high [2][x]
}

template <int KPT> struct Cfg {
  static constexpr int KC = 32 * KPT;
  static constexpr int STAGE_FLOATS = NCELL * KC;
  static constexpr int STAGE_BYTES = STAGE_FLOATS * 4;
  static constexpr int PX_FLOATS = (TX + 2) * TY * KC; // x faces: [y][x+1][k]
  static constexpr int PY_FLOATS = TX * (TY + 2) * KC; // y faces: [y+1][x][k]
  static constexpr size_t SMEM =
      (size_t)(NST * STAGE_FLOATS + 2 * (PX_FLOATS + PY_FLOATS) + 4 * KC + 2 * NW * kMac) * 4 +
      2 * NTHREADS * sizeof(int4) + NST * 8;
};

struct Tma3Args {
  float *__restrict__ fn;
  const float *__restrict__ f;
  const float *__restrict__ mac;  // [ncell][kMac]
  const float *__restrict__ xi;   // [3][nvp]
  const float *__restrict__ w;    // [nvp]
  const float *__restrict__ finf; // [nvp]
  const uint8_t *__restrict__ cmask;
  const int *__restrict__ dslot;
  const int *__restrict__ dlinks;
  const float *__restrict__ lval; // [nlink][nvp]
  float *__restrict__ part;       // [nchunk][NM][ncell]
  int *__restrict__ err;
  long long ncell;
  int nx, ny, nz, nvp, nv, zrows;
  float dt, rdx, rdy, rdz;
};

__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                        uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}
// half the van Leer slope times the cell width from the one-sided differences
// a = f - f_up and b = f_dn - f along the direction of motion (Eq. limiter)
__device__ __forceinline__ float vl_half(float a, float b) {
  const float p = a * b;
  const float v = p * rcp_approx(a + b);
  return p > 0.f ? v : 0.f;
}
// downwind face value: f plus half the slope along the motion
__device__ __forceinline__ float face(float f, float up, float dn) { return f + vl_half(f - up, dn - f); }

__device__ __forceinline__ float2 lds2(const float *base, int kk) { return *reinterpret_cast<const float2 *>(base + kk); }

__device__ __forceinline__ float link_value(const Tma3Args &A, long long c, int dir, int k) {
  const int s = A.dslot[c];
  const int l = (s >= 0) ? A.dlinks[s * 6 + dir] : -1;
  return (l >= 0) ? A.lval[(size_t)l * A.nvp + k] : A.finf[k];
}
// the link values of velocities k, k + 1 (k even)
__device__ __forceinline__ float2 link_value2(const Tma3Args &A, long long c, int dir, int k) {
  const int s = A.dslot[c];
  const int l = (s >= 0) ? A.dlinks[s * 6 + dir] : -1;
  return *reinterpret_cast<const float2 *>((l >= 0) ? A.lval + (size_t)l * A.nvp + k : A.finf + k);
}

enum : uint8_t { kNotFluid = 64, kGhostAny = 63 };

template <int KPT> using Ring = float2[KPT / 2];

// Every thread owns two halo faces per plane, both for chunk velocity
// kk = threadIdx.x % KC: the downwind x face of the upwind x-halo cell of row
// threadIdx.x / KC, and the downwind y face of the upwind y-halo cell of column
// threadIdx.x / KC.  All but the cells' flags is the same for every plane and
// is packed once into shared memory (int4 per face):
//   x: stage offset of f | (offset of the upwind neighbour + 1) << 16
//   y: offset of the downwind neighbour + 1 | face buffer offset << 16
//      (a neighbour offset of 0 after the + 1 means the freestream value)
//   z: the halo cell's index within a plane, or -1 outside the domain
template <int KPT> struct March3 {
  const Tma3Args &A;
  const CUtensorMap *tc, *tx, *ty; // tensor maps: tile, x halo strip, y halo strip
  float *stage, *phx, *phy, *sfinf, *sxi, *syi, *smac;
  uint64_t *full;
  int warp, lane, ti, tj, x0, y0, x, y, k0, z0, z1, zlast;
  int st;
  unsigned pb;
  bool col_in;
  long long nc, plane;
  // per velocity pair: xi, weight, dt |xi_a| / dx_a, sign of xi_a
  float2 xix[KPT / 2], xiy[KPT / 2], xiz[KPT / 2], wk[KPT / 2], ax[KPT / 2], ay[KPT / 2], az[KPT / 2];
  float2 sx[KPT / 2], sy[KPT / 2], sz[KPT / 2];
  uint8_t mask_next;
  uint16_t hm_next;  // flags of this thread's two halo cells at plane z (x | y << 8)
  bool abort_local;
  bool inner_xy;     // the column is fluid-capable away from the x and y domain edges
  long long nxy;     // cells per plane
  // running pointers of the current plane z, advanced by one plane per step
  const uint8_t *cm_plane; // flags of plane z
  const float *mac_next;   // this lane's parameter of the cell at plane z + 1
  float *fn_cell;          // f^{n+1} of the own cell, first chunk velocity
  float *part_cell;        // moment partial sums of the own cell, sum index lane >> 1
  const int4 *duty; // [2][NTHREADS]: x faces, then y faces
};

// chunk-local index of the first velocity of pair j of the lane
template <int KPT> __device__ __forceinline__ int kp(const March3<KPT> &M, int j) { return 2 * M.lane + 64 * j; }

template <int KPT> __device__ __forceinline__ void issue_plane(March3<KPT> &M, int z, int st) {
  using C = Cfg<KPT>;
  float *dst = M.stage + st * C::STAGE_FLOATS;
  uint64_t *bar = &M.full[st];
  mbar_expect_tx(bar, C::STAGE_BYTES);
  const int kc = M.k0;
  tma_box(dst + slot(0, 0) * C::KC, M.tc, kc, M.x0, M.y0, z, bar);
  tma_box(dst + slot(-2, 0) * C::KC, M.tx, kc, M.x0 - 2, M.y0, z, bar);
  tma_box(dst + slot(TX, 0) * C::KC, M.tx, kc, M.x0 + TX, M.y0, z, bar);
  tma_box(dst + slot(0, -2) * C::KC, M.ty, kc, M.x0, M.y0 - 2, z, bar);
  tma_box(dst + slot(0, TY) * C::KC, M.ty, kc, M.x0, M.y0 + TY, z, bar);
}

template <int KPT> __device__ __forceinline__ uint8_t cmask3(const March3<KPT> &M, int cx, int cy, int cz) {
  const Tma3Args &A = M.A;
  if (cx < 0 || cx >= A.nx || cy < 0 || cy >= A.ny || cz < 0 || cz >= A.nz) return 0;
  return A.cmask[cx + (long long)A.nx * (cy + (long long)A.ny * cz)];
}

// downwind face along axis a (0: x, 1: y) of slab cell (i, j) at plane z for
// chunk velocity kk, general path: domain edge, ghost neighbours, non-fluid
template <int KPT>
__device__ __forceinline__ float face_general(const March3<KPT> &M, const float *sp, int a, int i, int j, int z,
                                              int kk, float xi) {
  using C = Cfg<KPT>;
  const Tma3Args &A = M.A;
  const int cx = M.x0 + i, cy = M.y0 + j;
  if (cx < 0 || cx >= A.nx || cy < 0 || cy >= A.ny) return M.sfinf[kk]; // halo: freestream, zero slope
  const uint8_t m = cmask3(M, cx, cy, z);
  if (m & kNotFluid) return 0.f;
  const int s = (xi >= 0.f) ? 1 : -1;
  const int di = (a == 0) ? s : 0, dj = (a == 1) ? s : 0;
  const float f = sp[slot(i, j) * C::KC + kk];
  const int ca = (a == 0) ? cx : cy, na = (a == 0) ? A.nx : A.ny;
  const long long c = cx + (long long)A.nx * (cy + (long long)A.ny * z);
  float up, dn;
  // upwind neighbour (against the motion) and downwind neighbour
  if (m & (1u << (2 * a + (s > 0 ? 0 : 1)))) up = link_value(A, c, 2 * a + (s > 0 ? 0 : 1), M.k0 + kk);
  else if (ca - s < 0 || ca - s >= na) up = M.sfinf[kk];
  else up = sp[slot(i - di, j - dj) * C::KC + kk];
  if (m & (1u << (2 * a + (s > 0 ? 1 : 0)))) dn = link_value(A, c, 2 * a + (s > 0 ? 1 : 0), M.k0 + kk);
  else if (ca + s < 0 || ca + s >= na) dn = M.sfinf[kk];
  else dn = sp[slot(i + di, j + dj) * C::KC + kk];
  return face(f, up, dn);
}

// the same for the velocity pair at chunk index kk of the own cell (i, j),
// from the low and high neighbours along the axis and the signs s
template <int KPT>
__device__ __forceinline__ float2 face_general2(const March3<KPT> &M, const float *sp, int a, int i, int j, int z,
                                                int kk, float2 s) {
  using C = Cfg<KPT>;
  const Tma3Args &A = M.A;
  const int cx = M.x0 + i, cy = M.y0 + j;
  if (cx < 0 || cx >= A.nx || cy < 0 || cy >= A.ny) return lds2(M.sfinf, kk);
  const uint8_t m = cmask3(M, cx, cy, z);
  if (m & kNotFluid) return make_float2(0.f, 0.f);
  const int di = (a == 0) ? 1 : 0, dj = (a == 1) ? 1 : 0;
  const float2 f = lds2(sp + slot(i, j) * C::KC, kk);
  const int ca = (a == 0) ? cx : cy, na = (a == 0) ? A.nx : A.ny;
  const long long c = cx + (long long)A.nx * (cy + (long long)A.ny * z);
  float2 lo, hi;
  if (m & (1u << (2 * a))) lo = link_value2(A, c, 2 * a, M.k0 + kk);
  else if (ca - 1 < 0) lo = lds2(M.sfinf, kk);
  else lo = lds2(sp + slot(i - di, j - dj) * C::KC, kk);
  if (m & (1u << (2 * a + 1))) hi = link_value2(A, c, 2 * a + 1, M.k0 + kk);
  else if (ca + 1 >= na) hi = lds2(M.sfinf, kk);
  else hi = lds2(sp + slot(i + di, j + dj) * C::KC, kk);
  return face2(f, lo, hi, s);
}

// downwind z face of plane r for the own column: fr = f(r), lo = f(r-1), hi = f(r+1)
template <int KPT>
__device__ __forceinline__ void phi_z(const March3<KPT> &M, int r, uint8_t m, const Ring<KPT> &fr,
                                      const Ring<KPT> &lo, const Ring<KPT> &hi, Ring<KPT> &out) {
  const Tma3Args &A = M.A;
  if (r < 0 || r >= A.nz || !M.col_in) {
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) out[j] = lds2(M.sfinf, kp(M, j));
    return;
  }
  if (m & kNotFluid) {
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) out[j] = make_float2(0.f, 0.f);
    return;
  }
  if (!(m & 48)) {
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) out[j] = face2(fr[j], lo[j], hi[j], M.sz[j]);
    return;
  }
  const long long c = M.plane + (long long)r * A.nx * A.ny;
#pragma unroll
  for (int j = 0; j < KPT / 2; ++j) {
    const float2 l = (m & 16) ? link_value2(A, c, 4, M.k0 + kp(M, j)) : lo[j];
    const float2 h = (m & 32) ? link_value2(A, c, 5, M.k0 + kp(M, j)) : hi[j];
    out[j] = face2(fr[j], l, h, M.sz[j]);
  }
}

// the halo face of axis a owned by this thread at plane z
// the general halo face of axis a owned by this thread at plane z (not fluid,
// or a ghost neighbour along the axis)
template <int KPT, int a>
__device__ __forceinline__ float halo_face_general(const March3<KPT> &M, const float *sp, int z) {
  using C = Cfg<KPT>;
  const int kk = threadIdx.x % C::KC;
  const float xi = (a == 0) ? M.sxi[kk] : M.syi[kk];
  const int line = threadIdx.x / C::KC;
  const int i = (a == 0) ? ((xi >= 0.f) ? -1 : TX) : line;
  const int j = (a == 0) ? line : ((xi >= 0.f) ? -1 : TY);
  return face_general(M, sp, a, i, j, z, kk, xi);
}

// the two halo faces this thread owns at plane z (x, then y), evaluated as one
// packed pair; hm = the flags of the two halo cells at plane z (or 0 outside)
template <int KPT>
__device__ __forceinline__ void halo_faces(const March3<KPT> &M, const float *sp, int z, uint16_t hm, float *phx,
                                           float *phy) {
  using C = Cfg<KPT>;
  const int4 dx = M.duty[threadIdx.x], dy = M.duty[NTHREADS + threadIdx.x];
  const int kk = threadIdx.x % C::KC;
  const float fin = M.sfinf[kk];
  const uint8_t mx = hm & 0xff, my = hm >> 8;
  // per face: freestream outside the domain, the general path where needed
  const bool gx = dx.z >= 0 && (mx & (kNotFluid | 3u)), gy = dy.z >= 0 && (my & (kNotFluid | 12u));
  const int ux = dx.x >> 16, nx = dx.y & 0xffff, uy = dy.x >> 16, ny = dy.y & 0xffff;
  const float2 f = make_float2(sp[dx.x & 0xffff], sp[dy.x & 0xffff]);
  const float2 up = make_float2(ux ? sp[ux - 1] : fin, uy ? sp[uy - 1] : fin);
  const float2 dn = make_float2(nx ? sp[nx - 1] : fin, ny ? sp[ny - 1] : fin);
  const float2 o = __fadd2_rn(f, vl_half2(sub2(f, up), sub2(dn, f)));
  phx[dx.y >> 16] = (dx.z < 0) ? fin : (gx ? halo_face_general<KPT, 0>(M, sp, z) : o.x);
  phy[dy.y >> 16] = (dy.z < 0) ? fin : (gy ? halo_face_general<KPT, 1>(M, sp, z) : o.y);
}

template <int KPT>
__device__ __forceinline__ bool plane_step(March3<KPT> &M, int z, int par, uint8_t &mc, Ring<KPT> &Ra,
                                           Ring<KPT> &Rb, Ring<KPT> &Rc, Ring<KPT> &Pa, Ring<KPT> &Pb,
                                           Ring<KPT> &Pc) {
  using C = Cfg<KPT>;
  const Tma3Args &A = M.A;
  const long long cell = M.plane + (long long)z * M.nxy;
  const uint8_t m0 = mc;
  const bool fluid = !(m0 & kNotFluid);
  const float pre_next = (M.lane < kMac && M.col_in && z + 1 < A.nz) ? __ldg(M.mac_next) : 0.f;
  const uint8_t mn = M.mask_next;
  const uint8_t mn2 = M.col_in ? ((z + 2 < A.nz) ? M.cm_plane[2 * M.nxy + M.plane] : 0) : kNotFluid;
  const int st = M.st;
  int st2 = st + 2;
  unsigned pb2 = M.pb;
  if (st2 >= NST) {
    st2 -= NST;
    pb2 ^= 1u;
  }
  // (1) own column at plane z + 2 (the z stencil)
  if (z + 2 < A.nz && !mbar_wait(&M.full[st2], pb2)) M.abort_local = true;
  if (z + 2 < A.nz && M.col_in) {
    const float *src = M.stage + st2 * C::STAGE_FLOATS + slot(M.ti, M.tj) * C::KC;
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) Rc[j] = lds2(src, kp(M, j));
  } else {
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) Rc[j] = lds2(M.sfinf, kp(M, j));
  }
  const float *sp = M.stage + st * C::STAGE_FLOATS;
  float *phx = M.phx + par * C::PX_FLOATS; // [TY][TX + 2][KC]
  float *phy = M.phy + par * C::PY_FLOATS; // [TY + 2][TX][KC]
  // (2) downwind x and y faces of the own cell
  float2 PX[KPT / 2], PY[KPT / 2];
  const bool fast = M.inner_xy && fluid && !(m0 & 15);
  if (fast) {
    const float *px_lo = sp + slot(M.ti - 1, M.tj) * C::KC, *px_hi = sp + slot(M.ti + 1, M.tj) * C::KC;
    const float *py_lo = sp + slot(M.ti, M.tj - 1) * C::KC, *py_hi = sp + slot(M.ti, M.tj + 1) * C::KC;
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) {
      const int kk = kp(M, j);
      PX[j] = face2(Ra[j], lds2(px_lo, kk), lds2(px_hi, kk), M.sx[j]);
      PY[j] = face2(Ra[j], lds2(py_lo, kk), lds2(py_hi, kk), M.sy[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) {
      PX[j] = face_general2(M, sp, 0, M.ti, M.tj, z, kp(M, j), M.sx[j]);
      PY[j] = face_general2(M, sp, 1, M.ti, M.tj, z, kp(M, j), M.sy[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < KPT / 2; ++j) {
    *reinterpret_cast<float2 *>(phx + (M.tj * (TX + 2) + M.ti + 1) * C::KC + kp(M, j)) = PX[j];
    *reinterpret_cast<float2 *>(phy + ((M.tj + 1) * TX + M.ti) * C::KC + kp(M, j)) = PY[j];
  }
  // halo faces on the upwind side of the tile (TY rows in x, TX columns in y)
  {
    const uint16_t hm = M.hm_next;
    // the flags of the two halo cells at the next plane, a plane ahead of use
    const int hx = M.duty[threadIdx.x].z, hy = M.duty[NTHREADS + threadIdx.x].z;
    M.hm_next = (z + 1 < A.nz) ? (uint16_t)((hx >= 0 ? M.cm_plane[M.nxy + hx] : 0) |
                                            ((hy >= 0 ? M.cm_plane[M.nxy + hy] : 0) << 8))
                               : (uint16_t)0;
    halo_faces(M, sp, z, hm, phx, phy);
  }
  // (3) downwind z face of plane z + 1
  phi_z(M, z + 1, mn, Rb, Ra, Rc, Pc);
  // (4) barrier: faces published, the stage of plane z - 1 released
  if (__syncthreads_or(M.abort_local ? 1 : 0)) return false;
  if (threadIdx.x == 0 && z + NST - 1 < M.zlast) {
    fence_proxy_async();
    issue_plane(M, z + NST - 1, st == 0 ? NST - 1 : st - 1);
  }
  // (5) update of the own cell and its moment sums (per velocity pair)
  float acc[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) acc[m] = 0.f;
  if (fluid) {
    const float4 *pm = reinterpret_cast<const float4 *>(M.smac + (par * NW + M.warp) * kMac);
    const float4 p0 = pm[0], p1 = pm[1], p2 = pm[2];
    const float pre = p0.x, U0 = p0.y, U1 = p0.z, U2 = p0.w;
    const float invT = p1.x, shA = p1.z, q0 = p1.w;
    const float q1 = p2.x, q2 = p2.y, dtau = p2.z;
    const float2 omd = dup(1.f - dtau), dt2 = dup(dtau);
    const bool ghosty = (m0 & kGhostAny) != 0;
    const float *xl = phx + (M.tj * (TX + 2) + M.ti) * C::KC, *xr = xl + 2 * C::KC;
    const float *yl = phy + (M.tj * TX + M.ti) * C::KC, *yr = yl + 2 * TX * C::KC;
    Ring<KPT> out;
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) {
      const int kk = kp(M, j);
      // inflow faces: the upwind neighbour's downwind face, per velocity
      const float2 fxl = lds2(xl, kk), fxr = lds2(xr, kk), fyl = lds2(yl, kk), fyr = lds2(yr, kk);
      float2 ix = make_float2(M.sx[j].x > 0.f ? fxl.x : fxr.x, M.sx[j].y > 0.f ? fxl.y : fxr.y);
      float2 iy = make_float2(M.sy[j].x > 0.f ? fyl.x : fyr.x, M.sy[j].y > 0.f ? fyl.y : fyr.y);
      float2 iz = make_float2(M.sz[j].x > 0.f ? Pa[j].x : Pc[j].x, M.sz[j].y > 0.f ? Pa[j].y : Pc[j].y);
      if (ghosty) { // ghost upwind neighbour: mean of its link value and this cell
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = M.k0 + kk + e;
          const float fc = e ? Ra[j].y : Ra[j].x;
          const int dx = ((e ? M.sx[j].y : M.sx[j].x) > 0.f) ? 0 : 1;
          const int dy = ((e ? M.sy[j].y : M.sy[j].x) > 0.f) ? 2 : 3;
          const int dz = ((e ? M.sz[j].y : M.sz[j].x) > 0.f) ? 4 : 5;
          if (m0 & (1u << dx)) (e ? ix.y : ix.x) = 0.5f * (link_value(A, cell, dx, k) + fc);
          if (m0 & (1u << dy)) (e ? iy.y : iy.x) = 0.5f * (link_value(A, cell, dy, k) + fc);
          if (m0 & (1u << dz)) (e ? iz.y : iz.x) = 0.5f * (link_value(A, cell, dz, k) + fc);
        }
      }
      // Shakhov equilibrium g (1 + A c.q (2 c^2/T - 5)) from the stored state
      const float2 cx = __fadd2_rn(M.xix[j], dup(-U0)), cy = __fadd2_rn(M.xiy[j], dup(-U1)),
                   cz = __fadd2_rn(M.xiz[j], dup(-U2));
      const float2 c2 = __ffma2_rn(cx, cx, __ffma2_rn(cy, cy, __fmul2_rn(cz, cz)));
      const float2 t = __fmul2_rn(c2, dup(invT));
      const float2 e = __fmul2_rn(dup(pre), make_float2(__expf(-t.x), __expf(-t.y)));
      const float2 cq = __ffma2_rn(cx, dup(q0), __ffma2_rn(cy, dup(q1), __fmul2_rn(cz, dup(q2))));
      const float2 g = __ffma2_rn(__fmul2_rn(__fmul2_rn(e, dup(shA)), cq), __ffma2_rn(dup(2.f), t, dup(-5.f)), e);
      float2 n = __ffma2_rn(Ra[j], omd, __fmul2_rn(dt2, g));
      n = __ffma2_rn(M.ax[j], sub2(ix, PX[j]), n);
      n = __ffma2_rn(M.ay[j], sub2(iy, PY[j]), n);
      n = __ffma2_rn(M.az[j], sub2(iz, Pb[j]), n);
      out[j] = n;
      const float2 wf = __fmul2_rn(M.wk[j], n), e2 = __fmul2_rn(c2, wf);
      const float2 cxw = __fmul2_rn(cx, wf), cyw = __fmul2_rn(cy, wf);
      const float2 czz = __fmul2_rn(cz, cz);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float w1 = e ? wf.y : wf.x, x1 = e ? cx.y : cx.x, y1 = e ? cy.y : cy.x, z1 = e ? cz.y : cz.x;
        const float xw = e ? cxw.y : cxw.x, yw = e ? cyw.y : cyw.x, ee = e ? e2.y : e2.x;
        acc[0] += w1;
        acc[1] += xw;
        acc[2] += yw;
        acc[3] = fmaf(z1, w1, acc[3]);
        acc[4] += ee;
        acc[5] = fmaf(x1, xw, acc[5]);
        acc[6] = fmaf(y1, xw, acc[6]);
        acc[7] = fmaf(z1, xw, acc[7]);
        acc[8] = fmaf(y1, yw, acc[8]);
        acc[9] = fmaf(z1, yw, acc[9]);
        acc[10] = fmaf(e ? czz.y : czz.x, w1, acc[10]);
        acc[11] = fmaf(x1, ee, acc[11]);
        acc[12] = fmaf(y1, ee, acc[12]);
        acc[13] = fmaf(z1, ee, acc[13]);
      }
    }
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) *reinterpret_cast<float2 *>(M.fn_cell + kp(M, j)) = out[j];
  }
  // (6) butterfly of the 16 (14 used) sums over the 32 lanes
  {
    const int lane = M.lane;
    float v8[8];
    const bool b16 = lane & 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float keep = b16 ? acc[8 + i] : acc[i];
      const float send = b16 ? acc[i] : acc[8 + i];
      v8[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float v4[4];
    const bool b8 = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float keep = b8 ? v8[4 + i] : v8[i];
      const float send = b8 ? v8[i] : v8[4 + i];
      v4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float v2[2];
    const bool b4 = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float keep = b4 ? v4[2 + i] : v4[i];
      const float send = b4 ? v4[i] : v4[2 + i];
      v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const bool b2 = lane & 2;
    float v1 = (b2 ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? v2[0] : v2[1], 2);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
    // lane l holds sum index 8 b4(l) + 4 b3(l) + 2 b2(l) + b1(l) = l >> 1
    if (M.col_in && (lane & 1) == 0 && (lane >> 1) < NM) *M.part_cell = v1;
  }
  if (M.lane < kMac) M.smac[((par ^ 1) * NW + M.warp) * kMac + M.lane] = pre_next;
  M.mask_next = mn2;
  mc = mn;
  M.cm_plane += M.nxy;
  M.mac_next += M.nxy * kMac;
  M.fn_cell += M.nxy * A.nvp;
  M.part_cell += M.nxy;
  if (++M.st == NST) {
    M.st = 0;
    M.pb ^= 1u;
  }
  return true;
}

// The march of one block over the tile of columns at (x0, y0), chunk
// velocities [k0, k0 + KC) and planes [z0, z1).  tm[0..2]: tensor maps of the
// tile and of the x and y halo strips.  reinit: the block's mbarriers hold an
// earlier march (all of whose copies have landed) and are invalidated first.
// Returns false when the block aborted on a timed-out wait.
template <int KPT>
__device__ __forceinline__ bool march3d(const Tma3Args &A, const CUtensorMap *tmc, const CUtensorMap *tmx,
                                        const CUtensorMap *tmy, int x0, int y0, int k0, int z0, int z1,
                                        unsigned char *smem_raw, bool reinit) {
  using C = Cfg<KPT>;
  March3<KPT> M{A, tmc, tmx, tmy};
  M.stage = reinterpret_cast<float *>(smem_raw);
  M.phx = M.stage + NST * C::STAGE_FLOATS;
  M.phy = M.phx + 2 * C::PX_FLOATS;
  M.sfinf = M.phy + 2 * C::PY_FLOATS;
  M.sxi = M.sfinf + C::KC;
  M.syi = M.sxi + C::KC;
  M.smac = M.syi + 2 * C::KC;
  M.duty = reinterpret_cast<const int4 *>(M.smac + 2 * NW * kMac);
  M.full = reinterpret_cast<uint64_t *>(const_cast<int4 *>(M.duty) + 2 * NTHREADS);
  M.warp = threadIdx.x >> 5;
  M.lane = threadIdx.x & 31;
  M.ti = M.warp % TX;
  M.tj = M.warp / TX;
  M.x0 = x0;
  M.y0 = y0;
  M.x = M.x0 + M.ti;
  M.y = M.y0 + M.tj;
  M.col_in = M.x < A.nx && M.y < A.ny;
  M.k0 = k0;
  M.z0 = z0;
  M.z1 = z1;
  M.zlast = min(A.nz, M.z1 + 2);
  M.nc = A.ncell;
  M.plane = M.x + (long long)A.nx * M.y;
  M.nxy = (long long)A.nx * A.ny;
  M.inner_xy = M.col_in && M.x > 0 && M.x + 1 < A.nx && M.y > 0 && M.y + 1 < A.ny;
  M.cm_plane = A.cmask + (long long)M.z0 * M.nxy;
  M.mac_next = A.mac + (M.plane + (long long)(M.z0 + 1) * M.nxy) * kMac + (M.lane < kMac ? M.lane : 0);
  M.fn_cell = A.fn + (size_t)(M.plane + (long long)M.z0 * M.nxy) * A.nvp + M.k0;
  M.part_cell = A.part + ((size_t)(M.k0 / C::KC) * NM + ((M.lane >> 1) < NM ? (M.lane >> 1) : 0)) * M.nc + M.plane +
                (long long)M.z0 * M.nxy;
  M.st = 0;
  M.pb = 0;
  M.abort_local = false;
#pragma unroll
  for (int j = 0; j < KPT / 2; ++j) {
    float v[10][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = M.k0 + kp(M, j) + e;
      const bool valid = k < A.nv;
      // padding velocities: an enormous speed makes the equilibrium vanish,
      // zero flux coefficients and zero weight keep them out of everything
      const float x = valid ? A.xi[k] : 1e18f, y = valid ? A.xi[A.nvp + k] : 1e18f,
                  zz = valid ? A.xi[2 * A.nvp + k] : 1e18f;
      v[0][e] = x;
      v[1][e] = y;
      v[2][e] = zz;
      v[3][e] = valid ? A.w[k] : 0.f;
      v[4][e] = valid ? A.dt * fabsf(x) * A.rdx : 0.f;
      v[5][e] = valid ? A.dt * fabsf(y) * A.rdy : 0.f;
      v[6][e] = valid ? A.dt * fabsf(zz) * A.rdz : 0.f;
      v[7][e] = copysignf(1.f, x);
      v[8][e] = copysignf(1.f, y);
      v[9][e] = copysignf(1.f, zz);
    }
    M.xix[j] = make_float2(v[0][0], v[0][1]);
    M.xiy[j] = make_float2(v[1][0], v[1][1]);
    M.xiz[j] = make_float2(v[2][0], v[2][1]);
    M.wk[j] = make_float2(v[3][0], v[3][1]);
    M.ax[j] = make_float2(v[4][0], v[4][1]);
    M.ay[j] = make_float2(v[5][0], v[5][1]);
    M.az[j] = make_float2(v[6][0], v[6][1]);
    M.sx[j] = make_float2(v[7][0], v[7][1]);
    M.sy[j] = make_float2(v[8][0], v[8][1]);
    M.sz[j] = make_float2(v[9][0], v[9][1]);
  }
  for (int i = threadIdx.x; i < C::KC; i += NTHREADS) {
    M.sfinf[i] = A.finf[M.k0 + i];
    M.sxi[i] = A.xi[M.k0 + i];
    M.syi[i] = A.xi[A.nvp + M.k0 + i];
  }
  {
    static_assert(TX * C::KC == NTHREADS && TY * C::KC == NTHREADS, "two halo faces per thread");
    const int kk = threadIdx.x % C::KC, line = threadIdx.x / C::KC;
    int4 *duty = const_cast<int4 *>(M.duty);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float xi = A.xi[a * A.nvp + M.k0 + kk];
      const int s = (xi >= 0.f) ? 1 : -1;
      const int i = (a == 0) ? ((s > 0) ? -1 : TX) : line;
      const int j = (a == 0) ? line : ((s > 0) ? -1 : TY);
      const int di = (a == 0) ? s : 0, dj = (a == 1) ? s : 0;
      const int cx = M.x0 + i, cy = M.y0 + j;
      const bool outside = cx < 0 || cx >= A.nx || cy < 0 || cy >= A.ny;
      const int ca = (a == 0) ? cx : cy, na = (a == 0) ? A.nx : A.ny;
      const int f_off = slot(i, j) * C::KC + kk;
      const int up = (outside || ca - s < 0 || ca - s >= na) ? 0 : slot(i - di, j - dj) * C::KC + kk + 1;
      const int dn = (outside || ca + s < 0 || ca + s >= na) ? 0 : slot(i + di, j + dj) * C::KC + kk + 1;
      const int out = (a == 0) ? (j * (TX + 2) + i + 1) * C::KC + kk : ((j + 1) * TX + i) * C::KC + kk;
      duty[a * NTHREADS + threadIdx.x] =
          make_int4(f_off | (up << 16), dn | (out << 16), outside ? -1 : cx + A.nx * cy, 0);
    }
  }
  {
    const int hx = M.duty[threadIdx.x].z, hy = M.duty[NTHREADS + threadIdx.x].z;
    M.hm_next = (uint16_t)((hx >= 0 ? M.cm_plane[hx] : 0) | ((hy >= 0 ? M.cm_plane[hy] : 0) << 8));
  }
  if (M.lane < kMac)
    M.smac[M.warp * kMac + M.lane] =
        M.col_in ? A.mac[(M.plane + (long long)M.z0 * A.nx * A.ny) * kMac + M.lane] : 0.f;
  M.mask_next = M.col_in ? ((M.z0 + 1 < A.nz) ? cmask3(M, M.x, M.y, M.z0 + 1) : 0) : kNotFluid;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      if (reinit) mbar_inval(&M.full[s]);
      mbar_init(&M.full[s], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int r = M.z0; r < min(M.zlast, M.z0 + NST - 1); ++r) issue_plane(M, r, r - M.z0);
  auto own = [&](int r, Ring<KPT> &v) {
    if (r < 0 || r >= A.nz || !M.col_in) {
#pragma unroll
      for (int j = 0; j < KPT / 2; ++j) v[j] = lds2(M.sfinf, kp(M, j));
    } else {
      const float *src = A.f + (size_t)(M.plane + (long long)r * A.nx * A.ny) * A.nvp + M.k0;
#pragma unroll
      for (int j = 0; j < KPT / 2; ++j) v[j] = *reinterpret_cast<const float2 *>(src + kp(M, j));
    }
  };
  Ring<KPT> R0, R1, R2, P0, P1, P2;
  {
    Ring<KPT> Rm2;
    own(M.z0 - 2, Rm2);
    own(M.z0 - 1, R2);
    own(M.z0, R0);
    own(M.z0 + 1, R1);
    phi_z(M, M.z0 - 1, M.col_in ? cmask3(M, M.x, M.y, M.z0 - 1) : kNotFluid, R2, Rm2, R0, P0);
    phi_z(M, M.z0, M.col_in ? cmask3(M, M.x, M.y, M.z0) : kNotFluid, R0, R2, R1, P1);
  }
  for (int r = M.z0; r < min(M.zlast, M.z0 + 2); ++r)
    if (!mbar_wait(&M.full[r - M.z0], 0)) M.abort_local = true;
  uint8_t mc = M.col_in ? cmask3(M, M.x, M.y, M.z0) : kNotFluid;
  int z = M.z0, par = 0;
  bool ok = true;
  // one copy of the plane body (a small kernel keeps the instruction cache
  // warm); the ring rotates by moves
  for (; z < M.z1; ++z) {
    ok = plane_step(M, z, par, mc, R0, R1, R2, P0, P1, P2);
    if (!ok) break;
#pragma unroll
    for (int j = 0; j < KPT / 2; ++j) {
      R0[j] = R1[j];
      R1[j] = R2[j];
      P0[j] = P1[j];
      P1[j] = P2[j];
    }
    par ^= 1;
  }
  if (!ok && threadIdx.x == 0) {
    atomicOr(A.err, kFlagTimeout);
    const int issued_end = min(M.zlast, z + NST - 1);
    for (int r = max(M.z0 + 2, z + 2); r < issued_end; ++r) {
      const int j = r - M.z0;
      mbar_wait(&M.full[j % NST], (j / NST) & 1);
    }
  }
  return ok;
}

template <int KPT>
__global__ void __launch_bounds__(NTHREADS, 1)
    sweep3d_tma_kernel(const __grid_constant__ CUtensorMap tmc, const __grid_constant__ CUtensorMap tmx,
                       const __grid_constant__ CUtensorMap tmy, Tma3Args A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ntx = (A.nx + TX - 1) / TX;
  const int z0 = blockIdx.z * A.zrows;
  march3d<KPT>(A, &tmc, &tmx, &tmy, (blockIdx.x % ntx) * TX, (blockIdx.x / ntx) * TY, blockIdx.y * Cfg<KPT>::KC,
               z0, min(A.nz, z0 + A.zrows), smem_raw, false);
}

// One item of the batched 3D sweep: a march of one member case.
struct WorkItem3 {
  int cas;        // member index
  int x0, y0, k0; // tile origin and first chunk velocity
  int z0, z1;     // planes
  int pad[2];
};

// The batched 3D sweep: a persistent grid whose blocks take work items in
// order from a shared counter.  Member c at step parity par uses
// args[2 c + par] and the tensor maps tmaps[3 (2 c + par) + 0..2].
__global__ void __launch_bounds__(NTHREADS, 1)
    sweep3d_tma_batch_kernel(const Tma3Args *__restrict__ args, const CUtensorMap *__restrict__ tmaps,
                             const WorkItem3 *__restrict__ items, int nitems, int *__restrict__ next, int par) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Tma3Args sA;
  __shared__ int s_item;
  bool reinit = false;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int i = s_item;
    if (i >= nitems) break;
    const WorkItem3 it = items[i];
    if (threadIdx.x == 0) sA = args[2 * it.cas + par];
    __syncthreads();
    const CUtensorMap *tm = tmaps + 3 * (2 * it.cas + par);
    const bool ok = march3d<4>(sA, tm, tm + 1, tm + 2, it.x0, it.y0, it.k0, it.z0, it.z1, smem_raw, reinit);
    if (!ok) break; // uniform: the abort vote is block-wide
    reinit = true;
    __syncthreads(); // the item's shared memory and arguments are released
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder3() {
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

constexpr int kKpt3 = 4;

} // namespace

bool tma3_sweep_applicable(const ibdvm_ctx *ctx) {
  return ctx->dim == 3 && ctx->precision == IBDVM_MIXED && (ctx->nvp % (32 * kKpt3)) == 0 && encoder3() != nullptr;
}

int tma3_sweep_nchunk(const ibdvm_ctx *ctx) { return ctx->nvp / (32 * kKpt3); }

cudaError_t tma3_sweep_prepare(ibdvm_ctx *ctx) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder3();
  if (!enc) return cudaErrorNotSupported;
  const int kc = 32 * kKpt3;
  const Geom &g = ctx->geom;
  for (int b = 0; b < 2; ++b) {
    cuuint64_t dims[4] = {(cuuint64_t)ctx->nvp, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    cuuint64_t strides[3] = {(cuuint64_t)ctx->nvp * 4, (cuuint64_t)g.n[0] * ctx->nvp * 4,
                             (cuuint64_t)g.n[1] * g.n[0] * ctx->nvp * 4};
    const cuuint32_t boxes[3][4] = {{(cuuint32_t)kc, TX, TY, 1}, {(cuuint32_t)kc, 2, TY, 1}, {(cuuint32_t)kc, TX, 2, 1}};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int m = 0; m < 3; ++m) {
      CUtensorMap *tm = reinterpret_cast<CUtensorMap *>(ctx->tmap3[b][m]);
      CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->f[b], dims, strides, boxes[m], estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  return cudaFuncSetAttribute(sweep3d_tma_kernel<kKpt3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<kKpt3>::SMEM);
}

cudaError_t tma3_sweep_launch(ibdvm_ctx *ctx) {
  Tma3Args A{};
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
  A.nz = ctx->geom.n[2];
  A.nvp = ctx->nvp;
  A.nv = ctx->nv;
  A.dt = (float)ctx->geom.dt;
  A.rdx = (float)(1.0 / ctx->geom.dx[0]);
  A.rdy = (float)(1.0 / ctx->geom.dx[1]);
  A.rdz = (float)(1.0 / ctx->geom.dx[2]);
  const int ntiles = ((A.nx + TX - 1) / TX) * ((A.ny + TY - 1) / TY);
  const int nchunk = ctx->nvp / (32 * kKpt3);
  int nzb = 1;
  while ((long long)ntiles * nchunk * nzb < 4LL * 152 && A.nz / (nzb * 2) >= 16) nzb *= 2;
  A.zrows = (A.nz + nzb - 1) / nzb;
  dim3 grid(ntiles, nchunk, (A.nz + A.zrows - 1) / A.zrows);
  const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(ctx->tmap3[ctx->cur][0]);
  sweep3d_tma_kernel<kKpt3><<<grid, NTHREADS, Cfg<kKpt3>::SMEM, ctx->stream>>>(tm[0], tm[1], tm[2], A);
  return cudaGetLastError();
}

cudaError_t tma3_batch_build(const std::vector<ibdvm_ctx *> &cases, int zrows, int *flags, SweepTables &t,
                             cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder3();
  if (!enc) return cudaErrorNotSupported;
  const int n = static_cast<int>(cases.size());
  const int kc = 32 * kKpt3;
  std::vector<Tma3Args> args(2 * n);
  std::vector<CUtensorMap> maps(6 * n);
  std::vector<WorkItem3> items;
  for (int i = 0; i < n; ++i) {
    const ibdvm_ctx *ctx = cases[i];
    const Geom &g = ctx->geom;
    for (int p = 0; p < 2; ++p) {
      const int cur = ctx->cur ^ p;
      Tma3Args &A = args[2 * i + p];
      A = Tma3Args{};
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
      A.nx = g.n[0];
      A.ny = g.n[1];
      A.nz = g.n[2];
      A.nvp = ctx->nvp;
      A.nv = ctx->nv;
      A.zrows = 0;
      A.dt = (float)g.dt;
      A.rdx = (float)(1.0 / g.dx[0]);
      A.rdy = (float)(1.0 / g.dx[1]);
      A.rdz = (float)(1.0 / g.dx[2]);
      cuuint64_t dims[4] = {(cuuint64_t)ctx->nvp, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
      cuuint64_t strides[3] = {(cuuint64_t)ctx->nvp * 4, (cuuint64_t)g.n[0] * ctx->nvp * 4,
                               (cuuint64_t)g.n[1] * g.n[0] * ctx->nvp * 4};
      const cuuint32_t boxes[3][4] = {{(cuuint32_t)kc, TX, TY, 1}, {(cuuint32_t)kc, 2, TY, 1}, {(cuuint32_t)kc, TX, 2, 1}};
      cuuint32_t estr[4] = {1, 1, 1, 1};
      for (int m = 0; m < 3; ++m) {
        CUresult r = enc(&maps[3 * (2 * i + p) + m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->f[cur], dims, strides,
                         boxes[m], estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
      }
    }
    const int nz = g.n[2];
    const int nzb = (zrows <= 0 || zrows >= nz) ? 1 : (nz + zrows - 1) / zrows;
    const int per = (nz + nzb - 1) / nzb;
    for (int y0 = 0; y0 < g.n[1]; y0 += TY)
      for (int x0 = 0; x0 < g.n[0]; x0 += TX)
        for (int k0 = 0; k0 < ctx->nvp; k0 += kc)
          for (int z0 = 0; z0 < nz; z0 += per) {
            WorkItem3 it{};
            it.cas = i;
            it.x0 = x0;
            it.y0 = y0;
            it.k0 = k0;
            it.z0 = z0;
            it.z1 = std::min(nz, z0 + per);
            items.push_back(it);
          }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const WorkItem3 &a, const WorkItem3 &b) { return a.z1 - a.z0 > b.z1 - b.z0; });
  cudaError_t e;
  auto up = [&](const void *h, size_t bytes, void *&d) -> cudaError_t {
    cudaError_t r = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (r != cudaSuccess || bytes == 0) return r;
    return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
  };
  if ((e = up(args.data(), args.size() * sizeof(Tma3Args), t.args)) != cudaSuccess) return e;
  if ((e = up(maps.data(), maps.size() * sizeof(CUtensorMap), t.tmaps)) != cudaSuccess) return e;
  if ((e = up(items.data(), items.size() * sizeof(WorkItem3), t.items)) != cudaSuccess) return e;
  void *nx = nullptr;
  if ((e = cudaMalloc(&nx, sizeof(int))) != cudaSuccess) return e;
  t.next = static_cast<int *>(nx);
  t.nitems = static_cast<int>(items.size());
  t.dim = 3;
  const int smem = (int)Cfg<kKpt3>::SMEM;
  if ((e = cudaFuncSetAttribute(sweep3d_tma_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
      cudaSuccess)
    return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep3d_tma_batch_kernel, NTHREADS, smem)) !=
      cudaSuccess)
    return e;
  t.grid = std::max(1, std::min(t.nitems, nsm * std::max(per_sm, 1)));
  return cudaStreamSynchronize(s); // the host tables go out of scope
}

cudaError_t tma3_batch_launch(const SweepTables &t, int par, cudaStream_t s) {
  if (t.nitems == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.next, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  sweep3d_tma_batch_kernel<<<t.grid, NTHREADS, Cfg<kKpt3>::SMEM, s>>>(
      static_cast<const Tma3Args *>(t.args), static_cast<const CUtensorMap *>(t.tmaps),
      static_cast<const WorkItem3 *>(t.items), t.nitems, t.next, par);
  return cudaGetLastError();
}

} // namespace ibdvm
