// sweep3d_tma.cu -- the transport / relaxation / moments sweep of 3D cases in
// FP32 storage (the mixed path), staged through shared memory by TMA.
//
// Same arithmetic as sweep_kernel in kernels.cu (Sec. 2.2 Eqs. reconstruction
// and limiter, the Shakhov equilibrium of Sec. 2.1 in the non-dimensional
// form of Sec. 4, forward Euler, Eqs. moments1-3 by quadrature), organised for
// GB300 around the octant layout of the velocities:
//
//   * velocities are stored grouped by the signs of their three components,
//     each group padded to a whole number of chunks of KC = 32 VPL velocities,
//     so every velocity of a chunk has the same upwind direction along x, y
//     and z: the upwind halo side, the inflow faces and the march direction
//     are the same for the whole block, and no per-velocity selection remains;
//   * a block owns a 4 x 4 tile of (x, y) columns of cells (16 warps, one per
//     column) and one chunk; lane l owns the velocities 4 l + 128 g + e
//     (g < VPL / 4, e < 4), so stage reads, face exchange and stores are
//     16-byte accesses and the arithmetic runs on pairs of velocities with
//     Blackwell's packed FP32 instructions (__ffma2_rn and friends);
//   * the block marches along z in the direction of the chunk's z velocities,
//     so the z inflow face of a plane is the z outflow face of the previous
//     one (kept in registers with the z stencil);
//   * every plane arrives in shared memory by three TMA tensor copies
//     (cp.async.bulk.tensor.4d) on one mbarrier per stage of a 3-stage ring:
//     the tile's rows extended by two upwind cells and one downwind cell in x
//     (one box), and two upwind rows and one downwind row in y (two boxes);
//   * x and y outflow faces are exchanged through shared memory (two buffers):
//     while a plane is updated the faces of the next plane are published, so
//     one block barrier per plane suffices; the faces of the upwind halo cells
//     (one column in x, one row in y) are spread over the warps;
//   * the moment sums (about the stored bulk velocity) are accumulated per
//     lane, reduced over the warp by a butterfly once per plane and written as
//     FP32 partial sums per chunk; the finalize kernel adds the chunks with a
//     compensated sum and widens them to FP64.
//
// Padding positions of the layout carry zero weight and a huge flux
// coefficient, so their equilibrium vanishes and their f stays zero.
// Conditions that hold for a whole warp (ghost neighbours, the domain edge, a
// cell that is not fluid) select a general path per warp.  Every mbarrier
// wait is bounded: on timeout the block sets an error flag, drains its copies
// (bounded) and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "ctx.h"
#include "tma_sync.cuh"

namespace ibdvm {
namespace {

using namespace dev;

constexpr int TX = 4, TY = 4;          // tile of columns, one warp each
constexpr int NW = TX * TY;            // warps per block
constexpr int NTHREADS = NW * 32;
constexpr int NST = 3;                 // TMA plane stages
constexpr int NM = 14;                 // moment sums (3D)
constexpr int XW = TX + 3;             // an x-extended row of a stage: 2 upwind cells, the tile row, 1 downwind
constexpr int NSLOT = XW * TY + 3 * TX; // cells of a stage: the extended rows and three y halo rows (40)
constexpr float kLn2 = 0.693147180559945309f;
constexpr float kLog2e = 1.442695040888963407f;

template <int VPL> struct Cfg {
  static_assert(VPL == 4 || VPL == 8, "four or eight velocities per lane");
  static constexpr int NG = VPL / 4;            // groups of four consecutive velocities per lane
  static constexpr int KC = 32 * VPL;           // velocities of a chunk
  static constexpr int STAGE = NSLOT * KC;      // floats of a plane stage
  static constexpr int FX = TY * (TX + 2) * KC; // x outflow faces [y][x + 1][k]
  static constexpr int FY = (TY + 2) * TX * KC; // y outflow faces [y + 1][x][k]
  static constexpr int CONST = NG * 4 * 128;    // per group and quantity a float4 per lane
  static constexpr size_t SMEM = (size_t)(NST * STAGE + 2 * FX + 2 * FY + CONST + KC + 2 * NW * kMac) * 4 + NST * 8;
};
static_assert(Cfg<8>::SMEM <= 232448, "shared memory of a block");

struct Oct3Args {
  float *__restrict__ fn;
  const float *__restrict__ f;
  const float *__restrict__ mac;     // [ncell][kMac]
  const float *__restrict__ vconst;  // [nvp][4]: |a_x|, |a_y|, |a_z|, w with |a_a| = dt |xi_a| / dx_a
  const uint8_t *__restrict__ csign; // [nchunk]: bit a when component a of the chunk's velocities is negative
  const float *__restrict__ finf;    // [nvp]
  const uint8_t *__restrict__ cmask;
  const int *__restrict__ dslot;
  const int *__restrict__ dlinks;
  const float *__restrict__ lval;    // [nlink][nvp]
  float *__restrict__ part;          // [nchunk][NM][ncell]
  int *__restrict__ err;
  long long ncell;
  int nx, ny, nz, nvp, zrows;
  int kc;       // velocities of a chunk (256 or 128)
  float sig[3]; // dx_a / dt: |xi_a| = |a_a| sig[a]
  // diffuse domain walls: faces 2a + (s > 0) in wmask, the halo values of
  // their boundary cells [slot][nvp] from the first slot woff[face]; the slot
  // of a boundary cell is its transverse index (y + ny z, x + nx z, x + nx y)
  const float *__restrict__ whalo;
  long long woff[6];
  int wmask;
};

enum : uint8_t { kNotFluid = 64 };

__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                        uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
// 2^x (the hardware base-2 exponential)
__device__ __forceinline__ float ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// downwind face f + vl(f - up, dn - f): the upwind cell's value plus half its
// van Leer slope times the cell width (Eqs. reconstruction and limiter)
__device__ __forceinline__ float2 face2u(float2 f, float2 up, float2 dn) {
  return __fadd2_rn(f, vl_half2(sub2(f, up), sub2(dn, f)));
}
__device__ __forceinline__ float4 face4(float4 f, float4 up, float4 dn) {
  return cat4(face2u(lo2(f), lo2(up), lo2(dn)), face2u(hi2(f), hi2(up), hi2(dn)));
}
// downwind face from the one-sided differences a = f - f_up and b = f_dn - f
__device__ __forceinline__ float4 face4d(float4 f, float4 a, float4 b) {
  return cat4(__fadd2_rn(lo2(f), vl_half2(lo2(a), lo2(b))), __fadd2_rn(hi2(f), vl_half2(hi2(a), hi2(b))));
}
__device__ __forceinline__ float4 sub4(float4 x, float4 y) { return cat4(sub2(lo2(x), lo2(y)), sub2(hi2(x), hi2(y))); }
// moment accumulators of a lane: scalars (packed pairs of accumulators cost
// thirteen more registers, which the block does not have)
using ACC = float;
__device__ __forceinline__ void acc_add(float &a, float2 v) { a += v.x + v.y; }
__device__ __forceinline__ void acc_fma(float &a, float2 u, float2 v) { a = fmaf(u.y, v.y, fmaf(u.x, v.x, a)); }
__device__ __forceinline__ float acc_value(float a) { return a; }
__device__ __forceinline__ float4 mean4(float4 a, float4 b) {
  return make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.5f * (a.w + b.w));
}
__device__ __forceinline__ float2 mean2(float2 a, float2 b) { return make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y)); }
// ghost values of the link across face dir (bit numbering of cmask) of cell c
// for the four velocities from stored position k
__device__ __forceinline__ float4 link4(const Oct3Args &A, long long c, int dir, int k) {
  const int s = A.dslot[c];
  const int l = (s >= 0) ? A.dlinks[s * 6 + dir] : -1;
  return *reinterpret_cast<const float4 *>((l >= 0) ? A.lval + (size_t)l * A.nvp + k : A.finf + k);
}
// the value of the halo cell across domain face i = 2a + (s > 0) of the
// boundary cell with transverse slot t, for the four velocities at offset o of
// the chunk from k0: a diffuse wall's slot of this step, or the freestream
// (both halo layers hold the same values)
__device__ __forceinline__ float4 halo3(const Oct3Args &A, int i, long long t, int k0, int o, const float *sfinf) {
  if ((A.wmask >> i) & 1) return *reinterpret_cast<const float4 *>(A.whalo + (size_t)(A.woff[i] + t) * A.nvp + k0 + o);
  return *reinterpret_cast<const float4 *>(sfinf + o);
}
__device__ __forceinline__ float2 link2(const Oct3Args &A, long long c, int dir, int k) {
  const int s = A.dslot[c];
  const int l = (s >= 0) ? A.dlinks[s * 6 + dir] : -1;
  return *reinterpret_cast<const float2 *>((l >= 0) ? A.lval + (size_t)l * A.nvp + k : A.finf + k);
}

// The march of one block over the tile of columns at (x0, y0), chunk `chunk`
// and planes [za, zb), in the direction of the chunk's z velocities.
// tm[0..2]: tensor maps of the x-extended rows (TX + 3 cells x TY rows), of a
// pair of y halo rows and of a single y halo row (TX cells each).  reinit: the
// block's mbarriers hold an earlier march (all of whose copies have landed)
// and are invalidated first.  Returns false when the block aborted on a
// timed-out wait.
template <int VPL>
__device__ __forceinline__ bool march3o(const Oct3Args &A, const CUtensorMap *tmx, const CUtensorMap *tmp,
                                        const CUtensorMap *tms, int x0, int y0, int chunk, int za, int zb,
                                        unsigned char *smem_raw, bool reinit) {
  using C = Cfg<VPL>;
  constexpr int NG = C::NG, KC = C::KC;
  float *stage = reinterpret_cast<float *>(smem_raw);
  float *fxb = stage + NST * C::STAGE; // two buffers of x faces, then two of y faces
  float *fyb = fxb + 2 * C::FX;
  float *scon = fyb + 2 * C::FY;
  float *sfinf = scon + C::CONST;
  float *smac = sfinf + KC;
  uint64_t *full = reinterpret_cast<uint64_t *>(smac + 2 * NW * kMac);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = warp % TX, tj = warp / TX;
  const int k0 = chunk * KC;
  const unsigned sg = A.csign[chunk];
  const int sx = (sg & 1u) ? -1 : 1, sy = (sg & 2u) ? -1 : 1, d = (sg & 4u) ? -1 : 1; // d: the march direction
  const float2 sigx = dup(sx * A.sig[0]), sigy = dup(sy * A.sig[1]), sigz = dup(d * A.sig[2]);
  const int ox = (sx > 0) ? 2 : 1; // position of tile column 0 in an extended row
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const long long nxy = (long long)nx * ny;
  // stage slot of tile-relative cell (i, j)
  auto slot = [&](int i, int j) -> int {
    if (j >= 0 && j < TY) return j * XW + i + ox;
    const int yr = (sy > 0) ? ((j < 0) ? j + 2 : 2) : ((j < 0) ? 0 : j - TY + 1);
    return XW * TY + yr * TX + i;
  };
  // flag bits of a ghost across the upwind / downwind face along each axis
  const unsigned gux = 1u << (sx < 0), gdx = 1u << (sx > 0);
  const unsigned guy = 4u << (sy < 0), gdy = 4u << (sy > 0);
  const unsigned guz = 16u << (d < 0), gdz = 16u << (d > 0);
  const int dux = 0 + (sx < 0), ddx = 0 + (sx > 0), duy = 2 + (sy < 0), ddy = 2 + (sy > 0);
  const int duz = 4 + (d < 0), ddz = 4 + (d > 0);

  // the own column
  const int x = x0 + ti, y = y0 + tj;
  const bool col_in = x < nx && y < ny;
  const bool inner = col_in && x - 1 >= 0 && x + 1 < nx && y - 1 >= 0 && y + 1 < ny;
  const int so = slot(ti, tj), syu = slot(ti, tj - sy), syd = slot(ti, tj + sy);
  const long long plane0 = x + (long long)nx * y;
  const int fx_own = (tj * (TX + 2) + ti + 1) * KC, fx_in = fx_own - sx * KC;
  const int fy_own = ((tj + 1) * TX + ti) * KC, fy_in = fy_own - sy * TX * KC;

  // the halo duty of this warp: the upwind halo cell h of the tile (x halo
  // column for h < 4, y halo row for h >= 4) and the group hg of its velocities
  const bool hduty = (VPL == 8) || warp < 8;
  const int h = (VPL == 8) ? (warp >> 1) : (warp & 7), hg = (VPL == 8) ? (warp & 1) : 0;
  const bool hxa = h < TX; // a face along x
  const int hi = hxa ? ((sx > 0) ? -1 : TX) : h - TX;
  const int hj = hxa ? h : ((sy > 0) ? -1 : TY);
  const int hs = hxa ? sx : sy;
  const int hc = slot(hi, hj), hup = hxa ? hc - sx : slot(hi, hj - sy), hdn = hxa ? hc + sx : slot(hi, hj + sy);
  const int hx = x0 + hi, hy = y0 + hj;
  const bool h_in = hduty && hx >= 0 && hx < nx && hy >= 0 && hy < ny;
  const bool h_up_in = hxa ? (hx - hs >= 0 && hx - hs < nx) : (hy - hs >= 0 && hy - hs < ny);
  const unsigned hgu = hxa ? gux : guy, hgd = hxa ? gdx : gdy;
  const int hdu = hxa ? dux : duy, hdd = hxa ? ddx : ddy;
  const int hout = hxa ? (hj * (TX + 2) + hi + 1) * KC : 2 * C::FX + ((hj + 1) * TX + hi) * KC; // from fxb
  const long long hplane0 = h_in ? hx + (long long)nx * hy : 0;
  const int ho = 128 * hg + 4 * lane;

  // planes: march index m = 0..M-1 is plane p0 + d m; stage m holds plane
  // p0 + d m (also m = M: the z neighbour of the last plane)
  const int M = zb - za;
  const int p0 = (d > 0) ? za : zb - 1;
  auto plane_in = [&](int m) { const int p = p0 + d * m; return p >= 0 && p < nz; };

  // velocity constants (quantity-major per group) and the free stream of the chunk
  for (int t = threadIdx.x; t < NG * 32; t += NTHREADS) {
    const int g = t >> 5, l = t & 31;
    const float4 *src = reinterpret_cast<const float4 *>(A.vconst) + (k0 + 128 * g + 4 * l);
    const float4 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
    sts4(scon + ((g * 4 + 0) * 32 + l) * 4, make_float4(v0.x, v1.x, v2.x, v3.x));
    sts4(scon + ((g * 4 + 1) * 32 + l) * 4, make_float4(v0.y, v1.y, v2.y, v3.y));
    sts4(scon + ((g * 4 + 2) * 32 + l) * 4, make_float4(v0.z, v1.z, v2.z, v3.z));
    sts4(scon + ((g * 4 + 3) * 32 + l) * 4, make_float4(v0.w, v1.w, v2.w, v3.w));
  }
  for (int i = threadIdx.x; i < KC; i += NTHREADS) sfinf[i] = A.finf[k0 + i];
  __shared__ int s_seg[2]; // first and last special row (march indices)
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      if (reinit) mbar_inval(&full[s]);
      mbar_init(&full[s], 1);
    }
    fence_mbar_init();
    s_seg[0] = INT_MAX;
    s_seg[1] = -1;
  }
  __syncthreads();
  const int ys_pair = (sy > 0) ? y0 - 2 : y0 + TY, ys_single = (sy > 0) ? y0 + TY : y0 - 1;
  const int yr_pair = (sy > 0) ? 0 : 1, yr_single = (sy > 0) ? 2 : 0;
  auto issue = [&](int m, int st) { // stage m into slot st = m mod NST
    float *dst = stage + st * C::STAGE;
    uint64_t *bar = &full[st];
    const int z = p0 + d * m;
    mbar_expect_tx(bar, C::STAGE * 4);
    tma_box(dst, tmx, k0, x0 - ox, y0, z, bar);
    tma_box(dst + (XW * TY + yr_pair * TX) * KC, tmp, k0, x0, ys_pair, z, bar);
    tma_box(dst + (XW * TY + yr_single * TX) * KC, tms, k0, x0, ys_single, z, bar);
  };
  int issued = -1; // the last stage issued (thread 0)
  if (threadIdx.x == 0 && M > 0)
    for (int m = 0; m < NST && m <= M && plane_in(m); ++m) {
      issue(m, m);
      issued = m;
    }

  // halo values beyond the domain faces for this lane's groups: x faces at
  // (y, plane p), y faces at (x, plane p), z faces at (x, y)
  auto hx_face = [&](int xo, int yy, int p, int o) { // xo: the x index beyond the edge
    return halo3(A, xo < 0 ? 0 : 1, yy + (long long)ny * p, k0, o, sfinf);
  };
  auto hy_face = [&](int xx, int yo, int p, int o) {
    return halo3(A, yo < 0 ? 2 : 3, xx + (long long)nx * p, k0, o, sfinf);
  };
  auto own = [&](int p, float4 *v) {
    if (!col_in) {
#pragma unroll
      for (int g = 0; g < NG; ++g) v[g] = lds4(sfinf + 128 * g + 4 * lane);
    } else if (p < 0 || p >= nz) {
#pragma unroll
      for (int g = 0; g < NG; ++g) v[g] = halo3(A, p < 0 ? 4 : 5, plane0, k0, 128 * g + 4 * lane, sfinf);
    } else {
      const float *src = A.f + (size_t)(plane0 + (long long)p * nxy) * A.nvp + k0 + 4 * lane;
#pragma unroll
      for (int g = 0; g < NG; ++g) v[g] = __ldg(reinterpret_cast<const float4 *>(src + 128 * g));
    }
  };
  auto cflag = [&](int p) -> unsigned {
    return (col_in && p >= 0 && p < nz) ? A.cmask[plane0 + (long long)p * nxy] : kNotFluid;
  };
  auto hflag = [&](int p) -> unsigned {
    return (h_in && p >= 0 && p < nz) ? A.cmask[hplane0 + (long long)p * nxy] : kNotFluid;
  };
  // the z stencil of the own column, per group: the difference D = f(p) -
  // f(p - d) of the current plane p and its upwind neighbour, and the z
  // outflow face of plane p - d (the inflow of plane p)
  // (as pairs of velocities: unit u = 2 g + q holds velocities 2 q, 2 q + 1 of group g)
  float2 D[2 * NG], P[2 * NG];
  {
    float4 Rpp[NG], Rp[NG], Rc[NG];
    own(p0 - 2 * d, Rpp);
    own(p0 - d, Rp);
    own(p0, Rc);
    const int r = p0 - d;
    const unsigned mr = cflag(r);
    const long long cr = plane0 + (long long)r * nxy;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int k = k0 + 128 * g + 4 * lane;
      float4 P4;
      if (!col_in) P4 = lds4(sfinf + 128 * g + 4 * lane);
      else if (r < 0 || r >= nz) P4 = Rp[g]; // a halo plane: its value, zero slope
      else if (mr & kNotFluid) P4 = make_float4(0.f, 0.f, 0.f, 0.f);
      else P4 = face4(Rp[g], (mr & guz) ? link4(A, cr, duz, k) : Rpp[g], (mr & gdz) ? link4(A, cr, ddz, k) : Rc[g]);
      const float4 D4 = sub4(Rc[g], Rp[g]);
      P[2 * g] = lo2(P4);
      P[2 * g + 1] = hi2(P4);
      D[2 * g] = lo2(D4);
      D[2 * g + 1] = hi2(D4);
    }
  }
  if (lane < kMac)
    smac[warp * kMac + lane] = col_in ? A.mac[(plane0 + (long long)p0 * nxy) * kMac + lane] : 0.f;

  // x and y outflow faces of plane index m (own cell and the warp's halo
  // cell) from stage m into face buffer b
  auto publish = [&](auto plain, int m, int st, unsigned mcm, unsigned hmm, int b) { // st: slot of stage m
    constexpr bool PL = decltype(plain)::value;
    const int p = p0 + d * m;
    const float *sp = stage + st * C::STAGE;
    const long long cell = plane0 + (long long)p * nxy;
    float *fxo = fxb + b * C::FX + fx_own, *fyo = fyb + b * C::FY + fy_own;
    const float *rc = (PL || col_in) ? sp + so * KC + 4 * lane : sfinf + 4 * lane;
    if (PL || (inner && !(mcm & (kNotFluid | 15u)))) {
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const int o = 128 * g + 4 * lane;
        const float4 fc = lds4(rc + 128 * g);
        sts4(fxo + 128 * g + 4 * lane, face4(fc, lds4(sp + (so - sx) * KC + o), lds4(sp + (so + sx) * KC + o)));
        sts4(fyo + 128 * g + 4 * lane, face4(fc, lds4(sp + syu * KC + o), lds4(sp + syd * KC + o)));
      }
    } else {
      const bool fluid = col_in && !(mcm & kNotFluid);
      const bool xu_in = x - sx >= 0 && x - sx < nx, xd_in = x + sx >= 0 && x + sx < nx;
      const bool yu_in = y - sy >= 0 && y - sy < ny, yd_in = y + sy >= 0 && y + sy < ny;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const int o = 128 * g + 4 * lane, k = k0 + o;
        float4 FX, FY;
        if (!col_in) {
          // a column past the x or y edge: the halo value (zero slope) across
          // that edge; the face along the other axis is never read
          FX = (x >= nx && y < ny) ? hx_face(x, y, p, o) : lds4(sfinf + o);
          FY = (y >= ny && x < nx) ? hy_face(x, y, p, o) : lds4(sfinf + o);
        } else if (!fluid) {
          FX = FY = make_float4(0.f, 0.f, 0.f, 0.f); // never read: neighbours see the link values
        } else {
          const float4 xu = (mcm & gux) ? link4(A, cell, dux, k) : (xu_in ? lds4(sp + (so - sx) * KC + o) : hx_face(x - sx, y, p, o));
          const float4 xd = (mcm & gdx) ? link4(A, cell, ddx, k) : (xd_in ? lds4(sp + (so + sx) * KC + o) : hx_face(x + sx, y, p, o));
          const float4 yu = (mcm & guy) ? link4(A, cell, duy, k) : (yu_in ? lds4(sp + syu * KC + o) : hy_face(x, y - sy, p, o));
          const float4 yd = (mcm & gdy) ? link4(A, cell, ddy, k) : (yd_in ? lds4(sp + syd * KC + o) : hy_face(x, y + sy, p, o));
          const float4 fc = lds4(rc + 128 * g);
          FX = face4(fc, xu, xd);
          FY = face4(fc, yu, yd);
        }
        sts4(fxo + o, FX);
        sts4(fyo + o, FY);
      }
    }
    if (hduty) {
      float4 out;
      if (PL || (h_in && h_up_in && !(hmm & (kNotFluid | hgu | hgd)))) {
        out = face4(lds4(sp + hc * KC + ho), lds4(sp + hup * KC + ho), lds4(sp + hdn * KC + ho));
      } else if (!h_in) {
        // a halo cell beyond the domain edge of its axis: the halo value; one
        // beyond the other axis's edge as well is never read
        if (hxa) out = (hy >= 0 && hy < ny) ? hx_face(hx, hy, p, ho) : lds4(sfinf + ho);
        else out = (hx >= 0 && hx < nx) ? hy_face(hx, hy, p, ho) : lds4(sfinf + ho);
      } else if (hmm & kNotFluid) {
        out = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const long long hcell = hplane0 + (long long)p * nxy;
        const float4 up = (hmm & hgu) ? link4(A, hcell, hdu, k0 + ho)
                          : h_up_in ? lds4(sp + hup * KC + ho)
                          : hxa     ? hx_face(hx - hs, hy, p, ho)
                                    : hy_face(hx, hy - hs, p, ho);
        const float4 dn = (hmm & hgd) ? link4(A, hcell, hdd, k0 + ho) : lds4(sp + hdn * KC + ho);
        out = face4(lds4(sp + hc * KC + ho), up, dn);
      }
      // the halo cell's face goes into buffer b of its axis
      sts4(fxb + b * (hxa ? C::FX : C::FY) + hout + ho, out);
    }
  };

  // Special planes: a cell of the tile's columns that is not fluid or has a
  // ghost neighbour (along its axis for a halo cell); every plane when a
  // column or halo cell lies at an x or y edge of the domain.  Planes from
  // the one before the first special plane to the last run the general copy
  // of the plane body, the others the plain one (no per-plane flags).
  {
    int lo = INT_MAX, hi = -1;
    const bool edge = !inner || (hduty && !(h_in && h_up_in));
    if (edge) {
      lo = 0;
      hi = M - 1;
    } else {
      for (int r = za + lane; r < zb; r += 32) {
        unsigned fl = A.cmask[plane0 + (long long)r * nxy] & (kNotFluid | 63u);
        if (hduty) fl |= A.cmask[hplane0 + (long long)r * nxy] & (kNotFluid | hgu | hgd);
        if (fl) {
          const int mr = (r - p0) * d;
          lo = min(lo, mr);
          hi = max(hi, mr);
        }
      }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0 && hi >= 0) {
      atomicMin(&s_seg[0], lo);
      atomicMax(&s_seg[1], hi);
    }
  }
  __syncthreads();
  const int gs = (s_seg[1] >= 0) ? max(0, s_seg[0] - 1) : M, ge = (s_seg[1] >= 0) ? s_seg[1] + 1 : M;

  bool abort_local = false;
  int waited = -1; // the last stage this thread waited for successfully
  unsigned mc0 = cflag(p0), mc1 = cflag(p0 + d);
  unsigned hm1 = hflag(p0 + d);
  if (M > 0) {
    if (mbar_wait(&full[0], 0)) waited = 0;
    else abort_local = true;
    publish(std::false_type{}, 0, 0, mc0, hflag(p0), 0);
  }
  float *fn_cell = A.fn + (size_t)(plane0 + (long long)p0 * nxy) * A.nvp + k0 + 4 * lane;
  float *part_cell =
      A.part + ((size_t)chunk * NM + ((lane >> 1) < NM ? (lane >> 1) : 0)) * A.ncell + plane0 + (long long)p0 * nxy;
  const long long step_cells = d * nxy;
  bool ok = !__syncthreads_or(abort_local ? 1 : 0);
  // planes [mb, me), in two copies: plain (no flags), and general
  auto planes = [&](auto plain_tag, int mb, int me) {
    constexpr bool PL = decltype(plain_tag)::value;
    if (!PL && mb < me) { // the flags of the segment's first planes
      mc0 = cflag(p0 + d * mb);
      mc1 = cflag(p0 + d * (mb + 1));
      hm1 = hflag(p0 + d * (mb + 1));
    }
  // stage slots of planes m and m + 1, and the parity of the latter
  int st0 = mb % NST, st1 = (mb + 1) % NST;
  unsigned ph1 = ((mb + 1) / NST) & 1;
  for (int m = mb; ok && m < me; ++m) {
    const int p = p0 + d * m, par = m & 1;
    const bool nin = plane_in(m + 1);
    const long long cell = plane0 + (long long)p * nxy;
    // prefetch: flags two planes ahead, the Shakhov parameters of the next plane
    const unsigned mc2 = PL ? 0u : cflag(p + 2 * d), hm2 = PL ? 0u : hflag(p + 2 * d);
    const float macn = (lane < kMac && (PL || col_in) && nin) ? __ldg(A.mac + (cell + d * nxy) * kMac + lane) : 0.f;
    if (nin) {
      if (mbar_wait(&full[st1], ph1)) waited = m + 1;
      else abort_local = true;
    }
    // (1) the faces of the next plane, into the other buffer
    if (m + 1 < M && !abort_local) publish(plain_tag, m + 1, st1, mc1, hm1, par ^ 1);
    // (2) update of the own cell at plane p and its moment sums (13 independent
    // sums: the sum of w c^2 f is the trace of the second moments)
    const float *sp = stage + st0 * C::STAGE;
    float *sp1 = stage + st1 * C::STAGE;
    const float *rc = (PL || col_in) ? sp + so * KC + 4 * lane : sfinf + 4 * lane;
    const float *rn = (PL || col_in) ? sp1 + so * KC + 4 * lane : sfinf + 4 * lane;
    if (!nin && (PL || col_in)) {
      // past the domain edge: the halo value of the own column, written into
      // the unused slot of that plane (each lane reads back only what it wrote)
#pragma unroll
      for (int g = 0; g < NG; ++g)
        sts4(sp1 + so * KC + 128 * g + 4 * lane, halo3(A, d > 0 ? 5 : 4, plane0, k0, 128 * g + 4 * lane, sfinf));
    }
    const float *fxo_b = fxb + par * C::FX, *fyo_b = fyb + par * C::FY;
    const bool fluid = PL ? !abort_local : (col_in && !(mc0 & kNotFluid) && !abort_local);
    ACC acc[13];
#pragma unroll
    for (int i = 0; i < 13; ++i) acc[i] = ACC{};
    if (fluid) {
      const float4 *pm = reinterpret_cast<const float4 *>(smac + (par * NW + warp) * kMac);
      const float4 c0v = pm[0], c1v = pm[1], c2v = pm[2];
      const float2 mUx = dup(-c0v.y), mUy = dup(-c0v.z), mUz = dup(-c0v.w);
      const float2 nl2 = dup(-c1v.x * kLog2e); // -log2(e) / T
      // the Shakhov factor A (1 - Pr) folded into the heat flux
      const float2 q0 = dup(c1v.z * c1v.w), q1 = dup(c1v.z * c2v.x), q2 = dup(c1v.z * c2v.y);
      const float2 dt2 = dup(c2v.z);
      const float2 pre2 = dup(c0v.x);
      // the plane body, in two copies: GEN = a ghost neighbour (links for
      // the faces and the inflow), else the plain stencil
      auto body = [&](auto gen) {
        constexpr bool GEN = decltype(gen)::value;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        float2 out[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          // velocities 2 q, 2 q + 1 of group g: one 8-byte access each
          const int u = 2 * g + q;
          const int o = 128 * g + 4 * lane + 2 * q;
          const float2 ax = lds2(scon + ((g * 4 + 0) * 32 + lane) * 4 + 2 * q);
          const float2 ay = lds2(scon + ((g * 4 + 1) * 32 + lane) * 4 + 2 * q);
          const float2 az = lds2(scon + ((g * 4 + 2) * 32 + lane) * 4 + 2 * q);
          const float2 wk = lds2(scon + ((g * 4 + 3) * 32 + lane) * 4 + 2 * q);
          const float2 f = lds2(rc + 128 * g + 2 * q), fnx = lds2(rn + 128 * g + 2 * q);
          const float2 Dn = sub2(fnx, f);
          const float2 fxo = lds2(fxo_b + fx_own + o), fyo = lds2(fyo_b + fy_own + o);
          float2 fxi = lds2(fxo_b + fx_in + o), fyi = lds2(fyo_b + fy_in + o), fzi = P[u];
          // z outflow face of this plane (the inflow of the next)
          float2 fzo;
          if constexpr (!GEN) {
            fzo = __fadd2_rn(f, vl_half2(D[u], Dn));
          } else {
            const float2 a = (mc0 & guz) ? sub2(f, link2(A, cell, duz, k0 + o)) : D[u];
            const float2 b = (mc0 & gdz) ? sub2(link2(A, cell, ddz, k0 + o), f) : Dn;
            fzo = __fadd2_rn(f, vl_half2(a, b));
            // a ghost upwind neighbour: the mean of its link value and this cell (one-sided slope)
            if (mc0 & gux) fxi = mean2(link2(A, cell, dux, k0 + o), f);
            if (mc0 & guy) fyi = mean2(link2(A, cell, duy, k0 + o), f);
            if (mc0 & guz) fzi = mean2(link2(A, cell, duz, k0 + o), f);
          }
          P[u] = fzo;
          D[u] = Dn; // f(p + d) - f(p): the upwind difference of the next plane
          // Shakhov equilibrium g (1 + A c.q (2 c^2 / T - 5)) from the stored state
          const float2 cx = __ffma2_rn(ax, sigx, mUx), cy = __ffma2_rn(ay, sigy, mUy), cz = __ffma2_rn(az, sigz, mUz);
          const float2 c2 = __ffma2_rn(cx, cx, __ffma2_rn(cy, cy, __fmul2_rn(cz, cz)));
          const float2 tn = __fmul2_rn(c2, nl2); // -c^2 / T log2(e)
          const float2 e = __fmul2_rn(pre2, make_float2(ex2(tn.x), ex2(tn.y)));
          const float2 cq = __ffma2_rn(cx, q0, __ffma2_rn(cy, q1, __fmul2_rn(cz, q2)));
          const float2 poly = __ffma2_rn(tn, dup(-2.f * kLn2), dup(-5.f)); // 2 c^2 / T - 5
          const float2 geq = __ffma2_rn(__fmul2_rn(e, cq), poly, e);
          // forward Euler: relaxation, then the flux differences along x, y, z
          float2 n = __ffma2_rn(dt2, sub2(geq, f), f);
          n = __ffma2_rn(ax, sub2(fxi, fxo), n);
          n = __ffma2_rn(ay, sub2(fyi, fyo), n);
          n = __ffma2_rn(az, sub2(fzi, fzo), n);
          out[q] = n;
          // moment sums about the stored bulk velocity (Eqs. moments1-3)
          const float2 wf = __fmul2_rn(wk, n);
          const float2 cxw = __fmul2_rn(cx, wf), cyw = __fmul2_rn(cy, wf), czw = __fmul2_rn(cz, wf);
          const float2 e2 = __fmul2_rn(c2, wf);
          acc_add(acc[0], wf);
          acc_add(acc[1], cxw);
          acc_add(acc[2], cyw);
          acc_add(acc[3], czw);
          acc_fma(acc[4], cx, cxw);
          acc_fma(acc[5], cy, cxw);
          acc_fma(acc[6], cz, cxw);
          acc_fma(acc[7], cy, cyw);
          acc_fma(acc[8], cz, cyw);
          acc_fma(acc[9], cz, czw);
          acc_fma(acc[10], cx, e2);
          acc_fma(acc[11], cy, e2);
          acc_fma(acc[12], cz, e2);
          // the next unit's loads after this unit: the units run one after the
          // other instead of interleaved (fewer live registers, no spills)
          asm volatile("" ::: "memory");
        }
        *reinterpret_cast<float4 *>(fn_cell + 128 * g) = cat4(out[0], out[1]);
      }
      };
      if (!PL && (mc0 & 63u))
        body(std::true_type{});
      else
        body(std::false_type{});
    } else {
#pragma unroll
      for (int u = 0; u < 2 * NG; ++u) {
        const int ou = 128 * (u >> 1) + 2 * (u & 1);
        P[u] = col_in ? make_float2(0.f, 0.f) : lds2(sfinf + ou + 4 * lane);
        D[u] = col_in ? sub2(lds2(rn + ou), lds2(rc + ou)) : make_float2(0.f, 0.f);
      }
    }
    // (3) butterfly of the 16 (14 used) sums over the 32 lanes, in the order of
    // the finalize kernel: 1, c, c^2, c_a c_b (xx xy xz yy yz zz), c c^2
    {
      float v16[16];
#pragma unroll
      for (int i = 0; i < 4; ++i) v16[i] = acc_value(acc[i]);
#pragma unroll
      for (int i = 4; i < 13; ++i) v16[i + 1] = acc_value(acc[i]);
      v16[4] = v16[5] + v16[8] + v16[10];
      v16[14] = v16[15] = 0.f;
      float v8[8];
      const bool b16 = lane & 16;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float keep = b16 ? v16[8 + i] : v16[i];
        const float send = b16 ? v16[i] : v16[8 + i];
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
      if ((PL || col_in) && (lane & 1) == 0 && (lane >> 1) < NM) *part_cell = v1;
    }
    // (4) advance: the flags and parameters of the next planes
    if (lane < kMac) smac[((par ^ 1) * NW + warp) * kMac + lane] = macn;
    mc0 = mc1;
    mc1 = mc2;
    hm1 = hm2;
    fn_cell += step_cells * A.nvp;
    part_cell += step_cells;
    // faces of the next plane published, this plane's buffer and stage m consumed
    if (__syncthreads_or(abort_local ? 1 : 0)) {
      ok = false;
      break;
    }
    // the stage of plane index m + NST into the slot of stage m
    if (threadIdx.x == 0 && m + NST <= M && plane_in(m + NST)) {
      fence_proxy_async();
      issue(m + NST, st0);
      issued = m + NST;
    }
    st0 = st1;
    if (++st1 == NST) {
      st1 = 0;
      ph1 ^= 1u;
    }
  }
  };
  planes(std::true_type{}, 0, gs);
  planes(std::false_type{}, gs, ge);
  planes(std::true_type{}, ge, M);
  if (!ok && threadIdx.x == 0) {
    atomicOr(A.err, kFlagTimeout);
    for (int q = waited + 1; q <= issued; ++q) mbar_wait(&full[q % NST], (q / NST) & 1);
  }
  return ok;
}

template <int VPL>
__global__ void __launch_bounds__(NTHREADS, 1)
    sweep3d_tma_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmp,
                       const __grid_constant__ CUtensorMap tms, Oct3Args A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ntx = (A.nx + TX - 1) / TX;
  const int za = blockIdx.z * A.zrows;
  march3o<VPL>(A, &tmx, &tmp, &tms, (blockIdx.x % ntx) * TX, (blockIdx.x / ntx) * TY, blockIdx.y, za,
               min(A.nz, za + A.zrows), smem_raw, false);
}

// One item of the batched 3D sweep: a march of one member case.
struct WorkItem3 {
  int cas;     // member index
  int x0, y0;  // tile origin
  int chunk;   // velocity chunk
  int za, zb;  // planes
  int pad[2];
};

// The batched 3D sweep: a persistent grid whose blocks take work items in
// order from a shared counter.  Member c at step parity par uses
// args[2 c + par] and the tensor maps tmaps[3 (2 c + par) + 0..2].  VPL = 0:
// the members have chunks of either width, chosen per item.
template <int VPL>
__global__ void __launch_bounds__(NTHREADS, 1)
    sweep3d_tma_batch_kernel(const Oct3Args *__restrict__ args, const CUtensorMap *__restrict__ tmaps,
                             const WorkItem3 *__restrict__ items, int nitems, int *__restrict__ next, int par) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Oct3Args sA;
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
    bool ok;
    if constexpr (VPL == 0)
      ok = (sA.kc == 256) ? march3o<8>(sA, tm, tm + 1, tm + 2, it.x0, it.y0, it.chunk, it.za, it.zb, smem_raw, reinit)
                          : march3o<4>(sA, tm, tm + 1, tm + 2, it.x0, it.y0, it.chunk, it.za, it.zb, smem_raw, reinit);
    else
      ok = march3o<VPL>(sA, tm, tm + 1, tm + 2, it.x0, it.y0, it.chunk, it.za, it.zb, smem_raw, reinit);
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

// the three tensor maps of a state buffer: x-extended rows, a pair of y rows, a single y row
CUresult encode_maps(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *out, void *f, const Geom &g, int nvp,
                     int kc) {
  cuuint64_t dims[4] = {(cuuint64_t)nvp, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
  cuuint64_t strides[3] = {(cuuint64_t)nvp * 4, (cuuint64_t)g.n[0] * nvp * 4, (cuuint64_t)g.n[1] * g.n[0] * nvp * 4};
  const cuuint32_t boxes[3][4] = {{(cuuint32_t)kc, XW, TY, 1}, {(cuuint32_t)kc, TX, 2, 1}, {(cuuint32_t)kc, TX, 1, 1}};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int m = 0; m < 3; ++m) {
    CUresult r = enc(&out[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, f, dims, strides, boxes[m], estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return r;
  }
  return CUDA_SUCCESS;
}

Oct3Args oct_args(const ibdvm_ctx *ctx, int cur, int *err) {
  Oct3Args A{};
  A.f = static_cast<const float *>(ctx->f[cur]);
  A.fn = static_cast<float *>(ctx->f[1 - cur]);
  A.mac = static_cast<const float *>(ctx->mac);
  A.vconst = ctx->oct_const;
  A.csign = ctx->oct_sign;
  A.finf = static_cast<const float *>(ctx->finf);
  A.cmask = ctx->cmask;
  A.dslot = ctx->dslot;
  A.dlinks = ctx->dlinks;
  A.lval = static_cast<const float *>(ctx->lval);
  A.part = ctx->partf;
  A.err = err;
  A.ncell = ctx->ncell;
  A.nx = ctx->geom.n[0];
  A.ny = ctx->geom.n[1];
  A.nz = ctx->geom.n[2];
  A.nvp = ctx->nvp;
  A.zrows = 0;
  A.kc = ctx->oct_kc;
  for (int a = 0; a < 3; ++a) A.sig[a] = (float)(ctx->geom.dx[a] / ctx->geom.dt);
  A.whalo = static_cast<const float *>(ctx->whalo);
  A.wmask = ctx->wall_mask;
  for (int i = 0; i < 6; ++i) A.woff[i] = ctx->wall_off[i];
  return A;
}

} // namespace

bool tma_encoder_available() { return encoder3() != nullptr; }

bool tma3_sweep_applicable(const ibdvm_ctx *ctx) {
  return ctx->dim == 3 && ctx->precision == IBDVM_MIXED && ctx->oct_kc > 0 && encoder3() != nullptr;
}

int tma3_sweep_nchunk(const ibdvm_ctx *ctx) { return ctx->nvp / ctx->oct_kc; }

cudaError_t tma3_sweep_prepare(ibdvm_ctx *ctx) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder3();
  if (!enc || ctx->oct_kc <= 0) return cudaErrorNotSupported;
  for (int b = 0; b < 2; ++b)
    if (encode_maps(enc, reinterpret_cast<CUtensorMap *>(ctx->tmap3[b][0]), ctx->f[b], ctx->geom, ctx->nvp,
                    ctx->oct_kc) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(sweep3d_tma_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg<8>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sweep3d_tma_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<4>::SMEM);
}

cudaError_t tma3_sweep_launch(ibdvm_ctx *ctx) {
  Oct3Args A = oct_args(ctx, ctx->cur, ctx->d_flags);
  const int ntiles = ((A.nx + TX - 1) / TX) * ((A.ny + TY - 1) / TY);
  const int nchunk = ctx->nvp / ctx->oct_kc;
  // planes split when the grid is too small to fill the GPU
  int nzb = 1;
  while ((long long)ntiles * nchunk * nzb < 2LL * 152 && A.nz / (nzb * 2) >= 16) nzb *= 2;
  A.zrows = (A.nz + nzb - 1) / nzb;
  dim3 grid(ntiles, nchunk, (A.nz + A.zrows - 1) / A.zrows);
  const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(ctx->tmap3[ctx->cur][0]);
  if (ctx->oct_kc == 256)
    sweep3d_tma_kernel<8><<<grid, NTHREADS, Cfg<8>::SMEM, ctx->stream>>>(tm[0], tm[1], tm[2], A);
  else
    sweep3d_tma_kernel<4><<<grid, NTHREADS, Cfg<4>::SMEM, ctx->stream>>>(tm[0], tm[1], tm[2], A);
  return cudaGetLastError();
}

cudaError_t tma3_batch_build(const std::vector<ibdvm_ctx *> &cases, int zrows, int *flags, SweepTables &t,
                             cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder3();
  if (!enc) return cudaErrorNotSupported;
  const int n = static_cast<int>(cases.size());
  std::vector<Oct3Args> args(2 * n);
  std::vector<CUtensorMap> maps(6 * n);
  std::vector<WorkItem3> items;
  bool all8 = true, all4 = true;
  for (int i = 0; i < n; ++i) {
    const ibdvm_ctx *ctx = cases[i];
    if (ctx->oct_kc <= 0) return cudaErrorInvalidValue;
    all8 = all8 && ctx->oct_kc == 256;
    all4 = all4 && ctx->oct_kc == 128;
    const Geom &g = ctx->geom;
    for (int p = 0; p < 2; ++p) {
      const int cur = ctx->cur ^ p;
      args[2 * i + p] = oct_args(ctx, cur, flags + i);
      if (encode_maps(enc, &maps[3 * (2 * i + p)], ctx->f[cur], g, ctx->nvp, ctx->oct_kc) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
    const int nz = g.n[2];
    const int nzb = (zrows <= 0 || zrows >= nz) ? 1 : (nz + zrows - 1) / zrows;
    const int per = (nz + nzb - 1) / nzb;
    for (int y0 = 0; y0 < g.n[1]; y0 += TY)
      for (int x0 = 0; x0 < g.n[0]; x0 += TX)
        for (int c = 0; c < ctx->nvp / ctx->oct_kc; ++c)
          for (int za = 0; za < nz; za += per) {
            WorkItem3 it{};
            it.cas = i;
            it.x0 = x0;
            it.y0 = y0;
            it.chunk = c;
            it.za = za;
            it.zb = std::min(nz, za + per);
            items.push_back(it);
          }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const WorkItem3 &a, const WorkItem3 &b) { return a.zb - a.za > b.zb - b.za; });
  cudaError_t e;
  auto up = [&](const void *h, size_t bytes, void *&d) -> cudaError_t {
    cudaError_t r = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (r != cudaSuccess || bytes == 0) return r;
    return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
  };
  if ((e = up(args.data(), args.size() * sizeof(Oct3Args), t.args)) != cudaSuccess) return e;
  if ((e = up(maps.data(), maps.size() * sizeof(CUtensorMap), t.tmaps)) != cudaSuccess) return e;
  if ((e = up(items.data(), items.size() * sizeof(WorkItem3), t.items)) != cudaSuccess) return e;
  void *nx = nullptr;
  if ((e = cudaMalloc(&nx, sizeof(int))) != cudaSuccess) return e;
  t.next = static_cast<int *>(nx);
  t.nitems = static_cast<int>(items.size());
  t.dim = 3;
  t.ksel = all8 ? 8 : (all4 ? 4 : 0);
  const void *fn = all8 ? (const void *)sweep3d_tma_batch_kernel<8>
                   : all4 ? (const void *)sweep3d_tma_batch_kernel<4> : (const void *)sweep3d_tma_batch_kernel<0>;
  const int smem = all4 ? (int)Cfg<4>::SMEM : (int)Cfg<8>::SMEM;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTHREADS, smem)) != cudaSuccess) return e;
  t.grid = std::max(1, std::min(t.nitems, nsm * std::max(per_sm, 1)));
  return cudaStreamSynchronize(s); // the host tables go out of scope
}

cudaError_t tma3_batch_launch(const SweepTables &t, int par, cudaStream_t s) {
  if (t.nitems == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.next, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const Oct3Args *a = static_cast<const Oct3Args *>(t.args);
  const CUtensorMap *m = static_cast<const CUtensorMap *>(t.tmaps);
  const WorkItem3 *it = static_cast<const WorkItem3 *>(t.items);
  if (t.ksel == 8)
    sweep3d_tma_batch_kernel<8><<<t.grid, NTHREADS, Cfg<8>::SMEM, s>>>(a, m, it, t.nitems, t.next, par);
  else if (t.ksel == 4)
    sweep3d_tma_batch_kernel<4><<<t.grid, NTHREADS, Cfg<4>::SMEM, s>>>(a, m, it, t.nitems, t.next, par);
  else
    sweep3d_tma_batch_kernel<0><<<t.grid, NTHREADS, Cfg<8>::SMEM, s>>>(a, m, it, t.nitems, t.next, par);
  return cudaGetLastError();
}

} // namespace ibdvm
