// sweep_tma.cu -- the transport / relaxation / moments sweep of 2D cases in
// FP32 storage (the mixed path), staged through shared memory by TMA, and the
// work lists of the batched sweeps.
//
// Same arithmetic as sweep_kernel in kernels.cu (Sec. 2.2 Eqs. reconstruction
// and limiter, the reduced Shakhov equilibria of Sec. 4, forward Euler, Eqs.
// moments1-3 by quadrature), organised for GB300 around the quadrant layout
// of the velocities (layout.cpp):
//
//   * velocities are stored grouped by the signs of their two components, each
//     group padded to a whole number of chunks of KC = 32 VPL velocities, so
//     every velocity of a chunk has the same upwind direction along x and y:
//     the upwind halo side, the inflow faces and the march direction are the
//     same for the whole block, and no per-velocity selection remains;
//   * a block owns TX = 8 columns of cells (one warp each) and one chunk; lane
//     l owns the velocity pairs 2 l + 64 g, 2 l + 64 g + 1 (g < VPL / 2), so
//     every access of a warp is 16 bytes per lane, (h, b) of two velocities,
//     over 512 contiguous bytes; the arithmetic runs on packed FP32 pairs,
//     (h, b) for the transport and two velocities for the equilibrium;
//   * the block marches along y in the direction of the chunk's y velocities,
//     so the y inflow face of a row is the y outflow face of the previous one
//     (kept in registers with f one row back);
//   * every row arrives in shared memory by one TMA tensor copy
//     (cp.async.bulk.tensor.4d over 16-byte velocity pairs) of the TX columns
//     extended by two upwind cells and one downwind cell, on one mbarrier per
//     stage of a 4-stage ring;
//   * x outflow faces are exchanged through two shared buffers: while a row is
//     updated the faces of the next row are published, so one block barrier per
//     row suffices; the faces of the upwind halo column are spread over the
//     first VPL / 2 warps;
//   * the nine moment sums (about the stored bulk velocity) are accumulated per
//     lane, reduced over the warp by a butterfly once per row and written as
//     FP32 partial sums per chunk; the finalize kernel adds the chunks with a
//     compensated sum and widens them to FP64.
//
// Values beyond the domain edge come from the freestream or, for a diffuse
// domain wall (Sec. 2.3 on the domain faces, reading C24), from the wall's
// halo slot of that boundary cell; only the general paths read them.
// Conditions that hold for a whole warp (ghost neighbours, the domain edge, a
// cell that is not fluid) select a general path per warp.  Every mbarrier
// wait is bounded: on timeout the block sets an error flag, drains its copies
// (bounded) and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "ctx.h"
#include "tma_sync.cuh"

namespace ibdvm {
namespace {

using namespace dev;

constexpr int TX = 8;        // columns per block, one warp each
constexpr int NTHREADS = TX * 32;
constexpr int NST = 4;       // TMA row stages
constexpr int NM = 9;        // moment sums (2D)
constexpr int XW = TX + 3;   // cells of a staged row: two upwind, the TX columns, one downwind
constexpr float kLn2 = 0.693147180559945309f;
constexpr float kLog2e = 1.442695040888963407f;

template <int VPL> struct Cfg {
  static_assert(VPL == 2 || VPL == 4 || VPL == 6, "two, four or six velocities per lane");
  static constexpr int G = VPL / 2;            // groups of two velocities (a float4 of (h, b) pairs) per lane
  static constexpr int KC = 32 * VPL;          // velocities of a chunk
  static constexpr int KC2 = 2 * KC;           // floats of one cell of a chunk
  static constexpr int STAGE = XW * KC2;       // floats of a staged row
  static constexpr int FX = (TX + 2) * KC2;    // x outflow faces [x + 1][k][comp], one buffer
  static constexpr int CONST = G * 3 * 64;     // per group and quantity a float2 per lane
  static constexpr size_t SMEM = (size_t)(NST * STAGE + 2 * FX + CONST + KC2 + 2 * TX * kMac) * 4 + NST * 8;
};
static_assert(Cfg<6>::SMEM <= 113 * 1024, "two blocks per SM");

struct Oct2Args {
  float *__restrict__ fn;
  const float *__restrict__ f;
  const float *__restrict__ mac;     // [ncell][kMac]
  const float *__restrict__ vconst;  // [nvp][4]: |a_x|, |a_y|, w, 0 with |a_a| = dt |xi_a| / dx_a
  const uint8_t *__restrict__ csign; // [nchunk]: bit a when component a of the chunk's velocities is negative
  const float *__restrict__ finf;    // [nvp][2]
  const uint8_t *__restrict__ cmask;
  const int *__restrict__ dslot;
  const int *__restrict__ dlinks;
  const float *__restrict__ lval;    // [nlink][nvp][2]
  float *__restrict__ part;          // [nchunk][NM][ncell]
  int *__restrict__ err;
  long long ncell;
  int nx, ny, nvp, rows;
  int kc;        // velocities of a chunk (192, 128 or 64)
  float sig[2];  // dx_a / dt: |xi_a| = |a_a| sig[a]
  // diffuse domain walls: faces 2a + (s > 0) in wmask, the halo values of
  // their boundary cells [slot][nvp][2] from the first slot woff[face]
  const float *__restrict__ whalo;
  long long woff[4];
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
// downwind face f + vl(f - up, dn - f) of (h, b) pairs (Eqs. reconstruction and limiter)
__device__ __forceinline__ float2 face2u(float2 f, float2 up, float2 dn) {
  return __fadd2_rn(f, vl_half2(sub2(f, up), sub2(dn, f)));
}
__device__ __forceinline__ float4 face4(float4 f, float4 up, float4 dn) {
  return cat4(face2u(lo2(f), lo2(up), lo2(dn)), face2u(hi2(f), hi2(up), hi2(dn)));
}
__device__ __forceinline__ float4 mean4(float4 a, float4 b) {
  return make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.5f * (a.w + b.w));
}
// ghost values of the link across face dir (bit numbering of cmask) of cell c
// for the two velocities from stored position k
__device__ __forceinline__ float4 link4(const Oct2Args &A, long long c, int dir, int k) {
  const int s = A.dslot[c];
  const int l = (s >= 0) ? A.dlinks[s * 6 + dir] : -1;
  return *reinterpret_cast<const float4 *>((l >= 0) ? A.lval + ((size_t)l * A.nvp + k) * 2 : A.finf + (size_t)k * 2);
}
__device__ __forceinline__ float2 link2(const Oct2Args &A, long long c, int dir, int k) {
  const int s = A.dslot[c];
  const int l = (s >= 0) ? A.dlinks[s * 6 + dir] : -1;
  return *reinterpret_cast<const float2 *>((l >= 0) ? A.lval + ((size_t)l * A.nvp + k) * 2 : A.finf + (size_t)k * 2);
}
// downwind face from the one-sided differences a = f - f_up and b = f_dn - f
__device__ __forceinline__ float4 face4d(float4 f, float4 a, float4 b) {
  return cat4(__fadd2_rn(lo2(f), vl_half2(lo2(a), lo2(b))), __fadd2_rn(hi2(f), vl_half2(hi2(a), hi2(b))));
}
__device__ __forceinline__ float4 sub4(float4 x, float4 y) { return cat4(sub2(lo2(x), lo2(y)), sub2(hi2(x), hi2(y))); }
__device__ __forceinline__ void sts2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
// moment accumulators: scalars
__device__ __forceinline__ void acc_add(float &a, float2 v) { a += v.x + v.y; }
__device__ __forceinline__ void acc_fma(float &a, float2 u, float2 v) { a = fmaf(u.y, v.y, fmaf(u.x, v.x, a)); }

// The march of one block over columns [x0, x0 + TX), chunk `chunk` and rows
// [ya, yb), in the direction of the chunk's y velocities.  reinit: the
// block's mbarriers hold an earlier march (all of whose copies have landed)
// and are invalidated first.  Returns false when the block aborted on a
// timed-out wait.
template <int VPL>
__device__ __forceinline__ bool march2o(const Oct2Args &A, const CUtensorMap *tm, int x0, int chunk, int ya, int yb,
                                        unsigned char *smem_raw, bool reinit) {
  using C = Cfg<VPL>;
  constexpr int G = C::G, KC = C::KC, KC2 = C::KC2;
  float *stage = reinterpret_cast<float *>(smem_raw);
  float *fxb = stage + NST * C::STAGE; // two buffers of x faces
  float *scon = fxb + 2 * C::FX;
  float *sfinf = scon + C::CONST;
  float *smac = sfinf + KC2;
  uint64_t *full = reinterpret_cast<uint64_t *>(smac + 2 * TX * kMac);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = chunk * KC;
  const unsigned sg = A.csign[chunk];
  const int sx = (sg & 1u) ? -1 : 1, d = (sg & 2u) ? -1 : 1; // d: the march direction
  const float2 sigx = dup(sx * A.sig[0]), sigy = dup(d * A.sig[1]);
  const int ox = (sx > 0) ? 2 : 1; // position of column x0 in a staged row
  const int nx = A.nx, ny = A.ny;
  // flag bits of a ghost across the upwind / downwind face along each axis
  const unsigned gux = 1u << (sx < 0), gdx = 1u << (sx > 0);
  const unsigned guy = 4u << (d < 0), gdy = 4u << (d > 0);
  const int dux = (sx < 0), ddx = (sx > 0), duy = 2 + (d < 0), ddy = 2 + (d > 0);
  // halo faces of the domain edges (i = 2a + (s > 0)) beyond the upwind and
  // downwind neighbours along x and along y
  const int hxu = (sx > 0) ? 0 : 1, hxd = 1 - hxu, hyu = (d > 0) ? 2 : 3, hyd = 5 - hyu;

  // the own column
  const int x = x0 + warp;
  const bool col_in = x < nx;
  const bool inner = col_in && x - 1 >= 0 && x + 1 < nx;
  const int so = warp + ox;
  const int fx_own = (warp + 1) * KC2, fx_in = fx_own - sx * KC2;
  // the halo duty: thread j < KC takes velocity j of the upwind halo column's
  // face (the first VPL warps, one (h, b) pair each)
  const bool hduty = threadIdx.x < KC;
  const int hj = threadIdx.x;
  const int hi = (sx > 0) ? -1 : TX;
  const int hc = hi + ox, hup = hc - sx, hdn = hc + sx;
  const int hx = x0 + hi;
  const bool h_in = hduty && hx >= 0 && hx < nx;
  const bool h_up_in = hx - sx >= 0 && hx - sx < nx;
  const int hout = (hi + 1) * KC2;
  const int ho = 2 * hj;

  // the value of the halo cell across face i of the boundary cell at
  // transverse index t, this lane's group at offset o: a diffuse wall's slot
  // of this step, or the freestream (both halo layers hold the same values)
  auto halo4 = [&](int i, int t, int o) -> float4 {
    if ((A.wmask >> i) & 1) return *reinterpret_cast<const float4 *>(A.whalo + ((size_t)(A.woff[i] + t) * A.nvp + k0) * 2 + o);
    return lds4(sfinf + o);
  };
  auto halo2 = [&](int i, int t, int o) -> float2 {
    if ((A.wmask >> i) & 1) return *reinterpret_cast<const float2 *>(A.whalo + ((size_t)(A.woff[i] + t) * A.nvp + k0) * 2 + o);
    return lds2(sfinf + o);
  };

  // rows: march index m = 0..M-1 is row p0 + d m; stage m holds row p0 + d m
  // (also m = M: the y neighbour of the last row)
  const int M = yb - ya;
  const int p0 = (d > 0) ? ya : yb - 1;
  auto row_in = [&](int m) { const int p = p0 + d * m; return p >= 0 && p < ny; };

  // velocity constants (quantity-major per group) and the free stream of the chunk
  for (int t = threadIdx.x; t < G * 32; t += NTHREADS) {
    const int g = t >> 5, l = t & 31;
    const float4 *src = reinterpret_cast<const float4 *>(A.vconst) + (k0 + 64 * g + 2 * l);
    const float4 v0 = src[0], v1 = src[1];
    *reinterpret_cast<float2 *>(scon + ((g * 3 + 0) * 32 + l) * 2) = make_float2(v0.x, v1.x);
    *reinterpret_cast<float2 *>(scon + ((g * 3 + 1) * 32 + l) * 2) = make_float2(v0.y, v1.y);
    *reinterpret_cast<float2 *>(scon + ((g * 3 + 2) * 32 + l) * 2) = make_float2(v0.z, v1.z);
  }
  for (int i = threadIdx.x; i < KC2; i += NTHREADS) sfinf[i] = A.finf[2 * k0 + i];
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
  auto issue = [&](int m) {
    mbar_expect_tx(&full[m % NST], C::STAGE * 4);
    tma_box(stage + (m % NST) * C::STAGE, tm, 0, k0 / 2, x0 - ox, p0 + d * m, &full[m % NST]);
  };
  int issued = -1; // the last stage issued (thread 0)
  if (threadIdx.x == 0 && reinit) fence_proxy_async(); // the stages were read (and written) by threads
  if (threadIdx.x == 0 && M > 0)
    for (int m = 0; m < NST && m <= M && row_in(m); ++m) {
      issue(m);
      issued = m;
    }

  auto own = [&](int p, float4 *v) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int o = 128 * g + 4 * lane;
      if (!col_in) v[g] = lds4(sfinf + o);
      else if (p < 0 || p >= ny) v[g] = halo4(p < 0 ? 2 : 3, x, o);
      else v[g] = __ldg(reinterpret_cast<const float4 *>(A.f + ((size_t)(x + (long long)nx * p) * A.nvp + k0) * 2 + o));
    }
  };
  auto cflag = [&](int p) -> unsigned {
    return (col_in && p >= 0 && p < ny) ? A.cmask[x + (long long)nx * p] : kNotFluid;
  };
  auto hflag = [&](int p) -> unsigned {
    return (h_in && p >= 0 && p < ny) ? A.cmask[hx + (long long)nx * p] : kNotFluid;
  };
  // the y stencil of the own column, per group: the difference D = f(p) -
  // f(p - d) of the current row p and its upwind neighbour, and the y outflow
  // face of row p - d (the inflow of row p)
  float4 D[G], P[G];
  {
    float4 Rpp[G], Rp[G], Rc[G];
    own(p0 - 2 * d, Rpp);
    own(p0 - d, Rp);
    own(p0, Rc);
    const int r = p0 - d;
    const unsigned mr = cflag(r);
    const long long cr = x + (long long)nx * r;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int o = 128 * g + 4 * lane, k = k0 + 64 * g + 2 * lane;
      if (!col_in) P[g] = lds4(sfinf + o);
      else if (r < 0 || r >= ny) P[g] = Rp[g]; // a halo row: its value, zero slope
      else if (mr & kNotFluid) P[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      else P[g] = face4(Rp[g], (mr & guy) ? link4(A, cr, duy, k) : Rpp[g], (mr & gdy) ? link4(A, cr, ddy, k) : Rc[g]);
      D[g] = sub4(Rc[g], Rp[g]);
    }
  }
  if (lane < kMac) smac[warp * kMac + lane] = col_in ? A.mac[(x + (long long)nx * p0) * kMac + lane] : 0.f;

  // x outflow faces of row index m (own cell and the halo duty) from stage m
  // into face buffer b; PL (plain): no cell of the march is special
  auto publish = [&](auto plain, int m, unsigned mcm, unsigned hmm, int b) {
    constexpr bool PL = decltype(plain)::value;
    const int p = p0 + d * m;
    const float *sp = stage + (m % NST) * C::STAGE;
    float *fb = fxb + b * C::FX;
    if (PL || (inner && !(mcm & (kNotFluid | 3u)))) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int o = 128 * g + 4 * lane;
        sts4(fb + fx_own + o, face4(lds4(sp + so * KC2 + o), lds4(sp + (so - sx) * KC2 + o), lds4(sp + (so + sx) * KC2 + o)));
      }
    } else {
      const bool fluid = col_in && !(mcm & kNotFluid);
      const long long cell = x + (long long)nx * p;
      const bool xu_in = x - sx >= 0 && x - sx < nx, xd_in = x + sx >= 0 && x + sx < nx;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int o = 128 * g + 4 * lane, k = k0 + 64 * g + 2 * lane;
        float4 FX;
        if (!col_in) {
          FX = halo4(1, p, o); // a column past the right edge: the halo value, zero slope
        } else if (!fluid) {
          FX = make_float4(0.f, 0.f, 0.f, 0.f); // never read: neighbours see the link values
        } else {
          const float4 xu = (mcm & gux) ? link4(A, cell, dux, k) : (xu_in ? lds4(sp + (so - sx) * KC2 + o) : halo4(hxu, p, o));
          const float4 xd = (mcm & gdx) ? link4(A, cell, ddx, k) : (xd_in ? lds4(sp + (so + sx) * KC2 + o) : halo4(hxd, p, o));
          FX = face4(lds4(sp + so * KC2 + o), xu, xd);
        }
        sts4(fb + fx_own + o, FX);
      }
    }
    if (hduty) {
      float2 out;
      if (PL || (h_in && h_up_in && !(hmm & (kNotFluid | 3u)))) {
        out = face2u(lds2(sp + hc * KC2 + ho), lds2(sp + hup * KC2 + ho), lds2(sp + hdn * KC2 + ho));
      } else if (!h_in) {
        out = halo2(hxu, p, ho); // the halo column beyond the domain edge: its value
      } else if (hmm & kNotFluid) {
        out = make_float2(0.f, 0.f);
      } else {
        const long long hcell = hx + (long long)nx * p;
        const int k = k0 + hj;
        const float2 up = (hmm & gux) ? link2(A, hcell, dux, k) : (h_up_in ? lds2(sp + hup * KC2 + ho) : halo2(hxu, p, ho));
        const float2 dn = (hmm & gdx) ? link2(A, hcell, ddx, k) : lds2(sp + hdn * KC2 + ho);
        out = face2u(lds2(sp + hc * KC2 + ho), up, dn);
      }
      sts2(fb + hout + ho, out);
    }
  };

  // Special rows: a cell of the block's columns that is not fluid or has a
  // ghost neighbour (along x for the upwind halo column); every row when a
  // column lies at an x edge of the domain.  Rows from the one before the
  // first special row to the last run the general copy of the row body, the
  // others the plain one (no per-row flags).
  {
    int lo = INT_MAX, hi = -1;
    bool edge = !inner;
    if (warp == 0) edge = edge || !(hx >= 0 && hx < nx && h_up_in);
    if (edge) {
      lo = 0;
      hi = M - 1;
    } else {
      for (int r = ya + lane; r < yb; r += 32) {
        unsigned fl = A.cmask[x + (long long)nx * r] & (kNotFluid | 15u);
        if (warp == 0) fl |= A.cmask[hx + (long long)nx * r] & (kNotFluid | 3u);
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
    publish(std::false_type{}, 0, mc0, hflag(p0), 0);
  }
  float *fn_cell = A.fn + ((size_t)(x + (long long)nx * p0) * A.nvp + k0) * 2 + 4 * lane;
  // lanes 4 i write sum i (i < 8); lane 1 writes the ninth sum
  const int sidx = ((lane & 3) == 0) ? (lane >> 2) : 8;
  float *part_cell = A.part + ((size_t)chunk * NM + sidx) * A.ncell + x + (long long)nx * p0;
  const long long step_cells = (long long)d * nx;
  bool ok = !__syncthreads_or(abort_local ? 1 : 0);
  // rows [mb, me), in two copies: plain (no flags), and general
  auto rows = [&](auto plain_tag, int mb, int me) {
    constexpr bool PL = decltype(plain_tag)::value;
    if (!PL && mb < me) { // the flags of the segment's first rows
      mc0 = cflag(p0 + d * mb);
      mc1 = cflag(p0 + d * (mb + 1));
      hm1 = hflag(p0 + d * (mb + 1));
    }
    for (int m = mb; ok && m < me; ++m) {
      const int p = p0 + d * m, par = m & 1;
      const bool nin = row_in(m + 1);
      const long long cell = x + (long long)nx * p;
      // prefetch: flags two rows ahead, the Shakhov parameters of the next row
      const unsigned mc2 = PL ? 0u : cflag(p + 2 * d), hm2 = PL ? 0u : hflag(p + 2 * d);
      const float macn = (lane < kMac && (PL || col_in) && nin) ? __ldg(A.mac + (cell + step_cells) * kMac + lane) : 0.f;
      if (nin) {
        if (mbar_wait(&full[(m + 1) % NST], ((m + 1) / NST) & 1)) waited = m + 1;
        else abort_local = true;
      }
      // (1) the x faces of the next row, into the other buffer
      if (m + 1 < M && !abort_local) publish(plain_tag, m + 1, mc1, hm1, par ^ 1);
      // (2) update of the own cell at row p and its moment sums
      const float *sp = stage + (m % NST) * C::STAGE;
      float *sp1 = stage + ((m + 1) % NST) * C::STAGE;
      if (!nin && (PL || col_in)) {
        // past the domain edge: the halo value of the own column, written into
        // the unused slot of that row (each lane reads back only what it wrote)
  #pragma unroll
        for (int g = 0; g < G; ++g) sts4(sp1 + so * KC2 + 128 * g + 4 * lane, halo4(hyd, x, 128 * g + 4 * lane));
      }
      const float *fb = fxb + par * C::FX;
      const bool fluid = PL ? !abort_local : (col_in && !(mc0 & kNotFluid) && !abort_local);
      float acc[NM];
  #pragma unroll
      for (int i = 0; i < NM; ++i) acc[i] = 0.f;
      if (fluid) {
        const float4 *pm = reinterpret_cast<const float4 *>(smac + (par * TX + warp) * kMac);
        const float4 c0v = pm[0], c1v = pm[1], c2v = pm[2];
        const float2 mU0 = dup(-c0v.y), mU1 = dup(-c0v.z);
        const float2 nl2 = dup(-c1v.x * kLog2e);                        // -log2(e) / T
        const float Tc = 2.f * c1v.y;                                    // T
        const float2 pH = dup(-2.f * kLn2), pB = dup(-Tc * kLn2), mT = dup(-Tc);
        const float2 hT = dup(c1v.y);                                    // T / 2
        const float2 q0 = dup(c1v.z * c1v.w), q1 = dup(c1v.z * c2v.x);   // the Shakhov factor folded into q
        const float2 dt2 = dup(c2v.z), pre2 = dup(c0v.x);
        // the row body, in two copies: GEN = a ghost neighbour (links for the
        // faces and the inflow), else the plain stencil
        auto body = [&](auto gen) {
          constexpr bool GEN = decltype(gen)::value;
  #pragma unroll
        for (int g = 0; g < G; ++g) {
          const int o = 128 * g + 4 * lane, k = k0 + 64 * g + 2 * lane;
          const float2 ax = lds2(scon + ((g * 3 + 0) * 32 + lane) * 2);
          const float2 ay = lds2(scon + ((g * 3 + 1) * 32 + lane) * 2);
          const float2 wk = lds2(scon + ((g * 3 + 2) * 32 + lane) * 2);
          const float4 fc = lds4(sp + so * KC2 + o);
          const float4 fnx = lds4(sp1 + so * KC2 + o);
          const float4 Dn = sub4(fnx, fc);
          const float4 fxo = lds4(fb + fx_own + o);
          float4 fxi = lds4(fb + fx_in + o), fyi = P[g];
          // y outflow face of this row (the inflow of the next)
          float4 fyo;
          if constexpr (!GEN) {
            (void)k;
            fyo = face4d(fc, D[g], Dn);
          } else {
            fyo = face4d(fc, (mc0 & guy) ? sub4(fc, link4(A, cell, duy, k)) : D[g],
                         (mc0 & gdy) ? sub4(link4(A, cell, ddy, k), fc) : Dn);
            // a ghost upwind neighbour: the mean of its link value and this cell (one-sided slope)
            if (mc0 & gux) fxi = mean4(link4(A, cell, dux, k), fc);
            if (mc0 & guy) fyi = mean4(link4(A, cell, duy, k), fc);
          }
          P[g] = fyo;
          D[g] = Dn; // f(p + d) - f(p): the upwind difference of the next row
          // reduced Shakhov equilibria of the two velocities (Sec. 4):
          // H = e (1 + A c.q (2t - 4)), B = T/2 e (1 + A c.q (2t - 2)), t = c^2 / T
          const float2 cx = __ffma2_rn(ax, sigx, mU0), cy = __ffma2_rn(ay, sigy, mU1);
          const float2 c2 = __ffma2_rn(cx, cx, __fmul2_rn(cy, cy));
          const float2 tn = __fmul2_rn(c2, nl2); // -t log2(e)
          const float2 e = __fmul2_rn(pre2, make_float2(ex2(tn.x), ex2(tn.y)));
          const float2 mm = __fmul2_rn(e, __ffma2_rn(cx, q0, __fmul2_rn(cy, q1)));
          const float2 H = __ffma2_rn(mm, __ffma2_rn(tn, pH, dup(-4.f)), e);
          const float2 B = __ffma2_rn(mm, __ffma2_rn(tn, pB, mT), __fmul2_rn(hT, e));
          // forward Euler per velocity on (h, b): relaxation, then the flux differences
          float2 n0 = __ffma2_rn(dt2, sub2(make_float2(H.x, B.x), lo2(fc)), lo2(fc));
          float2 n1 = __ffma2_rn(dt2, sub2(make_float2(H.y, B.y), hi2(fc)), hi2(fc));
          n0 = __ffma2_rn(dup(ax.x), sub2(lo2(fxi), lo2(fxo)), n0);
          n1 = __ffma2_rn(dup(ax.y), sub2(hi2(fxi), hi2(fxo)), n1);
          n0 = __ffma2_rn(dup(ay.x), sub2(lo2(fyi), lo2(fyo)), n0);
          n1 = __ffma2_rn(dup(ay.y), sub2(hi2(fyi), hi2(fyo)), n1);
          *reinterpret_cast<float4 *>(fn_cell + 128 * g) = cat4(n0, n1);
          // moment sums about the stored bulk velocity (Eqs. moments1-3, reduced)
          const float2 wh = __fmul2_rn(wk, make_float2(n0.x, n1.x));
          const float2 e2 = __ffma2_rn(c2, wh, __fmul2_rn(wk, make_float2(n0.y, n1.y))); // w (c^2 h + b)
          const float2 cxwh = __fmul2_rn(cx, wh);
          acc_add(acc[0], wh);
          acc_fma(acc[1], cx, wh);
          acc_fma(acc[2], cy, wh);
          acc_add(acc[3], e2);
          acc_fma(acc[4], cx, cxwh);
          acc_fma(acc[5], cy, cxwh);
          acc_fma(acc[6], cy, __fmul2_rn(cy, wh));
          acc_fma(acc[7], cx, e2);
          acc_fma(acc[8], cy, e2);
        }
        };
        if (!PL && (mc0 & 15u))
          body(std::true_type{});
        else
          body(std::false_type{});
      } else {
  #pragma unroll
        for (int g = 0; g < G; ++g) {
          const int o = 128 * g + 4 * lane;
          P[g] = col_in ? make_float4(0.f, 0.f, 0.f, 0.f) : lds4(sfinf + o);
          D[g] = col_in ? sub4(lds4(sp1 + so * KC2 + o), lds4(sp + so * KC2 + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      // (3) butterfly reduction of the sums over the 32 lanes: three rounds halve
      //     the eight values a lane holds, two more finish the one it keeps; the
      //     ninth sum is a plain xor tree
      {
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
        if (PL || col_in) {
          if ((lane & 3) == 0) *part_cell = v1;
          if (lane == 1) *part_cell = s8;
        }
      }
      // (4) advance: the flags and parameters of the next rows
      if (lane < kMac) smac[((par ^ 1) * TX + warp) * kMac + lane] = macn;
      mc0 = mc1;
      mc1 = mc2;
      hm1 = hm2;
      fn_cell += step_cells * A.nvp * 2;
      part_cell += step_cells;
      // faces of the next row published, this row's buffer and stage m consumed
      if (__syncthreads_or(abort_local ? 1 : 0)) {
        ok = false;
        break;
      }
      // the stage of row index m + NST into the slot of stage m
      if (threadIdx.x == 0 && m + NST <= M && row_in(m + NST)) {
        fence_proxy_async();
        issue(m + NST);
        issued = m + NST;
      }
    }
  };
  rows(std::true_type{}, 0, gs);
  rows(std::false_type{}, gs, ge);
  rows(std::true_type{}, ge, M);
  if (!ok && threadIdx.x == 0) {
    atomicOr(A.err, kFlagTimeout);
    for (int q = waited + 1; q <= issued; ++q) mbar_wait(&full[q % NST], (q / NST) & 1);
  }
  return ok;
}

template <int VPL>
__global__ void __launch_bounds__(NTHREADS, 2) sweep2d_tma_kernel(const __grid_constant__ CUtensorMap tmf,
                                                                  Oct2Args A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ya = blockIdx.z * A.rows;
  march2o<VPL>(A, &tmf, blockIdx.x * TX, blockIdx.y, ya, min(A.ny, ya + A.rows), smem_raw, false);
}

// One item of the batched sweep: a march of one member case.
struct WorkItem {
  int cas;    // member index
  int x0;     // first column
  int chunk;  // velocity chunk
  int ya, yb; // rows
  int vpl;    // velocities per lane of the member's layout
  int pad[2];
};

// The batched sweep: a persistent grid whose blocks take work items in order
// from a shared counter (items sorted by decreasing size), all of VPL
// velocities per lane.  Member c at step parity par uses args[2 c + par] and
// tmaps[2 c + par].
template <int VPL>
__global__ void __launch_bounds__(NTHREADS, 2)
    sweep2d_tma_batch_kernel(const Oct2Args *__restrict__ args, const CUtensorMap *__restrict__ tmaps,
                             const WorkItem *__restrict__ items, int nitems, int *__restrict__ next, int par) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Oct2Args sA;
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
    const bool ok = march2o<VPL>(sA, tm, it.x0, it.chunk, it.ya, it.yb, smem_raw, reinit);
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

// the tensor map of a state buffer: 16-byte velocity pairs (h, b of two
// velocities) x pairs x cells x rows; one box is a staged row of a chunk
CUresult encode_map(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *out, void *f, const Geom &g, int nvp, int kc) {
  cuuint64_t dims[4] = {4, (cuuint64_t)nvp / 2, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1]};
  cuuint64_t strides[3] = {16, (cuuint64_t)nvp * 8, (cuuint64_t)g.n[0] * nvp * 8};
  cuuint32_t box[4] = {4, (cuuint32_t)kc / 2, XW, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

Oct2Args oct2_args(const ibdvm_ctx *ctx, int cur, int *err) {
  Oct2Args A{};
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
  A.nvp = ctx->nvp;
  A.rows = 0;
  A.kc = ctx->oct_kc;
  for (int a = 0; a < 2; ++a) A.sig[a] = (float)(ctx->geom.dx[a] / ctx->geom.dt);
  A.whalo = static_cast<const float *>(ctx->whalo);
  A.wmask = ctx->wall_mask;
  for (int i = 0; i < 4; ++i) A.woff[i] = ctx->wall_off[i];
  return A;
}

template <int VPL> cudaError_t set_smem() {
  return cudaFuncSetAttribute(sweep2d_tma_kernel<VPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<VPL>::SMEM);
}

} // namespace

// The TMA sweep applies to 2D cases in FP32 storage with the quadrant layout.
bool tma_sweep_applicable(const ibdvm_ctx *ctx) {
  return ctx->dim == 2 && ctx->precision == IBDVM_MIXED && ctx->oct_kc > 0 && encoder() != nullptr;
}

int tma_sweep_nchunk(const ibdvm_ctx *ctx) { return ctx->nvp / ctx->oct_kc; }

cudaError_t tma_sweep_prepare(ibdvm_ctx *ctx) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc || ctx->oct_kc <= 0) return cudaErrorNotSupported;
  for (int b = 0; b < 2; ++b)
    if (encode_map(enc, reinterpret_cast<CUtensorMap *>(ctx->tmap[b]), ctx->f[b], ctx->geom, ctx->nvp,
                   ctx->oct_kc) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  switch (ctx->oct_kc) {
  case 192: return set_smem<6>();
  case 128: return set_smem<4>();
  default: return set_smem<2>();
  }
}

cudaError_t tma_sweep_launch(ibdvm_ctx *ctx) {
  Oct2Args A = oct2_args(ctx, ctx->cur, ctx->d_flags);
  const int nstrip = (A.nx + TX - 1) / TX;
  const int nchunk = ctx->nvp / ctx->oct_kc;
  // rows per block: about 64, and enough blocks for several waves of two
  // blocks per SM
  int nrb = (A.ny + 63) / 64;
  while ((long long)nstrip * nchunk * nrb < 8LL * 152 && A.ny / (nrb * 2) >= 16) nrb *= 2;
  A.rows = (A.ny + nrb - 1) / nrb;
  dim3 grid(nstrip, nchunk, (A.ny + A.rows - 1) / A.rows);
  const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(ctx->tmap[ctx->cur]);
  switch (ctx->oct_kc) {
  case 192: sweep2d_tma_kernel<6><<<grid, NTHREADS, Cfg<6>::SMEM, ctx->stream>>>(*tm, A); break;
  case 128: sweep2d_tma_kernel<4><<<grid, NTHREADS, Cfg<4>::SMEM, ctx->stream>>>(*tm, A); break;
  default: sweep2d_tma_kernel<2><<<grid, NTHREADS, Cfg<2>::SMEM, ctx->stream>>>(*tm, A); break;
  }
  return cudaGetLastError();
}

bool tma_batch_member_ok(const ibdvm_ctx *ctx) {
  if (ctx->precision != IBDVM_MIXED || ctx->partf == nullptr || encoder() == nullptr) return false;
  if (ctx->dim == 2) return tma_sweep_applicable(ctx);
  return tma3_sweep_applicable(ctx);
}

int tma_batch_kpt_max(const ibdvm_ctx *ctx) { return ctx->oct_kc / 32; }

void tma_batch_free(SweepTables &t) {
  void *ps[] = {t.args, t.tmaps, t.items, t.next};
  for (void *p : ps)
    if (p) cudaFree(p);
  t = SweepTables{};
}

cudaError_t tma_batch_build(const std::vector<ibdvm_ctx *> &cases, const std::vector<int> &kpt, int rows,
                            int *flags, SweepTables &t, cudaStream_t s) {
  (void)kpt; // the chunk of every member is that of its velocity layout
  tma_batch_free(t);
  if (!cases.empty() && cases[0]->dim == 3) return tma3_batch_build(cases, rows, flags, t, s);
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const int n = static_cast<int>(cases.size());
  std::vector<Oct2Args> args(2 * n);
  std::vector<CUtensorMap> maps(2 * n);
  std::vector<WorkItem> items;
  for (int i = 0; i < n; ++i) {
    const ibdvm_ctx *ctx = cases[i];
    if (ctx->oct_kc <= 0) return cudaErrorInvalidValue;
    const int vpl = ctx->oct_kc / 32;
    for (int p = 0; p < 2; ++p) {
      const int cur = ctx->cur ^ p;
      args[2 * i + p] = oct2_args(ctx, cur, flags + i);
      if (encode_map(enc, &maps[2 * i + p], ctx->f[cur], ctx->geom, ctx->nvp, ctx->oct_kc) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
    // items: column strips x velocity chunks x row ranges of about `rows` rows
    const int nx = ctx->geom.n[0], ny = ctx->geom.n[1];
    const int nrb = (rows <= 0 || rows >= ny) ? 1 : (ny + rows - 1) / rows;
    const int per = (ny + nrb - 1) / nrb;
    for (int x0 = 0; x0 < nx; x0 += TX)
      for (int c = 0; c < ctx->nvp / ctx->oct_kc; ++c)
        for (int ya = 0; ya < ny; ya += per) {
          WorkItem it{};
          it.cas = i;
          it.x0 = x0;
          it.chunk = c;
          it.ya = ya;
          it.yb = std::min(ny, ya + per);
          it.vpl = vpl;
          items.push_back(it);
        }
  }
  // grouped by velocities per lane (6, 4, 2), the largest items of a group
  // first, so the last items to start are the short ones
  std::stable_sort(items.begin(), items.end(), [](const WorkItem &a, const WorkItem &b) {
    if (a.vpl != b.vpl) return a.vpl > b.vpl;
    return (a.yb - a.ya) > (b.yb - b.ya);
  });
  static const int kVpl[3] = {6, 4, 2};
  for (int c = 0, i = 0; c < 3; ++c) {
    t.cls_off[c] = i;
    while (i < static_cast<int>(items.size()) && items[i].vpl == kVpl[c]) ++i;
    t.cls_off[c + 1] = i;
  }
  cudaError_t e;
  auto up = [&](const void *h, size_t bytes, void *&d) -> cudaError_t {
    cudaError_t r = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (r != cudaSuccess || bytes == 0) return r;
    return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
  };
  if ((e = up(args.data(), args.size() * sizeof(Oct2Args), t.args)) != cudaSuccess) return e;
  if ((e = up(maps.data(), maps.size() * sizeof(CUtensorMap), t.tmaps)) != cudaSuccess) return e;
  if ((e = up(items.data(), items.size() * sizeof(WorkItem), t.items)) != cudaSuccess) return e;
  void *nx = nullptr;
  if ((e = cudaMalloc(&nx, 3 * sizeof(int))) != cudaSuccess) return e;
  t.next = static_cast<int *>(nx);
  t.nitems = static_cast<int>(items.size());
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  t.grid = 0;
  for (int c = 0; c < 3; ++c) {
    const int n = t.cls_off[c + 1] - t.cls_off[c];
    t.cls_grid[c] = 0;
    if (n == 0) continue;
    const void *fn = (c == 0)   ? (const void *)sweep2d_tma_batch_kernel<6>
                     : (c == 1) ? (const void *)sweep2d_tma_batch_kernel<4>
                                : (const void *)sweep2d_tma_batch_kernel<2>;
    const int smem = (c == 0) ? (int)Cfg<6>::SMEM : (c == 1) ? (int)Cfg<4>::SMEM : (int)Cfg<2>::SMEM;
    int per_sm = 0;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTHREADS, smem)) != cudaSuccess) return e;
    t.cls_grid[c] = std::max(1, std::min(n, nsm * std::max(per_sm, 1)));
    t.grid = std::max(t.grid, t.cls_grid[c]);
  }
  return cudaStreamSynchronize(s); // the host tables go out of scope
}

cudaError_t tma_batch_launch(const SweepTables &t, int par, cudaStream_t s) {
  if (t.dim == 3) return tma3_batch_launch(t, par, s);
  if (t.nitems == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.next, 0, 3 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const Oct2Args *a = static_cast<const Oct2Args *>(t.args);
  const CUtensorMap *m = static_cast<const CUtensorMap *>(t.tmaps);
  const WorkItem *it = static_cast<const WorkItem *>(t.items);
  for (int c = 0; c < 3; ++c) {
    const int off = t.cls_off[c], n = t.cls_off[c + 1] - off;
    if (n == 0) continue;
    if (c == 0)
      sweep2d_tma_batch_kernel<6><<<t.cls_grid[c], NTHREADS, Cfg<6>::SMEM, s>>>(a, m, it + off, n, t.next + c, par);
    else if (c == 1)
      sweep2d_tma_batch_kernel<4><<<t.cls_grid[c], NTHREADS, Cfg<4>::SMEM, s>>>(a, m, it + off, n, t.next + c, par);
    else
      sweep2d_tma_batch_kernel<2><<<t.cls_grid[c], NTHREADS, Cfg<2>::SMEM, s>>>(a, m, it + off, n, t.next + c, par);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

} // namespace ibdvm
