// capi.cpp -- the C-ABI of libibdvm.so (declared in include/ibdvm.h).
//
// Owns the device memory of a solver context, validates every argument,
// uploads the host geometry (geom.cpp) and drives the kernels (kernels.cu).
// No call aborts: failures come back as an ibdvm_status with a one-line
// reason in ibdvm_last_error().
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"

using namespace ibdvm;

namespace {

constexpr double kPi = 3.14159265358979323846;
thread_local std::string g_geom_err;

struct Fail {
  ibdvm_status st;
};

void cfree(void *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}
template <typename T> void cfree_t(T *&p) {
  void *q = p;
  cfree(q);
  p = nullptr;
}

// cudaMalloc with bookkeeping; throws Fail on error
template <typename T> T *dalloc(ibdvm_ctx *ctx, size_t count, const char *what) {
  void *p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = std::string("device allocation of ") + what + " (" + std::to_string(bytes) +
               " bytes) failed: " + cudaGetErrorString(e);
    throw Fail{IBDVM_E_NOMEM};
  }
  ctx->dev_bytes += bytes;
  return static_cast<T *>(p);
}

void check(ibdvm_ctx *ctx, cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    throw Fail{IBDVM_E_CUDA};
  }
}

template <typename T> void upload(ibdvm_ctx *ctx, T *dst, const std::vector<T> &src, const char *what) {
  if (src.empty()) return;
  check(ctx, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream), what);
}

void harvest(ibdvm_ctx *ctx);
void sync(ibdvm_ctx *ctx, const char *what) {
  check(ctx, cudaStreamSynchronize(ctx->stream), what);
  harvest(ctx);
}

int nmoments(int dim) { return dim == 2 ? 9 : 14; }

// Maxwellian at every node (2D reduced H, B = T/2 H; 3D g), Sec. 4
std::vector<double> maxwellian(const Geom &G, double rho, const double *U, double T) {
  std::vector<double> out(static_cast<size_t>(G.nvp) * G.ncomp, 0.0);
  const double norm = (G.dim == 2) ? rho / (kPi * T) : rho / std::pow(kPi * T, 1.5);
  for (int k = 0; k < G.nv; ++k) {
    double c2 = 0.0;
    for (int a = 0; a < G.dim; ++a) {
      double c = G.xi[3 * k + a] - U[a];
      c2 += c * c;
    }
    double g = norm * std::exp(-c2 / T);
    out[static_cast<size_t>(k) * G.ncomp] = g;
    if (G.dim == 2) out[static_cast<size_t>(k) * 2 + 1] = 0.5 * T * g;
  }
  return out;
}

template <typename T> std::vector<T> cast(const std::vector<double> &v) {
  return std::vector<T>(v.begin(), v.end());
}

void free_body(ibdvm_ctx *ctx) {
  void *ps[] = {ctx->dslot, ctx->dlinks, ctx->l_int, ctx->l_dbl, ctx->l_wg, ctx->g_int, ctx->s_int,
                ctx->s_dbl, ctx->lval, ctx->fi_scr, ctx->fsp_scr, ctx->rhow, ctx->fpart, ctx->gw_unit};
  for (void *p : ps)
    if (p) cudaFree(p);
  ctx->dslot = ctx->dlinks = ctx->l_int = ctx->g_int = ctx->s_int = nullptr;
  ctx->l_dbl = ctx->l_wg = ctx->s_dbl = ctx->rhow = ctx->fpart = ctx->gw_unit = nullptr;
  ctx->lval = ctx->fi_scr = ctx->fsp_scr = nullptr;
}

void drop_graphs(ibdvm_ctx *ctx) {
  for (int i = 0; i < 4; ++i) {
    if (ctx->graph2[i]) cudaGraphExecDestroy(ctx->graph2[i]);
    ctx->graph2[i] = nullptr;
  }
}

void free_all(ibdvm_ctx *ctx) {
  drop_graphs(ctx);
  free_body(ctx);
  cfree(ctx->f[0]);
  cfree(ctx->f[1]);
  cfree(ctx->mac);
  cfree_t(ctx->W[0]);
  cfree_t(ctx->W[1]);
  cfree_t(ctx->part);
  cfree_t(ctx->resblk);
  cfree_t(ctx->d_res);
  cfree_t(ctx->d_flags);
  cfree(ctx->xiT);
  cfree(ctx->wT);
  cfree(ctx->finf);
  cfree_t(ctx->xiD);
  cfree_t(ctx->wD);
  cfree_t(ctx->kst);
  cfree_t(ctx->oct_const);
  cfree_t(ctx->oct_sign);
  cfree_t(ctx->ctype);
  cfree_t(ctx->cmask);
  cfree_t(ctx->tree_sti);
  cfree_t(ctx->tree_stg);
  cfree_t(ctx->tree_lrec);
  cfree_t(ctx->tree_far);
  cfree_t(ctx->tree_sched);
  cfree_t(ctx->partf);
  cfree_t(ctx->d_forces);
  cfree_t(ctx->d_step_forces);
  cfree(ctx->whalo);
  for (cudaEvent_t &e : ctx->copy_ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (ctx->copy_stream) {
    cudaStreamDestroy(ctx->copy_stream);
    ctx->copy_stream = nullptr;
  }
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  ctx->ev_pool.clear();
  ctx->ev_marks.clear();
  ctx->ev_used = 0;
}

// adds the elapsed times of the recorded launch events (after a sync)
void harvest(ibdvm_ctx *ctx) {
  for (const auto &m : ctx->ev_marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_pool[m.second], ctx->ev_pool[m.second + 1]) == cudaSuccess)
      ctx->kernel_ms[m.first] += ms;
  }
  cudaGetLastError();
  ctx->ev_marks.clear();
  ctx->ev_used = 0;
}

// Uploads the cell classes, links, surface cells and cut table of ctx->geom.
// A tree (C29) passes the finest grid GV the body was placed on and the leaf
// of each of its cells (vmap): ctx->geom then holds the ghost band in leaf
// indices, and the surface vectors and neighbour codes come from GV.
void upload_body(ibdvm_ctx *ctx, const Geom *GV = nullptr, const std::vector<int> *vmap = nullptr) {
  const Geom &G = ctx->geom;
  const Geom &GS = GV ? *GV : G; // the grid of the surface cells
  auto cell_of = [&](long long v) { return vmap ? (*vmap)[static_cast<size_t>(v)] : static_cast<int>(v); };
  const int D = G.dim;
  const size_t nl = G.links.size();
  const int nvp = ctx->nvp;
  // donor slots: (donor, direction toward the ghost) -> link
  std::vector<int> dslot(G.ncell, -1), dlinks;
  for (size_t l = 0; l < nl; ++l) {
    const Link &L = G.links[l];
    int &slot = dslot[L.donor];
    if (slot < 0) {
      slot = static_cast<int>(dlinks.size() / 6);
      dlinks.insert(dlinks.end(), 6, -1);
    }
    const int dir = 2 * L.axis + ((-L.side) > 0 ? 1 : 0);
    dlinks[static_cast<size_t>(slot) * 6 + dir] = static_cast<int>(l);
  }
  std::vector<int> l_int(8 * nl);
  std::vector<double> l_dbl(8 * nl, 0.0), l_wg(nl * static_cast<size_t>(nvp), 0.0);
  for (size_t l = 0; l < nl; ++l) {
    const Link &L = G.links[l];
    int *li = &l_int[8 * l];
    li[0] = L.gidx;
    li[1] = L.donor;
    li[2] = L.aux;
    li[3] = L.axis;
    li[4] = L.side;
    li[5] = L.ghost;
    li[6] = G.surf_off[L.gidx];
    li[7] = G.surf_off[L.gidx + 1];
    double *ld = &l_dbl[8 * l];
    ld[0] = L.c_sp;
    ld[1] = L.c_iw;
    ld[2] = L.c_gc;
    for (int a = 0; a < 3; ++a) ld[3 + a] = L.nw[a];
    double S = 1.0;
    for (int b = 0; b < D; ++b)
      if (b != L.axis) S *= G.dx[b];
    ld[6] = S;
    for (int i = 0; i < G.nv; ++i) l_wg[l * nvp + ctx->kst_h[i]] = G.wg[l * G.nv + i];
  }
  // surface entries: neighbour codes and the vectors of the weights and slopes
  const int mode = (G.gas.flags & IBDVM_RHAT_GHOST_TO_FLUID) ? 2 : 1;
  const size_t ns = G.surf_cell.size();
  std::vector<int> s_int(8 * ns, -2);
  std::vector<double> s_dbl(8 * ns, 0.0);
  auto ijk_of = [&](long long c, int *o) {
    o[0] = static_cast<int>(c % GS.n[0]);
    o[1] = static_cast<int>((c / GS.n[0]) % GS.n[1]);
    o[2] = static_cast<int>(c / (static_cast<long long>(GS.n[0]) * GS.n[1]));
  };
  for (size_t gi = 0; gi < GS.ghosts.size(); ++gi) {
    int ig[3];
    ijk_of(GS.ghosts[gi], ig);
    for (int e = GS.surf_off[gi]; e < GS.surf_off[gi + 1]; ++e) {
      const int j = GS.surf_cell[e];
      int ij[3];
      ijk_of(j, ij);
      int *si = &s_int[8 * e];
      double *sd = &s_dbl[8 * e];
      si[0] = cell_of(j);
      for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s) {
          int code = -2;
          if (a < D) {
            int q[3] = {ij[0], ij[1], ij[2]};
            q[a] += s ? 1 : -1;
            if (q[a] < 0 || q[a] >= GS.n[a]) {
              code = -1; // domain halo: freestream or a diffuse domain wall
            } else {
              long long nb = q[0] + GS.n[0] * (q[1] + static_cast<long long>(GS.n[1]) * q[2]);
              if (GS.type[nb] == IBDVM_CELL_FLUID) code = cell_of(nb);
            }
          }
          si[1 + 2 * a + s] = code;
        }
      double rl = 0.0;
      for (int a = 0; a < D; ++a) {
        const int o = (mode == 2) ? (ij[a] - ig[a]) : (ig[a] - ij[a]);
        sd[a] = o * G.dx[a];
        rl += sd[a] * sd[a];
      }
      sd[3] = std::sqrt(rl);
      for (int a = 0; a < D; ++a) sd[4 + a] = (ij[a] - ig[a]) * G.dx[a];
      sd[7] = 1.0 / sd[3];
    }
  }
  std::vector<uint8_t> ctype(G.type.begin(), G.type.end());
  // per-cell flags of the sweeps: a ghost across face (a, s) sets bit 2a + (s > 0)
  std::vector<uint8_t> cmask(G.ncell, 0);
  for (long long c = 0; c < G.ncell; ++c) {
    if (G.type[c] != IBDVM_CELL_FLUID) {
      cmask[c] = 64;
      continue;
    }
    if (GV) continue; // a tree: the tree sweep reads ghost faces from its stencil tables
    int ijk[3];
    ijk_of(c, ijk);
    for (int a = 0; a < D; ++a)
      for (int s = 0; s < 2; ++s) {
        int q[3] = {ijk[0], ijk[1], ijk[2]};
        q[a] += s ? 1 : -1;
        if (q[a] < 0 || q[a] >= G.n[a]) continue;
        long long nb = q[0] + G.n[0] * (q[1] + static_cast<long long>(G.n[1]) * q[2]);
        if (G.type[nb] == IBDVM_CELL_GHOST) cmask[c] |= static_cast<uint8_t>(1u << (2 * a + s));
      }
  }
  // allocate the new band first, so that a failure leaves the old one intact
  ibdvm_ctx tmp;
  tmp.stream = ctx->stream;
  try {
    tmp.dslot = dalloc<int>(&tmp, dslot.size(), "donor slots");
    tmp.dlinks = dalloc<int>(&tmp, dlinks.size(), "donor links");
    tmp.l_int = dalloc<int>(&tmp, l_int.size(), "link table");
    tmp.l_dbl = dalloc<double>(&tmp, l_dbl.size(), "link coefficients");
    tmp.l_wg = dalloc<double>(&tmp, l_wg.size(), "cut table");
    tmp.s_int = dalloc<int>(&tmp, s_int.size(), "surface table");
    tmp.s_dbl = dalloc<double>(&tmp, s_dbl.size(), "surface vectors");
    const size_t band = nl * static_cast<size_t>(nvp) * ctx->ncomp * ctx->esize;
    tmp.lval = dalloc<char>(&tmp, band, "ghost values");
    tmp.fi_scr = dalloc<char>(&tmp, band, "incident scratch");
    tmp.fsp_scr = dalloc<char>(&tmp, band, "shifted-point scratch");
    tmp.rhow = dalloc<double>(&tmp, nl, "wall density");
    tmp.fpart = dalloc<double>(&tmp, 4 * nl, "force partial sums");
    tmp.gw_unit = dalloc<double>(&tmp, nvp, "wall Maxwellian");
  } catch (const Fail &f) {
    ctx->err = tmp.err;
    free_body(&tmp);
    throw;
  }
  free_body(ctx);
  ctx->dev_bytes += tmp.dev_bytes;
  ctx->dslot = tmp.dslot;
  ctx->dlinks = tmp.dlinks;
  ctx->l_int = tmp.l_int;
  ctx->l_dbl = tmp.l_dbl;
  ctx->l_wg = tmp.l_wg;
  ctx->s_int = tmp.s_int;
  ctx->s_dbl = tmp.s_dbl;
  ctx->lval = tmp.lval;
  ctx->fi_scr = tmp.fi_scr;
  ctx->fsp_scr = tmp.fsp_scr;
  ctx->rhow = tmp.rhow;
  ctx->fpart = tmp.fpart;
  ctx->gw_unit = tmp.gw_unit;
  tmp.dslot = tmp.dlinks = tmp.l_int = tmp.s_int = nullptr;
  tmp.l_dbl = tmp.l_wg = tmp.s_dbl = tmp.rhow = tmp.fpart = tmp.gw_unit = nullptr;
  tmp.lval = tmp.fi_scr = tmp.fsp_scr = nullptr;
  ctx->nlink = static_cast<int>(nl);
  ctx->nghost = static_cast<int>(G.ghosts.size());
  ctx->nsurf = static_cast<int>(ns);
  upload(ctx, ctx->dslot, dslot, "upload donor slots");
  upload(ctx, ctx->dlinks, dlinks, "upload donor links");
  upload(ctx, ctx->l_int, l_int, "upload link table");
  upload(ctx, ctx->l_dbl, l_dbl, "upload link coefficients");
  upload(ctx, ctx->l_wg, l_wg, "upload cut table");
  upload(ctx, ctx->s_int, s_int, "upload surface table");
  upload(ctx, ctx->s_dbl, s_dbl, "upload surface vectors");
  {
    // unit-density wall Maxwellian per velocity (Eq. boundary maxwell; the 2D
    // reduced H_w of Sec. 4): depends on the wall only, so tabulated once
    std::vector<double> gw(nvp, 0.0);
    const double Tw = G.body.T_w;
    const double norm = (D == 2) ? 1.0 / (kPi * Tw) : 1.0 / std::pow(kPi * Tw, 1.5);
    for (int k = 0; k < G.nv; ++k) {
      double c2 = 0.0;
      for (int a = 0; a < D; ++a) {
        const double c = G.xi[3 * k + a] - G.body.U_w[a];
        c2 += c * c;
      }
      gw[ctx->kst_h[k]] = norm * std::exp(-c2 / Tw);
    }
    upload(ctx, ctx->gw_unit, gw, "upload wall Maxwellian");
  }
  upload(ctx, ctx->ctype, ctype, "upload cell classes");
  upload(ctx, ctx->cmask, cmask, "upload cell flags");
  if (nl) {
    const size_t band = nl * static_cast<size_t>(nvp) * ctx->ncomp * ctx->esize;
    check(ctx, cudaMemsetAsync(ctx->lval, 0, band, ctx->stream), "clear ghost values");
    check(ctx, cudaMemsetAsync(ctx->fi_scr, 0, band, ctx->stream), "clear scratch");
    check(ctx, cudaMemsetAsync(ctx->fsp_scr, 0, band, ctx->stream), "clear scratch");
  }
  sync(ctx, "upload body");
}

// moments of the current state in two passes (about zero, then about the
// bulk velocity just found), so the macroscopic state matches f exactly
void refresh_moments(ibdvm_ctx *ctx) {
  check(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream), "clear flags");
  check(ctx, launch_refresh_range(ctx, 0, ctx->ncell), "moments kernel");
}

// f^n from host memory in kUploadParts cell ranges on a copy stream; the
// moments of each range are taken on the context's stream as soon as its
// bytes have arrived (a cell's moments depend on its own row only), so the
// refresh hides behind the copy. Small states take one copy.
void upload_refresh(ibdvm_ctx *ctx, const void *host, size_t bytes) {
  const long long nc = ctx->ncell;
  const size_t row = static_cast<size_t>(ctx->nvp) * ctx->ncomp * ctx->esize;
  char *dst = static_cast<char *>(ctx->f[ctx->cur]);
  const char *src = static_cast<const char *>(host);
  check(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream), "clear flags");
  if (bytes < (size_t(64) << 20) || nc < kUploadParts) {
    check(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy f");
    check(ctx, launch_refresh_range(ctx, 0, nc), "moments kernel");
    return;
  }
  if (!ctx->copy_stream) {
    check(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (cudaEvent_t &e : ctx->copy_ev) check(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "copy event");
  }
  // the copy starts after the work already on the context's stream
  check(ctx, cudaEventRecord(ctx->copy_ev[kUploadParts], ctx->stream), "record");
  check(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev[kUploadParts], 0), "wait");
  for (int i = 0; i < kUploadParts; ++i) {
    const long long c0 = nc * i / kUploadParts, c1 = nc * (i + 1) / kUploadParts;
    check(ctx, cudaMemcpyAsync(dst + c0 * row, src + c0 * row, (c1 - c0) * row, cudaMemcpyHostToDevice,
                               ctx->copy_stream), "copy f");
    check(ctx, cudaEventRecord(ctx->copy_ev[i], ctx->copy_stream), "record");
    check(ctx, cudaStreamWaitEvent(ctx->stream, ctx->copy_ev[i], 0), "wait");
    check(ctx, launch_refresh_range(ctx, c0, c1), "moments kernel");
  }
}

int read_flags(ibdvm_ctx *ctx) {
  int fl = 0;
  check(ctx, cudaMemcpyAsync(&fl, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read flags");
  sync(ctx, "read flags");
  return fl;
}

ibdvm_status status_of_flags(ibdvm_ctx *ctx, int fl) {
  if (fl & kFlagTimeout) {
    ctx->err = "a bounded device wait in the sweep gave up (TMA copy did not arrive)";
    return IBDVM_E_TIMEOUT;
  }
  if (fl & kFlagNonFinite) {
    ctx->err = "non-finite or non-positive density/temperature in the moments";
    return IBDVM_E_NONFINITE;
  }
  if (fl & kFlagUnstable) {
    ctx->err = "dt / tau > 1: the explicit relaxation is unstable; lower the CFL number or dt";
    return IBDVM_E_UNSTABLE;
  }
  return IBDVM_OK;
}

// staging of FP64 dense host arrays through a bounded device buffer
ibdvm_status transfer_f(ibdvm_ctx *ctx, double *host, bool to_state) {
  const size_t per_cell = static_cast<size_t>(ctx->nv) * ctx->ncomp;
  const size_t max_bytes = size_t(256) << 20;
  long long cells_per = std::max<long long>(1, static_cast<long long>(max_bytes / (per_cell * 8)));
  cells_per = std::min(cells_per, ctx->ncell);
  double *stage = dalloc<double>(ctx, cells_per * per_cell, "staging buffer");
  ctx->dev_bytes -= std::max<size_t>(cells_per * per_cell, 1) * sizeof(double);
  ibdvm_status st = IBDVM_OK;
  try {
    for (long long c0 = 0; c0 < ctx->ncell; c0 += cells_per) {
      long long nc = std::min(cells_per, ctx->ncell - c0);
      size_t bytes = nc * per_cell * sizeof(double);
      double *h = host + c0 * per_cell;
      if (to_state) {
        check(ctx, cudaMemcpyAsync(stage, h, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy f to device");
        check(ctx, launch_convert(ctx, stage, c0, nc, true), "convert f");
        // keep the other buffer in step for the cells the sweep does not write
        ctx->cur = 1 - ctx->cur;
        check(ctx, launch_convert(ctx, stage, c0, nc, true), "convert f");
        ctx->cur = 1 - ctx->cur;
      } else {
        check(ctx, launch_convert(ctx, stage, c0, nc, false), "convert f");
        check(ctx, cudaMemcpyAsync(h, stage, bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy f to host");
      }
      sync(ctx, "transfer f");
    }
  } catch (const Fail &f) {
    st = f.st;
  }
  cudaFree(stage);
  return st;
}

double default_lref(const Geom &G) {
  const ibdvm_body_desc &b = G.body;
  if (b.L_ref > 0.0) return b.L_ref;
  switch (b.kind) {
  case IBDVM_BODY_CIRCLE:
    return 2.0 * b.radii[0];
  case IBDVM_BODY_ELLIPSE:
    return 2.0 * std::max(b.radii[0], b.radii[1]);
  case IBDVM_BODY_SPHERE:
    return kPi * b.radii[0] * b.radii[0];
  case IBDVM_BODY_POLYGON: {
    double mn = 1e300, mx = -1e300;
    for (size_t i = 0; i < G.verts.size(); i += 2) {
      mn = std::min(mn, G.verts[i]);
      mx = std::max(mx, G.verts[i]);
    }
    return mx - mn;
  }
  default:
    return 1.0;
  }
}


void fill_forces(ibdvm_ctx *ctx, const double *h, double *F, double *Q, double *CD, double *CL) {
  if (F)
    for (int a = 0; a < 3; ++a) F[a] = (a < ctx->dim) ? h[a] : 0.0;
  if (Q) *Q = h[3];
  const Geom &G = ctx->geom;
  double U2 = 0.0;
  for (int a = 0; a < 3; ++a) U2 += G.Uinf[a] * G.Uinf[a];
  const double qdyn = 0.5 * G.gas.rho_inf * U2 * default_lref(G);
  double cd = 0.0, cl = 0.0;
  if (U2 > 0.0 && qdyn > 0.0) {
    const double Um = std::sqrt(U2);
    const double e[3] = {G.Uinf[0] / Um, G.Uinf[1] / Um, G.Uinf[2] / Um};
    cd = (h[0] * e[0] + h[1] * e[1] + (ctx->dim == 3 ? h[2] * e[2] : 0.0)) / qdyn;
    cl = (-h[0] * e[1] + h[1] * e[0]) / qdyn;
  }
  if (CD) *CD = cd;
  if (CL) *CL = cl;
}

#define IBDVM_GUARD(ctx)                                                                            \
  if (!(ctx)) return IBDVM_E_INVAL;                                                                 \
  ctx->err.clear();                                                                                 \
  try {
#define IBDVM_END                                                                                   \
  }                                                                                                 \
  catch (const Fail &f) {                                                                           \
    return f.st;                                                                                    \
  }                                                                                                 \
  catch (const std::bad_alloc &) {                                                                  \
    ctx->err = "host allocation failed";                                                            \
    return IBDVM_E_NOMEM;                                                                           \
  }

} // namespace

namespace ibdvm {
// message returned by ibdvm_last_error(NULL) for calls that have no context
void set_thread_error(const std::string &e) { g_geom_err = e; }
} // namespace ibdvm

struct ibdvm_geom {
  Geom g;
};

namespace {

// the stencil tables of the tree sweep for the leaf classes and ghost links of
// ctx->geom, and the row beyond each donor for the surface force
void upload_tree_tables(ibdvm_ctx *ctx, const std::vector<int> &glink, const std::vector<int> &far) {
  std::vector<int> sti, lrec;
  std::vector<double> stg;
  build_tree_stencils(ctx->dim, ctx->tree_lev_h, ctx->tree_nb_h, ctx->tree_h0, ctx->geom.type, glink, sti, stg,
                      lrec);
  upload(ctx, ctx->tree_sti, sti, "upload tree stencils");
  upload(ctx, ctx->tree_stg, stg, "upload tree stencil geometry");
  upload(ctx, ctx->tree_lrec, lrec, "upload tree leaf records");
  upload(ctx, ctx->tree_sched, tree_schedule(ctx->dim, lrec), "upload tree leaf schedule");
  cfree_t(ctx->tree_far);
  if (!far.empty()) {
    ctx->tree_far = dalloc<int>(ctx, far.size(), "tree donor rows");
    upload(ctx, ctx->tree_far, far, "upload tree donor rows");
  }
}

// a body on a tree-refined grid (C29): placed on the finest grid, moved onto
// the leaves when its ghost band lies in the finest level
ibdvm_status tree_set_body(ibdvm_ctx *ctx, const ibdvm_body_desc *body) {
  Geom Gv = ctx->tree_vgeom;
  std::string err;
  if (!place_body(*body, Gv, err)) {
    ctx->err = err;
    return IBDVM_E_INVAL;
  }
  Geom Gt = ctx->geom;
  std::vector<int> glink, far;
  if (!map_tree_body(Gv, ctx->tree_own, ctx->tree_lev_h, ctx->tree_L, Gt, glink, far, err)) {
    ctx->err = err;
    return IBDVM_E_INVAL;
  }
  drop_graphs(ctx);
  ++ctx->body_gen;
  Geom old = std::move(ctx->geom);
  ctx->geom = std::move(Gt);
  try {
    upload_body(ctx, &Gv, &ctx->tree_own);
    upload_tree_tables(ctx, glink, far);
  } catch (const Fail &f) {
    std::string e = ctx->err;
    ctx->geom = std::move(old);
    ctx->err = e;
    return f.st;
  }
  refresh_moments(ctx);
  return status_of_flags(ctx, read_flags(ctx));
}

} // namespace

extern "C" {

const char *ibdvm_status_string(ibdvm_status s) {
  switch (s) {
  case IBDVM_OK: return "ok";
  case IBDVM_E_INVAL: return "invalid argument";
  case IBDVM_E_NOMEM: return "out of memory";
  case IBDVM_E_CUDA: return "CUDA error";
  case IBDVM_E_UNSTABLE: return "unstable time step";
  case IBDVM_E_NONFINITE: return "non-finite state";
  case IBDVM_E_NOTCONVERGED: return "not converged";
  case IBDVM_E_TIMEOUT: return "device wait timed out";
  case IBDVM_E_STATE: return "invalid state";
  }
  return "unknown status";
}

// a context on a uniform grid, or (tree != NULL) on the leaves of a
// tree-refined 2D grid over the root grid `grid`
static ibdvm_status create_ctx(const ibdvm_grid_desc *grid, const ibdvm_tree_desc *tree,
                               const ibdvm_vgrid_desc *vgrid, const ibdvm_gas_desc *gas, void *cuda_stream,
                               ibdvm_ctx **out) {
  if (!out) return IBDVM_E_INVAL;
  *out = nullptr;
  if (!grid || !vgrid || !gas) return IBDVM_E_INVAL;
  ibdvm_ctx *ctx = new (std::nothrow) ibdvm_ctx();
  if (!ctx) return IBDVM_E_NOMEM;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ibdvm_status st = IBDVM_OK;
  try {
    std::string err;
    ibdvm_grid_desc gd = *grid;
    std::vector<int> tlev, tnb, town;
    if (tree) {
      // the velocity grid, the gas and the time step of the finest level (dt by
      // the CFL of the smallest leaf); the cells are the leaves
      if (!build_tree_mesh(*grid, *tree, tlev, tnb, town, err)) {
        ctx->err = err;
        throw Fail{IBDVM_E_INVAL};
      }
      for (int a = 0; a < grid->dim; ++a) gd.n[a] = grid->n[a] << tree->maxlevel;
    }
    if (!build_grid(gd, *vgrid, *gas, ctx->geom, err)) {
      ctx->err = err;
      throw Fail{IBDVM_E_INVAL};
    }
    if (tree) {
      ctx->tree_vgeom = ctx->geom; // the finest grid: a body is placed there (C29)
      ctx->tree_own = std::move(town);
      ctx->tree_lev_h = tlev;
      ctx->tree_L = tree->maxlevel;
      Geom &Gt = ctx->geom;
      Gt.ncell = tree->nleaf;
      Gt.n[0] = tree->nleaf;
      Gt.n[1] = Gt.n[2] = 1;
      Gt.type.assign(static_cast<size_t>(tree->nleaf), IBDVM_CELL_FLUID);
      Gt.nfluid = tree->nleaf;
      ctx->tree = true;
      for (int a = 0; a < grid->dim; ++a) ctx->tree_h0[a] = (grid->hi[a] - grid->lo[a]) / grid->n[a];
    }
    const Geom &G = ctx->geom;
    ctx->precision = gas->precision;
    ctx->dim = G.dim;
    ctx->ncomp = G.ncomp;
    ctx->nv = G.nv;
    ctx->nvp = G.nvp;
    ctx->ncell = G.ncell;
    // the stored order of the velocities: natural, or grouped by orthant for
    // the FP32 TMA sweeps (IBDVM_NO_TMA=1 keeps the plain sweep and the natural order)
    const char *no_tma = std::getenv("IBDVM_NO_TMA");
    const bool tma_off = (no_tma && no_tma[0] == '1') || tree != nullptr; // trees: the generic tree sweep
    ctx->kst_h.resize(G.nv);
    for (int i = 0; i < G.nv; ++i) ctx->kst_h[i] = i;
    if (tree) {
      // trees: grouped by orthant (bit a: component a < 0), packed, so that
      // the threads of a warp of the tree sweep share upwind sides
      int pos = 0;
      for (int o = 0; o < (1 << G.dim); ++o) {
        if (o > 0 && o < 4) ctx->tree_qb[o - 1] = pos;
        for (int i = 0; i < G.nv; ++i) {
          int oi = 0;
          for (int a = 0; a < G.dim; ++a) oi |= (G.xi[3 * i + a] < 0.0) ? (1 << a) : 0;
          if (oi == o) ctx->kst_h[i] = pos++;
        }
      }
    }
    if (!tma_off && gas->precision == IBDVM_MIXED && tma_encoder_available()) {
      std::vector<int> kst;
      int nvp = 0;
      const int kc = orthant_layout(G, kst, nvp);
      ctx->oct_kc = kc;
      ctx->kst_h = std::move(kst);
      ctx->nvp = nvp;
    }
    ctx->esize = (ctx->precision == IBDVM_FP64) ? sizeof(double) : sizeof(float);
    // velocity chunks: one chunk per cell unless the grid is too small to fill the GPU
    const long long cell_blocks = (ctx->ncell + 3) / 4;
    const int kblocks = ctx->nvp / 64;
    int nchunk = static_cast<int>(std::min<long long>(kblocks, std::max<long long>(1, (4 * 152 + cell_blocks - 1) / cell_blocks)));
    ctx->kloop = (kblocks + nchunk - 1) / nchunk;
    ctx->nchunk = (kblocks + ctx->kloop - 1) / ctx->kloop;
    const int NW = G.dim + 2;
    const int NM = nmoments(G.dim);
    // memory check before allocating
    const size_t fbytes = static_cast<size_t>(ctx->ncell) * ctx->nvp * ctx->ncomp * ctx->esize;
    const size_t need = 2 * fbytes + static_cast<size_t>(ctx->ncell) * (ctx->nvp / 64 + 1) * 4 * (G.dim == 2 ? 9 : 14) +
                        static_cast<size_t>(ctx->ncell) *
                                         (kMac * ctx->esize + 2 * (NW + G.dim) * 8 + ctx->nchunk * NM * 8 + 8);
    int dev = 0;
    check(ctx, cudaGetDevice(&dev), "cudaGetDevice");
    size_t freeb = 0, totb = 0;
    check(ctx, cudaMemGetInfo(&freeb, &totb), "cudaMemGetInfo");
    if (need > freeb) {
      ctx->err = "the case needs " + std::to_string(need) + " bytes of device memory, " +
                 std::to_string(freeb) + " are free";
      throw Fail{IBDVM_E_NOMEM};
    }
    ctx->f[0] = dalloc<char>(ctx, fbytes, "f");
    ctx->f[1] = dalloc<char>(ctx, fbytes, "f");
    ctx->mac = dalloc<char>(ctx, static_cast<size_t>(kMac) * ctx->ncell * ctx->esize, "macroscopic state");
    for (int i = 0; i < 2; ++i) ctx->W[i] = dalloc<double>(ctx, static_cast<size_t>(NW + G.dim) * ctx->ncell, "W");
    ctx->part = dalloc<double>(ctx, static_cast<size_t>(ctx->nchunk) * NM * ctx->ncell, "moment sums");
    ctx->nresblk = static_cast<int>((ctx->ncell + 255) / 256);
    ctx->resblk = dalloc<double>(ctx, static_cast<size_t>(ctx->nresblk) * 2 * NW, "residual sums");
    ctx->d_res = dalloc<double>(ctx, 1, "residual");
    ctx->d_flags = dalloc<int>(ctx, 1, "flags");
    ctx->d_forces = dalloc<double>(ctx, 4, "forces");
    ctx->d_step_forces = dalloc<double>(ctx, 4, "step forces");
    check(ctx, cudaMemsetAsync(ctx->d_step_forces, 0, 4 * sizeof(double), ctx->stream), "clear");
    ctx->ctype = dalloc<uint8_t>(ctx, ctx->ncell, "cell classes");
    ctx->cmask = dalloc<uint8_t>(ctx, ctx->ncell, "cell flags");
    if (tree) {
      std::vector<int> sti, lrec;
      std::vector<double> stg;
      build_tree_stencils(G.dim, tlev, tnb, ctx->tree_h0, {}, {}, sti, stg, lrec);
      ctx->tree_sti = dalloc<int>(ctx, sti.size(), "tree stencils");
      ctx->tree_stg = dalloc<double>(ctx, stg.size(), "tree stencil geometry");
      ctx->tree_lrec = dalloc<int>(ctx, lrec.size(), "tree leaf records");
      ctx->tree_sched = dalloc<int>(ctx, lrec.size() / 8, "tree leaf schedule");
      upload(ctx, ctx->tree_sti, sti, "upload tree stencils");
      upload(ctx, ctx->tree_stg, stg, "upload tree stencil geometry");
      upload(ctx, ctx->tree_lrec, lrec, "upload tree leaf records");
      upload(ctx, ctx->tree_sched, tree_schedule(G.dim, lrec), "upload tree leaf schedule");
      ctx->tree_nb_h = std::move(tnb);
    }
    ctx->kst = dalloc<int>(ctx, G.nv, "velocity positions");
    upload(ctx, ctx->kst, ctx->kst_h, "upload velocity positions");
    if (ctx->oct_kc) {
      std::vector<float> vconst;
      std::vector<uint8_t> sign;
      orthant_tables(G, ctx->kst_h, ctx->nvp, ctx->oct_kc, vconst, sign);
      ctx->oct_const = dalloc<float>(ctx, vconst.size(), "velocity constants");
      ctx->oct_sign = dalloc<uint8_t>(ctx, sign.size(), "chunk signs");
      upload(ctx, ctx->oct_const, vconst, "upload velocity constants");
      upload(ctx, ctx->oct_sign, sign, "upload chunk signs");
    }
    // the TMA sweeps of FP32 cases
    if (!tma_off && (tma_sweep_applicable(ctx) || tma3_sweep_applicable(ctx))) {
      const bool two = G.dim == 2;
      ctx->tma_nchunk = two ? tma_sweep_nchunk(ctx) : tma3_sweep_nchunk(ctx);
      const size_t nch = static_cast<size_t>(ctx->tma_nchunk);
      ctx->partf = dalloc<float>(ctx, nch * nmoments(G.dim) * ctx->ncell, "FP32 moment sums");
      check(ctx, two ? tma_sweep_prepare(ctx) : tma3_sweep_prepare(ctx), "TMA sweep set-up");
      ctx->use_tma = true;
      ctx->tma_ok = true;
    }
    // velocity tables
    // (stored positions; padding positions hold zeros)
    std::vector<double> xi3(3 * static_cast<size_t>(ctx->nvp), 0.0), w(ctx->nvp, 0.0);
    for (int i = 0; i < G.nv; ++i) {
      const size_t k = ctx->kst_h[i];
      for (int a = 0; a < 3; ++a) xi3[a * static_cast<size_t>(ctx->nvp) + k] = G.xi[3 * i + a];
      w[k] = G.w[i];
    }
    std::vector<double> finf(static_cast<size_t>(ctx->nvp) * G.ncomp, 0.0);
    {
      const std::vector<double> nat = maxwellian(G, gas->rho_inf, G.Uinf, gas->T_inf);
      for (int i = 0; i < G.nv; ++i)
        for (int m = 0; m < G.ncomp; ++m)
          finf[static_cast<size_t>(ctx->kst_h[i]) * G.ncomp + m] = nat[static_cast<size_t>(i) * G.ncomp + m];
    }
    ctx->xiD = dalloc<double>(ctx, xi3.size(), "velocities");
    upload(ctx, ctx->xiD, xi3, "upload velocities");
    {
      // the weights, followed by their reciprocals (zero at padding positions)
      std::vector<double> w2(2 * w.size(), 0.0);
      for (size_t k = 0; k < w.size(); ++k) {
        w2[k] = w[k];
        w2[w.size() + k] = (w[k] > 0.0) ? 1.0 / w[k] : 0.0;
      }
      ctx->wD = dalloc<double>(ctx, w2.size(), "weights");
      upload(ctx, ctx->wD, w2, "upload weights");
    }
    if (ctx->precision == IBDVM_FP64) {
      double *a = dalloc<double>(ctx, xi3.size(), "velocities");
      double *b = dalloc<double>(ctx, w.size(), "weights");
      double *c = dalloc<double>(ctx, finf.size(), "freestream");
      ctx->xiT = a;
      ctx->wT = b;
      ctx->finf = c;
      upload(ctx, a, xi3, "upload velocities");
      upload(ctx, b, w, "upload weights");
      upload(ctx, c, finf, "upload freestream");
    } else {
      float *a = dalloc<float>(ctx, xi3.size(), "velocities");
      float *b = dalloc<float>(ctx, w.size(), "weights");
      float *c = dalloc<float>(ctx, finf.size(), "freestream");
      ctx->xiT = a;
      ctx->wT = b;
      ctx->finf = c;
      upload(ctx, a, cast<float>(xi3), "upload velocities");
      upload(ctx, b, cast<float>(w), "upload weights");
      upload(ctx, c, cast<float>(finf), "upload freestream");
    }
    check(ctx, cudaMemsetAsync(ctx->mac, 0, static_cast<size_t>(kMac) * ctx->ncell * ctx->esize, ctx->stream), "clear");
    for (int i = 0; i < 2; ++i)
      check(ctx, cudaMemsetAsync(ctx->W[i], 0, static_cast<size_t>(NW + G.dim) * ctx->ncell * 8, ctx->stream), "clear");
    upload_body(ctx);
    check(ctx, launch_init_state(ctx), "init kernel");
    refresh_moments(ctx);
    st = status_of_flags(ctx, read_flags(ctx));
    if (st != IBDVM_OK) throw Fail{st};
  } catch (const Fail &f) {
    st = f.st;
  } catch (const std::bad_alloc &) {
    st = IBDVM_E_NOMEM;
  }
  if (st != IBDVM_OK) {
    g_geom_err = ctx->err;
    free_all(ctx);
    delete ctx;
    return st;
  }
  *out = ctx;
  return IBDVM_OK;
}

ibdvm_status ibdvm_create_grid(const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid,
                               const ibdvm_gas_desc *gas, void *cuda_stream, ibdvm_ctx **out) {
  return create_ctx(grid, nullptr, vgrid, gas, cuda_stream, out);
}

ibdvm_status ibdvm_create_tree(const ibdvm_grid_desc *root, const ibdvm_tree_desc *tree,
                               const ibdvm_vgrid_desc *vgrid, const ibdvm_gas_desc *gas, void *cuda_stream,
                               ibdvm_ctx **out) {
  if (!tree) {
    if (out) *out = nullptr;
    return IBDVM_E_INVAL;
  }
  return create_ctx(root, tree, vgrid, gas, cuda_stream, out);
}

ibdvm_status ibdvm_tree_neighbours(const ibdvm_ctx *ctx, long long *nb) {
  if (!ctx || !nb) return IBDVM_E_INVAL;
  if (!ctx->tree) return IBDVM_E_STATE;
  for (size_t i = 0; i < ctx->tree_nb_h.size(); ++i) nb[i] = ctx->tree_nb_h[i];
  return IBDVM_OK;
}

ibdvm_status ibdvm_set_body(ibdvm_ctx *ctx, const ibdvm_body_desc *body) {
  IBDVM_GUARD(ctx)
  if (!body) {
    ctx->err = "body is NULL";
    return IBDVM_E_INVAL;
  }
  if (ctx->tree) return tree_set_body(ctx, body);
  Geom G2 = ctx->geom;
  std::string err;
  if (!place_body(*body, G2, err)) {
    ctx->err = err;
    return IBDVM_E_INVAL;
  }
  drop_graphs(ctx);
  ++ctx->body_gen;
  Geom old = std::move(ctx->geom);
  ctx->geom = std::move(G2);
  try {
    upload_body(ctx);
  } catch (const Fail &f) {
    std::string e = ctx->err;
    ctx->geom = std::move(old);
    ctx->err = e;
    return f.st;
  }
  refresh_moments(ctx);
  return status_of_flags(ctx, read_flags(ctx));
  IBDVM_END
}

ibdvm_status ibdvm_set_domain(ibdvm_ctx *ctx, const ibdvm_domain_desc *d) {
  IBDVM_GUARD(ctx)
  if (ctx->tree) {
    ctx->err = "set_domain: a tree-refined grid keeps freestream domain faces";
    return IBDVM_E_STATE;
  }
  if (!d) {
    ctx->err = "domain description is NULL";
    return IBDVM_E_INVAL;
  }
  if (ctx->batch) {
    ctx->err = "set_domain: the context is a member of a batch; remove it first";
    return IBDVM_E_STATE;
  }
  const int D = ctx->dim;
  int mask = 0;
  for (int i = 0; i < 6; ++i) {
    const int kind = d->kind[i];
    if (kind != IBDVM_FACE_FREESTREAM && kind != IBDVM_FACE_DIFFUSE_WALL) {
      ctx->err = "set_domain: kind must be IBDVM_FACE_FREESTREAM or IBDVM_FACE_DIFFUSE_WALL";
      return IBDVM_E_INVAL;
    }
    if (kind != IBDVM_FACE_DIFFUSE_WALL) continue;
    if (i >= 2 * D) {
      ctx->err = "set_domain: a 2D grid has no z faces";
      return IBDVM_E_INVAL;
    }
    if (!(d->T_w[i] > 0.0) || !std::isfinite(d->T_w[i]) || !std::isfinite(d->U_w[i][0]) ||
        !std::isfinite(d->U_w[i][1]) || !std::isfinite(d->U_w[i][2])) {
      ctx->err = "set_domain: a wall needs T_w > 0 and a finite U_w";
      return IBDVM_E_INVAL;
    }
    mask |= 1 << i;
  }
  const Geom &G = ctx->geom;
  long long off[7] = {};
  for (int i = 0; i < 6; ++i) off[i + 1] = off[i] + ((i < 2 * D) ? ctx->ncell / G.n[i >> 1] : 0);
  void *halo = nullptr;
  if (mask) {
    const size_t bytes = static_cast<size_t>(off[6]) * ctx->nvp * ctx->ncomp * ctx->esize;
    if (cudaMalloc(&halo, bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "set_domain: device allocation of the wall halo (" + std::to_string(bytes) + " bytes) failed";
      return IBDVM_E_NOMEM;
    }
    ctx->dev_bytes += bytes;
  }
  if (ctx->whalo) {
    sync(ctx, "drain before replacing the wall halo");
    cudaFree(ctx->whalo);
    ctx->dev_bytes -= static_cast<size_t>(ctx->wall_off[6]) * ctx->nvp * ctx->ncomp * ctx->esize;
  }
  ctx->whalo = halo;
  ctx->wall_mask = mask;
  for (int i = 0; i < 7; ++i) ctx->wall_off[i] = mask ? off[i] : 0;
  for (int i = 0; i < 6; ++i) {
    ctx->wall_T[i] = (mask >> i & 1) ? d->T_w[i] : 1.0;
    for (int a = 0; a < 3; ++a) ctx->wall_U[i][a] = (mask >> i & 1) ? d->U_w[i][a] : 0.0;
  }
  // the TMA sweeps read the wall halo at the domain faces
  ctx->use_tma = ctx->tma_ok;
  drop_graphs(ctx);
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_step(ibdvm_ctx *ctx, int nsteps, double *residual_out) {
  IBDVM_GUARD(ctx)
  if (nsteps < 0) {
    ctx->err = "nsteps must be >= 0";
    return IBDVM_E_INVAL;
  }
  if (nsteps == 0) {
    if (residual_out) *residual_out = 0.0;
    return IBDVM_OK;
  }
  check(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream), "clear flags");
  // one step: the ghost band on f^n, the surface force of the fluxes this
  // step applies, then transport, relaxation and the moments of f^{n+1}
  auto one_step = [&]() {
    check(ctx, launch_ghost_band(ctx, nullptr), "ghost band kernel");
    check(ctx, launch_forces(ctx, ctx->d_step_forces), "forces kernel");
    check(ctx, launch_sweep(ctx), "sweep kernel");
  };
  int done = 0;
  // pairs of steps replay a captured CUDA graph (not while profiling, and
  // not on the legacy default stream, which cannot be captured)
  if (nsteps >= 2 && ctx->graphs_enabled && !ctx->profiling && ctx->stream != nullptr) {
    const int key = ctx->cur * 2 + ctx->wcur;
    if (!ctx->graph2[key]) {
      long long before[8];
      for (int i = 0; i < 8; ++i) before[i] = ctx->kernel_launches[i];
      cudaGraph_t g = nullptr;
      check(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin graph capture");
      try {
        one_step();
        one_step();
      } catch (const Fail &) {
        cudaStreamEndCapture(ctx->stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      check(ctx, cudaStreamEndCapture(ctx->stream, &g), "end graph capture");
      cudaError_t e = cudaGraphInstantiate(&ctx->graph2[key], g, 0);
      cudaGraphDestroy(g);
      check(ctx, e, "instantiate step graph");
      for (int i = 0; i < 8; ++i) {
        ctx->graph2_launches[key][i] = ctx->kernel_launches[i] - before[i];
        ctx->kernel_launches[i] = before[i]; // counted when replayed
      }
    }
    for (; done + 2 <= nsteps; done += 2) {
      check(ctx, cudaGraphLaunch(ctx->graph2[key], ctx->stream), "replay step graph");
      for (int i = 0; i < 8; ++i) ctx->kernel_launches[i] += ctx->graph2_launches[key][i];
    }
  }
  for (; done < nsteps; ++done) {
    one_step();
    if (ctx->ev_used > 4096) sync(ctx, "step"); // keep the event pool bounded on long calls
  }
  double res = 0.0;
  int fl = 0;
  check(ctx, cudaMemcpyAsync(&res, ctx->d_res, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read residual");
  check(ctx, cudaMemcpyAsync(&fl, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read flags");
  sync(ctx, "step");
  ctx->steps += nsteps;
  if (residual_out) *residual_out = res;
  ibdvm_status st = status_of_flags(ctx, fl);
  if (st == IBDVM_OK && !std::isfinite(res)) {
    ctx->err = "non-finite residual";
    return IBDVM_E_NONFINITE;
  }
  return st;
  IBDVM_END
}

ibdvm_status ibdvm_moments(ibdvm_ctx *ctx, double *W, double *q, unsigned char *celltype) {
  IBDVM_GUARD(ctx)
  const int D = ctx->dim, NW = D + 2;
  const long long nc = ctx->ncell;
  if (W || q) {
    // rows per cell are formed on the device, in the moment partial-sum
    // buffer (free between steps, at least (D + 2 + D) ncell doubles)
    double *Wo = ctx->part, *qo = ctx->part + static_cast<size_t>(NW) * nc;
    check(ctx, launch_interleave(ctx, W ? Wo : nullptr, q ? qo : nullptr), "interleave W");
    if (W)
      check(ctx, cudaMemcpyAsync(W, Wo, static_cast<size_t>(NW) * nc * 8, cudaMemcpyDeviceToHost, ctx->stream),
            "read W");
    if (q)
      check(ctx, cudaMemcpyAsync(q, qo, static_cast<size_t>(D) * nc * 8, cudaMemcpyDeviceToHost, ctx->stream),
            "read q");
    sync(ctx, "read W");
  }
  if (celltype) std::copy(ctx->geom.type.begin(), ctx->geom.type.end(), celltype);
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_forces(ibdvm_ctx *ctx, double F[3], double *Q, double *CD, double *CL) {
  IBDVM_GUARD(ctx)
  check(ctx, launch_ghost_band(ctx, nullptr), "ghost band kernel");
  check(ctx, launch_forces(ctx, ctx->d_forces), "forces kernel");
  double h[4] = {0, 0, 0, 0};
  check(ctx, cudaMemcpyAsync(h, ctx->d_forces, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "read forces");
  sync(ctx, "forces");
  fill_forces(ctx, h, F, Q, CD, CL);
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_step_forces(ibdvm_ctx *ctx, double F[3], double *Q, double *CD, double *CL) {
  IBDVM_GUARD(ctx)
  double h[4] = {0, 0, 0, 0};
  check(ctx, cudaMemcpyAsync(h, ctx->d_step_forces, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "read forces");
  sync(ctx, "step forces");
  fill_forces(ctx, h, F, Q, CD, CL);
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_set_profiling(ibdvm_ctx *ctx, int on) {
  IBDVM_GUARD(ctx)
  sync(ctx, "profiling");
  ctx->profiling = (on != 0);
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_get_kernel_times(ibdvm_ctx *ctx, double *ms, long long *launches) {
  IBDVM_GUARD(ctx)
  sync(ctx, "kernel times");
  for (int i = 0; i < 8; ++i) {
    if (ms) ms[i] = ctx->kernel_ms[i];
    if (launches) launches[i] = ctx->kernel_launches[i];
  }
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_reset_kernel_times(ibdvm_ctx *ctx) {
  IBDVM_GUARD(ctx)
  sync(ctx, "kernel times");
  for (int i = 0; i < 8; ++i) {
    ctx->kernel_ms[i] = 0.0;
    ctx->kernel_launches[i] = 0;
  }
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_get_f(ibdvm_ctx *ctx, double *f) {
  IBDVM_GUARD(ctx)
  if (!f) return IBDVM_E_INVAL;
  return transfer_f(ctx, f, false);
  IBDVM_END
}

ibdvm_status ibdvm_set_f(ibdvm_ctx *ctx, const double *f) {
  IBDVM_GUARD(ctx)
  if (!f) return IBDVM_E_INVAL;
  ibdvm_status st = transfer_f(ctx, const_cast<double *>(f), true);
  if (st != IBDVM_OK) return st;
  refresh_moments(ctx);
  return status_of_flags(ctx, read_flags(ctx));
  IBDVM_END
}

ibdvm_status ibdvm_get_f_native(ibdvm_ctx *ctx, void *host, size_t bytes) {
  IBDVM_GUARD(ctx)
  const size_t want = static_cast<size_t>(ctx->ncell) * ctx->nvp * ctx->ncomp * ctx->esize;
  if (!host || bytes != want) {
    ctx->err = "get_f_native: bytes must be ncell * nvel_padded * ncomp * element size";
    return IBDVM_E_INVAL;
  }
  check(ctx, cudaMemcpyAsync(host, ctx->f[ctx->cur], bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy f");
  sync(ctx, "copy f");
  return IBDVM_OK;
  IBDVM_END
}

ibdvm_status ibdvm_set_f_native(ibdvm_ctx *ctx, const void *host, size_t bytes) {
  IBDVM_GUARD(ctx)
  const size_t want = static_cast<size_t>(ctx->ncell) * ctx->nvp * ctx->ncomp * ctx->esize;
  if (!host || bytes != want) {
    ctx->err = "set_f_native: bytes must be ncell * nvel_padded * ncomp * element size";
    return IBDVM_E_INVAL;
  }
  upload_refresh(ctx, host, bytes);
  return status_of_flags(ctx, read_flags(ctx));
  IBDVM_END
}

ibdvm_status ibdvm_velocity_positions(const ibdvm_ctx *ctx, int *pos) {
  if (!ctx || !pos) return IBDVM_E_INVAL;
  std::copy(ctx->kst_h.begin(), ctx->kst_h.end(), pos);
  return IBDVM_OK;
}

ibdvm_status ibdvm_ghost_band(ibdvm_ctx *ctx, double *fiw, double *fstarw, double *fstargc, double *rhow) {
  IBDVM_GUARD(ctx)
  const size_t nl = ctx->nlink;
  if (nl == 0) return IBDVM_OK;
  const size_t nvp = ctx->nvp, nc = ctx->ncomp, nv = ctx->nv;
  double *dbg = dalloc<double>(ctx, nl * nvp * nc, "ghost-band debug buffer");
  ctx->dev_bytes -= nl * nvp * nc * sizeof(double);
  ibdvm_status st = IBDVM_OK;
  try {
    check(ctx, launch_ghost_band(ctx, dbg), "ghost band kernel");
    std::vector<double> hs(nl * nvp * nc);
    std::vector<char> hi(nl * nvp * nc * ctx->esize), hg(nl * nvp * nc * ctx->esize);
    std::vector<double> hr(nl);
    check(ctx, cudaMemcpyAsync(hs.data(), dbg, hs.size() * 8, cudaMemcpyDeviceToHost, ctx->stream), "read");
    check(ctx, cudaMemcpyAsync(hi.data(), ctx->fi_scr, hi.size(), cudaMemcpyDeviceToHost, ctx->stream), "read");
    check(ctx, cudaMemcpyAsync(hg.data(), ctx->lval, hg.size(), cudaMemcpyDeviceToHost, ctx->stream), "read");
    check(ctx, cudaMemcpyAsync(hr.data(), ctx->rhow, nl * 8, cudaMemcpyDeviceToHost, ctx->stream), "read");
    sync(ctx, "ghost band");
    auto val = [&](const std::vector<char> &v, size_t i) -> double {
      if (ctx->esize == 8) return reinterpret_cast<const double *>(v.data())[i];
      return reinterpret_cast<const float *>(v.data())[i];
    };
    for (size_t l = 0; l < nl; ++l)
      for (size_t k = 0; k < nv; ++k)
        for (size_t m = 0; m < nc; ++m) {
          size_t src = (l * nvp + ctx->kst_h[k]) * nc + m, dst = (l * nv + k) * nc + m;
          if (fiw) fiw[dst] = val(hi, src);
          if (fstarw) fstarw[dst] = hs[src];
          if (fstargc) fstargc[dst] = val(hg, src);
        }
    if (rhow) std::copy(hr.begin(), hr.end(), rhow);
  } catch (const Fail &f) {
    st = f.st;
  }
  cudaFree(dbg);
  return st;
  IBDVM_END
}

ibdvm_status ibdvm_wall(ibdvm_ctx *ctx, double *out) {
  IBDVM_GUARD(ctx)
  if (!out) {
    ctx->err = "wall: out is NULL";
    return IBDVM_E_INVAL;
  }
  static_assert(IBDVM_WALL_COLS == kWallCols, "wall columns");
  const size_t nl = ctx->nlink;
  if (nl == 0) return IBDVM_OK;
  const size_t scr = nl * ctx->nvp * ctx->ncomp + nl * kWallCols;
  double *fstar = dalloc<double>(ctx, scr, "wall-point scratch buffer");
  ctx->dev_bytes -= scr * sizeof(double);
  double *dout = fstar + nl * ctx->nvp * ctx->ncomp;
  ibdvm_status st = IBDVM_OK;
  try {
    check(ctx, launch_ghost_band(ctx, fstar), "ghost band kernel");
    check(ctx, launch_wall(ctx, fstar, dout), "wall kernel");
    check(ctx, cudaMemcpyAsync(out, dout, nl * kWallCols * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
          "read wall quantities");
    sync(ctx, "wall quantities");
  } catch (const Fail &f) {
    st = f.st;
  }
  cudaFree(fstar);
  return st;
  IBDVM_END
}

ibdvm_status ibdvm_get_info(const ibdvm_ctx *ctx, ibdvm_info *info) {
  if (!ctx || !info) return IBDVM_E_INVAL;
  info->dim = ctx->dim;
  info->ncomp = ctx->ncomp;
  info->ncell = ctx->ncell;
  info->nfluid = ctx->geom.nfluid;
  info->nvel = ctx->nv;
  info->nvel_padded = ctx->nvp;
  info->nlink = ctx->nlink;
  info->nghost = ctx->nghost;
  info->dt = ctx->geom.dt;
  info->precision = ctx->precision;
  info->steps_done = ctx->steps;
  info->device_bytes = ctx->dev_bytes;
  info->sweep_variant = ctx->tree ? 3 : ctx->use_tma ? (ctx->dim == 2 ? 1 : 2) : 0;
  return IBDVM_OK;
}

ibdvm_status ibdvm_set_stream(ibdvm_ctx *ctx, void *cuda_stream) {
  IBDVM_GUARD(ctx)
  if (ctx->batch && static_cast<cudaStream_t>(cuda_stream) != ctx->stream) {
    ctx->err = "a batch member stays on the batch's stream";
    return IBDVM_E_STATE;
  }
  sync(ctx, "drain the old stream");
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return IBDVM_OK;
  IBDVM_END
}

const ibdvm_geom *ibdvm_get_geom(const ibdvm_ctx *ctx) {
  return ctx ? reinterpret_cast<const ibdvm_geom *>(&ctx->geom) : nullptr;
}

void ibdvm_destroy(ibdvm_ctx *ctx) {
  if (!ctx) return;
  if (ctx->batch) batch_detach(ctx);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
}

const char *ibdvm_last_error(const ibdvm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_geom_err.c_str(); }

// ---------------------------------------------------------------------------
// host-only geometry
// ---------------------------------------------------------------------------

ibdvm_status ibdvm_geom_build(const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid,
                              const ibdvm_gas_desc *gas, const ibdvm_body_desc *body, ibdvm_geom **out) {
  if (!out || !grid || !vgrid || !gas) return IBDVM_E_INVAL;
  *out = nullptr;
  try {
    ibdvm_geom *g = new ibdvm_geom();
    std::string err;
    if (!build_grid(*grid, *vgrid, *gas, g->g, err) || (body && !place_body(*body, g->g, err))) {
      g_geom_err = err;
      delete g;
      return IBDVM_E_INVAL;
    }
    *out = g;
    return IBDVM_OK;
  } catch (const std::bad_alloc &) {
    g_geom_err = "host allocation failed";
    return IBDVM_E_NOMEM;
  }
}

static const Geom &G_of(const ibdvm_geom *g) { return reinterpret_cast<const Geom &>(*g); }

ibdvm_status ibdvm_geom_sizes(const ibdvm_geom *g, long long *s) {
  if (!g || !s) return IBDVM_E_INVAL;
  const Geom &G = G_of(g);
  s[0] = G.ncell;
  s[1] = G.nv;
  s[2] = G.ncomp;
  s[3] = static_cast<long long>(G.links.size());
  s[4] = static_cast<long long>(G.ghosts.size());
  s[5] = G.nfluid;
  s[6] = static_cast<long long>(G.surf_cell.size());
  s[7] = G.nvp;
  return IBDVM_OK;
}

ibdvm_status ibdvm_geom_cells(const ibdvm_geom *g, unsigned char *types) {
  if (!g || !types) return IBDVM_E_INVAL;
  const Geom &G = G_of(g);
  std::copy(G.type.begin(), G.type.end(), types);
  return IBDVM_OK;
}

ibdvm_status ibdvm_geom_links(const ibdvm_geom *g, int *ghost, int *donor, int *aux, int *axis,
                              int *side, double *xw, double *nw) {
  if (!g) return IBDVM_E_INVAL;
  const Geom &G = G_of(g);
  for (size_t l = 0; l < G.links.size(); ++l) {
    const Link &L = G.links[l];
    if (ghost) ghost[l] = L.ghost;
    if (donor) donor[l] = L.donor;
    if (aux) aux[l] = L.aux;
    if (axis) axis[l] = L.axis;
    if (side) side[l] = L.side;
    for (int a = 0; a < 3; ++a) {
      if (xw) xw[3 * l + a] = L.xw[a];
      if (nw) nw[3 * l + a] = L.nw[a];
    }
  }
  return IBDVM_OK;
}

ibdvm_status ibdvm_geom_cut_table(const ibdvm_geom *g, double *wg) {
  if (!g || !wg) return IBDVM_E_INVAL;
  const Geom &G = G_of(g);
  std::copy(G.wg.begin(), G.wg.end(), wg);
  return IBDVM_OK;
}

ibdvm_status ibdvm_geom_velocities(const ibdvm_geom *g, double *xi, double *w) {
  if (!g) return IBDVM_E_INVAL;
  const Geom &G = G_of(g);
  if (xi) std::copy(G.xi.begin(), G.xi.end(), xi);
  if (w) std::copy(G.w.begin(), G.w.end(), w);
  return IBDVM_OK;
}

ibdvm_status ibdvm_geom_surface(const ibdvm_geom *g, int *ghost_cell, int *offsets, int *cells) {
  if (!g) return IBDVM_E_INVAL;
  const Geom &G = G_of(g);
  if (ghost_cell) std::copy(G.ghosts.begin(), G.ghosts.end(), ghost_cell);
  if (offsets) std::copy(G.surf_off.begin(), G.surf_off.end(), offsets);
  if (cells) std::copy(G.surf_cell.begin(), G.surf_cell.end(), cells);
  return IBDVM_OK;
}

double ibdvm_geom_dt(const ibdvm_geom *g) { return g ? G_of(g).dt : 0.0; }

void ibdvm_geom_destroy(ibdvm_geom *g) { delete g; }

const char *ibdvm_geom_last_error(void) { return g_geom_err.c_str(); }

} // extern "C"

namespace ibdvm {
size_t estimate_ctx_bytes(const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid, const ibdvm_gas_desc *gas) {
  Geom G;
  std::string err;
  if (!build_grid(*grid, *vgrid, *gas, G, err)) return 0;
  const size_t es = (gas->precision == IBDVM_FP64) ? 8 : 4;
  size_t nvp = static_cast<size_t>(G.nvp);
  if (gas->precision == IBDVM_MIXED) { // the orthant layout of the TMA sweeps
    std::vector<int> kst;
    int np = 0;
    if (orthant_layout(G, kst, np) > 0) nvp = std::max(nvp, static_cast<size_t>(np));
  }
  const size_t nc = static_cast<size_t>(G.ncell);
  const int D = G.dim, NW = D + 2, NM = nmoments(D);
  size_t b = 2 * nc * nvp * G.ncomp * es;                               // f^n, f^{n+1}
  b += nc * (nvp / 64 + 1) * 4 * NM;                                     // FP32 moment partial sums
  b += nc * (kMac * es + 2 * (NW + D) * 8 + (nvp / 64 + 1) * NM * 8 + 16); // per-cell state, FP64 sums
  // the ghost band: at most D n^(D-1) links for a body that fits the domain
  const double nl = D * std::pow(static_cast<double>(nc), (D - 1.0) / D);
  b += static_cast<size_t>(nl) * (nvp * (3 * G.ncomp * es + 8) + 256);
  return b + nvp * 64 + (1u << 20);
}

void force_outputs(const ibdvm_ctx *ctx, const double *h, double *F, double *Q, double *CD, double *CL) {
  fill_forces(const_cast<ibdvm_ctx *>(ctx), h, F, Q, CD, CL);
}
} // namespace ibdvm
