// batch.cpp -- the batched form of the C-ABI (declared in include/ibdvm.h).
//
// A batch advances many FP32 contexts of uneven size (all 2D or all 3D) with
// one launch per kernel class and step: the grouped ghost-band, force and
// finalize kernels (kernels.cu) and the persistent TMA sweep over a packed
// work list (sweep_tma.cu, sweep3d_tma.cu).  The batch keeps per-member device tables with two argument
// blocks each (the buffer parities after an even and an odd number of steps),
// rebuilt when the membership, a member's body or the tiling changes, and
// replays pairs of steps from captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"

using namespace ibdvm;

struct ibdvm_batch {
  cudaStream_t stream = nullptr;
  std::vector<ibdvm_ctx *> members;
  std::vector<unsigned> gens;   // members' body_gen at the last table build
  std::vector<char> stepped;    // member has stepped in this batch
  bool dirty = true;
  int par = 0;                  // steps since the tables were built, mod 2
  int rows = 0, kpt = 0;        // tiling of the sweep's work items (kpt: kept, no effect)
  GroupTables gt;
  SweepTables st;
  double *d_res = nullptr;      // [cap] residual of each member's last step
  int *d_flags = nullptr;       // [cap] flags of each member
  double *d_forces = nullptr;   // [cap][4] step forces of each member
  int cap = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  long long graph_launches[2][8] = {};
  bool graphs_enabled = true;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> marks;
  double kernel_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long kernel_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::string err;
};

namespace {

struct BFail {
  ibdvm_status st;
};

void bcheck(ibdvm_batch *b, cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
    throw BFail{IBDVM_E_CUDA};
  }
}

void drop_graphs(ibdvm_batch *b) {
  for (int i = 0; i < 2; ++i) {
    if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
    b->graph[i] = nullptr;
  }
}

void harvest(ibdvm_batch *b) {
  for (const auto &m : b->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev_pool[m.second], b->ev_pool[m.second + 1]) == cudaSuccess)
      b->kernel_ms[m.first] += ms;
  }
  cudaGetLastError();
  b->marks.clear();
  b->ev_used = 0;
}

void bsync(ibdvm_batch *b, const char *what) {
  bcheck(b, cudaStreamSynchronize(b->stream), what);
  harvest(b);
}

// CUDA events around one launch class while profiling
struct BTimed {
  ibdvm_batch *b;
  int cls;
  size_t start = 0;
  bool on;
  BTimed(ibdvm_batch *bb, int k) : b(bb), cls(k), on(bb->profiling) {
    if (!on) return;
    if (b->ev_used + 2 > b->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          on = false;
          return;
        }
        b->ev_pool.push_back(e);
      }
    }
    start = b->ev_used;
    b->ev_used += 2;
    cudaEventRecord(b->ev_pool[start], b->stream);
  }
  ~BTimed() {
    if (!on) return;
    cudaEventRecord(b->ev_pool[start + 1], b->stream);
    b->marks.emplace_back(cls, start);
  }
};

void free_tables(ibdvm_batch *b) {
  group_free(b->gt);
  tma_batch_free(b->st);
}

void ensure_capacity(ibdvm_batch *b) {
  const int n = static_cast<int>(b->members.size());
  if (n <= b->cap) return;
  const int cap = std::max(n, std::max(16, 2 * b->cap));
  if (b->d_res) cudaFree(b->d_res);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->d_forces) cudaFree(b->d_forces);
  b->d_res = nullptr;
  b->d_flags = nullptr;
  b->d_forces = nullptr;
  b->cap = 0;
  void *p = nullptr;
  bcheck(b, cudaMalloc(&p, cap * sizeof(double)), "allocate batch residuals");
  b->d_res = static_cast<double *>(p);
  bcheck(b, cudaMalloc(&p, cap * sizeof(int)), "allocate batch flags");
  b->d_flags = static_cast<int *>(p);
  bcheck(b, cudaMalloc(&p, 4 * cap * sizeof(double)), "allocate batch forces");
  b->d_forces = static_cast<double *>(p);
  bcheck(b, cudaMemsetAsync(b->d_forces, 0, 4 * cap * sizeof(double), b->stream), "clear batch forces");
  b->cap = cap;
}

// velocities per lane of a member's sweep: those of its orthant layout's chunk
int member_kpt(const ibdvm_ctx *ctx) { return tma_batch_kpt_max(ctx); }

// (re)builds the device tables when the membership, a body or the tiling changed
void build(ibdvm_batch *b) {
  const size_t n = b->members.size();
  bool stale = b->dirty || b->gens.size() != n;
  for (size_t i = 0; !stale && i < n; ++i) stale = b->gens[i] != b->members[i]->body_gen;
  if (!stale) return;
  bsync(b, "drain before rebuilding the batch tables");
  drop_graphs(b);
  free_tables(b);
  ensure_capacity(b);
  std::vector<int> kpt(n), nchunk(n);
  for (size_t i = 0; i < n; ++i) {
    kpt[i] = member_kpt(b->members[i]);
    nchunk[i] = b->members[i]->tma_nchunk;
  }
  bcheck(b, group_build(b->members, nchunk, b->d_res, b->d_flags, b->d_forces, b->gt, b->stream),
         "build the grouped launch tables");
  bcheck(b, tma_batch_build(b->members, kpt, b->rows, b->d_flags, b->st, b->stream), "build the sweep work list");
  // member indices may have moved: the step forces start over
  bcheck(b, cudaMemsetAsync(b->d_forces, 0, 4 * b->cap * sizeof(double), b->stream), "clear batch forces");
  std::fill(b->stepped.begin(), b->stepped.end(), 0);
  b->gens.resize(n);
  for (size_t i = 0; i < n; ++i) b->gens[i] = b->members[i]->body_gen;
  b->par = 0;
  b->dirty = false;
}

// one batched step at parity p: ghost band on f^n, the forces of the fluxes
// the step applies, transport / relaxation / moments, finalize and residual
void one_step(ibdvm_batch *b, int p) {
  {
    BTimed t(b, kKGhost);
    bcheck(b, group_ghost(b->gt, p, b->stream), "grouped ghost-band kernel");
    b->kernel_launches[kKGhost] += b->gt.link_blocks ? 1 : 0;
  }
  {
    BTimed t(b, kKForces);
    bcheck(b, group_forces(b->gt, p, b->stream), "grouped force kernels");
    b->kernel_launches[kKForces] += (b->gt.link_blocks ? 1 : 0) + 1;
  }
  {
    BTimed t(b, kKSweep);
    bcheck(b, tma_batch_launch(b->st, p, b->stream), "batched sweep kernel");
    int nl = 0; // 2D: one launch per chunk width present; 3D: one
    for (int c = 0; c < 3; ++c) nl += (b->st.cls_off[c + 1] > b->st.cls_off[c]) ? 1 : 0;
    b->kernel_launches[kKSweep] += (b->st.dim == 3) ? (b->st.nitems ? 1 : 0) : nl;
  }
  {
    BTimed t(b, kKMoments);
    bcheck(b, group_finalize(b->gt, p, b->stream), "grouped finalize kernels");
    b->kernel_launches[kKMoments] += 2;
  }
}

// enqueues nsteps steps (no synchronisation, except a table rebuild)
void advance(ibdvm_batch *b, int nsteps) {
  build(b);
  int done = 0;
  if (nsteps >= 2 && b->graphs_enabled && !b->profiling && b->stream != nullptr) {
    const int key = b->par;
    if (!b->graph[key]) {
      long long before[8];
      for (int i = 0; i < 8; ++i) before[i] = b->kernel_launches[i];
      cudaGraph_t g = nullptr;
      bcheck(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin graph capture");
      try {
        one_step(b, key);
        one_step(b, key ^ 1);
      } catch (const BFail &) {
        cudaStreamEndCapture(b->stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      bcheck(b, cudaStreamEndCapture(b->stream, &g), "end graph capture");
      cudaError_t e = cudaGraphInstantiate(&b->graph[key], g, 0);
      cudaGraphDestroy(g);
      bcheck(b, e, "instantiate batch step graph");
      for (int i = 0; i < 8; ++i) {
        b->graph_launches[key][i] = b->kernel_launches[i] - before[i];
        b->kernel_launches[i] = before[i];
      }
    }
    for (; done + 2 <= nsteps; done += 2) {
      bcheck(b, cudaGraphLaunch(b->graph[key], b->stream), "replay batch step graph");
      for (int i = 0; i < 8; ++i) b->kernel_launches[i] += b->graph_launches[key][i];
    }
  }
  for (; done < nsteps; ++done) {
    one_step(b, b->par);
    b->par ^= 1;
    if (b->ev_used > 4096) bsync(b, "batch step");
  }
  for (ibdvm_ctx *ctx : b->members) {
    ctx->cur ^= (nsteps & 1);
    ctx->wcur ^= (nsteps & 1);
    ctx->steps += nsteps;
  }
  std::fill(b->stepped.begin(), b->stepped.end(), 1);
}

ibdvm_status member_status(ibdvm_batch *b, int fl, int m) {
  const std::string who = "member " + std::to_string(m) + ": ";
  if (fl & kFlagTimeout) {
    b->err = who + "a bounded device wait in the sweep gave up (TMA copy did not arrive)";
    return IBDVM_E_TIMEOUT;
  }
  if (fl & kFlagNonFinite) {
    b->err = who + "non-finite or non-positive density or temperature";
    return IBDVM_E_NONFINITE;
  }
  if (fl & kFlagUnstable) {
    b->err = who + "dt / tau > 1: the explicit relaxation is unstable at this time step";
    return IBDVM_E_UNSTABLE;
  }
  return IBDVM_OK;
}

// reads residuals and flags after the enqueued steps
ibdvm_status collect(ibdvm_batch *b, double *residuals, int *statuses) {
  const int n = static_cast<int>(b->members.size());
  std::vector<double> res(n, 0.0);
  std::vector<int> fl(n, 0);
  if (n) {
    bcheck(b, cudaMemcpyAsync(res.data(), b->d_res, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
           "read residuals");
    bcheck(b, cudaMemcpyAsync(fl.data(), b->d_flags, n * sizeof(int), cudaMemcpyDeviceToHost, b->stream),
           "read flags");
  }
  bsync(b, "batch step");
  ibdvm_status first = IBDVM_OK;
  std::string first_err;
  for (int m = 0; m < n; ++m) {
    ibdvm_status st = member_status(b, fl[m], m);
    if (st == IBDVM_OK && !std::isfinite(res[m])) {
      b->err = "member " + std::to_string(m) + ": non-finite residual";
      st = IBDVM_E_NONFINITE;
    }
    if (st != IBDVM_OK && first == IBDVM_OK) {
      first = st;
      first_err = b->err;
    }
    if (residuals) residuals[m] = res[m];
    if (statuses) statuses[m] = st;
  }
  b->err = first_err;
  return first;
}

#define BATCH_GUARD(b)                                                                              \
  if (!(b)) return IBDVM_E_INVAL;                                                                   \
  (b)->err.clear();                                                                                 \
  try {
#define BATCH_END                                                                                   \
  }                                                                                                 \
  catch (const BFail &f) {                                                                          \
    return f.st;                                                                                    \
  }                                                                                                 \
  catch (const std::bad_alloc &) {                                                                  \
    b->err = "host allocation failed";                                                              \
    return IBDVM_E_NOMEM;                                                                           \
  }

} // namespace

namespace ibdvm {
void batch_detach(ibdvm_ctx *ctx) {
  ibdvm_batch *b = ctx->batch;
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i] == ctx) {
      b->members.erase(b->members.begin() + i);
      b->stepped.erase(b->stepped.begin() + i);
      break;
    }
  ctx->batch = nullptr;
  b->dirty = true;
  drop_graphs(b);
}
} // namespace ibdvm

namespace ibdvm {
ibdvm_status batch_enqueue(ibdvm_batch *b, int nsteps) {
  BATCH_GUARD(b)
  if (b->members.empty() || nsteps <= 0) return IBDVM_OK;
  build(b);
  bcheck(b, cudaMemsetAsync(b->d_flags, 0, b->members.size() * sizeof(int), b->stream), "clear flags");
  advance(b, nsteps);
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status batch_collect(ibdvm_batch *b, double *residuals, int *statuses) {
  BATCH_GUARD(b)
  return collect(b, residuals, statuses);
  BATCH_END
}
} // namespace ibdvm

extern "C" {

ibdvm_status ibdvm_batch_create(void *cuda_stream, ibdvm_batch **out) {
  if (!out) return IBDVM_E_INVAL;
  *out = nullptr;
  ibdvm_batch *b = new (std::nothrow) ibdvm_batch();
  if (!b) return IBDVM_E_NOMEM;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = b;
  return IBDVM_OK;
}

ibdvm_status ibdvm_batch_add(ibdvm_batch *b, ibdvm_ctx *ctx) {
  BATCH_GUARD(b)
  if (!ctx) {
    b->err = "context is NULL";
    return IBDVM_E_INVAL;
  }
  if (ctx->batch) {
    b->err = "the context is already a member of a batch";
    return IBDVM_E_STATE;
  }
  if (!ctx->use_tma || !tma_batch_member_ok(ctx) || ctx->wall_mask) {
    b->err = "batch members are contexts in FP32 storage with the TMA sweep (no diffuse domain walls)";
    return IBDVM_E_INVAL;
  }
  if (!b->members.empty() && b->members[0]->dim != ctx->dim) {
    b->err = "the members of a batch have one dimension";
    return IBDVM_E_INVAL;
  }
  if (ctx->stream != b->stream) {
    b->err = "the context is bound to another stream than the batch";
    return IBDVM_E_INVAL;
  }
  b->members.push_back(ctx);
  b->stepped.push_back(0);
  ctx->batch = b;
  b->dirty = true;
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status ibdvm_batch_remove(ibdvm_batch *b, ibdvm_ctx *ctx) {
  BATCH_GUARD(b)
  if (!ctx || ctx->batch != b) {
    b->err = "the context is not a member of this batch";
    return IBDVM_E_INVAL;
  }
  batch_detach(ctx);
  return IBDVM_OK;
  BATCH_END
}

int ibdvm_batch_size(const ibdvm_batch *b) { return b ? static_cast<int>(b->members.size()) : -1; }

ibdvm_ctx *ibdvm_batch_member(const ibdvm_batch *b, int i) {
  if (!b || i < 0 || i >= static_cast<int>(b->members.size())) return nullptr;
  return b->members[i];
}

ibdvm_status ibdvm_batch_step(ibdvm_batch *b, int nsteps, double *residuals, int *statuses) {
  BATCH_GUARD(b)
  if (nsteps < 0) {
    b->err = "nsteps must be >= 0";
    return IBDVM_E_INVAL;
  }
  if (b->members.empty() || nsteps == 0) {
    for (size_t m = 0; m < b->members.size(); ++m) {
      if (residuals) residuals[m] = 0.0;
      if (statuses) statuses[m] = IBDVM_OK;
    }
    return IBDVM_OK;
  }
  build(b);
  bcheck(b, cudaMemsetAsync(b->d_flags, 0, b->members.size() * sizeof(int), b->stream), "clear flags");
  advance(b, nsteps);
  return collect(b, residuals, statuses);
  BATCH_END
}

ibdvm_status ibdvm_batch_forces(ibdvm_batch *b, double *F, double *Q, double *CD, double *CL) {
  BATCH_GUARD(b)
  const int n = static_cast<int>(b->members.size());
  std::vector<double> h(4 * static_cast<size_t>(n), 0.0);
  if (n && b->d_forces && b->cap >= n) {
    bcheck(b, cudaMemcpyAsync(h.data(), b->d_forces, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
           "read forces");
    bsync(b, "read forces");
  }
  for (int m = 0; m < n; ++m) {
    double z[4] = {0, 0, 0, 0};
    const double *hm = b->stepped[m] ? &h[4 * m] : z;
    force_outputs(b->members[m], hm, F ? F + 3 * m : nullptr, Q ? Q + m : nullptr, CD ? CD + m : nullptr,
                  CL ? CL + m : nullptr);
  }
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status ibdvm_batch_set_tiling(ibdvm_batch *b, int rows, int kpt) {
  BATCH_GUARD(b)
  if (rows < 0 || !(kpt == 0 || kpt == 2 || kpt == 4)) {
    b->err = "rows must be >= 0 and kpt one of 0, 2, 4";
    return IBDVM_E_INVAL;
  }
  b->kpt = kpt; // no effect: every member takes the chunk of its velocity layout
  if (rows != b->rows) {
    b->rows = rows;
    b->dirty = true;
  }
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status ibdvm_batch_get_tiling(const ibdvm_batch *b, ibdvm_batch_tiling *out) {
  if (!b || !out) return IBDVM_E_INVAL;
  out->rows = b->rows;
  out->kpt = b->members.empty() ? 0 : member_kpt(b->members[0]);
  out->nitems = b->dirty ? 0 : b->st.nitems;
  out->grid = b->dirty ? 0 : b->st.grid;
  out->graphs = (b->graphs_enabled && !b->profiling && b->stream != nullptr) ? 1 : 0;
  return IBDVM_OK;
}

ibdvm_status ibdvm_batch_tune(ibdvm_batch *b, int steps_per_trial, double *best_ms) {
  BATCH_GUARD(b)
  if (steps_per_trial < 2 || (steps_per_trial & 1)) {
    b->err = "steps_per_trial must be even and >= 2";
    return IBDVM_E_INVAL;
  }
  if (b->members.empty()) {
    b->err = "the batch has no members";
    return IBDVM_E_STATE;
  }
  const int rows_c[5] = {16, 32, 64, 128, 0};
  cudaEvent_t e0, e1;
  bcheck(b, cudaEventCreate(&e0), "create event");
  bcheck(b, cudaEventCreate(&e1), "create event");
  double best = 1e300;
  int best_rows = b->rows;
  ibdvm_status st = IBDVM_OK;
  try {
    for (int r : rows_c) {
      b->rows = r;
      b->dirty = true;
      build(b);
      bcheck(b, cudaMemsetAsync(b->d_flags, 0, b->members.size() * sizeof(int), b->stream), "clear flags");
      advance(b, 2); // warm-up pair: captures the graphs of this tiling
      bcheck(b, cudaEventRecord(e0, b->stream), "record event");
      advance(b, steps_per_trial);
      bcheck(b, cudaEventRecord(e1, b->stream), "record event");
      st = collect(b, nullptr, nullptr);
      if (st != IBDVM_OK) throw BFail{st};
      float ms = 0.f;
      bcheck(b, cudaEventElapsedTime(&ms, e0, e1), "event time");
      const double per = ms / steps_per_trial;
      if (per < best) {
        best = per;
        best_rows = r;
      }
    }
  } catch (const BFail &) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->rows = best_rows;
  b->dirty = true;
  build(b);
  if (best_ms) *best_ms = best;
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status ibdvm_batch_set_profiling(ibdvm_batch *b, int on) {
  BATCH_GUARD(b)
  bsync(b, "drain");
  b->profiling = on != 0;
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status ibdvm_batch_get_kernel_times(ibdvm_batch *b, double *ms, long long *launches) {
  BATCH_GUARD(b)
  bsync(b, "kernel times");
  for (int i = 0; i < 8; ++i) {
    if (ms) ms[i] = b->kernel_ms[i];
    if (launches) launches[i] = b->kernel_launches[i];
  }
  return IBDVM_OK;
  BATCH_END
}

ibdvm_status ibdvm_batch_reset_kernel_times(ibdvm_batch *b) {
  BATCH_GUARD(b)
  bsync(b, "kernel times");
  for (int i = 0; i < 8; ++i) {
    b->kernel_ms[i] = 0.0;
    b->kernel_launches[i] = 0;
  }
  return IBDVM_OK;
  BATCH_END
}

void ibdvm_batch_destroy(ibdvm_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (ibdvm_ctx *ctx : b->members) ctx->batch = nullptr;
  b->members.clear();
  drop_graphs(b);
  free_tables(b);
  if (b->d_res) cudaFree(b->d_res);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->d_forces) cudaFree(b->d_forces);
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
  delete b;
}

const char *ibdvm_batch_last_error(const ibdvm_batch *b) { return b ? b->err.c_str() : "batch is NULL"; }

} // extern "C"
