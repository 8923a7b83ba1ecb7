// server.cpp -- the serving loop of the C-ABI (declared in include/ibdvm.h).
//
// Requests are queued on submission and admitted first come first served
// while the device bytes of the admitted cases stay within the HBM budget.
// An admitted request is a context in FP32 storage that joins the 2D or the
// 3D batch (two streams, so the two batches' launches overlap on the device);
// a poll enqueues a round of steps on both batches before it waits for
// either, then retires converged, failed and capped requests, freeing their
// memory for the queue.  In the sequential FP64 mode one request at a time
// runs alone in the FP64 path (the plain form the batched one is compared
// with).  Contexts that cannot join a batch step alone after the batches are
// enqueued.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "ctx.h"

using namespace ibdvm;

namespace {

struct Req {
  long long id = 0;
  ibdvm_grid_desc grid{};
  ibdvm_vgrid_desc vgrid{};
  ibdvm_gas_desc gas{};
  ibdvm_body_desc body{};
  bool has_body = false;
  std::vector<double> verts;
  std::vector<double> vnodes[3]; // velocity nodes of IBDVM_RULE_NODES (the request owns a copy)
  ibdvm_ctx *ctx = nullptr;
  bool batched = false;
  size_t bytes = 0;
  ibdvm_result r{};
};

} // namespace

struct ibdvm_server {
  ibdvm_server_desc d{};
  cudaStream_t stream[2] = {nullptr, nullptr}; // 2D, 3D
  ibdvm_batch *batch[2] = {nullptr, nullptr};
  std::deque<Req *> queue;
  std::vector<Req *> active;
  std::unordered_map<long long, Req *> all;
  long long next_id = 0;
  size_t used = 0, budget = 0;
  std::chrono::steady_clock::time_point t0;
  std::string err;
};

namespace {

double now(const ibdvm_server *s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void release(ibdvm_server *s, Req *q) {
  if (!q->ctx) return;
  if (q->batched) ibdvm_batch_remove(s->batch[q->grid.dim == 3 ? 1 : 0], q->ctx);
  ibdvm_destroy(q->ctx);
  q->ctx = nullptr;
  q->batched = false;
  s->used -= std::min(s->used, q->bytes);
}

// final outputs of a request and its release
void finish(ibdvm_server *s, Req *q, int status) {
  q->r.status = status;
  if (q->ctx && (status == IBDVM_OK || status == IBDVM_E_NOTCONVERGED)) {
    double F[3] = {0, 0, 0}, Q = 0, CD = 0, CL = 0;
    if (ibdvm_forces(q->ctx, F, &Q, &CD, &CL) == IBDVM_OK) {
      for (int a = 0; a < 3; ++a) q->r.F[a] = F[a];
      q->r.Q = Q;
      q->r.CD = CD;
      q->r.CL = CL;
    }
  }
  release(s, q);
  q->r.done = 1;
  q->r.t_done = now(s);
}

// admits queued requests while the budget and the cap allow; returns the
// number of requests that failed at admission (retired at once)
int admit(ibdvm_server *s) {
  int failed = 0;
  while (!s->queue.empty()) {
    if (s->d.sequential_fp64 && !s->active.empty()) break;
    if (s->d.max_active > 0 && static_cast<int>(s->active.size()) >= s->d.max_active) break;
    Req *q = s->queue.front();
    const size_t est = estimate_ctx_bytes(&q->grid, &q->vgrid, &q->gas);
    if (!s->active.empty() && s->used + est > s->budget) break; // wait for memory to free up
    s->queue.pop_front();
    const int di = q->grid.dim == 3 ? 1 : 0;
    ibdvm_ctx *ctx = nullptr;
    ibdvm_status st = ibdvm_create_grid(&q->grid, &q->vgrid, &q->gas, s->stream[di], &ctx);
    if (st == IBDVM_E_NOMEM && !s->active.empty()) { // retry when a request has left
      s->queue.push_front(q);
      break;
    }
    q->r.t_admit = now(s);
    if (st != IBDVM_OK) {
      q->r.status = st;
      q->r.done = 1;
      q->r.t_done = now(s);
      ++failed;
      continue;
    }
    q->ctx = ctx;
    if (q->has_body) {
      q->body.verts = q->verts.empty() ? nullptr : q->verts.data();
      st = ibdvm_set_body(ctx, &q->body);
      if (st != IBDVM_OK) {
        finish(s, q, st);
        ++failed;
        continue;
      }
    }
    q->bytes = ctx->dev_bytes;
    s->used += q->bytes;
    q->r.device_bytes = q->bytes;
    if (!s->d.sequential_fp64 && ibdvm_batch_add(s->batch[di], ctx) == IBDVM_OK) q->batched = true;
    s->active.push_back(q);
  }
  return failed;
}

} // namespace

extern "C" {

ibdvm_status ibdvm_server_create(const ibdvm_server_desc *desc, ibdvm_server **out) {
  if (!out) return IBDVM_E_INVAL;
  *out = nullptr;
  if (!desc || !(desc->tol >= 0.0) || desc->max_steps < 1 || desc->steps_per_round < 2 ||
      (desc->steps_per_round & 1) || desc->max_active < 0)
    return IBDVM_E_INVAL;
  ibdvm_server *s = new (std::nothrow) ibdvm_server();
  if (!s) return IBDVM_E_NOMEM;
  s->d = *desc;
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < 2; ++i) {
    if (cudaStreamCreateWithFlags(&s->stream[i], cudaStreamNonBlocking) != cudaSuccess ||
        ibdvm_batch_create(s->stream[i], &s->batch[i]) != IBDVM_OK) {
      cudaGetLastError();
      ibdvm_server_destroy(s);
      return IBDVM_E_CUDA;
    }
  }
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) {
    cudaGetLastError();
    ibdvm_server_destroy(s);
    return IBDVM_E_CUDA;
  }
  s->budget = desc->hbm_budget ? desc->hbm_budget : static_cast<size_t>(0.9 * static_cast<double>(freeb));
  *out = s;
  return IBDVM_OK;
}

ibdvm_status ibdvm_server_submit(ibdvm_server *s, const ibdvm_grid_desc *grid, const ibdvm_vgrid_desc *vgrid,
                                 const ibdvm_gas_desc *gas, const ibdvm_body_desc *body, long long *id) {
  if (!s) return IBDVM_E_INVAL;
  s->err.clear();
  if (!grid || !vgrid || !gas) {
    s->err = "grid, velocity grid and gas are required";
    return IBDVM_E_INVAL;
  }
  try {
    Req *q = new Req();
    q->grid = *grid;
    q->vgrid = *vgrid;
    q->gas = *gas;
    if (vgrid->rule == IBDVM_RULE_NODES)
      for (int a = 0; a < grid->dim && a < 3; ++a) {
        if (vgrid->nodes[a] && vgrid->n[a] > 0) q->vnodes[a].assign(vgrid->nodes[a], vgrid->nodes[a] + vgrid->n[a]);
        q->vgrid.nodes[a] = q->vnodes[a].empty() ? nullptr : q->vnodes[a].data();
      }
    q->gas.precision = s->d.sequential_fp64 ? IBDVM_FP64 : IBDVM_MIXED;
    if (estimate_ctx_bytes(&q->grid, &q->vgrid, &q->gas) == 0) {
      delete q;
      s->err = "invalid grid, velocity grid or gas descriptor";
      return IBDVM_E_INVAL;
    }
    if (body && body->kind != IBDVM_BODY_NONE) {
      q->body = *body;
      q->has_body = true;
      if (body->verts && body->nverts > 0) q->verts.assign(body->verts, body->verts + 2 * body->nverts);
    }
    q->id = s->next_id++;
    q->r.id = q->id;
    q->r.t_submit = now(s);
    q->r.t_admit = -1.0;
    q->r.t_done = -1.0;
    s->all[q->id] = q;
    s->queue.push_back(q);
    if (id) *id = q->id;
  } catch (const std::bad_alloc &) {
    s->err = "host allocation failed";
    return IBDVM_E_NOMEM;
  }
  return IBDVM_OK;
}

ibdvm_status ibdvm_server_poll(ibdvm_server *s, int *nactive, int *nqueued, int *nfinished) {
  if (!s) return IBDVM_E_INVAL;
  s->err.clear();
  int finished = admit(s);
  const int k = s->d.steps_per_round;
  // enqueue both batches before waiting for either
  for (int i = 0; i < 2; ++i) {
    ibdvm_status st = batch_enqueue(s->batch[i], k);
    if (st != IBDVM_OK) {
      s->err = std::string("batch step: ") + ibdvm_batch_last_error(s->batch[i]);
      return st;
    }
  }
  // requests that step alone (sequential mode, or a context that cannot join a batch)
  for (Req *q : s->active) {
    if (q->batched) continue;
    double res = 0.0;
    ibdvm_status st = ibdvm_step(q->ctx, k, &res);
    q->r.steps += k;
    q->r.residual = res;
    if (st != IBDVM_OK) {
      finish(s, q, st);
      ++finished;
    }
  }
  for (int i = 0; i < 2; ++i) {
    const int n = ibdvm_batch_size(s->batch[i]);
    std::vector<double> res(std::max(n, 1));
    std::vector<int> sts(std::max(n, 1));
    ibdvm_status st = batch_collect(s->batch[i], res.data(), sts.data());
    if (st == IBDVM_E_CUDA) {
      s->err = std::string("batch step: ") + ibdvm_batch_last_error(s->batch[i]);
      return st;
    }
    std::vector<ibdvm_ctx *> members(n);
    for (int m = 0; m < n; ++m) members[m] = ibdvm_batch_member(s->batch[i], m);
    for (Req *q : s->active) {
      if (!q->batched || (q->grid.dim == 3) != (i == 1)) continue;
      for (int m = 0; m < n; ++m)
        if (members[m] == q->ctx) {
          q->r.steps += k;
          q->r.residual = res[m];
          if (sts[m] != IBDVM_OK) {
            finish(s, q, sts[m]);
            ++finished;
          }
          break;
        }
    }
  }
  // convergence and the step cap
  for (Req *q : s->active) {
    if (q->r.done) continue;
    if (q->r.residual < s->d.tol) {
      finish(s, q, IBDVM_OK);
      ++finished;
    } else if (q->r.steps >= s->d.max_steps) {
      finish(s, q, IBDVM_E_NOTCONVERGED);
      ++finished;
    }
  }
  s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](Req *q) { return q->r.done != 0; }),
                  s->active.end());
  if (nactive) *nactive = static_cast<int>(s->active.size());
  if (nqueued) *nqueued = static_cast<int>(s->queue.size());
  if (nfinished) *nfinished = finished;
  return IBDVM_OK;
}

ibdvm_status ibdvm_server_cancel(ibdvm_server *s, long long id) {
  if (!s) return IBDVM_E_INVAL;
  s->err.clear();
  auto it = s->all.find(id);
  if (it == s->all.end()) {
    s->err = "unknown request id";
    return IBDVM_E_INVAL;
  }
  Req *q = it->second;
  if (q->r.done) return IBDVM_OK;
  auto qi = std::find(s->queue.begin(), s->queue.end(), q);
  if (qi != s->queue.end()) { // not admitted yet
    s->queue.erase(qi);
    q->r.status = IBDVM_E_STATE;
    q->r.done = 1;
    q->r.t_done = now(s);
    return IBDVM_OK;
  }
  // on the device: its batch is idle between polls, so it leaves at once
  finish(s, q, IBDVM_E_STATE);
  s->active.erase(std::remove(s->active.begin(), s->active.end(), q), s->active.end());
  return IBDVM_OK;
}

ibdvm_status ibdvm_server_result(ibdvm_server *s, long long id, ibdvm_result *out) {
  if (!s || !out) return IBDVM_E_INVAL;
  auto it = s->all.find(id);
  if (it == s->all.end()) {
    s->err = "unknown request id";
    return IBDVM_E_INVAL;
  }
  *out = it->second->r;
  return IBDVM_OK;
}

double ibdvm_server_clock(const ibdvm_server *s) { return s ? now(s) : 0.0; }

void ibdvm_server_destroy(ibdvm_server *s) {
  if (!s) return;
  for (Req *q : s->active) release(s, q);
  for (auto &kv : s->all) delete kv.second;
  for (int i = 0; i < 2; ++i) {
    if (s->batch[i]) ibdvm_batch_destroy(s->batch[i]);
    if (s->stream[i]) cudaStreamDestroy(s->stream[i]);
  }
  delete s;
}

const char *ibdvm_server_last_error(const ibdvm_server *s) { return s ? s->err.c_str() : "server is NULL"; }

} // extern "C"
