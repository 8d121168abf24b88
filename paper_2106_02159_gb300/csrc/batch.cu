// batch.cu -- continuous-batching solve server on one device (host code).
// Requests -- a mesh, an initial state and a final time each -- are admitted
// first come, first served while their device memory fits a budget next to
// the running ones, and their states stay resident on the device.
//
// Merged mode (the default): the running requests are the instances of ONE
// batched context (eh_set_instances on their block-diagonal union), so a step
// of the batch is one set of kernel launches -- one CUDA-graph replay -- for
// all of them, each request with its own CFL step and its own final time.
// Requests join and leave between eh_batch_advance calls: the union is rebuilt
// ("repacked") on the device from the requests' resident mesh data and current
// states by device-to-device copies, and a request that reached its final time
// stays frozen (tau = 0) until then.
//
// Per-request-stream mode (the comparison): every request keeps a context of
// its own on its own stream, and an advance launches one step of each request
// in turn, so that their launches overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "../../include/euler_hyp.h"
#include "internal.cuh"

namespace {

struct Slot {
  int64_t ticket;
  eh_ctx *ctx;       // merged mode: the request's mesh data and state; else its own full context
  uint64_t bytes;
  double t_final;
  double t;
  int64_t steps;       // steps taken with tau > 0
  int64_t steps_base;  // merged mode: steps taken before the current repack
  bool finished;     // reached t_final, or failed (status)
  bool in_union;     // merged mode: an instance of the batch's current context
  eh_status status;  // EH_OK, or the error that stopped the request
};

// device bytes of one context: the arrays eh_upload_mesh allocates per CSR
// entry and per node (static mesh data, per-stage work arrays, limiter and
// line-search queues), with 10% and 1 MiB of headroom
uint64_t estimate_bytes(int dim, int precision, int64_t n, int64_t nnz) {
  const int64_t S = dim + 2, SP = dim == 2 ? 4 : 6;
  int64_t per_entry = 4 + 4 + 8 * dim + 8 * 4 + 8 * SP * 2 + 8 * 3 + 8 + 5;
  int64_t per_node = 8 * (24 + 8 * SP + 3 * S + 13);
  if (precision == EH_PRECISION_MIXED) {
    per_entry += 4 * (dim + 2 + SP + 1);
    per_node += 4 * (40 + SP);
  }
  return (uint64_t)(1.1 * (double)(per_entry * nnz + per_node * n)) + (1u << 20);
}

}  // namespace

struct eh_batch {
  eh_config cfg;
  int mode = EH_BATCH_MERGED;
  uint64_t budget = 0, used = 0;
  int64_t next_ticket = 1;
  std::vector<Slot> slots;
  std::string err;
  // merged mode: the batch's context and whether its member set is stale
  eh_ctx *uni = nullptr;
  bool dirty = false;
  int64_t repacks = 0;
};

namespace {

eh_status bfail(eh_batch *b, eh_status st, const char *fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->err = buf;
  }
  return st;
}

Slot *find(eh_batch *b, int64_t ticket) {
  for (Slot &s : b->slots)
    if (s.ticket == ticket) return &s;
  return nullptr;
}

// the current members of the merged context, in order
std::vector<Slot *> members(eh_batch *b) {
  std::vector<Slot *> out;
  for (Slot &s : b->slots)
    if (s.in_union) out.push_back(&s);
  return out;
}

// merged mode: copies the members' states out of the batch's context and
// rebuilds it from the requests that still run (finished ones leave with
// their final state in their own buffers)
eh_status repack(eh_batch *b) {
  std::vector<Slot *> old = members(b);
  if (!old.empty()) {
    std::vector<eh_ctx *> parts;
    for (Slot *s : old) parts.push_back(s->ctx);
    const eh_status st = ehi::scatter(b->uni, parts.data(), (int)parts.size());
    if (st) return bfail(b, st, "repack (copy out): %s", eh_last_error(b->uni));
    for (Slot *s : old) {
      s->in_union = false;
      s->steps_base = s->steps;
    }
  }
  std::vector<eh_ctx *> parts;
  std::vector<double> t, tf;
  std::vector<Slot *> run;
  for (Slot &s : b->slots)
    if (!s.finished) {
      run.push_back(&s);
      parts.push_back(s.ctx);
      t.push_back(s.t);
      tf.push_back(s.t_final);
    }
  b->dirty = false;
  if (run.empty()) return EH_OK;
  const eh_status st = ehi::assemble(b->uni, parts.data(), (int)parts.size(), t.data(), tf.data());
  if (st) return bfail(b, st, "repack: %s", eh_last_error(b->uni));
  for (Slot *s : run) s->in_union = true;
  ++b->repacks;
  return EH_OK;
}

eh_status advance_merged(eh_batch *b, int32_t steps) {
  if (b->dirty) {
    const eh_status st = repack(b);
    if (st) return st;
  }
  std::vector<Slot *> mem = members(b);
  if (mem.empty()) return EH_OK;
  eh_status st = eh_run(b->uni, steps, 0.0);
  std::vector<double> t(mem.size(), 0.0);
  std::vector<int64_t> taken(mem.size(), 0);
  if (!st) st = eh_get_instances(b->uni, t.data(), nullptr, nullptr);  // synchronises
  if (!st) st = eh_get_instance_steps(b->uni, taken.data());
  if (st) {
    // one context steps every member: its failure stops all of them
    for (Slot *s : mem) {
      s->finished = true;
      s->status = st;
    }
    b->dirty = true;
    return EH_OK;
  }
  for (size_t k = 0; k < mem.size(); ++k) {
    Slot *s = mem[k];
    s->steps = s->steps_base + taken[k];
    s->t = t[k];
    if (t[k] >= s->t_final) {
      s->finished = true;
      b->dirty = true;  // it leaves at the next repack (frozen until then)
    }
  }
  return EH_OK;
}

eh_status advance_streams(eh_batch *b, int32_t steps) {
  // step by step over the running requests: each launch is asynchronous on
  // the request's own stream, so the requests overlap on the device
  for (int32_t k = 0; k < steps; ++k)
    for (Slot &s : b->slots) {
      if (s.finished) continue;
      const eh_status st = eh_run(s.ctx, 1, 0.0);
      if (st) {
        s.finished = true;
        s.status = st;
      }
    }
  for (Slot &s : b->slots) {
    if (s.finished) continue;
    double t = 0.0;
    eh_status st = eh_get_instances(s.ctx, &t, nullptr, nullptr);  // synchronises this request
    if (!st) st = eh_get_instance_steps(s.ctx, &s.steps);
    if (st) {
      s.finished = true;
      s.status = st;
    } else {
      s.t = t;
      if (t >= s.t_final) s.finished = true;
    }
  }
  return EH_OK;
}

}  // namespace

extern "C" {

eh_status eh_estimate_device_bytes(int32_t dim, int32_t precision, int32_t n, int64_t nnz, uint64_t *bytes) {
  if ((dim != 2 && dim != 3) || (precision != EH_PRECISION_FP64 && precision != EH_PRECISION_MIXED) || n < 1 ||
      nnz < n || !bytes)
    return EH_ERR_INVALID_ARG;
  *bytes = estimate_bytes(dim, precision, n, nnz);
  return EH_OK;
}

eh_status eh_estimate_request_bytes(int32_t dim, int32_t precision, int32_t mode, int32_t n, int64_t nnz,
                                    int32_t n_bnd, uint64_t *bytes) {
  if ((dim != 2 && dim != 3) || (precision != EH_PRECISION_FP64 && precision != EH_PRECISION_MIXED) || n < 1 ||
      nnz < n || n_bnd < 0 || !bytes || (mode != EH_BATCH_MERGED && mode != EH_BATCH_PER_REQUEST_STREAMS))
    return EH_ERR_INVALID_ARG;
  *bytes = estimate_bytes(dim, precision, n, nnz) +
           (mode == EH_BATCH_MERGED ? ehi::part_bytes(dim, precision, n, nnz, n_bnd) : 0);
  return EH_OK;
}

eh_status eh_batch_create(const eh_config *cfg, uint64_t hbm_budget_bytes, eh_batch **out) {
  if (!out) return EH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->stream || hbm_budget_bytes == 0) return EH_ERR_INVALID_ARG;
  // the batch's own context (merged mode) also checks the configuration
  eh_ctx *uni = nullptr;
  eh_status st = eh_create(cfg, &uni);
  if (st) return st;
  eh_batch *b = new (std::nothrow) eh_batch;
  if (!b) {
    eh_destroy(uni);
    return EH_ERR_OOM;
  }
  b->cfg = *cfg;
  b->budget = hbm_budget_bytes;
  b->uni = uni;
  *out = b;
  return EH_OK;
}

eh_status eh_batch_set_mode(eh_batch *b, int32_t mode) {
  if (!b) return EH_ERR_INVALID_ARG;
  if (mode != EH_BATCH_MERGED && mode != EH_BATCH_PER_REQUEST_STREAMS)
    return bfail(b, EH_ERR_INVALID_ARG, "unknown batch mode %d", mode);
  if (!b->slots.empty()) return bfail(b, EH_ERR_STATE, "the mode is set while the batch is empty");
  b->mode = mode;
  return EH_OK;
}

eh_status eh_batch_admit(eh_batch *b, int32_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                         const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                         const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                         const double *bnd_state, const double *U0, double t_final, int64_t *ticket) {
  if (!b) return EH_ERR_INVALID_ARG;
  if (!ticket || !U0 || !(t_final > 0.0) || n < 1 || nnz < n)
    return bfail(b, EH_ERR_INVALID_ARG, "invalid request arguments");
  const bool merged = b->mode == EH_BATCH_MERGED;
  // merged: the request's share of the batch context plus its own mesh copy
  uint64_t need = 0;
  if (eh_estimate_request_bytes(b->cfg.dim, b->cfg.precision, b->mode, n, nnz, n_bnd, &need))
    return bfail(b, EH_ERR_INVALID_ARG, "invalid request sizes");
  if (need > b->budget)
    return bfail(b, EH_ERR_INVALID_ARG, "request needs %llu bytes, more than the whole budget of %llu",
                 (unsigned long long)need, (unsigned long long)b->budget);
  if (b->used + need > b->budget)
    return bfail(b, EH_ERR_OOM, "request needs %llu bytes, %llu of %llu in use", (unsigned long long)need,
                 (unsigned long long)b->used, (unsigned long long)b->budget);
  size_t free_b = 0, total_b = 0;
  if (cudaSetDevice(b->cfg.device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, EH_ERR_CUDA, "cudaMemGetInfo failed");
  }
  if (need > free_b)
    return bfail(b, EH_ERR_OOM, "request needs %llu bytes, %llu free on the device", (unsigned long long)need,
                 (unsigned long long)free_b);
  eh_ctx *c = nullptr;
  eh_status st;
  if (merged) {
    st = ehi::create_part(&b->cfg, ehi::stream_of(b->uni), n, nnz, row_ptr, col, cij, mij, mi, n_bnd, bnd_node,
                          bnd_kind, bnd_normal, bnd_state, U0, &c);
    if (st) return bfail(b, st, "request not admitted: %s", eh_status_string(st));
  } else {
    st = eh_create(&b->cfg, &c);
    if (st) return bfail(b, st, "eh_create: %s", eh_status_string(st));
    const int64_t off[2] = {0, n};
    if (!st) st = eh_upload_mesh(c, n, nnz, row_ptr, col, cij, mij, mi, n_bnd, bnd_node, bnd_kind, bnd_normal,
                                 bnd_state);
    if (!st) st = eh_set_instances(c, 1, off, &t_final);
    if (!st) st = eh_set_state(c, U0, 0);
    if (!st) st = eh_apply_boundary_conditions(c);
    if (st) {
      bfail(b, st, "request not admitted: %s", eh_last_error(c));
      eh_destroy(c);
      return st;
    }
  }
  Slot s{};
  s.ticket = b->next_ticket++;
  s.ctx = c;
  s.bytes = need;
  s.t_final = t_final;
  s.status = EH_OK;
  b->slots.push_back(s);
  b->used += need;
  b->dirty = true;
  *ticket = s.ticket;
  return EH_OK;
}

eh_status eh_batch_advance(eh_batch *b, int32_t steps, int32_t *n_finished) {
  if (!b) return EH_ERR_INVALID_ARG;
  if (steps < 1) return bfail(b, EH_ERR_INVALID_ARG, "steps must be >= 1");
  const eh_status st = b->mode == EH_BATCH_MERGED ? advance_merged(b, steps) : advance_streams(b, steps);
  if (st) return st;
  int32_t fin = 0;
  for (Slot &s : b->slots)
    if (s.finished) ++fin;
  if (n_finished) *n_finished = fin;
  return EH_OK;
}

eh_status eh_batch_poll(eh_batch *b, int64_t ticket, int32_t *done, double *U_out, double *t, int64_t *steps) {
  if (!b || !done) return EH_ERR_INVALID_ARG;
  Slot *s = find(b, ticket);
  if (!s) return bfail(b, EH_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
  *done = s->finished ? 1 : 0;
  if (!s->finished) return EH_OK;
  if (t) *t = s->t;
  if (steps) *steps = s->steps;
  eh_status st = s->status;
  if (s->in_union) {  // its final state is still in the batch's context: copy the members' states out
    const eh_status rs = repack(b);
    if (rs && !st) st = rs;
  }
  if (!st && U_out) st = eh_get_state(s->ctx, U_out, 0);
  if (st) bfail(b, st, "request %lld: %s", (long long)ticket, eh_last_error(s->ctx));
  eh_destroy(s->ctx);
  b->used -= s->bytes;
  b->slots.erase(b->slots.begin() + (s - b->slots.data()));
  return st;
}

eh_status eh_batch_active(const eh_batch *b, int32_t *n_requests, uint64_t *bytes_in_use) {
  if (!b) return EH_ERR_INVALID_ARG;
  if (n_requests) *n_requests = (int32_t)b->slots.size();
  if (bytes_in_use) *bytes_in_use = b->used;
  return EH_OK;
}

eh_status eh_batch_repacks(const eh_batch *b, int64_t *repacks) {
  if (!b || !repacks) return EH_ERR_INVALID_ARG;
  *repacks = b->repacks;
  return EH_OK;
}

const char *eh_batch_last_error(const eh_batch *b) { return b ? b->err.c_str() : "null batch"; }

void eh_batch_destroy(eh_batch *b) {
  if (!b) return;
  for (Slot &s : b->slots) eh_destroy(s.ctx);
  eh_destroy(b->uni);
  delete b;
}

}  // extern "C"
