// batch.cu -- continuous-batching solve server on one device, over the
// context API of include/euler_hyp.h (host code only). Requests -- a mesh, an
// initial state and a final time each -- are admitted first come, first served
// while their device memory fits a budget next to the running ones; every
// admitted request keeps its mesh and state resident in a context of its own,
// on the context's own stream, and eh_batch_advance launches one SSPRK(3,3)
// step (a CUDA-graph replay) for every running request in turn, so that the
// requests' launches overlap on the device. A request stops on the device at
// its final time (eh_set_instances shortens its last step); eh_batch_poll hands
// its state back and frees its memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "../../include/euler_hyp.h"

namespace {

struct Slot {
  int64_t ticket;
  eh_ctx *ctx;
  uint64_t bytes;
  double t_final;
  double t;
  int64_t steps;
  bool finished;     // reached t_final, or failed (status)
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
  uint64_t budget = 0, used = 0;
  int64_t next_ticket = 1;
  std::vector<Slot> slots;
  std::string err;
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

}  // namespace

extern "C" {

eh_status eh_estimate_device_bytes(int32_t dim, int32_t precision, int32_t n, int64_t nnz, uint64_t *bytes) {
  if ((dim != 2 && dim != 3) || (precision != EH_PRECISION_FP64 && precision != EH_PRECISION_MIXED) || n < 1 ||
      nnz < n || !bytes)
    return EH_ERR_INVALID_ARG;
  *bytes = estimate_bytes(dim, precision, n, nnz);
  return EH_OK;
}

eh_status eh_batch_create(const eh_config *cfg, uint64_t hbm_budget_bytes, eh_batch **out) {
  if (!out) return EH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->stream || hbm_budget_bytes == 0) return EH_ERR_INVALID_ARG;
  // the configuration is checked once here, by a context that is not kept
  eh_ctx *probe = nullptr;
  eh_status st = eh_create(cfg, &probe);
  if (st) return st;
  eh_destroy(probe);
  eh_batch *b = new (std::nothrow) eh_batch;
  if (!b) return EH_ERR_OOM;
  b->cfg = *cfg;
  b->budget = hbm_budget_bytes;
  *out = b;
  return EH_OK;
}

eh_status eh_batch_admit(eh_batch *b, int32_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                         const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                         const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                         const double *bnd_state, const double *U0, double t_final, int64_t *ticket) {
  if (!b) return EH_ERR_INVALID_ARG;
  if (!ticket || !U0 || !(t_final > 0.0) || n < 1 || nnz < n)
    return bfail(b, EH_ERR_INVALID_ARG, "invalid request arguments");
  const uint64_t need = estimate_bytes(b->cfg.dim, b->cfg.precision, n, nnz);
  if (!b->slots.empty() && b->used + need > b->budget)
    return bfail(b, EH_ERR_OOM, "request needs %llu bytes, %llu of %llu in use", (unsigned long long)need,
                 (unsigned long long)b->used, (unsigned long long)b->budget);
  eh_ctx *c = nullptr;
  eh_status st = eh_create(&b->cfg, &c);
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
  Slot s{};
  s.ticket = b->next_ticket++;
  s.ctx = c;
  s.bytes = need;
  s.t_final = t_final;
  s.status = EH_OK;
  b->slots.push_back(s);
  b->used += need;
  *ticket = s.ticket;
  return EH_OK;
}

eh_status eh_batch_advance(eh_batch *b, int32_t steps, int32_t *n_finished) {
  if (!b) return EH_ERR_INVALID_ARG;
  if (steps < 1) return bfail(b, EH_ERR_INVALID_ARG, "steps must be >= 1");
  // step by step over the running requests: each launch is asynchronous on
  // the request's own stream, so the requests overlap on the device
  for (int32_t k = 0; k < steps; ++k)
    for (Slot &s : b->slots) {
      if (s.finished) continue;
      const eh_status st = eh_run(s.ctx, 1, 0.0);
      if (st) {
        s.finished = true;
        s.status = st;
        continue;
      }
      s.steps += 1;
    }
  int32_t fin = 0;
  for (Slot &s : b->slots) {
    if (!s.finished) {
      double t = 0.0;
      const eh_status st = eh_get_instances(s.ctx, &t, nullptr, nullptr);  // synchronises this request
      if (st) {
        s.finished = true;
        s.status = st;
      } else {
        s.t = t;
        if (t >= s.t_final) s.finished = true;
      }
    }
    if (s.finished) ++fin;
  }
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

const char *eh_batch_last_error(const eh_batch *b) { return b ? b->err.c_str() : "null batch"; }

void eh_batch_destroy(eh_batch *b) {
  if (!b) return;
  for (Slot &s : b->slots) eh_destroy(s.ctx);
  delete b;
}

}  // extern "C"
