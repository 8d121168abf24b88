// internal.cuh -- functions of capi.cu that the served batch (batch.cu) uses
// to merge its requests into one batched context. Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/euler_hyp.h"

namespace ehi {

// A context that holds one request's mesh data and state on the device and no
// per-stage work arrays: it is never stepped itself, only placed into a
// merged batch. The state is U0 with the boundary post-processing of Sec. 4
// applied. Runs on 'stream'. Arguments and errors as eh_upload_mesh and
// eh_set_state.
eh_status create_part(const eh_config *cfg, cudaStream_t stream, int32_t n, int64_t nnz, const int64_t *row_ptr,
                      const int32_t *col, const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                      const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                      const double *bnd_state, const double *U0, eh_ctx **out);

// Rebuilds 'uni' as the block-diagonal union of parts[0..count): their mesh
// data and current states, instance k = parts[k] with simulated time t[k] and
// end time t_final[k] (eh_set_instances). Device-to-device copies on uni's
// stream (the arrays are reallocated only when the union outgrows them; the
// CUDA graph is rebuilt at the next eh_run). Synchronises.
eh_status assemble(eh_ctx *uni, eh_ctx *const *parts, int count, const double *t, const double *t_final);

// Copies the state of instance k of 'uni' back into parts[k], for every k.
// Synchronises.
eh_status scatter(eh_ctx *uni, eh_ctx *const *parts, int count);

// The stream of a context.
cudaStream_t stream_of(const eh_ctx *c);

// Device bytes of the mesh data and state a part holds (dim, precision, n,
// nnz, boundary nodes).
uint64_t part_bytes(int dim, int precision, int64_t n, int64_t nnz, int64_t n_bnd);

}  // namespace ehi
