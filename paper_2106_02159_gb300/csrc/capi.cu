// capi.cu -- host side of the C ABI declared in include/euler_hyp.h: mesh
// validation and preprocessing, device memory, the SSPRK(3,3) stage schedule
// (Sec. 4.1, eq. SPPRK33), CUDA-graph replay and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/euler_hyp.h"
#include "internal.cuh"
#include "kernels.cuh"
#include "parabolic.cuh"

using namespace eh;

struct eh_ctx {
  eh_config cfg{};
  Params prm{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // mesh
  bool have_mesh = false, have_state = false;
  int n = 0;
  int64_t nnz = 0;
  int n_bnd = 0;
  std::vector<void *> allocs;  // every device allocation
  MeshView mv{};
  Work wk{};
  // state [S][n], stage state, trace buffers
  double *U = nullptr, *W = nullptr;
  // trace buffers, allocated by the first eh_stage: symmetrised limiter of
  // the first and of the last pass, state after the first pass, state before
  // the post-processing, P_ij of the first pass ([nnz][SP])
  double *trace_lsym = nullptr, *trace_upass = nullptr, *trace_pre = nullptr, *trace_llast = nullptr,
         *trace_P = nullptr;
  DevStatus *st = nullptr;
  DevStatus *st_host = nullptr;  // pinned
  // host bookkeeping
  int64_t steps = 0;
  double last_dt = 0.0;
  bool last_stage_traced = false;
  // graph cache for eh_run
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  // optional per-kernel event timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;  // kernel, (start, stop) event indices
  double prof_ms[EH_KERNEL_COUNT] = {0};
  int64_t prof_count[EH_KERNEL_COUNT] = {0};
  // block size (rows per block) of every kernel kind
  int tpb[EH_KERNEL_COUNT] = {128, 128, 128, 1024, 128, 128, 128, 256};
  // rows in flight per SM of the grid-stride kernels (lim1, pass, final); 0:
  // one thread per row
  int rows_per_sm[EH_KERNEL_COUNT] = {0};
  int nsm = 0;  // multiprocessors of the device
  // independent instances
  int ninst = 1;
  std::vector<void *> inst_allocs;
  double *Usave = nullptr;  // state saved while autotuning
  double *stat_part = nullptr, *stat_out = nullptr;  // state statistics of eh_get_diagnostics
  // parabolic sub-step (Sec. 5): finite-element data, constants, work arrays
  bool have_visc = false;
  ParView pv{};
  ParWork pw{};
  double cg_tol = 1e-13;
  int cg_max_iter = 2000;
  std::vector<void *> par_allocs;
  double *host_scal = nullptr;  // pinned, two doubles
  int *host_ctl = nullptr;      // pinned, the CG control pair
  int cg_last[3] = {8, 8, 8};   // iterations of the last velocity, energy and low-order solves
  // a request of a merged served batch: mesh data and state on the device, no
  // work arrays (it is stepped inside the batch's own context)
  bool static_only = false;
  // a merged batch's context: the sizes its arrays were allocated for
  int64_t cap_n = 0, cap_nnz = 0, cap_bnd = 0;
  int64_t rec_n = 0;  // nodes the record array was allocated for
};

namespace {

const char *kStatusNames[] = {"EH_OK",         "EH_ERR_INVALID_ARG", "EH_ERR_OOM",  "EH_ERR_BAD_MESH",
                              "EH_ERR_NOT_ADMISSIBLE", "EH_ERR_CFL",  "EH_ERR_CUDA", "EH_ERR_STATE"};

eh_status fail(eh_ctx *c, eh_status st, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

#define CUDA_TRY(c, expr)                                                                                     \
  do {                                                                                                        \
    cudaError_t e_ = (expr);                                                                                  \
    if (e_ != cudaSuccess) {                                                                                  \
      eh_status s_ = e_ == cudaErrorMemoryAllocation ? EH_ERR_OOM : EH_ERR_CUDA;                              \
      return fail(c, s_, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__);       \
    }                                                                                                         \
  } while (0)

template <typename T> eh_status dalloc(eh_ctx *c, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? EH_ERR_OOM : EH_ERR_CUDA, "cudaMalloc of %zu bytes: %s",
                count * sizeof(T), cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *p = (T *)q;
  return EH_OK;
}

void free_instances(eh_ctx *c) {
  for (void *q : c->inst_allocs) cudaFree(q);
  c->inst_allocs.clear();
}

void free_parabolic(eh_ctx *c) {
  for (void *p : c->par_allocs) cudaFree(p);
  c->par_allocs.clear();
  c->have_visc = false;
}

void free_mesh(eh_ctx *c) {
  free_parabolic(c);
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  free_instances(c);
  for (void *q : c->allocs) cudaFree(q);
  c->allocs.clear();
  c->mv = MeshView{};
  c->wk = Work{};
  c->U = c->W = nullptr;
  c->trace_lsym = c->trace_upass = c->trace_pre = c->trace_llast = c->trace_P = nullptr;
  c->have_mesh = c->have_state = false;
}

int S_of(const eh_ctx *c) { return c->cfg.dim + 2; }
int SP_of(const eh_ctx *c) { return c->cfg.dim == 2 ? Layout<2>::SP : Layout<3>::SP; }

eh_status check_device_error(eh_ctx *c) {
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  CUDA_TRY(c, cudaMemcpy(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  int e = c->st_host->err;
  if (e == EH_ERR_CFL) return fail(c, EH_ERR_CFL, "prescribed dt exceeds the invariant-domain limit of the first stage");
  if (e == EH_ERR_NOT_ADMISSIBLE)
    return fail(c, EH_ERR_NOT_ADMISSIBLE, "%llu non-admissible nodes after a step",
                (unsigned long long)c->st_host->not_admissible);
  if (e) return fail(c, EH_ERR_CUDA, "device error code %d", e);
  return EH_OK;
}

// Event pair around one kernel launch when profiling is on.
struct ProfScope {
  eh_ctx *c;
  int kernel;
  size_t a = 0;
  ProfScope(eh_ctx *c_, int k) : c(c_), kernel(k) {
    if (!c->profiling) return;
    a = next_event();
    cudaEventRecord(c->ev_pool[a], c->stream);
  }
  size_t next_event() {
    size_t idx = 0;
    for (auto &m : c->ev_marks) idx = std::max(idx, std::max(m.second.first, m.second.second) + 1);
    if (idx >= c->ev_pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev_pool.push_back(e);
    }
    return idx;
  }
  ~ProfScope() {
    if (!c->profiling) return;
    c->ev_marks.push_back({kernel, {a, a}});
    size_t b = next_event();
    c->ev_marks.back().second.second = b;
    cudaEventRecord(c->ev_pool[b], c->stream);
  }
};

void flush_profile(eh_ctx *c) {
  if (c->ev_marks.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto &m : c->ev_marks) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_pool[m.second.first], c->ev_pool[m.second.second]);
    c->prof_ms[m.first] += ms;
    c->prof_count[m.first] += 1;
  }
  c->ev_marks.clear();
}

// One forward-Euler stage on the component-major state Uin, written as
// out = BC(FE(Uin)) (coef < 0) or out = U0 + coef (BC(FE(Uin)) - U0).
// grid cap of a grid-stride kernel kind (0: one thread per row)
int max_blocks(const eh_ctx *c, int kernel) {
  const int r = c->rows_per_sm[kernel];
  if (r <= 0 || c->nsm <= 0) return 0;
  return c->nsm * std::max(1, r / c->tpb[kernel]);
}

template <int DIM, typename T>
void enqueue_stage(eh_ctx *c, const double *Uin, int stage, double dt_given, const double *U0, double coef, double *out,
                   bool trace) {
  cudaStream_t s = c->stream;
  const MeshView &m = c->mv;
  const Params &p = c->prm;
  const Work &w = c->wk;
  const int *tpb = c->tpb;
  { ProfScope ps(c, EH_KERNEL_PREP); launch_prep<DIM, T>(m, p, Uin, w, tpb[EH_KERNEL_PREP], s); }
  {
    ProfScope ps(c, EH_KERNEL_VISC);
    launch_visc<DIM, T>(m, p, w, tpb[EH_KERNEL_VISC], s);
    launch_alpha<DIM, T>(m, p, w, tpb[EH_KERNEL_VISC], s);
  }
  { ProfScope ps(c, EH_KERNEL_LOW); launch_low<DIM, T>(m, p, w, tpb[EH_KERNEL_LOW], s); }
  { ProfScope ps(c, EH_KERNEL_TAU); launch_tau(m, w, stage, dt_given, p.cfl, !trace, s); }
  {
    ProfScope ps(c, EH_KERNEL_LIM1);
    launch_lim1<DIM, T>(m, p, w, trace ? c->trace_P : nullptr, tpb[EH_KERNEL_LIM1], max_blocks(c, EH_KERNEL_LIM1), s);
  }
  { ProfScope ps(c, EH_KERNEL_LSEARCH); launch_ls_deferred<DIM>(m, p, w, w.UL, 0, w.la, tpb[EH_KERNEL_LSEARCH], s); }
  const double *ucur = w.UL;
  double *lcur = w.la, *lnext = w.lb;
  double *unext = w.Ua;
  for (int pass = 1; pass < c->cfg.limiter_passes; ++pass) {
    {
      ProfScope ps(c, EH_KERNEL_PASS);
      launch_pass<DIM>(m, p, w, ucur, unext, lcur, lnext, (trace && pass == 1) ? c->trace_lsym : nullptr, pass,
                       tpb[EH_KERNEL_PASS], max_blocks(c, EH_KERNEL_PASS), s);
    }
    {
      ProfScope ps(c, EH_KERNEL_LSEARCH);
      launch_ls_deferred<DIM>(m, p, w, unext, pass, lnext, tpb[EH_KERNEL_LSEARCH], s);
    }
    if (trace && pass == 1) {
      cudaMemcpyAsync(c->trace_upass, unext, sizeof(double) * (size_t)c->n * SP_of(c), cudaMemcpyDeviceToDevice, s);
    }
    ucur = unext;
    unext = (unext == w.Ua) ? w.Ub : w.Ua;
    std::swap(lcur, lnext);
  }
  {
    ProfScope ps(c, EH_KERNEL_FINAL);
    launch_final<DIM>(m, p, w, ucur, lcur, U0, coef, out, trace ? c->trace_pre : nullptr,
                      trace ? c->trace_llast : nullptr, tpb[EH_KERNEL_FINAL],
                      max_blocks(c, EH_KERNEL_FINAL), s);
  }
}

template <int DIM, typename T> void enqueue_step(eh_ctx *c, double dt) {
  // w1 = BC(FE(u)); w2 = u + 1/4 (BC(FE(w1)) - u); u <- u + 2/3 (BC(FE(w2)) - u)
  enqueue_stage<DIM, T>(c, c->U, 0, dt, nullptr, -1.0, c->W, false);
  enqueue_stage<DIM, T>(c, c->W, 1, dt, c->U, 0.25, c->W, false);
  enqueue_stage<DIM, T>(c, c->W, 2, dt, c->U, 2.0 / 3.0, c->U, false);
}

bool mixed(const eh_ctx *c) { return c->cfg.precision == EH_PRECISION_MIXED; }

void enqueue_step_any(eh_ctx *c, double dt) {
  if (c->cfg.dim == 2) {
    if (mixed(c)) enqueue_step<2, float>(c, dt); else enqueue_step<2, double>(c, dt);
  } else {
    if (mixed(c)) enqueue_step<3, float>(c, dt); else enqueue_step<3, double>(c, dt);
  }
}

void enqueue_stage_any(eh_ctx *c, double tau) {
  if (c->cfg.dim == 2) {
    if (mixed(c)) enqueue_stage<2, float>(c, c->U, 0, tau, nullptr, -1.0, c->U, true);
    else enqueue_stage<2, double>(c, c->U, 0, tau, nullptr, -1.0, c->U, true);
  } else {
    if (mixed(c)) enqueue_stage<3, float>(c, c->U, 0, tau, nullptr, -1.0, c->U, true);
    else enqueue_stage<3, double>(c, c->U, 0, tau, nullptr, -1.0, c->U, true);
  }
}

template <int DIM, typename T> void enqueue_cfl(eh_ctx *c) {
  launch_prep<DIM, T>(c->mv, c->prm, c->U, c->wk, c->tpb[EH_KERNEL_PREP], c->stream);
  launch_visc<DIM, T>(c->mv, c->prm, c->wk, c->tpb[EH_KERNEL_VISC], c->stream);
  launch_alpha<DIM, T>(c->mv, c->prm, c->wk, c->tpb[EH_KERNEL_VISC], c->stream);
  launch_low<DIM, T>(c->mv, c->prm, c->wk, c->tpb[EH_KERNEL_LOW], c->stream);
}

// (Re)allocates the per-instance arrays for 'ninst' instances with row offsets
// 'off' (host, ninst+1 entries) and end times 'tf' (host, or NULL = none).
eh_status setup_instances(eh_ctx *c, int ninst, const int64_t *off, const double *tf) {
  free_instances(c);
  auto ialloc = [&](void **p, size_t bytes) -> eh_status {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 8));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, EH_ERR_OOM, "cudaMalloc of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    c->inst_allocs.push_back(*p);
    return EH_OK;
  };
  eh_status st;
  void *p_off, *p_tau, *p_bound, *p_t, *p_tf, *p_bits, *p_steps, *p_inst = nullptr;
  if ((st = ialloc(&p_off, sizeof(int64_t) * (ninst + 1)))) return st;
  if ((st = ialloc(&p_tau, sizeof(double) * ninst))) return st;
  if ((st = ialloc(&p_bound, sizeof(double) * 3 * ninst))) return st;
  if ((st = ialloc(&p_t, sizeof(double) * ninst))) return st;
  if ((st = ialloc(&p_tf, sizeof(double) * ninst))) return st;
  if ((st = ialloc(&p_bits, sizeof(unsigned long long) * ninst))) return st;
  if ((st = ialloc(&p_steps, sizeof(unsigned long long) * ninst))) return st;
  CUDA_TRY(c, cudaMemset(p_steps, 0, sizeof(unsigned long long) * ninst));
  std::vector<unsigned long long> inf_bits(ninst, 0x7FF0000000000000ull);
  CUDA_TRY(c, cudaMemcpy(p_bits, inf_bits.data(), sizeof(unsigned long long) * ninst, cudaMemcpyHostToDevice));
  std::vector<double> tfinal(ninst, INFINITY);
  if (tf)
    for (int k = 0; k < ninst; ++k) tfinal[k] = tf[k] > 0.0 ? tf[k] : INFINITY;
  CUDA_TRY(c, cudaMemcpy(p_off, off, sizeof(int64_t) * (ninst + 1), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemset(p_tau, 0, sizeof(double) * ninst));
  CUDA_TRY(c, cudaMemset(p_bound, 0, sizeof(double) * 3 * ninst));
  CUDA_TRY(c, cudaMemset(p_t, 0, sizeof(double) * ninst));
  CUDA_TRY(c, cudaMemcpy(p_tf, tfinal.data(), sizeof(double) * ninst, cudaMemcpyHostToDevice));
  if (ninst > 1) {
    std::vector<int32_t> inst(c->n);
    for (int k = 0; k < ninst; ++k)
      for (int64_t i = off[k]; i < off[k + 1]; ++i) inst[i] = k;
    if ((st = ialloc(&p_inst, sizeof(int32_t) * c->n))) return st;
    CUDA_TRY(c, cudaMemcpy(p_inst, inst.data(), sizeof(int32_t) * c->n, cudaMemcpyHostToDevice));
  }
  if (c->cfg.bound_relaxation) {
    // r_i = (m_i / |D|)^(1.5/dim) with |D| the measure of the node's own
    // instance, not of the whole block-diagonal mesh
    const int n = c->n, dim = c->cfg.dim;
    std::vector<double> mi(n), relax(n);
    CUDA_TRY(c, cudaMemcpy(mi.data(), c->mv.mi, sizeof(double) * n, cudaMemcpyDeviceToHost));
    for (int k = 0; k < ninst; ++k) {
      double area = 0.0;
      for (int64_t i = off[k]; i < off[k + 1]; ++i) area += mi[i];
      for (int64_t i = off[k]; i < off[k + 1]; ++i) relax[i] = std::pow(mi[i] / area, 1.5 / dim);
    }
    CUDA_TRY(c, cudaMemcpy((void *)c->mv.relax, relax.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  }
  c->ninst = ninst;
  c->mv.ninst = ninst;
  c->mv.inst = (const int32_t *)p_inst;
  c->mv.inst_row_off = (const int64_t *)p_off;
  c->wk.tau_inst = (double *)p_tau;
  c->wk.bound_inst = (double *)p_bound;
  c->wk.t_inst = (double *)p_t;
  c->wk.tfinal_inst = (double *)p_tf;
  c->wk.bound_bits = (unsigned long long *)p_bits;
  c->wk.steps_inst = (unsigned long long *)p_steps;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return EH_OK;
}

// Device arrays of the static mesh data for (up to) n nodes, nnz entries and
// n_bnd boundary nodes; sets the MeshView pointers (contents not written).
eh_status alloc_static(eh_ctx *c, int64_t n, int64_t nnz, int64_t n_bnd) {
  const int dim = c->cfg.dim, S = S_of(c);
  MeshView &m = c->mv;
  eh_status st;
  int64_t *row = nullptr;
  int32_t *col = nullptr, *tr = nullptr, *bidx = nullptr, *bnode = nullptr, *bkind = nullptr;
  double *cij = nullptr, *cn = nullptr, *cinv = nullptr, *betat = nullptr, *mi = nullptr, *imi = nullptr,
         *relax = nullptr, *lam = nullptr, *bnorm = nullptr, *bstate = nullptr;
  unsigned char *isb = nullptr;
  if ((st = dalloc(c, &row, (size_t)n + 1)) || (st = dalloc(c, &col, (size_t)nnz)) ||
      (st = dalloc(c, &tr, (size_t)nnz)) || (st = dalloc(c, &cij, (size_t)dim * nnz)) ||
      (st = dalloc(c, &cn, (size_t)nnz)) || (st = dalloc(c, &cinv, (size_t)nnz)) ||
      (st = dalloc(c, &betat, (size_t)nnz)) || (st = dalloc(c, &mi, (size_t)n)) || (st = dalloc(c, &imi, (size_t)n)) ||
      (st = dalloc(c, &relax, (size_t)n)) || (st = dalloc(c, &lam, (size_t)n)) || (st = dalloc(c, &isb, (size_t)n)) ||
      (st = dalloc(c, &bidx, (size_t)n)) || (st = dalloc(c, &bnode, (size_t)n_bnd)) ||
      (st = dalloc(c, &bkind, (size_t)n_bnd)) || (st = dalloc(c, &bnorm, (size_t)dim * n_bnd)) ||
      (st = dalloc(c, &bstate, (size_t)S * n_bnd)))
    return st;
  m.row_ptr = row;
  m.col = col;
  m.tr = tr;
  m.cij = cij;
  m.cn = cn;
  m.cinv = cinv;
  m.betat = betat;
  m.mi = mi;
  m.inv_mi = imi;
  m.relax = relax;
  m.lam = lam;
  m.isb = isb;
  m.bnd_index = bidx;
  m.bnd_node = bnode;
  m.bnd_kind = bkind;
  m.bnd_normal = bnorm;
  m.bnd_state = bstate;
  m.vcij = cij;
  m.vcn = cn;
  m.vcinv = cinv;
  if (mixed(c)) {  // FP32 c_ij, |c_ij|, 1/|c_ij|
    float *fc = nullptr, *fn = nullptr, *fi = nullptr;
    if ((st = dalloc(c, &fc, (size_t)dim * nnz)) || (st = dalloc(c, &fn, (size_t)nnz)) ||
        (st = dalloc(c, &fi, (size_t)nnz)))
      return st;
    m.vcij = fc;
    m.vcn = fn;
    m.vcinv = fi;
  }
  return EH_OK;
}

// Node records as all-ones bit patterns (NaN), which no admissible state
// matches: k_prep then remakes every record, and k_visc skips no edge (its
// skip relies on edge values stored from the same states on the same mesh).
// Called when the arrays are allocated and when a merged batch's context is
// rebuilt over another set of meshes.
cudaError_t invalidate_records(eh_ctx *c) {
  if (!c->wk.rec || c->rec_n <= 0) return cudaSuccess;
  return cudaMemsetAsync(c->wk.rec, 0xFF, sizeof(double) * (size_t)c->rec_n * REC_MAX, c->stream);
}

// The per-stage work arrays for (up to) n nodes and nnz entries, and the
// state buffers. A static-only context (a request of a merged served batch)
// gets the state only: it is stepped as part of the batch's context.
eh_status alloc_work(eh_ctx *c, int64_t n, int64_t nnz) {
  const int dim = c->cfg.dim, S = S_of(c), SP = SP_of(c);
  Work &w = c->wk;
  eh_status st;
#define ALLOC(ptr, cnt) \
  if ((st = dalloc(c, &ptr, (size_t)(cnt))) != EH_OK) return st;
  ALLOC(c->U, (size_t)S * n);
  w.st = c->st;
  if (c->static_only) return EH_OK;
  ALLOC(w.rec, (size_t)n * REC_MAX);
  ALLOC(c->stat_part, (size_t)7 * STAT_BLOCKS);
  ALLOC(c->stat_out, 8);
  ALLOC(w.alpha, n);
  ALLOC(w.rough, n);
  ALLOC(w.rough2, n);
  ALLOC(w.steady, n);
  ALLOC(w.lone, 2 * n);
  ALLOC(w.inc, (size_t)n * SP);
  if (mixed(c)) {
    // FP32 node record, packed w_ij/a_ij/d_ij slots and F^H
    float *f_rec, *f_w, *f_fh;
    ALLOC(f_rec, (size_t)n * VREC_MAX);
    ALLOC(f_fh, (size_t)n * SP);
    static_assert(EdgeLayout<2, float>::packed && EdgeLayout<3, float>::packed, "FP32 edge slots are packed");
    constexpr int spw_f = EdgeLayout<2, float>::SPW;
    ALLOC(f_w, (size_t)nnz * spw_f);
    w.va = nullptr;
    w.vrec = f_rec;
    w.vw = f_w;
    w.vd = nullptr;
    w.vFH = f_fh;
    ALLOC(w.G64, (size_t)n * SP);
  } else {
    ALLOC(w.FH, (size_t)n * SP);
    double *d_a = nullptr;
    if (dim == 3) {  // packed slots [w (5), a, d, 0]
      constexpr int spw3 = EdgeLayout<3, double>::SPW;
      ALLOC(w.w, (size_t)nnz * spw3);
      w.d = nullptr;
    } else {
      constexpr int spw2 = EdgeLayout<2, double>::SPW;
      ALLOC(w.w, (size_t)nnz * spw2);
      ALLOC(w.d, nnz);
      ALLOC(d_a, nnz);
    }
    w.va = d_a;
    w.vrec = w.rec;
    w.vw = w.w;
    w.vd = w.d;
    w.vFH = w.FH;
    w.G64 = w.FH;
  }
  ALLOC(w.bounds, (size_t)n * 4);
  ALLOC(w.UL, (size_t)n * SP);
  ALLOC(w.Ua, (size_t)n * SP);
  ALLOC(w.Ub, (size_t)n * SP);
  ALLOC(w.P, (size_t)nnz * SP);
  ALLOC(w.rem, nnz);
  ALLOC(w.la, nnz);
  ALLOC(w.lb, nnz);
  ALLOC(w.lsq, nnz);  // every entry can be queued once per pass
  ALLOC(w.lsq_count, LSQ_SLOTS);
  w.lsq_cap = (unsigned)nnz;
  // iterations: a small share of the searches; a full queue falls back to
  // iterating in k_ls_deferred
  w.lsq2_cap = (unsigned)std::max<int64_t>(nnz / 8, 4096);
  ALLOC(w.lsq2, w.lsq2_cap);
  ALLOC(w.lsq2_count, LSQ_SLOTS);
  ALLOC(c->Usave, (size_t)S * n);
  ALLOC(c->W, (size_t)S * n);
#undef ALLOC
  CUDA_TRY(c, cudaMemset(w.lsq_count, 0, sizeof(unsigned) * LSQ_SLOTS));
  CUDA_TRY(c, cudaMemset(w.lsq2_count, 0, sizeof(unsigned) * LSQ_SLOTS));
  c->rec_n = n;
  CUDA_TRY(c, invalidate_records(c));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return EH_OK;
}

void enqueue_cfl_any(eh_ctx *c) {
  if (c->cfg.dim == 2) {
    if (mixed(c)) enqueue_cfl<2, float>(c); else enqueue_cfl<2, double>(c);
  } else {
    if (mixed(c)) enqueue_cfl<3, float>(c); else enqueue_cfl<3, double>(c);
  }
}

eh_status require_ready(eh_ctx *c) {
  if (!c) return EH_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, EH_ERR_STATE, "no mesh uploaded");
  if (!c->have_state) return fail(c, EH_ERR_STATE, "no state set");
  return EH_OK;
}

// the trace buffers of eh_stage, allocated on first use (they are freed with
// the mesh)
eh_status ensure_trace_buffers(eh_ctx *c) {
  if (c->trace_P) return EH_OK;
  const int SP = SP_of(c);
  eh_status st;
  if ((st = dalloc(c, &c->trace_lsym, (size_t)c->nnz))) return st;
  if ((st = dalloc(c, &c->trace_llast, (size_t)c->nnz))) return st;
  if ((st = dalloc(c, &c->trace_upass, (size_t)c->n * SP))) return st;
  if ((st = dalloc(c, &c->trace_pre, (size_t)c->n * SP))) return st;
  return dalloc(c, &c->trace_P, (size_t)c->nnz * SP);
}

eh_status reset_status(eh_ctx *c) {
  CUDA_TRY(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
  return EH_OK;
}

// The cached CUDA graph of one SSPRK(3,3) step with dt (captured again when
// dt differs from the one it holds).
eh_status ensure_graph(eh_ctx *c, double dt) {
  if (c->graph && c->graph_dt == dt) return EH_OK;
  if (c->graph) {
    CUDA_TRY(c, cudaGraphExecDestroy(c->graph));
    c->graph = nullptr;
  }
  cudaGraph_t g;
  CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_step_any(c, dt);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess) return fail(c, EH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, EH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graph_dt = dt;
  return EH_OK;
}

}  // namespace

extern "C" {

void eh_config_default(eh_config *cfg) {
  if (!cfg) return;
  cfg->dim = 2;
  cfg->gamma = 1.4;
  cfg->cfl = 0.5;
  cfg->limiter_passes = 2;
  cfg->bound_relaxation = 0;
  cfg->precision = EH_PRECISION_FP64;
  cfg->device = 0;
  cfg->stream = nullptr;
}

const char *eh_status_string(eh_status st) {
  int k = (int)st;
  if (k < 0 || k > 7) return "EH_UNKNOWN";
  return kStatusNames[k];
}

const char *eh_last_error(const eh_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

eh_status eh_create(const eh_config *cfg, eh_ctx **out) {
  if (!out) return EH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return EH_ERR_INVALID_ARG;
  if (cfg->dim != 2 && cfg->dim != 3) return EH_ERR_INVALID_ARG;
  if (!(cfg->gamma > 1.0 && cfg->gamma <= 5.0 / 3.0)) return EH_ERR_INVALID_ARG;
  if (!(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) return EH_ERR_INVALID_ARG;
  if (cfg->limiter_passes < 1 || cfg->limiter_passes > 8) return EH_ERR_INVALID_ARG;
  if (cfg->precision != EH_PRECISION_FP64 && cfg->precision != EH_PRECISION_MIXED) return EH_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return EH_ERR_CUDA;
  }
  eh_ctx *c = new eh_ctx();
  c->cfg = *cfg;
  c->device = cfg->device;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    delete c;
    return EH_ERR_CUDA;
  }
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return EH_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaMalloc(&c->st, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->st_host, sizeof(DevStatus)) != cudaSuccess) {
    if (c->st) cudaFree(c->st);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return EH_ERR_OOM;
  }
  cudaMemset(c->st, 0, sizeof(DevStatus));
  if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) c->nsm = 0;
  if (cfg->dim == 3) {
    // 3D: eh_autotune on a 6.0M-vertex extruded cylinder (after 100 steps
    // and on a perturbed state, FP64 and mixed), with k_pass reading P only
    // where a limiter is below 1: every kernel uncapped (2-3% over a cap of
    // 512 rows in flight per SM on k_pass, which kept a 27-entry row's lines
    // of P in L1 while its second walk still re-read all of them)
    c->tpb[EH_KERNEL_PREP] = 64;
    c->tpb[EH_KERNEL_VISC] = 64;
    c->tpb[EH_KERNEL_LOW] = 64;
    c->tpb[EH_KERNEL_LIM1] = 128;
    c->tpb[EH_KERNEL_PASS] = 256;
    c->tpb[EH_KERNEL_FINAL] = 64;
    c->tpb[EH_KERNEL_LSEARCH] = 64;
  } else {
    // 2D: eh_autotune on the 4.0M cylinder (bench window and a perturbed
    // state, FP64 and mixed) picks 64 rows per block and no cap on the rows
    // in flight for the row kernels (1-2% faster than 128 with caps)
    for (int k = 0; k < EH_KERNEL_COUNT; ++k)
      if (k != EH_KERNEL_TAU) c->tpb[k] = 64;
    c->tpb[EH_KERNEL_LSEARCH] = 128;
  }
  Params &p = c->prm;
  p.gamma = cfg->gamma;
  p.cfl = cfg->cfl;
  p.gamma75 = cfg->gamma == 1.4 ? 1 : 0;
  p.limiter_passes = cfg->limiter_passes;
  p.gm1 = cfg->gamma - 1.0;
  p.z = (cfg->gamma - 1.0) / (2.0 * cfg->gamma);
  p.inv_z = 1.0 / p.z;
  p.kshock = (cfg->gamma + 1.0) / (2.0 * cfg->gamma);
  p.inv_gm1 = 1.0 / (cfg->gamma - 1.0);
  *out = c;
  return EH_OK;
}

void eh_destroy(eh_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_mesh(c);
  if (c->st) cudaFree(c->st);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->host_scal) cudaFreeHost(c->host_scal);
  if (c->host_ctl) cudaFreeHost(c->host_ctl);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

eh_status eh_upload_mesh(eh_ctx *c, int32_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                         const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                         const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                         const double *bnd_state) {
  if (!c) return EH_ERR_INVALID_ARG;
  if (n <= 0 || nnz <= 0 || nnz >= ((int64_t)1 << 31) || !row_ptr || !col || !cij || !mij || !mi || n_bnd < 0 ||
      (n_bnd > 0 && (!bnd_node || !bnd_kind || !bnd_normal)))
    return fail(c, EH_ERR_INVALID_ARG, "invalid mesh arguments");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  free_mesh(c);
  const int dim = c->cfg.dim, S = S_of(c);
  // ---- validation (host) ----
  if (row_ptr[0] != 0 || row_ptr[n] != nnz) return fail(c, EH_ERR_BAD_MESH, "row_ptr must start at 0 and end at nnz");
  for (int i = 0; i < n; ++i) {
    if (row_ptr[i + 1] - row_ptr[i] < 2) return fail(c, EH_ERR_BAD_MESH, "row %d has fewer than 2 entries", i);
    bool diag = false;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n) return fail(c, EH_ERR_BAD_MESH, "column out of range in row %d", i);
      if (k > row_ptr[i] && col[k] <= col[k - 1]) return fail(c, EH_ERR_BAD_MESH, "row %d not sorted/unique", i);
      if (col[k] == i) diag = true;
    }
    if (!diag) return fail(c, EH_ERR_BAD_MESH, "row %d has no diagonal entry", i);
    if (!(mi[i] > 0.0)) return fail(c, EH_ERR_BAD_MESH, "m_%d <= 0", i);
  }
  std::vector<int32_t> tr(nnz);
  for (int i = 0; i < n; ++i) {
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const int j = col[k];
      const int32_t *b = col + row_ptr[j], *e = col + row_ptr[j + 1];
      const int32_t *f = std::lower_bound(b, e, i);
      if (f == e || *f != i) return fail(c, EH_ERR_BAD_MESH, "pattern not symmetric at (%d,%d)", i, j);
      tr[k] = (int32_t)(row_ptr[j] + (f - b));
    }
  }
  std::vector<double> cn(nnz), cinv(nnz), betat(nnz);
  for (int i = 0; i < n; ++i) {
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double s2 = 0.0;
      for (int d = 0; d < dim; ++d) s2 += cij[(int64_t)d * nnz + k] * cij[(int64_t)d * nnz + k];
      cn[k] = std::sqrt(s2);
      cinv[k] = cn[k] > 0.0 ? 1.0 / cn[k] : 0.0;
      if (col[k] != i && !(cn[k] > 0.0)) return fail(c, EH_ERR_BAD_MESH, "c_ij = 0 at an off-diagonal entry");
      // the consistent mass matrix is symmetric (m_ij = int phi_i phi_j);
      // k_lim1 relies on it, with the mean of the two entries
      const double a = mij[k], b = mij[tr[k]];
      if (std::fabs(a - b) > 1e-12 * std::max(std::fabs(a), std::fabs(b)))
        return fail(c, EH_ERR_BAD_MESH, "consistent mass not symmetric at (%d,%d)", i, col[k]);
      betat[k] = 0.5 * (a + b) / mi[i];
    }
  }
  std::vector<double> inv_mi(n), relax(n, 0.0), lam(n);
  double area = 0.0;
  for (int i = 0; i < n; ++i) area += mi[i];
  for (int i = 0; i < n; ++i) {
    inv_mi[i] = 1.0 / mi[i];
    lam[i] = 1.0 / (double)(row_ptr[i + 1] - row_ptr[i] - 1);
    if (c->cfg.bound_relaxation) relax[i] = std::pow(mi[i] / area, 1.5 / dim);
  }
  std::vector<unsigned char> isb(n, 0);
  std::vector<int32_t> bidx(n, -1);
  for (int b = 0; b < n_bnd; ++b) {
    const int i = bnd_node[b];
    if (i < 0 || i >= n || bidx[i] >= 0) return fail(c, EH_ERR_BAD_MESH, "boundary node %d invalid or repeated", i);
    if (bnd_kind[b] < EH_BC_SLIP || bnd_kind[b] > EH_BC_GODUNOV)
      return fail(c, EH_ERR_BAD_MESH, "boundary kind %d invalid", bnd_kind[b]);
    if (bnd_kind[b] != EH_BC_SLIP && bnd_kind[b] != EH_BC_DO_NOTHING && !bnd_state)
      return fail(c, EH_ERR_BAD_MESH, "boundary kind %d needs a Dirichlet state", bnd_kind[b]);
    isb[i] = 1;
    bidx[i] = b;
  }
  // ---- device arrays ----
  eh_status st;
  if ((st = alloc_static(c, n, nnz, n_bnd)) != EH_OK) {
    free_mesh(c);
    return st;
  }
  MeshView &m = c->mv;
  auto up = [&](const void *dst, const void *src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpy(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = up(m.row_ptr, row_ptr, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = up(m.col, col, sizeof(int32_t) * nnz);
  if (e == cudaSuccess) e = up(m.tr, tr.data(), sizeof(int32_t) * nnz);
  if (e == cudaSuccess) e = up(m.cij, cij, sizeof(double) * dim * nnz);
  if (e == cudaSuccess) e = up(m.cn, cn.data(), sizeof(double) * nnz);
  if (e == cudaSuccess) e = up(m.cinv, cinv.data(), sizeof(double) * nnz);
  if (e == cudaSuccess) e = up(m.betat, betat.data(), sizeof(double) * nnz);
  if (e == cudaSuccess) e = up(m.mi, mi, sizeof(double) * n);
  if (e == cudaSuccess) e = up(m.inv_mi, inv_mi.data(), sizeof(double) * n);
  if (e == cudaSuccess) e = up(m.relax, relax.data(), sizeof(double) * n);
  if (e == cudaSuccess) e = up(m.lam, lam.data(), sizeof(double) * n);
  if (e == cudaSuccess) e = up(m.isb, isb.data(), n);
  if (e == cudaSuccess) e = up(m.bnd_index, bidx.data(), sizeof(int32_t) * n);
  if (e == cudaSuccess) e = up(m.bnd_node, bnd_node, sizeof(int32_t) * n_bnd);
  if (e == cudaSuccess) e = up(m.bnd_kind, bnd_kind, sizeof(int32_t) * n_bnd);
  if (e == cudaSuccess) e = up(m.bnd_normal, bnd_normal, sizeof(double) * dim * n_bnd);
  if (e == cudaSuccess && bnd_state) e = up(m.bnd_state, bnd_state, sizeof(double) * S * n_bnd);
  if (e == cudaSuccess && mixed(c)) {
    std::vector<float> tmp((size_t)dim * nnz);
    for (size_t q = 0; q < tmp.size(); ++q) tmp[q] = (float)cij[q];
    e = up(m.vcij, tmp.data(), sizeof(float) * tmp.size());
    tmp.resize(nnz);
    for (int64_t k = 0; e == cudaSuccess && k < nnz; ++k) tmp[k] = (float)cn[k];
    if (e == cudaSuccess) e = up(m.vcn, tmp.data(), sizeof(float) * nnz);
    for (int64_t k = 0; e == cudaSuccess && k < nnz; ++k) tmp[k] = (float)cinv[k];
    if (e == cudaSuccess) e = up(m.vcinv, tmp.data(), sizeof(float) * nnz);
  }
  if (e != cudaSuccess) {
    free_mesh(c);
    return fail(c, EH_ERR_CUDA, "mesh upload: %s", cudaGetErrorString(e));
  }
  m.n = n;
  m.nnz = nnz;
  m.n_bnd = n_bnd;
  m.n_nonreflecting = 0;
  for (int b = 0; b < n_bnd; ++b)
    if (bnd_kind[b] == EH_BC_CHARACTERISTIC || bnd_kind[b] == EH_BC_GODUNOV) ++m.n_nonreflecting;
  c->n = n;
  c->nnz = nnz;
  c->n_bnd = n_bnd;
  if ((st = alloc_work(c, n, nnz)) != EH_OK) {
    free_mesh(c);
    return st;
  }
  const int64_t one[2] = {0, (int64_t)n};
  if ((st = setup_instances(c, 1, one, nullptr)) != EH_OK) {
    free_mesh(c);
    return st;
  }
  c->have_mesh = true;
  c->steps = 0;
  return EH_OK;
}

eh_status eh_set_state(eh_ctx *c, const double *U, int is_device_ptr) {
  if (!c || !U) return EH_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, EH_ERR_STATE, "no mesh uploaded");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const size_t bytes = sizeof(double) * S_of(c) * c->n;
  CUDA_TRY(c, cudaMemcpyAsync(c->U, U, bytes, is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
  eh_status st = reset_status(c);
  if (st) return st;
  if (c->cfg.dim == 2) launch_count_not_admissible<2>(c->n, c->U, c->st, c->stream);
  else launch_count_not_admissible<3>(c->n, c->U, c->st, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  CUDA_TRY(c, cudaMemcpy(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  if (c->st_host->not_admissible) {
    c->have_state = false;
    return fail(c, EH_ERR_NOT_ADMISSIBLE, "%llu nodes with rho <= 0 or internal energy <= 0",
                (unsigned long long)c->st_host->not_admissible);
  }
  st = reset_status(c);
  if (st) return st;
  c->have_state = true;
  return EH_OK;
}

eh_status eh_get_state(eh_ctx *c, double *U_out, int is_device_ptr) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (!U_out) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  const size_t bytes = sizeof(double) * S_of(c) * c->n;
  CUDA_TRY(c, cudaMemcpyAsync(U_out, c->U, bytes, is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->stream));
  return check_device_error(c);
}

eh_status eh_apply_boundary_conditions(eh_ctx *c) {
  eh_status st = require_ready(c);
  if (st) return st;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (c->cfg.dim == 2) launch_apply_bc<2>(c->mv, c->prm, c->U, c->stream);
  else launch_apply_bc<3>(c->mv, c->prm, c->U, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  return EH_OK;
}

eh_status eh_cfl_dt(eh_ctx *c, double *dt) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (!dt) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if ((st = check_device_error(c))) return st;
  enqueue_cfl_any(c);
  launch_tau(c->mv, c->wk, 0, 0.0, c->prm.cfl, false, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  if ((st = check_device_error(c))) return st;
  *dt = c->st_host->stage_bound[0];
  return EH_OK;
}

eh_status eh_stage(eh_ctx *c, double tau, double *tau_used) {
  eh_status st = require_ready(c);
  if (st) return st;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if ((st = check_device_error(c))) return st;
  if ((st = ensure_trace_buffers(c))) return st;
  enqueue_stage_any(c, tau);
  CUDA_TRY(c, cudaGetLastError());
  c->last_stage_traced = true;
  if (tau_used) {
    if ((st = check_device_error(c))) return st;
    *tau_used = c->st_host->tau;
  }
  return EH_OK;
}

eh_status eh_step(eh_ctx *c, double dt, double *dt_used) {
  eh_status st = require_ready(c);
  if (st) return st;
  CUDA_TRY(c, cudaSetDevice(c->device));
  // the CFL step, or a prescribed dt the cached graph was captured with, is
  // one graph replay (as eh_run); another prescribed dt launches the step's
  // kernels one by one rather than capturing a graph for a single use
  if (c->profiling || (dt > 0.0 && !(c->graph && c->graph_dt == dt))) {
    enqueue_step_any(c, dt);
  } else {
    if ((st = ensure_graph(c, dt))) return st;
    CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
  }
  CUDA_TRY(c, cudaGetLastError());
  c->steps += 1;
  c->last_stage_traced = false;
  if (dt_used) {
    if ((st = check_device_error(c))) return st;
    *dt_used = c->st_host->tau;
    c->last_dt = *dt_used;
  }
  return EH_OK;
}

eh_status eh_run(eh_ctx *c, int32_t nsteps, double dt) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (nsteps < 0) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (c->profiling) {  // eager launches with event pairs
    for (int32_t k = 0; k < nsteps; ++k) enqueue_step_any(c, dt);
    CUDA_TRY(c, cudaGetLastError());
    c->steps += nsteps;
    c->last_stage_traced = false;
    return EH_OK;
  }
  if ((st = ensure_graph(c, dt))) return st;
  for (int32_t k = 0; k < nsteps; ++k) CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
  c->steps += nsteps;
  c->last_stage_traced = false;
  return EH_OK;
}

eh_status eh_step_adaptive(eh_ctx *c, double cfl_max, double *dt_used, double *cfl_used, int32_t *restarts) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (!(cfl_max > 0.0 && cfl_max <= 64.0)) return EH_ERR_INVALID_ARG;
  if (c->ninst != 1) return fail(c, EH_ERR_STATE, "eh_step_adaptive runs one instance");
  CUDA_TRY(c, cudaSetDevice(c->device));
  if ((st = check_device_error(c))) return st;
  const size_t bytes = sizeof(double) * S_of(c) * c->n;
  double t0 = 0.0;
  unsigned long long steps0 = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->Usave, c->U, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpy(&t0, c->wk.t_inst, sizeof(double), cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(&steps0, c->wk.steps_inst, sizeof(steps0), cudaMemcpyDeviceToHost));
  double cfl = cfl_max;
  int32_t r = 0;
  for (;;) {
    c->prm.cfl = cfl;
    CUDA_TRY(c, cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(&c->st->low_not_admissible, 0, sizeof(unsigned long long), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(&c->st->not_admissible, 0, sizeof(unsigned long long), c->stream));
    enqueue_step_any(c, 0.0);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpy(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    const int e = c->st_host->err;
    const bool failed = e == EH_ERR_NOT_ADMISSIBLE || c->st_host->low_not_admissible > 0;
    if (e && !failed) {
      c->prm.cfl = c->cfg.cfl;
      return check_device_error(c);
    }
    if (!failed) break;
    // put the state and the time back; clear the failure
    CUDA_TRY(c, cudaMemcpyAsync(c->U, c->Usave, bytes, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->wk.t_inst, &t0, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->wk.steps_inst, &steps0, sizeof(steps0), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (cfl <= 1.0) {  // cannot happen for an admissible state: U^L is then invariant-domain preserving
      c->prm.cfl = c->cfg.cfl;
      return fail(c, EH_ERR_NOT_ADMISSIBLE, "no admissible step down to c_cfl = %g", cfl);
    }
    cfl *= 0.5;
    ++r;
  }
  c->prm.cfl = c->cfg.cfl;
  c->steps += 1;
  c->last_stage_traced = false;
  if (dt_used) *dt_used = c->st_host->tau;
  if (cfl_used) *cfl_used = cfl;
  if (restarts) *restarts = r;
  return EH_OK;
}

// ---------------------------------------------------------------------------
// Sec. 5: the parabolic sub-step and the Strang-split Navier-Stokes step
// ---------------------------------------------------------------------------
eh_status eh_set_viscosity(eh_ctx *c, double mu, double lambda, double kappa_cv, const double *L, const double *G,
                           int32_t n_cells, int32_t nv, int32_t nq, const int32_t *cells, const double *qw,
                           const double *qphi, const double *qgrad, int32_t n_wall, const int32_t *wall, double cg_tol,
                           int32_t cg_max_iter) {
  if (!c) return EH_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, EH_ERR_STATE, "no mesh uploaded");
  if (c->cfg.dim != 2) return fail(c, EH_ERR_INVALID_ARG, "the parabolic step is implemented for 2D meshes");
  if (!(mu >= 0.0 && lambda >= 0.0 && kappa_cv >= 0.0) || !L || !G || n_cells <= 0 || (nv != 3 && nv != 4) ||
      nq < 1 || nq > 16 || !cells || !qw || !qphi || !qgrad || n_wall < 0 || (n_wall > 0 && !wall) ||
      !(cg_tol > 0.0 && cg_tol < 1.0) || cg_max_iter < 1)
    return fail(c, EH_ERR_INVALID_ARG, "invalid viscosity arguments");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int n = c->n;
  const int64_t nnz = c->nnz;
  for (int64_t q = 0; q < (int64_t)n_cells * nv; ++q)
    if (cells[q] < 0 || cells[q] >= n) return fail(c, EH_ERR_BAD_MESH, "cell node %d out of range", cells[q]);
  for (int q = 0; q < n_wall; ++q)
    if (wall[q] < 0 || wall[q] >= n) return fail(c, EH_ERR_BAD_MESH, "wall node %d out of range", wall[q]);
  free_parabolic(c);
  // host tables: diagonal positions, cells around every node, wall mask
  std::vector<int64_t> rp(n + 1), diag(n, -1);
  std::vector<int32_t> col(nnz);
  CUDA_TRY(c, cudaMemcpy(rp.data(), c->mv.row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(col.data(), c->mv.col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] == i) diag[i] = k;
  std::vector<int64_t> nc_ptr(n + 1, 0);
  for (int64_t q = 0; q < (int64_t)n_cells * nv; ++q) nc_ptr[cells[q] + 1]++;
  for (int i = 0; i < n; ++i) nc_ptr[i + 1] += nc_ptr[i];
  std::vector<int32_t> nc_cell(nc_ptr[n]), nc_local(nc_ptr[n]);
  std::vector<int64_t> fill(nc_ptr.begin(), nc_ptr.end() - 1);
  for (int e = 0; e < n_cells; ++e)
    for (int a = 0; a < nv; ++a) {
      const int i = cells[(int64_t)e * nv + a];
      nc_cell[fill[i]] = e;
      nc_local[fill[i]++] = a;
    }
  std::vector<unsigned char> wm(n, 0);
  for (int q = 0; q < n_wall; ++q) wm[wall[q]] = 1;
  auto palloc = [&](void **ptr, size_t bytes) -> eh_status {
    cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 8));
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_parabolic(c);
      return fail(c, EH_ERR_OOM, "cudaMalloc of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    c->par_allocs.push_back(*ptr);
    return EH_OK;
  };
  auto upload = [&](void **ptr, const void *src, size_t bytes) -> eh_status {
    eh_status st = palloc(ptr, bytes);
    if (st) return st;
    if (cudaMemcpy(*ptr, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      free_parabolic(c);
      return fail(c, EH_ERR_CUDA, "parabolic data upload");
    }
    return EH_OK;
  };
  ParView &v = c->pv;
  ParWork &w = c->pw;
  v = ParView{};
  w = ParWork{};
  void *p;
  eh_status st;
#define UP(field, type, src, count)                                            \
  if ((st = upload(&p, src, sizeof(type) * (size_t)(count)))) return st; \
  field = (type *)p;
  UP(v.diag, const int64_t, diag.data(), n);
  UP(v.L, const double, L, nnz);
  UP(v.cells, const int32_t, cells, (int64_t)n_cells * nv);
  UP(v.qw, const double, qw, (int64_t)n_cells * nq);
  UP(v.qphi, const double, qphi, (int64_t)n_cells * nq * nv);
  UP(v.qgrad, const double, qgrad, (int64_t)n_cells * nq * 2 * nv);
  UP(v.nc_ptr, const int64_t, nc_ptr.data(), n + 1);
  UP(v.nc_cell, const int32_t, nc_cell.data(), nc_ptr[n]);
  UP(v.nc_local, const int32_t, nc_local.data(), nc_ptr[n]);
  UP(v.wall, const unsigned char, wm.data(), n);
#undef UP
  v.n = n;
  v.nnz = nnz;
  v.row_ptr = c->mv.row_ptr;
  v.col = c->mv.col;
  v.mi = c->mv.mi;
  v.n_cells = n_cells;
  v.nv = nv;
  v.nq = nq;
  v.mu = mu;
  v.lam = lambda;
  v.kc = kappa_cv;
  {
    // the velocity operator's coefficients, formed once from G (not kept)
    if ((st = palloc(&p, sizeof(double) * 4 * (size_t)nnz))) return st;
    v.A = (const double *)p;
    void *g = nullptr;
    cudaError_t e = cudaMalloc(&g, sizeof(double) * 4 * (size_t)nnz);
    if (e == cudaSuccess) e = cudaMemcpy(g, G, sizeof(double) * 4 * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      par_vel_coef(v, (const double *)g, (double *)p, c->stream);
      e = cudaStreamSynchronize(c->stream);
    }
    if (g) cudaFree(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_parabolic(c);
      return fail(c, e == cudaErrorMemoryAllocation ? EH_ERR_OOM : EH_ERR_CUDA, "velocity coefficients: %s",
                  cudaGetErrorString(e));
    }
  }
#define WA(field, count)                                                  \
  if ((st = palloc(&p, sizeof(double) * (size_t)(count)))) return st; \
  field = (double *)p;
  WA(w.D, n);
  WA(w.V, 2 * n);
  WA(w.Vh, 2 * n);
  WA(w.x, 2 * n);
  WA(w.b, 2 * n);
  WA(w.iPd, 2 * n);
  WA(w.r, 2 * n);
  WA(w.z, 2 * n);
  WA(w.d, 2 * n);
  WA(w.q, 2 * n);
  WA(w.en, n);
  WA(w.eH, n);
  WA(w.eL, n);
  WA(w.K, n);
  WA(w.Rp, n);
  WA(w.Rm, n);
  WA(w.ce, (int64_t)n_cells * nv);
  WA(w.part, 3 * kRedBlocks);
  WA(w.scal, 8);
#undef WA
  if ((st = palloc(&p, sizeof(int)))) return st;
  w.flag = (int *)p;
  if ((st = palloc(&p, sizeof(int) * 2))) return st;
  w.ctl = (int *)p;
  if ((st = palloc(&p, sizeof(unsigned)))) return st;
  w.count = (unsigned *)p;
  if (cudaMemset(w.count, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    free_parabolic(c);
    return fail(c, EH_ERR_CUDA, "reduction counter");
  }
  if ((!c->host_scal && cudaMallocHost(&c->host_scal, sizeof(double) * 2) != cudaSuccess) ||
      (!c->host_ctl && cudaMallocHost(&c->host_ctl, sizeof(int) * 2) != cudaSuccess)) {
    cudaGetLastError();
    free_parabolic(c);
    return fail(c, EH_ERR_OOM, "pinned scalars");
  }
  c->cg_tol = cg_tol;
  c->cg_max_iter = cg_max_iter;
  c->have_visc = true;
  return EH_OK;
}

namespace {

// reads one device scalar (synchronises)
eh_status read_scal(eh_ctx *c, int slot, double *out) {
  CUDA_TRY(c, cudaMemcpyAsync(c->host_scal, c->pw.scal + slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *out = c->host_scal[0];
  return EH_OK;
}

// Diagonally preconditioned CG on (D + coef A) x = b (velocity, m = 2n) or
// (D + coef L) x = b (energy, m = n); x holds the initial guess. Stops when
// ||r|| <= tol ||b||; *iters = the iteration count (-1: no convergence).
// Iterations are queued in batches (the first as long as the last solve of
// the same system took, then two at a time) and the host reads the device's
// control pair after each batch; iterations queued past convergence do
// nothing, so the result does not depend on the batching.
eh_status run_pcg(eh_ctx *c, bool velocity, double coef, int which, int *iters) {
  const ParView &v = c->pv;
  const ParWork &w = c->pw;
  cudaStream_t s = c->stream;
  const int64_t m = velocity ? 2 * (int64_t)c->n : c->n;
  const int *skip = w.ctl + CTL_DONE;
  auto apply = [&](const double *x, double *y, const int *sk) {
    if (velocity) par_vel_apply(v, w, coef, x, y, sk, s); else par_en_apply(v, w, coef, x, y, sk, s);
  };
  apply(w.x, w.q, nullptr);
  par_cg_init(w, m, c->cg_tol, s);
  int k = 0, batch = std::max(1, c->cg_last[which]);
  while (k < c->cg_max_iter) {
    const int nb = std::min(batch, c->cg_max_iter - k);
    for (int b = 0; b < nb; ++b) {
      apply(w.d, w.q, skip);
      par_cg_alpha(w, m, s);
      par_cg_update(w, m, s);
      par_cg_dir(w, m, s);
    }
    k += nb;
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(c->host_ctl, w.ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (c->host_ctl[CTL_DONE]) {
      *iters = c->host_ctl[CTL_IT];
      c->cg_last[which] = *iters;
      return EH_OK;
    }
    batch = 2;
  }
  *iters = -1;
  return EH_OK;
}

}  // namespace

eh_status eh_parabolic_step(eh_ctx *c, double dt, eh_parabolic_info *info) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (!c->have_visc) return fail(c, EH_ERR_STATE, "no viscosity data (eh_set_viscosity)");
  if (!(dt > 0.0)) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if ((st = check_device_error(c))) return st;
  const ParView &v = c->pv;
  const ParWork &w = c->pw;
  cudaStream_t s = c->stream;
  eh_parabolic_info out{};
  // velocity (eq. mt_parabolic_discrete): (D + dt/2 A) V^{n+1/2} = D V^n
  par_init(v, w, c->U, dt, s);
  int it;
  if ((st = run_pcg(c, true, 0.5 * dt, 0, &it))) return st;
  if (it < 0) return fail(c, EH_ERR_NOT_ADMISSIBLE, "velocity CG did not converge");
  out.cg_iter_velocity = it;
  CUDA_TRY(c, cudaMemcpyAsync(w.Vh, w.x, sizeof(double) * 2 * c->n, cudaMemcpyDeviceToDevice, s));
  // internal energy (eqs. def_Ki_nplusone, high_int_energy_CN)
  par_cell_source(v, w, w.Vh, s);
  par_source(v, w, s);
  par_en_rhs(v, w, 0.5 * dt, 0.5 * dt * v.kc, s);
  if ((st = run_pcg(c, false, 0.5 * dt * v.kc, 1, &it))) return st;
  if (it < 0) return fail(c, EH_ERR_NOT_ADMISSIBLE, "energy CG did not converge");
  out.cg_iter_energy = it;
  CUDA_TRY(c, cudaMemsetAsync(w.flag, 0, sizeof(int), s));
  par_en_extrapolate(v, w, s);
  int flag = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&flag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  if (flag) {
    // low-order update and FCT (eqs. low_order_update_internal_energy, Aij_for_internal_energy)
    par_en_rhs(v, w, dt, dt * v.kc, s);
    if ((st = run_pcg(c, false, dt * v.kc, 2, &it))) return st;
    if (it < 0) return fail(c, EH_ERR_NOT_ADMISSIBLE, "low-order energy CG did not converge");
    out.cg_iter_low = it;
    out.limited = 1;
    CUDA_TRY(c, cudaMemcpyAsync(w.eL, w.x, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
    par_fct(v, w, dt, s);
  }
  par_final(v, w, c->U, s);
  par_min_e(v, w, SC_TMP, s);
  CUDA_TRY(c, cudaGetLastError());
  if ((st = read_scal(c, SC_TMP, &out.min_e))) return st;
  if (info) *info = out;
  return EH_OK;
}

eh_status eh_step_ns(eh_ctx *c, double dt, double *tau_used, eh_parabolic_info *info) {
  if (!c) return EH_ERR_INVALID_ARG;
  if (!c->have_visc) return fail(c, EH_ERR_STATE, "no viscosity data (eh_set_viscosity)");
  double tau = 0.0;
  eh_status st = eh_step(c, dt, &tau);  // H(tau)
  if (st) return st;
  if ((st = eh_parabolic_step(c, 2.0 * tau, info))) return st;  // P(2 tau)
  if ((st = eh_step(c, tau, nullptr))) return st;  // H(tau)
  if ((st = check_device_error(c))) return st;
  if (tau_used) *tau_used = tau;
  return EH_OK;
}

eh_status eh_synchronize(eh_ctx *c) {
  if (!c) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  return check_device_error(c);
}

eh_status eh_get_diagnostics(eh_ctx *c, eh_diagnostics *out) {
  if (!c || !out) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  eh_status st = check_device_error(c);
  memset(out, 0, sizeof(*out));
  double t0 = 0.0;  // simulated time of instance 0, advanced on the device
  CUDA_TRY(c, cudaMemcpy(&t0, c->wk.t_inst, sizeof(double), cudaMemcpyDeviceToHost));
  out->t = t0;
  out->steps = c->steps;
  out->last_dt = c->st_host->tau;
  for (int q = 0; q < 3; ++q) out->last_stage_bound[q] = c->st_host->stage_bound[q];
  out->cfl_violations = (int64_t)c->st_host->cfl_violations;
  out->not_admissible = (int64_t)c->st_host->not_admissible;
  out->line_searches_deferred = (int64_t)c->st_host->line_searches_deferred;
  out->line_searches_iterated = (int64_t)c->st_host->line_searches_iterated;
  out->low_order_not_admissible = (int64_t)c->st_host->low_not_admissible;
  if (c->have_state) {
    double stats[8] = {0.0};
    if (c->cfg.dim == 2) launch_state_stats<2>(c->n, c->U, c->mv.mi, c->stat_part, c->stat_out, c->stream);
    else launch_state_stats<3>(c->n, c->U, c->mv.mi, c->stat_part, c->stat_out, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(stats, c->stat_out, sizeof(double) * (c->cfg.dim + 4), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    out->rho_min = stats[0];
    out->e_min = stats[1];
    for (int q = 0; q < c->cfg.dim + 2; ++q) out->total[q] = stats[2 + q];
  }
  return st;
}

eh_status eh_set_instances(eh_ctx *c, int32_t ninst, const int64_t *row_offset, const double *t_final) {
  if (!c || ninst < 1 || !row_offset) return EH_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, EH_ERR_STATE, "no mesh uploaded");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (row_offset[0] != 0 || row_offset[ninst] != c->n)
    return fail(c, EH_ERR_INVALID_ARG, "instance offsets must start at 0 and end at n");
  for (int k = 0; k < ninst; ++k)
    if (row_offset[k + 1] <= row_offset[k]) return fail(c, EH_ERR_INVALID_ARG, "instance %d is empty", k);
  // no CSR entry may couple two instances
  std::vector<int64_t> rp(c->n + 1);
  std::vector<int32_t> col(c->nnz);
  CUDA_TRY(c, cudaMemcpy(rp.data(), c->mv.row_ptr, sizeof(int64_t) * (c->n + 1), cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(col.data(), c->mv.col, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToHost));
  for (int k = 0; k < ninst; ++k)
    for (int64_t i = row_offset[k]; i < row_offset[k + 1]; ++i)
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (col[q] < row_offset[k] || col[q] >= row_offset[k + 1])
          return fail(c, EH_ERR_BAD_MESH, "row %lld couples instances", (long long)i);
  return setup_instances(c, ninst, row_offset, t_final);
}

eh_status eh_get_instances(eh_ctx *c, double *t, double *last_dt, double *stage_bound) {
  if (!c) return EH_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, EH_ERR_STATE, "no mesh uploaded");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const size_t b = sizeof(double) * c->ninst;
  if (t) CUDA_TRY(c, cudaMemcpy(t, c->wk.t_inst, b, cudaMemcpyDeviceToHost));
  if (last_dt) CUDA_TRY(c, cudaMemcpy(last_dt, c->wk.tau_inst, b, cudaMemcpyDeviceToHost));
  if (stage_bound) CUDA_TRY(c, cudaMemcpy(stage_bound, c->wk.bound_inst, 3 * b, cudaMemcpyDeviceToHost));
  return check_device_error(c);
}

eh_status eh_get_instance_steps(eh_ctx *c, int64_t *steps) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (!steps) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<unsigned long long> tmp(c->ninst);
  CUDA_TRY(c, cudaMemcpy(tmp.data(), c->wk.steps_inst, sizeof(unsigned long long) * c->ninst, cudaMemcpyDeviceToHost));
  for (int k = 0; k < c->ninst; ++k) steps[k] = (int64_t)tmp[k];
  return EH_OK;
}

eh_status eh_autotune(eh_ctx *c, int32_t steps_per_candidate, int32_t *chosen) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (steps_per_candidate < 1) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if ((st = check_device_error(c))) return st;
  const size_t bytes = sizeof(double) * S_of(c) * c->n;
  const size_t tb = sizeof(double) * c->ninst;
  std::vector<double> t_saved(c->ninst);
  std::vector<unsigned long long> steps_saved(c->ninst);
  CUDA_TRY(c, cudaMemcpyAsync(c->Usave, c->U, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpy(t_saved.data(), c->wk.t_inst, tb, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(steps_saved.data(), c->wk.steps_inst, sizeof(unsigned long long) * c->ninst,
                         cudaMemcpyDeviceToHost));
  // candidates: block sizes 64/128/256, each with the grid-stride kernels
  // (lim1, pass, final) at one thread per row or 8/16/24 warps in flight per SM
  const int cands[3] = {64, 128, 256};
  const int caps[4] = {0, 256, 512, 768};
  double best_ms[EH_KERNEL_COUNT];
  int best[EH_KERNEL_COUNT], best_cap[EH_KERNEL_COUNT];
  for (int k = 0; k < EH_KERNEL_COUNT; ++k) {
    best_ms[k] = INFINITY;
    best[k] = c->tpb[k];
    best_cap[k] = c->rows_per_sm[k];
  }
  const bool was_profiling = c->profiling;
  for (int q = 0; q < 3; ++q) {
    for (int r = 0; r < 4; ++r) {
      for (int k = 0; k < EH_KERNEL_COUNT; ++k) {
        if (k != EH_KERNEL_TAU) c->tpb[k] = cands[q];
        c->rows_per_sm[k] = (k == EH_KERNEL_LIM1 || k == EH_KERNEL_PASS || k == EH_KERNEL_FINAL) ? caps[r] : 0;
      }
      if ((st = eh_profile_enable(c, 1))) return st;
      CUDA_TRY(c, cudaMemcpyAsync(c->U, c->Usave, bytes, cudaMemcpyDeviceToDevice, c->stream));
      for (int32_t it = 0; it < steps_per_candidate; ++it) enqueue_step_any(c, 0.0);
      CUDA_TRY(c, cudaGetLastError());
      flush_profile(c);
      for (int k = 0; k < EH_KERNEL_COUNT; ++k)
        if (k != EH_KERNEL_TAU && c->prof_count[k] && c->prof_ms[k] < best_ms[k]) {
          best_ms[k] = c->prof_ms[k];
          best[k] = cands[q];
          best_cap[k] = c->rows_per_sm[k];
        }
    }
  }
  eh_profile_enable(c, was_profiling ? 1 : 0);
  for (int k = 0; k < EH_KERNEL_COUNT; ++k) {
    c->tpb[k] = best[k];
    c->rows_per_sm[k] = best_cap[k];
    if (chosen) chosen[k] = best[k];
  }
  // put the state and the instance times back
  CUDA_TRY(c, cudaMemcpyAsync(c->U, c->Usave, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->wk.t_inst, t_saved.data(), tb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->wk.steps_inst, steps_saved.data(), sizeof(unsigned long long) * c->ninst,
                              cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return check_device_error(c);
}

eh_status eh_profile_enable(eh_ctx *c, int enable) {
  if (!c) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  flush_profile(c);
  c->profiling = enable != 0;
  for (int k = 0; k < EH_KERNEL_COUNT; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_count[k] = 0;
  }
  return EH_OK;
}

eh_status eh_profile_read(eh_ctx *c, int kernel, double *total_ms, int64_t *launches) {
  if (!c || kernel < 0 || kernel >= EH_KERNEL_COUNT || !total_ms || !launches) return EH_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  flush_profile(c);
  *total_ms = c->prof_ms[kernel];
  *launches = c->prof_count[kernel];
  return EH_OK;
}

eh_status eh_get_block_sizes(const eh_ctx *c, int32_t *tpb) {
  if (!c || !tpb) return EH_ERR_INVALID_ARG;
  for (int k = 0; k < EH_KERNEL_COUNT; ++k) tpb[k] = c->tpb[k];
  return EH_OK;
}

eh_status eh_get_rows_per_sm(const eh_ctx *c, int32_t *rows) {
  if (!c || !rows) return EH_ERR_INVALID_ARG;
  for (int k = 0; k < EH_KERNEL_COUNT; ++k) rows[k] = c->rows_per_sm[k];
  return EH_OK;
}

eh_status eh_set_launch_shape(eh_ctx *c, int32_t kernel, int32_t threads_per_block, int32_t rows_per_sm) {
  if (!c || kernel < 0 || kernel >= EH_KERNEL_COUNT || kernel == EH_KERNEL_TAU) return EH_ERR_INVALID_ARG;
  if (threads_per_block != 64 && threads_per_block != 128 && threads_per_block != 256) return EH_ERR_INVALID_ARG;
  if (rows_per_sm < 0 || rows_per_sm > 2048) return EH_ERR_INVALID_ARG;
  if (rows_per_sm > 0 && kernel != EH_KERNEL_LIM1 && kernel != EH_KERNEL_PASS && kernel != EH_KERNEL_FINAL)
    return EH_ERR_INVALID_ARG;
  c->tpb[kernel] = threads_per_block;
  c->rows_per_sm[kernel] = rows_per_sm;
  if (c->graph) {  // the captured graph holds the old launch shapes
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return EH_OK;
}

int32_t eh_launches_per_step(const eh_ctx *c) {
  if (!c) return 0;
  // prep, visc, alpha, low, tau, lim1, (passes - 1) x pass, final; three stages
  // per stage: prep, visc, alpha, low, tau, lim1, final, one k_pass per
  // further pass and k_ls_deferred + k_ls_iterate per pass
  return 3 * (7 + (c->cfg.limiter_passes - 1) + 2 * c->cfg.limiter_passes + (c->mv.n_nonreflecting > 0 ? 1 : 0));
}

eh_status eh_get_mesh_index(eh_ctx *c, int64_t *row_ptr, int32_t *col, int32_t *transpose) {
  if (!c) return EH_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, EH_ERR_STATE, "no mesh uploaded");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (row_ptr)
    CUDA_TRY(c, cudaMemcpy(row_ptr, c->mv.row_ptr, sizeof(int64_t) * (c->n + 1), cudaMemcpyDeviceToHost));
  if (col) CUDA_TRY(c, cudaMemcpy(col, c->mv.col, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToHost));
  if (transpose) CUDA_TRY(c, cudaMemcpy(transpose, c->mv.tr, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToHost));
  return EH_OK;
}

eh_status eh_trace(eh_ctx *c, int what, double *host_out, int64_t count) {
  eh_status st = require_ready(c);
  if (st) return st;
  if (!host_out) return EH_ERR_INVALID_ARG;
  if (!c->last_stage_traced) return fail(c, EH_ERR_STATE, "eh_trace needs a preceding eh_stage");
  CUDA_TRY(c, cudaSetDevice(c->device));
  if ((st = check_device_error(c))) return st;
  const int S = S_of(c), SP = SP_of(c);
  const int64_t n = c->n, nnz = c->nnz;
  auto aos_to_soa = [&](const double *dev, int stride, int comps) -> eh_status {
    if (count != comps * n) return fail(c, EH_ERR_INVALID_ARG, "count must be %lld", (long long)(comps * n));
    std::vector<double> tmp((size_t)n * stride);
    CUDA_TRY(c, cudaMemcpy(tmp.data(), dev, sizeof(double) * n * stride, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
      for (int s = 0; s < comps; ++s) host_out[s * n + i] = tmp[i * stride + s];
    return EH_OK;
  };
  auto plain = [&](const double *dev, int64_t len) -> eh_status {
    if (count != len) return fail(c, EH_ERR_INVALID_ARG, "count must be %lld", (long long)len);
    CUDA_TRY(c, cudaMemcpy(host_out, dev, sizeof(double) * len, cudaMemcpyDeviceToHost));
    return EH_OK;
  };
  // d_ij and F^H live in the viscosity precision (float in mixed mode)
  auto vcopy = [&](const void *dev, int64_t len, std::vector<double> &dst) -> eh_status {
    dst.resize(len);
    if (mixed(c)) {
      std::vector<float> tmp(len);
      CUDA_TRY(c, cudaMemcpy(tmp.data(), dev, sizeof(float) * len, cudaMemcpyDeviceToHost));
      for (int64_t q = 0; q < len; ++q) dst[q] = tmp[q];
    } else {
      CUDA_TRY(c, cudaMemcpy(dst.data(), dev, sizeof(double) * len, cudaMemcpyDeviceToHost));
    }
    return EH_OK;
  };
  std::vector<double> buf;
  switch (what) {
    case EH_TRACE_D_IJ:
      if (count != nnz) return fail(c, EH_ERR_INVALID_ARG, "count must be %lld", (long long)nnz);
      if (c->cfg.dim == 3 || mixed(c)) {  // packed slots [w (S), a, d, 0...]
        const int spw = 8, dpos = c->cfg.dim + 3;
        if ((st = vcopy(c->wk.vw, nnz * spw, buf))) return st;
        for (int64_t k = 0; k < nnz; ++k) host_out[k] = buf[k * spw + dpos];
        return EH_OK;
      }
      if ((st = vcopy(c->wk.vd, nnz, buf))) return st;
      std::copy(buf.begin(), buf.end(), host_out);
      return EH_OK;
    case EH_TRACE_ALPHA:  // stored halved
      if ((st = plain(c->wk.alpha, n))) return st;
      for (int64_t i = 0; i < n; ++i) host_out[i] *= 2.0;
      return EH_OK;
    case EH_TRACE_U_LOW: return aos_to_soa(c->wk.UL, SP, S);
    case EH_TRACE_F_HIGH: {  // stored as F^H_i / m_i
      if (count != S * n) return fail(c, EH_ERR_INVALID_ARG, "count must be %lld", (long long)(S * n));
      if ((st = vcopy(c->wk.vFH, n * SP, buf))) return st;
      std::vector<double> mi_host(n);
      CUDA_TRY(c, cudaMemcpy(mi_host.data(), c->mv.mi, sizeof(double) * n, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < n; ++i)
        for (int s = 0; s < S; ++s) host_out[s * n + i] = buf[i * SP + s] * mi_host[i];
      return EH_OK;
    }
    case EH_TRACE_BOUNDS: return aos_to_soa(c->wk.bounds, 4, 3);
    case EH_TRACE_L_PASS1:
      if (c->cfg.limiter_passes < 2) return fail(c, EH_ERR_STATE, "L_PASS1 needs limiter_passes >= 2");
      return plain(c->trace_lsym, nnz);
    case EH_TRACE_U_PASS1:
      return aos_to_soa(c->cfg.limiter_passes >= 2 ? c->trace_upass : c->trace_pre, SP, S);
    case EH_TRACE_P_PASS1: {
      if (count != S * nnz) return fail(c, EH_ERR_INVALID_ARG, "count must be %lld", (long long)(S * nnz));
      std::vector<double> tmp((size_t)nnz * SP);
      CUDA_TRY(c, cudaMemcpy(tmp.data(), c->trace_P, sizeof(double) * nnz * SP, cudaMemcpyDeviceToHost));
      for (int64_t k = 0; k < nnz; ++k)
        for (int s = 0; s < S; ++s) host_out[s * nnz + k] = tmp[k * SP + s];
      return EH_OK;
    }
    case EH_TRACE_L_LAST: return plain(c->trace_llast, nnz);
    case EH_TRACE_TAU:
      if (count != 1) return EH_ERR_INVALID_ARG;
      host_out[0] = c->st_host->tau;
      return EH_OK;
    case EH_TRACE_TAU_BOUND:
      if (count != 1) return EH_ERR_INVALID_ARG;
      host_out[0] = c->st_host->stage_bound[0];
      return EH_OK;
    default: return fail(c, EH_ERR_INVALID_ARG, "unknown trace selector %d", what);
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// merged served batch (internal.cuh)
// ---------------------------------------------------------------------------
namespace ehi {

cudaStream_t stream_of(const eh_ctx *c) { return c->stream; }

uint64_t part_bytes(int dim, int precision, int64_t n, int64_t nnz, int64_t n_bnd) {
  const int64_t S = dim + 2;
  int64_t per_entry = 4 + 4 + 8 * dim + 8 * 3, per_node = 8 + 8 * 4 + 1 + 4 + 8 * S + 8 * 4;
  if (precision == EH_PRECISION_MIXED) per_entry += 4 * (dim + 2);
  return (uint64_t)(per_entry * nnz + per_node * n + (8 + 8 * dim + 8 * S) * n_bnd) + (1u << 16);
}

eh_status create_part(const eh_config *cfg, cudaStream_t stream, int32_t n, int64_t nnz, const int64_t *row_ptr,
                      const int32_t *col, const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                      const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                      const double *bnd_state, const double *U0, eh_ctx **out) {
  *out = nullptr;
  eh_config c2 = *cfg;
  c2.stream = (void *)stream;
  eh_ctx *p = nullptr;
  eh_status st = eh_create(&c2, &p);
  if (st) return st;
  p->static_only = true;
  if (!st) st = eh_upload_mesh(p, n, nnz, row_ptr, col, cij, mij, mi, n_bnd, bnd_node, bnd_kind, bnd_normal, bnd_state);
  if (!st) st = eh_set_state(p, U0, 0);
  if (!st) st = eh_apply_boundary_conditions(p);
  if (!st) st = eh_synchronize(p);
  if (st) {
    eh_destroy(p);
    return st;
  }
  *out = p;
  return EH_OK;
}

eh_status assemble(eh_ctx *uni, eh_ctx *const *parts, int count, const double *t, const double *t_final) {
  if (!uni || count < 1) return EH_ERR_INVALID_ARG;
  CUDA_TRY(uni, cudaSetDevice(uni->device));
  CUDA_TRY(uni, cudaStreamSynchronize(uni->stream));
  const int dim = uni->cfg.dim, S = S_of(uni);
  int64_t N = 0, NNZ = 0, NB = 0;
  for (int k = 0; k < count; ++k) {
    N += parts[k]->n;
    NNZ += parts[k]->nnz;
    NB += parts[k]->n_bnd;
  }
  if (N > INT32_MAX || NNZ >= ((int64_t)1 << 31)) return fail(uni, EH_ERR_INVALID_ARG, "merged batch too large");
  eh_status st;
  if (!uni->have_mesh || N > uni->cap_n || NNZ > uni->cap_nnz || NB > uni->cap_bnd) {
    free_mesh(uni);
    // room to grow: the next arrivals are placed without reallocating
    uni->cap_n = std::min<int64_t>(INT32_MAX, N + N / 4 + 1024);
    uni->cap_nnz = std::min<int64_t>(((int64_t)1 << 31) - 1, NNZ + NNZ / 4 + 16384);
    uni->cap_bnd = NB + NB / 4 + 256;
    if ((st = alloc_static(uni, uni->cap_n, uni->cap_nnz, uni->cap_bnd)) ||
        (st = alloc_work(uni, uni->cap_n, uni->cap_nnz))) {
      free_mesh(uni);
      uni->cap_n = uni->cap_nnz = uni->cap_bnd = 0;
      return st;
    }
  }
  MeshView &m = uni->mv;
  cudaStream_t s = uni->stream;
  auto cp = [&](const void *dst, const void *src, size_t bytes) {
    if (bytes) cudaMemcpyAsync(const_cast<void *>(dst), src, bytes, cudaMemcpyDeviceToDevice, s);
  };
  const size_t vsz = mixed(uni) ? sizeof(float) : sizeof(double);
  int64_t ro = 0, eo = 0, bo = 0;
  int nonrefl = 0;
  for (int k = 0; k < count; ++k) {
    const eh_ctx *p = parts[k];
    const MeshView &pm = p->mv;
    const int64_t n = p->n, nnz = p->nnz, nb = p->n_bnd;
    launch_offset_copy<int64_t>(const_cast<int64_t *>(m.row_ptr) + ro, pm.row_ptr, n, eo, false, s);
    launch_offset_copy<int32_t>(const_cast<int32_t *>(m.col) + eo, pm.col, nnz, (int32_t)ro, false, s);
    launch_offset_copy<int32_t>(const_cast<int32_t *>(m.tr) + eo, pm.tr, nnz, (int32_t)eo, false, s);
    for (int q = 0; q < dim; ++q) {
      cp(m.cij + (int64_t)q * NNZ + eo, pm.cij + (int64_t)q * nnz, sizeof(double) * nnz);
      cp((const char *)m.vcij + vsz * ((int64_t)q * NNZ + eo), (const char *)pm.vcij + vsz * (int64_t)q * nnz,
         vsz * nnz);
    }
    cp(m.cn + eo, pm.cn, sizeof(double) * nnz);
    cp(m.cinv + eo, pm.cinv, sizeof(double) * nnz);
    cp(m.betat + eo, pm.betat, sizeof(double) * nnz);
    if (mixed(uni)) {
      cp((const char *)m.vcn + vsz * eo, pm.vcn, vsz * nnz);
      cp((const char *)m.vcinv + vsz * eo, pm.vcinv, vsz * nnz);
    }
    cp(m.mi + ro, pm.mi, sizeof(double) * n);
    cp(m.inv_mi + ro, pm.inv_mi, sizeof(double) * n);
    cp(m.relax + ro, pm.relax, sizeof(double) * n);
    cp(m.lam + ro, pm.lam, sizeof(double) * n);
    cp(m.isb + ro, pm.isb, n);
    launch_offset_copy<int32_t>(const_cast<int32_t *>(m.bnd_index) + ro, pm.bnd_index, n, (int32_t)bo, true, s);
    launch_offset_copy<int32_t>(const_cast<int32_t *>(m.bnd_node) + bo, pm.bnd_node, nb, (int32_t)ro, false, s);
    cp(m.bnd_kind + bo, pm.bnd_kind, sizeof(int32_t) * nb);
    for (int q = 0; q < dim; ++q) cp(m.bnd_normal + (int64_t)q * NB + bo, pm.bnd_normal + (int64_t)q * nb, 8 * nb);
    for (int c = 0; c < S; ++c) cp(m.bnd_state + (int64_t)c * NB + bo, pm.bnd_state + (int64_t)c * nb, 8 * nb);
    for (int c = 0; c < S; ++c) cp(uni->U + (int64_t)c * N + ro, p->U + (int64_t)c * n, 8 * n);
    nonrefl += pm.n_nonreflecting;
    ro += n;
    eo += nnz;
    bo += nb;
  }
  CUDA_TRY(uni, cudaGetLastError());
  CUDA_TRY(uni, cudaMemcpyAsync(const_cast<int64_t *>(m.row_ptr) + N, &NNZ, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(uni, cudaStreamSynchronize(s));
  m.n = (int)N;
  m.nnz = NNZ;
  m.n_bnd = (int)NB;
  m.n_nonreflecting = nonrefl;
  uni->n = (int)N;
  uni->nnz = NNZ;
  uni->n_bnd = (int)NB;
  std::vector<int64_t> off(count + 1, 0);
  for (int k = 0; k < count; ++k) off[k + 1] = off[k] + parts[k]->n;
  if ((st = setup_instances(uni, count, off.data(), t_final))) return st;
  CUDA_TRY(uni, cudaMemcpy(uni->wk.t_inst, t, sizeof(double) * count, cudaMemcpyHostToDevice));
  if ((st = reset_status(uni))) return st;
  CUDA_TRY(uni, invalidate_records(uni));  // other meshes at the same rows
  CUDA_TRY(uni, cudaStreamSynchronize(s));
  uni->have_mesh = uni->have_state = true;
  uni->steps = 0;
  uni->last_stage_traced = false;
  return EH_OK;
}

eh_status scatter(eh_ctx *uni, eh_ctx *const *parts, int count) {
  CUDA_TRY(uni, cudaSetDevice(uni->device));
  const int S = S_of(uni);
  const int64_t N = uni->n;
  int64_t ro = 0;
  for (int k = 0; k < count; ++k) {
    const int64_t n = parts[k]->n;
    for (int c = 0; c < S; ++c)
      CUDA_TRY(uni, cudaMemcpyAsync(parts[k]->U + (int64_t)c * n, uni->U + (int64_t)c * N + ro, 8 * n,
                                    cudaMemcpyDeviceToDevice, uni->stream));
    ro += n;
  }
  CUDA_TRY(uni, cudaStreamSynchronize(uni->stream));
  return EH_OK;
}

}  // namespace ehi
