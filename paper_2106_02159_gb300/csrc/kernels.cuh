// kernels.cuh -- device data views and kernel launchers of the forward-Euler
// stage (Algorithm 1 of arXiv:2106.02159, Appendix B) for sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eh {

// Padded state stride: 4 doubles in 2D (rho, m1, m2, E), 6 in 3D (5 used),
// so that every per-node / per-edge state vector starts on 16 bytes.
template <int DIM> struct Layout {
  static constexpr int S = DIM + 2;
  static constexpr int SP = DIM == 2 ? 4 : 6;
};

// Per-entry quantities of the viscosity kernel: w_ij (S values), a_ij, d_ij,
// in precision T. FP64 2D: w_ij in a 4-value slot (one 32-byte sector), a_ij
// and d_ij in arrays of their own. Otherwise (3D, and FP32 2D) one 8-value
// slot [w_ij (S), a_ij, d_ij, 0...] per entry, so that the write of an edge
// and its mirrored copy cover whole 32-byte sectors (partial slots and
// separate a/d writes left partial sectors that the L2 completed from DRAM).
template <int DIM, typename T> struct EdgeLayout {
  static constexpr bool packed = DIM == 3 || sizeof(T) == 4;
  static constexpr int SPW = packed ? 8 : 4;
  static constexpr int A = DIM + 2;  // packed: slot index of a_ij
  static constexpr int D = DIM + 3;  // packed: slot index of d_ij
};

// Node record written once per stage by k_prep and gathered by the edge loops:
// [0..S) state, then the primitive and derived quantities below. 2D: 16
// values (one 128-byte line), 3D: 24. The FP32 copy of mixed mode appends
// the flux f(U) (S x DIM, row-major) at F, rounded from FP64.
template <int DIM> struct Rec {
  static constexpr int V = DIM + 2;       // v_1..v_dim
  static constexpr int P = 2 * DIM + 2;   // pressure p
  static constexpr int A = 2 * DIM + 3;   // sound speed a
  static constexpr int AZ = 2 * DIM + 4;  // a p^{-z}, z = (gamma-1)/(2 gamma)
  static constexpr int IP = 2 * DIM + 5;  // 1/p
  static constexpr int PHI = 2 * DIM + 6; // Phi = eps rho^-gamma
  static constexpr int ETA = 2 * DIM + 7; // eta = -rho s
  static constexpr int EPS = 2 * DIM + 8; // internal energy eps
  static constexpr int H = 2 * DIM + 9;   // E + p
  static constexpr int IRHO = 2 * DIM + 10;  // 1/rho
  static constexpr int IEPS = 2 * DIM + 11;  // 1/eps
  static constexpr int SIZE = DIM == 2 ? 16 : 24;
  static_assert(IEPS < SIZE, "node record too small");
  static constexpr int F = SIZE;                                     // FP32 copy only
  static constexpr int VSIZE = SIZE + ((DIM + 2) * DIM + 7) / 8 * 8;  // FP32 copy: 24 (2D), 40 (3D)
};
constexpr int REC_MAX = 24;   // FP64 record stride allocated for either dimension
constexpr int VREC_MAX = 40;  // FP32 record stride allocated for either dimension
// stride of the record in the viscosity precision T
template <int DIM, typename T> __host__ __device__ constexpr int vrec_stride() {
  return sizeof(T) == 8 ? Rec<DIM>::SIZE : Rec<DIM>::VSIZE;
}

struct DevStatus {
  int err;                       // eh_status of a device-detected failure, 0 if none
  int pad;
  double tau;                    // the step's tau (fixed at the first stage)
  double stage_bound[3];         // c_cfl min_i m_i/(2|d_ii|) of the three stages
  unsigned long long cfl_violations;
  unsigned long long not_admissible;
  unsigned long long line_searches_deferred;  // searches the l = 1 check left open (cumulative)
  unsigned long long line_searches_iterated;  // of those, searches that ran the bracketing iteration
  unsigned long long low_not_admissible;      // rows whose low-order update U^L left the admissible set
};

struct MeshView {
  int n;
  int64_t nnz;
  const int64_t *row_ptr;
  const int32_t *col;
  const int32_t *tr;         // transpose position of every entry
  const double *cij;         // [dim][nnz]
  const double *cn;          // |c_ij|
  const double *cinv;        // 1/|c_ij|
  const double *betat;       // m_ij / m_i (the consistent mass matrix is symmetric)
  const double *mi;
  const double *inv_mi;
  const double *relax;       // r_i (0 when the bounds are strict)
  const double *lam;         // lambda_i = 1 / (card I(i) - 1)
  const unsigned char *isb;  // 1 for boundary nodes
  // arrays in the precision of the viscosity / flux part (double in FP64 mode,
  // float in mixed mode): c_ij [dim][nnz], |c_ij|, 1/|c_ij|
  const void *vcij;
  const void *vcn;
  const void *vcinv;
  const int32_t *bnd_index;  // per node: index into the boundary arrays, -1 inside
  const int32_t *bnd_node;   // [n_bnd] node of every boundary entry
  int n_nonreflecting;       // boundary nodes of the two non-reflecting kinds
  const int32_t *bnd_kind;   // [n_bnd]
  const double *bnd_normal;  // [dim][n_bnd]
  const double *bnd_state;   // [S][n_bnd]
  int n_bnd;
  // independent instances (block-diagonal CSR): rows [inst_row_off[k], inst_row_off[k+1])
  int ninst;
  const int32_t *inst;          // instance of every row
  const int64_t *inst_row_off;  // [ninst + 1]
};

struct Params {
  double gamma, cfl;
  int gamma75;               // gamma == 7/5 exactly: root/power fast paths
  double gm1;                // gamma - 1
  double z;                  // (gamma-1)/(2 gamma)
  double inv_z;              // 2 gamma/(gamma-1)
  double kshock;             // (gamma+1)/(2 gamma)
  double inv_gm1;            // 1/(gamma - 1)
  int limiter_passes;        // 1 + the passes of k_pass (k_final reads rem when >= 2)
};

struct Work {
  double *rec;     // [n][Rec<DIM>::SIZE]
  double *alpha;   // [n]      alpha_i / 2 (so that d^H_ij = (alpha_i/2 + alpha_j/2) d_ij, exactly as 0.5 (alpha_i + alpha_j) d_ij)
  // identical-state stencils (exact shortcuts, see k_visc): rough[i] = 1 when
  // some neighbour's state differs from U_i in any bit (zeroed by k_prep, set
  // by k_visc); rough2[i] = 1 when row i or one of its neighbours is rough
  // (written by k_low). A row with rough2 = 0 has P_ij = 0 on every entry.
  unsigned char *rough;   // [n]
  unsigned char *rough2;  // [n]
  // steady[i] (written by k_prep): bit 0 = U_i has the bits it had at the
  // previous k_prep (its record was kept), bit 1 = that, and node i was not
  // rough at the previous k_visc. An edge between two kept nodes one of
  // which also has bit 1 joins equal states whose edge values k_visc already
  // stored: it is skipped.
  unsigned char *steady;  // [n]
  // lone[q * n + i] = 1 when every limiter of row i in a pass is 1 (no entry
  // of the row went to the queued searches): written by k_lim1 (q = 0) and by
  // k_pass of pass p (q = p & 1), read by the next pass, which then needs no
  // gather of the transposed limiter for an entry between two such rows
  unsigned char *lone;    // [2][n]
  double *w;       // [nnz][SP]  (f(U_j) - f(U_i)) c_ij
  double *d;       // [nnz]      d^L_ij (diagonal: d_ii)
  double *inc;     // [n][SP]    sum_{j != i} d_ij (U_j - U_i) - w_ij
  double *FH;      // [n][SP]    F^H_i / m_i
  double *bounds;  // [n][4]     rho_min, rho_max, Phi_min
  double *UL;      // [n][SP]
  double *Ua;      // [n][SP]    limited state, ping
  double *Ub;      // [n][SP]    limited state, pong
  double *P;       // [nnz][SP]
  // rem[k] = 1 - l_ij of the last limiter pass (written by k_pass): that
  // pass leaves the remainder rem[k] P[k] for the next one, formed where it
  // is read and never stored (rem = 0: nothing left of P_ij); from the third
  // pass on, k_pass first writes its own input back to P
  double *rem;     // [nnz]
  double *la;      // [nnz]      limiter, ping
  double *lb;      // [nnz]      limiter, pong
  unsigned long long *bound_bits;  // [ninst] running minimum of c_cfl m_i / (2 sum_j d_ij) over the
                                   // instance's rows, as the bit pattern of a positive double (+inf between stages)
  double *tau_inst; // [ninst]   tau of each instance (fixed at the first stage)
  double *bound_inst;  // [3][ninst] CFL bound of each stage and instance
  double *t_inst;   // [ninst]   simulated time of each instance
  double *tfinal_inst; // [ninst] end time of each instance (+inf: none)
  unsigned long long *steps_inst;  // [ninst] steps taken with tau > 0
  DevStatus *st;
  // viscosity / flux precision arrays (aliases of rec, w, d, FH in FP64 mode;
  // float arrays in mixed mode)
  void *vrec;      // [n][Rec::SIZE] node record in that precision
  void *vw;        // [nnz][EdgeLayout::SPW] w_ij (and, packed, a_ij and d_ij)
  void *vd;        // [nnz]      d_ij (not packed)
  void *va;        // [nnz]      (q(U_j) - q(U_i)) . c_ij of the indicator (not packed)
  void *vFH;       // [n][SP]    F^H_i / m_i
  double *G64;     // [n][SP]    F^H_i / m_i in FP64 (mixed mode: the FP32 value widened once per node,
                   //            so that k_lim1 converts nothing per entry; FP64 mode: alias of FH)
  // line searches that the fast check at l = 1 left open, run by
  // k_ls_deferred after each limiter pass (one queue, reused by every pass)
  int2 *lsq;             // [lsq_cap] (row i, entry k)
  unsigned *lsq_count;   // [LSQ_SLOTS] entries queued by pass 0, 1, ... of the stage (zeroed by k_tau)
  unsigned lsq_cap;
  // the searches among those that need the bracketing iteration, queued by
  // k_ls_deferred for k_ls_iterate
  struct LsItem *lsq2;   // [lsq2_cap]
  unsigned *lsq2_count;  // [LSQ_SLOTS]
  unsigned lsq2_cap;
};

// a line search left to the bracketing iteration: row i, entry k, the bracket
// [0, l] with psi(0) = pl > 0, psi(l) = pr < 0 and rR = rho(l)^(-1/5)
struct LsItem {
  int i, k;
  double l, pl, pr, rR;
};
constexpr int LSQ_SLOTS = 8;  // limiter passes per stage, at most

// Launchers (all asynchronous on 'stream'). T is the precision of the
// viscosity / high-order-flux part: double (FP64 mode) or float (mixed mode).
// 'tpb' is the block size (threads = rows per block): 64, 128 or 256.
constexpr int TPB_MAX = 256;
template <int DIM, typename T>
void launch_prep(const MeshView &m, const Params &p, const double *U, const Work &w, int tpb, cudaStream_t s);
template <int DIM, typename T>
void launch_visc(const MeshView &m, const Params &p, const Work &w, int tpb, cudaStream_t s);
template <int DIM, typename T>
void launch_alpha(const MeshView &m, const Params &p, const Work &w, int tpb, cudaStream_t s);
template <int DIM, typename T>
void launch_low(const MeshView &m, const Params &p, const Work &w, int tpb, cudaStream_t s);
// per-instance minimum of the row bounds; stage 0 fixes tau (dt_given > 0:
// that step, else the bound), clipped to reach t_final; stage 2 advances t
void launch_tau(const MeshView &m, const Work &w, int stage, double dt_given, double cfl, bool advance_time,
                cudaStream_t s);
// lim1, pass and final loop over rows with a grid stride; max_blocks > 0 caps
// their grid (fewer rows in flight: less cache pressure from the gathers of
// long rows), 0 runs one thread per row
// P_trace (or NULL): P_ij of the pass, [nnz][SP], 0 on the diagonal
template <int DIM, typename T>
void launch_lim1(const MeshView &m, const Params &p, const Work &w, double *P_trace, int tpb, int max_blocks,
                 cudaStream_t s);
template <int DIM>
void launch_pass(const MeshView &m, const Params &p, const Work &w, const double *Uin, double *Uout, const double *lin,
                 double *lout, double *lsym_trace, int slot, int tpb, int max_blocks, cudaStream_t s);
// the queued line searches of pass 'slot' from the states ub ([n][SP]) and the
// stored P_ij; writes their limiters to lout
template <int DIM>
void launch_ls_deferred(const MeshView &m, const Params &p, const Work &w, const double *ub, int slot, double *lout,
                        int tpb, cudaStream_t s);
// out = SSP combination of U0 and BC(Uin + sum lambda l P): coef < 0 -> out = BC(...),
// else out = U0 + coef (BC(...) - U0). U0 / out are component-major [S][n].
template <int DIM>
void launch_final(const MeshView &m, const Params &p, const Work &w, const double *Uin, const double *lin,
                  const double *U0, double coef, double *out, double *Upre_trace, double *lsym_trace, int tpb,
                  int max_blocks, cudaStream_t s);
template <int DIM> void launch_apply_bc(const MeshView &m, const Params &p, double *U, cudaStream_t s);
template <int DIM> void launch_count_not_admissible(int n, const double *U, DevStatus *st, cudaStream_t s);
// out[0] = min rho, out[1] = min specific internal energy, out[2 + s] =
// sum_i m_i U_i[s] of the state U[S][n] (deterministic); part holds
// (DIM + 4) x STAT_BLOCKS partials
constexpr int STAT_BLOCKS = 304;
template <int DIM>
void launch_state_stats(int n, const double *U, const double *mi, double *part, double *out, cudaStream_t s);

// dst[i] = src[i] + add over count entries (nonneg_only: negative entries
// copied unchanged); int32_t and int64_t
template <typename I>
void launch_offset_copy(I *dst, const I *src, int64_t count, I add, bool nonneg_only, cudaStream_t s);

}  // namespace eh
