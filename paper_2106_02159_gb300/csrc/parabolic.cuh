// parabolic.cuh -- device views and launchers of the parabolic sub-step of
// arXiv:2106.02159 (Sec. 5): Crank-Nicolson velocity and internal-energy
// solves, the viscous energy source and the FCT limiting of the internal
// energy, on 2D P1/Q1 meshes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eh {

struct ParView {
  int n;
  int64_t nnz;
  const int64_t *row_ptr;
  const int32_t *col;
  const int64_t *diag;    // position of the diagonal entry of every row
  const double *mi;
  const double *L;        // [nnz] int grad phi_i . grad phi_j
  const double *A;        // [nnz][2][2] A_ij[a][m] of the velocity operator, zero in wall columns
  int n_cells, nv, nq;
  const int32_t *cells;   // [n_cells][nv]
  const double *qw;       // [n_cells][nq]
  const double *qphi;     // [n_cells][nq][nv]
  const double *qgrad;    // [n_cells][nq][2][nv]
  const int64_t *nc_ptr;  // [n+1] cells around every node
  const int32_t *nc_cell; // cell ids
  const int32_t *nc_local;  // the node's index in that cell
  const unsigned char *wall;  // no-slip nodes
  double mu, lam, kc;     // shear and bulk viscosity, kappa / c_v
};

struct ParWork {
  double *D;              // [n] rho_i m_i
  double *V, *Vh;         // [n][2] velocity at t^n and the Crank-Nicolson midpoint value
  double *x, *b, *iPd, *r, *z, *d, *q;  // [2n] CG vectors, iPd the inverse diagonal preconditioner
                          // (the energy solves use the first n)
  double *en, *eH, *eL, *K;  // [n]
  double *Rp, *Rm;        // [n] FCT ratios
  double *ce;             // [n_cells][nv] the cells' shares of m_i K_i
  double *part;           // [3][kRedBlocks] reduction partials
  double *scal;           // [8] device scalars (see enum below)
  unsigned *count;        // [1] blocks of the running reduction that are done (0 between kernels)
  int *ctl;               // [2] CG control: converged flag, iterations done
  int *flag;              // [1] a non-positive internal energy was met
};
enum { SC_RZ = 0, SC_ALPHA = 1, SC_BETA = 2, SC_STOP = 3, SC_TMP = 4 };
enum { CTL_DONE = 0, CTL_IT = 1 };
constexpr int kRedBlocks = 608;  // 4 blocks of 256 threads per SM: the grid of every reduction

// A from L, the gradient integrals G ([2][2][nnz], int d_k phi_i d_m phi_j) and
// the wall mask of v (once per eh_set_viscosity)
void par_vel_coef(const ParView &v, const double *G, double *A, cudaStream_t s);
void par_init(const ParView &v, const ParWork &w, const double *U, double dt, cudaStream_t s);
// y = D x + coef (operator) x; nothing when skip && *skip
void par_vel_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, const int *skip,
                   cudaStream_t s);
void par_en_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, const int *skip,
                  cudaStream_t s);
// Diagonally preconditioned CG on vectors of length m, with q = (operator) x
// already applied: r = b - q, z = d = iPd r; scal[SC_STOP] = tol ||b||,
// ctl = {||r|| <= tol ||b||, 0}. Reductions in a fixed grid and fixed trees
// (deterministic); the last block to finish a reduction forms the scalars.
void par_cg_init(const ParWork &w, int64_t m, double tol, cudaStream_t s);
// with q = (operator) d: alpha = (r.z) / (d.q)
void par_cg_alpha(const ParWork &w, int64_t m, cudaStream_t s);
// x += alpha d, r -= alpha q, z = iPd r; one more iteration done; converged
// when ||r|| <= tol ||b||, else beta = (r.z)_new / (r.z)
void par_cg_update(const ParWork &w, int64_t m, cudaStream_t s);
// d = z + beta d
void par_cg_dir(const ParWork &w, int64_t m, cudaStream_t s);
// the three CG kernels do nothing once ctl[CTL_DONE] is set
void par_cell_source(const ParView &v, const ParWork &w, const double *vh, cudaStream_t s);  // ce
void par_source(const ParView &v, const ParWork &w, cudaStream_t s);                         // K from ce
// energy system: b = D e^n + src m K, x = e^n, iPd = 1 / (D + coefL L_ii)
void par_en_rhs(const ParView &v, const ParWork &w, double src, double coefL, cudaStream_t s);
void par_en_extrapolate(const ParView &v, const ParWork &w, cudaStream_t s);  // eH = 2 x - en; flag if <= 0
void par_fct(const ParView &v, const ParWork &w, double dt, cudaStream_t s);  // eH <- limited update from eL
void par_final(const ParView &v, const ParWork &w, double *U, cudaStream_t s);  // momentum, total energy from Vh, eH
void par_min_e(const ParView &v, const ParWork &w, int slot, cudaStream_t s);   // scal[slot] = min eH

}  // namespace eh
