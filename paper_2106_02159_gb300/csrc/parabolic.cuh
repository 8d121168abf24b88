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
  const double *G;        // [2][2][nnz] int d_k phi_i d_m phi_j
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
  double *x, *b, *Pd, *r, *z, *d, *q;  // [2n] CG vectors (the energy solves use the first n)
  double *en, *eH, *eL, *K;  // [n]
  double *Rp, *Rm;        // [n] FCT ratios
  double *part;           // [kRedBlocks] reduction partials
  double *scal;           // [8] device scalars (see enum below)
  int *flag;              // [1] a non-positive internal energy was met
};
enum { SC_DOT = 0, SC_RZ = 1, SC_ALPHA = 2, SC_BETA = 3, SC_RN2 = 4, SC_BN2 = 5, SC_TMP = 6 };
constexpr int kRedBlocks = 608;

void par_init(const ParView &v, const ParWork &w, const double *U, double dt, cudaStream_t s);
void par_vel_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, cudaStream_t s);
void par_en_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, cudaStream_t s);
// scal[slot] = a . b (deterministic: fixed grid, fixed reduction trees)
void par_dot(const ParWork &w, const double *a, const double *b, int64_t m, int slot, cudaStream_t s);
void par_sub(const double *b, const double *q, double *r, int64_t m, cudaStream_t s);             // r = b - q
void par_precond(const double *r, const double *Pd, double *z, double *d, int64_t m, cudaStream_t s);  // z = r/Pd (d = z if d)
void par_ratio(const ParWork &w, int num, int den, int out, cudaStream_t s);                         // scal[out] = scal[num]/scal[den]
void par_copy_scal(const ParWork &w, int from, int to, cudaStream_t s);
void par_xr_update(const ParWork &w, double *x, double *r, const double *d, const double *q, int64_t m,
                   cudaStream_t s);  // x += alpha d, r -= alpha q
void par_d_update(const ParWork &w, double *d, const double *z, int64_t m, cudaStream_t s);  // d = z + beta d
void par_source(const ParView &v, const ParWork &w, const double *vh, cudaStream_t s);      // K
// energy system: b = D e^n + src m K, x = e^n, Pd = D + coefL L_ii
void par_en_rhs(const ParView &v, const ParWork &w, double src, double coefL, cudaStream_t s);
void par_en_extrapolate(const ParView &v, const ParWork &w, cudaStream_t s);  // eH = 2 x - en; flag if <= 0
void par_fct(const ParView &v, const ParWork &w, double dt, cudaStream_t s);  // eH <- limited update from eL
void par_final(const ParView &v, const ParWork &w, double *U, cudaStream_t s);  // momentum, total energy from Vh, eH
void par_min_e(const ParView &v, const ParWork &w, int slot, cudaStream_t s);   // scal[slot] = min eH

}  // namespace eh
