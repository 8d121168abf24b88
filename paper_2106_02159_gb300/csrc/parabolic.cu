// parabolic.cu -- sm_103a kernels of the parabolic sub-step S_P of
// arXiv:2106.02159 (Sec. 5) on 2D P1/Q1 meshes: the operators of the
// Crank-Nicolson velocity system (eq. mt_parabolic_discrete) and of the
// internal-energy systems (eqs. high_int_energy_CN,
// low_order_update_internal_energy), the pieces of diagonally preconditioned
// conjugate gradients, the viscous energy source K_i (eq. def_Ki_nplusone),
// the FCT limiting of the internal energy (eq. Aij_for_internal_energy) and
// the final update (eqs. vel_parabolic_discrete, energy_parabolic_discrete).
// The iteration itself is driven by the host (capi.cu). State layout [S][n]
// with S = 4; velocity vectors [n][2].
#include "parabolic.cuh"

#include <cmath>

namespace eh {
namespace {

constexpr int kT = 256;
inline unsigned grid_for(int64_t m) { return (unsigned)((m + kT - 1) / kT); }

__global__ void k_par_init(ParView v, ParWork w, const double *__restrict__ U, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int n = v.n;
  const double rho = U[i];
  const double D = rho * v.mi[i];
  const double vx = U[n + i] / rho, vy = U[2 * n + i] / rho;
  w.D[i] = D;
  w.V[2 * i] = vx;
  w.V[2 * i + 1] = vy;
  w.en[i] = U[3 * n + i] / rho - 0.5 * (vx * vx + vy * vy);
  const bool wl = v.wall[i] != 0;
  const int64_t kd = v.diag[i];
  const double lm = v.lam - 2.0 * v.mu / 3.0;
  const double c = 0.5 * dt;
  const double vv[2] = {vx, vy};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    w.b[2 * i + a] = wl ? 0.0 : D * vv[a];
    w.x[2 * i + a] = wl ? 0.0 : vv[a];
    const double Gaa = v.G[(a * 2 + a) * v.nnz + kd];
    w.Pd[2 * i + a] = wl ? 1.0 : D + c * (v.mu * v.L[kd] + v.mu * Gaa + lm * Gaa);
  }
}

// y = D x + coef A x with A_ij[a][m] = mu delta_am L_ij + mu G_ij[m][a] + (lambda - 2 mu/3) G_ij[a][m];
// wall rows are the identity, wall columns drop out
__global__ void k_vel_apply(ParView v, ParWork w, double coef, const double *__restrict__ x, double *__restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  if (v.wall[i]) {
    y[2 * i] = x[2 * i];
    y[2 * i + 1] = x[2 * i + 1];
    return;
  }
  const double lm = v.lam - 2.0 * v.mu / 3.0;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
    const int j = v.col[k];
    if (v.wall[j]) continue;
    const double L = v.L[k], g00 = v.G[k], g01 = v.G[v.nnz + k], g10 = v.G[2 * v.nnz + k], g11 = v.G[3 * v.nnz + k];
    const double x0 = x[2 * j], x1 = x[2 * j + 1];
    a0 += (v.mu * L + v.mu * g00 + lm * g00) * x0 + (v.mu * g10 + lm * g01) * x1;
    a1 += (v.mu * g01 + lm * g10) * x0 + (v.mu * L + v.mu * g11 + lm * g11) * x1;
  }
  const double D = w.D[i];
  y[2 * i] = D * x[2 * i] + coef * a0;
  y[2 * i + 1] = D * x[2 * i + 1] + coef * a1;
}

__global__ void k_en_apply(ParView v, ParWork w, double coef, const double *__restrict__ x, double *__restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  double acc = 0.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) acc += v.L[k] * x[v.col[k]];
  y[i] = w.D[i] * x[i] + coef * acc;
}

// block sums in a fixed tree; one partial per block
__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t m,
                              double *__restrict__ part) {
  __shared__ double sh[kT];
  double acc = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * kT + threadIdx.x; q < m; q += (int64_t)gridDim.x * kT) acc += a[q] * b[q];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double *__restrict__ part, int np, double *out) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) acc += part[q];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_min_partial(const double *__restrict__ a, int64_t m, double *__restrict__ part) {
  __shared__ double sh[kT];
  double acc = INFINITY;
  for (int64_t q = (int64_t)blockIdx.x * kT + threadIdx.x; q < m; q += (int64_t)gridDim.x * kT) acc = fmin(acc, a[q]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_min_partials(const double *__restrict__ part, int np, double *out) {
  double acc = INFINITY;
  for (int q = 0; q < np; ++q) acc = fmin(acc, part[q]);
  *out = acc;
}

__global__ void k_sub(const double *__restrict__ b, const double *__restrict__ q, double *__restrict__ r, int64_t m) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) r[s] = b[s] - q[s];
}

__global__ void k_precond(const double *__restrict__ r, const double *__restrict__ Pd, double *__restrict__ z,
                          double *__restrict__ d, int64_t m) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m) return;
  const double zz = r[s] / Pd[s];
  z[s] = zz;
  if (d) d[s] = zz;
}

__global__ void k_ratio(double *scal, int num, int den, int out) { scal[out] = scal[num] / scal[den]; }
__global__ void k_copy_scal(double *scal, int from, int to) { scal[to] = scal[from]; }

__global__ void k_xr_update(const double *__restrict__ scal, double *__restrict__ x, double *__restrict__ r,
                            const double *__restrict__ d, const double *__restrict__ q, int64_t m) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m) return;
  const double alpha = scal[SC_ALPHA];
  x[s] += alpha * d[s];
  r[s] -= alpha * q[s];
}

__global__ void k_d_update(const double *__restrict__ scal, double *__restrict__ d, const double *__restrict__ z,
                           int64_t m) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) d[s] = z[s] + scal[SC_BETA] * d[s];
}

// K_i = (1/m_i) int sigma(v):eps(v) phi_i over the cells around i (the
// quadrature values of sigma:eps recomputed per node; fixed order)
__global__ void k_source(ParView v, ParWork w, const double *__restrict__ vh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double lm = v.lam - 2.0 * v.mu / 3.0;
  double acc = 0.0;
  for (int64_t t = v.nc_ptr[i]; t < v.nc_ptr[i + 1]; ++t) {
    const int e = v.nc_cell[t], loc = v.nc_local[t];
    const int32_t *cn = v.cells + (int64_t)e * v.nv;
    for (int q = 0; q < v.nq; ++q) {
      const double *gr = v.qgrad + ((int64_t)e * v.nq + q) * 2 * v.nv;
      double d00 = 0.0, d01 = 0.0, d10 = 0.0, d11 = 0.0;  // d_km = d_m v_k
      for (int a = 0; a < v.nv; ++a) {
        const double g0 = gr[a], g1 = gr[v.nv + a];
        const double u0 = vh[2 * cn[a]], u1 = vh[2 * cn[a] + 1];
        d00 += u0 * g0;
        d01 += u0 * g1;
        d10 += u1 * g0;
        d11 += u1 * g1;
      }
      const double e01 = 0.5 * (d01 + d10), div = d00 + d11;
      const double se = 2.0 * v.mu * (d00 * d00 + 2.0 * e01 * e01 + d11 * d11) + lm * div * div;
      acc += v.qw[(int64_t)e * v.nq + q] * v.qphi[((int64_t)e * v.nq + q) * v.nv + loc] * se;
    }
  }
  w.K[i] = acc / v.mi[i];
}

__global__ void k_en_rhs(ParView v, ParWork w, double src, double coefL) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double D = w.D[i];
  w.b[i] = D * w.en[i] + src * v.mi[i] * w.K[i];
  w.x[i] = w.en[i];
  w.Pd[i] = D + coefL * v.L[v.diag[i]];
}

__global__ void k_en_extrapolate(ParView v, ParWork w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double e = 2.0 * w.x[i] - w.en[i];
  w.eH[i] = e;
  if (!(e > 0.0)) atomicExch(w.flag, 1);
}

// Zalesak's ratios with the bounds of the low-order solution on the stencil
__global__ void k_fct_ratios(ParView v, ParWork w, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double c = -0.5 * dt * v.kc;
  const double xi = w.eH[i] + w.en[i] - 2.0 * w.eL[i];
  double lo = w.eL[i], hi = w.eL[i], pp = 0.0, pm = 0.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
    const int j = v.col[k];
    if (j == i) continue;
    lo = fmin(lo, w.eL[j]);
    hi = fmax(hi, w.eL[j]);
    const double A = c * v.L[k] * ((w.eH[j] + w.en[j] - 2.0 * w.eL[j]) - xi);
    if (A > 0.0) pp += A; else pm += A;
  }
  const double D = w.D[i];
  w.Rp[i] = pp > 0.0 ? fmin(1.0, D * (hi - w.eL[i]) / pp) : 1.0;
  w.Rm[i] = pm < 0.0 ? fmin(1.0, D * (lo - w.eL[i]) / pm) : 1.0;
}

// limited update into x (eH still read by neighbours), then copied
__global__ void k_fct_apply(ParView v, ParWork w, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double c = -0.5 * dt * v.kc;
  const double xi = w.eH[i] + w.en[i] - 2.0 * w.eL[i];
  double acc = 0.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
    const int j = v.col[k];
    if (j == i) continue;
    const double A = c * v.L[k] * ((w.eH[j] + w.en[j] - 2.0 * w.eL[j]) - xi);
    const double l = A > 0.0 ? fmin(w.Rp[i], w.Rm[j]) : fmin(w.Rm[i], w.Rp[j]);
    acc += l * A;
  }
  w.x[i] = w.eL[i] + acc / w.D[i];
}

__global__ void k_final(ParView v, ParWork w, double *__restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int n = v.n;
  const double rho = U[i];
  const double v0 = 2.0 * w.Vh[2 * i] - w.V[2 * i], v1 = 2.0 * w.Vh[2 * i + 1] - w.V[2 * i + 1];
  U[n + i] = rho * v0;
  U[2 * n + i] = rho * v1;
  U[3 * n + i] = rho * w.eH[i] + 0.5 * rho * (v0 * v0 + v1 * v1);
}

}  // namespace

void par_init(const ParView &v, const ParWork &w, const double *U, double dt, cudaStream_t s) {
  k_par_init<<<grid_for(v.n), kT, 0, s>>>(v, w, U, dt);
}
void par_vel_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, cudaStream_t s) {
  k_vel_apply<<<grid_for(v.n), kT, 0, s>>>(v, w, coef, x, y);
}
void par_en_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, cudaStream_t s) {
  k_en_apply<<<grid_for(v.n), kT, 0, s>>>(v, w, coef, x, y);
}
void par_dot(const ParWork &w, const double *a, const double *b, int64_t m, int slot, cudaStream_t s) {
  k_dot_partial<<<kRedBlocks, kT, 0, s>>>(a, b, m, w.part);
  k_sum_partials<<<1, 1024, 0, s>>>(w.part, kRedBlocks, w.scal + slot);
}
void par_sub(const double *b, const double *q, double *r, int64_t m, cudaStream_t s) {
  k_sub<<<grid_for(m), kT, 0, s>>>(b, q, r, m);
}
void par_precond(const double *r, const double *Pd, double *z, double *d, int64_t m, cudaStream_t s) {
  k_precond<<<grid_for(m), kT, 0, s>>>(r, Pd, z, d, m);
}
void par_ratio(const ParWork &w, int num, int den, int out, cudaStream_t s) {
  k_ratio<<<1, 1, 0, s>>>(w.scal, num, den, out);
}
void par_copy_scal(const ParWork &w, int from, int to, cudaStream_t s) { k_copy_scal<<<1, 1, 0, s>>>(w.scal, from, to); }
void par_xr_update(const ParWork &w, double *x, double *r, const double *d, const double *q, int64_t m,
                   cudaStream_t s) {
  k_xr_update<<<grid_for(m), kT, 0, s>>>(w.scal, x, r, d, q, m);
}
void par_d_update(const ParWork &w, double *d, const double *z, int64_t m, cudaStream_t s) {
  k_d_update<<<grid_for(m), kT, 0, s>>>(w.scal, d, z, m);
}
void par_source(const ParView &v, const ParWork &w, const double *vh, cudaStream_t s) {
  k_source<<<grid_for(v.n), kT, 0, s>>>(v, w, vh);
}
void par_en_rhs(const ParView &v, const ParWork &w, double src, double coefL, cudaStream_t s) {
  k_en_rhs<<<grid_for(v.n), kT, 0, s>>>(v, w, src, coefL);
}
void par_en_extrapolate(const ParView &v, const ParWork &w, cudaStream_t s) {
  k_en_extrapolate<<<grid_for(v.n), kT, 0, s>>>(v, w);
}
void par_fct(const ParView &v, const ParWork &w, double dt, cudaStream_t s) {
  k_fct_ratios<<<grid_for(v.n), kT, 0, s>>>(v, w, dt);
  k_fct_apply<<<grid_for(v.n), kT, 0, s>>>(v, w, dt);
  cudaMemcpyAsync(w.eH, w.x, sizeof(double) * v.n, cudaMemcpyDeviceToDevice, s);
}
void par_final(const ParView &v, const ParWork &w, double *U, cudaStream_t s) {
  k_final<<<grid_for(v.n), kT, 0, s>>>(v, w, U);
}
void par_min_e(const ParView &v, const ParWork &w, int slot, cudaStream_t s) {
  k_min_partial<<<kRedBlocks, kT, 0, s>>>(w.eH, v.n, w.part);
  k_min_partials<<<1, 1, 0, s>>>(w.part, kRedBlocks, w.scal + slot);
}

}  // namespace eh
