// parabolic.cu -- sm_103a kernels of the parabolic sub-step S_P of
// arXiv:2106.02159 (Sec. 5) on 2D P1/Q1 meshes: the operators of the
// Crank-Nicolson velocity system (eq. mt_parabolic_discrete) and of the
// internal-energy systems (eqs. high_int_energy_CN,
// low_order_update_internal_energy), the pieces of diagonally preconditioned
// conjugate gradients, the viscous energy source K_i (eq. def_Ki_nplusone),
// the FCT limiting of the internal energy (eq. Aij_for_internal_energy) and
// the final update (eqs. vel_parabolic_discrete, energy_parabolic_discrete).
// The CG iterations are queued by the host (capi.cu) in batches; their scalars
// live on the device. State layout [S][n] with S = 4; velocity vectors [n][2].
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
  const double c = 0.5 * dt;
  const double vv[2] = {vx, vy};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    w.b[2 * i + a] = wl ? 0.0 : D * vv[a];
    w.x[2 * i + a] = wl ? 0.0 : vv[a];
    w.iPd[2 * i + a] = wl ? 1.0 : 1.0 / (D + c * v.A[4 * kd + 3 * a]);
  }
}

// A_ij[a][m] = mu delta_am L_ij + mu G_ij[m][a] + (lambda - 2 mu/3) G_ij[a][m]
// (eq. mt_parabolic_discrete), zero where j is a wall node: the wall values
// are held at 0 and drop out of every row
__global__ void k_vel_coef(ParView v, const double *__restrict__ G, double *__restrict__ A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double lm = v.lam - 2.0 * v.mu / 3.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
    double *a = A + 4 * k;
    if (v.wall[v.col[k]]) {
      a[0] = a[1] = a[2] = a[3] = 0.0;
      continue;
    }
    const double L = v.L[k], g00 = G[k], g01 = G[v.nnz + k], g10 = G[2 * v.nnz + k], g11 = G[3 * v.nnz + k];
    a[0] = v.mu * L + v.mu * g00 + lm * g00;
    a[1] = v.mu * g10 + lm * g01;
    a[2] = v.mu * g01 + lm * g10;
    a[3] = v.mu * L + v.mu * g11 + lm * g11;
  }
}

// y = D x + coef A x; wall rows are the identity
__global__ void k_vel_apply(ParView v, ParWork w, double coef, const double *__restrict__ x, double *__restrict__ y,
                            const int *skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double2 xi = *(const double2 *)(x + 2 * i);
  if (v.wall[i]) {
    *(double2 *)(y + 2 * i) = xi;
    return;
  }
  double a0 = 0.0, a1 = 0.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
    const int j = v.col[k];
    const double2 r0 = *(const double2 *)(v.A + 4 * k), r1 = *(const double2 *)(v.A + 4 * k + 2);
    const double2 xj = *(const double2 *)(x + 2 * j);
    a0 += r0.x * xj.x + r0.y * xj.y;
    a1 += r1.x * xj.x + r1.y * xj.y;
  }
  const double D = w.D[i];
  *(double2 *)(y + 2 * i) = make_double2(D * xi.x + coef * a0, D * xi.y + coef * a1);
}

__global__ void k_en_apply(ParView v, ParWork w, double coef, const double *__restrict__ x, double *__restrict__ y,
                           const int *skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  double acc = 0.0;
  for (int64_t k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) acc += v.L[k] * x[v.col[k]];
  y[i] = w.D[i] * x[i] + coef * acc;
}

// ---------------------------------------------------------------------------
// conjugate-gradient kernels: grid-stride over kRedBlocks blocks of kT
// threads, block sums by fixed shuffle and shared-memory trees, and the block
// that finishes last sums the partials in a fixed order and forms the scalars
// ---------------------------------------------------------------------------
template <int NV> __device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0) sh[q][warp] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      v[q] = lane < kT / 32 ? sh[q][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
  }
  __syncthreads();
}

// thread 0 of every block passes its sums in v; returns true in the block that
// finishes last, whose thread 0 then holds the totals in v
template <int NV> __device__ __forceinline__ bool grid_sum(const ParWork &w, double (&v)[NV]) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) w.part[q * kRedBlocks + blockIdx.x] = v[q];
    __threadfence();
    last = atomicAdd(w.count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < kRedBlocks; t += kT) acc += __ldcg(w.part + q * kRedBlocks + t);
    v[q] = acc;
  }
  block_sum<NV>(v);
  if (threadIdx.x == 0) *w.count = 0u;
  return true;
}

__global__ void __launch_bounds__(kT, 4) k_cg_init(ParWork w, int64_t m, double tol) {
  double v[3] = {0.0, 0.0, 0.0};  // b.b, r.r, r.z
  for (int64_t s = (int64_t)blockIdx.x * kT + threadIdx.x; s < m; s += (int64_t)kRedBlocks * kT) {
    const double bs = w.b[s], rs = bs - w.q[s], zs = rs * w.iPd[s];
    w.r[s] = rs;
    w.z[s] = zs;
    w.d[s] = zs;
    v[0] += bs * bs;
    v[1] += rs * rs;
    v[2] += rs * zs;
  }
  block_sum<3>(v);
  if (grid_sum<3>(w, v) && threadIdx.x == 0) {
    const double stop = tol * sqrt(v[0]);
    w.scal[SC_STOP] = stop;
    w.scal[SC_RZ] = v[2];
    w.ctl[CTL_DONE] = sqrt(v[1]) <= stop;
    w.ctl[CTL_IT] = 0;
  }
}

__global__ void __launch_bounds__(kT, 4) k_cg_alpha(ParWork w, int64_t m) {
  if (w.ctl[CTL_DONE]) return;
  double v[1] = {0.0};  // d.q
  for (int64_t s = (int64_t)blockIdx.x * kT + threadIdx.x; s < m; s += (int64_t)kRedBlocks * kT) v[0] += w.d[s] * w.q[s];
  block_sum<1>(v);
  if (grid_sum<1>(w, v) && threadIdx.x == 0) w.scal[SC_ALPHA] = w.scal[SC_RZ] / v[0];
}

__global__ void __launch_bounds__(kT, 4) k_cg_update(ParWork w, int64_t m) {
  if (w.ctl[CTL_DONE]) return;
  const double alpha = w.scal[SC_ALPHA];
  double v[2] = {0.0, 0.0};  // r.r, r.z
  for (int64_t s = (int64_t)blockIdx.x * kT + threadIdx.x; s < m; s += (int64_t)kRedBlocks * kT) {
    w.x[s] += alpha * w.d[s];
    const double rs = w.r[s] - alpha * w.q[s], zs = rs * w.iPd[s];
    w.r[s] = rs;
    w.z[s] = zs;
    v[0] += rs * rs;
    v[1] += rs * zs;
  }
  block_sum<2>(v);
  if (grid_sum<2>(w, v) && threadIdx.x == 0) {
    w.ctl[CTL_IT] += 1;
    if (sqrt(v[0]) <= w.scal[SC_STOP]) {
      w.ctl[CTL_DONE] = 1;
    } else {
      w.scal[SC_BETA] = v[1] / w.scal[SC_RZ];
      w.scal[SC_RZ] = v[1];
    }
  }
}

__global__ void __launch_bounds__(kT, 4) k_cg_dir(ParWork w, int64_t m) {
  if (w.ctl[CTL_DONE]) return;
  const double beta = w.scal[SC_BETA];
  for (int64_t s = (int64_t)blockIdx.x * kT + threadIdx.x; s < m; s += (int64_t)kRedBlocks * kT)
    w.d[s] = w.z[s] + beta * w.d[s];
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

// every cell's share of int sigma(v):eps(v) phi_a for its nv nodes a, by the
// cell's quadrature, with sigma = 2 mu eps + (lambda - 2 mu/3) div v I
// (eq. def_Ki_nplusone)
template <int NV>
__global__ void k_cell_source(ParView v, ParWork w, const double *__restrict__ vh) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= v.n_cells) return;
  const double lm = v.lam - 2.0 * v.mu / 3.0;
  const int32_t *cn = v.cells + (int64_t)e * NV;
  double2 u[NV];
  double ce[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    u[a] = *(const double2 *)(vh + 2 * cn[a]);
    ce[a] = 0.0;
  }
  for (int q = 0; q < v.nq; ++q) {
    const int64_t eq = (int64_t)e * v.nq + q;
    const double *gr = v.qgrad + eq * 2 * NV;
    double d00 = 0.0, d01 = 0.0, d10 = 0.0, d11 = 0.0;  // d_km = d_m v_k
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const double g0 = gr[a], g1 = gr[NV + a];
      d00 += u[a].x * g0;
      d01 += u[a].x * g1;
      d10 += u[a].y * g0;
      d11 += u[a].y * g1;
    }
    const double e01 = 0.5 * (d01 + d10), div = d00 + d11;
    const double se = 2.0 * v.mu * (d00 * d00 + 2.0 * e01 * e01 + d11 * d11) + lm * div * div;
#pragma unroll
    for (int a = 0; a < NV; ++a) ce[a] += v.qw[eq] * v.qphi[eq * NV + a] * se;
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) w.ce[(int64_t)e * NV + a] = ce[a];
}

// K_i = (1/m_i) int sigma(v):eps(v) phi_i: the shares of the cells around i
// in a fixed order
__global__ void k_source(ParView v, ParWork w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  double acc = 0.0;
  for (int64_t t = v.nc_ptr[i]; t < v.nc_ptr[i + 1]; ++t) acc += w.ce[(int64_t)v.nc_cell[t] * v.nv + v.nc_local[t]];
  w.K[i] = acc / v.mi[i];
}

__global__ void k_en_rhs(ParView v, ParWork w, double src, double coefL) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double D = w.D[i];
  w.b[i] = D * w.en[i] + src * v.mi[i] * w.K[i];
  w.x[i] = w.en[i];
  w.iPd[i] = 1.0 / (D + coefL * v.L[v.diag[i]]);
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

void par_vel_coef(const ParView &v, const double *G, double *A, cudaStream_t s) {
  k_vel_coef<<<grid_for(v.n), kT, 0, s>>>(v, G, A);
}
void par_init(const ParView &v, const ParWork &w, const double *U, double dt, cudaStream_t s) {
  k_par_init<<<grid_for(v.n), kT, 0, s>>>(v, w, U, dt);
}
void par_vel_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, const int *skip,
                   cudaStream_t s) {
  k_vel_apply<<<grid_for(v.n), kT, 0, s>>>(v, w, coef, x, y, skip);
}
void par_en_apply(const ParView &v, const ParWork &w, double coef, const double *x, double *y, const int *skip,
                  cudaStream_t s) {
  k_en_apply<<<grid_for(v.n), kT, 0, s>>>(v, w, coef, x, y, skip);
}
void par_cg_init(const ParWork &w, int64_t m, double tol, cudaStream_t s) {
  k_cg_init<<<kRedBlocks, kT, 0, s>>>(w, m, tol);
}
void par_cg_alpha(const ParWork &w, int64_t m, cudaStream_t s) { k_cg_alpha<<<kRedBlocks, kT, 0, s>>>(w, m); }
void par_cg_update(const ParWork &w, int64_t m, cudaStream_t s) { k_cg_update<<<kRedBlocks, kT, 0, s>>>(w, m); }
void par_cg_dir(const ParWork &w, int64_t m, cudaStream_t s) { k_cg_dir<<<kRedBlocks, kT, 0, s>>>(w, m); }
void par_cell_source(const ParView &v, const ParWork &w, const double *vh, cudaStream_t s) {
  if (v.nv == 3)
    k_cell_source<3><<<grid_for(v.n_cells), kT, 0, s>>>(v, w, vh);
  else
    k_cell_source<4><<<grid_for(v.n_cells), kT, 0, s>>>(v, w, vh);
}
void par_source(const ParView &v, const ParWork &w, cudaStream_t s) { k_source<<<grid_for(v.n), kT, 0, s>>>(v, w); }
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
