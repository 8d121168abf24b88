// noalloc.cu -- eh_cfl_dt_noalloc: the CFL time step computed from caller-owned
// device arrays without allocating anything.
//
// Why it exists: some callers cannot call cudaMalloc at the point where they
// need a time step -- a host framework that owns every byte of device memory
// through its own pool and forbids allocation from plug-in libraries, or a
// real-time loop where an allocation (which may synchronise the device and
// take milliseconds) is not allowed. They cannot create an eh_ctx either,
// since eh_upload_mesh allocates. This entry point needs only their own device
// arrays: its one piece of scratch memory, the per-block minima of the
// reduction, is the file-scope array below, sized for EH_CFL_NOALLOC_MAX_ROWS
// rows and kept by every GPU that loads the library until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/euler_hyp.h"

namespace {

constexpr int kThreads = 128;
constexpr int kMaxBlocks = EH_CFL_NOALLOC_MAX_ROWS / kThreads;
constexpr int kMaxDevices = 64;

// The scratch: one double per block of kThreads rows (512 KiB).
static __device__ __align__(256) double g_cfl_block_min[kMaxBlocks];

// Device address of g_cfl_block_min, looked up once per device and context:
// the address belongs to the module loaded into one CUDA context, so the cache
// is keyed on that context's process-unique id (a device reset or a new
// primary context gets a new id, and the address is looked up again).
struct ScratchEntry {
  unsigned long long ctx_id;
  double *addr;
};
ScratchEntry g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mutex;

struct Prim {
  double un, p, a, az, ip;
};

// Normal velocity, pressure, sound speed, a p^-z and 1/p of state U[.][i]
// along the unit vector (c * cinv).
template <int DIM>
__device__ inline Prim primitives(const double *U, int n, int i, const double *c, double cinv, double gamma) {
  double rho = U[i];
  double m2 = 0.0, mn = 0.0;
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    double mq = U[(int64_t)(1 + q) * n + i];
    m2 += mq * mq;
    mn += mq * (c[q] * cinv);
  }
  double eps = U[(int64_t)(DIM + 1) * n + i] - m2 / (2.0 * rho);
  Prim r;
  r.un = mn / rho;
  r.p = (gamma - 1.0) * eps;
  r.a = sqrt(gamma * r.p / rho);
  r.az = r.a * pow(r.p, -(gamma - 1.0) / (2.0 * gamma));
  r.ip = 1.0 / r.p;
  return r;
}

// Upper bound on the maximum wave speed (two-rarefaction pressure, then the
// outer shock speeds evaluated there).
__device__ inline double wave_bound(const Prim &l, const Prim &r, double gamma) {
  double num = fmax(l.a + r.a - 0.5 * (gamma - 1.0) * (r.un - l.un), 0.0);
  double ptr = pow(num / (l.az + r.az), 2.0 * gamma / (gamma - 1.0));
  double k = (gamma + 1.0) / (2.0 * gamma);
  double sl = ptr > l.p ? sqrt(1.0 + k * (ptr - l.p) * l.ip) : 1.0;
  double sr = ptr > r.p ? sqrt(1.0 + k * (ptr - r.p) * r.ip) : 1.0;
  return fmax(fmax(-(l.un - l.a * sl), 0.0), fmax(r.un + r.a * sr, 0.0));
}

// d_ij of the entry k = (i, j), evaluated in its canonical orientation
// (from the row of min(i, j)), with the maximum over both directions when
// both nodes are boundary nodes.
template <int DIM>
__device__ inline double graph_viscosity(int lo, int hi, int64_t k_lohi, int64_t k_hilo, const double *cij, int64_t nnz,
                                         int n, const double *U, const unsigned char *isb, double gamma) {
  double c[DIM], ct[DIM], s2 = 0.0, t2 = 0.0;
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    c[q] = cij[(int64_t)q * nnz + k_lohi];
    ct[q] = cij[(int64_t)q * nnz + k_hilo];
    s2 += c[q] * c[q];
    t2 += ct[q] * ct[q];
  }
  double cn = sqrt(s2), ci = 1.0 / cn;
  double d = wave_bound(primitives<DIM>(U, n, lo, c, ci, gamma), primitives<DIM>(U, n, hi, c, ci, gamma), gamma) * cn;
  if (isb && isb[lo] && isb[hi]) {
    double tn = sqrt(t2), ti = 1.0 / tn;
    double dt = wave_bound(primitives<DIM>(U, n, hi, ct, ti, gamma), primitives<DIM>(U, n, lo, ct, ti, gamma), gamma) * tn;
    d = fmax(d, dt);
  }
  return d;
}

// min(a, b) that keeps a NaN: a row whose state is not admissible (rho <= 0 or
// internal energy <= 0) gives a NaN bound, which must reach dt_out instead of
// being dropped by the reduction
__device__ __forceinline__ double nan_min(double a, double b) { return (a < b || a != a) ? a : b; }

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_cfl_rows(int n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                                                       const double *cij, const double *mi, const unsigned char *isb,
                                                       const double *U, double gamma, double cfl, double *block_min) {
  __shared__ double smin[kThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double bound = INFINITY;
  if (i < n) {
    double dsum = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const int j = col[k];
      if (j == i) continue;
      // position of (j, i) by binary search in the sorted row j
      int64_t lo = row_ptr[j], hi = row_ptr[j + 1] - 1, kt = -1;
      while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int cm = col[mid];
        if (cm == i) {
          kt = mid;
          break;
        }
        if (cm < i) lo = mid + 1; else hi = mid - 1;
      }
      if (kt < 0) continue;  // unreachable for a symmetric pattern
      dsum += j > i ? graph_viscosity<DIM>(i, j, k, kt, cij, nnz, n, U, isb, gamma)
                    : graph_viscosity<DIM>(j, i, kt, k, cij, nnz, n, U, isb, gamma);
    }
    bound = cfl * mi[i] / (2.0 * dsum);
    // the row's own state must be admissible (rho > 0, internal energy > 0):
    // otherwise the wave speeds are undefined and the step is NaN
    double m2 = 0.0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) m2 += U[(int64_t)(1 + q) * n + i] * U[(int64_t)(1 + q) * n + i];
    const double rho = U[i];
    if (!(rho > 0.0 && U[(int64_t)(DIM + 1) * n + i] - m2 / (2.0 * rho) > 0.0)) bound = NAN;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) bound = nan_min(bound, __shfl_xor_sync(0xffffffffu, bound, off));
  if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = bound;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = smin[0];
#pragma unroll
    for (int q = 1; q < kThreads / 32; ++q) b = nan_min(b, smin[q]);
    block_min[blockIdx.x] = b;
  }
}

__global__ void __launch_bounds__(1024) k_cfl_reduce(const double *block_min, int nb, double *dt_out) {
  __shared__ double sm[32];
  double b = INFINITY;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) b = nan_min(b, block_min[q]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) b = nan_min(b, __shfl_xor_sync(0xffffffffu, b, off));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sm[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = nan_min(m, sm[q]);
    *dt_out = m;
  }
}

// The id of the CUDA context current on the calling thread, through driver
// entry points fetched by the runtime (the library does not link libcuda).
// Called with g_scratch_mutex held.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

eh_status current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return EH_ERR_CUDA;
    }
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS) return EH_ERR_CUDA;
  return EH_OK;
}

// The scratch's device address in the current device's current context. The
// lookup (cudaGetSymbolAddress, which allocates nothing) runs on the first
// call in each context and is cached for the later ones.
eh_status scratch_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return EH_ERR_CUDA;
  }
  // makes the device's primary context current if no context is yet
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return EH_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);  // also guards the entry points cached below
  unsigned long long ctx_id = 0;
  if (current_context_id(&ctx_id) != EH_OK) return EH_ERR_CUDA;
  ScratchEntry &e = g_scratch[dev];
  if (!e.addr || e.ctx_id != ctx_id) {
    void *p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_cfl_block_min);
    if (err != cudaSuccess || !p) {
      cudaGetLastError();
      return EH_ERR_CUDA;
    }
    e.addr = (double *)p;
    e.ctx_id = ctx_id;
  }
  *out = e.addr;
  return EH_OK;
}

}  // namespace

extern "C" eh_status eh_cfl_dt_noalloc(int32_t dim, double gamma, double cfl, int32_t n, int64_t nnz,
                                       const int64_t *row_ptr, const int32_t *col, const double *cij, const double *mi,
                                       const unsigned char *is_boundary, const double *U, double *dt_out,
                                       void *stream) {
  if ((dim != 2 && dim != 3) || !(gamma > 1.0 && gamma <= 5.0 / 3.0) || !(cfl > 0.0 && cfl <= 1.0))
    return EH_ERR_INVALID_ARG;
  if (n <= 0 || n > EH_CFL_NOALLOC_MAX_ROWS || nnz <= 0 || !row_ptr || !col || !cij || !mi || !U || !dt_out)
    return EH_ERR_INVALID_ARG;
  // an error left by earlier work of the caller is reported, not consumed:
  // the caller still finds it with its own cudaGetLastError
  if (cudaPeekAtLastError() != cudaSuccess) return EH_ERR_CUDA;
  double *scratch = nullptr;
  eh_status st = scratch_for_current_device(&scratch);
  if (st != EH_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (n + kThreads - 1) / kThreads;
  if (dim == 2)
    k_cfl_rows<2><<<nb, kThreads, 0, s>>>(n, nnz, row_ptr, col, cij, mi, is_boundary, U, gamma, cfl, scratch);
  else
    k_cfl_rows<3><<<nb, kThreads, 0, s>>>(n, nnz, row_ptr, col, cij, mi, is_boundary, U, gamma, cfl, scratch);
  if (cudaGetLastError() != cudaSuccess) return EH_ERR_CUDA;  // this launch's error only (none was pending)
  k_cfl_reduce<<<1, 1024, 0, s>>>(scratch, nb, dt_out);
  if (cudaGetLastError() != cudaSuccess) return EH_ERR_CUDA;
  return EH_OK;
}
