// kernels.cu -- sm_103a kernels of one forward-Euler stage of the hyperbolic
// (Euler) operator of arXiv:2106.02159 (Appendix B, Algorithm 1) and of the
// boundary post-processing of Sec. 4.
//
// Design: on GB300 an FP64 FMA issues at 1/72 of the FP32 rate, so this path
// is bound by FP64 instruction issue, not by HBM. Every edge loop therefore
// runs one thread per CSR row (no idle lanes in 7/9/27-entry rows), sums in
// the row's column order (bitwise reproducible), and trades bytes for FP64
// work: per-node quantities (primitives, a p^-z, Phi, eta, E + p; in the FP32
// record of mixed mode also the flux f(U)) are computed once per stage in
// k_prep and gathered; |c_ij|, 1/|c_ij|, m_ij/m_j and m_ji/m_i are static
// per-edge arrays; (f(U_j) - f(U_i)) c_ij is computed once per edge in k_visc
// and reused by k_low; the limiter directions P_ij are stored.
//
// Work that cannot change a result is skipped, exactly: an edge between two
// bit-identical states takes the closed form of its values; a node record made
// from the same state bits is kept, and an edge between two kept states that
// were equal at the previous stage keeps its stored values; a row none of whose
// neighbours differs has P_ij = 0 and every limiter 1; a limiter pass leaves
// its remainder (1 - l) P_ij as the factor 1 - l (nothing is read where it is
// 0); a row whose limiters are all 1 stores none and says so in a flag.
#include "kernels.cuh"

#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace eh {

// threads (= rows) per block of the row kernels: chosen per kernel at run time
// (eh_create's defaults, eh_autotune, eh_set_launch_shape), at most TPB_MAX

__host__ __device__ inline unsigned nblocks(int64_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// ---------------------------------------------------------------------------
// comparisons and min/max of doubles of known sign, on the bit patterns: a
// non-negative double orders like its bit pattern read as a signed 64-bit
// integer, and every negative double reads as a negative integer. An FP64
// compare or min/max issues on the FP64 pipe (2 lanes per SM and clock on
// GB300); the integer form runs on the ALUs. No operand is NaN on these paths.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// x > y and x < y for y > 0, x of either sign
__device__ __forceinline__ bool gt_pos(double x, double y) { return dbits(x) > dbits(y); }
__device__ __forceinline__ bool lt_pos(double x, double y) { return dbits(x) < dbits(y); }
// an integer key with the order of the doubles (either sign)
__device__ __forceinline__ long long order_key(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
// max(x, 0); a > b and max(a, b) for a, b >= 0 (FP32: the plain instructions)
__device__ __forceinline__ double pos_part(double x) { return dbits(x) > 0 ? x : 0.0; }
__device__ __forceinline__ float pos_part(float x) { return fmaxf(x, 0.0f); }
__device__ __forceinline__ bool gt_nonneg(double a, double b) { return dbits(a) > dbits(b); }
__device__ __forceinline__ bool gt_nonneg(float a, float b) { return a > b; }
__device__ __forceinline__ double max_nonneg(double a, double b) { return dbits(a) > dbits(b) ? a : b; }
__device__ __forceinline__ float max_nonneg(float a, float b) { return fmaxf(a, b); }
// x > 0 and x < 0 (strict: false for both zeros)
__device__ __forceinline__ bool pos_strict(double x) { return dbits(x) > 0; }
__device__ __forceinline__ bool neg_strict(double x) { return dbits(x) < 0 && (dbits(x) << 1) != 0; }
// min(max(x, 0), 1)
__device__ __forceinline__ double clamp01(double x) { return dbits(x) <= 0 ? 0.0 : (gt_pos(x, 1.0) ? 1.0 : x); }
// |x| by clearing the sign bit
__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(dbits(x) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ float abs_bits(float x) { return fabsf(x); }

// the per-entry viscosity quantities (layout: EdgeLayout)
template <int DIM, typename T> __device__ __forceinline__ T *w_slot(const Work &w, int64_t k) {
  return (T *)w.vw + k * EdgeLayout<DIM, T>::SPW;
}
template <int DIM, typename T> __device__ __forceinline__ T *d_ptr(const Work &w, int64_t k) {
  return EdgeLayout<DIM, T>::packed ? w_slot<DIM, T>(w, k) + EdgeLayout<DIM, T>::D : (T *)w.vd + k;
}
template <int DIM, typename T> __device__ __forceinline__ T *a_ptr(const Work &w, int64_t k) {
  return EdgeLayout<DIM, T>::packed ? w_slot<DIM, T>(w, k) + EdgeLayout<DIM, T>::A : (T *)w.va + k;
}
// one packed slot [w (S), a, d, 0...] of 8 values in whole-sector vector stores
template <int S> __device__ __forceinline__ void store_slot(double *p, const double *wv, double a, double d) {
  double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int s = 0; s < S; ++s) v[s] = wv[s];
  v[S] = a;
  v[S + 1] = d;
  double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
  for (int h = 0; h < 4; ++h) q[h] = make_double2(v[2 * h], v[2 * h + 1]);
}
// one 32-byte sector of FP64 values
__device__ __forceinline__ void store_sector(double *p, double x0, double x1, double x2, double x3) {
  double2 *q = reinterpret_cast<double2 *>(p);
  q[0] = make_double2(x0, x1);
  q[1] = make_double2(x2, x3);
}
template <int S> __device__ __forceinline__ void store_slot(float *p, const float *wv, float a, float d) {
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int s = 0; s < S; ++s) v[s] = wv[s];
  v[S] = a;
  v[S + 1] = d;
  float4 *q = reinterpret_cast<float4 *>(p);
  q[0] = make_float4(v[0], v[1], v[2], v[3]);
  q[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// the entry k of an edge between equal states: w = 0, a = 0, and d
template <int DIM, typename T> __device__ __forceinline__ void store_zero_edge(const Work &w, int64_t k, T d) {
  constexpr int S = DIM + 2;
  if constexpr (!EdgeLayout<DIM, T>::packed) {
    store_sector((double *)w_slot<DIM, T>(w, k), 0.0, 0.0, 0.0, 0.0);
    *a_ptr<DIM, T>(w, k) = T(0);
    *d_ptr<DIM, T>(w, k) = d;
  } else if constexpr (sizeof(T) == 8) {  // FP64 3D: two sectors [w0..w3], [w4, a, d, 0]
    store_sector((double *)w_slot<DIM, T>(w, k), 0.0, 0.0, 0.0, 0.0);
    store_sector((double *)w_slot<DIM, T>(w, k) + 4, 0.0, 0.0, (double)d, 0.0);
  } else {
    T z[S];
#pragma unroll
    for (int s = 0; s < S; ++s) z[s] = T(0);
    store_slot<S>(w_slot<DIM, T>(w, k), z, T(0), d);
  }
}

// ---------------------------------------------------------------------------
// roots and powers for gamma = 7/5 (division-free Newton iterations from an
// FP32 seed; two steps take the ~2^-21 seed error below double rounding)
// ---------------------------------------------------------------------------

// x^(-1/5): Newton's method on r^-5 = x, r <- r (6 - x r^5) / 5.
__device__ __forceinline__ double rroot5(double x) {
  if (!(gt_pos(x, 1e-30) && lt_pos(x, 1e30))) return pow(x, -0.2);
  double r = (double)exp2f(-0.2f * log2f((float)x));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    double r2 = r * r;
    double r5 = r2 * r2 * r;
    r = r * (6.0 - x * r5) * 0.2;
  }
  return r;
}

// x^(-1/7): Newton's method on r^-7 = x, r <- r (8 - x r^7) / 7.
__device__ __forceinline__ double rroot7(double x) {
  if (!(gt_pos(x, 1e-30) && lt_pos(x, 1e30))) return pow(x, -1.0 / 7.0);
  double r = (double)exp2f((-1.0f / 7.0f) * log2f((float)x));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    double r2 = r * r;
    double r7 = r2 * r2 * r2 * r;
    r = r * (8.0 - x * r7) * (1.0 / 7.0);
  }
  return r;
}

// rho^gamma
__device__ __forceinline__ double pow_gamma(const Params &p, double rho) {
  if (p.gamma75) {
    double r = rroot5(rho);  // rho^(-1/5); rho^(7/5) = rho^2 r^3
    return rho * rho * (r * r * r);
  }
  return pow(rho, p.gamma);
}

// rho^(gamma - 1)
__device__ __forceinline__ double pow_gamma_m1(const Params &p, double rho) {
  if (p.gamma75) {
    double r = rroot5(rho);  // rho^(2/5) = rho r^3
    return rho * (r * r * r);
  }
  return pow(rho, p.gamma - 1.0);
}

// ---------------------------------------------------------------------------
// Sec. 3.1: guaranteed upper bound on the maximum wave speed
// ---------------------------------------------------------------------------
// Two-rarefaction pressure p_tr >= p* (1 < gamma <= 5/3), then the outer wave
// speeds of the 1- and 3-waves evaluated at p_tr. Inputs per side: normal
// velocity, p, a, a p^-z, 1/p.
template <typename T>
__device__ __forceinline__ T lambda_max(const Params &p, T unl, T pl, T al, T azl, T ipl, T unr, T pr, T ar, T azr,
                                        T ipr) {
  T num = al + ar - T(0.5) * T(p.gm1) * (unr - unl);
  num = pos_part(num);
  T x = num / (azl + azr);
  T ptr;
  if (p.gamma75) {
    T x2 = x * x;
    T x4 = x2 * x2;
    ptr = x4 * x2 * x;  // x^(2 gamma/(gamma-1)) = x^7
  } else {
    ptr = pow(x, T(p.inv_z));
  }
  const T ks = T(p.kshock);
  T sl = gt_nonneg(ptr, pl) ? sqrt(T(1) + ks * (ptr - pl) * ipl) : T(1);
  T sr = gt_nonneg(ptr, pr) ? sqrt(T(1) + ks * (ptr - pr) * ipr) : T(1);
  T lam1 = unl - al * sl;
  T lam3 = unr + ar * sr;
  return max_nonneg(pos_part(-lam1), pos_part(lam3));
}

// ---------------------------------------------------------------------------
// Sec. 3.3: line search for the largest l in [0,1] within the local bounds
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double psi(const Params &p, const double *ub, const double *P, double l, double phimin) {
  constexpr int S = DIM + 2;
  double u[S];
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = ub[s] + l * P[s];
  double m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) m2 += u[1 + k] * u[1 + k];
  double eps = u[S - 1] - m2 / (2.0 * u[0]);
  return eps - phimin * pow_gamma(p, u[0]);
}

template <int DIM>
__device__ __forceinline__ double dpsi(const Params &p, const double *ub, const double *P, double l, double phimin) {
  constexpr int S = DIM + 2;
  double u[S];
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = ub[s] + l * P[s];
  double irho = 1.0 / u[0];
  double v2 = 0.0, vP = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    double v = u[1 + k] * irho;
    v2 += v * v;
    vP += v * P[1 + k];
  }
  double deps = P[S - 1] - vP + 0.5 * v2 * P[0];
  return deps - phimin * p.gamma * pow_gamma_m1(p, u[0]) * P[0];
}

constexpr int LINE_SEARCH_ITERATIONS = 6;

// gamma = 7/5: psi(l) as psi() above, also returning r = rho(l)^(-1/5), so
// that psi'(lR) reuses the root of the psi(lR) evaluation (rho^(2/5) = rho r^3);
// the values are those of psi()/dpsi() bit for bit.
template <int DIM>
__device__ __forceinline__ double psi_g75(const double *ub, const double *P, double l, double phimin, double *r_out) {
  constexpr int S = DIM + 2;
  double u[S];
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = ub[s] + l * P[s];
  double m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) m2 += u[1 + k] * u[1 + k];
  const double eps = u[S - 1] - m2 / (2.0 * u[0]);
  const double r = rroot5(u[0]);
  *r_out = r;
  return eps - phimin * (u[0] * u[0] * (r * r * r));
}

template <int DIM>
__device__ __forceinline__ double dpsi_g75(const double *ub, const double *P, double l, double r, double phimin) {
  constexpr int S = DIM + 2;
  double u[S];
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = ub[s] + l * P[s];
  const double irho = 1.0 / u[0];
  double v2 = 0.0, vP = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const double v = u[1 + k] * irho;
    v2 += v * v;
    vP += v * P[1 + k];
  }
  const double deps = P[S - 1] - vP + 0.5 * v2 * P[0];
  return deps - phimin * 1.4 * (u[0] * (r * r * r)) * P[0];
}

// The line search in two parts. line_search_start takes every exit that needs
// no iteration (P = 0, the density limit, the entropy bound met at that limit,
// psi(0) <= 0) and otherwise returns the bracket [0, l] with psi at both ends;
// line_search_iterate runs the fixed number of secant (feasible side) / Newton
// (infeasible side) steps on that bracket and returns its feasible end. For
// gamma = 7/5 the root of rho is shared between psi(lR) and psi'(lR), and psi
// is evaluated once when the Newton and secant points coincide.
struct LsBracket {
  double l;   // the result when done; else the right end of the bracket
  double pl;  // psi(0) > 0
  double pr;  // psi(l) < 0
  double rR;  // rho(l)^(-1/5) (gamma = 7/5)
  bool done;
};

// phimin5 = phimin^5 (used by the gamma = 7/5 fast check only).
template <int DIM>
__device__ LsBracket line_search_start(const Params &p, const double *ub, const double *P, double rmin, double rmax,
                                       double phimin, double phimin5) {
  constexpr int S = DIM + 2;
  LsBracket b{1.0, 0.0, 0.0, 0.0, true};
  // P = 0 (every edge whose previous limiter was 1, uniform flow): every l gives
  // the same state; the largest, 1, is returned without any FP64 work
  bool zero = true;
#pragma unroll
  for (int s = 0; s < S; ++s) zero &= (__double_as_longlong(P[s]) << 1) == 0;
  if (zero) return b;
  // (compares on the bit patterns; the density bounds are positive)
  double l = 1.0;
  const double rb = ub[0], rp = P[0];
  // density: the division is needed only when l = 1 leaves [rho_min, rho_max]
  if (pos_strict(rp)) {
    if (gt_pos(rb + rp, rmax)) l = clamp01((rmax - rb) / rp);
  } else if (neg_strict(rp)) {
    if (lt_pos(rb + rp, rmin)) l = clamp01((rmin - rb) / rp);
  }
  b.l = l;
  if (p.gamma75) {
    // entropy at l: psi(l) >= 0 <=> (eps rho)^5 >= Phi_min^5 rho^12 when
    // eps rho > 0 -- no division and no root on the common path
    double u[S];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = ub[s] + l * P[s];
    const double rho = u[0];
    if (gt_pos(rho, 1e-6) && lt_pos(rho, 1e6)) {
      double m2 = 0.0;
#pragma unroll
      for (int q = 0; q < DIM; ++q) m2 += u[1 + q] * u[1 + q];
      const double er = u[S - 1] * rho - 0.5 * m2;
      if (pos_strict(er)) {
        const double r2 = rho * rho, r4 = r2 * r2, r12 = r4 * r4 * r4;
        const double e2 = er * er;
        const double lhs = e2 * e2 * er, rhs = phimin5 * r12;  // lhs > 0, rhs >= 0
        if (lt_pos(rhs, 1e300) && dbits(lhs) >= dbits(rhs)) return b;
      }
    }
    double r0;
    b.pr = psi_g75<DIM>(ub, P, l, phimin, &b.rR);
    if (!neg_strict(b.pr)) return b;
    b.pl = psi_g75<DIM>(ub, P, 0.0, phimin, &r0);
  } else {
    b.pr = psi<DIM>(p, ub, P, l, phimin);
    if (!neg_strict(b.pr)) return b;
    b.pl = psi<DIM>(p, ub, P, 0.0, phimin);
  }
  if (!pos_strict(b.pl)) {
    b.l = 0.0;
    return b;
  }
  b.done = false;
  return b;
}

template <int DIM>
__device__ double line_search_iterate(const Params &p, const double *ub, const double *P, double phimin,
                                      const LsBracket &b) {
  double lL = 0.0, lR = b.l, pl = b.pl, pr = b.pr, rR = b.rR;
  for (int it = 0; it < LINE_SEARCH_ITERATIONS; ++it) {
    double ls = lL + pl * (lR - lL) / (pl - pr);
    double dr = p.gamma75 ? dpsi_g75<DIM>(ub, P, lR, rR, phimin) : dpsi<DIM>(p, ub, P, lR, phimin);
    double ln = neg_strict(dr) ? lR - pr / dr : lR;
    if (order_key(ln) < order_key(ls)) ln = ls;
    double ps, pn, rs, rn;
    if (p.gamma75) {
      ps = psi_g75<DIM>(ub, P, ls, phimin, &rs);
      pn = ps;
      rn = rs;
      if (dbits(ln) != dbits(ls)) pn = psi_g75<DIM>(ub, P, ln, phimin, &rn);
    } else {
      ps = psi<DIM>(p, ub, P, ls, phimin);
      pn = psi<DIM>(p, ub, P, ln, phimin);
      rn = 0.0;
    }
    if (!neg_strict(ps)) {
      lL = ls;
      pl = ps;
    }
    if (neg_strict(pn)) {
      lR = ln;
      pr = pn;
      rR = rn;
    } else {
      lL = ln;
      pl = pn;
    }
  }
  return lL;
}

// FP32 pre-decision of the entropy test at l = 1 (gamma = 7/5): with
// u = ub + P, does (rho E - |m|^2/2)^5 >= Phi_min^5 rho^12 hold, for the FP64
// inputs, in exact arithmetic? The FP32 evaluation carries error bounds built
// from the inputs' magnitudes (every conversion and operation rounds by at most
// 2^-24 relative): +1 = holds with a margin that covers them, -1 = fails with
// such a margin, 0 = too close to call (or outside the range where the FP32
// powers can neither overflow nor underflow). Every error term is
// over-estimated by a third or more (3 units for a chain that rounds twice, 8
// and 16 for chains of 3 and 6 roundings, B scaled by 1.01), so a decided
// outcome holds with a relative margin of at least ~1e-7 -- far beyond the
// FP64 test's own rounding (~1e-15): it is the outcome the FP64 test reaches,
// and the FP64 test runs only where this returns 0.
struct RowF32 {
  float u[5];   // ub rounded to FP32
  float phi5;   // Phi_min^5 rounded to FP32 (0 when out of range)
};
// The row's FP32 data of the pre-decision. Rows whose density bounds are
// within 1e-6 of each other (near-uniform neighbourhoods) skip it: there psi(1)
// sits within the FP32 error of 0 almost always (on the Mach-3 cylinder most
// such rows differ from their neighbours by a few ulps, and psi(1) is within
// 1e-13 of 0), and a warp with one undecided lane pays for both tests.
template <int DIM>
__device__ __forceinline__ RowF32 row_f32(const double *ub, double rmin, double rmax, double phimin5) {
  RowF32 r;
#pragma unroll
  for (int s = 0; s < DIM + 2; ++s) r.u[s] = 0.0f;
  r.phi5 = 0.0f;
  // 2^-40 <= Phi_min^5 <= 2^40 (else no pre-decision)
  if (!(gt_pos(rmax - rmin, 1e-6 * rmax) && gt_pos(phimin5, 9.094947017729282e-13) &&
        lt_pos(phimin5, 1.099511627776e12)))
    return r;
#pragma unroll
  for (int s = 0; s < DIM + 2; ++s) r.u[s] = (float)ub[s];
  r.phi5 = (float)phimin5;
  return r;
}

template <int DIM> __device__ __forceinline__ int entropy_at_one_f32(const RowF32 &r, const double *P) {
  constexpr int S = DIM + 2;
  constexpr float u24 = 5.9604645e-8f;  // 2^-24
  if (r.phi5 == 0.0f) return 0;
  float u[S], e[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float pf = (float)P[s];
    u[s] = r.u[s] + pf;
    // |u_f - u| <= 2^-24 (|ub| + |P| + |u_f|) (two conversions, one add)
    e[s] = 3.0f * u24 * (fabsf(r.u[s]) + fabsf(pf));
  }
  const float rho = u[0], E = u[S - 1];
  // 2^-6 <= rho <= 2^6 with its error: rho^12 stays within FP32's range
  if (!(rho - e[0] >= 0.015625f && rho + e[0] <= 64.0f)) return 0;
  float m2h = 0.0f, em = 0.0f;
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    m2h += u[1 + q] * u[1 + q];
    em += fabsf(u[1 + q]) * e[1 + q] + 0.5f * e[1 + q] * e[1 + q];
  }
  m2h *= 0.5f;
  const float rE = rho * E;
  const float er = rE - m2h;
  // |er_f - er| <= propagated input errors + 8 roundings of the magnitudes
  const float B = 1.01f * (rho * e[S - 1] + fabsf(E) * e[0] + e[0] * e[S - 1] + em +
                           8.0f * u24 * (fabsf(rE) + m2h));
  const float elo = er - B, ehi = er + B;
  // 2^-24 <= er <= 2^24 with its error: er^5 stays within FP32's range
  if (!(elo >= 5.9604645e-8f && ehi <= 16777216.0f)) return 0;
  const float rlo = rho - e[0], rhi = rho + e[0];
  const float l2 = elo * elo, h2 = ehi * ehi;
  const float lhs_lo = l2 * l2 * elo * (1.0f - 8.0f * u24);
  const float lhs_hi = h2 * h2 * ehi * (1.0f + 8.0f * u24);
  const float a2 = rlo * rlo, a4 = a2 * a2, b2 = rhi * rhi, b4 = b2 * b2;
  const float rhs_lo = r.phi5 * (a4 * a4 * a4) * (1.0f - 16.0f * u24);
  const float rhs_hi = r.phi5 * (b4 * b4 * b4) * (1.0f + 16.0f * u24);
  if (lhs_lo > rhs_hi) return 1;
  if (lhs_hi < rhs_lo) return -1;
  return 0;
}

// The common outcome of the line search, decided with a short branch-free
// sequence: P = 0, or l = 1 inside the density bounds and (gamma = 7/5) inside
// the entropy bound. Returns true exactly where line_search returns 1 through
// one of these exits; false leaves the entry to the full search. (A warp whose
// lanes took the search's other exits -- density clipping, psi evaluations,
// the secant/Newton loop -- inline would issue each of them for all 32 lanes.)
// The entropy test is pre-decided in FP32 (entropy_at_one_f32) and evaluated
// in FP64 only where that is too close to call.
template <int DIM>
__device__ __forceinline__ bool line_search_at_one(const Params &p, const double *ub, const double *P, double rmin,
                                                   double rmax, double phimin5, const RowF32 &rf) {
  constexpr int S = DIM + 2;
  bool zero = true;
#pragma unroll
  for (int s = 0; s < S; ++s) zero &= (__double_as_longlong(P[s]) << 1) == 0;
  if (zero) return true;
  if (!p.gamma75) return false;
  // the compares below run on the bit patterns (all thresholds are positive);
  // rp = -0 may take the density test, which can only send the entry to the
  // full search
  const double rb = ub[0], rp = P[0];
  if (dbits(rp) > 0) {
    if (gt_pos(rb + rp, rmax)) return false;
  } else if (dbits(rp) < 0) {
    if (lt_pos(rb + rp, rmin)) return false;
  }
  const int pre = entropy_at_one_f32<DIM>(rf, P);
  if (pre != 0) return pre > 0;
  double u[S];
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = ub[s] + P[s];
  const double rho = u[0];
  if (!(gt_pos(rho, 1e-6) && lt_pos(rho, 1e6))) return false;
  double m2 = 0.0;
#pragma unroll
  for (int q = 0; q < DIM; ++q) m2 += u[1 + q] * u[1 + q];
  const double er = u[S - 1] * rho - 0.5 * m2;
  if (!(dbits(er) > 0)) return false;
  const double r2 = rho * rho, r4 = r2 * r2, r12 = r4 * r4 * r4;
  const double e2 = er * er;
  const double lhs = e2 * e2 * er, rhs = phimin5 * r12;  // lhs > 0, rhs >= 0
  return lt_pos(rhs, 1e300) && dbits(lhs) >= dbits(rhs);
}

// Queues the line searches of row i's entries k0 + b for every bit b of 'mask'
// for k_ls_deferred: one atomic per group of converged lanes (normally once
// per warp and kernel). The queue holds nnz entries and a pass queues each
// entry at most once, so it cannot fill; the bounds check only guards memory
// (an overflow would be reported as EH_ERR_STATE).
__device__ __forceinline__ void defer_line_searches(const Work &w, int slot, int i, int64_t k0, uint64_t mask) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  const unsigned cnt = (unsigned)__popcll(mask);
  const unsigned off = cg::exclusive_scan(g, cnt);
  const unsigned total = g.shfl(off + cnt, g.size() - 1);
  if (total == 0) return;
  unsigned base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&w.lsq_count[slot], total);
  base = g.shfl(base, 0) + off;
  while (mask) {
    const int b = __ffsll((long long)mask) - 1;
    mask &= mask - 1;
    if (base < w.lsq_cap)
      w.lsq[base++] = make_int2(i, (int)(k0 + b));
    else
      atomicExch(&w.st->err, 7);  // EH_ERR_STATE
  }
}

// ---------------------------------------------------------------------------
// flux f(U) = (m, m v^T + p I, v (E + p)) of one node (Sec. 2.1), row s =
// component, from its momentum, velocity, pressure and E + p
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__device__ __forceinline__ void node_flux(const T *mv, const T *v, T pr, T H, T f[DIM + 2][DIM]) {
#pragma unroll
  for (int q = 0; q < DIM; ++q) f[0][q] = mv[q];
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int b = 0; b < DIM; ++b) f[1 + a][b] = mv[a] * v[b] + (a == b ? pr : T(0));
#pragma unroll
  for (int q = 0; q < DIM; ++q) f[DIM + 1][q] = v[q] * H;
}

// ---------------------------------------------------------------------------
// k_prep: node records (primitives and derived quantities), once per stage
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void __launch_bounds__(TPB_MAX) k_prep(MeshView m, Params p, const double *__restrict__ U,
                                              double *__restrict__ rec, T *__restrict__ vrec,
                                              unsigned char *__restrict__ rough,
                                              unsigned char *__restrict__ steady, const DevStatus *st) {
  constexpr int S = DIM + 2;
  using R = Rec<DIM>;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.n || st->err) return;
  const unsigned char was_rough = rough[i];  // as the previous k_visc left it
  rough[i] = 0;  // set by k_visc where a neighbour's state differs
  double u[S];
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = U[(int64_t)s * m.n + i];
  double *Rr = rec + (int64_t)i * R::SIZE;
  {
    // the record (both precisions) is a function of U_i and gamma alone, so
    // where the stored one was made from the same bits it stands as it is:
    // nodes of a uniform region keep their state exactly from stage to stage
    // (every P_ij and increment is 0). The records start as NaN bit patterns,
    // which no admissible state matches.
    bool same = true;
#pragma unroll
    for (int s = 0; s < S; ++s) same &= dbits(Rr[s]) == dbits(u[s]);
    steady[i] = same ? (unsigned char)(was_rough ? 1 : 3) : (unsigned char)0;
    if (same) return;
  }
  double rho = u[0];
  double irho = 1.0 / rho;
  double v[DIM], m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    v[k] = u[1 + k] * irho;
    m2 += u[1 + k] * u[1 + k];
  }
  double eps = u[S - 1] - 0.5 * m2 * irho;
  double pr = p.gm1 * eps;
  double a = sqrt(p.gamma * pr * irho);
  double az, phi;
  if (p.gamma75) {
    az = a * rroot7(pr);
    double r = rroot5(rho);  // rho^(-1/5); rho^(-7/5) = r^7
    double r2 = r * r;
    phi = eps * (r2 * r2 * r2 * r);
  } else {
    az = a * pow(pr, -p.z);
    phi = eps * pow(rho, -p.gamma);
  }
  double eta = -rho * (log(phi) * p.inv_gm1);
#pragma unroll
  for (int s = 0; s < S; ++s) Rr[s] = u[s];
#pragma unroll
  for (int k = 0; k < DIM; ++k) Rr[R::V + k] = v[k];
  Rr[R::P] = pr;
  Rr[R::A] = a;
  Rr[R::AZ] = az;
  Rr[R::IP] = 1.0 / pr;
  Rr[R::PHI] = phi;
  Rr[R::ETA] = eta;
  Rr[R::EPS] = eps;
  Rr[R::H] = u[S - 1] + pr;
  Rr[R::IRHO] = irho;
  Rr[R::IEPS] = 1.0 / eps;
  if constexpr (!std::is_same<T, double>::value) {
    // the same record in the viscosity precision (mixed mode), with the flux
    T *Rv = vrec + (int64_t)i * R::VSIZE;
#pragma unroll
    for (int q = 0; q <= R::IEPS; ++q) Rv[q] = (T)Rr[q];
    double f[S][DIM];
    node_flux<DIM, double>(u + 1, v, pr, Rr[R::H], f);
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < DIM; ++q) Rv[R::F + s * DIM + q] = (T)f[s][q];
  }
}

// ---------------------------------------------------------------------------
// k_visc: Algorithm 1 step 1 -- d_ij (j > i, mirrored through the transpose
// index), the flux differences w_ij and the indicator alpha_i
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void __launch_bounds__(TPB_MAX) k_visc(MeshView m, Params p, Work w) {
  constexpr int S = DIM + 2;
  using R = Rec<DIM>;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.n || w.st->err) return;
  const T *rec = (const T *)w.vrec;
  const T *cij = (const T *)m.vcij;
  const T *cn = (const T *)m.vcn;
  const T *cinv = (const T *)m.vcinv;
  constexpr bool packed = EdgeLayout<DIM, T>::packed;
  constexpr int RS = vrec_stride<DIM, T>();
  const T *Ri = rec + (int64_t)i * RS;
  T vi[DIM], mi[DIM];
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    vi[k] = Ri[R::V + k];
    mi[k] = Ri[1 + k];
  }
  const T pi = Ri[R::P], ai = Ri[R::A], azi = Ri[R::AZ], ipi = Ri[R::IP], etai = Ri[R::ETA], Hi = Ri[R::H];
  // FP64: w_ij from v.c_ij of both nodes (fewest FP64 operations). FP32: as
  // differences of the two nodes' fluxes (rounded from FP64 by k_prep), then
  // dotted with c_ij -- products taken per entry in FP32 (m_i (v_i.c_ij), or
  // the flux formed in FP32) carry rounding errors that the difference of
  // rounded fluxes does not: they left ~20x more of the limiter's l = 1
  // checks failing on the Mach-3 cylinder and raised the error against FP64
  constexpr bool flux_diff = sizeof(T) == 4;
  T fi[DIM + 2][DIM], qi[DIM];
  if constexpr (flux_diff) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < DIM; ++q) fi[s][q] = Ri[R::F + s * DIM + q];
#pragma unroll
    for (int q = 0; q < DIM; ++q) qi[q] = vi[q] * etai;
  }
  const bool bi = m.isb[i] != 0;
  // the FP64 state of node i as bit patterns (the identical-state test below
  // compares FP64 bits in either precision)
  long long ubi[S];
  {
    const double *Ri64 = w.rec + (int64_t)i * R::SIZE;
#pragma unroll
    for (int s = 0; s < S; ++s) ubi[s] = dbits(Ri64[s]);
  }
  const unsigned char sti = w.steady[i];
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  for (int64_t k = k0; k < k1; ++k) {
    const int j = m.col[k];
    if (j <= i) continue;  // each unique edge once, from the row of min(i, j)
    if (sti & 1) {
      // both states unchanged since the previous k_visc, which stored this
      // edge's values from the same bits; they were equal then (one of the
      // two nodes had no differing neighbour), so they are now: nothing to
      // store and no rough mark to set
      const unsigned char stj = w.steady[j];
      if ((stj & 1) && ((sti | stj) & 2)) continue;
    }
    const T *Rj = rec + (int64_t)j * RS;
    const int32_t kt = m.tr[k];
    {
      // U_j = U_i bit for bit: the flux and entropy-flux differences vanish,
      // w_ij = a_ij = 0 exactly, and the two-rarefaction bound of Sec. 3.1
      // reduces to lambda_max = |v.n_ij| + a (p_tr = p, both outer waves
      // rarefactions), so d_ij = |v.c_ij| + a |c_ij| with no division, power
      // or root. Any other edge marks both of its nodes rough.
      const double *Rj64 = w.rec + (int64_t)j * R::SIZE;
      bool same = true;
#pragma unroll
      for (int s = 0; s < S; ++s) same &= dbits(Rj64[s]) == ubi[s];
      if (same) {
        T vc = T(0);
#pragma unroll
        for (int q = 0; q < DIM; ++q) vc += vi[q] * cij[(int64_t)q * m.nnz + k];
        T dij = abs_bits(vc) + ai * cn[k];
        if (bi && m.isb[j]) {  // c_ji != -c_ij: the max over both directions
          T vct = T(0);
#pragma unroll
          for (int q = 0; q < DIM; ++q) vct += vi[q] * cij[(int64_t)q * m.nnz + kt];
          dij = max_nonneg(dij, abs_bits(vct) + ai * cn[kt]);
        }
        store_zero_edge<DIM, T>(w, k, dij);
        store_zero_edge<DIM, T>(w, kt, dij);
        continue;
      }
      w.rough[i] = 1;
      w.rough[j] = 1;
    }
    T vj[DIM], mj[DIM], c[DIM];
    const T pj = Rj[R::P], etaj = Rj[R::ETA], Hj = Rj[R::H];
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      vj[q] = Rj[R::V + q];
      mj[q] = Rj[1 + q];
      c[q] = cij[(int64_t)q * m.nnz + k];
    }
    // w_ij = (f(U_j) - f(U_i)) c_ij with f = (m, m v^T + p I, v (E + p));
    // a_ij = (q_j - q_i) . c_ij with q = eta v
    T vjc = T(0), vic = T(0);
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      vjc += vj[q] * c[q];
      vic += vi[q] * c[q];
    }
    const T dp = pj - pi;
    T wv[S], a_ = T(0), dm[DIM];
    if constexpr (flux_diff) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < DIM; ++q) acc += (Rj[R::F + s * DIM + q] - fi[s][q]) * c[q];
        wv[s] = acc;
      }
      T qj[DIM];
#pragma unroll
      for (int q = 0; q < DIM; ++q) qj[q] = vj[q] * etaj;
#pragma unroll
      for (int q = 0; q < DIM; ++q) a_ += (qj[q] - qi[q]) * c[q];
    } else {
      // X_j (v_j.c) - X_i (v_i.c) as (X_j - X_i) (v_j.c) + X_i (v_j.c - v_i.c):
      // exactly 0 when the two states are equal (a contracted X_j v_j.c -
      // X_i v_i.c leaves the rounding error of one product), so that uniform
      // regions keep P_ij = 0 and the limiter's cheapest exit
      T w0 = T(0);
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        dm[q] = mj[q] - mi[q];
        w0 += dm[q] * c[q];
      }
      const T dv = vjc - vic;
      wv[0] = w0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) wv[1 + a] = dm[a] * vjc + mi[a] * dv + dp * c[a];
      wv[S - 1] = (Hj - Hi) * vjc + Hi * dv;
      a_ = (etaj - etai) * vjc + etai * dv;
    }
    const bool both = bi && m.isb[j];
    // the transposed entry: c_ji = -c_ij unless both nodes lie on the boundary
    // (Sec. 3.1), so w_ji = w_ij and a_ji = a_ij; otherwise evaluate with c_ji.
    // Packed slots are stored whole once d_ij is known; otherwise each value
    // is stored as soon as it is computed (fewer live registers).
    // FP64 3D slots are two sectors: [w0..w3] stored at once, [w4, a, d, 0]
    // once d_ij is known
    constexpr bool two_sectors = packed && sizeof(T) == 8;
    T wt[S], at = a_, vjct = T(0), vict = T(0);
    if constexpr (!packed) {
      T *wk = w_slot<DIM, T>(w, k);
#pragma unroll
      for (int s = 0; s < S; ++s) wk[s] = wv[s];
      *a_ptr<DIM, T>(w, k) = a_;
    } else if constexpr (two_sectors) {
      store_sector((double *)w_slot<DIM, T>(w, k), wv[0], wv[1], wv[2], wv[3]);
    }
    if (!both) {
#pragma unroll
      for (int s = 0; s < S; ++s) wt[s] = wv[s];
    } else {
      T ct[DIM];
#pragma unroll
      for (int q = 0; q < DIM; ++q) ct[q] = cij[(int64_t)q * m.nnz + kt];
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        vjct += vj[q] * ct[q];
        vict += vi[q] * ct[q];
      }
      if constexpr (flux_diff) {
        at = T(0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          T acc = T(0);
#pragma unroll
          for (int q = 0; q < DIM; ++q) acc += (fi[s][q] - Rj[R::F + s * DIM + q]) * ct[q];
          wt[s] = acc;
        }
#pragma unroll
        for (int q = 0; q < DIM; ++q) at += (qi[q] - vj[q] * etaj) * ct[q];  // q_j as above
      } else {
        // (f_i - f_j) . c_ji = -[(f_j . c_ji) - (f_i . c_ji)], in the form above
        T w0t = T(0);
#pragma unroll
        for (int q = 0; q < DIM; ++q) w0t += dm[q] * ct[q];
        const T dvt = vjct - vict;
        wt[0] = -w0t;
#pragma unroll
        for (int a = 0; a < DIM; ++a) wt[1 + a] = -(dm[a] * vjct + mi[a] * dvt + dp * ct[a]);
        wt[S - 1] = -((Hj - Hi) * vjct + Hi * dvt);
        at = -((etaj - etai) * vjct + etai * dvt);
      }
    }
    if constexpr (!packed) {
      T *wtk = w_slot<DIM, T>(w, kt);
#pragma unroll
      for (int s = 0; s < S; ++s) wtk[s] = wt[s];
      *a_ptr<DIM, T>(w, kt) = at;
    } else if constexpr (two_sectors) {
      store_sector((double *)w_slot<DIM, T>(w, kt), wt[0], wt[1], wt[2], wt[3]);
    }
    // d_ij (Sec. 3.1), mirrored; normal velocities v . c_ij / |c_ij| (FP32:
    // v . (c_ij / |c_ij|))
    const T ci = cinv[k];
    T unl = vic * ci, unr = vjc * ci;
    if constexpr (flux_diff) {
      unl = unr = T(0);
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        unl += vi[q] * (c[q] * ci);
        unr += vj[q] * (c[q] * ci);
      }
    }
    T dij = lambda_max<T>(p, unl, pi, ai, azi, ipi, unr, pj, Rj[R::A], Rj[R::AZ], Rj[R::IP]) * cn[k];
    if (both) {
      const T cit = cinv[kt];
      T unj = vjct * cit, uni = vict * cit;
      if constexpr (flux_diff) {
        unj = uni = T(0);
#pragma unroll
        for (int q = 0; q < DIM; ++q) {
          T nq = cij[(int64_t)q * m.nnz + kt] * cit;
          unj += vj[q] * nq;
          uni += vi[q] * nq;
        }
      }
      T dji = lambda_max<T>(p, unj, pj, Rj[R::A], Rj[R::AZ], Rj[R::IP], uni, pi, ai, azi, ipi) * cn[kt];
      dij = max_nonneg(dij, dji);
    }
    if constexpr (two_sectors) {
      // values 4..7 of [w (S), a, d, 0...]
      double hi[4] = {0.0, 0.0, 0.0, 0.0}, hit[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int s = 4; s < S; ++s) {
        hi[s - 4] = wv[s];
        hit[s - 4] = wt[s];
      }
      hi[S - 4] = a_;
      hi[S - 3] = dij;
      hit[S - 4] = at;
      hit[S - 3] = dij;
      store_sector((double *)w_slot<DIM, T>(w, k) + 4, hi[0], hi[1], hi[2], hi[3]);
      store_sector((double *)w_slot<DIM, T>(w, kt) + 4, hit[0], hit[1], hit[2], hit[3]);
    } else if constexpr (packed) {
      store_slot<S>(w_slot<DIM, T>(w, k), wv, a_, dij);
      store_slot<S>(w_slot<DIM, T>(w, kt), wt, at, dij);
    } else {
      *d_ptr<DIM, T>(w, k) = dij;
      *d_ptr<DIM, T>(w, kt) = dij;
    }
  }
}

// ---------------------------------------------------------------------------
// k_alpha: the indicator alpha_i (Sec. 3.2) from the row's w_ij and a_ij
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void __launch_bounds__(TPB_MAX) k_alpha(MeshView m, Params p, Work w) {
  constexpr int S = DIM + 2;
  using R = Rec<DIM>;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.n || w.st->err) return;
  if (!w.rough[i]) {  // every w_ij and a_ij of the row is 0: N_i = D_i = 0
    w.alpha[i] = 0.0;
    return;
  }
  const T *Ri = (const T *)w.vrec + (int64_t)i * vrec_stride<DIM, T>();
  // eta'(U_i)
  T deta[S];
  {
    // eta' = (-s - rho/(gamma-1) (|v|^2/(2 eps) - gamma/rho), g1 v, -g1), g1 = rho/((gamma-1) eps)
    const T igm1 = T(p.inv_gm1);
    const T rho = Ri[0], irho = Ri[R::IRHO], ieps = Ri[R::IEPS];
    T s_i = -Ri[R::ETA] * irho;
    T g1 = rho * igm1 * ieps;
    T v2 = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) v2 += Ri[R::V + k] * Ri[R::V + k];
    deta[0] = -s_i - rho * igm1 * (T(0.5) * v2 * ieps - T(p.gamma) * irho);
#pragma unroll
    for (int k = 0; k < DIM; ++k) deta[1 + k] = g1 * Ri[R::V + k];
    deta[S - 1] = -g1;
  }
  T N = T(0), D = T(0);
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  for (int64_t k = k0; k < k1; ++k) {
    if (m.col[k] == i) continue;
    const T *wk = w_slot<DIM, T>(w, k);
    const T a_ = *a_ptr<DIM, T>(w, k);
    T b_ = T(0);
#pragma unroll
    for (int s = 0; s < S; ++s) b_ += deta[s] * wk[s];
    N += a_ - b_;
    D += abs_bits(a_) + abs_bits(b_);
  }
  w.alpha[i] = D > T(0) ? 0.5 * (double)(fabs(N) / D) : 0.0;  // alpha_i / 2 (exact): d^H_ij = (a_i/2 + a_j/2) d_ij
}

// Algorithm 1 steps 2-3 for one row; returns the row's CFL bound
// c_cfl m_i / (2 sum_{j != i} d_ij)
template <int DIM, typename T>
__device__ __forceinline__ double low_row(const MeshView &m, const Params &p, const Work &w, int i) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  using R = Rec<DIM>;
  const double *Ri = w.rec + (int64_t)i * R::SIZE;
  double ui[S];
#pragma unroll
  for (int s = 0; s < S; ++s) ui[s] = Ri[s];
  const double alphai = w.alpha[i];

  // U^L increment and the bounds in FP64; F^H in the viscosity precision T
  // U^L increment in FP64 (also in mixed mode); the sum of the w_ij in their
  // own precision T (FP32 values summed in FP32 in mixed mode, converted once)
  double inc[S];
  T wsum[S];
  T fh[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    inc[s] = 0.0;
    wsum[s] = T(0);
    fh[s] = T(0);
  }
  // bar-state densities rho_bar = num / den, den = 2 d_ij > 0; the running
  // minimum / maximum is kept as a fraction and compared by cross-multiplication
  double nmin = ui[0], dmin = 1.0, nmax = ui[0], dmax = 1.0;
  double phimin = Ri[R::PHI], dsum = 0.0;
  int64_t kd = -1;
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  for (int64_t k = k0; k < k1; ++k) {
    const int j = m.col[k];
    if (j == i) {
      kd = k;
      continue;
    }
    const double *Rj = w.rec + (int64_t)j * R::SIZE;
    const T *wk = w_slot<DIM, T>(w, k);
    const T dkT = *d_ptr<DIM, T>(w, k);
    const double dk = (double)dkT;
    const T dH = T(alphai + w.alpha[j]) * dkT;  // w.alpha holds alpha / 2
    const double w0 = (double)wk[0];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const double du = Rj[s] - ui[s];
      inc[s] += dk * du;  // sum_j d_ij (U_j - U_i); the sum of w_ij is subtracted once
      fh[s] += dH * (T)du;
      wsum[s] += wk[s];
    }
    if (dbits(dk) > 0) {  // dk >= 0
      const double num = dk * (ui[0] + Rj[0]) - w0;
      const double den = 2.0 * dk;
      const long long knew_min = order_key(num * dmin), kmin = order_key(nmin * den);
      const long long knew_max = order_key(num * dmax), kmax = order_key(nmax * den);
      if (knew_min < kmin) {
        nmin = num;
        dmin = den;
      }
      if (knew_max > kmax) {
        nmax = num;
        dmax = den;
      }
    }
    // Phi > 0: the integer order of the bit patterns is the numeric order
    const long long pj = __double_as_longlong(Rj[R::PHI]), pm = __double_as_longlong(phimin);
    phimin = __longlong_as_double(pj < pm ? pj : pm);
    dsum += dk;
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    inc[s] -= (double)wsum[s];
    fh[s] -= wsum[s];
  }
  *d_ptr<DIM, T>(w, kd) = (T)(-dsum);
  double *inci = w.inc + (int64_t)i * SP;
  T *fhi = (T *)w.vFH + (int64_t)i * SP;  // stored as F^H_i / m_i
  const T imi = T(m.inv_mi[i]);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    inci[s] = inc[s];
    fhi[s] = fh[s] * imi;
    if constexpr (sizeof(T) == 4) w.G64[(int64_t)i * SP + s] = (double)fhi[s];
  }
  const double rmin = dmin == 1.0 ? nmin : nmin / dmin;
  const double rmax = dmax == 1.0 ? nmax : nmax / dmax;
  const double r = m.relax[i];
  double *bi = w.bounds + (int64_t)i * 4;
  bi[0] = (1.0 - r) * rmin;
  bi[1] = (1.0 + r) * rmax;
  bi[2] = (1.0 - r) * phimin;
  w.rough2[i] = 1;
  return p.cfl * m.mi[i] / (2.0 * dsum);
}

// The same for a row whose neighbours all carry U_i bit for bit (rough[i] =
// 0): every w_ij is 0 and U_j - U_i = 0, so the increment and F^H vanish,
// every bar state is U_i (rho_min = rho_max = rho_i) and Phi_min = Phi_i --
// the values the general row gives, bit for bit. Only sum_j d_ij remains
// (same order). rough2[i] records whether a neighbour is rough.
template <int DIM, typename T>
__device__ __forceinline__ double low_row_smooth(const MeshView &m, const Params &p, const Work &w, int i) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  using R = Rec<DIM>;
  double dsum = 0.0;
  int64_t kd = -1;
  unsigned char r2 = 0;
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  for (int64_t k = k0; k < k1; ++k) {
    const int j = m.col[k];
    if (j == i) {
      kd = k;
      continue;
    }
    dsum += (double)*d_ptr<DIM, T>(w, k);
    r2 |= w.rough[j];
  }
  *d_ptr<DIM, T>(w, kd) = (T)(-dsum);
  double *inci = w.inc + (int64_t)i * SP;
  T *fhi = (T *)w.vFH + (int64_t)i * SP;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    inci[s] = 0.0;
    fhi[s] = T(0);
    if constexpr (sizeof(T) == 4) w.G64[(int64_t)i * SP + s] = 0.0;
  }
  const double *Ri = w.rec + (int64_t)i * R::SIZE;
  const double rho = Ri[0];
  const double r = m.relax[i];
  double *bi = w.bounds + (int64_t)i * 4;
  bi[0] = (1.0 - r) * rho;
  bi[1] = (1.0 + r) * rho;
  bi[2] = (1.0 - r) * Ri[R::PHI];
  w.rough2[i] = r2;
  return p.cfl * m.mi[i] / (2.0 * dsum);
}

// ---------------------------------------------------------------------------
// k_low: Algorithm 1 steps 2-3 -- d_ii, CFL bound, low-order increment, local
// bounds and high-order fluxes
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void __launch_bounds__(TPB_MAX) k_low(MeshView m, Params p, Work w) {
  __shared__ double smin[TPB_MAX / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double bound = INFINITY;
  if (i < m.n && !w.st->err) bound = w.rough[i] ? low_row<DIM, T>(m, p, w, i) : low_row_smooth<DIM, T>(m, p, w, i);
  // per-instance minimum of the CFL bound (exact and order independent: the
  // bit patterns of positive doubles order like their values). A block whose
  // rows lie in one instance reduces first and issues one atomic.
  const int first = blockIdx.x * blockDim.x;
  const int last = min(first + (int)blockDim.x, m.n) - 1;
  const int k_first = m.inst ? m.inst[first] : 0;
  const int k_last = m.inst ? m.inst[last] : 0;
  if (k_first == k_last) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bound = fmin(bound, __shfl_xor_sync(0xffffffffu, bound, off));
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = bound;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = smin[0];
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q) b = fmin(b, smin[q]);
      if (b < INFINITY) atomicMin(&w.bound_bits[k_first], (unsigned long long)__double_as_longlong(b));
    }
  } else if (i < m.n && bound < INFINITY) {
    atomicMin(&w.bound_bits[m.inst[i]], (unsigned long long)__double_as_longlong(bound));
  }
}

// ---------------------------------------------------------------------------
// k_tau: each instance's CFL bound (the minimum gathered by k_low); fixes the
// instance's tau at the first stage (Sec. 3.1) and resets the minimum
// ---------------------------------------------------------------------------
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

__global__ void __launch_bounds__(256) k_tau(MeshView m, Work w, int stage, double dt_given, double cfl,
                                             int advance_time) {
  DevStatus *st = w.st;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < LSQ_SLOTS) {  // the stage's queued line searches start empty
    w.lsq_count[k] = 0;
    w.lsq2_count[k] = 0;
  }
  if (k >= m.ninst || st->err) return;
  const double bound = __longlong_as_double((long long)w.bound_bits[k]);
  w.bound_bits[k] = kInfBits;
  w.bound_inst[stage * m.ninst + k] = bound;
  if (k == 0) st->stage_bound[stage] = bound;
  const double limit = bound / cfl;  // invariant-domain limit, c_cfl = 1
  if (stage == 0) {
    double tau;
    if (dt_given > 0.0) {
      if (dt_given > limit) {
        atomicExch(&st->err, 5);  // EH_ERR_CFL
        return;
      }
      tau = dt_given;
    } else {
      tau = bound;
    }
    const double left = w.tfinal_inst[k] - w.t_inst[k];
    if (tau > left) tau = left > 0.0 ? left : 0.0;  // land on t_final; finished instances stay frozen
    w.tau_inst[k] = tau;
    if (k == 0) st->tau = tau;
  } else {
    if (w.tau_inst[k] > limit) atomicAdd(&st->cfl_violations, 1ull);
    if (advance_time && stage == 2) {
      w.t_inst[k] += w.tau_inst[k];
      if (w.tau_inst[k] > 0.0) w.steps_inst[k] += 1ull;
    }
  }
}

// ---------------------------------------------------------------------------
// k_lim1: Algorithm 1 step 4 -- U^L, P_ij and the first line search
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__device__ __forceinline__ void lim1_row(const MeshView &m, const Params &p, const Work &w, double *P_trace, int i) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  using R = Rec<DIM>;
  if (!w.rough2[i]) {
    // row and neighbours without a differing neighbour state: the increment
    // is 0 (U^L = U_i) and every P_ij = (tc m_ij/m_i)(0 - 0) + (.)(U_j - U_i)
    // is 0, so every search returns 1 (reading R5b) -- as the general row
    const double *Ri = w.rec + (int64_t)i * R::SIZE;
    double *ULi = w.UL + (int64_t)i * SP;
#pragma unroll
    for (int s = 0; s < S; ++s) ULi[s] = Ri[s];
    const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
    if (P_trace) {
      for (int64_t k = k0; k < k1; ++k) {
#pragma unroll
        for (int s = 0; s < S; ++s) P_trace[k * SP + s] = 0.0;
      }
    }
    w.lone[i] = 1;  // every limiter is 1; la is not written (readers check lone first)
    return;
  }
  const double tau = w.tau_inst[m.inst ? m.inst[i] : 0];
  const double *Ri = w.rec + (int64_t)i * R::SIZE;
  double ui[S], ul[S], gi[S];
  const double *inci = w.inc + (int64_t)i * SP;
  const double *Garr = w.G64;  // G = F^H / m per node, in FP64 (widened once per node in mixed mode)

  const double *Gi = Garr + (int64_t)i * SP;
  const double tm = tau * m.inv_mi[i];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    ui[s] = Ri[s];
    ul[s] = ui[s] + tm * inci[s];
    gi[s] = Gi[s];
  }
  double *ULi = w.UL + (int64_t)i * SP;
#pragma unroll
  for (int s = 0; s < S; ++s) ULi[s] = ul[s];
  {
    // U^L admissible: rho > 0 and rho E - |M|^2/2 > 0 (no division); with
    // c_cfl <= 1 it always is (invariant-domain property), above 1 the
    // adaptive step restarts on it
    double m2 = 0.0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) m2 += ul[1 + q] * ul[1 + q];
    if (!(pos_strict(ul[0]) && pos_strict(ul[S - 1] * ul[0] - 0.5 * m2)))
      atomicAdd(&w.st->low_not_admissible, 1ull);
  }
  const double *bi = w.bounds + (int64_t)i * 4;
  const double rmin = bi[0], rmax = bi[1], phimin = bi[2];
  const double phimin2 = phimin * phimin, phimin5 = phimin2 * phimin2 * phimin;
  const RowF32 rf = row_f32<DIM>(ul, rmin, rmax, phimin5);
  const double alphai = w.alpha[i];
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  // P_ij = tau/(m_i lambda_i) (b_ij F^H_j - b_ji F^H_i + (d^H_ij - d_ij)(U_j - U_i))
  // with b_ij = -m_ij/m_j, b_ji = -m_ji/m_i and m_ij = m_ji:
  //      = (tc m_ij/m_i) (G_i - G_j) + (tc/m_i) (d^H_ij - d_ij)(U_j - U_i),
  // G = F^H/m, tc = tau (card I(i) - 1)
  const double tc = tau * (double)(k1 - k0 - 1);
  const double coef = tc * m.inv_mi[i];
  uint64_t defer = 0;  // entries whose line search goes to k_ls_deferred
  bool long_deferred = false;
  const bool longrow = k1 - k0 > 64;  // limiters stored as they are known
  for (int64_t k = k0; k < k1; ++k) {
    const int j = m.col[k];
    double *Pk = w.P + k * SP;
    if (j == i) {
#pragma unroll
      for (int s = 0; s < S; ++s) Pk[s] = 0.0;
      if (P_trace) {
#pragma unroll
        for (int s = 0; s < S; ++s) P_trace[k * SP + s] = 0.0;
      }
      if (longrow) w.la[k] = 1.0;
      continue;
    }
    const double *Rj = w.rec + (int64_t)j * R::SIZE;
    const double *Gj = Garr + (int64_t)j * SP;
    const double dk = (double)*d_ptr<DIM, T>(w, k);
    const double dH = (alphai + w.alpha[j]) * dk;  // w.alpha holds alpha / 2
    const double cm = tc * m.betat[k], cd = coef * (dH - dk);
    double P[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      P[s] = cm * (gi[s] - Gj[s]) + cd * (Rj[s] - ui[s]);
      Pk[s] = P[s];
    }
    if (P_trace) {
#pragma unroll
      for (int s = 0; s < S; ++s) P_trace[k * SP + s] = P[s];
    }
    if (line_search_at_one<DIM>(p, ul, P, rmin, rmax, phimin5, rf)) {
      if (longrow) w.la[k] = 1.0;
    } else if (k - k0 < 64) {
      defer |= 1ull << (k - k0);
    } else {
      defer_line_searches(w, 0, i, k, 1ull);  // rows longer than 64 entries
      long_deferred = true;
    }
  }
  const bool lone = defer == 0 && !long_deferred;
  w.lone[i] = lone ? 1 : 0;
  // a row with a queued search stores its other limiters (1); a row without
  // one stores none (every limiter of it is 1, and its lone flag says so)
  if (!lone && !longrow)
    for (int64_t k = k0; k < k1; ++k)
      if (!((defer >> (k - k0)) & 1ull)) w.la[k] = 1.0;
  defer_line_searches(w, 0, i, k0, defer);
}

// rows i, i + grid size, ... (the grid may be capped to limit the rows in
// flight; one row per thread otherwise)
template <int DIM, typename T>
__global__ void __launch_bounds__(TPB_MAX) k_lim1(MeshView m, Params p, Work w, double *P_trace) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n; i += gridDim.x * blockDim.x) {
    if (w.st->err) return;
    lim1_row<DIM, T>(m, p, w, P_trace, i);
  }
}

// min of two limiters in [0, 1]: non-negative doubles order like their bit
// patterns, so an integer min (no FP64 instruction) gives the same value
__device__ __forceinline__ double lmin(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x < y ? x : y);
}

// The symmetrised limiters l_ij = min(l_k, l_tr[k]) of the cnt <= LCHUNK
// entries kb, kb + 1, ... of row i (diag[q]: the entry is the diagonal); a
// row whose lone flag is set has every limiter 1 (and none stored). Every
// load of the chunk is issued before the first use: the transposed value is a
// dependent gather (tr[k], then l at tr[k]), and issuing a chunk's gathers
// together overlaps their latencies instead of paying them one entry at a time.
constexpr int LCHUNK = 3;  // measured on the 4.0M cylinder: 3 shortens k_final by 7%; 4 and 9 lengthen it
                           // (one limiter pass; after two or more k_final gathers only where rem != 0)
__device__ __forceinline__ void sym_limiters(const MeshView &m, const double *__restrict__ lin,
                                             const unsigned char *__restrict__ lone, int64_t kb, int cnt, int i,
                                             double *ls, bool *diag) {
  int32_t t[LCHUNK], c[LCHUNK];
#pragma unroll
  for (int q = 0; q < LCHUNK; ++q)
    if (q < cnt) {
      t[q] = m.tr[kb + q];
      c[q] = m.col[kb + q];
    }
  const bool one_i = lone[i] != 0;
  double a[LCHUNK], b[LCHUNK];
#pragma unroll
  for (int q = 0; q < LCHUNK; ++q)
    if (q < cnt) {
      a[q] = one_i ? 1.0 : lin[kb + q];
      b[q] = lone[c[q]] ? 1.0 : lin[t[q]];
    }
#pragma unroll
  for (int q = 0; q < LCHUNK; ++q)
    if (q < cnt) {
      ls[q] = lmin(a[q], b[q]);
      diag[q] = c[q] == i;
    }
}

// ---------------------------------------------------------------------------
// k_pass: symmetrise the limiter, update, shrink P and search again
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void pass_row(const MeshView &m, const Params &p, const Work &w, const double *__restrict__ Uin,
                                         double *__restrict__ Uout, const double *__restrict__ lin,
                                         double *__restrict__ lout, double *lsym_trace, int slot, int i) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  const double lambda_i = m.lam[i];
  double u[S];
  const double *Ui = Uin + (int64_t)i * SP;
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = Ui[s];
  const unsigned char *lone_in = w.lone + (int64_t)((slot - 1) & 1) * m.n;
  unsigned char *lone_out = w.lone + (int64_t)(slot & 1) * m.n;
  if (!w.rough2[i]) {  // every P_ij is 0 (see lim1_row): the state stays, every next search returns 1
    double *Uo = Uout + (int64_t)i * SP;
#pragma unroll
    for (int s = 0; s < S; ++s) Uo[s] = u[s];
    if (lsym_trace) {
      for (int64_t k = k0; k < k1; ++k) {
        const int j = m.col[k];
        lsym_trace[k] = j == i ? 1.0 : lmin(lone_in[i] ? 1.0 : lin[k], lone_in[j] ? 1.0 : lin[m.tr[k]]);
      }
    }
    lone_out[i] = 1;  // every next limiter is 1; lout is not written
    return;
  }
  const bool one_i = lone_in[i] != 0;
  // slot = the pass (1, 2, ...): pass 1 starts from k_lim1's P_ij, a later
  // pass from the remainder rem[k] P[k] that the previous one left
  for (int64_t k = k0; k < k1; ++k) {
    const int j = m.col[k];
    if (j == i) {
      if (lsym_trace) lsym_trace[k] = 1.0;
      continue;
    }
    // a row whose limiters are all 1 has none stored: its side is 1, and an
    // entry between two such rows needs no gather of the transposed limiter
    const double l = lmin(one_i ? 1.0 : lin[k], lone_in[j] ? 1.0 : lin[m.tr[k]]);
    if (lsym_trace) lsym_trace[k] = l;
    double *Pk = w.P + k * SP;
    double P[S];
    if (slot > 1) {
      const double r = w.rem[k];
      if (dbits(r) == 0) continue;  // nothing left of P_ij (rem stays 0)
#pragma unroll
      for (int s = 0; s < S; ++s) {
        P[s] = r * Pk[s];
        Pk[s] = P[s];  // this pass's P_ij, for the remainder it leaves
      }
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) P[s] = Pk[s];
    }
    // the update with l P; the remainder (1 - l) P is left as rem[k] (a
    // store of (1 - l) P here costs more than forming it where it is read,
    // and for l = 1 -- most entries -- nothing is read at all)
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] += lambda_i * l * P[s];
    w.rem[k] = 1.0 - l;
  }
  double *Uo = Uout + (int64_t)i * SP;
#pragma unroll
  for (int s = 0; s < S; ++s) Uo[s] = u[s];
  const double *bi = w.bounds + (int64_t)i * 4;
  const double rmin = bi[0], rmax = bi[1], phimin = bi[2];
  const double phimin2 = phimin * phimin, phimin5 = phimin2 * phimin2 * phimin;
  const RowF32 rf = row_f32<DIM>(u, rmin, rmax, phimin5);
  uint64_t defer = 0;
  bool long_deferred = false;
  const bool longrow = k1 - k0 > 64;  // limiters stored as they are known
  for (int64_t k = k0; k < k1; ++k) {
    if (m.col[k] == i) {
      if (longrow) lout[k] = 1.0;
      continue;
    }
    const double r = w.rem[k];
    if (dbits(r) == 0) {  // the remainder is 0: every l gives the same state, the largest is 1
      if (longrow) lout[k] = 1.0;
      continue;
    }
    const double *Pk = w.P + k * SP;
    double P[S];
#pragma unroll
    for (int s = 0; s < S; ++s) P[s] = r * Pk[s];
    if (line_search_at_one<DIM>(p, u, P, rmin, rmax, phimin5, rf)) {
      if (longrow) lout[k] = 1.0;
    } else if (k - k0 < 64) {
      defer |= 1ull << (k - k0);
    } else {
      defer_line_searches(w, slot, i, k, 1ull);
      long_deferred = true;
    }
  }
  const bool lone = defer == 0 && !long_deferred;
  lone_out[i] = lone ? 1 : 0;
  if (!lone && !longrow)  // as in k_lim1: only a row with a queued search stores its limiters
    for (int64_t k = k0; k < k1; ++k)
      if (!((defer >> (k - k0)) & 1ull)) lout[k] = 1.0;
  defer_line_searches(w, slot, i, k0, defer);
}

template <int DIM>
__global__ void __launch_bounds__(TPB_MAX) k_pass(MeshView m, Params p, Work w, const double *__restrict__ Uin,
                                              double *__restrict__ Uout, const double *__restrict__ lin,
                                              double *__restrict__ lout, double *lsym_trace, int slot) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n; i += gridDim.x * blockDim.x) {
    if (w.st->err) return;
    pass_row<DIM>(m, p, w, Uin, Uout, lin, lout, lsym_trace, slot, i);
  }
}

// ---------------------------------------------------------------------------
// k_ls_deferred / k_ls_iterate: the queued line searches of one pass, one per
// thread, from the pass's start state ub, the stored P_ij and the row's
// bounds. The first kernel takes every exit without iteration and queues the
// rest for the second, whose threads then all run the same iteration count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool queue_iteration(const Work &w, int slot, const LsItem &it) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&w.lsq2_count[slot], g.size());
  base = g.shfl(base, 0) + g.thread_rank();
  if (base >= w.lsq2_cap) return false;  // full: the caller iterates itself
  w.lsq2[base] = it;
  return true;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_ls_deferred(MeshView m, Params p, Work w, const double *__restrict__ ub,
                                                     int slot, double *__restrict__ lout) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  if (w.st->err) return;
  const unsigned cnt = min(w.lsq_count[slot], w.lsq_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.st->line_searches_deferred, (unsigned long long)cnt);
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
    const int2 it = w.lsq[q];
    const double *bi = w.bounds + (int64_t)it.x * 4;
    const double phimin = bi[2], phimin2 = phimin * phimin, phimin5 = phimin2 * phimin2 * phimin;
    double u[S], P[S];
    const double r = slot > 0 ? w.rem[it.y] : 1.0;  // a later pass: the remainder rem P
#pragma unroll
    for (int s = 0; s < S; ++s) {
      u[s] = ub[(int64_t)it.x * SP + s];
      P[s] = slot > 0 ? r * w.P[(int64_t)it.y * SP + s] : w.P[(int64_t)it.y * SP + s];
    }
    const LsBracket b = line_search_start<DIM>(p, u, P, bi[0], bi[1], phimin, phimin5);
    if (b.done)
      lout[it.y] = b.l;
    else if (!queue_iteration(w, slot, LsItem{it.x, it.y, b.l, b.pl, b.pr, b.rR}))
      lout[it.y] = line_search_iterate<DIM>(p, u, P, phimin, b);
  }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_ls_iterate(MeshView m, Params p, Work w, const double *__restrict__ ub,
                                                    int slot, double *__restrict__ lout) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  if (w.st->err) return;
  const unsigned cnt = min(w.lsq2_count[slot], w.lsq2_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.st->line_searches_iterated, (unsigned long long)cnt);
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
    const LsItem it = w.lsq2[q];
    const double phimin = w.bounds[(int64_t)it.i * 4 + 2];
    double u[S], P[S];
    const double r = slot > 0 ? w.rem[it.k] : 1.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      u[s] = ub[(int64_t)it.i * SP + s];
      P[s] = slot > 0 ? r * w.P[(int64_t)it.k * SP + s] : w.P[(int64_t)it.k * SP + s];
    }
    const LsBracket b{it.l, it.pl, it.pr, it.rR, false};
    lout[it.k] = line_search_iterate<DIM>(p, u, P, phimin, b);
  }
}

// ---------------------------------------------------------------------------
// k_final: last limited update, boundary post-processing (Sec. 4), SSP
// combination (Sec. 4.1) and admissibility check
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Sec. 4.2: non-reflecting post-processing of one state along the unit
// outward normal nv with the far-field (Dirichlet) state ud
// ---------------------------------------------------------------------------
template <int DIM> struct NormalState {
  double rho, un, ut[DIM], p, c;  // density, normal and tangential velocity, pressure, sound speed
};

template <int DIM>
__device__ NormalState<DIM> split_normal(const double *u, const double *nv, double gamma) {
  NormalState<DIM> w;
  w.rho = u[0];
  const double ir = 1.0 / u[0];
  double un = 0.0, v2 = 0.0;
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    const double v = u[1 + q] * ir;
    un += v * nv[q];
    v2 += v * v;
  }
  w.un = un;
#pragma unroll
  for (int q = 0; q < DIM; ++q) w.ut[q] = u[1 + q] * ir - un * nv[q];
  w.p = (gamma - 1.0) * (u[DIM + 1] - 0.5 * u[0] * v2);
  w.c = sqrt(gamma * w.p * ir);
  return w;
}

template <int DIM>
__device__ void join_normal(double rho, double un, const double *ut, double pr, const double *nv, double gamma,
                            double *u) {
  u[0] = rho;
  double v2 = 0.0;
#pragma unroll
  for (int q = 0; q < DIM; ++q) {
    const double v = ut[q] + un * nv[q];
    u[1 + q] = rho * v;
    v2 += v * v;
  }
  u[DIM + 1] = pr / (gamma - 1.0) + 0.5 * rho * v2;
}

// Sec. 4.2.2: incoming characteristics (C_1 = u_n - 2c/(gamma-1) at speed
// u_n - c; entropy p rho^-gamma and tangential velocity at u_n; C_3 = u_n +
// 2c/(gamma-1) at u_n + c) take the far-field values, outgoing ones keep the
// node's: eqs. Supersonic_inflow, Subsonic_inflow, Subsonic_outflow,
// Supersonic_outflow.
template <int DIM>
__device__ void bc_characteristic(double *u, const double *nv, const double *ud, double gamma) {
  const NormalState<DIM> in = split_normal<DIM>(u, nv, gamma);
  if (in.un < 0.0 && -in.un > in.c) {  // every wave enters
#pragma unroll
    for (int s = 0; s < DIM + 2; ++s) u[s] = ud[s];
    return;
  }
  if (in.un >= 0.0 && in.un >= in.c) return;  // every wave leaves
  const NormalState<DIM> far = split_normal<DIM>(ud, nv, gamma);
  const double k = 2.0 / (gamma - 1.0);
  const double c3 = in.un + k * in.c, c1 = far.un - k * far.c;
  const NormalState<DIM> &up = in.un < 0.0 ? far : in;  // source of entropy and tangential velocity
  const double ent = up.p * pow(up.rho, -gamma);
  const double cp = 0.25 * (gamma - 1.0) * (c3 - c1);
  const double rho = pow(cp * cp / (gamma * ent), 1.0 / (gamma - 1.0));
  join_normal<DIM>(rho, 0.5 * (c1 + c3), up.ut, ent * pow(rho, gamma), nv, gamma, u);
}

// wave curve of side w through its state: the jump in normal velocity across
// a 1- or 3-wave that leads to pressure p, and its derivative in p
template <int DIM>
__device__ void wave_curve(double p, const NormalState<DIM> &w, double gamma, double *f, double *df) {
  if (p > w.p) {  // shock (Rankine-Hugoniot)
    const double A = 2.0 / ((gamma + 1.0) * w.rho), B = w.p * (gamma - 1.0) / (gamma + 1.0);
    const double r = sqrt(A / (B + p));
    *f = (p - w.p) * r;
    *df = r * (1.0 - 0.5 * (p - w.p) / (B + p));
  } else {  // rarefaction (isentropic)
    const double e = 0.5 * (gamma - 1.0) / gamma;
    const double q = pow(p / w.p, e);
    *f = 2.0 * w.c / (gamma - 1.0) * (q - 1.0);
    *df = q * w.c / (gamma * p);
  }
}

// Sec. 4.2.1, eq. Godunov_bc: the exact solution at x/t = 0 of the Riemann
// problem along nv with the node's state on the inside (left) and the far
// field outside (right)
template <int DIM>
__device__ void bc_godunov(double *u, const double *nv, const double *ud, double gamma) {
  const NormalState<DIM> L = split_normal<DIM>(u, nv, gamma), R = split_normal<DIM>(ud, nv, gamma);
  const double gm = gamma - 1.0, gp = gamma + 1.0, e = 0.5 * gm / gamma;
  const double jump = R.un - L.un;
  double rho, un, pr;
  const double *ut;
  if (2.0 * (L.c + R.c) / gm <= jump) {  // vacuum between two rarefactions
    const double head_l = L.un - L.c, edge_l = L.un + 2.0 * L.c / gm;
    const double edge_r = R.un - 2.0 * R.c / gm, head_r = R.un + R.c;
    if (head_l >= 0.0) {
      rho = L.rho; un = L.un; pr = L.p; ut = L.ut;
    } else if (edge_l > 0.0) {
      const double c = 2.0 / gp * (L.c + 0.5 * gm * L.un);
      rho = L.rho * pow(c / L.c, 2.0 / gm); un = c; pr = L.p * pow(c / L.c, 1.0 / e); ut = L.ut;
    } else if (edge_r >= 0.0) {
      rho = 0.0; un = 0.0; pr = 0.0; ut = L.ut;
    } else if (head_r > 0.0) {
      const double c = 2.0 / gp * (R.c - 0.5 * gm * R.un);
      rho = R.rho * pow(c / R.c, 2.0 / gm); un = -c; pr = R.p * pow(c / R.c, 1.0 / e); ut = R.ut;
    } else {
      rho = R.rho; un = R.un; pr = R.p; ut = R.ut;
    }
    join_normal<DIM>(rho, un, ut, pr, nv, gamma, u);
    if (rho == 0.0) {
#pragma unroll
      for (int s = 0; s < DIM + 2; ++s) u[s] = 0.0;
    }
    return;
  }
  // star pressure: Newton from the two-rarefaction value to a relative change of 1e-15
  double ps = pow((L.c + R.c - 0.5 * gm * jump) / (L.c * pow(L.p, -e) + R.c * pow(R.p, -e)), 1.0 / e);
  for (int it = 0; it < 100; ++it) {
    double fl, dl, fr, dr;
    wave_curve<DIM>(ps, L, gamma, &fl, &dl);
    wave_curve<DIM>(ps, R, gamma, &fr, &dr);
    double pn = ps - (fl + fr + jump) / (dl + dr);
    if (!(pn > 0.0)) pn = 0.5 * ps;
    const double rel = fabs(pn - ps) / (0.5 * (pn + ps));
    ps = pn;
    if (rel < 1e-15) break;
  }
  double fl, dl, fr, dr;
  wave_curve<DIM>(ps, L, gamma, &fl, &dl);
  wave_curve<DIM>(ps, R, gamma, &fr, &dr);
  const double us = 0.5 * (L.un + R.un + fr - fl);  // contact speed
  const bool left = us >= 0.0;
  const NormalState<DIM> &K = left ? L : R;
  const double sgn = left ? 1.0 : -1.0;  // mirror the right side onto the left
  ut = K.ut;
  const double uk = sgn * K.un, ustar = sgn * us;
  if (ps > K.p) {  // shock moving away from the contact
    const double speed = uk - K.c * sqrt(0.5 * gp / gamma * ps / K.p + e);
    if (speed >= 0.0) {
      rho = K.rho; un = K.un; pr = K.p;
    } else {
      const double r = ps / K.p, g6 = gm / gp;
      rho = K.rho * (r + g6) / (g6 * r + 1.0); un = us; pr = ps;
    }
  } else if (uk - K.c >= 0.0) {  // rarefaction entirely on the far side of x = 0
    rho = K.rho; un = K.un; pr = K.p;
  } else if (ustar - K.c * pow(ps / K.p, e) < 0.0) {  // x = 0 in the star region
    rho = K.rho * pow(ps / K.p, 1.0 / gamma); un = us; pr = ps;
  } else {  // x = 0 inside the rarefaction fan
    const double c = 2.0 / gp * (K.c + 0.5 * gm * uk);
    rho = K.rho * pow(c / K.c, 2.0 / gm); un = sgn * c; pr = K.p * pow(c / K.c, 1.0 / e);
  }
  join_normal<DIM>(rho, un, ut, pr, nv, gamma, u);
}

// Sec. 4 without the non-reflecting kinds: slip and Dirichlet applied, the
// return value tells whether the node is a non-reflecting one (its
// post-processing then runs in k_final_nonreflecting, out of the row kernel,
// whose register budget it would otherwise set)
template <int DIM>
__device__ __forceinline__ bool apply_bc_node_local(const MeshView &m, int i, double *u) {
  const int b = m.bnd_index[i];
  if (b < 0) return false;
  const int kind = m.bnd_kind[b];
  if (kind == 1) {  // slip: M <- M - (M . n^s) n^s
    double mn = 0.0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) mn += u[1 + q] * m.bnd_normal[(int64_t)q * m.n_bnd + b];
#pragma unroll
    for (int q = 0; q < DIM; ++q) u[1 + q] -= mn * m.bnd_normal[(int64_t)q * m.n_bnd + b];
  } else if (kind == 2) {  // supersonic inflow: U <- U^D
#pragma unroll
    for (int s = 0; s < DIM + 2; ++s) u[s] = m.bnd_state[(int64_t)s * m.n_bnd + b];
  }
  return kind == 4 || kind == 5;
}

// Sec. 4: slip (M <- M - (M . n^s) n^s), Dirichlet / supersonic inflow
// (U <- U^D), do nothing, and the two non-reflecting post-processings
template <int DIM>
__device__ __forceinline__ void apply_bc_node(const MeshView &m, const Params &p, int i, double *u) {
  const int b = m.bnd_index[i];
  if (b < 0) return;
  const int kind = m.bnd_kind[b];
  if (kind == 1) {  // slip: M <- M - (M . n^s) n^s
    double mn = 0.0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) mn += u[1 + q] * m.bnd_normal[(int64_t)q * m.n_bnd + b];
#pragma unroll
    for (int q = 0; q < DIM; ++q) u[1 + q] -= mn * m.bnd_normal[(int64_t)q * m.n_bnd + b];
  } else if (kind == 2) {  // supersonic inflow: U <- U^D
#pragma unroll
    for (int s = 0; s < DIM + 2; ++s) u[s] = m.bnd_state[(int64_t)s * m.n_bnd + b];
  } else if (kind == 4 || kind == 5) {
    double nv[DIM], ud[DIM + 2];
#pragma unroll
    for (int q = 0; q < DIM; ++q) nv[q] = m.bnd_normal[(int64_t)q * m.n_bnd + b];
#pragma unroll
    for (int s = 0; s < DIM + 2; ++s) ud[s] = m.bnd_state[(int64_t)s * m.n_bnd + b];
    if (kind == 4)
      bc_characteristic<DIM>(u, nv, ud, p.gamma);
    else
      bc_godunov<DIM>(u, nv, ud, p.gamma);
  }
}

template <int DIM>
__device__ __forceinline__ bool admissible(const double *u) {
  double m2 = 0.0;
#pragma unroll
  for (int q = 0; q < DIM; ++q) m2 += u[1 + q] * u[1 + q];
  return u[0] > 0.0 && (u[DIM + 1] - m2 / (2.0 * u[0])) > 0.0;
}

template <int DIM>
__device__ __forceinline__ void final_row(const MeshView &m, const Params &p, const Work &w, const double *__restrict__ Uin,
                                          const double *__restrict__ lin, const double *U0, double coef, double *out,
                                          double *Upre_trace, double *lsym_trace, int i) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  const int64_t k0 = m.row_ptr[i], k1 = m.row_ptr[i + 1];
  const double lambda_i = m.lam[i];
  double u[S];
  const double *Ui = Uin + (int64_t)i * SP;
#pragma unroll
  for (int s = 0; s < S; ++s) u[s] = Ui[s];
  const unsigned char *lone = w.lone + (int64_t)((p.limiter_passes - 1) & 1) * m.n;  // of the last pass
  if (w.rough2[i] && p.limiter_passes >= 2) {
    // the remainder rem P that the last k_pass left: where rem = 0 (most
    // entries) the update adds nothing, and the symmetrised limiter -- a
    // dependent gather of the transposed one -- is not needed
    for (int64_t k = k0; k < k1; ++k) {
      if (m.col[k] == i) {
        if (lsym_trace) lsym_trace[k] = 1.0;
        continue;
      }
      const double r = w.rem[k];
      if (dbits(r) == 0 && !lsym_trace) continue;
      const int j = m.col[k];
      const double l = lmin(lone[i] ? 1.0 : lin[k], lone[j] ? 1.0 : lin[m.tr[k]]);
      if (lsym_trace) lsym_trace[k] = l;
      if (dbits(r) == 0) continue;
      const double *Pk = w.P + k * SP;
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] += lambda_i * l * (r * Pk[s]);
    }
  } else if (w.rough2[i]) {  // else every P_ij is 0 (see lim1_row) and the update adds nothing
    for (int64_t kb = k0; kb < k1; kb += LCHUNK) {
      const int cnt = (int)min((int64_t)LCHUNK, k1 - kb);
      double ls[LCHUNK];
      bool dg[LCHUNK];
      sym_limiters(m, lin, lone, kb, cnt, i, ls, dg);
#pragma unroll
      for (int q = 0; q < LCHUNK; ++q) {
        if (q >= cnt) break;
        const int64_t k = kb + q;
        if (dg[q]) {
          if (lsym_trace) lsym_trace[k] = 1.0;
          continue;
        }
        if (lsym_trace) lsym_trace[k] = ls[q];
        const double *Pk = w.P + k * SP;
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] += lambda_i * ls[q] * Pk[s];
      }
    }
  } else if (lsym_trace) {
    for (int64_t k = k0; k < k1; ++k) {
      const int j = m.col[k];
      lsym_trace[k] = j == i ? 1.0 : lmin(lone[i] ? 1.0 : lin[k], lone[j] ? 1.0 : lin[m.tr[k]]);
    }
  }
  if (Upre_trace) {
#pragma unroll
    for (int s = 0; s < S; ++s) Upre_trace[(int64_t)i * SP + s] = u[s];
  }
  // a finished instance (tau = 0) keeps its state bit for bit: the stage is
  // the identity there, and re-applying the post-processing would not be
  if (w.tau_inst[m.inst ? m.inst[i] : 0] != 0.0 && apply_bc_node_local<DIM>(m, i, u)) {
    // non-reflecting node: hand the state to k_final_nonreflecting (the
    // low-order increment rows are free at this point of the stage)
    double *h = w.inc + (int64_t)i * SP;
#pragma unroll
    for (int s = 0; s < S; ++s) h[s] = u[s];
    return;
  }
  if (coef >= 0.0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const double u0 = U0[(int64_t)s * m.n + i];
      u[s] = u0 + coef * (u[s] - u0);
    }
  }
  if (!admissible<DIM>(u)) {
    atomicAdd(&w.st->not_admissible, 1ull);
    atomicExch(&w.st->err, 4);  // EH_ERR_NOT_ADMISSIBLE
  }
#pragma unroll
  for (int s = 0; s < S; ++s) out[(int64_t)s * m.n + i] = u[s];
}

template <int DIM>
__global__ void __launch_bounds__(TPB_MAX) k_final(MeshView m, Params p, Work w, const double *__restrict__ Uin,
                                               const double *__restrict__ lin, const double *U0, double coef,
                                               double *out, double *Upre_trace, double *lsym_trace) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n; i += gridDim.x * blockDim.x) {
    if (w.st->err) return;
    final_row<DIM>(m, p, w, Uin, lin, U0, coef, out, Upre_trace, lsym_trace, i);
  }
}

// the non-reflecting boundary nodes of a stage: post-processing (Sec. 4.2),
// SSP combination and admissibility, as k_final does for the other nodes
template <int DIM>
__global__ void __launch_bounds__(256) k_final_nonreflecting(MeshView m, Params p, Work w, const double *U0,
                                                             double coef, double *out) {
  constexpr int S = DIM + 2;
  constexpr int SP = Layout<DIM>::SP;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m.n_bnd || w.st->err) return;
  const int kind = m.bnd_kind[b];
  if (kind != 4 && kind != 5) return;
  const int i = m.bnd_node[b];
  if (w.tau_inst[m.inst ? m.inst[i] : 0] == 0.0) return;  // frozen instance: k_final wrote it
  double u[S], nv[DIM], ud[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    u[s] = w.inc[(int64_t)i * SP + s];
    ud[s] = m.bnd_state[(int64_t)s * m.n_bnd + b];
  }
#pragma unroll
  for (int q = 0; q < DIM; ++q) nv[q] = m.bnd_normal[(int64_t)q * m.n_bnd + b];
  if (kind == 4)
    bc_characteristic<DIM>(u, nv, ud, p.gamma);
  else
    bc_godunov<DIM>(u, nv, ud, p.gamma);
  if (coef >= 0.0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const double u0 = U0[(int64_t)s * m.n + i];
      u[s] = u0 + coef * (u[s] - u0);
    }
  }
  if (!admissible<DIM>(u)) {
    atomicAdd(&w.st->not_admissible, 1ull);
    atomicExch(&w.st->err, 4);  // EH_ERR_NOT_ADMISSIBLE
  }
#pragma unroll
  for (int s = 0; s < S; ++s) out[(int64_t)s * m.n + i] = u[s];
}

template <int DIM> __global__ void k_apply_bc(MeshView m, Params p, double *U) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.n || m.bnd_index[i] < 0) return;
  double u[DIM + 2];
#pragma unroll
  for (int s = 0; s < DIM + 2; ++s) u[s] = U[(int64_t)s * m.n + i];
  apply_bc_node<DIM>(m, p, i, u);
#pragma unroll
  for (int s = 0; s < DIM + 2; ++s) U[(int64_t)s * m.n + i] = u[s];
}

template <int DIM> __global__ void k_count_not_admissible(int n, const double *U, DevStatus *st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double u[DIM + 2];
#pragma unroll
  for (int s = 0; s < DIM + 2; ++s) u[s] = U[(int64_t)s * n + i];
  if (!admissible<DIM>(u)) atomicAdd(&st->not_admissible, 1ull);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int DIM, typename T>
void launch_prep(const MeshView &m, const Params &p, const double *U, const Work &w, int tpb, cudaStream_t s) {
  k_prep<DIM, T><<<nblocks(m.n, tpb), tpb, 0, s>>>(m, p, U, w.rec, (T *)w.vrec, w.rough, w.steady, w.st);
}
template <int DIM, typename T>
void launch_visc(const MeshView &m, const Params &p, const Work &w, int tpb, cudaStream_t s) {
  k_visc<DIM, T><<<nblocks(m.n, tpb), tpb, 0, s>>>(m, p, w);
}
template <int DIM, typename T>
void launch_alpha(const MeshView &m, const Params &p, const Work &w, int tpb, cudaStream_t s) {
  k_alpha<DIM, T><<<nblocks(m.n, tpb), tpb, 0, s>>>(m, p, w);
}
template <int DIM, typename T>
void launch_low(const MeshView &m, const Params &p, const Work &w, int tpb, cudaStream_t s) {
  k_low<DIM, T><<<nblocks(m.n, tpb), tpb, 0, s>>>(m, p, w);
}
void launch_tau(const MeshView &m, const Work &w, int stage, double dt_given, double cfl, bool advance_time,
                cudaStream_t s) {
  k_tau<<<nblocks(m.ninst, 256), 256, 0, s>>>(m, w, stage, dt_given, cfl, advance_time ? 1 : 0);
}
// grid of the grid-stride row kernels: one thread per row, or at most
// max_blocks blocks (max_blocks > 0)
inline unsigned capped_grid(int64_t n, int tpb, int max_blocks) {
  const unsigned g = nblocks(n, tpb);
  return (max_blocks > 0 && g > (unsigned)max_blocks) ? (unsigned)max_blocks : g;
}
template <int DIM, typename T>
void launch_lim1(const MeshView &m, const Params &p, const Work &w, double *P_trace, int tpb, int max_blocks,
                 cudaStream_t s) {
  k_lim1<DIM, T><<<capped_grid(m.n, tpb, max_blocks), tpb, 0, s>>>(m, p, w, P_trace);
}
template <int DIM>
void launch_pass(const MeshView &m, const Params &p, const Work &w, const double *Uin, double *Uout, const double *lin,
                 double *lout, double *lsym_trace, int slot, int tpb, int max_blocks, cudaStream_t s) {
  k_pass<DIM><<<capped_grid(m.n, tpb, max_blocks), tpb, 0, s>>>(m, p, w, Uin, Uout, lin, lout, lsym_trace, slot);
}
template <int DIM>
void launch_ls_deferred(const MeshView &m, const Params &p, const Work &w, const double *ub, int slot, double *lout,
                        int tpb, cudaStream_t s) {
  // a fixed grid (1024 threads per SM of a 152-SM GB300) that strides over
  // however many searches were queued; the count stays on the device
  k_ls_deferred<DIM><<<152 * 1024 / tpb, tpb, 0, s>>>(m, p, w, ub, slot, lout);
  k_ls_iterate<DIM><<<152 * 1024 / tpb, tpb, 0, s>>>(m, p, w, ub, slot, lout);
}
template <int DIM>
void launch_final(const MeshView &m, const Params &p, const Work &w, const double *Uin, const double *lin,
                  const double *U0, double coef, double *out, double *Upre_trace, double *lsym_trace, int tpb,
                  int max_blocks, cudaStream_t s) {
  k_final<DIM><<<capped_grid(m.n, tpb, max_blocks), tpb, 0, s>>>(m, p, w, Uin, lin, U0, coef, out, Upre_trace,
                                                                 lsym_trace);
  if (m.n_nonreflecting > 0)
    k_final_nonreflecting<DIM><<<nblocks(m.n_bnd, 256), 256, 0, s>>>(m, p, w, U0, coef, out);
}
template <int DIM> void launch_apply_bc(const MeshView &m, const Params &p, double *U, cudaStream_t s) {
  k_apply_bc<DIM><<<nblocks(m.n, 256), 256, 0, s>>>(m, p, U);
}
// min_i rho_i, min_i e_i (e = E/rho - |m|^2/(2 rho^2)) and sum_i m_i U_i over
// the whole state: a fixed grid of STAT_BLOCKS blocks with a grid stride,
// fixed shuffle and shared-memory trees per block, then one block summing the
// partials in a fixed order -- the same bits on every run
template <int DIM> __global__ void __launch_bounds__(256) k_state_partial(int n, const double *__restrict__ U,
                                                                        const double *__restrict__ mi,
                                                                        double *__restrict__ part) {
  constexpr int S = DIM + 2, NV = S + 2;
  double v[NV];
  v[0] = INFINITY;
  v[1] = INFINITY;
#pragma unroll
  for (int s = 0; s < S; ++s) v[2 + s] = 0.0;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += STAT_BLOCKS * 256) {
    double u[S];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = U[(int64_t)s * n + i];
    const double irho = 1.0 / u[0];
    double m2 = 0.0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) m2 += u[1 + q] * u[1 + q];
    v[0] = fmin(v[0], u[0]);
    v[1] = fmin(v[1], u[S - 1] * irho - 0.5 * m2 * irho * irho);
    const double m = mi[i];
#pragma unroll
    for (int s = 0; s < S; ++s) v[2 + s] += m * u[s];
  }
  __shared__ double sh[NV][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_down_sync(0xffffffffu, v[q], o);
      v[q] = q < 2 ? fmin(v[q], x) : v[q] + x;
    }
    if (lane == 0) sh[q][warp] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int q = threadIdx.x;
    double acc = sh[q][0];
    for (int w = 1; w < 8; ++w) acc = q < 2 ? fmin(acc, sh[q][w]) : acc + sh[q][w];
    part[q * STAT_BLOCKS + blockIdx.x] = acc;
  }
}

__global__ void k_state_final(int nv, const double *__restrict__ part, double *__restrict__ out) {
  const int q = threadIdx.x;
  if (q >= nv) return;
  double acc = part[q * STAT_BLOCKS];
  for (int b = 1; b < STAT_BLOCKS; ++b) acc = q < 2 ? fmin(acc, part[q * STAT_BLOCKS + b]) : acc + part[q * STAT_BLOCKS + b];
  out[q] = acc;
}

template <int DIM>
void launch_state_stats(int n, const double *U, const double *mi, double *part, double *out, cudaStream_t s) {
  k_state_partial<DIM><<<STAT_BLOCKS, 256, 0, s>>>(n, U, mi, part);
  k_state_final<<<1, 32, 0, s>>>(DIM + 4, part, out);
}
template <int DIM> void launch_count_not_admissible(int n, const double *U, DevStatus *st, cudaStream_t s) {
  k_count_not_admissible<DIM><<<nblocks(n, 256), 256, 0, s>>>(n, U, st);
}

// dst[i] = src[i] + add (nonneg_only: only where src[i] >= 0; -1 entries
// stay): the index arrays of one instance placed into a block-diagonal union
template <typename I> __global__ void k_offset_copy(I *dst, const I *src, int64_t count, I add, int nonneg_only) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    const I v = src[q];
    dst[q] = (nonneg_only && v < 0) ? v : v + add;
  }
}
template <typename I>
void launch_offset_copy(I *dst, const I *src, int64_t count, I add, bool nonneg_only, cudaStream_t s) {
  if (count <= 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 16);
  k_offset_copy<I><<<grid, 256, 0, s>>>(dst, src, count, add, nonneg_only ? 1 : 0);
}
template void launch_offset_copy<int32_t>(int32_t *, const int32_t *, int64_t, int32_t, bool, cudaStream_t);
template void launch_offset_copy<int64_t>(int64_t *, const int64_t *, int64_t, int64_t, bool, cudaStream_t);

#define EH_INSTANTIATE_T(DIM, T)                                                                                     \
  template void launch_prep<DIM, T>(const MeshView &, const Params &, const double *, const Work &, int, cudaStream_t); \
  template void launch_visc<DIM, T>(const MeshView &, const Params &, const Work &, int, cudaStream_t);               \
  template void launch_alpha<DIM, T>(const MeshView &, const Params &, const Work &, int, cudaStream_t);              \
  template void launch_low<DIM, T>(const MeshView &, const Params &, const Work &, int, cudaStream_t);                \
  template void launch_lim1<DIM, T>(const MeshView &, const Params &, const Work &, double *, int, int, cudaStream_t);

EH_INSTANTIATE_T(2, double)
EH_INSTANTIATE_T(3, double)
EH_INSTANTIATE_T(2, float)
EH_INSTANTIATE_T(3, float)

#define EH_INSTANTIATE(DIM)                                                                                          \
  template void launch_pass<DIM>(const MeshView &, const Params &, const Work &, const double *, double *,            \
                                 const double *, double *, double *, int, int, int, cudaStream_t);                    \
  template void launch_ls_deferred<DIM>(const MeshView &, const Params &, const Work &, const double *, int, double *, \
                                        int, cudaStream_t);                                                          \
  template void launch_final<DIM>(const MeshView &, const Params &, const Work &, const double *, const double *,     \
                                  const double *, double, double *, double *, double *, int, int, cudaStream_t);      \
  template void launch_apply_bc<DIM>(const MeshView &, const Params &, double *, cudaStream_t);                       \
  template void launch_count_not_admissible<DIM>(int, const double *, DevStatus *, cudaStream_t);            \
  template void launch_state_stats<DIM>(int, const double *, const double *, double *, double *, cudaStream_t);

EH_INSTANTIATE(2)
EH_INSTANTIATE(3)

}  // namespace eh
