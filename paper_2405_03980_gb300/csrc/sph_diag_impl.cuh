// Per-particle accumulation and block reduction of the FP64 conservation
// diagnostics, shared by every reduction kernel that produces them.
#pragma once
#include <math.h>

#include "sph_internal.h"

namespace sphgb {

constexpr int kRedThreads = 256;
// Fields: 0 N (count), 1 N_s, 2 N_n, 3-5 momentum, 6-8 L_orb, 9-11 L_spin,
// 12 E_kin, 13 E_rot, 14 E_int, 15 n_pairs; 16 rho_min, 17 rho_max, 18 v_max.
// The counts become masses M = m_s N_s + m_n N_n in diag_finish().
constexpr int kSumFields = 16;

__device__ __forceinline__ double diag_ipow(double x, int e) {
  double r = 1.0;
  for (int t = 0; t < e; ++t) r *= x;
  return r;
}

// Tait internal energy per unit mass, e(rho) = int_{rho0}^{rho} P(s)/s^2 ds.
__device__ __forceinline__ double tait_energy(const InstDev& P, double rho) {
  const double x = rho * P.inv_rho0;
  double e1;
  if (P.alphaP == 1) e1 = P.p0 * P.inv_rho0 * log(x);
  else e1 = P.p0 / ((double)(P.alphaP - 1) * P.rho0) * (diag_ipow(x, P.alphaP - 1) - 1.0);
  return e1 + P.beta_P * (1.0 / rho - P.inv_rho0);
}

struct DiagAcc {
  double v[kSumFields];
  double rmin, rmax, vmax;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int a = 0; a < kSumFields; ++a) v[a] = 0.0;
    rmin = INFINITY;
    rmax = -INFINITY;
    vmax = 0.0;
  }
  // One fluid particle: position p, velocity u, spin w, density rho,
  // neighbour count npairs; inviscid selects the species.
  __device__ __forceinline__ void add(const InstDev& P, bool inviscid, const double* p,
                                      const double* u, const double* w, double rho,
                                      double npairs) {
    const double m = inviscid ? P.m_s : P.m_n;
    const double I = 1.0 / (inviscid ? P.inv_I_s : P.inv_I_n);
    v[0] += 1.0;
    v[1] += inviscid ? 1.0 : 0.0;
    v[2] += inviscid ? 0.0 : 1.0;
    v[3] += m * u[0];
    v[4] += m * u[1];
    v[5] += m * u[2];
    v[6] += m * (p[1] * u[2] - p[2] * u[1]);
    v[7] += m * (p[2] * u[0] - p[0] * u[2]);
    v[8] += m * (p[0] * u[1] - p[1] * u[0]);
    v[9] += I * w[0];
    v[10] += I * w[1];
    v[11] += I * w[2];
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    v[12] += 0.5 * m * u2;
    v[13] += 0.5 * I * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    v[14] += m * tait_energy(P, rho);
    v[15] += npairs;
    rmin = fmin(rmin, rho);
    rmax = fmax(rmax, rho);
    vmax = fmax(vmax, sqrt(u2));
  }
};

// Fixed-order tree sum of NV doubles per thread across a kRedThreads block.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  const int t = threadIdx.x;
#pragma unroll
  for (int a = 0; a < NV; ++a) sh[a * kRedThreads + t] = v[a];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (t < s) {
#pragma unroll
      for (int a = 0; a < NV; ++a) sh[a * kRedThreads + t] += sh[a * kRedThreads + t + s];
    }
    __syncthreads();
  }
}

// Reduce the block's accumulators in a fixed order and write one partial of
// kDiagFields doubles (sums, then min rho, max rho, max |v|).
__device__ __forceinline__ void diag_block_write(DiagAcc& acc, double* out) {
  __shared__ double sh[kSumFields * kRedThreads];
  __shared__ double mx[3][kRedThreads];
  block_sum<kSumFields>(acc.v, sh);
  const int t = threadIdx.x;
  mx[0][t] = acc.rmin;
  mx[1][t] = acc.rmax;
  mx[2][t] = acc.vmax;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (t < s) {
      mx[0][t] = fmin(mx[0][t], mx[0][t + s]);
      mx[1][t] = fmax(mx[1][t], mx[1][t + s]);
      mx[2][t] = fmax(mx[2][t], mx[2][t + s]);
    }
    __syncthreads();
  }
  if (t < kSumFields) out[t] = sh[t * kRedThreads];
  if (t < 3) out[kSumFields + t] = mx[t][0];
}

// Add n_chunks partials in chunk order; counts become masses.
__device__ __forceinline__ void diag_finish(const InstDev& P, const double* partials,
                                            int64_t n_chunks, double* o) {
  double s[kSumFields];
  for (int a = 0; a < kSumFields; ++a) s[a] = 0.0;
  double rmin = INFINITY, rmax = -INFINITY, vmax = 0.0;
  for (int64_t c = 0; c < n_chunks; ++c) {
    const double* q = partials + c * kDiagFields;
    for (int a = 0; a < kSumFields; ++a) s[a] += q[a];
    rmin = fmin(rmin, q[kSumFields]);
    rmax = fmax(rmax, q[kSumFields + 1]);
    vmax = fmax(vmax, q[kSumFields + 2]);
  }
  for (int a = 0; a < kSumFields; ++a) o[a] = s[a];
  o[1] = P.m_s * s[1];
  o[2] = P.m_n * s[2];
  o[0] = o[1] + o[2];
  o[kSumFields] = rmin;
  o[kSumFields + 1] = rmax;
  o[kSumFields + 2] = vmax;
}

}  // namespace sphgb
