// Deterministic FP64 reductions: the wall torque of each force evaluation
// (angular-momentum budget of the driven vessel) and the conservation
// diagnostics (total mass M = M_s + M_n of Sec. 2.1, momentum, orbital and spin
// angular momentum, energies).  Both state forms are read in FP64.
//
// Each instance's particle range is cut into fixed chunks of kStateChunk
// particles counted from the instance's first particle (small enough that
// the chunks of a 20M-particle state fill the GPU in several even waves);
// one block reduces one chunk in a fixed tree order and a second kernel adds
// the chunk partials of an instance in a fixed order.  The result therefore depends only on the
// instance's own sorted particles, not on launch shapes or on the other
// instances of a batch.
#include <math.h>

#include "sph_kernels.h"

namespace sphgb {
namespace {

constexpr int kRedThreads = 256;

// Read-only FP64 views of the two state forms.
struct Fp64View {
  Fp64Buf b;
  Fp64Fields f;
  __device__ __forceinline__ int species(int64_t i) const { return (int)b.pos[i].w; }
  __device__ __forceinline__ void pos(int64_t i, const InstDev&, double* r) const {
    const dvec4 p = b.pos[i];
    r[0] = p.x;
    r[1] = p.y;
    r[2] = p.z;
  }
  __device__ __forceinline__ void vel(int64_t i, double* v) const {
    const dvec4 p = b.vel[i];
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
  __device__ __forceinline__ void spin(int64_t i, double* v) const {
    const dvec4 p = b.spin[i];
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
  __device__ __forceinline__ double rho(int64_t i, const InstDev&) const { return f.rho[i]; }
  // 1 / rho from the stored volume V = m / rho (one multiply, no division)
  __device__ __forceinline__ double inv_rho(int64_t i, double, double inv_m) const {
    return b.vel[i].w * inv_m;
  }
  __device__ __forceinline__ double pres(int64_t i) const { return f.P[i]; }
  // The wall torque record of particle i, whether it is not zero (it is zero
  // for every particle without a wall neighbour, walls included; the test
  // looks at the bits, so that no FP64 instruction is spent on the zeros),
  // and its value.
  typedef dvec4 TwRec;
  __device__ __forceinline__ TwRec tw(int64_t i) const { return f.tw[i]; }
  __device__ __forceinline__ static bool tw_nonzero(const TwRec& p) {
    const unsigned long long any = ((unsigned long long)__double_as_longlong(p.x) |
                                    (unsigned long long)__double_as_longlong(p.y) |
                                    (unsigned long long)__double_as_longlong(p.z)) << 1;
    return any != 0ull;  // not +0 or -0 in every component
  }
  __device__ __forceinline__ static void tw_value(const TwRec& p, double* v) {
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
};

struct MixView {
  MixBuf b;
  MixFields f;
  __device__ __forceinline__ int species(int64_t i) const { return (int)b.off[i].w; }
  __device__ __forceinline__ void pos(int64_t i, const InstDev& P, double* r) const {
    const uint32_t c = b.cell[i];
    const float4 o = b.off[i];
    const int cx = (int)(c & ((1u << kCellBitsX) - 1));
    const int cy = (int)((c >> kCellBitsX) & ((1u << kCellBitsY) - 1));
    const int cz = (int)(c >> (kCellBitsX + kCellBitsY));
    r[0] = P.lo[0] + (double)cx * P.cell[0] + (double)o.x;
    r[1] = P.lo[1] + (double)cy * P.cell[1] + (double)o.y;
    r[2] = fold_z(P, P.lo[2] + (double)cz * P.cell[2] + (double)o.z);
  }
  __device__ __forceinline__ void vel(int64_t i, double* v) const {
    const float4 p = b.vel(i);
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
  __device__ __forceinline__ void spin(int64_t i, double* v) const {
    const float4 p = b.spin(i);
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
  __device__ __forceinline__ double rho(int64_t i, const InstDev& P) const {
    return P.rho0 * (1.0 + (double)f.delta[i]);
  }
  // the stored FP32 volume is too coarse for 1/rho - 1/rho0: divide in FP64
  __device__ __forceinline__ double inv_rho(int64_t, double rho, double) const {
    return 1.0 / rho;
  }
  __device__ __forceinline__ double pres(int64_t i) const { return (double)f.P[i]; }
  // The wall torque record of particle i (see Fp64View).
  typedef float4 TwRec;
  __device__ __forceinline__ TwRec tw(int64_t i) const { return f.tw[i]; }
  __device__ __forceinline__ static bool tw_nonzero(const TwRec& p) {
    return ((__float_as_uint(p.x) | __float_as_uint(p.y) | __float_as_uint(p.z)) << 1) != 0u;
  }
  __device__ __forceinline__ static void tw_value(const TwRec& p, double* v) {
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
};

struct ChunkRange {
  int64_t begin, end;
  int32_t inst;
};

__device__ __forceinline__ ChunkRange chunk_range(const InstDev* inst, int32_t n_inst,
                                                  int64_t c) {
  // instances are few; a linear scan keeps this simple and exact
  int32_t k = 0;
  while (k + 1 < n_inst && inst[k + 1].chunk_base <= c) ++k;
  const InstDev& P = inst[k];
  ChunkRange r;
  r.inst = k;
  r.begin = P.p_begin + (c - P.chunk_base) * (int64_t)kStateChunk;
  r.end = r.begin + kStateChunk;
  if (r.end > P.p_end) r.end = P.p_end;
  return r;
}

// Fixed-order tree sum of NV doubles per thread across the block.
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

template <class View>
__global__ void __launch_bounds__(kRedThreads)
k_wall_torque_chunks(int32_t n_inst, const InstDev* __restrict__ inst, View V,
                     double* __restrict__ partials) {
  __shared__ double sh[3 * kRedThreads];
  const ChunkRange r = chunk_range(inst, n_inst, blockIdx.x);
  double v[3] = {0.0, 0.0, 0.0};
  // walls carry a zero wall torque, as does every particle without a wall
  // neighbour: only the others are added (adding a zero changes no sum).
  // Four records per round are all loaded (an index past the chunk reads
  // its first record and is not added) before any is tested, then added in
  // the same order as one at a time.
  for (int64_t i0 = r.begin + threadIdx.x; i0 < r.end; i0 += 4 * kRedThreads) {
    typename View::TwRec rec[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + (int64_t)u * kRedThreads;
      rec[u] = V.tw(i < r.end ? i : r.begin);
    }
    // the tests on the integer pipe give a mask of the records to add; the
    // conversions and FP64 adds run for those only (a few in a hundred)
    uint32_t nz = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + (int64_t)u * kRedThreads;
      if (i < r.end && View::tw_nonzero(rec[u])) nz |= 1u << u;
    }
    while (nz != 0u) {
      const int u = __ffs(nz) - 1;
      nz &= nz - 1u;
      const typename View::TwRec p = u == 0 ? rec[0] : (u == 1 ? rec[1] : (u == 2 ? rec[2] : rec[3]));
      double t[3];
      View::tw_value(p, t);
      v[0] += t[0];
      v[1] += t[1];
      v[2] += t[2];
    }
  }
  block_sum<3>(v, sh);
  if (threadIdx.x < 3)
    partials[(int64_t)blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x * kRedThreads];
}

// One warp per instance: lane l adds chunks l, l + 32, ... in order, then a
// fixed butterfly combines the lanes (deterministic, independent of batching).
__global__ void k_wall_torque_final(int32_t n_inst, const InstDev* __restrict__ inst,
                                    InstState* __restrict__ ist,
                                    const double* __restrict__ partials, int advance) {
  const int32_t k = blockIdx.x;
  if (k >= n_inst) return;
  const int lane = threadIdx.x;
  const InstDev& P = inst[k];
  double T[3] = {0.0, 0.0, 0.0};
  for (int64_t c = lane; c < P.n_chunks; c += 32)
    for (int a = 0; a < 3; ++a) T[a] += partials[(P.chunk_base + c) * 3 + a];
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 3; ++a) T[a] += __shfl_xor_sync(0xffffffffu, T[a], o);
  if (lane != 0) return;
  InstState s = ist[k];
  if (advance) {
    for (int a = 0; a < 3; ++a) s.J_wall[a] += P.hdt * (s.T_wall[a] + T[a]);
    s.theta = __dadd_rn(s.theta, __dmul_rn(P.Omega, P.dt));
    s.step += 1;
  }
  for (int a = 0; a < 3; ++a) s.T_wall[a] = T[a];
  ist[k] = s;
}

// x^e for an integer e >= 0 by repeated squaring (three multiplies for the
// e = 6 of the alpha_P = 7 Tait law).
__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  for (; e > 0; e >>= 1) {
    if (e & 1) r *= x;
    x *= x;
  }
  return r;
}

// Tait internal energy per unit mass, e(rho) = int_{rho0}^{rho} P(s)/s^2 ds,
// from rho and 1/rho; ecoef = p0 / ((alpha_P - 1) rho0).
__device__ __forceinline__ double tait_energy(const InstDev& P, double rho, double inv_rho,
                                             double ecoef) {
  const double x = rho * P.inv_rho0;
  double e1;
  if (P.alphaP == 1) e1 = P.p0 * P.inv_rho0 * log(x);
  else e1 = ecoef * (ipow(x, P.alphaP - 1) - 1.0);
  return e1 + P.beta_P * (inv_rho - P.inv_rho0);
}

// The bits of a double >= 0 order like its value: min/max of densities and
// squared speeds on the integer pipe.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// Fields: 0 M, 1 M_s, 2 M_n, 3-5 momentum, 6-8 L_orb, 9-11 L_spin, 12 E_kin,
// 13 E_rot, 14 E_int, 15 n_pairs; 16 rho_min, 17 rho_max, 18 v_max.
constexpr int kSumFields = 16;

template <class View>
__global__ void __launch_bounds__(kRedThreads)
k_diag_chunks(int32_t n_inst, const InstDev* __restrict__ inst, View V, NbrWs nw,
              double* __restrict__ partials) {
  __shared__ double sh[kSumFields * kRedThreads];
  __shared__ double mx[3][kRedThreads];
  const ChunkRange r = chunk_range(inst, n_inst, blockIdx.x);
  const InstDev& P = inst[r.inst];
  double v[kSumFields];
#pragma unroll
  for (int a = 0; a < kSumFields; ++a) v[a] = 0.0;
  // the extrema as bits (all values >= 0), the counts as integers: both on
  // the integer pipe, leaving the FP64 pipe to the sums
  long long rmin_b = dbits(INFINITY), rmax_b = 0, vmax2_b = 0;
  uint32_t n_all = 0, n_s = 0;
  uint64_t pairs = 0;
  // per-species constants: mass, 1/mass, spin inertia; Tait energy factor
  const double I_s = 1.0 / P.inv_I_s, I_n = 1.0 / P.inv_I_n;
  const double inv_ms = 1.0 / P.m_s, inv_mn = 1.0 / P.m_n;
  const double ecoef = P.alphaP > 1 ? P.p0 / ((double)(P.alphaP - 1) * P.rho0) : 0.0;
  for (int64_t i = r.begin + threadIdx.x; i < r.end; i += kRedThreads) {
    const int sp = V.species(i);
    if (sp >= 2) continue;
    const bool inv = sp == 0;
    const double m = inv ? P.m_s : P.m_n;
    const double I = inv ? I_s : I_n;
    double p[3], u[3], w[3];
    V.pos(i, P, p);
    V.vel(i, u);
    V.spin(i, w);
    const double rho = V.rho(i, P);
    const double inv_rho = V.inv_rho(i, rho, inv ? inv_ms : inv_mn);
    // particle counts (exact integers): M_s = m_s N_s and M_n = m_n N_n are
    // formed at the end, so the total mass is conserved bit for bit
    ++n_all;
    n_s += inv ? 1u : 0u;
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
    v[14] += m * tait_energy(P, rho, inv_rho, ecoef);
    pairs += nw.count[i];
    const long long rb = dbits(rho), ub = dbits(u2);
    rmin_b = rb < rmin_b ? rb : rmin_b;
    rmax_b = rb > rmax_b ? rb : rmax_b;
    vmax2_b = ub > vmax2_b ? ub : vmax2_b;  // the square root of the largest, once
  }
  v[0] = (double)n_all;
  v[1] = (double)n_s;
  v[2] = (double)(n_all - n_s);
  v[15] = (double)pairs;
  const double rmin = n_all ? __longlong_as_double(rmin_b) : INFINITY;
  const double rmax = n_all ? __longlong_as_double(rmax_b) : -INFINITY;
  const double vmax = sqrt(__longlong_as_double(vmax2_b));
  block_sum<kSumFields>(v, sh);
  const int t = threadIdx.x;
  mx[0][t] = rmin;
  mx[1][t] = rmax;
  mx[2][t] = vmax;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (t < s) {
      mx[0][t] = fmin(mx[0][t], mx[0][t + s]);
      mx[1][t] = fmax(mx[1][t], mx[1][t + s]);
      mx[2][t] = fmax(mx[2][t], mx[2][t + s]);
    }
    __syncthreads();
  }
  double* out = partials + (int64_t)blockIdx.x * kDiagFields;
  if (t < kSumFields) out[t] = sh[t * kRedThreads];
  if (t < 3) out[kSumFields + t] = mx[t][0];
}

// One warp per instance: lane l adds chunks l, l + 32, ... in order, then a
// fixed butterfly combines the lanes (as for the wall torque).
__global__ void k_diag_final(int32_t n_inst, const InstDev* __restrict__ inst,
                             const double* __restrict__ partials, double* __restrict__ out) {
  const int32_t k = blockIdx.x;
  if (k >= n_inst) return;
  const int lane = threadIdx.x;
  const InstDev& P = inst[k];
  double s[kSumFields];
  for (int a = 0; a < kSumFields; ++a) s[a] = 0.0;
  double rmin = INFINITY, rmax = -INFINITY, vmax = 0.0;
  for (int64_t c = lane; c < P.n_chunks; c += 32) {
    const double* q = partials + (P.chunk_base + c) * kDiagFields;
    for (int a = 0; a < kSumFields; ++a) s[a] += q[a];
    rmin = fmin(rmin, q[kSumFields]);
    rmax = fmax(rmax, q[kSumFields + 1]);
    vmax = fmax(vmax, q[kSumFields + 2]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int a = 0; a < kSumFields; ++a) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
    rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  if (lane != 0) return;
  double* o = out + (int64_t)k * kDiagFields;
  for (int a = 0; a < kSumFields; ++a) o[a] = s[a];
  o[1] = P.m_s * s[1];
  o[2] = P.m_n * s[2];
  o[0] = o[1] + o[2];
  o[kSumFields] = rmin;
  o[kSumFields + 1] = rmax;
  o[kSumFields + 2] = vmax;
}

template <class View>
cudaError_t wall_torque(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                        InstState* ist, const View& V, double* partials, int advance,
                        cudaStream_t s, int* launches) {
  k_wall_torque_chunks<View><<<(unsigned)total_chunks, kRedThreads, 0, s>>>(n_inst, inst, V,
                                                                            partials);
  k_wall_torque_final<<<n_inst, 32, 0, s>>>(n_inst, inst, ist, partials, advance);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

template <class View>
cudaError_t diag(int32_t n_inst, int64_t total_chunks, const InstDev* inst, const View& V,
                 const NbrWs& nw, double* partials, double* out, cudaStream_t s) {
  k_diag_chunks<View><<<(unsigned)total_chunks, kRedThreads, 0, s>>>(n_inst, inst, V, nw,
                                                                     partials);
  k_diag_final<<<n_inst, 32, 0, s>>>(n_inst, inst, partials, out);
  return cudaGetLastError();
}

// Per-term force magnitudes (the force breakdown the paper reports for its
// runs, Sec. 4): for every fluid particle i the five pair terms (pressure
// M3, interfacial M4, shear M5, rotational M6, local interaction M7) are
// summed separately over i's neighbour list, in FP64 from the state as
// stored, and sum_i |f_i^term| is accumulated per term.
template <class View>
__global__ void __launch_bounds__(kRedThreads)
k_breakdown_chunks(int32_t n_inst, int64_t n, const InstDev* __restrict__ inst, View V,
                   NbrWs nw, double* __restrict__ partials) {
  __shared__ double sh[5 * kRedThreads];
  const ChunkRange r = chunk_range(inst, n_inst, blockIdx.x);
  const InstDev& P = inst[r.inst];
  const uint32_t fl = P.flags;
  double mag[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = r.begin + threadIdx.x; i < r.end; i += kRedThreads) {
    const int sp_i = V.species(i);
    if (sp_i >= 2) continue;
    const bool inv_i = sp_i == 0;
    double pi[3], vi[3], wi[3];
    V.pos(i, P, pi);
    V.vel(i, vi);
    V.spin(i, wi);
    const double rho_i = V.rho(i, P);
    const double m_i = inv_i ? P.m_s : P.m_n;
    const double Vi = m_i / rho_i, Pri = V.pres(i) / (rho_i * rho_i);
    double fs[5][3];
#pragma unroll
    for (int q = 0; q < 5; ++q) fs[q][0] = fs[q][1] = fs[q][2] = 0.0;
    // list lengths and entries clamped to their ranges (a diagnostic pass:
    // a corrupt list gives wrong magnitudes, never an out-of-range access)
    const uint32_t cnt = min(nw.count[i], (uint32_t)nw.cap);
    for (uint32_t t = 0; t < cnt; ++t) {
      uint32_t j = nw.list[nbr_slot(n, i, t)] & kNbrIndexMask;
      if ((int64_t)j >= n) j = 0;
      double pj[3], vj[3], wj[3];
      V.pos(j, P, pj);
      V.vel(j, vj);
      V.spin(j, wj);
      double d[3] = {pi[0] - pj[0], pi[1] - pj[1], pi[2] - pj[2]};
      if (P.periodic_z) {
        if (d[2] > P.half_Hz) d[2] -= P.Hz;
        else if (d[2] < -P.half_Hz) d[2] += P.Hz;
      }
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 > 0.0)) continue;
      const double rr = sqrt(r2);
      const double e[3] = {d[0] / rr, d[1] / rr, d[2] / rr};
      const double q = rr * P.inv_h, t1 = 1.0 - 0.5 * q, t2 = t1 * t1;
      const double F = P.cF * t2 * t1, W = P.aD * t2 * t2 * (2.0 * q + 1.0);
      const int sp_j = V.species(j);
      const bool inv_j = sp_j == 0;
      const double m_j = inv_j ? P.m_s : P.m_n;
      const double rho_j = V.rho(j, P);
      const double Vj = m_j / rho_j, Prj = V.pres(j) / (rho_j * rho_j);
      const bool chiX = inv_i != inv_j, chiV = !inv_i && !inv_j;
      const double vij[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
      const double ws[3] = {wi[0] + wj[0], wi[1] + wj[1], wi[2] + wj[2]};
      const double u[3] = {vij[0] + 0.5 * (d[1] * ws[2] - d[2] * ws[1]),
                           vij[1] + 0.5 * (d[2] * ws[0] - d[0] * ws[2]),
                           vij[2] + 0.5 * (d[0] * ws[1] - d[1] * ws[0])};
      if (fl & SPH_TERM_P) {  // M3
        const double sP = m_i * m_j * (Pri + Prj) * F;
        for (int a = 0; a < 3; ++a) fs[0][a] += sP * d[a];
      }
      if ((fl & SPH_TERM_T) && chiX) {  // M4, horizontal unless disabled
        const double sT = P.C_T * Vi * Vj * F;
        fs[1][0] += sT * d[0];
        fs[1][1] += sT * d[1];
        if (!(fl & SPH_HPROJ)) fs[1][2] += sT * d[2];
      }
      if ((fl & SPH_TERM_SH) && chiV) {  // M5
        const double ev = e[0] * vij[0] + e[1] * vij[1] + e[2] * vij[2];
        const double sA = -P.A * Vi * Vj * F * ev;
        for (int a = 0; a < 3; ++a) fs[2][a] += sA * e[a];
      }
      if ((fl & SPH_TERM_ROT) && chiV) {  // M6
        const double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        const double sB = -P.B * Vi * Vj * F;
        for (int a = 0; a < 3; ++a) fs[3][a] += sB * (u[a] - eu * e[a]);
      }
      if ((fl & SPH_TERM_SN) && chiX) {  // M7
        const double sN = -P.C_l * Vi * Vj * W;
        const double* w = (fl & SPH_SN_LITERAL) ? vij : u;
        for (int a = 0; a < 3; ++a) fs[4][a] += sN * w[a];
      }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q)
      mag[q] += sqrt(fs[q][0] * fs[q][0] + fs[q][1] * fs[q][1] + fs[q][2] * fs[q][2]);
  }
  block_sum<5>(mag, sh);
  if (threadIdx.x < 5)
    partials[(int64_t)blockIdx.x * kDiagFields + threadIdx.x] = sh[threadIdx.x * kRedThreads];
}

// Per-instance sums of the chunk partials, in chunk order.
__global__ void k_breakdown_final(int32_t n_inst, const InstDev* __restrict__ inst,
                                  const double* __restrict__ partials, double* __restrict__ out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_inst) return;
  const InstDev& P = inst[k];
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t c = 0; c < P.n_chunks; ++c)
    for (int a = 0; a < 5; ++a) s[a] += partials[(P.chunk_base + c) * kDiagFields + a];
  for (int a = 0; a < 5; ++a) out[(int64_t)k * kDiagFields + a] = s[a];
}

template <class View>
cudaError_t breakdown(int32_t n_inst, int64_t n, int64_t total_chunks, const InstDev* inst,
                      const View& V, const NbrWs& nw, double* partials, double* out,
                      cudaStream_t s) {
  k_breakdown_chunks<View><<<(unsigned)total_chunks, kRedThreads, 0, s>>>(n_inst, n, inst, V, nw,
                                                                          partials);
  k_breakdown_final<<<(n_inst + 127) / 128, 128, 0, s>>>(n_inst, inst, partials, out);
  return cudaGetLastError();
}

// Neighbour-pair census: ordered pairs (fluid row i, listed neighbour j) by
// species class, 0 both inviscid, 1 unlike fluid, 2 both viscous, 3 inviscid
// and wall, 4 viscous and wall; exact integer counts carried in doubles, per
// chunk, then per instance in chunk order.
template <class View>
__global__ void __launch_bounds__(kRedThreads)
k_census_chunks(int32_t n_inst, int64_t n, const InstDev* __restrict__ inst, View V, NbrWs nw,
                double* __restrict__ partials) {
  __shared__ double sh[5 * kRedThreads];
  const ChunkRange r = chunk_range(inst, n_inst, blockIdx.x);
  uint32_t c[5] = {0u, 0u, 0u, 0u, 0u};
  for (int64_t i = r.begin + threadIdx.x; i < r.end; i += kRedThreads) {
    const int sp_i = V.species(i);
    if (sp_i >= 2) continue;
    const uint32_t cnt = min(nw.count[i], (uint32_t)nw.cap);
    for (uint32_t t = 0; t < cnt; ++t) {
      uint32_t j = nw.list[nbr_slot(n, i, t)] & kNbrIndexMask;
      if ((int64_t)j >= n) j = 0;
      const int sp_j = V.species(j);
      const int k = sp_j >= 2 ? (sp_i == 0 ? 3 : 4) : (sp_i + sp_j == 0 ? 0 : (sp_i + sp_j == 1 ? 1 : 2));
      c[k] += 1u;
    }
  }
  for (int q = 0; q < 5; ++q) sh[q * kRedThreads + threadIdx.x] = (double)c[q];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 5; ++q) sh[q * kRedThreads + threadIdx.x] += sh[q * kRedThreads + threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5)
    partials[(int64_t)blockIdx.x * kDiagFields + threadIdx.x] = sh[threadIdx.x * kRedThreads];
}

__global__ void k_census_final(int32_t n_inst, const InstDev* __restrict__ inst,
                               const double* __restrict__ partials, double* __restrict__ out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_inst) return;
  const InstDev& P = inst[k];
  double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t ch = 0; ch < P.n_chunks; ++ch)
    for (int q = 0; q < 5; ++q) c[q] += partials[(P.chunk_base + ch) * kDiagFields + q];
  for (int q = 0; q < 5; ++q) out[(int64_t)k * kDiagFields + q] = c[q];
}

template <class View>
cudaError_t census(int32_t n_inst, int64_t n, int64_t total_chunks, const InstDev* inst,
                   const View& V, const NbrWs& nw, double* partials, double* out,
                   cudaStream_t s) {
  k_census_chunks<View><<<(unsigned)total_chunks, kRedThreads, 0, s>>>(n_inst, n, inst, V, nw,
                                                                       partials);
  k_census_final<<<(n_inst + 127) / 128, 128, 0, s>>>(n_inst, inst, partials, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_census_fp64(int32_t n_inst, int64_t n, int64_t total_chunks,
                               const InstDev* inst, const Fp64Buf& b, const Fp64Fields& f,
                               const NbrWs& nw, double* partials, double* out, cudaStream_t s) {
  return census(n_inst, n, total_chunks, inst, Fp64View{b, f}, nw, partials, out, s);
}

cudaError_t launch_census_mixed(int32_t n_inst, int64_t n, int64_t total_chunks,
                                const InstDev* inst, const MixBuf& b, const MixFields& f,
                                const NbrWs& nw, double* partials, double* out, cudaStream_t s) {
  return census(n_inst, n, total_chunks, inst, MixView{b, f}, nw, partials, out, s);
}

cudaError_t launch_wall_torque_fp64(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                                    InstState* ist, const Fp64Buf& b, const Fp64Fields& f,
                                    double* partials, int advance, cudaStream_t s,
                                    int* launches) {
  return wall_torque(n_inst, total_chunks, inst, ist, Fp64View{b, f}, partials, advance, s,
                     launches);
}

cudaError_t launch_wall_torque_mixed(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                                     InstState* ist, const MixBuf& b, const MixFields& f,
                                     double* partials, int advance, cudaStream_t s,
                                     int* launches) {
  return wall_torque(n_inst, total_chunks, inst, ist, MixView{b, f}, partials, advance, s,
                     launches);
}

cudaError_t launch_diag_fp64(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                             const Fp64Buf& b, const Fp64Fields& f, const NbrWs& nw,
                             double* partials, double* out, cudaStream_t s) {
  return diag(n_inst, total_chunks, inst, Fp64View{b, f}, nw, partials, out, s);
}

cudaError_t launch_diag_mixed(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                              const MixBuf& b, const MixFields& f, const NbrWs& nw,
                              double* partials, double* out, cudaStream_t s) {
  return diag(n_inst, total_chunks, inst, MixView{b, f}, nw, partials, out, s);
}

cudaError_t launch_breakdown_fp64(int32_t n_inst, int64_t n, int64_t total_chunks,
                                  const InstDev* inst, const Fp64Buf& b, const Fp64Fields& f,
                                  const NbrWs& nw, double* partials, double* out,
                                  cudaStream_t s) {
  return breakdown(n_inst, n, total_chunks, inst, Fp64View{b, f}, nw, partials, out, s);
}

cudaError_t launch_breakdown_mixed(int32_t n_inst, int64_t n, int64_t total_chunks,
                                   const InstDev* inst, const MixBuf& b, const MixFields& f,
                                   const NbrWs& nw, double* partials, double* out,
                                   cudaStream_t s) {
  return breakdown(n_inst, n, total_chunks, inst, MixView{b, f}, nw, partials, out, s);
}

}  // namespace sphgb
