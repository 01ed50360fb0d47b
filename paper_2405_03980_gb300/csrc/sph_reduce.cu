// Deterministic FP64 reductions: the wall torque of each force evaluation
// (angular-momentum budget of the driven vessel) and the conservation
// diagnostics (total mass M = M_s + M_n of Sec. 2.1, momentum, orbital and spin
// angular momentum, energies).  Both state forms are read in FP64.
//
// Each instance's particle range is cut into fixed chunks of kReduceChunk
// particles counted from the instance's first particle; one block reduces one
// chunk in a fixed tree order and a second kernel adds the chunk partials of an
// instance in chunk order.  The result therefore depends only on the
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
  __device__ __forceinline__ void tw(int64_t i, double* v) const {
    const dvec4 p = f.tw[i];
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
    r[2] = P.lo[2] + (double)cz * P.cell[2] + (double)o.z;
  }
  __device__ __forceinline__ void vel(int64_t i, double* v) const {
    const float4 p = b.vel[i];
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
  __device__ __forceinline__ void spin(int64_t i, double* v) const {
    const float4 p = b.spin[i];
    v[0] = p.x;
    v[1] = p.y;
    v[2] = p.z;
  }
  __device__ __forceinline__ double rho(int64_t i, const InstDev& P) const {
    return P.rho0 * (1.0 + (double)f.delta[i]);
  }
  __device__ __forceinline__ void tw(int64_t i, double* v) const {
    const float4 p = f.tw[i];
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
  r.begin = P.p_begin + (c - P.chunk_base) * (int64_t)kReduceChunk;
  r.end = r.begin + kReduceChunk;
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
  for (int64_t i = r.begin + threadIdx.x; i < r.end; i += kRedThreads) {
    if (V.species(i) >= 2) continue;
    double t[3];
    V.tw(i, t);
    v[0] += t[0];
    v[1] += t[1];
    v[2] += t[2];
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

__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  for (int t = 0; t < e; ++t) r *= x;
  return r;
}

// Tait internal energy per unit mass, e(rho) = int_{rho0}^{rho} P(s)/s^2 ds.
__device__ __forceinline__ double tait_energy(const InstDev& P, double rho) {
  const double x = rho * P.inv_rho0;
  double e1;
  if (P.alphaP == 1) e1 = P.p0 * P.inv_rho0 * log(x);
  else e1 = P.p0 / ((double)(P.alphaP - 1) * P.rho0) * (ipow(x, P.alphaP - 1) - 1.0);
  return e1 + P.beta_P * (1.0 / rho - P.inv_rho0);
}

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
  double rmin = INFINITY, rmax = -INFINITY, vmax = 0.0;
  for (int64_t i = r.begin + threadIdx.x; i < r.end; i += kRedThreads) {
    const int sp = V.species(i);
    if (sp >= 2) continue;
    const bool inv = sp == 0;
    const double m = inv ? P.m_s : P.m_n;
    const double I = 1.0 / (inv ? P.inv_I_s : P.inv_I_n);
    double p[3], u[3], w[3];
    V.pos(i, P, p);
    V.vel(i, u);
    V.spin(i, w);
    const double rho = V.rho(i, P);
    // particle counts (exact integers): M_s = m_s N_s and M_n = m_n N_n are
    // formed at the end, so the total mass is conserved bit for bit
    v[0] += 1.0;
    v[1] += inv ? 1.0 : 0.0;
    v[2] += inv ? 0.0 : 1.0;
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
    v[15] += (double)nw.count[i];
    rmin = fmin(rmin, rho);
    rmax = fmax(rmax, rho);
    vmax = fmax(vmax, sqrt(u2));
  }
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

__global__ void k_diag_final(int32_t n_inst, const InstDev* __restrict__ inst,
                             const double* __restrict__ partials, double* __restrict__ out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_inst) return;
  const InstDev& P = inst[k];
  double s[kSumFields];
  for (int a = 0; a < kSumFields; ++a) s[a] = 0.0;
  double rmin = INFINITY, rmax = -INFINITY, vmax = 0.0;
  for (int64_t c = 0; c < P.n_chunks; ++c) {
    const double* q = partials + (P.chunk_base + c) * kDiagFields;
    for (int a = 0; a < kSumFields; ++a) s[a] += q[a];
    rmin = fmin(rmin, q[kSumFields]);
    rmax = fmax(rmax, q[kSumFields + 1]);
    vmax = fmax(vmax, q[kSumFields + 2]);
  }
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
  k_diag_final<<<(n_inst + 127) / 128, 128, 0, s>>>(n_inst, inst, partials, out);
  return cudaGetLastError();
}

}  // namespace

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

}  // namespace sphgb
