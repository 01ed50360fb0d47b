// FP64 form of the two-fluid spin-SPH step (every stored field and every
// arithmetic operation in double precision).
//
// Model (Sec. 2.1, Eqs. 1, 2, 4; Algorithm 1; Sec. 3 boundary set-up):
//   density   rho_i = sum_j m_j W_ij (self included), Wendland C2, support 2h,
//             for fluid and inner-wall particles; outer walls keep rho0;
//   pressure  Eq. 4, P = p0 (rho/rho0)^alpha_P - beta_P;
//   pair pass per neighbour j of a fluid particle i, r_ij = r_i - r_j,
//             F = -(1/r) dW/dr, V = m/rho, e = r_ij / r:
//     pressure      m_i m_j (P_i/rho_i^2 + P_j/rho_j^2) F r_ij
//     interfacial   C_T V_i V_j F (x_ij, y_ij, 0)        unlike species only
//     shear         -10 (eta - 0.6 eta_r) V_i V_j F (e.v_ij) e  neither inviscid
//     rotational    -4 eta_r V_i V_j F (I - ee) u_ij,       neither inviscid
//                   u_ij = v_ij + 1/2 r_ij x (w_i + w_j)
//     F_sn          -C_l V_i V_j W u_ij                    unlike species only
//     spin torque   -1/2 r_ij x (rotational + F_sn), I_i dw_i/dt = tau_i;
//   integrator kick-drift-kick velocity Verlet, rigid walls rotating at Omega,
//   periodic z (slip top/bottom).  Walls count as the viscous species.
#include <math.h>

#include <type_traits>

#include "sph_kernels.h"
#include "sph_partition.cuh"

namespace sphgb {
namespace {

__device__ __forceinline__ void latch(uint32_t* err, uint32_t bit) {
  if ((*(volatile uint32_t*)err & bit) == 0u) atomicOr(err, bit);
}

__device__ __forceinline__ bool finite3(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// Cell of a position.  A particle outside the interior cell range (or with a
// non-finite coordinate) is clamped into it and ERR_ESCAPED is latched, so
// every later access stays inside the cell arrays.
__device__ __forceinline__ uint32_t cell_key(const InstDev& P, double x, double y, double z,
                                             uint32_t* err) {
  int c[3];
  const double r[3] = {x, y, z};
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double t = floor((r[a] - P.lo[a]) * P.inv_cell[a]);
    if (a == 2 && P.periodic_z) {
      // z was wrapped into [lo, lo + Hz); rounding may give nz for z just
      // below the top, which belongs to the last cell
      bad |= !(r[a] >= P.lo[a] && r[a] < P.lo[a] + P.Hz);
      c[a] = (t >= 0.0) ? ((t <= (double)(P.nz - 1)) ? (int)t : P.nz - 1) : 0;
    } else if (t >= (double)P.clo[a] && t <= (double)P.chi[a]) {
      c[a] = (int)t;
    } else {
      bad = true;
      c[a] = (t > (double)P.chi[a]) ? P.chi[a] : P.clo[a];  // NaN -> clo
    }
  }
  if (bad) latch(err, ERR_ESCAPED);
  // x-slab of the particle inside its cell
  int slab = (int)floor(((r[0] - P.lo[0]) * P.inv_cell[0] - (double)c[0]) * P.slabs);
  slab = slab < 0 ? 0 : (slab >= P.slabs ? P.slabs - 1 : slab);
  return (uint32_t)(P.cell_base +
                    ((int64_t)c[0] + (int64_t)P.nx * (c[1] + (int64_t)P.ny * c[2])) * P.slabs +
                    slab);
}

inline int grid_for(int64_t n, int threads, int sm_count, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------- integrator

__global__ void k_kick_drift_fp64(int64_t n, Fp64Buf b, Fp64Fields f,
                                  const InstDev* __restrict__ inst,
                                  const InstState* __restrict__ ist, CellWs cw,
                                  uint32_t* err, int mode) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = b.inst[i];
    const InstDev& P = inst[k];
    dvec4 p = b.pos[i];
    dvec4 v = b.vel[i];
    dvec4 w = b.spin[i];
    const int sp = (int)p.w;
    if (sp < 2) {
      if (mode == 1) {
        const dvec4 a = f.acc[i];
        const dvec4 al = f.dspin[i];
        v.x += P.hdt * a.x;
        v.y += P.hdt * a.y;
        v.z += P.hdt * a.z;
        w.x += P.hdt * al.x;
        w.y += P.hdt * al.y;
        w.z += P.hdt * al.z;
        p.x += P.dt * v.x;
        p.y += P.dt * v.y;
        p.z += P.dt * v.z;
        if (P.periodic_z) {
          if (p.z >= P.Hz + P.lo[2]) p.z -= P.Hz;
          else if (p.z < P.lo[2]) p.z += P.Hz;
        }
        b.vel[i] = v;
        b.spin[i] = w;
        b.pos[i] = p;
      }
      if (!finite3(p.x, p.y, p.z) || !finite3(v.x, v.y, v.z) || !finite3(w.x, w.y, w.z))
        latch(err, ERR_NONFINITE);
    } else {
      // rigid vessel: phase theta_n (mode 0) or theta_n + Omega dt (mode 1)
      double th = ist[k].theta;
      if (mode == 1) th = __dadd_rn(th, __dmul_rn(P.Omega, P.dt));
      double s, c;
      sincos(th, &s, &c);
      const dvec2 r0 = b.ref[i];
      p.x = __dsub_rn(__dmul_rn(c, r0.x), __dmul_rn(s, r0.y));
      p.y = __dadd_rn(__dmul_rn(s, r0.x), __dmul_rn(c, r0.y));
      v.x = -P.Omega * p.y;
      v.y = P.Omega * p.x;
      v.z = 0.0;
      w.x = 0.0;
      w.y = 0.0;
      w.z = P.Omega;
      b.pos[i] = p;
      b.vel[i] = v;
      b.spin[i] = w;
    }
    const uint32_t key = cell_key(P, p.x, p.y, p.z, err);
    cw.key[i] = key;
    cw.slot[i] = atomicAdd(&cw.count[key], 1u);
  }
}

__global__ void k_kick_fp64(int64_t n, Fp64Buf b, Fp64Fields f,
                            const InstDev* __restrict__ inst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double spw = b.pos[i].w;
    if (spw >= 2.0) continue;
    const double hdt = inst[b.inst[i]].hdt;
    const dvec4 a = f.acc[i];
    const dvec4 al = f.dspin[i];
    dvec4 v = b.vel[i];
    dvec4 w = b.spin[i];
    v.x += hdt * a.x;
    v.y += hdt * a.y;
    v.z += hdt * a.z;
    w.x += hdt * al.x;
    w.y += hdt * al.y;
    w.z += hdt * al.z;
    b.vel[i] = v;
    b.spin[i] = w;
  }
}

// -------------------------------------------------------------------- reorder

__global__ void k_reorder_fp64(int64_t n, Fp64Buf src, Fp64Buf dst, CellWs cw, NbrWs nw) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = checked_index(cw.perm[k], n, cw.err);
    const dvec4 p = src.pos[j];
    dst.pos[k] = p;
    dst.vel[k] = src.vel[j];
    dst.spin[k] = src.spin[j];
    dst.ref[k] = src.ref[j];
    dst.id[k] = src.id[j];
    dst.inst[k] = src.inst[j];
    cw.skey[k] = cw.key[j];
    nw.posf[k] = make_float4((float)p.x, (float)p.y, (float)p.z, (float)p.w);
  }
}

// Species and wrap tests without FP64 instructions (the FP64 pipe is the
// bottleneck of this form): the species codes 0..3 are stored as doubles, so
// the high word orders them (0.0 -> 0, 1.0 -> 0x3ff00000, 2.0 -> 0x40000000,
// 3.0 -> 0x40080000).
__device__ __forceinline__ bool inviscid(double w) { return __double2hiint(w) == 0; }
__device__ __forceinline__ bool is_wall(double w) { return __double2hiint(w) >= 0x40000000; }
// Species classes and wall-row zeroing of the FP64 state, for the partition.
struct Fp64Species {
  Fp64Buf b;
  Fp64Fields f;
  __device__ __forceinline__ int cls(int64_t i) const {  // 0 inviscid, 1 viscous, 2 wall
    const double w = b.pos[i].w;
    return inviscid(w) ? 0 : (is_wall(w) ? 2 : 1);
  }
  __device__ __forceinline__ void zero(int64_t i) const {
    const dvec4 z = {0.0, 0.0, 0.0, 0.0};
    f.acc[i] = z;
    f.dspin[i] = z;
    f.tw[i] = z;
  }
};

// z period crossed by the pair (i, j): +1 if j's image lies one period above
// i's cell row (i in the bottom row, cell code dz + 1 = 2), -1 if below (i in
// the top row, code 0), else 0.  The code is c_i - c_j + 1 per axis.
__device__ __forceinline__ int z_wrap(uint32_t ent, int cz_i, int nz) {
  const uint32_t cz = ent >> (kNbrIndexBits + 4);
  return (cz_i == 0 && cz == 2u) ? 1 : ((cz_i == nz - 1 && cz == 0u) ? -1 : 0);
}

// ------------------------------------------------- square roots of distances

// sqrt(x) for the pair distances of the density pass, with few FP64
// instructions (the FP64 pipe bounds that pass).  The FP32 hardware
// estimate of 1/sqrt(x) is taken on the top 20 mantissa bits of x;
// operand and estimate move between the formats by integer operations on
// their bits, so no conversion instruction is issued.  One step of the
// third-order iteration y <- y + y e (1/2 + 3e/8), e = 1 - x y^2 (the first
// terms of the binomial series (1 - e)^(-1/2) = 1 / (y sqrt(x))) takes the
// estimate's relative error, below 2^-19, to about (5/16) |e|^3 < 2^-55:
// x times the refined 1/sqrt(x) is within about an ulp of sqrt(x).  An
// argument whose FP32 form would not be normal (zero, tiny, huge) takes
// CUDA's sqrt.
__device__ __forceinline__ bool fp32_range(int hi) {
  return hi >= 0x38100000 && hi < 0x47F00000;  // 2^-126 <= x < 2^128
}
__device__ __forceinline__ double rsqrt_seed_step(double x, int hi) {
  const float xf = __int_as_float((int)(((unsigned)hi - (896u << 20)) << 3));
  const unsigned yb = (unsigned)__float_as_int(rsqrtf(xf));
  const double y = __hiloint2double((int)((yb >> 3) + (896u << 20)), (int)(yb << 29));
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}
__device__ __forceinline__ double sqrt_dist(double x) {
  const int hi = __double2hiint(x);
  return fp32_range(hi) ? x * rsqrt_seed_step(x, hi) : sqrt(x);
}

// -------------------------------------------------------------------- density

__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  for (int t = 0; t < e; ++t) r *= x;
  return r;
}

// Density and Tait pressure (Eq. 4), one thread per particle, from the hit
// bits of the FP32 prefilter of the neighbour search (sph_search.cu): every
// candidate whose bit is set is re-tested exactly in FP64 (no fused
// multiply-add in r^2, strict <); the neighbours are summed and written as
// i's neighbour list for the pair pass, a fluid particle's inviscid
// neighbours first (in candidate order, count_a of them) and then the others
// (in candidate order, from a second walk over the bits set aside for them).
// The walk takes 4 candidates at a time: their table entries, then their
// position records, are loaded together before they are tested.
// kFilter: some instance uses the pressure filter; the kernel shape of every
// list entry is then stored beside the list (nw.wsh_d) for the filter.
template <int BLOCK, bool kFilter>
__global__ void __launch_bounds__(BLOCK)
k_density_fp64(int64_t n, Fp64Buf b, Fp64Fields f, const InstDev* __restrict__ inst, CellWs cw,
               NbrWs nw, uint32_t* err) {
  __shared__ uint32_t smask[BLOCK * kMaxCandWords];
  __shared__ uint32_t stage[BLOCK * kStageWords];
  const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const InstDev& P = inst[b.inst[i]];
  const dvec4 pi = b.pos[i];
  const int sp = (int)pi.w;
  const double m_i = sp == 0 ? P.m_s : P.m_n;
  double rho;
  uint32_t cnt = 0, count_a = kUnsplit;
  if (sp == 3) {
    rho = P.rho0;
  } else {
    const int64_t g = (int64_t)cw.skey[i] / P.slabs;  // grid cell
    const int cz_i = (int)((g - P.cell_base / P.slabs) / ((int64_t)P.nx * P.ny));
    const bool per = P.periodic_z != 0;
    MaskWalk mk(nw, n, i, g, smask + threadIdx.x, BLOCK);
    ListWriter out(nw, n, i, stage + threadIdx.x, BLOCK);
    // fluid rows without the filter: the inviscid neighbours are listed
    // first; the others are set aside as mask bits and listed after them by a
    // second walk (the pair pass then runs one specialised loop per part)
    const bool split = !kFilter && sp < 2;
    MaskKeep keep_b(mk);
    const double half_inv_h = 0.5 * P.inv_h, two_inv_h = 2.0 * P.inv_h;
    const double mD_s = P.m_s * P.aD, mD_n = P.m_n * P.aD;
    const long long cut2_bits = __double_as_longlong(P.cut2);
    rho = m_i * P.aD;  // self term W(0)
    uint32_t e[4], q[4];
    for (uint32_t m; (m = mk.next(e, q)) != 0u;) {
      dvec4 pj[4];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u)
        if (u < m) pj[u] = b.pos[checked_index(e[u] & kNbrIndexMask, n, err)];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        if (u < m) {
          const double dx = __dsub_rn(pi.x, pj[u].x);
          const double dy = __dsub_rn(pi.y, pj[u].y);
          double dz = __dsub_rn(pi.z, pj[u].z);
          if (per) {  // minimum image across the z period
            const int wz = z_wrap(e[u], cz_i, P.nz);
            if (wz > 0) dz = __dadd_rn(dz, P.Hz);
            else if (wz < 0) dz = __dsub_rn(dz, P.Hz);
          }
          const double r2 =
              __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          // r2 < (2h)^2 on the integer pipe: r2 is a sum of squares (+0 or
          // positive, or NaN), and such doubles order as their bit patterns
          const bool keep = __double_as_longlong(r2) < cut2_bits;
          const bool inv_j = inviscid(pj[u].w);
          if (split && keep && !inv_j) keep_b.set(q[u]);
          out.push(e[u], keep && (inv_j || !split));  // index and cell-displacement code
          if (keep) {
            // m_j W(r) = (m_j aD) t^4 (2q + 1), t = 1 - q/2, q = r / h
            const double r = sqrt_dist(r2);
            const double t1 = fma(-half_inv_h, r, 1.0);
            const double t2 = t1 * t1;
            const double mD = inv_j ? mD_s : mD_n;
            const double Wt = t2 * t2 * fma(two_inv_h, r, 1.0);
            rho += mD * Wt;
            if (kFilter) {  // the shape of this list entry, in the list's layout
              const uint32_t t = out.total() - 1u;
              if (t < (uint32_t)nw.cap) nw.wsh_d[nbr_slot(n, i, t)] = Wt;
            }
          }
        }
      }
      if (out.pend >= (uint32_t)kDrainAt) out.drain();
    }
    if (split) {
      count_a = out.total();
      keep_b.finish();  // the set-aside bits now stand in the staged mask words
      MaskWalk mk2 = mk;
      mk2.k = 0;
      mk2.w = mk2.sw[0];
      for (uint32_t m; (m = mk2.next(e)) != 0u;) {
        for (uint32_t u = 0; u < m; ++u) out.push(e[u], true);
        if (out.pend >= (uint32_t)kDrainAt) out.drain();
      }
    }
    cnt = out.finish();
    if (out.overflow()) latch(err, ERR_NEIGHBORS);
  }
  nw.count[i] = cnt;
  nw.count_a[i] = count_a;
  const double Pres = P.p0 * ipow(rho * P.inv_rho0, P.alphaP) - P.beta_P;
  f.rho[i] = rho;
  f.P[i] = Pres;
  const double V = m_i / rho;
  b.vel[i].w = V;
  b.spin[i].w = Pres / (rho * rho);
  if (P.flags & SPH_PFILTER) f.vp[i] = sp == 3 ? dvec2{0.0, 0.0} : dvec2{V, V * Pres};
  if (!isfinite(rho) || !isfinite(Pres)) latch(err, ERR_NONFINITE);
}

// ------------------------------------------------------------ pressure filter

// Pressure filter of Algorithm 1 (its formula is not printed; read as the
// zeroth-order kernel average): P_i <- sum_j V_j P_j W_ij / sum_j V_j W_ij
// over i itself and its neighbour list, for fluid and inner-wall particles of
// the instances that enable it.  The inputs (V, P) come from the density
// pass's separate array, as (V, V P), and the outputs go to f.P and spin.w,
// so rows never read a value another row writes.  W enters through its shape
// t^4 (2q + 1) (the constant aD cancels), which the density pass stored for
// every list entry: the pass streams the list and the shapes and gathers
// (V, V P) only, leaving two FP64 fused multiply-adds per neighbour (the FP64
// pipe, not memory, bounds it).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_pfilter_fp64(int64_t n, Fp64Buf b, Fp64Fields f, const InstDev* __restrict__ inst, NbrWs nw,
               uint32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const InstDev& P = inst[b.inst[i]];
  if (!(P.flags & SPH_PFILTER) || b.pos[i].w == 3.0) return;  // outer walls keep P
  const dvec2 own = f.vp[i];
  double num = own.y, den = own.x;  // self term, W(0) / aD = 1
  const uint32_t cnt = checked_count(nw.count[i], nw.cap, err);
  const uint4* __restrict__ groups = reinterpret_cast<const uint4*>(nw.list);
  const dvec2* __restrict__ shapes = reinterpret_cast<const dvec2*>(nw.wsh_d);
  for (uint32_t t0 = 0; t0 < cnt; t0 += 8) {
    const int64_t g = (int64_t)(t0 >> 3) * n + i;
    const uint4 ga = groups[2 * g], gb = groups[2 * g + 1];
    const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
    const uint32_t m = cnt - t0 < 8u ? cnt - t0 : 8u;
    dvec2 w2[4];
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q)
      if (2 * q < m) w2[q] = shapes[4 * g + q];
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      if (u >= m) break;
      const dvec2 vj = f.vp[checked_index(e[u] & kNbrIndexMask, n, err)];
      const double w = (u & 1) ? w2[u >> 1].y : w2[u >> 1].x;
      num = fma(w, vj.y, num);
      den = fma(w, vj.x, den);
    }
  }
  const double Pf = num / den;
  const double rho = f.rho[i];
  f.P[i] = Pf;
  b.spin[i].w = Pf / (rho * rho);
  if (!isfinite(Pf)) latch(err, ERR_NONFINITE);
}

// ------------------------------------------------------------------ pair pass

// The pair terms a neighbour brings depend on the species of the pair
// (walls count as viscous): two inviscid particles exchange the pressure
// term alone; unlike species the pressure, interfacial and local-interaction
// terms (and the latter's spin torque); two viscous particles the pressure,
// shear and rotational terms and the rotational torque.  The density pass
// lists a fluid particle's inviscid neighbours first (count_a of them), and
// the pair pass runs over the fluid particles in species order (all inviscid
// ones, then all viscous ones), so that each warp walks the two parts of its
// lists with one specialised loop each: kPathII, kPathIX, kPathVV.  kPathAll
// is the unspecialised loop for unsplit lists (the pressure filter's runs).
enum { kPathAll = 0, kPathII = 1, kPathIX = 2, kPathVV = 3 };

// Per-particle constants of the pair pass, with the term switches, V_i and
// the kernel constants folded in.
struct PairCtx {
  dvec4 pi, vi, wi;          // own records: position+species, velocity+V, spin+P/rho^2
  double cP0, cP1;           // pressure coefficient for an inviscid / other j
  double cT0, cT1;           // interfacial, j inviscid / other (zero for like species)
  double cBA1, cB1;          // shear - rotational along r, rotational along u (j other)
  double cN0, cN1;           // local interaction (zero for like species)
  double half_inv_h, two_inv_h;
  double hwx, hwy, hwz;      // half the own spin
  long long col2b;           // collision distance^2 bits (0: off)
  int si, cz_i;
  bool hproj, literal, per;
};

struct PairSums {
  double fx = 0.0, fy = 0.0, fz = 0.0;  // force
  double tx = 0.0, ty = 0.0, tz = 0.0;  // spin torque (times -2)
  double wx = 0.0, wy = 0.0, wz = 0.0;  // torque of the walls on the particle
};

// Entries t_begin .. t_end of particle i's list, one 32-byte group at a time.
template <int kPath, int kOpt>
__device__ __forceinline__ void pair_loop(const PairCtx& C, const InstDev& P, const Fp64Buf& b,
                                          const NbrWs& nw, int64_t n, int64_t i,
                                          uint32_t t_begin, uint32_t t_end, uint32_t* err,
                                          PairSums& S) {
  const uint4* __restrict__ groups = reinterpret_cast<const uint4*>(nw.list);
  const dvec4 pi = C.pi, vi = C.vi, wi = C.wi;
  for (uint32_t t = t_begin; t < t_end;) {
    const uint32_t g0 = t >> 3;
    const int64_t gi = 2 * ((int64_t)g0 * n + i);
    const uint4 ga = groups[gi], gb = groups[gi + 1];
    const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
    const uint32_t u0 = t & 7u;
    const uint32_t u1 = t_end - (g0 << 3) < 8u ? t_end - (g0 << 3) : 8u;
    t = (g0 + 1) << 3;
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      if (u < u0) continue;
      if (u >= u1) break;
      const uint32_t j = checked_index(e[u] & kNbrIndexMask, n, err);
      const dvec4 pj = b.pos[j];
      const double dx = pi.x - pj.x, dy = pi.y - pj.y;
      double dz = pi.z - pj.z;
      if (C.per) {  // minimum image across the z period
        const int wz = z_wrap(e[u], C.cz_i, P.nz);
        if (wz > 0) dz += P.Hz;
        else if (wz < 0) dz -= P.Hz;
      }
      const double r2 = dx * dx + dy * dy + dz * dz;
      // coincident particles (r2 = 0) count for the density only; r2 > 0 is
      // tested on the bits (r2 >= 0 or NaN)
      const long long r2b = __double_as_longlong(r2);
      if (!(r2b > 0 && r2b <= 0x7ff0000000000000LL)) continue;
      const double inv_r = rsqrt(r2);
      const double r = r2 * inv_r;
      const double t1 = fma(-C.half_inv_h, r, 1.0);  // 1 - q/2
      const double t2 = t1 * t1;
      const double F = t2 * t1;                      // F / cF
      if (kPath == kPathII) {
        // two inviscid particles: the pressure term alone (and a collision);
        // j is fluid, so no wall torque
        const double Prj = b.spin[j].w;
        double al = C.cP0 * (wi.w + Prj) * F;
        if (kOpt & kOptCollision) {
          const dvec4 vj = b.vel[j];
          const double dv = dx * (vi.x - vj.x) + dy * (vi.y - vj.y) + dz * (vi.z - vj.z);
          if (r2b < C.col2b && __double2hiint(dv) < 0) al += P.cC[0] * dv * (inv_r * inv_r);
        }
        S.fx = fma(al, dx, S.fx);
        S.fy = fma(al, dy, S.fy);
        S.fz = fma(al, dz, S.fz);
        continue;
      }
      const dvec4 vj = b.vel[j];
      const dvec4 wj = b.spin[j];
      // whether j is viscous (or a wall): fixed by the list part except in
      // the unspecialised loop (unlike species: j is viscous iff i is not)
      const bool vis_j = kPath == kPathVV ? true
                       : kPath == kPathIX ? C.si == 0
                                          : !inviscid(pj.w);
      // relative velocity v_ij and spin-corrected u_ij = v_ij + 1/2 r_ij x (w_i + w_j),
      // with s = (w_i + w_j) / 2
      const double vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
      const double sx = fma(0.5, wj.x, C.hwx), sy = fma(0.5, wj.y, C.hwy),
                   sz = fma(0.5, wj.z, C.hwz);
      const double ux = fma(dy, sz, fma(-dz, sy, vx));
      const double uy = fma(dz, sx, fma(-dx, sz, vy));
      const double uz = fma(dx, sy, fma(-dy, sx, vz));
      // The five pair terms collected along r_ij and u_ij (and v_ij for the
      // literal F_sn): shear -A V_iV_j F (e.v) e = -A V_iV_j F dv/r^2 r_ij,
      // rotational -B V_iV_j F (u - (e.u) e) = -B V_iV_j F u + B V_iV_j F dv/r^2 r_ij
      // (r_ij . u_ij = r_ij . v_ij: the spin part of u_ij is normal to r_ij).
      const double VF = vj.w * F;
      double aP, aT = 0.0, aV = 0.0, bR = 0.0, bN = 0.0, dv = 0.0;
      const bool need_dv = kPath != kPathIX || (kOpt & kOptCollision);
      if (need_dv) dv = dx * vx + dy * vy + dz * vz;  // r_ij . v_ij
      if (kPath == kPathIX) {  // unlike species: pressure, interfacial, F_sn
        const double W = t2 * t2 * fma(C.two_inv_h, r, 1.0);  // W / aD
        aP = (vis_j ? C.cP1 : C.cP0) * (wi.w + wj.w) * F;
        aT = (vis_j ? C.cT1 : C.cT0) * VF;
        bN = (vis_j ? C.cN1 : C.cN0) * vj.w * W;
      } else if (kPath == kPathVV) {  // like viscous species: pressure, shear, rotational
        aP = C.cP1 * (wi.w + wj.w) * F;
        aV = VF * (inv_r * inv_r) * (C.cBA1 * dv);
        bR = C.cB1 * VF;
      } else {  // any pair
        const double W = t2 * t2 * fma(C.two_inv_h, r, 1.0);
        aP = (vis_j ? C.cP1 : C.cP0) * (wi.w + wj.w) * F;
        aT = (vis_j ? C.cT1 : C.cT0) * VF;
        aV = vis_j ? VF * (inv_r * inv_r) * (C.cBA1 * dv) : 0.0;
        bR = vis_j ? C.cB1 * VF : 0.0;
        bN = (vis_j ? C.cN1 : C.cN0) * vj.w * W;
      }
      // (a class loop adds only the terms its class carries: no FP64 addition
      // of a zero term, as the FP64 pipe bounds this loop)
      double base = kPath == kPathIX ? aP : aP + aV;  // the z component drops aT
      // collision of an approaching pair closer than col_dist: the central
      // force m_i dv_i / dt = -(1 + e) mu_ij (r_ij . v_ij) / (r^2 dt) r_ij;
      // both tests on the bits (dv < 0: its sign bit; -0 adds nothing)
      if ((kOpt & kOptCollision) && r2b < C.col2b && __double2hiint(dv) < 0)
        base += P.cC[C.si + (vis_j ? 1 : 0)] * dv * (inv_r * inv_r);
      const double al = kPath == kPathVV ? base : base + aT;
      const double alz = C.hproj ? base : al;
      // coefficient of u_ij
      const double bu = kPath == kPathIX ? (C.literal ? 0.0 : bN)
                      : kPath == kPathVV ? bR
                                         : (C.literal ? bR : bR + bN);
      // The pair force al r_ij + bu u_ij (+ bN v_ij) goes into the sums one
      // fused multiply-add per term, and so does the spin torque
      // -1/2 r_ij x (f_rot + f_sn) = -1/2 bu (r_ij x u_ij), whose factor
      // -1/2 (exact) is applied to the sums: the FP64 pipe bounds this loop.
      const double cx = dy * uz - dz * uy, cy = dz * ux - dx * uz, cz = dx * uy - dy * ux;
      S.fx = fma(al, dx, fma(bu, ux, S.fx));
      S.fy = fma(al, dy, fma(bu, uy, S.fy));
      S.fz = fma(alz, dz, fma(bu, uz, S.fz));
      if ((kOpt & kOptLiteral) && C.literal) {  // coefficient bN of v_ij
        S.fx = fma(bN, vx, S.fx);
        S.fy = fma(bN, vy, S.fy);
        S.fz = fma(bN, vz, S.fz);
      }
      S.tx = fma(bu, cx, S.tx);
      S.ty = fma(bu, cy, S.ty);
      S.tz = fma(bu, cz, S.tz);
      if (is_wall(pj.w)) {  // torque exerted by the wall on particle i
        double pfx = al * dx + bu * ux;
        double pfy = al * dy + bu * uy;
        double pfz = alz * dz + bu * uz;
        if ((kOpt & kOptLiteral) && C.literal) {
          pfx += bN * vx;
          pfy += bN * vy;
          pfz += bN * vz;
        }
        S.wx += fma(-0.5, bu * cx, pi.y * pfz - pi.z * pfy);
        S.wy += fma(-0.5, bu * cy, pi.z * pfx - pi.x * pfz);
        S.wz += fma(-0.5, bu * cz, pi.x * pfy - pi.y * pfx);
      }
    }
  }
}

// kOpt: kOptLiteral if some instance uses the literal F_sn (coefficient of
// v_ij), kOptCollision if some instance uses the collision model; the
// default form (0) has neither and drops both at compile time.  Thread t
// takes the fluid particle order[t]: t < n_inv are the inviscid ones, and
// the threads from the fluid count on (the grid covers all n) return.
template <int BLOCK, int kOpt>
__global__ void __launch_bounds__(BLOCK, kOpt ? 512 / BLOCK : 0)
k_forces_fp64(int64_t n, Fp64Buf b, Fp64Fields f, const InstDev* __restrict__ inst, CellWs cw,
              NbrWs nw, uint32_t* err, int64_t part_totals) {
  const int64_t t = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (t >= (int64_t)nw.part[part_totals + 1]) return;
  const int64_t n_inv = nw.part[part_totals];
  const int64_t i = checked_index(nw.order[t], n, err);
  PairCtx C;
  C.pi = b.pos[i];
  const int sp_i = (int)C.pi.w;
  const InstDev& P = inst[b.inst[i]];
  C.vi = b.vel[i];   // w = V_i
  C.wi = b.spin[i];  // w = P_i / rho_i^2
  const double m_i = sp_i == 0 ? P.m_s : P.m_n;
  const double inv_I = sp_i == 0 ? P.inv_I_s : P.inv_I_n;
  const uint32_t fl = P.flags;
  const double cP = (fl & SPH_TERM_P) ? m_i : 0.0;
  const double cT = (fl & SPH_TERM_T) ? P.C_T * C.vi.w : 0.0;
  const double cA = (fl & SPH_TERM_SH) ? P.A * C.vi.w : 0.0;
  const double cB = (fl & SPH_TERM_ROT) ? P.B * C.vi.w : 0.0;
  const double cN = (fl & SPH_TERM_SN) ? P.C_l * C.vi.w : 0.0;
  C.literal = (kOpt & kOptLiteral) && (fl & SPH_SN_LITERAL) != 0;
  const bool inv_i = sp_i == 0;
  // collision model: the bits of col_dist^2 (0 when off; r^2 > 0 orders like
  // its bits); its coefficient -(1 + e) mu_ij / dt is read, for the rare
  // colliding pair only, from the table indexed by the species sum, so both
  // sides of a pair read one value
  C.col2b = (kOpt & kOptCollision) ? __double_as_longlong(P.col2) : 0ll;
  C.si = inv_i ? 0 : 1;
  // The species factors of the pair terms depend on j only through whether
  // j is inviscid (suffix 0) or not (suffix 1): mX = 1 for unlike species
  // (interfacial force, F_sn), mV = 1 for two viscous particles (shear,
  // rotational); walls count as viscous.
  const double mX0 = inv_i ? 0.0 : 1.0, mX1 = inv_i ? 1.0 : 0.0;
  const double mV1 = inv_i ? 0.0 : 1.0;
  // The kernel constants cF (in F) and aD (in W) are folded in here, so
  // that the pair loop forms only the shapes t^3 and t^4 (2q + 1).
  C.cP0 = cP * P.m_s * P.cF;
  C.cP1 = cP * P.m_n * P.cF;
  C.cT0 = cT * mX0 * P.cF;
  C.cT1 = cT * mX1 * P.cF;
  C.cBA1 = mV1 != 0.0 ? (cB - cA) * P.cF : 0.0;
  C.cB1 = -cB * mV1 * P.cF;
  C.cN0 = -cN * mX0 * P.aD;
  C.cN1 = -cN * mX1 * P.aD;
  C.hproj = (fl & SPH_HPROJ) != 0;
  C.half_inv_h = 0.5 * P.inv_h;
  C.two_inv_h = 2.0 * P.inv_h;
  C.hwx = 0.5 * C.wi.x;
  C.hwy = 0.5 * C.wi.y;
  C.hwz = 0.5 * C.wi.z;
  const int64_t g = (int64_t)cw.skey[i] / P.slabs;  // grid cell
  C.cz_i = (int)((g - P.cell_base / P.slabs) / ((int64_t)P.nx * P.ny));
  C.per = P.periodic_z != 0;
  PairSums S;
  const uint32_t cnt = checked_count(nw.count[i], nw.cap, err);
  const uint32_t ca = nw.count_a[i];
  if (ca == kUnsplit) {
    pair_loop<kPathAll, kOpt>(C, P, b, nw, n, i, 0u, cnt, err, S);
  } else {
    const uint32_t na = ca < cnt ? ca : cnt;
    // the inviscid neighbours, then the others: the warp's particles are of
    // one species except at the boundary of the two parts of the order
    if (t < n_inv) {
      pair_loop<kPathII, kOpt>(C, P, b, nw, n, i, 0u, na, err, S);
      pair_loop<kPathIX, kOpt>(C, P, b, nw, n, i, na, cnt, err, S);
    } else {
      pair_loop<kPathIX, kOpt>(C, P, b, nw, n, i, 0u, na, err, S);
      pair_loop<kPathVV, kOpt>(C, P, b, nw, n, i, na, cnt, err, S);
    }
  }
  const double inv_m = 1.0 / m_i;
  f.acc[i] = dvec4{S.fx * inv_m, S.fy * inv_m, S.fz * inv_m, 0.0};
  const double tx = -0.5 * S.tx, ty = -0.5 * S.ty, tz = -0.5 * S.tz;
  f.dspin[i] = dvec4{tx * inv_I, ty * inv_I, tz * inv_I, 0.0};
  f.tw[i] = dvec4{S.wx, S.wy, S.wz, 0.0};
  if (!finite3(S.fx, S.fy, S.fz) || !finite3(tx, ty, tz)) latch(err, ERR_NONFINITE);
}

// ----------------------------------------------------------- load / unload

__global__ void k_load_fp64(int64_t n, Fp64Buf b, const double* __restrict__ pos,
                            const double* __restrict__ vel, const double* __restrict__ spin,
                            const uint8_t* __restrict__ sp, const InstDev* __restrict__ inst,
                            int32_t n_inst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double s = (double)sp[i];
    b.pos[i] = dvec4{pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], s};
    b.vel[i] = dvec4{vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.0};
    b.spin[i] = dvec4{spin[3 * i], spin[3 * i + 1], spin[3 * i + 2], 0.0};
    b.ref[i] = dvec2{pos[3 * i], pos[3 * i + 1]};
    b.id[i] = (uint32_t)i;
    b.inst[i] = instance_of(inst, n_inst, i);
  }
}

__global__ void k_unsort_fp64(int64_t n, Fp64Buf b, Fp64Fields f, double* pos, double* vel,
                              double* spin, double* rho, double* P, double* acc,
                              double* dspin) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b.id[k];
    if (pos) {
      const dvec4 p = b.pos[k];
      pos[3 * o] = p.x;
      pos[3 * o + 1] = p.y;
      pos[3 * o + 2] = p.z;
    }
    if (vel) {
      const dvec4 v = b.vel[k];
      vel[3 * o] = v.x;
      vel[3 * o + 1] = v.y;
      vel[3 * o + 2] = v.z;
    }
    if (spin) {
      const dvec4 w = b.spin[k];
      spin[3 * o] = w.x;
      spin[3 * o + 1] = w.y;
      spin[3 * o + 2] = w.z;
    }
    if (rho) rho[o] = f.rho[k];
    if (P) P[o] = f.P[k];
    if (acc) {
      const dvec4 a = f.acc[k];
      acc[3 * o] = a.x;
      acc[3 * o + 1] = a.y;
      acc[3 * o + 2] = a.z;
    }
    if (dspin) {
      const dvec4 a = f.dspin[k];
      dspin[3 * o] = a.x;
      dspin[3 * o + 1] = a.y;
      dspin[3 * o + 2] = a.z;
    }
  }
}

}  // namespace

cudaError_t launch_kick_drift_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                                   const InstDev* inst, const InstState* ist,
                                   const CellWs& cw, uint32_t* err, int mode,
                                   cudaStream_t s, const LaunchCfg& lc, int* launches) {
  k_kick_drift_fp64<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, inst, ist, cw,
                                                                       err, mode);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_reorder_fp64(int64_t n, const Fp64Buf& src, const Fp64Buf& dst,
                                const CellWs& cw, const NbrWs& nw, cudaStream_t s,
                                const LaunchCfg& lc, int* launches) {
  k_reorder_fp64<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, src, dst, cw, nw);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_density_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                                const InstDev* inst, const CellWs& cw, const NbrWs& nw,
                                uint32_t* err, cudaStream_t s, const LaunchCfg& lc,
                                int* launches) {
  const unsigned g32 = (unsigned)((n + 31) / 32), g64 = (unsigned)((n + 63) / 64),
                 g128 = (unsigned)((n + 127) / 128);
  if (lc.any_filter) {
    if (lc.block_density == 32)
      k_density_fp64<32, true><<<g32, 32, 0, s>>>(n, b, f, inst, cw, nw, err);
    else if (lc.block_density == 64)
      k_density_fp64<64, true><<<g64, 64, 0, s>>>(n, b, f, inst, cw, nw, err);
    else
      k_density_fp64<128, true><<<g128, 128, 0, s>>>(n, b, f, inst, cw, nw, err);
  } else {
    if (lc.block_density == 32)
      k_density_fp64<32, false><<<g32, 32, 0, s>>>(n, b, f, inst, cw, nw, err);
    else if (lc.block_density == 64)
      k_density_fp64<64, false><<<g64, 64, 0, s>>>(n, b, f, inst, cw, nw, err);
    else
      k_density_fp64<128, false><<<g128, 128, 0, s>>>(n, b, f, inst, cw, nw, err);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_forces_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                               const InstDev* inst, const CellWs& cw, const NbrWs& nw,
                               uint32_t* err, cudaStream_t s, const LaunchCfg& lc,
                               int* launches) {
  // the species partition of the fluid particles, then the pair pass over it
  const int64_t nt = (n + kPartTile - 1) / kPartTile;
  cudaError_t e = launch_partition(n, Fp64Species{b, f}, nw, s, launches);
  if (e != cudaSuccess) return e;
  const unsigned g256 = (unsigned)((n + 255) / 256), g128 = (unsigned)((n + 127) / 128),
                 g64 = (unsigned)((n + 63) / 64);
  // the pair pass carries only the options some instance uses
  const int opt = (lc.any_literal ? kOptLiteral : 0) | (lc.any_collision ? kOptCollision : 0);
  auto go = [&](auto kopt) {
    constexpr int O = decltype(kopt)::value;
    if (lc.block_forces == 256)
      k_forces_fp64<256, O><<<g256, 256, 0, s>>>(n, b, f, inst, cw, nw, err, 2 * nt);
    else if (lc.block_forces == 64)
      k_forces_fp64<64, O><<<g64, 64, 0, s>>>(n, b, f, inst, cw, nw, err, 2 * nt);
    else
      k_forces_fp64<128, O><<<g128, 128, 0, s>>>(n, b, f, inst, cw, nw, err, 2 * nt);
  };
  if (opt == 0)
    go(std::integral_constant<int, 0>());
  else if (opt == kOptCollision)
    go(std::integral_constant<int, kOptCollision>());
  else  // the literal F_sn, with or without collisions
    go(std::integral_constant<int, kOptLiteral | kOptCollision>());
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_pfilter_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                                const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                cudaStream_t s, int* launches) {
  k_pfilter_fp64<128><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, b, f, inst, nw, err);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_kick_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                             const InstDev* inst, cudaStream_t s, const LaunchCfg& lc,
                             int* launches) {
  k_kick_fp64<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, inst);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_unsort_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                               double* pos, double* vel, double* spin, double* rho,
                               double* P, double* acc, double* dspin, cudaStream_t s,
                               const LaunchCfg& lc) {
  k_unsort_fp64<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, pos, vel, spin, rho,
                                                                   P, acc, dspin);
  return cudaGetLastError();
}

cudaError_t launch_load_fp64(int64_t n, const Fp64Buf& b, const double* pos,
                             const double* vel, const double* spin, const uint8_t* sp,
                             const InstDev* inst, int32_t n_inst, cudaStream_t s,
                             const LaunchCfg& lc) {
  k_load_fp64<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, pos, vel, spin, sp, inst,
                                                                 n_inst);
  return cudaGetLastError();
}

}  // namespace sphgb
