// Mixed-precision form of the two-fluid spin-SPH step.
//
// Same model as the FP64 form (density summation + Eq. 4 Tait pressure, the
// fused pair pass of Eqs. 1-2 with the spin torque, kick-drift-kick with
// rigid rotating walls, Algorithm 1), stored and computed differently:
//  - a position is an integer cell (the neighbour-grid cell, side >= 2h) plus
//    an FP32 offset inside that cell; pair vectors are formed as
//    (c_i - c_j) L + (o_i - o_j), exactly antisymmetric, with the cell
//    difference folded into {-1, 0, 1} (periodic z included);
//  - velocities, spins, density deviation delta = rho/rho0 - 1, pressure and
//    all pair arithmetic are FP32; the pair terms are written so that
//    f_ji == -f_ij bit for bit, and every per-particle sum is Kahan-compensated;
//  - the Tait pressure is evaluated in binomial form from delta, avoiding the
//    cancellation of (rho/rho0)^alpha - 1;
//  - the wall phase stays FP64, walls are placed in FP64 and then converted;
//    conservation reductions read this state in FP64 (sph_reduce.cu).
#include <math.h>

#include <type_traits>

#include "sph_f32x2.cuh"
#include "sph_kernels.h"

namespace sphgb {
namespace {

__device__ __forceinline__ void latch(uint32_t* err, uint32_t bit) {
  if ((*(volatile uint32_t*)err & bit) == 0u) atomicOr(err, bit);
}

inline int grid_for(int64_t n, int threads, int sm_count, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

__device__ __forceinline__ uint32_t pack_cell(int cx, int cy, int cz) {
  return (uint32_t)cx | ((uint32_t)cy << kCellBitsX) | ((uint32_t)cz << (kCellBitsX + kCellBitsY));
}
__device__ __forceinline__ int cell_x(uint32_t c) { return (int)(c & ((1u << kCellBitsX) - 1)); }
__device__ __forceinline__ int cell_y(uint32_t c) {
  return (int)((c >> kCellBitsX) & ((1u << kCellBitsY) - 1));
}
__device__ __forceinline__ int cell_z(uint32_t c) { return (int)(c >> (kCellBitsX + kCellBitsY)); }

// Kahan-compensated FP32 accumulation.
struct Kahan {
  float s, c;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s - c; }
};

// Double position -> (cell, FP32 offset) on one axis.  Returns false if the
// cell falls outside the interior range (the cell is then clamped).
__device__ __forceinline__ bool to_cell(const InstDev& P, int a, double x, int& c, float& o) {
  const double u = (x - P.lo[a]) * P.inv_cell[a];
  double t = floor(u);
  bool ok = true;
  const int lo = P.clo[a], hi = P.chi[a];
  if (!(t >= (double)lo && t <= (double)hi)) {
    ok = false;
    t = (t > (double)hi) ? (double)hi : (double)lo;  // NaN -> lo
  }
  c = (int)t;
  double r = (x - P.lo[a]) - t * P.cell[a];
  if (!(r >= 0.0)) r = 0.0;
  o = (float)r;
  if (o >= P.cellf[a]) o = nextafterf(P.cellf[a], 0.f);
  return ok;
}

// Keep o in [0, L) by moving whole cells; periodic axes wrap c modulo n.
__device__ __forceinline__ bool normalize(float& o, int& c, float L, int lo, int hi,
                                          bool periodic, int n) {
  for (int k = 0; k < 4; ++k) {
    if (o >= L) {
      o -= L;
      c += 1;
    } else if (o < 0.f) {
      o += L;
      c -= 1;
      if (o >= L) {  // |o| below half an ulp of L: the particle sits on the face
        o = 0.f;
        c += 1;
      }
    } else {
      break;
    }
  }
  bool ok = (o >= 0.f && o < L);
  if (!ok) o = 0.f;
  if (periodic) {
    c = ((c % n) + n) % n;
  } else if (c < lo || c > hi) {
    ok = false;
    c = c < lo ? lo : hi;
  }
  return ok;
}

// Pair vector r_i - r_j = (c_i - c_j) L + (o_i - o_j) from a neighbour-list
// entry (whose top bits carry c_i - c_j + 1 per axis) and the two offsets;
// exactly antisymmetric, and bit-identical to the candidate test that wrote
// the entry.  The unit displacement d of an axis is decoded on the integer
// and FP32 pipes without a table: the float with the bits of 2^23 + (d + 1)
// is exactly 2^23 + d + 1, and subtracting 2^23 + 1 leaves d exactly.
// d L is exact, so the fused multiply-add gives the same bits as the
// candidate test's (c_i - c_j) L + (o_i - o_j).  (A 64-entry table of unit
// displacements in shared memory cost more: its bank-conflicted lookups
// shared the L1 data path with the neighbour gathers.)
__device__ __forceinline__ float unit_disp(uint32_t code, int axis) {
  return __int_as_float(0x4B000000 | ((code >> (2 * axis)) & 3u)) - 8388609.0f;
}

__device__ __forceinline__ void entry_vec(const InstDev& P, uint32_t ent, const float4& oi,
                                          const float4& oj, float& dx, float& dy, float& dz) {
  const uint32_t c = ent >> kNbrIndexBits;
  dx = fmaf(unit_disp(c, 0), P.cellf[0], oi.x - oj.x);
  dy = fmaf(unit_disp(c, 1), P.cellf[1], oi.y - oj.y);
  dz = fmaf(unit_disp(c, 2), P.cellf[2], oi.z - oj.z);
}

// The velocity and spin records of neighbour j: its 32-byte record in one
// 256-bit load through the read-only path (the pair pass does not write the
// state; the record is 32-byte aligned: the state buffer is 256-byte aligned
// and the records are carved from it in multiples of 256 bytes).
__device__ __forceinline__ void load_vs(const MixBuf& b, uint32_t j, float4& v, float4& w) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w), "=f"(w.x), "=f"(w.y), "=f"(w.z), "=f"(w.w)
      : "l"(b.vs + 2 * (int64_t)j));
}

// The same record loaded and stored whole by the kernels that update or move
// it (plain coherent accesses).
__device__ __forceinline__ void ld_vs(const MixBuf& b, int64_t i, float4& v, float4& w) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w), "=f"(w.x), "=f"(w.y), "=f"(w.z),
                 "=f"(w.w)
               : "l"(b.vs + 2 * i)
               : "memory");
}
__device__ __forceinline__ void st_vs(const MixBuf& b, int64_t i, const float4& v,
                                      const float4& w) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               :
               : "l"(b.vs + 2 * i), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "f"(w.x), "f"(w.y),
                 "f"(w.z), "f"(w.w)
               : "memory");
}

__device__ __forceinline__ bool finite3f(float a, float b, float c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// ---------------------------------------------------------------- integrator

// v += dt/2 a, w += dt/2 alpha with explicit rounding: the closing half kick
// of a step, whether run alone (k_kick_mixed) or fused into the next step's
// drift, gives the same bits.
__device__ __forceinline__ void half_kick(float hdt, const float4& a, const float4& al, float4& v,
                                          float4& w) {
  v.x = __fmaf_rn(hdt, a.x, v.x);
  v.y = __fmaf_rn(hdt, a.y, v.y);
  v.z = __fmaf_rn(hdt, a.z, v.z);
  w.x = __fmaf_rn(hdt, al.x, w.x);
  w.y = __fmaf_rn(hdt, al.y, w.y);
  w.z = __fmaf_rn(hdt, al.z, w.z);
}

// A gate word: kernels of the list build run only while it is non-zero
// (null: always).
__device__ __forceinline__ bool gate_closed(const uint32_t* gate) {
  return gate != nullptr && *(const volatile uint32_t*)gate == 0u;
}

// Wall placement at the step's phase: the rigid rotation of the reference
// position, in FP64.
__device__ __forceinline__ void wall_xy(const InstDev& P, const InstState& S, const dvec2& r0,
                                        int mode, double& x, double& y) {
  double th = S.theta;
  if (mode == 1) th = __dadd_rn(th, __dmul_rn(P.Omega, P.dt));
  double s, cs;
  sincos(th, &s, &cs);
  x = __dsub_rn(__dmul_rn(cs, r0.x), __dmul_rn(s, r0.y));
  y = __dadd_rn(__dmul_rn(s, r0.x), __dmul_rn(cs, r0.y));
}

// Half kick and drift (mode 1; mode 2: the previous step's closing half
// kick, then this step's opening one, then the drift, so that a run of steps
// passes over the velocities once per step), or the walls' placement alone
// (mode 0), with every particle's cell held fixed: between list builds the offsets may leave
// [0, L), which keeps the cell-displacement codes of the lists valid.  A
// particle that departed more than half the skin from its build position
// carried along by the vessel's rigid rotation since the build (rotation
// keeps every pair distance), or whose offset left [-L, 2L), marks its
// instance for a rebuild in this step (and opens the step's rebuild gate).
__global__ void k_drift_mixed(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst,
                              InstState* __restrict__ ist, uint32_t* err, int mode) {
  // the vessel's rotation since the build, per instance: formed (FP64 phase
  // difference, then FP32 sine and cosine) once per thread and instance
  uint32_t kr = 0xFFFFFFFFu;
  float sn = 0.f, cs = 1.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = b.inst[i];
    const InstDev& P = inst[k];
    float4 o = b.off[i];
    const int sp = (int)o.w;
    if (sp < 2) {
      if (mode >= 1) {
        float4 v, w;
        ld_vs(b, i, v, w);
        const float4 a = f.acc[i];
        const float4 al = f.dspin[i];
        const int kicks = mode == 2 ? 2 : 1;  // the previous step's closing half kick first
        for (int q = 0; q < kicks; ++q) half_kick(P.hdt_f, a, al, v, w);
        o.x = __fmaf_rn(P.dt_f, v.x, o.x);
        o.y = __fmaf_rn(P.dt_f, v.y, o.y);
        o.z = __fmaf_rn(P.dt_f, v.z, o.z);
        st_vs(b, i, v, w);
        b.off[i] = o;
        if (!finite3f(v.x, v.y, v.z) || !finite3f(w.x, w.y, w.z)) latch(err, ERR_NONFINITE);
      }
    } else {
      double x, y;
      wall_xy(P, ist[k], b.ref[i], mode >= 1 ? 1 : 0, x, y);
      const uint32_t cc = b.cell[i];
      o.x = (float)((x - P.lo[0]) - (double)cell_x(cc) * P.cell[0]);
      o.y = (float)((y - P.lo[1]) - (double)cell_y(cc) * P.cell[1]);
      b.off[i] = o;
      float4 v, w;
      ld_vs(b, i, v, w);
      st_vs(b, i, make_float4((float)(-P.Omega * y), (float)(P.Omega * x), 0.f, v.w),
            make_float4(0.f, 0.f, P.Omega_f, w.w));
    }
    const float4 r = f.oref[i];
    const uint32_t cc = b.cell[i];
    // the cell's corner in FP32 (within about 2e-5 dx: the test's margin is
    // 1e-3 dx)
    const float cx = fmaf((float)cell_x(cc), P.cellf[0], P.lof[0]);
    const float cy = fmaf((float)cell_y(cc), P.cellf[1], P.lof[1]);
    if (k != kr) {
      double th = ist[k].theta;
      if (mode >= 1) th = __dadd_rn(th, __dmul_rn(P.Omega, P.dt));
      sincosf((float)(th - ist[k].theta_ref), &sn, &cs);
      kr = k;
    }
    const float xr = cx + r.x, yr = cy + r.y;
    const float dx = (cx + o.x) - (cs * xr - sn * yr);
    const float dy = (cy + o.y) - (sn * xr + cs * yr);
    const float dz = o.z - r.z;
    const float om = P.skin_omax_f;
    const bool inside = o.x >= -om && o.x <= P.cellf[0] + om && o.y >= -om &&
                        o.y <= P.cellf[1] + om && o.z >= -om && o.z <= P.cellf[2] + om;
    if (!(dx * dx + dy * dy + dz * dz <= P.skin_disp2_f && inside) && ist[k].rebuild == 0) {
      ist[k].rebuild = 1;
      err[kErrRebuild] = 1u;
    }
  }
}

// Sort keys of a list build (the rebuild gate open): particles of the
// instances that rebuild get their offsets back into [0, L) (moving whole
// cells; walls are placed exactly at the step's phase) and the key of their
// new cell; the other instances keep the keys of their last sort, so that
// the sort leaves their order, and with it their lists, unchanged.  Every
// particle takes an arrival slot in its key's count.
__global__ void k_keys_mixed(int64_t n, MixBuf b, const InstDev* __restrict__ inst,
                             const InstState* __restrict__ ist, CellWs cw, uint32_t* err,
                             int mode) {
  if (gate_closed(err + kErrRebuild)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = b.inst[i];
    uint32_t key;
    if (ist[k].rebuild) {
      const InstDev& P = inst[k];
      float4 o = b.off[i];
      const uint32_t cc = b.cell[i];
      int c[3] = {cell_x(cc), cell_y(cc), cell_z(cc)};
      bool ok = true;
      if ((int)o.w < 2) {
        ok &= normalize(o.x, c[0], P.cellf[0], P.clo[0], P.chi[0], false, P.nx);
        ok &= normalize(o.y, c[1], P.cellf[1], P.clo[1], P.chi[1], false, P.ny);
        ok &= normalize(o.z, c[2], P.cellf[2], P.clo[2], P.chi[2], P.periodic_z != 0, P.nz);
      } else {  // a wall keeps its z cell and offset; x, y follow the rotation
        double x, y;
        wall_xy(P, ist[k], b.ref[i], mode, x, y);
        ok &= to_cell(P, 0, x, c[0], o.x);
        ok &= to_cell(P, 1, y, c[1], o.y);
      }
      if (!ok) latch(err, ERR_ESCAPED);
      b.off[i] = o;
      b.cell[i] = pack_cell(c[0], c[1], c[2]);
      int slab = (int)(o.x * ((float)P.slabs / P.cellf[0]));
      slab = slab < 0 ? 0 : (slab >= P.slabs ? P.slabs - 1 : slab);
      key = (uint32_t)(P.cell_base +
                       ((int64_t)c[0] + (int64_t)P.nx * (c[1] + (int64_t)P.ny * c[2])) * P.slabs +
                       slab);
    } else {
      key = cw.skey[i];
    }
    cw.key[i] = key;
    cw.slot[i] = atomicAdd(&cw.count[key], 1u);
  }
}

// Keys of the current order recomputed from the cells and the offsets of the
// last build (after a checkpoint load, whose workspace holds no lists): the
// order is already sorted by them, so the counts, their scan and the sorted
// keys are all a relist needs.
__global__ void k_relist_keys_mixed(int64_t n, MixBuf b, MixFields f,
                                    const InstDev* __restrict__ inst, CellWs cw) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const InstDev& P = inst[b.inst[i]];
    const uint32_t cc = b.cell[i];
    int slab = (int)(f.oref[i].x * ((float)P.slabs / P.cellf[0]));
    slab = slab < 0 ? 0 : (slab >= P.slabs ? P.slabs - 1 : slab);
    const uint32_t key = (uint32_t)(
        P.cell_base +
        ((int64_t)cell_x(cc) + (int64_t)P.nx * (cell_y(cc) + (int64_t)P.ny * cell_z(cc))) *
            P.slabs +
        slab);
    cw.skey[i] = key;
    atomicAdd(&cw.count[key], 1u);
  }
}

// Open the rebuild gate of every instance (initial evaluation, a standalone
// cell build) / close it at the end of a step, counting the builds.
__global__ void k_gate_force(int32_t n_inst, InstState* ist, uint32_t* err) {
  for (int32_t k = threadIdx.x; k < n_inst; k += blockDim.x) ist[k].rebuild = 1;
  if (threadIdx.x == 0) err[kErrRebuild] = 1u;
}
__global__ void k_gate_close(int32_t n_inst, const InstDev* __restrict__ inst, InstState* ist,
                             uint32_t* err, int mode) {
  for (int32_t k = threadIdx.x; k < n_inst; k += blockDim.x)
    if (ist[k].rebuild) {  // the wall phase the new lists were built at
      double th = ist[k].theta;
      if (mode == 1) th = __dadd_rn(th, __dmul_rn(inst[k].Omega, inst[k].dt));
      ist[k].theta_ref = th;
      ist[k].rebuild = 0;
      ist[k].rebuilds += 1;
    }
  if (threadIdx.x == 0) err[kErrRebuild] = 0u;
}

__global__ void k_kick_mixed(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (b.off[i].w >= 2.f) continue;
    const float hdt = inst[b.inst[i]].hdt_f;
    const float4 a = f.acc[i];
    const float4 al = f.dspin[i];
    float4 v, w;
    ld_vs(b, i, v, w);
    half_kick(hdt, a, al, v, w);
    st_vs(b, i, v, w);
  }
}

__global__ void k_reorder_mixed(int64_t n, MixBuf src, MixBuf dst, CellWs cw,
                                const uint32_t* gate) {
  if (gate_closed(gate)) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = checked_index(cw.perm[k], n, cw.err);
    dst.cell[k] = src.cell[j];
    dst.off[k] = src.off[j];
    float4 v, w;
    ld_vs(src, j, v, w);
    st_vs(dst, k, v, w);
    dst.ref[k] = src.ref[j];
    dst.id[k] = src.id[j];
    dst.inst[k] = src.inst[j];
    cw.skey[k] = cw.key[j];
  }
}

// The sorted state back into the main buffer (the step's kernels all read
// one buffer); the instances that rebuilt record their offsets as the
// reference of the new lists.
__global__ void k_copyback_mixed(int64_t n, MixBuf src, MixBuf dst, MixFields f,
                                 const InstState* __restrict__ ist, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float4 o = src.off[k];
    const uint32_t q = src.inst[k];
    dst.cell[k] = src.cell[k];
    dst.off[k] = o;
    float4 v, w;
    ld_vs(src, k, v, w);
    st_vs(dst, k, v, w);
    dst.ref[k] = src.ref[k];
    dst.id[k] = src.id[k];
    dst.inst[k] = q;
    if (ist[q].rebuild) f.oref[k] = o;
  }
}

// The reused candidate list of every particle of the instances that rebuild
// (all instances without a gate): the set bits of its candidate mask, in
// order, as candidate-table entries, 8 per 32-byte group.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_skin_list_mixed(int64_t n, MixBuf b, const InstDev* __restrict__ inst,
                  const InstState* __restrict__ ist, CellWs cw, NbrWs nw, uint32_t* err,
                  int gated) {
  __shared__ uint32_t smask[BLOCK * kMaxCandWords];
  if (gated && gate_closed(err + kErrRebuild)) return;  // no instance rebuilds
  for (int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * BLOCK) {
    const uint32_t k = b.inst[i];
    if (gated && !ist[k].rebuild) continue;
    const InstDev& P = inst[k];
    uint32_t cnt = 0;
    if (b.off[i].w != 3.f) {  // outer-wall particles keep no list
      MaskWalk mk(nw, n, i, (int64_t)cw.skey[i] / P.slabs, smask + threadIdx.x, BLOCK);
      const uint32_t groups = (uint32_t)nw.skin_cap >> 3;
      uint32_t e[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      for (uint32_t m, g = 0; (m = mk.next(e)) != 0u; ++g) {
        if (g < groups) {
          uint4* dst = reinterpret_cast<uint4*>(nw.skin + nbr_slot(n, i, g << 3));
          dst[0] = make_uint4(e[0], e[1], e[2], e[3]);
          dst[1] = make_uint4(e[4], e[5], e[6], e[7]);
        }
        cnt += m;
      }
      if (cnt > (groups << 3)) {
        latch(err, ERR_NEIGHBORS);
        cnt = groups << 3;
      }
    }
    nw.skin_count[i] = cnt;
  }
}

// -------------------------------------------------------------------- density

// The list builder with a float per kept entry (the kernel shape the
// pressure filter reads) staged beside it, with the entries' stride, and
// written group by group to the same slots of wl as full sectors.
struct ShapedListWriter : ListWriter {
  float* wl;
  float* sw;
  __device__ __forceinline__ ShapedListWriter(const NbrWs& nw, int64_t n_, int64_t i_,
                                              uint32_t* st_, float* sw_, uint32_t stride_)
      : ListWriter(nw, n_, i_, st_, stride_), wl(nw.wsh_f), sw(sw_) {}
  __device__ __forceinline__ void push(uint32_t e, float w) {
    st[pend * stride] = e;
    sw[pend * stride] = w;
    ++pend;
  }
  __device__ __forceinline__ void write_group(uint32_t from) {
    if (written < groups) {
      const int64_t slot = nbr_slot(n, i, written << 3);
      const float* r = sw + from * stride;
      float4* dw = reinterpret_cast<float4*>(wl + slot);
      dw[0] = make_float4(r[0], r[stride], r[2 * stride], r[3 * stride]);
      dw[1] = make_float4(r[4 * stride], r[5 * stride], r[6 * stride], r[7 * stride]);
    }
    ListWriter::write_group(from);
  }
  __device__ __forceinline__ void drain() {
    const uint32_t g = pend >> 3;
    for (uint32_t k = 0; k < g; ++k) write_group(k << 3);
    const uint32_t rem = pend & 7u;
    for (uint32_t r = 0; r < rem; ++r) {
      st[r * stride] = st[((g << 3) + r) * stride];
      sw[r * stride] = sw[((g << 3) + r) * stride];
    }
    pend = rem;
  }
  __device__ __forceinline__ uint32_t finish() {
    drain();
    const uint32_t t = total();
    if (pend) write_group(0);
    return t < (groups << 3) ? t : (groups << 3);
  }
};

template <bool kShaped>
__device__ __forceinline__ auto make_writer(const NbrWs& nw, int64_t n, int64_t i, uint32_t* st,
                                            float* sw, uint32_t stride) {
  if constexpr (kShaped) return ShapedListWriter(nw, n, i, st, sw, stride);
  else return ListWriter(nw, n, i, st, stride);
}

// r^2 of a pair vector with an explicit rounding sequence: the same bits as
// the neighbour search's test, so that a list rebuilt every step (skin 0)
// keeps exactly the search's neighbours.
__device__ __forceinline__ float pair_r2f(float dx, float dy, float dz) {
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Density deviation and Tait pressure, one thread per particle, summed over
// the entries of its reused list that lie within 2h now (r^2 < (2h)^2 on the
// current offsets and the entry's cell-displacement code), which are also
// written, in order, as the particle's neighbour list for the pair pass.
// The list is read one 32-byte group of 8 entries at a time, and the 8
// offset records are loaded together before the 8 pairs are tested.
// kFilter: some instance uses the pressure filter; the kernel shape of every
// list entry is then stored beside the list (nw.wsh_f) for the filter, staged
// with the entries and written with them as full sectors (drained at 16
// entries, so that the two stagings take the shared memory of one).
template <int BLOCK, bool kFilter>
__global__ void __launch_bounds__(BLOCK)
k_density_mixed(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst, NbrWs nw,
                uint32_t* err) {
  constexpr int kDrain = kFilter ? 16 : kDrainAt;
  constexpr int kWords = kFilter ? 24 : kStageWords;
  static_assert(kWords >= kDrain - 1 + 8, "staging holds a drain's remainder and a batch");
  __shared__ uint32_t stage[BLOCK * kWords];
  __shared__ float wstage[kFilter ? BLOCK * kWords : 1];
  const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const InstDev& P = inst[b.inst[i]];
  const float4 oi = b.off[i];
  const int sp = (int)oi.w;
  const int si = sp == 0 ? 0 : 1;
  float delta;
  uint32_t cnt = 0;
  if (sp == 3) {
    delta = 0.f;
  } else {
    // delta = sum_j (m_j/rho0) W_ij + (m_i/rho0) W(0) - 1, Kahan-compensated,
    // starting from the self term minus one carried as a float pair
    Kahan acc{P.self_hi[si], -P.self_lo[si]};
    using Writer = typename std::conditional<kFilter, ShapedListWriter, ListWriter>::type;
    Writer out = make_writer<kFilter>(nw, n, i, stage + threadIdx.x, wstage + threadIdx.x, BLOCK);
    const float half_inv_h = 0.5f * P.inv_h_f, two_inv_h = 2.f * P.inv_h_f;
    const float mrD0 = P.mr_f[0] * P.aD_f, mrD1 = P.mr_f[1] * P.aD_f;
    const float cut2 = P.cut2_f;
    const uint32_t scnt = checked_count(nw.skin_count[i], nw.skin_cap, err);
    const uint4* __restrict__ groups = reinterpret_cast<const uint4*>(nw.skin);
    for (uint32_t t0 = 0; t0 < scnt; t0 += 8) {
      const int64_t g = 2 * ((int64_t)(t0 >> 3) * n + i);
      const uint4 ga = groups[g], gb = groups[g + 1];
      const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
      const uint32_t m = scnt - t0 < 8u ? scnt - t0 : 8u;
      float4 o[8];
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u)
        if (u < m) o[u] = b.off[checked_index(e[u] & kNbrIndexMask, n, err)];
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        if (u < m) {
          float dx, dy, dz;
          entry_vec(P, e[u], oi, o[u], dx, dy, dz);
          const float r2 = pair_r2f(dx, dy, dz);
          const bool keep = r2 < cut2;
          if constexpr (!kFilter) out.push(e[u], keep);
          if (keep) {
            // r = r2 / sqrt(r2) from the approximate reciprocal square root
            const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
            // (m_j / rho0) W(r) = (m_j aD / rho0) t^4 (2q + 1), t = 1 - q/2
            const float t1 = fmaf(-half_inv_h, r, 1.f);
            const float t2 = t1 * t1;
            const float Wt = t2 * t2 * fmaf(two_inv_h, r, 1.f);
            acc.add((o[u].w == 0.f ? mrD0 : mrD1) * Wt);
            if constexpr (kFilter) out.push(e[u], Wt);  // with the shape of this entry
          }
        }
      }
      if (out.pend >= (uint32_t)kDrain) out.drain();
    }
    cnt = out.finish();
    if (out.overflow()) latch(err, ERR_NEIGHBORS);
    delta = acc.value();
  }
  nw.count[i] = cnt;
  // Tait pressure in binomial form: P = p0 sum_k C(a,k) delta^k + (p0 - beta_P)
  float h = P.binom[P.alphaP];
  for (int k = P.alphaP - 1; k >= 1; --k) h = h * delta + P.binom[k];
  const float Pres = P.p0_f * (delta * h) + P.p0mb_f;
  const float rho = P.rho0_f * (1.f + delta);
  f.delta[i] = delta;
  f.P[i] = Pres;
  const float V = P.m_f[si] / rho;
  b.vel(i).w = V;
  b.spin(i).w = Pres / (rho * rho);
  if (P.flags & SPH_PFILTER) f.vp[i] = sp == 3 ? make_float2(0.f, 0.f) : make_float2(V, Pres);
  if (!isfinite(delta) || !isfinite(Pres)) latch(err, ERR_NONFINITE);
}

// ------------------------------------------------------------ pressure filter

// Pressure filter of Algorithm 1 (its formula is not printed; read as the
// zeroth-order kernel average): P_i <- sum_j V_j P_j W_ij / sum_j V_j W_ij
// over i itself and its neighbour list, for fluid and inner-wall particles of
// the instances that enable it.  The inputs (V, P) come from the density
// pass's separate array and the outputs go to f.P and spin.w, so rows never
// read a value another row writes.  W enters through its shape t^4 (2q + 1)
// (the constant aD cancels), which the density pass stored for every list
// entry: the pass streams the list and the shapes and gathers (V, P) only.
// The sums are compensated across groups of 8 neighbours like the pair pass.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_pfilter_mixed(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst, NbrWs nw,
                uint32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const InstDev& P = inst[b.inst[i]];
  if (!(P.flags & SPH_PFILTER) || b.off[i].w == 3.f) return;  // outer walls keep P
  const float2 own = f.vp[i];
  Kahan num{own.x * own.y, 0.f}, den{own.x, 0.f};  // self term, W(0) / aD = 1
  const uint32_t cnt = checked_count(nw.count[i], nw.cap, err);
  const uint4* __restrict__ groups = reinterpret_cast<const uint4*>(nw.list);
  const float4* __restrict__ shapes = reinterpret_cast<const float4*>(nw.wsh_f);
  for (uint32_t t0 = 0; t0 < cnt; t0 += 8) {
    const int64_t g = 2 * ((int64_t)(t0 >> 3) * n + i);
    const uint4 ga = groups[g], gb = groups[g + 1];
    const float4 wa = shapes[g], wb = shapes[g + 1];
    const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
    const float ws[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    const uint32_t m = cnt - t0 < 8u ? cnt - t0 : 8u;
    float2 vj[8];
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u)
      if (u < m) vj[u] = f.vp[checked_index(e[u] & kNbrIndexMask, n, err)];
    float gn = 0.f, gd = 0.f;
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      if (u < m) {
        const float w = vj[u].x * ws[u];
        gn += w * vj[u].y;
        gd += w;
      }
    }
    num.add(gn);
    den.add(gd);
  }
  const float Pf = num.value() / den.value();
  const float rho = P.rho0_f * (1.f + f.delta[i]);
  f.P[i] = Pf;
  b.spin(i).w = Pf / (rho * rho);
  if (!isfinite(Pf)) latch(err, ERR_NONFINITE);
}

// ------------------------------------------------------------------ pair pass

// The pair pass with the optional terms, one neighbour per step.  kOpt:
// kOptLiteral if some instance uses the literal F_sn (coefficient of v_ij),
// kOptCollision if some instance uses the collision model.  (The default
// form, with neither, runs k_forces_mixed_x2 below.)
template <int BLOCK, int kOpt>
__global__ void __launch_bounds__(BLOCK)
k_forces_mixed(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst, NbrWs nw,
               uint32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const float4 oi = b.off[i];
  const int sp_i = (int)oi.w;
  if (sp_i >= 2) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    f.acc[i] = z;
    f.dspin[i] = z;
    f.tw[i] = z;
    return;
  }
  const InstDev& P = inst[b.inst[i]];
  const uint32_t ci = b.cell[i];
  float4 vi, wi;  // w: V_i and P_i / rho_i^2
  load_vs(b, i, vi, wi);
  const int si = sp_i == 0 ? 0 : 1;
  const float m_i = P.m_f[si];
  const uint32_t fl = P.flags;
  const float kP = (fl & SPH_TERM_P) ? 1.f : 0.f;
  const float kT = (fl & SPH_TERM_T) ? P.C_T_f : 0.f;
  const float kA = (fl & SPH_TERM_SH) ? P.A_f : 0.f;
  const float kB = (fl & SPH_TERM_ROT) ? P.B_f : 0.f;
  const float kN = (fl & SPH_TERM_SN) ? P.C_l_f : 0.f;
  const float hz = (fl & SPH_HPROJ) ? 0.f : 1.f;
  const bool lit = (kOpt & kOptLiteral) && (fl & SPH_SN_LITERAL) != 0;
  // collision model: col_dist^2 (0 when off); its coefficient
  // -(1 + e) mu_ij / dt is read, for the rare colliding pair only, from the
  // table indexed by the species sum, so both sides of a pair read one value
  const float col2 = (kOpt & kOptCollision) ? P.col2_f : 0.f;
  const bool inv_i = sp_i == 0;
  // The species factors of the pair terms depend on j only through whether
  // j is inviscid (suffix 0) or not (suffix 1): mX = 1 for unlike species
  // (interfacial force, F_sn), mV = 1 for two viscous particles (shear,
  // rotational); walls count as viscous.
  const float mX0 = inv_i ? 0.f : 1.f;  // j inviscid
  const float mX1 = inv_i ? 1.f : 0.f;  // j viscous or wall
  const float mV1 = inv_i ? 0.f : 1.f;  // (mV = 0 for an inviscid j)
  // The kernel constants cF (in F) and aD (in W) are folded in here, so
  // that the pair loop forms only the shapes t^3 and t^4 (2q + 1).
  const float cF = P.cF_f, aD = P.aD_f;
  const float cP0 = kP * (m_i * P.m_f[0]) * cF, cP1 = kP * (m_i * P.m_f[1]) * cF;
  const float cT0 = kT * mX0 * cF, cT1 = kT * mX1 * cF;
  const float cBA1 = mV1 != 0.f ? (kB - kA) * cF : 0.f;
  const float cB0 = -kB * 0.f, cB1 = -kB * mV1 * cF;
  const float cN0 = -kN * mX0 * aD, cN1 = -kN * mX1 * aD;
  const bool hproj = hz == 0.f;
  const float half_inv_h = 0.5f * P.inv_h_f, two_inv_h = 2.f * P.inv_h_f;
  const float hwx = 0.5f * wi.x, hwy = 0.5f * wi.y, hwz = 0.5f * wi.z;
  // absolute position of i about the rotation axis (wall torque only)
  const double xi = P.lo[0] + (double)cell_x(ci) * P.cell[0] + (double)oi.x;
  const double yi = P.lo[1] + (double)cell_y(ci) * P.cell[1] + (double)oi.y;
  const double zi = fold_z(P, P.lo[2] + (double)cell_z(ci) * P.cell[2] + (double)oi.z);
  const float pxi = (float)xi, pyi = (float)yi, pzi = (float)zi;
  // compensated sums across groups of 8 neighbours, plain FP32 sums inside
  // a group
  Kahan fx{0.f, 0.f}, fy{0.f, 0.f}, fz{0.f, 0.f}, tx{0.f, 0.f}, ty{0.f, 0.f}, tz{0.f, 0.f};
  float gfx = 0.f, gfy = 0.f, gfz = 0.f, gtx = 0.f, gty = 0.f, gtz = 0.f;
  float wx = 0.f, wy = 0.f, wz = 0.f;
  const uint32_t cnt = checked_count(nw.count[i], nw.cap, err);
  // The list is read one group of 8 entries (one 32-byte sector) at a time,
  // the next group while the current one is evaluated; the neighbour record
  // of the next entry is loaded one pair ahead.
  const uint4* __restrict__ groups = reinterpret_cast<const uint4*>(nw.list);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  uint4 ga = make_uint4(0u, 0u, 0u, 0u), gb = ga;
  float4 oj_n = zero4, vj_n = zero4, wj_n = zero4;
  if (cnt > 0) {
    ga = groups[2 * i];
    gb = groups[2 * i + 1];
    const uint32_t j0 = checked_index(ga.x & kNbrIndexMask, n, err);
    oj_n = b.off[j0];
    load_vs(b, j0, vj_n, wj_n);
  }
  for (uint32_t t0 = 0; t0 < cnt; t0 += 8) {
    const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
    if (t0 + 8 < cnt) {
      const int64_t g = 2 * ((int64_t)((t0 >> 3) + 1) * n + i);
      ga = groups[g];
      gb = groups[g + 1];
    }
    const uint32_t m = cnt - t0 < 8u ? cnt - t0 : 8u;
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      if (u >= m) break;
      const uint32_t ent = e[u];
      const float4 oj = oj_n, vj = vj_n, wj = wj_n;
      if (t0 + u + 1 < cnt) {
        const uint32_t jn = checked_index((u < 7 ? e[u + 1] : ga.x) & kNbrIndexMask, n, err);
        oj_n = b.off[jn];
        load_vs(b, jn, vj_n, wj_n);
      }
      float dx, dy, dz;
      entry_vec(P, ent, oi, oj, dx, dy, dz);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 > 0.f)) continue;  // coincident particles: density only
      const float inv_r = rsqrtf(r2);
      const float r = r2 * inv_r;
      const float inv_r2 = inv_r * inv_r;
      const float t1 = fmaf(-half_inv_h, r, 1.f);         // 1 - q/2
      const float t2 = t1 * t1;
      const float F = t2 * t1;                            // F / cF
      const float W = (t2 * t2) * fmaf(two_inv_h, r, 1.f);  // W / aD
      const bool vis_j = oj.w != 0.f;
      // symmetric pair scalars (products taken in an order independent of i, j)
      const float VV = vi.w * vj.w;
      const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
      // half the spin sum, (w_i + w_j) / 2, the same bits from either side
      const float sx = fmaf(0.5f, wj.x, hwx), sy = fmaf(0.5f, wj.y, hwy),
                  sz = fmaf(0.5f, wj.z, hwz);
      const float ux = fmaf(dy, sz, fmaf(-dz, sy, vx));
      const float uy = fmaf(dz, sx, fmaf(-dx, sz, vy));
      const float uz = fmaf(dx, sy, fmaf(-dy, sx, vz));
      const float dv = dx * vx + dy * vy + dz * vz;  // r_ij . v_ij (symmetric)
      // the five terms collected along r_ij, u_ij and (literal F_sn) v_ij:
      // shear -A VV F dv/r^2 r_ij; rotational -B VV F u_ij + B VV F dv/r^2 r_ij
      // (r_ij . u_ij = r_ij . v_ij: the spin part of u_ij is normal to r_ij)
      const float VF = VV * F;
      const float aP = (vis_j ? cP1 : cP0) * ((wi.w + wj.w) * F);
      const float aT = (vis_j ? cT1 : cT0) * VF;
      const float aV = (VF * inv_r2) * ((vis_j ? cBA1 : 0.f) * dv);
      const float bR = (vis_j ? cB1 : cB0) * VF;
      const float bN = (vis_j ? cN1 : cN0) * (VV * W);
      float base = aP + aV;  // the z component drops aT under the projection
      // collision of an approaching pair closer than col_dist: the central
      // force m_i dv_i / dt = -(1 + e) mu_ij (r_ij . v_ij) / (r^2 dt) r_ij
      if ((kOpt & kOptCollision) && r2 < col2 && dv < 0.f)
        base += P.cC_f[si + (vis_j ? 1 : 0)] * (dv * inv_r2);
      const float al = base + aT;
      const float alz = hproj ? base : al;
      const float bu = lit ? bR : bR + bN;
      float pfx = al * dx + bu * ux;
      float pfy = al * dy + bu * uy;
      float pfz = alz * dz + bu * uz;
      if ((kOpt & kOptLiteral) && lit) {
        pfx += bN * vx;
        pfy += bN * vy;
        pfz += bN * vz;
      }
      gfx += pfx;
      gfy += pfy;
      gfz += pfz;
      // spin torque -1/2 r_ij x (f_rot + f_sn) = -1/2 bu (r_ij x u_ij); the
      // factor -1/2 (exact) is applied to the sums
      const float qx = bu * (dy * uz - dz * uy);
      const float qy = bu * (dz * ux - dx * uz);
      const float qz = bu * (dx * uy - dy * ux);
      gtx += qx;
      gty += qy;
      gtz += qz;
      if (oj.w >= 2.f) {
        wx += fmaf(-0.5f, qx, pyi * pfz - pzi * pfy);
        wy += fmaf(-0.5f, qy, pzi * pfx - pxi * pfz);
        wz += fmaf(-0.5f, qz, pxi * pfy - pyi * pfx);
      }
    }
    fx.add(gfx);
    fy.add(gfy);
    fz.add(gfz);
    tx.add(gtx);
    ty.add(gty);
    tz.add(gtz);
    gfx = gfy = gfz = gtx = gty = gtz = 0.f;
  }
  const float inv_m = P.inv_m_f[si], inv_I = P.inv_I_f[si];
  const float ax = fx.value(), ay = fy.value(), az = fz.value();
  const float bx = -0.5f * tx.value(), by = -0.5f * ty.value(), bz = -0.5f * tz.value();
  f.acc[i] = make_float4(ax * inv_m, ay * inv_m, az * inv_m, 0.f);
  f.dspin[i] = make_float4(bx * inv_I, by * inv_I, bz * inv_I, 0.f);
  f.tw[i] = make_float4(wx, wy, wz, 0.f);
  if (!finite3f(ax, ay, az) || !finite3f(bx, by, bz)) latch(err, ERR_NONFINITE);
}

// The pair pass of the default form (neither the literal F_sn nor the
// collision model) with two neighbours of particle i per step, their FP32
// arithmetic in packed pairs (f32x2: one instruction, two independent
// operations each rounded as its scalar form), where the thread-per-pair
// loop above issues one instruction per operation.  Every pair scalar is
// formed in an order independent of (i, j) as there, so f_ji == -f_ij bit
// for bit.  A neighbour slot past the list's end, or a coincident particle
// (r = 0: density only), is evaluated on stand-in values and masked out.
// The packed form wants more registers (140) than the scalar loop; bounding
// them at 128 keeps the scalar loop's 16 warps per SM at the cost of a few
// spilled loop constants (with 12 warps the pass waited on its gathers).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK)
k_forces_mixed_x2(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst, NbrWs nw,
                  uint32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const float4 oi = b.off[i];
  const int sp_i = (int)oi.w;
  if (sp_i >= 2) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    f.acc[i] = z;
    f.dspin[i] = z;
    f.tw[i] = z;
    return;
  }
  const InstDev& P = inst[b.inst[i]];
  const uint32_t ci = b.cell[i];
  float4 vi, wi;  // w: V_i and P_i / rho_i^2
  load_vs(b, i, vi, wi);
  const int si = sp_i == 0 ? 0 : 1;
  const float m_i = P.m_f[si];
  const uint32_t fl = P.flags;
  const float kP = (fl & SPH_TERM_P) ? 1.f : 0.f;
  const float kT = (fl & SPH_TERM_T) ? P.C_T_f : 0.f;
  const float kA = (fl & SPH_TERM_SH) ? P.A_f : 0.f;
  const float kB = (fl & SPH_TERM_ROT) ? P.B_f : 0.f;
  const float kN = (fl & SPH_TERM_SN) ? P.C_l_f : 0.f;
  const bool hproj = (fl & SPH_HPROJ) != 0;
  const bool inv_i = sp_i == 0;
  // species factors and kernel constants as in k_forces_mixed
  const float mX0 = inv_i ? 0.f : 1.f, mX1 = inv_i ? 1.f : 0.f, mV1 = inv_i ? 0.f : 1.f;
  const float cF = P.cF_f, aD = P.aD_f;
  const float cP0 = kP * (m_i * P.m_f[0]) * cF, cP1 = kP * (m_i * P.m_f[1]) * cF;
  const float cT0 = kT * mX0 * cF, cT1 = kT * mX1 * cF;
  const float cBA1 = mV1 != 0.f ? (kB - kA) * cF : 0.f;
  const float cB0 = -kB * 0.f, cB1 = -kB * mV1 * cF;
  const float cN0 = -kN * mX0 * aD, cN1 = -kN * mX1 * aD;
  const double xi = P.lo[0] + (double)cell_x(ci) * P.cell[0] + (double)oi.x;
  const double yi = P.lo[1] + (double)cell_y(ci) * P.cell[1] + (double)oi.y;
  const double zi = fold_z(P, P.lo[2] + (double)cell_z(ci) * P.cell[2] + (double)oi.z);
  const float pxi = (float)xi, pyi = (float)yi, pzi = (float)zi;
  // packed constants; the differences with i's own records are formed as two
  // scalar operations each (the same roundings), which keeps those records
  // out of packed registers and the kernel within its register bound
  const f2 LX = f2_splat(P.cellf[0]), LY = f2_splat(P.cellf[1]), LZ = f2_splat(P.cellf[2]);
  const f2 ONE = f2_splat(1.f), MAGIC = f2_splat(8388609.0f);
  const f2 NHIH = f2_splat(-0.5f * P.inv_h_f), TIH = f2_splat(2.f * P.inv_h_f);
  const float hwx = 0.5f * wi.x, hwy = 0.5f * wi.y, hwz = 0.5f * wi.z;
  Kahan fx{0.f, 0.f}, fy{0.f, 0.f}, fz{0.f, 0.f}, tx{0.f, 0.f}, ty{0.f, 0.f}, tz{0.f, 0.f};
  float wx = 0.f, wy = 0.f, wz = 0.f;
  const uint32_t cnt = checked_count(nw.count[i], nw.cap, err);
  const uint4* __restrict__ groups = reinterpret_cast<const uint4*>(nw.list);
  // records of the next two entries, loaded one step ahead; a slot past the
  // list's end takes the first entry's records
  uint4 ga = make_uint4(0u, 0u, 0u, 0u), gb = ga;
  float4 oa_n, va_n, wa_n, ob_n, vb_n, wb_n;
  auto fetch2 = [&](uint32_t ea, uint32_t eb, bool has_b) {
    const uint32_t ja = checked_index(ea & kNbrIndexMask, n, err);
    const uint32_t jb = has_b ? checked_index(eb & kNbrIndexMask, n, err) : ja;
    oa_n = b.off[ja];
    load_vs(b, ja, va_n, wa_n);
    ob_n = b.off[jb];
    load_vs(b, jb, vb_n, wb_n);
  };
  if (cnt > 0) {
    ga = groups[2 * i];
    gb = groups[2 * i + 1];
    fetch2(ga.x, ga.y, cnt > 1);
  }
  for (uint32_t t0 = 0; t0 < cnt; t0 += 8) {
    const uint32_t e[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
    if (t0 + 8 < cnt) {
      const int64_t gi = 2 * ((int64_t)((t0 >> 3) + 1) * n + i);
      ga = groups[gi];
      gb = groups[gi + 1];
    }
    const uint32_t m = cnt - t0 < 8u ? cnt - t0 : 8u;
    f2 GFX = 0ull, GFY = 0ull, GFZ = 0ull, GTX = 0ull, GTY = 0ull, GTZ = 0ull;
#pragma unroll
    for (uint32_t u = 0; u < 8; u += 2) {
      if (u >= m) break;
      const bool has_b = u + 1 < m;
      const uint32_t ea = e[u], eb = has_b ? e[u + 1] : e[u];
      const float4 oa = oa_n, va = va_n, wa = wa_n, ob = ob_n, vb = vb_n, wb = wb_n;
      if (t0 + u + 2 < cnt) {
        const uint32_t na = u < 6 ? e[u + 2] : ga.x;
        const uint32_t nb = u < 6 ? e[u + 3] : ga.y;
        fetch2(na, nb, t0 + u + 3 < cnt);
      }
      // pair vectors (c_i - c_j) L + (o_i - o_j), the unit displacement of
      // each axis decoded as in entry_vec
      const uint32_t ca = ea >> kNbrIndexBits, cb = eb >> kNbrIndexBits;
      const f2 EX = f2_sub(f2_make(__int_as_float(0x4B000000 | (ca & 3u)),
                                   __int_as_float(0x4B000000 | (cb & 3u))), MAGIC);
      const f2 EY = f2_sub(f2_make(__int_as_float(0x4B000000 | ((ca >> 2) & 3u)),
                                   __int_as_float(0x4B000000 | ((cb >> 2) & 3u))), MAGIC);
      const f2 EZ = f2_sub(f2_make(__int_as_float(0x4B000000 | (ca >> 4)),
                                   __int_as_float(0x4B000000 | (cb >> 4))), MAGIC);
      const f2 dX = f2_fma(EX, LX, f2_make(oi.x - oa.x, oi.x - ob.x));
      const f2 dY = f2_fma(EY, LY, f2_make(oi.y - oa.y, oi.y - ob.y));
      const f2 dZ = f2_fma(EZ, LZ, f2_make(oi.z - oa.z, oi.z - ob.z));
      const f2 R2 = f2_fma(dZ, dZ, f2_fma(dY, dY, f2_mul(dX, dX)));
      float r2a, r2b;
      f2_split(R2, r2a, r2b);
      const bool oka = r2a > 0.f, okb = has_b && r2b > 0.f;
      const float ira = rsqrtf(oka ? r2a : 1.f), irb = rsqrtf(okb ? r2b : 1.f);
      const f2 IR = f2_make(ira, irb);
      const f2 R = f2_mul(f2_make(oka ? r2a : 1.f, okb ? r2b : 1.f), IR);
      const f2 IR2 = f2_mul(IR, IR);
      const f2 T1 = f2_fma(NHIH, R, ONE);  // 1 - q/2
      const f2 Q2 = f2_fma(TIH, R, ONE);
      const f2 T2 = f2_mul(T1, T1);
      const f2 F = f2_mul(T2, T1);
      const f2 W = f2_mul(f2_mul(T2, T2), Q2);
      const bool visa = oa.w != 0.f, visb = ob.w != 0.f;
      const f2 VV = f2_make(vi.w * va.w, vi.w * vb.w);
      const f2 vX = f2_make(vi.x - va.x, vi.x - vb.x);
      const f2 vY = f2_make(vi.y - va.y, vi.y - vb.y);
      const f2 vZ = f2_make(vi.z - va.z, vi.z - vb.z);
      const f2 SX = f2_make(fmaf(0.5f, wa.x, hwx), fmaf(0.5f, wb.x, hwx));
      const f2 SY = f2_make(fmaf(0.5f, wa.y, hwy), fmaf(0.5f, wb.y, hwy));
      const f2 SZ = f2_make(fmaf(0.5f, wa.z, hwz), fmaf(0.5f, wb.z, hwz));
      // u = v_ij + r_ij x s, each component one product added to the other's
      // negative (the sign of -(dz sy) taken from the product, exactly)
      const f2 uX = f2_fma(dY, SZ, f2_sub(vX, f2_mul(dZ, SY)));
      const f2 uY = f2_fma(dZ, SX, f2_sub(vY, f2_mul(dX, SZ)));
      const f2 uZ = f2_fma(dX, SY, f2_sub(vZ, f2_mul(dY, SX)));
      const f2 DV = f2_fma(dZ, vZ, f2_fma(dY, vY, f2_mul(dX, vX)));
      const f2 VF = f2_mul(VV, F);
      const f2 aP = f2_mul(f2_make(visa ? cP1 : cP0, visb ? cP1 : cP0),
                           f2_mul(f2_make(wi.w + wa.w, wi.w + wb.w), F));
      const f2 aT = f2_mul(f2_make(visa ? cT1 : cT0, visb ? cT1 : cT0), VF);
      const f2 aV = f2_mul(f2_mul(VF, IR2),
                           f2_mul(f2_make(visa ? cBA1 : 0.f, visb ? cBA1 : 0.f), DV));
      const f2 bR = f2_mul(f2_make(visa ? cB1 : cB0, visb ? cB1 : cB0), VF);
      const f2 bN = f2_mul(f2_make(visa ? cN1 : cN0, visb ? cN1 : cN0), f2_mul(VV, W));
      const f2 MK = f2_make(oka ? 1.f : 0.f, okb ? 1.f : 0.f);
      const f2 base = f2_add(aP, aV);
      const f2 AL = f2_mul(f2_add(base, aT), MK);
      const f2 ALZ = hproj ? f2_mul(base, MK) : AL;
      const f2 BU = f2_mul(f2_add(bR, bN), MK);
      const f2 pX = f2_fma(AL, dX, f2_mul(BU, uX));
      const f2 pY = f2_fma(AL, dY, f2_mul(BU, uY));
      const f2 pZ = f2_fma(ALZ, dZ, f2_mul(BU, uZ));
      GFX = f2_add(GFX, pX);
      GFY = f2_add(GFY, pY);
      GFZ = f2_add(GFZ, pZ);
      const f2 qX = f2_mul(BU, f2_sub(f2_mul(dY, uZ), f2_mul(dZ, uY)));
      const f2 qY = f2_mul(BU, f2_sub(f2_mul(dZ, uX), f2_mul(dX, uZ)));
      const f2 qZ = f2_mul(BU, f2_sub(f2_mul(dX, uY), f2_mul(dY, uX)));
      GTX = f2_add(GTX, qX);
      GTY = f2_add(GTY, qY);
      GTZ = f2_add(GTZ, qZ);
      if (oa.w >= 2.f || ob.w >= 2.f) {  // wall neighbours: torque about the axis
        float p[2][3], q[2][3];
        f2_split(pX, p[0][0], p[1][0]);
        f2_split(pY, p[0][1], p[1][1]);
        f2_split(pZ, p[0][2], p[1][2]);
        f2_split(qX, q[0][0], q[1][0]);
        f2_split(qY, q[0][1], q[1][1]);
        f2_split(qZ, q[0][2], q[1][2]);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if ((s == 0 ? oa.w : ob.w) >= 2.f) {
            wx += fmaf(-0.5f, q[s][0], pyi * p[s][2] - pzi * p[s][1]);
            wy += fmaf(-0.5f, q[s][1], pzi * p[s][0] - pxi * p[s][2]);
            wz += fmaf(-0.5f, q[s][2], pxi * p[s][1] - pyi * p[s][0]);
          }
        }
      }
    }
    // the group's two partial sums, then the compensated sums
    float a0, a1;
    f2_split(GFX, a0, a1);
    fx.add(a0 + a1);
    f2_split(GFY, a0, a1);
    fy.add(a0 + a1);
    f2_split(GFZ, a0, a1);
    fz.add(a0 + a1);
    f2_split(GTX, a0, a1);
    tx.add(a0 + a1);
    f2_split(GTY, a0, a1);
    ty.add(a0 + a1);
    f2_split(GTZ, a0, a1);
    tz.add(a0 + a1);
  }
  const float inv_m = P.inv_m_f[si], inv_I = P.inv_I_f[si];
  const float ax = fx.value(), ay = fy.value(), az = fz.value();
  const float bx = -0.5f * tx.value(), by = -0.5f * ty.value(), bz = -0.5f * tz.value();
  f.acc[i] = make_float4(ax * inv_m, ay * inv_m, az * inv_m, 0.f);
  f.dspin[i] = make_float4(bx * inv_I, by * inv_I, bz * inv_I, 0.f);
  f.tw[i] = make_float4(wx, wy, wz, 0.f);
  if (!finite3f(ax, ay, az) || !finite3f(bx, by, bz)) latch(err, ERR_NONFINITE);
}

// ----------------------------------------------------------- load / unload

__global__ void k_load_mixed(int64_t n, MixBuf b, const InstDev* __restrict__ inst,
                             int32_t n_inst, const double* __restrict__ pos,
                             const double* __restrict__ vel, const double* __restrict__ spin,
                             const uint8_t* __restrict__ sp, uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = instance_of(inst, n_inst, i);
    const InstDev& P = inst[k];
    int c[3];
    float4 o;
    bool ok = true;
    ok &= to_cell(P, 0, pos[3 * i], c[0], o.x);
    ok &= to_cell(P, 1, pos[3 * i + 1], c[1], o.y);
    ok &= to_cell(P, 2, pos[3 * i + 2], c[2], o.z);
    o.w = (float)sp[i];
    if (!ok) latch(err, ERR_ESCAPED);
    b.cell[i] = pack_cell(c[0], c[1], c[2]);
    b.off[i] = o;
    b.vel(i) = make_float4((float)vel[3 * i], (float)vel[3 * i + 1], (float)vel[3 * i + 2], 0.f);
    b.spin(i) =
        make_float4((float)spin[3 * i], (float)spin[3 * i + 1], (float)spin[3 * i + 2], 0.f);
    b.ref[i] = dvec2{pos[3 * i], pos[3 * i + 1]};
    b.id[i] = (uint32_t)i;
    b.inst[i] = k;
  }
}

__global__ void k_unsort_mixed(int64_t n, MixBuf b, MixFields f, const InstDev* __restrict__ inst,
                               double* pos, double* vel, double* spin, double* rho, double* P,
                               double* acc, double* dspin) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b.id[k];
    const InstDev& Q = inst[b.inst[k]];
    if (pos) {
      const uint32_t c = b.cell[k];
      const float4 of = b.off[k];
      pos[3 * o] = Q.lo[0] + (double)cell_x(c) * Q.cell[0] + (double)of.x;
      pos[3 * o + 1] = Q.lo[1] + (double)cell_y(c) * Q.cell[1] + (double)of.y;
      pos[3 * o + 2] = fold_z(Q, Q.lo[2] + (double)cell_z(c) * Q.cell[2] + (double)of.z);
    }
    if (vel) {
      const float4 v = b.vel(k);
      vel[3 * o] = v.x;
      vel[3 * o + 1] = v.y;
      vel[3 * o + 2] = v.z;
    }
    if (spin) {
      const float4 w = b.spin(k);
      spin[3 * o] = w.x;
      spin[3 * o + 1] = w.y;
      spin[3 * o + 2] = w.z;
    }
    if (rho) rho[o] = Q.rho0 * (1.0 + (double)f.delta[k]);
    if (P) P[o] = f.P[k];
    if (acc) {
      const float4 a = f.acc[k];
      acc[3 * o] = a.x;
      acc[3 * o + 1] = a.y;
      acc[3 * o + 2] = a.z;
    }
    if (dspin) {
      const float4 a = f.dspin[k];
      dspin[3 * o] = a.x;
      dspin[3 * o + 1] = a.y;
      dspin[3 * o + 2] = a.z;
    }
  }
}

}  // namespace

cudaError_t launch_drift_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                               const InstDev* inst, InstState* ist, uint32_t* err, int mode,
                               cudaStream_t s, const LaunchCfg& lc, int* launches) {
  k_drift_mixed<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, inst, ist, err, mode);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// (The gated streaming kernels of the list build run on grids of 8 blocks
// per SM, striding over the particles: a step that keeps its lists pays a
// few microseconds for each instead of about twelve.)
cudaError_t launch_keys_mixed(int64_t n, const MixBuf& b, const InstDev* inst,
                              const InstState* ist, const CellWs& cw, uint32_t* err, int mode,
                              cudaStream_t s, const LaunchCfg& lc, int* launches) {
  k_keys_mixed<<<grid_for(n, 256, lc.sm_count, 8), 256, 0, s>>>(n, b, inst, ist, cw, err, mode);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_relist_keys_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                     const InstDev* inst, const CellWs& cw, cudaStream_t s,
                                     const LaunchCfg& lc) {
  k_relist_keys_mixed<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, inst, cw);
  return cudaGetLastError();
}

cudaError_t launch_gate(bool open, int32_t n_inst, const InstDev* inst, InstState* ist,
                        uint32_t* err, int mode, cudaStream_t s, int* launches) {
  if (open)
    k_gate_force<<<1, 128, 0, s>>>(n_inst, ist, err);
  else
    k_gate_close<<<1, 128, 0, s>>>(n_inst, inst, ist, err, mode);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_reorder_mixed(int64_t n, const MixBuf& src, const MixBuf& dst,
                                 const CellWs& cw, const uint32_t* gate, cudaStream_t s,
                                 const LaunchCfg& lc, int* launches) {
  k_reorder_mixed<<<grid_for(n, 256, lc.sm_count, 8), 256, 0, s>>>(n, src, dst, cw, gate);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_copyback_mixed(int64_t n, const MixBuf& src, const MixBuf& dst,
                                  const MixFields& f, const InstState* ist, const uint32_t* gate,
                                  cudaStream_t s, const LaunchCfg& lc, int* launches) {
  k_copyback_mixed<<<grid_for(n, 256, lc.sm_count, 8), 256, 0, s>>>(n, src, dst, f, ist, gate);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_skin_list_mixed(int64_t n, const MixBuf& b, const InstDev* inst,
                                   const InstState* ist, const CellWs& cw, const NbrWs& nw,
                                   uint32_t* err, int gated, cudaStream_t s,
                                   const LaunchCfg& lc, int* launches) {
  k_skin_list_mixed<64><<<grid_for(n, 64, lc.sm_count, 16), 64, 0, s>>>(n, b, inst, ist, cw, nw,
                                                                          err, gated);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_density_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                 const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                 cudaStream_t s, const LaunchCfg& lc, int* launches) {
  const unsigned g32 = (unsigned)((n + 31) / 32), g64 = (unsigned)((n + 63) / 64),
                 g128 = (unsigned)((n + 127) / 128);
  if (lc.any_filter) {
    if (lc.block_density == 32)
      k_density_mixed<32, true><<<g32, 32, 0, s>>>(n, b, f, inst, nw, err);
    else if (lc.block_density == 64)
      k_density_mixed<64, true><<<g64, 64, 0, s>>>(n, b, f, inst, nw, err);
    else
      k_density_mixed<128, true><<<g128, 128, 0, s>>>(n, b, f, inst, nw, err);
  } else {
    if (lc.block_density == 32)
      k_density_mixed<32, false><<<g32, 32, 0, s>>>(n, b, f, inst, nw, err);
    else if (lc.block_density == 64)
      k_density_mixed<64, false><<<g64, 64, 0, s>>>(n, b, f, inst, nw, err);
    else
      k_density_mixed<128, false><<<g128, 128, 0, s>>>(n, b, f, inst, nw, err);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_forces_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                cudaStream_t s, const LaunchCfg& lc, int* launches) {
  const unsigned g256 = (unsigned)((n + 255) / 256), g128 = (unsigned)((n + 127) / 128),
                 g64 = (unsigned)((n + 63) / 64);
  // the pair pass carries only the options some instance uses
  const int opt = (lc.any_literal ? kOptLiteral : 0) | (lc.any_collision ? kOptCollision : 0);
  if (opt == 0) {  // the default form: two neighbours per step in packed FP32
    if (lc.block_forces == 256)
      k_forces_mixed_x2<256><<<g256, 256, 0, s>>>(n, b, f, inst, nw, err);
    else if (lc.block_forces == 64)
      k_forces_mixed_x2<64><<<g64, 64, 0, s>>>(n, b, f, inst, nw, err);
    else
      k_forces_mixed_x2<128><<<g128, 128, 0, s>>>(n, b, f, inst, nw, err);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  auto go = [&](auto kopt) {
    constexpr int O = decltype(kopt)::value;
    if (lc.block_forces == 256)
      k_forces_mixed<256, O><<<g256, 256, 0, s>>>(n, b, f, inst, nw, err);
    else if (lc.block_forces == 64)
      k_forces_mixed<64, O><<<g64, 64, 0, s>>>(n, b, f, inst, nw, err);
    else
      k_forces_mixed<128, O><<<g128, 128, 0, s>>>(n, b, f, inst, nw, err);
  };
  if (opt == kOptCollision)
    go(std::integral_constant<int, kOptCollision>());
  else  // the literal F_sn, with or without collisions
    go(std::integral_constant<int, kOptLiteral | kOptCollision>());
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_pfilter_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                 const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                 cudaStream_t s, int* launches) {
  k_pfilter_mixed<128><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, b, f, inst, nw, err);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_kick_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                              const InstDev* inst, cudaStream_t s, const LaunchCfg& lc,
                              int* launches) {
  k_kick_mixed<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, inst);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_load_mixed(int64_t n, const MixBuf& b, const InstDev* inst, int32_t n_inst,
                              const double* pos, const double* vel, const double* spin,
                              const uint8_t* sp, uint32_t* err, cudaStream_t s,
                              const LaunchCfg& lc) {
  k_load_mixed<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, inst, n_inst, pos, vel,
                                                                  spin, sp, err);
  return cudaGetLastError();
}

cudaError_t launch_unsort_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                const InstDev* inst, double* pos, double* vel, double* spin,
                                double* rho, double* P, double* acc, double* dspin,
                                cudaStream_t s, const LaunchCfg& lc) {
  k_unsort_mixed<<<grid_for(n, 256, lc.sm_count, 32), 256, 0, s>>>(n, b, f, inst, pos, vel, spin,
                                                                    rho, P, acc, dspin);
  return cudaGetLastError();
}

}  // namespace sphgb
