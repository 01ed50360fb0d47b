// Internal data layout shared by the host driver and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph.h"

namespace sphgb {

// 32-byte aligned four-double record (one particle's xyz + one scalar) and a
// 16-byte pair; own types so that the alignment is explicit.
struct alignas(32) dvec4 {
  double x, y, z, w;
};
struct alignas(16) dvec2 {
  double x, y;
};

constexpr int kScanChunk = 4096;       // elements per block of the cell-count scan
constexpr int kReduceChunk = 32768;    // particles per partial of the FP64 reductions
constexpr int kDiagFields = 24;        // doubles per diagnostics partial
constexpr int kMaxInst = 65535;
constexpr int kSlabs = 4;              // x-slabs per cell in the sort key

// Error bits latched on the device.
enum : uint32_t {
  ERR_ESCAPED = 1u,
  ERR_NONFINITE = 2u,
  ERR_NEIGHBORS = 4u,
  ERR_TIMEOUT = 8u,
};

// Derived per-instance constants (host computed, read-only on the device).
struct InstDev {
  double h, inv_h, cut2;          // smoothing length, 1/h, (2h)^2
  double aD, cF;                  // Wendland C2: W = aD t^4 (2q+1), F = cF t^3
  double m_s, m_n;                // particle masses (inviscid, viscous/wall)
  double inv_I_s, inv_I_n;        // 1 / spin inertia
  double rho0, inv_rho0, p0, beta_P;
  double A, B;                    // shear 10(eta - 0.6 eta_r), rotational 4 eta_r
  double C_l, C_T;
  double Omega, dt, hdt;
  double Hz, half_Hz;             // z period
  double lo[3], inv_cell[3];      // grid origin (ghost cells included), 1 / side
  double cell[3];                 // cell side per axis (>= 2h)
  float cut2f_margin;             // FP32 prefilter bound (>= every FP64 neighbour)
  float Hzf, half_Hzf;
  int32_t nx, ny, nz;             // cells per axis (ghost ring except periodic z)
  int32_t clo[3], chi[3];         // interior cell range per axis (inclusive)
  int32_t alphaP;                 // integer Tait exponent
  uint32_t flags;
  int32_t periodic_z;
  int32_t slabs;                  // x-slabs per cell: sort key = cell * slabs + slab
  int64_t cell_base;              // first global sort key of the instance
  int64_t p_begin, p_end;         // particle range (fixed across sorts)
  int64_t chunk_base;             // first reduction chunk of the instance
  int64_t n_chunks;
  // ---- FP32 copies for the mixed form ----
  float cellf[3];                 // cell side per axis
  float cut2_f;                   // (2h)^2 rounded to float (strict < test)
  float inv_h_f, aD_f, cF_f;
  float m_f[2];                   // particle mass: [0] inviscid, [1] viscous/wall
  float mr_f[2];                  // m / rho0
  float inv_m_f[2], inv_I_f[2];
  float self_hi[2], self_lo[2];   // m aD / rho0 - 1 as an unevaluated float sum
  float p0_f, p0mb_f;             // p0 and p0 - beta_P
  float binom[17];                // binomial coefficients C(alpha_P, k)
  float rho0_f, A_f, B_f, C_l_f, C_T_f;
  float dt_f, hdt_f, Omega_f;
};

// Mutable per-instance scalars that live on the device.
struct InstState {
  double theta;                   // wall phase
  double T_wall[3];               // wall torque of the last force evaluation
  double J_wall[3];               // trapezoidal impulse of T_wall
  int64_t step;
  int64_t pad;
};

// One copy of the sorted FP64 particle state (double-buffered for the reorder).
// pos.w holds the species code; vel.w and spin.w receive V = m/rho and
// Pr = P/rho^2 from the density pass so that the pair pass gathers a
// neighbour with three 32-byte loads.
struct Fp64Buf {
  dvec4* pos;         // x, y, z, species
  dvec4* vel;         // vx, vy, vz, V
  dvec4* spin;        // wx, wy, wz, Pr
  dvec2* ref;         // wall reference (phase-0) x, y
  uint32_t* id;         // input index
  uint32_t* inst;       // instance index
};

struct Fp64Fields {
  dvec4* acc;         // acceleration (w unused)
  dvec4* dspin;       // spin angular acceleration (w unused)
  double* rho;
  double* P;
  dvec4* tw;          // torque of wall neighbours on each fluid particle
};

// One copy of the sorted mixed-precision state: an integer cell plus an FP32
// offset inside the cell for the position, FP32 everything else.
// off.w holds the species code; vel.w and spin.w receive V = m/rho and
// Pr = P/rho^2 from the density pass.
struct MixBuf {
  uint32_t* cell;       // cx | cy << 11 | cz << 22 (cell coordinates in the instance)
  float4* off;          // offset in [0, cell side) per axis, species
  float4* vel;          // vx, vy, vz, V
  float4* spin;         // wx, wy, wz, Pr
  dvec2* ref;           // wall reference (phase-0) x, y in FP64
  uint32_t* id;
  uint32_t* inst;
};

struct MixFields {
  float4* acc;
  float4* dspin;
  float4* tw;           // torque of wall neighbours on each fluid particle
  float* delta;         // rho / rho0 - 1
  float* P;
};

constexpr uint32_t kCellBitsX = 11, kCellBitsY = 11, kCellBitsZ = 10;

struct CellWs {
  uint32_t* key;        // global cell of each particle (pre-sort order)
  uint32_t* slot;       // arrival slot within the cell (atomic order)
  uint32_t* perm;       // sorted position -> pre-sort index
  uint32_t* skey;       // key in sorted order
  uint32_t* count;      // particles per cell
  uint32_t* start;      // exclusive scan of count, n_cells + 1 entries
  uint32_t* bsum;       // per-chunk sums of the scan
  int64_t n_cells;
  int64_t n_scan_blocks;
};

// Neighbour lists.  Entry t of particle i lives at nbr_slot(n, i, t): groups
// of 8 consecutive entries of one particle form one 32-byte sector, and the
// groups of consecutive particles are adjacent ([cap/8][n][8]), so a warp
// writes whole sectors and reads 1 KB contiguous per group.  An entry holds
// the neighbour's sorted index in its low 26 bits and, in the top 6 bits, the
// cell displacement code (dx+1) | (dy+1) << 2 | (dz+1) << 4 of the neighbour's
// cell relative to the particle's own (used by the mixed form).
constexpr int kNbrGroup = 8;
constexpr uint32_t kNbrIndexBits = 26;
constexpr uint32_t kNbrIndexMask = (1u << kNbrIndexBits) - 1u;
constexpr int64_t kMaxParticles = (int64_t)1 << kNbrIndexBits;  // 67,108,864

__host__ __device__ __forceinline__ int64_t nbr_slot(int64_t n, int64_t i, uint32_t t) {
  return (((int64_t)(t >> 3) * n + i) << 3) + (int64_t)(t & 7u);
}

struct NbrWs {
  uint32_t* list;       // neighbour entries, layout above
  uint32_t* count;      // neighbours per particle
  float4* posf;         // FP32 copy of sorted positions (FP64-form prefilter)
  int32_t cap;          // slots per particle (multiple of 8)
};

#ifdef __CUDACC__
// Per-thread neighbour-list builder.  push() stores every candidate entry in
// the thread's shared-memory staging and advances the fill only if it is a
// neighbour (no branch per candidate); drain(), called by all lanes of a warp
// at the same points (every kDrainEvery pushes), writes the complete groups
// of 8 as full 32-byte sectors and keeps the remainder.  Entries beyond
// nw.cap are counted but dropped.
constexpr int kDrainEvery = 32;
constexpr int kStageWords = 40;  // >= 7 + kDrainEvery
constexpr int kStageStride = 41;  // odd stride spreads the threads over banks

struct ListWriter {
  uint32_t* list;
  int64_t n, i;
  uint32_t* st;
  uint32_t groups;       // cap / 8
  uint32_t pend = 0;     // staged entries not yet written
  uint32_t written = 0;  // groups written (or dropped beyond the capacity)
  __device__ __forceinline__ ListWriter(const NbrWs& nw, int64_t n_, int64_t i_, uint32_t* st_)
      : list(nw.list), n(n_), i(i_), st(st_), groups((uint32_t)nw.cap >> 3) {}
  __device__ __forceinline__ void push(uint32_t e, bool keep) {
    if (keep) st[pend++] = e;  // a predicated store, no branch
  }
  __device__ __forceinline__ void write_group(uint32_t from) {
    if (written < groups) {
      uint4* dst = reinterpret_cast<uint4*>(list + nbr_slot(n, i, written << 3));
      dst[0] = make_uint4(st[from], st[from + 1], st[from + 2], st[from + 3]);
      dst[1] = make_uint4(st[from + 4], st[from + 5], st[from + 6], st[from + 7]);
    }
    ++written;
  }
  __device__ __forceinline__ void drain() {
    const uint32_t g = pend >> 3;
    for (uint32_t k = 0; k < g; ++k) write_group(k << 3);
    const uint32_t rem = pend & 7u;
    for (uint32_t r = 0; r < rem; ++r) st[r] = st[(g << 3) + r];
    pend = rem;
  }
  __device__ __forceinline__ uint32_t total() const { return (written << 3) + pend; }
  __device__ __forceinline__ bool overflow() const { return total() > (groups << 3); }
  // Write everything (the last group partially); returns the stored count.
  __device__ __forceinline__ uint32_t finish() {
    drain();
    const uint32_t t = total();
    if (pend) write_group(0);
    return t < (groups << 3) ? t : (groups << 3);
  }
};

// Visits the candidates of one particle: the 9 rows (dy, dz) of the 27-cell
// stencil, each row the 3 x-adjacent cells cx-1..cx+1, which the sort keeps
// as one run of S x-slabs per cell.  With window, a row out of reach (its
// nearest y-z distance >= the cutoff) is skipped and within a row only the
// slabs overlapping the x-window |x_j - x_i| <= sqrt(cut^2 - d_yz^2) (+ a
// margin) are visited.  Runs are split at the cell boundaries, so the cell
// displacement c_i - c_j of every candidate is known: visit(j, exL, eyL, ezL,
// code) gets it as -1/0/+1 times the cell side per axis and as its 6-bit
// code.  (ox, oy, oz) are the particle's FP32 offsets inside its cell
// (cx, cy, cz); cut2 is the squared cutoff of the candidate test.
template <class Visit>
__device__ __forceinline__ void visit_candidates(const uint32_t* __restrict__ start, int64_t base,
                                                 int nx, int ny, int nz, int S, bool periodic,
                                                 int cx, int cy, int cz, float Lx, float Ly,
                                                 float Lz, float ox, float oy, float oz,
                                                 float cut2, bool window, Visit&& visit) {
  const float inv_slab = (float)S / Lx;
  for (int dz = -1; dz <= 1; ++dz) {
    int z2 = cz + dz;
    if (periodic) z2 = z2 < 0 ? z2 + nz : (z2 >= nz ? z2 - nz : z2);
    const float rz = dz < 0 ? oz : (dz > 0 ? Lz - oz : 0.f);
    const float ezL = (float)(-dz) * Lz;
    for (int dy = -1; dy <= 1; ++dy) {
      int slo = 0, shi = 3 * S - 1;
      if (window) {
        const float ry = dy < 0 ? oy : (dy > 0 ? Ly - oy : 0.f);
        const float d2 = ry * ry + rz * rz;
        if (d2 >= cut2 + 1e-3f) continue;  // row out of reach
        const float w = sqrtf(fmaxf(cut2 - d2, 0.f)) + 2e-3f;
        const float xr = Lx + ox;  // x relative to the start of cell cx-1
        const int lo = (int)floorf((xr - w) * inv_slab);
        const int hi = (int)floorf((xr + w) * inv_slab);
        slo = lo < 0 ? 0 : lo;
        shi = hi > 3 * S - 1 ? 3 * S - 1 : hi;
      }
      const int64_t rowkey =
          base + ((int64_t)(cx - 1) + (int64_t)nx * ((cy + dy) + (int64_t)ny * z2)) * S;
      const float eyL = (float)(-dy) * Ly;
      const uint32_t code_yz = ((uint32_t)(1 - dy) << 2) | ((uint32_t)(1 - dz) << 4);
      for (int kc = slo / S; kc < 3 && kc * S <= shi; ++kc) {
        const int a = kc * S > slo ? kc * S : slo;
        const int b = kc * S + S - 1 < shi ? kc * S + S - 1 : shi;
        const uint32_t j0 = start[rowkey + a];
        const uint32_t j1 = start[rowkey + b + 1];
        const float exL = (float)(1 - kc) * Lx;
        const uint32_t code = ((uint32_t)(2 - kc) | code_yz) << kNbrIndexBits;
        for (uint32_t j = j0; j < j1; ++j) visit(j, exL, eyL, ezL, code);
      }
    }
  }
}
#endif

}  // namespace sphgb
