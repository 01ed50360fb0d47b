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
  int64_t cell_base;              // first global cell index of the instance
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
// Per-thread neighbour-list builder: entries are staged in shared memory and
// written to global memory 8 at a time as one full 32-byte sector.  Entries
// beyond nw.cap are counted (total) but dropped.
constexpr int kStageStride = 9;  // words of shared staging per thread (8 used)

struct ListWriter {
  uint32_t* list;
  int64_t n, i;
  uint32_t* st;
  uint32_t groups;  // cap / 8
  uint32_t cnt = 0;  // entries appended (may exceed the capacity)
  __device__ __forceinline__ ListWriter(const NbrWs& nw, int64_t n_, int64_t i_, uint32_t* st_)
      : list(nw.list), n(n_), i(i_), st(st_), groups((uint32_t)nw.cap >> 3) {}
  __device__ __forceinline__ void flush(uint32_t group) {
    if (group >= groups) return;  // beyond the capacity: dropped
    uint4* dst = reinterpret_cast<uint4*>(list + nbr_slot(n, i, group << 3));
    dst[0] = make_uint4(st[0], st[1], st[2], st[3]);
    dst[1] = make_uint4(st[4], st[5], st[6], st[7]);
  }
  __device__ __forceinline__ void append(uint32_t e) {
    st[cnt & 7u] = e;
    ++cnt;
    if ((cnt & 7u) == 0u) flush((cnt >> 3) - 1u);
  }
  __device__ __forceinline__ bool overflow() const { return cnt > (groups << 3); }
  // Flush the last partial group; returns the number of stored entries.
  __device__ __forceinline__ uint32_t finish() {
    if (cnt & 7u) flush(cnt >> 3);
    return cnt < (groups << 3) ? cnt : (groups << 3);
  }
};

// Walks the candidates of one particle's 27 neighbour cells as one flat
// sequence: 9 rows (dy, dz) of 3 x-adjacent cells, each row a contiguous run
// of the sorted order split at the cell starts.  For the current candidate
// it provides the cell displacement c_i - c_j (as -1/0/+1 times the cell
// side per axis) and its 6-bit code.  One flat loop per thread keeps the
// lanes of a warp in step even when they sit in different cells.
struct CellWalker {
  const uint32_t* start;
  int64_t base;
  int nx, ny, nz, cx, cy, cz;
  bool periodic;
  float Lx, Ly, Lz;
  int kx = 2, ky = 2, kz = -1;
  uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
  uint32_t j = 0, e = 0;
  float exL = 0.f, eyL = 0.f, ezL = 0.f;
  uint32_t code_yz = 0, code = 0;
  __device__ __forceinline__ CellWalker(const uint32_t* start_, int64_t base_, int nx_, int ny_,
                                        int nz_, int cx_, int cy_, int cz_, bool periodic_,
                                        float Lx_, float Ly_, float Lz_)
      : start(start_), base(base_), nx(nx_), ny(ny_), nz(nz_), cx(cx_), cy(cy_), cz(cz_),
        periodic(periodic_), Lx(Lx_), Ly(Ly_), Lz(Lz_) {}
  // Next candidate index in *jj; false when all 27 cells are done.
  __device__ __forceinline__ bool next(uint32_t* jj) {
    while (j == e) {
      if (++kx == 3) {
        kx = 0;
        if (++ky == 3) {
          ky = 0;
          if (++kz == 3) return false;
        }
        int z2 = cz + kz - 1;
        if (periodic) z2 = z2 < 0 ? z2 + nz : (z2 >= nz ? z2 - nz : z2);
        const int64_t row = base + (int64_t)nx * ((cy + ky - 1) + (int64_t)ny * z2);
        r0 = start[row + cx - 1];
        r1 = start[row + cx];
        r2 = start[row + cx + 1];
        r3 = start[row + cx + 2];
        eyL = (float)(1 - ky) * Ly;
        ezL = (float)(1 - kz) * Lz;
        code_yz = ((uint32_t)(2 - ky) << 2) | ((uint32_t)(2 - kz) << 4);
      }
      j = kx == 0 ? r0 : (kx == 1 ? r1 : r2);
      e = kx == 0 ? r1 : (kx == 1 ? r2 : r3);
      exL = (float)(1 - kx) * Lx;
      code = ((uint32_t)(2 - kx) | code_yz) << kNbrIndexBits;
    }
    *jj = j++;
    return true;
  }
};
#endif

}  // namespace sphgb
