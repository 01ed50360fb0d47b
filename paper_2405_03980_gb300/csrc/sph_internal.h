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
constexpr int kReduceChunk = 32768;    // particles per partial of the plain-array diagnostics
constexpr int kStateChunk = 8192;      // particles per partial of the state's FP64 reductions
constexpr int kDiagFields = 24;        // doubles per diagnostics partial
constexpr int kMaxInst = 65535;
constexpr int kSlabs = 4;              // x-slabs per cell in the sort key

// Error bits latched on the device.
enum : uint32_t {
  ERR_ESCAPED = 1u,
  ERR_NONFINITE = 2u,
  ERR_NEIGHBORS = 4u,
  ERR_TIMEOUT = 8u,
  ERR_BOUNDS = 16u,         // an index failed a bounds check (checked build)
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
  double col2;                    // collision model: col_dist^2, 0 when it is off
  double cC[3];                   // -(1 + col_e) m_a m_b / ((m_a + m_b) dt) for the
                                  // species pairs a + b = 0 (inviscid, inviscid),
                                  // 1 (inviscid, other), 2 (other, other)
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
  float lof[3];                   // grid origin lo per axis
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
  float col2_f, cC_f[3];
  // Reused neighbour lists of the mixed form: the lists are built with the
  // radius 2h + skin (cell side >= 2h + skin) and kept while every particle
  // of the instance stays within skin/2 of where the vessel's rigid rotation
  // since the build has carried its build position (rotation keeps every
  // pair distance, so only the departure from it can bring a new pair inside
  // 2h); every step re-tests r < 2h.  skin 0: rebuilt every step.
  double skin;
  float skin_cut2_f;              // (2h + skin)^2: the list-build test
  float skin_disp2_f;             // rebuild when |departure|^2 exceeds this (< 0: always)
  float skin_omax_f;              // rebuild when an offset leaves [-omax, L + omax]
};

// Mutable per-instance scalars that live on the device.
struct InstState {
  double theta;                   // wall phase
  double T_wall[3];               // wall torque of the last force evaluation
  double J_wall[3];               // trapezoidal impulse of T_wall
  int64_t step;
  int32_t rebuild;                // mixed form: the lists are rebuilt in this step
  int32_t rebuilds;               // mixed form: list builds so far
  double theta_ref;               // mixed form: wall phase at the last list build
  double pad;
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
  dvec2* vp;          // pressure filter input (V, V P) of the density pass;
                      // (0, 0) for outer walls
};

// One copy of the sorted mixed-precision state: an integer cell plus an FP32
// offset inside the cell for the position, FP32 everything else.
// off.w holds the species code; vel.w and spin.w receive V = m/rho and
// Pr = P/rho^2 from the density pass.
struct MixBuf {
  uint32_t* cell;       // cx | cy << 11 | cz << 22 (cell coordinates in the instance)
  float4* off;          // offset in [0, cell side) per axis, species
  // velocity (vx, vy, vz, V) and spin (wx, wy, wz, P / rho^2) of particle i
  // side by side in one 32-byte record, vs[2i] and vs[2i + 1], so that a
  // neighbour's two records arrive in one sector (one 256-bit load)
  float4* vs;
  dvec2* ref;           // wall reference (phase-0) x, y in FP64
  uint32_t* id;
  uint32_t* inst;
#ifdef __CUDACC__
  __device__ __forceinline__ float4& vel(int64_t i) const { return vs[2 * i]; }
  __device__ __forceinline__ float4& spin(int64_t i) const { return vs[2 * i + 1]; }
#endif
};

struct MixFields {
  float4* acc;
  float4* dspin;
  float4* tw;           // torque of wall neighbours on each fluid particle
  float* delta;         // rho / rho0 - 1
  float* P;
  float2* vp;           // pressure filter input (V, P); (0, 0) for outer walls
  float4* oref;         // offsets (and species) at the last list build; the
                        // cells stay fixed until the next build
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
  uint32_t* err;        // the device error word (bounds checks of the checked build)
};

// Neighbour sets.  The neighbour search writes, for every grid cell, its
// candidate table: the particles of the 27-cell stencil in candidate order
// (rows dz, dy, cells kc, sorted index), at most kMaxCand entries, each the
// candidate's sorted index in the low 26 bits and, in the top 6 bits, the
// cell displacement code (dx+1) | (dy+1) << 2 | (dz+1) << 4 of the particle's
// cell relative to the candidate's (used by the mixed form).  Per particle it
// writes one bit per candidate of its cell: word k of particle i, at
// mask[k * n + i], covers candidates 32k .. 32k + 31.  The density pass walks
// the set bits in order (the FP64 form re-tests each exactly) and writes the
// neighbours as i's neighbour list for the pair pass.
constexpr uint32_t kNbrIndexBits = 26;
constexpr uint32_t kNbrIndexMask = (1u << kNbrIndexBits) - 1u;
constexpr int64_t kMaxParticles = (int64_t)1 << kNbrIndexBits;  // 67,108,864
constexpr int kMaxCand = 1024;
constexpr int kMaxCandWords = kMaxCand / 32;

// Neighbour lists.  Entry t of particle i lives at nbr_slot(n, i, t): groups
// of 8 consecutive entries of one particle form one 32-byte sector, and the
// groups of consecutive particles are adjacent ([cap/8][n][8]), so a warp
// writes whole sectors and reads 1 KB contiguous per group.  An entry is a
// candidate-table entry (index | displacement code).
constexpr int kNbrGroup = 8;
constexpr uint32_t kUnsplit = 0xFFFFFFFFu;
constexpr int kPartTile = 4096;  // particles per tile of the species partition

// Compile-time options of the pair pass (template argument kOpt).
constexpr int kOptLiteral = 1;    // literal F_sn on v_ij (SPH_SN_LITERAL)
constexpr int kOptCollision = 2;  // collision model (SPH_COLLISION)

__host__ __device__ __forceinline__ int64_t nbr_slot(int64_t n, int64_t i, uint32_t t) {
  return (((int64_t)(t >> 3) * n + i) << 3) + (int64_t)(t & 7u);
}

struct NbrWs {
  uint32_t* list;       // neighbour entries, layout above
  uint32_t* count;      // neighbours per particle (list length)
  // FP64 form: the list of a fluid particle holds its inviscid neighbours
  // first; count_a is their number (kUnsplit: not ordered, when the
  // pressure filter is on).  Species partition of the fluid particles for
  // the pair pass: order[0 .. n_inv) inviscid, then the viscous ones, each in
  // sorted order.
  uint32_t* count_a;
  uint32_t* order;
  uint32_t* part;       // per-tile counts of the partition, then its totals
  float4* posf;         // FP32 copy of sorted positions (FP64-form prefilter)
  uint32_t* mask;       // [kMaxCandWords][n] candidate hit bits
  uint32_t* cand;       // [grid cells][kMaxCand] candidate table of each cell
  uint32_t* ncand;      // [grid cells] candidates of each cell
  // Pressure filter only (null otherwise): the kernel shape t^4 (2q + 1) of
  // every list entry, written by the density pass in the list's layout
  // (nbr_slot), so the filter neither gathers positions nor re-evaluates W.
  double* wsh_d;        // FP64 form
  float* wsh_f;         // mixed form
  int32_t cap;          // list slots per particle (multiple of 8)
  // Mixed form: the reused candidate lists (entries within 2h + skin at the
  // last build, candidate-table entries in the layout of nbr_slot with
  // skin_cap slots) and their lengths; the density pass re-tests them.
  uint32_t* skin;
  uint32_t* skin_count;
  int32_t skin_cap;
};

// Error-word slots: err[0] latched error bits; err[1] (mixed form) non-zero
// while some instance rebuilds its lists in the current step.
constexpr int kErrRebuild = 1;

#ifdef __CUDACC__
// The instance that particle i (in input order) belongs to: instances hold
// consecutive ranges [p_begin, p_end) in order, so a binary search over their
// first particles finds it.
__device__ __forceinline__ uint32_t instance_of(const InstDev* __restrict__ inst, int32_t n_inst,
                                                int64_t i) {
  int32_t lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (inst[mid].p_begin <= i) lo = mid;
    else hi = mid - 1;
  }
  return (uint32_t)lo;
}

// z of an absolute position folded into the period [lo, lo + Hz) when z is
// periodic (mixed form: between list builds an offset may carry a particle
// past the period's end; it is folded when positions are formed).
__device__ __forceinline__ double fold_z(const InstDev& P, double z) {
  if (P.periodic_z) {
    if (z >= P.lo[2] + P.Hz) z -= P.Hz;
    else if (z < P.lo[2]) z += P.Hz;
  }
  return z;
}

// Checked build (compiled with -DSPH_CHECKED): the indices the kernels take
// from data (cell keys, sorted positions, candidate runs, neighbour entries,
// list lengths) are bounds-checked before use; a failed check latches
// ERR_BOUNDS and a safe index is used instead, so the run ends with
// SPH_ERR_BOUNDS rather than an out-of-range access.  In the default build
// the checks compile to nothing.
#ifdef SPH_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool bounds_ok(bool ok, uint32_t* err) {
  if (kChecked && !ok) {
    atomicOr(err, (uint32_t)ERR_BOUNDS);
    return false;
  }
  return true;
}

// A neighbour-list length, capped at the list's capacity (checked build).
__device__ __forceinline__ uint32_t checked_count(uint32_t c, int32_t cap, uint32_t* err) {
  return bounds_ok(c <= (uint32_t)cap, err) ? c : (uint32_t)cap;
}

// j if j < n, else (checked build) 0 with ERR_BOUNDS latched.
__device__ __forceinline__ uint32_t checked_index(uint32_t j, int64_t n, uint32_t* err) {
  return bounds_ok((int64_t)j < n, err) ? j : 0u;
}

// Walks the set bits of one particle's candidate mask in candidate order and
// yields the candidate-table entries, B at a time: the B table loads of a
// batch are independent and in flight together.  The K mask words are first
// copied, also all in flight together, to the thread's column of shared
// memory (word k at sw[k * stride]).
struct MaskWalk {
  const uint32_t* __restrict__ tab;
  uint32_t* sw;
  uint32_t stride, K;
  uint32_t k = 0, w = 0;
  __device__ __forceinline__ MaskWalk(const NbrWs& nw, int64_t n, int64_t i, int64_t g,
                                      uint32_t* sw_, uint32_t stride_)
      : tab(nw.cand + g * kMaxCand), sw(sw_), stride(stride_) {
    K = (nw.ncand[g] + 31u) >> 5;
    const uint32_t* __restrict__ mw = nw.mask + i;
#pragma unroll 4
    for (uint32_t t = 0; t < K; ++t) sw[t * stride] = mw[(int64_t)t * n];
    w = sw[0];
  }
  // Fills e[0 .. m) with the next m <= B entries; m = 0 at the end.
  template <int B>
  __device__ __forceinline__ uint32_t next(uint32_t (&e)[B]) {
    uint32_t m = 0;
#pragma unroll
    for (int u = 0; u < B; ++u) {
      while (w == 0u && k + 1 < K) w = sw[++k * stride];
      if (w != 0u) {
        const uint32_t bit = (uint32_t)__ffs(w) - 1u;
        w &= w - 1u;
        e[u] = tab[(k << 5) + bit];
        m = (uint32_t)u + 1u;
      }
    }
    return m;
  }
  // The same, also giving each entry's candidate position q = 32 word + bit.
  template <int B>
  __device__ __forceinline__ uint32_t next(uint32_t (&e)[B], uint32_t (&q)[B]) {
    uint32_t m = 0;
#pragma unroll
    for (int u = 0; u < B; ++u) {
      while (w == 0u && k + 1 < K) w = sw[++k * stride];
      if (w != 0u) {
        const uint32_t bit = (uint32_t)__ffs(w) - 1u;
        w &= w - 1u;
        q[u] = (k << 5) + bit;
        e[u] = tab[q[u]];
        m = (uint32_t)u + 1u;
      }
    }
    return m;
  }
};

// Candidate positions set aside during a mask walk, as bits, written back
// over the walk's own staged mask words once the walk has passed them (a
// word is staged before any of its bits is returned), so that a second walk
// over the same words yields the set-aside entries in candidate order.
struct MaskKeep {
  uint32_t* sw;
  uint32_t stride, K;
  uint32_t k = 0, acc = 0;
  __device__ __forceinline__ MaskKeep(const MaskWalk& mk) : sw(mk.sw), stride(mk.stride), K(mk.K) {}
  __device__ __forceinline__ void set(uint32_t q) {  // q ascending over the calls
    const uint32_t kq = q >> 5;
    while (k < kq) {
      sw[k * stride] = acc;
      acc = 0u;
      ++k;
    }
    acc |= 1u << (q & 31u);
  }
  __device__ __forceinline__ void finish() {  // the remaining words: set-aside bits or none
    for (; k < K; ++k) {
      sw[k * stride] = acc;
      acc = 0u;
    }
  }
};

// Per-thread neighbour-list builder.  push() stores an entry in the thread's
// shared-memory staging and advances the fill only if it is kept (a
// predicated store, no branch); drain(), called whenever 32 or more entries
// are staged, writes the complete groups of 8 as full 32-byte sectors and
// keeps the remainder.  Entries beyond nw.cap are counted but dropped.
// Staged word k of thread t lives at st[k * stride] with st = stage + t and
// stride = the block size (a multiple of 32), so the threads of a warp always
// touch distinct banks, whatever their fill.
constexpr int kDrainAt = 32;
constexpr int kStageWords = 40;   // >= kDrainAt - 1 + the largest batch pushed

struct ListWriter {
  uint32_t* list;
  int64_t n, i;
  uint32_t* st;
  uint32_t stride;       // words between a thread's staged entries
  uint32_t groups;       // cap / 8
  uint32_t pend = 0;     // staged entries not yet written
  uint32_t written = 0;  // groups written (or dropped beyond the capacity)
  __device__ __forceinline__ ListWriter(const NbrWs& nw, int64_t n_, int64_t i_, uint32_t* st_,
                                        uint32_t stride_)
      : list(nw.list), n(n_), i(i_), st(st_), stride(stride_), groups((uint32_t)nw.cap >> 3) {}
  __device__ __forceinline__ void push(uint32_t e, bool keep) {
    if (keep) st[(pend++) * stride] = e;
  }
  __device__ __forceinline__ void write_group(uint32_t from) {
    if (written < groups) {
      uint4* dst = reinterpret_cast<uint4*>(list + nbr_slot(n, i, written << 3));
      const uint32_t* q = st + from * stride;
      dst[0] = make_uint4(q[0], q[stride], q[2 * stride], q[3 * stride]);
      dst[1] = make_uint4(q[4 * stride], q[5 * stride], q[6 * stride], q[7 * stride]);
    }
    ++written;
  }
  __device__ __forceinline__ void drain() {
    const uint32_t g = pend >> 3;
    for (uint32_t k = 0; k < g; ++k) write_group(k << 3);
    const uint32_t rem = pend & 7u;
    for (uint32_t r = 0; r < rem; ++r) st[r * stride] = st[((g << 3) + r) * stride];
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
#endif

}  // namespace sphgb
