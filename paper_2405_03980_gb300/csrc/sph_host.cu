// Host side of the C ABI: parameter validation, the layout of the caller-owned
// device buffers, the step pipeline and its capture into CUDA graphs.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sph_kernels.h"

using namespace sphgb;

namespace {

// NVTX range around a public entry point (host side; the kernels a call
// enqueues, graph replays included, are attributed to it by the profilers).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kAlign = 256;

// Bump allocator over one caller buffer (or a null base to measure sizes).
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class T>
  T* take(int64_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = base ? (T*)(base + off) : nullptr;
    off += sizeof(T) * (size_t)(count > 0 ? count : 1);
    return p;
  }
};

bool is_int(double v) { return v == floor(v); }

// Sum of the Wendland C2 kernel over the integer lattice (host copy used for
// the particle mass m = rho0 / sum).
double lattice_kernel_sum(double dx, double h) {
  const double aD = 21.0 / (16.0 * kPi * h * h * h);
  const int m = (int)ceil(2.0 * h / dx) + 1;
  double s = 0.0;
  for (int a = -m; a <= m; ++a)
    for (int b = -m; b <= m; ++b)
      for (int c = -m; c <= m; ++c) {
        const double r = dx * sqrt((double)(a * a + b * b + c * c));
        const double q = r / h;
        if (!(q < 2.0)) continue;
        const double t = 1.0 - 0.5 * q;
        s += aD * t * t * t * t * (2.0 * q + 1.0);
      }
  return s;
}

sph_status derive(const sph_params& p, InstDev& d) {
  if (!(p.dx > 0) || !(p.h > 0) || !(p.rho0 > 0) || !(p.dt > 0) || !(p.p0 >= 0) ||
      !(p.inertia_coef > 0) || !(p.mass_ratio > 0) || !isfinite(p.Omega) ||
      !isfinite(p.beta_P) || !isfinite(p.eta_bar) || !isfinite(p.eta_r) ||
      !isfinite(p.C_l) || !isfinite(p.C_T))
    return SPH_ERR_ARG;
  if (!(p.alpha_P >= 1 && p.alpha_P <= 16 && is_int(p.alpha_P))) return SPH_ERR_ARG;
  if (p.precision != SPH_FP64 && p.precision != SPH_MIXED) return SPH_ERR_ARG;
  if (p.flags & ~511u) return SPH_ERR_ARG;
  if ((p.flags & SPH_COLLISION) &&
      !(p.col_dist > 0.0 && p.col_dist < 2.0 * p.h && p.col_e >= 0.0 && p.col_e <= 1.0))
    return SPH_ERR_ARG;
  memset(&d, 0, sizeof d);
  const double h = p.h;
  d.h = h;
  d.inv_h = 1.0 / h;
  d.cut2 = (2.0 * h) * (2.0 * h);
  d.aD = 21.0 / (16.0 * kPi * h * h * h);
  d.cF = 5.0 * d.aD / (h * h);
  const double S = lattice_kernel_sum(p.dx, h);
  d.m_n = p.rho0 / S;
  d.m_s = p.mass_ratio * d.m_n;
  d.inv_I_n = 1.0 / (p.inertia_coef * d.m_n * p.dx * p.dx);
  d.inv_I_s = 1.0 / (p.inertia_coef * d.m_s * p.dx * p.dx);
  d.rho0 = p.rho0;
  d.inv_rho0 = 1.0 / p.rho0;
  d.p0 = p.p0;
  d.beta_P = p.beta_P;
  d.A = 10.0 * (p.eta_bar - 0.6 * p.eta_r);
  d.B = 4.0 * p.eta_r;
  d.C_l = p.C_l;
  d.C_T = p.C_T;
  d.Omega = p.Omega;
  d.dt = p.dt;
  d.hdt = 0.5 * p.dt;
  d.alphaP = (int32_t)p.alpha_P;
  d.flags = p.flags;
  if (p.flags & SPH_COLLISION) {  // binary collision with restitution col_e
    d.col2 = p.col_dist * p.col_dist;
    const double ms[2] = {d.m_s, d.m_n};
    for (int k = 0; k < 3; ++k) {
      const double ma = ms[k > 1 ? 1 : 0], mb = ms[k > 0 ? 1 : 0];
      d.cC[k] = -(1.0 + p.col_e) * (ma * mb / (ma + mb)) / p.dt;
    }
  }
  d.periodic_z = p.periodic_z ? 1 : 0;
  d.slabs = kSlabs;
  // mixed form: neighbour lists kept across steps with a skin (0 = 0.5 dx,
  // negative = none); the cells must hold the 2h + skin stencil
  if (!isfinite(p.skin)) return SPH_ERR_ARG;
  d.skin = 0.0;
  if (p.precision == SPH_MIXED) d.skin = p.skin == 0.0 ? 0.3 * p.dx : (p.skin > 0.0 ? p.skin : 0.0);
  if (!(d.skin <= 2.0 * h)) return SPH_ERR_ARG;
  // The cells split each axis evenly with a side >= 2h + skin.  A periodic z
  // needs 3 cells; and where the even split would make the cells more than
  // 5 % deeper than 2h + skin (a short axis), one more cell with a narrower
  // skin keeps the 27-cell stencil's candidates within the table.
  for (int pass = 0; pass < 8 && d.skin > 0.0; ++pass) {
    double s2 = d.skin;
    for (int a = 0; a < 3; ++a) {
      const double L = p.box_hi[a] - p.box_lo[a];
      if (!(L > 0) || !isfinite(L)) return SPH_ERR_ARG;
      const double want = 2.0 * h + s2;
      const double nc = floor(L / want);
      double cells = -1.0;  // the cell count to fit, if any
      if (a == 2 && d.periodic_z && nc < 3) cells = 3.0;
      else if (nc >= 1 && L / nc > 1.05 * want) cells = nc + 1.0;
      if (cells > 0) {
        const double s3 = L / cells * (1.0 - 1e-12) - 2.0 * h;
        s2 = s3 > 0.0 ? s3 : 0.0;
      }
    }
    if (s2 == d.skin) break;
    d.skin = s2;
  }
  const double side = 2.0 * h + d.skin;
  double xmax = 0.0;
  int32_t n[3];
  for (int a = 0; a < 3; ++a) {
    const double L = p.box_hi[a] - p.box_lo[a];
    if (!(L > 0) || !isfinite(L)) return SPH_ERR_ARG;
    const double ncell = floor(L / side);
    const bool per = (a == 2 && d.periodic_z);
    if (per) {
      if (ncell < 3) return SPH_ERR_ARG;  // the 27-cell stencil needs 3 z cells
      if (ncell > 1 << 20) return SPH_ERR_GRID_OVERFLOW;
      n[a] = (int32_t)ncell;
      d.cell[a] = L / ncell;
      d.lo[a] = p.box_lo[a];
      d.clo[a] = 0;
      d.chi[a] = n[a] - 1;
    } else {
      const double ni = ncell < 1 ? 1 : ncell;
      if (ni > 1 << 20) return SPH_ERR_GRID_OVERFLOW;
      n[a] = (int32_t)ni + 2;  // ghost cell on both sides
      d.cell[a] = L / ni;
      d.lo[a] = p.box_lo[a] - d.cell[a];
      d.clo[a] = 1;
      d.chi[a] = n[a] - 2;
    }
    d.inv_cell[a] = 1.0 / d.cell[a];
    xmax = fmax(xmax, fmax(fabs(p.box_lo[a]), fabs(p.box_hi[a])) + d.cell[a]);
  }
  d.nx = n[0];
  d.ny = n[1];
  d.nz = n[2];
  const double Hz = p.box_hi[2] - p.box_lo[2];
  d.Hz = Hz;
  d.half_Hz = 0.5 * Hz;
  d.Hzf = (float)Hz;
  d.half_Hzf = (float)(0.5 * Hz);
  // FP32 prefilter bound: with coordinates rounded to float (|x| <= xmax) the
  // float r^2 of every true neighbour stays below cut2 + margin.
  const double eps = (2.0 * xmax + 2.0 * side) * ldexp(1.0, -24);
  const double margin = 4.0 * (2.0 * sqrt(3.0) * side * eps + 3.0 * eps * eps +
                               6.0 * d.cut2 * ldexp(1.0, -24));
  d.cut2f_margin = nextafterf((float)(d.cut2 + margin), INFINITY);

  // FP32 constants of the mixed form
  if (p.precision == SPH_MIXED &&
      (d.nx > (1 << kCellBitsX) || d.ny > (1 << kCellBitsY) || d.nz > (1 << kCellBitsZ)))
    return SPH_ERR_GRID_OVERFLOW;
  for (int a = 0; a < 3; ++a) {
    d.cellf[a] = (float)d.cell[a];
    d.lof[a] = (float)d.lo[a];
  }
  d.cut2_f = (float)d.cut2;
  d.inv_h_f = (float)d.inv_h;
  d.aD_f = (float)d.aD;
  d.cF_f = (float)d.cF;
  const double m[2] = {d.m_s, d.m_n};
  const double invI[2] = {d.inv_I_s, d.inv_I_n};
  for (int k = 0; k < 2; ++k) {
    d.m_f[k] = (float)m[k];
    d.mr_f[k] = (float)(m[k] / p.rho0);
    d.inv_m_f[k] = (float)(1.0 / m[k]);
    d.inv_I_f[k] = (float)invI[k];
    const double self = m[k] * d.aD / p.rho0 - 1.0;
    d.self_hi[k] = (float)self;
    d.self_lo[k] = (float)(self - (double)d.self_hi[k]);
  }
  d.p0_f = (float)p.p0;
  d.p0mb_f = (float)(p.p0 - p.beta_P);
  double binom = 1.0;
  for (int k = 0; k <= 16; ++k) {
    d.binom[k] = (k <= d.alphaP) ? (float)binom : 0.f;
    binom = binom * (double)(d.alphaP - k) / (double)(k + 1);
  }
  d.rho0_f = (float)p.rho0;
  d.A_f = (float)d.A;
  d.B_f = (float)d.B;
  d.C_l_f = (float)p.C_l;
  d.C_T_f = (float)p.C_T;
  d.dt_f = (float)p.dt;
  d.hdt_f = (float)(0.5 * p.dt);
  d.Omega_f = (float)p.Omega;
  d.col2_f = (float)d.col2;
  for (int k = 0; k < 3; ++k) d.cC_f[k] = (float)d.cC[k];
  // the list-build test keeps every pair within 2h + skin (rounded up, so
  // that no pair the exact test can accept later is lost to rounding); a
  // rebuild is due once a particle moved 0.495 skin (both ends of a pair
  // together less than the skin)
  if (d.skin > 0.0) {
    d.skin_cut2_f = nextafterf((float)((2.0 * h + d.skin) * (2.0 * h + d.skin)), INFINITY);
    // the departure is formed from FP32 positions of up to |x| ~ 2^11 dx:
    // 1e-3 dx of the half skin covers their rounding
    d.skin_disp2_f = (float)((0.5 * d.skin - 1e-3 * p.dx) * (0.5 * d.skin - 1e-3 * p.dx));
  } else {
    d.skin_cut2_f = d.cut2_f;
    d.skin_disp2_f = -1.0f;
  }
  // between builds the offsets may leave the cell by one cell side: their
  // FP32 resolution stays that of [0, 2L)
  d.skin_omax_f = d.cellf[0] < d.cellf[2] ? d.cellf[0] : d.cellf[2];
  return SPH_OK;
}

}  // namespace

sph_status sphgb::derive_instance(const sph_params& p, InstDev& d) { return derive(p, d); }

struct sph_ctx {
  int32_t n_inst = 0;
  int64_t n = 0;
  int32_t precision = SPH_FP64;
  int32_t cap = 160;
  std::vector<InstDev> inst_h;
  InstDev* inst = nullptr;
  InstState* ist = nullptr;
  uint32_t* err = nullptr;
  Fp64Buf buf[2];    // FP64 form
  Fp64Fields f;
  MixBuf mbuf[2];    // mixed form
  MixFields mf;
  int cur = 0;
  CellWs cw;
  NbrWs nw;
  int64_t total_chunks = 0;
  double* part_tw = nullptr;
  double* part_diag = nullptr;
  double* diag_out = nullptr;
  char* backup = nullptr;        // autotuner copy of acc, dspin, wall torque, InstState
  void* staging = nullptr;
  size_t staging_bytes = 0;
  void* state = nullptr;          // the caller's state buffer (checkpoints copy it)
  size_t state_bytes = 0;         // bytes of it in use
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool forces_valid = false;
  bool lists_valid = false;      // neighbour lists of the current sorted order
  bool skin_valid = false;       // mixed form: the reused lists of the workspace
                                 // belong to the state (not after a checkpoint load)
  int launches_per_step = 0;
  int64_t max_cells = 0;         // largest cell grid of an instance
  LaunchCfg lc;
};

namespace {

struct Carved {
  Fp64Buf buf[2];
  Fp64Fields f;
  MixBuf mbuf[2];
  MixFields mf;
  CellWs cw;
  NbrWs nw;
  InstDev* inst;
  InstState* ist;
  uint32_t* err;
  double *part_tw, *part_diag, *diag_out;
  char* backup;
  char* staging;
  size_t staging_bytes;
  size_t state_bytes, ws_bytes;
};

// Per-particle fields the pair pass writes (acc, dspin, wall torque) and the
// per-instance scalars: what sph_autotune saves and restores.
int64_t field_bytes(int32_t precision, int64_t n) {
  return (int64_t)(precision == SPH_FP64 ? sizeof(dvec4) : sizeof(float4)) * n;
}
int64_t backup_bytes(int32_t precision, int64_t n, int32_t n_inst) {
  return 3 * field_bytes(precision, n) + (int64_t)sizeof(InstState) * n_inst + 3 * 256;
}

void carve(void* state, void* ws, int32_t n_inst, int64_t n, int64_t n_cells,
           int64_t total_chunks, int32_t cap, int32_t skin_cap, int32_t precision, bool filter,
           Carved& c) {
  memset(&c, 0, sizeof c);
  Carver s(state);
  c.inst = s.take<InstDev>(n_inst);
  c.ist = s.take<InstState>(n_inst);
  c.err = s.take<uint32_t>(4);
  if (precision == SPH_FP64) {
    for (int b = 0; b < 2; ++b) {
      c.buf[b].pos = s.take<dvec4>(n);
      c.buf[b].vel = s.take<dvec4>(n);
      c.buf[b].spin = s.take<dvec4>(n);
      c.buf[b].ref = s.take<dvec2>(n);
      c.buf[b].id = s.take<uint32_t>(n);
      c.buf[b].inst = s.take<uint32_t>(n);
    }
    c.f.acc = s.take<dvec4>(n);
    c.f.dspin = s.take<dvec4>(n);
    c.f.tw = s.take<dvec4>(n);
    c.f.rho = s.take<double>(n);
    c.f.P = s.take<double>(n);
  } else {
    for (int b = 0; b < 2; ++b) {
      c.mbuf[b].cell = s.take<uint32_t>(n);
      c.mbuf[b].off = s.take<float4>(n);
      c.mbuf[b].vs = s.take<float4>(2 * n);
      c.mbuf[b].ref = s.take<dvec2>(n);
      c.mbuf[b].id = s.take<uint32_t>(n);
      c.mbuf[b].inst = s.take<uint32_t>(n);
    }
    c.mf.acc = s.take<float4>(n);
    c.mf.dspin = s.take<float4>(n);
    c.mf.tw = s.take<float4>(n);
    c.mf.delta = s.take<float>(n);
    c.mf.P = s.take<float>(n);
    c.mf.oref = s.take<float4>(n);
  }
  c.state_bytes = s.off + kAlign;

  Carver w(ws);
  c.cw.key = w.take<uint32_t>(n);
  c.cw.slot = w.take<uint32_t>(n);
  c.cw.perm = w.take<uint32_t>(n);
  c.cw.skey = w.take<uint32_t>(n);
  c.cw.count = w.take<uint32_t>(n_cells);
  c.cw.start = w.take<uint32_t>(n_cells + 1);
  c.cw.n_cells = n_cells;
  c.cw.err = c.err;
  c.cw.n_scan_blocks = (n_cells + kScanChunk - 1) / kScanChunk;
  c.cw.bsum = w.take<uint32_t>(c.cw.n_scan_blocks + 1);
  c.nw.list = w.take<uint32_t>((int64_t)cap * n);
  c.nw.count = w.take<uint32_t>(n);
  c.nw.posf = precision == SPH_FP64 ? w.take<float4>(n) : nullptr;
  c.nw.mask = w.take<uint32_t>((int64_t)kMaxCandWords * n);
  c.nw.ncand = w.take<uint32_t>(n_cells / kSlabs);
  c.nw.cand = w.take<uint32_t>(n_cells / kSlabs * kMaxCand);
  c.nw.cap = cap;
  if (precision == SPH_MIXED) {  // the reused candidate lists of the mixed form
    c.nw.skin = w.take<uint32_t>((int64_t)skin_cap * n);
    c.nw.skin_count = w.take<uint32_t>(n);
    c.nw.skin_cap = skin_cap;
  }
  if (precision == SPH_FP64) {
    c.f.vp = w.take<dvec2>(n);
    // the split lists and the species order of the FP64 pair pass
    c.nw.count_a = w.take<uint32_t>(n);
    c.nw.order = w.take<uint32_t>(n);
    c.nw.part = w.take<uint32_t>(2 * ((n + kPartTile - 1) / kPartTile) + 2);
  } else {
    c.mf.vp = w.take<float2>(n);
  }
  if (filter) {  // kernel shapes of the list entries, for the pressure filter
    if (precision == SPH_FP64)
      c.nw.wsh_d = w.take<double>((int64_t)cap * n);
    else
      c.nw.wsh_f = w.take<float>((int64_t)cap * n);
  }
  c.part_tw = w.take<double>(3 * total_chunks);
  c.part_diag = w.take<double>((int64_t)kDiagFields * total_chunks);
  c.diag_out = w.take<double>((int64_t)kDiagFields * n_inst);
  c.backup = w.take<char>(backup_bytes(precision, n, n_inst));
  // host arrays in and out: at most 17 doubles per particle (sph_get_state),
  // each array aligned
  c.staging_bytes = sizeof(double) * 17 * (size_t)n + 8 * kAlign;
  c.staging = w.take<char>((int64_t)c.staging_bytes);
  c.ws_bytes = w.off + kAlign;
}

struct Plan {
  std::vector<InstDev> inst;
  int64_t n = 0, n_cells = 0, total_chunks = 0;
  int32_t cap = 160;
  int32_t skin_cap = 0;          // slots of the mixed form's reused lists
  int32_t precision = SPH_FP64;
  bool any_filter = false;       // some instance uses the pressure filter
};

sph_status plan(int32_t n_inst, const sph_params* params, const int64_t* counts, Plan& pl) {
  if (n_inst < 1 || n_inst > kMaxInst || !params || !counts) return SPH_ERR_ARG;
  pl.inst.resize(n_inst);
  pl.precision = params[0].precision;
  pl.cap = params[0].nbr_cap ? params[0].nbr_cap : 160;
  if (pl.cap < 64 || pl.cap > 1024 || pl.cap % kNbrGroup) return SPH_ERR_ARG;
  int64_t pb = 0, cb = 0, kb = 0;
  for (int32_t k = 0; k < n_inst; ++k) {
    if (params[k].precision != pl.precision) return SPH_ERR_ARG;
    if ((params[k].nbr_cap ? params[k].nbr_cap : 160) != pl.cap) return SPH_ERR_ARG;
    if (counts[k] < 1) return SPH_ERR_ARG;
    sph_status st = derive(params[k], pl.inst[k]);
    if (st != SPH_OK) return st;
    if (params[k].flags & SPH_PFILTER) pl.any_filter = true;
    InstDev& d = pl.inst[k];
    d.cell_base = cb;
    d.p_begin = pb;
    d.p_end = pb + counts[k];
    d.chunk_base = kb;
    d.n_chunks = (counts[k] + kStateChunk - 1) / kStateChunk;
    cb += (int64_t)d.nx * d.ny * d.nz * d.slabs;
    pb += counts[k];
    kb += d.n_chunks;
  }
  if (pb > kMaxParticles || cb >= (int64_t)0xFFFFFFF0ll) return SPH_ERR_GRID_OVERFLOW;
  // the reused lists hold the pairs within 2h + skin: the capacity of the
  // exact lists scaled by the volume ratio of the two spheres, in groups of 8
  if (pl.precision == SPH_MIXED) {
    double ratio = 1.0;
    for (const InstDev& d : pl.inst) {
      const double q = (2.0 * d.h + d.skin) / (2.0 * d.h);
      ratio = std::max(ratio, q * q * q);
    }
    pl.skin_cap = (int32_t)(ceil(pl.cap * ratio / kNbrGroup) * kNbrGroup);
  }
  pl.n = pb;
  pl.n_cells = cb;
  pl.total_chunks = kb;
  return SPH_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define CK(x)                                       \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return SPH_ERR_CUDA;     \
  } while (0)

sph_status decode_err(uint32_t e) {
  if (e & ERR_NONFINITE) return SPH_ERR_NONFINITE;
  if (e & ERR_ESCAPED) return SPH_ERR_ESCAPED;
  if (e & ERR_NEIGHBORS) return SPH_ERR_NEIGHBORS;
  if (e & ERR_TIMEOUT) return SPH_ERR_TIMEOUT;
  if (e & ERR_BOUNDS) return SPH_ERR_BOUNDS;
  return SPH_OK;
}

// ---- pipeline pieces (enqueue only) -----------------------------------------

// Optional stage markers: an event is recorded before each stage and after
// the last one, so that consecutive events bracket one stage.
struct Marks {
  cudaEvent_t* ev = nullptr;
  int k = 0;
};

inline void mark(Marks* m, cudaStream_t s) {
  if (m) cudaEventRecord(m->ev[m->k++], s);
}

constexpr int kStages = 10;
const char* const kStageNames[kStages] = {
    "kick_drift_keys", "cell_scan", "scatter_cell_sort", "reorder", "cell_search",
    "density",         "pressure_filter", "forces",      "kick",    "wall_torque"};

bool mixed(const sph_ctx* c) { return c->precision == SPH_MIXED; }

// FP64 form: kick + drift (mode 1) or wall placement (mode 0) with the cell
// keys, scan, scatter and cell sort, and the reorder into the other buffer.
sph_status enqueue_cells(sph_ctx* c, cudaStream_t s, int mode, int* launches,
                         Marks* m = nullptr) {
  const int a = c->cur, b = 1 - c->cur;
  mark(m, s);
  CK(cudaMemsetAsync(c->cw.count, 0, sizeof(uint32_t) * (size_t)c->cw.n_cells, s));
  CK(launch_kick_drift_fp64(c->n, c->buf[a], c->f, c->inst, c->ist, c->cw, c->err, mode, s,
                            c->lc, launches));
  mark(m, s);
  CK(launch_scan(c->cw, s, c->lc, launches));
  mark(m, s);
  CK(launch_scatter_sort(c->cw, c->buf[a].id, c->n, s, c->lc, launches));
  mark(m, s);
  CK(launch_reorder_fp64(c->n, c->buf[a], c->buf[b], c->cw, c->nw, s, c->lc, launches));
  return SPH_OK;
}

// Neighbour search: the FP64 form's prefilter on the rounded positions; the
// mixed form's list-build test on the offsets of the last build (gate: only
// the instances that rebuild in this step; null: all).
sph_status enqueue_search(sph_ctx* c, cudaStream_t s, int* launches,
                          const InstState* gate = nullptr) {
  const float4* rec = mixed(c) ? c->mf.oref : c->nw.posf;
  const uint32_t* inst_of = mixed(c) ? c->mbuf[c->cur].inst : c->buf[c->cur].inst;
  CK(launch_cell_search(mixed(c), c->n, rec, inst_of, c->inst, c->n_inst, c->max_cells, c->cw,
                        c->nw, c->err, s, c->lc, launches, gate));
  return SPH_OK;
}

// Mixed form: the gated list build of a step after the drift (keys, scan,
// scatter and cell sort, reorder and copy-back, then per instance the search
// and the compaction into the reused lists), and the gate closed.
sph_status enqueue_build_mixed(sph_ctx* c, cudaStream_t s, int mode, int* launches,
                               Marks* m = nullptr) {
  const uint32_t* gate = c->err + kErrRebuild;
  CK(launch_keys_mixed(c->n, c->mbuf[0], c->inst, c->ist, c->cw, c->err, mode, s, c->lc,
                       launches));
  mark(m, s);
  CK(launch_scan(c->cw, s, c->lc, launches, gate));
  mark(m, s);
  CK(launch_scatter_sort(c->cw, c->mbuf[0].id, c->n, s, c->lc, launches, gate));
  mark(m, s);
  CK(launch_reorder_mixed(c->n, c->mbuf[0], c->mbuf[1], c->cw, gate, s, c->lc, launches));
  CK(launch_copyback_mixed(c->n, c->mbuf[1], c->mbuf[0], c->mf, c->ist, gate, s, c->lc,
                           launches));
  mark(m, s);
  sph_status st = enqueue_search(c, s, launches, c->ist);
  if (st != SPH_OK) return st;
  CK(launch_skin_list_mixed(c->n, c->mbuf[0], c->inst, c->ist, c->cw, c->nw, c->err, 1, s,
                            c->lc, launches));
  CK(launch_gate(false, c->n_inst, c->inst, c->ist, c->err, mode, s, launches));
  c->skin_valid = true;
  return SPH_OK;
}

// Mixed form: a build of every instance's lists at the current positions
// (initial evaluation, a standalone cell build): walls placed at the current
// phase, no kick or drift.
sph_status enqueue_forced_build_mixed(sph_ctx* c, cudaStream_t s, int* launches) {
  CK(launch_gate(true, c->n_inst, c->inst, c->ist, c->err, 0, s, launches));
  CK(launch_drift_mixed(c->n, c->mbuf[0], c->mf, c->inst, c->ist, c->err, 0, s, c->lc,
                        launches));
  return enqueue_build_mixed(c, s, 0, launches);
}

// Mixed form: the reused lists again from the cells and the offsets of the
// last build, in the stored order (after a checkpoint load, whose workspace
// holds none): the same masks and so the same lists as at that build.
sph_status enqueue_relist_mixed(sph_ctx* c, cudaStream_t s) {
  CK(cudaMemsetAsync(c->cw.count, 0, sizeof(uint32_t) * (size_t)c->cw.n_cells, s));
  CK(launch_relist_keys_mixed(c->n, c->mbuf[0], c->mf, c->inst, c->cw, s, c->lc));
  CK(launch_scan(c->cw, s, c->lc, nullptr));
  sph_status st = enqueue_search(c, s, nullptr);
  if (st != SPH_OK) return st;
  CK(launch_skin_list_mixed(c->n, c->mbuf[0], c->inst, c->ist, c->cw, c->nw, c->err, 0, s,
                            c->lc, nullptr));
  c->skin_valid = true;
  return SPH_OK;
}

sph_status enqueue_density_only(sph_ctx* c, cudaStream_t s, int* launches) {
  if (mixed(c))
    CK(launch_density_mixed(c->n, c->mbuf[c->cur], c->mf, c->inst, c->nw, c->err, s, c->lc,
                            launches));
  else
    CK(launch_density_fp64(c->n, c->buf[c->cur], c->f, c->inst, c->cw, c->nw, c->err, s,
                           c->lc, launches));
  return SPH_OK;
}

// Pressure filter of the instances that enable it (nothing if none does).
sph_status enqueue_pfilter(sph_ctx* c, cudaStream_t s, int* launches) {
  if (!c->lc.any_filter) return SPH_OK;
  if (mixed(c))
    CK(launch_pfilter_mixed(c->n, c->mbuf[c->cur], c->mf, c->inst, c->nw, c->err, s, launches));
  else
    CK(launch_pfilter_fp64(c->n, c->buf[c->cur], c->f, c->inst, c->nw, c->err, s, launches));
  return SPH_OK;
}

// Neighbour search (FP64 form; the mixed form searches in its list builds
// and reuses the lists, rebuilt first if a checkpoint load dropped them),
// then density and pressure, then the pressure filter.
sph_status enqueue_density(sph_ctx* c, cudaStream_t s, int* launches, Marks* m = nullptr) {
  sph_status st = SPH_OK;
  if (!mixed(c)) {
    mark(m, s);
    st = enqueue_search(c, s, launches);
  } else if (!c->skin_valid) {
    st = enqueue_relist_mixed(c, s);
  }
  if (st != SPH_OK) return st;
  mark(m, s);
  st = enqueue_density_only(c, s, launches);
  if (st != SPH_OK) return st;
  mark(m, s);
  st = enqueue_pfilter(c, s, launches);
  if (st != SPH_OK) return st;
  c->lists_valid = true;
  return SPH_OK;
}

// advance: a step's pair pass (then the closing half kick, unless kick is
// false, and the wall phase advanced); 0: an evaluation at the current state.
sph_status enqueue_forces(sph_ctx* c, cudaStream_t s, int advance, int* launches,
                          Marks* m = nullptr, bool kick = true) {
  const int k = c->cur;
  mark(m, s);
  if (mixed(c))
    CK(launch_forces_mixed(c->n, c->mbuf[k], c->mf, c->inst, c->nw, c->err, s, c->lc,
                           launches));
  else
    CK(launch_forces_fp64(c->n, c->buf[k], c->f, c->inst, c->cw, c->nw, c->err, s, c->lc,
                          launches));
  mark(m, s);
  if (advance && kick) {
    if (mixed(c))
      CK(launch_kick_mixed(c->n, c->mbuf[k], c->mf, c->inst, s, c->lc, launches));
    else
      CK(launch_kick_fp64(c->n, c->buf[k], c->f, c->inst, s, c->lc, launches));
  }
  mark(m, s);
  if (mixed(c))
    CK(launch_wall_torque_mixed(c->n_inst, c->total_chunks, c->inst, c->ist, c->mbuf[k], c->mf,
                                c->part_tw, advance, s, launches));
  else
    CK(launch_wall_torque_fp64(c->n_inst, c->total_chunks, c->inst, c->ist, c->buf[k], c->f,
                               c->part_tw, advance, s, launches));
  mark(m, s);
  return SPH_OK;
}

// One kick-drift-kick step.  FP64 form: flips c->cur (the reorder target
// becomes current).  Mixed form: the drift, the gated list build, then the
// passes over the reused lists; c->cur stays 0.  The mixed step leaves its
// closing half kick out: the next step's drift applies it first (fused_kick)
// or enqueue_closing_kick does, so a run of steps passes over the velocities
// once per step with the same bits as separate kicks.
sph_status enqueue_step(sph_ctx* c, cudaStream_t s, int* launches, Marks* m = nullptr,
                        bool fused_kick = false) {
  sph_status st;
  if (mixed(c)) {
    mark(m, s);
    CK(launch_drift_mixed(c->n, c->mbuf[0], c->mf, c->inst, c->ist, c->err, fused_kick ? 2 : 1, s,
                          c->lc, launches));
    st = enqueue_build_mixed(c, s, 1, launches, m);
  } else {
    st = enqueue_cells(c, s, 1, launches, m);
    c->cur = 1 - c->cur;
  }
  if (st != SPH_OK) return st;
  st = enqueue_density(c, s, launches, m);
  if (st != SPH_OK) return st;
  return enqueue_forces(c, s, 1, launches, m, !mixed(c));
}

// The closing half kick of the last step of a run (mixed form).
sph_status enqueue_closing_kick(sph_ctx* c, cudaStream_t s, int* launches) {
  CK(launch_kick_mixed(c->n, c->mbuf[0], c->mf, c->inst, s, c->lc, launches));
  return SPH_OK;
}

// FP64 form: one graph per starting buffer.  Mixed form: graph[0] the first
// step of a run, graph[1] a later one (its drift applies the previous step's
// closing half kick); sph_step adds the last step's closing kick.
sph_status capture_graphs(sph_ctx* c) {
  const int saved = c->cur;
  for (int g = 0; g < 2; ++g) {
    c->cur = mixed(c) ? 0 : (saved + g) & 1;
    const int start_cur = mixed(c) ? g : c->cur;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    sph_status st = enqueue_step(c, c->cap_stream, &launches, nullptr, mixed(c) && g == 1);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st != SPH_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      c->cur = saved;
      return st != SPH_OK ? st : SPH_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->cur = saved;
      return SPH_ERR_CUDA;
    }
    c->graph[start_cur] = exec;
    // launches of sph_step(ctx, 1) (mixed form: with its closing kick)
    c->launches_per_step = launches + (mixed(c) ? 1 : 0);
  }
  c->cur = saved;
  return SPH_OK;
}

}  // namespace

extern "C" {

const char* sph_status_string(sph_status s) {
  switch (s) {
    case SPH_OK: return "ok";
    case SPH_ERR_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA runtime error";
    case SPH_ERR_WORKSPACE: return "state or workspace buffer too small or misaligned";
    case SPH_ERR_GRID_OVERFLOW: return "cell grid or particle count too large";
    case SPH_ERR_ESCAPED: return "a particle left the cell grid";
    case SPH_ERR_NONFINITE: return "non-finite value in the state";
    case SPH_ERR_TIMEOUT: return "a bounded device wait gave up";
    case SPH_ERR_STATE: return "call out of order";
    case SPH_ERR_NEIGHBORS: return "neighbour list overflow (raise nbr_cap)";
    case SPH_ERR_BOUNDS: return "an index failed a bounds check (checked build)";
  }
  return "unknown status";
}

sph_status sph_params_default(sph_params* p, double R, double H, double Omega) {
  if (!p || !(R > 0) || !(H > 0) || !(Omega > 0)) return SPH_ERR_ARG;
  memset(p, 0, sizeof *p);
  const double dx = 1.0, h = 1.3 * dx, rho0 = 1.0, gamma = 7.0;
  const double cs = 10.0 * Omega * R;
  p->dx = dx;
  p->h = h;
  p->rho0 = rho0;
  p->alpha_P = gamma;
  p->p0 = rho0 * cs * cs / gamma;
  p->beta_P = p->p0;
  p->eta_bar = rho0 * Omega * R * R / 100.0;
  p->eta_r = p->eta_bar;
  p->C_l = 1e-3 * rho0 * Omega;
  p->C_T = 0.01 * p->p0;
  p->C_omega = 0.016;
  p->mass_ratio = 1.0;
  p->inertia_coef = 0.1;
  p->Omega = Omega;
  p->dt = 0.25 * h / cs;
  const double ext = R + 2.0 * dx + 2.0 * h;
  p->box_lo[0] = p->box_lo[1] = -ext;
  p->box_hi[0] = p->box_hi[1] = ext;
  p->box_lo[2] = 0.0;
  p->box_hi[2] = H;
  p->periodic_z = 1;
  p->precision = SPH_FP64;
  p->flags = SPH_FLAGS_DEFAULT;
  p->nbr_cap = 160;
  p->col_dist = 0.8 * dx;
  p->col_e = 0.2;
  return SPH_OK;
}

size_t sph_state_bytes(int32_t n_inst, const sph_params* params, const int64_t* counts) {
  Plan pl;
  if (plan(n_inst, params, counts, pl) != SPH_OK) return 0;
  Carved c;
  carve(nullptr, nullptr, n_inst, pl.n, pl.n_cells, pl.total_chunks, pl.cap, pl.skin_cap,
        pl.precision, pl.any_filter, c);
  return c.state_bytes;
}

size_t sph_workspace_bytes(int32_t n_inst, const sph_params* params, const int64_t* counts) {
  Plan pl;
  if (plan(n_inst, params, counts, pl) != SPH_OK) return 0;
  Carved c;
  carve(nullptr, nullptr, n_inst, pl.n, pl.n_cells, pl.total_chunks, pl.cap, pl.skin_cap,
        pl.precision, pl.any_filter, c);
  return c.ws_bytes;
}

sph_status sph_init_batch(sph_ctx** out, int32_t n_inst, const sph_params* params,
                          const int64_t* counts, const double* pos, const double* vel,
                          const double* spin, const uint8_t* species, void* dev_state,
                          size_t state_bytes, void* dev_workspace, size_t workspace_bytes,
                          void* stream) {
  NvtxRange range("sph_init");
  if (!out) return SPH_ERR_ARG;
  *out = nullptr;
  if (!pos || !vel || !spin || !species || !dev_state || !dev_workspace) return SPH_ERR_ARG;
  Plan pl;
  sph_status st = plan(n_inst, params, counts, pl);
  if (st != SPH_OK) return st;
  if (((uintptr_t)dev_state % kAlign) || ((uintptr_t)dev_workspace % kAlign))
    return SPH_ERR_WORKSPACE;
  Carved cv;
  carve(dev_state, dev_workspace, n_inst, pl.n, pl.n_cells, pl.total_chunks, pl.cap,
        pl.skin_cap, pl.precision, pl.any_filter, cv);
  if (state_bytes < cv.state_bytes || workspace_bytes < cv.ws_bytes) return SPH_ERR_WORKSPACE;

  sph_ctx* c = new (std::nothrow) sph_ctx();
  if (!c) return SPH_ERR_ARG;
  c->n_inst = n_inst;
  c->n = pl.n;
  c->precision = pl.precision;
  c->cap = pl.cap;
  c->inst_h = pl.inst;
  c->inst = cv.inst;
  c->ist = cv.ist;
  c->err = cv.err;
  c->buf[0] = cv.buf[0];
  c->buf[1] = cv.buf[1];
  c->f = cv.f;
  c->mbuf[0] = cv.mbuf[0];
  c->mbuf[1] = cv.mbuf[1];
  c->mf = cv.mf;
  c->cw = cv.cw;
  c->nw = cv.nw;
  c->total_chunks = pl.total_chunks;
  c->part_tw = cv.part_tw;
  c->part_diag = cv.part_diag;
  c->diag_out = cv.diag_out;
  c->backup = cv.backup;
  c->staging = cv.staging;
  c->staging_bytes = cv.staging_bytes;
  c->state = dev_state;
  c->state_bytes = cv.state_bytes;
  c->stream = (cudaStream_t)stream;
  int dev = 0;
  auto fail = [&](sph_status s) {
    sph_destroy(c);
    return s;
  };
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPH_ERR_CUDA);
  if (cudaDeviceGetAttribute(&c->lc.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SPH_ERR_CUDA);
  c->lc.block_density = 128;
  c->lc.block_forces = 128;
  c->lc.search_warps = 4;
  c->lc.search_depth = 512;
  c->lc.any_literal = false;
  c->lc.any_collision = false;
  c->lc.any_filter = false;
  for (const InstDev& d : pl.inst) {
    c->max_cells = std::max(c->max_cells, (int64_t)d.nx * d.ny * d.nz);
    if (d.flags & SPH_SN_LITERAL) c->lc.any_literal = true;
    if (d.flags & SPH_COLLISION) c->lc.any_collision = true;
    if (d.flags & SPH_PFILTER) c->lc.any_filter = true;
  }
  {
    static std::once_flag once;
    static cudaError_t prep = cudaSuccess;
    std::call_once(once, [] { prep = prepare_search_kernels(); });
    if (prep != cudaSuccess) return fail(SPH_ERR_CUDA);
  }
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(SPH_ERR_CUDA);

  cudaStream_t s = c->stream;
  const int64_t n = pl.n;
  // inputs: device pointers are used in place, host pointers go through the
  // staging area
  char* stg = (char*)c->staging;
  size_t off = 0;
  auto stage = [&](const void* src, size_t bytes, const void** dst) -> sph_status {
    off = (off + kAlign - 1) / kAlign * kAlign;
    if (off + bytes > c->staging_bytes) return SPH_ERR_WORKSPACE;
    if (is_device_ptr(src)) {
      *dst = src;
      return SPH_OK;
    }
    if (cudaMemcpyAsync(stg + off, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return SPH_ERR_CUDA;
    *dst = stg + off;
    off += bytes;
    return SPH_OK;
  };
  const void *dpos, *dvel, *dspin, *dsp;
  if ((st = stage(pos, sizeof(double) * 3 * n, &dpos)) != SPH_OK) return fail(st);
  if ((st = stage(vel, sizeof(double) * 3 * n, &dvel)) != SPH_OK) return fail(st);
  if ((st = stage(spin, sizeof(double) * 3 * n, &dspin)) != SPH_OK) return fail(st);
  if ((st = stage(species, (size_t)n, &dsp)) != SPH_OK) return fail(st);
  if (cudaMemcpyAsync(c->inst, pl.inst.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return fail(SPH_ERR_CUDA);
  if (cudaMemsetAsync(c->ist, 0, sizeof(InstState) * n_inst, s) != cudaSuccess ||
      cudaMemsetAsync(c->err, 0, sizeof(uint32_t) * 4, s) != cudaSuccess)
    return fail(SPH_ERR_CUDA);
  cudaError_t le;
  if (mixed(c))
    le = launch_load_mixed(n, c->mbuf[0], c->inst, n_inst, (const double*)dpos,
                           (const double*)dvel, (const double*)dspin, (const uint8_t*)dsp, c->err,
                           s, c->lc);
  else
    le = launch_load_fp64(n, c->buf[0], (const double*)dpos, (const double*)dvel,
                          (const double*)dspin, (const uint8_t*)dsp, c->inst, n_inst, s, c->lc);
  if (le != cudaSuccess) return fail(SPH_ERR_CUDA);
  c->cur = 0;
  // initial evaluation: walls at phase 0, cells, density, forces (a_0, alpha_0)
  if (mixed(c)) {
    if (cudaMemsetAsync(c->mf.oref, 0, sizeof(float4) * (size_t)n, s) != cudaSuccess ||
        cudaMemsetAsync(c->cw.count, 0, sizeof(uint32_t) * (size_t)c->cw.n_cells, s) !=
            cudaSuccess)
      return fail(SPH_ERR_CUDA);
    if ((st = enqueue_forced_build_mixed(c, s, nullptr)) != SPH_OK) return fail(st);
  } else {
    if ((st = enqueue_cells(c, s, 0, nullptr)) != SPH_OK) return fail(st);
    c->cur = 1;
  }
  if ((st = enqueue_density(c, s, nullptr)) != SPH_OK) return fail(st);
  if ((st = enqueue_forces(c, s, 0, nullptr)) != SPH_OK) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(SPH_ERR_CUDA);
  c->forces_valid = true;
  uint32_t e = 0;
  if (cudaMemcpy(&e, c->err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(SPH_ERR_CUDA);
  if (e) return fail(decode_err(e));
  *out = c;
  return SPH_OK;
}

sph_status sph_init(sph_ctx** ctx, const sph_params* params, int64_t n, const double* pos,
                    const double* vel, const double* spin, const uint8_t* species,
                    void* dev_state, size_t state_bytes, void* dev_workspace,
                    size_t workspace_bytes, void* stream) {
  return sph_init_batch(ctx, 1, params, &n, pos, vel, spin, species, dev_state, state_bytes,
                        dev_workspace, workspace_bytes, stream);
}

sph_status sph_build_cells(sph_ctx* c) {
  NvtxRange range("sph_build_cells");
  if (!c) return SPH_ERR_ARG;
  sph_status st;
  if (mixed(c)) {  // the mixed form builds its reused lists with the cells
    st = enqueue_forced_build_mixed(c, c->stream, nullptr);
  } else {
    st = enqueue_cells(c, c->stream, 0, nullptr);
    c->cur = 1 - c->cur;
  }
  if (st != SPH_OK) return st;
  c->forces_valid = false;
  c->lists_valid = false;
  return SPH_OK;
}

sph_status sph_density(sph_ctx* c) {
  NvtxRange range("sph_density");
  if (!c) return SPH_ERR_ARG;
  return enqueue_density(c, c->stream, nullptr);
}

sph_status sph_forces(sph_ctx* c) {
  NvtxRange range("sph_forces");
  if (!c) return SPH_ERR_ARG;
  if (!c->lists_valid) return SPH_ERR_STATE;  // needs sph_density first
  sph_status st = enqueue_forces(c, c->stream, 0, nullptr);
  if (st == SPH_OK) c->forces_valid = true;
  return st;
}

sph_status sph_step(sph_ctx* c, int32_t nsteps) {
  NvtxRange range("sph_step");
  if (!c || nsteps < 0) return SPH_ERR_ARG;
  if (nsteps == 0) return SPH_OK;
  if (!c->forces_valid) {
    // a standalone cell build reordered the particles: re-evaluate a and alpha
    sph_status st = enqueue_density(c, c->stream, nullptr);
    if (st == SPH_OK) st = enqueue_forces(c, c->stream, 0, nullptr);
    if (st != SPH_OK) return st;
    c->forces_valid = true;
  }
  if (mixed(c) && !c->skin_valid) {  // a checkpoint load dropped the reused lists
    sph_status st = enqueue_relist_mixed(c, c->stream);
    if (st != SPH_OK) return st;
  }
  if (!c->graph[0]) {
    sph_status st = capture_graphs(c);
    if (st != SPH_OK) return st;
  }
  if (mixed(c)) {  // one state buffer; the closing half kick fused into the next step
    for (int32_t t = 0; t < nsteps; ++t) CK(cudaGraphLaunch(c->graph[t ? 1 : 0], c->stream));
    return enqueue_closing_kick(c, c->stream, nullptr);
  }
  for (int32_t t = 0; t < nsteps; ++t) {
    CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
    c->cur = 1 - c->cur;
  }
  return SPH_OK;
}

sph_status sph_check(sph_ctx* c) {
  if (!c) return SPH_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  uint32_t e = 0;
  CK(cudaMemcpy(&e, c->err, sizeof e, cudaMemcpyDeviceToHost));
  return decode_err(e);
}

sph_status sph_force_breakdown(sph_ctx* c, int32_t inst, double out[5]) {
  if (!c || !out || inst < 0 || inst >= c->n_inst) return SPH_ERR_ARG;
  if (!c->lists_valid) return SPH_ERR_STATE;  // needs the lists of a density pass
  if (mixed(c))
    CK(launch_breakdown_mixed(c->n_inst, c->n, c->total_chunks, c->inst, c->mbuf[c->cur], c->mf,
                              c->nw, c->part_diag, c->diag_out, c->stream));
  else
    CK(launch_breakdown_fp64(c->n_inst, c->n, c->total_chunks, c->inst, c->buf[c->cur], c->f,
                             c->nw, c->part_diag, c->diag_out, c->stream));
  CK(cudaMemcpyAsync(out, c->diag_out + (int64_t)inst * kDiagFields, sizeof(double) * 5,
                     cudaMemcpyDeviceToHost, c->stream));
  return sph_check(c);
}

sph_status sph_pair_census(sph_ctx* c, int32_t inst, int64_t out[5]) {
  if (!c || !out || inst < 0 || inst >= c->n_inst) return SPH_ERR_ARG;
  if (!c->lists_valid) return SPH_ERR_STATE;  // needs the lists of a density pass
  if (mixed(c))
    CK(launch_census_mixed(c->n_inst, c->n, c->total_chunks, c->inst, c->mbuf[c->cur], c->mf,
                           c->nw, c->part_diag, c->diag_out, c->stream));
  else
    CK(launch_census_fp64(c->n_inst, c->n, c->total_chunks, c->inst, c->buf[c->cur], c->f, c->nw,
                          c->part_diag, c->diag_out, c->stream));
  double d[5];
  CK(cudaMemcpyAsync(d, c->diag_out + (int64_t)inst * kDiagFields, sizeof d,
                     cudaMemcpyDeviceToHost, c->stream));
  const sph_status st = sph_check(c);
  for (int q = 0; q < 5; ++q) out[q] = (int64_t)d[q];
  return st;
}

sph_status sph_diagnostics(sph_ctx* c, int32_t inst, sph_diag* out) {
  NvtxRange range("sph_diagnostics");
  if (!c || !out || inst < 0 || inst >= c->n_inst) return SPH_ERR_ARG;
  if (mixed(c))
    CK(launch_diag_mixed(c->n_inst, c->total_chunks, c->inst, c->mbuf[c->cur], c->mf, c->nw,
                         c->part_diag, c->diag_out, c->stream));
  else
    CK(launch_diag_fp64(c->n_inst, c->total_chunks, c->inst, c->buf[c->cur], c->f, c->nw,
                        c->part_diag, c->diag_out, c->stream));
  double d[kDiagFields];
  InstState s;
  CK(cudaMemcpyAsync(d, c->diag_out + (int64_t)inst * kDiagFields, sizeof d,
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&s, c->ist + inst, sizeof s, cudaMemcpyDeviceToHost, c->stream));
  sph_status st = sph_check(c);
  memset(out, 0, sizeof *out);
  out->mass = d[0];
  out->mass_s = d[1];
  out->mass_n = d[2];
  for (int a = 0; a < 3; ++a) {
    out->mom[a] = d[3 + a];
    out->L_orb[a] = d[6 + a];
    out->L_spin[a] = d[9 + a];
    out->T_wall[a] = s.T_wall[a];
    out->J_wall[a] = s.J_wall[a];
  }
  out->E_kin = d[12];
  out->E_rot = d[13];
  out->E_int = d[14];
  out->n_pairs = (int64_t)d[15];
  out->rho_min = d[16];
  out->rho_max = d[17];
  out->v_max = d[18];
  out->step = s.step;
  out->theta = s.theta;
  return st;
}

}  // extern "C"

namespace {

// Checkpoint header; the verbatim state buffer follows it.
struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t precision;
  int32_t n_inst;
  int32_t cur;
  int64_t n;
  uint64_t state_bytes;
  uint64_t inst_bytes;     // InstDev array at the start of the state buffer
  uint64_t forces_valid;   // the stored accelerations belong to the stored order
  uint64_t reserved[2];
};
constexpr char kCkptMagic[8] = {'S', 'P', 'H', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 2;  // 2: mixed velocity and spin in one record

}  // namespace

extern "C" {

size_t sph_checkpoint_bytes(const sph_ctx* c) {
  return c ? sizeof(CkptHeader) + c->state_bytes : 0;
}

sph_status sph_save_checkpoint(sph_ctx* c, void* buf, size_t bytes) {
  NvtxRange range("sph_save_checkpoint");
  if (!c || !buf || bytes < sph_checkpoint_bytes(c)) return SPH_ERR_ARG;
  sph_status st = sph_check(c);  // synchronises; a latched error is not saved
  if (st != SPH_OK) return st;
  CkptHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kCkptMagic, sizeof h.magic);
  h.version = kCkptVersion;
  h.precision = c->precision;
  h.n_inst = c->n_inst;
  h.cur = c->cur;
  h.n = c->n;
  h.state_bytes = c->state_bytes;
  h.inst_bytes = sizeof(InstDev) * (uint64_t)c->n_inst;
  h.forces_valid = c->forces_valid ? 1u : 0u;
  char* out = static_cast<char*>(buf);
  CK(cudaMemcpyAsync(out, &h, sizeof h, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(out + sizeof h, c->state, c->state_bytes, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SPH_OK;
}

sph_status sph_load_checkpoint(sph_ctx* c, const void* buf, size_t bytes) {
  NvtxRange range("sph_load_checkpoint");
  if (!c || !buf || bytes < sph_checkpoint_bytes(c)) return SPH_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  const char* in = static_cast<const char*>(buf);
  CkptHeader h;
  CK(cudaMemcpy(&h, in, sizeof h, cudaMemcpyDefault));
  if (memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0 || h.version != kCkptVersion ||
      h.precision != c->precision || h.n_inst != c->n_inst || h.n != c->n ||
      h.state_bytes != c->state_bytes || (h.cur != 0 && h.cur != 1) ||
      h.inst_bytes != sizeof(InstDev) * (uint64_t)c->n_inst ||
      (const char*)c->inst != (const char*)c->state)
    return SPH_ERR_ARG;
  // the instance constants (derived from the parameters and counts) must match
  std::vector<InstDev> saved((size_t)c->n_inst);
  CK(cudaMemcpy(saved.data(), in + sizeof h, h.inst_bytes, cudaMemcpyDefault));
  if (memcmp(saved.data(), c->inst_h.data(), h.inst_bytes) != 0) return SPH_ERR_ARG;
  CK(cudaMemcpyAsync(c->state, in + sizeof h, c->state_bytes, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->cur = h.cur;
  c->forces_valid = h.forces_valid != 0;  // the accelerations came with the state
  c->lists_valid = false;                 // neighbour lists live in the workspace
  c->skin_valid = false;                  // so do the mixed form's reused lists
  return sph_check(c);
}

sph_status sph_get_state(sph_ctx* c, double* pos, double* vel, double* spin, double* rho,
                         double* P, double* acc, double* dspin) {
  if (!c) return SPH_ERR_ARG;
  const int64_t n = c->n;
  double* outs[7] = {pos, vel, spin, rho, P, acc, dspin};
  const int width[7] = {3, 3, 3, 1, 1, 3, 3};
  double* dev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t off = 0;
  char* stg = (char*)c->staging;
  for (int k = 0; k < 7; ++k) {
    if (!outs[k]) continue;
    if (is_device_ptr(outs[k])) {
      dev[k] = outs[k];
    } else {
      const size_t bytes = sizeof(double) * (size_t)width[k] * (size_t)n;
      off = (off + kAlign - 1) / kAlign * kAlign;
      if (off + bytes > c->staging_bytes) return SPH_ERR_WORKSPACE;
      dev[k] = (double*)(stg + off);
      off += bytes;
    }
  }
  if (mixed(c))
    CK(launch_unsort_mixed(n, c->mbuf[c->cur], c->mf, c->inst, dev[0], dev[1], dev[2], dev[3],
                           dev[4], dev[5], dev[6], c->stream, c->lc));
  else
    CK(launch_unsort_fp64(n, c->buf[c->cur], c->f, dev[0], dev[1], dev[2], dev[3], dev[4],
                          dev[5], dev[6], c->stream, c->lc));
  for (int k = 0; k < 7; ++k)
    if (outs[k] && dev[k] != outs[k])
      CK(cudaMemcpyAsync(outs[k], dev[k], sizeof(double) * (size_t)width[k] * (size_t)n,
                         cudaMemcpyDeviceToHost, c->stream));
  return sph_check(c);
}

sph_status sph_get_neighbors(sph_ctx* c, int64_t* offsets, int64_t* nbr, int64_t cap) {
  if (!c || !offsets) return SPH_ERR_ARG;
  if (!c->lists_valid) return SPH_ERR_STATE;
  const int64_t n = c->n;
  std::vector<uint32_t> cnt((size_t)n), id((size_t)n), list((size_t)c->cap * (size_t)n);
  CK(cudaMemcpyAsync(cnt.data(), c->nw.count, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(id.data(), mixed(c) ? c->mbuf[c->cur].id : c->buf[c->cur].id,
                     sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(list.data(), c->nw.list, sizeof(uint32_t) * list.size(),
                     cudaMemcpyDeviceToHost, c->stream));
  sph_status st = sph_check(c);
  std::vector<int64_t> where((size_t)n);
  for (int64_t k = 0; k < n; ++k) where[id[k]] = k;
  int64_t tot = 0;
  for (int64_t o = 0; o < n; ++o) {
    offsets[o] = tot;
    tot += cnt[(size_t)where[o]];
  }
  offsets[n] = tot;
  if (!nbr || cap < tot) return st != SPH_OK ? st : SPH_ERR_ARG;
  std::vector<int64_t> tmp;
  for (int64_t o = 0; o < n; ++o) {
    const int64_t k = where[o];
    tmp.clear();
    for (uint32_t t = 0; t < cnt[(size_t)k]; ++t)
      tmp.push_back(id[list[(size_t)nbr_slot(n, k, t)] & kNbrIndexMask]);
    std::sort(tmp.begin(), tmp.end());
    for (size_t t = 0; t < tmp.size(); ++t) nbr[offsets[o] + (int64_t)t] = tmp[t];
  }
  return st;
}

sph_status sph_profile_steps(sph_ctx* c, int32_t nsteps, double* stage_ms, int32_t n_stages) {
  if (!c || nsteps < 1 || !stage_ms || n_stages < kStages) return SPH_ERR_ARG;
  if (!c->forces_valid) {
    sph_status st = enqueue_density(c, c->stream, nullptr);
    if (st == SPH_OK) st = enqueue_forces(c, c->stream, 0, nullptr);
    if (st != SPH_OK) return st;
    c->forces_valid = true;
  }
  std::vector<cudaEvent_t> ev((size_t)nsteps * (kStages + 1), nullptr);
  sph_status st = SPH_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) st = SPH_ERR_CUDA;
  for (int32_t t = 0; t < nsteps && st == SPH_OK; ++t) {
    Marks m;
    m.ev = ev.data() + (size_t)t * (kStages + 1);
    st = enqueue_step(c, c->stream, nullptr, &m, t > 0);
  }
  // (mixed form: the kicks between the steps ran inside the drifts, in the
  // first stage; the last step's closing kick follows, unmeasured)
  if (st == SPH_OK && mixed(c)) st = enqueue_closing_kick(c, c->stream, nullptr);
  if (st == SPH_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = SPH_ERR_CUDA;
  for (int k = 0; k < n_stages; ++k) stage_ms[k] = 0.0;
  for (int32_t t = 0; t < nsteps && st == SPH_OK; ++t)
    for (int k = 0; k < kStages; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[(size_t)t * (kStages + 1) + k],
                               ev[(size_t)t * (kStages + 1) + k + 1]) != cudaSuccess)
        st = SPH_ERR_CUDA;
      stage_ms[k] += ms / nsteps;
    }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (st != SPH_OK) return st;
  return sph_check(c);
}

sph_status sph_autotune(sph_ctx* c, int32_t reps, int32_t* block_density, int32_t* block_forces) {
  if (!c || reps < 1) return SPH_ERR_ARG;
  cudaStream_t s = c->stream;
  // The density pass is a function of the positions alone, so repeating it
  // reproduces the same lists and fields.  The pair pass of a step used the
  // half-step velocities, which are gone after the step: its outputs (acc,
  // dspin, wall torque and the per-instance torque record) are saved first
  // and restored after the trials.
  sph_status st = SPH_OK;
  if (!c->lists_valid) st = enqueue_density(c, s, nullptr);
  if (st != SPH_OK) return st;
  const size_t fb = (size_t)field_bytes(c->precision, c->n);
  void* fields[3];
  if (mixed(c)) {
    fields[0] = c->mf.acc;
    fields[1] = c->mf.dspin;
    fields[2] = c->mf.tw;
  } else {
    fields[0] = c->f.acc;
    fields[1] = c->f.dspin;
    fields[2] = c->f.tw;
  }
  char* bk[4];
  {
    size_t off = 0;
    for (int k = 0; k < 4; ++k) {
      bk[k] = c->backup + off;
      off += ((k < 3 ? fb : sizeof(InstState) * (size_t)c->n_inst) + 255) / 256 * 256;
    }
  }
  for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(bk[k], fields[k], fb, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(bk[3], c->ist, sizeof(InstState) * c->n_inst, cudaMemcpyDeviceToDevice, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SPH_ERR_CUDA;
  }
  const int cand[3] = {64, 128, 256};   // pair pass
  const int dcand[3] = {32, 64, 128};   // density pass
  // neighbour search: warp per cell with 2, 4 or 8 cells per block and a
  // segment depth of 256 or 512 candidates, or (0) thread per particle; all
  // write the same masks and tables
  const int wcand[7] = {2, 4, 8, 2, 4, 8, 0};
  const int scand[7] = {256, 256, 256, 512, 512, 512, 512};
  float best[3] = {INFINITY, INFINITY, INFINITY};
  LaunchCfg pick = c->lc;
  // trials 0-6: mapping and shape of the neighbour search (timed alone);
  // 7-9: density block size (timed with the search before it, which rebuilds
  // the lists it compacts); 10-12: pair-pass block size
  for (int trial = 0; trial < 13 && st == SPH_OK; ++trial) {
    const int kind = trial < 7 ? 0 : (trial < 10 ? 1 : 2);
    const int opt = trial < 7 ? trial : (trial < 10 ? trial - 7 : trial - 10);
    LaunchCfg saved = c->lc;
    if (kind == 0) {
      c->lc.search_warps = wcand[opt];
      c->lc.search_depth = scand[opt];
    }
    if (kind == 1) c->lc.block_density = dcand[opt];
    if (kind == 2) c->lc.block_forces = cand[opt];
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == SPH_OK; ++r) {
      if (kind == 0) st = enqueue_search(c, s, nullptr);
      else if (kind == 1) st = enqueue_density(c, s, nullptr);
      else st = enqueue_forces(c, s, 0, nullptr);
    }
    // (mixed form: the search trials write only the masks and tables of a
    // build, which its lists do not read; its density trials re-test the
    // reused lists, so the trials leave the lists as they were)
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (st == SPH_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = SPH_ERR_CUDA;
    if (ms < best[kind]) {
      best[kind] = ms;
      if (kind == 0) {
        pick.search_warps = c->lc.search_warps;
        pick.search_depth = c->lc.search_depth;
      }
      if (kind == 1) pick.block_density = c->lc.block_density;
      if (kind == 2) pick.block_forces = c->lc.block_forces;
    }
    c->lc = saved;
    // the density trials must see the chosen search shape
    if (kind == 0 && trial == 6) {
      c->lc.search_warps = pick.search_warps;
      c->lc.search_depth = pick.search_depth;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SPH_OK) return st;
  c->lc = pick;
  const int bd = pick.block_density, bf = pick.block_forces;
  // restore the pair-pass outputs, and drop the graphs captured with the old
  // shapes; they are captured again by the next sph_step
  st = enqueue_density(c, s, nullptr);
  if (st != SPH_OK) return st;
  for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(fields[k], bk[k], fb, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->ist, bk[3], sizeof(InstState) * c->n_inst, cudaMemcpyDeviceToDevice, s));
  for (int g = 0; g < 2; ++g)
    if (c->graph[g]) {
      cudaGraphExecDestroy(c->graph[g]);
      c->graph[g] = nullptr;
    }
  if (block_density) *block_density = bd;
  if (block_forces) *block_forces = bf;
  return sph_check(c);
}

sph_status sph_get_launch_config(const sph_ctx* c, int32_t* block_density, int32_t* block_forces,
                                 int32_t* search_warps, int32_t* search_depth) {
  if (!c) return SPH_ERR_ARG;
  if (block_density) *block_density = c->lc.block_density;
  if (block_forces) *block_forces = c->lc.block_forces;
  if (search_warps) *search_warps = c->lc.search_warps;
  if (search_depth) *search_depth = c->lc.search_depth;
  return SPH_OK;
}

int32_t sph_stage_count(void) { return kStages; }

const char* sph_stage_name(int32_t stage) {
  return (stage >= 0 && stage < kStages) ? kStageNames[stage] : "";
}

int32_t sph_launches_per_step(const sph_ctx* c) { return c ? c->launches_per_step : 0; }

sph_status sph_list_builds(sph_ctx* c, int32_t inst, int64_t* builds) {
  if (!c || !builds || inst < 0 || inst >= c->n_inst) return SPH_ERR_ARG;
  InstState st;
  CK(cudaMemcpyAsync(&st, c->ist + inst, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  const sph_status e = sph_check(c);
  // the FP64 form builds its lists at the start and in every step
  *builds = mixed(c) ? (int64_t)st.rebuilds : st.step + 1;
  return e;
}

sph_status sph_set_launch_config(sph_ctx* c, int32_t block_density, int32_t block_forces,
                                 int32_t search_warps, int32_t search_depth) {
  if (!c) return SPH_ERR_ARG;
  const bool bd = block_density == 32 || block_density == 64 || block_density == 128;
  const bool bf = block_forces == 64 || block_forces == 128 || block_forces == 256;
  const bool sw = search_warps == 0 || search_warps == 2 || search_warps == 4 ||
                  search_warps == 8;
  const bool sd = search_depth == 256 || search_depth == 512;
  if (!bd || !bf || !sw || !sd) return SPH_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  c->lc.block_density = block_density;
  c->lc.block_forces = block_forces;
  c->lc.search_warps = search_warps;
  c->lc.search_depth = search_depth;
  for (int g = 0; g < 2; ++g)
    if (c->graph[g]) {
      cudaGraphExecDestroy(c->graph[g]);
      c->graph[g] = nullptr;
    }
  return SPH_OK;
}

sph_status sph_destroy(sph_ctx* c) {
  if (!c) return SPH_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int g = 0; g < 2; ++g)
    if (c->graph[g]) cudaGraphExecDestroy(c->graph[g]);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return SPH_OK;
}

}  // extern "C"
