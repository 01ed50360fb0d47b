// Host-side launchers of the device kernels (one translation unit each).
#pragma once
#include "sph_internal.h"

namespace sphgb {

// Validate one instance's parameters and derive its device constants (cell
// grid, kernel and EOS constants, masses); host only (sph_host.cu).
sph_status derive_instance(const sph_params& p, InstDev& d);

struct LaunchCfg {
  int sm_count;          // multiprocessors of the device
  int block_density;     // threads per block of the density pass (32, 64, 128)
  int block_forces;      // threads per block of the pair pass
  int search_warps;      // warps (cells) per block of the neighbour search; 0: one
                         // thread per particle instead
  int search_depth;      // candidates per staged segment of the warp search (256, 512)
  bool any_literal;      // some instance uses the literal F_sn (SPH_SN_LITERAL)
  bool any_collision;    // some instance uses the collision model (SPH_COLLISION)
  bool any_filter;       // some instance uses the pressure filter (SPH_PFILTER)
};

// ---- cell build (sph_cells.cu) --------------------------------------------
// Exclusive scan of cw.count into cw.start (n_cells + 1 entries); the counts
// are left at zero for the next build.  gate: the kernels do nothing while
// *gate is zero (null: always run).
cudaError_t launch_scan(const CellWs& cw, cudaStream_t s, const LaunchCfg& lc, int* launches,
                        const uint32_t* gate = nullptr);
// perm[start[key[i]] + slot[i]] = i, then sort each cell by particle id.
cudaError_t launch_scatter_sort(const CellWs& cw, const uint32_t* id, int64_t n,
                                cudaStream_t s, const LaunchCfg& lc, int* launches,
                                const uint32_t* gate = nullptr);

// ---- neighbour search (sph_search.cu) ---------------------------------------
// One warp per cell of every instance (grid.y = instance); writes the
// candidate tables and candidate masks of nw, from which the density pass
// builds the neighbour lists.  rec: the per-particle FP32 records (mixed: cell offset
// and species, FP64 form: the rounded position and species).  mixed_form:
// exact FP32 test with cell-displacement codes; otherwise the FP32 prefilter.
// lc.search_warps = 0 selects the thread-per-particle mapping (inst_of: the
// instance of each sorted particle), which writes the same output.
// gate (mixed form): only the instances whose InstState::rebuild is set are
// searched (null: all).  The mixed form's test is r^2 < (2h + skin)^2.
cudaError_t launch_cell_search(bool mixed_form, int64_t n, const float4* rec,
                               const uint32_t* inst_of, const InstDev* inst, int32_t n_inst,
                               int64_t max_cells, const CellWs& cw, const NbrWs& nw,
                               uint32_t* err, cudaStream_t s, const LaunchCfg& lc,
                               int* launches, const InstState* gate = nullptr);
// Raise the dynamic shared-memory limit of the search kernels (once, before
// any launch or stream capture).
cudaError_t prepare_search_kernels();
int search_max_warps();

// ---- FP64 path (sph_fp64.cu) ------------------------------------------------
// mode 0: initial placement (walls at the current phase, no kick/drift);
// mode 1: half kick + drift + wall rotation to the next phase.
cudaError_t launch_kick_drift_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                                   const InstDev* inst, const InstState* ist,
                                   const CellWs& cw, uint32_t* err, int mode,
                                   cudaStream_t s, const LaunchCfg& lc, int* launches);
cudaError_t launch_reorder_fp64(int64_t n, const Fp64Buf& src, const Fp64Buf& dst,
                                const CellWs& cw, const NbrWs& nw, cudaStream_t s,
                                const LaunchCfg& lc, int* launches);
cudaError_t launch_density_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                                const InstDev* inst, const CellWs& cw, const NbrWs& nw,
                                uint32_t* err, cudaStream_t s, const LaunchCfg& lc,
                                int* launches);
// Pressure filter (instances with SPH_PFILTER) over the density pass's lists.
cudaError_t launch_pfilter_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                                const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                cudaStream_t s, int* launches);
cudaError_t launch_forces_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                               const InstDev* inst, const CellWs& cw, const NbrWs& nw,
                               uint32_t* err,
                               cudaStream_t s, const LaunchCfg& lc, int* launches);
cudaError_t launch_kick_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                             const InstDev* inst, cudaStream_t s, const LaunchCfg& lc,
                             int* launches);
// Gather the sorted state back to input order into device arrays (any may be null).
cudaError_t launch_unsort_fp64(int64_t n, const Fp64Buf& b, const Fp64Fields& f,
                               double* pos, double* vel, double* spin, double* rho,
                               double* P, double* acc, double* dspin, cudaStream_t s,
                               const LaunchCfg& lc);
// Scatter AoS input (input order) into the sorted-buffer layout (identity order);
// each particle's instance is found from the instances' particle ranges.
cudaError_t launch_load_fp64(int64_t n, const Fp64Buf& b, const double* pos,
                             const double* vel, const double* spin, const uint8_t* sp,
                             const InstDev* inst, int32_t n_inst, cudaStream_t s,
                             const LaunchCfg& lc);

// ---- mixed-precision path (sph_mixed.cu) -------------------------------------
// The mixed form keeps its neighbour lists across steps (a skin, InstDev::skin)
// and advances one state buffer (mbuf[0]; mbuf[1] is the reorder's scratch).
// A step: drift (cells fixed; sets the rebuild gate err[kErrRebuild] and
// InstState::rebuild of the instances that moved too far), then, gated, keys,
// scan, scatter/sort, reorder, copy-back and (per instance) search and list
// compaction, then density over the reused lists, pressure filter, pair pass,
// kick, wall torque, and the gate closed.
// mode 0: walls placed at the current phase, no kick/drift; mode 1: half kick
// + drift + walls at the next phase; mode 2: as 1, after the previous step's
// closing half kick (which the step graphs leave to the next step's drift).
cudaError_t launch_drift_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                               const InstDev* inst, InstState* ist, uint32_t* err, int mode,
                               cudaStream_t s, const LaunchCfg& lc, int* launches);
cudaError_t launch_keys_mixed(int64_t n, const MixBuf& b, const InstDev* inst,
                              const InstState* ist, const CellWs& cw, uint32_t* err, int mode,
                              cudaStream_t s, const LaunchCfg& lc, int* launches);
// Sorted keys and cell counts of the current order from the cells and the
// offsets of the last build (relist after a checkpoint load; counts zero).
cudaError_t launch_relist_keys_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                     const InstDev* inst, const CellWs& cw, cudaStream_t s,
                                     const LaunchCfg& lc);
// open: every instance rebuilds (the gate opened); otherwise close the gate,
// recording the wall phase of the step's builds (mode as for the drift).
cudaError_t launch_gate(bool open, int32_t n_inst, const InstDev* inst, InstState* ist,
                        uint32_t* err, int mode, cudaStream_t s, int* launches);
cudaError_t launch_reorder_mixed(int64_t n, const MixBuf& src, const MixBuf& dst,
                                 const CellWs& cw, const uint32_t* gate, cudaStream_t s,
                                 const LaunchCfg& lc, int* launches);
cudaError_t launch_copyback_mixed(int64_t n, const MixBuf& src, const MixBuf& dst,
                                  const MixFields& f, const InstState* ist, const uint32_t* gate,
                                  cudaStream_t s, const LaunchCfg& lc, int* launches);
// gated: only the instances that rebuild (InstState::rebuild); 0: all.
cudaError_t launch_skin_list_mixed(int64_t n, const MixBuf& b, const InstDev* inst,
                                   const InstState* ist, const CellWs& cw, const NbrWs& nw,
                                   uint32_t* err, int gated, cudaStream_t s,
                                   const LaunchCfg& lc, int* launches);
cudaError_t launch_density_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                 const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                 cudaStream_t s, const LaunchCfg& lc, int* launches);
cudaError_t launch_pfilter_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                 const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                 cudaStream_t s, int* launches);
cudaError_t launch_forces_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                const InstDev* inst, const NbrWs& nw, uint32_t* err,
                                cudaStream_t s, const LaunchCfg& lc, int* launches);
cudaError_t launch_kick_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                              const InstDev* inst, cudaStream_t s, const LaunchCfg& lc,
                              int* launches);
cudaError_t launch_load_mixed(int64_t n, const MixBuf& b, const InstDev* inst, int32_t n_inst,
                              const double* pos, const double* vel, const double* spin,
                              const uint8_t* sp, uint32_t* err, cudaStream_t s,
                              const LaunchCfg& lc);
cudaError_t launch_unsort_mixed(int64_t n, const MixBuf& b, const MixFields& f,
                                const InstDev* inst, double* pos, double* vel, double* spin,
                                double* rho, double* P, double* acc, double* dspin,
                                cudaStream_t s, const LaunchCfg& lc);

// ---- FP64 reductions (sph_reduce.cu) -----------------------------------------
cudaError_t launch_wall_torque_mixed(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                                     InstState* ist, const MixBuf& b, const MixFields& f,
                                     double* partials, int advance, cudaStream_t s,
                                     int* launches);
cudaError_t launch_diag_mixed(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                              const MixBuf& b, const MixFields& f, const NbrWs& nw,
                              double* partials, double* out, cudaStream_t s);
// Per-instance wall torque of the last force pass; then
// J += dt/2 (T_old + T_new), T = T_new, and (advance) theta += Omega dt, step++.
cudaError_t launch_wall_torque_fp64(int32_t n_inst, int64_t total_chunks,
                                    const InstDev* inst, InstState* ist,
                                    const Fp64Buf& b, const Fp64Fields& f,
                                    double* partials, int advance, cudaStream_t s,
                                    int* launches);
// Per-instance diagnostics partials, then final sums into out[n_inst * kDiagFields].
cudaError_t launch_diag_fp64(int32_t n_inst, int64_t total_chunks, const InstDev* inst,
                             const Fp64Buf& b, const Fp64Fields& f, const NbrWs& nw,
                             double* partials, double* out, cudaStream_t s);

// Per-instance force breakdown: out[k * kDiagFields + q] = sum over the fluid
// particles of instance k of |sum_j f_ij^q| for the pair terms q = pressure,
// interfacial, shear, rotational, local interaction (FP64, current state and
// neighbour lists).
cudaError_t launch_breakdown_fp64(int32_t n_inst, int64_t n, int64_t total_chunks,
                                  const InstDev* inst, const Fp64Buf& b, const Fp64Fields& f,
                                  const NbrWs& nw, double* partials, double* out,
                                  cudaStream_t s);
cudaError_t launch_breakdown_mixed(int32_t n_inst, int64_t n, int64_t total_chunks,
                                   const InstDev* inst, const MixBuf& b, const MixFields& f,
                                   const NbrWs& nw, double* partials, double* out,
                                   cudaStream_t s);

// Per-instance neighbour-pair census of the current lists: ordered (fluid
// row, neighbour) pairs by species class into out[k * kDiagFields + q],
// q = 0 inviscid-inviscid, 1 unlike fluid, 2 viscous-viscous, 3 inviscid-wall,
// 4 viscous-wall.
cudaError_t launch_census_fp64(int32_t n_inst, int64_t n, int64_t total_chunks,
                               const InstDev* inst, const Fp64Buf& b, const Fp64Fields& f,
                               const NbrWs& nw, double* partials, double* out, cudaStream_t s);
cudaError_t launch_census_mixed(int32_t n_inst, int64_t n, int64_t total_chunks,
                                const InstDev* inst, const MixBuf& b, const MixFields& f,
                                const NbrWs& nw, double* partials, double* out, cudaStream_t s);

}  // namespace sphgb
