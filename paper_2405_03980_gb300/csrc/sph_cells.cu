// Cell-list build: exclusive scan of the cell counts, stable scatter and the
// per-cell ordering by particle id (the neighbour-particle-list construction
// of Algorithm 1; particle sorting keeps the pair search O(N), Sec. 2.3).
//
// The counts come from atomics in the kick/drift kernel, so the arrival slot
// of a particle inside its cell is not deterministic; sorting every cell by
// particle id afterwards makes the sorted order a pure function of the cell
// assignment, identical from run to run and between batched and single runs.
#include "sph_kernels.h"

namespace sphgb {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kPerThread = kScanChunk / kScanThreads;  // 4
static_assert(kPerThread == 4, "scan layout assumes 4 elements per thread");

// The kernels of the cell build do nothing while a gate word is zero (the
// mixed form's steps that reuse their lists); a null gate always runs.
__device__ __forceinline__ bool closed(const uint32_t* gate) {
  return gate != nullptr && *(const volatile uint32_t*)gate == 0u;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_chunks(uint32_t* __restrict__ count, uint32_t* __restrict__ start,
              uint32_t* __restrict__ bsum, int64_t n, const uint32_t* gate) {
  __shared__ uint32_t warp_ex[32];
  __shared__ uint32_t block_total;
  if (closed(gate)) return;
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kPerThread;
  uint32_t v[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    v[k] = (base + k < n) ? count[base + k] : 0u;
    if (base + k < n) count[base + k] = 0u;  // zero for the next build
  }
  uint32_t s = v[0] + v[1] + v[2] + v[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(s);
  if (lane == 31) warp_ex[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = warp_ex[lane];
    uint32_t wi = warp_incl_scan(w);
    warp_ex[lane] = wi - w;
    if (lane == 31) block_total = wi;
  }
  __syncthreads();
  uint32_t run = warp_ex[warp] + inc - s;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    if (base + k < n) start[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = block_total;
}

// One block: exclusive scan of the chunk sums in place, total to start[n].
__global__ void __launch_bounds__(kScanThreads)
k_scan_top(uint32_t* __restrict__ bsum, int64_t nb, uint32_t* __restrict__ start, int64_t n,
           const uint32_t* gate) {
  __shared__ uint32_t warp_ex[32];
  __shared__ uint32_t tile_total;
  if (closed(gate)) return;
  uint32_t carry = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t0 = 0; t0 < nb; t0 += kScanThreads) {
    const int64_t i = t0 + threadIdx.x;
    uint32_t v = (i < nb) ? bsum[i] : 0u;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) warp_ex[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = warp_ex[lane];
      uint32_t wi = warp_incl_scan(w);
      warp_ex[lane] = wi - w;
      if (lane == 31) tile_total = wi;
    }
    __syncthreads();
    if (i < nb) bsum[i] = carry + warp_ex[warp] + inc - v;
    carry += tile_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_scan_add(uint32_t* __restrict__ start, const uint32_t* __restrict__ bsum,
                           int64_t n, const uint32_t* gate) {
  if (closed(gate)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    start[i] += bsum[i / kScanChunk];
}

__global__ void k_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ slot,
                          const uint32_t* __restrict__ start, uint32_t* __restrict__ perm,
                          int64_t n, int64_t n_cells, uint32_t* err, const uint32_t* gate) {
  if (closed(gate)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = key[i];
    if (!bounds_ok((int64_t)k < n_cells, err)) continue;
    const uint32_t d = start[k] + slot[i];
    if (!bounds_ok((int64_t)d < n, err)) continue;
    perm[d] = (uint32_t)i;
  }
}

// Sort the entries of every cell by particle id (insertion sort; cells hold
// about 18 particles at a cell side of 2h = 2.6 dx).
__global__ void k_cell_sort(const uint32_t* __restrict__ start, uint32_t* __restrict__ perm,
                            const uint32_t* __restrict__ id, int64_t n_cells, int64_t n,
                            uint32_t* err, const uint32_t* gate) {
  if (closed(gate)) return;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = start[c], e = start[c + 1];
    if (!bounds_ok(s <= e && (int64_t)e <= n, err)) continue;
    const uint32_t m = e - s;
    if (m <= 1) continue;
    if (m <= 32) {
      uint32_t kk[32], vv[32];
      for (uint32_t t = 0; t < m; ++t) {
        vv[t] = checked_index(perm[s + t], n, err);
        kk[t] = id[vv[t]];
      }
      for (uint32_t t = 1; t < m; ++t) {
        uint32_t k = kk[t], v = vv[t];
        int32_t u = (int32_t)t - 1;
        while (u >= 0 && kk[u] > k) {
          kk[u + 1] = kk[u];
          vv[u + 1] = vv[u];
          --u;
        }
        kk[u + 1] = k;
        vv[u + 1] = v;
      }
      for (uint32_t t = 0; t < m; ++t) perm[s + t] = vv[t];
    } else {
      for (uint32_t t = s + 1; t < e; ++t) {
        uint32_t v = checked_index(perm[t], n, err), k = id[v];
        uint32_t u = t;
        while (u > s && id[checked_index(perm[u - 1], n, err)] > k) {
          perm[u] = perm[u - 1];
          --u;
        }
        perm[u] = v;
      }
    }
  }
}

inline int grid_for(int64_t n, int threads, int sm_count, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_scan(const CellWs& cw, cudaStream_t s, const LaunchCfg& lc, int* launches,
                        const uint32_t* gate) {
  const int64_t nb = cw.n_scan_blocks;
  k_scan_chunks<<<(unsigned)nb, kScanThreads, 0, s>>>(cw.count, cw.start, cw.bsum, cw.n_cells,
                                                      gate);
  k_scan_top<<<1, kScanThreads, 0, s>>>(cw.bsum, nb, cw.start, cw.n_cells, gate);
  k_scan_add<<<grid_for(cw.n_cells, 256, lc.sm_count, 8), 256, 0, s>>>(cw.start, cw.bsum,
                                                                       cw.n_cells, gate);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_scatter_sort(const CellWs& cw, const uint32_t* id, int64_t n,
                                cudaStream_t s, const LaunchCfg& lc, int* launches,
                                const uint32_t* gate) {
  k_scatter<<<grid_for(n, 256, lc.sm_count, 16), 256, 0, s>>>(cw.key, cw.slot, cw.start,
                                                                cw.perm, n, cw.n_cells, cw.err,
                                                                gate);
  k_cell_sort<<<grid_for(cw.n_cells, 128, lc.sm_count, 16), 128, 0, s>>>(
      cw.start, cw.perm, id, cw.n_cells, n, cw.err, gate);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

}  // namespace sphgb
