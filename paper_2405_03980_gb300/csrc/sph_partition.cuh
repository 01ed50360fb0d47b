// Stable, deterministic partition of the fluid particles by species for the
// pair passes (no atomics): per tile of kPartTile sorted particles the
// counts of inviscid and viscous fluid; their exclusive scans over the tiles
// (inviscid first); then each tile writes its particles' indices in order,
// nw.order[0 .. n_inv) the inviscid ones and nw.order[n_inv .. n_fluid) the
// viscous ones, with nw.part[2 nt] = n_inv and nw.part[2 nt + 1] = n_fluid.
// Wall rows, which the pair passes do not visit, get zero accelerations and
// wall torque here.  A View gives cls(i) (0 inviscid, 1 viscous, 2 wall) and
// zero(i).
#pragma once
#include "sph_kernels.h"

namespace sphgb {
namespace {

constexpr int kPartThreads = 256;
constexpr int kPartPer = kPartTile / kPartThreads;  // 16 consecutive particles per thread

// Exclusive block scan of two counts at once (kPartThreads threads).
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t v, uint32_t& ea, uint32_t& ev,
                                            uint32_t& ta, uint32_t& tv) {
  __shared__ uint32_t wa[32], wv[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ia = a, iv = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t xa = __shfl_up_sync(~0u, ia, o), xv = __shfl_up_sync(~0u, iv, o);
    if (lane >= o) {
      ia += xa;
      iv += xv;
    }
  }
  if (lane == 31) {
    wa[warp] = ia;
    wv[warp] = iv;
  }
  __syncthreads();
  if (warp == 0) {
    const int nwarp = kPartThreads / 32;
    uint32_t sa = lane < nwarp ? wa[lane] : 0u, sv = lane < nwarp ? wv[lane] : 0u;
    uint32_t ja = sa, jv = sv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t xa = __shfl_up_sync(~0u, ja, o), xv = __shfl_up_sync(~0u, jv, o);
      if (lane >= o) {
        ja += xa;
        jv += xv;
      }
    }
    if (lane < nwarp) {
      wa[lane] = ja - sa;
      wv[lane] = jv - sv;
    }
    if (lane == nwarp - 1) {
      wa[31] = ja;
      wv[31] = jv;
    }
  }
  __syncthreads();
  ea = wa[warp] + ia - a;
  ev = wv[warp] + iv - v;
  ta = wa[31];
  tv = wv[31];
  __syncthreads();
}

template <class View>
__global__ void __launch_bounds__(kPartThreads)
k_part_count(int64_t n, View V, uint32_t* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * kPartTile + (int64_t)threadIdx.x * kPartPer;
  uint32_t a = 0, v = 0;
  for (int k = 0; k < kPartPer; ++k)
    if (base + k < n) {
      const int c = V.cls(base + k);
      a += c == 0;
      v += c == 1;
    }
  uint32_t ea, ev, ta, tv;
  block_scan2(a, v, ea, ev, ta, tv);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ta;
    part[2 * blockIdx.x + 1] = tv;
  }
}

// One block: the tile offsets (inviscid from 0, viscous after all inviscid)
// in place, and the totals part[2 nt] = inviscid, part[2 nt + 1] = fluid.
__global__ void __launch_bounds__(kPartThreads)
k_part_scan(int64_t nt, uint32_t* __restrict__ part) {
  __shared__ uint32_t carry[2];
  if (threadIdx.x == 0) carry[0] = carry[1] = 0u;
  __syncthreads();
  for (int64_t t0 = 0; t0 < nt; t0 += kPartThreads) {
    const int64_t t = t0 + threadIdx.x;
    const uint32_t a = t < nt ? part[2 * t] : 0u, v = t < nt ? part[2 * t + 1] : 0u;
    uint32_t ea, ev, ta, tv;
    block_scan2(a, v, ea, ev, ta, tv);
    const uint32_t ca = carry[0], cv = carry[1];
    if (t < nt) {
      part[2 * t] = ca + ea;
      part[2 * t + 1] = cv + ev;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] = ca + ta;
      carry[1] = cv + tv;
    }
    __syncthreads();
  }
  // the viscous offsets start after every inviscid particle
  const uint32_t n_inv = carry[0];
  for (int64_t t = threadIdx.x; t < nt; t += kPartThreads) part[2 * t + 1] += n_inv;
  if (threadIdx.x == 0) {
    part[2 * nt] = n_inv;
    part[2 * nt + 1] = n_inv + carry[1];
  }
}

template <class View>
__global__ void __launch_bounds__(kPartThreads)
k_part_scatter(int64_t n, View V, const uint32_t* __restrict__ part,
               uint32_t* __restrict__ order) {
  const int64_t base = (int64_t)blockIdx.x * kPartTile + (int64_t)threadIdx.x * kPartPer;
  int cls[kPartPer];
  uint32_t a = 0, v = 0;
#pragma unroll
  for (int k = 0; k < kPartPer; ++k) {
    cls[k] = base + k < n ? V.cls(base + k) : 3;
    a += cls[k] == 0;
    v += cls[k] == 1;
  }
  uint32_t ea, ev, ta, tv;
  block_scan2(a, v, ea, ev, ta, tv);
  uint32_t oa = part[2 * blockIdx.x] + ea, ov = part[2 * blockIdx.x + 1] + ev;
#pragma unroll
  for (int k = 0; k < kPartPer; ++k) {
    const int64_t i = base + k;
    if (cls[k] == 0) order[oa++] = (uint32_t)i;
    else if (cls[k] == 1) order[ov++] = (uint32_t)i;
    else if (cls[k] == 2) V.zero(i);
  }
}

template <class View>
cudaError_t launch_partition(int64_t n, const View& V, const NbrWs& nw, cudaStream_t s,
                             int* launches) {
  const int64_t nt = (n + kPartTile - 1) / kPartTile;
  k_part_count<View><<<(unsigned)nt, kPartThreads, 0, s>>>(n, V, nw.part);
  k_part_scan<<<1, kPartThreads, 0, s>>>(nt, nw.part);
  k_part_scatter<View><<<(unsigned)nt, kPartThreads, 0, s>>>(n, V, nw.part, nw.order);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace
}  // namespace sphgb
