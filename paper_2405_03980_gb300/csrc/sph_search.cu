// Neighbour search of the density pass (Sec. 2.3: all particles within the
// kernel support 2h), one warp per grid cell, shared by both state forms.
//
// Every particle of a cell has the same 27-cell candidate set: the 9 rows
// (dy, dz) of x-adjacent cells cx-1..cx+1, each row one contiguous run of the
// sorted order per cell.  A warp takes one cell, writes its candidate
// sequence (rows dz, dy, cells kc, index j) once as the cell's candidate
// table, and tests the candidates with the lanes spread over the CANDIDATES:
// for each target particle t of the cell, the 32 lanes test 32 candidates at
// once and a ballot gives the 32-bit hit mask of (t, chunk), so no lane idles
// on a short cell and the control flow never diverges.  The output is one
// bit per (particle, candidate): mask word k of particle i covers candidates
// 32k .. 32k+31 of its cell's table.  The density pass walks these bits in
// order, which is the neighbour order of the lists it writes for the pair
// pass.
//
// Mixed form: the test is exact, r^2 < (2h)^2 in FP32 on the pair vector
// (c_i - c_j) L + (o_i - o_j), which every later use of the entry recomputes
// bit for bit; the test of (j, i) negates that of (i, j), so the neighbour
// sets are symmetric.  Table entries carry the cell-displacement code.
// FP64 form: an FP32 prefilter on rounded absolute positions (the periodic
// image in z taken per run) against a widened bound, a superset of the FP64
// neighbours; the density pass re-tests every candidate it is given in FP64.
#include "sph_f32x2.cuh"
#include "sph_kernels.h"

namespace sphgb {
namespace {

// kSeg, the segment depth: candidates staged in shared memory at a time (256
// or 512, chosen by the autotuner; a cell of the 2.6 dx grid has about 470)
constexpr int kMaskRow = 36;  // mask words of one chunk: 4 targets per 16-byte store, and
                              // lane t reading word t of chunk k hits bank (4k + t) % 32
constexpr int kMaxSearchWarps = 8;

template <int kSeg>
struct WarpSmem {
  static_assert(kMaxCand % kSeg == 0, "segments tile the candidate table");
  static constexpr int kSegChunks = kSeg / 32;
  uint32_t ent[kSeg];                 // candidate index | cell-displacement code
  // coordinates of the current targets by axis, so that two consecutive
  // targets load as one 8-byte pair
  alignas(16) float tx[32];
  alignas(16) float ty[32];
  alignas(16) float tz[32];
  alignas(16) uint32_t mask[kSegChunks * kMaskRow];  // hit mask of (chunk, target)
};

__device__ __forceinline__ void latch(uint32_t* err, uint32_t bit) {
  if ((*(volatile uint32_t*)err & bit) == 0u) atomicOr(err, bit);
}

// r^2 of a pair vector with an explicit rounding sequence, so that both
// search mappings below classify every candidate with the same bits.
__device__ __forceinline__ float pair_r2(float dx, float dy, float dz) {
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// rec: per sorted particle (x, y, z, species); mixed: the offset inside the
// cell, FP64 form: the FP32-rounded absolute position.
template <bool kMixed, int kSeg>
__global__ void __launch_bounds__(32 * kMaxSearchWarps, 3)
k_cell_search(int64_t n, const float4* __restrict__ rec, const InstDev* __restrict__ inst,
              CellWs cw, NbrWs nw, uint32_t* err, const InstState* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate && gate[blockIdx.y].rebuild == 0) return;  // the instance keeps its lists
  const int lane = threadIdx.x & 31;
  WarpSmem<kSeg>& sm = reinterpret_cast<WarpSmem<kSeg>*>(smem_raw)[threadIdx.x >> 5];
  const InstDev& P = inst[blockIdx.y];
  const int64_t ncells = (int64_t)P.nx * P.ny * P.nz;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  // the warps of a bounded grid take the instance's cells in turn, so that a
  // step whose gate is closed costs a few thousand empty blocks at most
  for (int64_t l = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < ncells;
       l += wstride) {
    const int S = P.slabs;
    const int64_t key0 = P.cell_base + l * S;
    const uint32_t i0 = cw.start[key0], i1 = cw.start[key0 + S];
    if (i0 == i1) continue;
    const int cx = (int)(l % P.nx);
    const int cy = (int)((l / P.nx) % P.ny);
    const int cz = (int)(l / ((int64_t)P.nx * P.ny));

    // run table: lane r < 27 holds run r = (dz + 1) 9 + (dy + 1) 3 + kc, the
    // particles of cell (cx - 1 + kc, cy + dy, cz + dz)
    uint32_t rj0 = 0, rlen = 0, rcode = 0;
    if (lane < 27) {
      const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, kc = lane % 3;
      int z2 = cz + dz;
      if (P.periodic_z) z2 = z2 < 0 ? z2 + P.nz : (z2 >= P.nz ? z2 - P.nz : z2);
      const int64_t key =
          P.cell_base +
          ((int64_t)(cx - 1 + kc) + (int64_t)P.nx * ((cy + dy) + (int64_t)P.ny * z2)) * S;
      rj0 = cw.start[key];
      rlen = cw.start[key + S] - rj0;
      if (!bounds_ok((int64_t)rj0 + rlen <= n, err)) rlen = 0;
      rcode = ((uint32_t)(2 - kc) | ((uint32_t)(1 - dy) << 2) | ((uint32_t)(1 - dz) << 4))
              << kNbrIndexBits;
    }
    uint32_t incl = rlen;  // inclusive scan of the run lengths over the lanes
  #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t rpre = incl - rlen;
    uint32_t total = __shfl_sync(~0u, incl, 31);
    const int64_t g = key0 / S;  // grid cell over all instances
    if (total > (uint32_t)kMaxCand) {  // more candidates than the table holds
      if (lane == 0) latch(err, ERR_NEIGHBORS);
      total = kMaxCand;
    }
    if (lane == 0) nw.ncand[g] = total;
    uint32_t* __restrict__ table = nw.cand + g * kMaxCand;
    const uint32_t pre_self = __shfl_sync(~0u, rpre, 13);  // the cell's own run
    const float cut2 = kMixed ? P.skin_cut2_f : P.cut2f_margin;

    bool table_done = false;
    for (uint32_t tb = i0; tb < i1; tb += 32) {
      const uint32_t nt = min(32u, i1 - tb);
      const uint32_t i = tb + lane;
      float4 mine = make_float4(0.f, 0.f, 0.f, 3.f);
      if (lane < nt) mine = rec[i];
      sm.tx[lane] = mine.x;
      sm.ty[lane] = mine.y;
      sm.tz[lane] = mine.z;
      const bool active = lane < nt && mine.w != 3.f;  // outer-wall particles keep no list
      if (__ballot_sync(~0u, active) == 0u) {
        if (lane < nt) nw.count[i] = 0u;
        continue;
      }
      const uint32_t self_q = pre_self + (i - i0);  // candidate position of i itself
      uint32_t hits = 0;
      for (uint32_t s0 = 0; s0 < total; s0 += kSeg) {
        const uint32_t nseg = min((uint32_t)kSeg, total - s0);
        __syncwarp();
        if (lane < 27) {  // lane r writes the entries of run r that fall in this segment
          const uint32_t e0 = s0 > rpre ? s0 - rpre : 0u;
          const uint32_t end = s0 + nseg - rpre;  // used only if the run starts before it
          const uint32_t e1 = s0 + nseg > rpre ? (rlen < end ? rlen : end) : 0u;
          for (uint32_t e = e0; e < e1; ++e) sm.ent[rpre + e - s0] = (rj0 + e) | rcode;
        }
        __syncwarp();
        if (!table_done)  // the cell's candidate table, once per cell
          for (uint32_t q = lane; q < nseg; q += 32) table[s0 + q] = sm.ent[q];
        const uint32_t nch = (nseg + 31) >> 5;
        // each lane's candidate record, the next chunk's loaded one chunk ahead
        uint32_t ent_n = sm.ent[lane < nseg ? lane : 0u];
        float4 c_n = rec[ent_n & kNbrIndexMask];
        for (uint32_t k = 0; k < nch; ++k) {
          const uint32_t q = (k << 5) + lane;
          const bool valid = q < nseg;
          const uint32_t ent = ent_n;
          float4 c = c_n;
          if (k + 1 < nch) {
            const uint32_t qn = q + 32u;
            ent_n = sm.ent[qn < nseg ? qn : 0u];
            c_n = rec[ent_n & kNbrIndexMask];
          }
          const uint32_t code = ent >> kNbrIndexBits;
          float ex = 0.f, ey = 0.f, ez = 0.f;
          if (kMixed) {  // (c_i - c_j) L per axis; exact
            ex = (float)((int)(code & 3u) - 1) * P.cellf[0];
            ey = (float)((int)((code >> 2) & 3u) - 1) * P.cellf[1];
            ez = (float)((int)(code >> 4) - 1) * P.cellf[2];
          } else if (P.periodic_z) {  // image of a candidate across the z period
            const int z2 = cz + 1 - (int)(code >> 4);
            if (z2 < 0) c.z -= P.Hzf;
            else if (z2 >= P.nz) c.z += P.Hzf;
          }
          // the pair vector e + (o_t - c) of the mixed form is the one every
          // later use of the entry recomputes; two targets per packed FP32
          // instruction, four per round, ahead of their ballots
          auto hit = [&](uint32_t t) {
            float dx = sm.tx[t] - c.x, dy = sm.ty[t] - c.y, dz = sm.tz[t] - c.z;
            if (kMixed) {
              dx = ex + dx;
              dy = ey + dy;
              dz = ez + dz;
            }
            return valid && pair_r2(dx, dy, dz) < cut2;
          };
          const f2 CX = f2_splat(c.x), CY = f2_splat(c.y), CZ = f2_splat(c.z);
          const f2 EX = f2_splat(ex), EY = f2_splat(ey), EZ = f2_splat(ez);
          auto hit2 = [&](uint32_t t, bool& h0, bool& h1) {  // targets t, t + 1 (t even)
            f2 dx = f2_sub(*reinterpret_cast<const f2*>(sm.tx + t), CX);
            f2 dy = f2_sub(*reinterpret_cast<const f2*>(sm.ty + t), CY);
            f2 dz = f2_sub(*reinterpret_cast<const f2*>(sm.tz + t), CZ);
            if (kMixed) {
              dx = f2_add(EX, dx);
              dy = f2_add(EY, dy);
              dz = f2_add(EZ, dz);
            }
            const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
            float r0, r1;
            f2_split(r2, r0, r1);
            h0 = valid && r0 < cut2;
            h1 = valid && r1 < cut2;
          };
          uint32_t* mk = sm.mask + k * kMaskRow;
          uint32_t t = 0;
          for (; t + 4 <= nt; t += 4) {
            bool h0, h1, h2, h3;
            hit2(t, h0, h1);
            hit2(t + 2, h2, h3);
            const uint32_t m0 = __ballot_sync(~0u, h0), m1 = __ballot_sync(~0u, h1);
            const uint32_t m2 = __ballot_sync(~0u, h2), m3 = __ballot_sync(~0u, h3);
            if (lane == 0) {
              *reinterpret_cast<uint4*>(mk + t) = make_uint4(m0, m1, m2, m3);
            }
          }
          for (; t < nt; ++t) {
            const uint32_t m0 = __ballot_sync(~0u, hit(t));
            if (lane == 0) mk[t] = m0;
          }
        }
        __syncwarp();
        if (active) {  // lane t stores its mask words, without the self bit
          const uint32_t* mcol = sm.mask + lane;
          uint32_t* out = nw.mask + (int64_t)(s0 >> 5) * n + i;
          for (uint32_t k = 0; k < nch; ++k) {
            uint32_t m = mcol[k * kMaskRow];
            const uint32_t qs = self_q - s0 - (k << 5);  // < 32 iff i itself is in chunk k
            if (qs < 32u) m &= ~(1u << qs);
            out[(int64_t)k * n] = m;
            hits += __popc(m);
          }
        }
      }
      table_done = true;
      if (lane < nt) nw.count[i] = hits;
    }
  }
}

// The same search with the other mapping: one thread per particle walks the
// 27 runs of its cell's stencil in candidate order and tests each candidate
// itself (the same FP32 expression as above, so the same bits), setting bit q
// of its mask words; the first particle of each cell writes the cell's
// candidate table and its length.  Lanes of one cell load the same candidate
// record (a broadcast); lanes of neighbouring cells walk runs of different
// lengths.  The output is identical to the warp-per-cell kernel's.
template <bool kMixed>
__global__ void __launch_bounds__(128)
k_cell_search_tpp(int64_t n, const float4* __restrict__ rec,
                  const uint32_t* __restrict__ inst_of, const InstDev* __restrict__ inst,
                  CellWs cw, NbrWs nw, uint32_t* err, const InstState* __restrict__ gate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (gate && gate[inst_of[i]].rebuild == 0) continue;  // the instance keeps its lists
    const InstDev& P = inst[inst_of[i]];
    const int S = P.slabs;
    const int64_t g = (int64_t)cw.skey[i] / S;  // grid cell over all instances
    const int64_t l = g - P.cell_base / S;      // cell inside the instance
    const int cx = (int)(l % P.nx);
    const int cy = (int)((l / P.nx) % P.ny);
    const int cz = (int)(l / ((int64_t)P.nx * P.ny));
    const uint32_t i0 = cw.start[g * S];
    const bool writer = (uint32_t)i == i0;  // writes the cell's candidate table
    const float4 mine = rec[i];
    const bool active = mine.w != 3.f;      // outer-wall particles keep no list
    if (!active && !writer) {
      nw.count[i] = 0u;
      continue;
    }
    uint32_t* __restrict__ table = nw.cand + g * kMaxCand;
    uint32_t* __restrict__ out = nw.mask + i;
    const float cut2 = kMixed ? P.skin_cut2_f : P.cut2f_margin;
    uint32_t q = 0, word = 0, hits = 0, self_q = ~0u;
    bool over = false;
    for (int r = 0; r < 27 && !over; ++r) {
      const int dz = r / 9 - 1, dy = (r / 3) % 3 - 1, kc = r % 3;
      const int zu = cz + dz;  // unwrapped z cell of the run
      int z2 = zu;
      if (P.periodic_z) z2 = z2 < 0 ? z2 + P.nz : (z2 >= P.nz ? z2 - P.nz : z2);
      const int64_t key =
          P.cell_base +
          ((int64_t)(cx - 1 + kc) + (int64_t)P.nx * ((cy + dy) + (int64_t)P.ny * z2)) * S;
      const uint32_t rj0 = cw.start[key];
      uint32_t rlen = cw.start[key + S] - rj0;
      if (!bounds_ok((int64_t)rj0 + rlen <= n, err)) rlen = 0;
      if (r == 13) self_q = q + ((uint32_t)i - rj0);  // run 13 is the particle's own cell
      const uint32_t code = ((uint32_t)(2 - kc) | ((uint32_t)(1 - dy) << 2) |
                             ((uint32_t)(1 - dz) << 4)) << kNbrIndexBits;
      // (c_i - c_j) L per axis (exact): the run's cell is c_i + (kc - 1, dy, dz),
      // so the displacement is -(kc - 1, dy, dz), the code minus one per axis
      const float ex = (float)(1 - kc) * P.cellf[0];
      const float ey = (float)(-dy) * P.cellf[1];
      const float ez = (float)(-dz) * P.cellf[2];
      const float zs = (!kMixed && P.periodic_z) ? (zu < 0 ? -1.f : (zu >= P.nz ? 1.f : 0.f)) : 0.f;
      for (uint32_t e = 0; e < rlen; ++e, ++q) {
        if (q >= (uint32_t)kMaxCand) {  // more candidates than the table holds
          over = true;
          break;
        }
        const uint32_t j = rj0 + e;
        if (writer) table[q] = j | code;
        if (active) {
          float4 c = rec[j];
          if (!kMixed) {  // image of the candidate across the z period
            if (zs < 0.f) c.z -= P.Hzf;
            else if (zs > 0.f) c.z += P.Hzf;
          }
          float dx = mine.x - c.x, dyv = mine.y - c.y, dzv = mine.z - c.z;
          if (kMixed) {
            dx = ex + dx;
            dyv = ey + dyv;
            dzv = ez + dzv;
          }
          if (pair_r2(dx, dyv, dzv) < cut2) word |= 1u << (q & 31u);
          if ((q & 31u) == 31u) {  // a full mask word, without the self bit
            const uint32_t qs = self_q - (q & ~31u);
            if (qs < 32u) word &= ~(1u << qs);
            out[(int64_t)(q >> 5) * n] = word;
            hits += __popc(word);
            word = 0u;
          }
        }
      }
    }
    if (over) latch(err, ERR_NEIGHBORS);
    if (active && (q & 31u) != 0u) {  // the last, partial word
      const uint32_t qs = self_q - (q & ~31u);
      if (qs < 32u) word &= ~(1u << qs);
      out[(int64_t)(q >> 5) * n] = word;
      hits += __popc(word);
    }
    if (writer) nw.ncand[g] = q;
    nw.count[i] = active ? hits : 0u;
  }
}

size_t search_smem(int warps, int seg) {
  return (seg == 256 ? sizeof(WarpSmem<256>) : sizeof(WarpSmem<512>)) * (size_t)warps;
}

}  // namespace

int search_max_warps() { return kMaxSearchWarps; }

cudaError_t prepare_search_kernels() {
  const void* fns[4] = {(const void*)k_cell_search<true, 256>,
                        (const void*)k_cell_search<false, 256>,
                        (const void*)k_cell_search<true, 512>,
                        (const void*)k_cell_search<false, 512>};
  for (int k = 0; k < 4; ++k) {
    const int bytes = (int)search_smem(kMaxSearchWarps, k < 2 ? 256 : 512);
    const cudaError_t e =
        cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_cell_search(bool mixed_form, int64_t n, const float4* rec,
                               const uint32_t* inst_of, const InstDev* inst, int32_t n_inst,
                               int64_t max_cells, const CellWs& cw, const NbrWs& nw,
                               uint32_t* err, cudaStream_t s, const LaunchCfg& lc,
                               int* launches, const InstState* gate) {
  if (lc.search_warps == 0) {  // thread-per-particle mapping
    const int64_t want = (n + 127) / 128, cap = (int64_t)lc.sm_count * 16;
    const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    if (mixed_form)
      k_cell_search_tpp<true><<<blocks, 128, 0, s>>>(n, rec, inst_of, inst, cw, nw, err, gate);
    else
      k_cell_search_tpp<false><<<blocks, 128, 0, s>>>(n, rec, inst_of, inst, cw, nw, err, gate);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  int warps = lc.search_warps;
  if (warps < 1 || warps > kMaxSearchWarps) warps = 4;
  const int64_t want = (max_cells + warps - 1) / warps, cap = (int64_t)lc.sm_count * 16;
  const dim3 grid((unsigned)(want < cap ? want : cap), (unsigned)n_inst);
  const int seg = lc.search_depth == 256 ? 256 : 512;
  const size_t smem = search_smem(warps, seg);
  if (seg == 256) {
    if (mixed_form)
      k_cell_search<true, 256><<<grid, 32 * warps, smem, s>>>(n, rec, inst, cw, nw, err, gate);
    else
      k_cell_search<false, 256><<<grid, 32 * warps, smem, s>>>(n, rec, inst, cw, nw, err, gate);
  } else {
    if (mixed_form)
      k_cell_search<true, 512><<<grid, 32 * warps, smem, s>>>(n, rec, inst, cw, nw, err, gate);
    else
      k_cell_search<false, 512><<<grid, 32 * warps, smem, s>>>(n, rec, inst, cw, nw, err, gate);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace sphgb
