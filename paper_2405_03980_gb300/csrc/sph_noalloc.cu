// Conservation sums for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs as a plug-in inside a
// host application that owns every device allocation (an in-situ analysis
// hook of a larger simulation, a process that reserved its whole memory budget
// up front), or that must not touch the allocator at all.  They still hold
// the particle arrays on the device and want the same FP64 totals that
// sph_diagnostics reports.  sph_diag_sums_noalloc computes them from plain
// input arrays; the scratch it needs (one partial per chunk of particles) is
// the file-scope array below.  The CUDA runtime loads this file's module on a
// device lazily, at the first use of one of its symbols there: the first
// call on a device, which looks up the array's address, is when the array's
// device memory is reserved (so that call can fail with SPH_ERR_CUDA on a
// device whose memory is already used up).  It is held until the process
// exits.
#include <mutex>

#include "sph_diag_impl.cuh"
#include "sph_kernels.h"

namespace sphgb {
namespace {

constexpr int64_t kNoAllocMaxChunks = 2048;
constexpr int64_t kNoAllocMaxParticles = kNoAllocMaxChunks * kReduceChunk;  // 67,108,864
constexpr int kNoAllocMaxDevices = 64;

// Chunk partials, then one record for the final sums: 2049 x 24 doubles
// (393,408 bytes) on every device that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxChunks + 1) * kDiagFields];

std::mutex g_scratch_mutex;
double* g_scratch_addr[kNoAllocMaxDevices] = {};

struct PlainArrays {
  const double* pos;
  const double* vel;
  const double* spin;
  const uint8_t* species;
  const double* rho;
};

__global__ void __launch_bounds__(kRedThreads)
k_diag_chunks_plain(InstDev P, PlainArrays A, int64_t n, double* __restrict__ partials) {
  const int64_t begin = (int64_t)blockIdx.x * kReduceChunk;
  const int64_t end = begin + kReduceChunk < n ? begin + kReduceChunk : n;
  DiagAcc acc;
  acc.init();
  for (int64_t i = begin + threadIdx.x; i < end; i += kRedThreads) {
    const int sp = A.species[i];
    if (sp >= 2) continue;
    const double p[3] = {A.pos[3 * i], A.pos[3 * i + 1], A.pos[3 * i + 2]};
    const double u[3] = {A.vel[3 * i], A.vel[3 * i + 1], A.vel[3 * i + 2]};
    const double w[3] = {A.spin[3 * i], A.spin[3 * i + 1], A.spin[3 * i + 2]};
    acc.add(P, sp == 0, p, u, w, A.rho[i], 0.0);
  }
  diag_block_write(acc, partials + (int64_t)blockIdx.x * kDiagFields);
}

__global__ void k_diag_final_plain(InstDev P, const double* __restrict__ partials,
                                   int64_t n_chunks, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) diag_finish(P, partials, n_chunks, out);
}

// Where a pointer points, seen from device `dev`: memory that kernels on dev
// may read or write (dev's own device memory, or managed memory), another
// device's memory (not reachable without peer access), or host memory.
enum class Mem { kDevice, kOtherDevice, kHost };
Mem mem_kind(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return Mem::kHost;
  }
  if (a.type == cudaMemoryTypeManaged) return Mem::kDevice;
  if (a.type == cudaMemoryTypeDevice) return a.device == dev ? Mem::kDevice : Mem::kOtherDevice;
  return Mem::kHost;
}
bool device_accessible(const void* p, int dev) { return mem_kind(p, dev) == Mem::kDevice; }

// Device address of the scratch array on device dev (the current one),
// looked up once per device: the host-side name of the array is not a
// device address.  The cached address is that of the device's context at
// the first call; a cudaDeviceReset ends that context and makes it stale.
sph_status scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SPH_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    double* ptr = nullptr;
    if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return SPH_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return SPH_OK;
}

}  // namespace
}  // namespace sphgb

using namespace sphgb;

extern "C" sph_status sph_diag_sums_noalloc(const sph_params* params, int64_t n,
                                            const double* pos, const double* vel,
                                            const double* spin, const uint8_t* species,
                                            const double* rho, double* out, void* stream) {
  if (!params || !pos || !vel || !spin || !species || !rho || !out) return SPH_ERR_ARG;
  if (n < 1 || n > kNoAllocMaxParticles) return SPH_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
  if (!device_accessible(pos, dev) || !device_accessible(vel, dev) ||
      !device_accessible(spin, dev) || !device_accessible(species, dev) ||
      !device_accessible(rho, dev))
    return SPH_ERR_ARG;
  if (mem_kind(out, dev) == Mem::kOtherDevice) return SPH_ERR_ARG;
  InstDev P;
  sph_status st = derive_instance(*params, P);
  if (st != SPH_OK) return st;
  double* scratch = nullptr;
  if ((st = scratch_address(dev, &scratch)) != SPH_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n_chunks = (n + kReduceChunk - 1) / kReduceChunk;
  const PlainArrays A{pos, vel, spin, species, rho};
  k_diag_chunks_plain<<<(unsigned)n_chunks, kRedThreads, 0, s>>>(P, A, n, scratch);
  const bool dev_out = device_accessible(out, dev);
  double* final_rec = dev_out ? out : scratch + kNoAllocMaxChunks * kDiagFields;
  k_diag_final_plain<<<1, 32, 0, s>>>(P, scratch, n_chunks, final_rec);
  if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
  if (!dev_out) {
    if (cudaMemcpyAsync(out, final_rec, sizeof(double) * SPH_DIAG_SUMS, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SPH_ERR_CUDA;
  }
  return SPH_OK;
}
