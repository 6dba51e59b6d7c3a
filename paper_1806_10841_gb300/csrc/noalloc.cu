// Allocation-free kinetic energy and momentum (see adress_kinetic_noalloc in adress.h).
//
// Some callers cannot allocate device memory at the point where they need this
// observable: code running inside a memory pool whose budget is fixed up front, a host
// that forbids cudaMalloc while another framework owns the allocator, or a monitoring
// hook that must not perturb the allocation pattern of the simulation it observes.  This
// entry point therefore needs neither a handle (whose creation allocates) nor any call
// that allocates: its per-block partial sums live in a file-scope device array of fixed
// size that every GPU loading the library holds until the process exits.
#include <mutex>
#include <string>

#include "internal.cuh"

namespace adress {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 1024;   // partial-sum slots in the static scratch array
constexpr int kNoAllocAtomsPerThread = 64;
constexpr long long kNoAllocMaxAtoms = (long long)kNoAllocMaxBlocks * kNoAllocThreads * kNoAllocAtomsPerThread;
constexpr int kNoAllocMaxDevices = 64;

// 1024 blocks x 4 partial sums (KE, Px, Py, Pz) = 32 KiB of scratch per device.
static __device__ __align__(256) double g_kinetic_scratch[kNoAllocMaxBlocks * 4];

struct NoAllocMasses {
  double m[kMaxNA];
  int na;
};

// Each block sums its grid-stride share of atoms into slot blockIdx.x of the scratch.
__global__ void __launch_bounds__(kNoAllocThreads) k_kinetic_partials(const double* __restrict__ v, long long n,
                                                                      NoAllocMasses ms, double* scratch) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double m = ms.m[i % ms.na];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double u = v[d * n + i];
      acc[0] += 0.5 * m * u * u;
      acc[1 + d] += m * u;
    }
  }
  __shared__ double sm[kNoAllocThreads / 32][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) sm[threadIdx.x >> 5][j] = acc[j];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double t = 0.0;
      for (int w = 0; w < kNoAllocThreads / 32; ++w) t += sm[w][j];
      scratch[blockIdx.x * 4 + j] = t;
    }
}

// One block adds the partial sums of the first `nblocks` slots in a fixed order.
__global__ void __launch_bounds__(kNoAllocThreads) k_kinetic_final(const double* scratch, int nblocks, double* out) {
  __shared__ double sm[kNoAllocThreads / 32][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += scratch[k * 4 + j];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) sm[threadIdx.x >> 5][j] = acc[j];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double t = 0.0;
      for (int w = 0; w < kNoAllocThreads / 32; ++w) t += sm[w][j];
      out[j] = t;
    }
}

// Device address of the scratch array, looked up once per device with that device current
// and kept for the life of the process (the device's primary context is assumed never to be
// reset while the library is loaded).
static std::mutex g_scratch_mutex;
static double* g_scratch_ptr[kNoAllocMaxDevices] = {};

static cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_kinetic_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace adress

using namespace adress;

extern "C" adress_status adress_kinetic_noalloc(const double* v, int64_t n_atoms, int32_t atoms_per_mol,
                                                const double* mass, void* stream, double* out) {
  if (!v || !out || !mass) return set_global_error(ADRESS_ERR_ARG, "adress_kinetic_noalloc: NULL pointer");
  if (atoms_per_mol < 1 || atoms_per_mol > kMaxNA)
    return set_global_error(ADRESS_ERR_ARG, "adress_kinetic_noalloc: atoms_per_mol must be in 1..4");
  if (n_atoms < 1 || n_atoms > kNoAllocMaxAtoms)
    return set_global_error(ADRESS_ERR_ARG, "adress_kinetic_noalloc: n_atoms must be in 1.." +
                                                std::to_string(kNoAllocMaxAtoms) +
                                                " (the fixed scratch holds 1024 blocks x 256 threads x 64 atoms)");
  NoAllocMasses ms{};
  ms.na = atoms_per_mol;
  for (int k = 0; k < atoms_per_mol; ++k) ms.m[k] = mass[k];
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return set_global_error(ADRESS_ERR_CUDA, std::string("adress_kinetic_noalloc: scratch address: ") +
                                                 cudaGetErrorString(e));
  const long long want = (n_atoms + kNoAllocThreads - 1) / kNoAllocThreads;
  const int nblocks = (int)(want < kNoAllocMaxBlocks ? want : kNoAllocMaxBlocks);
  cudaStream_t st = (cudaStream_t)stream;
  // every slot the final pass reads is written by this call's first pass, so no clearing
  // is needed; slots past nblocks keep an earlier call's values and are never read
  k_kinetic_partials<<<nblocks, kNoAllocThreads, 0, st>>>(v, (long long)n_atoms, ms, scratch);
  k_kinetic_final<<<1, kNoAllocThreads, 0, st>>>(scratch, nblocks, out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_global_error(ADRESS_ERR_CUDA, std::string("adress_kinetic_noalloc: launch: ") + cudaGetErrorString(e));
  return ADRESS_OK;
}
