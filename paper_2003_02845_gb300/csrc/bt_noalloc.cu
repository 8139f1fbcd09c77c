// bt_noalloc.cu -- weighted totals of a distribution without any device
// allocation.
//
// This entry point exists for callers that cannot allocate device memory:
// a host code whose own allocator owns all device memory and forbids raw
// cudaMalloc, a real-time loop that must not allocate, or a process whose
// memory budget is fixed before the transport library is loaded.  The
// per-block partial sums live in a file-scope __device__ array of fixed size
// instead of a workspace; every GPU that loads this library holds that array
// until the process exits.
//
// The array's name in host code is a host-side stand-in, not a device
// address, so the first call on each device looks up the real address with
// cudaGetSymbolAddress (with that device current) and caches it.  That first
// call should therefore happen before any stream capture begins.
//
// All calls share the one array and the kernel overwrites every slot it later
// reads, so no clearing is needed between calls; calls that overlap on the
// GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "bt.h"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kZonesPerBlock = 64;

// the scratch: one compensated partial (sum, compensation) per block
__device__ __align__(256) double g_noalloc_partials[2 * BT_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices];   // device address of the array, per device
std::mutex g_partials_mutex;


__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

// block (species s, zone chunk) -> partial of sum w_za[z][b] w_e[i] f[s][z][i][b]
template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) k_partials(const T* f, const double* w_za, const double* w_e,
                                                               int n_zone, int n_e, int n_ang, int chunks,
                                                               double* partials) {
  __shared__ double ss[kNoAllocThreads], cc[kNoAllocThreads];
  const int s = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
  const int z0 = chunk * kZonesPerBlock, z1 = min(z0 + kZonesPerBlock, n_zone);
  const size_t per_zone = (size_t)n_e * n_ang;
  double sum = 0.0, comp = 0.0;
  for (size_t q = threadIdx.x; q < (size_t)(z1 - z0) * per_zone; q += kNoAllocThreads) {
    const int z = z0 + (int)(q / per_zone);
    const int r = (int)(q % per_zone);
    const int i = r / n_ang, b = r % n_ang;
    const double v = w_za[(size_t)z * n_ang + b] * w_e[i] * (double)f[((size_t)s * n_zone + z) * per_zone + r];
    neumaier_add(sum, comp, v);
  }
  ss[threadIdx.x] = sum;
  cc[threadIdx.x] = comp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int t = 0; t < kNoAllocThreads; ++t) { neumaier_add(S, C, ss[t]); C += cc[t]; }
    partials[2 * blockIdx.x] = S;
    partials[2 * blockIdx.x + 1] = C;
  }
}

// out[s] = compensated sum of the species' partials
__global__ void __launch_bounds__(kNoAllocThreads) k_finish(const double* partials, int chunks, double* out) {
  __shared__ double ss[kNoAllocThreads], cc[kNoAllocThreads];
  const int s = blockIdx.x;
  double sum = 0.0, comp = 0.0;
  for (int c = threadIdx.x; c < chunks; c += kNoAllocThreads) {
    neumaier_add(sum, comp, partials[2 * (s * chunks + c)]);
    comp += partials[2 * (s * chunks + c) + 1];
  }
  ss[threadIdx.x] = sum;
  cc[threadIdx.x] = comp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int t = 0; t < kNoAllocThreads; ++t) { neumaier_add(S, C, ss[t]); C += cc[t]; }
    out[s] = S + C;
  }
}

int noalloc_fail(int code, const std::string&) { return code; }

}  // namespace

extern "C" int bt_weighted_totals_noalloc(const void* f, int precision, int n_s, int n_zone, int n_e, int n_ang,
                                          const double* w_za, const double* w_e, double* out, void* stream) {
  if (!f || !w_za || !w_e || !out) return noalloc_fail(BT_ERR_ARG, "NULL pointer");
  if (n_s < 1 || n_zone < 1 || n_e < 1 || n_ang < 1) return noalloc_fail(BT_ERR_ARG, "sizes must be >= 1");
  if (precision != BT_FP64 && precision != BT_MIXED) return noalloc_fail(BT_ERR_ARG, "precision");
  const int chunks = (n_zone + kZonesPerBlock - 1) / kZonesPerBlock;
  if ((long long)n_s * chunks > BT_NOALLOC_MAX_PARTIALS)
    return noalloc_fail(BT_ERR_ARG, "n_species * ceil(n_zone / 64) exceeds BT_NOALLOC_MAX_PARTIALS (" +
                                        std::to_string(BT_NOALLOC_MAX_PARTIALS) + ")");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(BT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(BT_ERR_ARG, "device index out of range");
  double* partials;
  {
    std::lock_guard<std::mutex> lock(g_partials_mutex);
    if (!g_partials_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_partials);   // device `dev` is current
      if (e != cudaSuccess)
        return noalloc_fail(BT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_partials_addr[dev] = static_cast<double*>(p);
    }
    partials = g_partials_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == BT_FP64)
    k_partials<double><<<n_s * chunks, kNoAllocThreads, 0, s>>>(static_cast<const double*>(f), w_za, w_e, n_zone,
                                                                  n_e, n_ang, chunks, partials);
  else
    k_partials<float><<<n_s * chunks, kNoAllocThreads, 0, s>>>(static_cast<const float*>(f), w_za, w_e, n_zone, n_e,
                                                                 n_ang, chunks, partials);
  k_finish<<<n_s, kNoAllocThreads, 0, s>>>(partials, chunks, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(BT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return BT_OK;
}
