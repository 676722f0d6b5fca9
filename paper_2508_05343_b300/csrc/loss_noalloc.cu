// A variant of the photometric-loss reduction that needs no caller-provided scratch.
//
// gabsplat_loss() asks the caller for a scratch buffer that holds one partial sum per CTA.  Some
// callers cannot hand out device memory: a plug-in running inside another engine's frame loop
// whose allocator owns the whole device heap, or a service under a fixed memory budget that
// forbids allocations once it is running.  gabsplat_loss_noalloc() keeps those partial sums in a
// fixed array compiled into the library instead, so the caller passes only inputs and outputs.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace gs {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_ITEMS = 16;                                        // values per thread
constexpr long long NOALLOC_CHUNK = (long long)NOALLOC_THREADS * NOALLOC_ITEMS;   // values per CTA

// One double per CTA, 64 KB in total.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_loss_partials[GS_LOSS_NOALLOC_MAX_COUNT / NOALLOC_CHUNK];

// Each CTA reduces one contiguous chunk of NOALLOC_CHUNK values and writes its own slot, so every
// slot the final kernel reads was written by this call: nothing has to start at zero.
__global__ void __launch_bounds__(NOALLOC_THREADS) k_loss_noalloc_partial(const float* __restrict__ img,
                                                                        const float* __restrict__ tgt,
                                                                        long long count, int kind,
                                                                        float* __restrict__ dL,
                                                                        double* __restrict__ partials) {
  __shared__ double s_sum[NOALLOC_THREADS / 32];
  const double invN = 1.0 / (double)count;
  const long long base = (long long)blockIdx.x * NOALLOC_CHUNK;
  double acc = 0.0;
#pragma unroll 4
  for (int it = 0; it < NOALLOC_ITEMS; ++it) {
    const long long i = base + (long long)it * NOALLOC_THREADS + threadIdx.x;
    if (i < count) {
      const float d = img[i] - tgt[i];
      if (kind == GS_LOSS_L1) {
        acc += fabs((double)d);
        dL[i] = (float)((d > 0.f ? 1.0 : (d < 0.f ? -1.0 : 0.0)) * invN);
      } else {
        acc += (double)d * (double)d;
        dL[i] = (float)(2.0 * (double)d * invN);
      }
    }
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NOALLOC_THREADS / 32; ++w) s += s_sum[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void k_loss_noalloc_final(const double* __restrict__ partials, int n, long long count, double* out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += partials[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] / (double)count;
}

// Device address of the partials array, looked up once per device with that device current.
// In host code the symbol g_loss_partials is only a host-side stand-in, never a device address.
// The cached address belongs to the device's primary context as it was at the lookup: after a
// cudaDeviceReset of that device it is stale (the header says so).  Reads take no lock; the
// mutex only serialises the first lookup on a device.
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::atomic<double*> g_partials_dev[NOALLOC_MAX_DEVICES];
static std::mutex g_partials_mutex;

static cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  double* p = g_partials_dev[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_partials_mutex);
    p = g_partials_dev[dev].load(std::memory_order_relaxed);
    if (!p) {
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_loss_partials);
      if (e != cudaSuccess) return e;
      p = reinterpret_cast<double*>(a);
      g_partials_dev[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return cudaSuccess;
}

}  // namespace gs

extern "C" gs_status gabsplat_loss_noalloc(const float* image, const float* target, long long count, int kind,
                                           double* loss_out, float* dL_dimage, gs_stream stream) {
  using namespace gs;
  if (!image || !target || !loss_out || !dL_dimage || count <= 0) return GS_ERR_INVALID_ARG;
  if (kind != GS_LOSS_L1 && kind != GS_LOSS_L2) return GS_ERR_INVALID_ARG;
  if (count > GS_LOSS_NOALLOC_MAX_COUNT) return GS_ERR_INVALID_ARG;   // beyond the fixed scratch
  double* partials = nullptr;
  if (partials_address(&partials) != cudaSuccess) return GS_ERR_CUDA;
  const int blocks = (int)((count + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_loss_noalloc_partial<<<blocks, NOALLOC_THREADS, 0, s>>>(image, target, count, kind, dL_dimage, partials);
  k_loss_noalloc_final<<<1, 256, 0, s>>>(partials, blocks, count, loss_out);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
