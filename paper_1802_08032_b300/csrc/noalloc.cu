// calcTotalProbNoAlloc: the total-probability reduction with no device
// allocation, for callers that must not call cudaMalloc.
//
// Some host programs cannot allocate device memory at the point where they
// need a norm: code running inside a framework that owns every byte of the
// device through its own pool, plug-ins handed a fixed buffer, or callers
// that must not trigger the device-wide synchronisation an allocation can
// cause.  calcTotalProb needs an environment, whose creation allocates its
// scratch; this entry point needs none.  Its scratch (one FP64 partial sum
// per CTA) lives in a file-scope __device__ array of fixed size that every
// GPU using the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "runtime.h"

namespace {

// Each CTA sums a fixed chunk of amplitudes; the scratch holds one partial per
// CTA, so it bounds the largest accepted array.
constexpr int kNaThreads = 512;
constexpr int64_t kNaChunk = int64_t(1) << 14;     // amplitudes per CTA
constexpr int kNaMaxPartials = 1 << 16;            // 65536 doubles = 512 KiB
constexpr int64_t kNaMaxAmps = kNaChunk * kNaMaxPartials;  // 2^30 amplitudes

static __device__ __align__(256) double g_na_partials[kNaMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
double* g_na_ptr[kMaxDevices] = {};

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// CTA b sums |a_j|^2 over j in [b*chunk, min((b+1)*chunk, n)) into partial[b].
template <typename V>
__global__ void __launch_bounds__(kNaThreads) k_na_chunks(const V* __restrict__ a, int64_t n,
                                                          double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t begin = int64_t(blockIdx.x) * kNaChunk;
  const int64_t end = begin + kNaChunk < n ? begin + kNaChunk : n;
  double acc = 0.0;
  for (int64_t j = begin + threadIdx.x; j < end; j += kNaThreads) {
    const V v = a[j];
    const double re = double(v.x), im = double(v.y);
    acc = fma(re, re, acc);
    acc = fma(im, im, acc);
  }
  const double s = na_block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[0] = sum of partial[0..count) in a fixed order.
__global__ void __launch_bounds__(1024) k_na_final(const double* __restrict__ partial, int count,
                                                   double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
  const double s = na_block_sum(acc, sh);
  if (threadIdx.x == 0) out[0] = s;
}

int na_fail(int code, const std::string& msg) {
  qs::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" {

int calcTotalProbNoAlloc(const void* amps, int precision, int64_t numAmps, double* out,
                         void* stream) {
  if (!amps || !out) return na_fail(QS_E_ARG, "null amplitude or output pointer");
  if (precision != QS_C64 && precision != QS_C128)
    return na_fail(QS_E_ARG, "precision must be QS_C64 or QS_C128");
  // the kernels read 16-byte (complex128) or 8-byte (complex64) amplitudes
  // and write one double: a misaligned pointer would fault on the device
  const uintptr_t amp_align = precision == QS_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(amps) % amp_align != 0)
    return na_fail(QS_E_ARG, "amps is not aligned to " + std::to_string(amp_align) +
                                 " bytes (one amplitude)");
  if (reinterpret_cast<uintptr_t>(out) % 8 != 0)
    return na_fail(QS_E_ARG, "out is not aligned to 8 bytes (one double)");
  if (numAmps < 1 || numAmps > kNaMaxAmps)
    return na_fail(QS_E_ARG, "numAmps " + std::to_string(numAmps) + " outside [1, " +
                                 std::to_string(kNaMaxAmps) +
                                 "]: the fixed scratch holds one partial per 16384 amplitudes, "
                                 "65536 partials at most");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(QS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(QS_E_CUDA, "device index beyond the supported range");
  double* scratch = nullptr;
  {
    // first call on this device: device address of the scratch array, taken
    // with the device current (the host-side name is not a device address).
    // The address is kept for the life of the process; cudaDeviceReset
    // unloads the module and invalidates it.
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_partials);
      if (e != cudaSuccess)
        return na_fail(QS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  // An error left pending by earlier, unrelated work belongs to its owner:
  // report it without clearing it and launch nothing, so that the error
  // checked after the launches below is this call's own.
  e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return na_fail(QS_E_CUDA, std::string("a CUDA error from earlier work is pending (not cleared): ") +
                                  cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = int((numAmps + kNaChunk - 1) / kNaChunk);
  // every partial the final kernel reads is written by this call first, so
  // nothing in the scratch needs clearing
  if (precision == QS_C128)
    k_na_chunks<double2><<<blocks, kNaThreads, 0, s>>>(static_cast<const double2*>(amps), numAmps, scratch);
  else
    k_na_chunks<float2><<<blocks, kNaThreads, 0, s>>>(static_cast<const float2*>(amps), numAmps, scratch);
  k_na_final<<<1, 1024, 0, s>>>(scratch, blocks, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(QS_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return QS_OK;
}

}  // extern "C"
