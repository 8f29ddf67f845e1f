// Field energies without any memory allocation (pic_field_energy_noalloc in include/pic.h).
//
// Some callers cannot allocate device memory at the point where they want the energies: plugins
// whose host application owns every device allocation (its own pool, cudaMalloc not theirs to
// call), monitoring hooks that must not change the memory footprint of the run they observe, and
// code that runs when the device is nearly full, where an allocation could fail or evict. This
// entry point serves them: the caller passes the six field arrays and a host array for the three
// results, and the per-block partial sums live in one fixed array of this library's device memory
// (kFeScratchBlocks x 3 doubles, 96 KiB, held by every GPU that loads the library until the
// process exits).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pic.h"

namespace {

constexpr int kFeThreads = 256;
constexpr long long kFeCellsPerBlock = 4096;  // each block sums a fixed chunk, in a fixed order
constexpr int kFeScratchBlocks = 4096;        // => at most 16,777,216 cells per call
constexpr int kFeMaxDevices = 64;

// [0, 3*kFeScratchBlocks): block partials (sum E^2, sum B^2, sum Ex^2+Ey^2+Bx^2+By^2);
// [3*kFeScratchBlocks, +3): the final sums. Shared by every call on a device.
static __device__ __align__(256) double g_fe_scratch[3 * kFeScratchBlocks + 4];

std::mutex g_fe_mu;
double* g_fe_addr[kFeMaxDevices] = {};  // device address of g_fe_scratch, per device

__device__ __forceinline__ double fe_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kFeThreads) k_fe_partials(const T* __restrict__ ex, const T* __restrict__ ey,
                                                            const T* __restrict__ ez, const T* __restrict__ bx,
                                                            const T* __restrict__ by, const T* __restrict__ bz,
                                                            long long ncell, double* scratch) {
  const long long c0 = blockIdx.x * kFeCellsPerBlock;
  const long long c1 = c0 + kFeCellsPerBlock < ncell ? c0 + kFeCellsPerBlock : ncell;
  double se = 0, sb = 0, sp = 0;
  for (long long c = c0 + threadIdx.x; c < c1; c += kFeThreads) {
    const double x2 = (double)ex[c] * ex[c], y2 = (double)ey[c] * ey[c], z2 = (double)ez[c] * ez[c];
    const double u2 = (double)bx[c] * bx[c], v2 = (double)by[c] * by[c], w2 = (double)bz[c] * bz[c];
    se += x2 + y2 + z2;
    sb += u2 + v2 + w2;
    sp += x2 + y2 + u2 + v2;
  }
  __shared__ double red[3][kFeThreads / 32];
  se = fe_warp_sum(se);
  sb = fe_warp_sum(sb);
  sp = fe_warp_sum(sp);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = se;
    red[1][w] = sb;
    red[2][w] = sp;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0;
    for (int q = 0; q < kFeThreads / 32; ++q) t += red[threadIdx.x][q];
    scratch[3 * blockIdx.x + threadIdx.x] = t;  // every used slot is overwritten by every call
  }
}

__global__ void k_fe_final(double* scratch, int nblocks) {
  const int r = threadIdx.x;  // 3 threads, one per sum, blocks added in order
  if (r >= 3) return;
  double t = 0;
  for (int b = 0; b < nblocks; ++b) t += scratch[3 * b + r];
  scratch[3 * kFeScratchBlocks + r] = t;
}

// Address of g_fe_scratch on the current device, looked up once per device (on the first call there)
// and kept for the life of the process; a cudaDeviceReset of that device invalidates it.
int fe_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kFeMaxDevices) return PIC_E_CUDA;
  std::lock_guard<std::mutex> lock(g_fe_mu);
  if (!g_fe_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fe_scratch) != cudaSuccess || !p) return PIC_E_CUDA;
    g_fe_addr[dev] = static_cast<double*>(p);
  }
  *out = g_fe_addr[dev];
  return PIC_OK;
}

}  // namespace

extern "C" int pic_field_energy_noalloc(const void* const fields[6], long long ncell, int precision, double dv,
                                        double out[3], void* stream) {
  if (!fields || !out || ncell < 1 || !(dv > 0) || (precision != PIC_FP32 && precision != PIC_FP64)) return PIC_E_ARG;
  for (int q = 0; q < 6; ++q)
    if (!fields[q]) return PIC_E_ARG;
  if (ncell > kFeCellsPerBlock * kFeScratchBlocks) return PIC_E_ARG;  // beyond the fixed scratch
  double* scratch = nullptr;
  int rc = fe_scratch(&scratch);
  if (rc != PIC_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nblocks = (int)((ncell + kFeCellsPerBlock - 1) / kFeCellsPerBlock);
  if (precision == PIC_FP32) {
    const float* const* f = reinterpret_cast<const float* const*>(fields);
    k_fe_partials<float><<<nblocks, kFeThreads, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5], ncell, scratch);
  } else {
    const double* const* f = reinterpret_cast<const double* const*>(fields);
    k_fe_partials<double><<<nblocks, kFeThreads, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5], ncell, scratch);
  }
  k_fe_final<<<1, 32, 0, st>>>(scratch, nblocks);
  double sums[3];
  // peek, not get: an error the caller left pending stays theirs to read (and fails this call too)
  if (cudaPeekAtLastError() != cudaSuccess) return PIC_E_CUDA;
  if (cudaMemcpyAsync(sums, scratch + 3 * kFeScratchBlocks, sizeof sums, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIC_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_E_CUDA;
  for (int r = 0; r < 3; ++r) out[r] = 0.5 * sums[r] * dv;
  return PIC_OK;
}
