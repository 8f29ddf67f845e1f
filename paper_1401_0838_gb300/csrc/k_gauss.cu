// Charge-conservation diagnostic: the residual of Gauss's law div E - F rho on the integer nodes.
//
// The Esirkepov deposit (cited in Sec. 2) makes the current satisfy the discrete continuity equation
// with the charge density rho of the particles' own shapes, and the Yee E update subtracts the
// filtered current F J, so div E - F rho keeps its initial value (zero for the neutral beam) up to
// rounding. These kernels compute that residual in FP64 from the live state: rho deposited from the
// particle bins with the B-spline of the run's shape order, filtered by the current filter's taps
// (the separable stencil kernel in FP64), then reduced node by node.
#include "common.cuh"
#include "launch.h"

namespace picgb {

constexpr int RHO_THREADS = 256;
constexpr int GR_THREADS = 256;
constexpr int GR_BLOCKS = 4 * 152;

// Weights of the nodes base, base + 1, ... for offset o in [0, 1) inside the cell: order 1 on the
// cell's two nodes (base = cell), order 3 the cubic B-spline on four nodes (base = cell - 1).
__device__ __forceinline__ void node_weights(int order, double o, double (&w)[4]) {
  if (order == 3) {
    const double p = 1.0 - o;
    w[0] = p * p * p / 6.0;
    w[1] = (4.0 - 6.0 * o * o + 3.0 * o * o * o) / 6.0;
    w[2] = (4.0 - 6.0 * p * p + 3.0 * p * p * p) / 6.0;
    w[3] = o * o * o / 6.0;
  } else {
    w[0] = 1.0 - o;
    w[1] = o;
    w[2] = 0.0;
    w[3] = 0.0;
  }
}

__device__ __forceinline__ int wrap_any(int g, int n) {
  g %= n;
  return g < 0 ? g + n : g;
}

// rho += q w S(x - x_node) / dV for every particle: one warp per cell, lanes over its slots.
template <typename T>
__global__ void __launch_bounds__(RHO_THREADS) k_rho(const __grid_constant__ RunDev<T> r, int order, double inv_dv,
                                                     double* __restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (RHO_THREADS / 32);
  const long long nxy = (long long)r.nx * r.ny;
  const int nn = order == 3 ? 4 : 2, lo = order == 3 ? -1 : 0;
  for (long long cell = blockIdx.x * (long long)(RHO_THREADS / 32) + (threadIdx.x >> 5); cell < r.ncell;
       cell += warps) {
    const int i = (int)(cell % r.nx), j = (int)((cell / r.nx) % r.ny), k = (int)(cell / nxy);
    for (int s = 0; s < 2; ++s) {
      const SpeciesBuf<T>& b = s ? r.in[1] : r.in[0];
      const int n = min(b.cnt[cell], r.cap);
      const double q = s ? 1.0 : -1.0;
      for (int slot = lane; slot < n; slot += 32) {
        const long long o = cell * r.cap + slot;
        const double qw = q * (b.w ? (double)b.w[o] : (double)r.wconst) * inv_dv;
        double wx[4], wy[4] = {1.0, 0.0, 0.0, 0.0}, wz[4];
        node_weights(order, (double)b.ox[o], wx);
        if (r.ndim == 3) node_weights(order, (double)b.oy[o], wy);
        node_weights(order, (double)b.oz[o], wz);
        const int ny_n = r.ndim == 3 ? nn : 1;
        for (int c = 0; c < nn; ++c) {
          const long long kz = wrap_any(k + lo + c, r.nz);
          for (int bb = 0; bb < ny_n; ++bb) {
            const long long jy = r.ndim == 3 ? wrap_any(j + lo + bb, r.ny) : 0;
            const double wyz = qw * wy[bb] * wz[c];
            for (int a = 0; a < nn; ++a)
              atomicAdd(rho + (kz * r.ny + jy) * r.nx + wrap_any(i + lo + a, r.nx), wyz * wx[a]);
          }
        }
      }
    }
  }
}

// Node residual res = div E - rho_f (FP64 from the stored precision). Per thread: max |res|, sum
// res^2, max |rho_f|; per block: tree into scratch[3 * block + r]; the last block to finish combines
// the partials in a fixed order and writes out = (max |res|, rms res, max |rho_f|).
template <typename T>
__global__ void __launch_bounds__(GR_THREADS) k_gauss_residual(const T* __restrict__ ex, const T* __restrict__ ey,
                                                               const T* __restrict__ ez,
                                                               const double* __restrict__ rhof, int nx, int ny,
                                                               int nz, double idx, double idy, double idz,
                                                               double* scratch, double* out) {
  const long long nxy = (long long)nx * ny, n = nxy * nz;
  double mres = 0.0, ssq = 0.0, mrho = 0.0;
  for (long long c = blockIdx.x * (long long)GR_THREADS + threadIdx.x; c < n; c += (long long)gridDim.x * GR_THREADS) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / nxy);
    const long long im = c - i + (i == 0 ? nx - 1 : i - 1);
    const long long jm = c + ((j == 0 ? ny - 1 : j - 1) - j) * (long long)nx;
    const long long km = c + ((k == 0 ? nz - 1 : k - 1) - k) * nxy;
    const double dive = ((double)ex[c] - (double)ex[im]) * idx + ((double)ey[c] - (double)ey[jm]) * idy +
                        ((double)ez[c] - (double)ez[km]) * idz;
    const double res = dive - rhof[c];
    mres = fmax(mres, fabs(res));
    ssq += res * res;
    mrho = fmax(mrho, fabs(rhof[c]));
  }
  __shared__ double red[3][GR_THREADS / 32];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mres = fmax(mres, __shfl_xor_sync(0xffffffffu, mres, o));
    ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
    mrho = fmax(mrho, __shfl_xor_sync(0xffffffffu, mrho, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = mres;
    red[1][w] = ssq;
    red[2][w] = mrho;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, s = 0.0, m = 0.0;
    for (int q = 0; q < GR_THREADS / 32; ++q) {
      a = fmax(a, red[0][q]);
      s += red[1][q];
      m = fmax(m, red[2][q]);
    }
    scratch[3 * blockIdx.x + 0] = a;
    scratch[3 * blockIdx.x + 1] = s;
    scratch[3 * blockIdx.x + 2] = m;
  }
  __threadfence();
  __syncthreads();
  unsigned* done = reinterpret_cast<unsigned*>(scratch + 3 * GR_BLOCKS);
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* v = scratch;
    double a = 0.0, s = 0.0, m = 0.0;
    for (unsigned q = 0; q < gridDim.x; ++q) {
      a = fmax(a, v[3 * q + 0]);
      s += v[3 * q + 1];
      m = fmax(m, v[3 * q + 2]);
    }
    out[0] = a;
    out[1] = sqrt(s / (double)n);
    out[2] = m;
    *done = 0u;
  }
}

size_t gauss_scratch_bytes() { return sizeof(double) * (3 * GR_BLOCKS + 2); }

template <typename T>
cudaError_t launch_rho(const RunDev<T>& r, int order, double inv_dv, double* rho, cudaStream_t st) {
  const long long want = (r.ncell + RHO_THREADS / 32 - 1) / (RHO_THREADS / 32);
  const int blocks = (int)(want < 8 * 152 ? (want < 1 ? 1 : want) : 8 * 152);
  k_rho<T><<<blocks, RHO_THREADS, 0, st>>>(r, order, inv_dv, rho);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gauss_residual(const T* ex, const T* ey, const T* ez, const double* rhof, int nx, int ny, int nz,
                                  double idx, double idy, double idz, double* scratch, double* out, cudaStream_t st) {
  const long long n = (long long)nx * ny * nz;
  const long long want = (n + GR_THREADS - 1) / GR_THREADS;
  const int blocks = (int)(want < GR_BLOCKS ? (want < 1 ? 1 : want) : GR_BLOCKS);
  k_gauss_residual<T><<<blocks, GR_THREADS, 0, st>>>(ex, ey, ez, rhof, nx, ny, nz, idx, idy, idz, scratch, out);
  return cudaGetLastError();
}

template cudaError_t launch_rho<float>(const RunDev<float>&, int, double, double*, cudaStream_t);
template cudaError_t launch_rho<double>(const RunDev<double>&, int, double, double*, cudaStream_t);
template cudaError_t launch_gauss_residual<float>(const float*, const float*, const float*, const double*, int, int,
                                                  int, double, double, double, double*, double*, cudaStream_t);
template cudaError_t launch_gauss_residual<double>(const double*, const double*, const double*, const double*, int,
                                                   int, int, double, double, double, double*, double*, cudaStream_t);

}  // namespace picgb
