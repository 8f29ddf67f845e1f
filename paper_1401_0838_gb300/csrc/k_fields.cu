// Grid kernels: the Psi z-stencil + binomial/compensation filter (one separable stencil kernel),
// the Yee curl updates and the FP64 energy reductions.
#include "common.cuh"
#include "launch.h"

#include <mutex>
#include <unordered_map>

namespace picgb {

cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> enabled;
  std::lock_guard<std::mutex> lock(mu);
  auto it = enabled.find(kernel);
  if (it != enabled.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) enabled[kernel] = bytes;
  return e;
}

// ---------------------------------------------------------------------------------------------
// Separable periodic stencil. One CTA computes a CX x CY x CZ output tile of one component:
// the input tile plus halos is staged in shared memory, then reduced along z, y and x in turn.
// Sec. 2 (Psi(D_z), 9 taps) and Sec. 3 Eq. 6 / Sec. 4 (filter) are combined into these taps on
// the host, in FP64.
// ---------------------------------------------------------------------------------------------
constexpr int SEP_THREADS = 256;
constexpr int SEP2_CX = 64, SEP2_CZ = 16;               // 2D tile
constexpr int SEP3_CX = 32, SEP3_CY = 4, SEP3_CZ = 8;   // 3D tile

template <typename T>
__global__ void __launch_bounds__(SEP_THREADS) k_sep(SepArgs<T> a, int CX, int CY, int CZ, int ntx, int nty) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* s0 = reinterpret_cast<T*>(smraw);
  const int comp = blockIdx.y;
  const T* __restrict__ src = a.src[comp];
  T* __restrict__ dst = a.dst[comp];
  const int zs = a.zset[comp];
  const int hz = a.hz[zs], hx = a.hx, hy = a.ndim == 3 ? a.hy : 0;
  const int tile = blockIdx.x;
  const int tix = tile % ntx, tiy = (tile / ntx) % nty, tiz = tile / (ntx * nty);
  const int X0 = tix * CX, Y0 = tiy * CY, Z0 = tiz * CZ;
  const int LX = CX + 2 * hx, LY = CY + 2 * hy, LZ = CZ + 2 * hz;
  const long long nxy = (long long)a.nx * a.ny;

  for (int e = threadIdx.x; e < LX * LY * LZ; e += SEP_THREADS) {
    int lx = e % LX, ly = (e / LX) % LY, lz = e / (LX * LY);
    int gx = wrapi(X0 - hx + lx, a.nx);
    int gy = a.ndim == 3 ? wrapi(Y0 - hy + ly, a.ny) : 0;
    int gz = wrapi(Z0 - hz + lz, a.nz);
    s0[e] = __ldg(src + gz * nxy + (long long)gy * a.nx + gx);
  }
  __syncthreads();
  // z pass: LX x LY x CZ
  T* s1 = s0 + LX * LY * LZ;
  const T* zt = a.zt[zs];
  for (int e = threadIdx.x; e < LX * LY * CZ; e += SEP_THREADS) {
    int lx = e % LX, ly = (e / LX) % LY, lz = e / (LX * LY);
    const T* p = s0 + (lz * LY + ly) * LX + lx;
    T acc = T(0);
    for (int m = 0; m <= 2 * hz; ++m) acc += zt[m] * p[m * LX * LY];
    s1[e] = acc;
  }
  __syncthreads();
  // y pass (3D): LX x CY x CZ
  T* s2 = s1;
  if (a.ndim == 3) {
    s2 = s1 + LX * LY * CZ;
    for (int e = threadIdx.x; e < LX * CY * CZ; e += SEP_THREADS) {
      int lx = e % LX, ly = (e / LX) % CY, lz = e / (LX * CY);
      const T* p = s1 + (lz * LY + ly) * LX + lx;
      T acc = T(0);
      for (int m = 0; m <= 2 * hy; ++m) acc += a.yt[m] * p[m * LX];
      s2[e] = acc;
    }
    __syncthreads();
  }
  const int SY = a.ndim == 3 ? CY : LY;  // y extent of s2 (LY = 1 in 2D)
  // x pass -> global
  for (int e = threadIdx.x; e < CX * CY * CZ; e += SEP_THREADS) {
    int lx = e % CX, ly = (e / CX) % CY, lz = e / (CX * CY);
    int gx = X0 + lx, gy = Y0 + ly, gz = Z0 + lz;
    if (gx >= a.nx || gy >= (a.ndim == 3 ? a.ny : 1) || gz >= a.nz) continue;
    const T* p = s2 + (lz * SY + ly) * LX + lx;
    T acc = T(0);
    for (int m = 0; m <= 2 * hx; ++m) acc += a.xt[m] * p[m];
    dst[gz * nxy + (long long)gy * a.nx + gx] = acc;
  }
}

template <typename T>
cudaError_t launch_sep(const SepArgs<T>& a, cudaStream_t st) {
  int CX, CY, CZ;
  if (a.ndim == 2) {
    CX = SEP2_CX; CY = 1; CZ = SEP2_CZ;
  } else {
    CX = SEP3_CX; CY = SEP3_CY; CZ = SEP3_CZ;
  }
  int hzmax = a.hz[0] > a.hz[1] ? a.hz[0] : a.hz[1];
  int hy = a.ndim == 3 ? a.hy : 0;
  int LX = CX + 2 * a.hx, LY = CY + 2 * hy, LZ = CZ + 2 * hzmax;
  size_t sm = sizeof(T) * ((size_t)LX * LY * LZ + (size_t)LX * LY * CZ + (a.ndim == 3 ? (size_t)LX * CY * CZ : 0));
  int ntx = (a.nx + CX - 1) / CX, nty = a.ndim == 3 ? (a.ny + CY - 1) / CY : 1, ntz = (a.nz + CZ - 1) / CZ;
  cudaError_t e = ensure_dynamic_smem((const void*)k_sep<T>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(ntx * nty * ntz), (unsigned)a.ncomp);
  k_sep<T><<<grid, SEP_THREADS, sm, st>>>(a, CX, CY, CZ, ntx, nty);
  return cudaGetLastError();
}
template cudaError_t launch_sep<float>(const SepArgs<float>&, cudaStream_t);
template cudaError_t launch_sep<double>(const SepArgs<double>&, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Yee updates on the periodic staggered mesh (x fastest). One thread per cell.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_yee_b(YeeArgs<T> a) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nxy = (long long)a.nx * a.ny, n = nxy * a.nz;
  if (c >= n) return;
  int i = (int)(c % a.nx), j = (int)((c / a.nx) % a.ny), k = (int)(c / nxy);
  long long ip = c - i + (i + 1 == a.nx ? 0 : i + 1);
  long long jp = c + ((j + 1 == a.ny ? 0 : j + 1) - j) * (long long)a.nx;
  long long kp = c + ((k + 1 == a.nz ? 0 : k + 1) - k) * nxy;
  T ex = a.ex[c], ey = a.ey[c], ez = a.ez[c];
  // B -= h curl E
  a.bx[c] -= a.cy * (a.ez[jp] - ez) - a.cz * (a.ey[kp] - ey);
  a.by[c] -= a.cz * (a.ex[kp] - ex) - a.cx * (a.ez[ip] - ez);
  a.bz[c] -= a.cx * (a.ey[ip] - ey) - a.cy * (a.ex[jp] - ex);
}

template <typename T>
__global__ void k_yee_e(YeeArgs<T> a) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nxy = (long long)a.nx * a.ny, n = nxy * a.nz;
  if (c >= n) return;
  int i = (int)(c % a.nx), j = (int)((c / a.nx) % a.ny), k = (int)(c / nxy);
  long long im = c - i + (i == 0 ? a.nx - 1 : i - 1);
  long long jm = c + ((j == 0 ? a.ny - 1 : j - 1) - j) * (long long)a.nx;
  long long km = c + ((k == 0 ? a.nz - 1 : k - 1) - k) * nxy;
  T bx = a.bx[c], by = a.by[c], bz = a.bz[c];
  // E += h (curl B - J)
  a.ex[c] += a.cy * (bz - a.bz[jm]) - a.cz * (by - a.by[km]) - a.h * a.jx[c];
  a.ey[c] += a.cz * (bx - a.bx[km]) - a.cx * (bz - a.bz[im]) - a.h * a.jy[c];
  a.ez[c] += a.cx * (by - a.by[im]) - a.cy * (bx - a.bx[jm]) - a.h * a.jz[c];
}

template <typename T>
cudaError_t launch_yee_b(const YeeArgs<T>& a, cudaStream_t st) {
  long long n = (long long)a.nx * a.ny * a.nz;
  k_yee_b<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_yee_e(const YeeArgs<T>& a, cudaStream_t st) {
  long long n = (long long)a.nx * a.ny * a.nz;
  k_yee_e<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_yee_b<float>(const YeeArgs<float>&, cudaStream_t);
template cudaError_t launch_yee_b<double>(const YeeArgs<double>&, cudaStream_t);
template cudaError_t launch_yee_e<float>(const YeeArgs<float>&, cudaStream_t);
template cudaError_t launch_yee_e<double>(const YeeArgs<double>&, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// FP64 reductions
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void k_field_energy(const T* __restrict__ ex, const T* __restrict__ ey, const T* __restrict__ ez,
                               const T* __restrict__ bx, const T* __restrict__ by, const T* __restrict__ bz,
                               long long n, double* out) {
  double se = 0, sb = 0, sp = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    double x2 = (double)ex[c] * ex[c], y2 = (double)ey[c] * ey[c], z2 = (double)ez[c] * ez[c];
    double u2 = (double)bx[c] * bx[c], v2 = (double)by[c] * by[c], w2 = (double)bz[c] * bz[c];
    se += x2 + y2 + z2;
    sb += u2 + v2 + w2;
    sp += x2 + y2 + u2 + v2;
  }
  __shared__ double red[3][32];
  se = warp_sum(se);
  sb = warp_sum(sb);
  sp = warp_sum(sp);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = se;
    red[1][w] = sb;
    red[2][w] = sp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0, 0, 0};
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
      for (int r = 0; r < 3; ++r) t[r] += red[r][q];
    atomicAdd(out + 0, t[0]);
    atomicAdd(out + 1, t[1]);
    atomicAdd(out + 2, t[2]);
  }
}

template <typename T>
cudaError_t launch_field_energy(const T* const f6[6], long long ncell, double* out, cudaStream_t st) {
  int blocks = (int)((ncell + 255) / 256);
  if (blocks > 4 * 152 * 8) blocks = 4 * 152 * 8;
  if (blocks < 1) blocks = 1;
  k_field_energy<T><<<blocks, 256, 0, st>>>(f6[0], f6[1], f6[2], f6[3], f6[4], f6[5], ncell, out);
  return cudaGetLastError();
}
template cudaError_t launch_field_energy<float>(const float* const*, long long, double*, cudaStream_t);
template cudaError_t launch_field_energy<double>(const double* const*, long long, double*, cudaStream_t);

template <typename T>
__global__ void k_kinetic(RunDev<T> r, double* out) {
  double acc = 0;
  for (int s = 0; s < 2; ++s) {
    const SpeciesBuf<T> b = r.in[s];
    for (long long c = blockIdx.x * (long long)blockDim.y + threadIdx.y; c < r.ncell;
         c += (long long)gridDim.x * blockDim.y) {
      int n = b.cnt[c];
      n = n > r.cap ? r.cap : n;
      for (int j = threadIdx.x; j < n; j += 32) {
        long long o = c * r.cap + j;
        double ux = b.dux[o], uy = b.duy[o], uz = (double)r.u0 + (double)b.duz[o];
        double u2 = ux * ux + uy * uy + uz * uz;
        double w = b.w ? (double)b.w[o] : (double)r.wconst;
        acc += w * u2 / (sqrt(1.0 + u2) + 1.0);
      }
    }
  }
  acc = warp_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

template <typename T>
cudaError_t launch_kinetic(const RunDev<T>& r, double* out, cudaStream_t st) {
  dim3 blk(32, 8);
  long long blocks = (r.ncell + 7) / 8;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  k_kinetic<T><<<(unsigned)blocks, blk, 0, st>>>(r, out);
  return cudaGetLastError();
}
template cudaError_t launch_kinetic<float>(const RunDev<float>&, double*, cudaStream_t);
template cudaError_t launch_kinetic<double>(const RunDev<double>&, double*, cudaStream_t);

}  // namespace picgb
