// Grid kernels: the Psi z-stencil + binomial/compensation filter (one separable stencil kernel),
// the Yee curl updates and the FP64 energy reductions.
#include <cudaTypedefs.h>

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

// The driver's tensor-map encoder, looked up once through the runtime (no link to the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    (void)cudaGetLastError();  // a failed lookup leaves the element-copy staging in use
  });
  return fn;
}

bool tma_encode(CUtensorMap* m, const void* base, int es, int ndim, int nx, int ny, int nz, int bx, int by, int bz) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tma_encoder();
  if (!fn || !base || (es != 4 && es != 8)) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((long long)nx * es) % 16 != 0) return false;
  if (bx < 1 || by < 1 || bz < 1 || bx > 256 || by > 256 || bz > 256 || (bx * es) % 16 != 0) return false;
  const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  cuuint32_t rank;
  if (ndim == 2) {  // (x, z), one y plane
    rank = 2;
    dims[0] = (cuuint64_t)nx;
    dims[1] = (cuuint64_t)nz;
    strides[0] = (cuuint64_t)nx * es;
    box[0] = (cuuint32_t)bx;
    box[1] = (cuuint32_t)bz;
  } else {
    rank = 3;
    dims[0] = (cuuint64_t)nx;
    dims[1] = (cuuint64_t)ny;
    dims[2] = (cuuint64_t)nz;
    strides[0] = (cuuint64_t)nx * es;
    strides[1] = (cuuint64_t)nx * ny * es;
    box[0] = (cuuint32_t)bx;
    box[1] = (cuuint32_t)by;
    box[2] = (cuuint32_t)bz;
  }
  const CUresult r = fn(m, dt, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------------------------
// Separable periodic stencil. One CTA computes a CX x CY x CZ output tile of one component:
// the input tile plus halos is staged in shared memory, then reduced along z, y and x in turn.
// Sec. 2 (Psi(D_z), 9 taps) and Sec. 3 Eq. 6 / Sec. 4 (filter) are combined into these taps on
// the host, in FP64.
// ---------------------------------------------------------------------------------------------
constexpr int SEP_THREADS = 256;
constexpr int SEP2_CX = 128, SEP2_CZ = 32;              // 2D tile
constexpr int SEP3_CX = 32, SEP3_CY = 8, SEP3_CZ = 8;   // 3D tile

// Element-wise asynchronous global -> shared copies (all loads of a staging loop in flight at once).
__device__ __forceinline__ void cp_async_el(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_el(double* dst, const double* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all_fields() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Periodic index of any g: one compare and add in the common case g in [-n, 2n); a modulo only when
// a tile and its halo are wider than the grid (tiles are staged whole, even past the grid's end).
__device__ __forceinline__ int wrap_near(int g, int n) {
  if (g < 0) {
    g += n;
    if (g < 0) g = wrapi(g, n);
  } else if (g >= n) {
    g -= n;
    if (g >= n) g %= n;
  }
  return g;
}

// Periodic index of g in [-n, 2n) with one compare and add (WrapOnce), or of any g (WrapNear). Tile
// staging takes WrapOnce when the grid is at least as wide as the staged tile in every direction
// (then every staged index lies in [-n, 2n)), behind a block-uniform branch.
struct WrapOnce {
  __device__ __forceinline__ int operator()(int g, int n) const { return g < 0 ? g + n : (g >= n ? g - n : g); }
};
struct WrapNear {
  __device__ __forceinline__ int operator()(int g, int n) const { return wrap_near(g, n); }
};

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

  // rows of LX consecutive x, one (ly, lz) pair per row
  for (int row = threadIdx.x / 32; row < LY * LZ; row += SEP_THREADS / 32) {
    const int ly = row % LY, lz = row / LY;
    const int gy = a.ndim == 3 ? wrap_near(Y0 - hy + ly, a.ny) : 0;
    const int gz = wrap_near(Z0 - hz + lz, a.nz);
    const T* srow = src + gz * nxy + (long long)gy * a.nx;
    T* drow = s0 + row * LX;
    for (int lx = threadIdx.x & 31; lx < LX; lx += 32) {
      cp_async_el(drow + lx, srow + wrap_near(X0 - hx + lx, a.nx));
    }
  }
  cp_async_wait_all_fields();
  __syncthreads();
  // z pass: LX x LY x CZ
  T* s1 = s0 + LX * LY * LZ;
  const T* zt = a.zt[zs];
  for (int e = threadIdx.x; e < LX * LY * CZ; e += SEP_THREADS) {
    const int lx = e % LX, ly = (e / LX) % LY, lz = e / (LX * LY);
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
      const int lx = e % LX, ly = (e / LX) % CY, lz = e / (LX * CY);
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
    const int lx = e % CX, ly = (e / CX) % CY, lz = e / (CX * CY);
    const int gx = X0 + lx, gy = Y0 + ly, gz = Z0 + lz;
    if (gx >= a.nx || gy >= (a.ndim == 3 ? a.ny : 1) || gz >= a.nz) continue;
    const T* p = s2 + (lz * SY + ly) * LX + lx;
    T acc = T(0);
    for (int m = 0; m <= 2 * hx; ++m) acc += a.xt[m] * p[m];
    const long long o = gz * nxy + (long long)gy * a.nx + gx;
    dst[o] = acc;
    if (comp == 0 && a.zero[0]) {
      a.zero[0][o] = T(0);
      a.zero[1][o] = T(0);
      a.zero[2][o] = T(0);
    }
  }
}

template <typename T>
cudaError_t launch_sep_generic(const SepArgs<T>& a, cudaStream_t st) {
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

// Fast separable stencil with compile-time tap counts (2*HZ+1 along z, 2*HX+1 along x and y) and
// a fixed 2D thread map: no integer division by runtime sizes, taps in registers. Valid when
// every halo fits in one period of the grid (the dispatcher checks; tiny grids use the generic
// kernel above).
// Staged x range of a tile: from X0 - XA to X0 + CX + XA, XA = HX rounded up to a 16-byte multiple
// of elements, so that the start of every staged row (and a TMA box's x coordinate) is 16-byte
// aligned when X0 is; the stencil reads the columns from XA - HX on.
// An int known at compile time, passed where a runtime extent is otherwise taken.
template <int V>
struct CInt {
  __host__ __device__ constexpr operator int() const { return V; }
};

// Tile extents of a field kernel over a grid n: the kernel's tile c, halved along z, then x, then y
// (each not below lo) while twice the blocks (tiles x mult) still fit in `spread`; a halving that
// adds no tile is skipped. spread = 0 keeps c. e: cells per tile; nt: tiles per direction.
static long long field_tiles(const int n[3], const int c[3], const int lo[3], int mult, int spread, int e[3],
                             int nt[3]) {
  for (int d = 0; d < 3; ++d) e[d] = c[d];
  auto count = [&]() {
    long long t = 1;
    for (int d = 0; d < 3; ++d) {
      nt[d] = (n[d] + e[d] - 1) / e[d];
      t *= nt[d];
    }
    return t;
  };
  long long tiles = count();
  const int order[3] = {2, 0, 1};
  for (int k = 0; k < 3 && spread > 0 && 2 * tiles * mult <= spread;) {
    const int d = order[k];
    if (e[d] / 2 < lo[d]) {
      ++k;
      continue;
    }
    e[d] /= 2;
    const long long t2 = count();
    if (t2 == tiles) {  // no more tiles along d: undo, next direction
      e[d] *= 2;
      count();
      ++k;
      continue;
    }
    tiles = t2;
  }
  return tiles;
}

template <typename T, int HX>
struct SepPitch {
  static constexpr int AL = 16 / (int)sizeof(T);
  static constexpr int XA = (HX + AL - 1) / AL * AL;
};

template <typename T, int NDIM, int HZ, int HX>
struct SepGeom {
  static constexpr int CX = NDIM == 2 ? SEP2_CX : SEP3_CX, CY = NDIM == 2 ? 1 : SEP3_CY;
  static constexpr int CZ = NDIM == 2 ? SEP2_CZ : SEP3_CZ;
  static constexpr int HY = NDIM == 3 ? HX : 0;
  static constexpr int XA = SepPitch<T, HX>::XA;
  static constexpr int PX = CX + 2 * XA, LY = CY + 2 * HY, LZ = CZ + 2 * HZ;
  static constexpr size_t STAGE_BYTES = sizeof(T) * (size_t)LZ * LY * PX;
  // dynamic shared memory: the staged tile (128-byte aligned for TMA), the y-pass output in 3D
  static constexpr size_t SMEM_BYTES = 128 + STAGE_BYTES + (NDIM == 3 ? sizeof(T) * (size_t)CZ * CY * PX : 0);
};

// Overwrite the staged elements that lie outside the grid (a TMA box reads them as zero) with their
// periodic images: columns, rows and (3D) planes past either end. The grid is at least as wide as
// the staged region in every direction, so every index is within one period of the grid. Elements
// on two edges are written twice, with the same value.
template <typename T, int NDIM, int NT>
__device__ __forceinline__ void patch_wrapped(T* s0, const T* __restrict__ src, int xs, int ys, int zs, int PX, int LY,
                                              int LZ, int nx, int ny, int nz) {
  const WrapOnce w;
  const int xlo = max(0, -xs), xhi = max(0, xs + PX - nx);
  const int ylo = NDIM == 3 ? max(0, -ys) : 0, yhi = NDIM == 3 ? max(0, ys + LY - ny) : 0;
  const int zlo = max(0, -zs), zhi = max(0, zs + LZ - nz);
  if (!(xlo | xhi | ylo | yhi | zlo | zhi)) return;
  const long long nxy = (long long)nx * ny;
  auto fix = [&](int lx, int ly, int lz) {
    const int gx = w(xs + lx, nx), gy = NDIM == 3 ? w(ys + ly, ny) : 0, gz = w(zs + lz, nz);
    s0[(lz * LY + ly) * PX + lx] = src[gz * nxy + (long long)gy * nx + gx];
  };
  const int nxe = xlo + xhi;  // outside columns, every row
  for (int i = threadIdx.x; i < nxe * LY * LZ; i += NT) {
    const int c = i % nxe, row = i / nxe;
    fix(c < xlo ? c : PX - xhi + (c - xlo), row % LY, row / LY);
  }
  const int nze = zlo + zhi;  // outside rows, every column
  for (int i = threadIdx.x; i < nze * LY * PX; i += NT) {
    const int lx = i % PX, r = i / PX;
    const int zr = r / LY;
    fix(lx, r % LY, zr < zlo ? zr : LZ - zhi + (zr - zlo));
  }
  if constexpr (NDIM == 3) {
    const int nye = ylo + yhi;  // outside y planes
    for (int i = threadIdx.x; i < nye * LZ * PX; i += NT) {
      const int lx = i % PX, r = i / PX;
      const int yr = r % nye, lz = r / nye;
      fix(lx, yr < ylo ? yr : LY - yhi + (yr - ylo), lz);
    }
  }
}

template <typename T, int NDIM, int HZ, int HX>
__device__ __forceinline__ void sep_tile(const SepArgs<T>& a, const int tile, const int comp, const int ntx,
                                         const int nty, const int ex, const int ey, const int ez) {
  using G = SepGeom<T, NDIM, HZ, HX>;
  constexpr int CX = G::CX, CY = G::CY, CZ = G::CZ, HY = G::HY, XA = G::XA;
  constexpr int PX = G::PX, LY = G::LY, LZ = G::LZ;
  constexpr int TXN = CX < 32 ? 32 : CX, TYN = SEP_THREADS / TXN;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long mbar;
  // [LZ][LY][PX]; the z pass leaves its output in rows [0, CZ)
  T* s0 = reinterpret_cast<T*>(smraw + ((128 - (smem_u32(smraw) & 127)) & 127));
  T* s1 = s0;                   // [CZ][LY][PX] (z pass output, in place)
  T* s2 = s0 + LZ * LY * PX;    // [CZ][CY][PX] (3D)
  const T* __restrict__ src = a.src[comp];
  T* __restrict__ dst = a.dst[comp];
  const int zs = a.zset[comp];
  const int tx = threadIdx.x % TXN, ty = threadIdx.x / TXN;
  const int tix = tile % ntx, tiy = (tile / ntx) % nty, tiz = tile / (ntx * nty);
  const bool zero_j = comp == 0 && a.zero[0] != nullptr;
  // tiles of ex * ey * ez cells (at most the compile-time tile); this one writes wx * wy * wz of them
  const int X0 = tix * ex, Y0 = tiy * ey, Z0 = tiz * ez;
  const int wx = min(ex, a.nx - X0), wy = NDIM == 3 ? min(ey, a.ny - Y0) : 1, wz = min(ez, a.nz - Z0);
  const long long nxy = (long long)a.nx * a.ny;
  // z pass tasks: (x, y) columns of the staged tile that the y and x passes read, times segments of
  // ZS output rows covering the wz written ones
  constexpr int C0 = XA - HX, NSEG = NDIM == 2 ? 2 : 1, ZS = CZ / NSEG;
  static_assert(CZ % NSEG == 0, "z segments must tile the output rows");
  const int ncx = wx + 2 * HX, ncy = NDIM == 3 ? wy + 2 * HY : 1;
  const int nseg = (wz + ZS - 1) / ZS, rows_staged = min(LZ, nseg * ZS + 2 * HZ);
  T zt[2 * HZ + 1], xt[2 * HX + 1], yt[2 * HY + 1];
#pragma unroll
  for (int m = 0; m <= 2 * HZ; ++m) zt[m] = a.zt[zs][m];
#pragma unroll
  for (int m = 0; m <= 2 * HX; ++m) xt[m] = a.xt[m];
#pragma unroll
  for (int m = 0; m <= 2 * HY; ++m) yt[m] = a.yt[m];
  // stage the tile and its halos: x from X0 - XA (16-byte aligned), y from Y0 - HY, z from Z0 - HZ
  const int xs = X0 - XA, ys = Y0 - HY, zs0 = Z0 - HZ;
  if (a.use_tma) {
    // one box for the whole region (periodic images patched below); the host enabled TMA only
    // where the grid spans the region in every direction
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      mbar_expect_tx(&mbar, (unsigned)G::STAGE_BYTES);
      if (NDIM == 2) tma_load_2d(s0, &a.tm[comp], xs, zs0, &mbar);
      else tma_load_3d(s0, &a.tm[comp], xs, ys, zs0, &mbar);
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    const bool ok = __syncthreads_and(mbar_wait(&mbar, 0, TMA_WAIT_POLLS));
    if (!ok) {  // give up: record it, let the copy land (bounded), and leave the tile
      if (threadIdx.x == 0) flag_error(a.err, ERR_TIMEOUT);
      mbar_wait(&mbar, 0, TMA_WAIT_POLLS);
      return;
    }
    patch_wrapped<T, NDIM, SEP_THREADS>(s0, src, xs, ys, zs0, PX, LY, LZ, a.nx, a.ny, a.nz);
  } else {
    auto stage = [&](auto wrap) {  // the rows and columns the passes read
      for (int row = ty; row < rows_staged * LY; row += TYN) {
        const int ly = row % LY, lz = row / LY;
        if (ly >= ncy) continue;
        const int gy = NDIM == 3 ? wrap(ys + ly, a.ny) : 0;
        const int gz = wrap(zs0 + lz, a.nz);
        const T* srow = src + gz * nxy + (long long)gy * a.nx;
        for (int lx = C0 + tx; lx < C0 + ncx; lx += TXN)
          cp_async_el(s0 + row * PX + lx, srow + wrap(xs + lx, a.nx));
      }
    };
    if (a.nx >= PX && a.nz >= LZ && (NDIM == 2 || a.ny >= LY)) stage(WrapOnce{});
    else stage(WrapNear{});
    cp_async_wait_all_fields();
  }
  __syncthreads();
  // the passes, on the written extent: compile-time constants for a full tile (constant divisions
  // and loop bounds), the tile's own extents otherwise
  auto passes = [&](auto wx_, auto wy_, auto wz_) {
    // z pass in place. A task is one (x, y) column of the staged tile and a segment of ZS output rows;
    // it reads its ZS + 2 HZ inputs into registers before any task of its round writes, and a column's
    // segment 0 (rows [0, ZS + 2 HZ) read, [0, ZS) written) always runs in a round no later than its
    // segment 1 (rows [ZS, 2 ZS + 2 HZ) read), so no task reads a row that another has overwritten.
    // The columns before XA - HX and past wx + XA + HX are staged for alignment only (or not at all)
    // and skipped; rows past wz are not computed.
    {
      const int ncx = wx_ + 2 * HX, ncy = NDIM == 3 ? wy_ + 2 * HY : 1, nseg = (wz_ + ZS - 1) / ZS;
      const int ncol = ncx * ncy, ntask = ncol * nseg;
      for (int t0 = 0; t0 < ntask; t0 += SEP_THREADS) {
        const int t = t0 + threadIdx.x;
        const bool act = t < ntask;
        const int col = t % ncol, seg = t / ncol;
        T* base = s0 + seg * ZS * LY * PX + (col / ncx) * PX + C0 + col % ncx;
        T w[ZS + 2 * HZ];
        if (act) {
#pragma unroll
          for (int m = 0; m < ZS + 2 * HZ; ++m) w[m] = base[m * LY * PX];
        }
        __syncthreads();
        if (act) {
#pragma unroll
          for (int r = 0; r < ZS; ++r) {
            if (seg * ZS + r >= wz_) break;
            T acc = T(0);
#pragma unroll
            for (int m = 0; m <= 2 * HZ; ++m) acc += zt[m] * w[r + m];
            base[r * LY * PX] = acc;
          }
        }
        __syncthreads();
      }
    }
    const T* sx = s1;
    if (NDIM == 3) {  // y pass
      for (int row = ty; row < CZ * CY; row += TYN) {
        const int ly = row % CY, lz = row / CY;
        if (ly >= wy_ || lz >= wz_) continue;
        for (int lx = XA - HX + tx; lx < XA + HX + wx_; lx += TXN) {
          const T* p = s1 + (lz * LY + ly) * PX + lx;
          T acc = T(0);
#pragma unroll
          for (int m = 0; m <= 2 * HY; ++m) acc += yt[m] * p[m * PX];
          s2[row * PX + lx] = acc;
        }
      }
      __syncthreads();
      sx = s2;
    }
    for (int row = ty; row < CZ * CY; row += TYN) {  // x pass -> global
      const int ly = row % CY, lz = row / CY;
      if (ly >= wy_ || lz >= wz_) continue;
      const int gy = Y0 + ly, gz = Z0 + lz;
      for (int lx = tx; lx < wx_; lx += TXN) {
        const int gx = X0 + lx;
        const T* p = sx + row * PX + XA - HX + lx;
        T acc = T(0);
#pragma unroll
        for (int m = 0; m <= 2 * HX; ++m) acc += xt[m] * p[m];
        const long long o = gz * nxy + (long long)gy * a.nx + gx;
        dst[o] = acc;
        if (zero_j) {
          a.zero[0][o] = T(0);
          a.zero[1][o] = T(0);
          a.zero[2][o] = T(0);
        }
      }
    }
  };
  if (wx == CX && wy == CY && wz == CZ) passes(CInt<CX>{}, CInt<CY>{}, CInt<CZ>{});
  else passes(wx, wy, wz);
}

template <typename T, int NDIM, int HZ, int HX>
__global__ void __launch_bounds__(SEP_THREADS) k_sep_t(const __grid_constant__ SepArgs<T> a, int ntx, int nty,
                                                       int ex, int ey, int ez) {
  pdl_wait();
  sep_tile<T, NDIM, HZ, HX>(a, blockIdx.x, blockIdx.y, ntx, nty, ex, ey, ez);
}

// Run of a flat tile index: largest r with tile_base[r] <= t.
__device__ __forceinline__ int run_of_tile(const int* tile_base, int nruns, int t) {
  int lo = 0, hi = nruns;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_base[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename T, int NDIM, int HZ, int HX>
__global__ void __launch_bounds__(SEP_THREADS) k_sep_batch(const SepArgs<T>* __restrict__ args,
                                                           const int* __restrict__ tile_base, int nruns) {
  constexpr int CX = NDIM == 2 ? SEP2_CX : SEP3_CX, CY = NDIM == 2 ? 1 : SEP3_CY;
  constexpr int CZ = NDIM == 2 ? SEP2_CZ : SEP3_CZ;
  pdl_wait();
  const int run = run_of_tile(tile_base, nruns, blockIdx.x);
  const SepArgs<T>& a = args[run];
  const int ntx = (a.nx + CX - 1) / CX, nty = NDIM == 3 ? (a.ny + CY - 1) / CY : 1;
  sep_tile<T, NDIM, HZ, HX>(a, blockIdx.x - tile_base[run], blockIdx.y, ntx, nty, CX, CY, CZ);
}

template <typename T, int NDIM, int HZ, int HX>
static cudaError_t launch_sep_t(const SepArgs<T>& a_in, cudaStream_t st) {
  using G = SepGeom<T, NDIM, HZ, HX>;
  constexpr int CX = G::CX, CY = G::CY, CZ = G::CZ;
  const size_t sm = G::SMEM_BYTES;
  // a small grid's tiles shrink (z first, down to 8 rows in 2D; x not below a warp's 32 columns)
  const int n[3] = {a_in.nx, a_in.ny, a_in.nz}, c[3] = {CX, CY, CZ};
  const int lo[3] = {32, NDIM == 3 ? 2 : 1, NDIM == 3 ? 2 : 8};
  int te[3], nt[3];
  field_tiles(n, c, lo, a_in.ncomp, a_in.spread, te, nt);
  const int ntx = nt[0], nty = nt[1], ntz = nt[2];
  // TMA staging where the grid spans a staged region in every direction (its periodic images are
  // then one period away) and the rows are 16-byte multiples; element copies otherwise
  SepArgs<T> a = a_in;
  a.use_tma = 0;
  if (a.nx >= G::PX && a.nz >= G::LZ && (NDIM == 2 || a.ny >= G::LY)) {
    bool ok = true;
    for (int c = 0; c < a.ncomp && ok; ++c)
      ok = tma_encode(&a.tm[c], a.src[c], (int)sizeof(T), NDIM, a.nx, a.ny, a.nz, G::PX, G::LY, G::LZ);
    a.use_tma = ok ? 1 : 0;
  }
  cudaError_t e = ensure_dynamic_smem((const void*)k_sep_t<T, NDIM, HZ, HX>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(ntx * nty * ntz), (unsigned)a.ncomp);
  return launch_pdl(k_sep_t<T, NDIM, HZ, HX>, grid, dim3(SEP_THREADS), sm, st, a, ntx, nty, te[0], te[1], te[2]);
}

template <typename T, int NDIM, int HX>
static cudaError_t sep_pick_hz(const SepArgs<T>& a, cudaStream_t st) {
  if (a.hz[0] == HX) return launch_sep_t<T, NDIM, HX, HX>(a, st);          // current filter
  if (a.hz[0] == HX + 4) return launch_sep_t<T, NDIM, HX + 4, HX>(a, st);  // Psi (9 taps) * filter
  return launch_sep_generic<T>(a, st);
}

bool sep_fast_ok(int ndim, int nx, int ny, int nz, int hz, int hx) {
  return hx <= 4 && (hz == hx || hz == hx + 4) && nx >= hx && nz >= hz && (ndim == 2 || ny >= hx);
}
int sep_tiles(int ndim, int nx, int ny, int nz) {
  if (ndim == 2) return ((nx + SEP2_CX - 1) / SEP2_CX) * ((nz + SEP2_CZ - 1) / SEP2_CZ);
  return ((nx + SEP3_CX - 1) / SEP3_CX) * ((ny + SEP3_CY - 1) / SEP3_CY) * ((nz + SEP3_CZ - 1) / SEP3_CZ);
}

template <typename T, int NDIM, int HZ, int HX>
static cudaError_t launch_sep_batch_t(const SepArgs<T>* args, const int* tile_base, int nruns, int total_tiles,
                                      int ncomp, cudaStream_t st) {
  const size_t sm = SepGeom<T, NDIM, HZ, HX>::SMEM_BYTES;  // the tables carry use_tma = 0
  cudaError_t e = ensure_dynamic_smem((const void*)k_sep_batch<T, NDIM, HZ, HX>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)total_tiles, (unsigned)ncomp);
  return launch_pdl(k_sep_batch<T, NDIM, HZ, HX>, grid, dim3(SEP_THREADS), sm, st, args, tile_base, nruns);
}

template <typename T, int NDIM, int HX>
static cudaError_t sep_batch_pick_hz(const SepArgs<T>* args, const int* tb, int nruns, int tot, int ncomp, int hz,
                                     cudaStream_t st) {
  if (hz == HX) return launch_sep_batch_t<T, NDIM, HX, HX>(args, tb, nruns, tot, ncomp, st);
  return launch_sep_batch_t<T, NDIM, HX + 4, HX>(args, tb, nruns, tot, ncomp, st);
}

template <typename T>
cudaError_t launch_sep_batch(const SepArgs<T>* args, const int* tile_base, int nruns, int total_tiles, int ncomp,
                             int ndim, int hz, int hx, cudaStream_t st) {
  if (hx < 0 || hx > 4 || (hz != hx && hz != hx + 4)) return cudaErrorInvalidValue;
#define PIC_SEP_CASE(D, X) \
  if (ndim == D && hx == X) return sep_batch_pick_hz<T, D, X>(args, tile_base, nruns, total_tiles, ncomp, hz, st);
  PIC_SEP_CASE(2, 0) PIC_SEP_CASE(2, 1) PIC_SEP_CASE(2, 2) PIC_SEP_CASE(2, 3) PIC_SEP_CASE(2, 4)
  PIC_SEP_CASE(3, 0) PIC_SEP_CASE(3, 1) PIC_SEP_CASE(3, 2) PIC_SEP_CASE(3, 3) PIC_SEP_CASE(3, 4)
#undef PIC_SEP_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_sep_batch<float>(const SepArgs<float>*, const int*, int, int, int, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_sep_batch<double>(const SepArgs<double>*, const int*, int, int, int, int, int, int,
                                              cudaStream_t);

template <typename T>
cudaError_t launch_sep(const SepArgs<T>& a, cudaStream_t st) {
  const int hz = a.hz[0];
  const bool fits = a.hz[0] == a.hz[1] && sep_fast_ok(a.ndim, a.nx, a.ny, a.nz, hz, a.hx);
  if (!fits) return launch_sep_generic<T>(a, st);
  if (a.ndim == 2) {
    switch (a.hx) {
      case 0: return sep_pick_hz<T, 2, 0>(a, st);
      case 1: return sep_pick_hz<T, 2, 1>(a, st);
      case 2: return sep_pick_hz<T, 2, 2>(a, st);
      case 3: return sep_pick_hz<T, 2, 3>(a, st);
      default: return sep_pick_hz<T, 2, 4>(a, st);
    }
  }
  switch (a.hx) {
    case 0: return sep_pick_hz<T, 3, 0>(a, st);
    case 1: return sep_pick_hz<T, 3, 1>(a, st);
    case 2: return sep_pick_hz<T, 3, 2>(a, st);
    case 3: return sep_pick_hz<T, 3, 3>(a, st);
    default: return sep_pick_hz<T, 3, 4>(a, st);
  }
}
template cudaError_t launch_sep<float>(const SepArgs<float>&, cudaStream_t);
template cudaError_t launch_sep<double>(const SepArgs<double>&, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Field energies: per-thread sums of exact squares and the deterministic block / grid reduction.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int FE_THREADS = 256;
constexpr int FE_BLOCKS = 8 * 152;  // partial sums per launch; scratch holds 3 * FE_BLOCKS + 1

// FP32 sum of exact squares with an error-free running sum: x^2 = hi + lo exactly (lo from an FMA);
// hi is added by TwoSum (s + hi = t + err exactly) and the small terms err and lo accumulate in c,
// whose own rounding is O(eps^2) of the sum.
struct FSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_sq(float x) {
    const float hi = x * x;
    const float lo = fmaf(x, x, -hi);
    const float t = s + hi;
    const float bb = t - s;
    const float err = (s - (t - bb)) + (hi - bb);
    s = t;
    c += err + lo;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};


// Per-thread sums of squares of the six field components: FP32 fields through FSum (exact squares,
// error-free running sums), FP64 fields with FMAs.
template <typename T>
struct EnergyAcc {
  FSum e2, b2, e2x, e2y, b2x, b2y;  // FP32 fields
  double se = 0, sb = 0, sp = 0;    // FP64 fields
  __device__ __forceinline__ void add(T x, T y, T z, T u, T v, T w) {
    if (sizeof(T) == 4) {
      e2x.add_sq((float)x);
      e2y.add_sq((float)y);
      e2.add_sq((float)z);
      b2x.add_sq((float)u);
      b2y.add_sq((float)v);
      b2.add_sq((float)w);
    } else {
      const double dx = x, dy = y, dz = z, du = u, dv = v, dw = w;
      const double t = fma(dx, dx, dy * dy), tb = fma(du, du, dv * dv);
      se += fma(dz, dz, t);
      sb += fma(dw, dw, tb);
      sp += t + tb;
    }
  }
  // FP32 fields: the same three sums as FP32 pairs (FP64 fields: unused)
  __device__ __forceinline__ void pairs(FPair& oe, FPair& ob, FPair& op) const {
    const FPair ax{e2x.s, e2x.c}, ay{e2y.s, e2y.c}, bxs{b2x.s, b2x.c}, bys{b2y.s, b2y.c};
    const FPair exy = pair_add(ax, ay), bxy = pair_add(bxs, bys);
    oe = pair_add(exy, FPair{e2.s, e2.c});
    ob = pair_add(bxy, FPair{b2.s, b2.c});
    op = pair_add(exy, bxy);
  }
  // (sum E^2, sum B^2, sum Ex^2 + Ey^2 + Bx^2 + By^2) of this thread
  __device__ __forceinline__ void get(double& oe, double& ob, double& op) const {
    if (sizeof(T) == 4) {
      const double ax = e2x.get(), ay = e2y.get(), bxs = b2x.get(), bys = b2y.get();
      oe = ax + ay + e2.get();
      ob = bxs + bys + b2.get();
      op = ax + ay + bxs + bys;
    } else {
      oe = se;
      ob = sb;
      op = sp;
    }
  }
};

// Block and grid stage of the energy sums (FE_THREADS threads per block): FP64 tree per block into
// scratch[3 * block + r]; the last block to finish (counter at scratch + 3 * slots, slots >= the
// grid size) adds the block partials in a fixed order and writes (sum E^2, sum B^2, sum Ex^2 + Ey^2
// + Bx^2 + By^2) to out[0..2], or, with a history ring, into its next slot with the kinetic sums.
// The grid stage: thread r < 3 holds the block's partial r in `part`; it stores it and fences, the
// block counts itself done, and the last block adds every block's partials in FP64.
__device__ __forceinline__ void energy_grid_finish(double part, double* scratch, unsigned slots, double* out,
                                                   const HistCtl& hc) {
  __shared__ double red[3][FE_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned* done = reinterpret_cast<unsigned*>(scratch + 3 * (size_t)slots);
  if (threadIdx.x < 3) {
    scratch[3 * blockIdx.x + threadIdx.x] = part;
    __threadfence();  // the partial is visible before the block counts itself done
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) {  // the whole last block adds the partials: strided per thread, then a fixed tree
    __threadfence();
    double t[3] = {0, 0, 0};
    for (unsigned q = threadIdx.x; q < gridDim.x; q += FE_THREADS)
      for (int r = 0; r < 3; ++r) t[r] += ((volatile double*)scratch)[3 * q + r];
    for (int r = 0; r < 3; ++r) t[r] = warp_sum(t[r]);
    __syncthreads();
    if (lane == 0)
      for (int r = 0; r < 3; ++r) red[r][w] = t[r];
    __syncthreads();
    if (hc.hist) {
      double* slot = hc.hist + 8 * (*hc.count % hc.cap);
      if (threadIdx.x < 3) {
        double acc = 0;
        for (int q = 0; q < FE_THREADS / 32; ++q) acc += red[threadIdx.x][q];
        slot[threadIdx.x] = acc;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        slot[3] = hc.kin[0];
        slot[4] = hc.kin[1];
        hc.kin[0] = 0.0;
        hc.kin[1] = 0.0;
        *hc.count += 1;
      }
    } else if (threadIdx.x < 3) {
      double acc = 0;
      for (int q = 0; q < FE_THREADS / 32; ++q) acc += red[threadIdx.x][q];
      out[threadIdx.x] = acc;
    }
    if (threadIdx.x == 0) *done = 0u;  // ready for the next launch
  }
}

// Block stage, FP64 per-thread sums: FP64 tree per block, then the grid stage.
__device__ __forceinline__ void energy_finish(double se, double sb, double sp, double* scratch, unsigned slots,
                                              double* out, const HistCtl& hc) {
  __shared__ double redb[3][FE_THREADS / 32];
  const double dse = warp_sum(se), dsb = warp_sum(sb), dsp = warp_sum(sp);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    redb[0][w] = dse;
    redb[1][w] = dsb;
    redb[2][w] = dsp;
  }
  __syncthreads();
  double part = 0;
  if (threadIdx.x < 3)
    for (int q = 0; q < FE_THREADS / 32; ++q) part += redb[threadIdx.x][q];
  energy_grid_finish(part, scratch, slots, out, hc);
}

// Block stage, FP32 pair sums: pair trees per warp and block, FP64 only for the block's partials.
__device__ __forceinline__ void energy_finish(FPair e, FPair b, FPair p, double* scratch, unsigned slots,
                                              double* out, const HistCtl& hc) {
  __shared__ FPair redp[3][FE_THREADS / 32];
  e = warp_sum_pair(e);
  b = warp_sum_pair(b);
  p = warp_sum_pair(p);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    redp[0][w] = e;
    redp[1][w] = b;
    redp[2][w] = p;
  }
  __syncthreads();
  double part = 0;
  if (threadIdx.x < 3) {
    FPair t = redp[threadIdx.x][0];
    for (int q = 1; q < FE_THREADS / 32; ++q) t = pair_add(t, redp[threadIdx.x][q]);
    part = (double)t.s + (double)t.c;
  }
  energy_grid_finish(part, scratch, slots, out, hc);
}

// The block's energy sums from each thread's accumulator, then the grid stage.
template <typename T>
__device__ __forceinline__ void energy_finish(const EnergyAcc<T>& acc, double* scratch, unsigned slots, double* out,
                                              const HistCtl& hc) {
  if constexpr (sizeof(T) == 4) {
    FPair e, b, p;
    acc.pairs(e, b, p);
    energy_finish(e, b, p, scratch, slots, out, hc);
  } else {
    double se, sb, sp;
    acc.get(se, sb, sp);
    energy_finish(se, sb, sp, scratch, slots, out, hc);
  }
}

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
// Fused Yee step: B -= dt/2 curl E, E += dt (curl B - J), B -= dt/2 curl E on one tile, with the
// fields staged in shared memory over [-HL, C+2) per direction: B^{n+1/2} is formed on [-HB, C+1),
// E^{n+1} on [-HE, C+1), B^{n+1} on [0, C), and E, B are written back on [0, C). Same arithmetic and
// order as the three separate updates; one read and one write of E and B per step.
// Yee: HL = 1, HB = 1, HE = 0. Cole-Karkkainen (2D): the B updates average each forward difference
// over the two transverse neighbours, which widens every stage by one cell: HL = 3, HB = 2, HE = 1.
// ---------------------------------------------------------------------------------------------
constexpr int YEE_THREADS = 256;
constexpr int YEE2_CX = 32, YEE2_CZ = 32;
constexpr int YEE3_CX = 16, YEE3_CY = 8, YEE3_CZ = 8;

template <bool CK>
struct YeeHalo {
  static constexpr int HL = CK ? 3 : 1, HB = CK ? 2 : 1, HE = CK ? 1 : 0;
};

// Staged region of a Yee tile: x from X0 - XAL (HL rounded up to a 16-byte multiple of elements, so
// that a TMA box starts on a 16-byte boundary) over PX columns, local column OX = XAL - HL holding
// x = X0 - HL; y from Y0 - 1 over LY, z from Z0 - HL over LZ.
template <typename T, int NDIM, bool CK>
struct YeeGeom {
  static constexpr int HL = YeeHalo<CK>::HL;
  static constexpr int CX = NDIM == 2 ? YEE2_CX : YEE3_CX, CY = NDIM == 2 ? 1 : YEE3_CY;
  static constexpr int CZ = NDIM == 2 ? YEE2_CZ : YEE3_CZ;
  static constexpr int AL = 16 / (int)sizeof(T);
  static constexpr int XAL = (HL + AL - 1) / AL * AL, OX = XAL - HL;
  static constexpr int PX = (XAL + CX + 2 + AL - 1) / AL * AL;
  static constexpr int LY = NDIM == 2 ? 1 : CY + 3, LZ = CZ + HL + 2;
  static constexpr size_t BOX_BYTES = sizeof(T) * (size_t)PX * LY * LZ;
  // arrays spaced by whole 128-byte units: a bulk tensor copy's shared-memory destination must start
  // on a 128-byte boundary
  static constexpr int LN = (int)((BOX_BYTES + 127) / 128 * 128 / sizeof(T));
  static constexpr size_t SMEM_BYTES = 128 + 9 * sizeof(T) * (size_t)LN;
};

template <typename T, int NDIM, bool CK, bool DIAG>
__device__ __forceinline__ void yee_tile(const YeeArgs<T>& a, const int tile, const int ntx, const int nty,
                                         const int ex, const int ey, const int ez, double* escratch = nullptr,
                                         const HistCtl* hc = nullptr) {
  static_assert(!CK || NDIM == 2, "the Cole-Karkkainen curl is built for 2D x-z runs");
  using G = YeeGeom<T, NDIM, CK>;
  constexpr int HL = YeeHalo<CK>::HL, HB = YeeHalo<CK>::HB, HE = YeeHalo<CK>::HE;
  constexpr int LX = G::PX, LY = G::LY, LZ = G::LZ, LN = G::LN, OX = G::OX;
  constexpr int OY = NDIM == 2 ? 0 : 1;  // local offset of the -1 halo along y
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long mbar;
  T* sm = reinterpret_cast<T*>(smraw + ((128 - (smem_u32(smraw) & 127)) & 127));
  T* e[3] = {sm, sm + LN, sm + 2 * LN};
  T* b[3] = {sm + 3 * LN, sm + 4 * LN, sm + 5 * LN};
  T* j[3] = {sm + 6 * LN, sm + 7 * LN, sm + 8 * LN};
  const int tix = tile % ntx, tiy = (tile / ntx) % nty, tiz = tile / (ntx * nty);
  // tiles of ex * ey * ez cells (at most the compile-time tile); this one updates wx * wy * wz of them
  const int X0 = tix * ex, Y0 = tiy * ey, Z0 = tiz * ez;
  const int wx = min(ex, a.nx - X0), wy = NDIM == 3 ? min(ey, a.ny - Y0) : 1, wz = min(ez, a.nz - Z0);
  const long long nxy = (long long)a.nx * a.ny;
  const int xs = X0 - G::XAL, ys = NDIM == 3 ? Y0 - 1 : 0, zs = Z0 - HL;
  // wrap_near takes any index, so the halos may wrap around grids smaller than the tile
  auto gsrc = [&](int c) -> const T* {
    switch (c) {
      case 0: return a.ex;
      case 1: return a.ey;
      case 2: return a.ez;
      case 3: return a.bx;
      case 4: return a.by;
      case 5: return a.bz;
      case 6: return a.jx;
      case 7: return a.jy;
      default: return a.jz;
    }
  };
  if (a.use_tma) {
    // one box per array (periodic images patched below); the host enabled TMA only where the grid
    // spans the staged region in every direction
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      mbar_expect_tx(&mbar, (unsigned)(9 * G::BOX_BYTES));
      for (int c = 0; c < 9; ++c) {
        if (NDIM == 2) tma_load_2d(sm + c * LN, &a.tm[c], xs, zs, &mbar);
        else tma_load_3d(sm + c * LN, &a.tm[c], xs, ys, zs, &mbar);
      }
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    const bool ok = __syncthreads_and(mbar_wait(&mbar, 0, TMA_WAIT_POLLS));
    if (!ok) {  // give up: record it, let the copies land (bounded), and leave the tile unchanged
      if (threadIdx.x == 0) flag_error(a.err, ERR_TIMEOUT);
      mbar_wait(&mbar, 0, TMA_WAIT_POLLS);
      if (DIAG) energy_finish(0.0, 0.0, 0.0, escratch, gridDim.x, nullptr, *hc);
      return;
    }
    for (int c = 0; c < 9; ++c)
      patch_wrapped<T, NDIM, YEE_THREADS>(sm + c * LN, gsrc(c), xs, ys, zs, LX, LY, LZ, a.nx, a.ny, a.nz);
  } else {
    auto stage = [&](auto wrap) {
      // the region the phases read: columns [0, XAL + wx + 2), y rows [0, wy + 3), z rows [0, wz + HL + 2)
      const int nbx = G::XAL + wx + 2, nby = NDIM == 3 ? wy + 3 : 1, nbz = wz + HL + 2;
      const int nb = nbx * nby * nbz;
      for (int idx = threadIdx.x; idx < 9 * nb; idx += YEE_THREADS) {  // flat: rows are wider than a warp
        const int c = idx / nb, r3 = idx - c * nb;
        const int lx = r3 % nbx, r2 = r3 / nbx;
        const int ly = r2 % nby, lz = r2 / nby;
        const int gy = NDIM == 3 ? wrap(ys + ly, a.ny) : 0;
        const int gz = wrap(zs + lz, a.nz);
        cp_async_el(sm + c * LN + (lz * LY + ly) * LX + lx,
                    gsrc(c) + gz * nxy + (long long)gy * a.nx + wrap(xs + lx, a.nx));
      }
    };
    if (a.nx >= LX && a.nz >= LZ && (NDIM == 2 || a.ny >= LY)) stage(WrapOnce{});
    else stage(WrapNear{});
    cp_async_wait_all_fields();
  }
  __syncthreads();
  const int sx = 1, sy = NDIM == 3 ? LX : 0, sz = LX * LY;  // sy = 0 in 2D: y differences vanish
  const T hcx = a.cx * T(0.5), hcy = a.cy * T(0.5), hcz = a.cz * T(0.5);
  // CK averaged forward differences at local node l (2D): along z averaged over x, along x over z
  auto ck_dz = [&](const T* f, int l) -> T {
    return a.wz0 * (f[l + sz] - f[l]) + a.wz1 * ((f[l + sz - 1] - f[l - 1]) + (f[l + sz + 1] - f[l + 1]));
  };
  auto ck_dx = [&](const T* f, int l) -> T {
    return a.wx0 * (f[l + 1] - f[l]) + a.wx1 * ((f[l + 1 - sz] - f[l - sz]) + (f[l + 1 + sz] - f[l + sz]));
  };
  // B^{n+1/2} on cells [-HB, w+1) in x and z ([-1, w+1) in y)
  const int ny2 = NDIM == 3 ? wy + 2 : 1, ny1 = NDIM == 3 ? wy + 1 : 1;
  const int nbx = wx + 1 + HB, nbz = wz + 1 + HB;
  // each phase walks its cells with one flat index over all threads (rows are wider than a warp)
  for (int idx = threadIdx.x; idx < ny2 * nbz * nbx; idx += YEE_THREADS) {
    const int q = idx % nbx, row = idx / nbx;
    const int lx = OX + HL - HB + q, ly = row % ny2, lz = HL - HB + row / ny2;
    const int l = (lz * LY + ly) * LX + lx;
    if (CK) {
      b[0][l] += hcz * ck_dz(e[1], l);
      b[1][l] -= hcz * ck_dz(e[0], l) - hcx * ck_dx(e[2], l);
      b[2][l] -= hcx * ck_dx(e[1], l);
    } else {
      const T ex = e[0][l], ey = e[1][l], ez = e[2][l];
      b[0][l] -= hcy * (e[2][l + sy] - ez) - hcz * (e[1][l + sz] - ey);
      b[1][l] -= hcz * (e[0][l + sz] - ex) - hcx * (e[2][l + sx] - ez);
      b[2][l] -= hcx * (e[1][l + sx] - ey) - hcy * (e[0][l + sy] - ex);
    }
  }
  __syncthreads();
  // E^{n+1} on cells [-HE, w+1) in x and z ([0, w+1) in y)
  const int nex = wx + 1 + HE, nez = wz + 1 + HE;
  for (int idx = threadIdx.x; idx < ny1 * nez * nex; idx += YEE_THREADS) {
    const int q = idx % nex, row = idx / nex;
    const int lx = OX + HL - HE + q, ly = NDIM == 3 ? 1 + row % ny1 : 0, lz = HL - HE + row / ny1;
    const int l = (lz * LY + ly) * LX + lx;
    const T bx = b[0][l], by = b[1][l], bz = b[2][l];
    e[0][l] += a.cy * (bz - b[2][l - sy]) - a.cz * (by - b[1][l - sz]) - a.h * j[0][l];
    e[1][l] += a.cz * (bx - b[0][l - sz]) - a.cx * (bz - b[2][l - sx]) - a.h * j[1][l];
    e[2][l] += a.cx * (by - b[1][l - sx]) - a.cy * (bx - b[0][l - sy]) - a.h * j[2][l];
  }
  __syncthreads();
  // B^{n+1} on cells [0, w), then write E and B of the tile (and, with DIAG, sum their energies)
  EnergyAcc<T> en;
  for (int idx = threadIdx.x; idx < wy * wz * wx; idx += YEE_THREADS) {
    const int cx = idx % wx, row = idx / wx;
    const int cy = row % wy, cz = row / wy;
    const int gx = X0 + cx, gy = Y0 + cy, gz = Z0 + cz;
    const int l = ((cz + HL) * LY + cy + OY) * LX + cx + HL + OX;
    const T ex = e[0][l], ey = e[1][l], ez = e[2][l];
    T nbx, nby, nbz;
    if (CK) {
      nbx = b[0][l] + hcz * ck_dz(e[1], l);
      nby = b[1][l] - (hcz * ck_dz(e[0], l) - hcx * ck_dx(e[2], l));
      nbz = b[2][l] - hcx * ck_dx(e[1], l);
    } else {
      nbx = b[0][l] - (hcy * (e[2][l + sy] - ez) - hcz * (e[1][l + sz] - ey));
      nby = b[1][l] - (hcz * (e[0][l + sz] - ex) - hcx * (e[2][l + sx] - ez));
      nbz = b[2][l] - (hcx * (e[1][l + sx] - ey) - hcy * (e[0][l + sy] - ex));
    }
    const long long o = gz * nxy + (long long)gy * a.nx + gx;
    a.oex[o] = ex;
    a.oey[o] = ey;
    a.oez[o] = ez;
    a.obx[o] = nbx;
    a.oby[o] = nby;
    a.obz[o] = nbz;
    if (DIAG) en.add(ex, ey, ez, nbx, nby, nbz);
  }
  if (DIAG) energy_finish(en, escratch, gridDim.x, nullptr, *hc);  // every thread reaches this
}

template <typename T, int NDIM, bool CK, bool DIAG>
__global__ void __launch_bounds__(YEE_THREADS) k_yee_fused(const __grid_constant__ YeeArgs<T> a, int ntx, int nty,
                                                           int ex, int ey, int ez, double* escratch,
                                                           const __grid_constant__ HistCtl hc) {
  pdl_wait();
  yee_tile<T, NDIM, CK, DIAG>(a, blockIdx.x, ntx, nty, ex, ey, ez, escratch, &hc);
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(YEE_THREADS) k_yee_batch(const YeeArgs<T>* __restrict__ args,
                                                           const int* __restrict__ tile_base, int nruns) {
  constexpr int CX = NDIM == 2 ? YEE2_CX : YEE3_CX, CY = NDIM == 2 ? 1 : YEE3_CY;
  constexpr int CZ = NDIM == 2 ? YEE2_CZ : YEE3_CZ;
  pdl_wait();
  const int run = run_of_tile(tile_base, nruns, blockIdx.x);
  const YeeArgs<T>& a = args[run];
  const int ntx = (a.nx + CX - 1) / CX, nty = NDIM == 3 ? (a.ny + CY - 1) / CY : 1;
  yee_tile<T, NDIM, false, false>(a, blockIdx.x - tile_base[run], ntx, nty, CX, CY, CZ);
}

int yee_tiles(int ndim, int nx, int ny, int nz) {
  if (ndim == 2) return ((nx + YEE2_CX - 1) / YEE2_CX) * ((nz + YEE2_CZ - 1) / YEE2_CZ);
  return ((nx + YEE3_CX - 1) / YEE3_CX) * ((ny + YEE3_CY - 1) / YEE3_CY) * ((nz + YEE3_CZ - 1) / YEE3_CZ);
}

template <typename T>
cudaError_t launch_yee_batch(const YeeArgs<T>* args, const int* tile_base, int nruns, int total_tiles, int ndim,
                             cudaStream_t st) {
  if (ndim == 2) {  // the tables carry use_tma = 0: element-copy staging
    const size_t sm = YeeGeom<T, 2, false>::SMEM_BYTES;
    cudaError_t e = ensure_dynamic_smem((const void*)k_yee_batch<T, 2>, sm);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_yee_batch<T, 2>, dim3(total_tiles), dim3(YEE_THREADS), sm, st, args, tile_base, nruns);
    if (e != cudaSuccess) return e;
  } else {
    const size_t sm = YeeGeom<T, 3, false>::SMEM_BYTES;
    cudaError_t e = ensure_dynamic_smem((const void*)k_yee_batch<T, 3>, sm);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_yee_batch<T, 3>, dim3(total_tiles), dim3(YEE_THREADS), sm, st, args, tile_base, nruns);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}
template cudaError_t launch_yee_batch<float>(const YeeArgs<float>*, const int*, int, int, int, cudaStream_t);
template cudaError_t launch_yee_batch<double>(const YeeArgs<double>*, const int*, int, int, int, cudaStream_t);

bool yee_records_energy(int ndim, int nx, int ny, int nz, int ck) {
  return ck || !(nx < 3 || nz < 3 || (ndim == 3 && ny < 3));
}
// Tiles of the fused Yee launch: a small grid's tiles shrink (not below 8 cells in x and z, 2 in y).
static long long yee_launch_tiles(int ndim, int nx, int ny, int nz, int spread, int te[3], int nt[3]) {
  const int n[3] = {nx, ny, nz};
  const int c[3] = {ndim == 2 ? YEE2_CX : YEE3_CX, ndim == 2 ? 1 : YEE3_CY, ndim == 2 ? YEE2_CZ : YEE3_CZ};
  const int lo[3] = {8, ndim == 2 ? 1 : 2, ndim == 2 ? 8 : 2};
  return field_tiles(n, c, lo, 1, spread, te, nt);
}

size_t yee_energy_scratch_bytes(int ndim, int nx, int ny, int nz, int spread) {
  int te[3], nt[3];
  return sizeof(double) * (3 * (size_t)yee_launch_tiles(ndim, nx, ny, nz, spread, te, nt) + 2);
}

template <typename T, int NDIM, bool CK>
static cudaError_t launch_yee_tiles(const YeeArgs<T>& a_in, double* escratch, const HistCtl* hc, cudaStream_t st) {
  using G = YeeGeom<T, NDIM, CK>;
  const size_t sm = G::SMEM_BYTES;
  int te[3], nt[3];
  const int ntiles = (int)yee_launch_tiles(NDIM, a_in.nx, a_in.ny, a_in.nz, a_in.spread, te, nt);
  const int ntx = nt[0], nty = nt[1];
  const HistCtl none{nullptr, 0, nullptr, nullptr};
  // TMA staging where the grid spans the staged region in every direction and the rows are 16-byte
  // multiples; element copies otherwise
  YeeArgs<T> a = a_in;
  a.use_tma = 0;
  if (a.nx >= G::PX && a.nz >= G::LZ && (NDIM == 2 || a.ny >= G::LY)) {
    const T* src[9] = {a.ex, a.ey, a.ez, a.bx, a.by, a.bz, a.jx, a.jy, a.jz};
    bool ok = true;
    for (int c = 0; c < 9 && ok; ++c)
      ok = tma_encode(&a.tm[c], src[c], (int)sizeof(T), NDIM, a.nx, a.ny, a.nz, G::PX, G::LY, G::LZ);
    a.use_tma = ok ? 1 : 0;
  }
  if (hc) {
    cudaError_t e = ensure_dynamic_smem((const void*)k_yee_fused<T, NDIM, CK, true>, sm);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_yee_fused<T, NDIM, CK, true>, dim3(ntiles), dim3(YEE_THREADS), sm, st, a, ntx, nty, te[0], te[1],
                   te[2], escratch, *hc);
    if (e != cudaSuccess) return e;
  } else {
    cudaError_t e = ensure_dynamic_smem((const void*)k_yee_fused<T, NDIM, CK, false>, sm);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_yee_fused<T, NDIM, CK, false>, dim3(ntiles), dim3(YEE_THREADS), sm, st, a, ntx, nty, te[0],
                   te[1], te[2], (double*)nullptr, none);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_yee_fused(const YeeArgs<T>& a, int ndim, cudaStream_t st, double* escratch, const HistCtl* hc) {
  if (hc && (!escratch || !yee_records_energy(ndim, a.nx, a.ny, a.nz, a.ck))) return cudaErrorInvalidValue;
  if (ndim == 2 && a.ck) return launch_yee_tiles<T, 2, true>(a, escratch, hc, st);  // any grid: the halos wrap
  if (a.ck) return cudaErrorInvalidValue;  // 3D CK is not built (pic_create rejects it)
  if (a.nx < 3 || a.nz < 3 || (ndim == 3 && a.ny < 3)) {
    // tiny grids: the inputs copied to the outputs, then the three separate updates in place there
    const size_t bytes = sizeof(T) * (size_t)a.nx * a.ny * a.nz;
    const T* in[6] = {a.ex, a.ey, a.ez, a.bx, a.by, a.bz};
    T* out[6] = {a.oex, a.oey, a.oez, a.obx, a.oby, a.obz};
    for (int q = 0; q < 6; ++q) {
      cudaError_t e = cudaMemcpyAsync(out[q], in[q], bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    YeeArgs<T> o = a;
    o.ex = a.oex;
    o.ey = a.oey;
    o.ez = a.oez;
    o.bx = a.obx;
    o.by = a.oby;
    o.bz = a.obz;
    YeeArgs<T> hb = o;
    hb.cx = a.cx * T(0.5);
    hb.cy = a.cy * T(0.5);
    hb.cz = a.cz * T(0.5);
    hb.h = a.h * T(0.5);
    cudaError_t e = launch_yee_b<T>(hb, st);
    if (e == cudaSuccess) e = launch_yee_e<T>(o, st);
    if (e == cudaSuccess) e = launch_yee_b<T>(hb, st);
    return e;
  }
  if (ndim == 2) return launch_yee_tiles<T, 2, false>(a, escratch, hc, st);
  return launch_yee_tiles<T, 3, false>(a, escratch, hc, st);
}
template cudaError_t launch_yee_fused<float>(const YeeArgs<float>&, int, cudaStream_t, double*, const HistCtl*);
template cudaError_t launch_yee_fused<double>(const YeeArgs<double>&, int, cudaStream_t, double*, const HistCtl*);

// ---------------------------------------------------------------------------------------------
// FP64 reductions
// ---------------------------------------------------------------------------------------------
// Field energies of a whole grid: per-thread sums of exact squares over a grid-stride set of cells,
// then energy_finish (deterministic block and grid stages).
template <typename T>
__device__ __forceinline__ void field_energy_body(const T* __restrict__ ex, const T* __restrict__ ey,
                                                  const T* __restrict__ ez, const T* __restrict__ bx,
                                                  const T* __restrict__ by, const T* __restrict__ bz, long long n,
                                                  double* out, double* scratch, const HistCtl& hc) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  EnergyAcc<T> acc;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += stride)
    acc.add(ex[c], ey[c], ez[c], bx[c], by[c], bz[c]);
  energy_finish(acc, scratch, FE_BLOCKS, out, hc);
}

template <typename T>
__global__ void __launch_bounds__(FE_THREADS) k_field_energy(const T* __restrict__ ex, const T* __restrict__ ey,
                                                             const T* __restrict__ ez, const T* __restrict__ bx,
                                                             const T* __restrict__ by, const T* __restrict__ bz,
                                                             long long n, double* out, double* scratch, HistCtl hc) {
  field_energy_body<T>(ex, ey, ez, bx, by, bz, n, out, scratch, hc);
}

template <typename T>
__global__ void __launch_bounds__(FE_THREADS) k_field_energy_batch(const EnergyArgs<T>* __restrict__ args) {
  pdl_wait();
  const EnergyArgs<T>& a = args[blockIdx.y];
  field_energy_body<T>(a.f[0], a.f[1], a.f[2], a.f[3], a.f[4], a.f[5], a.ncell, nullptr, a.scratch, a.hc);
}

template <typename T>
cudaError_t launch_field_energy_batch(const EnergyArgs<T>* args, int nruns, cudaStream_t st) {
  dim3 grid(2 * 152 / (nruns < 8 ? 1 : nruns / 8) + 1, (unsigned)nruns);  // about 2 waves in all
  return launch_pdl(k_field_energy_batch<T>, grid, dim3(FE_THREADS), 0, st, args);
}
template cudaError_t launch_field_energy_batch<float>(const EnergyArgs<float>*, int, cudaStream_t);
template cudaError_t launch_field_energy_batch<double>(const EnergyArgs<double>*, int, cudaStream_t);

template <typename T>
cudaError_t launch_field_energy(const T* const f6[6], long long ncell, double* out, double* scratch, HistCtl hc,
                                cudaStream_t st) {
  long long want = (ncell + 8 * FE_THREADS - 1) / (8 * FE_THREADS);  // about 8 cells per thread
  const int blocks = (int)(want < 1 ? 1 : (want > FE_BLOCKS ? FE_BLOCKS : want));
  k_field_energy<T><<<blocks, FE_THREADS, 0, st>>>(f6[0], f6[1], f6[2], f6[3], f6[4], f6[5], ncell, out, scratch,
                                                     hc);
  return cudaGetLastError();
}
template cudaError_t launch_field_energy<float>(const float* const*, long long, double*, double*, HistCtl,
                                                cudaStream_t);
template cudaError_t launch_field_energy<double>(const double* const*, long long, double*, double*, HistCtl,
                                                 cudaStream_t);
size_t field_energy_scratch_bytes() { return sizeof(double) * (3 * FE_BLOCKS + 2); }

template <typename T>
__global__ void k_kinetic(const __grid_constant__ RunDev<T> r, double* out) {
  double acc = 0;
  for (int s = 0; s < 2; ++s) {
    const SpeciesBuf<T>& b = s ? r.in[1] : r.in[0];  // constant indices: no local copy of r
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

namespace picgb {

// ---------------------------------------------------------------------------------------------
// Psi_E(D_z) Psi_B(D_z)^-1 along z (the exact rational multiplier, Sec. 2): one thread per z-line
// and component, FP64 (complex) arithmetic; the FP32 copy stencil in front applies the filter only. Each factor 4 lam (1 - lam S)^-1 (1 - lam S^-1)^-1 of the
// inverse is a causal then an anticausal first-order recursion with the periodic start value
// sum_m lam^m x_(start - m) / (1 - lam^nz); the factor 4 lam and 1 / b_deg are applied at the end
// (their product is real).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_inverse_psi_z(InvPsiArgs<T> a) {
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int comp = blockIdx.y;
  if (l >= a.nxy) return;
  T* f = comp == 0 ? a.f[0] : a.f[1];
  double2* w = a.work + (size_t)comp * a.nz * a.nxy;
  const long long nxy = a.nxy;
  const int nz = a.nz;
  // Psi_E(D_z) (9 taps, periodic) in FP64 into the complex work line
  for (int k = 0; k < nz; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      int kk = k + m - 4;
      kk = kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk);
      if (kk < 0 || kk >= nz) kk = wrapi(kk, nz);  // lines shorter than 4 cells
      acc += a.pe_taps[m] * (double)f[kk * nxy + l];
    }
    w[k * nxy + l] = make_double2(acc, 0.0);
  }
  for (int i = 0; i < a.nf; ++i) {
    const double lr = a.lam_re[i], li = a.lam_im[i];
    // causal: y_k = x_k + lam y_(k-1), periodic
    double sr = 0.0, si = 0.0, pr = 1.0, pi = 0.0;
    for (int m = 0; m < nz; ++m) {
      const double2 x = w[(m == 0 ? 0 : nz - m) * nxy + l];
      sr += pr * x.x - pi * x.y;
      si += pr * x.y + pi * x.x;
      const double tr = pr * lr - pi * li;
      pi = pr * li + pi * lr;
      pr = tr;
    }
    // (pr, pi) = lam^nz; start value s / (1 - lam^nz)
    double dr = 1.0 - pr, di = -pi, dd = dr * dr + di * di;
    double yr = (sr * dr + si * di) / dd, yi = (si * dr - sr * di) / dd;
    w[l] = make_double2(yr, yi);
    for (int k = 1; k < nz; ++k) {
      const double2 x = w[k * nxy + l];
      const double nr = x.x + lr * yr - li * yi, ni = x.y + lr * yi + li * yr;
      yr = nr;
      yi = ni;
      w[k * nxy + l] = make_double2(yr, yi);
    }
    // anticausal: z_k = y_k + lam z_(k+1), periodic
    sr = 0.0;
    si = 0.0;
    pr = 1.0;
    pi = 0.0;
    for (int m = 0; m < nz; ++m) {
      const double2 x = w[(m == 0 ? nz - 1 : m - 1) * nxy + l];
      sr += pr * x.x - pi * x.y;
      si += pr * x.y + pi * x.x;
      const double tr = pr * lr - pi * li;
      pi = pr * li + pi * lr;
      pr = tr;
    }
    dr = 1.0 - pr;
    di = -pi;
    dd = dr * dr + di * di;
    yr = (sr * dr + si * di) / dd;
    yi = (si * dr - sr * di) / dd;
    w[(nz - 1) * nxy + l] = make_double2(yr, yi);
    for (int k = nz - 2; k >= 0; --k) {
      const double2 x = w[k * nxy + l];
      const double nr = x.x + lr * yr - li * yi, ni = x.y + lr * yi + li * yr;
      yr = nr;
      yi = ni;
      w[k * nxy + l] = make_double2(yr, yi);
    }
  }
  for (int k = 0; k < nz; ++k) f[k * nxy + l] = (T)(a.scale * w[k * nxy + l].x);
}

// The same operator with one warp per z-line and the line in shared memory (FP64 complex, one
// padding slot per 32 elements against bank conflicts). Each periodic first-order recursion
// y_k = x_k + lam y_(k-1) is a blocked scan: every lane runs it over its own chunk of L = ceil(nz/32)
// elements from zero, the 32 chunk maps y -> lam^len y + e are composed around the ring by a cyclic
// doubling scan (Y_j = A_j Y_j + B_j after the full window, so Y_j = B_j / (1 - lam^nz)), and each
// lane adds lam^(i+1) times the previous chunk's end value to its elements.
constexpr int IPZ_LINES = 8;  // z-lines (warps) per block

__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_fma(double2 a, double2 b, double2 c) {  // a b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_shfl(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ int ipz_pad(int k) { return k + (k >> 5); }

__device__ __forceinline__ void periodic_recursion(double2* w, int nz, double2 lam, bool rev, int lane) {
  const int L = (nz + 31) >> 5;
  const int k0 = min(lane * L, nz), k1 = min(k0 + L, nz);
  // 1. the chunk's recursion from zero; mu = lam^len
  double2 y = make_double2(0.0, 0.0), mu = make_double2(1.0, 0.0);
  for (int k = k0; k < k1; ++k) {
    double2& v = w[ipz_pad(rev ? nz - 1 - k : k)];
    y = c_fma(lam, y, v);
    v = y;
    mu = c_mul(mu, lam);
  }
  // 2. cyclic composition of the chunk maps: Y_j = A Y_(j - window) + B
  double2 A = mu, B = y;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const double2 Ap = c_shfl(A, (lane - s) & 31), Bp = c_shfl(B, (lane - s) & 31);
    B = c_fma(A, Bp, B);
    A = c_mul(A, Ap);
  }
  const double dr = 1.0 - A.x, di = -A.y, dd = dr * dr + di * di;
  const double2 Y = make_double2((B.x * dr + B.y * di) / dd, (B.y * dr - B.x * di) / dd);
  // 3. the previous chunk's end value carried into this chunk
  const double2 cin = c_shfl(Y, (lane - 1) & 31);
  double2 p = lam;
  for (int k = k0; k < k1; ++k) {
    double2& v = w[ipz_pad(rev ? nz - 1 - k : k)];
    v = c_fma(p, cin, v);
    p = c_mul(p, lam);
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * IPZ_LINES) k_inverse_psi_lines(const __grid_constant__ InvPsiArgs<T> a) {
  extern __shared__ __align__(16) unsigned char ipz_raw[];
  const int nz = a.nz, lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int stride = ipz_pad(nz - 1) + 1;  // padded line length
  double2* lines = reinterpret_cast<double2*>(ipz_raw);
  T* f = blockIdx.y == 0 ? a.f[0] : a.f[1];
  const long long l0 = (long long)blockIdx.x * IPZ_LINES;
  const int nl = (int)min((long long)IPZ_LINES, a.nxy - l0);
  // load the block's lines (consecutive l for each k: 8 values side by side) into the imaginary
  // slots, which the Psi_E pass reads while it writes the real slots
  for (int e = threadIdx.x; e < nz * IPZ_LINES; e += blockDim.x) {
    const int k = e / IPZ_LINES, li = e % IPZ_LINES;
    if (li < nl) lines[li * stride + ipz_pad(k)] = make_double2(0.0, (double)f[k * a.nxy + l0 + li]);
  }
  __syncthreads();
  if (wl < nl) {
    double2* w = lines + wl * stride;
    for (int k = lane; k < nz; k += 32) {  // Psi_E(D_z), 9 taps, periodic, FP64
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 9; ++m) acc += a.pe_taps[m] * w[ipz_pad(wrapi(k + m - 4, nz))].y;
      w[ipz_pad(k)].x = acc;
    }
    __syncwarp();
    for (int k = lane; k < nz; k += 32) w[ipz_pad(k)].y = 0.0;
    __syncwarp();
    for (int i = 0; i < a.nf; ++i) {
      const double2 lam = make_double2(a.lam_re[i], a.lam_im[i]);
      periodic_recursion(w, nz, lam, false, lane);  // causal
      __syncwarp();
      periodic_recursion(w, nz, lam, true, lane);   // anticausal
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nz * IPZ_LINES; e += blockDim.x) {
    const int k = e / IPZ_LINES, li = e % IPZ_LINES;
    if (li < nl) f[k * a.nxy + l0 + li] = (T)(a.scale * lines[li * stride + ipz_pad(k)].x);
  }
}

size_t inverse_psi_lines_smem(int nz) {
  return sizeof(double2) * (size_t)IPZ_LINES * (size_t)((nz - 1) + ((nz - 1) >> 5) + 1);
}

template <typename T>
cudaError_t launch_inverse_psi_z(const InvPsiArgs<T>& a, cudaStream_t st) {
  if (a.nxy <= 0 || a.nz <= 0) return cudaSuccess;
  const size_t sm = inverse_psi_lines_smem(a.nz);
  if (sm <= 200 * 1024) {  // lines up to about 1500 cells: the warp-per-line kernel
    cudaError_t e = ensure_dynamic_smem((const void*)k_inverse_psi_lines<T>, sm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.nxy + IPZ_LINES - 1) / IPZ_LINES), 2);
    k_inverse_psi_lines<T><<<grid, 32 * IPZ_LINES, sm, st>>>(a);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((a.nxy + 63) / 64), 2);  // longer lines: one thread per line in global memory
  k_inverse_psi_z<T><<<grid, 64, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_inverse_psi_z<float>(const InvPsiArgs<float>&, cudaStream_t);
template cudaError_t launch_inverse_psi_z<double>(const InvPsiArgs<double>&, cudaStream_t);

}  // namespace picgb
