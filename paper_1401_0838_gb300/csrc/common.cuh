// Internal definitions shared by the CUDA translation units of the PIC library.
// Nothing here is part of the public C ABI (include/pic.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace picgb {

// Sticky error bits written by kernels (read by the host at pic_sync / pic_energy).
enum : int {
  ERR_OVERFLOW = 1,   // a particle found its bin full and no room in the spill or leaver list: dropped
  ERR_NONFINITE = 2,  // a particle position or momentum became NaN/Inf or moved > 1 cell
  ERR_IMPORT = 4,     // an imported particle had an invalid cell or species
  ERR_TIMEOUT = 8,    // a bounded device wait gave up
  ERR_IDS = 16,       // particle ids are not a permutation of 0 .. N-1 (adjoint tape)
};

constexpr int MAX_ZTAPS = 33;  // combined z stencil: Psi (9 taps) convolved with the filter
constexpr int MAX_XTAPS = 25;  // filter stencil along x or y

// One species' particle storage in one of the two ping-pong buffers. Slot s of the arrays
// belongs to cell s / cap; cell c holds cnt[c] particles in slots [c*cap, c*cap + cnt[c]).
template <typename T>
struct SpeciesBuf {
  T *ox, *oy, *oz;     // offsets in [0,1) inside the cell (oy unused in 2D)
  T *dux, *duy, *duz;  // u - u0 z_hat
  T* w;                // per-particle weight or nullptr
  unsigned* id;        // particle id or nullptr
  int* cnt;            // particles per cell
};

// Particles that left their tile in a push (appended by the push kernel, inserted into their
// destination bins by the migrate kernel). key = destination cell * 2 + species. The same layout
// holds the spill list: particles whose destination bin was full when they were inserted (by the
// migrate kernel or the import); the next step pushes them from there (k_push_spill), and the
// host moves them into larger bins at its next synchronising call.
template <typename T>
struct LeaverList {
  int* key;
  T *ox, *oy, *oz, *dux, *duy, *duz, *w;
  unsigned* id;
};

// Entry o of a leaver or spill list (the arrays a run does not carry are null).
template <typename T>
__device__ __forceinline__ void list_put(const LeaverList<T>& l, long long o, int key, T ox, T oy, T oz, T ux, T uy,
                                         T uz, T w, unsigned id) {
  l.key[o] = key;
  l.ox[o] = ox;
  if (l.oy) l.oy[o] = oy;
  l.oz[o] = oz;
  l.dux[o] = ux;
  l.duy[o] = uy;
  l.duz[o] = uz;
  if (l.w) l.w[o] = w;
  if (l.id) l.id[o] = id;
}

// A sum held as an FP32 pair s + c, added with s by TwoSum and its rounding error into c. The block
// stages of the FP32 field energy sums reduce pairs, so no FP64 arithmetic runs until a block's
// partials leave it: GB300's FP64 pipe is narrow, and a one-wave launch's blocks all reach that stage
// at once.
struct FPair {
  float s, c;
};
__device__ __forceinline__ FPair pair_add(FPair a, FPair b) {
  const float t = a.s + b.s;
  const float bb = t - a.s;
  const float err = (a.s - (t - bb)) + (b.s - bb);
  return FPair{t, a.c + b.c + err};
}
__device__ __forceinline__ FPair warp_sum_pair(FPair v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = pair_add(v, FPair{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)});
  return v;
}

// Programmatic dependent launch. The kernels of a step are launched with launch_pdl, so a kernel's
// launch overlaps the completion of the kernel before it in the stream; pdl_wait, the first thing
// each of them does, holds it until that kernel has completed and its memory is visible (outside
// such a launch it returns at once). No kernel triggers its dependents early: measured, letting the
// next grid's blocks take SM resources while a kernel still runs cost 2 % of the step.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Particle tile of the linear push (cells per direction, the shared-memory tiles' size). A run's
// tiles are at most this (push_tiles); the launchers check it. Tall and narrow, along the drift:
// few particles leave a tile through a z face per step, and a warp's cell group spans several z
// rows, so a particle crossing into the next z cell mostly lands in a cell of its own group (one
// slot reservation for both). 3D FP64 keeps a cube: its shared-memory tiles are twice as large.
template <typename T, int NDIM>
struct PTile;
template <typename T>
struct PTile<T, 2> {
  static constexpr int TX = 4, TY = 1, TZ = 64;
};
template <>
struct PTile<float, 3> {
  static constexpr int TX = 2, TY = 2, TZ = 128;
};
template <>
struct PTile<double, 3> {
  static constexpr int TX = 8, TY = 8, TZ = 8;
};

// Particle tile of the cubic and momentum-conserving push (k_push_ho): tall along the drift in 2D
// too (the momentum-conserving push measured 14 % faster than on 16x16 tiles, the cubic the same).
template <typename T, int NDIM>
struct HoTile;
template <typename T>
struct HoTile<T, 2> {
  static constexpr int TX = 4, TY = 1, TZ = 64;
};
template <typename T>
struct HoTile<T, 3> {
  static constexpr int TX = 8, TY = 8, TZ = 8;
};

// Everything a kernel needs about one simulation (passed by value as a kernel parameter).
template <typename T>
struct RunDev {
  int ndim, nx, ny, nz;
  long long ncell;
  int ntx, nty, ntz;  // particle tiles per direction
  int tex, tey, tez;  // cells per particle tile and direction (at most PTile; origins at multiples)
  int cap;            // slots per cell per species
  int scheme;         // 0 Galerkin, 1 Uniform, 2 momentum-conserving
  T dtdx, dtdy, dtdz; // dt / d (grid units per unit velocity)
  T u0;               // drift momentum sqrt(gamma^2 - 1)
  T hq;               // dt / 2 (Boris half-kick for unit charge and mass)
  T wconst;           // weight when per-particle weights are absent
  T jfx, jfy, jfz;    // -d_a / (dV dt): Esirkepov current per unit (q w) and unit W
  T jfy2d;            // 1 / dV: 2D out-of-plane current per unit (q w v_y)
  T* g[6];            // field copies seen by the particles (Ex Ey Ez Bx By Bz)
  T* j[3];            // current accumulator
  SpeciesBuf<T> in[2], out[2];
  LeaverList<T> lv;
  int* lv_count;       // leavers appended in this step
  int* lv_other;       // the other parity's leaver counter (zeroed by this step's migrate)
  long long lv_cap;    // capacity of the leaver list
  LeaverList<T> sp;    // spill list
  int* sp_in;          // spilled particles waiting for this step's push (read by k_push_spill)
  int* sp_out;         // particles spilled by this step's insertions (zeroed by k_push_spill)
  long long sp_cap;    // capacity of the spill list
  unsigned long long* sp_total;  // insertions that found their bin full, since creation
  int* err;
  double* kin;        // FP64 accumulators of this step: [0] sum w (gamma - 1), [1] particle count
                      // (nullptr: not recorded)
};

// A run's tile extents lie within a push kernel's compile-time tile TL (its shared-memory size).
template <template <typename, int> class TL, typename T>
inline bool tiles_fit(const RunDev<T>& r) {
  if (r.tex < 1 || r.tey < 1 || r.tez < 1) return false;
  if (r.ndim == 2) return r.tex <= TL<T, 2>::TX && r.tey == 1 && r.tez <= TL<T, 2>::TZ;
  return r.tex <= TL<T, 3>::TX && r.tey <= TL<T, 3>::TY && r.tez <= TL<T, 3>::TZ;
}

// Device-side energy history of one run: the energy kernel writes sample (*count % cap) from its
// field sums and the kinetic accumulator kin[0..1] (filled by the push kernel), zeroes kin and
// increments *count, so a captured step needs no host bookkeeping.
struct HistCtl {
  double* hist;  // cap x 8 doubles
  int cap;
  int* count;
  double* kin;
};

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the multiply-xor round
// function with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,
// 0xBB67AE85.
// ---------------------------------------------------------------------------------------------
struct u32x4 {
  uint32_t v[4];
};

__host__ __device__ inline u32x4 philox10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint64_t a = (uint64_t)0xD2511F53u * c.v[0];
    uint64_t b = (uint64_t)0xCD9E8D57u * c.v[2];
    u32x4 n;
    n.v[0] = (uint32_t)(b >> 32) ^ c.v[1] ^ k0;
    n.v[1] = (uint32_t)b;
    n.v[2] = (uint32_t)(a >> 32) ^ c.v[3] ^ k1;
    n.v[3] = (uint32_t)a;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ---------------------------------------------------------------------------------------------
// Small math helpers
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T tri(T d) {  // linear spline max(0, 1 - |d|)
  T a = T(1) - (d < T(0) ? -d : d);
  return a > T(0) ? a : T(0);
}

__device__ __forceinline__ float dev_floor(float x) { return floorf(x); }
__device__ __forceinline__ double dev_floor(double x) { return floor(x); }
__device__ __forceinline__ float dev_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dev_sqrt(double x) { return sqrt(x); }

__device__ __forceinline__ void flag_error(int* err, int bit) {
  if (err) atomicOr(err, bit);
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// cp.async staging into shared memory: 16-byte copies through L2 only (particle packs), 4- or
// 8-byte copies through L1 (field tiles, counts); commit / wait of the thread's copy groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void copy4_async(float* dst, const float* src) { cp_async16(dst, src); }
__device__ __forceinline__ void copy4_async(double* dst, const double* src) {
  cp_async16(dst, src);
  cp_async16(dst + 2, src + 2);
}
__device__ __forceinline__ void copy4_async(unsigned* dst, const unsigned* src) { cp_async16(dst, src); }
__device__ __forceinline__ void copy1_async(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void copy1_async(int* dst, const int* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void copy1_async(double* dst, const double* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Tensor-memory-access (TMA) staging: one thread starts a tiled bulk copy of a box of a field into
// shared memory, completed on an mbarrier that every thread of the block waits on. The tensor map
// (a CUtensorMap encoded on the host) lives in the kernel's parameter space.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the copy engine
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// box of a 2D / 3D tensor at element coordinates (x, y[, z]); x * element size a multiple of 16 bytes
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
      : "memory");
}
// Wait for phase `parity` of the barrier to complete, giving up after `limit` polls (each poll may
// suspend the thread for a short, hardware-chosen time). Returns whether it completed.
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, unsigned parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
constexpr int TMA_WAIT_POLLS = 1 << 20;  // each poll returns within microseconds: a second or so in all

}  // namespace picgb
