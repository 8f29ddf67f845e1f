// Particle kernels: fused gather + Boris + move + Esirkepov deposition + rebin, beam
// initialisation, state import (binning) and export (compaction).
//
// Particle storage: per species, per cell, a bin of `cap` slots (SpeciesBuf). The push kernel
// reads the input buffer and writes every particle straight into its destination cell's bin of
// the output buffer (a counting-sort rebin fused into the push), so particles stay sorted by
// cell at no extra HBM pass. Positions are cell-relative offsets in [0,1); momenta are stored
// relative to the drift u0 z_hat so that FP32 keeps the thermal spread (u0 = 130, spread 1e-4).
#include "common.cuh"
#include "fastmath.cuh"
#include "launch.h"

namespace picgb {

// Threads per push block: 8 warps; the 3D FP32 kernel, one block per SM, takes 12 warps.
template <typename T, int NDIM>
struct PushThreads {
  static constexpr int value = (NDIM == 3 && sizeof(T) == 4) ? 384 : 256;
};

// Per-warp double-buffered stage: [stage][slot][lane][4] for the particle arrays (slots ox oz dux
// duy duz w in 2D; ox oy oz dux duy duz w in 3D), then [stage][lane][4] ids.
template <typename T, int NDIM>
struct PushStage {
  static constexpr int NSLOT = NDIM == 3 ? 7 : 6;
  // slot of array a (0 ox, 1 oy, 2 oz, 3 dux, 4 duy, 5 duz, 6 w); 2D stages no oy
  static constexpr __host__ __device__ int slot(int a) { return NDIM == 3 ? a : (a > 1 ? a - 1 : a); }
  static constexpr __host__ __device__ size_t per_warp_elems() {
    return 2 * NSLOT * 32 * 4 + (2 * 32 * 4 * sizeof(unsigned) + sizeof(T) - 1) / sizeof(T);
  }
  static __device__ __forceinline__ T* at(T* base, int stage, int arr, int lane) {
    return base + ((stage * NSLOT + slot(arr)) * 32 + lane) * 4;
  }
  static __device__ __forceinline__ unsigned* id_at(T* base, int stage, int lane) {
    return reinterpret_cast<unsigned*>(base + 2 * NSLOT * 32 * 4) + (stage * 32 + lane) * 4;
  }
};


template <typename T, int NDIM>
struct PushSmem {
  static constexpr int TX = PTile<T, NDIM>::TX, TY = PTile<T, NDIM>::TY, TZ = PTile<T, NDIM>::TZ;
  static constexpr int NCL = TX * TY * TZ;
  // gather tile: nodes [X0-1, X0+TX] per direction (y only in 3D)
  static constexpr int GX = TX + 2, GY = (NDIM == 3 ? TY + 2 : 1), GZ = TZ + 2, GN = GX * GY * GZ;
  // current tile: nodes [X0-1, X0+TX+1]
  static constexpr int JX = TX + 3, JY = (NDIM == 3 ? TY + 3 : 1), JZ = TZ + 3, JN = JX * JY * JZ;
  // particles leaving the tile, buffered per block: [7][LVB] values (ox oy oz dux duy duz w), LVB
  // keys, LVB ids and the buffer's counter; written to the global leaver list once per tile
  static constexpr int LVB = (NDIM == 3 && sizeof(T) == 8) ? 128 : 512;  // 3D FP64: within 227 KB
  static constexpr size_t lv_bytes() { return (size_t)LVB * (7 * sizeof(T) + 2 * sizeof(int)) + 16; }
  static constexpr size_t bytes() {
    return sizeof(T) * (6 * GN + 3 * JN) + sizeof(int) * (4 * NCL) + 16 +
           sizeof(T) * PushStage<T, NDIM>::per_warp_elems() * (PushThreads<T, NDIM>::value / 32) + 16 + lv_bytes();
  }
};

// Per-direction interpolation weights of a particle at cell-relative offset o:
// integer-node S1 (base 0: nodes 0, 1), half-node S1 (Uniform: base -1 or 0), half-node S0
// (Galerkin: node 0). Bases are relative to the particle's cell.
template <typename T>
struct DirW {
  T i0, i1;     // integer nodes 0 and 1
  int hb;       // half-node base (-1 or 0)
  T h0, h1;     // half nodes hb, hb+1
};

template <typename T>
__device__ __forceinline__ DirW<T> dir_weights(T o) {
  DirW<T> d;
  d.i0 = T(1) - o;
  d.i1 = o;
  if (o < T(0.5)) {
    d.hb = -1;
    T g = o + T(0.5);
    d.h0 = T(1) - g;
    d.h1 = g;
  } else {
    d.hb = 0;
    T g = o - T(0.5);
    d.h0 = T(1) - g;
    d.h1 = g;
  }
  return d;
}

// One direction of the gather: returns (base, w0, w1, two) for stagger st and scheme.
template <typename T, int SCHEME>
__device__ __forceinline__ void pick(const DirW<T>& d, int st, int& base, T& w0, T& w1, bool& two) {
  if (!st) {
    base = 0; w0 = d.i0; w1 = d.i1; two = true;
  } else if (SCHEME == 0) {  // Galerkin: S0 along a half-staggered direction
    base = 0; w0 = T(1); w1 = T(0); two = false;
  } else {                   // Uniform: S1 at the half-integer nodes
    base = d.hb; w0 = d.h0; w1 = d.h1; two = true;
  }
}

// Stagger of Ex Ey Ez Bx By Bz along x, y, z.
__device__ __constant__ int c_stag[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

template <typename T, int NDIM, int SCHEME>
__device__ __forceinline__ T gather_comp(const T* __restrict__ sgc, int c, int lx, int ly, int lz, const DirW<T>& dx,
                                         const DirW<T>& dy, const DirW<T>& dz) {
  using S = PushSmem<T, NDIM>;
  int bx, by = 0, bz;
  T x0, x1, y0 = T(1), y1 = T(0), z0, z1;
  bool tx, ty = false, tz;
  pick<T, SCHEME>(dx, c_stag[c][0], bx, x0, x1, tx);
  if (NDIM == 3) pick<T, SCHEME>(dy, c_stag[c][1], by, y0, y1, ty);
  pick<T, SCHEME>(dz, c_stag[c][2], bz, z0, z1, tz);
  // smem index of node (lx+bx, ly+by, lz+bz), +1 halo offset per direction
  const int ix = lx + bx + 1, iy = (NDIM == 3 ? ly + by + 1 : 0), iz = lz + bz + 1;
  const T* p = sgc + (iz * S::GY + iy) * S::GX + ix;
  T acc;
  {
    T r0 = x0 * p[0] + (tx ? x1 * p[1] : T(0));
    T r1 = T(0);
    if (ty) {
      const T* q = p + S::GX;
      r1 = x0 * q[0] + (tx ? x1 * q[1] : T(0));
    }
    acc = z0 * (y0 * r0 + y1 * r1);
  }
  if (tz) {
    const T* p2 = p + S::GX * S::GY;
    T r0 = x0 * p2[0] + (tx ? x1 * p2[1] : T(0));
    T r1 = T(0);
    if (ty) {
      const T* q = p2 + S::GX;
      r1 = x0 * q[0] + (tx ? x1 * q[1] : T(0));
    }
    acc += z1 * (y0 * r0 + y1 * r1);
  }
  return acc;
}

// One direction of an Esirkepov move of displacement d (|d| < 1 cell) from offset o in [0,1):
// the 3-node window (origin a = -1 or 0 relative to the cell), the start shapes S0 and the shape
// changes dS on it, and the new cell shift and offset. dS is formed from d itself (slope times
// the move on the linear piece of the spline), not as S(o + d) - S(o), so that moves far below one
// ulp of the offset (the transverse drift of a cold relativistic beam) keep full relative
// precision; the three dS always sum to zero (charge conservation).
template <typename T>
struct EsirDir {
  int a, shift;
  T off;
  T S0[3], dS[3];
};

// Comparisons of the push's values. FP64: integer tests on the IEEE bit patterns, exact for every
// value that is not a NaN (the offsets and displacements compared here are finite), which keeps
// them off the narrow FP64 pipe that bounds the FP64 push. FP32: plain comparisons.
template <typename T>
__device__ __forceinline__ bool is_neg(T x) {  // x < 0 (-0 is not)
  if constexpr (sizeof(T) == 8) return (unsigned long long)__double_as_longlong(x) > 0x8000000000000000ull;
  else return x < T(0);
}
template <typename T>
__device__ __forceinline__ bool is_pos(T x) {  // x > 0
  if constexpr (sizeof(T) == 8) return __double_as_longlong(x) > 0;
  else return x > T(0);
}
template <typename T>
__device__ __forceinline__ bool ge_one(T x) {  // x >= 1
  if constexpr (sizeof(T) == 8) return __double_as_longlong(x) >= 0x3FF0000000000000ll;
  else return x >= T(1);
}
template <typename T>
__device__ __forceinline__ bool is_zero(T x) {  // x == 0 (either sign)
  if constexpr (sizeof(T) == 8) return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) == 0;
  else return x == T(0);
}
template <typename T>
__device__ __forceinline__ bool abs_lt_one(T x) {  // -1 < x < 1; false for a NaN or an infinity
  if constexpr (sizeof(T) == 8) return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) < 0x3FF0000000000000ll;
  else return x > T(-1) && x < T(1);
}

template <typename T>
__device__ __forceinline__ EsirDir<T> esir_dir(T o, T d) {
  EsirDir<T> e;
  const T x1 = o + d;
  if (is_neg(x1)) {  // into the cell below: window nodes -1, 0, 1
    e.a = -1;
    e.S0[0] = T(0); e.S0[1] = T(1) - o; e.S0[2] = o;
    e.dS[0] = -x1; e.dS[2] = -o; e.dS[1] = -(e.dS[0] + e.dS[2]);
    e.off = T(1) + x1;
    e.shift = -1;
    if (ge_one(e.off)) { e.off = T(0); e.shift = 0; }
  } else {
    e.a = 0;
    e.S0[0] = T(1) - o; e.S0[1] = o; e.S0[2] = T(0);
    const T am = T(1) - o;  // distance to the upper face
    const T c = d - am;     // x1 - 1, without the rounding of x1
    if (ge_one(x1) && is_pos(c)) {  // into the cell above: nodes 0, 1, 2
      e.dS[0] = -am; e.dS[2] = c; e.dS[1] = -(e.dS[0] + e.dS[2]);
      e.off = c;
      e.shift = 1;
    } else {  // same cell (or onto the upper face within rounding)
      e.dS[0] = -d; e.dS[1] = d; e.dS[2] = T(0);
      if (ge_one(x1)) { e.off = T(0); e.shift = 1; }
      else { e.off = x1; e.shift = 0; }
    }
  }
  return e;
}

// Layout of one particle's current contributions: index i -> (component, node offset in the
// 3-node window). 2D: 6 Jx (b*2+a), 6 Jz (6+a*2+b), 9 Jy (12+b*3+a). 3D: 18 Jx ((c*3+b)*2+a),
// 18 Jy (18+(c*3+a)*2+b), 18 Jz (36+(b*3+a)*2+c); a, b, c are the x, y, z node offsets.
template <int NDIM>
struct DepLayout;
template <>
struct DepLayout<2> {
  static constexpr int NV = 21;
  static __device__ __forceinline__ void at(int i, int& comp, int& a, int& b, int& c) {
    b = 0;
    if (i < 6) { comp = 0; c = i >> 1; a = i & 1; }
    else if (i < 12) { comp = 2; a = (i - 6) >> 1; c = (i - 6) & 1; }
    else { comp = 1; c = (i - 12) / 3; a = (i - 12) % 3; }
  }
};
template <>
struct DepLayout<3> {
  static constexpr int NV = 54;
  static __device__ __forceinline__ void at(int i, int& comp, int& a, int& b, int& c) {
    if (i < 18) { comp = 0; a = i & 1; b = (i >> 1) % 3; c = (i >> 1) / 3; }
    else if (i < 36) { const int m = i - 18; comp = 1; b = m & 1; a = (m >> 1) % 3; c = (m >> 1) / 3; }
    else { const int m = i - 36; comp = 2; c = m & 1; a = (m >> 1) % 3; b = (m >> 1) / 3; }
  }
};

// Periodic index of g in [-n, 2n) without a modulo (callers guarantee the range: near_ok, or a
// neighbour cell index in [-1, n]).
__device__ __forceinline__ int wrap_near_p(int g, int n) { return g < 0 ? g + n : (g >= n ? g - n : g); }

// FP32 uses the hardware reciprocal square root and fast division (relative error ~1e-7, inside
// the 1e-5 per-step bar); FP64 keeps IEEE division and square root.

// Galerkin gather (order 0 along each half-staggered direction, order 1 elsewhere): the nodes are
// the same for every particle of a cell, so they are read once per lane and each component is an
// affine or bilinear function of the cell offsets. Node (a, b, c) of a component is its value at
// offsets (a, b, c) from the cell's own node in the shared-memory tile.
template <typename T, int NDIM>
struct GalCache;

template <typename T>
struct GalCache<T, 2> {
  // Ex: x half -> S0; z -> S1. Ey: S1 x, S1 z. Ez: S1 x; z half -> S0. Bx: S1 x; S0 z.
  // By: S0 x, S0 z. Bz: S0 x; S1 z.
  T ex0, ex1, ey00, ey10, ey01, ey11, ez0, ez1, bx0, bx1, by0, bz0, bz1;
  __device__ __forceinline__ void load(const T* sg, int lx, int ly, int lz) {
    using S = PushSmem<T, 2>;
    const int p = (lz + 1) * S::GX + lx + 1;
    const T* e = sg;
    ex0 = e[p]; ex1 = e[p + S::GX] - ex0;
    e = sg + S::GN;
    ey00 = e[p]; ey10 = e[p + 1] - ey00; ey01 = e[p + S::GX] - ey00; ey11 = e[p + S::GX + 1] - e[p + S::GX] - ey10;
    e = sg + 2 * S::GN;
    ez0 = e[p]; ez1 = e[p + 1] - ez0;
    e = sg + 3 * S::GN;
    bx0 = e[p]; bx1 = e[p + 1] - bx0;
    by0 = sg[4 * S::GN + p];
    e = sg + 5 * S::GN;
    bz0 = e[p]; bz1 = e[p + S::GX] - bz0;
  }
  __device__ __forceinline__ void interp(T ox, T, T oz, T (&F)[6]) const {
    F[0] = ex0 + oz * ex1;
    F[1] = ey00 + ox * ey10 + oz * (ey01 + ox * ey11);
    F[2] = ez0 + ox * ez1;
    F[3] = bx0 + ox * bx1;
    F[4] = by0;
    F[5] = bz0 + oz * bz1;
  }
};

template <typename T>
struct GalCache<T, 3> {
  // Ex: S0 x, bilinear (y, z). Ey: S0 y, bilinear (x, z). Ez: S0 z, bilinear (x, y).
  // Bx: S0 y, z, linear x. By: S0 x, z, linear y. Bz: S0 x, y, linear z.
  T e[3][4], b[3][2];
  __device__ __forceinline__ void bil(const T* f, int p, int s1, int s2, T (&o)[4]) {
    o[0] = f[p];
    o[1] = f[p + s1] - o[0];
    o[2] = f[p + s2] - o[0];
    o[3] = f[p + s1 + s2] - f[p + s2] - o[1];
  }
  __device__ __forceinline__ void load(const T* sg, int lx, int ly, int lz) {
    using S = PushSmem<T, 3>;
    const int p = ((lz + 1) * S::GY + ly + 1) * S::GX + lx + 1;
    const int sx = 1, sy = S::GX, sz = S::GX * S::GY;
    bil(sg, p, sy, sz, e[0]);
    bil(sg + S::GN, p, sx, sz, e[1]);
    bil(sg + 2 * S::GN, p, sx, sy, e[2]);
    b[0][0] = sg[3 * S::GN + p]; b[0][1] = sg[3 * S::GN + p + sx] - b[0][0];
    b[1][0] = sg[4 * S::GN + p]; b[1][1] = sg[4 * S::GN + p + sy] - b[1][0];
    b[2][0] = sg[5 * S::GN + p]; b[2][1] = sg[5 * S::GN + p + sz] - b[2][0];
  }
  __device__ __forceinline__ void interp(T ox, T oy, T oz, T (&F)[6]) const {
    F[0] = e[0][0] + oy * e[0][1] + oz * (e[0][2] + oy * e[0][3]);
    F[1] = e[1][0] + ox * e[1][1] + oz * (e[1][2] + ox * e[1][3]);
    F[2] = e[2][0] + ox * e[2][1] + oy * (e[2][2] + ox * e[2][3]);
    F[3] = b[0][0] + ox * b[0][1];
    F[4] = b[1][0] + oy * b[1][1];
    F[5] = b[2][0] + oz * b[2][1];
  }
};

// Esirkepov contributions of one particle, written as sums into the 3-node window of its own
// cell (layout of DepLayout). With f = S0 + dS/2 per direction, the 2D out-of-plane weight
// S0x S0z + dSx S0z/2 + S0x dSz/2 + dSx dSz/3 equals fx fz + dSx dSz / 12, and the running sums
// of the in-plane weights at the two half-nodes are dS[0] and -dS[2] times the transverse factor.
template <typename T, int NVP>
__device__ __forceinline__ void deposit2(T (&acc)[NVP], const EsirDir<T>& X, const EsirDir<T>& Z, T cx, T cy, T cz) {
  T fx[3], fz[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fx[a] = X.S0[a] + T(0.5) * X.dS[a];
    fz[a] = Z.S0[a] + T(0.5) * Z.dS[a];
  }
  const T gx0 = cx * X.dS[0], gx1 = -cx * X.dS[2];
  const T gz0 = cz * Z.dS[0], gz1 = -cz * Z.dS[2];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    acc[b * 2 + 0] += gx0 * fz[b];
    acc[b * 2 + 1] += gx1 * fz[b];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc[6 + a * 2 + 0] += gz0 * fx[a];
    acc[6 + a * 2 + 1] += gz1 * fx[a];
  }
  T hx[3], kx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hx[a] = cy * fx[a];
    kx[a] = cy * X.dS[a] * T(1.0 / 12.0);
  }
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[12 + b * 3 + a] += hx[a] * fz[b] + kx[a] * Z.dS[b];
}

// Same contributions added to shared memory at the window origin (wx, wz) (tile indices).
template <typename T, int NDIM>
__device__ __noinline__ void deposit2_smem(T* sj, int wx, int wz, EsirDir<T> X, EsirDir<T> Z, T cx, T cy, T cz) {
  using S = PushSmem<T, NDIM>;
  T v[DepLayout<2>::NV];
#pragma unroll
  for (int i = 0; i < DepLayout<2>::NV; ++i) v[i] = T(0);
  deposit2<T, DepLayout<2>::NV>(v, X, Z, cx, cy, cz);
  const int key = wz * S::JX + wx;
#pragma unroll
  for (int i = 0; i < DepLayout<2>::NV; ++i) {
    int comp, a, b, c;
    DepLayout<2>::at(i, comp, a, b, c);
    atomicAdd(sj + comp * S::JN + key + c * S::JX + a, v[i]);
  }
}

// 3D: W_a = dS_a T(b1, b2) with T = f f + dS dS / 12 over the two transverse directions.
template <typename T, int NVP>
__device__ __forceinline__ void deposit3(T (&acc)[NVP], const EsirDir<T>& X, const EsirDir<T>& Y, const EsirDir<T>& Z,
                                         T cx, T cy, T cz) {
  T fx[3], fy[3], fz[3], kx[3], ky[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fx[a] = X.S0[a] + T(0.5) * X.dS[a];
    fy[a] = Y.S0[a] + T(0.5) * Y.dS[a];
    fz[a] = Z.S0[a] + T(0.5) * Z.dS[a];
    kx[a] = X.dS[a] * T(1.0 / 12.0);
    ky[a] = Y.dS[a] * T(1.0 / 12.0);
  }
  const T gx0 = cx * X.dS[0], gx1 = -cx * X.dS[2];
  const T gy0 = cy * Y.dS[0], gy1 = -cy * Y.dS[2];
  const T gz0 = cz * Z.dS[0], gz1 = -cz * Z.dS[2];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {  // Jx(a+1/2, b, c)
      const T t = fy[b] * fz[c] + ky[b] * Z.dS[c];
      acc[(c * 3 + b) * 2 + 0] += gx0 * t;
      acc[(c * 3 + b) * 2 + 1] += gx1 * t;
    }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // Jy(a, b+1/2, c)
      const T t = fx[a] * fz[c] + kx[a] * Z.dS[c];
      acc[18 + (c * 3 + a) * 2 + 0] += gy0 * t;
      acc[18 + (c * 3 + a) * 2 + 1] += gy1 * t;
    }
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // Jz(a, b, c+1/2)
      const T t = fx[a] * fy[b] + kx[a] * Y.dS[b];
      acc[36 + (b * 3 + a) * 2 + 0] += gz0 * t;
      acc[36 + (b * 3 + a) * 2 + 1] += gz1 * t;
    }
}

template <typename T, int NDIM>
__device__ __noinline__ void deposit3_smem(T* sj, int wx, int wy, int wz, EsirDir<T> X, EsirDir<T> Y, EsirDir<T> Z,
                                           T cx, T cy, T cz) {
  using S = PushSmem<T, NDIM>;
  T v[DepLayout<3>::NV];
#pragma unroll
  for (int i = 0; i < DepLayout<3>::NV; ++i) v[i] = T(0);
  deposit3<T, DepLayout<3>::NV>(v, X, Y, Z, cx, cy, cz);
  const int key = (wz * S::JY + wy) * S::JX + wx;
#pragma unroll
  for (int i = 0; i < DepLayout<3>::NV; ++i) {
    int comp, a, b, c;
    DepLayout<3>::at(i, comp, a, b, c);
    atomicAdd(sj + comp * S::JN + key + (c * S::JY + b) * S::JX + a, v[i]);
  }
}

// The sums each lane keeps in registers: the Esirkepov window of a particle that starts in its own
// cell, does not step back across a face, and does not cross its cell's upper face in x (nor, in
// 3D, in y). Such a particle's shape changes vanish at the window's third transverse node (S0 and
// dS are zero there), so its contributions there are exactly zero: of the 3-node window only
// x nodes 0-1 (2D: 13 of the 21 sums; 3D: y nodes 0-1 too, 20 of the 54) carry it. Every other
// particle (a transverse face crossed, or a step back) adds its full window to shared memory.
// 2D layout: 3 Jx (node a = 0, z node c = i), 4 Jz (3 + a*2 + c), 6 Jy (7 + c*2 + a).
// 3D layout: 6 Jx (a = 0; c*2 + b), 6 Jy (b = 0; 6 + c*2 + a), 8 Jz (12 + (b*2 + a)*2 + c).
template <int NDIM>
struct RegLayout;
template <>
struct RegLayout<2> {
  static constexpr int NV = 13;
  static __device__ __forceinline__ void at(int i, int& comp, int& a, int& b, int& c) {
    b = 0;
    if (i < 3) { comp = 0; a = 0; c = i; }
    else if (i < 7) { comp = 2; a = (i - 3) >> 1; c = (i - 3) & 1; }
    else { comp = 1; c = (i - 7) >> 1; a = (i - 7) & 1; }
  }
};
template <>
struct RegLayout<3> {
  static constexpr int NV = 20;
  static __device__ __forceinline__ void at(int i, int& comp, int& a, int& b, int& c) {
    if (i < 6) { comp = 0; a = 0; b = i & 1; c = i >> 1; }
    else if (i < 12) { const int k = i - 6; comp = 1; b = 0; a = k & 1; c = k >> 1; }
    else { const int k = i - 12; comp = 2; c = k & 1; a = (k >> 1) & 1; b = k >> 2; }
  }
};

// Whether a particle's window fits the register sums (see RegLayout).
template <typename T, int NDIM>
__device__ __forceinline__ bool reg_window(const EsirDir<T>& X, const EsirDir<T>& Y, const EsirDir<T>& Z) {
  if (NDIM == 3) return (X.a | Y.a | Z.a) == 0 && is_zero(X.dS[2]) && is_zero(Y.dS[2]);
  return (X.a | Z.a) == 0 && is_zero(X.dS[2]);
}

// The contributions of deposit2 / deposit3 that can be nonzero for such a particle, into the
// register layout (the same products and sums as the full window).
template <typename T, int NVP>
__device__ __forceinline__ void deposit2_reg(T (&acc)[NVP], const EsirDir<T>& X, const EsirDir<T>& Z, T cx, T cy,
                                             T cz) {
  const T fx0 = X.S0[0] + T(0.5) * X.dS[0], fx1 = X.S0[1] + T(0.5) * X.dS[1];
  T fz[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) fz[b] = Z.S0[b] + T(0.5) * Z.dS[b];
  const T gx0 = cx * X.dS[0];
#pragma unroll
  for (int b = 0; b < 3; ++b) acc[b] += gx0 * fz[b];
  const T gz0 = cz * Z.dS[0], gz1 = -cz * Z.dS[2];
  acc[3] += gz0 * fx0;
  acc[4] += gz1 * fx0;
  acc[5] += gz0 * fx1;
  acc[6] += gz1 * fx1;
  const T hx0 = cy * fx0, hx1 = cy * fx1;
  const T kx0 = cy * X.dS[0] * T(1.0 / 12.0), kx1 = cy * X.dS[1] * T(1.0 / 12.0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    acc[7 + 2 * b] += hx0 * fz[b] + kx0 * Z.dS[b];
    acc[8 + 2 * b] += hx1 * fz[b] + kx1 * Z.dS[b];
  }
}

template <typename T, int NVP>
__device__ __forceinline__ void deposit3_reg(T (&acc)[NVP], const EsirDir<T>& X, const EsirDir<T>& Y,
                                             const EsirDir<T>& Z, T cx, T cy, T cz) {
  T fx[2], fy[2], fz[3], kx[2], ky[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    fx[a] = X.S0[a] + T(0.5) * X.dS[a];
    fy[a] = Y.S0[a] + T(0.5) * Y.dS[a];
    kx[a] = X.dS[a] * T(1.0 / 12.0);
    ky[a] = Y.dS[a] * T(1.0 / 12.0);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) fz[c] = Z.S0[c] + T(0.5) * Z.dS[c];
  const T gx0 = cx * X.dS[0], gy0 = cy * Y.dS[0];
  const T gz0 = cz * Z.dS[0], gz1 = -cz * Z.dS[2];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[c * 2 + b] += gx0 * (fy[b] * fz[c] + ky[b] * Z.dS[c]);  // Jx(1/2, b, c)
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int a = 0; a < 2; ++a) acc[6 + c * 2 + a] += gy0 * (fx[a] * fz[c] + kx[a] * Z.dS[c]);  // Jy(a, 1/2, c)
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) {  // Jz(a, b, c + 1/2)
      const T t = fx[a] * fy[b] + kx[a] * Y.dS[b];
      acc[12 + (b * 2 + a) * 2 + 0] += gz0 * t;
      acc[12 + (b * 2 + a) * 2 + 1] += gz1 * t;
    }
}

// Work assignment of the push kernel: a warp takes CPW = 32/LPC cells of its tile at a time,
// LPC lanes per cell. The cell's particles are split into packs of 4 consecutive slots of one
// species (electron packs first); lane l of the cell takes packs l, l + LPC, ... . Each lane sums
// the Esirkepov contributions of its particles in registers (the window of RegLayout: every
// particle that neither steps back across a face nor crosses a transverse face); at the end one
// segmented butterfly transpose-reduction over the cell's LPC lanes leaves PER = NVP/LPC of the
// cell's NVP (padded) sums in each lane, added to shared memory with distinct addresses. The other
// particles add their full 3-node window to shared memory directly.
template <int NDIM, int LPC>
struct PushPlan {
  static constexpr int NV = RegLayout<NDIM>::NV;
  static constexpr int PER = (NV + LPC - 1) / LPC;
  static constexpr int NVP = PER * LPC;
  static constexpr int CPW = 32 / LPC;
};

// Resident blocks per SM the push kernel is compiled for (register budget): FP32 2D fits two.
template <typename T, int NDIM>
struct PushMinBlocks {
  static constexpr int value = (sizeof(T) == 4 && NDIM == 2) ? 2 : 1;
};

// FP32 2D: each lane takes the particles of its pack two at a time, with the arithmetic of the pair
// in packed FP32x2 instructions (one instruction advances both particles) and the two rebins
// interleaved, so one dependent chain carries two particles.
template <typename T, int NDIM>
struct PushPaired {
  static constexpr bool value = sizeof(T) == 4 && NDIM == 2;
};

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <typename T, int NDIM, int SCHEME, int LPC>
__device__ __forceinline__ void push_tile(const RunDev<T>& r, const int tile) {
  using S = PushSmem<T, NDIM>;
  using PL = PushPlan<NDIM, LPC>;
  constexpr int TX = S::TX, TY = S::TY, NCL = S::NCL;
  constexpr int NV = PL::NV, PER = PL::PER, NVP = PL::NVP, CPW = PL::CPW;
  constexpr int PUSH_THREADS = PushThreads<T, NDIM>::value, NWARP = PUSH_THREADS / 32;
  static_assert(NCL % CPW == 0, "cells per tile must be a multiple of the cells per warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sg = reinterpret_cast<T*>(smem_raw);
  T* sj = sg + 6 * S::GN;
  int* sn = reinterpret_cast<int*>(sj + 3 * S::JN);  // [species][cell] particle counts (input)
  int* scnt = sn + 2 * NCL;                          // [species][cell] output counts of this tile

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // per-warp stages start on a 16-byte boundary after the counts (cp.async destinations)
  const size_t stage_off = ((size_t)(reinterpret_cast<unsigned char*>(scnt + 2 * NCL) - smem_raw) + 15) & ~(size_t)15;
  using SG = PushStage<T, NDIM>;
  T* stg = reinterpret_cast<T*>(smem_raw + stage_off) + (size_t)warp * SG::per_warp_elems();
  // the tile's leaver buffer follows every warp's stage
  const size_t lv_off = (stage_off + sizeof(T) * SG::per_warp_elems() * NWARP + 15) & ~(size_t)15;
  T* lvv = reinterpret_cast<T*>(smem_raw + lv_off);
  int* lvk = reinterpret_cast<int*>(lvv + 7 * S::LVB);
  unsigned* lvi = reinterpret_cast<unsigned*>(lvk + S::LVB);
  int* lvn = reinterpret_cast<int*>(lvi + S::LVB);
  const int tix = tile % r.ntx;
  const int tiy = (tile / r.ntx) % r.nty;
  const int tiz = tile / (r.ntx * r.nty);
  // the run's tile extents (r.tex <= TX ...): cells past them stay empty, as at the grid's edge
  const int X0 = tix * r.tex, Y0 = tiy * r.tey, Z0 = tiz * r.tez;
  const int wx = min(r.tex, r.nx - X0), wy = min(r.tey, r.ny - Y0), wz = min(r.tez, r.nz - Z0);
  const long long nxy = (long long)r.nx * r.ny;

  const bool has_w = r.in[0].w != nullptr;
  const bool has_id = r.in[0].id != nullptr;
  const int sl = lane % LPC;  // lane within its cell group

  // 1. field copies of the tile and its halo into shared memory (periodic wrap); zero the current
  const bool near_ok = r.nx >= S::TX + 2 && r.nz >= S::TZ + 2 && (NDIM == 2 || r.ny >= S::TY + 2);
  for (int e = tid; e < 6 * S::GN; e += PUSH_THREADS) {
    int c = e / S::GN, rem = e - c * S::GN;
    int lz = rem / (S::GX * S::GY);
    int ly = (rem / S::GX) % S::GY;
    int lx = rem % S::GX;
    // tile + halo lies within one period of the grid when the grid has at least TX+2 cells
    int gx = near_ok ? wrap_near_p(X0 - 1 + lx, r.nx) : wrapi(X0 - 1 + lx, r.nx);
    int gy = NDIM == 3 ? (near_ok ? wrap_near_p(Y0 - 1 + ly, r.ny) : wrapi(Y0 - 1 + ly, r.ny)) : 0;
    int gz = near_ok ? wrap_near_p(Z0 - 1 + lz, r.nz) : wrapi(Z0 - 1 + lz, r.nz);
    const T* src = r.g[0];
    switch (c) {  // constant-indexed parameter reads (no local copy of r.g)
      case 1: src = r.g[1]; break;
      case 2: src = r.g[2]; break;
      case 3: src = r.g[3]; break;
      case 4: src = r.g[4]; break;
      case 5: src = r.g[5]; break;
      default: break;
    }
    copy1_async(sg + e, src + (long long)gz * nxy + (long long)gy * r.nx + gx);
  }
  for (int e = tid; e < 3 * S::JN; e += PUSH_THREADS) sj[e] = T(0);
  // 2. particle counts of the tile's cells, copied in the same asynchronous batch as the fields (one
  // global round trip for both); then clamped, and the input counts zeroed (they are the next
  // step's output counts). Each thread reads back only the counts it copied itself.
  for (int cl = tid; cl < NCL; cl += PUSH_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    if (lx < wx && ly < wy && lz < wz) {
      const long long cell = (long long)(Z0 + lz) * nxy + (long long)(Y0 + ly) * r.nx + X0 + lx;
      copy1_async(sn + cl, r.in[0].cnt + cell);
      copy1_async(sn + NCL + cl, r.in[1].cnt + cell);
    } else {
      sn[cl] = 0;
      sn[NCL + cl] = 0;
    }
    scnt[cl] = 0;
    scnt[NCL + cl] = 0;
  }
  // The first item of the warp's first cell group, in the same batch although the counts are not in
  // yet: lane sl takes pack sl of species 0, as it does whenever its cell holds more than 4 sl
  // particles of species 0 (slots below cap: inside the cell's own bin). A lane whose first pack is
  // of species 1 copies it again once the counts are known.
  {
    const int c = warp * CPW + lane / LPC;  // every warp has a first group (NCL / CPW >= NWARP)
    const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    if (lx < wx && ly < wy && lz < wz && 4 * sl + 4 <= r.cap) {
      const long long slot0 =
          ((long long)(Z0 + lz) * nxy + (long long)(Y0 + ly) * r.nx + X0 + lx) * r.cap + 4 * sl;
      const SpeciesBuf<T>& pin = r.in[0];
      const T* src[7] = {pin.ox, pin.oy, pin.oz, pin.dux, pin.duy, pin.duz, pin.w};
#pragma unroll
      for (int arr = 0; arr < 7; ++arr) {
        if (arr == 1 && NDIM == 2) continue;
        if (arr == 6 && !has_w) continue;
        copy4_async(SG::at(stg, 0, arr, lane), src[arr] + slot0);
      }
      if (has_id) copy4_async(SG::id_at(stg, 0, lane), pin.id + slot0);
    }
  }
  static_assert(NCL / CPW >= NWARP, "every warp needs a first cell group");
  cp_async_commit();
  cp_async_wait_all();
  for (int cl = tid; cl < NCL; cl += PUSH_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    if (lx < wx && ly < wy && lz < wz) {
      const long long cell = (long long)(Z0 + lz) * nxy + (long long)(Y0 + ly) * r.nx + X0 + lx;
      sn[cl] = min(sn[cl], r.cap);  // the excess of a full bin waits in the spill list
      sn[NCL + cl] = min(sn[NCL + cl], r.cap);
      r.in[0].cnt[cell] = 0;
      r.in[1].cnt[cell] = 0;
    }
  }
  // cell groups after each warp's first one are handed out in the order warps ask for them, so
  // warps whose groups hold more packs do fewer groups
  __shared__ int s_next_group;
  if (tid == 0) {
    *lvn = 0;
    s_next_group = PUSH_THREADS / 32;
  }
  __syncthreads();

  T kin = T(0);
  int npush = 0;

  // Items of this warp: (cell group, pack round). The packs of the next item are copied into the
  // warp's shared-memory stage with cp.async while the current item is computed.
  constexpr int NGRP = NCL / CPW;
  auto group_iters = [&](int g) -> int {
    const int c = g * CPW + lane / LPC;
    const int nq = ((sn[c] + 3) >> 2) + ((sn[NCL + c] + 3) >> 2);
    return __reduce_max_sync(0xffffffffu, (nq + LPC - 1) / LPC);
  };
  // fix: only the packs the speculative first copy did not cover (species 1, or slots past cap)
  auto issue = [&](int g, int it, int stage, bool fix) {
    const int c = g * CPW + lane / LPC;
    const int n0 = sn[c], n1 = sn[NCL + c];
    const int nq0 = (n0 + 3) >> 2, nq = nq0 + ((n1 + 3) >> 2);
    const int q = sl + it * LPC;
    if (q >= nq) return;
    const int s = q >= nq0 ? 1 : 0;
    const int q4 = 4 * (s ? q - nq0 : q);
    if (fix && s == 0 && q4 + 4 <= r.cap) return;
    const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    const long long slot0 = ((long long)(Z0 + lz) * nxy + (long long)(Y0 + ly) * r.nx + X0 + lx) * r.cap + q4;
    const SpeciesBuf<T> pin = s ? r.in[1] : r.in[0];
    const T* src[7] = {pin.ox, pin.oy, pin.oz, pin.dux, pin.duy, pin.duz, pin.w};
#pragma unroll
    for (int arr = 0; arr < 7; ++arr) {
      if (arr == 1 && NDIM == 2) continue;
      if (arr == 6 && !has_w) continue;
      copy4_async(SG::at(stg, stage, arr, lane), src[arr] + slot0);
    }
    if (has_id) copy4_async(SG::id_at(stg, stage, lane), pin.id + slot0);
  };

  auto take_group = [&]() -> int {
    int v = 0;
    if (lane == 0) v = atomicAdd(&s_next_group, 1);
    return __shfl_sync(0xffffffffu, v, 0);
  };
  int g = warp, it = 0;
  int giters = g < NGRP ? group_iters(g) : 0;
  while (g < NGRP && giters == 0) {
    g = take_group();
    giters = g < NGRP ? group_iters(g) : 0;
  }
  int stage = 0;
  if (g < NGRP) issue(g, 0, 0, g == warp);  // the first group's first item was copied speculatively
  cp_async_commit();
  T acc[NVP];
  GalCache<T, NDIM> gc;  // Galerkin nodes of the lane's cell, loaded once per cell group
  while (g < NGRP) {
    // prefetch the next item
    int ng = g, nit = it + 1, niters = giters;
    if (nit >= giters) {
      nit = 0;
      do {
        ng = take_group();
        niters = ng < NGRP ? group_iters(ng) : 0;
      } while (ng < NGRP && niters == 0);
    }
    if (ng < NGRP) issue(ng, nit, stage ^ 1, false);
    cp_async_commit();
    cp_async_wait_1();
    __syncwarp();

    const int cl = g * CPW + lane / LPC;
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    const int gi = X0 + lx, gj = Y0 + ly, gk = Z0 + lz;
    const int n0 = sn[cl], n1 = sn[NCL + cl];
    const int nq0 = (n0 + 3) >> 2, nq = nq0 + ((n1 + 3) >> 2);
    const int okey = ((lz + 1) * S::JY + (NDIM == 3 ? ly + 1 : 0)) * S::JX + lx + 1;  // cell-origin window
    if (it == 0) {
      if (SCHEME == 0) gc.load(sg, lx, ly, lz);
#pragma unroll
      for (int i = 0; i < NVP; ++i) acc[i] = T(0);
    }
    {
      const int q = sl + it * LPC;
      const bool has = q < nq;
      const int s = (has && q >= nq0) ? 1 : 0;
      const int q4 = 4 * (s ? q - nq0 : q);
      const int cnt = has ? min(4, (s ? n1 : n0) - q4) : 0;
      const SpeciesBuf<T> pout = s ? r.out[1] : r.out[0];
      const T qs = s ? T(1) : T(-1);
      const T* st_x = SG::at(stg, stage, 0, lane);  // array a of the lane's pack at st_x + slot(a) * 128
      const unsigned* st_id = SG::id_at(stg, stage, lane);
      if constexpr (PushPaired<T, NDIM>::value) {
        const float2 hh = make_float2(qs * r.hq, qs * r.hq);
        const float2 u02 = make_float2(r.u0, r.u0), one2 = make_float2(1.f, 1.f);
        const float2 dtdx2 = make_float2(r.dtdx, r.dtdx), dtdz2 = make_float2(r.dtdz, r.dtdz);
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll 1
        for (int rp = 0; rp < 4; rp += 2) {
          // the pack elements (ja, ja + 1) of this pair, one 8-byte load per array; lanes 8-15 and
          // 24-31 take the other pair first, so a half-warp's loads cover all 32 banks
          const int ja = 2 * (((rp >> 1) + (lane >> 3)) & 1), jb = ja + 1;
          const bool va = ja < cnt, vb = jb < cnt;
          const float2 pox = *reinterpret_cast<const float2*>(st_x + ja);
          const float2 poz = *reinterpret_cast<const float2*>(st_x + SG::slot(2) * 128 + ja);
          const float2 pux = *reinterpret_cast<const float2*>(st_x + SG::slot(3) * 128 + ja);
          const float2 puy = *reinterpret_cast<const float2*>(st_x + SG::slot(4) * 128 + ja);
          const float2 puz = *reinterpret_cast<const float2*>(st_x + SG::slot(5) * 128 + ja);
          // an empty slot stands in as a particle at rest with no weight (finite, deposits nothing)
          const float oxa = va ? pox.x : 0.5f, oza = va ? poz.x : 0.5f;
          const float uxa = va ? pux.x : 0.f, uya = va ? puy.x : 0.f, uza = va ? puz.x : 0.f;
          const float oxb = vb ? pox.y : 0.5f, ozb = vb ? poz.y : 0.5f;
          const float uxb = vb ? pux.y : 0.f, uyb = vb ? puy.y : 0.f, uzb = vb ? puz.y : 0.f;
          float wa = 0.f, wb = 0.f;
          if (has_w) {
            const float2 pw = *reinterpret_cast<const float2*>(st_x + SG::slot(6) * 128 + ja);
            wa = va ? pw.x : 0.f;
            wb = vb ? pw.y : 0.f;
          } else {
            wa = va ? r.wconst : 0.f;
            wb = vb ? r.wconst : 0.f;
          }
          // gather
          float Fa[6], Fb[6];
          if (SCHEME == 0) {
            gc.interp(oxa, 0.f, oza, Fa);
            gc.interp(oxb, 0.f, ozb, Fb);
          } else {
            const DirW<float> xa = dir_weights(oxa), za = dir_weights(oza), xb = dir_weights(oxb),
                              zb = dir_weights(ozb), y0 = dir_weights(0.f);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              Fa[c] = gather_comp<float, 2, SCHEME>(sg + c * S::GN, c, lx, 0, lz, xa, y0, za);
              Fb[c] = gather_comp<float, 2, SCHEME>(sg + c * S::GN, c, lx, 0, lz, xb, y0, zb);
            }
          }
          const float2 Ex = make_float2(Fa[0], Fb[0]), Ey = make_float2(Fa[1], Fb[1]), Ez = make_float2(Fa[2], Fb[2]);
          const float2 Bx = make_float2(Fa[3], Fb[3]), By = make_float2(Fa[4], Fb[4]), Bz = make_float2(Fa[5], Fb[5]);
          // relativistic Boris of the pair, momenta relative to the drift u0 z_hat
          const float2 mx = fma2(hh, Ex, make_float2(uxa, uxb));
          const float2 my = fma2(hh, Ey, make_float2(uya, uyb));
          const float2 mz = fma2(hh, Ez, make_float2(uza, uzb));
          const float2 Mz = add2(u02, mz);
          float2 m2 = fma2(mx, mx, one2);
          m2 = fma2(my, my, m2);
          m2 = fma2(Mz, Mz, m2);
          const float2 hig = mul2(hh, make_float2(fast_rsqrt(m2.x), fast_rsqrt(m2.y)));
          const float2 tx = mul2(hig, Bx), ty = mul2(hig, By), tz = mul2(hig, Bz);
          float2 t2 = fma2(tx, tx, one2);
          t2 = fma2(ty, ty, t2);
          t2 = fma2(tz, tz, t2);
          const float2 sf = make_float2(fast_div(2.f, t2.x), fast_div(2.f, t2.y));
          const float2 sx = mul2(sf, tx), sy = mul2(sf, ty), sz = mul2(sf, tz);
          const float2 qx = fma2(my, tz, fma2(neg2(Mz), ty, mx));
          const float2 qy = fma2(Mz, tx, fma2(neg2(mx), tz, my));
          const float2 qz = fma2(mx, ty, fma2(neg2(my), tx, Mz));
          const float2 ux2 = fma2(qy, sz, fma2(neg2(qz), sy, fma2(hh, Ex, mx)));
          const float2 uy2 = fma2(qz, sx, fma2(neg2(qx), sz, fma2(hh, Ey, my)));
          const float2 uz2 = fma2(qx, sy, fma2(neg2(qy), sx, fma2(hh, Ez, mz)));
          const float2 Uz = add2(u02, uz2);
          float2 u2 = mul2(ux2, ux2);
          u2 = fma2(uy2, uy2, u2);
          u2 = fma2(Uz, Uz, u2);
          const float2 gp = add2(one2, u2);
          const float2 ign = make_float2(fast_rsqrt(gp.x), fast_rsqrt(gp.y));
          const float2 g1 = fma2(gp, ign, one2);  // gamma + 1; gamma - 1 = u^2 / (gamma + 1)
          kin = fmaf(wa, fast_div(u2.x, g1.x), kin);
          kin = fmaf(wb, fast_div(u2.y, g1.y), kin);
          npush += (va ? 1 : 0) + (vb ? 1 : 0);
          const float2 vy2 = mul2(uy2, ign);
          const float2 ddx2 = mul2(dtdx2, mul2(ux2, ign)), ddz2 = mul2(dtdz2, mul2(Uz, ign));
          float dxa = ddx2.x, dza = ddz2.x, dxb = ddx2.y, dzb = ddz2.y;
          float nuxa = ux2.x, nuya = uy2.x, nuza = uz2.x, vya = vy2.x;
          float nuxb = ux2.y, nuyb = uy2.y, nuzb = uz2.y, vyb = vy2.y;
          if (!(dxa > -1.f && dxa < 1.f && dza > -1.f && dza < 1.f)) {
            flag_error(r.err, ERR_NONFINITE);
            dxa = dza = nuxa = nuya = nuza = vya = 0.f;
          }
          if (!(dxb > -1.f && dxb < 1.f && dzb > -1.f && dzb < 1.f)) {
            flag_error(r.err, ERR_NONFINITE);
            dxb = dzb = nuxb = nuyb = nuzb = vyb = 0.f;
          }
          // Esirkepov deposits
          const EsirDir<float> exa = esir_dir(oxa, dxa), eza = esir_dir(oza, dza);
          const EsirDir<float> exb = esir_dir(oxb, dxb), ezb = esir_dir(ozb, dzb);
          if (va) {
            const float qw = qs * wa;
            const float cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vya * r.jfy2d;
            if (reg_window<float, 2>(exa, exa, eza)) deposit2_reg<float, NVP>(acc, exa, eza, cx, cy, cz);
            else deposit2_smem<float, NDIM>(sj, lx + exa.a + 1, lz + eza.a + 1, exa, eza, cx, cy, cz);
          }
          if (vb) {
            const float qw = qs * wb;
            const float cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vyb * r.jfy2d;
            if (reg_window<float, 2>(exb, exb, ezb)) deposit2_reg<float, NVP>(acc, exb, ezb, cx, cy, cz);
            else deposit2_smem<float, NDIM>(sj, lx + exb.a + 1, lz + ezb.a + 1, exb, ezb, cx, cy, cz);
          }
          // destinations: a cell of this tile (key (cell * 2 + species) in the tile) or, leaving
          // the tile, the global cell (key global cell * 2 + species)
          int dka = -1 - lane, dkb = -1 - lane;
          bool lva = false, lvb = false;
          if (va) {
            const int nlx = lx + exa.shift, nlz = lz + eza.shift;
            if (nlx >= 0 && nlx < wx && nlz >= 0 && nlz < wz) {
              dka = (nlz * TX + nlx) * 2 + s;
            } else {
              lva = true;
              dka = (wrap_near_p(gk + eza.shift, r.nz) * r.nx + wrap_near_p(gi + exa.shift, r.nx)) * 2 + s;
            }
          }
          if (vb) {
            const int nlx = lx + exb.shift, nlz = lz + ezb.shift;
            if (nlx >= 0 && nlx < wx && nlz >= 0 && nlz < wz) {
              dkb = (nlz * TX + nlx) * 2 + s;
            } else {
              lvb = true;
              dkb = (wrap_near_p(gk + ezb.shift, r.nz) * r.nx + wrap_near_p(gi + exb.shift, r.nx)) * 2 + s;
            }
          }
          // rebin of the pair: consecutive slots per (destination, species) for each particle of the
          // pair, the two reservations interleaved
          const bool sta = va && !lva, stb = vb && !lvb;
          const unsigned pa = __match_any_sync(0xffffffffu, sta ? dka : -1 - lane);
          const unsigned pb = __match_any_sync(0xffffffffu, stb ? dkb : -1 - lane);
          const int lda = __ffs(pa) - 1, ldb = __ffs(pb) - 1;
          int ba = 0, bb = 0;
          if (sta && lane == lda) ba = atomicAdd(scnt + (dka & 1) * NCL + (dka >> 1), __popc(pa));
          if (stb && lane == ldb) bb = atomicAdd(scnt + (dkb & 1) * NCL + (dkb >> 1), __popc(pb));
          ba = __shfl_sync(0xffffffffu, ba, lda) + __popc(pa & lt);
          bb = __shfl_sync(0xffffffffu, bb, ldb) + __popc(pb & lt);
          const bool fa = sta && ba >= r.cap, fb = stb && bb >= r.cap;  // full bins: on to k_migrate
          // leavers: the tile's shared buffer (one reservation for the pair), then the global list
          // for full bins and once the shared buffer is full
          const unsigned lma = __ballot_sync(0xffffffffu, lva), lmb = __ballot_sync(0xffffffffu, lvb);
          int lsa = 0, lsb = 0;
          if (lma | lmb) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(lvn, __popc(lma) + __popc(lmb));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            lsa = b0 + __popc(lma & lt);
            lsb = b0 + __popc(lma) + __popc(lmb & lt);
          }
          const bool ga = fa || (lva && lsa >= S::LVB), gb = fb || (lvb && lsb >= S::LVB);
          const unsigned gma = __ballot_sync(0xffffffffu, ga), gmb = __ballot_sync(0xffffffffu, gb);
          long long goa = 0, gob = 0;
          if (gma | gmb) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(r.lv_count, __popc(gma) + __popc(gmb));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            goa = (long long)b0 + __popc(gma & lt);
            gob = (long long)b0 + __popc(gma) + __popc(gmb & lt);
          }
          const int gcell = gk * r.nx + gi;  // cells < 2^30
          auto place = [&](bool st, bool full, bool lv, bool g, int dk, int jo, int ls, long long go, float nox,
                           float noz, float ux, float uy, float uz, float w, unsigned id, int shx, int shz) {
            const int dcell = gcell + shz * r.nx + shx;  // a cell of this tile when st
            if (st && !full) {
              const long long o = (long long)dcell * r.cap + jo;
              pout.ox[o] = nox;
              pout.oz[o] = noz;
              pout.dux[o] = ux;
              pout.duy[o] = uy;
              pout.duz[o] = uz;
              if (has_w) pout.w[o] = w;
              if (has_id) pout.id[o] = id;
            } else if (g) {
              if (go < r.lv_cap) list_put(r.lv, go, full ? dcell * 2 + (dk & 1) : dk, nox, 0.f, noz, ux, uy, uz, w, id);
              else flag_error(r.err, ERR_OVERFLOW);
            } else if (lv) {
              lvk[ls] = dk;
              lvv[ls] = nox;
              lvv[2 * S::LVB + ls] = noz;
              lvv[3 * S::LVB + ls] = ux;
              lvv[4 * S::LVB + ls] = uy;
              lvv[5 * S::LVB + ls] = uz;
              if (has_w) lvv[6 * S::LVB + ls] = w;
              if (has_id) lvi[ls] = id;
            }
          };
          if (va)
            place(sta, fa, lva, ga, dka, ba, lsa, goa, exa.off, eza.off, nuxa, nuya, nuza, wa, has_id ? st_id[ja] : 0u,
                  exa.shift, eza.shift);
          if (vb)
            place(stb, fb, lvb, gb, dkb, bb, lsb, gob, exb.off, ezb.off, nuxb, nuyb, nuzb, wb, has_id ? st_id[jb] : 0u,
                  exb.shift, ezb.shift);
        }
      } else {
#pragma unroll 1
      for (int rnd = 0; rnd < 4; ++rnd) {
        // pack element of this round, rotated by lane / 8 so the 32 lanes' shared-memory reads of
        // one array fall in distinct banks
        const int jj = (rnd + (lane >> 3)) & 3;
        const bool valid = jj < cnt;
        int dkey = -1 - lane;  // unique per lane when there is no particle
        bool leave = false;
        T nox = T(0), noy = T(0), noz = T(0), ux = T(0), uy = T(0), uz = T(0);
        const T w = (has_w && valid) ? st_x[SG::slot(6) * 128 + jj] : r.wconst;
        if (valid) {
          const T o_x = st_x[jj], o_y = NDIM == 3 ? st_x[SG::slot(1) * 128 + jj] : T(0), o_z = st_x[SG::slot(2) * 128 + jj];
          ux = st_x[SG::slot(3) * 128 + jj];
          uy = st_x[SG::slot(4) * 128 + jj];
          uz = st_x[SG::slot(5) * 128 + jj];
          // gather
          T F[6];
          if (SCHEME == 0) {
            gc.interp(o_x, o_y, o_z, F);
          } else {
            const DirW<T> dwx = dir_weights(o_x), dwy = dir_weights(o_y), dwz = dir_weights(o_z);
#pragma unroll
            for (int c = 0; c < 6; ++c)
              F[c] = gather_comp<T, NDIM, SCHEME>(sg + c * S::GN, c, lx, ly, lz, dwx, dwy, dwz);
          }
          // relativistic Boris, momenta relative to the drift u0 z_hat
          const T h = qs * r.hq;
          const T mx = ux + h * F[0], my = uy + h * F[1], mz = uz + h * F[2];
          const T Mz = r.u0 + mz;
          const T ig = fast_rsqrt(T(1) + mx * mx + my * my + Mz * Mz);
          const T tx = h * F[3] * ig, ty = h * F[4] * ig, tz = h * F[5] * ig;
          const T sf = fast_div(T(2), T(1) + tx * tx + ty * ty + tz * tz);
          const T sx = sf * tx, sy = sf * ty, sz = sf * tz;
          const T qx = mx + (my * tz - Mz * ty);
          const T qy = my + (Mz * tx - mx * tz);
          const T qz = Mz + (mx * ty - my * tx);
          ux = mx + (qy * sz - qz * sy) + h * F[0];
          uy = my + (qz * sx - qx * sz) + h * F[1];
          uz = mz + (qx * sy - qy * sx) + h * F[2];
          const T Uz = r.u0 + uz;
          const T u2 = ux * ux + uy * uy + Uz * Uz;
          const T ign = fast_rsqrt(T(1) + u2);
          T vx = ux * ign, vy = uy * ign;
          const T vz = Uz * ign;
          kin += w * fast_div(u2, (T(1) + u2) * ign + T(1));  // gamma - 1 = u^2 / (gamma + 1)
          ++npush;
          // move (cell-relative displacement in grid units)
          T ddx = r.dtdx * vx, ddy = NDIM == 3 ? r.dtdy * vy : T(0), ddz = r.dtdz * vz;
          if (!(abs_lt_one(ddx) && abs_lt_one(ddy) && abs_lt_one(ddz))) {
            flag_error(r.err, ERR_NONFINITE);
            ddx = ddy = ddz = T(0);
            ux = uy = uz = T(0);
            vy = T(0);
          }
          const EsirDir<T> ex_ = esir_dir(o_x, ddx);
          const EsirDir<T> ez_ = esir_dir(o_z, ddz);
          EsirDir<T> ey_;
          if (NDIM == 3) ey_ = esir_dir(o_y, ddy);
          else { ey_.a = 0; ey_.shift = 0; ey_.off = T(0); }
          // Esirkepov deposit: summed in registers when the window fits RegLayout (no step back across
          // a face and no transverse crossing), else straight to shared memory
          const T qw = qs * w;
          const bool own = reg_window<T, NDIM>(ex_, NDIM == 3 ? ey_ : ex_, ez_);
          if (NDIM == 2) {
            const T cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vy * r.jfy2d;
            if (own) deposit2_reg<T, NVP>(acc, ex_, ez_, cx, cy, cz);
            else deposit2_smem<T, NDIM>(sj, lx + ex_.a + 1, lz + ez_.a + 1, ex_, ez_, cx, cy, cz);
          } else {
            const T cx = qw * r.jfx, cy = qw * r.jfy, cz = qw * r.jfz;
            if (own) deposit3_reg<T, NVP>(acc, ex_, ey_, ez_, cx, cy, cz);
            else deposit3_smem<T, NDIM>(sj, lx + ex_.a + 1, ly + ey_.a + 1, lz + ez_.a + 1, ex_, ey_, ez_, cx, cy, cz);
          }
          // new cell and offsets
          nox = ex_.off;
          noy = NDIM == 3 ? ey_.off : T(0);
          noz = ez_.off;
          const int nlx = lx + ex_.shift, nly = NDIM == 3 ? ly + ey_.shift : 0, nlz = lz + ez_.shift;
          if (nlx >= 0 && nlx < wx && nly >= 0 && nly < wy && nlz >= 0 && nlz < wz) {
            dkey = ((nlz * TY + nly) * TX + nlx) * 2 + s;  // stays in this tile
          } else {
            leave = true;  // global destination, as cell * 2 + species
            // one cell across a face: the index stays within [-1, n] (cells < 2^30: int keys)
            const int ni = wrap_near_p(gi + ex_.shift, r.nx);
            const int nj = NDIM == 3 ? wrap_near_p(gj + ey_.shift, r.ny) : 0;
            const int nk = wrap_near_p(gk + ez_.shift, r.nz);
            dkey = ((nk * r.ny + nj) * r.nx + ni) * 2 + s;
          }
        }
        // rebin. Destination in this tile: lanes with the same (cell, species) reserve consecutive
        // slots with one shared-memory atomic on the tile's output counts. Destination in another
        // tile: the particle is appended to the leaver list (one global atomic per warp), which
        // k_migrate inserts after this kernel.
        const bool stay = valid && !leave;
        const unsigned peers = __match_any_sync(0xffffffffu, stay ? dkey : -1 - lane);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int base = 0;
        if (stay && lane == leader) base = atomicAdd(scnt + (dkey & 1) * NCL + (dkey >> 1), __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        // a full destination bin: the particle goes through the global leaver list instead, and
        // k_migrate spills it when the bin is still full there (nothing is dropped)
        const bool full = stay && base + rank >= r.cap;
        const unsigned fmask = __ballot_sync(0xffffffffu, full);
        long long fglob = 0;
        if (fmask) {
          const int fl = __ffs(fmask) - 1;
          int fb = 0;
          if (lane == fl) fb = atomicAdd(r.lv_count, __popc(fmask));
          fb = __shfl_sync(0xffffffffu, fb, fl);
          fglob = (long long)fb + __popc(fmask & ((1u << lane) - 1u));
        }
        // leavers: a slot in the tile's shared-memory buffer (one shared atomic per warp), or, once
        // the buffer is full, straight in the global list
        const unsigned lmask = __ballot_sync(0xffffffffu, valid && leave);
        int lslot = 0;
        long long lglob = 0;
        if (lmask) {
          const int lleader = __ffs(lmask) - 1;
          int b = 0;
          if (lane == lleader) b = atomicAdd(lvn, __popc(lmask));
          b = __shfl_sync(0xffffffffu, b, lleader);
          lslot = b + __popc(lmask & ((1u << lane) - 1u));
          const unsigned gmask = __ballot_sync(0xffffffffu, valid && leave && lslot >= S::LVB);
          if (gmask) {
            const int gl = __ffs(gmask) - 1;
            int gb = 0;
            if (lane == gl) gb = atomicAdd(r.lv_count, __popc(gmask));
            gb = __shfl_sync(0xffffffffu, gb, gl);
            lglob = (long long)gb + __popc(gmask & ((1u << lane) - 1u));
          }
        }
        if (stay) {
          const int j = base + rank;
          const int dl = dkey >> 1;
          const int dx = dl % TX, dy = (dl / TX) % TY, dz = dl / (TX * TY);
          const int dcell = ((Z0 + dz) * r.ny + Y0 + dy) * r.nx + X0 + dx;  // cells < 2^30
          if (!full) {
            const long long o = (long long)dcell * r.cap + j;
            pout.ox[o] = nox;
            if (NDIM == 3) pout.oy[o] = noy;
            pout.oz[o] = noz;
            pout.dux[o] = ux;
            pout.duy[o] = uy;
            pout.duz[o] = uz;
            if (has_w) pout.w[o] = w;
            if (has_id) pout.id[o] = st_id[jj];
          } else if (fglob < r.lv_cap) {
            list_put(r.lv, fglob, dcell * 2 + (dkey & 1), nox, noy, noz, ux, uy, uz, w, has_id ? st_id[jj] : 0u);
          } else {
            flag_error(r.err, ERR_OVERFLOW);
          }
        } else if (valid && lslot < S::LVB) {
          lvk[lslot] = dkey;
          lvv[lslot] = nox;
          if (NDIM == 3) lvv[S::LVB + lslot] = noy;
          lvv[2 * S::LVB + lslot] = noz;
          lvv[3 * S::LVB + lslot] = ux;
          lvv[4 * S::LVB + lslot] = uy;
          lvv[5 * S::LVB + lslot] = uz;
          if (has_w) lvv[6 * S::LVB + lslot] = w;
          if (has_id) lvi[lslot] = st_id[jj];
        } else if (valid) {
          const long long o = lglob;
          if (o < r.lv_cap) {
            r.lv.key[o] = dkey;
            r.lv.ox[o] = nox;
            if (NDIM == 3) r.lv.oy[o] = noy;
            r.lv.oz[o] = noz;
            r.lv.dux[o] = ux;
            r.lv.duy[o] = uy;
            r.lv.duz[o] = uz;
            if (has_w) r.lv.w[o] = w;
            if (has_id) r.lv.id[o] = st_id[jj];
          } else {
            flag_error(r.err, ERR_OVERFLOW);
          }
        }
      }
      }
    }
    if (it == giters - 1) {
      // 3. segmented transpose-reduction of the cell's register sums over its LPC lanes
#pragma unroll
      for (int sh = LPC / 2; sh >= 1; sh >>= 1) {
        const bool up = (lane & sh) != 0;
#pragma unroll
        for (int j = 0; j < PER * sh; ++j) {
          const T send = up ? acc[j] : acc[j + PER * sh];
          const T keep = up ? acc[j + PER * sh] : acc[j];
          acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
        }
      }
#pragma unroll
      for (int m = 0; m < PER; ++m) {
        const int i = sl * PER + m;
        if (i < NV && acc[m] != T(0)) {
          int comp, a, b, c;
          RegLayout<NDIM>::at(i, comp, a, b, c);
          atomicAdd(sj + comp * S::JN + okey + (c * S::JY + b) * S::JX + a, acc[m]);
        }
      }
    }
    __syncwarp();  // the stage just read is refilled by the next iteration's prefetch
    g = ng;
    it = nit;
    giters = niters;
    stage ^= 1;
  }
  cp_async_wait_all();
  __syncthreads();

  // 4. the tile's buffered leavers: one reservation in the global list, then a coalesced copy
  __shared__ int lv_base;
  const int nlv = min(*lvn, S::LVB);
  if (tid == 0) lv_base = nlv > 0 ? atomicAdd(r.lv_count, nlv) : 0;
  __syncthreads();
  for (int e = tid; e < nlv; e += PUSH_THREADS) {
    const long long o = (long long)lv_base + e;
    if (o < r.lv_cap) {
      r.lv.key[o] = lvk[e];
      r.lv.ox[o] = lvv[e];
      if (NDIM == 3) r.lv.oy[o] = lvv[S::LVB + e];
      r.lv.oz[o] = lvv[2 * S::LVB + e];
      r.lv.dux[o] = lvv[3 * S::LVB + e];
      r.lv.duy[o] = lvv[4 * S::LVB + e];
      r.lv.duz[o] = lvv[5 * S::LVB + e];
      if (has_w) r.lv.w[o] = lvv[6 * S::LVB + e];
      if (has_id) r.lv.id[o] = lvi[e];
    } else {
      flag_error(r.err, ERR_OVERFLOW);
    }
  }

  // 5. output counts of the tile's cells (leavers from other tiles are added by k_migrate); a count
  // past the capacity (particles sent on through the leaver list) is stored as the capacity
  for (int cl = tid; cl < NCL; cl += PUSH_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    if (lx < wx && ly < wy && lz < wz) {
      const long long cell = (long long)(Z0 + lz) * nxy + (long long)(Y0 + ly) * r.nx + X0 + lx;
      r.out[0].cnt[cell] = min(scnt[cl], r.cap);
      r.out[1].cnt[cell] = min(scnt[NCL + cl], r.cap);
    }
  }

  // 6. flush the tile's current to global memory
  for (int e = tid; e < 3 * S::JN; e += PUSH_THREADS) {
    T v = sj[e];
    if (v == T(0)) continue;
    int c = e / S::JN, rem = e - c * S::JN;
    int lz = rem / (S::JX * S::JY);
    int ly = (rem / S::JX) % S::JY;
    int lx = rem % S::JX;
    int gx = near_ok ? wrap_near_p(X0 - 1 + lx, r.nx) : wrapi(X0 - 1 + lx, r.nx);
    int gy = NDIM == 3 ? (near_ok ? wrap_near_p(Y0 - 1 + ly, r.ny) : wrapi(Y0 - 1 + ly, r.ny)) : 0;
    int gz = near_ok ? wrap_near_p(Z0 - 1 + lz, r.nz) : wrapi(Z0 - 1 + lz, r.nz);
    atomicAdd(r.j[c] + (long long)gz * nxy + (long long)gy * r.nx + gx, v);
  }

  // 7. kinetic energy and particle count of this step: per-thread partial sums in the working
  // precision, FP64 across the block and the grid
  if (r.kin) {
    double kd = (double)kin;
    int nd = npush;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kd += __shfl_xor_sync(0xffffffffu, kd, o);
      nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    __shared__ double skin[NWARP];
    __shared__ int swcnt[NWARP];
    if (lane == 0) {
      skin[warp] = kd;
      swcnt[warp] = nd;
    }
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      long long c = 0;
      for (int w2 = 0; w2 < NWARP; ++w2) {
        t += skin[w2];
        c += swcnt[w2];
      }
      atomicAdd(r.kin, t);
      atomicAdd(r.kin + 1, (double)c);
    }
  }
}

// One tile per block.
template <typename T, int NDIM, int SCHEME, int LPC>
__global__ void __launch_bounds__(PushThreads<T, NDIM>::value, PushMinBlocks<T, NDIM>::value)
    k_push(const __grid_constant__ RunDev<T> r) {
  pdl_wait();
  push_tile<T, NDIM, SCHEME, LPC>(r, blockIdx.x);
}

// Persistent form for many runs: each block takes (run, tile) work items from a global counter
// (items grouped by run, so a block mostly stays on one run) and copies the run's descriptor into
// shared memory when the run changes. Work-list counter reset: the caller zeroes *queue before the
// launch.
template <typename T, int NDIM, int SCHEME, int LPC>
__global__ void __launch_bounds__(PushThreads<T, NDIM>::value, PushMinBlocks<T, NDIM>::value)
    k_push_batch(const RunDev<T>* __restrict__ runs, const int2* __restrict__ items, int nitems, int* queue) {
  pdl_wait();
  __shared__ RunDev<T> rs;
  __shared__ int cur, cur_run;
  if (threadIdx.x == 0) cur_run = -1;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) cur = atomicAdd(queue, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) break;
    const int2 w = items[it];
    if (w.x != cur_run) {  // warp 0 copies the descriptor as 32-bit words
      __syncthreads();
      constexpr int NW = (int)(sizeof(RunDev<T>) / 4);
      const int* src = reinterpret_cast<const int*>(runs + w.x);
      int* dst = reinterpret_cast<int*>(&rs);
      for (int k = threadIdx.x; k < NW; k += PushThreads<T, NDIM>::value) dst[k] = src[k];
      __syncthreads();
      if (threadIdx.x == 0) cur_run = w.x;
    }
    __syncthreads();
    push_tile<T, NDIM, SCHEME, LPC>(rs, w.y);
  }
}

// Lanes per cell from the expected particles per cell (both species): packs of 4 per lane.
static int lanes_per_cell(int ndim, int ppc_total) {
  const int packs = 2 * ((ppc_total / 2 + 3) / 4);  // packs of 4 per species
  // 2D: four lanes per cell up to 8 packs (two packs per lane halve the per-cell reduction cost;
  // measured 3 % faster than eight lanes at 16 particles/cell/species on GB300)
  // 3D up to 4 packs: two lanes per cell (a lane's two packs halve the per-cell reduction and
  // Galerkin loads per particle; measured 5 % faster than four lanes at 8 particles/cell/species)
  if (ndim == 3 && packs <= 4) return 2;
  if (packs <= 4 || (ndim == 2 && packs <= 8)) return 4;
  if (packs <= 8) return 8;
  return 16;
}

template <typename T, int NDIM, int SCHEME>
static cudaError_t launch_push_t(const RunDev<T>& r, int lpc, cudaStream_t st) {
  using S = PushSmem<T, NDIM>;
  const size_t sm = S::bytes();
  const int ntiles = r.ntx * r.nty * r.ntz;
  auto go = [&](void (*kern)(const RunDev<T>)) -> cudaError_t {
    cudaError_t e = ensure_dynamic_smem((const void*)kern, sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, dim3(ntiles), dim3(PushThreads<T, NDIM>::value), sm, st, r);
  };
  if constexpr (NDIM == 3) {
    if (lpc == 2) return go(k_push<T, NDIM, SCHEME, 2>);
  }
  if (lpc == 4) return go(k_push<T, NDIM, SCHEME, 4>);
  if (lpc == 8) return go(k_push<T, NDIM, SCHEME, 8>);
  return go(k_push<T, NDIM, SCHEME, 16>);
}

template <typename T>
cudaError_t launch_push(const RunDev<T>& r, int ppc_total, cudaStream_t st) {
  if (!tiles_fit<PTile>(r)) return cudaErrorInvalidValue;
  const int lpc = lanes_per_cell(r.ndim, ppc_total);
  if (r.ndim == 2)
    return r.scheme == 0 ? launch_push_t<T, 2, 0>(r, lpc, st) : launch_push_t<T, 2, 1>(r, lpc, st);
  return r.scheme == 0 ? launch_push_t<T, 3, 0>(r, lpc, st) : launch_push_t<T, 3, 1>(r, lpc, st);
}
template cudaError_t launch_push<float>(const RunDev<float>&, int, cudaStream_t);

template <typename T, int NDIM, int SCHEME>
static cudaError_t launch_push_batch_t(const RunDev<T>* runs, const int2* items, int nitems, int* queue, int lpc,
                                       int blocks, cudaStream_t st) {
  using S = PushSmem<T, NDIM>;
  const size_t sm = S::bytes();
  auto go = [&](void (*kern)(const RunDev<T>*, const int2*, int, int*)) -> cudaError_t {
    cudaError_t e = ensure_dynamic_smem((const void*)kern, sm);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, dim3(blocks), dim3(PushThreads<T, NDIM>::value), sm, st, runs, items, nitems, queue);
  };
  if (lpc == 4) return go(k_push_batch<T, NDIM, SCHEME, 4>);
  if (lpc == 8) return go(k_push_batch<T, NDIM, SCHEME, 8>);
  return go(k_push_batch<T, NDIM, SCHEME, 16>);
}

template <typename T>
cudaError_t launch_push_batch(const RunDev<T>* runs, const int2* items, int nitems, int* queue, int ndim, int scheme,
                              int lpc, int blocks, cudaStream_t st) {
  if (ndim == 2)
    return scheme == 0 ? launch_push_batch_t<T, 2, 0>(runs, items, nitems, queue, lpc, blocks, st)
                       : launch_push_batch_t<T, 2, 1>(runs, items, nitems, queue, lpc, blocks, st);
  return scheme == 0 ? launch_push_batch_t<T, 3, 0>(runs, items, nitems, queue, lpc, blocks, st)
                     : launch_push_batch_t<T, 3, 1>(runs, items, nitems, queue, lpc, blocks, st);
}
template cudaError_t launch_push_batch<float>(const RunDev<float>*, const int2*, int, int*, int, int, int, int,
                                              cudaStream_t);
template cudaError_t launch_push_batch<double>(const RunDev<double>*, const int2*, int, int*, int, int, int, int,
                                               cudaStream_t);

// The batched kernel is built for 4, 8 and 16 lanes per cell.
int push_lanes_per_cell(int ndim, int ppc_total) {
  const int l = lanes_per_cell(ndim, ppc_total);
  return l < 4 ? 4 : l;
}

template <typename T>
int push_max_blocks_per_sm(int ndim, int scheme, int lpc) {
  int n = 0;
  size_t sm = ndim == 2 ? PushSmem<T, 2>::bytes() : PushSmem<T, 3>::bytes();
  const void* k = nullptr;
  if (ndim == 2)
    k = scheme == 0 ? (lpc == 4 ? (const void*)k_push_batch<T, 2, 0, 4> : lpc == 8 ? (const void*)k_push_batch<T, 2, 0, 8> : (const void*)k_push_batch<T, 2, 0, 16>)
                    : (lpc == 4 ? (const void*)k_push_batch<T, 2, 1, 4> : lpc == 8 ? (const void*)k_push_batch<T, 2, 1, 8> : (const void*)k_push_batch<T, 2, 1, 16>);
  else
    k = scheme == 0 ? (lpc == 4 ? (const void*)k_push_batch<T, 3, 0, 4> : lpc == 8 ? (const void*)k_push_batch<T, 3, 0, 8> : (const void*)k_push_batch<T, 3, 0, 16>)
                    : (lpc == 4 ? (const void*)k_push_batch<T, 3, 1, 4> : lpc == 8 ? (const void*)k_push_batch<T, 3, 1, 8> : (const void*)k_push_batch<T, 3, 1, 16>);
  if (ensure_dynamic_smem(k, sm) != cudaSuccess) return 1;
  const int nt = ndim == 2 ? PushThreads<T, 2>::value : PushThreads<T, 3>::value;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, nt, sm) != cudaSuccess || n < 1) return 1;
  return n;
}
template int push_max_blocks_per_sm<float>(int, int, int);
template int push_max_blocks_per_sm<double>(int, int, int);
template cudaError_t launch_push<double>(const RunDev<double>&, int, cudaStream_t);

// The compile-time tile TL of the working precision T.
template <template <typename, int> class TL, typename T>
static void tile_of(int ndim, int te[3]) {
  if (ndim == 2) {
    te[0] = TL<T, 2>::TX;
    te[1] = 1;
    te[2] = TL<T, 2>::TZ;
  } else {
    te[0] = TL<T, 3>::TX;
    te[1] = TL<T, 3>::TY;
    te[2] = TL<T, 3>::TZ;
  }
}

void push_tiles(int ndim, int es, bool ho, int nx, int ny, int nz, int spread, int nt[3], int te[3]) {
  const int n[3] = {nx, ndim == 3 ? ny : 1, nz};
  if (es == 4) ho ? tile_of<HoTile, float>(ndim, te) : tile_of<PTile, float>(ndim, te);
  else ho ? tile_of<HoTile, double>(ndim, te) : tile_of<PTile, double>(ndim, te);
  auto count = [&]() {
    long long t = 1;
    for (int d = 0; d < 3; ++d) {
      nt[d] = (n[d] + te[d] - 1) / te[d];
      t *= nt[d];
    }
    return t;
  };
  long long tiles = count();
  while (spread > 0 && 2 * tiles <= spread) {
    int d = -1;  // the longest extent above 4 that still splits the grid further
    for (int k = 0; k < 3; ++k)
      if (te[k] > 4 && n[k] > te[k] / 2 && (d < 0 || te[k] > te[d])) d = k;
    if (d < 0) break;
    te[d] /= 2;
    tiles = count();
  }
}

// ---------------------------------------------------------------------------------------------
// Migrate: insert the particles that left their tile in this step (leaver list of the push
// kernel) into their destination bins, then zero the other parity's list counter for the next
// step's push.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void migrate_body(const RunDev<T>& r, int* other_count, int bid, int nblk) {
  const long long n = min((long long)*r.lv_count, r.lv_cap);
  const int lane = threadIdx.x & 31;
  // whole warps iterate together (leavers of one source cell are consecutive and mostly share their
  // destination, so one atomic per destination group reserves their slots)
  const long long stride = (long long)nblk * blockDim.x;
  for (long long base = bid * (long long)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const long long i = base + lane;
    const bool valid = i < n;
    int key = -1 - lane;
    T ox = T(0), oy = T(0), oz = T(0), ux = T(0), uy = T(0), uz = T(0), w = T(0);
    unsigned id = 0;
    if (valid) {
      key = r.lv.key[i];
      ox = r.lv.ox[i];
      if (r.ndim == 3) oy = r.lv.oy[i];
      oz = r.lv.oz[i];
      ux = r.lv.dux[i];
      uy = r.lv.duy[i];
      uz = r.lv.duz[i];
      if (r.lv.w) w = r.lv.w[i];
      if (r.lv.id) id = r.lv.id[i];
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int s = key & 1;
    const long long cell = key >> 1;
    const SpeciesBuf<T> b = s ? r.out[1] : r.out[0];
    int j0 = 0;
    if (valid && lane == leader) j0 = atomicAdd(b.cnt + cell, __popc(peers));
    j0 = __shfl_sync(0xffffffffu, j0, leader);
    // a full bin: the particle goes to the spill list, which the next step pushes from (the count
    // keeps the excess, so the host sees how large the bin has to grow)
    const bool full = valid && j0 + rank >= r.cap;
    const unsigned fmask = __ballot_sync(0xffffffffu, full);
    long long so = 0;
    if (fmask) {
      const int fl = __ffs(fmask) - 1;
      int sb = 0;
      if (lane == fl) {
        sb = atomicAdd(r.sp_out, __popc(fmask));
        atomicAdd(r.sp_total, (unsigned long long)__popc(fmask));
      }
      sb = __shfl_sync(0xffffffffu, sb, fl);
      so = (long long)sb + __popc(fmask & ((1u << lane) - 1u));
    }
    if (!valid) continue;
    if (full) {
      if (so < r.sp_cap) list_put(r.sp, so, key, ox, oy, oz, ux, uy, uz, w, id);
      else flag_error(r.err, ERR_OVERFLOW);
      continue;
    }
    const int j = j0 + rank;
    const long long o = cell * r.cap + j;
    b.ox[o] = ox;
    if (r.ndim == 3) b.oy[o] = oy;
    b.oz[o] = oz;
    b.dux[o] = ux;
    b.duy[o] = uy;
    b.duz[o] = uz;
    if (b.w) b.w[o] = w;
    if (b.id) b.id[o] = id;
  }
  if (bid == 0 && threadIdx.x == 0) *other_count = 0;
}

template <typename T>
__global__ void k_migrate(const __grid_constant__ RunDev<T> r, int* other_count) {
  pdl_wait();
  migrate_body<T>(r, other_count, blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void k_migrate_batch(const RunDev<T>* __restrict__ runs) {
  pdl_wait();
  const RunDev<T>& r = runs[blockIdx.y];
  migrate_body<T>(r, r.lv_other, blockIdx.x, gridDim.x);
}

template <typename T>
cudaError_t launch_migrate(const RunDev<T>& r, int* other_count, cudaStream_t st) {
  return launch_pdl(k_migrate<T>, dim3(152 * 4), dim3(256), 0, st, r, other_count);
}

template <typename T>
cudaError_t launch_migrate_batch(const RunDev<T>* runs, int nruns, cudaStream_t st) {
  dim3 grid(4 * 152 / (nruns < 4 ? 1 : nruns / 4) + 1, (unsigned)nruns);
  return launch_pdl(k_migrate_batch<T>, grid, dim3(256), 0, st, runs);
}
template cudaError_t launch_migrate_batch<float>(const RunDev<float>*, int, cudaStream_t);
template cudaError_t launch_migrate_batch<double>(const RunDev<double>*, int, cudaStream_t);
template cudaError_t launch_migrate<float>(const RunDev<float>&, int*, cudaStream_t);
template cudaError_t launch_migrate<double>(const RunDev<double>&, int*, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Insert one particle of species s into its cell bin of the input buffers (used by init and
// import); a full bin puts it in the spill list that the next step pushes from.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void insert_particle(const RunDev<T>& r, int s, long long cell, T ox, T oy, T oz, T ux,
                                                T uy, T uz, T w, unsigned id) {
  const SpeciesBuf<T>& b = s ? r.in[1] : r.in[0];
  const int cap = r.cap;
  int j = atomicAdd(b.cnt + cell, 1);
  if (j >= cap) {
    const long long o = atomicAdd(r.sp_in, 1);
    atomicAdd(r.sp_total, 1ull);
    if (o < r.sp_cap) list_put(r.sp, o, (int)(cell * 2 + s), ox, oy, oz, ux, uy, uz, w, id);
    else flag_error(r.err, ERR_OVERFLOW);
    return;
  }
  long long o = cell * cap + j;
  b.ox[o] = ox;
  if (b.oy) b.oy[o] = oy;
  b.oz[o] = oz;
  b.dux[o] = ux;
  b.duy[o] = uy;
  b.duz[o] = uz;
  if (b.w) b.w[o] = w;
  if (b.id) b.id[o] = id;
}

// Fold a position (cell index per direction + offset, offset possibly outside [0,1)) into range.
template <typename T>
__device__ __forceinline__ void fold(int& i, T& o, int n) {
  T f = dev_floor(o);
  i += (int)f;
  o -= f;
  if (o >= T(1)) { o = T(0); i += 1; }
  if (o < T(0)) o = T(0);
  i = wrapi(i, n);
}

// ---------------------------------------------------------------------------------------------
// Seeded beam: one thread per lattice point p (cell-major, ppc points per cell on an lx x ly x lz
// lattice at offsets (l + 1/2) / n). Philox4x32-10 keyed by the seed with counter (p, 0, 0, 0) gives
// the position jitter, uniform in +-jitter cells per coordinate; counter (p, 1 + s, 0, 0) gives
// species s's two Box-Muller pairs for the thermal momenta (spread u_th per component, relative to
// the drift). The electron and the positron of a point share its position, and with transverse
// Gaussian weights w = w0 exp(-r_perp^2 / (2 sigma^2)) about the box axis. All random numbers and
// the derived positions and momenta are computed in FP64 and rounded once.
// ---------------------------------------------------------------------------------------------
struct BeamDev {
  int ppc, lx, ly, lz;
  double u0, w0, jitter, u_th, sigma_perp;
  uint32_t k0, k1;
};

__device__ __forceinline__ double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

template <typename T>
__global__ void k_init_beam(const __grid_constant__ RunDev<T> r, BeamDev b, long long npoints) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= npoints) return;
  const long long nxy = (long long)r.nx * r.ny;
  long long cell = p / b.ppc;
  int l = (int)(p - cell * b.ppc);
  int i = (int)(cell % r.nx), j = (int)((cell / r.nx) % r.ny), k = (int)(cell / nxy);
  int lx = l % b.lx, ly = (l / b.lx) % b.ly, lz = l / (b.lx * b.ly);
  u32x4 c = {{(uint32_t)((unsigned long long)p & 0xffffffffu), (uint32_t)((unsigned long long)p >> 32), 0u, 0u}};
  u32x4 rr = philox10(c, b.k0, b.k1);
  double ox = (lx + 0.5) / b.lx + b.jitter * (2.0 * u01(rr.v[0]) - 1.0);
  double oy = r.ndim == 3 ? (ly + 0.5) / b.ly + b.jitter * (2.0 * u01(rr.v[1]) - 1.0) : 0.0;
  double oz = (lz + 0.5) / b.lz + b.jitter * (2.0 * u01(rr.v[2]) - 1.0);
  double w = b.w0;
  if (b.sigma_perp > 0) {
    double X = i + ox, Y = r.ndim == 3 ? j + oy : 0.0;
    X = X - r.nx * floor(X / r.nx);
    if (r.ndim == 3) Y = Y - r.ny * floor(Y / r.ny);
    double rx = X - 0.5 * r.nx, ry = r.ndim == 3 ? Y - 0.5 * r.ny : 0.0;
    w = b.w0 * exp(-(rx * rx + ry * ry) / (2.0 * b.sigma_perp * b.sigma_perp));
  }
  // fold in FP64, then round the offsets
  double fxd = floor(ox), fyd = floor(oy), fzd = floor(oz);
  int ci = wrapi(i + (int)fxd, r.nx), cj = r.ndim == 3 ? wrapi(j + (int)fyd, r.ny) : 0, ck = wrapi(k + (int)fzd, r.nz);
  T tox = (T)(ox - fxd), toy = (T)(oy - fyd), toz = (T)(oz - fzd);
  if (tox >= T(1)) { tox = T(0); ci = wrapi(ci + 1, r.nx); }
  if (r.ndim == 3 && toy >= T(1)) { toy = T(0); cj = wrapi(cj + 1, r.ny); }
  if (toz >= T(1)) { toz = T(0); ck = wrapi(ck + 1, r.nz); }
  long long dcell = (long long)ck * nxy + (long long)cj * r.nx + ci;
  const double two_pi = 6.283185307179586476925286766559;
  for (int s = 0; s < 2; ++s) {
    c.v[2] = (uint32_t)(1 + s);
    u32x4 t = philox10(c, b.k0, b.k1);
    double ra = sqrt(-2.0 * log(u01(t.v[0]))), ta = two_pi * u01(t.v[1]);
    double rb = sqrt(-2.0 * log(u01(t.v[2]))), tb = two_pi * u01(t.v[3]);
    T ux = (T)(b.u_th * ra * cos(ta));
    T uy = (T)(b.u_th * ra * sin(ta));
    T uz = (T)(b.u_th * rb * cos(tb));
    insert_particle(r, s, dcell, tox, toy, toz, ux, uy, uz, (T)w, (unsigned)(p * 2 + s));
  }
}

template <typename T>
cudaError_t launch_init_beam(const RunDev<T>& r, int ppc, const int lat[3], double u0, double w0, double jitter,
                             double u_th, double sigma_perp, unsigned long long seed, cudaStream_t st) {
  BeamDev b;
  b.ppc = ppc;
  b.lx = lat[0];
  b.ly = lat[1];
  b.lz = lat[2];
  b.u0 = u0;
  b.w0 = w0;
  b.jitter = jitter;
  b.u_th = u_th;
  b.sigma_perp = sigma_perp;
  b.k0 = (uint32_t)(seed & 0xffffffffull);
  b.k1 = (uint32_t)(seed >> 32);
  long long np = r.ncell * ppc;
  int threads = 256;
  long long blocks = (np + threads - 1) / threads;
  if (blocks > 0) k_init_beam<T><<<(unsigned)blocks, threads, 0, st>>>(r, b, np);
  return cudaGetLastError();
}
template cudaError_t launch_init_beam<float>(const RunDev<float>&, int, const int*, double, double, double, double,
                                             double, unsigned long long, cudaStream_t);
template cudaError_t launch_init_beam<double>(const RunDev<double>&, int, const int*, double, double, double, double,
                                              double, unsigned long long, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Import: flat particle arrays (device) -> cell bins of the input buffers.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_import(const __grid_constant__ RunDev<T> r, const __grid_constant__ FlatDev<T> f) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= f.np) return;
  int s = f.species[p];
  long long cell = f.cell[p];
  if ((s != 0 && s != 1) || cell < 0 || cell >= r.ncell) {
    flag_error(r.err, ERR_IMPORT);
    return;
  }
  const long long nxy = (long long)r.nx * r.ny;
  int i = (int)(cell % r.nx), j = (int)((cell / r.nx) % r.ny), k = (int)(cell / nxy);
  T ox = f.ox[p], oy = (r.ndim == 3 && f.oy) ? f.oy[p] : T(0), oz = f.oz[p];
  const T lim = T(1 << 20);
  if (!(ox > -lim && ox < lim && oy > -lim && oy < lim && oz > -lim && oz < lim)) {
    flag_error(r.err, ERR_IMPORT);
    return;
  }
  fold(i, ox, r.nx);
  if (r.ndim == 3) fold(j, oy, r.ny);
  fold(k, oz, r.nz);
  long long dcell = (long long)k * nxy + (long long)j * r.nx + i;
  T w = f.w ? f.w[p] : r.wconst;
  unsigned id = f.id ? f.id[p] : (unsigned)p;
  insert_particle(r, s, dcell, ox, oy, oz, f.dux[p], f.duy[p], f.duz[p], w, id);
}

template <typename T>
cudaError_t launch_import(const RunDev<T>& r, const FlatDev<T>& f, cudaStream_t st) {
  if (f.np <= 0) return cudaSuccess;
  int threads = 256;
  long long blocks = (f.np + threads - 1) / threads;
  k_import<T><<<(unsigned)blocks, threads, 0, st>>>(r, f);
  return cudaGetLastError();
}
template cudaError_t launch_import<float>(const RunDev<float>&, const FlatDev<float>&, cudaStream_t);
template cudaError_t launch_import<double>(const RunDev<double>&, const FlatDev<double>&, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Export: bins -> flat arrays, species 0 first, cells in order. `offs` is the exclusive prefix of
// the (clamped) counts over cells of this species, `base` the species' first flat index.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_export(const __grid_constant__ RunDev<T> r, int s, const long long* __restrict__ offs, long long base,
                         const __grid_constant__ FlatDev<T> f) {
  long long cell = blockIdx.x * (long long)blockDim.y + threadIdx.y;
  if (cell >= r.ncell) return;
  const SpeciesBuf<T>& b = s ? r.in[1] : r.in[0];  // constant indices: no local copy of r
  int n = b.cnt[cell];
  n = n > r.cap ? r.cap : n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    long long src = cell * r.cap + j;
    long long d = base + offs[cell] + j;
    if (d >= f.np) return;
    f.cell[d] = (int)cell;
    f.species[d] = s;
    f.ox[d] = b.ox[src];
    if (f.oy) f.oy[d] = r.ndim == 3 ? b.oy[src] : T(0);
    f.oz[d] = b.oz[src];
    f.dux[d] = b.dux[src];
    f.duy[d] = b.duy[src];
    f.duz[d] = b.duz[src];
    if (f.w) f.w[d] = b.w ? b.w[src] : r.wconst;
    if (f.id) f.id[d] = b.id ? b.id[src] : 0u;
  }
}

template <typename T>
cudaError_t launch_export(const RunDev<T>& r, int s, const long long* offs, long long base, const FlatDev<T>& f,
                          cudaStream_t st) {
  dim3 blk(32, 8);
  long long blocks = (r.ncell + 7) / 8;
  if (blocks > 0) k_export<T><<<(unsigned)blocks, blk, 0, st>>>(r, s, offs, base, f);
  return cudaGetLastError();
}
template cudaError_t launch_export<float>(const RunDev<float>&, int, const long long*, long long, const FlatDev<float>&,
                                          cudaStream_t);
template cudaError_t launch_export<double>(const RunDev<double>&, int, const long long*, long long,
                                           const FlatDev<double>&, cudaStream_t);

// Spill list entries [0, n) -> flat arrays at [base, base + n) (cell and species from the key).
template <typename T>
__global__ void k_spill_export(const __grid_constant__ RunDev<T> r, long long n, long long base,
                               const __grid_constant__ FlatDev<T> f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n || base + i >= f.np) return;
  const long long d = base + i;
  const int key = r.sp.key[i];
  f.cell[d] = key >> 1;
  f.species[d] = key & 1;
  f.ox[d] = r.sp.ox[i];
  if (f.oy) f.oy[d] = r.ndim == 3 ? r.sp.oy[i] : T(0);
  f.oz[d] = r.sp.oz[i];
  f.dux[d] = r.sp.dux[i];
  f.duy[d] = r.sp.duy[i];
  f.duz[d] = r.sp.duz[i];
  if (f.w) f.w[d] = r.sp.w ? r.sp.w[i] : r.wconst;
  if (f.id) f.id[d] = r.sp.id ? r.sp.id[i] : 0u;
}

template <typename T>
cudaError_t launch_spill_export(const RunDev<T>& r, long long n, long long base, const FlatDev<T>& f,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_spill_export<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r, n, base, f);
  return cudaGetLastError();
}
template cudaError_t launch_spill_export<float>(const RunDev<float>&, long long, long long, const FlatDev<float>&,
                                                cudaStream_t);
template cudaError_t launch_spill_export<double>(const RunDev<double>&, long long, long long,
                                                 const FlatDev<double>&, cudaStream_t);

// Largest insertion count over the cells of two count arrays (counts keep every insertion, the
// spilled ones too) into *out, which the caller zeroes.
__global__ void k_max_count(const int* __restrict__ c0, const int* __restrict__ c1, long long ncell, int* out) {
  int m = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x)
    m = max(m, max(c0[c], c1[c]));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

cudaError_t launch_max_count(const int* c0, const int* c1, long long ncell, int* out, cudaStream_t st) {
  if (ncell <= 0) return cudaSuccess;
  long long blocks = (ncell + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_max_count<<<(unsigned)blocks, 256, 0, st>>>(c0, c1, ncell, out);
  return cudaGetLastError();
}

// Exclusive prefix of min(cnt, cap) over cells (two-level, block sums then scan), into offs.
__global__ void k_count_blocks(const int* __restrict__ cnt, long long ncell, int cap, long long* bsum) {
  __shared__ long long s[256];
  long long c = blockIdx.x * 256ll + threadIdx.x;
  long long v = 0;
  if (c < ncell) {
    int n = cnt[c];
    v = n > cap ? cap : n;
  }
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

__global__ void k_scan_blocks(long long* bsum, long long nb, long long* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long acc = 0;
  for (long long b = 0; b < nb; ++b) {
    long long v = bsum[b];
    bsum[b] = acc;
    acc += v;
  }
  *total = acc;
}

__global__ void k_scan_within(const int* __restrict__ cnt, long long ncell, int cap, const long long* bsum,
                              long long* offs) {
  __shared__ long long s[256];
  long long c = blockIdx.x * 256ll + threadIdx.x;
  long long v = 0;
  if (c < ncell) {
    int n = cnt[c];
    v = n > cap ? cap : n;
  }
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    long long t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (c < ncell) offs[c] = bsum[blockIdx.x] + s[threadIdx.x] - v;
}

cudaError_t launch_count_prefix(const int* cnt, long long ncell, int cap, long long* offs, long long* bsum,
                                long long* total, cudaStream_t st) {
  long long nb = (ncell + 255) / 256;
  if (nb == 0) return cudaSuccess;
  k_count_blocks<<<(unsigned)nb, 256, 0, st>>>(cnt, ncell, cap, bsum);
  k_scan_blocks<<<1, 32, 0, st>>>(bsum, nb, total);
  k_scan_within<<<(unsigned)nb, 256, 0, st>>>(cnt, ncell, cap, bsum, offs);
  return cudaGetLastError();
}

long long count_prefix_blocks(long long ncell) { return (ncell + 255) / 256; }

}  // namespace picgb
