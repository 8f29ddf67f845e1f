// Particle kernels: fused gather + Boris + move + Esirkepov deposition + rebin, beam
// initialisation, state import (binning) and export (compaction).
//
// Particle storage: per species, per cell, a bin of `cap` slots (SpeciesBuf). The push kernel
// reads the input buffer and writes every particle straight into its destination cell's bin of
// the output buffer (a counting-sort rebin fused into the push), so particles stay sorted by
// cell at no extra HBM pass. Positions are cell-relative offsets in [0,1); momenta are stored
// relative to the drift u0 z_hat so that FP32 keeps the thermal spread (u0 = 130, spread 1e-4).
#include "common.cuh"
#include "launch.h"

namespace picgb {

template <int NDIM>
struct PTile;
template <>
struct PTile<2> {
  static constexpr int TX = 16, TY = 1, TZ = 16;
};
template <>
struct PTile<3> {
  static constexpr int TX = 8, TY = 8, TZ = 8;
};

constexpr int PUSH_THREADS = 256;

template <typename T, int NDIM>
struct PushSmem {
  static constexpr int TX = PTile<NDIM>::TX, TY = PTile<NDIM>::TY, TZ = PTile<NDIM>::TZ;
  static constexpr int NCL = TX * TY * TZ;
  // gather tile: nodes [X0-1, X0+TX] per direction (y only in 3D)
  static constexpr int GX = TX + 2, GY = (NDIM == 3 ? TY + 2 : 1), GZ = TZ + 2, GN = GX * GY * GZ;
  // current tile: nodes [X0-1, X0+TX+1]
  static constexpr int JX = TX + 3, JY = (NDIM == 3 ? TY + 3 : 1), JZ = TZ + 3, JN = JX * JY * JZ;
  static constexpr size_t bytes() {
    return sizeof(T) * (6 * GN + 3 * JN) + sizeof(int) * (NCL + 1 + PUSH_THREADS / 32 + 1);
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

// Largest c in [0, n) with pre[c] <= f (pre is a nondecreasing exclusive prefix, pre[0] = 0).
__device__ __forceinline__ int find_cell(const int* pre, int n, int f) {
  int lo = 0, hi = n;  // invariant pre[lo] <= f < pre[hi] (pre[n] = total > f)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= f) lo = mid; else hi = mid;
  }
  return lo;
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

template <typename T>
__device__ __forceinline__ EsirDir<T> esir_dir(T o, T d) {
  EsirDir<T> e;
  const T x1 = o + d;
  if (x1 < T(0)) {  // into the cell below: window nodes -1, 0, 1
    e.a = -1;
    e.S0[0] = T(0); e.S0[1] = T(1) - o; e.S0[2] = o;
    e.dS[0] = -x1; e.dS[2] = -o; e.dS[1] = -(e.dS[0] + e.dS[2]);
    e.off = T(1) + x1;
    e.shift = -1;
    if (e.off >= T(1)) { e.off = T(0); e.shift = 0; }
  } else {
    e.a = 0;
    e.S0[0] = T(1) - o; e.S0[1] = o; e.S0[2] = T(0);
    const T am = T(1) - o;  // distance to the upper face
    const T c = d - am;     // x1 - 1, without the rounding of x1
    if (x1 >= T(1) && c > T(0)) {  // into the cell above: nodes 0, 1, 2
      e.dS[0] = -am; e.dS[2] = c; e.dS[1] = -(e.dS[0] + e.dS[2]);
      e.off = c;
      e.shift = 1;
    } else {  // same cell (or onto the upper face within rounding)
      e.dS[0] = -d; e.dS[1] = d; e.dS[2] = T(0);
      if (x1 >= T(1)) { e.off = T(0); e.shift = 1; }
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

// Add the NV contributions of every valid lane into shared memory. Lanes are grouped by window
// origin `key`; per group and per round of 32 values, a butterfly transpose-reduction leaves in
// lane l the group's sum of value l, which that lane adds with one shared-memory atomic (the 32
// lanes of a round touch distinct addresses).
template <typename T, int NDIM>
__device__ __forceinline__ void deposit_warp(T* sj, const T (&dv)[DepLayout<NDIM>::NV], int key, bool valid,
                                             int lane) {
  using S = PushSmem<T, NDIM>;
  constexpr int NV = DepLayout<NDIM>::NV;
  constexpr int ROUNDS = (NV + 31) / 32;
  unsigned pending = __ballot_sync(0xffffffffu, valid);
  while (pending) {
    const int src = __ffs(pending) - 1;
    const int k = __shfl_sync(0xffffffffu, key, src);
    const bool mine = valid && key == k;
    pending &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
    for (int rd = 0; rd < ROUNDS; ++rd) {
      T x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = (mine && rd * 32 + i < NV) ? dv[rd * 32 + i] : T(0);
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const bool up = (lane & sh) != 0;
#pragma unroll
        for (int j = 0; j < sh; ++j) {
          const T send = up ? x[j] : x[j + sh];
          const T keep = up ? x[j + sh] : x[j];
          x[j] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
        }
      }
      const int i = rd * 32 + lane;
      if (i < NV && x[0] != T(0)) {
        int comp, a, b, c;
        DepLayout<NDIM>::at(i, comp, a, b, c);
        atomicAdd(sj + comp * S::JN + k + (c * S::JY + b) * S::JX + a, x[0]);
      }
    }
  }
}

template <typename T, int NDIM, int SCHEME, bool HAS_W, bool HAS_ID>
__global__ void __launch_bounds__(PUSH_THREADS) k_push(RunDev<T> r) {
  using S = PushSmem<T, NDIM>;
  constexpr int TX = S::TX, TY = S::TY, TZ = S::TZ, NCL = S::NCL;
  constexpr int PER = NCL / PUSH_THREADS;
  static_assert(NCL % PUSH_THREADS == 0, "cells per tile must be a multiple of the block size");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sg = reinterpret_cast<T*>(smem_raw);
  T* sj = sg + 6 * S::GN;
  int* spre = reinterpret_cast<int*>(sj + 3 * S::JN);
  int* swarp = spre + NCL + 1;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x;
  const int tix = tile % r.ntx;
  const int tiy = (tile / r.ntx) % r.nty;
  const int tiz = tile / (r.ntx * r.nty);
  const int X0 = tix * TX, Y0 = tiy * TY, Z0 = tiz * TZ;
  const int wx = min(TX, r.nx - X0), wy = min(TY, r.ny - Y0), wz = min(TZ, r.nz - Z0);
  const long long nxy = (long long)r.nx * r.ny;

  // 1. field copies of the tile and its halo into shared memory (periodic wrap)
  for (int e = tid; e < 6 * S::GN; e += PUSH_THREADS) {
    int c = e / S::GN, rem = e - c * S::GN;
    int lz = rem / (S::GX * S::GY);
    int ly = (rem / S::GX) % S::GY;
    int lx = rem % S::GX;
    int gx = wrapi(X0 - 1 + lx, r.nx);
    int gy = NDIM == 3 ? wrapi(Y0 - 1 + ly, r.ny) : 0;
    int gz = wrapi(Z0 - 1 + lz, r.nz);
    sg[e] = __ldg(r.g[c] + (long long)gz * nxy + (long long)gy * r.nx + gx);
  }
  for (int e = tid; e < 3 * S::JN; e += PUSH_THREADS) sj[e] = T(0);

  T kin = T(0);  // per-thread partial sum of w (gamma - 1)
  int npush = 0;  // particles pushed by this thread
  for (int s = 0; s < 2; ++s) {
    const SpeciesBuf<T> pin = r.in[s];
    const SpeciesBuf<T> pout = r.out[s];
    const T q = s == 0 ? T(-1) : T(1);
    // 2. particle counts of the tile's cells -> exclusive prefix (cells x-fastest in the tile)
    int loc[PER];
    int mysum = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      int cl = tid * PER + u;
      int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
      int n = 0;
      if (lx < wx && ly < wy && lz < wz) {
        long long cell = (long long)(Z0 + lz) * nxy + (long long)(Y0 + ly) * r.nx + X0 + lx;
        n = pin.cnt[cell];
        n = n > r.cap ? r.cap : n;  // an overflow was flagged when it happened
        pin.cnt[cell] = 0;          // this count array is the next step's output
      }
      loc[u] = mysum;
      mysum += n;
    }
    int incl = mysum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) swarp[warp] = incl;
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int w = 0; w < PUSH_THREADS / 32; ++w) {
        int v = swarp[w];
        swarp[w] = acc;
        acc += v;
      }
      spre[NCL] = acc;
    }
    __syncthreads();
    {
      int base = swarp[warp] + incl - mysum;
#pragma unroll
      for (int u = 0; u < PER; ++u) spre[tid * PER + u] = base + loc[u];
    }
    __syncthreads();
    const int N = spre[NCL];

    // 3. particles of the tile, flattened over its cells
    for (int fb = 0; fb < N; fb += PUSH_THREADS) {
      const int f = fb + tid;
      const bool valid = f < N;
      int dst = -1 - lane;  // unique per lane when invalid
      T nox = 0, noy = 0, noz = 0, ux = 0, uy = 0, uz = 0, w = 0;
      unsigned pid = 0;
      constexpr int NV = DepLayout<NDIM>::NV;
      T dv[NV];
      int wkey = -1;
      if (valid) {
        const int cl = find_cell(spre, NCL, f);
        const int j = f - spre[cl];
        const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
        const int gi = X0 + lx, gj = Y0 + ly, gk = Z0 + lz;
        const long long slot = ((long long)gk * nxy + (long long)gj * r.nx + gi) * r.cap + j;
        T ox = __ldg(pin.ox + slot);
        T oy = NDIM == 3 ? __ldg(pin.oy + slot) : T(0);
        T oz = __ldg(pin.oz + slot);
        ux = __ldg(pin.dux + slot);
        uy = __ldg(pin.duy + slot);
        uz = __ldg(pin.duz + slot);
        w = HAS_W ? __ldg(pin.w + slot) : r.wconst;
        if (HAS_ID) pid = __ldg(pin.id + slot);

        // gather
        const DirW<T> dwx = dir_weights(ox), dwy = dir_weights(oy), dwz = dir_weights(oz);
        T F[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) F[c] = gather_comp<T, NDIM, SCHEME>(sg + c * S::GN, c, lx, ly, lz, dwx, dwy, dwz);

        // relativistic Boris, momenta relative to the drift u0 z_hat
        const T h = q * r.hq;
        T mx = ux + h * F[0], my = uy + h * F[1], mz = uz + h * F[2];
        T Mz = r.u0 + mz;
        T ig = T(1) / dev_sqrt(T(1) + mx * mx + my * my + Mz * Mz);
        T tx = h * F[3] * ig, ty = h * F[4] * ig, tz = h * F[5] * ig;
        T sf = T(2) / (T(1) + tx * tx + ty * ty + tz * tz);
        T sx = sf * tx, sy = sf * ty, sz = sf * tz;
        T px = mx + (my * tz - Mz * ty);
        T py = my + (Mz * tx - mx * tz);
        T pz = Mz + (mx * ty - my * tx);
        ux = mx + (py * sz - pz * sy) + h * F[0];
        uy = my + (pz * sx - px * sz) + h * F[1];
        uz = mz + (px * sy - py * sx) + h * F[2];
        T Uz = r.u0 + uz;
        T u2 = ux * ux + uy * uy + Uz * Uz;
        T gn = dev_sqrt(T(1) + u2);
        T ign = T(1) / gn;
        T vx = ux * ign, vy = uy * ign, vz = Uz * ign;
        kin += w * (u2 / (gn + T(1)));
        ++npush;

        // move (cell-relative displacement in grid units)
        T ddx = r.dtdx * vx;
        T ddy = NDIM == 3 ? r.dtdy * vy : T(0);
        T ddz = r.dtdz * vz;
        if (!(ddx > T(-1) && ddx < T(1) && ddy > T(-1) && ddy < T(1) && ddz > T(-1) && ddz < T(1))) {
          flag_error(r.err, ERR_NONFINITE);
          ddx = ddy = ddz = T(0);
          ux = uy = uz = T(0);
          vx = vy = T(0);
        }
        const EsirDir<T> ex_ = esir_dir(ox, ddx);
        const EsirDir<T> ez_ = esir_dir(oz, ddz);
        EsirDir<T> ey_;
        if (NDIM == 3) ey_ = esir_dir(oy, ddy);
        else { ey_.a = 0; ey_.shift = 0; ey_.off = T(0); }
        const int ax = ex_.a, ay = NDIM == 3 ? ey_.a : 0, az = ez_.a;
        T S0x[3], dSx[3], S0y[3], dSy[3], S0z[3], dSz[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          S0x[a] = ex_.S0[a]; dSx[a] = ex_.dS[a];
          S0z[a] = ez_.S0[a]; dSz[a] = ez_.dS[a];
          if (NDIM == 3) { S0y[a] = ey_.S0[a]; dSy[a] = ey_.dS[a]; }
        }
        const T qw = q * w;
        // per-particle current contributions v[i] to the smem tile at offset dep_off<NDIM>(i)
        // from the window origin (bx, by, bz)
        const int bx = lx + ax + 1, by = NDIM == 3 ? ly + ay + 1 : 0, bz = lz + az + 1;
        wkey = (bz * S::JY + by) * S::JX + bx;
        if (NDIM == 2) {
          const T cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vy * r.jfy2d;
#pragma unroll
          for (int b = 0; b < 3; ++b) {  // Jx(a+1/2, b): running sum over a
            T fz = S0z[b] + T(0.5) * dSz[b];
            T a0 = dSx[0] * fz, a1 = a0 + dSx[1] * fz;
            dv[b * 2 + 0] = cx * a0;
            dv[b * 2 + 1] = cx * a1;
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {  // Jz(a, b+1/2): running sum over b
            T fx = S0x[a] + T(0.5) * dSx[a];
            T a0 = dSz[0] * fx, a1 = a0 + dSz[1] * fx;
            dv[6 + a * 2 + 0] = cz * a0;
            dv[6 + a * 2 + 1] = cz * a1;
          }
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a)  // Jy(a, b): out-of-plane weight
              dv[12 + b * 3 + a] = cy * (S0x[a] * S0z[b] + T(0.5) * dSx[a] * S0z[b] + T(0.5) * S0x[a] * dSz[b] +
                                         dSx[a] * dSz[b] * T(1.0 / 3.0));
        } else {
          const T cx = qw * r.jfx, cy = qw * r.jfy, cz = qw * r.jfz;
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b) {  // Jx(a+1/2, b, c)
              T tr = S0y[b] * S0z[c] + T(0.5) * dSy[b] * S0z[c] + T(0.5) * S0y[b] * dSz[c] +
                     dSy[b] * dSz[c] * T(1.0 / 3.0);
              T a0 = dSx[0] * tr, a1 = a0 + dSx[1] * tr;
              dv[(c * 3 + b) * 2 + 0] = cx * a0;
              dv[(c * 3 + b) * 2 + 1] = cx * a1;
            }
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int a = 0; a < 3; ++a) {  // Jy(a, b+1/2, c)
              T tr = S0x[a] * S0z[c] + T(0.5) * dSx[a] * S0z[c] + T(0.5) * S0x[a] * dSz[c] +
                     dSx[a] * dSz[c] * T(1.0 / 3.0);
              T a0 = dSy[0] * tr, a1 = a0 + dSy[1] * tr;
              dv[18 + (c * 3 + a) * 2 + 0] = cy * a0;
              dv[18 + (c * 3 + a) * 2 + 1] = cy * a1;
            }
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {  // Jz(a, b, c+1/2)
              T tr = S0x[a] * S0y[b] + T(0.5) * dSx[a] * S0y[b] + T(0.5) * S0x[a] * dSy[b] +
                     dSx[a] * dSy[b] * T(1.0 / 3.0);
              T a0 = dSz[0] * tr, a1 = a0 + dSz[1] * tr;
              dv[36 + (b * 3 + a) * 2 + 0] = cz * a0;
              dv[36 + (b * 3 + a) * 2 + 1] = cz * a1;
            }
        }

        // new cell and offsets
        nox = ex_.off;
        noy = NDIM == 3 ? ey_.off : T(0);
        noz = ez_.off;
        const int ni = wrapi(gi + ex_.shift, r.nx);
        const int nj = NDIM == 3 ? wrapi(gj + ey_.shift, r.ny) : 0;
        const int nk = wrapi(gk + ez_.shift, r.nz);
        dst = (int)((long long)nk * nxy + (long long)nj * r.nx + ni);
      }
      // deposit: lanes that share a window origin sum their contributions by a warp transpose-
      // reduction, then every lane adds one distinct value to shared memory (no atomic conflicts)
      deposit_warp<T, NDIM>(sj, dv, wkey, valid, lane);

      // 4. rebin: warp-aggregated slot reservation in the destination cell's bin
      const unsigned peers = __match_any_sync(0xffffffffu, dst);
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int base = 0;
      if (valid && lane == leader) base = atomicAdd(pout.cnt + dst, __popc(peers));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (valid) {
        const int j = base + rank;
        if (j < r.cap) {
          const long long o = (long long)dst * r.cap + j;
          pout.ox[o] = nox;
          if (NDIM == 3) pout.oy[o] = noy;
          pout.oz[o] = noz;
          pout.dux[o] = ux;
          pout.duy[o] = uy;
          pout.duz[o] = uz;
          if (HAS_W) pout.w[o] = w;
          if (HAS_ID) pout.id[o] = pid;
        } else {
          flag_error(r.err, ERR_OVERFLOW);
        }
      }
    }
    __syncthreads();  // spre / swarp are reused by the next species
  }

  // 5. flush the tile's current to global memory
  for (int e = tid; e < 3 * S::JN; e += PUSH_THREADS) {
    T v = sj[e];
    if (v == T(0)) continue;
    int c = e / S::JN, rem = e - c * S::JN;
    int lz = rem / (S::JX * S::JY);
    int ly = (rem / S::JX) % S::JY;
    int lx = rem % S::JX;
    int gx = wrapi(X0 - 1 + lx, r.nx);
    int gy = NDIM == 3 ? wrapi(Y0 - 1 + ly, r.ny) : 0;
    int gz = wrapi(Z0 - 1 + lz, r.nz);
    atomicAdd(r.j[c] + (long long)gz * nxy + (long long)gy * r.nx + gx, v);
  }

  // 6. kinetic energy and particle count of this step: per-thread partial sums in the working
  // precision, FP64 across the block and the grid
  if (r.kin) {
    double kd = (double)kin;
    int nd = npush;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kd += __shfl_xor_sync(0xffffffffu, kd, o);
      nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    __shared__ double skin[PUSH_THREADS / 32];
    __shared__ int scnt[PUSH_THREADS / 32];
    if (lane == 0) {
      skin[warp] = kd;
      scnt[warp] = nd;
    }
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      long long c = 0;
      for (int w2 = 0; w2 < PUSH_THREADS / 32; ++w2) {
        t += skin[w2];
        c += scnt[w2];
      }
      atomicAdd(r.kin, t);
      atomicAdd(r.kin + 1, (double)c);
    }
  }
}

template <typename T, int NDIM, int SCHEME>
static cudaError_t launch_push_t(const RunDev<T>& r, bool has_w, bool has_id, cudaStream_t st) {
  using S = PushSmem<T, NDIM>;
  const size_t sm = S::bytes();
  const int ntiles = r.ntx * r.nty * r.ntz;
  auto go = [&](void (*kern)(RunDev<T>)) -> cudaError_t {
    cudaError_t e = ensure_dynamic_smem((const void*)kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, PUSH_THREADS, sm, st>>>(r);
    return cudaGetLastError();
  };
  if (has_w && has_id) return go(k_push<T, NDIM, SCHEME, true, true>);
  if (has_w) return go(k_push<T, NDIM, SCHEME, true, false>);
  if (has_id) return go(k_push<T, NDIM, SCHEME, false, true>);
  return go(k_push<T, NDIM, SCHEME, false, false>);
}

template <typename T>
cudaError_t launch_push(const RunDev<T>& r, bool has_w, bool has_id, cudaStream_t st) {
  if (r.ndim == 2)
    return r.scheme == 0 ? launch_push_t<T, 2, 0>(r, has_w, has_id, st) : launch_push_t<T, 2, 1>(r, has_w, has_id, st);
  return r.scheme == 0 ? launch_push_t<T, 3, 0>(r, has_w, has_id, st) : launch_push_t<T, 3, 1>(r, has_w, has_id, st);
}
template cudaError_t launch_push<float>(const RunDev<float>&, bool, bool, cudaStream_t);
template cudaError_t launch_push<double>(const RunDev<double>&, bool, bool, cudaStream_t);

void push_tiles(int ndim, int nx, int ny, int nz, int* ntx, int* nty, int* ntz) {
  if (ndim == 2) {
    *ntx = (nx + PTile<2>::TX - 1) / PTile<2>::TX;
    *nty = 1;
    *ntz = (nz + PTile<2>::TZ - 1) / PTile<2>::TZ;
  } else {
    *ntx = (nx + PTile<3>::TX - 1) / PTile<3>::TX;
    *nty = (ny + PTile<3>::TY - 1) / PTile<3>::TY;
    *ntz = (nz + PTile<3>::TZ - 1) / PTile<3>::TZ;
  }
}

// ---------------------------------------------------------------------------------------------
// Insert one particle into its cell bin (used by init and import).
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void insert_particle(const SpeciesBuf<T>& b, int cap, long long cell, T ox, T oy, T oz,
                                                T ux, T uy, T uz, T w, unsigned id, int* err) {
  int j = atomicAdd(b.cnt + cell, 1);
  if (j >= cap) {
    flag_error(err, ERR_OVERFLOW);
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
// Seeded beam: one thread per lattice point; see pic.h / the oracle for the recipe. All random
// numbers and the derived positions and momenta are computed in FP64 and rounded once.
// ---------------------------------------------------------------------------------------------
struct BeamDev {
  int ppc, lx, ly, lz;
  double u0, w0, jitter, u_th, sigma_perp;
  uint32_t k0, k1;
};

__device__ __forceinline__ double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

template <typename T>
__global__ void k_init_beam(RunDev<T> r, BeamDev b, long long npoints) {
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
    insert_particle(r.in[s], r.cap, dcell, tox, toy, toz, ux, uy, uz, (T)w, (unsigned)(p * 2 + s), r.err);
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
__global__ void k_import(RunDev<T> r, FlatDev<T> f) {
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
  insert_particle(r.in[s], r.cap, dcell, ox, oy, oz, f.dux[p], f.duy[p], f.duz[p], w, id, r.err);
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
__global__ void k_export(RunDev<T> r, int s, const long long* __restrict__ offs, long long base, FlatDev<T> f) {
  long long cell = blockIdx.x * (long long)blockDim.y + threadIdx.y;
  if (cell >= r.ncell) return;
  const SpeciesBuf<T> b = r.in[s];
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
