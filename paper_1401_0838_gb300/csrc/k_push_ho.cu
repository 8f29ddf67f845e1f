// Particle step for cubic shapes (Sec. 3 runs with cubic interpolation) and for the
// momentum-conserving gather (the scheme Eq. 5 belongs to): gather, Boris push, move, Esirkepov
// deposition and rebin in one kernel, for any (shape order 1 or 3) x (Galerkin, Uniform,
// momentum-conserving) combination in 2D and 3D. The linear Galerkin / Uniform step has its own,
// more specialised kernel (k_particles.cu). Here: one CTA per particle tile with the field copies
// and the tile's current in shared memory; in 2D one warp per cell (lanes over the cell's
// particles, the deposit reduced over the warp), in 3D one thread per cell walking the cell's
// particles with the deposit added by shared-memory atomics.
//
// Shapes: centred B-splines S_n (S0 box, S1 hat, S2 quadratic, S3 cubic). Gather along a
// direction: Uniform uses the particle shape order n at the component's own (staggered) nodes;
// Galerkin uses order n-1 along each direction in which the component is half staggered; the
// momentum-conserving scheme averages every component from its Yee location to the nodes and
// interpolates with S_n there. Deposit: Esirkepov's W from S_n at the old position and the shape
// change dS, formed from the displacement on each polynomial piece (exact, full relative
// precision for small moves), the plain difference across a knot.
#include "common.cuh"
#include "launch.h"

namespace picgb {

namespace {

constexpr int HO_THREADS = 256;


// Geometry of the shared-memory tiles for shape order ORDER: the field tile holds nodes
// [-H, T + H) per direction, the current tile nodes [-H, T + H + 1), H = (ORDER + 1) / 2.
template <typename T, int NDIM, int ORDER>
struct HoGeom {
  using TL = HoTile<T, NDIM>;
  static constexpr int H = (ORDER + 1) / 2;
  static constexpr int GX = TL::TX + 2 * H, GY = NDIM == 3 ? TL::TY + 2 * H : 1, GZ = TL::TZ + 2 * H;
  static constexpr int GN = GX * GY * GZ;
  static constexpr int JX = TL::TX + 2 * H + 1, JY = NDIM == 3 ? TL::TY + 2 * H + 1 : 1, JZ = TL::TZ + 2 * H + 1;
  static constexpr int JN = JX * JY * JZ;
  static constexpr int NCL = TL::TX * TL::TY * TL::TZ;
  static constexpr int NW = ORDER == 3 ? 6 : 4;   // deposit window nodes per direction
  static constexpr int K0 = ORDER == 3 ? -2 : -1;  // first window node relative to the start cell
  static constexpr size_t bytes() {
    return sizeof(T) * (6 * (size_t)GN + 3 * (size_t)JN) + sizeof(int) * 4 * (size_t)NCL;
  }
};

// Periodic index of any g.
__device__ __forceinline__ int wrap_any(int g, int n) {
  if (g < 0) {
    g += n;
    if (g < 0) g = wrapi(g, n);
  } else if (g >= n) {
    g -= n;
    if (g >= n) g %= n;
  }
  return g;
}

// Centred B-splines.
template <typename T>
__device__ __forceinline__ T bspl(int n, T t) {
  const T a = t < T(0) ? -t : t;
  if (n == 0) return (t >= T(-0.5) && t < T(0.5)) ? T(1) : T(0);
  if (n == 1) return a < T(1) ? T(1) - a : T(0);
  if (n == 2) {
    if (a <= T(0.5)) return T(0.75) - a * a;
    if (a < T(1.5)) return T(0.5) * (T(1.5) - a) * (T(1.5) - a);
    return T(0);
  }
  if (a <= T(1)) return T(2.0 / 3.0) - a * a + T(0.5) * a * a * a;
  if (a < T(2)) return (T(2) - a) * (T(2) - a) * (T(2) - a) * T(1.0 / 6.0);
  return T(0);
}

// S_n(a0 - d) - S_n(a0) for the particle shape (n = 1 or 3): on one polynomial piece from the
// displacement (linear: slope times -d; cubic: the terminating Taylor series), else the difference.
template <typename T>
__device__ __forceinline__ T shape_change(int n, T a0, T d) {
  const T a1 = a0 - d;
  if (n == 1) {
    const int p0 = (a0 > T(-1)) + (a0 > T(0)) + (a0 >= T(1)), p1 = (a1 > T(-1)) + (a1 > T(0)) + (a1 >= T(1));
    if (p0 == p1) return p0 == 1 ? -d : (p0 == 2 ? d : T(0));
    return bspl(1, a1) - bspl(1, a0);
  }
  const int p0 = (a0 > T(-2)) + (a0 > T(-1)) + (a0 > T(0)) + (a0 > T(1)) + (a0 >= T(2));
  const int p1 = (a1 > T(-2)) + (a1 > T(-1)) + (a1 > T(0)) + (a1 > T(1)) + (a1 >= T(2));
  if (p0 != p1) return bspl(3, a1) - bspl(3, a0);
  T d1, d2, d3;  // P', P'', P''' of the piece at a0
  switch (p0) {
    case 1: d1 = T(0.5) * (T(2) + a0) * (T(2) + a0); d2 = T(2) + a0; d3 = T(1); break;
    case 2: d1 = -T(2) * a0 - T(1.5) * a0 * a0; d2 = -T(2) - T(3) * a0; d3 = T(-3); break;
    case 3: d1 = -T(2) * a0 + T(1.5) * a0 * a0; d2 = -T(2) + T(3) * a0; d3 = T(3); break;
    case 4: d1 = -T(0.5) * (T(2) - a0) * (T(2) - a0); d2 = T(2) - a0; d3 = T(-1); break;
    default: return T(0);
  }
  return -d * (d1 - d * (T(0.5) * d2 - d * d3 * T(1.0 / 6.0)));
}

// Gather weights along one direction for a position at cell-relative offset o: order `ord`
// on the integer lattice (st = 0) or the half-integer lattice (st = 1). first = the first node
// relative to the cell; w[0..ord].
template <typename T>
__device__ __forceinline__ void gweights(T o, int st, int ord, int& first, T (&w)[4]) {
  const T xs = st ? o - T(0.5) : o;  // position in units of the component's node lattice, rel. to the cell
  if (ord & 1) {
    const int fl = xs < T(0) ? -1 : 0;
    first = fl - (ord - 1) / 2;
  } else {
    const int fl = xs + T(0.5) >= T(1) ? 1 : (xs + T(0.5) < T(0) ? -1 : 0);
    first = fl - ord / 2;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = q <= ord ? bspl(ord, xs - T(first + q)) : T(0);
}

// Stagger of Ex Ey Ez Bx By Bz along x, y, z (compile-time, so that the gather's orders and loop
// bounds fold for each unrolled component).
__host__ __device__ constexpr int stag_ho(int c, int axis) {
  return axis == 0 ? (c == 0 || c == 4 || c == 5) : (axis == 1 ? (c == 1 || c == 3 || c == 5) : (c == 2 || c == 3 || c == 4));
}

template <typename T, int NDIM, int ORDER, int SCHEME, int C>
__device__ __forceinline__ T gather_comp(const T* sgc, int lx, int ly, int lz, T ox, T oy, T oz) {
  using G = HoGeom<T, NDIM, ORDER>;
  // momentum-conserving: integer nodes of the averaged tile; Galerkin: one order lower along the
  // component's half-staggered directions; Uniform: the shape order at the component's nodes
  constexpr int SX = SCHEME == 2 ? 0 : stag_ho(C, 0), SY = SCHEME == 2 ? 0 : stag_ho(C, 1);
  constexpr int SZ = SCHEME == 2 ? 0 : stag_ho(C, 2);
  constexpr int OX = SCHEME == 0 ? ORDER - SX : ORDER, OZ = SCHEME == 0 ? ORDER - SZ : ORDER;
  constexpr int OY = NDIM == 3 ? (SCHEME == 0 ? ORDER - SY : ORDER) : 0;
  int fx, fy = 0, fz;
  T wx[4], wy[4] = {T(1), T(0), T(0), T(0)}, wz[4];
  gweights(ox, SX, OX, fx, wx);
  if (NDIM == 3) gweights(oy, SY, OY, fy, wy);
  gweights(oz, SZ, OZ, fz, wz);
  T acc = T(0);
#pragma unroll
  for (int c3 = 0; c3 <= OZ; ++c3) {
    const int iz = lz + fz + c3 + G::H;
#pragma unroll
    for (int c2 = 0; c2 <= OY; ++c2) {
      const int iy = NDIM == 3 ? ly + fy + c2 + G::H : 0;
      const T* row = sgc + (iz * G::GY + iy) * G::GX + lx + fx + G::H;
      T r = T(0);
#pragma unroll
      for (int c1 = 0; c1 <= OX; ++c1) r += wx[c1] * row[c1];
      acc += wz[c3] * wy[c2] * r;
    }
  }
  return acc;
}

template <typename T, int NDIM, int ORDER, int SCHEME>
__device__ __forceinline__ void gather6(const T* sg, int lx, int ly, int lz, T ox, T oy, T oz, T (&F)[6]) {
  using G = HoGeom<T, NDIM, ORDER>;
  F[0] = gather_comp<T, NDIM, ORDER, SCHEME, 0>(sg, lx, ly, lz, ox, oy, oz);
  F[1] = gather_comp<T, NDIM, ORDER, SCHEME, 1>(sg + G::GN, lx, ly, lz, ox, oy, oz);
  F[2] = gather_comp<T, NDIM, ORDER, SCHEME, 2>(sg + 2 * G::GN, lx, ly, lz, ox, oy, oz);
  F[3] = gather_comp<T, NDIM, ORDER, SCHEME, 3>(sg + 3 * G::GN, lx, ly, lz, ox, oy, oz);
  F[4] = gather_comp<T, NDIM, ORDER, SCHEME, 4>(sg + 4 * G::GN, lx, ly, lz, ox, oy, oz);
  F[5] = gather_comp<T, NDIM, ORDER, SCHEME, 5>(sg + 5 * G::GN, lx, ly, lz, ox, oy, oz);
}

// Tile geometry shared by the step's phases.
struct HoTileRef {
  int X0, Y0, Z0, wx, wy, wz, nxy;
};

template <typename T>
__device__ __forceinline__ HoTileRef ho_tile(const RunDev<T>& r) {
  const int tile = blockIdx.x;
  const int tix = tile % r.ntx, tiy = (tile / r.ntx) % r.nty, tiz = tile / (r.ntx * r.nty);
  HoTileRef t;  // the run's tile extents are at most HoTile's; cells past them stay empty
  t.X0 = tix * r.tex;
  t.Y0 = tiy * r.tey;
  t.Z0 = tiz * r.tez;
  t.wx = min(r.tex, r.nx - t.X0);
  t.wy = min(r.tey, r.ny - t.Y0);
  t.wz = min(r.tez, r.nz - t.Z0);
  t.nxy = r.nx * r.ny;  // cells < 2^30
  return t;
}

// Phases 1-2: field copies of the tile and halo into shared memory (node-averaged for the
// momentum scheme), the tile's current zeroed, input counts read (and zeroed), output counts zeroed.
template <typename T, int NDIM, int ORDER, int SCHEME>
__device__ __forceinline__ void ho_prologue(const RunDev<T>& r, const HoTileRef& t, T* sg, T* sj, int* sn,
                                            int* scnt) {
  using G = HoGeom<T, NDIM, ORDER>;
  using TL = HoTile<T, NDIM>;
  constexpr int TX = TL::TX, TY = TL::TY, NCL = G::NCL, H = G::H;
  const int tid = threadIdx.x;
  const int X0 = t.X0, Y0 = t.Y0, Z0 = t.Z0, wx = t.wx, wy = t.wy, wz = t.wz, nxy = t.nxy;
  // 1. field copies of the tile and its halo (periodic) and the cells' particle counts, as one
  // asynchronous batch (one global round trip); current tile and output counts zeroed
  for (int e = tid; e < 6 * G::GN; e += HO_THREADS) {
    const int c = e / G::GN, rem = e - c * G::GN;
    const int lz = rem / (G::GX * G::GY), ly = (rem / G::GX) % G::GY, lx = rem % G::GX;
    const int gx = wrap_any(X0 - H + lx, r.nx);
    const int gy = NDIM == 3 ? wrap_any(Y0 - H + ly, r.ny) : 0;
    const int gz = wrap_any(Z0 - H + lz, r.nz);
    const T* src = r.g[0];
    switch (c) {  // constant-indexed parameter reads
      case 1: src = r.g[1]; break;
      case 2: src = r.g[2]; break;
      case 3: src = r.g[3]; break;
      case 4: src = r.g[4]; break;
      case 5: src = r.g[5]; break;
      default: break;
    }
    copy1_async(sg + e, src + (long long)gz * nxy + (long long)gy * r.nx + gx);
  }
  for (int e = tid; e < 3 * G::JN; e += HO_THREADS) sj[e] = T(0);
  for (int cl = tid; cl < NCL; cl += HO_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    if (lx < wx && ly < wy && lz < wz) {
      const int cell = (Z0 + lz) * nxy + (Y0 + ly) * r.nx + X0 + lx;
      copy1_async(sn + cl, r.in[0].cnt + cell);
      copy1_async(sn + NCL + cl, r.in[1].cnt + cell);
    } else {
      sn[cl] = 0;
      sn[NCL + cl] = 0;
    }
    scnt[cl] = 0;
    scnt[NCL + cl] = 0;
  }
  cp_async_commit();
  cp_async_wait_all();
  // 2. counts clamped (the excess of a full bin is in the spill list) and the input counts zeroed (they
  // become the next step's output counts); each thread reads back only the counts it copied
  for (int cl = tid; cl < NCL; cl += HO_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    if (lx < wx && ly < wy && lz < wz) {
      const int cell = (Z0 + lz) * nxy + (Y0 + ly) * r.nx + X0 + lx;
      sn[cl] = min(sn[cl], r.cap);
      sn[NCL + cl] = min(sn[NCL + cl], r.cap);
      r.in[0].cnt[cell] = 0;
      r.in[1].cnt[cell] = 0;
    }
  }
  __syncthreads();
  if (SCHEME == 2) {
    // average each component from its Yee location to the nodes along its half-staggered
    // directions: node i gets (v[i-1] + v[i]) / 2, rows walked from the top so v[i-1] is unchanged
    for (int axis = 0; axis < 3; ++axis) {
      if (axis == 1 && NDIM == 2) continue;
      const int len = axis == 0 ? G::GX : (axis == 1 ? G::GY : G::GZ);
      const int stride = axis == 0 ? 1 : (axis == 1 ? G::GX : G::GX * G::GY);
      const int nrows = G::GN / len;
      for (int e = tid; e < 6 * nrows; e += HO_THREADS) {
        const int c = e / nrows, row = e - c * nrows;
        if (!stag_ho(c, axis)) continue;
        int base;  // first element of the row
        if (axis == 0) base = row * G::GX;
        else if (axis == 1) base = (row / G::GX) * G::GX * G::GY + row % G::GX;
        else base = row;
        T* v = sg + c * G::GN + base;
        for (int i = len - 1; i >= 1; --i) v[i * stride] = T(0.5) * (v[i * stride] + v[(i - 1) * stride]);
      }
      __syncthreads();
    }
  }
}

// Phases 4-6: output counts, the tile's current into global memory, the step's kinetic sums.
template <typename T, int NDIM, int ORDER>
__device__ __forceinline__ void ho_epilogue(const RunDev<T>& r, const HoTileRef& t, T* sj, int* scnt, T kin,
                                            int npush) {
  using G = HoGeom<T, NDIM, ORDER>;
  using TL = HoTile<T, NDIM>;
  constexpr int TX = TL::TX, TY = TL::TY, NCL = G::NCL, H = G::H;
  const int tid = threadIdx.x;
  const int X0 = t.X0, Y0 = t.Y0, Z0 = t.Z0, wx = t.wx, wy = t.wy, wz = t.wz, nxy = t.nxy;
  __syncthreads();
  // 4. output counts of the tile's cells (a count past the capacity, whose excess went on through
  // the leaver list, is stored as the capacity)
  for (int cl = tid; cl < NCL; cl += HO_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    if (lx < wx && ly < wy && lz < wz) {
      const int cell = (Z0 + lz) * nxy + (Y0 + ly) * r.nx + X0 + lx;
      r.out[0].cnt[cell] = min(scnt[cl], r.cap);
      r.out[1].cnt[cell] = min(scnt[NCL + cl], r.cap);
    }
  }
  // 5. the tile's current into global memory
  for (int e = tid; e < 3 * G::JN; e += HO_THREADS) {
    const T v = sj[e];
    if (v == T(0)) continue;
    const int c = e / G::JN, rem = e - c * G::JN;
    const int lz = rem / (G::JX * G::JY), ly = (rem / G::JX) % G::JY, lx = rem % G::JX;
    const int gx = wrap_any(X0 - H + lx, r.nx);
    const int gy = NDIM == 3 ? wrap_any(Y0 - H + ly, r.ny) : 0;
    const int gz = wrap_any(Z0 - H + lz, r.nz);
    T* dst = c == 0 ? r.j[0] : (c == 1 ? r.j[1] : r.j[2]);
    atomicAdd(dst + (long long)gz * nxy + (long long)gy * r.nx + gx, v);
  }
  // 6. kinetic energy and particle count of the step (FP64 across the block and the grid)
  if (r.kin) {
    double kd = (double)kin;
    int nd = npush;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kd += __shfl_xor_sync(0xffffffffu, kd, o);
      nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    __shared__ double skin[HO_THREADS / 32];
    __shared__ int scn[HO_THREADS / 32];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
      skin[warp] = kd;
      scn[warp] = nd;
    }
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      long long c = 0;
      for (int w2 = 0; w2 < HO_THREADS / 32; ++w2) {
        t += skin[w2];
        c += scn[w2];
      }
      atomicAdd(r.kin, t);
      atomicAdd(r.kin + 1, (double)c);
    }
  }
}

template <typename T, int NDIM, int ORDER, int SCHEME>
__global__ void __launch_bounds__(HO_THREADS) k_push_ho(const __grid_constant__ RunDev<T> r) {
  using G = HoGeom<T, NDIM, ORDER>;
  using TL = HoTile<T, NDIM>;
  constexpr int TX = TL::TX, TY = TL::TY, NCL = G::NCL, NW = G::NW, K0 = G::K0, H = G::H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sg = reinterpret_cast<T*>(smem_raw);
  T* sj = sg + 6 * G::GN;
  int* sn = reinterpret_cast<int*>(sj + 3 * G::JN);  // [species][cell] input counts
  int* scnt = sn + 2 * NCL;                          // [species][cell] output counts
  const int tid = threadIdx.x;
  const HoTileRef tr = ho_tile(r);
  const int X0 = tr.X0, Y0 = tr.Y0, Z0 = tr.Z0, wx = tr.wx, wy = tr.wy, wz = tr.wz;
  ho_prologue<T, NDIM, ORDER, SCHEME>(r, tr, sg, sj, sn, scnt);
  const bool has_w = r.in[0].w != nullptr, has_id = r.in[0].id != nullptr;
  T kin = T(0);
  int npush = 0;
  // 3. one thread per cell, the cell's particles in turn
  for (int cl = tid; cl < NCL; cl += HO_THREADS) {
    const int lx = cl % TX, ly = (cl / TX) % TY, lz = cl / (TX * TY);
    const int gi = X0 + lx, gj = Y0 + ly, gk = Z0 + lz;
    const int cell = (gk * r.ny + gj) * r.nx + gi;
    for (int s = 0; s < 2; ++s) {
      const SpeciesBuf<T>& pin = s ? r.in[1] : r.in[0];
      const SpeciesBuf<T>& pout = s ? r.out[1] : r.out[0];
      const T qs = s ? T(1) : T(-1);
      const int n = sn[s * NCL + cl];
      for (int j = 0; j < n; ++j) {
        const long long slot = (long long)cell * r.cap + j;
        const T ox = pin.ox[slot], oy = NDIM == 3 ? pin.oy[slot] : T(0), oz = pin.oz[slot];
        T ux = pin.dux[slot], uy = pin.duy[slot], uz = pin.duz[slot];
        const T w = has_w ? pin.w[slot] : r.wconst;
        const unsigned id = has_id ? pin.id[slot] : 0u;
        // gather
        T F[6];
        gather6<T, NDIM, ORDER, SCHEME>(sg, lx, ly, lz, ox, oy, oz, F);
        // relativistic Boris, momenta relative to the drift u0 z_hat
        const T h = qs * r.hq;
        const T mx = ux + h * F[0], my = uy + h * F[1], mz = uz + h * F[2];
        const T Mz = r.u0 + mz;
        const T ig = T(1) / sqrt(T(1) + mx * mx + my * my + Mz * Mz);
        const T tx = h * F[3] * ig, ty = h * F[4] * ig, tz = h * F[5] * ig;
        const T sf = T(2) / (T(1) + tx * tx + ty * ty + tz * tz);
        const T sx = sf * tx, sy = sf * ty, sz = sf * tz;
        const T qx = mx + (my * tz - Mz * ty);
        const T qy = my + (Mz * tx - mx * tz);
        const T qz = Mz + (mx * ty - my * tx);
        ux = mx + (qy * sz - qz * sy) + h * F[0];
        uy = my + (qz * sx - qx * sz) + h * F[1];
        uz = mz + (qx * sy - qy * sx) + h * F[2];
        const T Uz = r.u0 + uz;
        const T u2 = ux * ux + uy * uy + Uz * Uz;
        const T gam = sqrt(T(1) + u2);
        const T ign = T(1) / gam;
        kin += w * u2 / (gam + T(1));
        ++npush;
        T ddx = r.dtdx * ux * ign, ddy = NDIM == 3 ? r.dtdy * uy * ign : T(0), ddz = r.dtdz * Uz * ign;
        T vy = uy * ign;
        if (!(ddx > T(-1) && ddx < T(1) && ddy > T(-1) && ddy < T(1) && ddz > T(-1) && ddz < T(1))) {
          flag_error(r.err, ERR_NONFINITE);
          ddx = ddy = ddz = T(0);
          ux = uy = uz = T(0);
          vy = T(0);  // nothing non-finite reaches the current
        }
        // Esirkepov on the window nodes K0 .. K0 + NW - 1 of the start cell
        T S0x[NW], dSx[NW], S0y[NW], dSy[NW], S0z[NW], dSz[NW];
#pragma unroll
        for (int a = 0; a < NW; ++a) {
          const T node = T(K0 + a);
          S0x[a] = bspl(ORDER, node - ox);
          dSx[a] = shape_change(ORDER, node - ox, ddx);
          S0z[a] = bspl(ORDER, node - oz);
          dSz[a] = shape_change(ORDER, node - oz, ddz);
          if (NDIM == 3) {
            S0y[a] = bspl(ORDER, node - oy);
            dSy[a] = shape_change(ORDER, node - oy, ddy);
          } else {
            S0y[a] = T(0);
            dSy[a] = T(0);
          }
        }
        const T qw = qs * w;
        // window node a of the start cell is current-tile index (cell + K0 + a) + H
        const int bx = lx + K0 + H, by = NDIM == 3 ? ly + K0 + H : 0, bz = lz + K0 + H;
        if (NDIM == 2) {
          const T cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vy * r.jfy2d;
          T Tx[NW], Tz[NW];
#pragma unroll
          for (int a = 0; a < NW; ++a) {
            Tx[a] = S0x[a] + T(0.5) * dSx[a];
            Tz[a] = S0z[a] + T(0.5) * dSz[a];
          }
          // Jx(i+1/2, k): running sum over the x window
#pragma unroll
          for (int b = 0; b < NW; ++b) {
            T acc = T(0);
#pragma unroll
            for (int a = 0; a < NW - 1; ++a) {
              acc += dSx[a];
              const T v = cx * acc * Tz[b];
              if (v != T(0)) atomicAdd(sj + (bz + b) * G::JX + bx + a, v);
            }
          }
          // Jz(i, k+1/2): running sum over the z window
#pragma unroll
          for (int a = 0; a < NW; ++a) {
            T acc = T(0);
#pragma unroll
            for (int b = 0; b < NW - 1; ++b) {
              acc += dSz[b];
              const T v = cz * acc * Tx[a];
              if (v != T(0)) atomicAdd(sj + 2 * G::JN + (bz + b) * G::JX + bx + a, v);
            }
          }
          // Jy(i, k): out-of-plane weight Tx Tz + dSx dSz / 12
#pragma unroll
          for (int b = 0; b < NW; ++b)
#pragma unroll
            for (int a = 0; a < NW; ++a) {
              const T v = cy * (Tx[a] * Tz[b] + dSx[a] * dSz[b] * T(1.0 / 12.0));
              if (v != T(0)) atomicAdd(sj + G::JN + (bz + b) * G::JX + bx + a, v);
            }
        } else {
          T Tx[NW], Ty[NW], Tz[NW];
#pragma unroll
          for (int a = 0; a < NW; ++a) {
            Tx[a] = S0x[a] + T(0.5) * dSx[a];
            Ty[a] = S0y[a] + T(0.5) * dSy[a];
            Tz[a] = S0z[a] + T(0.5) * dSz[a];
          }
          const T cxq = qw * r.jfx, cyq = qw * r.jfy, czq = qw * r.jfz;
          // J_axis: running sum along the axis of dS times the transverse weight
          // T1 T2 + dS1 dS2 / 12 over the other two directions
          for (int t2 = 0; t2 < NW; ++t2)
            for (int t1 = 0; t1 < NW; ++t1) {
              const T wx_ = Ty[t1] * Tz[t2] + dSy[t1] * dSz[t2] * T(1.0 / 12.0);  // Jx: (y, z) = (t1, t2)
              const T wy_ = Tx[t1] * Tz[t2] + dSx[t1] * dSz[t2] * T(1.0 / 12.0);  // Jy: (x, z) = (t1, t2)
              const T wz_ = Tx[t1] * Ty[t2] + dSx[t1] * dSy[t2] * T(1.0 / 12.0);  // Jz: (x, y) = (t1, t2)
              T ax_ = T(0), ay_ = T(0), az_ = T(0);
              for (int a = 0; a < NW - 1; ++a) {
                ax_ += dSx[a];
                ay_ += dSy[a];
                az_ += dSz[a];
                const T vx = cxq * ax_ * wx_, vyv = cyq * ay_ * wy_, vz = czq * az_ * wz_;
                if (vx != T(0)) atomicAdd(sj + ((bz + t2) * G::JY + by + t1) * G::JX + bx + a, vx);
                if (vyv != T(0)) atomicAdd(sj + G::JN + ((bz + t2) * G::JY + by + a) * G::JX + bx + t1, vyv);
                if (vz != T(0)) atomicAdd(sj + 2 * G::JN + ((bz + a) * G::JY + by + t2) * G::JX + bx + t1, vz);
              }
            }
        }
        // new cell and offsets
        auto fold = [](T o, T d, int& sh) -> T {
          const T t = o + d;
          sh = t < T(0) ? -1 : (t >= T(1) ? 1 : 0);
          T no = t - T(sh);
          if (no >= T(1)) {  // rounding of t - sh
            no = T(0);
            sh += 1;
          }
          if (no < T(0)) no = T(0);
          return no;
        };
        int shx, shy = 0, shz;
        const T nox = fold(ox, ddx, shx);
        const T noy = NDIM == 3 ? fold(oy, ddy, shy) : T(0);
        const T noz = fold(oz, ddz, shz);
        const int nlx = lx + shx, nly = ly + shy, nlz = lz + shz;
        if (nlx >= 0 && nlx < wx && nly >= 0 && nly < wy && nlz >= 0 && nlz < wz) {
          const int ncl = (nlz * TY + nly) * TX + nlx;
          const int jj = atomicAdd(scnt + s * NCL + ncl, 1);
          const int dcell = ((Z0 + nlz) * r.ny + Y0 + nly) * r.nx + X0 + nlx;
          if (jj < r.cap) {
            const long long o = (long long)dcell * r.cap + jj;
            pout.ox[o] = nox;
            if (NDIM == 3) pout.oy[o] = noy;
            pout.oz[o] = noz;
            pout.dux[o] = ux;
            pout.duy[o] = uy;
            pout.duz[o] = uz;
            if (has_w) pout.w[o] = w;
            if (has_id) pout.id[o] = id;
          } else {  // bin full: on through the leaver list (k_migrate spills it if still full)
            const long long o = atomicAdd(r.lv_count, 1);
            if (o < r.lv_cap) list_put(r.lv, o, dcell * 2 + s, nox, noy, noz, ux, uy, uz, w, id);
            else flag_error(r.err, ERR_OVERFLOW);
          }
        } else {  // to another tile: the leaver list (inserted by k_migrate)
          const int ni = wrap_any(gi + shx, r.nx), nj = NDIM == 3 ? wrap_any(gj + shy, r.ny) : 0;
          const int nk = wrap_any(gk + shz, r.nz);
          const long long o = atomicAdd(r.lv_count, 1);
          if (o < r.lv_cap) {
            r.lv.key[o] = ((nk * r.ny + nj) * r.nx + ni) * 2 + s;
            r.lv.ox[o] = nox;
            if (NDIM == 3) r.lv.oy[o] = noy;
            r.lv.oz[o] = noz;
            r.lv.dux[o] = ux;
            r.lv.duy[o] = uy;
            r.lv.duz[o] = uz;
            if (has_w) r.lv.w[o] = w;
            if (has_id) r.lv.id[o] = id;
          } else {
            flag_error(r.err, ERR_OVERFLOW);
          }
        }
      }
    }
  }
  ho_epilogue<T, NDIM, ORDER>(r, tr, sj, scnt, kin, npush);
}

// 2D, one warp per cell: lanes take the cell's particles (consecutive slots, both species), so the
// loads are coalesced and every lane's Esirkepov window is the cell's window (nodes K0 .. K0+NW-1
// per direction, which holds any move of less than a cell). The NV window sums are reduced over
// the warp in chunks of 32 by a butterfly transpose (lane L ends with the warp's total of entry L
// of the chunk) and added to the tile's current with one shared-memory atomic per lane and chunk.
template <typename T, int ORDER, int SCHEME>
__global__ void __launch_bounds__(HO_THREADS) k_push_ho_w2(const __grid_constant__ RunDev<T> r) {
  using G = HoGeom<T, 2, ORDER>;
  constexpr int TX = HoTile<T, 2>::TX, NCL = G::NCL, NW = G::NW, K0 = G::K0, H = G::H;
  constexpr int NVX = (NW - 1) * NW, NVZ = NW * (NW - 1), NVY = NW * NW, NV = NVX + NVZ + NVY;
  constexpr int NCH = (NV + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sg = reinterpret_cast<T*>(smem_raw);
  T* sj = sg + 6 * G::GN;
  int* sn = reinterpret_cast<int*>(sj + 3 * G::JN);
  int* scnt = sn + 2 * NCL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const HoTileRef tr = ho_tile(r);
  const int X0 = tr.X0, Z0 = tr.Z0, wx = tr.wx, wz = tr.wz;
  ho_prologue<T, 2, ORDER, SCHEME>(r, tr, sg, sj, sn, scnt);
  const bool has_w = r.in[0].w != nullptr, has_id = r.in[0].id != nullptr;
  T kin = T(0);
  int npush = 0;
  for (int cl = warp; cl < NCL; cl += HO_THREADS / 32) {
    const int lx = cl % TX, lz = cl / TX;
    const int gi = X0 + lx, gk = Z0 + lz;
    const int cell = gk * r.nx + gi;
    const int n0 = sn[cl], ntot = n0 + sn[NCL + cl];
    const int bx = lx + K0 + H, bz = lz + K0 + H;  // current-tile index of window node 0
    for (int base = 0; base < ntot; base += 32) {
      const int idx = base + lane;
      const bool valid = idx < ntot;
      const int s = idx >= n0 ? 1 : 0;
      const int j = s ? idx - n0 : idx;
      const SpeciesBuf<T>& pin = s ? r.in[1] : r.in[0];
      T ox = T(0.5), oz = T(0.5), ux = T(0), uy = T(0), uz = T(0), w = T(0);
      unsigned id = 0u;
      if (valid) {
        const long long slot = (long long)cell * r.cap + j;
        ox = pin.ox[slot];
        oz = pin.oz[slot];
        ux = pin.dux[slot];
        uy = pin.duy[slot];
        uz = pin.duz[slot];
        w = has_w ? pin.w[slot] : r.wconst;
        if (has_id) id = pin.id[slot];
      }
      const T qs = s ? T(1) : T(-1);
      // gather and relativistic Boris (momenta relative to the drift u0 z_hat)
      T F[6];
      gather6<T, 2, ORDER, SCHEME>(sg, lx, 0, lz, ox, T(0), oz, F);
      const T h = qs * r.hq;
      const T mx = ux + h * F[0], my = uy + h * F[1], mz = uz + h * F[2];
      const T Mz = r.u0 + mz;
      const T ig = T(1) / sqrt(T(1) + mx * mx + my * my + Mz * Mz);
      const T tx = h * F[3] * ig, ty = h * F[4] * ig, tz = h * F[5] * ig;
      const T sf = T(2) / (T(1) + tx * tx + ty * ty + tz * tz);
      const T sx = sf * tx, sy = sf * ty, sz = sf * tz;
      const T qx = mx + (my * tz - Mz * ty);
      const T qy = my + (Mz * tx - mx * tz);
      const T qz = Mz + (mx * ty - my * tx);
      ux = mx + (qy * sz - qz * sy) + h * F[0];
      uy = my + (qz * sx - qx * sz) + h * F[1];
      uz = mz + (qx * sy - qy * sx) + h * F[2];
      const T Uz = r.u0 + uz;
      const T u2 = ux * ux + uy * uy + Uz * Uz;
      const T gam = sqrt(T(1) + u2);
      const T ign = T(1) / gam;
      if (valid) {
        kin += w * u2 / (gam + T(1));
        ++npush;
      }
      T ddx = r.dtdx * ux * ign, ddz = r.dtdz * Uz * ign;
      T vy = uy * ign;
      if (valid && !(ddx > T(-1) && ddx < T(1) && ddz > T(-1) && ddz < T(1))) {
        flag_error(r.err, ERR_NONFINITE);
        ddx = ddz = T(0);
        ux = uy = uz = T(0);
        vy = T(0);  // nothing non-finite reaches the current
      }
      if (!valid) ddx = ddz = T(0);
      // Esirkepov on the cell's window
      T S0x[NW], dSx[NW], S0z[NW], dSz[NW], Tx[NW], Tz[NW];
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        const T node = T(K0 + a);
        S0x[a] = bspl(ORDER, node - ox);
        dSx[a] = shape_change(ORDER, node - ox, ddx);
        S0z[a] = bspl(ORDER, node - oz);
        dSz[a] = shape_change(ORDER, node - oz, ddz);
        Tx[a] = S0x[a] + T(0.5) * dSx[a];
        Tz[a] = S0z[a] + T(0.5) * dSz[a];
      }
      T PX[NW - 1], PZ[NW - 1];  // running sums of dS (the last, over the whole window, is 0)
      PX[0] = dSx[0];
      PZ[0] = dSz[0];
#pragma unroll
      for (int a = 1; a < NW - 1; ++a) {
        PX[a] = PX[a - 1] + dSx[a];
        PZ[a] = PZ[a - 1] + dSz[a];
      }
      const T qw = valid ? qs * w : T(0);
      const T cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vy * r.jfy2d;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        T v[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int i = ch * 32 + t;
          if (i < NVX) {  // Jx(a + 1/2, b): i = b (NW - 1) + a
            v[t] = cx * PX[i % (NW - 1)] * Tz[i / (NW - 1)];
          } else if (i < NVX + NVZ) {  // Jz(a, b + 1/2): i - NVX = a (NW - 1) + b
            const int k = i - NVX;
            v[t] = cz * PZ[k % (NW - 1)] * Tx[k / (NW - 1)];
          } else if (i < NV) {  // Jy(a, b): i - NVX - NVZ = b NW + a
            const int k = i - NVX - NVZ;
            v[t] = cy * (Tx[k % NW] * Tz[k / NW] + dSx[k % NW] * dSz[k / NW] * T(1.0 / 12.0));
          } else {
            v[t] = T(0);
          }
        }
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) {
          const bool up = (lane & sh) != 0;
#pragma unroll
          for (int q = 0; q < sh; ++q) {
            const T send = up ? v[q] : v[q + sh];
            const T keep = up ? v[q + sh] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
          }
        }
        const int i = ch * 32 + lane;
        if (i < NV && v[0] != T(0)) {
          int comp, a, b;
          if (i < NVX) {
            comp = 0;
            a = i % (NW - 1);
            b = i / (NW - 1);
          } else if (i < NVX + NVZ) {
            comp = 2;
            a = (i - NVX) / (NW - 1);
            b = (i - NVX) % (NW - 1);
          } else {
            comp = 1;
            a = (i - NVX - NVZ) % NW;
            b = (i - NVX - NVZ) / NW;
          }
          atomicAdd(sj + comp * G::JN + (bz + b) * G::JX + bx + a, v[0]);
        }
      }
      // new cell and offsets; rebin
      int shx, shz;
      T nox = ox + ddx, noz = oz + ddz;
      shx = nox < T(0) ? -1 : (nox >= T(1) ? 1 : 0);
      shz = noz < T(0) ? -1 : (noz >= T(1) ? 1 : 0);
      nox -= T(shx);
      noz -= T(shz);
      if (nox >= T(1)) { nox = T(0); shx += 1; }
      if (noz >= T(1)) { noz = T(0); shz += 1; }
      if (nox < T(0)) nox = T(0);
      if (noz < T(0)) noz = T(0);
      const int nlx = lx + shx, nlz = lz + shz;
      const bool stay = valid && nlx >= 0 && nlx < wx && nlz >= 0 && nlz < wz;
      const bool leave = valid && !stay;
      const int dkey = stay ? ((nlz * TX + nlx) * 2 + s) : -1 - lane;
      const unsigned peers = __match_any_sync(0xffffffffu, dkey);
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int slot_base = 0;
      if (stay && lane == leader) slot_base = atomicAdd(scnt + s * NCL + (dkey >> 1), __popc(peers));
      slot_base = __shfl_sync(0xffffffffu, slot_base, leader);
      // a full destination bin sends the particle on through the leaver list too (k_migrate spills
      // it if the bin is still full there)
      const bool full = stay && slot_base + rank >= r.cap;
      const unsigned lmask = __ballot_sync(0xffffffffu, leave || full);
      int lbase = 0;
      if (lmask) {
        const int ll = __ffs(lmask) - 1;
        if (lane == ll) lbase = atomicAdd(r.lv_count, __popc(lmask));
        lbase = __shfl_sync(0xffffffffu, lbase, ll);
      }
      if (stay) {
        const SpeciesBuf<T>& pout = s ? r.out[1] : r.out[0];
        const int jj = slot_base + rank;
        const int dcell = (Z0 + nlz) * r.nx + X0 + nlx;
        if (!full) {
          const long long o = (long long)dcell * r.cap + jj;
          pout.ox[o] = nox;
          pout.oz[o] = noz;
          pout.dux[o] = ux;
          pout.duy[o] = uy;
          pout.duz[o] = uz;
          if (has_w) pout.w[o] = w;
          if (has_id) pout.id[o] = id;
        } else {
          const long long o = lbase + __popc(lmask & ((1u << lane) - 1u));
          if (o < r.lv_cap) list_put(r.lv, o, dcell * 2 + s, nox, T(0), noz, ux, uy, uz, w, id);
          else flag_error(r.err, ERR_OVERFLOW);
        }
      } else if (leave) {
        const long long o = lbase + __popc(lmask & ((1u << lane) - 1u));
        if (o < r.lv_cap) {
          const int ni = wrap_any(gi + shx, r.nx), nk = wrap_any(gk + shz, r.nz);
          r.lv.key[o] = (nk * r.nx + ni) * 2 + s;
          r.lv.ox[o] = nox;
          r.lv.oz[o] = noz;
          r.lv.dux[o] = ux;
          r.lv.duy[o] = uy;
          r.lv.duz[o] = uz;
          if (has_w) r.lv.w[o] = w;
          if (has_id) r.lv.id[o] = id;
        } else {
          flag_error(r.err, ERR_OVERFLOW);
        }
      }
    }
  }
  ho_epilogue<T, 2, ORDER>(r, tr, sj, scnt, kin, npush);
}

// ---------------------------------------------------------------------------------------------
// Spilled particles: those whose destination bin was full when they were inserted wait in the
// spill list. One thread per spilled particle runs the step of the tile kernels on it (the same
// gather rule, Boris push, move and Esirkepov deposit), with the field copies read from global
// memory and the current added by global atomics, and hands it to the leaver list, from which
// k_migrate inserts it (or spills it again while its bin is still full). Nothing is dropped; the
// host grows the bins at its next synchronising call, so the list stays short.
// ---------------------------------------------------------------------------------------------

// Field copy at integer node (x, y, z) of the periodic grid, for a component with staggers
// (sx, sy, sz); for the momentum-conserving gather the average from the component's Yee location to
// the node, formed in the order of the tile prologue (x, then y, then z; upper neighbour first).
template <typename T, int NDIM>
__device__ __noinline__ T node_value(const T* g, const RunDev<T>& r, int scheme, int sx, int sy, int sz, int x, int y,
                                     int z) {
  const long long nxy = (long long)r.nx * r.ny;
  auto at = [&](int a, int b, int c) -> T {
    return g[(long long)wrap_any(c, r.nz) * nxy + (long long)(NDIM == 3 ? wrap_any(b, r.ny) : 0) * r.nx +
             wrap_any(a, r.nx)];
  };
  if (scheme != 2) return at(x, y, z);
  if (NDIM == 2) sy = 0;
  T v[2][2];  // [z offset][y offset], x already averaged
#pragma unroll 1
  for (int dz = 0; dz <= sz; ++dz)
#pragma unroll 1
    for (int dy = 0; dy <= sy; ++dy)
      v[dz][dy] = sx ? T(0.5) * (at(x, y - dy, z - dz) + at(x - 1, y - dy, z - dz)) : at(x, y - dy, z - dz);
  if (sy) {
    v[0][0] = T(0.5) * (v[0][0] + v[0][1]);
    if (sz) v[1][0] = T(0.5) * (v[1][0] + v[1][1]);
  }
  return sz ? T(0.5) * (v[0][0] + v[1][0]) : v[0][0];
}

// Component c of the gather at offsets (ox, oy, oz) in cell (gi, gj, gk), from global memory (the
// weights and node rule of gather_comp, with the order and scheme given at run time).
template <typename T, int NDIM>
__device__ __noinline__ T gather_global(const T* g, const RunDev<T>& r, int order, int scheme, int c, int gi, int gj,
                                       int gk, T ox, T oy, T oz) {
  const int stx = stag_ho(c, 0), sty = stag_ho(c, 1), stz = stag_ho(c, 2);
  const int SX = scheme == 2 ? 0 : stx, SY = scheme == 2 ? 0 : sty, SZ = scheme == 2 ? 0 : stz;
  const int OX = scheme == 0 ? order - SX : order, OZ = scheme == 0 ? order - SZ : order;
  const int OY = NDIM == 3 ? (scheme == 0 ? order - SY : order) : 0;
  int fx, fy = 0, fz;
  T wx[4], wy[4] = {T(1), T(0), T(0), T(0)}, wz[4];
  gweights(ox, SX, OX, fx, wx);
  if (NDIM == 3) gweights(oy, SY, OY, fy, wy);
  gweights(oz, SZ, OZ, fz, wz);
  T acc = T(0);
#pragma unroll 1
  for (int c3 = 0; c3 <= OZ; ++c3) {
#pragma unroll 1
    for (int c2 = 0; c2 <= OY; ++c2) {
      T row = T(0);
#pragma unroll 1
      for (int c1 = 0; c1 <= OX; ++c1)
        row += wx[c1] * node_value<T, NDIM>(g, r, scheme, stx, sty, stz, gi + fx + c1, gj + fy + c2, gk + fz + c3);
      acc += wz[c3] * wy[c2] * row;
    }
  }
  return acc;
}

template <typename T, int NDIM>
__device__ __forceinline__ void push_spill_body(const RunDev<T>& r, int order, int scheme, int bid, int nblk) {
  constexpr int NWMAX = 6;
  const int NW = order == 3 ? 6 : 4, K0 = order == 3 ? -2 : -1;  // deposit window (as HoGeom)
  const int tid = threadIdx.x;
  if (bid == 0 && tid == 0) *r.sp_out = 0;  // this step's k_migrate spills into a fresh list
  const long long n = min((long long)*r.sp_in, r.sp_cap);
  if (n == 0) return;
  const long long nxy = (long long)r.nx * r.ny;
  T kin = T(0);
  int npush = 0;
  for (long long i = (long long)bid * blockDim.x + tid; i < n; i += (long long)nblk * blockDim.x) {
    const int key = r.sp.key[i];
    const int s = key & 1;
    const int cell = key >> 1;  // cells < 2^30
    const int gi = cell % r.nx, gj = (cell / r.nx) % r.ny, gk = (int)(cell / nxy);
    const T ox = r.sp.ox[i], oy = NDIM == 3 ? r.sp.oy[i] : T(0), oz = r.sp.oz[i];
    T ux = r.sp.dux[i], uy = r.sp.duy[i], uz = r.sp.duz[i];
    const T w = r.sp.w ? r.sp.w[i] : r.wconst;
    const unsigned id = r.sp.id ? r.sp.id[i] : 0u;
    const T qs = s ? T(1) : T(-1);
    T F[6];
#pragma unroll 1
    for (int c = 0; c < 6; ++c) F[c] = gather_global<T, NDIM>(r.g[c], r, order, scheme, c, gi, gj, gk, ox, oy, oz);
    // relativistic Boris, momenta relative to the drift u0 z_hat
    const T h = qs * r.hq;
    const T mx = ux + h * F[0], my = uy + h * F[1], mz = uz + h * F[2];
    const T Mz = r.u0 + mz;
    const T ig = T(1) / sqrt(T(1) + mx * mx + my * my + Mz * Mz);
    const T tx = h * F[3] * ig, ty = h * F[4] * ig, tz = h * F[5] * ig;
    const T sf = T(2) / (T(1) + tx * tx + ty * ty + tz * tz);
    const T sx = sf * tx, sy = sf * ty, sz = sf * tz;
    const T qx = mx + (my * tz - Mz * ty);
    const T qy = my + (Mz * tx - mx * tz);
    const T qz = Mz + (mx * ty - my * tx);
    ux = mx + (qy * sz - qz * sy) + h * F[0];
    uy = my + (qz * sx - qx * sz) + h * F[1];
    uz = mz + (qx * sy - qy * sx) + h * F[2];
    const T Uz = r.u0 + uz;
    const T u2 = ux * ux + uy * uy + Uz * Uz;
    const T gam = sqrt(T(1) + u2);
    const T ign = T(1) / gam;
    kin += w * u2 / (gam + T(1));
    ++npush;
    T ddx = r.dtdx * ux * ign, ddy = NDIM == 3 ? r.dtdy * uy * ign : T(0), ddz = r.dtdz * Uz * ign;
    T vy = uy * ign;
    if (!(ddx > T(-1) && ddx < T(1) && ddy > T(-1) && ddy < T(1) && ddz > T(-1) && ddz < T(1))) {
      flag_error(r.err, ERR_NONFINITE);
      ddx = ddy = ddz = T(0);
      ux = uy = uz = T(0);
      vy = T(0);  // nothing non-finite reaches the current
    }
    // Esirkepov on the window nodes K0 .. K0 + NW - 1 of the start cell, straight into J
    T S0x[NWMAX], dSx[NWMAX], dSy[NWMAX], dSz[NWMAX], Tx[NWMAX], Ty[NWMAX], Tz[NWMAX];
    int xs[NWMAX], ys[NWMAX], zs[NWMAX];  // periodic indices of the window nodes
#pragma unroll 1
    for (int a = 0; a < NW; ++a) {
      const T node = T(K0 + a);
      S0x[a] = bspl(order, node - ox);
      dSx[a] = shape_change(order, node - ox, ddx);
      Tx[a] = S0x[a] + T(0.5) * dSx[a];
      const T s0z = bspl(order, node - oz);
      dSz[a] = shape_change(order, node - oz, ddz);
      Tz[a] = s0z + T(0.5) * dSz[a];
      if (NDIM == 3) {
        const T s0y = bspl(order, node - oy);
        dSy[a] = shape_change(order, node - oy, ddy);
        Ty[a] = s0y + T(0.5) * dSy[a];
      } else {
        dSy[a] = T(0);
        Ty[a] = T(0);
      }
      xs[a] = wrap_any(gi + K0 + a, r.nx);
      ys[a] = NDIM == 3 ? wrap_any(gj + K0 + a, r.ny) : 0;
      zs[a] = wrap_any(gk + K0 + a, r.nz);
    }
    const T qw = qs * w;
    T* const J0 = r.j[0];
    T* const J1 = r.j[1];
    T* const J2 = r.j[2];
    auto idx = [&](int x, int y, int z) -> long long { return (long long)z * nxy + (long long)y * r.nx + x; };
    if (NDIM == 2) {
      const T cx = qw * r.jfx, cz = qw * r.jfz, cy = qw * vy * r.jfy2d;
#pragma unroll 1
      for (int b = 0; b < NW; ++b) {  // Jx(a + 1/2, b): running sum over the x window
        T acc = T(0);
#pragma unroll 1
        for (int a = 0; a < NW - 1; ++a) {
          acc += dSx[a];
          const T v = cx * acc * Tz[b];
          if (v != T(0)) atomicAdd(J0 + idx(xs[a], 0, zs[b]), v);
        }
      }
#pragma unroll 1
      for (int a = 0; a < NW; ++a) {  // Jz(a, b + 1/2): running sum over the z window
        T acc = T(0);
#pragma unroll 1
        for (int b = 0; b < NW - 1; ++b) {
          acc += dSz[b];
          const T v = cz * acc * Tx[a];
          if (v != T(0)) atomicAdd(J2 + idx(xs[a], 0, zs[b]), v);
        }
      }
#pragma unroll 1
      for (int b = 0; b < NW; ++b)  // Jy(a, b): out-of-plane weight Tx Tz + dSx dSz / 12
#pragma unroll 1
        for (int a = 0; a < NW; ++a) {
          const T v = cy * (Tx[a] * Tz[b] + dSx[a] * dSz[b] * T(1.0 / 12.0));
          if (v != T(0)) atomicAdd(J1 + idx(xs[a], 0, zs[b]), v);
        }
    } else {
      const T cxq = qw * r.jfx, cyq = qw * r.jfy, czq = qw * r.jfz;
#pragma unroll 1
      for (int t2 = 0; t2 < NW; ++t2)
#pragma unroll 1
        for (int t1 = 0; t1 < NW; ++t1) {
          const T wx_ = Ty[t1] * Tz[t2] + dSy[t1] * dSz[t2] * T(1.0 / 12.0);  // Jx: (y, z) = (t1, t2)
          const T wy_ = Tx[t1] * Tz[t2] + dSx[t1] * dSz[t2] * T(1.0 / 12.0);  // Jy: (x, z) = (t1, t2)
          const T wz_ = Tx[t1] * Ty[t2] + dSx[t1] * dSy[t2] * T(1.0 / 12.0);  // Jz: (x, y) = (t1, t2)
          T ax_ = T(0), ay_ = T(0), az_ = T(0);
#pragma unroll 1
          for (int a = 0; a < NW - 1; ++a) {
            ax_ += dSx[a];
            ay_ += dSy[a];
            az_ += dSz[a];
            const T vx = cxq * ax_ * wx_, vyv = cyq * ay_ * wy_, vz = czq * az_ * wz_;
            if (vx != T(0)) atomicAdd(J0 + idx(xs[a], ys[t1], zs[t2]), vx);
            if (vyv != T(0)) atomicAdd(J1 + idx(xs[t1], ys[a], zs[t2]), vyv);
            if (vz != T(0)) atomicAdd(J2 + idx(xs[t1], ys[t2], zs[a]), vz);
          }
        }
    }
    // new cell and offsets, then on to k_migrate through the leaver list
    auto fold = [](T o, T d, int& sh) -> T {
      const T t = o + d;
      sh = t < T(0) ? -1 : (t >= T(1) ? 1 : 0);
      T no = t - T(sh);
      if (no >= T(1)) {  // rounding of t - sh
        no = T(0);
        sh += 1;
      }
      if (no < T(0)) no = T(0);
      return no;
    };
    int shx, shy = 0, shz;
    const T nox = fold(ox, ddx, shx);
    const T noy = NDIM == 3 ? fold(oy, ddy, shy) : T(0);
    const T noz = fold(oz, ddz, shz);
    const int ni = wrap_any(gi + shx, r.nx), nj = NDIM == 3 ? wrap_any(gj + shy, r.ny) : 0;
    const int nk = wrap_any(gk + shz, r.nz);
    const long long o = atomicAdd(r.lv_count, 1);
    if (o < r.lv_cap) list_put(r.lv, o, ((nk * r.ny + nj) * r.nx + ni) * 2 + s, nox, noy, noz, ux, uy, uz, w, id);
    else flag_error(r.err, ERR_OVERFLOW);
  }
  // kinetic energy and particle count of the step (FP64, one atomic per warp)
  if (r.kin) {
    double kd = (double)kin;
    int nd = npush;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kd += __shfl_xor_sync(0xffffffffu, kd, o);
      nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    if ((tid & 31) == 0 && nd > 0) {
      atomicAdd(r.kin, kd);
      atomicAdd(r.kin + 1, (double)nd);
    }
  }
}

constexpr int SPILL_THREADS = 256;

template <typename T, int NDIM>
__global__ void __launch_bounds__(SPILL_THREADS) k_push_spill(const __grid_constant__ RunDev<T> r, int order,
                                                              int scheme) {
  pdl_wait();
  push_spill_body<T, NDIM>(r, order, scheme, blockIdx.x, gridDim.x);
}

// Many runs: run blockIdx.y (the batched step covers linear shapes).
template <typename T, int NDIM>
__global__ void __launch_bounds__(SPILL_THREADS) k_push_spill_batch(const RunDev<T>* __restrict__ runs, int scheme) {
  pdl_wait();
  push_spill_body<T, NDIM>(runs[blockIdx.y], 1, scheme, blockIdx.x, gridDim.x);
}

template <typename T, int NDIM, int ORDER, int SCHEME>
cudaError_t launch_ho_t(const RunDev<T>& r, cudaStream_t st) {
  using G = HoGeom<T, NDIM, ORDER>;
  const size_t sm = G::bytes();
  const int ntiles = r.ntx * r.nty * r.ntz;
  if (NDIM == 2) {  // one warp per cell
    cudaError_t e = ensure_dynamic_smem((const void*)k_push_ho_w2<T, ORDER, SCHEME>, sm);
    if (e != cudaSuccess) return e;
    if (ntiles > 0) k_push_ho_w2<T, ORDER, SCHEME><<<ntiles, HO_THREADS, sm, st>>>(r);
    return cudaGetLastError();
  }
  cudaError_t e = ensure_dynamic_smem((const void*)k_push_ho<T, NDIM, ORDER, SCHEME>, sm);
  if (e != cudaSuccess) return e;
  if (ntiles > 0) k_push_ho<T, NDIM, ORDER, SCHEME><<<ntiles, HO_THREADS, sm, st>>>(r);
  return cudaGetLastError();
}

template <typename T, int NDIM, int ORDER>
cudaError_t launch_ho_scheme(const RunDev<T>& r, int scheme, cudaStream_t st) {
  if (scheme == 0) return launch_ho_t<T, NDIM, ORDER, 0>(r, st);
  if (scheme == 1) return launch_ho_t<T, NDIM, ORDER, 1>(r, st);
  return launch_ho_t<T, NDIM, ORDER, 2>(r, st);
}

}  // namespace

template <typename T>
cudaError_t launch_push_ho(const RunDev<T>& r, int order, int scheme, cudaStream_t st) {
  if (!tiles_fit<HoTile>(r)) return cudaErrorInvalidValue;
  if (r.ndim == 2) return order == 3 ? launch_ho_scheme<T, 2, 3>(r, scheme, st) : launch_ho_scheme<T, 2, 1>(r, scheme, st);
  return order == 3 ? launch_ho_scheme<T, 3, 3>(r, scheme, st) : launch_ho_scheme<T, 3, 1>(r, scheme, st);
}
template cudaError_t launch_push_ho<float>(const RunDev<float>&, int, int, cudaStream_t);
template cudaError_t launch_push_ho<double>(const RunDev<double>&, int, int, cudaStream_t);

template <typename T>
cudaError_t launch_push_spill(const RunDev<T>& r, int order, int scheme, cudaStream_t st) {
  // a fixed grid (the count is on the device): every block exits at once when the list is empty
  constexpr int blocks = 152;
  if (r.ndim == 2) return launch_pdl(k_push_spill<T, 2>, dim3(blocks), dim3(SPILL_THREADS), 0, st, r, order, scheme);
  return launch_pdl(k_push_spill<T, 3>, dim3(blocks), dim3(SPILL_THREADS), 0, st, r, order, scheme);
}
template cudaError_t launch_push_spill<float>(const RunDev<float>&, int, int, cudaStream_t);
template cudaError_t launch_push_spill<double>(const RunDev<double>&, int, int, cudaStream_t);

template <typename T>
cudaError_t launch_push_spill_batch(const RunDev<T>* runs, int nruns, int ndim, int scheme, cudaStream_t st) {
  if (nruns <= 0) return cudaSuccess;
  const dim3 grid(152 / (nruns < 8 ? 1 : nruns / 8) + 1, (unsigned)nruns);
  if (ndim == 2) return launch_pdl(k_push_spill_batch<T, 2>, grid, dim3(SPILL_THREADS), 0, st, runs, scheme);
  return launch_pdl(k_push_spill_batch<T, 3>, grid, dim3(SPILL_THREADS), 0, st, runs, scheme);
}
template cudaError_t launch_push_spill_batch<float>(const RunDev<float>*, int, int, int, cudaStream_t);
template cudaError_t launch_push_spill_batch<double>(const RunDev<double>*, int, int, int, cudaStream_t);

}  // namespace picgb
