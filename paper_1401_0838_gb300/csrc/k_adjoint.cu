// Adjoint (reverse-mode) kernels of the 2D step: the transposes of the gather, Boris push, move
// and Esirkepov deposition for one particle per thread, the id-ordered particle tape, the seed of
// the final transverse field energy, and the Psi(D_z) transpose with the coefficient gradients.
//
// Forward step being differentiated (all passes linear in the fields except the particle ones):
//   G = Psi(D_z) F_filter E          gather copies (Sec. 2 last paragraph, Sec. 3 Eq. 6)
//   f_p = sum W(x_p) G               field gather, linear shapes (Sec. 2, Eq. 3-4)
//   u' = Boris(u, f_p)               relativistic Boris
//   x' = x + dt u'/gamma'            move
//   J = Esirkepov(x, x' - x, v'_y)   current deposition, shape change from the displacement
//   E, B <- Yee(E, B, F_filter J)    B half, E full, B half
// Reverse order per step: Yee^T (host: the curl kernels with negated coefficients), filter^T = the
// filter (symmetric taps), then k_adj_particles (this file), then copies^T = filter then Psi(D_z)
// (symmetric taps), the last fused with the coefficient gradient in k_adj_psi.
#include <climits>

#include "launch.h"

namespace picgb {

// ---------------------------------------------------------------------------------------------
// Tape: bins (current buffers) -> flat arrays indexed by particle id. With `seen` (one bit per id,
// zeroed by the caller) ids that are out of range or repeated raise ERR_IDS.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_tape(const __grid_constant__ RunDev<T> r, const __grid_constant__ FlatDev<T> f,
                                              unsigned long long* seen) {
  // eight lanes per (cell, species) bin, four bins per warp (bins hold about ppc particles)
  const long long cs = blockIdx.x * 32LL + (threadIdx.x >> 3);
  const long long cell = cs >> 1;
  if (cell >= r.ncell) return;
  const int s = (int)(cs & 1);
  const SpeciesBuf<T>& b = s ? r.in[1] : r.in[0];  // constant indices: no local copy of r
  const int n = min(b.cnt[cell], r.cap);
  for (int j = threadIdx.x & 7; j < n; j += 8) {
  const long long src = cell * r.cap + j;
  const unsigned id = b.id[src];
  if ((long long)id >= f.np) {
    flag_error(r.err, ERR_IDS);
    continue;
  }
  if (seen) {
    const unsigned long long bit = 1ull << (id & 63u);
    if (atomicOr(seen + (id >> 6), bit) & bit) flag_error(r.err, ERR_IDS);
  }
  f.cell[id] = (int)cell;
  f.species[id] = s;
  f.ox[id] = b.ox[src];
  if (f.oy) f.oy[id] = r.ndim == 3 ? b.oy[src] : T(0);
  f.oz[id] = b.oz[src];
  f.dux[id] = b.dux[src];
  f.duy[id] = b.duy[src];
  f.duz[id] = b.duz[src];
  if (f.w) f.w[id] = b.w ? b.w[src] : r.wconst;
  }
}

template <typename T>
cudaError_t launch_tape(const RunDev<T>& r, const FlatDev<T>& f, unsigned long long* seen, cudaStream_t st) {
  const long long blocks = (2 * r.ncell + 31) / 32;
  if (blocks > 0) k_tape<T><<<(unsigned)blocks, 256, 0, st>>>(r, f, seen);
  return cudaGetLastError();
}
template cudaError_t launch_tape<float>(const RunDev<float>&, const FlatDev<float>&, unsigned long long*,
                                        cudaStream_t);
template cudaError_t launch_tape<double>(const RunDev<double>&, const FlatDev<double>&, unsigned long long*,
                                         cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Seed: adjoint of the final fields for L = scale_w * W_perp, W_perp = 1/2 dV sum(Ex^2+Ey^2+Bx^2+By^2)
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_adj_seed(AdjSeedArgs<T> a) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= a.ncell) return;
  const T s = a.scale;
  a.lam[0][c] = s * a.f[0][c];
  a.lam[1][c] = s * a.f[1][c];
  a.lam[2][c] = T(0);
  a.lam[3][c] = s * a.f[3][c];
  a.lam[4][c] = s * a.f[4][c];
  a.lam[5][c] = T(0);
}

template <typename T>
cudaError_t launch_adj_seed(const AdjSeedArgs<T>& a, cudaStream_t st) {
  const long long blocks = (a.ncell + 255) / 256;
  if (blocks > 0) k_adj_seed<T><<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_adj_seed<float>(const AdjSeedArgs<float>&, cudaStream_t);
template cudaError_t launch_adj_seed<double>(const AdjSeedArgs<double>&, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Particle adjoint, 2D x-z, one particle per thread in id order.
// ---------------------------------------------------------------------------------------------
// Stagger of Ex, Ey, Ez, Bx, By, Bz along x and z (Yee, y-invariant).
__device__ __constant__ int kStagX[6] = {1, 0, 0, 0, 1, 1};
__device__ __constant__ int kStagZ[6] = {0, 0, 1, 1, 1, 0};

// Gather weights along one direction at cell-relative offset o in [0, 1): S1 on two nodes
// (weights 1-f, f; derivatives -1, +1 in o) or S0 on one node (derivative 0).
template <typename T>
struct Gw {
  int i0, i1;  // node indices (periodic)
  int fl;      // first node relative to the start cell
  T w0, w1;
  bool two;
};

// Periodic index of i in [-n, 2n).
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// nodes[k] = periodic index of start cell + k - 1, k = 0..3
template <typename T>
__device__ __forceinline__ Gw<T> gweights(T o, int st, int order, const int nodes[4]) {
  Gw<T> g;
  if (order == 1) {
    const T xs = st ? o - T(0.5) : o;
    const int fl = xs < T(0) ? -1 : 0;
    const T fr = xs - T(fl);
    g.i0 = fl < 0 ? nodes[0] : nodes[1];
    g.i1 = fl < 0 ? nodes[1] : nodes[2];
    g.fl = fl;
    g.w0 = T(1) - fr;
    g.w1 = fr;
    g.two = true;
  } else {
    const T xs = st ? o : o + T(0.5);  // the box of the node floor(x - st/2 + 1/2)
    const int fl = xs >= T(1) ? 1 : 0;
    g.i0 = g.i1 = fl ? nodes[2] : nodes[1];
    g.fl = fl;
    g.w0 = T(1);
    g.w1 = T(0);
    g.two = false;
  }
  return g;
}

// slope of S1(t) = max(0, 1 - |t|) on the pieces (-inf,-1], (-1,0], (0,1), [1,inf)
template <typename T>
__device__ __forceinline__ T s1_slope(T t) {
  return (t > T(-1) && t <= T(0)) ? T(1) : ((t > T(0) && t < T(1)) ? T(-1) : T(0));
}
__device__ __forceinline__ int s1_piece_d(double t) { return (t > -1.0) + (t > 0.0) + (t >= 1.0); }
__device__ __forceinline__ int s1_piece_d(float t) { return (t > -1.f) + (t > 0.f) + (t >= 1.f); }
template <typename T>
__device__ __forceinline__ T s1v(T t) {
  const T a = T(1) - (t < T(0) ? -t : t);
  return a > T(0) ? a : T(0);
}

// Shapes on the window nodes -1..2 of the start cell: S0 = S1(node - o), the change dS when the
// particle moves by d (from the displacement on one linear piece, else the difference), and the
// partial derivatives of both in o and d.
template <typename T>
struct Win {
  T S0[4], dS[4], dS0o[4], dSo[4], dSd[4];
};

template <typename T>
__device__ __forceinline__ void shape_win(T o, T d, Win<T>& w) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const T t0 = T(a - 1) - o, t1 = t0 - d;
    const T sl0 = s1_slope(t0), sl1 = s1_slope(t1);
    w.S0[a] = s1v(t0);
    w.dS0o[a] = -sl0;
    if (s1_piece_d(t0) == s1_piece_d(t1)) {
      w.dS[a] = sl0 * (-d);
      w.dSd[a] = -sl0;
      w.dSo[a] = T(0);
    } else {
      w.dS[a] = s1v(t1) - s1v(t0);
      w.dSd[a] = -sl1;
      w.dSo[a] = sl0 - sl1;
    }
  }
}

template <typename T>
__device__ __forceinline__ void atomic_add(T* p, T v) {
  atomicAdd(p, v);
}

constexpr int ADJ_THREADS = 128;

// Inclusive sum of v over the run of consecutive lanes that hold the same key (the run starts at
// lane `start`); the last lane of a run ends with the run's total. All 32 lanes take part.
template <typename T>
__device__ __forceinline__ T run_sum(T v, int start, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= start) v += t;
  }
  return v;
}

template <typename T, int SCHEME>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_particles(const __grid_constant__ AdjPartArgs<T> a) {
  // Consecutive ids start close together (the beam keeps its lattice order), so neighbouring lanes
  // mostly add into the same nodes of the copies' adjoint: each node's contributions are summed over
  // the run of lanes that share it, and the run's last lane adds the total to global memory.
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nx = a.nx, nz = a.nz;
  bool active = p < a.n;
  int cell = 0, s = 0;
  if (active) {
    cell = a.cell[p];
    s = a.species[p];
    if (cell < 0 || cell >= nx * nz || (s != 0 && s != 1)) {  // a particle the recomputed step lost
      flag_error(a.err, ERR_IDS);
      active = false;
      cell = 0;
      s = 0;
    }
  }
  const int ck = cell / nx, ci = cell - ck * nx;
  int ix[4], iz[4];  // periodic node indices of the start cell - 1 .. + 2
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ix[q] = wrap1(ci + q - 1, nx);
    iz[q] = wrap1(ck + q - 1, nz);
  }
  T lF[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  T ox = T(0), oz = T(0);
  if (active) {
  ox = a.ox[p];
  oz = a.oz[p];
  const T ux0 = a.dux[p], uy0 = a.duy[p], uz0 = a.duz[p];
  const T w = a.w ? a.w[p] : a.wconst;
  const T qs = s ? T(1) : T(-1);

  // 1. gather at x^n (recomputed) with the derivatives of each component in ox and oz
  T F[6], dFx[6], dFz[6];
  Gw<T> gx[6], gz[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int sx = kStagX[c], sz = kStagZ[c];
    gx[c] = gweights(ox, sx, SCHEME == 0 ? 1 - sx : 1, ix);
    gz[c] = gweights(oz, sz, SCHEME == 0 ? 1 - sz : 1, iz);
    const T* G0 = a.g[c] + gz[c].i0 * nx;  // 32-bit offsets: the launcher caps the cell count
    const T* G1 = a.g[c] + gz[c].i1 * nx;
    const T g00 = G0[gx[c].i0], g01 = G0[gx[c].i1], g10 = G1[gx[c].i0], g11 = G1[gx[c].i1];
    const T zx0 = gz[c].w0 * gx[c].w0, zx1 = gz[c].w0 * gx[c].w1, zx2 = gz[c].w1 * gx[c].w0, zx3 = gz[c].w1 * gx[c].w1;
    F[c] = zx0 * g00 + zx1 * g01 + zx2 * g10 + zx3 * g11;
    dFx[c] = gx[c].two ? gz[c].w0 * (g01 - g00) + gz[c].w1 * (g11 - g10) : T(0);
    dFz[c] = gz[c].two ? gx[c].w0 * (g10 - g00) + gx[c].w1 * (g11 - g01) : T(0);
  }

  // 2. Boris u^{n-1/2} -> u^{n+1/2} (recomputed; momenta relative to the drift u0 z_hat)
  const T h = qs * a.hq;
  const T mx = ux0 + h * F[0], my = uy0 + h * F[1], mz = uz0 + h * F[2];
  const T Mz = a.u0 + mz;
  const T gm = sqrt(T(1) + mx * mx + my * my + Mz * Mz);
  const T igm = T(1) / gm;
  const T tx = h * F[3] * igm, ty = h * F[4] * igm, tz = h * F[5] * igm;
  const T tt = tx * tx + ty * ty + tz * tz;
  const T den = T(1) + tt;
  const T iden = T(1) / den;
  const T sx = T(2) * tx * iden, sy = T(2) * ty * iden, sz = T(2) * tz * iden;
  const T px = mx + (my * tz - Mz * ty), py = my + (Mz * tx - mx * tz), pz = Mz + (mx * ty - my * tx);
  const T ux = mx + (py * sz - pz * sy) + h * F[0];
  const T uy = my + (pz * sx - px * sz) + h * F[1];
  const T uz = mz + (px * sy - py * sx) + h * F[2];
  const T Uz = a.u0 + uz;
  const T ux2 = ux * ux, uy2 = uy * uy, uz2 = Uz * Uz;
  const T gam = sqrt(T(1) + ux2 + uy2 + uz2);
  const T ig = T(1) / gam;
  const T vx = ux * ig, vy = uy * ig, vz = Uz * ig;
  const T ddx = a.dtdx * vx, ddz = a.dtdz * vz;

  // 3. Esirkepov transpose: lambda_J . J as a function of (ox, ddx, oz, ddz, vy)
  Win<T> wx, wz;
  shape_win(ox, ddx, wx);
  shape_win(oz, ddz, wz);
  const T qw = qs * w;
  const T cx = qw * a.jfx, cz = qw * a.jfz, cyc = qw * a.jfy2d;
  T gS0x[4] = {}, gdSx[4] = {}, gS0z[4] = {}, gdSz[4] = {};
  T Tx[4], Tz[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Tx[q] = wx.S0[q] + T(0.5) * wx.dS[q];
    Tz[q] = wz.S0[q] + T(0.5) * wz.dS[q];
  }
  T gTx[4] = {}, gTz[4] = {};
  // Jx on the edges i+1/2 of the window nodes -1..1 (the running sum closes to 0 at node 2)
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const T* row = a.lj[0] + iz[b] * nx;
    const T l0 = row[ix[0]], l1 = row[ix[1]], l2 = row[ix[2]];
    const T L2 = l2, L1 = l1 + l2, L0 = l0 + l1 + l2;  // suffix sums: dJ/dW over the edges at or right of a
    gdSx[0] += cx * Tz[b] * L0;
    gdSx[1] += cx * Tz[b] * L1;
    gdSx[2] += cx * Tz[b] * L2;
    gTz[b] += cx * (wx.dS[0] * L0 + wx.dS[1] * L1 + wx.dS[2] * L2);
  }
  // Jz on the edges k+1/2 of the window nodes -1..1
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T l0 = a.lj[2][iz[0] * nx + ix[q]];
    const T l1 = a.lj[2][iz[1] * nx + ix[q]];
    const T l2 = a.lj[2][iz[2] * nx + ix[q]];
    const T L2 = l2, L1 = l1 + l2, L0 = l0 + l1 + l2;
    gdSz[0] += cz * Tx[q] * L0;
    gdSz[1] += cz * Tx[q] * L1;
    gdSz[2] += cz * Tx[q] * L2;
    gTx[q] += cz * (wz.dS[0] * L0 + wz.dS[1] * L1 + wz.dS[2] * L2);
  }
  // Jy at the nodes, coefficient q w vy / dV, weight S0x S0z + dSx S0z/2 + S0x dSz/2 + dSx dSz/3,
  // which is Tx Tz + dSx dSz / 12 with T = S0 + dS/2
  T Aq[4] = {}, Bq[4] = {}, Cb[4] = {}, Db[4] = {};
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const T* row = a.lj[1] + iz[b] * nx;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T l = row[ix[q]];
      Aq[q] += l * Tz[b];
      Bq[q] += l * wz.dS[b];
      Cb[b] += l * Tx[q];
      Db[b] += l * wx.dS[q];
    }
  }
  T gcy = T(0);
  const T lvy = cyc * vy, k12 = T(1.0 / 12.0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    gcy += Tx[q] * Aq[q] + k12 * wx.dS[q] * Bq[q];
    gS0x[q] += lvy * Aq[q];
    gdSx[q] += lvy * (T(0.5) * Aq[q] + k12 * Bq[q]);
    gS0z[q] += lvy * Cb[q];
    gdSz[q] += lvy * (T(0.5) * Cb[q] + k12 * Db[q]);
  }
  gcy *= cyc;
  T lox_dep = T(0), lddx = T(0), loz_dep = T(0), lddz = T(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    gS0x[q] += gTx[q];
    gdSx[q] += T(0.5) * gTx[q];
    gS0z[q] += gTz[q];
    gdSz[q] += T(0.5) * gTz[q];
    lox_dep += gS0x[q] * wx.dS0o[q] + gdSx[q] * wx.dSo[q];
    lddx += gdSx[q] * wx.dSd[q];
    loz_dep += gS0z[q] * wz.dS0o[q] + gdSz[q] * wz.dSo[q];
    lddz += gdSz[q] * wz.dSd[q];
  }

  // 4. move transpose: x^{n+1} = x^n + d, d = (dt/dx) u / gamma
  const T lx1 = a.lox[p], lz1 = a.loz[p];
  lddx += lx1;
  lddz += lz1;
  const T gxv = lddx * a.dtdx, gyv = gcy, gzv = lddz * a.dtdz;  // adjoints of vx, vy, vz
  // d(u_i/gamma)/du_j = (delta_ij (1 + |u|^2) - u_i u_j) / gamma^3, with 1 + |u|^2 - u_i^2 summed
  // from the other components (no cancellation at large gamma)
  const T ig3 = ig * ig * ig;
  T lux = a.lux[p] + ((T(1) + uy2 + uz2) * gxv - ux * (uy * gyv + Uz * gzv)) * ig3;
  T luy = a.luy[p] + ((T(1) + ux2 + uz2) * gyv - uy * (ux * gxv + Uz * gzv)) * ig3;
  T luz = a.luz[p] + ((T(1) + ux2 + uy2) * gzv - Uz * (ux * gxv + uy * gyv)) * ig3;

  // 5. Boris transpose
  T lE[3], lB[3];
  lE[0] = h * lux;
  lE[1] = h * luy;
  lE[2] = h * luz;
  // u+ = m + p x s
  T lmx = lux, lmy = luy, lmz = luz;
  const T lpx = sy * luz - sz * luy, lpy = sz * lux - sx * luz, lpz = sx * luy - sy * lux;  // s x lu
  const T lsx = luy * pz - luz * py, lsy = luz * px - lux * pz, lsz = lux * py - luy * px;  // lu x p
  // p = m + m x t
  lmx += lpx + (ty * lpz - tz * lpy);
  lmy += lpy + (tz * lpx - tx * lpz);
  lmz += lpz + (tx * lpy - ty * lpx);
  T ltx = lpy * Mz - lpz * my, lty = lpz * mx - lpx * Mz, ltz = lpx * my - lpy * mx;  // lp x m
  // s = 2 t / (1 + |t|^2)
  const T ts = tx * lsx + ty * lsy + tz * lsz;
  const T f2 = T(2) * iden, f4 = T(4) * ts * iden * iden;
  ltx += f2 * lsx - f4 * tx;
  lty += f2 * lsy - f4 * ty;
  ltz += f2 * lsz - f4 * tz;
  // t = h B / gm
  const T hg = h * igm;
  lB[0] = hg * ltx;
  lB[1] = hg * lty;
  lB[2] = hg * ltz;
  const T lgm = -(tx * ltx + ty * lty + tz * ltz) * igm * igm;
  lmx += lgm * mx;
  lmy += lgm * my;
  lmz += lgm * Mz;
  // m = u + h E
  lE[0] += h * lmx;
  lE[1] += h * lmy;
  lE[2] += h * lmz;
  a.lux[p] = lmx;
  a.luy[p] = lmy;
  a.luz[p] = lmz;

  // 6. gather transpose: the weights' dependence on x^n here, the copies' adjoint below
  T lox = lx1 + lox_dep, loz = lz1 + loz_dep;
  const T lFv[6] = {lE[0], lE[1], lE[2], lB[0], lB[1], lB[2]};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    lF[c] = lFv[c];
    lox += lF[c] * dFx[c];
    loz += lF[c] * dFz[c];
  }
  a.lox[p] = lox;
  a.loz[p] = loz;
  }  // active
  // adjoint of the copies: lambda_F times the gather weights, summed over runs of lanes that share
  // the component's base node (inactive lanes carry zeros under keys of their own)
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int sx = kStagX[c], sz = kStagZ[c];
    const Gw<T> wx = gweights(ox, sx, SCHEME == 0 ? 1 - sx : 1, ix);
    const Gw<T> wz = gweights(oz, sz, SCHEME == 0 ? 1 - sz : 1, iz);
    const int key = active ? wz.i0 * nx + wx.i0 : -1 - lane;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const bool tail = active && (lane == 31 || next != key);
    T* LG = a.lg[c];
    const T v = lF[c];
    const T s00 = run_sum(v * wz.w0 * wx.w0, start, lane);
    if (tail) atomic_add(LG + wz.i0 * nx + wx.i0, s00);
    if (wx.two) {  // the same for every lane (the order depends on the component only)
      const T s01 = run_sum(v * wz.w0 * wx.w1, start, lane);
      if (tail) atomic_add(LG + wz.i0 * nx + wx.i1, s01);
    }
    if (wz.two) {
      const T s10 = run_sum(v * wz.w1 * wx.w0, start, lane);
      if (tail) atomic_add(LG + wz.i1 * nx + wx.i0, s10);
      if (wx.two) {
        const T s11 = run_sum(v * wz.w1 * wx.w1, start, lane);
        if (tail) atomic_add(LG + wz.i1 * nx + wx.i1, s11);
      }
    }
  }
}

template <typename T>
cudaError_t launch_adj_particles(const AdjPartArgs<T>& a, int scheme, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((a.n + ADJ_THREADS - 1) / ADJ_THREADS);
  if (scheme == 0) k_adj_particles<T, 0><<<blocks, ADJ_THREADS, 0, st>>>(a);
  else k_adj_particles<T, 1><<<blocks, ADJ_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_adj_particles<float>(const AdjPartArgs<float>&, int, cudaStream_t);
template cudaError_t launch_adj_particles<double>(const AdjPartArgs<double>&, int, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Psi(D_z) transpose and coefficient gradient, per cell and component q (blockIdx.y):
//   lf_q += Psi_q(D_z) y_q          (y = F_filter applied to the adjoint of the copies)
//   dots[n] += f_q . D_z^n y_q      (n = 0..4; Psi_E rows for q < 2, Psi_B rows for q >= 2)
// since G_q = Psi_q(D_z) F_filter f_q with Psi_q = sum_n a_n D^n, every operator symmetric.
// Block partial sums in FP64, one atomic per block and coefficient.
// ---------------------------------------------------------------------------------------------
constexpr int PSI_BLOCKS = 304;  // blocks per component (grid-stride), partial sums per block

template <typename T>
__global__ void __launch_bounds__(256) k_adj_psi(const __grid_constant__ AdjPsiArgs<T> a) {
  const int q = blockIdx.y;
  const T* __restrict__ Y = a.y[q];
  const T* __restrict__ Fq = a.f[q];
  T* __restrict__ L = a.lf[q];
  const int zs = q < 2 ? 0 : 1;
  T taps[9], dp[5][9];
#pragma unroll
  for (int m = 0; m < 9; ++m) {
    taps[m] = a.taps[zs][m];
#pragma unroll
    for (int n = 0; n < 5; ++n) dp[n][m] = a.dpow[n][m];
  }
  double dn[5] = {0, 0, 0, 0, 0};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long k = c / a.nxy, base = c - k * a.nxy;
    T y[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      int kk = (int)k + m - 4;
      kk = kk < 0 ? kk + a.nz : (kk >= a.nz ? kk - a.nz : kk);
      if (kk < 0 || kk >= a.nz) kk = wrapi(kk, a.nz);  // grids shorter than 4 cells
      y[m] = Y[(long long)kk * a.nxy + base];
    }
    T psi = T(0);
#pragma unroll
    for (int m = 0; m < 9; ++m) psi += taps[m] * y[m];
    L[c] += psi;
    const double f = (double)Fq[c];
#pragma unroll
    for (int n = 0; n < 5; ++n) {
      T v = T(0);
#pragma unroll
      for (int m = 0; m < 9; ++m) v += dp[n][m] * y[m];
      dn[n] += f * (double)v;
    }
  }
  __shared__ double red[5][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    double v = dn[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[n][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    a.partial[((long long)q * gridDim.x + blockIdx.x) * 5 + threadIdx.x] = t;
  }
}

// dots[n] += the Psi_E rows (components 0, 1), dots[5 + n] += the Psi_B rows (2..5), in a fixed order
// One warp per output: lanes stride over the blocks, then a fixed-order shuffle tree.
__global__ void k_adj_psi_final(const double* __restrict__ partial, int nblocks, double* dots) {
  const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (t >= 10) return;
  const int n = t % 5, q0 = t < 5 ? 0 : 2, q1 = t < 5 ? 2 : 6;
  double s = 0;
  for (int q = q0; q < q1; ++q)
    for (int b = lane; b < nblocks; b += 32) s += partial[((long long)q * nblocks + b) * 5 + n];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) dots[t] += s;
}

template <typename T>
cudaError_t launch_adj_psi(const AdjPsiArgs<T>& a, cudaStream_t st) {
  if (a.ncell <= 0) return cudaSuccess;
  long long nb = (a.ncell + 255) / 256;
  nb = nb < PSI_BLOCKS ? nb : PSI_BLOCKS;
  dim3 grid((unsigned)nb, 6);
  k_adj_psi<T><<<grid, 256, 0, st>>>(a);
  k_adj_psi_final<<<1, 320, 0, st>>>(a.partial, (int)nb, a.dots);
  return cudaGetLastError();
}
size_t adj_psi_partial_doubles() { return (size_t)6 * PSI_BLOCKS * 5; }
template cudaError_t launch_adj_psi<float>(const AdjPsiArgs<float>&, cudaStream_t);
template cudaError_t launch_adj_psi<double>(const AdjPsiArgs<double>&, cudaStream_t);

}  // namespace picgb
