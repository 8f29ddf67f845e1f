// Host-side launchers of the CUDA kernels (internal; the public ABI is include/pic.h).
#pragma once
#include <cuda.h>  // CUtensorMap (the encoder is fetched from the driver at run time)
#include <cuda_runtime.h>
#include <utility>

#include "common.cuh"

namespace picgb {

// Flat (compact) particle arrays used by state import / export.
template <typename T>
struct FlatDev {
  long long np;
  int* cell;
  int* species;
  T *ox, *oy, *oz, *dux, *duy, *duz, *w;
  unsigned* id;
};

// Separable periodic stencil over up to 6 components: out = X(Y(Z(in))) with per-component
// z taps (one of two sets) and shared x / y taps. Taps are odd-length, centred.
template <typename T>
struct SepArgs {
  const T* src[6];
  T* dst[6];
  int zset[6];
  int ncomp;
  T* zero[3];  // optional: arrays zeroed at this kernel's output cells (the current, before a push)
  int nx, ny, nz, ndim;
  int hz[2], hx, hy;
  T zt[2][MAX_ZTAPS];
  T xt[MAX_XTAPS];
  T yt[MAX_XTAPS];
  int spread;  // blocks to spread a small grid over (the SM count); 0: the kernel's full tiles
  // TMA staging (set by launch_sep when the grid allows it): one tensor map per source component
  int use_tma;
  int* err;  // device error flags (ERR_TIMEOUT when a staging wait gives up)
  CUtensorMap tm[6];
};

template <typename T>
struct YeeArgs {
  T *ex, *ey, *ez, *bx, *by, *bz;  // fields at the start of the step (the separate updates: in place)
  // the fused step's output E^{n+1}, B^{n+1}: arrays other than the inputs, because a tile reads
  // its neighbours' cells as halo while they may already have written theirs
  T *oex = nullptr, *oey = nullptr, *oez = nullptr, *obx = nullptr, *oby = nullptr, *obz = nullptr;
  const T *jx, *jy, *jz;
  int nx, ny, nz;
  T cx, cy, cz;  // h / d for the curl differences (h = dt or dt/2)
  T h;           // coefficient of J in the E update
  int ck = 0;                // 1: Cole-Karkkainen curl of E in the B updates (2D fused kernel only)
  T wx0 = T(1), wx1 = T(0);  // CK weights of the x differences at z offsets 0 and +-1 (1 - 2 beta_x, beta_x)
  T wz0 = T(1), wz1 = T(0);  // CK weights of the z differences at x offsets 0 and +-1 (1 - 2 beta_z, beta_z)
  // TMA staging of the fused kernel (set by launch_yee_fused when the grid allows it): tensor maps of
  // Ex Ey Ez Bx By Bz Jx Jy Jz
  int spread = 0;      // blocks to spread a small grid over (the SM count); 0: the kernel's full tiles
  int use_tma = 0;
  int* err = nullptr;  // device error flags (ERR_TIMEOUT when a staging wait gives up)
  CUtensorMap tm[9];
};

// Tensor map of a periodic field array (x fastest; nx*ny*nz elements of es bytes) for boxes of
// (bx, by[, bz]) elements: rank 2 for ndim 2 (x, z), 3 for ndim 3. Out-of-range box elements read
// as zero. Returns false when the layout does not allow TMA (row bytes not a multiple of 16, an
// unaligned base, a box past the limits) or the driver has no encoder.
bool tma_encode(CUtensorMap* m, const void* base, int es, int ndim, int nx, int ny, int nz, int bx, int by, int bz);

// Launch with programmatic stream serialization (see pdl_wait): the kernel must call pdl_wait before
// it reads or writes anything its predecessor in the stream touches.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Particle tiles of a grid: the push kernel's tile (PTile, or HoTile for the cubic and momentum-
// conserving push) for the precision (es bytes per value), halved (down to 4 cells, the longest
// extent first) while twice the tiles still fit in `spread` blocks, so that a small grid spreads over
// the SMs. spread = 0 keeps the full tile. te: cells per tile and direction.
void push_tiles(int ndim, int es, bool ho, int nx, int ny, int nz, int spread, int nt[3], int te[3]);

// Raise a kernel's dynamic shared memory limit to `bytes` (once per kernel and size).
cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes);

// ppc_total: expected particles per cell (both species), used to pick the lanes per cell.
template <typename T>
cudaError_t launch_push(const RunDev<T>& r, int ppc_total, cudaStream_t st);
template <typename T>
cudaError_t launch_migrate(const RunDev<T>& r, int* other_count, cudaStream_t st);
// Particle step for shape order 3 and/or the momentum-conserving gather (k_push_ho.cu).
template <typename T>
cudaError_t launch_push_ho(const RunDev<T>& r, int order, int scheme, cudaStream_t st);
// Many runs in one persistent launch: work items (run, tile), *queue zeroed by the launcher.
template <typename T>
cudaError_t launch_push_batch(const RunDev<T>* runs, const int2* items, int nitems, int* queue, int ndim, int scheme,
                              int lpc, int blocks, cudaStream_t st);
// Lanes per cell of the batched push (4, 8 or 16) for the expected particles per cell.
int push_lanes_per_cell(int ndim, int ppc_total);
template <typename T>
int push_max_blocks_per_sm(int ndim, int scheme, int lpc);
template <typename T>
cudaError_t launch_init_beam(const RunDev<T>& r, int ppc, const int lat[3], double u0, double w0, double jitter,
                             double u_th, double sigma_perp, unsigned long long seed, cudaStream_t st);
template <typename T>
cudaError_t launch_import(const RunDev<T>& r, const FlatDev<T>& f, cudaStream_t st);
// Spilled particles (full bins): the step of the tile kernels, one thread per spilled particle
// (k_push_ho.cu); zeroes *r.sp_out for this step's k_migrate. Batched: one run per blockIdx.y,
// linear shapes, Galerkin or Uniform.
template <typename T>
cudaError_t launch_push_spill(const RunDev<T>& r, int order, int scheme, cudaStream_t st);
template <typename T>
cudaError_t launch_push_spill_batch(const RunDev<T>* runs, int nruns, int ndim, int scheme, cudaStream_t st);
// spill list entries [0, n) into flat arrays at [base, base + n)
template <typename T>
cudaError_t launch_spill_export(const RunDev<T>& r, long long n, long long base, const FlatDev<T>& f,
                                cudaStream_t st);
// *out = max(*out, max over cells of c0, c1)
cudaError_t launch_max_count(const int* c0, const int* c1, long long ncell, int* out, cudaStream_t st);
template <typename T>
cudaError_t launch_export(const RunDev<T>& r, int s, const long long* offs, long long base, const FlatDev<T>& f,
                          cudaStream_t st);
cudaError_t launch_count_prefix(const int* cnt, long long ncell, int cap, long long* offs, long long* bsum,
                                long long* total, cudaStream_t st);
long long count_prefix_blocks(long long ncell);

template <typename T>
cudaError_t launch_sep(const SepArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_yee_b(const YeeArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_yee_e(const YeeArgs<T>& a, cudaStream_t st);

// (sum E^2, sum B^2, sum Ex^2+Ey^2+Bx^2+By^2) in FP64 into out[0..2], or, when hc.hist is set, into
// the run's device history (see HistCtl); scratch holds field_energy_scratch_bytes() and starts
// zeroed (the kernel leaves it ready for the next launch)
template <typename T>
cudaError_t launch_field_energy(const T* const f6[6], long long ncell, double* out, double* scratch, HistCtl hc,
                                cudaStream_t st);
template <typename T>
struct EnergyArgs {
  const T* f[6];
  long long ncell;
  double* scratch;
  HistCtl hc;
};
template <typename T>
cudaError_t launch_field_energy_batch(const EnergyArgs<T>* args, int nruns, cudaStream_t st);
// Many runs: tile_base[run] = first flat tile of the run (prefix over runs, tile_base[nruns] = total)
template <typename T>
cudaError_t launch_sep_batch(const SepArgs<T>* args, const int* tile_base, int nruns, int total_tiles, int ncomp,
                             int ndim, int hz, int hx, cudaStream_t st);
template <typename T>
cudaError_t launch_yee_batch(const YeeArgs<T>* args, const int* tile_base, int nruns, int total_tiles, int ndim,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_migrate_batch(const RunDev<T>* runs, int nruns, cudaStream_t st);
// tiles of the fast stencil / Yee kernels for a grid (the kernels' full tiles, as the batched launches use)
int sep_tiles(int ndim, int nx, int ny, int nz);
int yee_tiles(int ndim, int nx, int ny, int nz);
bool sep_fast_ok(int ndim, int nx, int ny, int nz, int hz, int hx);
size_t field_energy_scratch_bytes();
// B half step, E step, B half step in one launch. With hc, the same launch also records the field
// energies of the new E, B into the history ring (block partials in escratch, of
// yee_energy_scratch_bytes, zeroed once); only where yee_records_energy (cudaErrorInvalidValue else).
bool yee_records_energy(int ndim, int nx, int ny, int nz, int ck);
size_t yee_energy_scratch_bytes(int ndim, int nx, int ny, int nz, int spread);
template <typename T>
cudaError_t launch_yee_fused(const YeeArgs<T>& a, int ndim, cudaStream_t st, double* escratch = nullptr,
                             const HistCtl* hc = nullptr);
// out[0] += sum w (gamma - 1) over both species of the input buffers
template <typename T>
cudaError_t launch_kinetic(const RunDev<T>& r, double* out, cudaStream_t st);

// Gauss-law residual (k_gauss.cu): rho += q w S / dV from the particle bins of r.in (shape order 1 or
// 3, FP64 atomics; rho zeroed by the caller), and (max |div E - rhof|, rms, max |rhof|) into out[0..2]
// (scratch of gauss_scratch_bytes, zeroed once).
template <typename T>
cudaError_t launch_rho(const RunDev<T>& r, int order, double inv_dv, double* rho, cudaStream_t st);
template <typename T>
cudaError_t launch_gauss_residual(const T* ex, const T* ey, const T* ez, const double* rhof, int nx, int ny, int nz,
                                  double idx, double idy, double idz, double* scratch, double* out, cudaStream_t st);
size_t gauss_scratch_bytes();

// Psi_E(D_z) Psi_B(D_z)^-1 applied in place to the two transverse E copies (k_fields.cu); work:
// 2 x ncell complex doubles of scratch
template <typename T>
struct InvPsiArgs {
  T* f[2];
  double2* work;
  long long nxy;
  int nz;
  int nf;  // factors (the degree of Psi_B)
  double lam_re[4], lam_im[4];
  double scale;
  double pe_taps[9];  // Psi_E(D_z), applied first
};
template <typename T>
cudaError_t launch_inverse_psi_z(const InvPsiArgs<T>& a, cudaStream_t st);

// ---- adjoint of the 2D step (k_adjoint.cu) ----
// bins of the current buffers -> flat arrays indexed by particle id (f.np = number of ids);
// `seen` (optional, one zeroed bit per id) flags repeated ids
template <typename T>
cudaError_t launch_tape(const RunDev<T>& r, const FlatDev<T>& f, unsigned long long* seen, cudaStream_t st);
template <typename T>
struct AdjSeedArgs {
  const T* f[6];  // final E, B
  T* lam[6];      // out: adjoint of the final E, B for L = W_perp scaled (scale = dL/dW_perp * dV)
  long long ncell;
  T scale;
};
template <typename T>
cudaError_t launch_adj_seed(const AdjSeedArgs<T>& a, cudaStream_t st);
template <typename T>
struct AdjPartArgs {
  long long n;  // particles (ids 0 .. n-1)
  int nx, nz;
  const int* cell;  // start state of the step, id order
  const int* species;
  const T *ox, *oz, *dux, *duy, *duz, *w;  // w: NULL = wconst
  const T* g[6];                           // gather copies of the step's E, B
  const T* lj[3];                          // adjoint of the unfiltered current J^{n+1/2}
  T* lg[6];                                // adjoint of the gather copies (accumulated atomically)
  T *lox, *loz, *lux, *luy, *luz;          // in: adjoint of x^{n+1}, u^{n+1/2}; out: of x^n, u^{n-1/2}
  T dtdx, dtdz, u0, hq, wconst, jfx, jfz, jfy2d;
  int* err;  // device error flags (ERR_IDS for an invalid taped particle)
};
template <typename T>
cudaError_t launch_adj_particles(const AdjPartArgs<T>& a, int scheme, cudaStream_t st);
template <typename T>
struct AdjPsiArgs {
  const T* y[6];  // filtered adjoint of the gather copies
  const T* f[6];  // the step's E, B
  T* lf[6];       // adjoint of E, B (accumulated)
  long long ncell, nxy;
  int nz;
  T taps[2][9];   // Psi_E, Psi_B z-stencils
  T dpow[5][9];   // D^n, n = 0..4
  double* dots;     // [10]: d/d a_n of Psi_E (0..4) and Psi_B (5..9), accumulated
  double* partial;  // adj_psi_partial_doubles() of block partial sums (scratch)
};
template <typename T>
cudaError_t launch_adj_psi(const AdjPsiArgs<T>& a, cudaStream_t st);
size_t adj_psi_partial_doubles();

}  // namespace picgb
