/*
 * pic.h -- C ABI of a GB300 (sm_103a) implementation of the stabilised FDTD-Esirkepov
 * particle-in-cell time step of Godfrey & Vay, "Suppressing the Numerical Cherenkov
 * Instability in FDTD PIC Codes" (arXiv 1401.0838).
 *
 * One step (Sec. 2 and Sec. 3 of the paper, in the order its loop implies):
 *   1. copies of E and B as seen by the particles: Psi_E(D_z) on Ex, Ey and Psi_B(D_z) on
 *      Ez, Bx, By, Bz (Sec. 2, last paragraph), D = -(1,-2,1)/4 along z, then the gather share
 *      of the binomial + compensation filter (Sec. 3, Eq. 6; Sec. 4);
 *   2. gather at x^n with the Galerkin or Uniform shapes (Sec. 2, Eq. 3-4);
 *   3. relativistic Boris push u^{n-1/2} -> u^{n+1/2};
 *   4. move x^n -> x^{n+1};
 *   5. Esirkepov current deposition J^{n+1/2} (cited in Sec. 2);
 *   6. current filter (Eq. 6 / Sec. 4);
 *   7. Yee update: B half step, E full step with -J, B half step.
 *
 * Conventions
 *   - Units c = eps0 = mu0 = 1; particle mass 1; charges -1 (species 0, electrons) and
 *     +1 (species 1, positrons). Positions are in grid units.
 *   - Fields live on the standard periodic Yee mesh; element [(k*ny + j)*nx + i] of a field
 *     array holds Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2), Bx(i,j+1/2,k+1/2),
 *     By(i+1/2,j,k+1/2), Bz(i+1/2,j+1/2,k). A 2D run is x-z with ny = 1.
 *   - Every function returns PIC_OK (0) or a negative PIC_E_* code; pic_last_error() gives text.
 *   - The handle owns all device memory it allocates. Caller arrays are only read or written
 *     during the call (device-side copies are ordered on the handle's stream) and never kept.
 *   - pic_step and the state copies are asynchronous on the handle's stream. Errors raised by
 *     kernels (a non-finite particle, an invalid import) are sticky and reported by the next
 *     pic_sync, pic_energy or pic_get_state.
 *   - Particle bins never lose a particle: a particle whose cell bin is full waits in a spill
 *     list of the handle, which every step pushes from (the same gather, push, move and deposit),
 *     and the next synchronising call (or the next pic_step, once the previous one has finished)
 *     re-bins every particle into larger bins. A run whose beam bunches (the instability this
 *     library studies) therefore completes at any initial bin capacity.
 *   - A handle is not thread safe; different handles are independent.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_E_ARG (-1)        /* invalid argument or configuration */
#define PIC_E_CFL (-2)        /* dt violates the Courant limit of the field solver */
#define PIC_E_SINGULAR (-3)   /* rational interpolation singular / ill-conditioned */
#define PIC_E_OOM (-4)        /* device or host allocation failed */
#define PIC_E_CUDA (-5)       /* a CUDA runtime call failed */
#define PIC_E_TIMEOUT (-6)    /* a bounded device wait gave up */
#define PIC_E_NONFINITE (-7)  /* NaN/Inf found in the state */
#define PIC_E_OVERFLOW (-8)   /* a particle found no room in a bin, the spill or the leaver list */
#define PIC_E_STATE (-9)      /* call not valid in the handle's current state */

#define PIC_GALERKIN 0
#define PIC_UNIFORM 1
#define PIC_MOMENTUM 2 /* momentum-conserving gather: fields averaged to the nodes (Eq. 5 multiplier) */

#define PIC_FP32 0
#define PIC_FP64 1

#define PIC_FILTER_J 1      /* filter the deposited current */
#define PIC_FILTER_GATHER 2 /* filter the field copies seen by the particles */

#define PIC_HOST 0
#define PIC_DEVICE 1

typedef struct pic_handle pic_handle;

/* Run configuration. pic_config_default() fills the values of the paper's 2D beam problem. */
typedef struct pic_config {
  int ndim;                 /* 2 (x-z, three velocity components) or 3 */
  int nx, ny, nz;           /* cells per direction; ny is forced to 1 in 2D */
  double dx, dy, dz, dt;    /* cell sizes and time step (c = 1); dy forced to 1 in 2D */
  double gamma;             /* Lorentz factor of the beam drift along +z */
  int scheme;               /* field gather: PIC_GALERKIN, PIC_UNIFORM or PIC_MOMENTUM */
  int shape_order;          /* particle shape: 1 (linear) or 3 (cubic B-spline, the Sec. 3 setting) */
  int precision;            /* PIC_FP32 or PIC_FP64 (fields, particles and kernels) */
  int ppc_per_species;      /* lattice points per cell per species of the initial beam, 0 .. 2^20 */
  double omega_p_dz;        /* total plasma frequency (both species) times dz / c */
  double jitter;            /* uniform position jitter half-width, cells */
  double u_th;              /* Gaussian spread of each momentum component (u = gamma v) */
  double sigma_perp;        /* > 0: per-particle weight exp(-r_perp^2/(2 sigma^2)), cells */
  int filter_nbin;          /* bilinear passes per direction per side (paper's WARP runs: 1) */
  int filter_ncomp;         /* compensation passes per direction per side (paper: 1) */
  double filter_comp_alpha; /* compensation centre weight a: taps (-(a-1)/2, a, -(a-1)/2) */
  int filter_targets;       /* PIC_FILTER_J | PIC_FILTER_GATHER */
  unsigned long long seed;  /* Philox4x32-10 key of the initial beam */
  int init_beam;            /* 1: pic_create fills the seeded beam; 0: start empty */
  int bin_capacity;         /* initial particle slots per cell per species, up to 2^24;
                               0: automatic (2 ppc_per_species + 8); bins grow as cells fill */
  int track_ids;            /* 1: carry a 32-bit id per particle (for tests) */
  int diag_every;           /* > 0: record the energies on the device every diag_every steps */
  int diag_capacity;        /* ring size of the energy history; 0: 4096 samples */
  int correction_mode;      /* PIC_CORR_SPLIT (0): Psi_E on the transverse E copies, Psi_B on the
                               other copies, as WARP does (Sec. 2); PIC_CORR_RATIONAL (1): the
                               rational multiplier Psi_E / Psi_B on the transverse E copies only,
                               Psi_B applied exactly by inverting it along z (Sec. 2; the variant
                               of Sec. 3 with the multiplier on E only) */
  int field_solver;         /* PIC_YEE (0) or PIC_CK (1): the Cole-Karkkainen solver named in Sec. 2
                               for Fig. 1 (beta_z = 1/8, c dt/dz = 0.9). 2D only. Its B updates use a
                               curl of E whose forward difference along z is averaged over the x
                               neighbours with weights (beta_z, 1 - 2 beta_z, beta_z), and along x over
                               the z neighbours with beta_x; the E update is Yee's. Stable while
                               dt^2 max(1/dx^2, 1/dz^2, (1-4 beta_x)/dx^2 + (1-4 beta_z)/dz^2) < 1
                               (c dt < dz at beta = 1/8, dx = dz) */
  double ck_beta_x, ck_beta_z; /* CK averaging weights in [0, 1/4]; pic_config_default: 1/8 each */
} pic_config;

#define PIC_CORR_SPLIT 0
#define PIC_CORR_RATIONAL 1
#define PIC_YEE 0
#define PIC_CK 1

/* Energies, all FP64 sums over the whole grid / all particles (c = 1, m = 1). */
typedef struct pic_energy_t {
  double w_e;    /* 1/2 sum E^2 dV */
  double w_b;    /* 1/2 sum B^2 dV (B at integer time) */
  double w_perp; /* 1/2 sum (Ex^2 + Ey^2 + Bx^2 + By^2) dV: the growth-rate observable */
  double k;      /* sum w (gamma - 1), u at the last half step */
  double total;  /* w_e + w_b + k */
  long long np;  /* number of particles */
} pic_energy_t;

/*
 * State in the handle's native layout. Element type of the void* arrays is float (PIC_FP32
 * handle) or double (PIC_FP64). `where` says whether every pointer is host or device memory.
 * Particle i: cell index cell[i] = (k*ny + j)*nx + i, species[i] in {0, 1}, position
 * (i + ox, j + oy, k + oz) with offsets in [0, 1), momentum u = (dux, duy, u_drift + duz) with
 * u_drift = sqrt(gamma^2 - 1).
 */
typedef struct pic_state {
  int where;                        /* PIC_HOST or PIC_DEVICE */
  void *ex, *ey, *ez, *bx, *by, *bz; /* nx*ny*nz each; NULL skips that component */
  long long np;                     /* set: particle count; get: in = array capacity, out = count */
  int* cell;
  int* species;
  void *ox, *oy, *oz;               /* oy unused (may be NULL) in 2D */
  void *dux, *duy, *duz;
  void* w;                          /* per-particle weights; NULL: the uniform beam weight */
  unsigned int* id;                 /* optional (NULL); kept only when track_ids = 1 */
  double u_drift;                   /* filled by pic_get_state */
} pic_state;

/* Fills *cfg with the defaults: 2D 64x128, dx = dz = 1, dt = 0.5, gamma = 130, Galerkin, FP64,
 * 4 particles/cell/species, omega_p dz = 0.3868, jitter 0.1, u_th 1e-4, filter (1, 1, a = 3)
 * on J and on the gather copies, seed 1, init_beam 1. */
void pic_config_default(pic_config* cfg);

/*
 * Correction coefficients (Sec. 2, Eq. 3-4 and the rational interpolation that follows):
 * the (4,4) rational interpolant Psi_E(xi)/Psi_B(xi), xi = sin^2(k_z dz/2), of the Galerkin
 * (Eq. 3) or Uniform (Eq. 4) multiplier (or Eq. 5 for PIC_MOMENTUM) at alpha = c dt / dz, on the
 * nine nodes xi_j = j/8, with Psi_B(0) = 1. Coefficients are in powers of xi, constant first.
 * Host only, FP64. Returns PIC_E_SINGULAR when the 9x9 system is singular and the multiplier is
 * not constant, when its condition estimate exceeds 1e12, or when Psi_B has a zero on [0, 1];
 * when the multiplier is identically 1 (Uniform at alpha = 1/2) it returns Psi_E = Psi_B = 1.
 */
int pic_compute_correction_coeffs(int scheme, double alpha, double psi_e[5], double psi_b[5]);

/* Validates cfg (PIC_E_ARG; PIC_E_CFL: Yee dt >= 1/sqrt(sum 1/d^2), CK the bound stated at
 * field_solver), allocates device memory, fills the seeded beam (Philox4x32-10, counter = lattice point) when cfg->init_beam, zero fields.
 * The correction starts off (Psi = 1); set it with pic_set_correction_stencil. */
int pic_create(const pic_config* cfg, pic_handle** out);

/* Uses `stream` (a cudaStream_t; NULL = the handle's own stream) for all later work. */
int pic_set_stream(pic_handle* h, void* stream);

/* Sets the Psi_E / Psi_B polynomial coefficients (Sec. 2), powers of xi, constant first.
 * Both NULL turns the correction off (Psi = 1). The 9-tap z-stencils sum_n a_n D^n are built on
 * the host in FP64 and combined with the gather filter taps. */
int pic_set_correction_stencil(pic_handle* h, const double psi_e[5], const double psi_b[5]);

/* Advances nsteps >= 0 time steps (asynchronous on the handle's stream). */
int pic_step(pic_handle* h, int nsteps);

/* Waits for the handle's stream and returns any sticky kernel error. */
int pic_sync(pic_handle* h);

/* Energies (FP64 device reductions); synchronises the stream. */
int pic_energy(pic_handle* h, pic_energy_t* out);

/* Current number of particles (synchronises). */
int pic_num_particles(pic_handle* h, long long* np);

/* Particle storage: *cap = the current slots per cell and species of the bins (the initial
 * bin_capacity rounded up to 64 bytes, larger after the bins have grown); *spilled = the particle
 * insertions since pic_create that found their bin full and went to the spill list (each such
 * particle was still pushed every step). Either pointer may be NULL; reading *spilled
 * synchronises. No counterpart in the paper: storage bookkeeping. */
int pic_bin_stats(pic_handle* h, int* cap, long long* spilled);

/* Copies the state out (s->np in: capacity of the particle arrays; PIC_E_ARG when too small,
 * with s->np set to the count needed). With every particle pointer NULL only the non-NULL fields
 * are copied and s->np returns the particle count. Particles come out grouped by species, then by
 * cell. Synchronises. */
int pic_get_state(pic_handle* h, pic_state* s);

/* Replaces the state: the fields that are non-NULL, and all particles (re-binned by cell on the
 * device; offsets outside [0, 1) are folded into the cell index, periodically). s->np = -1 leaves
 * the particles untouched; s->np = 0 removes them all. Without per-particle weights (sigma_perp
 * <= 0) every particle carries the beam weight (omega_p_dz/dz)^2 dx dy dz / (2 ppc_per_species). */
int pic_set_state(pic_handle* h, const pic_state* s);

/* Test hooks. Copy out the six field copies the particles saw in the last step (after Psi and
 * the gather filter; order Ex Ey Ez Bx By Bz) or the three components of the (filtered) current
 * J^{n+1/2} of the last step. `out` holds 6 (resp. 3) pointers of nx*ny*nz elements. */
int pic_debug_gather_copies(pic_handle* h, int where, void* const* out6);
int pic_debug_current(pic_handle* h, int where, void* const* out3);

/* Charge conservation of the step (Sec. 2 cites Esirkepov's charge-conserving deposit; Eq. 6's
 * filter acts on the current): the Yee E update with the filtered current keeps
 * div E - F rho at its initial value, zero for the neutral beam, up to rounding. Computes, in FP64
 * on the device from the current state, rho on the integer nodes from the particles' shapes (order
 * shape_order B-splines, weight q w / dV), F rho with the current filter (identity when
 * filter_targets lacks PIC_FILTER_J), and out[0] = max |div E - F rho|, out[1] = its RMS over the
 * nodes, out[2] = max |F rho| (the scale). Synchronous; allocates 16 B per cell of device scratch on
 * first use (PIC_E_OOM). */
int pic_charge_residual(pic_handle* h, double out[3]);

/* Maximum instability growth rate (Fig. 2/4 captions: from the transverse field energy):
 * Gamma = 1/2 d ln W / dt by an FP64 least-squares fit over the window from the first sample
 * two decades above the noise floor (median of log10 W over the first tenth of the samples) to
 * the first later sample within one decade of the maximum; if that window has fewer than 5
 * samples, the steepest window of max(5, n/5) samples after the first tenth. Samples with w <= 0 or
 * non-finite w are skipped; *i0, *i1 (either may be NULL) receive the window's first and last sample
 * as indices into t and w. PIC_E_ARG when t is not finite and strictly increasing or fewer than 5
 * samples are kept. Host only. */
int pic_fit_growth_rate(const double* t, const double* w, int n, double* gamma_out, int* i0, int* i1);

/* Energies recorded on the device every cfg.diag_every steps (fused into the step: the kinetic
 * sum and particle count come from the push kernel, the field sums from one reduction launch;
 * no host synchronisation). Copies out the most recent min(max, recorded, diag_capacity) samples,
 * oldest first; *count receives that number. Synchronises. */
int pic_energy_history(pic_handle* h, pic_energy_t* out, int max, int* count);

/* Kernel classes of pic_kernel_times. */
#define PIC_K_COPIES 0 /* Psi + gather-filter stencil of the field copies */
#define PIC_K_PUSH 1   /* fused gather + Boris + move + Esirkepov deposition + rebin */
#define PIC_K_FILTER 2 /* current filter */
#define PIC_K_YEE 3    /* Yee updates */
#define PIC_K_DIAG 4    /* energy reductions */
#define PIC_K_OTHER 5   /* initialisation, import, export */
#define PIC_K_MIGRATE 6 /* insertion of the particles that left their tile into their new bins */
#define PIC_K_SPILL 7   /* push of the particles waiting in the spill list (their bin was full) */
#define PIC_NKERNEL 8

/* on = 1: bracket every later kernel launch with CUDA events on the handle's stream and reset the
 * totals; on = 0: stop. */
int pic_enable_timing(pic_handle* h, int on);

/* Device milliseconds and launch counts per kernel class since pic_enable_timing(h, 1).
 * Synchronises. */
int pic_kernel_times(pic_handle* h, double ms[PIC_NKERNEL], long long launches[PIC_NKERNEL]);

/* Kernel launches made by this handle since it was created. */
int pic_launch_count(pic_handle* h, long long* n);

/*
 * Field energies with no memory allocation. The paper has no counterpart: this entry point is for
 * callers that cannot allocate device memory where they need the energies (a plugin whose host
 * application owns every device allocation, a monitor that must not change the memory footprint of
 * the run it watches, code running when the device is nearly full). It returns the same W_E, W_B,
 * W_perp as pic_energy
 * (1/2 sum E^2 dV, 1/2 sum B^2 dV, 1/2 sum (Ex^2+Ey^2+Bx^2+By^2) dV, FP64 sums) for six device
 * arrays of ncell elements each (Ex Ey Ez Bx By Bz; float for PIC_FP32, double for PIC_FP64) and
 * writes them to the host array out[3]; dv is the cell volume. It calls no cudaMalloc or cudaFree:
 * the block partial sums live in one fixed array of this library's device memory (96 KiB, held by
 * every GPU that loads the library until the process exits), which limits a call to
 * 16,777,216 cells (larger ncell: PIC_E_ARG). The first call on a device looks that array's address
 * up (cudaGetSymbolAddress) with the device current, so make it before any stream capture on that
 * device; the address is kept for the life of the process, so do not call this entry point on a
 * device after a cudaDeviceReset of it. Every call shares the array: calls that overlap on the GPU
 * (other streams or threads) race and must be serialised by the caller; nothing in it has to start
 * at zero, because each call overwrites every partial sum it reads. Work is queued on `stream` (a
 * cudaStream_t; NULL = the default stream); the call synchronises that stream and copies the three
 * sums into out before returning. A CUDA error pending before the call makes it return PIC_E_CUDA
 * and is left pending.
 */
int pic_field_energy_noalloc(const void* const fields[6], long long ncell, int precision, double dv,
                             double out[3], void* stream);

/*
 * Batched runs (the sweeps of Sec. 3: growth rate against c dt/dz, gamma and the correction): many
 * independent simulations of possibly different grid sizes advanced together. Every step is one
 * set of multi-run launches (a persistent push kernel per lanes-per-cell group takes (run, tile)
 * items from a work list; one stencil, migrate, Yee and energy launch cover all runs) replayed from
 * a CUDA graph. The runs must agree on ndim, precision, scheme, shape order, filter and diagnostic
 * settings, per-particle weights, id tracking, correction mode and field solver (PIC_E_ARG
 * otherwise); grids, ppc, gamma, dt, seeds and corrections may differ. Each grid needs at least as
 * many cells per direction as the stencil halos (PIC_E_ARG otherwise). Batched runs use linear
 * shapes with the Galerkin or Uniform gather, the split correction and the Yee solver (cubic
 * shapes, the momentum-conserving gather, the rational multiplier or CK: PIC_E_ARG).
 */
typedef struct pic_batch pic_batch;
int pic_batch_create(const pic_config* cfgs, int nruns, pic_batch** out);
int pic_batch_size(const pic_batch* b);
/* The handle of one run (owned by the batch): for state import/export and energies between steps.
 * Stepping a run on its own desynchronises it from the batch (pic_batch_step then fails). */
pic_handle* pic_batch_run(pic_batch* b, int run);
int pic_batch_set_correction_stencil(pic_batch* b, int run, const double psi_e[5], const double psi_b[5]);
int pic_batch_set_stream(pic_batch* b, void* stream);
int pic_batch_step(pic_batch* b, int nsteps);
int pic_batch_sync(pic_batch* b);
int pic_batch_energy_history(pic_batch* b, int run, pic_energy_t* out, int max, int* count);
/* Autotuner: for every lanes-per-cell group, times 2*trial_steps batched steps with each candidate
 * (4, 8 or 16 lanes per cell; 1 or 2 resident blocks of the push kernel per SM) and keeps the
 * fastest (written to lpc_out[group] when not NULL; the runs are grouped by their default lanes per
 * cell, 4, 8 or 16, so lpc_out needs at most 3 entries); then every run is put back into its seeded
 * initial state (fields zero, beam from the seed), so tune before importing other states. */
int pic_batch_autotune(pic_batch* b, int trial_steps, int* lpc_out);
void pic_batch_destroy(pic_batch* b);
const char* pic_batch_last_error(const pic_batch* b);

/*
 * Adjoint (reverse mode) of the 2D step: the gradient of the final transverse field energy
 * W_perp(T) = 1/2 sum (Ex^2 + Ey^2 + Bx^2 + By^2) dV (the quantity whose growth Sec. 4 measures)
 * with respect to the Psi_E / Psi_B polynomial coefficients a_0..a_4 (Sec. 2) and the initial E,
 * B, from hand-written transposes of every pass of the step: the gather copies Psi(D_z) and the
 * filter (Sec. 2 last paragraph, Sec. 3 Eq. 6), the gather with the Galerkin or Uniform shapes
 * (Sec. 2, Eq. 3-4), the Boris push, the move, the Esirkepov deposition and the Yee update.
 * Derivatives are exact almost everywhere (the linear shapes have kinks).
 *
 * pic_adjoint_forward advances the run nsteps from its current state (as pic_step would) and
 * returns W_perp(T) in *w_perp. On the way it stores the full state (fields, particles by id)
 * every checkpoint_every steps and at the end, in device memory the handle keeps until
 * pic_adjoint_release or pic_destroy: (nsteps / checkpoint_every + 2 + checkpoint_every) states of
 * about N x (8 + 5 x element size) bytes for N particles, plus 6 field arrays each.
 * 2D runs with linear shapes, the Galerkin or Uniform gather, the split correction and the Yee
 * solver only (PIC_E_ARG otherwise), and
 * cfg.track_ids = 1 with ids 0 .. N-1, as the seeded beam
 * and any import without explicit ids have (PIC_E_STATE otherwise).
 *
 * pic_adjoint_backward, with the state still the final state of the recorded run (no step, state
 * or correction change in between; PIC_E_STATE otherwise), writes for L = dw x W_perp(T):
 * dL/da_n of Psi_E and Psi_B into grad_psi_e[5] / grad_psi_b[5] (host; either may be NULL), and
 * dL/dE^0, dL/dB^0 into grad_fields[6] (device arrays of the handle's precision and layout, order
 * Ex Ey Ez Bx By Bz; NULL or NULL entries skip them). Each segment between checkpoints is
 * recomputed once, so the call costs about one more forward run plus the transposed passes. It
 * leaves the state at the recorded final state again (the order of the particles inside a cell may
 * differ) and synchronises the stream. The particle adjoints are carried in the handle's
 * precision.
 */
int pic_adjoint_forward(pic_handle* h, int nsteps, int checkpoint_every, double* w_perp);
int pic_adjoint_backward(pic_handle* h, double dw, double grad_psi_e[5], double grad_psi_b[5],
                         void* const grad_fields[6]);
/* Frees the adjoint's checkpoint and work storage (no-op when there is none; NULL is a no-op). */
void pic_adjoint_release(pic_handle* h);

/* Frees everything the handle owns. NULL is a no-op. */
void pic_destroy(pic_handle* h);

/* Text of the last error on this handle (never NULL); with h = NULL, the reason the calling
 * thread's last pic_create failed. */
const char* pic_last_error(const pic_handle* h);

/* Static text for a PIC_E_* code. */
const char* pic_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
