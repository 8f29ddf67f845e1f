// C ABI (include/pic.h): handle management, the per-step launch sequence, state import/export,
// diagnostics, batched runs and the adjoint's checkpoint / recompute schedule. All arithmetic of
// the step and of its adjoint runs in the CUDA kernels of k_fields.cu, k_particles.cu and
// k_adjoint.cu; this file only allocates, marshals and orders launches on one stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/pic.h"
#include "common.cuh"
#include "host_math.h"
#include "launch.h"

using namespace picgb;

struct pic_handle {
  pic_config cfg;
  size_t es = 8;  // element size of fields and particle reals
  cudaStream_t own = nullptr, stream = nullptr;
  long long ncell = 0;
  int cap = 0;
  int ntx = 1, nty = 1, ntz = 1;
  int tex = 16, tey = 1, tez = 16;  // cells per particle tile and direction
  int nsm = 0;                       // the device's SMs: small grids spread their tiles over them
  double u0 = 0, w0 = 0;
  bool has_w = false, has_id = false;
  std::vector<void*> allocs;
  void* f[9] = {};   // ex ey ez bx by bz jx jy jz (E and B: the current step's)
  void* fb[6] = {};  // the other E, B buffers: the fused Yee update writes there, then the two swap
  void* g[6] = {};   // gather copies
  void* jf[3] = {};  // filtered current (aliases f[6..8] when J is not filtered)
  void* parr[2][2][8] = {};  // [species][buffer][ox oy oz dux duy duz w id]
  int* cnt[2][2] = {};
  int parity = 0;
  int* d_err = nullptr;
  void* lv[10] = {};        // leaver list: key, ox, oy, oz, dux, duy, duz, w, id
  int* d_lv_count = nullptr;  // two counters, one per step parity
  long long lv_cap = 0;
  // spill list (particles whose bin was full; same layout as the leaver list), two counters by
  // parity: [p] = waiting for the next step of parity p
  void* sp[10] = {};
  int* d_sp_count = nullptr;
  long long sp_cap = 0;
  int* d_maxc = nullptr;        // scratch of the bin growth (largest count)
  unsigned long long* d_sp_total = nullptr;  // insertions that found their bin full, since creation
  int* h_sp_mirror = nullptr;   // pinned copy of the waiting count, written after each pic_step
  cudaEvent_t ev_sp = nullptr;  // completion of that copy
  bool sp_pending = false;
  int grow_gen = 0;             // reallocations of bins or lists (batched runs re-upload their tables)
  double* d_acc = nullptr;  // 8 doubles of reduction scratch
  double* d_red = nullptr;  // block partials of the field-energy reduction
  double* d_red_yee = nullptr;  // block partials of the energies recorded by the Yee launch
  double* d_rho = nullptr;      // Gauss-law diagnostic: rho and F rho (FP64), then its scratch
  double* d_gauss = nullptr;
  long long* d_offs = nullptr;
  long long* d_bsum = nullptr;
  long long* d_total = nullptr;
  // import / export staging (device)
  void* stage[10] = {};
  long long stage_n = 0;
  // taps (FP64, host) of the copy and current stencils
  double pe[5] = {1, 0, 0, 0, 0}, pb[5] = {1, 0, 0, 0, 0};
  std::vector<double> zt_e, zt_b, xt_g, zt_j, xt_j;
  // rational correction mode: factors of Psi_B(D_z)^-1 and the complex scratch of the z-solves
  double inv_lr[4] = {}, inv_li[4] = {}, inv_scale = 1.0;
  int inv_nf = 0;
  void* inv_work = nullptr;
  // energy history (device ring of 8 doubles per sample: sum E^2, sum B^2, sum perp^2, K, np)
  double* d_hist = nullptr;
  int hist_cap = 0;
  int* d_hist_count = nullptr;  // samples written by the device (mirrors nhist)
  double* d_kin = nullptr;      // kinetic-energy / particle-count accumulator of the recorded step
  long long nhist = 0;
  long long nstep = 0;
  // CUDA graph of graph_len consecutive steps starting at an even step index
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  cudaStream_t graph_stream = nullptr;
  int graph_parity = 0;               // parity of the first captured step
  void* graph_f0 = nullptr;           // Ex buffer current when the graph was captured
  long long graph_launch_count = 0;   // kernel launches in one replay
  long long graph_counts[PIC_NKERNEL] = {};
  // kernel timing
  bool timing = false;
  struct Pending {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  double tms[PIC_NKERNEL] = {};
  long long tcount[PIC_NKERNEL] = {};
  long long launches = 0;
  // adjoint: checkpoints of the forward run, the recomputed segment's tape, adjoint work arrays
  struct Flat {
    void* a[9] = {};  // cell, species, ox, oy, oz, dux, duy, duz, w (id order)
  };
  struct Adj {
    bool ready = false;  // a forward run was recorded and the state has not changed since
    int nsteps = 0, every = 0, nseg = 0;
    long long np = 0, final_step = 0, final_hist = 0;
    int cap_ck = 0, cap_tape = 0;
    long long cap_np = 0;
    std::vector<void*> ck_f;    // (nseg + 1) x 6 fields at the checkpoints (the last: final state)
    std::vector<Flat> ck_p;     // nseg + 1 particle states
    std::vector<void*> tape_f;  // every x 6: fields at the start of each step of a segment
    std::vector<Flat> tape_p;   // every: particles at the start of each step of a segment
    void* lam[6] = {};          // adjoint of E, B
    void* lj[3] = {};           // adjoint of J
    void* lg[6] = {};           // adjoint of the gather copies
    void* y[6] = {};            // filtered lg
    void* lp[5] = {};           // particle adjoints: ox, oz, ux, uy, uz (id order)
    double* dots = nullptr;     // 10 coefficient-gradient accumulators
    double* partial = nullptr;  // block partial sums of the coefficient gradient
    unsigned long long* seen = nullptr;
    std::vector<void*> mem;
  } adj;
  bool no_diag = false;  // the adjoint's recomputed steps record no diagnostics
  std::string err;
};

static void drop_graph(pic_handle* h);
static thread_local std::string g_create_err;  // why the last pic_create / pic_batch_create failed

namespace {

int fail(pic_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(pic_handle* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? PIC_E_OOM : PIC_E_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                               \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

cudaEvent_t take_event(pic_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Accumulate the elapsed times of every bracketed launch (synchronises the stream).
cudaError_t collect_times(pic_handle* h) {
  if (h->pending.empty()) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->tms[p.cls] += ms;
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->pending.clear();
  return cudaSuccess;
}

// NVTX ranges for profilers (a no-op unless one is attached): one per kernel launch, named by its
// class, and one around each pic_step / pic_batch_step call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
const char* const kKernelClassName[PIC_NKERNEL] = {"copies", "push", "filter", "yee", "diag", "other", "migrate",
                                                   "spill"};

// Launch one kernel of class `cls`, counted, and bracketed by events when timing is on.
template <class F>
cudaError_t launch(pic_handle* h, int cls, F&& go) {
  NvtxRange range(kKernelClassName[cls]);
  (void)cudaGetLastError();  // a failed earlier query must not be reported as this launch's error
  h->launches++;
  h->tcount[cls]++;
  if (!h->timing) return go();
  if (h->pending.size() > 200000) {
    cudaError_t e = collect_times(h);
    if (e != cudaSuccess) return e;
  }
  pic_handle::Pending p{take_event(h), take_event(h), cls};
  cudaEventRecord(p.a, h->stream);
  cudaError_t e = go();
  cudaEventRecord(p.b, h->stream);
  h->pending.push_back(p);
  return e;
}

void* dalloc(pic_handle* h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();  // reported by the null return; a later launch check must not see it
    return nullptr;
  }
  h->allocs.push_back(p);
  return p;
}

// Free one allocation of the handle's list.
void dfree(pic_handle* h, void*& p) {
  if (!p) return;
  cudaFree(p);
  for (auto& q : h->allocs)
    if (q == p) q = nullptr;
  p = nullptr;
}

// Leaver and spill lists with room for n particles each (every particle of the run fits, so a
// step can hand all of them on, and nothing is dropped however many bins are full).
int alloc_lists(pic_handle* h, long long n) {
  const pic_config& c = h->cfg;
  long long want = (long long)h->ncell * h->cap / 4;
  if (want < n) want = n;
  if (want < 65536) want = 65536;
  if (want <= h->lv_cap && want <= h->sp_cap) return PIC_OK;
  for (int a = 0; a < 9; ++a) {
    dfree(h, h->lv[a]);
    dfree(h, h->sp[a]);
  }
  h->lv_cap = h->sp_cap = 0;
  for (int a = 0; a < 9; ++a) {
    if (a == 2 && c.ndim == 2) continue;
    if (a == 7 && !h->has_w) continue;
    if (a == 8 && !h->has_id) continue;
    const size_t bytes = (size_t)want * (a == 0 || a == 8 ? 4 : h->es);
    if (!(h->lv[a] = dalloc(h, bytes)) || !(h->sp[a] = dalloc(h, bytes)))
      return fail(h, PIC_E_OOM, "leaver / spill list allocation failed");
  }
  h->lv_cap = h->sp_cap = want;
  h->grow_gen++;  // new list addresses: batched runs re-upload their tables
  return PIC_OK;
}

void lattice_dims(int ndim, int ppc, int out[3]) {
  out[0] = out[1] = out[2] = 1;
  if (ndim == 2) {
    int d = (int)floor(sqrt((double)ppc));
    while (d > 1 && ppc % d) --d;
    out[0] = d;
    out[2] = ppc / d;
    return;
  }
  // most even split a <= b <= c of ppc = a b c (smallest c - a)
  int best = 1 << 30;
  for (int a = 1; a * a * a <= ppc; ++a) {
    if (ppc % a) continue;
    for (int b = a; a * b * b <= ppc; ++b) {
      if ((ppc / a) % b) continue;
      int c = ppc / (a * b);
      if (c - a < best) {
        best = c - a;
        out[0] = a;
        out[1] = b;
        out[2] = c;
      }
    }
  }
}

void rebuild_taps(pic_handle* h) {
  const pic_config& c = h->cfg;
  std::vector<double> F = filter_taps(c.filter_nbin, c.filter_ncomp, c.filter_comp_alpha);
  std::vector<double> one{1.0};
  const std::vector<double>& Fg = (c.filter_targets & PIC_FILTER_GATHER) ? F : one;
  const std::vector<double>& Fj = (c.filter_targets & PIC_FILTER_J) ? F : one;
  double te[9], tb[9];
  psi_stencil(h->pe, te);
  if (c.correction_mode == PIC_CORR_RATIONAL) {  // Psi_E Psi_B^-1 on E in the FP64 z-line pass
    const double one[5] = {1, 0, 0, 0, 0};
    psi_stencil(one, tb);
    psi_stencil(one, te);
  } else {
    psi_stencil(h->pb, tb);
  }
  h->zt_e = convolve(std::vector<double>(te, te + 9), Fg);
  h->zt_b = convolve(std::vector<double>(tb, tb + 9), Fg);
  h->xt_g = Fg;
  h->zt_j = Fj;
  h->xt_j = Fj;
}

// Particle tiles of the run's grid (push_tiles), spread over up to `spread` blocks.
static void set_tiles(pic_handle* h, int spread) {
  int nt[3], te[3];
  const bool ho = h->cfg.shape_order != 1 || h->cfg.scheme == PIC_MOMENTUM;  // the run's push is k_push_ho
  push_tiles(h->cfg.ndim, h->es, ho, h->cfg.nx, h->cfg.ny, h->cfg.nz, spread, nt, te);
  h->ntx = nt[0];
  h->nty = nt[1];
  h->ntz = nt[2];
  h->tex = te[0];
  h->tey = te[1];
  h->tez = te[2];
}

template <typename T>
RunDev<T> make_run(pic_handle* h, int parity) {
  RunDev<T> r;
  memset(&r, 0, sizeof r);
  const pic_config& c = h->cfg;
  r.ndim = c.ndim;
  r.nx = c.nx;
  r.ny = c.ny;
  r.nz = c.nz;
  r.ncell = h->ncell;
  r.ntx = h->ntx;
  r.nty = h->nty;
  r.ntz = h->ntz;
  r.tex = h->tex;
  r.tey = h->tey;
  r.tez = h->tez;
  r.cap = h->cap;
  r.scheme = c.scheme;
  r.dtdx = (T)(c.dt / c.dx);
  r.dtdy = (T)(c.dt / c.dy);
  r.dtdz = (T)(c.dt / c.dz);
  r.u0 = (T)h->u0;
  r.hq = (T)(0.5 * c.dt);
  r.wconst = (T)h->w0;
  const double dV = c.dx * c.dy * c.dz;
  r.jfx = (T)(-c.dx / (dV * c.dt));
  r.jfy = (T)(-c.dy / (dV * c.dt));
  r.jfz = (T)(-c.dz / (dV * c.dt));
  r.jfy2d = (T)(1.0 / dV);
  for (int q = 0; q < 6; ++q) r.g[q] = (T*)h->g[q];
  for (int q = 0; q < 3; ++q) r.j[q] = (T*)h->f[6 + q];
  for (int s = 0; s < 2; ++s)
    for (int io = 0; io < 2; ++io) {
      int b = io == 0 ? parity : 1 - parity;
      SpeciesBuf<T> sb;
      sb.ox = (T*)h->parr[s][b][0];
      sb.oy = (T*)h->parr[s][b][1];
      sb.oz = (T*)h->parr[s][b][2];
      sb.dux = (T*)h->parr[s][b][3];
      sb.duy = (T*)h->parr[s][b][4];
      sb.duz = (T*)h->parr[s][b][5];
      sb.w = (T*)h->parr[s][b][6];
      sb.id = (unsigned*)h->parr[s][b][7];
      sb.cnt = h->cnt[s][b];
      if (io == 0) r.in[s] = sb; else r.out[s] = sb;
    }
  r.lv.key = (int*)h->lv[0];
  r.lv.ox = (T*)h->lv[1];
  r.lv.oy = (T*)h->lv[2];
  r.lv.oz = (T*)h->lv[3];
  r.lv.dux = (T*)h->lv[4];
  r.lv.duy = (T*)h->lv[5];
  r.lv.duz = (T*)h->lv[6];
  r.lv.w = (T*)h->lv[7];
  r.lv.id = (unsigned*)h->lv[8];
  r.lv_count = h->d_lv_count + parity;
  r.lv_other = h->d_lv_count + (1 - parity);
  r.lv_cap = h->lv_cap;
  r.sp.key = (int*)h->sp[0];
  r.sp.ox = (T*)h->sp[1];
  r.sp.oy = (T*)h->sp[2];
  r.sp.oz = (T*)h->sp[3];
  r.sp.dux = (T*)h->sp[4];
  r.sp.duy = (T*)h->sp[5];
  r.sp.duz = (T*)h->sp[6];
  r.sp.w = (T*)h->sp[7];
  r.sp.id = (unsigned*)h->sp[8];
  r.sp_in = h->d_sp_count + parity;
  r.sp_out = h->d_sp_count + (1 - parity);
  r.sp_cap = h->sp_cap;
  r.sp_total = h->d_sp_total;
  r.err = h->d_err;
  r.kin = nullptr;
  return r;
}

template <typename T>
SepArgs<T> sep_args(pic_handle* h, bool copies) {
  SepArgs<T> a;
  memset(&a, 0, sizeof a);
  const pic_config& c = h->cfg;
  a.nx = c.nx;
  a.ny = c.ny;
  a.nz = c.nz;
  a.ndim = c.ndim;
  a.err = h->d_err;
  a.spread = h->nsm;
  auto put = [](T* dst, const std::vector<double>& v) {
    for (size_t i = 0; i < v.size(); ++i) dst[i] = (T)v[i];
  };
  if (copies) {
    a.ncomp = 6;
    for (int q = 0; q < 3; ++q) a.zero[q] = (T*)h->f[6 + q];  // the current, zeroed before the push
    for (int q = 0; q < 6; ++q) {
      a.src[q] = (const T*)h->f[q];
      a.dst[q] = (T*)h->g[q];
      a.zset[q] = q < 2 ? 0 : 1;  // Psi_E on Ex, Ey; Psi_B on Ez, Bx, By, Bz
    }
    a.hz[0] = (int)(h->zt_e.size() / 2);
    a.hz[1] = (int)(h->zt_b.size() / 2);
    put(a.zt[0], h->zt_e);
    put(a.zt[1], h->zt_b);
    a.hx = a.hy = (int)(h->xt_g.size() / 2);
    put(a.xt, h->xt_g);
    put(a.yt, h->xt_g);
  } else {
    a.ncomp = 3;
    for (int q = 0; q < 3; ++q) {
      a.src[q] = (const T*)h->f[6 + q];
      a.dst[q] = (T*)h->jf[q];
      a.zset[q] = 0;
    }
    a.hz[0] = a.hz[1] = (int)(h->zt_j.size() / 2);
    put(a.zt[0], h->zt_j);
    put(a.zt[1], h->zt_j);
    a.hx = a.hy = (int)(h->xt_j.size() / 2);
    put(a.xt, h->xt_j);
    put(a.yt, h->xt_j);
  }
  return a;
}

template <typename T>
YeeArgs<T> yee_args(pic_handle* h, double hstep) {
  YeeArgs<T> a;
  const pic_config& c = h->cfg;
  a.ex = (T*)h->f[0];
  a.ey = (T*)h->f[1];
  a.ez = (T*)h->f[2];
  a.bx = (T*)h->f[3];
  a.by = (T*)h->f[4];
  a.bz = (T*)h->f[5];
  a.oex = (T*)h->fb[0];
  a.oey = (T*)h->fb[1];
  a.oez = (T*)h->fb[2];
  a.obx = (T*)h->fb[3];
  a.oby = (T*)h->fb[4];
  a.obz = (T*)h->fb[5];
  void* const* js = (h->cfg.filter_targets & PIC_FILTER_J) ? h->jf : h->f + 6;
  a.jx = (const T*)js[0];
  a.jy = (const T*)js[1];
  a.jz = (const T*)js[2];
  a.nx = c.nx;
  a.ny = c.ny;
  a.nz = c.nz;
  a.cx = (T)(hstep / c.dx);
  a.cy = (T)(hstep / c.dy);
  a.cz = (T)(hstep / c.dz);
  a.h = (T)hstep;
  a.err = h->d_err;
  a.spread = h->nsm;
  if (c.field_solver == PIC_CK) {
    a.ck = 1;
    a.wx0 = (T)(1.0 - 2.0 * c.ck_beta_x);
    a.wx1 = (T)c.ck_beta_x;
    a.wz0 = (T)(1.0 - 2.0 * c.ck_beta_z);
    a.wz1 = (T)c.ck_beta_z;
  }
  return a;
}

void swap_fields(pic_handle* h);

template <typename T>
int step_once(pic_handle* h) {
  cudaStream_t st = h->stream;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  const bool rec = !h->no_diag && h->cfg.diag_every > 0 && (h->nstep + 1) % h->cfg.diag_every == 0;
  (void)fb;
  // 1. field copies seen by the particles: Psi(D_z) and the gather filter; zeroes J
  SepArgs<T> ca = sep_args<T>(h, true);
  CK(launch(h, PIC_K_COPIES, [&] { return launch_sep<T>(ca, st); }), "copy stencil");
  if (h->cfg.correction_mode == PIC_CORR_RATIONAL) {  // Psi_E / Psi_B on the Ex, Ey copies
    InvPsiArgs<T> ia;
    ia.f[0] = (T*)h->g[0];
    ia.f[1] = (T*)h->g[1];
    ia.work = (double2*)h->inv_work;
    ia.nxy = (long long)h->cfg.nx * h->cfg.ny;
    ia.nz = h->cfg.nz;
    ia.nf = h->inv_nf;
    for (int q = 0; q < 4; ++q) {
      ia.lam_re[q] = h->inv_lr[q];
      ia.lam_im[q] = h->inv_li[q];
    }
    ia.scale = h->inv_scale;
    psi_stencil(h->pe, ia.pe_taps);
    CK(launch(h, PIC_K_COPIES, [&] { return launch_inverse_psi_z<T>(ia, st); }), "inverse Psi_B");
  }
  // 2-5. gather, Boris, move, Esirkepov, rebin
  RunDev<T> r = make_run<T>(h, h->parity);
  r.kin = rec ? h->d_kin : nullptr;
  if (h->cfg.shape_order == 1 && h->cfg.scheme != PIC_MOMENTUM)
    CK(launch(h, PIC_K_PUSH, [&] { return launch_push<T>(r, 2 * h->cfg.ppc_per_species, st); }), "push");
  else
    CK(launch(h, PIC_K_PUSH, [&] { return launch_push_ho<T>(r, h->cfg.shape_order, h->cfg.scheme, st); }), "push");
  // particles waiting in the spill list (their bin was full): pushed one per thread, handed to the
  // leaver list
  CK(launch(h, PIC_K_SPILL,
            [&] { return launch_push_spill<T>(r, h->cfg.shape_order, h->cfg.scheme, st); }),
     "spill push");
  CK(launch(h, PIC_K_MIGRATE, [&] { return launch_migrate<T>(r, h->d_lv_count + (1 - h->parity), st); }),
     "migrate");
  // 6. current filter
  if (h->cfg.filter_targets & PIC_FILTER_J) {
    SepArgs<T> ja = sep_args<T>(h, false);
    CK(launch(h, PIC_K_FILTER, [&] { return launch_sep<T>(ja, st); }), "current filter");
  }
  // 7. Yee: B half, E full, B half (one fused launch); 8. on diagnostic steps the same launch records
  // the field energies of the new state into the history slot (a separate reduction on tiny grids)
  YeeArgs<T> ye = yee_args<T>(h, h->cfg.dt);
  const pic_config& c = h->cfg;
  HistCtl hc{h->d_hist, h->hist_cap, h->d_hist_count, h->d_kin};
  const bool fused_diag = rec && yee_records_energy(c.ndim, c.nx, c.ny, c.nz, ye.ck);
  CK(launch(h, PIC_K_YEE,
            [&] { return launch_yee_fused<T>(ye, c.ndim, st, h->d_red_yee, fused_diag ? &hc : nullptr); }),
     "yee");
  swap_fields(h);  // the new E, B are in the other buffers
  if (rec) {
    if (!fused_diag) {
      const T* f6[6];
      for (int q = 0; q < 6; ++q) f6[q] = (const T*)h->f[q];
      CK(launch(h, PIC_K_DIAG, [&] { return launch_field_energy<T>(f6, h->ncell, nullptr, h->d_red, hc, st); }),
         "field energy");
    }
    h->nhist++;
  }
  h->parity ^= 1;
  h->nstep++;
  return PIC_OK;
}

// E and B of the new step were written to the other buffers: they become the current ones.
void swap_fields(pic_handle* h) {
  for (int q = 0; q < 6; ++q) {
    void* t = h->f[q];
    h->f[q] = h->fb[q];
    h->fb[q] = t;
  }
}

int check_err(pic_handle* h) {
  int e = 0;
  CK(cudaStreamSynchronize(h->stream), "synchronize");
  CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
  if (!e) return PIC_OK;
  CK(cudaMemset(h->d_err, 0, sizeof(int)), "clear error flag");
  if (e & ERR_OVERFLOW) return fail(h, PIC_E_OVERFLOW, "a cell's particle bin overflowed; raise bin_capacity");
  if (e & ERR_NONFINITE) return fail(h, PIC_E_NONFINITE, "a particle became non-finite or moved more than a cell");
  if (e & ERR_IMPORT) return fail(h, PIC_E_ARG, "imported particle with invalid cell or species");
  if (e & ERR_TIMEOUT) return fail(h, PIC_E_TIMEOUT, "a bounded device wait gave up");
  if (e & ERR_IDS) return fail(h, PIC_E_STATE, "particle ids are not a permutation of 0 .. N-1");
  return fail(h, PIC_E_CUDA, "unknown device error flag");
}

template <typename T>
int init_beam(pic_handle* h) {
  const pic_config& c = h->cfg;
  int lat[3];
  lattice_dims(c.ndim, c.ppc_per_species, lat);
  RunDev<T> r = make_run<T>(h, h->parity);
  CK(launch(h, PIC_K_OTHER,
            [&] {
              return launch_init_beam<T>(r, c.ppc_per_species, lat, h->u0, h->w0, c.jitter, c.u_th, c.sigma_perp,
                                         c.seed, h->stream);
            }),
     "init beam");
  return PIC_OK;
}

int ensure_stage(pic_handle* h, long long n) {
  if (n <= h->stage_n) return PIC_OK;
  for (int q = 0; q < 10; ++q)
    if (h->stage[q]) {
      cudaFree(h->stage[q]);
      for (auto& p : h->allocs)
        if (p == h->stage[q]) p = nullptr;
      h->stage[q] = nullptr;
    }
  // cell, species, ox, oy, oz, dux, duy, duz, w, id
  const size_t sz[10] = {4, 4, h->es, h->es, h->es, h->es, h->es, h->es, h->es, 4};
  for (int q = 0; q < 10; ++q) {
    h->stage[q] = dalloc(h, sz[q] * (size_t)n);
    if (!h->stage[q]) return fail(h, PIC_E_OOM, "staging allocation failed");
  }
  h->stage_n = n;
  return PIC_OK;
}

template <typename T>
FlatDev<T> stage_view(pic_handle* h, long long n) {
  FlatDev<T> f;
  f.np = n;
  f.cell = (int*)h->stage[0];
  f.species = (int*)h->stage[1];
  f.ox = (T*)h->stage[2];
  f.oy = (T*)h->stage[3];
  f.oz = (T*)h->stage[4];
  f.dux = (T*)h->stage[5];
  f.duy = (T*)h->stage[6];
  f.duz = (T*)h->stage[7];
  f.w = (T*)h->stage[8];
  f.id = (unsigned*)h->stage[9];
  return f;
}

template <typename T>
int set_state_t(pic_handle* h, const pic_state* s) {
  cudaStream_t st = h->stream;
  drop_graph(h);
  const cudaMemcpyKind k = s->where == PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  void* const src[6] = {s->ex, s->ey, s->ez, s->bx, s->by, s->bz};
  for (int q = 0; q < 6; ++q)
    if (src[q]) CK(cudaMemcpyAsync(h->f[q], src[q], fb, k, st), "copy field in");
  const long long n = s->np;
  if (n == -1) return PIC_OK;  // fields only: particles untouched
  if (n < 0) return fail(h, PIC_E_ARG, "negative particle count");
  // particles: clear bins, leaver and spill counters, stage, bin
  for (int sp = 0; sp < 2; ++sp)
    for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(h->cnt[sp][b], 0, sizeof(int) * h->ncell, st), "clear counts");
  CK(cudaMemsetAsync(h->d_lv_count, 0, 2 * sizeof(int), st), "clear leaver counters");
  CK(cudaMemsetAsync(h->d_sp_count, 0, 2 * sizeof(int), st), "clear spill counters");
  h->parity = 0;
  h->sp_pending = false;
  if (n == 0) return PIC_OK;
  if (n > h->sp_cap) {  // room for every particle in the leaver and spill lists
    CK(cudaStreamSynchronize(st), "synchronize");
    int rc = alloc_lists(h, n);
    if (rc) return rc;
  }
  if (!s->cell || !s->species || !s->ox || !s->oz || !s->dux || !s->duy || !s->duz ||
      (h->cfg.ndim == 3 && !s->oy))
    return fail(h, PIC_E_ARG, "missing particle array");
  int rc = ensure_stage(h, n);
  if (rc) return rc;
  FlatDev<T> f = stage_view<T>(h, n);
  CK(cudaMemcpyAsync(f.cell, s->cell, 4 * (size_t)n, k, st), "copy cell");
  CK(cudaMemcpyAsync(f.species, s->species, 4 * (size_t)n, k, st), "copy species");
  CK(cudaMemcpyAsync(f.ox, s->ox, sizeof(T) * n, k, st), "copy ox");
  if (h->cfg.ndim == 3) CK(cudaMemcpyAsync(f.oy, s->oy, sizeof(T) * n, k, st), "copy oy");
  else f.oy = nullptr;
  CK(cudaMemcpyAsync(f.oz, s->oz, sizeof(T) * n, k, st), "copy oz");
  CK(cudaMemcpyAsync(f.dux, s->dux, sizeof(T) * n, k, st), "copy dux");
  CK(cudaMemcpyAsync(f.duy, s->duy, sizeof(T) * n, k, st), "copy duy");
  CK(cudaMemcpyAsync(f.duz, s->duz, sizeof(T) * n, k, st), "copy duz");
  if (s->w && h->has_w) CK(cudaMemcpyAsync(f.w, s->w, sizeof(T) * n, k, st), "copy w");
  else f.w = nullptr;
  if (s->id && h->has_id) CK(cudaMemcpyAsync(f.id, s->id, 4 * (size_t)n, k, st), "copy id");
  else f.id = nullptr;
  RunDev<T> r = make_run<T>(h, 0);
  CK(launch(h, PIC_K_OTHER, [&] { return launch_import<T>(r, f, st); }), "import");
  return PIC_OK;
}

// Particles per species in the bins of the current buffers (the spill list not included).
int count_bins(pic_handle* h, long long out[2]) {
  for (int s = 0; s < 2; ++s) {
    CK(launch_count_prefix(h->cnt[s][h->parity], h->ncell, h->cap, h->d_offs, h->d_bsum, h->d_total + s, h->stream),
       "count prefix");
  }
  CK(cudaMemcpyAsync(out, h->d_total, 2 * sizeof(long long), cudaMemcpyDeviceToHost, h->stream), "read counts");
  CK(cudaStreamSynchronize(h->stream), "synchronize");
  return PIC_OK;
}

// Empty the spill list into larger bins. Particles whose bin was full wait in the spill list (the
// step pushes them from there, so nothing is lost); here, at a synchronising call, every particle
// (bins and list) is exported to the staging arrays, the bins of both buffers are reallocated with
// a capacity a quarter above the fullest cell (and at least half again the old one), and the
// particles are imported back into the current buffers. The step parity is kept. A failed
// allocation keeps the old bins (and the list, which the step still pushes) and reports PIC_E_OOM.
template <typename T>
int settle(pic_handle* h) {
  cudaStream_t st = h->stream;
  int waiting = 0;
  CK(cudaMemcpyAsync(&waiting, h->d_sp_count + h->parity, sizeof(int), cudaMemcpyDeviceToHost, st),
     "read spill count");
  CK(cudaStreamSynchronize(st), "synchronize");
  h->sp_pending = false;
  if (waiting <= 0) return PIC_OK;
  const long long nsp = waiting < h->sp_cap ? waiting : h->sp_cap;
  // the fullest cell: the counts keep every insertion, the spilled ones included
  CK(cudaMemsetAsync(h->d_maxc, 0, sizeof(int), st), "clear max count");
  CK(launch(h, PIC_K_OTHER,
            [&] { return launch_max_count(h->cnt[0][h->parity], h->cnt[1][h->parity], h->ncell, h->d_maxc, st); }),
     "max count");
  int maxc = 0;
  CK(cudaMemcpyAsync(&maxc, h->d_maxc, sizeof(int), cudaMemcpyDeviceToHost, st), "read max count");
  long long cnts[2];
  int rc = count_bins(h, cnts);  // synchronises
  if (rc) return rc;
  const int align = (int)(64 / h->es);
  long long nc = (long long)maxc + maxc / 4 + 8;
  if (nc < (long long)h->cap + h->cap / 2) nc = (long long)h->cap + h->cap / 2;
  nc = (nc + align - 1) / align * align;
  if (nc > (1 << 24)) return fail(h, PIC_E_OOM, "a cell holds more particles than a bin can (2^24)");
  // every particle into the staging arrays: bins by species, then the list
  const long long n = cnts[0] + cnts[1] + nsp;
  rc = ensure_stage(h, n);
  if (rc) return rc;
  FlatDev<T> f = stage_view<T>(h, n);
  if (h->cfg.ndim != 3) f.oy = nullptr;
  if (!h->has_w) f.w = nullptr;
  if (!h->has_id) f.id = nullptr;
  RunDev<T> r = make_run<T>(h, h->parity);
  long long base = 0;
  for (int sp = 0; sp < 2; ++sp) {
    CK(launch_count_prefix(h->cnt[sp][h->parity], h->ncell, h->cap, h->d_offs, h->d_bsum, h->d_total, st),
       "count prefix");
    CK(launch(h, PIC_K_OTHER, [&] { return launch_export<T>(r, sp, h->d_offs, base, f, st); }), "export");
    base += cnts[sp];
  }
  CK(launch(h, PIC_K_OTHER, [&] { return launch_spill_export<T>(r, nsp, base, f, st); }), "spill export");
  CK(cudaStreamSynchronize(st), "synchronize");
  // new bins for both buffers and species; the old ones are freed only once all are in place
  const pic_config& c = h->cfg;
  const size_t slots = (size_t)h->ncell * (size_t)nc;
  void* np_[2][2][8] = {};
  bool ok = true;
  for (int sp = 0; sp < 2 && ok; ++sp)
    for (int b = 0; b < 2 && ok; ++b)
      for (int a = 0; a < 8 && ok; ++a) {
        if (!h->parr[sp][b][a]) continue;  // arrays the run does not carry
        ok = (np_[sp][b][a] = dalloc(h, slots * (a == 7 ? 4 : h->es))) != nullptr;
      }
  if (!ok) {
    for (int sp = 0; sp < 2; ++sp)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 8; ++a) dfree(h, np_[sp][b][a]);
    return fail(h, PIC_E_OOM, "particle bin growth: allocation failed");
  }
  for (int sp = 0; sp < 2; ++sp)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 8; ++a)
        if (h->parr[sp][b][a]) {
          dfree(h, h->parr[sp][b][a]);
          h->parr[sp][b][a] = np_[sp][b][a];
        }
  (void)c;
  h->cap = (int)nc;
  for (int sp = 0; sp < 2; ++sp)
    for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(h->cnt[sp][b], 0, sizeof(int) * h->ncell, st), "clear counts");
  CK(cudaMemsetAsync(h->d_sp_count, 0, 2 * sizeof(int), st), "clear spill counters");
  CK(cudaMemsetAsync(h->d_lv_count, 0, 2 * sizeof(int), st), "clear leaver counters");
  RunDev<T> r2 = make_run<T>(h, h->parity);
  CK(launch(h, PIC_K_OTHER, [&] { return launch_import<T>(r2, f, st); }), "re-bin");
  CK(cudaStreamSynchronize(st), "synchronize");
  drop_graph(h);
  h->grow_gen++;
  return PIC_OK;
}

template <typename T>
int count_particles(pic_handle* h, long long out[2]) {
  int rc = settle<T>(h);
  if (rc) return rc;
  return count_bins(h, out);
}

template <typename T>
int charge_residual_t(pic_handle* h, double out[3]) {
  int rc0 = settle<T>(h);
  if (rc0) return rc0;
  cudaStream_t st = h->stream;
  const pic_config& c = h->cfg;
  if (!h->d_rho) {
    h->d_rho = (double*)dalloc(h, 2 * sizeof(double) * (size_t)h->ncell);
    h->d_gauss = (double*)dalloc(h, gauss_scratch_bytes() + 4 * sizeof(double));
    if (!h->d_rho || !h->d_gauss) return fail(h, PIC_E_OOM, "residual scratch allocation failed");
    CK(cudaMemset(h->d_gauss, 0, gauss_scratch_bytes() + 4 * sizeof(double)), "clear residual scratch");
  }
  double* rho = h->d_rho;
  double* rhof = h->d_rho + h->ncell;
  double* dout = h->d_gauss + gauss_scratch_bytes() / sizeof(double);
  CK(cudaMemsetAsync(rho, 0, sizeof(double) * (size_t)h->ncell, st), "clear rho");
  RunDev<T> r = make_run<T>(h, h->parity);
  const double dV = c.dx * c.dy * c.dz;
  CK(launch(h, PIC_K_OTHER, [&] { return launch_rho<T>(r, c.shape_order, 1.0 / dV, rho, st); }), "rho");
  // F rho with the current filter's taps, in FP64
  SepArgs<double> a;
  memset(&a, 0, sizeof a);
  a.nx = c.nx;
  a.ny = c.ny;
  a.nz = c.nz;
  a.ndim = c.ndim;
  a.ncomp = 1;
  a.src[0] = rho;
  a.dst[0] = rhof;
  a.hz[0] = a.hz[1] = (int)(h->zt_j.size() / 2);
  for (size_t i = 0; i < h->zt_j.size(); ++i) a.zt[0][i] = a.zt[1][i] = h->zt_j[i];
  a.hx = a.hy = (int)(h->xt_j.size() / 2);
  for (size_t i = 0; i < h->xt_j.size(); ++i) a.xt[i] = a.yt[i] = h->xt_j[i];
  CK(launch(h, PIC_K_OTHER, [&] { return launch_sep<double>(a, st); }), "filter rho");
  CK(launch(h, PIC_K_OTHER,
            [&] {
              return launch_gauss_residual<T>((const T*)h->f[0], (const T*)h->f[1], (const T*)h->f[2], rhof, c.nx,
                                              c.ny, c.nz, 1.0 / c.dx, 1.0 / c.dy, 1.0 / c.dz, h->d_gauss, dout, st);
            }),
     "gauss residual");
  CK(cudaMemcpyAsync(out, dout, 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "read residual");
  CK(cudaStreamSynchronize(st), "synchronize");
  return check_err(h);
}

template <typename T>
int get_state_t(pic_handle* h, pic_state* s) {
  int rc = check_err(h);
  if (rc) return rc;
  rc = settle<T>(h);
  if (rc) return rc;
  cudaStream_t st = h->stream;
  const cudaMemcpyKind k = s->where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  void* const dst[6] = {s->ex, s->ey, s->ez, s->bx, s->by, s->bz};
  for (int q = 0; q < 6; ++q)
    if (dst[q]) CK(cudaMemcpyAsync(dst[q], h->f[q], fb, k, st), "copy field out");
  s->u_drift = h->u0;
  long long cnts[2];
  rc = count_particles<T>(h, cnts);
  if (rc) return rc;
  const long long n = cnts[0] + cnts[1];
  if (!s->cell && !s->species && !s->ox && !s->oy && !s->oz && !s->dux && !s->duy && !s->duz && !s->w && !s->id) {
    s->np = n;  // fields only
    CK(cudaStreamSynchronize(st), "synchronize");
    return check_err(h);
  }
  if (s->np < n) {
    s->np = n;
    return fail(h, PIC_E_ARG, "particle arrays too small (np updated to the required count)");
  }
  s->np = n;
  if (n == 0) return PIC_OK;
  rc = ensure_stage(h, n);
  if (rc) return rc;
  FlatDev<T> f = stage_view<T>(h, n);
  if (h->cfg.ndim != 3) f.oy = nullptr;
  RunDev<T> r = make_run<T>(h, h->parity);
  long long base = 0;
  for (int sp = 0; sp < 2; ++sp) {
    CK(launch_count_prefix(h->cnt[sp][h->parity], h->ncell, h->cap, h->d_offs, h->d_bsum, h->d_total, st),
       "count prefix");
    CK(launch(h, PIC_K_OTHER, [&] { return launch_export<T>(r, sp, h->d_offs, base, f, st); }), "export");
    base += cnts[sp];
  }
  if (s->cell) CK(cudaMemcpyAsync(s->cell, f.cell, 4 * (size_t)n, k, st), "copy cell out");
  if (s->species) CK(cudaMemcpyAsync(s->species, f.species, 4 * (size_t)n, k, st), "copy species out");
  if (s->ox) CK(cudaMemcpyAsync(s->ox, f.ox, sizeof(T) * n, k, st), "copy ox out");
  if (s->oy && f.oy) CK(cudaMemcpyAsync(s->oy, f.oy, sizeof(T) * n, k, st), "copy oy out");
  if (s->oz) CK(cudaMemcpyAsync(s->oz, f.oz, sizeof(T) * n, k, st), "copy oz out");
  if (s->dux) CK(cudaMemcpyAsync(s->dux, f.dux, sizeof(T) * n, k, st), "copy dux out");
  if (s->duy) CK(cudaMemcpyAsync(s->duy, f.duy, sizeof(T) * n, k, st), "copy duy out");
  if (s->duz) CK(cudaMemcpyAsync(s->duz, f.duz, sizeof(T) * n, k, st), "copy duz out");
  if (s->w) CK(cudaMemcpyAsync(s->w, f.w, sizeof(T) * n, k, st), "copy w out");
  if (s->id) CK(cudaMemcpyAsync(s->id, f.id, 4 * (size_t)n, k, st), "copy id out");
  CK(cudaStreamSynchronize(st), "synchronize");
  return check_err(h);
}

template <typename T>
int energy_t(pic_handle* h, pic_energy_t* out) {
  int rc0 = settle<T>(h);
  if (rc0) return rc0;
  cudaStream_t st = h->stream;
  CK(cudaMemsetAsync(h->d_acc, 0, 8 * sizeof(double), st), "zero accumulators");
  const T* f6[6];
  for (int q = 0; q < 6; ++q) f6[q] = (const T*)h->f[q];
  HistCtl none{nullptr, 0, nullptr, nullptr};
  CK(launch(h, PIC_K_DIAG, [&] { return launch_field_energy<T>(f6, h->ncell, h->d_acc, h->d_red, none, st); }),
     "field energy");
  RunDev<T> r = make_run<T>(h, h->parity);
  CK(launch(h, PIC_K_DIAG, [&] { return launch_kinetic<T>(r, h->d_acc + 3, st); }), "kinetic energy");
  double acc[8];
  CK(cudaMemcpyAsync(acc, h->d_acc, sizeof acc, cudaMemcpyDeviceToHost, st), "read energies");
  long long cnts[2];
  int rc = count_particles<T>(h, cnts);
  if (rc) return rc;
  const pic_config& c = h->cfg;
  const double dV = c.dx * c.dy * c.dz;
  out->w_e = 0.5 * acc[0] * dV;
  out->w_b = 0.5 * acc[1] * dV;
  out->w_perp = 0.5 * acc[2] * dV;
  out->k = acc[3];
  out->total = out->w_e + out->w_b + out->k;
  out->np = cnts[0] + cnts[1];
  return check_err(h);
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Public ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

void pic_config_default(pic_config* c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  c->ndim = 2;
  c->nx = 64;
  c->ny = 1;
  c->nz = 128;
  c->dx = c->dy = c->dz = 1.0;
  c->dt = 0.5;
  c->gamma = 130.0;
  c->scheme = PIC_GALERKIN;
  c->shape_order = 1;
  c->precision = PIC_FP64;
  c->ppc_per_species = 4;
  c->omega_p_dz = 0.3868;
  c->jitter = 0.1;
  c->u_th = 1e-4;
  c->sigma_perp = 0.0;
  c->filter_nbin = 1;
  c->filter_ncomp = 1;
  c->filter_comp_alpha = 3.0;
  c->filter_targets = PIC_FILTER_J | PIC_FILTER_GATHER;
  c->seed = 1;
  c->init_beam = 1;
  c->bin_capacity = 0;
  c->track_ids = 0;
  c->field_solver = PIC_YEE;
  c->ck_beta_x = c->ck_beta_z = 0.125;
}

int pic_compute_correction_coeffs(int scheme, double alpha, double psi_e[5], double psi_b[5]) {
  if (!psi_e || !psi_b) return PIC_E_ARG;
  return correction_coeffs(scheme, alpha, psi_e, psi_b);
}

int pic_create(const pic_config* cfg_in, pic_handle** out) {
  if (!cfg_in || !out) return PIC_E_ARG;
  *out = nullptr;
  pic_config c = *cfg_in;
  if (c.ndim == 2) {
    c.ny = 1;
    c.dy = 1.0;
  }
  if ((c.ndim != 2 && c.ndim != 3) || c.nx < 1 || c.ny < 1 || c.nz < 1 || !(c.dx > 0) || !(c.dy > 0) ||
      !(c.dz > 0) || !(c.dt > 0) || !(c.gamma >= 1.0) ||
      (c.scheme != PIC_GALERKIN && c.scheme != PIC_UNIFORM && c.scheme != PIC_MOMENTUM) ||
      (c.shape_order != 1 && c.shape_order != 3) || (c.precision != PIC_FP32 && c.precision != PIC_FP64) ||
      c.ppc_per_species < 0 || c.ppc_per_species > (1 << 20) || c.bin_capacity > (1 << 24) ||
      c.filter_nbin < 0 || c.filter_ncomp < 0 || c.filter_nbin + c.filter_ncomp > 12 || c.bin_capacity < 0 ||
      c.diag_every < 0 || c.diag_capacity < 0 ||
      (c.correction_mode != PIC_CORR_SPLIT && c.correction_mode != PIC_CORR_RATIONAL) ||
      (c.field_solver != PIC_YEE && c.field_solver != PIC_CK) ||
      (c.field_solver == PIC_CK &&
       (c.ndim != 2 || !(c.ck_beta_x >= 0.0 && c.ck_beta_x <= 0.25) || !(c.ck_beta_z >= 0.0 && c.ck_beta_z <= 0.25))) ||
      (long long)c.nx * c.ny * c.nz > (1ll << 30) - 1)
    return PIC_E_ARG;
  if (c.field_solver == PIC_CK) {
    // sin^2(w dt/2) = dt^2 [sz^2 (1 - 4 bz sx^2) / dz^2 + sx^2 (1 - 4 bx sz^2) / dx^2] is bilinear in
    // (sx^2, sz^2) in [0, 1]^2, so its largest value sits at a corner
    const double ix = 1.0 / (c.dx * c.dx), iz = 1.0 / (c.dz * c.dz);
    const double corner = (1.0 - 4.0 * c.ck_beta_x) * ix + (1.0 - 4.0 * c.ck_beta_z) * iz;
    const double m = fmax(fmax(ix, iz), corner);
    if (c.dt * c.dt * m >= 1.0) return PIC_E_CFL;
  } else {
    const double inv = 1.0 / (c.dx * c.dx) + (c.ndim == 3 ? 1.0 / (c.dy * c.dy) : 0.0) + 1.0 / (c.dz * c.dz);
    if (c.dt >= 1.0 / sqrt(inv)) return PIC_E_CFL;
  }
  pic_handle* h = new pic_handle();
  h->cfg = c;
  h->es = c.precision == PIC_FP32 ? 4 : 8;
  h->ncell = (long long)c.nx * c.ny * c.nz;
  {
    // a grid of few tiles takes smaller ones, spread over the SMs
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 0;
    h->nsm = nsm;
    set_tiles(h, nsm);
  }
  h->u0 = sqrt(c.gamma * c.gamma - 1.0);
  const double wp = c.omega_p_dz / c.dz;
  h->w0 = c.ppc_per_species > 0 ? wp * wp * c.dx * c.dy * c.dz / (2.0 * c.ppc_per_species) : 0.0;
  h->has_w = c.sigma_perp > 0;
  h->has_id = c.track_ids != 0;
  int cap = c.bin_capacity;
  if (cap == 0) cap = c.ppc_per_species * 2 + 8;
  const int align = (int)(64 / h->es);  // bins start on 64-byte boundaries
  cap = (cap + align - 1) / align * align;
  h->cap = cap;
  (void)cudaGetLastError();
  cudaError_t e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g_create_err = std::string("stream creation: ") + cudaGetErrorString(e);
    delete h;
    return PIC_E_CUDA;
  }
  h->stream = h->own;
  const size_t fb = (size_t)h->ncell * h->es;
  bool ok = true;
  for (int q = 0; q < 9 && ok; ++q) ok = (h->f[q] = dalloc(h, fb)) != nullptr;
  for (int q = 0; q < 6 && ok; ++q) ok = (h->fb[q] = dalloc(h, fb)) != nullptr;
  for (int q = 0; q < 6 && ok; ++q) ok = (h->g[q] = dalloc(h, fb)) != nullptr;
  for (int q = 0; q < 3 && ok; ++q) ok = (h->jf[q] = dalloc(h, fb)) != nullptr;
  if (ok && c.correction_mode == PIC_CORR_RATIONAL)  // complex scratch of the z-solves, two components
    ok = (h->inv_work = dalloc(h, 2 * sizeof(double) * 2 * (size_t)h->ncell)) != nullptr;
  const size_t slots = (size_t)h->ncell * cap;
  for (int s = 0; s < 2 && ok; ++s)
    for (int b = 0; b < 2 && ok; ++b) {
      for (int a = 0; a < 8 && ok; ++a) {
        if (a == 1 && c.ndim == 2) continue;
        if (a == 6 && !h->has_w) continue;
        if (a == 7 && !h->has_id) continue;
        ok = (h->parr[s][b][a] = dalloc(h, slots * (a == 7 ? 4 : h->es))) != nullptr;
      }
      if (ok) ok = (h->cnt[s][b] = (int*)dalloc(h, sizeof(int) * h->ncell)) != nullptr;
    }
  if (ok) ok = (h->d_err = (int*)dalloc(h, 16)) != nullptr;
  // leaver list (particles that leave their tile in one step) and spill list (particles whose bin
  // was full), each with room for every particle of the seeded beam
  if (ok) ok = alloc_lists(h, c.init_beam ? 2 * (long long)c.ppc_per_species * h->ncell : 0) == PIC_OK;
  if (ok) ok = (h->d_lv_count = (int*)dalloc(h, 2 * sizeof(int))) != nullptr;
  if (ok) ok = (h->d_sp_count = (int*)dalloc(h, 2 * sizeof(int))) != nullptr;
  if (ok) ok = (h->d_maxc = (int*)dalloc(h, 16)) != nullptr;
  if (ok) ok = (h->d_sp_total = (unsigned long long*)dalloc(h, 16)) != nullptr;
  if (ok) ok = cudaMemset(h->d_sp_total, 0, 16) == cudaSuccess;
  if (ok) ok = cudaHostAlloc((void**)&h->h_sp_mirror, 16, cudaHostAllocDefault) == cudaSuccess;
  if (ok) ok = cudaEventCreateWithFlags(&h->ev_sp, cudaEventDisableTiming) == cudaSuccess;
  if (ok) ok = (h->d_acc = (double*)dalloc(h, 8 * sizeof(double))) != nullptr;
  if (ok) ok = (h->d_red = (double*)dalloc(h, field_energy_scratch_bytes())) != nullptr;
  if (ok) ok = cudaMemset(h->d_red, 0, field_energy_scratch_bytes()) == cudaSuccess;
  if (ok) ok = (h->d_red_yee = (double*)dalloc(h, yee_energy_scratch_bytes(c.ndim, c.nx, c.ny, c.nz, h->nsm))) != nullptr;
  if (ok) ok = cudaMemset(h->d_red_yee, 0, yee_energy_scratch_bytes(c.ndim, c.nx, c.ny, c.nz, h->nsm)) == cudaSuccess;
  if (ok) ok = (h->d_offs = (long long*)dalloc(h, sizeof(long long) * h->ncell)) != nullptr;
  if (ok) ok = (h->d_bsum = (long long*)dalloc(h, sizeof(long long) * (count_prefix_blocks(h->ncell) + 1))) != nullptr;
  if (ok) ok = (h->d_total = (long long*)dalloc(h, 4 * sizeof(long long))) != nullptr;
  h->hist_cap = c.diag_capacity > 0 ? c.diag_capacity : 4096;
  if (ok) ok = (h->d_hist = (double*)dalloc(h, 8 * sizeof(double) * (size_t)h->hist_cap)) != nullptr;
  if (ok) ok = (h->d_hist_count = (int*)dalloc(h, 16)) != nullptr;
  if (ok) ok = (h->d_kin = (double*)dalloc(h, 2 * sizeof(double))) != nullptr;
  if (ok) ok = cudaMemset(h->d_hist_count, 0, 16) == cudaSuccess && cudaMemset(h->d_kin, 0, 2 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    g_create_err = "device allocation failed";
    pic_destroy(h);
    return PIC_E_OOM;
  }
  for (int q = 0; q < 9; ++q) cudaMemsetAsync(h->f[q], 0, fb, h->stream);
  for (int s = 0; s < 2; ++s)
    for (int b = 0; b < 2; ++b) cudaMemsetAsync(h->cnt[s][b], 0, sizeof(int) * h->ncell, h->stream);
  cudaMemsetAsync(h->d_err, 0, 16, h->stream);
  cudaMemsetAsync(h->d_lv_count, 0, 2 * sizeof(int), h->stream);
  cudaMemsetAsync(h->d_sp_count, 0, 2 * sizeof(int), h->stream);
  rebuild_taps(h);
  int rc = PIC_OK;
  if (c.init_beam && c.ppc_per_species > 0)
    rc = c.precision == PIC_FP32 ? init_beam<float>(h) : init_beam<double>(h);
  if (rc == PIC_OK) rc = check_err(h);
  if (rc != PIC_OK) {
    g_create_err = h->err;
    pic_destroy(h);
    return rc;
  }
  *out = h;
  return PIC_OK;
}

int pic_set_stream(pic_handle* h, void* stream) {
  if (!h) return PIC_E_ARG;
  h->stream = stream ? (cudaStream_t)stream : h->own;
  return PIC_OK;
}

int pic_set_correction_stencil(pic_handle* h, const double psi_e[5], const double psi_b[5]) {
  if (!h) return PIC_E_ARG;
  if ((psi_e == nullptr) != (psi_b == nullptr)) return fail(h, PIC_E_ARG, "give both Psi_E and Psi_B, or neither");
  for (int q = 0; q < 5; ++q) {
    h->pe[q] = psi_e ? psi_e[q] : (q == 0 ? 1.0 : 0.0);
    h->pb[q] = psi_b ? psi_b[q] : (q == 0 ? 1.0 : 0.0);
    if (!isfinite(h->pe[q]) || !isfinite(h->pb[q])) return fail(h, PIC_E_ARG, "non-finite coefficient");
  }
  if (h->cfg.correction_mode == PIC_CORR_RATIONAL) {
    int nf = 0;
    double lr[4], li[4], sc = 1.0;
    const int rc = psi_inverse_factors(h->pb, lr, li, &nf, &sc);
    if (rc) return fail(h, rc, "Psi_B has no inverse (a zero on [0, 1] or identically zero)");
    for (int q = 0; q < 4; ++q) {
      h->inv_lr[q] = q < nf ? lr[q] : 0.0;
      h->inv_li[q] = q < nf ? li[q] : 0.0;
    }
    h->inv_nf = nf;
    h->inv_scale = sc;
  }
  rebuild_taps(h);
  drop_graph(h);
  h->adj.ready = false;
  return PIC_OK;
}

}  // extern "C" (the graph helpers below have C++ linkage)

static void drop_graph(pic_handle* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_len = 0;
}

static int run_steps(pic_handle* h, int n) {
  for (int s = 0; s < n; ++s) {
    int rc = h->es == 4 ? step_once<float>(h) : step_once<double>(h);
    if (rc) return rc;
  }
  return PIC_OK;
}

// Capture graph_len steps (an even number covering whole diagnostic periods) on the handle's
// stream into one executable graph. Called with the step counter at a multiple of graph_len.
static int build_graph(pic_handle* h) {
  drop_graph(h);
  const int de = h->cfg.diag_every > 0 ? h->cfg.diag_every : 1;
  int len = 2;
  while (len % de && len <= 64) len += 2;  // past 64: no graph
  if (len > 64) return PIC_E_STATE;  // diagnostics too sparse to unroll into one graph
  const long long nstep0 = h->nstep, nhist0 = h->nhist;
  const int parity0 = h->parity;
  void* f0[6];
  void* fb0[6];
  for (int q = 0; q < 6; ++q) {
    f0[q] = h->f[q];
    fb0[q] = h->fb[q];
  }
  const long long launches0 = h->launches;
  long long counts0[PIC_NKERNEL];
  for (int q = 0; q < PIC_NKERNEL; ++q) counts0[q] = h->tcount[q];
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  int rc = run_steps(h, len);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  h->nstep = nstep0;
  h->nhist = nhist0;
  h->parity = parity0;
  for (int q = 0; q < 6; ++q) {  // an even number of steps: the captured swaps cancel
    h->f[q] = f0[q];
    h->fb[q] = fb0[q];
  }
  h->launches = launches0;
  for (int q = 0; q < PIC_NKERNEL; ++q) h->tcount[q] = counts0[q];
  if (rc != PIC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != PIC_OK ? rc : cuda_fail(h, e, "end capture");
  }
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  h->graph_len = len;
  h->graph_stream = h->stream;
  h->graph_parity = parity0;
  h->graph_f0 = f0[0];
  h->graph_launch_count = 0;
  for (int q = 0; q < PIC_NKERNEL; ++q) h->graph_counts[q] = 0;
  // launches per replay, for pic_launch_count / pic_kernel_times bookkeeping
  return PIC_OK;
}

// The spill list between pic_step calls: after a call, its waiting count is copied to pinned host
// memory behind an event; the next call reads it once the event has completed (no wait) and, when
// particles are waiting, grows the bins first. Under a caller's stream capture neither happens.
static bool capturing(pic_handle* h) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

static int spill_check(pic_handle* h) {
  if (!h->sp_pending || capturing(h)) return PIC_OK;
  const cudaError_t q = cudaEventQuery(h->ev_sp);
  if (q == cudaErrorNotReady) {
    (void)cudaGetLastError();
    return PIC_OK;  // the previous call is still running: look again next time
  }
  h->sp_pending = false;
  if (q != cudaSuccess) return cuda_fail(h, q, "spill count event");
  if (*h->h_sp_mirror <= 0) return PIC_OK;
  return h->es == 4 ? settle<float>(h) : settle<double>(h);
}

static void note_spill(pic_handle* h) {
  if (capturing(h)) return;
  if (cudaMemcpyAsync(h->h_sp_mirror, h->d_sp_count + h->parity, sizeof(int), cudaMemcpyDeviceToHost, h->stream) ==
          cudaSuccess &&
      cudaEventRecord(h->ev_sp, h->stream) == cudaSuccess)
    h->sp_pending = true;
}

static int step_calls(pic_handle* h, int nsteps) {
  // Graph replay when at least two whole graphs fit and timing is off; single steps otherwise.
  const int de = h->cfg.diag_every > 0 ? h->cfg.diag_every : 1;
  int len = 2;
  while (len % de && len <= 64) len += 2;  // past 64 the caller falls back to single steps
  if (h->timing || len > 64 || nsteps < 2 * len) return run_steps(h, nsteps);
  int lead = (int)((len - h->nstep % len) % len);
  int rc = run_steps(h, lead);
  if (rc) return rc;
  nsteps -= lead;
  if (!h->graph || h->graph_len != len || h->graph_stream != h->stream || h->graph_parity != h->parity ||
      h->graph_f0 != h->f[0]) {
    // counts of one replay: run one graph's worth of steps while counting, then capture
    const long long l0 = h->launches;
    long long c0[PIC_NKERNEL];
    for (int q = 0; q < PIC_NKERNEL; ++q) c0[q] = h->tcount[q];
    rc = run_steps(h, len);
    if (rc) return rc;
    nsteps -= len;
    const long long per_launch = h->launches - l0;
    long long per[PIC_NKERNEL];
    for (int q = 0; q < PIC_NKERNEL; ++q) per[q] = h->tcount[q] - c0[q];
    rc = build_graph(h);
    if (rc) return rc;
    h->graph_launch_count = per_launch;
    for (int q = 0; q < PIC_NKERNEL; ++q) h->graph_counts[q] = per[q];
  }
  while (nsteps >= len) {
    CK(cudaGraphLaunch(h->graph, h->stream), "graph launch");
    h->nstep += len;
    h->parity = (h->parity + len) & 1;
    const int de2 = h->cfg.diag_every;
    if (de2 > 0) h->nhist += len / de2;
    h->launches += h->graph_launch_count;
    for (int q = 0; q < PIC_NKERNEL; ++q) h->tcount[q] += h->graph_counts[q];
    nsteps -= len;
  }
  return run_steps(h, nsteps);
}

extern "C" {

int pic_step(pic_handle* h, int nsteps) {
  if (!h || nsteps < 0) return PIC_E_ARG;
  NvtxRange range("pic_step");
  int rc = spill_check(h);
  if (rc) return rc;
  rc = step_calls(h, nsteps);
  if (rc == PIC_OK && nsteps > 0) note_spill(h);
  return rc;
}

int pic_sync(pic_handle* h) {
  if (!h) return PIC_E_ARG;
  return check_err(h);
}

int pic_energy(pic_handle* h, pic_energy_t* out) {
  if (!h || !out) return PIC_E_ARG;
  return h->es == 4 ? energy_t<float>(h, out) : energy_t<double>(h, out);
}

int pic_num_particles(pic_handle* h, long long* np) {
  if (!h || !np) return PIC_E_ARG;
  long long c[2];
  int rc = h->es == 4 ? count_particles<float>(h, c) : count_particles<double>(h, c);
  if (rc) return rc;
  *np = c[0] + c[1];
  return check_err(h);
}

int pic_bin_stats(pic_handle* h, int* cap, long long* spilled) {
  if (!h) return PIC_E_ARG;
  if (cap) *cap = h->cap;
  if (spilled) {
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, h->d_sp_total, sizeof v, cudaMemcpyDeviceToHost, h->stream), "read spill total");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    *spilled = (long long)v;
  }
  return PIC_OK;
}

int pic_get_state(pic_handle* h, pic_state* s) {
  if (!h || !s || (s->where != PIC_HOST && s->where != PIC_DEVICE)) return PIC_E_ARG;
  return h->es == 4 ? get_state_t<float>(h, s) : get_state_t<double>(h, s);
}

int pic_set_state(pic_handle* h, const pic_state* s) {
  if (!h || !s || (s->where != PIC_HOST && s->where != PIC_DEVICE)) return PIC_E_ARG;
  h->adj.ready = false;
  return h->es == 4 ? set_state_t<float>(h, s) : set_state_t<double>(h, s);
}

static int debug_copy(pic_handle* h, int where, void* const* out, void* const* src, int n) {
  if (!h || !out || (where != PIC_HOST && where != PIC_DEVICE)) return PIC_E_ARG;
  const cudaMemcpyKind k = where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int q = 0; q < n; ++q)
    if (out[q]) CK(cudaMemcpyAsync(out[q], src[q], (size_t)h->ncell * h->es, k, h->stream), "debug copy");
  CK(cudaStreamSynchronize(h->stream), "synchronize");
  return PIC_OK;
}

int pic_debug_gather_copies(pic_handle* h, int where, void* const* out6) {
  if (!h) return PIC_E_ARG;
  return debug_copy(h, where, out6, h->g, 6);
}

int pic_debug_current(pic_handle* h, int where, void* const* out3) {
  if (!h) return PIC_E_ARG;
  void* src[3] = {h->jf[0], h->jf[1], h->jf[2]};
  if (!(h->cfg.filter_targets & PIC_FILTER_J))
    for (int q = 0; q < 3; ++q) src[q] = h->f[6 + q];
  return debug_copy(h, where, out3, src, 3);
}

int pic_charge_residual(pic_handle* h, double out[3]) {
  if (!h || !out) return PIC_E_ARG;
  int rc = check_err(h);
  if (rc) return rc;
  return h->es == 4 ? charge_residual_t<float>(h, out) : charge_residual_t<double>(h, out);
}

int pic_fit_growth_rate(const double* t, const double* w, int n, double* gamma_out, int* i0, int* i1) {
  if (!t || !w || !gamma_out || n < 5) return PIC_E_ARG;
  return growth_fit(t, w, n, gamma_out, i0, i1);
}

int pic_energy_history(pic_handle* h, pic_energy_t* out, int max, int* count) {
  if (!h || (!out && max > 0) || max < 0) return PIC_E_ARG;
  int rc = check_err(h);
  if (rc) return rc;
  long long avail = h->nhist < h->hist_cap ? h->nhist : h->hist_cap;
  long long n = avail < max ? avail : max;
  std::vector<double> buf(8 * (size_t)(n > 0 ? n : 1));
  const long long first = (h->nhist - n) % h->hist_cap;  // ring slot of the oldest sample wanted
  const long long run1 = n < h->hist_cap - first ? n : h->hist_cap - first;
  if (n > 0) {
    CK(cudaMemcpy(buf.data(), h->d_hist + 8 * first, 8 * sizeof(double) * run1, cudaMemcpyDeviceToHost),
       "read history");
    if (n > run1)
      CK(cudaMemcpy(buf.data() + 8 * run1, h->d_hist, 8 * sizeof(double) * (n - run1), cudaMemcpyDeviceToHost),
         "read history");
  }
  const pic_config& c = h->cfg;
  const double dV = c.dx * c.dy * c.dz;
  for (long long q = 0; q < n; ++q) {
    const double* v = buf.data() + 8 * q;  // oldest first
    out[q].w_e = 0.5 * v[0] * dV;
    out[q].w_b = 0.5 * v[1] * dV;
    out[q].w_perp = 0.5 * v[2] * dV;
    out[q].k = v[3];
    out[q].total = out[q].w_e + out[q].w_b + out[q].k;
    out[q].np = (long long)v[4];
  }
  if (count) *count = (int)n;
  return PIC_OK;
}

int pic_enable_timing(pic_handle* h, int on) {
  if (!h) return PIC_E_ARG;
  CK(collect_times(h), "collect timings");
  h->timing = on != 0;
  if (on)
    for (int q = 0; q < PIC_NKERNEL; ++q) {
      h->tms[q] = 0.0;
      h->tcount[q] = 0;
    }
  return PIC_OK;
}

int pic_kernel_times(pic_handle* h, double ms[PIC_NKERNEL], long long launches[PIC_NKERNEL]) {
  if (!h) return PIC_E_ARG;
  CK(collect_times(h), "collect timings");
  for (int q = 0; q < PIC_NKERNEL; ++q) {
    if (ms) ms[q] = h->tms[q];
    if (launches) launches[q] = h->tcount[q];
  }
  return PIC_OK;
}

int pic_launch_count(pic_handle* h, long long* n) {
  if (!h || !n) return PIC_E_ARG;
  *n = h->launches;
  return PIC_OK;
}

void pic_destroy(pic_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  for (void* p : h->allocs)
    if (p) cudaFree(p);
  for (void* p : h->adj.mem)
    if (p) cudaFree(p);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_sp) cudaEventDestroy(h->ev_sp);
  if (h->h_sp_mirror) cudaFreeHost(h->h_sp_mirror);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

const char* pic_last_error(const pic_handle* h) {
  if (!h) return g_create_err.c_str();  // no handle: the reason the last create failed
  return h->err.c_str();
}

const char* pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_E_ARG: return "invalid argument";
    case PIC_E_CFL: return "time step violates the Courant limit";
    case PIC_E_SINGULAR: return "singular or ill-conditioned rational interpolation";
    case PIC_E_OOM: return "out of memory";
    case PIC_E_CUDA: return "CUDA error";
    case PIC_E_TIMEOUT: return "device wait timed out";
    case PIC_E_NONFINITE: return "non-finite state";
    case PIC_E_OVERFLOW: return "particle bin overflow";
    case PIC_E_STATE: return "invalid call for the handle's state";
    default: return "unknown error";
  }
}

}  // extern "C"

// ================================================================================================
// Batched runs: many independent simulations advanced by one set of multi-run launches per step
// (persistent push over a work list of (run, tile) items, one launch per lanes-per-cell group),
// replayed from a CUDA graph. Each run is a full pic_handle; the batch only adds the device tables
// of per-run kernel arguments and the launch sequence.
// ================================================================================================
struct pic_batch {
  std::vector<pic_handle*> runs;
  cudaStream_t own = nullptr, stream = nullptr;
  size_t es = 8;
  int ndim = 2, scheme = 0, hz = 0, hx = 0, hzj = 0, hxj = 0;
  bool filter_j = false;
  int diag_every = 0;
  std::vector<void*> allocs;
  void* d_run[2][2] = {};  // RunDev<T>[nruns] by [parity][recording]
  void* d_sep_copy[2] = {};  // by step parity: the E, B buffers each run reads and (Yee) writes alternate
  void* d_sep_j = nullptr;
  void* d_yee[2] = {};
  void* d_energy[2] = {};
  int* d_sep_base = nullptr;
  int sep_total = 0;
  int* d_yee_base = nullptr;
  int yee_total = 0;
  struct Group {
    int lpc = 8, blocks = 0;
    int2* d_items = nullptr;
    int nitems = 0;
    int* d_queue = nullptr;
    std::vector<int> members;
  };
  std::vector<Group> groups;
  bool tables_dirty = true;
  std::vector<int> gens;  // each run's bin growths when its tables were uploaded
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0, graph_parity = 0;
  cudaStream_t graph_stream = nullptr;
  long long nstep = 0;
  int parity = 0;
  std::string err;
};

namespace {

int bfail(pic_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#define BCK(call, what)                                                                        \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, e_ == cudaErrorMemoryAllocation ? PIC_E_OOM : PIC_E_CUDA, \
                                        std::string(what) + ": " + cudaGetErrorString(e_));    \
  } while (0)

void* balloc(pic_batch* b, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    (void)cudaGetLastError();  // reported by the null return; a later launch check must not see it
    return nullptr;
  }
  b->allocs.push_back(p);
  return p;
}

void batch_drop_graph(pic_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_len = 0;
}

// Upload the per-run argument tables (after creation, a correction change or a tuning change).
template <typename T>
int batch_tables(pic_batch* b) {
  const int n = (int)b->runs.size();
  std::vector<RunDev<T>> rd(n);
  for (int p = 0; p < 2; ++p)
    for (int rec = 0; rec < 2; ++rec) {
      for (int i = 0; i < n; ++i) {
        rd[i] = make_run<T>(b->runs[i], p);
        rd[i].kin = rec ? b->runs[i]->d_kin : nullptr;
        if (!tiles_fit<PTile>(rd[i])) BCK(cudaErrorInvalidValue, "run tiles");
      }
      BCK(cudaMemcpy(b->d_run[p][rec], rd.data(), sizeof(RunDev<T>) * n, cudaMemcpyHostToDevice), "run table");
    }
  // the E, B buffers current now (X) are read by steps of the batch's present parity and written by
  // the other parity's steps; the other buffers (Y) the reverse
  std::vector<SepArgs<T>> sc(n), sj(n);
  std::vector<YeeArgs<T>> ya(n);
  std::vector<EnergyArgs<T>> ea(n);
  for (int p = 0; p < 2; ++p) {
    for (int i = 0; i < n; ++i) {
      pic_handle* h = b->runs[i];
      const bool cur = p == b->parity;
      void* const* in = cur ? h->f : h->fb;
      void* const* out = cur ? h->fb : h->f;
      sc[i] = sep_args<T>(h, true);
      for (int q = 0; q < 6; ++q) sc[i].src[q] = (const T*)in[q];
      ya[i] = yee_args<T>(h, h->cfg.dt);
      ya[i].ex = (T*)in[0];
      ya[i].ey = (T*)in[1];
      ya[i].ez = (T*)in[2];
      ya[i].bx = (T*)in[3];
      ya[i].by = (T*)in[4];
      ya[i].bz = (T*)in[5];
      ya[i].oex = (T*)out[0];
      ya[i].oey = (T*)out[1];
      ya[i].oez = (T*)out[2];
      ya[i].obx = (T*)out[3];
      ya[i].oby = (T*)out[4];
      ya[i].obz = (T*)out[5];
      for (int q = 0; q < 6; ++q) ea[i].f[q] = (const T*)out[q];  // the energies of the new step
      ea[i].ncell = h->ncell;
      ea[i].scratch = h->d_red;
      ea[i].hc = HistCtl{h->d_hist, h->hist_cap, h->d_hist_count, h->d_kin};
    }
    BCK(cudaMemcpy(b->d_sep_copy[p], sc.data(), sizeof(SepArgs<T>) * n, cudaMemcpyHostToDevice), "copy table");
    BCK(cudaMemcpy(b->d_yee[p], ya.data(), sizeof(YeeArgs<T>) * n, cudaMemcpyHostToDevice), "yee table");
    BCK(cudaMemcpy(b->d_energy[p], ea.data(), sizeof(EnergyArgs<T>) * n, cudaMemcpyHostToDevice), "energy table");
  }
  for (int i = 0; i < n; ++i) sj[i] = sep_args<T>(b->runs[i], false);
  BCK(cudaMemcpy(b->d_sep_j, sj.data(), sizeof(SepArgs<T>) * n, cudaMemcpyHostToDevice), "filter table");
  b->gens.resize(n);
  for (int i = 0; i < n; ++i) b->gens[i] = b->runs[i]->grow_gen;
  b->tables_dirty = false;
  return PIC_OK;
}

template <typename T>
int batch_step_once(pic_batch* b) {
  cudaStream_t st = b->stream;
  const int n = (int)b->runs.size();
  pic_handle* h0 = b->runs[0];
  const bool rec = b->diag_every > 0 && (h0->nstep + 1) % b->diag_every == 0;
  const RunDev<T>* runs = (const RunDev<T>*)b->d_run[b->parity][rec ? 1 : 0];
  BCK(launch_sep_batch<T>((const SepArgs<T>*)b->d_sep_copy[b->parity], b->d_sep_base, n, b->sep_total, 6, b->ndim,
                          b->hz, b->hx,
                          st),
      "batched copy stencil");
  for (auto& g : b->groups)
    BCK(launch_push_batch<T>(runs, g.d_items, g.nitems, g.d_queue, b->ndim, b->scheme, g.lpc, g.blocks, st),
        "batched push");
  BCK(launch_push_spill_batch<T>(runs, n, b->ndim, b->scheme, st), "batched spill push");
  BCK(launch_migrate_batch<T>(runs, n, st), "batched migrate");
  if (b->filter_j)
    BCK(launch_sep_batch<T>((const SepArgs<T>*)b->d_sep_j, b->d_sep_base, n, b->sep_total, 3, b->ndim, b->hzj, b->hxj,
                            st),
        "batched current filter");
  BCK(launch_yee_batch<T>((const YeeArgs<T>*)b->d_yee[b->parity], b->d_yee_base, n, b->yee_total, b->ndim, st),
      "batched yee");
  if (rec) BCK(launch_field_energy_batch<T>((const EnergyArgs<T>*)b->d_energy[b->parity], n, st), "batched energy");
  for (pic_handle* h : b->runs) {
    swap_fields(h);
    h->parity ^= 1;
    h->nstep++;
    if (rec) h->nhist++;
  }
  b->parity ^= 1;
  b->nstep++;
  return PIC_OK;
}

int batch_run_steps(pic_batch* b, int k) {
  for (int s = 0; s < k; ++s) {
    int rc = b->es == 4 ? batch_step_once<float>(b) : batch_step_once<double>(b);
    if (rc) return rc;
  }
  return PIC_OK;
}

int batch_graph_len(const pic_batch* b) {
  const int de = b->diag_every > 0 ? b->diag_every : 1;
  int len = 2;
  while (len % de && len <= 64) len += 2;  // past 64 the caller falls back to single steps
  return len;
}

int batch_build_graph(pic_batch* b) {
  batch_drop_graph(b);
  const int len = batch_graph_len(b);
  const long long nstep0 = b->nstep;
  const int parity0 = b->parity;
  std::vector<long long> ns(b->runs.size()), nh(b->runs.size());
  std::vector<int> pa(b->runs.size());
  std::vector<std::vector<void*>> fs(b->runs.size());
  for (size_t i = 0; i < b->runs.size(); ++i) {
    ns[i] = b->runs[i]->nstep;
    nh[i] = b->runs[i]->nhist;
    pa[i] = b->runs[i]->parity;
    fs[i].assign(b->runs[i]->f, b->runs[i]->f + 6);
    fs[i].insert(fs[i].end(), b->runs[i]->fb, b->runs[i]->fb + 6);
  }
  BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  int rc = batch_run_steps(b, len);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->nstep = nstep0;
  b->parity = parity0;
  for (size_t i = 0; i < b->runs.size(); ++i) {
    b->runs[i]->nstep = ns[i];
    b->runs[i]->nhist = nh[i];
    b->runs[i]->parity = pa[i];
    for (int q = 0; q < 6; ++q) {  // an even number of steps: the captured swaps cancel
      b->runs[i]->f[q] = fs[i][q];
      b->runs[i]->fb[q] = fs[i][6 + q];
    }
  }
  if (rc != PIC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != PIC_OK ? rc : bfail(b, PIC_E_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, PIC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  b->graph_len = len;
  b->graph_parity = parity0;
  b->graph_stream = b->stream;
  return PIC_OK;
}

// Work items (run, tile) of every group, runs in creation order.
int batch_items(pic_batch* b) {
  for (auto& g : b->groups) {
    std::vector<int2> items;
    for (int i : g.members) {
      pic_handle* h = b->runs[i];
      const int nt = h->ntx * h->nty * h->ntz;
      for (int t = 0; t < nt; ++t) items.push_back(make_int2(i, t));
    }
    g.nitems = (int)items.size();
    if (!g.d_items) {
      g.d_items = (int2*)balloc(b, sizeof(int2) * items.size());
      g.d_queue = (int*)balloc(b, 16);
      if (!g.d_items || !g.d_queue) return bfail(b, PIC_E_OOM, "work list allocation");
    }
    BCK(cudaMemcpy(g.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice), "work list");
  }
  return PIC_OK;
}

int batch_max_blocks(pic_batch* b, int lpc) {
  return b->es == 4 ? push_max_blocks_per_sm<float>(b->ndim, b->scheme, lpc)
                    : push_max_blocks_per_sm<double>(b->ndim, b->scheme, lpc);
}

int batch_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  return n > 0 ? n : 152;
}

// Back to the seeded initial state (fields, bins, counters, history), same as after pic_create.
template <typename T>
int reseed(pic_handle* h) {
  cudaStream_t st = h->stream;
  const size_t fb = (size_t)h->ncell * h->es;
  for (int q = 0; q < 9; ++q) CK(cudaMemsetAsync(h->f[q], 0, fb, st), "reseed fields");
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(h->cnt[s][k], 0, sizeof(int) * h->ncell, st), "reseed counts");
  CK(cudaMemsetAsync(h->d_lv_count, 0, 2 * sizeof(int), st), "reseed leavers");
  CK(cudaMemsetAsync(h->d_sp_count, 0, 2 * sizeof(int), st), "reseed spill list");
  CK(cudaMemsetAsync(h->d_sp_total, 0, sizeof(unsigned long long), st), "reseed spill total");
  h->sp_pending = false;
  CK(cudaMemsetAsync(h->d_hist_count, 0, 16, st), "reseed history");
  CK(cudaMemsetAsync(h->d_kin, 0, 2 * sizeof(double), st), "reseed kinetic");
  h->parity = 0;
  h->nstep = 0;
  h->nhist = 0;
  drop_graph(h);
  if (h->cfg.init_beam && h->cfg.ppc_per_species > 0) return init_beam<T>(h);
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_create(const pic_config* cfgs, int nruns, pic_batch** out) {
  if (!cfgs || nruns < 1 || !out) return PIC_E_ARG;
  *out = nullptr;
  const pic_config& c0 = cfgs[0];
  for (int i = 1; i < nruns; ++i) {
    const pic_config& c = cfgs[i];
    if (c.ndim != c0.ndim || c.precision != c0.precision || c.scheme != c0.scheme || c.shape_order != c0.shape_order ||
        c.filter_nbin != c0.filter_nbin || c.filter_ncomp != c0.filter_ncomp ||
        c.filter_comp_alpha != c0.filter_comp_alpha || c.filter_targets != c0.filter_targets ||
        c.diag_every != c0.diag_every || (c.sigma_perp > 0) != (c0.sigma_perp > 0) ||
        (c.track_ids != 0) != (c0.track_ids != 0) || c.correction_mode != c0.correction_mode ||
        c.field_solver != c0.field_solver)
      return PIC_E_ARG;  // these must agree across the runs of one batch
  }
  if (c0.shape_order != 1 || c0.scheme == PIC_MOMENTUM || c0.correction_mode != PIC_CORR_SPLIT ||
      c0.field_solver != PIC_YEE)
    return PIC_E_ARG;  // batched: linear Galerkin / Uniform with the split correction, Yee solver
  pic_batch* b = new pic_batch();
  b->es = c0.precision == PIC_FP32 ? 4 : 8;
  b->ndim = c0.ndim;
  b->scheme = c0.scheme;
  b->diag_every = c0.diag_every;
  b->filter_j = (c0.filter_targets & PIC_FILTER_J) != 0;
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return PIC_E_CUDA;
  }
  b->stream = b->own;
  int rc = PIC_OK;
  for (int i = 0; i < nruns && rc == PIC_OK; ++i) {
    pic_handle* h = nullptr;
    rc = pic_create(&cfgs[i], &h);
    if (rc == PIC_OK) {
      b->runs.push_back(h);
      h->stream = b->stream;
      set_tiles(h, 0);  // the sweep fills the GPU with many runs: full tiles
    }
  }
  if (rc != PIC_OK) {
    pic_batch_destroy(b);
    return rc;
  }
  pic_handle* h0 = b->runs[0];
  b->hz = (int)(h0->zt_e.size() / 2);
  b->hx = (int)(h0->xt_g.size() / 2);
  b->hzj = (int)(h0->zt_j.size() / 2);
  b->hxj = (int)(h0->xt_j.size() / 2);
  std::vector<int> sep_base{0}, yee_base{0};
  for (pic_handle* h : b->runs) {
    const pic_config& c = h->cfg;
    if (!sep_fast_ok(c.ndim, c.nx, c.ny, c.nz, b->hz, b->hx) ||
        (b->filter_j && !sep_fast_ok(c.ndim, c.nx, c.ny, c.nz, b->hzj, b->hxj)) || c.nx < 3 || c.nz < 3 ||
        (c.ndim == 3 && c.ny < 3)) {
      pic_batch_destroy(b);
      return PIC_E_ARG;  // grids too small for the batched stencil kernels
    }
    sep_base.push_back(sep_base.back() + sep_tiles(c.ndim, c.nx, c.ny, c.nz));
    yee_base.push_back(yee_base.back() + yee_tiles(c.ndim, c.nx, c.ny, c.nz));
  }
  b->sep_total = sep_base.back();
  b->yee_total = yee_base.back();
  size_t rd = b->es == 4 ? sizeof(RunDev<float>) : sizeof(RunDev<double>);
  size_t sa = b->es == 4 ? sizeof(SepArgs<float>) : sizeof(SepArgs<double>);
  size_t ya = b->es == 4 ? sizeof(YeeArgs<float>) : sizeof(YeeArgs<double>);
  size_t ea = b->es == 4 ? sizeof(EnergyArgs<float>) : sizeof(EnergyArgs<double>);
  bool ok = true;
  for (int p = 0; p < 2 && ok; ++p)
    for (int r = 0; r < 2 && ok; ++r) ok = (b->d_run[p][r] = balloc(b, rd * nruns)) != nullptr;
  for (int p = 0; p < 2 && ok; ++p)
    ok = (b->d_sep_copy[p] = balloc(b, sa * nruns)) && (b->d_yee[p] = balloc(b, ya * nruns)) &&
         (b->d_energy[p] = balloc(b, ea * nruns));
  if (ok) ok = (b->d_sep_j = balloc(b, sa * nruns)) &&
               (b->d_sep_base = (int*)balloc(b, sizeof(int) * (nruns + 1))) &&
               (b->d_yee_base = (int*)balloc(b, sizeof(int) * (nruns + 1)));
  if (!ok) {
    pic_batch_destroy(b);
    return PIC_E_OOM;
  }
  cudaMemcpy(b->d_sep_base, sep_base.data(), sizeof(int) * (nruns + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_yee_base, yee_base.data(), sizeof(int) * (nruns + 1), cudaMemcpyHostToDevice);
  // push groups by the default lanes per cell; two resident blocks per SM where they fit
  const int sms = batch_sm_count();
  for (int i = 0; i < nruns; ++i) {
    const int lpc = push_lanes_per_cell(b->ndim, 2 * b->runs[i]->cfg.ppc_per_species);
    pic_batch::Group* g = nullptr;
    for (auto& gg : b->groups)
      if (gg.lpc == lpc) g = &gg;
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
      g->lpc = lpc;
      const int mb = batch_max_blocks(b, lpc);
      g->blocks = sms * (mb < 2 ? mb : 2);
    }
    g->members.push_back(i);
  }
  rc = batch_items(b);
  if (rc == PIC_OK) rc = b->es == 4 ? batch_tables<float>(b) : batch_tables<double>(b);
  if (rc == PIC_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PIC_E_CUDA;
  if (rc != PIC_OK) {
    pic_batch_destroy(b);
    return rc;
  }
  *out = b;
  return PIC_OK;
}

pic_handle* pic_batch_run(pic_batch* b, int run) {
  if (!b || run < 0 || run >= (int)b->runs.size()) return nullptr;
  return b->runs[run];
}

int pic_batch_size(const pic_batch* b) { return b ? (int)b->runs.size() : 0; }

int pic_batch_set_correction_stencil(pic_batch* b, int run, const double psi_e[5], const double psi_b[5]) {
  if (!b || run < 0 || run >= (int)b->runs.size()) return PIC_E_ARG;
  int rc = pic_set_correction_stencil(b->runs[run], psi_e, psi_b);
  if (rc) return bfail(b, rc, pic_last_error(b->runs[run]));
  if ((int)(b->runs[run]->zt_e.size() / 2) != b->hz) return bfail(b, PIC_E_STATE, "stencil length changed");
  b->tables_dirty = true;
  batch_drop_graph(b);
  return PIC_OK;
}

int pic_batch_set_stream(pic_batch* b, void* stream) {
  if (!b) return PIC_E_ARG;
  b->stream = stream ? (cudaStream_t)stream : b->own;
  for (pic_handle* h : b->runs) h->stream = b->stream;
  batch_drop_graph(b);
  return PIC_OK;
}

}  // extern "C"

static int batch_steps(pic_batch* b, int nsteps);

extern "C" {

int pic_batch_step(pic_batch* b, int nsteps) {
  if (!b || nsteps < 0) return PIC_E_ARG;
  NvtxRange range("pic_batch_step");
  for (pic_handle* h : b->runs)
    if (h->parity != b->parity) return bfail(b, PIC_E_STATE, "a run was stepped or reset on its own");
  // runs with particles waiting in their spill list grow their bins first (see pic_step)
  for (pic_handle* h : b->runs) {
    const int rc = spill_check(h);
    if (rc) return bfail(b, rc, pic_last_error(h));
  }
  for (size_t i = 0; i < b->runs.size(); ++i)
    if (i >= b->gens.size() || b->gens[i] != b->runs[i]->grow_gen) {
      b->tables_dirty = true;
      batch_drop_graph(b);
    }
  if (b->tables_dirty) {
    int rc = b->es == 4 ? batch_tables<float>(b) : batch_tables<double>(b);
    if (rc) return rc;
  }
  const int rc = batch_steps(b, nsteps);
  if (rc == PIC_OK && nsteps > 0)
    for (pic_handle* h : b->runs) note_spill(h);
  return rc;
}

}  // extern "C"

static int batch_steps(pic_batch* b, int nsteps) {
  const int len = batch_graph_len(b);
  if (len > 64 || nsteps < 2 * len) return batch_run_steps(b, nsteps);
  int lead = (int)((len - b->nstep % len) % len);
  int rc = batch_run_steps(b, lead);
  if (rc) return rc;
  nsteps -= lead;
  if (!b->graph || b->graph_len != len || b->graph_stream != b->stream || b->graph_parity != b->parity) {
    rc = batch_run_steps(b, len);  // warm the kernel attributes before capturing
    if (rc) return rc;
    nsteps -= len;
    rc = batch_build_graph(b);
    if (rc) return rc;
  }
  while (nsteps >= len) {
    BCK(cudaGraphLaunch(b->graph, b->stream), "graph launch");
    for (pic_handle* h : b->runs) {
      h->nstep += len;
      if (b->diag_every > 0) h->nhist += len / b->diag_every;
    }
    b->nstep += len;
    nsteps -= len;
  }
  return batch_run_steps(b, nsteps);
}

extern "C" {

int pic_batch_sync(pic_batch* b) {
  if (!b) return PIC_E_ARG;
  BCK(cudaStreamSynchronize(b->stream), "synchronize");
  for (pic_handle* h : b->runs) {
    int rc = check_err(h);
    if (rc) return bfail(b, rc, pic_last_error(h));
  }
  return PIC_OK;
}

int pic_batch_energy_history(pic_batch* b, int run, pic_energy_t* out, int max, int* count) {
  if (!b || run < 0 || run >= (int)b->runs.size()) return PIC_E_ARG;
  return pic_energy_history(b->runs[run], out, max, count);
}

int pic_batch_autotune(pic_batch* b, int trial_steps, int* lpc_out) {
  if (!b || trial_steps < 1) return PIC_E_ARG;
  if (b->tables_dirty) {
    int rc = b->es == 4 ? batch_tables<float>(b) : batch_tables<double>(b);
    if (rc) return rc;
  }
  const int sms = batch_sm_count();
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "event");
  BCK(cudaEventCreate(&e1), "event");
  int rc = PIC_OK;
  for (size_t gi = 0; gi < b->groups.size() && rc == PIC_OK; ++gi) {
    auto& g = b->groups[gi];
    float best = 1e30f;
    int best_lpc = g.lpc, best_blocks = g.blocks;
    for (int lpc : {4, 8, 16}) {
      const int mb = batch_max_blocks(b, lpc);
      for (int bps = 1; bps <= mb && bps <= 2 && rc == PIC_OK; ++bps) {
        g.lpc = lpc;
        g.blocks = sms * bps;
        rc = batch_run_steps(b, 2);  // warm-up of this variant
        if (rc) break;
        cudaEventRecord(e0, b->stream);
        rc = batch_run_steps(b, 2 * trial_steps);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = PIC_E_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc == PIC_OK && ms < best) {
          best = ms;
          best_lpc = lpc;
          best_blocks = g.blocks;
        }
      }
    }
    g.lpc = best_lpc;
    g.blocks = best_blocks;
    if (lpc_out) lpc_out[gi] = best_lpc;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  // the trials advanced the runs: back to the seeded initial state
  for (pic_handle* h : b->runs) {
    rc = b->es == 4 ? reseed<float>(h) : reseed<double>(h);
    if (rc) return bfail(b, rc, pic_last_error(h));
  }
  b->parity = 0;
  b->nstep = 0;
  b->tables_dirty = true;  // the field buffers current at parity 0 may have changed roles
  batch_drop_graph(b);
  return pic_batch_sync(b);
}

void pic_batch_destroy(pic_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  for (pic_handle* h : b->runs) {
    h->stream = h->own;
    pic_destroy(h);
  }
  for (void* p : b->allocs)
    if (p) cudaFree(p);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

const char* pic_batch_last_error(const pic_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"

// ================================================================================================
// Adjoint of the 2D step with checkpoint and recompute. The forward run stores the full state
// (fields, particles in id order) every `every` steps. The backward pass walks the segments from
// the last: it restores the segment's checkpoint, recomputes the segment with the ordinary step
// while taping the state at the start of each step, then applies the transposed passes of each
// step in reverse (k_adjoint.cu), carrying the adjoints of E, B and of every particle's position
// and momentum from step to step.
// ================================================================================================
namespace {

void* adj_malloc(pic_handle* h, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    (void)cudaGetLastError();  // reported by the null return; a later launch check must not see it
    return nullptr;
  }
  h->adj.mem.push_back(p);
  return p;
}

void adj_release(pic_handle* h) {
  auto& A = h->adj;
  cudaStreamSynchronize(h->stream);
  for (void* p : A.mem)
    if (p) cudaFree(p);
  A = pic_handle::Adj();
}

int adj_flat(pic_handle* h, pic_handle::Flat& f, long long np) {
  const size_t n = (size_t)np;
  const size_t sz[9] = {4, 4, h->es, 0, h->es, h->es, h->es, h->es, h->has_w ? h->es : 0};
  for (int q = 0; q < 9; ++q) {
    if (!sz[q]) continue;
    f.a[q] = adj_malloc(h, sz[q] * n);
    if (!f.a[q]) return PIC_E_OOM;
    if (cudaMemset(f.a[q], 0, sz[q] * n) != cudaSuccess) return PIC_E_CUDA;  // valid cells until written
  }
  return PIC_OK;
}

// Storage for nck checkpoints, ntape taped steps and np particles (kept when large enough).
int adj_reserve(pic_handle* h, int nck, int ntape, long long np) {
  auto& A = h->adj;
  if (A.cap_ck >= nck && A.cap_tape >= ntape && A.cap_np >= np && A.dots) return PIC_OK;
  adj_release(h);
  const size_t fb = (size_t)h->ncell * h->es;
  A.ck_f.assign((size_t)nck * 6, nullptr);
  A.ck_p.assign(nck, pic_handle::Flat());
  A.tape_f.assign((size_t)ntape * 6, nullptr);
  A.tape_p.assign(ntape, pic_handle::Flat());
  bool ok = true;
  for (auto& p : A.ck_f) ok = ok && (p = adj_malloc(h, fb)) != nullptr;
  for (auto& p : A.tape_f) ok = ok && (p = adj_malloc(h, fb)) != nullptr;
  for (auto& f : A.ck_p) ok = ok && adj_flat(h, f, np) == PIC_OK;
  for (auto& f : A.tape_p) ok = ok && adj_flat(h, f, np) == PIC_OK;
  for (int q = 0; q < 6; ++q) ok = ok && (A.lam[q] = adj_malloc(h, fb)) && (A.lg[q] = adj_malloc(h, fb)) &&
                                   (A.y[q] = adj_malloc(h, fb));
  for (int q = 0; q < 3; ++q) ok = ok && (A.lj[q] = adj_malloc(h, fb));
  for (int q = 0; q < 5; ++q) ok = ok && (A.lp[q] = adj_malloc(h, h->es * (size_t)np));
  ok = ok && (A.dots = (double*)adj_malloc(h, 16 * sizeof(double)));
  ok = ok && (A.partial = (double*)adj_malloc(h, adj_psi_partial_doubles() * sizeof(double)));
  ok = ok && (A.seen = (unsigned long long*)adj_malloc(h, 8 * (size_t)(np / 64 + 1)));
  if (!ok) {
    adj_release(h);
    return fail(h, PIC_E_OOM, "adjoint storage allocation failed");
  }
  A.cap_ck = nck;
  A.cap_tape = ntape;
  A.cap_np = np;
  return PIC_OK;
}

template <typename T>
FlatDev<T> flat_view(const pic_handle::Flat& f, long long np) {
  FlatDev<T> v;
  v.np = np;
  v.cell = (int*)f.a[0];
  v.species = (int*)f.a[1];
  v.ox = (T*)f.a[2];
  v.oy = nullptr;
  v.oz = (T*)f.a[4];
  v.dux = (T*)f.a[5];
  v.duy = (T*)f.a[6];
  v.duz = (T*)f.a[7];
  v.w = (T*)f.a[8];
  v.id = nullptr;  // the flat index is the id
  return v;
}

// Fields and particles of the current state into (fields[6], flat) in id order.
template <typename T>
int adj_save(pic_handle* h, void* const* fields, const pic_handle::Flat& flat, bool check_ids) {
  int rc0 = settle<T>(h);  // the tape reads the bins: no particle may wait in the spill list
  if (rc0) return rc0;
  cudaStream_t st = h->stream;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  for (int q = 0; q < 6; ++q)
    if (fields) CK(cudaMemcpyAsync(fields[q], h->f[q], fb, cudaMemcpyDeviceToDevice, st), "save fields");
  unsigned long long* seen = nullptr;
  if (check_ids) {
    seen = h->adj.seen;
    CK(cudaMemsetAsync(seen, 0, 8 * (size_t)(h->adj.np / 64 + 1), st), "clear id bitmap");
  }
  RunDev<T> r = make_run<T>(h, h->parity);
  FlatDev<T> f = flat_view<T>(flat, h->adj.np);
  CK(launch(h, PIC_K_OTHER, [&] { return launch_tape<T>(r, f, seen, st); }), "tape");
  return PIC_OK;
}

// Back to checkpoint j: fields copied in, particles re-binned from the id-ordered arrays.
template <typename T>
int adj_restore(pic_handle* h, int j) {
  auto& A = h->adj;
  cudaStream_t st = h->stream;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  drop_graph(h);
  for (int q = 0; q < 6; ++q)
    CK(cudaMemcpyAsync(h->f[q], A.ck_f[(size_t)j * 6 + q], fb, cudaMemcpyDeviceToDevice, st), "restore fields");
  for (int sp = 0; sp < 2; ++sp)
    for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(h->cnt[sp][b], 0, sizeof(int) * h->ncell, st), "clear counts");
  CK(cudaMemsetAsync(h->d_lv_count, 0, 2 * sizeof(int), st), "clear leaver counters");
  CK(cudaMemsetAsync(h->d_sp_count, 0, 2 * sizeof(int), st), "clear spill counters");
  h->parity = 0;
  h->sp_pending = false;
  RunDev<T> r = make_run<T>(h, 0);
  FlatDev<T> f = flat_view<T>(A.ck_p[j], A.np);
  CK(launch(h, PIC_K_OTHER, [&] { return launch_import<T>(r, f, st); }), "restore particles");
  return PIC_OK;
}

template <typename T>
void put_taps(T* dst, const double* src, int n, double scale = 1.0) {
  for (int i = 0; i < n; ++i) dst[i] = (T)(src[i] * scale);
}

// Transposed passes of one step, in reverse order, for taped step s of the current segment.
template <typename T>
int adj_step(pic_handle* h, int s) {
  auto& A = h->adj;
  const pic_config& c = h->cfg;
  cudaStream_t st = h->stream;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  T* lam[6];
  T* lj[3];
  for (int q = 0; q < 6; ++q) lam[q] = (T*)A.lam[q];
  for (int q = 0; q < 3; ++q) lj[q] = (T*)A.lj[q];
  // Yee^T. Forward: B' = B - dt/2 C_E E; E' = E + dt C_B B' - dt J~; B'' = B' - dt/2 C_E E', and
  // C_E^T = C_B on the periodic Yee mesh. Reverse: lE -= dt/2 C_B lB; lJ~ = -dt lE;
  // lB += dt C_E lE; lE -= dt/2 C_B lB.
  YeeArgs<T> ya;
  ya.ex = lam[0];
  ya.ey = lam[1];
  ya.ez = lam[2];
  ya.bx = lam[3];
  ya.by = lam[4];
  ya.bz = lam[5];
  ya.jx = lj[0];
  ya.jy = lj[1];
  ya.jz = lj[2];
  ya.nx = c.nx;
  ya.ny = c.ny;
  ya.nz = c.nz;
  ya.h = T(0);
  auto coef = [&](double hs) {
    ya.cx = (T)(hs / c.dx);
    ya.cy = (T)(hs / c.dy);
    ya.cz = (T)(hs / c.dz);
  };
  coef(-0.5 * c.dt);
  CK(launch(h, PIC_K_YEE, [&] { return launch_yee_e<T>(ya, st); }), "adjoint yee (e half)");
  // lJ = F_J^T lJ~ = -dt F_J lE (symmetric filter taps, scaled by -dt)
  SepArgs<T> ja = sep_args<T>(h, false);
  for (int q = 0; q < 3; ++q) {
    ja.src[q] = lam[q];
    ja.dst[q] = lj[q];
  }
  put_taps(ja.zt[0], h->zt_j.data(), (int)h->zt_j.size(), -c.dt);
  put_taps(ja.zt[1], h->zt_j.data(), (int)h->zt_j.size(), -c.dt);
  CK(launch(h, PIC_K_FILTER, [&] { return launch_sep<T>(ja, st); }), "adjoint current filter");
  coef(-c.dt);
  CK(launch(h, PIC_K_YEE, [&] { return launch_yee_b<T>(ya, st); }), "adjoint yee (b)");
  coef(-0.5 * c.dt);
  CK(launch(h, PIC_K_YEE, [&] { return launch_yee_e<T>(ya, st); }), "adjoint yee (e half)");
  // gather copies of the taped fields (the forward's own copies, recomputed)
  SepArgs<T> ca = sep_args<T>(h, true);
  for (int q = 0; q < 6; ++q) ca.src[q] = (const T*)A.tape_f[(size_t)s * 6 + q];
  for (int q = 0; q < 3; ++q) ca.zero[q] = nullptr;
  CK(launch(h, PIC_K_COPIES, [&] { return launch_sep<T>(ca, st); }), "adjoint: copies");
  // particles
  for (int q = 0; q < 6; ++q) CK(cudaMemsetAsync(A.lg[q], 0, fb, st), "zero copy adjoint");
  const pic_handle::Flat& tp = A.tape_p[s];
  AdjPartArgs<T> pa;
  pa.n = A.np;
  pa.nx = c.nx;
  pa.nz = c.nz;
  pa.cell = (const int*)tp.a[0];
  pa.species = (const int*)tp.a[1];
  pa.ox = (const T*)tp.a[2];
  pa.oz = (const T*)tp.a[4];
  pa.dux = (const T*)tp.a[5];
  pa.duy = (const T*)tp.a[6];
  pa.duz = (const T*)tp.a[7];
  pa.w = h->has_w ? (const T*)tp.a[8] : nullptr;
  for (int q = 0; q < 6; ++q) pa.g[q] = (const T*)h->g[q];
  for (int q = 0; q < 3; ++q) pa.lj[q] = lj[q];
  for (int q = 0; q < 6; ++q) pa.lg[q] = (T*)A.lg[q];
  pa.lox = (T*)A.lp[0];
  pa.loz = (T*)A.lp[1];
  pa.lux = (T*)A.lp[2];
  pa.luy = (T*)A.lp[3];
  pa.luz = (T*)A.lp[4];
  const double dV = c.dx * c.dy * c.dz;
  pa.dtdx = (T)(c.dt / c.dx);
  pa.dtdz = (T)(c.dt / c.dz);
  pa.u0 = (T)h->u0;
  pa.hq = (T)(0.5 * c.dt);
  pa.wconst = (T)h->w0;
  pa.jfx = (T)(-c.dx / (dV * c.dt));
  pa.jfz = (T)(-c.dz / (dV * c.dt));
  pa.jfy2d = (T)(1.0 / dV);
  pa.err = h->d_err;
  CK(launch(h, PIC_K_PUSH, [&] { return launch_adj_particles<T>(pa, c.scheme, st); }), "adjoint: particles");
  // copies^T = Psi(D_z) F_gather: the filter here, Psi fused with the coefficient gradient
  const bool fg = (c.filter_targets & PIC_FILTER_GATHER) != 0;
  if (fg) {
    SepArgs<T> fa = sep_args<T>(h, true);
    for (int q = 0; q < 6; ++q) {
      fa.src[q] = (const T*)A.lg[q];
      fa.dst[q] = (T*)A.y[q];
    }
    for (int q = 0; q < 3; ++q) fa.zero[q] = nullptr;
    fa.hz[0] = fa.hz[1] = (int)(h->xt_g.size() / 2);
    put_taps(fa.zt[0], h->xt_g.data(), (int)h->xt_g.size());
    put_taps(fa.zt[1], h->xt_g.data(), (int)h->xt_g.size());
    CK(launch(h, PIC_K_COPIES, [&] { return launch_sep<T>(fa, st); }), "adjoint: copy filter");
  }
  AdjPsiArgs<T> ps;
  for (int q = 0; q < 6; ++q) {
    ps.y[q] = (const T*)(fg ? A.y[q] : A.lg[q]);
    ps.f[q] = (const T*)A.tape_f[(size_t)s * 6 + q];
    ps.lf[q] = lam[q];
  }
  ps.ncell = h->ncell;
  ps.nxy = (long long)c.nx * c.ny;
  ps.nz = c.nz;
  double te[9], tb[9];
  psi_stencil(h->pe, te);
  psi_stencil(h->pb, tb);
  put_taps(ps.taps[0], te, 9);
  put_taps(ps.taps[1], tb, 9);
  for (int n = 0; n < 5; ++n) {
    double e[5] = {0, 0, 0, 0, 0}, t[9];
    e[n] = 1.0;
    psi_stencil(e, t);
    put_taps(ps.dpow[n], t, 9);
  }
  ps.dots = A.dots;
  ps.partial = A.partial;
  CK(launch(h, PIC_K_DIAG, [&] { return launch_adj_psi<T>(ps, st); }), "adjoint: psi");
  return PIC_OK;
}

template <typename T>
int adjoint_forward_t(pic_handle* h, int nsteps, int every, double* w_perp) {
  auto& A = h->adj;
  A.ready = false;
  long long cnt[2];
  int rc = count_particles<T>(h, cnt);
  if (rc) return rc;
  rc = check_err(h);
  if (rc) return rc;
  const long long np = cnt[0] + cnt[1];
  const int nseg = nsteps > 0 ? (nsteps + every - 1) / every : 0;
  rc = adj_reserve(h, nseg + 1, nsteps < every ? (nsteps > 0 ? nsteps : 1) : every, np);
  if (rc) return rc;
  A.nsteps = nsteps;
  A.every = every;
  A.nseg = nseg;
  A.np = np;
  for (int j = 0; j < nseg; ++j) {
    rc = adj_save<T>(h, &A.ck_f[(size_t)j * 6], A.ck_p[j], j == 0);
    if (rc) return rc;
    const int len = nsteps - j * every < every ? nsteps - j * every : every;
    rc = pic_step(h, len);
    if (rc) return rc;
  }
  rc = adj_save<T>(h, &A.ck_f[(size_t)nseg * 6], A.ck_p[nseg], nseg == 0);
  if (rc) return rc;
  pic_energy_t e;
  rc = energy_t<T>(h, &e);  // synchronises and reads the device error flag (ids, overflow)
  if (rc) return rc;
  if (e.np != np) return fail(h, PIC_E_STATE, "particles were lost during the recorded run");
  *w_perp = e.w_perp;
  A.final_step = h->nstep;
  A.final_hist = h->nhist;
  A.ready = true;
  return PIC_OK;
}

template <typename T>
int adjoint_backward_t(pic_handle* h, double dw, double grad_psi_e[5], double grad_psi_b[5],
                       void* const grad_fields[6]) {
  auto& A = h->adj;
  if (!A.ready || h->nstep != A.final_step)
    return fail(h, PIC_E_STATE, "no recorded forward run for the current state (pic_adjoint_forward)");
  const pic_config& c = h->cfg;
  cudaStream_t st = h->stream;
  const size_t fb = (size_t)h->ncell * sizeof(T);
  const double dV = c.dx * c.dy * c.dz;
  // seed: adjoint of the final fields for dw * W_perp
  AdjSeedArgs<T> sa;
  for (int q = 0; q < 6; ++q) {
    sa.f[q] = (const T*)A.ck_f[(size_t)A.nseg * 6 + q];
    sa.lam[q] = (T*)A.lam[q];
  }
  sa.ncell = h->ncell;
  sa.scale = (T)(dw * dV);
  CK(launch(h, PIC_K_OTHER, [&] { return launch_adj_seed<T>(sa, st); }), "adjoint seed");
  for (int q = 0; q < 5; ++q) CK(cudaMemsetAsync(A.lp[q], 0, h->es * (size_t)A.np, st), "zero particle adjoint");
  for (int q = 0; q < 3; ++q) CK(cudaMemsetAsync(A.lj[q], 0, fb, st), "zero current adjoint");
  CK(cudaMemsetAsync(A.dots, 0, 16 * sizeof(double), st), "zero coefficient gradient");
  h->no_diag = true;
  int rc = PIC_OK;
  for (int j = A.nseg - 1; j >= 0 && rc == PIC_OK; --j) {
    const int len = A.nsteps - j * A.every < A.every ? A.nsteps - j * A.every : A.every;
    rc = adj_restore<T>(h, j);
    for (int s = 0; s < len && rc == PIC_OK; ++s) {
      rc = adj_save<T>(h, &A.tape_f[(size_t)s * 6], A.tape_p[s], false);
      if (rc == PIC_OK && s + 1 < len) rc = step_once<T>(h);
    }
    for (int s = len - 1; s >= 0 && rc == PIC_OK; --s) rc = adj_step<T>(h, s);
  }
  h->no_diag = false;
  if (rc) return rc;
  // back to the final state of the recorded run
  rc = adj_restore<T>(h, A.nseg);
  if (rc) return rc;
  h->nstep = A.final_step;
  h->nhist = A.final_hist;
  double dots[16];
  CK(cudaMemcpyAsync(dots, A.dots, sizeof dots, cudaMemcpyDeviceToHost, st), "read coefficient gradient");
  if (grad_fields)
    for (int q = 0; q < 6; ++q)
      if (grad_fields[q])
        CK(cudaMemcpyAsync(grad_fields[q], A.lam[q], fb, cudaMemcpyDeviceToDevice, st), "copy field gradient");
  rc = check_err(h);  // synchronises
  if (rc) return rc;
  for (int n = 0; n < 5; ++n) {
    if (grad_psi_e) grad_psi_e[n] = dots[n];
    if (grad_psi_b) grad_psi_b[n] = dots[5 + n];
  }
  A.ready = true;  // the state is the recorded run's final state again
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_adjoint_forward(pic_handle* h, int nsteps, int checkpoint_every, double* w_perp) {
  if (!h || nsteps < 0 || checkpoint_every < 1 || !w_perp) return PIC_E_ARG;
  if (h->cfg.ndim != 2) return fail(h, PIC_E_ARG, "the adjoint covers 2D runs");
  if (h->cfg.shape_order != 1 || h->cfg.scheme == PIC_MOMENTUM || h->cfg.correction_mode != PIC_CORR_SPLIT ||
      h->cfg.field_solver != PIC_YEE)
    return fail(h, PIC_E_ARG,
                "the adjoint covers linear shapes, the Galerkin or Uniform gather, the split correction, the Yee "
                "solver");
  if (!h->has_id) return fail(h, PIC_E_STATE, "the adjoint needs particle ids (cfg.track_ids = 1)");
  if (h->ncell >= (1LL << 31)) return fail(h, PIC_E_ARG, "the adjoint covers grids below 2^31 cells");
  return h->es == 4 ? adjoint_forward_t<float>(h, nsteps, checkpoint_every, w_perp)
                    : adjoint_forward_t<double>(h, nsteps, checkpoint_every, w_perp);
}

int pic_adjoint_backward(pic_handle* h, double dw, double grad_psi_e[5], double grad_psi_b[5],
                         void* const grad_fields[6]) {
  if (!h || !isfinite(dw)) return PIC_E_ARG;
  return h->es == 4 ? adjoint_backward_t<float>(h, dw, grad_psi_e, grad_psi_b, grad_fields)
                    : adjoint_backward_t<double>(h, dw, grad_psi_e, grad_psi_b, grad_fields);
}

void pic_adjoint_release(pic_handle* h) {
  if (h) adj_release(h);
}

}  // extern "C"
