// C ABI of the DD-4DVar GB300 library (include/dd4dvar.h): context, argument
// checks, decomposition tables, observation preprocessing and the host-side
// orchestration of the device kernels (sweep.cu, aux.cu).  Every numerical
// step runs in this library's CUDA kernels; the host only validates inputs,
// builds index tables and enqueues work.
#include "dd4dvar.h"
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

using namespace dd4dv;

namespace {

thread_local std::string g_create_error;

struct Fail {
  dd4dv_status st;
};

}  // namespace

namespace dd4dv {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace dd4dv

struct dd4dv_ctx {
  dd4dv_model m{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  long long launches = 0;

  // grid
  std::vector<RowConst> rows_h;
  RowConst* rows_d = nullptr;
  double Bth = 0, gBth = 0;
  size_t gstate = 0;          // 3*nlat*nlon
  size_t gtraj = 0;           // (nsteps+1)*gstate

  bool has_bg = false, has_berr = false, has_obs = false, has_dec = false;
  double* xb0 = nullptr;      // background initial state (FP64, one global state)
  double* gscratch = nullptr; // 3 global states: 2 RK3 stages + input/output staging
  double* gchunk = nullptr;   // gchunk_lv consecutive global levels (FP64): chunked global
  int gchunk_lv = 2;          // runs and host transfers of global trajectories

  double sigma_b[3] = {1, 1, 1};
  double corr_len = 0;
  int rf_passes = 4;
  double rf_alpha = 0, rf_c = 1;
  double* sigma_d = nullptr;

  std::vector<int> ob_level, ob_var;
  std::vector<double> ob_fi, ob_fj, ob_val, ob_so;

  // decomposition
  dd4dv_decomp dec{};
  std::vector<int> lon_cuts, lat_cuts, t_cuts;
  int n_sub = 0;
  std::vector<SubDesc> subs_h;
  SubDesc* subs_d = nullptr;
  int* order_d = nullptr;
  long long ctrl_total = 0, traj_elems = 0, ptraj_total = 0, pt_steps = 0;
  int max_nx = 0, max_ny = 0, min_ny = 0, max_levels = 0, max_pts = 0;
  int cl = 1, R = 1, W = 3, nthreads = 256;        // adjoint (and TLM base) sweep shape
  int cl_f = 1, R_f = 1, nt_f = 256;               // forward sweep shape
  double tune_ms = 0.0;
  double ckpt_ms = 0.0;       // ckpt_k = -2: measured evaluation time of the chosen storage
  int variant_f = 0;          // forward sweep: 0 = deep-halo FP32 sweep where it applies,
  int variant_a = 0;          // 1 = stripe sweep only; variant_a: the same for the adjoint
  size_t tsize = 8;

  void* traj = nullptr;
  void* seg = nullptr;        // checkpoint-segment buffers (ckpt_k > 0)
  int ckpt = 0;
  void* stg = nullptr;        // RK3 stage states (nullptr: the adjoint recomputes them)
  long long stg_elems = 0;
  void* stg1 = nullptr;       // x1 alone for some subdomains (see stg1_off), when stg is absent
  int stg1_subs = 0;          // subdomains with x1 stored
  double stg1_frac = 0.0;     // their share of the pt-steps
  bool use_stg = false;
  void* tgt = nullptr;
  void* bnd = nullptr;
  void* tgt0 = nullptr;       // copies of tgt and bnd at l = 0 (when they fit), so that
  void* bnd0 = nullptr;       // dd4dv_reset_exchange is two device copies
  double *xb_a = nullptr, *w = nullptr, *w_prev = nullptr, *g = nullptr, *wt = nullptr,
         *gt = nullptr, *p = nullptr, *S = nullptr, *Y = nullptr, *rho = nullptr;
  double *vw = nullptr, *vw2 = nullptr, *lam_a = nullptr, *J = nullptr, *Jt = nullptr,
         *parts = nullptr, *part = nullptr, *vconst = nullptr, *vpart = nullptr;
  double *io_a = nullptr, *io_b = nullptr, *io_c = nullptr, *io_p = nullptr;
  double* ptraj_io = nullptr;
  ObsRec* obs_d = nullptr;
  int* lvl_obs_d = nullptr;
  double* obs_force_d = nullptr;
  int *sc_tgt_d = nullptr, *sc_off_d = nullptr, *sc_obs_d = nullptr, *lvl_sc_d = nullptr;
  double* sc_w_d = nullptr;
  int *lon_cov_d = nullptr, *lat_cov_d = nullptr, *t_cov_d = nullptr;
  LbState* lbst = nullptr;
  // Gauss-Newton local solver (allocated on first use)
  double *cg_r = nullptr, *cg_p = nullptr, *cg_Ap = nullptr, *cg_dw = nullptr;
  CgState* cgst = nullptr;
  void* gn_dx = nullptr;
  int* phase_d = nullptr;
  int* owned_d = nullptr;     // [n_sub] 1 = this context evaluates and solves the subdomain
  std::vector<int> owned_h;
  bool owned_all = true;      // every subdomain owned (the default)
  int* counter_d = nullptr;
  int* counter_h = nullptr;   // pinned
  int* phase_h = nullptr;     // pinned
  double* scal_d = nullptr;
  double* scal_h = nullptr;   // pinned
  int* err_d = nullptr;
  int vblocks = 8;
  bool fwd_pending = false;
  LbState* lbst_h = nullptr;  // pinned
  // captured CUDA graphs of the outer iteration (start evaluation, L-BFGS
  // direction, one line-search trial, exchange), valid for one solver setting
  struct Graphs {
    cudaGraphExec_t start = nullptr, dir = nullptr, trial = nullptr, exch = nullptr, fin = nullptr;
    long long k_start = 0, k_dir = 0, k_trial = 0, k_exch = 0, k_fin = 0;
    dd4dv_solver key{};
    bool valid = false;
  } og;
  void drop_graphs();
  std::vector<void*> dec_allocs;

  ~dd4dv_ctx();
  void free_dec();
};

namespace {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) fail(ctx, DD4DV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define KL(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    ++ctx->launches;                                                                  \
    if (e_ != cudaSuccess) fail(ctx, DD4DV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

[[noreturn]] void fail(dd4dv_ctx* ctx, dd4dv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_error = buf;
  throw Fail{st};
}

template <typename F>
dd4dv_status guard(dd4dv_ctx* ctx, F&& f) {
  if (!ctx) return DD4DV_EINVAL;
  ctx->err.clear();
  try {
    return f();
  } catch (const Fail& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return DD4DV_ENOMEM;
  } catch (...) {
    ctx->err = "internal error";
    return DD4DV_EINVAL;
  }
}

template <typename T>
T* dalloc(dd4dv_ctx* ctx, size_t n, std::vector<void*>* list = nullptr) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, DD4DV_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
  }
  if (list) list->push_back(p);
  return static_cast<T*>(p);
}

void sync(dd4dv_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->st));
  int h = 0;
  CK(cudaMemcpy(&h, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    CK(cudaMemset(ctx->err_d, 0, sizeof(int)));
    fail(ctx, DD4DV_EINVAL, "device kernel rejected its launch configuration (code %d)", h);
  }
}

void h2d(dd4dv_ctx* ctx, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->st));
}
void d2h(dd4dv_ctx* ctx, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->st));
}

bool all_finite(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

// Recursive-filter coefficient and amplitude (see dd4dv_set_background_error):
// alpha from matching the variance 4 N alpha/(1-alpha)^2 of L L^T to ell^2;
// c^-2 = centre value of (F^T F)^(2N) applied to a unit impulse on a line long
// enough for the kernel to have decayed to below double precision.
void rf_coeffs(double ell, int npass, double* alpha, double* c) {
  const double E = 2.0 * npass / (ell * ell);
  const double a = 1.0 + E - std::sqrt(E * (E + 2.0));
  const int half = (int)(40 * ell) + 60;
  const int n = 2 * half + 1;
  std::vector<double> x(n, 0.0);
  x[half] = 1.0;
  for (int p = 0; p < 2 * npass; ++p) {
    double q = 0.0;
    for (int i = 0; i < n; ++i) { q = a * q + (1.0 - a) * x[i]; x[i] = q; }
    q = 0.0;
    for (int i = n - 1; i >= 0; --i) { q = a * q + (1.0 - a) * x[i]; x[i] = q; }
  }
  *alpha = a;
  *c = 1.0 / std::sqrt(x[half]);
}

void require_dec(dd4dv_ctx* ctx) {
  if (!ctx->has_dec) fail(ctx, DD4DV_ESTATE, "set_decomposition has not been called (or was invalidated)");
}

template <typename T>
SweepArgs<T> sweep_args(dd4dv_ctx* ctx) {
  SweepArgs<T> a{};
  a.subs = ctx->subs_d;
  a.order = ctx->order_d;
  a.n_sub = ctx->n_sub;
  a.traj = static_cast<T*>(ctx->traj);
  a.stg = ctx->use_stg ? static_cast<T*>(ctx->stg) : nullptr;
  a.stg1 = ctx->use_stg ? nullptr : static_cast<T*>(ctx->stg1);
  a.ckpt = ctx->ckpt;
  a.seg = static_cast<T*>(ctx->seg);
  a.tgt = static_cast<const T*>(ctx->tgt);
  a.bnd = static_cast<const T*>(ctx->bnd);
  a.rows = ctx->rows_d;
  a.Bth = ctx->Bth;
  a.gBth = ctx->gBth;
  a.dt = ctx->m.dt;
  a.h_ref = (sizeof(T) == 4) ? ctx->m.h_ref : 0.0;
  a.nlon = ctx->m.nlon;
  a.nlat = ctx->m.nlat;
  a.nsteps = ctx->m.nsteps;
  for (int v = 0; v < 3; ++v) a.isb2[v] = 1.0 / (ctx->sigma_b[v] * ctx->sigma_b[v]);
  a.lam = ctx->dec.lambda;
  a.mu = ctx->dec.mu;
  a.dt_s = (T)a.dt;
  a.Bth_s = (T)a.Bth;
  a.gBth_s = (T)a.gBth;
  a.href_s = (T)a.h_ref;
  for (int v = 0; v < 3; ++v) {
    a.isb2_s[v] = (T)a.isb2[v];
    a.musb2_s[v] = (T)(a.mu * a.isb2[v]);
  }
  a.obs = ctx->obs_d;
  a.lvl_obs = ctx->lvl_obs_d;
  a.obs_force = ctx->obs_force_d;
  a.sc_tgt = ctx->sc_tgt_d;
  a.sc_off = ctx->sc_off_d;
  a.sc_obs = ctx->sc_obs_d;
  a.sc_w = ctx->sc_w_d;
  a.lvl_sc = ctx->lvl_sc_d;
  a.part = ctx->part;
  a.cl_max = 16;   // part[] stride: room for the largest cluster
  a.active = nullptr;
  a.active_value = 0;
  a.lam_a = ctx->lam_a;
  a.yforce = nullptr;
  a.dx_out = nullptr;
  a.dx0 = nullptr;
  a.gn_dx = nullptr;
  a.R = ctx->R;
  a.W = ctx->W;
  a.err = ctx->err_d;
  a.min_ny = ctx->min_ny;
  a.variant = ctx->variant_a;   // adjoint (and tangent-linear) launches; forward_sweep sets its own
  return a;
}

double h_ref_of(dd4dv_ctx* ctx) { return ctx->m.precision == 1 ? ctx->m.h_ref : 0.0; }

// V w -> initial states (level 0 of every trajectory).  vw_buf receives L w.
// Largest ny * (nx | 1) plane of the decomposition (odd shared-memory row
// pitch), and whether it fits the fused shared-memory control-transform kernels.
static int max_plane(dd4dv_ctx* ctx) {
  int m = 0;
  for (const SubDesc& d : ctx->subs_h) m = std::max(m, d.ny * (d.nx | 1));
  return m;
}
static bool fused_v(dd4dv_ctx* ctx) { return (size_t)max_plane(ctx) * sizeof(double) <= 200 * 1024; }

template <typename T>
void init_states(dd4dv_ctx* ctx, const double* w, double* vw_buf, const int* active, int av) {
  if (fused_v(ctx)) {
    RFArgs ra{ctx->subs_d, ctx->n_sub, ctx->rf_alpha, ctx->rf_c, ctx->rf_passes, active, av};
    KL(launch_vinit<T>(ctx->subs_d, ctx->n_sub, ctx->xb_a, w, ctx->sigma_d, ra, ctx->corr_len > 0.0 ? 1 : 0,
                       h_ref_of(ctx), static_cast<T*>(ctx->traj), active, av, max_plane(ctx), ctx->st));
    return;
  }
  const double* src = w;
  if (ctx->corr_len > 0.0) {
    KL(launch_scale_copy(ctx->subs_d, ctx->n_sub, w, nullptr, vw_buf, active, av, ctx->max_pts, ctx->st));
    RFArgs ra{ctx->subs_d, ctx->n_sub, ctx->rf_alpha, ctx->rf_c, ctx->rf_passes, active, av};
    KL(launch_rf_rows(vw_buf, ra, ctx->max_ny, ctx->st));
    KL(launch_rf_cols(vw_buf, ra, ctx->max_nx, ctx->st));
    src = vw_buf;
  }
  KL(launch_init_state<T>(ctx->subs_d, ctx->n_sub, ctx->xb_a, src, ctx->sigma_d, 1, h_ref_of(ctx),
                          static_cast<T*>(ctx->traj), active, av, ctx->max_pts, ctx->st));
}

// out = V^T y  (+ w, times scale) for the subdomains in the mask.
void apply_VT(dd4dv_ctx* ctx, const double* y, const double* w, const double* scale, double* out,
              const int* active, int av) {
  if (fused_v(ctx)) {
    RFArgs ra{ctx->subs_d, ctx->n_sub, ctx->rf_alpha, ctx->rf_c, ctx->rf_passes, active, av};
    const int rf = ctx->corr_len > 0.0 ? 1 : 0;
    if (ctx->m.precision == 1)
      KL(launch_vgrad<float>(ctx->subs_d, ctx->n_sub, w, y, ctx->sigma_d, ra, rf, scale, out, active, av,
                             max_plane(ctx), ctx->st));
    else
      KL(launch_vgrad<double>(ctx->subs_d, ctx->n_sub, w, y, ctx->sigma_d, ra, rf, scale, out, active, av,
                              max_plane(ctx), ctx->st));
    return;
  }
  KL(launch_scale_copy(ctx->subs_d, ctx->n_sub, y, ctx->sigma_d, ctx->vw2, active, av, ctx->max_pts, ctx->st));
  if (ctx->corr_len > 0.0) {
    RFArgs ra{ctx->subs_d, ctx->n_sub, ctx->rf_alpha, ctx->rf_c, ctx->rf_passes, active, av};
    KL(launch_rf_cols(ctx->vw2, ra, ctx->max_nx, ctx->st));
    KL(launch_rf_rows(ctx->vw2, ra, ctx->max_ny, ctx->st));
  }
  KL(launch_grad_finish(ctx->subs_d, ctx->n_sub, w, ctx->vw2, scale, out, active, av, ctx->max_pts, ctx->st));
}

// full = true stores every level (exchange, trajectory export) even when the
// evaluations checkpoint.
template <typename T>
void forward_sweep(dd4dv_ctx* ctx, const int* active, int av, bool full = false) {
  SweepArgs<T> a = sweep_args<T>(ctx);
  a.active = active;
  a.active_value = av;
  if (full) {
    a.ckpt = 0;
    a.stg = nullptr;
    a.stg1 = nullptr;
  }
  a.R = ctx->R_f;
  a.variant = ctx->variant_f;
  KL(launch_forward<T>(a, ctx->cl_f, ctx->nt_f, ctx->st));
}

template <typename T>
void eval_T(dd4dv_ctx* ctx, const double* w, double* J, double* grad, double* parts, const int* active,
            int av, const double* scale) {
  init_states<T>(ctx, w, ctx->vw, active, av);
  forward_sweep<T>(ctx, active, av);
  KL(launch_finalize_J(ctx->subs_d, ctx->n_sub, w, ctx->part, ctx->cl_f, ctx->vconst, ctx->dec.lambda,
                       ctx->dec.mu, J, parts, active, av, ctx->st));
  if (grad) {
    SweepArgs<T> a = sweep_args<T>(ctx);
    a.active = active;
    a.active_value = av;
    KL(launch_adjoint<T>(a, ctx->cl, ctx->nthreads, ctx->st));
    apply_VT(ctx, ctx->lam_a, w, scale, grad, active, av);
  }
}

// Cluster size and rows per CTA of the tangent-linear sweep (six buffers):
// the smallest cluster (>= the evaluation's) whose stripes fit in shared memory.
void tlm_shape(dd4dv_ctx* ctx, int* cl, int* R) {
  for (int c = ctx->cl; c <= std::min(16, ctx->min_ny); ++c) {
    const int r = (ctx->max_ny + c - 1) / c;
    const size_t need = ctx->m.precision == 1 ? smem_tlm<float>(r, ctx->W) : smem_tlm<double>(r, ctx->W);
    if (need <= 232448) {
      *cl = c;
      *R = r;
      return;
    }
  }
  fail(ctx, DD4DV_EINVAL, "boxes too large for the tangent-linear sweep");
}

// out = V p (packed control layout) for the subdomains in the mask.
void apply_V(dd4dv_ctx* ctx, const double* p, double* out, const int* active, int av) {
  const double* src = p;
  if (ctx->corr_len > 0.0) {
    KL(launch_scale_copy(ctx->subs_d, ctx->n_sub, p, nullptr, ctx->vw2, active, av, ctx->max_pts, ctx->st));
    RFArgs ra{ctx->subs_d, ctx->n_sub, ctx->rf_alpha, ctx->rf_c, ctx->rf_passes, active, av};
    KL(launch_rf_rows(ctx->vw2, ra, ctx->max_ny, ctx->st));
    KL(launch_rf_cols(ctx->vw2, ra, ctx->max_nx, ctx->st));
    src = ctx->vw2;
  }
  KL(launch_scale_copy(ctx->subs_d, ctx->n_sub, src, ctx->sigma_d, out, active, av, ctx->max_pts, ctx->st));
}

// Work buffers of the Gauss-Newton solver, allocated with the decomposition's
// on first use.
void ensure_gn(dd4dv_ctx* ctx) {
  if (ctx->gn_dx) return;
  auto& L = ctx->dec_allocs;
  const size_t C = (size_t)ctx->ctrl_total;
  ctx->cg_r = dalloc<double>(ctx, C, &L);
  ctx->cg_p = dalloc<double>(ctx, C, &L);
  ctx->cg_Ap = dalloc<double>(ctx, C, &L);
  ctx->cg_dw = dalloc<double>(ctx, C, &L);
  ctx->cgst = dalloc<CgState>(ctx, ctx->n_sub, &L);
  ctx->gn_dx = dalloc<unsigned char>(ctx, std::max<long long>(1, ctx->traj_elems) * ctx->tsize, &L);
}

// Gauss-Newton product Ap = (I + G^T G) p for the subdomains in the mask, at
// the linearisation point whose trajectory (and stage states) the last
// forward sweep stored: V p, tangent-linear sweep (dx and H dx), adjoint sweep
// forced by dx, then p + V^T lambda(a).
template <typename T>
void gn_product_T(dd4dv_ctx* ctx, const double* p, double* Ap, const int* active, int av) {
  int tl_cl = 0, tl_R = 0;
  tlm_shape(ctx, &tl_cl, &tl_R);
  apply_V(ctx, p, ctx->io_c, active, av);
  SweepArgs<T> a = sweep_args<T>(ctx);
  a.active = active;
  a.active_value = av;
  a.dx0 = ctx->io_c;
  a.gn_dx = static_cast<T*>(ctx->gn_dx);
  a.R = tl_R;
  KL(launch_tlm<T>(a, tl_cl, ctx->nthreads, ctx->st));
  SweepArgs<T> b = sweep_args<T>(ctx);
  b.active = active;
  b.active_value = av;
  b.gn_dx = static_cast<T*>(ctx->gn_dx);
  KL(launch_adjoint<T>(b, ctx->cl, ctx->nthreads, ctx->st));
  apply_VT(ctx, ctx->lam_a, p, nullptr, Ap, active, av);
}

template <typename T>
void exchange_T(dd4dv_ctx* ctx, const double* w) {
  init_states<T>(ctx, w, ctx->vw, nullptr, 0);
  forward_sweep<T>(ctx, nullptr, 0, true);
  ExchArgs<T> x{};
  x.subs = ctx->subs_d;
  x.n_sub = ctx->n_sub;
  x.P1 = ctx->dec.P1;
  x.P2 = ctx->dec.P2;
  x.Q = ctx->dec.Q;
  x.nlon = ctx->m.nlon;
  x.nlat = ctx->m.nlat;
  x.nsteps = ctx->m.nsteps;
  x.traj = static_cast<const T*>(ctx->traj);
  x.tgt = static_cast<T*>(ctx->tgt);
  x.bnd = static_cast<T*>(ctx->bnd);
  for (int v = 0; v < 3; ++v) x.isb2[v] = 1.0 / (ctx->sigma_b[v] * ctx->sigma_b[v]);
  x.vpart = ctx->vpart;
  x.vblocks = ctx->vblocks;
  x.lon_cov = ctx->lon_cov_d;
  x.lat_cov = ctx->lat_cov_d;
  x.t_cov = ctx->t_cov_d;
  KL(launch_targets<T>(x, ctx->st));
  KL(launch_sum_vconst(ctx->vpart, ctx->n_sub, ctx->vblocks, ctx->vconst, ctx->st));
  KL(launch_assemble<T>(x, ctx->st));
  ctx->fwd_pending = false;
}

// The background trajectory (global model run of x_b(t0)), streamed through
// the chunk buffer into the frozen boundary trajectory B and the overlap
// targets (the state before the first exchange), and, with xb_a set, into the
// restricted background at each window's first level.
template <typename T>
void background_pass(dd4dv_ctx* ctx, bool xb_a);

template <typename T>
void reset_exchange_T(dd4dv_ctx* ctx) {
  if (ctx->bnd0 && ctx->tgt0) {
    CK(cudaMemcpyAsync(ctx->bnd, ctx->bnd0, ctx->gtraj * ctx->tsize, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->tgt, ctx->tgt0, ctx->traj_elems * ctx->tsize, cudaMemcpyDeviceToDevice, ctx->st));
  } else {
    background_pass<T>(ctx, false);
  }
  CK(cudaMemsetAsync(ctx->vconst, 0, ctx->n_sub * sizeof(double), ctx->st));
  ctx->fwd_pending = false;
}

// One RK3 step of the global model: x (device) -> nx (device), FP64.
void global_step(dd4dv_ctx* ctx, const double* x, double* nx) {
  double* s1 = ctx->gscratch;
  double* s2 = ctx->gscratch + ctx->gstate;
  KL(launch_global_stage(x, x, s1, 0.0, 1.0, ctx->rows_d, ctx->Bth, ctx->gBth, ctx->m.dt, ctx->m.nlon,
                         ctx->m.nlat, ctx->st));
  KL(launch_global_stage(x, s1, s2, 0.75, 0.25, ctx->rows_d, ctx->Bth, ctx->gBth, ctx->m.dt,
                         ctx->m.nlon, ctx->m.nlat, ctx->st));
  KL(launch_global_stage(x, s2, nx, 1.0 / 3.0, 2.0 / 3.0, ctx->rows_d, ctx->Bth, ctx->gBth, ctx->m.dt,
                         ctx->m.nlon, ctx->m.nlat, ctx->st));
}

// Global model run x0 (device) -> out trajectory (device, FP64).
void global_run(dd4dv_ctx* ctx, const double* x0, double* out) {
  const size_t G = ctx->gstate;
  CK(cudaMemcpyAsync(out, x0, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  for (int n = 0; n < ctx->m.nsteps; ++n) global_step(ctx, out + (size_t)n * G, out + (size_t)(n + 1) * G);
}

// Global model run from x0 (device) without a whole-trajectory buffer: the
// levels are produced in the chunk buffer, gchunk_lv at a time, and handed to
// sink(g0, g1, levels) (levels g0..g1, level-major FP64) in order.  The last
// level of a chunk is the first of the next.
template <typename Sink>
void global_run_chunked(dd4dv_ctx* ctx, const double* x0, Sink&& sink) {
  const size_t G = ctx->gstate;
  const int K = ctx->gchunk_lv - 1;
  double* c = ctx->gchunk;
  CK(cudaMemcpyAsync(c, x0, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  for (int g0 = 0;;) {
    const int g1 = std::min(g0 + K, ctx->m.nsteps);
    for (int n = g0; n < g1; ++n) global_step(ctx, c + (size_t)(n - g0) * G, c + (size_t)(n - g0 + 1) * G);
    sink(g0, g1, c);
    if (g1 >= ctx->m.nsteps) break;
    CK(cudaMemcpyAsync(c, c + (size_t)(g1 - g0) * G, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    g0 = g1;
  }
}

template <typename T>
void background_pass(dd4dv_ctx* ctx, bool xb_a) {
  const size_t G = ctx->gstate;
  const int nlon = ctx->m.nlon, nlat = ctx->m.nlat;
  global_run_chunked(ctx, ctx->xb0, [&](int g0, int g1, const double* lv) {
    const long long n = (long long)(g1 - g0 + 1) * G;
    KL(launch_bnd_from_global<T>(lv, n, h_ref_of(ctx), nlon, nlat, static_cast<T*>(ctx->bnd) + (size_t)g0 * G,
                                 ctx->st));
    KL(launch_restrict<T>(ctx->subs_d, ctx->n_sub, nlon, nlat, lv, g0, g1, h_ref_of(ctx),
                          static_cast<T*>(ctx->tgt), ctx->max_pts, ctx->st));
    if (xb_a) KL(launch_restrict_level(ctx->subs_d, ctx->n_sub, nlon, nlat, lv, g0, g1, ctx->xb_a, ctx->max_pts,
                                       ctx->st));
  });
}

// Ownership mask for evaluations: nullptr when the context owns every
// subdomain (the unmasked launches), else the device mask (value 1 = owned).
const int* own_mask(dd4dv_ctx* ctx) { return ctx->owned_all ? nullptr : ctx->owned_d; }

// Copies a host input into a device buffer when device_ptrs == 0.
const double* stage_in(dd4dv_ctx* ctx, const double* src, double* buf, size_t n, int device_ptrs) {
  if (device_ptrs) return src;
  h2d(ctx, buf, src, n * sizeof(double));
  return buf;
}

template <typename F>
auto by_precision(dd4dv_ctx* ctx, F&& f) {
  if (ctx->m.precision == 1) return f(float{});
  return f(double{});
}

// Kernel kinds (forward_kind / adjoint_kind: 0 = not launchable, 1 = stripe
// sweep, 2 = deep-halo FP32 sweep) of the sweeps at c CTAs per subdomain and
// nt threads per CTA, with the context's current stage-buffer use.
int fwd_kind_at(dd4dv_ctx* ctx, int c, int nt) {
  return by_precision(ctx, [&](auto t) {
    using T = decltype(t);
    SweepArgs<T> a = sweep_args<T>(ctx);
    a.R = (ctx->max_ny + c - 1) / c;
    a.variant = ctx->variant_f;
    return forward_kind<T>(a, c, nt);
  });
}
int adj_kind_at(dd4dv_ctx* ctx, int c, int nt) {
  return by_precision(ctx, [&](auto t) {
    using T = decltype(t);
    SweepArgs<T> a = sweep_args<T>(ctx);
    a.R = (ctx->max_ny + c - 1) / c;
    return adjoint_kind<T>(a, c, nt);
  });
}

// Frees one decomposition buffer ahead of dd4dv_destroy.
void free_dec_buffer(dd4dv_ctx* ctx, void*& p) {
  if (!p) return;
  auto it = std::find(ctx->dec_allocs.begin(), ctx->dec_allocs.end(), p);
  if (it != ctx->dec_allocs.end()) ctx->dec_allocs.erase(it);
  cudaFree(p);
  p = nullptr;
}

// The project's autotuner: for every feasible launch shape -- cluster size
// (CTAs per subdomain) x threads per CTA -- and, when the stage buffer exists,
// for stored and for recomputed stage states, it times the forward and the
// adjoint sweep separately (CUDA events around each launch, evaluation at
// w = 0) and keeps the fastest shape of each sweep and the faster stage mode.
// Thread counts include ones that divide a CTA's points evenly; FP32 sweeps
// are timed in their stripe and deep-halo forms, the adjoint also in its
// four-buffer form.  The search stops early when it has used a time budget of
// 80 evaluations (at least 2 s).  Results do not depend on the shapes except for the order of the
// per-CTA partial sums of J.
void autotune(dd4dv_ctx* ctx) {
  const bool f32 = ctx->m.precision == 1;
  int dev = 0, cap = 232448;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  CK(cudaMemsetAsync(ctx->io_a, 0, ctx->ctrl_total * sizeof(double), ctx->st));
  cudaEvent_t ev[4];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  auto smem_a = [&](int R) { return f32 ? smem_adjoint<float>(R, ctx->W) : smem_adjoint<double>(R, ctx->W); };
  // one evaluation's kernels at the shape (c, nt); returns false if not launchable
  auto run = [&](int c, int nt, float* tf, float* ta) -> bool {
    const int R = (ctx->max_ny + c - 1) / c;
    // the forward takes nt threads where its kernel allows them, else the
    // largest count its stripe kernel allows
    const int ntf = fwd_kind_at(ctx, c, nt) ? nt
                    : std::min(nt, f32 ? max_threads_forward<float>() : max_threads_forward<double>());
    if (!fwd_kind_at(ctx, c, ntf) || !adj_kind_at(ctx, c, nt)) return false;
    ctx->cl_f = ctx->cl = c;
    ctx->R_f = ctx->R = R;
    ctx->nthreads = nt;
    ctx->nt_f = ntf;
    try {
      by_precision(ctx, [&](auto tt) {
        using T = decltype(tt);
        init_states<T>(ctx, ctx->io_a, ctx->vw, nullptr, 0);
        CK(cudaEventRecord(ev[0], ctx->st));
        forward_sweep<T>(ctx, nullptr, 0);
        CK(cudaEventRecord(ev[1], ctx->st));
        SweepArgs<T> a = sweep_args<T>(ctx);
        CK(cudaEventRecord(ev[2], ctx->st));
        KL(launch_adjoint<T>(a, ctx->cl, ctx->nthreads, ctx->st));
        CK(cudaEventRecord(ev[3], ctx->st));
        return 0;
      });
    } catch (const Fail&) {
      cudaGetLastError();
      ctx->err.clear();
      return false;
    }
    CK(cudaEventSynchronize(ev[3]));
    CK(cudaEventElapsedTime(tf, ev[0], ev[1]));
    CK(cudaEventElapsedTime(ta, ev[2], ev[3]));
    return true;
  };
  std::vector<int> cls;
  {
    const int va = ctx->variant_a;
    ctx->variant_a = 2;   // the smallest footprint
    for (int c : {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16})
      if (c <= ctx->min_ny && (smem_a((ctx->max_ny + c - 1) / c) <= (size_t)cap || adj_kind_at(ctx, c, 512)))
        cls.push_back(c);
    ctx->variant_a = va;
  }
  // 1024 and 768 threads reach the FP64 forward and the stripe adjoints, 640
  // and 576 also the deep-halo FP32 sweeps
  const int nts[] = {1024, 768, 640, 576, 512, 448, 384, 320, 256, 192};
  // reference time of the starting shape sets the budget
  float tf0 = 0, ta0 = 0;
  const int c0 = ctx->cl, n0 = ctx->nthreads;
  run(c0, n0, &tf0, &ta0);
  run(c0, n0, &tf0, &ta0);
  const double budget_ms = std::max(2000.0, 80.0 * (tf0 + ta0));
  double spent = 0.0;
  struct Best { double t = 1e300; int c = 0, nt = 0, var = 0; };
  Best best_f[2], best_a[2];
  const bool have_stg = ctx->stg != nullptr;
  const int var0 = ctx->variant_f;   // the caller's choice: 1 keeps the stripe sweeps
  for (int use : {1, 0}) {
    if (use && !have_stg) continue;
    ctx->use_stg = use;
    for (int c : cls)
      for (int nt : nts)
        for (int var : {0, 1, 2}) {
          if (spent > budget_ms) break;
          if (var < var0) continue;
          ctx->variant_f = ctx->variant_a = var;
          // the stripe form is timed separately only where the deep form applied
          if (var == 1 && var0 == 0) {
            ctx->variant_f = ctx->variant_a = 0;
            const bool deep = fwd_kind_at(ctx, c, nt) == 2 || adj_kind_at(ctx, c, nt) == 2;
            ctx->variant_f = ctx->variant_a = 1;
            if (!deep) continue;
          }
          // the two-buffer forward and the four-buffer adjoint, where they
          // apply and the other variants did not already fall back to them
          bool new_f = false, new_a = false;
          if (var == 2) {
            ctx->variant_f = ctx->variant_a = 1;
            const bool a3 = adj_kind_at(ctx, c, nt) == 3;
            ctx->variant_f = ctx->variant_a = 2;
            new_f = fwd_kind_at(ctx, c, std::min(nt, f32 ? max_threads_forward<float>()
                                                       : max_threads_forward<double>())) == 4;
            new_a = !a3 && adj_kind_at(ctx, c, nt) == 3;
            if (!new_f) ctx->variant_f = 1;
            if (!new_f && !new_a) continue;
          }
          float tf = 0, ta = 0, tf2 = 0, ta2 = 0;
          if (!run(c, nt, &tf, &ta)) continue;
          if (!run(c, nt, &tf2, &ta2)) continue;
          spent += tf + ta + tf2 + ta2;
          tf = std::min(tf, tf2);
          ta = std::min(ta, ta2);
          if ((var != 2 || new_f) && tf < best_f[use].t) best_f[use] = {tf, c, ctx->nt_f, var};
          if ((var != 2 || new_a) && ta < best_a[use].t) best_a[use] = {ta, c, nt, var};
        }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  int use = 0;
  if (have_stg && best_f[1].c && best_a[1].c &&
      (!best_f[0].c || best_f[1].t + best_a[1].t < best_f[0].t + best_a[0].t))
    use = 1;
  if (!best_f[use].c || !best_a[use].c) {   // nothing measured: keep the starting shape
    best_f[use] = {tf0, c0, n0, var0};
    best_a[use] = {ta0, c0, n0, var0};
  }
  ctx->use_stg = use;
  ctx->variant_f = best_f[use].var;
  ctx->variant_a = best_a[use].var;
  ctx->cl_f = best_f[use].c;
  ctx->nt_f = best_f[use].nt;
  ctx->R_f = (ctx->max_ny + ctx->cl_f - 1) / ctx->cl_f;
  ctx->cl = best_a[use].c;
  ctx->nthreads = best_a[use].nt;
  ctx->R = (ctx->max_ny + ctx->cl - 1) / ctx->cl;
  ctx->dec.cluster = ctx->cl;
  ctx->tune_ms = best_f[use].t + best_a[use].t;
  sync(ctx);
  if (!use && ctx->stg && ctx->dec.ckpt_k != -2) {   // recomputing the stages won: give the memory back
    free_dec_buffer(ctx, ctx->stg);
    ctx->stg_elems = 0;
  }
}

// Checkpoint intervals the library tries for ckpt_k = -2.
constexpr int kTunedCkpt[3] = {8, 16, 32};

// ckpt_k = -2: time one forward + adjoint evaluation (w = 0, CUDA events,
// best of two) with stored stage states (when their buffer exists), with the
// stages recomputed, and with k-step checkpoints for k in kTunedCkpt, at the
// current launch shapes; keep the fastest and free the buffers it does not
// use.  Results do not depend on the choice.
void tune_checkpoint(dd4dv_ctx* ctx) {
  CK(cudaMemsetAsync(ctx->io_a, 0, ctx->ctrl_total * sizeof(double), ctx->st));
  cudaEvent_t ev[2];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  auto time_eval = [&](int k, bool stg) -> float {
    ctx->ckpt = k;
    ctx->use_stg = stg;
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      by_precision(ctx, [&](auto t) {
        using T = decltype(t);
        CK(cudaEventRecord(ev[0], ctx->st));
        eval_T<T>(ctx, ctx->io_a, ctx->io_p, ctx->io_b, nullptr, nullptr, 0, nullptr);
        CK(cudaEventRecord(ev[1], ctx->st));
        return 0;
      });
      CK(cudaEventSynchronize(ev[1]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      if (r > 0) best = std::min(best, ms);   // the first run warms up
    }
    return best;
  };
  struct Cand { int k; bool stg; float ms; };
  std::vector<Cand> c;
  if (ctx->stg) c.push_back({0, true, time_eval(0, true)});
  c.push_back({0, false, time_eval(0, false)});
  for (int k : kTunedCkpt) c.push_back({k, false, time_eval(k, false)});
  for (auto& e : ev) cudaEventDestroy(e);
  const Cand best = *std::min_element(c.begin(), c.end(), [](const Cand& a, const Cand& b) { return a.ms < b.ms; });
  ctx->ckpt = best.k;
  ctx->use_stg = best.stg;
  sync(ctx);
  if (!best.stg && ctx->stg) {
    free_dec_buffer(ctx, ctx->stg);
    ctx->stg_elems = 0;
  }
  if (best.k == 0 && ctx->seg) free_dec_buffer(ctx, ctx->seg);
  ctx->ckpt_ms = best.ms;
}

// ---------------------------------------------------------------------------
// Decomposition tables.
std::vector<int> make_cuts(dd4dv_ctx* ctx, const int* cuts, int n, int parts, const char* name) {
  std::vector<int> c(parts + 1);
  if (parts == 1) {   // one block: the whole axis, whatever was passed
    c[0] = 0;
    c[1] = n;
    return c;
  }
  if (cuts) {
    for (int k = 0; k <= parts; ++k) c[k] = cuts[k];
    if (c[0] != 0 || c[parts] != n) fail(ctx, DD4DV_EINVAL, "%s cuts must run from 0 to %d", name, n);
    for (int k = 0; k < parts; ++k)
      if (c[k + 1] <= c[k]) fail(ctx, DD4DV_EINVAL, "%s cuts must increase", name);
  } else {
    for (int k = 0; k <= parts; ++k) c[k] = (int)(((long long)k * n) / parts);
  }
  return c;
}

void build_decomposition(dd4dv_ctx* ctx, const dd4dv_decomp& d) {
  const int nlon = ctx->m.nlon, nlat = ctx->m.nlat, nsteps = ctx->m.nsteps;
  if (d.P1 < 1 || d.P2 < 1 || d.Q < 1) fail(ctx, DD4DV_EINVAL, "P1, P2, Q must be >= 1");
  if (d.o_lon < 0 || d.o_lat < 0 || d.o_t < 0) fail(ctx, DD4DV_EINVAL, "overlaps must be >= 0");
  if (!(d.mu >= 0.0) || !(d.lambda >= 0.0)) fail(ctx, DD4DV_EINVAL, "mu, lambda must be >= 0");
  if (d.Q > 1 && nsteps < 1) fail(ctx, DD4DV_EINVAL, "time split needs nsteps >= 1");
  ctx->lon_cuts = make_cuts(ctx, d.lon_cuts, nlon, d.P1, "lon");
  ctx->lat_cuts = make_cuts(ctx, d.lat_cuts, nlat, d.P2, "lat");
  ctx->t_cuts = make_cuts(ctx, d.t_cuts, nsteps, d.Q, "time");
  if (d.P1 > 1) {
    if (d.o_lon < 1) fail(ctx, DD4DV_EINVAL, "o_lon must be >= 1 when longitude is split");
    for (int k = 0; k < d.P1; ++k) {
      const int core = ctx->lon_cuts[k + 1] - ctx->lon_cuts[k];
      if (core < 2 * d.o_lon || core < 2) fail(ctx, DD4DV_EINVAL, "lon core block %d (%d) < 2*o_lon", k, core);
      if (core + 2 * d.o_lon >= nlon) fail(ctx, DD4DV_EINVAL, "extended lon box wraps onto itself");
    }
  }
  if (d.P2 > 1) {
    if (d.o_lat < 1) fail(ctx, DD4DV_EINVAL, "o_lat must be >= 1 when latitude is split");
    for (int k = 0; k < d.P2; ++k) {
      const int core = ctx->lat_cuts[k + 1] - ctx->lat_cuts[k];
      if (core < 2 * d.o_lat || core < 2) fail(ctx, DD4DV_EINVAL, "lat core block %d (%d) < 2*o_lat", k, core);
    }
  }
  if (d.Q > 1)
    for (int k = 0; k < d.Q; ++k) {
      const int core = ctx->t_cuts[k + 1] - ctx->t_cuts[k];
      if (core < 2 * d.o_t + 1) fail(ctx, DD4DV_EINVAL, "time core block %d (%d) < 2*o_t+1", k, core);
    }
  if (d.ckpt_k < -3) fail(ctx, DD4DV_EINVAL, "ckpt_k must be >= -3");
  // ckpt_k = -2: the segment buffers are sized for the largest interval tried
  const int seg_k = d.ckpt_k > 0 ? d.ckpt_k : (d.ckpt_k == -2 ? kTunedCkpt[2] : 0);

  const int n_sub = d.P1 * d.P2 * d.Q;
  std::vector<SubDesc> subs(n_sub);
  long long ctrl = 0, trj = 0, ptrj = 0, pts = 0, stgl = 0, segl = 0;
  int max_nx = 0, max_ny = 0, min_ny = 1 << 30, max_lv = 0, max_pts = 0;
  for (int q = 0; q < d.Q; ++q)
    for (int p2 = 0; p2 < d.P2; ++p2)
      for (int p1 = 0; p1 < d.P1; ++p1) {
        SubDesc s{};
        const int idx = (q * d.P2 + p2) * d.P1 + p1;
        if (d.Q == 1) { s.a = 0; s.b = nsteps; }
        else {
          s.a = std::max(0, ctx->t_cuts[q] - d.o_t);
          s.b = std::min(nsteps, ctx->t_cuts[q + 1] + d.o_t);
        }
        if (d.P2 == 1) { s.j0 = 0; s.ny = nlat; }
        else {
          s.j0 = std::max(0, ctx->lat_cuts[p2] - d.o_lat);
          s.ny = std::min(nlat, ctx->lat_cuts[p2 + 1] + d.o_lat) - s.j0;
        }
        s.flags = 0;
        if (d.P1 == 1) { s.i0 = 0; s.nx = nlon; s.flags |= F_PERIODIC; }
        else {
          s.i0 = ((ctx->lon_cuts[p1] - d.o_lon) % nlon + nlon) % nlon;
          s.nx = ctx->lon_cuts[p1 + 1] - ctx->lon_cuts[p1] + 2 * d.o_lon;
        }
        if (s.j0 == 0) s.flags |= F_SWALL;
        if (s.j0 + s.ny == nlat) s.flags |= F_NWALL;
        s.q = q; s.p2 = p2; s.p1 = p1;
        s.wL = s.wR = (d.P1 > 1) ? 2 * d.o_lon : 0;
        s.wS = (p2 > 0) ? 2 * d.o_lat : 0;
        s.wN = (p2 < d.P2 - 1) ? 2 * d.o_lat : 0;
        s.tA = (q > 0) ? 2 * d.o_t + 1 : 0;
        s.tB = (q < d.Q - 1) ? 2 * d.o_t + 1 : 0;
        if (s.ny < 2 || s.nx < 2) fail(ctx, DD4DV_EINVAL, "subdomain boxes need at least 2x2 points");
        s.nxp = (s.nx + 3) / 4 * 4;
        const int L = s.b - s.a;
        s.ctrl_off = ctrl;
        s.traj_off = trj;
        s.ptraj_off = ptrj;
        s.stg_off = stgl;
        s.stg1_off = -1;
        stgl += (long long)L * 2 * 3 * s.ny * s.nxp;
        s.seg_off = segl;
        if (seg_k > 0) segl += (long long)(std::min(seg_k, std::max(L, 1)) + 1) * 3 * s.ny * s.nxp;
        ctrl += 3LL * s.ny * s.nx;
        trj += (long long)(L + 1) * 3 * s.ny * s.nxp;
        ptrj += (long long)(L + 1) * 3 * s.ny * s.nx;
        pts += (long long)s.nx * s.ny * L;
        max_nx = std::max(max_nx, s.nx);
        max_ny = std::max(max_ny, s.ny);
        min_ny = std::min(min_ny, s.ny);
        max_lv = std::max(max_lv, L + 1);
        max_pts = std::max(max_pts, 3 * s.ny * s.nx);
        subs[idx] = s;
      }
  ctx->n_sub = n_sub;
  ctx->ctrl_total = ctrl;
  ctx->traj_elems = trj;
  ctx->ptraj_total = ptrj;
  ctx->pt_steps = pts;
  ctx->max_nx = max_nx;
  ctx->max_ny = max_ny;
  ctx->min_ny = min_ny;
  ctx->max_levels = max_lv;
  ctx->max_pts = max_pts;

  // observations -> per-subdomain records, per-level ranges, adjoint scatter plan
  const double href = h_ref_of(ctx);
  std::vector<std::vector<std::pair<int, ObsRec>>> per_sub(n_sub);   // (level, rec)
  const size_t nob = ctx->ob_level.size();
  std::vector<int> lon_in, lat_in, win_in;
  for (size_t k = 0; k < nob; ++k) {
    const double fi = ctx->ob_fi[k], fj = ctx->ob_fj[k];
    const int i0 = (int)std::floor(fi), j0 = (int)std::floor(fj);
    const double di = fi - i0, dj = fj - j0;
    const int i1 = (i0 + 1) % nlon;
    const int lev = ctx->ob_level[k];
    lon_in.clear(); lat_in.clear(); win_in.clear();
    for (int p1 = 0; p1 < d.P1; ++p1) {
      const SubDesc& s = subs[p1];
      const int k0 = ((i0 - s.i0) % nlon + nlon) % nlon;
      const int k1 = ((i1 - s.i0) % nlon + nlon) % nlon;
      if (k0 < s.nx && (di == 0.0 || k1 < s.nx)) lon_in.push_back(p1);
    }
    for (int p2 = 0; p2 < d.P2; ++p2) {
      const SubDesc& s = subs[p2 * d.P1];
      if (j0 >= s.j0 && j0 < s.j0 + s.ny && (dj == 0.0 || j0 + 1 < s.j0 + s.ny)) lat_in.push_back(p2);
    }
    for (int q = 0; q < d.Q; ++q) {
      const SubDesc& s = subs[q * d.P2 * d.P1];
      if (lev >= s.a && lev <= s.b) win_in.push_back(q);
    }
    const size_t cnt = lon_in.size() * lat_in.size() * win_in.size();
    if (cnt == 0) continue;
    const double omega = d.weight_obs ? 1.0 / (double)cnt : 1.0;
    for (int q : win_in)
      for (int p2 : lat_in)
        for (int p1 : lon_in) {
          const int sidx = (q * d.P2 + p2) * d.P1 + p1;
          const SubDesc& s = subs[sidx];
          ObsRec r{};
          r.var = ctx->ob_var[k];
          r.r0 = j0 - s.j0;
          r.k0 = ((i0 - s.i0) % nlon + nlon) % nlon;
          r.k1 = (di != 0.0) ? ((i1 - s.i0) % nlon + nlon) % nlon : r.k0;
          r.di = di;
          r.dj = dj;
          r.y = ctx->ob_val[k] - (r.var == 0 ? href : 0.0);
          r.w = omega / (ctx->ob_so[k] * ctx->ob_so[k]);
          per_sub[sidx].push_back({lev - s.a, r});
        }
  }
  std::vector<ObsRec> recs;
  std::vector<int> lvl_obs, lvl_sc, sc_tgt, sc_off, sc_obs;
  std::vector<double> sc_w;
  for (int sidx = 0; sidx < n_sub; ++sidx) {
    SubDesc& s = subs[sidx];
    const int L = s.b - s.a;
    auto& v = per_sub[sidx];
    std::stable_sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    s.obs_lvl = (int)lvl_obs.size();
    s.sc_lvl = (int)lvl_sc.size();
    size_t pos = 0;
    for (int l = 0; l <= L; ++l) {
      lvl_obs.push_back((int)recs.size());
      lvl_sc.push_back((int)sc_tgt.size());
      std::map<int, std::vector<std::pair<int, double>>> tg;   // target -> (record, weight)
      while (pos < v.size() && v[pos].first == l) {
        const int ridx = (int)recs.size();
        const ObsRec& r = v[pos].second;
        recs.push_back(r);
        const int plane = s.ny * s.nx;
        auto add = [&](int rr, int kk, double wgt) {
          tg[r.var * plane + rr * s.nx + kk].push_back({ridx, wgt});
        };
        add(r.r0, r.k0, (1.0 - r.dj) * (1.0 - r.di));
        if (r.di != 0.0) add(r.r0, r.k1, (1.0 - r.dj) * r.di);
        if (r.dj != 0.0) {
          add(r.r0 + 1, r.k0, r.dj * (1.0 - r.di));
          if (r.di != 0.0) add(r.r0 + 1, r.k1, r.dj * r.di);
        }
        ++pos;
      }
      for (auto& kv : tg) {
        sc_tgt.push_back(kv.first);
        sc_off.push_back((int)sc_obs.size());
        for (auto& c : kv.second) {
          sc_obs.push_back(c.first);
          sc_w.push_back(c.second);
        }
      }
    }
    lvl_obs.push_back((int)recs.size());
    lvl_sc.push_back((int)sc_tgt.size());
  }
  sc_off.push_back((int)sc_obs.size());

  // cover tables for the assembly
  std::vector<int> lon_cov(nlon * 4, -1), lat_cov(nlat * 4, -1), t_cov((nsteps + 1) * 4, -1);
  for (int i = 0; i < nlon; ++i) {
    int c = 0;
    for (int p1 = 0; p1 < d.P1 && c < 2; ++p1) {
      const SubDesc& s = subs[p1];
      const int kk = ((i - s.i0) % nlon + nlon) % nlon;
      if (kk < s.nx) { lon_cov[i * 4 + 2 * c] = p1; lon_cov[i * 4 + 2 * c + 1] = kk; ++c; }
    }
  }
  for (int j = 0; j < nlat; ++j) {
    int c = 0;
    for (int p2 = 0; p2 < d.P2 && c < 2; ++p2) {
      const SubDesc& s = subs[p2 * d.P1];
      if (j >= s.j0 && j < s.j0 + s.ny) { lat_cov[j * 4 + 2 * c] = p2; lat_cov[j * 4 + 2 * c + 1] = j - s.j0; ++c; }
    }
  }
  for (int n = 0; n <= nsteps; ++n) {
    int c = 0;
    for (int q = 0; q < d.Q && c < 2; ++q) {
      const SubDesc& s = subs[q * d.P2 * d.P1];
      if (n >= s.a && n <= s.b) { t_cov[n * 4 + 2 * c] = q; t_cov[n * 4 + 2 * c + 1] = n - s.a; ++c; }
    }
  }

  // cluster size: CTAs per subdomain
  const size_t smem_cap = 232448;
  const bool f32 = ctx->m.precision == 1;
  ctx->W = max_nx + 2;
  auto smem_need_min = [&](int R) {   // the four-buffer stripe adjoint
    return f32 ? smem_adjoint_rl<float>(R, ctx->W) : smem_adjoint_rl<double>(R, ctx->W);
  };
  int cl = d.cluster;
  ctx->nthreads = 256;
  if (cl > 0) {
    if (cl > 16 || cl > min_ny) fail(ctx, DD4DV_EINVAL, "cluster size %d must be <= 16 and <= smallest box height %d", cl, min_ny);
    ctx->R = (max_ny + cl - 1) / cl;
    if (smem_need_min(ctx->R) > smem_cap) fail(ctx, DD4DV_EINVAL, "cluster size %d needs too much shared memory", cl);
  } else {
    // Launch-shape model.  A cluster runs inside one GPC, so how many
    // subdomains run at once depends on how the GPCs' SMs divide by the
    // cluster size (asked of the runtime with the adjoint kernel's real
    // footprint), not only on CTAs per SM.  Estimated time = waves of
    // clusters x rows per CTA x CTAs sharing an SM (at least 1); the smallest
    // cluster within 3 % of the best wins (fewer CTAs, fewer barriers).
    // Threads: about 4 own points each, 128..512.
    int nsm = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    double best = 1e300;
    int best_cl = -1, best_nt = 256;
    for (int c = 1; c <= 16; ++c) {
      if (c > min_ny) break;
      const int R = (max_ny + c - 1) / c;
      if (smem_need_min(R) > smem_cap) continue;
      const int nt = std::min(512, std::max(128, 32 * ((R * max_nx + 127) / 128)));
      const int act = f32 ? active_clusters_adjoint<float>(R, ctx->W, c, nt)
                          : active_clusters_adjoint<double>(R, ctx->W, c, nt);
      if (act < 1) continue;
      const double waves = std::ceil((double)n_sub / act);
      const double share = std::max(1.0, (double)std::min(act, n_sub) * c / nsm);
      const double cost = waves * R * share;
      if (cost < best * 0.97) { best = cost; best_cl = c; best_nt = nt; }
    }
    if (best_cl < 0) fail(ctx, DD4DV_EINVAL, "subdomain boxes too large for the shared-memory sweep (max %dx%d)", max_nx, max_ny);
    cl = best_cl;
    ctx->R = (max_ny + cl - 1) / cl;
    ctx->nthreads = best_nt;
  }
  ctx->cl = cl;
  ctx->cl_f = cl;
  ctx->R_f = ctx->R;
  ctx->nt_f = std::min(ctx->nthreads, f32 ? max_threads_forward<float>() : max_threads_forward<double>());

  // device tables and buffers
  ctx->free_dec();
  auto& L = ctx->dec_allocs;
  ctx->tsize = f32 ? sizeof(float) : sizeof(double);
  ctx->subs_d = dalloc<SubDesc>(ctx, n_sub, &L);
  ctx->order_d = dalloc<int>(ctx, n_sub, &L);
  std::vector<int> order(n_sub);
  for (int s = 0; s < n_sub; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const long long wx = (long long)subs[x].nx * subs[x].ny * (subs[x].b - subs[x].a + 1);
    const long long wy = (long long)subs[y].nx * subs[y].ny * (subs[y].b - subs[y].a + 1);
    return wx > wy;
  });
  ctx->traj = dalloc<unsigned char>(ctx, ctx->traj_elems * ctx->tsize, &L);
  ctx->stg = nullptr;
  ctx->stg_elems = 0;
  ctx->use_stg = false;
  ctx->bnd0 = ctx->tgt0 = nullptr;
  ctx->cg_r = ctx->cg_p = ctx->cg_Ap = ctx->cg_dw = nullptr;
  ctx->cgst = nullptr;
  ctx->gn_dx = nullptr;
  ctx->ckpt = d.ckpt_k > 0 ? d.ckpt_k : 0;
  ctx->seg = nullptr;
  if (seg_k > 0) ctx->seg = dalloc<unsigned char>(ctx, std::max<long long>(1, segl) * ctx->tsize, &L);
  ctx->tgt = dalloc<unsigned char>(ctx, ctx->traj_elems * ctx->tsize, &L);
  ctx->bnd = dalloc<unsigned char>(ctx, ctx->gtraj * ctx->tsize, &L);
  const size_t C = (size_t)ctrl;
  ctx->xb_a = dalloc<double>(ctx, C, &L);
  ctx->w = dalloc<double>(ctx, C, &L);
  ctx->w_prev = dalloc<double>(ctx, C, &L);
  ctx->g = dalloc<double>(ctx, C, &L);
  ctx->wt = dalloc<double>(ctx, C, &L);
  ctx->gt = dalloc<double>(ctx, C, &L);
  ctx->p = dalloc<double>(ctx, C, &L);
  ctx->vw = dalloc<double>(ctx, C, &L);
  ctx->vw2 = dalloc<double>(ctx, C, &L);
  ctx->lam_a = dalloc<double>(ctx, C, &L);
  ctx->io_a = dalloc<double>(ctx, C, &L);
  ctx->io_b = dalloc<double>(ctx, C, &L);
  ctx->io_c = dalloc<double>(ctx, C, &L);
  ctx->J = dalloc<double>(ctx, n_sub, &L);
  ctx->Jt = dalloc<double>(ctx, n_sub, &L);
  ctx->io_p = dalloc<double>(ctx, 5 * n_sub, &L);
  ctx->parts = dalloc<double>(ctx, 3 * n_sub, &L);
  ctx->part = dalloc<double>(ctx, 2 * (size_t)n_sub * 16, &L);
  ctx->vconst = dalloc<double>(ctx, n_sub, &L);
  ctx->vpart = dalloc<double>(ctx, (size_t)n_sub * ctx->vblocks, &L);
  ctx->ptraj_io = nullptr;
  const int m = 8;   // history slots allocated (solver lbfgs_m <= 8)
  ctx->S = dalloc<double>(ctx, m * C, &L);
  ctx->Y = dalloc<double>(ctx, m * C, &L);
  ctx->rho = dalloc<double>(ctx, (size_t)m * n_sub, &L);
  ctx->lbst = dalloc<LbState>(ctx, n_sub, &L);
  ctx->phase_d = dalloc<int>(ctx, n_sub, &L);
  ctx->owned_d = dalloc<int>(ctx, n_sub, &L);
  ctx->owned_h.assign(n_sub, 1);
  ctx->owned_all = true;
  ctx->obs_d = dalloc<ObsRec>(ctx, recs.size(), &L);
  ctx->obs_force_d = dalloc<double>(ctx, recs.size(), &L);
  ctx->lvl_obs_d = dalloc<int>(ctx, lvl_obs.size(), &L);
  ctx->lvl_sc_d = dalloc<int>(ctx, lvl_sc.size(), &L);
  ctx->sc_tgt_d = dalloc<int>(ctx, sc_tgt.size(), &L);
  ctx->sc_off_d = dalloc<int>(ctx, sc_off.size(), &L);
  ctx->sc_obs_d = dalloc<int>(ctx, sc_obs.size(), &L);
  ctx->sc_w_d = dalloc<double>(ctx, sc_w.size(), &L);
  ctx->lon_cov_d = dalloc<int>(ctx, lon_cov.size(), &L);
  ctx->lat_cov_d = dalloc<int>(ctx, lat_cov.size(), &L);
  ctx->t_cov_d = dalloc<int>(ctx, t_cov.size(), &L);
  // Stored stage states (ckpt_k = 0) are twice the trajectory: allocate them
  // last, and only if they leave a reserve of 4 GB + 5 % of the device free;
  // otherwise the adjoint recomputes the stages.
  if (d.ckpt_k == 0 || d.ckpt_k == -2) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double need = (double)std::max<long long>(1, stgl) * ctx->tsize;
    const double reserve = 4.0 * (1ull << 30) + 0.05 * (double)total_b;
    if (need + reserve <= (double)free_b) {
      ctx->stg_elems = stgl;
      ctx->stg = dalloc<unsigned char>(ctx, std::max<long long>(1, stgl) * ctx->tsize, &L);
      ctx->use_stg = true;
    }
  }
  // FP64 path: where both stage states do not fit (ckpt_k = 0), or on
  // request (ckpt_k = -3), the first stage state x1 alone is stored for as
  // many subdomains as fit in the same reserve, longest first; their adjoint
  // then recomputes only x2.  Results are the same either way.  (The FP32
  // sweeps are compiled without this mode: the FP32 states are half the size
  // and both stage states fit where x1 alone would be needed in FP64.)
  ctx->stg1 = nullptr;
  ctx->stg1_subs = 0;
  ctx->stg1_frac = 0.0;
  if (!f32 && !ctx->stg && (d.ckpt_k == 0 || d.ckpt_k == -3)) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double reserve = 4.0 * (1ull << 30) + 0.05 * (double)total_b;
    const double budget = ((double)free_b - reserve) / (double)ctx->tsize;
    long long used = 0, pts_in = 0;
    for (int idx : order) {
      SubDesc& sd = subs[idx];
      const long long need = (long long)(sd.b - sd.a) * 3 * sd.ny * sd.nxp;
      if (need > 0 && (double)(used + need) <= budget) {
        sd.stg1_off = used;
        used += need;
        pts_in += (long long)sd.nx * sd.ny * (sd.b - sd.a);
        ++ctx->stg1_subs;
      }
    }
    if (used > 0) {
      ctx->stg1 = dalloc<unsigned char>(ctx, used * ctx->tsize, &L);
      ctx->stg1_frac = pts > 0 ? (double)pts_in / (double)pts : 0.0;
    }
  }
  h2d(ctx, ctx->subs_d, subs.data(), subs.size() * sizeof(SubDesc));
  h2d(ctx, ctx->order_d, order.data(), order.size() * sizeof(int));
  {
    const std::vector<int> ones(n_sub, 1);
    h2d(ctx, ctx->owned_d, ones.data(), n_sub * sizeof(int));
  }
  if (!recs.empty()) h2d(ctx, ctx->obs_d, recs.data(), recs.size() * sizeof(ObsRec));
  h2d(ctx, ctx->lvl_obs_d, lvl_obs.data(), lvl_obs.size() * sizeof(int));
  h2d(ctx, ctx->lvl_sc_d, lvl_sc.data(), lvl_sc.size() * sizeof(int));
  if (!sc_tgt.empty()) h2d(ctx, ctx->sc_tgt_d, sc_tgt.data(), sc_tgt.size() * sizeof(int));
  h2d(ctx, ctx->sc_off_d, sc_off.data(), sc_off.size() * sizeof(int));
  if (!sc_obs.empty()) {
    h2d(ctx, ctx->sc_obs_d, sc_obs.data(), sc_obs.size() * sizeof(int));
    h2d(ctx, ctx->sc_w_d, sc_w.data(), sc_w.size() * sizeof(double));
  }
  h2d(ctx, ctx->lon_cov_d, lon_cov.data(), lon_cov.size() * sizeof(int));
  h2d(ctx, ctx->lat_cov_d, lat_cov.data(), lat_cov.size() * sizeof(int));
  h2d(ctx, ctx->t_cov_d, t_cov.data(), t_cov.size() * sizeof(int));
  CK(cudaMemsetAsync(ctx->w, 0, C * sizeof(double), ctx->st));
  CK(cudaMemsetAsync(ctx->w_prev, 0, C * sizeof(double), ctx->st));
  CK(cudaMemsetAsync(ctx->traj, 0, ctx->traj_elems * ctx->tsize, ctx->st));
  CK(cudaMemsetAsync(ctx->obs_force_d, 0, std::max<size_t>(1, recs.size()) * sizeof(double), ctx->st));
  ctx->subs_h = subs;
  ctx->dec = d;
  ctx->dec.lon_cuts = ctx->dec.lat_cuts = ctx->dec.t_cuts = nullptr;
  ctx->dec.cluster = cl;
  by_precision(ctx, [&](auto t) {
    using T = decltype(t);
    background_pass<T>(ctx, true);
    return 0;
  });
  // keep the l = 0 exchange state for dd4dv_reset_exchange if it leaves the
  // same reserve as the stage buffer free; otherwise a reset reruns the
  // background forecast
  {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double need = (double)(ctx->gtraj + ctx->traj_elems) * ctx->tsize;
    if (need + 4.0 * (1ull << 30) + 0.05 * (double)total_b <= (double)free_b) {
      ctx->bnd0 = dalloc<unsigned char>(ctx, ctx->gtraj * ctx->tsize, &L);
      ctx->tgt0 = dalloc<unsigned char>(ctx, ctx->traj_elems * ctx->tsize, &L);
      CK(cudaMemcpyAsync(ctx->bnd0, ctx->bnd, ctx->gtraj * ctx->tsize, cudaMemcpyDeviceToDevice, ctx->st));
      CK(cudaMemcpyAsync(ctx->tgt0, ctx->tgt, ctx->traj_elems * ctx->tsize, cudaMemcpyDeviceToDevice, ctx->st));
    }
  }
  CK(cudaMemsetAsync(ctx->vconst, 0, n_sub * sizeof(double), ctx->st));
  ctx->fwd_pending = false;
  sync(ctx);
  ctx->has_dec = true;
  if (d.cluster < 0) autotune(ctx);
  if (d.ckpt_k == -2) tune_checkpoint(ctx);
}

}  // namespace

dd4dv_ctx::~dd4dv_ctx() {
  free_dec();
  cudaFree(rows_d);
  cudaFree(xb0);
  cudaFree(gscratch);
  cudaFree(gchunk);
  cudaFree(sigma_d);
  cudaFree(counter_d);
  cudaFree(scal_d);
  cudaFree(err_d);
  cudaFreeHost(counter_h);
  cudaFreeHost(phase_h);
  cudaFreeHost(scal_h);
  cudaFree(ptraj_io);
  if (own_stream && st) cudaStreamDestroy(st);
}

void dd4dv_ctx::drop_graphs() {
  for (cudaGraphExec_t* g : {&og.start, &og.dir, &og.trial, &og.exch, &og.fin})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  og.valid = false;
}

void dd4dv_ctx::free_dec() {
  if (st) cudaStreamSynchronize(st);
  drop_graphs();
  cudaFreeHost(lbst_h);
  lbst_h = nullptr;
  for (void* p : dec_allocs) cudaFree(p);
  dec_allocs.clear();
  cudaFreeHost(phase_h);
  phase_h = nullptr;
  cudaFree(ptraj_io);
  ptraj_io = nullptr;
  has_dec = false;
}

extern "C" {

dd4dv_status dd4dv_create(const dd4dv_model* model, void* cuda_stream, dd4dv_ctx** out) {
  g_create_error.clear();
  if (!model || !out) {
    g_create_error = "NULL argument";
    return DD4DV_EINVAL;
  }
  *out = nullptr;
  dd4dv_ctx* ctx = nullptr;
  try {
    const dd4dv_model& m = *model;
    if (m.nlon < 3 || m.nlat < 2 || !(m.dt > 0.0) || m.nsteps < 0 || !(m.radius > 0.0) ||
        !(m.gravity > 0.0) || !(m.lat_max_deg > m.lat_min_deg) || m.lat_min_deg <= -90.0 ||
        m.lat_max_deg >= 90.0 || (m.precision != 0 && m.precision != 1) || !std::isfinite(m.omega) ||
        !std::isfinite(m.h_ref)) {
      g_create_error = "invalid model parameters";
      return DD4DV_EINVAL;
    }
    ctx = new dd4dv_ctx();
    ctx->m = m;
    if (cuda_stream) {
      ctx->st = static_cast<cudaStream_t>(cuda_stream);
    } else {
      cudaError_t e = cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
        delete ctx;
        return DD4DV_ECUDA;
      }
      ctx->own_stream = true;
    }
    // row constants (Sec. 7): theta_j at cell centres between the walls
    const double pi = 3.14159265358979323846;
    const double dlam = 2.0 * pi / m.nlon;
    const double dth = (m.lat_max_deg - m.lat_min_deg) * pi / 180.0 / m.nlat;
    const double th0 = m.lat_min_deg * pi / 180.0;
    ctx->Bth = 1.0 / (2.0 * m.radius * dth);
    ctx->gBth = m.gravity * ctx->Bth;
    ctx->rows_h.resize(m.nlat);
    for (int j = 0; j < m.nlat; ++j) {
      const double th = th0 + (j + 0.5) * dth;
      RowConst r;
      r.c = std::cos(th);
      r.A = 1.0 / (2.0 * m.radius * r.c * dlam);
      r.f = 2.0 * m.omega * std::sin(th);
      r.tau = std::tan(th) / m.radius;
      r.BinvC = ctx->Bth / r.c;
      r.gA = m.gravity * r.A;
      ctx->rows_h[j] = r;
    }
    ctx->gstate = 3ULL * m.nlat * m.nlon;
    ctx->gtraj = (size_t)(m.nsteps + 1) * ctx->gstate;
    ctx->rows_d = dalloc<RowConst>(ctx, m.nlat);
    ctx->xb0 = dalloc<double>(ctx, ctx->gstate);
    ctx->gscratch = dalloc<double>(ctx, 3 * ctx->gstate);
    // chunk of global levels: at most 512 MB, at least 2 levels, at most the whole trajectory
    const size_t lv_bytes = ctx->gstate * sizeof(double);
    ctx->gchunk_lv = (int)std::max<size_t>(2, std::min<size_t>({(size_t)m.nsteps + 1, (512u << 20) / lv_bytes, 4096}));
    if (const char* e = std::getenv("DD4DV_GLOBAL_CHUNK_LEVELS")) {   // override (tests of the chunking)
      const int k = std::atoi(e);
      if (k >= 2 && k <= 4096) ctx->gchunk_lv = k;
    }
    ctx->gchunk = dalloc<double>(ctx, (size_t)ctx->gchunk_lv * ctx->gstate);
    ctx->sigma_d = dalloc<double>(ctx, 3);
    ctx->counter_d = dalloc<int>(ctx, 4);
    ctx->scal_d = dalloc<double>(ctx, 8);
    ctx->err_d = dalloc<int>(ctx, 1);
    if (cudaMallocHost(&ctx->counter_h, 4 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->scal_h, 8 * sizeof(double)) != cudaSuccess)
      fail(ctx, DD4DV_ENOMEM, "pinned host allocation failed");
    CK(cudaMemcpyAsync(ctx->rows_d, ctx->rows_h.data(), m.nlat * sizeof(RowConst),
                       cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(ctx->err_d, 0, sizeof(int), ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *out = ctx;
    return DD4DV_OK;
  } catch (const Fail& f) {
    if (ctx) {
      g_create_error = ctx->err;
      delete ctx;
    }
    return f.st;
  } catch (...) {
    delete ctx;
    g_create_error = "allocation failed";
    return DD4DV_ENOMEM;
  }
}

dd4dv_status dd4dv_destroy(dd4dv_ctx* ctx) {
  delete ctx;
  return DD4DV_OK;
}

const char* dd4dv_last_error(const dd4dv_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

dd4dv_status dd4dv_set_background(dd4dv_ctx* ctx, const double* xb0) {
  return guard(ctx, [&] {
    if (!xb0) fail(ctx, DD4DV_EINVAL, "xb0 is NULL");
    if (!all_finite(xb0, ctx->gstate)) fail(ctx, DD4DV_ENONFINITE, "background contains NaN or Inf");
    ctx->free_dec();
    h2d(ctx, ctx->xb0, xb0, ctx->gstate * sizeof(double));
    sync(ctx);
    ctx->has_bg = true;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_set_background_error(dd4dv_ctx* ctx, const double sigma_b[3], double corr_len,
                                        int rf_passes) {
  return guard(ctx, [&] {
    if (!sigma_b) fail(ctx, DD4DV_EINVAL, "sigma_b is NULL");
    for (int v = 0; v < 3; ++v)
      if (!(sigma_b[v] > 0.0) || !std::isfinite(sigma_b[v])) fail(ctx, DD4DV_EINVAL, "sigma_b must be > 0");
    if (!(corr_len >= 0.0) || !std::isfinite(corr_len)) fail(ctx, DD4DV_EINVAL, "corr_len must be >= 0");
    if (corr_len > 0.0 && (rf_passes < 1 || rf_passes > 8)) fail(ctx, DD4DV_EINVAL, "rf_passes must be 1..8");
    ctx->free_dec();
    for (int v = 0; v < 3; ++v) ctx->sigma_b[v] = sigma_b[v];
    ctx->corr_len = corr_len;
    ctx->rf_passes = rf_passes;
    if (corr_len > 0.0) rf_coeffs(corr_len, rf_passes, &ctx->rf_alpha, &ctx->rf_c);
    h2d(ctx, ctx->sigma_d, ctx->sigma_b, 3 * sizeof(double));
    sync(ctx);
    ctx->has_berr = true;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_set_observations(dd4dv_ctx* ctx, long long n, const int* level, const int* var,
                                    const double* fi, const double* fj, const double* value,
                                    const double* sigma_o) {
  return guard(ctx, [&] {
    if (n < 0) fail(ctx, DD4DV_EINVAL, "n < 0");
    if (n > 0 && (!level || !var || !fi || !fj || !value || !sigma_o)) fail(ctx, DD4DV_EINVAL, "NULL array");
    const int nlon = ctx->m.nlon, nlat = ctx->m.nlat;
    for (long long k = 0; k < n; ++k) {
      if (level[k] < 0 || level[k] > ctx->m.nsteps) fail(ctx, DD4DV_EINVAL, "obs %lld: level out of range", k);
      if (var[k] < 0 || var[k] > 2) fail(ctx, DD4DV_EINVAL, "obs %lld: var out of range", k);
      if (!std::isfinite(fi[k]) || !std::isfinite(fj[k]) || !std::isfinite(value[k]) || !std::isfinite(sigma_o[k]))
        fail(ctx, DD4DV_ENONFINITE, "obs %lld: NaN or Inf", k);
      if (!(fi[k] >= 0.0 && fi[k] < nlon)) fail(ctx, DD4DV_EINVAL, "obs %lld: fi out of [0, nlon)", k);
      if (!(fj[k] >= 0.0 && fj[k] <= nlat - 1)) fail(ctx, DD4DV_EINVAL, "obs %lld: fj out of [0, nlat-1]", k);
      if (!(sigma_o[k] > 0.0)) fail(ctx, DD4DV_EINVAL, "obs %lld: sigma_o must be > 0", k);
    }
    ctx->free_dec();
    ctx->ob_level.assign(level, level + n);
    ctx->ob_var.assign(var, var + n);
    ctx->ob_fi.assign(fi, fi + n);
    ctx->ob_fj.assign(fj, fj + n);
    ctx->ob_val.assign(value, value + n);
    ctx->ob_so.assign(sigma_o, sigma_o + n);
    ctx->has_obs = true;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_set_decomposition(dd4dv_ctx* ctx, const dd4dv_decomp* dec) {
  return guard(ctx, [&] {
    if (!dec) fail(ctx, DD4DV_EINVAL, "dec is NULL");
    if (!ctx->has_bg || !ctx->has_berr || !ctx->has_obs)
      fail(ctx, DD4DV_ESTATE, "set_background, set_background_error and set_observations must come first");
    build_decomposition(ctx, *dec);
    if (cudaMallocHost(&ctx->phase_h, ctx->n_sub * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->lbst_h, ctx->n_sub * sizeof(LbState)) != cudaSuccess)
      fail(ctx, DD4DV_ENOMEM, "pinned host allocation failed");
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_num_subdomains(const dd4dv_ctx* cctx, int* n) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!n) fail(ctx, DD4DV_EINVAL, "n is NULL");
    *n = ctx->n_sub;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_control_layout(const dd4dv_ctx* cctx, long long* offsets, int* boxes) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!offsets) fail(ctx, DD4DV_EINVAL, "offsets is NULL");
    for (int s = 0; s < ctx->n_sub; ++s) {
      const SubDesc& d = ctx->subs_h[s];
      offsets[s] = d.ctrl_off;
      if (boxes) {
        boxes[6 * s + 0] = d.i0; boxes[6 * s + 1] = d.nx; boxes[6 * s + 2] = d.j0;
        boxes[6 * s + 3] = d.ny; boxes[6 * s + 4] = d.a; boxes[6 * s + 5] = d.b;
      }
    }
    offsets[ctx->n_sub] = ctx->ctrl_total;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_traj_layout(const dd4dv_ctx* cctx, long long* offsets) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!offsets) fail(ctx, DD4DV_EINVAL, "offsets is NULL");
    for (int s = 0; s < ctx->n_sub; ++s) offsets[s] = ctx->subs_h[s].ptraj_off;
    offsets[ctx->n_sub] = ctx->ptraj_total;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_eval(dd4dv_ctx* ctx, const double* w_all, double* J_all, double* grad_all,
                        double* parts, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !J_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t C = ctx->ctrl_total;
    const double* w = stage_in(ctx, w_all, ctx->io_a, C, device_ptrs);
    double* J = device_ptrs ? J_all : ctx->io_p;
    double* pa = device_ptrs ? parts : (parts ? ctx->io_p + ctx->n_sub : nullptr);
    double* gr = grad_all ? (device_ptrs ? grad_all : ctx->io_b) : nullptr;
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      eval_T<T>(ctx, w, J, gr, pa, own_mask(ctx), 1, nullptr);
      return 0;
    });
    ctx->fwd_pending = false;
    if (!device_ptrs) {
      d2h(ctx, J_all, J, ctx->n_sub * sizeof(double));
      if (parts) d2h(ctx, parts, pa, 3 * ctx->n_sub * sizeof(double));
      if (grad_all) d2h(ctx, grad_all, gr, C * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_eval_forward(dd4dv_ctx* ctx, const double* w_all, double* J_all, double* parts,
                                int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !J_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t C = ctx->ctrl_total;
    // keep w for the backward pass in io_c
    if (device_ptrs) CK(cudaMemcpyAsync(ctx->io_c, w_all, C * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    else h2d(ctx, ctx->io_c, w_all, C * sizeof(double));
    double* J = device_ptrs ? J_all : ctx->io_p;
    double* pa = device_ptrs ? parts : (parts ? ctx->io_p + ctx->n_sub : nullptr);
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      init_states<T>(ctx, ctx->io_c, ctx->vw, own_mask(ctx), 1);
      forward_sweep<T>(ctx, own_mask(ctx), 1);
      KL(launch_finalize_J(ctx->subs_d, ctx->n_sub, ctx->io_c, ctx->part, ctx->cl_f, ctx->vconst,
                           ctx->dec.lambda, ctx->dec.mu, J, pa, own_mask(ctx), 1, ctx->st));
      return 0;
    });
    ctx->fwd_pending = true;
    if (!device_ptrs) {
      d2h(ctx, J_all, J, ctx->n_sub * sizeof(double));
      if (parts) d2h(ctx, parts, pa, 3 * ctx->n_sub * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_eval_backward(dd4dv_ctx* ctx, const double* scale, double* grad_all, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!ctx->fwd_pending) fail(ctx, DD4DV_ESTATE, "no pending dd4dv_eval_forward");
    if (!grad_all) fail(ctx, DD4DV_EINVAL, "grad_all is NULL");
    const double* sc = nullptr;
    if (scale) sc = stage_in(ctx, scale, ctx->io_p + 4 * ctx->n_sub, ctx->n_sub, device_ptrs);
    double* gr = device_ptrs ? grad_all : ctx->io_b;
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      SweepArgs<T> a = sweep_args<T>(ctx);
      a.active = own_mask(ctx);
      a.active_value = 1;
      KL(launch_adjoint<T>(a, ctx->cl, ctx->nthreads, ctx->st));
      apply_VT(ctx, ctx->lam_a, ctx->io_c, sc, gr, own_mask(ctx), 1);
      return 0;
    });
    ctx->fwd_pending = false;
    if (!device_ptrs) {
      d2h(ctx, grad_all, gr, ctx->ctrl_total * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

static double* ptraj_buf(dd4dv_ctx* ctx) {
  if (!ctx->ptraj_io) ctx->ptraj_io = dalloc<double>(ctx, ctx->ptraj_total);
  return ctx->ptraj_io;
}

dd4dv_status dd4dv_tlm(dd4dv_ctx* ctx, const double* w_all, const double* dw_all, double* dx_all,
                       int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !dw_all || !dx_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    int tl_cl = 0, tl_R = 0;
    tlm_shape(ctx, &tl_cl, &tl_R);
    const size_t C = ctx->ctrl_total;
    const double* w = stage_in(ctx, w_all, ctx->io_a, C, device_ptrs);
    const double* dw = stage_in(ctx, dw_all, ctx->io_b, C, device_ptrs);
    double* out = device_ptrs ? dx_all : ptraj_buf(ctx);
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      init_states<T>(ctx, w, ctx->vw, nullptr, 0);
      apply_V(ctx, dw, ctx->io_c, nullptr, 0);   // dx(a) = V dw
      SweepArgs<T> a = sweep_args<T>(ctx);
      a.dx0 = ctx->io_c;
      a.dx_out = out;
      a.R = tl_R;
      KL(launch_tlm<T>(a, tl_cl, ctx->nthreads, ctx->st));
      return 0;
    });
    ctx->fwd_pending = false;
    if (!device_ptrs) {
      d2h(ctx, dx_all, out, ctx->ptraj_total * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_adjoint(dd4dv_ctx* ctx, const double* w_all, const double* y_all, double* dw_all,
                           int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !y_all || !dw_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t C = ctx->ctrl_total;
    const double* w = stage_in(ctx, w_all, ctx->io_a, C, device_ptrs);
    const double* y = device_ptrs ? y_all : nullptr;
    if (!device_ptrs) {
      double* b = ptraj_buf(ctx);
      h2d(ctx, b, y_all, ctx->ptraj_total * sizeof(double));
      y = b;
    }
    double* out = device_ptrs ? dw_all : ctx->io_b;
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      init_states<T>(ctx, w, ctx->vw, nullptr, 0);
      forward_sweep<T>(ctx, nullptr, 0);
      SweepArgs<T> a = sweep_args<T>(ctx);
      a.yforce = y;
      KL(launch_adjoint<T>(a, ctx->cl, ctx->nthreads, ctx->st));
      apply_VT(ctx, ctx->lam_a, nullptr, nullptr, out, nullptr, 0);
      return 0;
    });
    ctx->fwd_pending = false;
    if (!device_ptrs) {
      d2h(ctx, dw_all, out, C * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_gn_hessvec(dd4dv_ctx* ctx, const double* w_all, const double* p_all, double* Ap_all,
                              int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !p_all || !Ap_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    ensure_gn(ctx);
    const size_t C = ctx->ctrl_total;
    const double* w = stage_in(ctx, w_all, ctx->io_a, C, device_ptrs);
    const double* pv = stage_in(ctx, p_all, ctx->io_b, C, device_ptrs);
    double* out = device_ptrs ? Ap_all : ctx->cg_Ap;
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      init_states<T>(ctx, w, ctx->vw, nullptr, 0);
      forward_sweep<T>(ctx, nullptr, 0);   // linearisation trajectory
      gn_product_T<T>(ctx, pv, out, nullptr, 0);
      return 0;
    });
    ctx->fwd_pending = false;
    if (!device_ptrs) {
      d2h(ctx, Ap_all, out, C * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_trajectories(dd4dv_ctx* ctx, const double* w_all, double* traj_all, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !traj_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const double* w = stage_in(ctx, w_all, ctx->io_a, ctx->ctrl_total, device_ptrs);
    double* out = device_ptrs ? traj_all : ptraj_buf(ctx);
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      init_states<T>(ctx, w, ctx->vw, nullptr, 0);
      forward_sweep<T>(ctx, nullptr, 0, true);
      KL(launch_export_traj<T>(ctx->subs_d, ctx->n_sub, static_cast<const T*>(ctx->traj), h_ref_of(ctx),
                               out, ctx->max_pts, ctx->max_levels, ctx->st));
      return 0;
    });
    ctx->fwd_pending = false;
    if (!device_ptrs) {
      d2h(ctx, traj_all, out, ctx->ptraj_total * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_exchange(dd4dv_ctx* ctx, const double* w_all, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const double* w = stage_in(ctx, w_all, ctx->io_a, ctx->ctrl_total, device_ptrs);
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      exchange_T<T>(ctx, w);
      return 0;
    });
    if (!device_ptrs) sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_reset_exchange(dd4dv_ctx* ctx) {
  return guard(ctx, [&] {
    require_dec(ctx);
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      reset_exchange_T<T>(ctx);
      return 0;
    });
    sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_boundary_trajectory(dd4dv_ctx* ctx, double* traj, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!traj) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t G = ctx->gstate;
    const int levels = ctx->m.nsteps + 1;
    const int chunk = device_ptrs ? levels : ctx->gchunk_lv;   // host output: through the chunk buffer
    for (int g0 = 0; g0 < levels; g0 += chunk) {
      const int nl = std::min(chunk, levels - g0);
      double* out = device_ptrs ? traj : ctx->gchunk;
      by_precision(ctx, [&](auto t) {
        using T = decltype(t);
        KL(launch_bnd_to_global<T>(static_cast<const T*>(ctx->bnd) + (size_t)g0 * G, (long long)nl * G,
                                   h_ref_of(ctx), ctx->m.nlon, ctx->m.nlat, out, ctx->st));
        return 0;
      });
      if (!device_ptrs) d2h(ctx, traj + (size_t)g0 * G, out, (size_t)nl * G * sizeof(double));
    }
    if (!device_ptrs) sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_analysis(dd4dv_ctx* ctx, double* xa0, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!xa0) fail(ctx, DD4DV_EINVAL, "NULL argument");
    double* out = device_ptrs ? xa0 : ctx->gscratch + 2 * ctx->gstate;
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      KL(launch_bnd_to_global<T>(static_cast<const T*>(ctx->bnd), (long long)ctx->gstate, h_ref_of(ctx),
                                 ctx->m.nlon, ctx->m.nlat, out, ctx->st));
      return 0;
    });
    if (!device_ptrs) {
      d2h(ctx, xa0, out, ctx->gstate * sizeof(double));
      sync(ctx);
    }
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_forward(dd4dv_ctx* ctx, const double* x0, double* traj, int device_ptrs) {
  return guard(ctx, [&] {
    if (!x0 || !traj) fail(ctx, DD4DV_EINVAL, "NULL argument");
    if (device_ptrs) {
      global_run(ctx, x0, traj);
      return DD4DV_OK;
    }
    if (!all_finite(x0, ctx->gstate)) fail(ctx, DD4DV_ENONFINITE, "x0 contains NaN or Inf");
    const size_t G = ctx->gstate;
    double* in = ctx->gscratch + 2 * G;
    h2d(ctx, in, x0, G * sizeof(double));
    global_run_chunked(ctx, in, [&](int g0, int g1, const double* lv) {
      d2h(ctx, traj + (size_t)g0 * G, lv, (size_t)(g1 - g0 + 1) * G * sizeof(double));
    });
    sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_observe(dd4dv_ctx* ctx, const double* traj, long long n, const int* level,
                           const int* var, const double* fi, const double* fj, double* out,
                           int device_ptrs) {
  return guard(ctx, [&] {
    if (n < 0) fail(ctx, DD4DV_EINVAL, "n < 0");
    if (n == 0) return DD4DV_OK;
    if (!traj || !level || !var || !fi || !fj || !out) fail(ctx, DD4DV_EINVAL, "NULL argument");
    if (device_ptrs) {
      KL(launch_observe(traj, 0, ctx->m.nsteps, n, level, var, fi, fj, ctx->m.nlon, ctx->m.nlat, out, ctx->st));
      return DD4DV_OK;
    }
    for (long long k = 0; k < n; ++k) {
      if (level[k] < 0 || level[k] > ctx->m.nsteps || var[k] < 0 || var[k] > 2 || !(fi[k] >= 0.0) ||
          !(fi[k] < ctx->m.nlon) || !(fj[k] >= 0.0) || !(fj[k] <= ctx->m.nlat - 1))
        fail(ctx, DD4DV_EINVAL, "observation site %lld out of range", k);
    }
    std::vector<void*> tmp;
    try {
      int* dl = dalloc<int>(ctx, n, &tmp);
      int* dv = dalloc<int>(ctx, n, &tmp);
      double* dfi = dalloc<double>(ctx, n, &tmp);
      double* dfj = dalloc<double>(ctx, n, &tmp);
      double* dout = dalloc<double>(ctx, n, &tmp);
      h2d(ctx, dl, level, n * sizeof(int));
      h2d(ctx, dv, var, n * sizeof(int));
      h2d(ctx, dfi, fi, n * sizeof(double));
      h2d(ctx, dfj, fj, n * sizeof(double));
      // the trajectory goes up a chunk of levels at a time
      const size_t G = ctx->gstate;
      const int levels = ctx->m.nsteps + 1;
      for (int g0 = 0; g0 < levels; g0 += ctx->gchunk_lv) {
        const int nl = std::min(ctx->gchunk_lv, levels - g0);
        h2d(ctx, ctx->gchunk, traj + (size_t)g0 * G, (size_t)nl * G * sizeof(double));
        KL(launch_observe(ctx->gchunk, g0, g0 + nl - 1, n, dl, dv, dfi, dfj, ctx->m.nlon, ctx->m.nlat, dout,
                          ctx->st));
      }
      d2h(ctx, out, dout, n * sizeof(double));
      sync(ctx);
    } catch (...) {
      for (void* p : tmp) cudaFree(p);
      throw;
    }
    for (void* p : tmp) cudaFree(p);
    return DD4DV_OK;
  });
}

static void check_solver(dd4dv_ctx* ctx, const dd4dv_solver* s) {
  if (!s) fail(ctx, DD4DV_EINVAL, "solver is NULL");
  if (s->lbfgs_m < 1 || s->lbfgs_m > 8) fail(ctx, DD4DV_EINVAL, "lbfgs_m must be 1..8");
  if (s->use_graphs != 0 && s->use_graphs != 1) fail(ctx, DD4DV_EINVAL, "use_graphs must be 0 or 1");
  if (s->max_local_iters < 0 || s->max_trials < 1 || s->max_outer < 0) fail(ctx, DD4DV_EINVAL, "bad iteration limits");
  if (!(s->c1 > 0.0 && s->c1 < 1.0)) fail(ctx, DD4DV_EINVAL, "c1 must be in (0,1)");
  if (!(s->gtol_rel >= 0.0) || !(s->eps_outer >= 0.0)) fail(ctx, DD4DV_EINVAL, "tolerances must be >= 0");
  if (s->local_solver != 0 && s->local_solver != 1) fail(ctx, DD4DV_EINVAL, "local_solver must be 0 or 1");
  if (s->local_solver == 1 && (s->gn_iters < 0 || s->cg_iters < 0 || !(s->cg_tol >= 0.0)))
    fail(ctx, DD4DV_EINVAL, "gn_iters, cg_iters and cg_tol must be >= 0");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The Turkel-Zwas scheme (Sec. 7, strides p, q, averaging weight alpha) on the
// undecomposed problem: global model runs, tangent-linear and adjoint runs,
// and the global 4D-Var functional with its gradient.  Kernels in tz.cu.
namespace {

TzArgs tz_args(dd4dv_ctx* ctx, int p, int q, double alpha) {
  const dd4dv_model& m = ctx->m;
  if (p < 1 || q < 1 || 2 * p >= m.nlon || q >= m.nlat || !(alpha >= 0.0 && alpha <= 1.0))
    fail(ctx, DD4DV_EINVAL, "Turkel-Zwas parameters need 1 <= p < nlon/2, 1 <= q < nlat, 0 <= alpha <= 1");
  TzArgs t;
  t.rows = ctx->rows_d;
  t.nlon = m.nlon;
  t.nlat = m.nlat;
  t.p = p;
  t.q = q;
  t.alpha = alpha;
  const double pi = 3.14159265358979323846;
  t.slon = 1.0 / (2.0 * m.radius * (2.0 * pi / m.nlon));
  t.slat = ctx->Bth;
  t.g = m.gravity;
  t.dt = m.dt;
  return t;
}

// Device scratch that lives for one call.
struct TzBufs {
  std::vector<void*> ptrs;
  dd4dv_ctx* ctx;
  explicit TzBufs(dd4dv_ctx* c) : ctx(c) {}
  double* get(size_t n) {
    double* p = dalloc<double>(ctx, n);
    ptrs.push_back(p);
    return p;
  }
  ~TzBufs() {
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    for (void* p : ptrs) cudaFree(p);
  }
};

void tz_step(dd4dv_ctx* ctx, const TzArgs& t, const double* x, double* s1, double* s2, double* nx) {
  KL(launch_tz_stage(t, x, x, s1, 0.0, 1.0, ctx->st));
  KL(launch_tz_stage(t, x, s1, s2, 0.75, 0.25, ctx->st));
  KL(launch_tz_stage(t, x, s2, nx, 1.0 / 3.0, 2.0 / 3.0, ctx->st));
}

void tz_run(dd4dv_ctx* ctx, const TzArgs& t, const double* x0, double* traj, double* s1, double* s2) {
  const size_t G = ctx->gstate;
  CK(cudaMemcpyAsync(traj, x0, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  for (int n = 0; n < ctx->m.nsteps; ++n) tz_step(ctx, t, traj + (size_t)n * G, s1, s2, traj + (size_t)(n + 1) * G);
}

// lam <- M_n^T lam for the step from x = x(n): the stage states recomputed,
// then mu2 = lam + dt F'(x2)^T lam, mu1 = mu2 + dt F'(x1)^T mu2,
// lam(n) = lam/3 + mu2/2 + (mu1 + dt F'(x)^T mu1)/6 (the transposed SSP-RK3
// step, as in the box sweeps).
void tz_adjoint_step(dd4dv_ctx* ctx, const TzArgs& t, const double* x, double* s1, double* s2, double* lam,
                     double* mu2, double* mu1, double* g3) {
  const size_t G = ctx->gstate;
  KL(launch_tz_stage(t, x, x, s1, 0.0, 1.0, ctx->st));
  KL(launch_tz_stage(t, x, s1, s2, 0.75, 0.25, ctx->st));
  CK(cudaMemcpyAsync(mu2, lam, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  KL(launch_tz_adj_scatter(t, s2, lam, mu2, t.dt, ctx->st));
  CK(cudaMemcpyAsync(mu1, mu2, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  KL(launch_tz_adj_scatter(t, s1, mu2, mu1, t.dt, ctx->st));
  CK(cudaMemcpyAsync(g3, mu1, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  KL(launch_tz_adj_scatter(t, x, mu1, g3, t.dt, ctx->st));
  KL(launch_tz_lincomb(lam, lam, mu2, g3, 1.0 / 3.0, 0.5, 1.0 / 6.0, (long long)G, ctx->st));
}

const double* tz_in(dd4dv_ctx* ctx, TzBufs& b, const double* src, size_t n, int device_ptrs) {
  if (device_ptrs) return src;
  double* d = b.get(n);
  h2d(ctx, d, src, n * sizeof(double));
  return d;
}

}  // namespace

extern "C" {

dd4dv_status dd4dv_tz_forward(dd4dv_ctx* ctx, int p, int q, double alpha, const double* x0, double* traj,
                              int device_ptrs) {
  return guard(ctx, [&] {
    const TzArgs t = tz_args(ctx, p, q, alpha);
    if (!x0 || !traj) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t G = ctx->gstate, T = (size_t)(ctx->m.nsteps + 1) * G;
    TzBufs b(ctx);
    const double* x = tz_in(ctx, b, x0, G, device_ptrs);
    double* out = device_ptrs ? traj : b.get(T);
    double* s = b.get(2 * G);
    tz_run(ctx, t, x, out, s, s + G);
    if (!device_ptrs) d2h(ctx, traj, out, T * sizeof(double));
    sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_tz_tlm(dd4dv_ctx* ctx, int p, int q, double alpha, const double* x0, const double* dx0,
                          double* dtraj, int device_ptrs) {
  return guard(ctx, [&] {
    const TzArgs t = tz_args(ctx, p, q, alpha);
    if (!x0 || !dx0 || !dtraj) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t G = ctx->gstate, T = (size_t)(ctx->m.nsteps + 1) * G;
    TzBufs b(ctx);
    const double* xin = tz_in(ctx, b, x0, G, device_ptrs);
    const double* dxin = tz_in(ctx, b, dx0, G, device_ptrs);
    double* dout = device_ptrs ? dtraj : b.get(T);
    double* w = b.get(6 * G);
    double *xa = w, *xb = w + G, *s1 = w + 2 * G, *s2 = w + 3 * G, *d1 = w + 4 * G, *d2 = w + 5 * G;
    CK(cudaMemcpyAsync(xa, xin, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(dout, dxin, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    for (int n = 0; n < ctx->m.nsteps; ++n) {
      const double* dx = dout + (size_t)n * G;
      double* dn = dout + (size_t)(n + 1) * G;
      KL(launch_tz_stage(t, xa, xa, s1, 0.0, 1.0, ctx->st));
      KL(launch_tz_tl_stage(t, xa, dx, dx, d1, 0.0, 1.0, ctx->st));
      KL(launch_tz_stage(t, xa, s1, s2, 0.75, 0.25, ctx->st));
      KL(launch_tz_tl_stage(t, s1, dx, d1, d2, 0.75, 0.25, ctx->st));
      KL(launch_tz_stage(t, xa, s2, xb, 1.0 / 3.0, 2.0 / 3.0, ctx->st));
      KL(launch_tz_tl_stage(t, s2, dx, d2, dn, 1.0 / 3.0, 2.0 / 3.0, ctx->st));
      std::swap(xa, xb);
    }
    if (!device_ptrs) d2h(ctx, dtraj, dout, T * sizeof(double));
    sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_tz_adjoint(dd4dv_ctx* ctx, int p, int q, double alpha, const double* x0, const double* ytraj,
                              double* dx0, int device_ptrs) {
  return guard(ctx, [&] {
    const TzArgs t = tz_args(ctx, p, q, alpha);
    if (!x0 || !ytraj || !dx0) fail(ctx, DD4DV_EINVAL, "NULL argument");
    const size_t G = ctx->gstate, T = (size_t)(ctx->m.nsteps + 1) * G;
    const int N = ctx->m.nsteps;
    TzBufs b(ctx);
    const double* xin = tz_in(ctx, b, x0, G, device_ptrs);
    const double* y = tz_in(ctx, b, ytraj, T, device_ptrs);
    double* traj = b.get(T);
    double* w = b.get(6 * G);
    double *s1 = w, *s2 = w + G, *lam = w + 2 * G, *mu2 = w + 3 * G, *mu1 = w + 4 * G, *g3 = w + 5 * G;
    tz_run(ctx, t, xin, traj, s1, s2);
    CK(cudaMemcpyAsync(lam, y + (size_t)N * G, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    for (int n = N - 1; n >= 0; --n) {
      tz_adjoint_step(ctx, t, traj + (size_t)n * G, s1, s2, lam, mu2, mu1, g3);
      KL(launch_tz_lincomb(lam, lam, y + (size_t)n * G, nullptr, 1.0, 1.0, 0.0, (long long)G, ctx->st));
    }
    if (device_ptrs) CK(cudaMemcpyAsync(dx0, lam, G * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    else d2h(ctx, dx0, lam, G * sizeof(double));
    sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_tz_eval(dd4dv_ctx* ctx, int p, int q, double alpha, const double* w_in, double* J_out,
                           double* grad_out, int device_ptrs) {
  return guard(ctx, [&] {
    const TzArgs t = tz_args(ctx, p, q, alpha);
    if (!w_in || !J_out) fail(ctx, DD4DV_EINVAL, "NULL argument");
    if (!ctx->has_bg || !ctx->has_berr) fail(ctx, DD4DV_ESTATE, "set_background and set_background_error first");
    if (ctx->corr_len > 0.0) fail(ctx, DD4DV_EINVAL, "dd4dv_tz_eval takes a diagonal B (corr_len_cells = 0)");
    const size_t G = ctx->gstate, T = (size_t)(ctx->m.nsteps + 1) * G;
    const int N = ctx->m.nsteps;
    const long long plane = (long long)ctx->m.nlat * ctx->m.nlon;
    TzBufs b(ctx);
    const double* w = tz_in(ctx, b, w_in, G, device_ptrs);
    double* traj = b.get(T);
    double* work = b.get(7 * G + 2);
    double *s1 = work, *s2 = work + G, *lam = work + 2 * G, *mu2 = work + 3 * G, *mu1 = work + 4 * G,
           *g3 = work + 5 * G, *x0 = work + 6 * G, *Jd = work + 7 * G, *Jo = work + 7 * G + 1;
    KL(launch_tz_scale_add(x0, ctx->xb0, w, ctx->sigma_d, plane, ctx->st));
    tz_run(ctx, t, x0, traj, s1, s2);
    // observations sorted by level, with the offsets of each level
    const size_t nob = ctx->has_obs ? ctx->ob_level.size() : 0;
    std::vector<size_t> ord(nob);
    for (size_t k = 0; k < nob; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t c) { return ctx->ob_level[a] < ctx->ob_level[c]; });
    std::vector<int> lv(nob), vr(nob);
    std::vector<double> fi(nob), fj(nob), yv(nob), so(nob);
    std::vector<long long> off(N + 2, 0);
    for (size_t k = 0; k < nob; ++k) {
      const size_t o = ord[k];
      lv[k] = ctx->ob_level[o];
      vr[k] = ctx->ob_var[o];
      fi[k] = ctx->ob_fi[o];
      fj[k] = ctx->ob_fj[o];
      yv[k] = ctx->ob_val[o];
      so[k] = ctx->ob_so[o];
      off[lv[k] + 1] += 1;
    }
    for (int n = 0; n <= N; ++n) off[n + 1] += off[n];
    const double* force = nullptr;
    const int* lvd = nullptr;
    const int* vrd = nullptr;
    const double *fid = nullptr, *fjd = nullptr;
    if (nob) {
      double* dbl = b.get(5 * nob);
      int* ints = reinterpret_cast<int*>(b.get(nob));   // 2 * nob ints
      h2d(ctx, ints, lv.data(), nob * sizeof(int));
      h2d(ctx, ints + nob, vr.data(), nob * sizeof(int));
      h2d(ctx, dbl, fi.data(), nob * sizeof(double));
      h2d(ctx, dbl + nob, fj.data(), nob * sizeof(double));
      h2d(ctx, dbl + 2 * nob, yv.data(), nob * sizeof(double));
      h2d(ctx, dbl + 3 * nob, so.data(), nob * sizeof(double));
      lvd = ints;
      vrd = ints + nob;
      fid = dbl;
      fjd = dbl + nob;
      force = dbl + 4 * nob;
      KL(launch_tz_obs_misfit(traj, (long long)nob, lvd, vrd, fid, fjd, dbl + 2 * nob, dbl + 3 * nob, ctx->m.nlon,
                              ctx->m.nlat, 1.0, dbl + 4 * nob, Jo, ctx->st));
    }
    KL(launch_tz_finish_J(w, (long long)G, nob ? Jo : nullptr, Jd, ctx->st));
    if (grad_out) {
      CK(cudaMemsetAsync(lam, 0, G * sizeof(double), ctx->st));
      if (nob) KL(launch_tz_obs_scatter(off[N], off[N + 1], vrd, fid, fjd, force, ctx->m.nlon, ctx->m.nlat, lam, ctx->st));
      for (int n = N - 1; n >= 0; --n) {
        tz_adjoint_step(ctx, t, traj + (size_t)n * G, s1, s2, lam, mu2, mu1, g3);
        if (nob) KL(launch_tz_obs_scatter(off[n], off[n + 1], vrd, fid, fjd, force, ctx->m.nlon, ctx->m.nlat, lam,
                                          ctx->st));
      }
      double* gd = device_ptrs ? grad_out : s1;
      KL(launch_tz_scale_add(gd, w, lam, ctx->sigma_d, plane, ctx->st));
      if (!device_ptrs) d2h(ctx, grad_out, gd, G * sizeof(double));
    }
    if (device_ptrs) CK(cudaMemcpyAsync(J_out, Jd, sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    else d2h(ctx, J_out, Jd, sizeof(double));
    sync(ctx);
    return DD4DV_OK;
  });
}

}  // extern "C"

// Captures the work enqueued by f on the context stream into an executable
// graph; *nk receives the number of this library's kernels in it.
template <typename F>
static cudaGraphExec_t capture_graph(dd4dv_ctx* ctx, F&& f, long long* nk) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
  const long long k0 = ctx->launches;
  try {
    f();
  } catch (...) {
    cudaStreamEndCapture(ctx->st, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  CK(cudaStreamEndCapture(ctx->st, &g));
  *nk = ctx->launches - k0;
  ctx->launches = k0;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) fail(ctx, DD4DV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  return ge;
}

// One outer iteration with the Gauss-Newton local solver: for each
// Gauss-Newton iteration, a batched J / grad J evaluation at w (which also
// stores the linearisation trajectory), CG on (I + G^T G) dw = -grad J with
// one batched Gauss-Newton product per CG iteration (masked to the
// subdomains still iterating), w += dw; a last evaluation for the
// statistics; then the Exchange.
template <typename T>
static void gn_outer_step_T(dd4dv_ctx* ctx, const dd4dv_solver& sv, dd4dv_stats* stats) {
  ensure_gn(ctx);
  CgArgs ca{};
  ca.subs = ctx->subs_d;
  ca.n_sub = ctx->n_sub;
  ca.g = ctx->g;
  ca.r = ctx->cg_r;
  ca.p = ctx->cg_p;
  ca.Ap = ctx->cg_Ap;
  ca.dw = ctx->cg_dw;
  ca.st = ctx->cgst;
  ca.phase = ctx->phase_d;
  ca.counter = ctx->counter_d;
  ca.max_iter = sv.cg_iters;
  ca.tol = sv.cg_tol;
  ca.gtol = sv.gtol_rel;
  std::vector<long long> sub_pts(ctx->n_sub);
  for (int s = 0; s < ctx->n_sub; ++s) {
    const SubDesc& d = ctx->subs_h[s];
    sub_pts[s] = (long long)d.nx * d.ny * (d.b - d.a);
  }
  long long evals = 0, sub_evals = 0, pts = 0;
  for (int it = 0;; ++it) {
    eval_T<T>(ctx, ctx->w, ctx->J, ctx->g, nullptr, nullptr, 0, nullptr);
    ++evals;
    sub_evals += ctx->n_sub;
    pts += ctx->pt_steps;
    const bool last = it >= sv.gn_iters;
    CgArgs c0 = ca;
    c0.first = it == 0;
    if (last) c0.max_iter = 0;   // norms for the statistics only
    KL(launch_cg_start(c0, ctx->st));
    if (last) break;
    d2h(ctx, ctx->counter_h, ctx->counter_d, sizeof(int));
    CK(cudaStreamSynchronize(ctx->st));
    if (ctx->counter_h[0] == 0) break;
    for (int k = 0; k < sv.cg_iters; ++k) {
      d2h(ctx, ctx->phase_h, ctx->phase_d, ctx->n_sub * sizeof(int));
      gn_product_T<T>(ctx, ctx->cg_p, ctx->cg_Ap, ctx->phase_d, 1);
      KL(launch_cg_step(ca, ctx->st));
      d2h(ctx, ctx->counter_h, ctx->counter_d, sizeof(int));
      CK(cudaStreamSynchronize(ctx->st));
      for (int s = 0; s < ctx->n_sub; ++s)
        if (ctx->phase_h[s] == 1) pts += sub_pts[s];
      if (ctx->counter_h[0] == 0) break;
    }
    KL(launch_axpy(ctx->w, ctx->cg_dw, ctx->ctrl_total, ctx->st));
  }
  exchange_T<T>(ctx, ctx->w);
  KL(launch_max_abs_diff(ctx->w, ctx->w_prev, ctx->ctrl_total, ctx->scal_d, ctx->st));
  CK(cudaMemcpyAsync(ctx->w_prev, ctx->w, ctx->ctrl_total * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
  d2h(ctx, ctx->scal_h, ctx->scal_d, sizeof(double));
  std::vector<double> J(ctx->n_sub);
  std::vector<CgState> cs(ctx->n_sub);
  d2h(ctx, J.data(), ctx->J, ctx->n_sub * sizeof(double));
  d2h(ctx, cs.data(), ctx->cgst, ctx->n_sub * sizeof(CgState));
  sync(ctx);
  if (stats) {
    stats->outer_iters += 1;
    stats->evals += evals;
    stats->sub_evals += sub_evals;
    stats->pt_steps += pts;
    stats->dw_inf = ctx->scal_h[0];
    double Js = 0.0, gmax = 0.0;
    for (int s = 0; s < ctx->n_sub; ++s) {
      Js += J[s];
      if (cs[s].g0n > 0.0) gmax = std::max(gmax, std::sqrt(cs[s].rr0) / cs[s].g0n);
    }
    stats->J_sum = Js;
    stats->gnorm_rel_max = gmax;
  }
}

// One outer iteration of Algorithm 1.  With L-BFGS the host loop only reads
// two counters per step (subdomains still in a line search / needing a
// direction); the device work of each step is one graph launch when
// sv.use_graphs is set.
template <typename T>
static void outer_step_T(dd4dv_ctx* ctx, const dd4dv_solver& sv, dd4dv_stats* stats, bool exchange = true) {
  if (sv.local_solver == 1) {
    gn_outer_step_T<T>(ctx, sv, stats);
    return;
  }
  LbArgs la{};
  la.subs = ctx->subs_d;
  la.n_sub = ctx->n_sub;
  la.w = ctx->w;
  la.g = ctx->g;
  la.wt = ctx->wt;
  la.gt = ctx->gt;
  la.p = ctx->p;
  la.S = ctx->S;
  la.Y = ctx->Y;
  la.rho = ctx->rho;
  la.total = ctx->ctrl_total;
  la.st = ctx->lbst;
  la.m = sv.lbfgs_m;
  la.max_iter = sv.max_local_iters;
  la.max_trials = sv.max_trials;
  la.gtol = sv.gtol_rel;
  la.c1 = sv.c1;
  la.counter = ctx->counter_d;
  la.phase = ctx->phase_d;
  la.owned = ctx->owned_d;

  auto q_start = [&] {   // evaluation at every owned local problem's start point
    eval_T<T>(ctx, ctx->w, ctx->J, ctx->g, nullptr, ctx->owned_d, 1, nullptr);
    LbArgs l2 = la;
    l2.J_eval = ctx->J;
    KL(launch_lb_start(l2, ctx->st));
  };
  auto q_dir = [&] {
    CK(cudaMemsetAsync(ctx->counter_d, 0, 2 * sizeof(int), ctx->st));
    LbArgs l2 = la;
    l2.J_eval = ctx->Jt;
    KL(launch_lb_direction(l2, ctx->st));
    d2h(ctx, ctx->counter_h, ctx->counter_d, 2 * sizeof(int));
  };
  auto q_trial = [&] {   // masked batched evaluation at the trial points + Armijo
    d2h(ctx, ctx->phase_h, ctx->phase_d, ctx->n_sub * sizeof(int));
    eval_T<T>(ctx, ctx->wt, ctx->Jt, ctx->gt, nullptr, ctx->phase_d, 1, nullptr);
    CK(cudaMemsetAsync(ctx->counter_d, 0, 2 * sizeof(int), ctx->st));
    LbArgs l2 = la;
    l2.J_eval = ctx->Jt;
    KL(launch_lb_linesearch(l2, ctx->st));
    d2h(ctx, ctx->counter_h, ctx->counter_d, 2 * sizeof(int));
  };
  auto q_fin = [&] {     // local solve only: the L-BFGS states for the statistics
    d2h(ctx, ctx->lbst_h, ctx->lbst, ctx->n_sub * sizeof(LbState));
  };
  auto q_exch = [&] {    // Exchange at the new local solutions, outer increment
    exchange_T<T>(ctx, ctx->w);
    KL(launch_max_abs_diff(ctx->w, ctx->w_prev, ctx->ctrl_total, ctx->scal_d, ctx->st));
    CK(cudaMemcpyAsync(ctx->w_prev, ctx->w, ctx->ctrl_total * sizeof(double), cudaMemcpyDeviceToDevice,
                       ctx->st));
    d2h(ctx, ctx->scal_h, ctx->scal_d, sizeof(double));
    d2h(ctx, ctx->lbst_h, ctx->lbst, ctx->n_sub * sizeof(LbState));
  };

  auto& og = ctx->og;
  const bool graphs = sv.use_graphs != 0;
  if (graphs && (!og.valid || std::memcmp(&og.key, &sv, sizeof(sv)) != 0)) {
    ctx->drop_graphs();
    og.start = capture_graph(ctx, q_start, &og.k_start);
    og.dir = capture_graph(ctx, q_dir, &og.k_dir);
    og.trial = capture_graph(ctx, q_trial, &og.k_trial);
    og.exch = capture_graph(ctx, q_exch, &og.k_exch);
    og.fin = capture_graph(ctx, q_fin, &og.k_fin);
    og.key = sv;
    og.valid = true;
  }
  auto run = [&](auto& q, cudaGraphExec_t ge, long long nk) {
    if (graphs) {
      CK(cudaGraphLaunch(ge, ctx->st));
      ctx->launches += nk;
    } else {
      q();
    }
  };

  long long evals = 0, sub_evals = 0, pts = 0;
  run(q_start, og.start, og.k_start);
  ++evals;
  std::vector<long long> sub_pts(ctx->n_sub);
  for (int s = 0; s < ctx->n_sub; ++s) {
    const SubDesc& d = ctx->subs_h[s];
    sub_pts[s] = (long long)d.nx * d.ny * (d.b - d.a);
    if (ctx->owned_h[s]) {
      ++sub_evals;
      pts += sub_pts[s];
    }
  }
  const int guard_iters = sv.max_local_iters + 2;
  for (int it = 0; it < guard_iters; ++it) {
    run(q_dir, og.dir, og.k_dir);
    CK(cudaStreamSynchronize(ctx->st));
    if (ctx->counter_h[0] == 0) break;
    for (int tr = 0; tr < sv.max_trials; ++tr) {
      run(q_trial, og.trial, og.k_trial);
      CK(cudaStreamSynchronize(ctx->st));
      ++evals;
      for (int s = 0; s < ctx->n_sub; ++s)
        if (ctx->phase_h[s] == 1) {
          ++sub_evals;
          pts += sub_pts[s];
        }
      if (ctx->counter_h[0] == 0) break;
    }
  }
  if (exchange) run(q_exch, og.exch, og.k_exch);
  else run(q_fin, og.fin, og.k_fin);
  sync(ctx);
  if (stats) {
    stats->outer_iters += exchange ? 1 : 0;
    stats->evals += evals;
    stats->sub_evals += sub_evals;
    stats->pt_steps += pts;
    if (exchange) stats->dw_inf = ctx->scal_h[0];
    double Js = 0.0, gmax = 0.0;
    int fails = 0;
    for (int s = 0; s < ctx->n_sub; ++s) {
      if (!ctx->owned_h[s]) continue;
      const LbState& l = ctx->lbst_h[s];
      Js += l.J;
      if (l.g0n > 0.0) gmax = std::max(gmax, l.gn / l.g0n);
      if (l.status == 3) ++fails;
    }
    stats->J_sum = Js;
    stats->gnorm_rel_max = gmax;
    stats->n_linesearch_fail += fails;
  }
}

extern "C" {

dd4dv_status dd4dv_set_owned(dd4dv_ctx* ctx, const int* owned) {
  return guard(ctx, [&] {
    require_dec(ctx);
    std::vector<int> m(ctx->n_sub, 1);
    if (owned)
      for (int s = 0; s < ctx->n_sub; ++s) {
        if (owned[s] != 0 && owned[s] != 1) fail(ctx, DD4DV_EINVAL, "owned[%d] must be 0 or 1", s);
        m[s] = owned[s];
      }
    h2d(ctx, ctx->owned_d, m.data(), ctx->n_sub * sizeof(int));
    sync(ctx);
    ctx->owned_h = m;
    ctx->owned_all = std::all_of(m.begin(), m.end(), [](int v) { return v == 1; });
    ctx->fwd_pending = false;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_local_solve(dd4dv_ctx* ctx, const dd4dv_solver* solver, dd4dv_stats* stats) {
  return guard(ctx, [&] {
    require_dec(ctx);
    check_solver(ctx, solver);
    if (solver->local_solver != 0) fail(ctx, DD4DV_EINVAL, "dd4dv_local_solve runs the L-BFGS local solver only");
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      outer_step_T<T>(ctx, *solver, stats, false);
      return 0;
    });
    ctx->fwd_pending = false;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_outer_step(dd4dv_ctx* ctx, const dd4dv_solver* solver, dd4dv_stats* stats) {
  return guard(ctx, [&] {
    require_dec(ctx);
    check_solver(ctx, solver);
    if (!ctx->owned_all)
      fail(ctx, DD4DV_ESTATE, "the context owns a subset of the subdomains: run dd4dv_local_solve, gather the "
                              "controls, dd4dv_set_controls and dd4dv_exchange instead");
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      outer_step_T<T>(ctx, *solver, stats);
      return 0;
    });
    ctx->fwd_pending = false;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_run(dd4dv_ctx* ctx, const dd4dv_solver* solver, double* xa0, dd4dv_stats* stats) {
  return guard(ctx, [&] {
    require_dec(ctx);
    check_solver(ctx, solver);
    if (!ctx->owned_all)
      fail(ctx, DD4DV_ESTATE, "the context owns a subset of the subdomains: drive the outer loop with "
                              "dd4dv_local_solve and dd4dv_exchange");
    dd4dv_stats local{};
    dd4dv_stats* stp = stats ? stats : &local;
    std::memset(stp, 0, sizeof(*stp));
    bool conv = false;
    for (int l = 0; l < solver->max_outer; ++l) {
      by_precision(ctx, [&](auto t) {
        using T = decltype(t);
        outer_step_T<T>(ctx, *solver, stp);
        return 0;
      });
      if (stp->dw_inf < solver->eps_outer) {
        conv = true;
        break;
      }
    }
    ctx->fwd_pending = false;
    if (xa0) {
      by_precision(ctx, [&](auto t) {
        using T = decltype(t);
        KL(launch_bnd_to_global<T>(static_cast<const T*>(ctx->bnd), (long long)ctx->gstate, h_ref_of(ctx),
                                   ctx->m.nlon, ctx->m.nlat, ctx->gscratch + 2 * ctx->gstate, ctx->st));
        return 0;
      });
      d2h(ctx, xa0, ctx->gscratch + 2 * ctx->gstate, ctx->gstate * sizeof(double));
      sync(ctx);
    }
    return conv ? DD4DV_OK : DD4DV_NOTCONV;
  });
}

dd4dv_status dd4dv_get_controls(dd4dv_ctx* ctx, double* w_all, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    CK(cudaMemcpyAsync(w_all, ctx->w, ctx->ctrl_total * sizeof(double),
                       device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->st));
    if (!device_ptrs) sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_set_controls(dd4dv_ctx* ctx, const double* w_all, int device_ptrs) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all) fail(ctx, DD4DV_EINVAL, "NULL argument");
    if (!device_ptrs && !all_finite(w_all, ctx->ctrl_total)) fail(ctx, DD4DV_ENONFINITE, "controls contain NaN or Inf");
    const auto kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ctx->w, w_all, ctx->ctrl_total * sizeof(double), kind, ctx->st));
    CK(cudaMemcpyAsync(ctx->w_prev, w_all, ctx->ctrl_total * sizeof(double), kind, ctx->st));
    sync(ctx);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_pt_steps(const dd4dv_ctx* cctx, long long* n) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!n) fail(ctx, DD4DV_EINVAL, "NULL argument");
    *n = ctx->pt_steps;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_launch_count(const dd4dv_ctx* ctx, long long* n) {
  if (!ctx || !n) return DD4DV_EINVAL;
  *n = ctx->launches;
  return DD4DV_OK;
}

dd4dv_status dd4dv_profile_sweeps(dd4dv_ctx* ctx, const double* w_all, int reps, double* ms) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!w_all || !ms || reps < 1) fail(ctx, DD4DV_EINVAL, "bad argument");
    h2d(ctx, ctx->io_a, w_all, ctx->ctrl_total * sizeof(double));
    cudaEvent_t ev[6];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    double tf = 0, ta = 0, te = 0;
    long long kernels = 0;
    by_precision(ctx, [&](auto t) {
      using T = decltype(t);
      for (int r = 0; r <= reps; ++r) {
        const long long k0 = ctx->launches;
        CK(cudaEventRecord(ev[4], ctx->st));
        init_states<T>(ctx, ctx->io_a, ctx->vw, nullptr, 0);
        CK(cudaEventRecord(ev[0], ctx->st));
        forward_sweep<T>(ctx, nullptr, 0);
        CK(cudaEventRecord(ev[1], ctx->st));
        KL(launch_finalize_J(ctx->subs_d, ctx->n_sub, ctx->io_a, ctx->part, ctx->cl_f, ctx->vconst,
                             ctx->dec.lambda, ctx->dec.mu, ctx->io_p, nullptr, nullptr, 0, ctx->st));
        SweepArgs<T> a = sweep_args<T>(ctx);
        CK(cudaEventRecord(ev[2], ctx->st));
        KL(launch_adjoint<T>(a, ctx->cl, ctx->nthreads, ctx->st));
        CK(cudaEventRecord(ev[3], ctx->st));
        apply_VT(ctx, ctx->lam_a, ctx->io_a, nullptr, ctx->io_b, nullptr, 0);
        CK(cudaEventRecord(ev[5], ctx->st));
        CK(cudaEventSynchronize(ev[5]));
        float f = 0, ad = 0, e = 0;
        CK(cudaEventElapsedTime(&f, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&ad, ev[2], ev[3]));
        CK(cudaEventElapsedTime(&e, ev[4], ev[5]));
        if (r > 0) { tf += f; ta += ad; te += e; }
        kernels = ctx->launches - k0;
      }
      return 0;
    });
    for (auto& e : ev) cudaEventDestroy(e);
    sync(ctx);
    ms[0] = tf / reps;
    ms[1] = ta / reps;
    ms[2] = te / reps;
    ms[3] = (double)kernels;
    ctx->fwd_pending = false;
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_sweep_config(const dd4dv_ctx* cctx, int* shape, double* eval_ms) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  if (!ctx) return DD4DV_EINVAL;
  if (!ctx->has_dec) return DD4DV_ESTATE;
  if (shape) {
    shape[0] = ctx->cl_f;
    shape[1] = ctx->nt_f;
    shape[2] = ctx->cl;
    shape[3] = ctx->nthreads;
    shape[4] = ctx->use_stg ? 1 : 0;
  }
  if (eval_ms) *eval_ms = ctx->tune_ms;
  return DD4DV_OK;
}

dd4dv_status dd4dv_set_sweep_config(dd4dv_ctx* ctx, const int* shape) {
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!shape) fail(ctx, DD4DV_EINVAL, "shape is NULL");
    const int cf = shape[0], tf = shape[1], ca = shape[2], ta = shape[3], sg = shape[4];
    for (int c : {cf, ca})
      if (c < 1 || c > 16 || c > ctx->min_ny)
        fail(ctx, DD4DV_EINVAL, "cluster sizes must be 1..16 and <= the smallest box height %d", ctx->min_ny);
    for (int t : {tf, ta})
      if (t < 64 || t > 1024 || t % 32) fail(ctx, DD4DV_EINVAL, "threads must be a multiple of 32 in 64..1024");
    if (sg && !ctx->stg) fail(ctx, DD4DV_EINVAL, "no stage buffer (ckpt_k != 0 or freed by the autotuner)");
    const int Rf = (ctx->max_ny + cf - 1) / cf, Ra = (ctx->max_ny + ca - 1) / ca;
    const bool stg0 = ctx->use_stg;
    ctx->use_stg = sg != 0;
    const int kf = fwd_kind_at(ctx, cf, tf), ka = adj_kind_at(ctx, ca, ta);
    ctx->use_stg = stg0;
    if (!kf || !ka)
      fail(ctx, DD4DV_EINVAL,
           "%s sweep shape cannot run: too much shared memory, or more threads than the stripe sweep allows "
           "(FP32 forward 384, else 1024) where the deep-halo FP32 sweep does not apply (it needs stripes of "
           ">= 3 rows, <= 4 own points per thread and <= 640 threads)",
           !kf ? "forward" : "adjoint");
    ctx->cl_f = cf; ctx->nt_f = tf; ctx->R_f = Rf;
    ctx->cl = ca; ctx->nthreads = ta; ctx->R = Ra;
    ctx->use_stg = sg != 0;
    ctx->dec.cluster = ca;
    ctx->drop_graphs();
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_checkpoint_interval(const dd4dv_ctx* cctx, int* k, double* eval_ms) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  if (!ctx) return DD4DV_EINVAL;
  if (!ctx->has_dec) return DD4DV_ESTATE;
  if (k) *k = ctx->use_stg ? 0 : (ctx->ckpt > 0 ? ctx->ckpt : (ctx->stg1 ? -3 : -1));
  if (eval_ms) *eval_ms = ctx->ckpt_ms;
  return DD4DV_OK;
}

dd4dv_status dd4dv_stage1_stored(const dd4dv_ctx* cctx, int* n_subs, double* pt_step_share) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  if (!ctx) return DD4DV_EINVAL;
  if (!ctx->has_dec) return DD4DV_ESTATE;
  const bool on = ctx->stg1 && !ctx->use_stg;
  if (n_subs) *n_subs = on ? ctx->stg1_subs : 0;
  if (pt_step_share) *pt_step_share = on ? ctx->stg1_frac : 0.0;
  return DD4DV_OK;
}

dd4dv_status dd4dv_set_sweep_variant(dd4dv_ctx* ctx, int forward, int adjoint) {
  return guard(ctx, [&] {
    if (forward < 0 || forward > 2 || adjoint < 0 || adjoint > 2)
      fail(ctx, DD4DV_EINVAL,
           "variants: 0 (automatic), 1 (stripe sweeps) or 2 (two-buffer stripe forward, four-buffer stripe "
           "adjoint)");
    ctx->variant_f = forward;
    ctx->variant_a = adjoint;
    ctx->drop_graphs();
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_sweep_kernels(const dd4dv_ctx* cctx, int* kinds) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  return guard(ctx, [&] {
    require_dec(ctx);
    if (!kinds) fail(ctx, DD4DV_EINVAL, "NULL argument");
    kinds[0] = fwd_kind_at(ctx, ctx->cl_f, ctx->nt_f);
    kinds[1] = adj_kind_at(ctx, ctx->cl, ctx->nthreads);
    return DD4DV_OK;
  });
}

dd4dv_status dd4dv_cluster_size(const dd4dv_ctx* cctx, int* n) {
  auto* ctx = const_cast<dd4dv_ctx*>(cctx);
  if (!ctx || !n) return DD4DV_EINVAL;
  if (!ctx->has_dec) return DD4DV_ESTATE;
  *n = ctx->cl;
  return DD4DV_OK;
}

}  // extern "C"
