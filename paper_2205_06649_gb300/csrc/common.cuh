// Internal declarations of the DD-4DVar GB300 library (not part of the C ABI).
//
// Device data layout (HBM):
//   * per-subdomain trajectories: traj[s] = [L+1 levels][3 vars][ny rows][nxp],
//     state type T (double, or float with h stored as h - h_ref), row pitch
//     nxp = nx rounded up to a multiple of 4 so every row starts on a 32-byte
//     boundary; subdomains are packed one after another (SubDesc::traj_off);
//   * overlap targets tgt[s]: same shape, the mean of the neighbours' values
//     at every point the subdomain shares with others (zero elsewhere);
//   * boundary trajectory bnd = [nsteps+1][3][nlat][nlon] (type T), the
//     partition-of-unity sum of the local trajectories (Eq. rest);
//   * stage states stg[s] = [L steps][2 stages][3 vars][ny][nxp]: the RK3
//     intermediate states x1, x2 of every step, stored by the forward sweep so
//     that the adjoint sweep loads them instead of recomputing them;
//   * controls, gradients, L-BFGS vectors: packed FP64 [3][ny][nx] per
//     subdomain (SubDesc::ctrl_off).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace dd4dv {

enum { F_PERIODIC = 1, F_SWALL = 2, F_NWALL = 4 };

struct SubDesc {
  int i0, nx, j0, ny, a, b;   // box [i0, i0+nx) (lon, mod nlon) x [j0, j0+ny), levels [a, b]
  int nxp;                    // trajectory row pitch (elements)
  int flags;                  // F_PERIODIC | F_SWALL | F_NWALL
  int q, p2, p1;              // block coordinates
  int wL, wR, wS, wN;         // overlap band widths: lon west/east, lat south/north
  int tA, tB;                 // overlap level counts at window start / end
  int obs_lvl;                // first entry of this subdomain in lvl_obs (L+2 entries)
  int sc_lvl;                 // first entry in lvl_sc (L+2 entries)
  long long ctrl_off;         // packed control offset (doubles)
  long long traj_off;         // trajectory offset (elements of T)
  long long ptraj_off;        // packed public trajectory offset (doubles, pitch nx)
  long long stg_off;          // stage-state offset (elements of T): [L][2][3][ny][nxp]
  long long stg1_off;         // offset of x1 alone (elements of T): [L][3][ny][nxp]; -1: not stored
  long long seg_off;          // checkpoint-segment buffer offset (elements of T): [k+1][3][ny][nxp]
};

struct ObsRec {               // one observation as seen by one subdomain
  int var, r0, k0, k1;        // local lower corner row/col, east corner col (wrapped)
  double di, dj;              // fractional offsets (0 = corner not used)
  double y;                   // observed value (h: minus h_ref on the FP32 path)
  double w;                   // omega / sigma_o^2
};

struct RowConst {             // per global latitude row j
  double A;                   // 1 / (2 a cos(theta_j) dlambda)
  double f;                   // 2 Omega sin(theta_j)
  double tau;                 // tan(theta_j) / a
  double c;                   // cos(theta_j)
  double BinvC;               // Bth / cos(theta_j)
  double gA;                  // g A
};

// Arguments shared by the sweep kernels (forward, adjoint, tangent-linear).
template <typename T>
struct SweepArgs {
  const SubDesc* subs;
  const int* order;           // cluster -> subdomain (longest first)
  int n_sub;
  T* traj;
  T* stg;                     // RK3 stage states x1, x2 of every step, or nullptr (recompute)
  T* stg1;                    // with stg == nullptr: x1 of every step of the subdomains whose
                              // stg1_off >= 0 (x2 recomputed), or nullptr
  int ckpt;                   // 0: every level stored; k > 0: levels 0, k, 2k, ... stored and
                              // each k-step segment recomputed in the adjoint
  T* seg;                     // per-subdomain segment buffers for the recomputation
  const T* tgt;
  const T* bnd;
  const RowConst* rows;       // [nlat]
  double Bth, gBth, dt, h_ref;
  int nlon, nlat, nsteps;
  double isb2[3];             // 1 / sigma_b^2 per variable
  double lam, mu;
  // the same constants rounded once to the state precision on the host, so
  // that the FP32 sweeps run no FP64 conversion per stage or level
  T dt_s, Bth_s, gBth_s, href_s;
  T isb2_s[3], musb2_s[3];    // 1 / sigma_b^2 and mu / sigma_b^2
  const ObsRec* obs;          // per-subdomain, per-level sorted
  const int* lvl_obs;         // obs ranges per (subdomain, level)
  double* obs_force;          // lambda * omega * d / sigma_o^2 per obs record
  const int* sc_tgt;          // adjoint scatter targets: var*ny*nx + r*nx + k
  const int* sc_off;          // contributions of each target
  const int* sc_obs;
  const double* sc_w;
  const int* lvl_sc;          // target ranges per (subdomain, level)
  double* part;               // [n_sub][cl_max][2] partial J_o, J_mu
  int cl_max;
  const int* active;          // per-subdomain mask (phase == active_value), or nullptr
  int active_value;
  double* lam_a;              // adjoint state at level a, packed control layout
  const double* yforce;       // external adjoint forcing (packed FP64 trajectories) or nullptr
  double* dx_out;             // tangent-linear output (packed FP64 trajectories)
  const double* dx0;          // tangent-linear initial perturbation (packed control layout)
  T* gn_dx;                   // Gauss-Newton products: the tangent-linear sweep stores dx here
                              // (trajectory layout) and sets obs_force = lambda w H dx; the
                              // adjoint sweep then takes its overlap forcing mu c dx / sb^2
                              // from it instead of mu c (x - m) / sb^2
  int R;                      // max rows per CTA
  int W;                      // shared-memory row pitch (>= max nx + 2)
  int* err;                   // device error word (0 = ok)
  int tgb_on;                 // set by the launcher: the FP32 sweep's shared memory holds a
                              // buffer of prefetched overlap targets (only if it still fits)
  int min_ny;                 // smallest box height of the decomposition
  int variant;                // 0: deep-halo FP32 sweeps where they apply, else the stripe
                              // sweeps; 1: stripe sweeps only; 2: the stripe adjoint with
                              // four state buffers (x(n) reloaded from HBM), the stripe
                              // forward with two (x(n) read from the stored level)
};

// Largest CTA of the stripe forward sweep: 384 threads on the FP32 path,
// whose forward kernel is compiled for up to 80 registers (2 CTAs of 384
// threads per SM), 1024 on the FP64 path (64 registers, one CTA of 1024 or two
// of 512 per SM).  The stripe adjoint takes up to 1024 threads (64 registers).
template <typename T> constexpr int max_threads_forward() { return sizeof(T) == 4 ? 384 : 1024; }
template <typename T> constexpr int min_blocks_forward() { return sizeof(T) == 4 ? 2 : 1; }
constexpr int kStripeAdjThreads = 1024;

// ---- launchers (sweep.cu) ----
// Which kernel a sweep launch with cl CTAs per subdomain and nthreads threads
// per CTA would run: 0 = none (shape not launchable), 1 = the stripe sweep
// (one halo row per stage), 2 = the deep-halo FP32 sweep (three halo rows, one
// exchange per step), 3 = the stripe adjoint with four state buffers, 4 =
// the stripe forward with two state buffers.
template <typename T> int forward_kind(const SweepArgs<T>& a, int cl, int nthreads);
template <typename T> int adjoint_kind(const SweepArgs<T>& a, int cl, int nthreads);
template <typename T> cudaError_t launch_forward(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st);
template <typename T> cudaError_t launch_adjoint(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st);
template <typename T> cudaError_t launch_tlm(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st);
template <typename T> size_t smem_forward(int R, int W);
template <typename T> size_t smem_adjoint(int R, int W);
template <typename T> size_t smem_adjoint_rl(int R, int W);
template <typename T> size_t smem_tlm(int R, int W);
// resident clusters of the stripe adjoint sweep at cl CTAs per cluster
template <typename T> int active_clusters_adjoint(int R, int W, int cl, int nthreads);

// ---- auxiliary kernels (aux.cu) ----
struct RFArgs {
  const SubDesc* subs; int n_sub;
  double alpha, c; int npass;
  const int* active; int active_value;
};
// in place: lines along lon (rows) or lat (columns) of each [3][ny][nx] block
cudaError_t launch_rf_rows(double* x, const RFArgs& a, int max_ny, cudaStream_t st);
cudaError_t launch_rf_cols(double* x, const RFArgs& a, int max_nx, cudaStream_t st);

// fused V / V^T (one CTA per subdomain and variable, plane in shared memory)
template <typename T>
cudaError_t launch_vinit(const SubDesc* subs, int n_sub, const double* xb_a, const double* w,
                         const double* sigma, const RFArgs& rf, int use_rf, double h_ref, T* traj,
                         const int* active, int active_value, int max_plane, cudaStream_t st);
// R = precision of the recursive filter (the state precision)
template <typename R>
cudaError_t launch_vgrad(const SubDesc* subs, int n_sub, const double* w, const double* y, const double* sigma,
                         const RFArgs& rf, int use_rf, const double* scale, double* grad, const int* active,
                         int active_value, int max_plane, cudaStream_t st);
template <typename T>
cudaError_t launch_init_state(const SubDesc* subs, int n_sub, const double* xb_a, const double* vw,
                              const double* sigma, int scale_sigma, double h_ref, T* traj,
                              const int* active, int active_value, int max_pts, cudaStream_t st);
cudaError_t launch_scale_copy(const SubDesc* subs, int n_sub, const double* in, const double* sigma,
                              double* out, const int* active, int active_value, int max_pts,
                              cudaStream_t st);
cudaError_t launch_grad_finish(const SubDesc* subs, int n_sub, const double* w, const double* vty,
                               const double* scale, double* grad, const int* active,
                               int active_value, int max_pts, cudaStream_t st);
cudaError_t launch_finalize_J(const SubDesc* subs, int n_sub, const double* w, const double* part,
                              int cl_max, const double* vconst, double lam, double mu, double* J,
                              double* parts, const int* active, int active_value, cudaStream_t st);

template <typename T>
struct ExchArgs {
  const SubDesc* subs; int n_sub;
  int P1, P2, Q;
  int nlon, nlat, nsteps;
  const T* traj; T* tgt; T* bnd;
  double isb2[3];
  double* vpart;              // [n_sub][blocks] partial sums of the overlap constant
  int vblocks;
  const int* lon_cov;         // [nlon][2][2] (p1, local col) or -1
  const int* lat_cov;         // [nlat][2][2]
  const int* t_cov;           // [nsteps+1][2][2]
};
template <typename T> cudaError_t launch_targets(const ExchArgs<T>& a, cudaStream_t st);
template <typename T> cudaError_t launch_assemble(const ExchArgs<T>& a, cudaStream_t st);
cudaError_t launch_sum_vconst(const double* vpart, int n_sub, int vblocks, double* vconst, cudaStream_t st);

template <typename T>
cudaError_t launch_restrict(const SubDesc* subs, int n_sub, int nlon, int nlat, const double* glob,
                            int g0, int g1, double h_ref, T* traj, int max_pts, cudaStream_t st);
template <typename T>
cudaError_t launch_export_traj(const SubDesc* subs, int n_sub, const T* traj, double h_ref,
                               double* out, int max_pts, int max_levels, cudaStream_t st);
template <typename T>
cudaError_t launch_bnd_from_global(const double* glob, long long n, double h_ref, int nlon, int nlat,
                                   T* bnd, cudaStream_t st);
template <typename T>
cudaError_t launch_bnd_to_global(const T* bnd, long long n, double h_ref, int nlon, int nlat,
                                 double* glob, cudaStream_t st);
cudaError_t launch_restrict_level(const SubDesc* subs, int n_sub, int nlon, int nlat, const double* glob,
                                  int g0, int g1, double* xb_a, int max_pts, cudaStream_t st);

// global model (whole sphere), FP64
cudaError_t launch_global_stage(const double* x, const double* y, double* out, double ca, double cb,
                                const RowConst* rows, double Bth, double gBth, double dt, int nlon,
                                int nlat, cudaStream_t st);
cudaError_t launch_observe(const double* traj, int g0, int g1, long long n, const int* level,
                           const int* var, const double* fi, const double* fj, int nlon, int nlat,
                           double* out, cudaStream_t st);

// L-BFGS (batched, one block per subdomain)
struct LbState {
  double J, Jt, gp, alpha, g0n, gn;
  int head, count, iter, trial, phase, status;
};
struct LbArgs {
  const SubDesc* subs; int n_sub;
  double* w; double* g; double* wt; double* gt; double* p;
  double* S; double* Y; double* rho;   // [m][total], [m][total], [n_sub][m]
  long long total;
  LbState* st;
  const double* J_eval;                // J of the last evaluation
  int m, max_iter, max_trials;
  double gtol, c1;
  int* counter;                        // [2]: # in line search, # needing a direction
  int* phase;                          // [n_sub] mirror of LbState::phase (sweep masks)
  const int* owned;                    // [n_sub] 1 = this context solves the subdomain, or nullptr
};
cudaError_t launch_lb_start(const LbArgs& a, cudaStream_t st);
cudaError_t launch_lb_direction(const LbArgs& a, cudaStream_t st);
cudaError_t launch_lb_linesearch(const LbArgs& a, cudaStream_t st);
// Batched conjugate gradients for the Gauss-Newton normal equations, one
// block per subdomain (fixed-order block reductions).
struct CgState {
  double rr, rr0, g0n;
  int k, status;   // status: 0 running, 1 converged, 2 iteration limit, 3 p.Ap <= 0, 4 skipped
};
struct CgArgs {
  const SubDesc* subs; int n_sub;
  const double* g;                     // gradient at the linearisation point (rhs = -g)
  double *r, *p, *Ap, *dw;             // packed control layout
  CgState* st;
  int* phase;                          // [n_sub] 1 = solving (sweep mask)
  int* counter;                        // # still solving
  int max_iter, first;                 // first: this is the first Gauss-Newton iteration
  double tol, gtol;
};
cudaError_t launch_cg_start(const CgArgs& a, cudaStream_t st);
cudaError_t launch_cg_step(const CgArgs& a, cudaStream_t st);
cudaError_t launch_axpy(double* y, const double* x, long long n, cudaStream_t st);   // y += x
cudaError_t launch_max_abs_diff(const double* a, const double* b, long long n, double* out,
                                cudaStream_t st);
cudaError_t launch_finite_check(const double* a, long long n, int* flag, cudaStream_t st);

// ---- Turkel-Zwas scheme on the whole sphere (tz.cu) ----
struct TzArgs {
  const RowConst* rows;       // [nlat]
  int nlon, nlat, p, q;
  double alpha, slon, slat, g, dt;
};
cudaError_t launch_tz_stage(const TzArgs& t, const double* X, const double* Y, double* out, double cx, double cy,
                            cudaStream_t st);
cudaError_t launch_tz_tl_stage(const TzArgs& t, const double* Y, const double* dX, const double* dY, double* dout,
                               double cx, double cy, cudaStream_t st);
cudaError_t launch_tz_adj_scatter(const TzArgs& t, const double* Y, const double* M, double* G, double scale,
                                  cudaStream_t st);
cudaError_t launch_tz_lincomb(double* out, const double* a, const double* b, const double* c, double ca, double cb,
                              double cc, long long n, cudaStream_t st);
cudaError_t launch_tz_scale_add(double* out, const double* a, const double* b, const double* sigma, long long plane,
                                cudaStream_t st);
cudaError_t launch_tz_obs_misfit(const double* traj, long long n, const int* level, const int* var, const double* fi,
                                 const double* fj, const double* y, const double* so, int nlon, int nlat, double lam,
                                 double* force, double* Jo, cudaStream_t st);
cudaError_t launch_tz_obs_scatter(long long k0, long long k1, const int* var, const double* fi, const double* fj,
                                  const double* force, int nlon, int nlat, double* lam, cudaStream_t st);
cudaError_t launch_tz_finish_J(const double* w, long long n, const double* Jo, double* J, cudaStream_t st);

}  // namespace dd4dv
