/*
 * dd4dvar.h -- C interface of the GB300 (sm_103a) library for space-time
 * domain-decomposed strong-constraint 4D-Var (DD-4DVar) on the shallow-water
 * equations on the sphere.
 *
 * Method: D'Amore, Constantinescu & Carracciuolo, "A scalable space-time
 * domain decomposition approach for solving large-scale nonlinear regularized
 * inverse ill-posed problems in 4D variational data assimilation"
 * (arXiv 2205.06649).  Section, equation and algorithm numbers below refer to
 * that paper.  The calls follow Algorithm 1's signature
 * DD-4DVar(in: M, u0b, {R_k}, B, H, v, Delta_M, Omega_K; out: u^DA):
 * set the model and grid, the background, B and the observations (with R),
 * set the decomposition and overlap, then evaluate the local functionals and
 * gradients or run the outer loop.
 *
 * Conventions (all calls)
 *   - Return value: dd4dv_status.  0 = success, negative = error (nothing
 *     of the requested output is valid), DD4DV_NOTCONV = finished without
 *     meeting the stopping test (outputs valid).  dd4dv_last_error() gives a
 *     message.  No C++ exception crosses this interface.
 *   - Ownership: the library copies every input at the call; the caller owns
 *     every buffer it passes and keeps ownership; outputs are written into
 *     caller buffers.  The context owns its device memory (cudaMalloc) and
 *     frees it in dd4dv_destroy.
 *   - Pointers: "host" arguments are ordinary host memory.  Where an entry
 *     point takes `device_ptrs`, 1 means every array argument of that call
 *     is CUDA device memory of the current device, read and written in
 *     stream order on the context's stream, and the call returns once the
 *     work is enqueued; 0 means host memory (the call copies in, runs, copies
 *     out and synchronises before it returns).
 *   - State layout: a state is [3][nlat][nlon] doubles, variables (h, u, v)
 *     in that order, row = latitude index j (south to north), column =
 *     longitude index i (eastward).  Trajectories are [nsteps+1][3][nlat][nlon].
 *   - Call order: create -> set_background, set_background_error,
 *     set_observations (any order) -> set_decomposition -> eval/run...
 *     A call made too early returns DD4DV_ESTATE.  Any set_* call after
 *     set_decomposition invalidates it (call set_decomposition again).
 *   - Threading: a context may be used by one host thread at a time.
 */
#ifndef DD4DVAR_H
#define DD4DVAR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd4dv_ctx dd4dv_ctx;      /* opaque, library-owned */

typedef enum {
  DD4DV_OK = 0,
  DD4DV_EINVAL = -1,       /* bad argument (size, range, NULL, layout)     */
  DD4DV_ENOMEM = -2,       /* device or pinned host allocation failed      */
  DD4DV_ECUDA = -3,        /* CUDA runtime error (message has the details) */
  DD4DV_ESTATE = -4,       /* call made before its prerequisites           */
  DD4DV_ETIMEOUT = -5,     /* reserved, never returned: no kernel of this
                              library spin-waits (the sweeps synchronise
                              only through hardware cluster barriers), so
                              there is no bounded wait that could run out  */
  DD4DV_ENONFINITE = -6,   /* NaN or Inf in an input                       */
  DD4DV_NOTCONV = 1        /* warning: stopping test not met, outputs valid */
} dd4dv_status;

/*
 * Model and grid (Sec. 7, Eqs. EquU-EquH; Definition "DA problem setup",
 * Sec. 2).  Regular lon-lat grid of nlon x nlat cell centres, periodic in
 * longitude, reflecting walls at lat_min_deg and lat_max_deg (the cell faces).
 * Centred second-order differences, flux-form continuity, SSP-RK3 steps of
 * dt seconds, nsteps steps in the assimilation window (levels 0..nsteps).
 * precision: 0 = FP64 state; 1 = FP32 state (h stored as h - h_ref) with
 * FP64 control, gradients, J and all reductions.
 */
typedef struct {
  int nlon, nlat;
  double lat_min_deg, lat_max_deg;
  double radius, gravity, omega;
  double dt;
  int nsteps;
  int precision;
  double h_ref;            /* FP32 path: reference depth removed from h   */
} dd4dv_model;

/*
 * Space-time decomposition DD(Delta x Omega) (Sec. 3.1, Eqs. DDOmega-decomall;
 * sizes per Sec. 7 Eq. nlocx: core block extended by o on each side).
 * P1 lon blocks x P2 lat blocks x Q time windows.  Cuts are core-block
 * boundaries (P1+1, P2+1, Q+1 increasing values from 0 to nlon / nlat /
 * nsteps), or NULL for equal blocks.  Requirements: every core lon/lat block
 * >= 2*o and >= 2 points, every core window > 2*o_t steps, o >= 1 where
 * the axis is split, extended lon box < nlon.  Subdomain numbering:
 * s = (q * P2 + p2) * P1 + p1.
 * mu, lambda: weights of the overlap and observation terms (Eq.
 * eq:cost:parallel1).  weight_obs = 1 weights each observation by
 * 1/(number of subdomains containing it), the restriction weights of
 * Definition "Restriction of a function"; 0 gives weight 1.
 * cluster: CTAs per subdomain in the sweep kernels (thread-block cluster
 * size, 1..16); 0 = chosen from a model of the launch; -1 = autotune: the
 * forward and adjoint sweeps are timed at every feasible (cluster size, threads
 * per CTA) shape, with stored and with recomputed stage states when
 * ckpt_k = 0, and the fastest shape of each and the faster mode are kept (see
 * dd4dv_sweep_config); if recomputation wins, the stage buffer is freed.
 * ckpt_k: trajectory storage for the adjoint.  0 = the forward sweep stores
 * every level and the two RK3 stage states of every step, and the adjoint
 * loads them (three times the memory of the states alone; on GB300 this
 * trades FP64 arithmetic for otherwise idle HBM bandwidth) -- the stage buffer
 * is allocated only if it leaves 4 GB + 5 % of the device memory free, else
 * the first stage state alone is stored as with -3; -1 = store every
 * level, the adjoint recomputes the stage states; -3 (FP64 path; as -1 on
 * the FP32-state path) = store every level and the first RK3 stage state x1
 * of every step, for as many subdomains as fit (longest first, same 4 GB +
 * 5 % reserve; dd4dv_stage1_stored reports them), whose adjoint then
 * recomputes only x2 (the others recompute both);
 * k > 0 = checkpointing:
 * evaluations store only the levels 0, k, 2k, ... and the adjoint
 * recomputes each k-step segment from its checkpoint before running back
 * through it (the exchange and dd4dv_trajectories still store every level);
 * -2 = choose by timing: after the launch shapes are set (or autotuned), one
 * evaluation is timed with stored stage states (when their buffer fits),
 * with recomputed stages and with checkpoints every 8, 16 and 32 levels, the
 * fastest is kept and the unused buffers are freed (dd4dv_checkpoint_interval
 * reports the choice).
 */
typedef struct {
  int P1, P2, Q;
  const int* lon_cuts;
  const int* lat_cuts;
  const int* t_cuts;
  int o_lon, o_lat, o_t;
  double mu, lambda;
  int weight_obs;
  int cluster;
  int ckpt_k;
} dd4dv_decomp;

/*
 * Local minimiser settings (Algorithm 2/3 with L-BFGS, Remark after
 * Algorithm 5) and outer loop (Algorithm 1).
 */
typedef struct {
  int lbfgs_m;             /* memory pairs (5)                             */
  int max_local_iters;     /* L-BFGS iterations per outer iteration (20)   */
  int max_trials;          /* Armijo trials per iteration (20)             */
  int max_outer;           /* outer iterations (10)                        */
  double eps_outer;        /* stop when max_s ||w_s^l - w_s^(l-1)||_inf < eps */
  double gtol_rel;         /* local stop when ||g|| / ||g_0|| < gtol       */
  double c1;               /* Armijo constant (1e-4)                       */
  int use_graphs;          /* 1: each step of the iteration (start evaluation,
                              L-BFGS direction, line-search trial, exchange) is
                              captured once as a CUDA graph and replayed;
                              0: launched eagerly.  Same results.        */
  int local_solver;        /* 0: L-BFGS (above); 1: Gauss-Newton (Algorithm 5
                              as Algorithm 6) with conjugate-gradient inner
                              solves of (I + G^T G) dw = -grad J_s in the
                              control variable (the B-preconditioned system
                              of Algorithm 7; CG gives the Lanczos iterates) */
  int gn_iters;            /* Gauss-Newton iterations per outer iteration
                              (each: one J/grad evaluation, one CG solve);
                              a subdomain stops early when
                              ||g|| <= gtol_rel ||g_0||                      */
  int cg_iters;            /* CG iterations per Gauss-Newton iteration; one
                              Gauss-Newton product (tangent-linear sweep +
                              adjoint sweep) each                            */
  double cg_tol;           /* CG stop: ||r|| <= cg_tol ||r_0||              */
} dd4dv_solver;

typedef struct {
  int outer_iters;         /* outer iterations done                        */
  long long evals;         /* batched J/grad evaluations                   */
  long long sub_evals;     /* subdomain evaluations (active subdomains)    */
  long long pt_steps;      /* grid-point steps, forward+adjoint, all evals */
  double dw_inf;           /* last max_s ||w^l - w^(l-1)||_inf             */
  double J_sum;            /* sum over subdomains of the final local J     */
  double gnorm_rel_max;    /* max_s ||g|| / ||g_0|| at the end             */
  int n_linesearch_fail;   /* local solves stopped by a failed line search */
} dd4dv_stats;

/* Create a context on the current CUDA device.  stream: a cudaStream_t to
 * order all work on (NULL = the context creates its own).  Device memory held
 * from here on: a few global states and a chunk of at most 512 MB of global
 * levels (global runs and host transfers of global trajectories go through
 * it; the environment variable DD4DV_GLOBAL_CHUNK_LEVELS = 2..4096, read
 * here, sets its number of levels instead).  Errors: EINVAL (sizes, dt <= 0,
 * nsteps < 0, lat range), ECUDA, ENOMEM. */
dd4dv_status dd4dv_create(const dd4dv_model* model, void* cuda_stream, dd4dv_ctx** out);

/* Free the context and all its device memory.  NULL is accepted. */
dd4dv_status dd4dv_destroy(dd4dv_ctx* ctx);

/* Background initial state u_0^b (Definition "DA problem setup"): host array
 * [3][nlat][nlon], copied.  The background forecast u^b = M(u_0^b) over the
 * window (Algorithm 1, background step) runs on the device when the
 * decomposition is set and at dd4dv_reset_exchange; it is streamed into the
 * boundary trajectory and the overlap targets a chunk of levels at a time, so
 * no separate global FP64 trajectory is kept.  ENONFINITE on NaN/Inf. */
dd4dv_status dd4dv_set_background(dd4dv_ctx* ctx, const double* xb0);

/* Background-error covariance B = V V^T (Sec. 4, Eq. EqV).  sigma_b[3]:
 * standard deviations of (h, u, v), > 0.  corr_len_cells = 0: diagonal B;
 * > 0: V = diag(sigma_b) L_lat L_lon with L a recursive filter of rf_passes
 * (1..8) forward/backward passes matched to a Gaussian of that length. */
dd4dv_status dd4dv_set_background_error(dd4dv_ctx* ctx, const double sigma_b[3],
                                        double corr_len_cells, int rf_passes);

/* Observations v and diagonal R_k (Definition "DA problem setup"; the
 * observation term of Eq. min3sec).  n records, host arrays: level in
 * [0, nsteps], var in {0,1,2} (h,u,v), fractional grid indices
 * fi in [0, nlon), fj in [0, nlat-1], value, sigma_o > 0.  H is bilinear
 * interpolation in index space, periodic in longitude. */
dd4dv_status dd4dv_set_observations(dd4dv_ctx* ctx, long long n, const int* level,
                                    const int* var, const double* fi, const double* fj,
                                    const double* value, const double* sigma_o);

/* Set the space-time decomposition and overlap (see dd4dv_decomp); builds
 * all device tables, puts the exchange state at l = 0 (boundary trajectory =
 * background trajectory, neighbour trajectories = background) and sets every
 * local control to 0. */
dd4dv_status dd4dv_set_decomposition(dd4dv_ctx* ctx, const dd4dv_decomp* dec);

/* Number of subdomains P1*P2*Q. */
dd4dv_status dd4dv_num_subdomains(const dd4dv_ctx* ctx, int* n);

/* Packed control layout.  offsets[n+1]: start of each subdomain's control
 * w_s (3*ny*nx doubles, layout [3][ny][nx]) in the packed vector, offsets[n]
 * = total.  boxes[6*n] (may be NULL): i0, nx, j0, ny, a, b per subdomain
 * (first global lon column, width, first lat row, height, window levels). */
dd4dv_status dd4dv_control_layout(const dd4dv_ctx* ctx, long long* offsets, int* boxes);

/* Evaluate every local functional J_s(w_s) (Sec. 3.3, Eq. eq:cost:parallel1
 * with halves of squared norms) and, when grad_all != NULL, its gradient
 * with respect to w_s (discrete adjoint, Algorithm 6 ADJ), with the current
 * boundary trajectory and neighbour data held fixed.
 *   w_all[total], grad_all[total]: packed controls (dd4dv_control_layout);
 *   J_all[n]; parts (may be NULL) [3*n]: J_b, J_o, J_mu per subdomain with
 *   J_s = J_b + lambda J_o + mu J_mu.
 * device_ptrs as in the conventions.  One batched launch per sweep covers
 * all subdomains. */
dd4dv_status dd4dv_eval(dd4dv_ctx* ctx, const double* w_all, double* J_all, double* grad_all,
                        double* parts, int device_ptrs);

/* Split evaluation for reverse-mode frameworks: dd4dv_eval_forward computes
 * J (and parts) and keeps what the adjoint needs; dd4dv_eval_backward then
 * writes grad_all = scale[s] * dJ_s/dw_s for that same w (scale: n doubles,
 * NULL = all ones).  ESTATE if no forward is pending. */
dd4dv_status dd4dv_eval_forward(dd4dv_ctx* ctx, const double* w_all, double* J_all,
                                double* parts, int device_ptrs);
dd4dv_status dd4dv_eval_backward(dd4dv_ctx* ctx, const double* scale, double* grad_all,
                                 int device_ptrs);

/* Tangent-linear model (Algorithm 6, TLM) of the map w -> local trajectory,
 * for every subdomain at once: dx_all = (d x_s / d w_s) dw_s.  dx_all is the
 * packed trajectory layout (dd4dv_traj_layout), FP64, full h. */
dd4dv_status dd4dv_tlm(dd4dv_ctx* ctx, const double* w_all, const double* dw_all,
                       double* dx_all, int device_ptrs);

/* Adjoint of the same map (Eq. Eq_propAdj): dw_all = (d x_s / d w_s)^T y_all
 * for a packed trajectory-shaped y_all, every subdomain at once. */
dd4dv_status dd4dv_adjoint(dd4dv_ctx* ctx, const double* w_all, const double* y_all,
                           double* dw_all, int device_ptrs);

/* Packed trajectory layout: offsets[n+1] of each subdomain's trajectory
 * [b-a+1][3][ny][nx] (doubles) in a packed vector; offsets[n] = total. */
dd4dv_status dd4dv_traj_layout(const dd4dv_ctx* ctx, long long* offsets);

/* Local trajectories at w_all (forward model only), packed layout, FP64, full h. */
dd4dv_status dd4dv_trajectories(dd4dv_ctx* ctx, const double* w_all, double* traj_all,
                                int device_ptrs);

/* Gauss-Newton product of every local problem (test instrument and building
 * block of local_solver = 1): Ap = (I + G^T G) p with G = dr/dw the
 * derivative, at w_all, of the weighted residuals of J_s = 1/2 w.w +
 * 1/2 r.r (observation misfits sqrt(lambda omega) (H x - y) / sigma_o and
 * overlap mismatches sqrt(mu) (x - x^t) / sigma_b per covering neighbour t).
 * Formed matrix-free: V p, the tangent-linear sweep (Algorithm 6 TLM), the
 * adjoint sweep forced by lambda H^T W H dx + mu c dx / sigma_b^2 (Algorithm 6
 * ADJ), V^T.  Packed control layout for w_all, p_all, Ap_all. */
dd4dv_status dd4dv_gn_hessvec(dd4dv_ctx* ctx, const double* w_all, const double* p_all, double* Ap_all,
                              int device_ptrs);

/* Exchange step of Algorithm 1 for given local controls: run every local
 * model at w_all, record the local trajectories as the neighbour data of the
 * next evaluations and assemble the boundary trajectory as their
 * partition-of-unity sum (Eq. rest). */
dd4dv_status dd4dv_exchange(dd4dv_ctx* ctx, const double* w_all, int device_ptrs);

/* Return the exchange state to l = 0 (background everywhere).  Two device
 * copies when dd4dv_set_decomposition could keep a copy of that state (it
 * does when the copy leaves 4 GB + 5 % of the device free), else a rerun of
 * the background forecast. */
dd4dv_status dd4dv_reset_exchange(dd4dv_ctx* ctx);

/* The current assembled (boundary) trajectory [nsteps+1][3][nlat][nlon]. */
dd4dv_status dd4dv_boundary_trajectory(dd4dv_ctx* ctx, double* traj, int device_ptrs);

/* Global model run (Sec. 7 model, whole sphere) from x0 [3][nlat][nlon];
 * traj [nsteps+1][3][nlat][nlon], FP64 on the device. */
dd4dv_status dd4dv_forward(dd4dv_ctx* ctx, const double* x0, double* traj, int device_ptrs);

/* The Turkel-Zwas scheme of Sec. 7 (the paper's discretisation, with
 * longitude stride p, latitude stride q and averaging weight alpha) on the
 * undecomposed problem (the whole sphere, P = Q = 1).  Pressure gradients
 * over i +- p and j +- q, the Coriolis terms of the u (v) equation averaged
 * over i +- p (j +- q), the divergence averaged over (i +- p, j +- q), with
 * weight alpha; advection with stride 1; walls mirror (h, u, -v) to depth q;
 * SSP-RK3 steps of dt.  Readings of the garbled print: the printed leapfrog
 * increments are semi-discrete tendencies with sigma_lon = 1/(2 a dlambda),
 * sigma_lat = 1/(2 a dtheta); the meridional advection of v uses v
 * differences; H carries the sigma factors and h / cos(theta).  FP64, global
 * memory, one thread per grid point; the decomposed sweeps keep the centred
 * scheme (p = q = 1, alpha = 0, flux-form continuity).
 * Arguments: 1 <= p < nlon/2, 1 <= q < nlat, 0 <= alpha <= 1 (else EINVAL);
 * states [3][nlat][nlon], trajectories [nsteps+1][3][nlat][nlon];
 * device_ptrs as in the conventions.
 *   dd4dv_tz_forward: traj = the model run from x0.
 *   dd4dv_tz_tlm: dtraj = the tangent-linear run from dx0 about the run from
 *     x0 (Algorithm 6, TLM).
 *   dd4dv_tz_adjoint: dx0 = sum_n (d x_n / d x_0)^T y_n (Algorithm 6, ADJ),
 *     the transpose of dd4dv_tz_tlm.
 *   dd4dv_tz_eval: the global functional J(w) = 1/2 w.w + 1/2 sum_obs
 *     (H x_n - y)^2 / sigma_o^2 with x_0 = u_0^b + sigma_b w (diagonal B:
 *     set_background_error with corr_len_cells = 0, else EINVAL; ESTATE
 *     before set_background / set_background_error), the context's
 *     observations, and its gradient w + sigma_b lambda_0 (grad may be NULL).
 * Each call allocates its trajectory and scratch for the call. */
dd4dv_status dd4dv_tz_forward(dd4dv_ctx* ctx, int p, int q, double alpha, const double* x0, double* traj,
                              int device_ptrs);
dd4dv_status dd4dv_tz_tlm(dd4dv_ctx* ctx, int p, int q, double alpha, const double* x0, const double* dx0,
                          double* dtraj, int device_ptrs);
dd4dv_status dd4dv_tz_adjoint(dd4dv_ctx* ctx, int p, int q, double alpha, const double* x0, const double* ytraj,
                              double* dx0, int device_ptrs);
dd4dv_status dd4dv_tz_eval(dd4dv_ctx* ctx, int p, int q, double alpha, const double* w, double* J, double* grad,
                           int device_ptrs);

/* Observation operator H (bilinear, as in dd4dv_set_observations) applied to
 * a global trajectory traj [nsteps+1][3][nlat][nlon]: out[k] = H_k traj. */
dd4dv_status dd4dv_observe(dd4dv_ctx* ctx, const double* traj, long long n, const int* level,
                           const int* var, const double* fi, const double* fj, double* out,
                           int device_ptrs);

/* One outer iteration of Algorithm 1: batched local L-BFGS on every
 * subdomain from its current control, then the Exchange.  stats may be NULL;
 * otherwise its counters are incremented (zero it before the first call). */
dd4dv_status dd4dv_outer_step(dd4dv_ctx* ctx, const dd4dv_solver* solver, dd4dv_stats* stats);

/* Sharding the subdomains of one problem over several contexts (one per GPU;
 * the outer loop of Algorithm 1 with the local problems distributed, as the
 * paper's processors own subdomains in Sec. 7).  owned: host array of n_sub
 * flags (1 = this context evaluates and solves the subdomain), NULL = all
 * (the default after dd4dv_set_decomposition).  With a subset owned,
 * dd4dv_eval, dd4dv_eval_forward / _backward and dd4dv_local_solve work on the
 * owned subdomains only (the J, parts and gradient entries of the others are
 * left as they were), dd4dv_exchange still uses every subdomain's control,
 * and dd4dv_outer_step / dd4dv_run return DD4DV_ESTATE.  EINVAL if a flag is
 * not 0 or 1. */
dd4dv_status dd4dv_set_owned(dd4dv_ctx* ctx, const int* owned);

/* The local part of one outer iteration of Algorithm 1: the batched L-BFGS
 * of dd4dv_outer_step on every owned subdomain from its current control,
 * without the Exchange.  A sharded outer iteration is: dd4dv_local_solve on
 * each context, an all-gather of the owned control blocks (layout of
 * dd4dv_control_layout), dd4dv_set_controls and dd4dv_exchange with the full
 * vector on each context; every context then holds the same exchange state
 * as one context running dd4dv_outer_step, bit for bit.  stats (may be NULL)
 * counts the owned subdomains' work and J; dw_inf and outer_iters are left
 * to the caller.  EINVAL for local_solver != 0. */
dd4dv_status dd4dv_local_solve(dd4dv_ctx* ctx, const dd4dv_solver* solver, dd4dv_stats* stats);

/* Algorithm 1: outer iterations until max_s ||w^l - w^(l-1)||_inf < eps_outer
 * or max_outer, then the Gather: xa0 [3][nlat][nlon] (host, may be NULL) is
 * the analysis at t0 = the partition-of-unity sum of the first window's
 * local states.  Starts from the context's current controls and exchange
 * state.  Returns DD4DV_NOTCONV if max_outer was reached. */
dd4dv_status dd4dv_run(dd4dv_ctx* ctx, const dd4dv_solver* solver, double* xa0,
                       dd4dv_stats* stats);

/* Current analysis at t0 (boundary trajectory level 0), [3][nlat][nlon]. */
dd4dv_status dd4dv_analysis(dd4dv_ctx* ctx, double* xa0, int device_ptrs);

/* Current packed controls (copy out) / replace them (copy in). */
dd4dv_status dd4dv_get_controls(dd4dv_ctx* ctx, double* w_all, int device_ptrs);
dd4dv_status dd4dv_set_controls(dd4dv_ctx* ctx, const double* w_all, int device_ptrs);

/* Subdomain pt-steps of one evaluation: sum_s nx_s ny_s (b_s - a_s). */
dd4dv_status dd4dv_pt_steps(const dd4dv_ctx* ctx, long long* n);

/* Number of this library's kernel launches on the context since it was
 * created (cumulative; take differences around a region to count it). */
dd4dv_status dd4dv_launch_count(const dd4dv_ctx* ctx, long long* n);

/* Kernel timing (diagnostics): evaluates J and grad J at w_all (host,
 * packed) reps times after one warm-up and returns in ms[4] the mean
 * duration of one forward-sweep launch, one adjoint-sweep launch, one whole
 * evaluation (all kernels of dd4dv_eval) and the number of kernels in one
 * evaluation; durations come from CUDA events recorded on the context's
 * stream around each launch. */
dd4dv_status dd4dv_profile_sweeps(dd4dv_ctx* ctx, const double* w_all, int reps, double* ms);

/* Launch shapes of the sweeps, shape[5] = {forward cluster size, forward
 * threads per CTA, adjoint cluster size, adjoint threads per CTA, stored stage
 * states (1) or recomputed (0)}; eval_ms (after autotuning, else 0) = the
 * measured forward + adjoint time of those shapes.  Either pointer may be NULL. */
dd4dv_status dd4dv_sweep_config(const dd4dv_ctx* ctx, int* shape, double* eval_ms);

/* Force launch shapes (e.g. ones an earlier autotuning run reported), same
 * layout as dd4dv_sweep_config: cluster sizes 1..16 (<= smallest box height),
 * threads a multiple of 32 in 64..1024 (the stripe sweeps take at most 1024,
 * 384 for the FP32-state forward; the deep-halo FP32 sweeps at most 640, see
 * dd4dv_set_sweep_variant), stored stages 1 only with ckpt_k = 0 and the
 * stage buffer present; DD4DV_EINVAL for a shape no kernel can run.  Results
 * are the same for every shape up to the order of the partial sums of J. */
dd4dv_status dd4dv_set_sweep_config(dd4dv_ctx* ctx, const int* shape);

/* Trajectory storage the evaluations use: *k = 0 stored stage states,
 * -1 stages recomputed, -3 x1 stored for some or all subdomains, k > 0
 * checkpoints every k levels (ckpt_k of dd4dv_decomp, or the choice made for
 * ckpt_k = -2); eval_ms (may be NULL) = the evaluation time measured for that
 * choice (0 unless ckpt_k = -2). */
dd4dv_status dd4dv_checkpoint_interval(const dd4dv_ctx* ctx, int* k, double* eval_ms);

/* Subdomains whose first RK3 stage state is stored (ckpt_k = -3, or 0 when
 * both stage states do not fit), and their share of the pt-steps of an
 * evaluation; 0 and 0.0 otherwise.  Either pointer may be NULL.  ESTATE
 * before dd4dv_set_decomposition. */
dd4dv_status dd4dv_stage1_stored(const dd4dv_ctx* ctx, int* n_subs, double* pt_step_share);

/* Sweep kernels (FP32-state path).  The library has two forms of the forward
 * and adjoint sweeps.  The stripe sweeps exchange one halo row between the
 * CTAs of a subdomain after every RK3 stage.  The deep-halo sweeps (FP32
 * state only) keep three halo rows, recompute the two rows next to each
 * neighbour edge in the first two stages and exchange once per step; they
 * run where every CTA stripe has at least 3 rows, a thread holds at most 4
 * own points and (adjoint) the stage states are stored (ckpt_k = 0, no
 * Gauss-Newton or external forcing).  Both give the same values bit for bit.
 * The stripe adjoint also has a four-buffer form (any precision): mu2 (the
 * adjoint of the second RK3 stage) takes the buffer of x(n) and x(n) is read
 * again from HBM for the last phase of the step, so a CTA needs four state
 * buffers in shared memory instead of five; same values bit for bit, one more
 * state read per step.  It lets larger stripes (fewer CTAs per subdomain) or
 * more CTAs per SM fit.
 * The stripe forward also has a two-buffer form: x2 is written over x(n)
 * and the last stage reads x(n) from the trajectory level stored the step
 * before (every level stored: ckpt_k 0, -1 or -3), so two CTAs per SM fit where
 * three buffers fit one; same values bit for bit.
 * forward: 0 = deep-halo sweep wherever it applies (default), 1 = stripe
 * sweep only, 2 = the two-buffer stripe forward where it applies (else as
 * 1).  adjoint: 0 and 1 as for the forward (the stripe adjoint takes its
 * four-buffer form where five buffers do not fit), 2 = the four-buffer
 * stripe adjoint.  EINVAL for other values.  The autotuner (cluster = -1 in
 * dd4dv_decomp) times every form that applies and keeps the fastest one for
 * each sweep; dd4dv_sweep_kernels reports which run. */
dd4dv_status dd4dv_set_sweep_variant(dd4dv_ctx* ctx, int forward, int adjoint);

/* Which kernels the current launch shapes run: kinds[0] forward, kinds[1]
 * adjoint; 1 = stripe sweep, 2 = deep-halo sweep, 3 = four-buffer stripe
 * adjoint, 4 = two-buffer stripe forward. */
dd4dv_status dd4dv_sweep_kernels(const dd4dv_ctx* ctx, int* kinds);

/* The cluster size (CTAs per subdomain) the sweeps use. */
dd4dv_status dd4dv_cluster_size(const dd4dv_ctx* ctx, int* n);

/* Global model run for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is an interface variant of dd4dv_forward.
 * Some callers cannot call cudaMalloc: a framework whose caching allocator
 * already holds the free device memory, code that may not allocate after
 * start-up, or a thread that must not trigger the device-wide
 * synchronisation cudaMalloc/cudaFree can cause.  dd4dv_create allocates, so
 * those callers cannot use dd4dv_forward; this call needs no context and
 * makes no cudaMalloc, cudaFree or other allocating call.
 *   model: as for dd4dv_create (precision and h_ref are ignored: FP64).
 *   x0: device pointer, [3][nlat][nlon] initial state.
 *   traj: device pointer, [nsteps+1][3][nlat][nlon] output (caller-owned).
 *   cuda_stream: cudaStream_t to order the work on (NULL = legacy stream).
 *     The call enqueues the whole run on that stream (a kernel that computes
 *     the grid constants, then the RK3 stages) and returns without waiting:
 *     it makes no host copy and no stream or device synchronisation.
 * Limit: 3*nlat*nlon <= 393216 doubles (e.g. 512 x 256 points) and
 * nlat <= 1024; larger grids return DD4DV_EINVAL.  Errors: EINVAL, ECUDA;
 * the message is dd4dv_last_error(NULL).
 * Scratch: the two RK3 stage states and the grid constants live in a fixed
 * 6.3 MB __device__ array of the library that every GPU which loads the
 * library keeps until the process exits.  The first call on a device (with
 * that device current) looks up the array's device address and keeps it for
 * the life of the process; make that first call before any stream capture.
 * A device reset (cudaDeviceReset) after it is not supported.  All calls on
 * a device share the array, so calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be ordered by the caller. */
dd4dv_status dd4dv_forward_noalloc(const dd4dv_model* model, const double* x0, double* traj,
                                   void* cuda_stream);

/* Message of the last error on this context (library-owned, valid until the
 * next call on the context); ctx == NULL gives the message of the calling
 * thread's last dd4dv_create or dd4dv_forward_noalloc call. */
const char* dd4dv_last_error(const dd4dv_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DD4DVAR_H */
