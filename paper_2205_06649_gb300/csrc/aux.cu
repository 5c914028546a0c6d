// Auxiliary kernels of the DD-4DVar library: the control transform V and its
// transpose (Sec. 4, Eq. EqV), the background term and J assembly (Sec. 3.3,
// Eq. eq:cost:parallel1), the overlap exchange (Algorithm 1 "Exchange", Eq.
// rest), the global model (Sec. 7), the observation operator H, and the
// batched local L-BFGS (Algorithm 2/3 with L-BFGS, Remark after Alg. 5).
#include "common.cuh"

#include <cfloat>
#include <mutex>
#include <set>
#include <utility>

namespace dd4dv {

namespace {

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Deterministic block sum (fixed shuffle tree, warps in order); result valid
// in every thread.
__device__ double block_sum(double x, double* sh) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w];
    sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

__device__ __forceinline__ bool is_active(const int* active, int value, int s) {
  return active == nullptr || active[s] == value;
}

// ---------------------------------------------------------------------------
// Recursive filter L_1D = c (F^T F)^N on lines of each [3][ny][nx] block:
// F: q_i = alpha q_(i-1) + (1-alpha) p_i from a zero start, F^T the same
// recursion run backwards; zero values beyond the box edges.
__device__ void rf_line(double* x, int n, int stride, double alpha, double c, int npass) {
  const double b = 1.0 - alpha;
  for (int p = 0; p < npass; ++p) {
    double q = 0.0;
    for (int i = 0; i < n; ++i) {
      q = alpha * q + b * x[(size_t)i * stride];
      x[(size_t)i * stride] = q;
    }
    q = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      q = alpha * q + b * x[(size_t)i * stride];
      x[(size_t)i * stride] = q;
    }
  }
  for (int i = 0; i < n; ++i) x[(size_t)i * stride] *= c;
}

__global__ void rf_rows_kernel(double* x, RFArgs a) {
  const int s = blockIdx.y;
  if (!is_active(a.active, a.active_value, s)) return;
  const SubDesc d = a.subs[s];
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= 3 * d.ny) return;
  rf_line(x + d.ctrl_off + (size_t)line * d.nx, d.nx, 1, a.alpha, a.c, a.npass);
}

__global__ void rf_cols_kernel(double* x, RFArgs a) {
  const int s = blockIdx.y;
  if (!is_active(a.active, a.active_value, s)) return;
  const SubDesc d = a.subs[s];
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= 3 * d.nx) return;
  const int v = line / d.nx, k = line - v * d.nx;
  rf_line(x + d.ctrl_off + (size_t)v * d.ny * d.nx + k, d.ny, d.nx, a.alpha, a.c, a.npass);
}

// x(a) = x_b(a) + diag(sigma) vw  -> trajectory level 0 (h - h_ref on FP32).
template <typename T>
__global__ void init_state_kernel(const SubDesc* subs, const double* xb_a, const double* vw,
                                  const double* sigma, int scale_sigma, double h_ref, T* traj,
                                  const int* active, int active_value) {
  const int s = blockIdx.y;
  if (!is_active(active, active_value, s)) return;
  const SubDesc d = subs[s];
  const int npt = 3 * d.ny * d.nx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npt; i += gridDim.x * blockDim.x) {
    const int v = i / (d.ny * d.nx);
    const int rem = i - v * d.ny * d.nx;
    const int r = rem / d.nx, k = rem - r * d.nx;
    double x = xb_a[d.ctrl_off + i] + (scale_sigma ? sigma[v] : 1.0) * vw[d.ctrl_off + i];
    if (v == 0) x -= h_ref;
    traj[d.traj_off + ((size_t)v * d.ny + r) * d.nxp + k] = (T)x;
  }
}

__global__ void scale_copy_kernel(const SubDesc* subs, const double* in, const double* sigma,
                                  double* out, const int* active, int active_value) {
  const int s = blockIdx.y;
  if (!is_active(active, active_value, s)) return;
  const SubDesc d = subs[s];
  const int npt = 3 * d.ny * d.nx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npt; i += gridDim.x * blockDim.x) {
    const int v = i / (d.ny * d.nx);
    out[d.ctrl_off + i] = (sigma ? sigma[v] : 1.0) * in[d.ctrl_off + i];
  }
}

// grad = scale_s * (w + V^T y)   (w may be null: grad = scale_s V^T y)
__global__ void grad_finish_kernel(const SubDesc* subs, const double* w, const double* vty,
                                   const double* scale, double* grad, const int* active,
                                   int active_value) {
  const int s = blockIdx.y;
  if (!is_active(active, active_value, s)) return;
  const SubDesc d = subs[s];
  const double sc = scale ? scale[s] : 1.0;
  const int npt = 3 * d.ny * d.nx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npt; i += gridDim.x * blockDim.x) {
    const size_t o = d.ctrl_off + i;
    const double gv = (w ? w[o] : 0.0) + vty[o];
    grad[o] = scale ? sc * gv : gv;
  }
}

// J_s = 1/2 w.w + lambda J_o + mu (J_mu + overlap constant)
__global__ void finalize_J_kernel(const SubDesc* subs, const double* w, const double* part, int ncl,
                                  const double* vconst, double lam, double mu, double* J,
                                  double* parts, const int* active, int active_value) {
  __shared__ double sh[33];
  const int s = blockIdx.x;
  if (!is_active(active, active_value, s)) return;
  const SubDesc d = subs[s];
  const int npt = 3 * d.ny * d.nx;
  double acc = 0.0;
  for (int i = threadIdx.x; i < npt; i += blockDim.x) {
    const double x = w[d.ctrl_off + i];
    acc += x * x;
  }
  const double ww = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    double Jo = 0.0, Jm = 0.0;
    for (int r = 0; r < ncl; ++r) {
      Jo += part[((size_t)s * 16 + r) * 2 + 0];   // stride: SweepArgs::cl_max = 16
      Jm += part[((size_t)s * 16 + r) * 2 + 1];
    }
    Jm += vconst[s];
    const double Jb = 0.5 * ww;
    J[s] = Jb + lam * Jo + mu * Jm;
    if (parts) {
      parts[3 * s + 0] = Jb;
      parts[3 * s + 1] = Jo;
      parts[3 * s + 2] = Jm;
    }
  }
}

// ---------------------------------------------------------------------------
// Exchange.  Overlap targets: for every point a subdomain shares with others,
// the mean m of the other subdomains' values, and the constant
// 1/2 sum_nb sum_v (x_nb - m)^2 / sb^2 so that the overlap term is
// 1/2 sum_v [c (x - m)^2 / sb^2] + constant (exact rewriting of
// 1/2 sum_nb (x - x_nb)^2 / sb^2).
template <typename T>
__global__ void targets_kernel(ExchArgs<T> a) {
  __shared__ double sh[33];
  const int s = blockIdx.y;
  const SubDesc d = a.subs[s];
  const int L = d.b - d.a;
  const long long npt = (long long)(L + 1) * d.ny * d.nx;
  double vacc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < npt;
       idx += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(idx / ((long long)d.ny * d.nx));
    const int rem = (int)(idx - (long long)l * d.ny * d.nx);
    const int r = rem / d.nx, k = rem - r * d.nx;
    const int t0 = (l < d.tA) ? -1 : 0, t1 = (l > L - d.tB) ? 1 : 0;
    const int y0 = (r < d.wS) ? -1 : 0, y1 = (r >= d.ny - d.wN) ? 1 : 0;
    const int x0 = (k < d.wL) ? -1 : 0, x1 = (k >= d.nx - d.wR) ? 1 : 0;
    const int c = (t1 - t0 + 1) * (y1 - y0 + 1) * (x1 - x0 + 1) - 1;
    if (c == 0) continue;
    const int n = d.a + l, gj = d.j0 + r, gi = (d.i0 + k) % a.nlon;
    double sum[3] = {0.0, 0.0, 0.0};
    for (int pass = 0; pass < 2; ++pass) {
      double m[3];
      if (pass == 1)
        for (int v = 0; v < 3; ++v) m[v] = sum[v] / c;
      for (int dq = t0; dq <= t1; ++dq)
        for (int dy = y0; dy <= y1; ++dy)
          for (int dx = x0; dx <= x1; ++dx) {
            if (dq == 0 && dy == 0 && dx == 0) continue;
            const int t = ((d.q + dq) * a.P2 + (d.p2 + dy)) * a.P1 + (d.p1 + dx + a.P1) % a.P1;
            const SubDesc e = a.subs[t];
            const int lt = n - e.a, rt = gj - e.j0, kt = (gi - e.i0 + a.nlon) % a.nlon;
            const T* src = a.traj + e.traj_off + (size_t)lt * 3 * e.ny * e.nxp;
            for (int v = 0; v < 3; ++v) {
              const double xv = (double)src[((size_t)v * e.ny + rt) * e.nxp + kt];
              if (pass == 0) {
                sum[v] += xv;
              } else {
                const double dv = xv - m[v];
                vacc += dv * dv * a.isb2[v];
              }
            }
          }
      if (pass == 1) {
        T* dst = a.tgt + d.traj_off + (size_t)l * 3 * d.ny * d.nxp;
        for (int v = 0; v < 3; ++v) dst[((size_t)v * d.ny + r) * d.nxp + k] = (T)m[v];
      }
    }
  }
  const double tot = block_sum(vacc, sh);
  if (threadIdx.x == 0) a.vpart[(size_t)s * gridDim.x + blockIdx.x] = 0.5 * tot;
}

__global__ void sum_vconst_kernel(const double* vpart, int n_sub, int vblocks, double* vconst) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sub) return;
  double acc = 0.0;
  for (int b = 0; b < vblocks; ++b) acc += vpart[(size_t)s * vblocks + b];
  vconst[s] = acc;
}

// Assembled boundary trajectory: B(n, v, j, i) = mean over the covering
// subdomains (partition-of-unity weights 1/count, Eq. rest).
template <typename T>
__global__ void assemble_kernel(ExchArgs<T> a) {
  const long long plane = (long long)a.nlat * a.nlon;
  const long long total = (long long)(a.nsteps + 1) * 3 * plane;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(idx / (3 * plane));
    const long long rem = idx - (long long)n * 3 * plane;
    const int v = (int)(rem / plane);
    const int jr = (int)(rem - (long long)v * plane);
    const int j = jr / a.nlon, i = jr - j * a.nlon;
    double sum = 0.0;
    int cnt = 0;
    for (int tq = 0; tq < 2; ++tq) {
      const int q = a.t_cov[(n * 2 + tq) * 2], l = a.t_cov[(n * 2 + tq) * 2 + 1];
      if (q < 0) continue;
      for (int ty = 0; ty < 2; ++ty) {
        const int p2 = a.lat_cov[(j * 2 + ty) * 2], r = a.lat_cov[(j * 2 + ty) * 2 + 1];
        if (p2 < 0) continue;
        for (int tx = 0; tx < 2; ++tx) {
          const int p1 = a.lon_cov[(i * 2 + tx) * 2], k = a.lon_cov[(i * 2 + tx) * 2 + 1];
          if (p1 < 0) continue;
          const SubDesc e = a.subs[(q * a.P2 + p2) * a.P1 + p1];
          sum += (double)a.traj[e.traj_off + (((size_t)l * 3 + v) * e.ny + r) * e.nxp + k];
          ++cnt;
        }
      }
    }
    a.bnd[idx] = (T)(sum / cnt);
  }
}

// Restriction of a global FP64 trajectory to every subdomain's window x box,
// for the global levels g0..g1 that `glob` holds (level g0 first).
template <typename T>
__global__ void restrict_kernel(const SubDesc* subs, int nlon, int nlat, const double* glob, int g0,
                                double h_ref, T* traj) {
  const int s = blockIdx.z;
  const SubDesc d = subs[s];
  const int n = g0 + (int)blockIdx.y;
  if (n < d.a || n > d.b) return;
  const int l = n - d.a;
  const int npt = 3 * d.ny * d.nx;
  const size_t plane = (size_t)nlat * nlon;
  const double* src = glob + (size_t)blockIdx.y * 3 * plane;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npt; i += gridDim.x * blockDim.x) {
    const int v = i / (d.ny * d.nx);
    const int rem = i - v * d.ny * d.nx;
    const int r = rem / d.nx, k = rem - r * d.nx;
    double x = src[((size_t)v * nlat + d.j0 + r) * nlon + (d.i0 + k) % nlon];
    if (v == 0) x -= h_ref;
    traj[d.traj_off + (((size_t)l * 3 + v) * d.ny + r) * d.nxp + k] = (T)x;
  }
}

template <typename T>
__global__ void export_traj_kernel(const SubDesc* subs, const T* traj, double h_ref, double* out) {
  const int s = blockIdx.z;
  const SubDesc d = subs[s];
  const int l = blockIdx.y;
  if (l > d.b - d.a) return;
  const int npt = 3 * d.ny * d.nx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npt; i += gridDim.x * blockDim.x) {
    const int v = i / (d.ny * d.nx);
    const int rem = i - v * d.ny * d.nx;
    const int r = rem / d.nx, k = rem - r * d.nx;
    double x = (double)traj[d.traj_off + (((size_t)l * 3 + v) * d.ny + r) * d.nxp + k];
    if (v == 0) x += h_ref;
    out[d.ptraj_off + (size_t)l * npt + i] = x;
  }
}

__global__ void restrict_level_kernel(const SubDesc* subs, int nlon, int nlat, const double* glob,
                                      int g0, int g1, double* xb_a) {
  const int s = blockIdx.y;
  const SubDesc d = subs[s];
  if (d.a < g0 || d.a > g1) return;
  const int npt = 3 * d.ny * d.nx;
  const size_t plane = (size_t)nlat * nlon;
  const double* src = glob + (size_t)(d.a - g0) * 3 * plane;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npt; i += gridDim.x * blockDim.x) {
    const int v = i / (d.ny * d.nx);
    const int rem = i - v * d.ny * d.nx;
    const int r = rem / d.nx, k = rem - r * d.nx;
    xb_a[d.ctrl_off + i] = src[((size_t)v * nlat + d.j0 + r) * nlon + (d.i0 + k) % nlon];
  }
}

template <typename T>
__global__ void bnd_from_global_kernel(const double* glob, long long n, double h_ref, long long plane,
                                       T* bnd) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)((i / plane) % 3);
    bnd[i] = (T)(glob[i] - (v == 0 ? h_ref : 0.0));
  }
}

template <typename T>
__global__ void bnd_to_global_kernel(const T* bnd, long long n, double h_ref, long long plane,
                                     double* glob) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)((i / plane) % 3);
    glob[i] = (double)bnd[i] + (v == 0 ? h_ref : 0.0);
  }
}

// ---------------------------------------------------------------------------
// Global model stage on the whole sphere: out = ca x + cb (y + dt F(y)).
__global__ void global_stage_kernel(const double* x, const double* y, double* out, double ca,
                                    double cb, const RowConst* rows, double Bth, double gBth,
                                    double dt, int nlon, int nlat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nlon) return;
  const size_t P = (size_t)nlat * nlon;
  const double* H = y;
  const double* U = y + P;
  const double* V = y + 2 * P;
  const int iE = (i + 1) % nlon, iW = (i - 1 + nlon) % nlon;
  const size_t o = (size_t)j * nlon + i;
  const RowConst rc = rows[j];
  const double h = H[o], u = U[o], v = V[o];
  const double hE = H[(size_t)j * nlon + iE], hW = H[(size_t)j * nlon + iW];
  const double uE = U[(size_t)j * nlon + iE], uW = U[(size_t)j * nlon + iW];
  const double vE = V[(size_t)j * nlon + iE], vW = V[(size_t)j * nlon + iW];
  double hN, uN, vN, cN, hS, uS, vS, cS;
  if (j + 1 < nlat) {
    const size_t q = (size_t)(j + 1) * nlon + i;
    hN = H[q]; uN = U[q]; vN = V[q]; cN = rows[j + 1].c;
  } else {
    hN = h; uN = u; vN = -v; cN = rc.c;
  }
  if (j > 0) {
    const size_t q = (size_t)(j - 1) * nlon + i;
    hS = H[q]; uS = U[q]; vS = V[q]; cS = rows[j - 1].c;
  } else {
    hS = h; uS = u; vS = -v; cS = rc.c;
  }
  const double fu = rc.f + rc.tau * u;
  const double Fu = -rc.A * u * (uE - uW) - Bth * v * (uN - uS) + fu * v - rc.gA * (hE - hW);
  const double Fv = -rc.A * u * (vE - vW) - Bth * v * (vN - vS) - fu * u - gBth * (hN - hS);
  const double Fh = -rc.A * (hE * uE - hW * uW) - rc.BinvC * (hN * vN * cN - hS * vS * cS);
  const double F[3] = {Fh, Fu, Fv};
  for (int c = 0; c < 3; ++c) {
    const size_t q = (size_t)c * P + o;
    out[q] = (ca == 0.0 ? 0.0 : ca * x[q]) + cb * (y[q] + dt * F[c]);
  }
}

// H: bilinear interpolation in index space (lon periodic), corners in the
// order (j0,i0), (j0,i1), (j1,i0), (j1,i1), zero-weight corners skipped.
// `traj` holds the global levels g0..g1; observations at other levels are
// left untouched.
__global__ void observe_kernel(const double* traj, int g0, int g1, long long n, const int* level,
                               const int* var, const double* fi, const double* fj, int nlon, int nlat,
                               double* out) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (level[k] < g0 || level[k] > g1) continue;
    const double x = fi[k], y = fj[k];
    const int i0 = (int)floor(x), j0 = (int)floor(y);
    const double di = x - i0, dj = y - j0;
    const int i1 = (i0 + 1) % nlon;
    const size_t P = (size_t)nlat * nlon;
    const double* src = traj + ((size_t)(level[k] - g0) * 3 + var[k]) * P;
    double acc = 0.0;
    acc += ((1.0 - dj) * (1.0 - di)) * src[(size_t)j0 * nlon + i0 % nlon];
    if (di != 0.0) acc += ((1.0 - dj) * di) * src[(size_t)j0 * nlon + i1];
    if (dj != 0.0) {
      acc += (dj * (1.0 - di)) * src[(size_t)(j0 + 1) * nlon + i0 % nlon];
      if (di != 0.0) acc += (dj * di) * src[(size_t)(j0 + 1) * nlon + i1];
    }
    out[k] = acc;
  }
}

// ---------------------------------------------------------------------------
// Batched L-BFGS, one block per subdomain (fixed-order block reductions).
__device__ double dot(const double* x, const double* y, int n, double* sh) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * y[i];
  return block_sum(acc, sh);
}

__global__ void lb_start_kernel(LbArgs a) {
  __shared__ double sh[33];
  const int s = blockIdx.x;
  const SubDesc d = a.subs[s];
  const int n = 3 * d.ny * d.nx;
  const double* g = a.g + d.ctrl_off;
  const double gg = dot(g, g, n, sh);
  if (threadIdx.x == 0) {
    LbState st;
    st.J = a.J_eval[s];
    st.Jt = st.J;
    st.gp = 0.0;
    st.g0n = sqrt(gg);
    st.gn = st.g0n;
    st.head = 0;
    st.count = 0;
    st.iter = 0;
    st.trial = 0;
    st.alpha = 1.0;
    st.phase = (st.g0n > 0.0) ? 0 : 2;
    st.status = (st.g0n > 0.0) ? 0 : 1;
    if (a.owned && !a.owned[s]) {   // solved by another context: done from the start
      st.phase = 2;
      st.status = 4;
    }
    a.st[s] = st;
    a.phase[s] = st.phase;
  }
}

// Stop test, then the two-loop recursion p = -H g and the first trial point.
// The state is read once into shared memory; only thread 0 writes it back.
__global__ void lb_direction_kernel(LbArgs a) {
  __shared__ double sh[33];
  __shared__ double alph[16];
  __shared__ LbState ls;
  __shared__ int stop;
  const int s = blockIdx.x;
  if (threadIdx.x == 0) {
    ls = a.st[s];
    stop = 0;
    if (ls.phase != 0) {
      stop = 1;
    } else if (ls.gn / ls.g0n < a.gtol) {
      ls.phase = 2; ls.status = 1; stop = 2;
    } else if (ls.iter >= a.max_iter) {
      ls.phase = 2; ls.status = 2; stop = 2;
    }
    if (stop == 2) {
      a.st[s] = ls;
      a.phase[s] = ls.phase;
    }
  }
  __syncthreads();
  if (stop) return;
  const SubDesc d = a.subs[s];
  const int n = 3 * d.ny * d.nx;
  const size_t off = d.ctrl_off;
  const double* g = a.g + off;
  double* p = a.p + off;
  const int cnt = ls.count, m = a.m, head = ls.head;
  if (cnt == 0) {
    const double inv = 1.0 / ls.gn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = -g[i] * inv;
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = g[i];   // q
    __syncthreads();
    for (int c = 0; c < cnt; ++c) {          // newest to oldest
      const int slot = (head - 1 - c + 2 * m) % m;
      const double* S = a.S + (size_t)slot * a.total + off;
      const double* Y = a.Y + (size_t)slot * a.total + off;
      const double al = a.rho[s * m + slot] * dot(S, p, n, sh);
      if (threadIdx.x == 0) alph[slot] = al;
      for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] -= al * Y[i];
      __syncthreads();
    }
    const int newest = (head - 1 + m) % m;
    const double* Sn = a.S + (size_t)newest * a.total + off;
    const double* Yn = a.Y + (size_t)newest * a.total + off;
    const double sy = dot(Sn, Yn, n, sh);
    const double yy = dot(Yn, Yn, n, sh);
    const double gamma = sy / yy;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] *= gamma;
    __syncthreads();
    for (int c = cnt - 1; c >= 0; --c) {     // oldest to newest
      const int slot = (head - 1 - c + 2 * m) % m;
      const double* S = a.S + (size_t)slot * a.total + off;
      const double* Y = a.Y + (size_t)slot * a.total + off;
      const double beta = a.rho[s * m + slot] * dot(Y, p, n, sh);
      const double al = alph[slot];
      for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] += (al - beta) * S[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = -p[i];
  }
  __syncthreads();
  double gp = dot(g, p, n, sh);
  int cleared = 0;
  if (!(gp < 0.0)) {      // not a descent direction: steepest descent, clear memory
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = -g[i];
    __syncthreads();
    gp = -ls.gn * ls.gn;
    cleared = 1;
  }
  const double* w = a.w + off;
  double* wt = a.wt + off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) wt[i] = w[i] + p[i];
  if (threadIdx.x == 0) {
    if (cleared) ls.count = 0;
    ls.gp = gp;
    ls.alpha = 1.0;
    ls.trial = 0;
    ls.phase = 1;
    a.st[s] = ls;
    a.phase[s] = 1;
    atomicAdd(&a.counter[0], 1);
  }
}

// Armijo test at the trial point; accept (update memory) or halve the step.
__global__ void lb_linesearch_kernel(LbArgs a) {
  __shared__ double sh[33];
  __shared__ LbState ls;
  const int s = blockIdx.x;
  if (threadIdx.x == 0) ls = a.st[s];
  __syncthreads();
  if (ls.phase != 1) return;
  const SubDesc d = a.subs[s];
  const int n = 3 * d.ny * d.nx;
  const size_t off = d.ctrl_off;
  const double Jt = a.J_eval[s];
  const bool accept = Jt <= ls.J + a.c1 * ls.alpha * ls.gp;
  double* w = a.w + off;
  double* g = a.g + off;
  double* wt = a.wt + off;
  const double* gt = a.gt + off;
  const double* p = a.p + off;
  if (accept) {
    const int m = a.m, slot = ls.head;
    double* S = a.S + (size_t)slot * a.total + off;
    double* Y = a.Y + (size_t)slot * a.total + off;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      S[i] = wt[i] - w[i];
      Y[i] = gt[i] - g[i];
    }
    __syncthreads();
    const double sy = dot(S, Y, n, sh);
    const double ss = dot(S, S, n, sh);
    const double yy = dot(Y, Y, n, sh);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      w[i] = wt[i];
      g[i] = gt[i];
    }
    const double gg = dot(gt, gt, n, sh);
    if (threadIdx.x == 0) {
      if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
        a.rho[s * m + slot] = 1.0 / sy;
        ls.head = (slot + 1) % m;
        ls.count = min(ls.count + 1, m);
      }
      ls.J = Jt;
      ls.gn = sqrt(gg);
      ls.iter += 1;
      ls.phase = 0;
      a.st[s] = ls;
      a.phase[s] = 0;
      atomicAdd(&a.counter[1], 1);
    }
  } else {
    const double al = 0.5 * ls.alpha;
    if (ls.trial + 1 >= a.max_trials) {
      if (threadIdx.x == 0) {
        ls.phase = 2;
        ls.status = 3;
        a.st[s] = ls;
        a.phase[s] = 2;
      }
      return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) wt[i] = w[i] + al * p[i];
    if (threadIdx.x == 0) {
      ls.alpha = al;
      ls.trial += 1;
      a.st[s] = ls;
      atomicAdd(&a.counter[0], 1);
    }
  }
}

__global__ void max_abs_diff_kernel(const double* a, const double* b, long long n,
                                    unsigned long long* out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i] - b[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void finite_check_kernel(const double* a, long long n, int* flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) atomicExch(flag, 1);
}

// Fused control transform, one CTA per (subdomain, variable) with the
// variable's ny x nx plane staged in shared memory:
//   forward (V):   x(a) = x_b(a) + sigma_v L_lat L_lon w  -> trajectory level 0
//   adjoint (V^T): grad = scale_s (w + L_lon L_lat (sigma_v y))
// Rows (lon lines) are filtered by one thread per row, columns by one thread
// per column, in the same operation order as the separate kernels.  The
// filter runs in the state precision R: FP64 on the FP64 path; on the
// FP32-state path in FP32, since L w only feeds an initial state that is
// stored in FP32 and L^T acts on an adjoint state computed in FP32 (the
// control, x_b, w and the gradient stay FP64).
template <typename R>
__device__ void rf_line_smem(R* x, int n, int stride, R alpha, R c, int npass) {
  const R b = (R)1 - alpha;
  for (int p = 0; p < npass; ++p) {
    R q = (R)0;
    for (int i = 0; i < n; ++i) {
      q = alpha * q + b * x[i * stride];
      x[i * stride] = q;
    }
    q = (R)0;
    for (int i = n - 1; i >= 0; --i) {
      q = alpha * q + b * x[i * stride];
      x[i * stride] = q;
    }
  }
  for (int i = 0; i < n; ++i) x[i * stride] *= c;
}

extern __shared__ __align__(16) unsigned char smem_plane[];

template <typename T>
__global__ void vinit_kernel(const SubDesc* subs, const double* xb_a, const double* w, const double* sigma,
                             RFArgs rf, int use_rf, double h_ref, T* traj, const int* active,
                             int active_value) {
  T* pl = reinterpret_cast<T*>(smem_plane);
  const int s = blockIdx.x, v = blockIdx.y;
  if (!is_active(active, active_value, s)) return;
  const SubDesc d = subs[s];
  const int n = d.ny * d.nx;
  const int pitch = d.nx | 1;   // odd row pitch: row-wise passes are free of bank conflicts
  const double* src = w + d.ctrl_off + (size_t)v * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i / d.nx, k = i - r * d.nx;
    pl[r * pitch + k] = (T)src[i];
  }
  __syncthreads();
  if (use_rf) {
    const T al = (T)rf.alpha, c = (T)rf.c;
    for (int r = threadIdx.x; r < d.ny; r += blockDim.x) rf_line_smem(pl + r * pitch, d.nx, 1, al, c, rf.npass);
    __syncthreads();
    for (int k = threadIdx.x; k < d.nx; k += blockDim.x) rf_line_smem(pl + k, d.ny, pitch, al, c, rf.npass);
    __syncthreads();
  }
  const double sg = sigma[v];
  const double* xb = xb_a + d.ctrl_off + (size_t)v * n;
  T* dst = traj + d.traj_off + (size_t)v * d.ny * d.nxp;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i / d.nx, k = i - r * d.nx;
    double x = xb[i] + sg * (double)pl[r * pitch + k];
    if (v == 0) x -= h_ref;
    dst[(size_t)r * d.nxp + k] = (T)x;
  }
}

template <typename R>
__global__ void vgrad_kernel(const SubDesc* subs, const double* w, const double* y, const double* sigma,
                             RFArgs rf, int use_rf, const double* scale, double* grad, const int* active,
                             int active_value) {
  R* pl = reinterpret_cast<R*>(smem_plane);
  const int s = blockIdx.x, v = blockIdx.y;
  if (!is_active(active, active_value, s)) return;
  const SubDesc d = subs[s];
  const int n = d.ny * d.nx;
  const int pitch = d.nx | 1;
  const size_t o = d.ctrl_off + (size_t)v * n;
  const double sg = sigma[v];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i / d.nx, k = i - r * d.nx;
    pl[r * pitch + k] = (R)(sg * y[o + i]);
  }
  __syncthreads();
  if (use_rf) {
    const R al = (R)rf.alpha, c = (R)rf.c;
    for (int k = threadIdx.x; k < d.nx; k += blockDim.x) rf_line_smem(pl + k, d.ny, pitch, al, c, rf.npass);
    __syncthreads();
    for (int r = threadIdx.x; r < d.ny; r += blockDim.x) rf_line_smem(pl + r * pitch, d.nx, 1, al, c, rf.npass);
    __syncthreads();
  }
  const double sc = scale ? scale[s] : 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i / d.nx, k = i - r * d.nx;
    const double gv = (w ? w[o + i] : 0.0) + (double)pl[r * pitch + k];
    grad[o + i] = scale ? sc * gv : gv;
  }
}

// Raises a kernel's dynamic shared-memory cap to the 227 KB opt-in maximum,
// once per (kernel, device): the attribute belongs to the device current at
// the call, so a context on another device sets it again.
template <typename K>
cudaError_t raise_smem_cap(K kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const std::pair<const void*, int> key{reinterpret_cast<const void*>(kernel), dev};
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e != cudaSuccess) return e;
  done.insert(key);
  return cudaSuccess;
}

inline unsigned blocks_for(long long n, int t, int cap = 152 * 16) {
  long long b = (n + t - 1) / t;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

}  // namespace

template <typename T>
cudaError_t launch_vinit(const SubDesc* subs, int n_sub, const double* xb_a, const double* w,
                         const double* sigma, const RFArgs& rf, int use_rf, double h_ref, T* traj,
                         const int* active, int active_value, int max_plane, cudaStream_t st) {
  const size_t smem = (size_t)max_plane * sizeof(T);
  cudaError_t e = raise_smem_cap(vinit_kernel<T>);
  if (e != cudaSuccess) return e;
  vinit_kernel<T><<<dim3(n_sub, 3), 256, smem, st>>>(subs, xb_a, w, sigma, rf, use_rf, h_ref, traj, active,
                                                      active_value);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_vgrad(const SubDesc* subs, int n_sub, const double* w, const double* y, const double* sigma,
                         const RFArgs& rf, int use_rf, const double* scale, double* grad, const int* active,
                         int active_value, int max_plane, cudaStream_t st) {
  const size_t smem = (size_t)max_plane * sizeof(R);
  cudaError_t e = raise_smem_cap(vgrad_kernel<R>);
  if (e != cudaSuccess) return e;
  vgrad_kernel<R><<<dim3(n_sub, 3), 256, smem, st>>>(subs, w, y, sigma, rf, use_rf, scale, grad, active,
                                                     active_value);
  return cudaGetLastError();
}

cudaError_t launch_rf_rows(double* x, const RFArgs& a, int max_ny, cudaStream_t st) {
  dim3 grid((3 * max_ny + 127) / 128, a.n_sub);
  rf_rows_kernel<<<grid, 128, 0, st>>>(x, a);
  return cudaGetLastError();
}
cudaError_t launch_rf_cols(double* x, const RFArgs& a, int max_nx, cudaStream_t st) {
  dim3 grid((3 * max_nx + 127) / 128, a.n_sub);
  rf_cols_kernel<<<grid, 128, 0, st>>>(x, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_state(const SubDesc* subs, int n_sub, const double* xb_a, const double* vw,
                              const double* sigma, int scale_sigma, double h_ref, T* traj,
                              const int* active, int active_value, int max_pts, cudaStream_t st) {
  dim3 grid(blocks_for(max_pts, 256, 64), n_sub);
  init_state_kernel<T><<<grid, 256, 0, st>>>(subs, xb_a, vw, sigma, scale_sigma, h_ref, traj, active,
                                             active_value);
  return cudaGetLastError();
}
cudaError_t launch_scale_copy(const SubDesc* subs, int n_sub, const double* in, const double* sigma,
                              double* out, const int* active, int active_value, int max_pts,
                              cudaStream_t st) {
  dim3 grid(blocks_for(max_pts, 256, 64), n_sub);
  scale_copy_kernel<<<grid, 256, 0, st>>>(subs, in, sigma, out, active, active_value);
  return cudaGetLastError();
}
cudaError_t launch_grad_finish(const SubDesc* subs, int n_sub, const double* w, const double* vty,
                               const double* scale, double* grad, const int* active,
                               int active_value, int max_pts, cudaStream_t st) {
  dim3 grid(blocks_for(max_pts, 256, 64), n_sub);
  grad_finish_kernel<<<grid, 256, 0, st>>>(subs, w, vty, scale, grad, active, active_value);
  return cudaGetLastError();
}
cudaError_t launch_finalize_J(const SubDesc* subs, int n_sub, const double* w, const double* part,
                              int ncl, const double* vconst, double lam, double mu, double* J,
                              double* parts, const int* active, int active_value, cudaStream_t st) {
  finalize_J_kernel<<<n_sub, 256, 0, st>>>(subs, w, part, ncl, vconst, lam, mu, J, parts, active,
                                           active_value);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_targets(const ExchArgs<T>& a, cudaStream_t st) {
  dim3 grid(a.vblocks, a.n_sub);
  targets_kernel<T><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_assemble(const ExchArgs<T>& a, cudaStream_t st) {
  const long long total = (long long)(a.nsteps + 1) * 3 * a.nlat * a.nlon;
  assemble_kernel<T><<<blocks_for(total, 256, 152 * 32), 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_sum_vconst(const double* vpart, int n_sub, int vblocks, double* vconst,
                              cudaStream_t st) {
  sum_vconst_kernel<<<(n_sub + 127) / 128, 128, 0, st>>>(vpart, n_sub, vblocks, vconst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const SubDesc* subs, int n_sub, int nlon, int nlat, const double* glob,
                            int g0, int g1, double h_ref, T* traj, int max_pts, cudaStream_t st) {
  dim3 grid(blocks_for(max_pts, 256, 16), g1 - g0 + 1, n_sub);
  restrict_kernel<T><<<grid, 256, 0, st>>>(subs, nlon, nlat, glob, g0, h_ref, traj);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_export_traj(const SubDesc* subs, int n_sub, const T* traj, double h_ref,
                               double* out, int max_pts, int max_levels, cudaStream_t st) {
  dim3 grid(blocks_for(max_pts, 256, 16), max_levels, n_sub);
  export_traj_kernel<T><<<grid, 256, 0, st>>>(subs, traj, h_ref, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_bnd_from_global(const double* glob, long long n, double h_ref, int nlon, int nlat,
                                   T* bnd, cudaStream_t st) {
  bnd_from_global_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(glob, n, h_ref,
                                                                 (long long)nlon * nlat, bnd);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_bnd_to_global(const T* bnd, long long n, double h_ref, int nlon, int nlat,
                                 double* glob, cudaStream_t st) {
  bnd_to_global_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(bnd, n, h_ref,
                                                               (long long)nlon * nlat, glob);
  return cudaGetLastError();
}
cudaError_t launch_restrict_level(const SubDesc* subs, int n_sub, int nlon, int nlat, const double* glob,
                                  int g0, int g1, double* xb_a, int max_pts, cudaStream_t st) {
  dim3 grid(blocks_for(max_pts, 256, 64), n_sub);
  restrict_level_kernel<<<grid, 256, 0, st>>>(subs, nlon, nlat, glob, g0, g1, xb_a);
  return cudaGetLastError();
}

cudaError_t launch_global_stage(const double* x, const double* y, double* out, double ca, double cb,
                                const RowConst* rows, double Bth, double gBth, double dt, int nlon,
                                int nlat, cudaStream_t st) {
  dim3 grid((nlon + 127) / 128, nlat);
  global_stage_kernel<<<grid, 128, 0, st>>>(x, y, out, ca, cb, rows, Bth, gBth, dt, nlon, nlat);
  return cudaGetLastError();
}
cudaError_t launch_observe(const double* traj, int g0, int g1, long long n, const int* level,
                           const int* var, const double* fi, const double* fj, int nlon, int nlat,
                           double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  observe_kernel<<<blocks_for(n, 256), 256, 0, st>>>(traj, g0, g1, n, level, var, fi, fj, nlon, nlat,
                                                     out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conjugate gradients (Hestenes-Stiefel) on (I + G^T G) dw = -g per subdomain,
// the inner solve of the Gauss-Newton iteration (Algorithm 7 in the control
// variable).  The products A p come from the sweeps between the kernels.
__global__ void cg_start_kernel(CgArgs a) {
  __shared__ double sh[33];
  __shared__ int go;
  const int s = blockIdx.x;
  const SubDesc d = a.subs[s];
  const int n = 3 * d.ny * d.nx;
  const size_t off = d.ctrl_off;
  const double* g = a.g + off;
  const double gg = dot(g, g, n, sh);
  if (threadIdx.x == 0) {
    CgState c = a.st[s];
    if (a.first) c.g0n = sqrt(gg);
    c.rr = c.rr0 = gg;
    c.k = 0;
    const bool run = c.g0n > 0.0 && sqrt(gg) > a.gtol * c.g0n && gg > 0.0 && a.max_iter > 0;
    c.status = run ? 0 : 4;
    a.st[s] = c;
    a.phase[s] = run ? 1 : 0;
    if (run) atomicAdd(a.counter, 1);
    go = run;
  }
  __syncthreads();
  double* r = a.r + off;
  double* p = a.p + off;
  double* dw = a.dw + off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dw[i] = 0.0;
    if (go) {
      r[i] = -g[i];
      p[i] = -g[i];
    }
  }
}

__global__ void cg_step_kernel(CgArgs a) {
  __shared__ double sh[33];
  __shared__ double alpha, beta;
  __shared__ int mode;   // 0 skip, 1 update and continue, 2 update and stop
  const int s = blockIdx.x;
  if (a.phase[s] != 1) return;
  const SubDesc d = a.subs[s];
  const int n = 3 * d.ny * d.nx;
  const size_t off = d.ctrl_off;
  double* r = a.r + off;
  double* p = a.p + off;
  double* dw = a.dw + off;
  const double* Ap = a.Ap + off;
  const double pAp = dot(p, Ap, n, sh);
  if (threadIdx.x == 0) {
    CgState c = a.st[s];
    if (!(pAp > 0.0)) {
      c.status = 3;
      a.st[s] = c;
      a.phase[s] = 0;
      mode = 0;
    } else {
      alpha = c.rr / pAp;
      mode = 1;
    }
  }
  __syncthreads();
  if (mode == 0) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dw[i] += alpha * p[i];
    r[i] -= alpha * Ap[i];
  }
  const double rr1 = dot(r, r, n, sh);   // block_sum barriers order the updates above
  if (threadIdx.x == 0) {
    CgState c = a.st[s];
    c.k += 1;
    if (rr1 <= a.tol * a.tol * c.rr0) {
      c.status = 1;
      mode = 2;
    } else if (c.k >= a.max_iter) {
      c.status = 2;
      mode = 2;
    } else {
      beta = rr1 / c.rr;
      mode = 1;
      atomicAdd(a.counter, 1);
    }
    c.rr = rr1;
    a.st[s] = c;
    if (mode == 2) a.phase[s] = 0;
  }
  __syncthreads();
  if (mode != 1) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = r[i] + beta * p[i];
}

__global__ void axpy_kernel(double* y, const double* x, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

cudaError_t launch_cg_start(const CgArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  cg_start_kernel<<<a.n_sub, 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_cg_step(const CgArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  cg_step_kernel<<<a.n_sub, 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_axpy(double* y, const double* x, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  axpy_kernel<<<blocks_for(n, 256), 256, 0, st>>>(y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_lb_start(const LbArgs& a, cudaStream_t st) {
  lb_start_kernel<<<a.n_sub, 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_lb_direction(const LbArgs& a, cudaStream_t st) {
  lb_direction_kernel<<<a.n_sub, 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_lb_linesearch(const LbArgs& a, cudaStream_t st) {
  lb_linesearch_kernel<<<a.n_sub, 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_max_abs_diff(const double* a, const double* b, long long n, double* out,
                                cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  max_abs_diff_kernel<<<blocks_for(n, 256), 256, 0, st>>>(a, b, n,
                                                           reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}
cudaError_t launch_finite_check(const double* a, long long n, int* flag, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  finite_check_kernel<<<blocks_for(n, 256), 256, 0, st>>>(a, n, flag);
  return cudaGetLastError();
}

#define DD4DV_INST(T)                                                                              \
  template cudaError_t launch_vgrad<T>(const SubDesc*, int, const double*, const double*,           \
                                       const double*, const RFArgs&, int, const double*, double*,  \
                                       const int*, int, int, cudaStream_t);                        \
  template cudaError_t launch_vinit<T>(const SubDesc*, int, const double*, const double*,           \
                                       const double*, const RFArgs&, int, double, T*, const int*,  \
                                       int, int, cudaStream_t);                                    \
  template cudaError_t launch_init_state<T>(const SubDesc*, int, const double*, const double*,     \
                                            const double*, int, double, T*, const int*, int, int,  \
                                            cudaStream_t);                                         \
  template cudaError_t launch_targets<T>(const ExchArgs<T>&, cudaStream_t);                        \
  template cudaError_t launch_assemble<T>(const ExchArgs<T>&, cudaStream_t);                       \
  template cudaError_t launch_restrict<T>(const SubDesc*, int, int, int, const double*, int, int,  \
                                          double, T*, int, cudaStream_t);                          \
  template cudaError_t launch_export_traj<T>(const SubDesc*, int, const T*, double, double*, int,  \
                                             int, cudaStream_t);                                   \
  template cudaError_t launch_bnd_from_global<T>(const double*, long long, double, int, int, T*,   \
                                                 cudaStream_t);                                    \
  template cudaError_t launch_bnd_to_global<T>(const T*, long long, double, int, int, double*,     \
                                               cudaStream_t);
DD4DV_INST(double)
DD4DV_INST(float)
#undef DD4DV_INST

}  // namespace dd4dv
