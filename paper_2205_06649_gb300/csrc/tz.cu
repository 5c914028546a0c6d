// The Turkel-Zwas scheme of Sec. 7 on the whole sphere: forward RK3 stages,
// tangent-linear stages and the transposed (adjoint) stages, FP64, one thread
// per grid point, global memory.
//
// Scheme (Sec. 7, the semi-discrete U_ij, V_ij, H_ij with longitude stride
// p, latitude stride q and averaging weight alpha; readings of the garbled
// print as in the oracle): advection with stride 1, pressure gradients over
// i +- p and j +- q, Coriolis terms of the u (v) equation averaged over
// i +- p (j +- q) with weight alpha, and the divergence of the continuity
// equation averaged over the diagonal points (i +- p, j +- q) with weight
// alpha.  Longitude is periodic; the walls mirror (h, u, -v) to depth q
// (ghost row -1 - s holds row s, row nlat + s holds row nlat - 1 - s, with
// the mirrored row's cos, f and tan).
//
// The tangent-linear stage is built from one list of partial derivatives per
// point (tz_jacobian: for each value of the state that F at the point reads,
// d F_out / d value_in), and the adjoint stage applies the same list
// transposed, scattering coef * m_out(point) into value_in (FP64 atomic
// additions); the adjoint is therefore the exact transpose of the
// tangent-linear model up to the order of the additions.
#include "common.cuh"

namespace dd4dv {

namespace {

struct Loc {
  int j, i;
  double vs;   // -1 for v read through a wall mirror
};

__device__ __forceinline__ Loc tz_resolve(const TzArgs& t, int j, int i) {
  Loc L;
  L.i = ((i % t.nlon) + t.nlon) % t.nlon;
  L.vs = 1.0;
  if (j < 0) {
    L.j = -1 - j;
    L.vs = -1.0;
  } else if (j >= t.nlat) {
    L.j = 2 * t.nlat - 1 - j;
    L.vs = -1.0;
  } else {
    L.j = j;
  }
  return L;
}

__device__ __forceinline__ double tz_val(const TzArgs& t, const double* Y, int var, int j, int i) {
  const Loc L = tz_resolve(t, j, i);
  const double x = Y[((size_t)var * t.nlat + L.j) * t.nlon + L.i];
  return var == 2 ? L.vs * x : x;
}

// Semi-discrete Turkel-Zwas tendencies at (j, i):
//   F_u = -s_lon u/c (u[i+1] - u[i-1]) - s_lat v (u[j+1] - u[j-1]) - s_lon g/(p c) (h[i+p] - h[i-p])
//         + (1-alpha) C v + alpha/2 ((C v)[i+p] + (C v)[i-p])
//   F_v = -s_lon u/c (v[i+1] - v[i-1]) - s_lat v (v[j+1] - v[j-1]) - s_lat g/q (h[j+q] - h[j-q])
//         - (1-alpha) C u - alpha/2 ((C u)[j+q] + (C u)[j-q])
//   F_h = -{ s_lon u/c (h[i+1] - h[i-1]) + s_lat v (h[j+1] - h[j-1]) + s_lon h/(p c) Du + s_lat h/(q c) Dv }
//   Du = (1-alpha) (u[i+p] - u[i-p]) + alpha/2 (u[i+p,j+q] - u[i-p,j+q] + u[i+p,j-q] - u[i-p,j-q])
//   Dv = (1-alpha) ((v c)[j+q] - (v c)[j-q])
//        + alpha/2 ((v c)[i+p,j+q] - (v c)[i+p,j-q] + (v c)[i-p,j+q] - (v c)[i-p,j-q])
// with C = f + u tan(theta)/a at the point it multiplies (its own row's f, tan).
__device__ void tz_F(const TzArgs& t, const double* Y, int j, int i, double& Fh, double& Fu, double& Fv) {
  const int p = t.p, q = t.q;
  const double al = t.alpha, sl = t.slon, st = t.slat, g = t.g;
  const RowConst rc = t.rows[j];
  const double c = rc.c, f = rc.f, tau = rc.tau;
  const RowConst rN = t.rows[tz_resolve(t, j + q, i).j], rS = t.rows[tz_resolve(t, j - q, i).j];
  const double h = tz_val(t, Y, 0, j, i), u = tz_val(t, Y, 1, j, i), v = tz_val(t, Y, 2, j, i);
  const double C = f + u * tau;
  double cor_u = (1.0 - al) * C * v;
  double cor_v = (1.0 - al) * C * u;
  if (al != 0.0) {
    const double uEp = tz_val(t, Y, 1, j, i + p), uWp = tz_val(t, Y, 1, j, i - p);
    cor_u += 0.5 * al * ((f + uEp * tau) * tz_val(t, Y, 2, j, i + p) + (f + uWp * tau) * tz_val(t, Y, 2, j, i - p));
    const double uNq = tz_val(t, Y, 1, j + q, i), uSq = tz_val(t, Y, 1, j - q, i);
    cor_v += 0.5 * al * ((rN.f + uNq * rN.tau) * uNq + (rS.f + uSq * rS.tau) * uSq);
  }
  Fu = -sl * u / c * (tz_val(t, Y, 1, j, i + 1) - tz_val(t, Y, 1, j, i - 1)) -
       st * v * (tz_val(t, Y, 1, j + 1, i) - tz_val(t, Y, 1, j - 1, i)) -
       sl * g / (p * c) * (tz_val(t, Y, 0, j, i + p) - tz_val(t, Y, 0, j, i - p)) + cor_u;
  Fv = -sl * u / c * (tz_val(t, Y, 2, j, i + 1) - tz_val(t, Y, 2, j, i - 1)) -
       st * v * (tz_val(t, Y, 2, j + 1, i) - tz_val(t, Y, 2, j - 1, i)) -
       st * g / q * (tz_val(t, Y, 0, j + q, i) - tz_val(t, Y, 0, j - q, i)) - cor_v;
  double du = (1.0 - al) * (tz_val(t, Y, 1, j, i + p) - tz_val(t, Y, 1, j, i - p));
  double dv = (1.0 - al) * (tz_val(t, Y, 2, j + q, i) * rN.c - tz_val(t, Y, 2, j - q, i) * rS.c);
  if (al != 0.0) {
    du += 0.5 * al * (tz_val(t, Y, 1, j + q, i + p) - tz_val(t, Y, 1, j + q, i - p) +
                      tz_val(t, Y, 1, j - q, i + p) - tz_val(t, Y, 1, j - q, i - p));
    dv += 0.5 * al * (tz_val(t, Y, 2, j + q, i + p) * rN.c - tz_val(t, Y, 2, j - q, i + p) * rS.c +
                      tz_val(t, Y, 2, j + q, i - p) * rN.c - tz_val(t, Y, 2, j - q, i - p) * rS.c);
  }
  Fh = -(sl * u / c * (tz_val(t, Y, 0, j, i + 1) - tz_val(t, Y, 0, j, i - 1)) +
         st * v * (tz_val(t, Y, 0, j + 1, i) - tz_val(t, Y, 0, j - 1, i)) + sl * h / (p * c) * du +
         st * h / (q * c) * dv);
}

// Partial derivatives of (F_h, F_u, F_v) at (j, i) with respect to every
// state value they read: vis(out_var, in_var, row, col, coef) with the
// location resolved through the periodic wrap and the wall mirror (a v read
// through a mirror enters with the sign flipped).  Derived from tz_F term by
// term; a location read by several terms (p = 1 or q = 1) gets one entry
// per term.
template <typename Vis>
__device__ void tz_jacobian(const TzArgs& t, const double* Y, int j, int i, Vis&& vis) {
  const int p = t.p, q = t.q;
  const double al = t.alpha, sl = t.slon, st = t.slat, g = t.g;
  const RowConst rc = t.rows[j];
  const double c = rc.c, f = rc.f, tau = rc.tau;
  const RowConst rN = t.rows[tz_resolve(t, j + q, i).j], rS = t.rows[tz_resolve(t, j - q, i).j];
  auto emit = [&](int vo, int vi, int dj, int di, double coef) {
    const Loc L = tz_resolve(t, j + dj, i + di);
    vis(vo, vi, L.j, L.i, vi == 2 ? coef * L.vs : coef);
  };
  const double h = tz_val(t, Y, 0, j, i), u = tz_val(t, Y, 1, j, i), v = tz_val(t, Y, 2, j, i);
  const double C = f + u * tau;
  // F_u
  const double dux1 = tz_val(t, Y, 1, j, i + 1) - tz_val(t, Y, 1, j, i - 1);
  const double duy1 = tz_val(t, Y, 1, j + 1, i) - tz_val(t, Y, 1, j - 1, i);
  emit(1, 1, 0, 0, -sl / c * dux1 + (1.0 - al) * tau * v);
  emit(1, 1, 0, 1, -sl * u / c);
  emit(1, 1, 0, -1, sl * u / c);
  emit(1, 2, 0, 0, -st * duy1 + (1.0 - al) * C);
  emit(1, 1, 1, 0, -st * v);
  emit(1, 1, -1, 0, st * v);
  emit(1, 0, 0, p, -sl * g / (p * c));
  emit(1, 0, 0, -p, sl * g / (p * c));
  if (al != 0.0) {
    const double uEp = tz_val(t, Y, 1, j, i + p), vEp = tz_val(t, Y, 2, j, i + p);
    const double uWp = tz_val(t, Y, 1, j, i - p), vWp = tz_val(t, Y, 2, j, i - p);
    emit(1, 1, 0, p, 0.5 * al * tau * vEp);
    emit(1, 2, 0, p, 0.5 * al * (f + uEp * tau));
    emit(1, 1, 0, -p, 0.5 * al * tau * vWp);
    emit(1, 2, 0, -p, 0.5 * al * (f + uWp * tau));
  }
  // F_v
  const double dvx1 = tz_val(t, Y, 2, j, i + 1) - tz_val(t, Y, 2, j, i - 1);
  const double dvy1 = tz_val(t, Y, 2, j + 1, i) - tz_val(t, Y, 2, j - 1, i);
  emit(2, 1, 0, 0, -sl / c * dvx1 - (1.0 - al) * (f + 2.0 * u * tau));
  emit(2, 2, 0, 1, -sl * u / c);
  emit(2, 2, 0, -1, sl * u / c);
  emit(2, 2, 0, 0, -st * dvy1);
  emit(2, 2, 1, 0, -st * v);
  emit(2, 2, -1, 0, st * v);
  emit(2, 0, q, 0, -st * g / q);
  emit(2, 0, -q, 0, st * g / q);
  if (al != 0.0) {
    const double uNq = tz_val(t, Y, 1, j + q, i), uSq = tz_val(t, Y, 1, j - q, i);
    emit(2, 1, q, 0, -0.5 * al * (rN.f + 2.0 * uNq * rN.tau));
    emit(2, 1, -q, 0, -0.5 * al * (rS.f + 2.0 * uSq * rS.tau));
  }
  // F_h
  const double dhx1 = tz_val(t, Y, 0, j, i + 1) - tz_val(t, Y, 0, j, i - 1);
  const double dhy1 = tz_val(t, Y, 0, j + 1, i) - tz_val(t, Y, 0, j - 1, i);
  double du = (1.0 - al) * (tz_val(t, Y, 1, j, i + p) - tz_val(t, Y, 1, j, i - p));
  double dv = (1.0 - al) * (tz_val(t, Y, 2, j + q, i) * rN.c - tz_val(t, Y, 2, j - q, i) * rS.c);
  if (al != 0.0) {
    du += 0.5 * al * (tz_val(t, Y, 1, j + q, i + p) - tz_val(t, Y, 1, j + q, i - p) +
                      tz_val(t, Y, 1, j - q, i + p) - tz_val(t, Y, 1, j - q, i - p));
    dv += 0.5 * al * (tz_val(t, Y, 2, j + q, i + p) * rN.c - tz_val(t, Y, 2, j - q, i + p) * rS.c +
                      tz_val(t, Y, 2, j + q, i - p) * rN.c - tz_val(t, Y, 2, j - q, i - p) * rS.c);
  }
  const double ku = sl * h / (p * c), kv = st * h / (q * c);
  emit(0, 1, 0, 0, -sl / c * dhx1);
  emit(0, 0, 0, 1, -sl * u / c);
  emit(0, 0, 0, -1, sl * u / c);
  emit(0, 2, 0, 0, -st * dhy1);
  emit(0, 0, 1, 0, -st * v);
  emit(0, 0, -1, 0, st * v);
  emit(0, 0, 0, 0, -(sl / (p * c) * du + st / (q * c) * dv));
  emit(0, 1, 0, p, -ku * (1.0 - al));
  emit(0, 1, 0, -p, ku * (1.0 - al));
  emit(0, 2, q, 0, -kv * (1.0 - al) * rN.c);
  emit(0, 2, -q, 0, kv * (1.0 - al) * rS.c);
  if (al != 0.0) {
    const double a2 = 0.5 * al;
    emit(0, 1, q, p, -ku * a2);
    emit(0, 1, q, -p, ku * a2);
    emit(0, 1, -q, p, -ku * a2);
    emit(0, 1, -q, -p, ku * a2);
    emit(0, 2, q, p, -kv * a2 * rN.c);
    emit(0, 2, -q, p, kv * a2 * rS.c);
    emit(0, 2, q, -p, -kv * a2 * rN.c);
    emit(0, 2, -q, -p, kv * a2 * rS.c);
  }
}

// out = cx X + cy (Y + dt F(Y))
__global__ void tz_stage_kernel(TzArgs t, const double* X, const double* Y, double* out, double cx, double cy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= t.nlon) return;
  double F[3];
  tz_F(t, Y, j, i, F[0], F[1], F[2]);
  const size_t pl = (size_t)t.nlat * t.nlon, o = (size_t)j * t.nlon + i;
  for (int v = 0; v < 3; ++v) {
    double r = cy * (Y[v * pl + o] + t.dt * F[v]);
    if (cx != 0.0) r += cx * X[v * pl + o];
    out[v * pl + o] = r;
  }
}

// dout = cx dX + cy (dY + dt F'(Y) dY)
__global__ void tz_tl_stage_kernel(TzArgs t, const double* Y, const double* dX, const double* dY, double* dout,
                                   double cx, double cy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= t.nlon) return;
  const size_t pl = (size_t)t.nlat * t.nlon, o = (size_t)j * t.nlon + i;
  double d[3] = {0.0, 0.0, 0.0};
  tz_jacobian(t, Y, j, i, [&](int vo, int vi, int jj, int ii, double coef) {
    d[vo] += coef * dY[vi * pl + (size_t)jj * t.nlon + ii];
  });
  for (int v = 0; v < 3; ++v) {
    double r = cy * (dY[v * pl + o] + t.dt * d[v]);
    if (cx != 0.0) r += cx * dX[v * pl + o];
    dout[v * pl + o] = r;
  }
}

// G += scale F'(Y)^T M (the transposed partial derivatives, scattered)
__global__ void tz_adj_scatter_kernel(TzArgs t, const double* Y, const double* M, double* G, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= t.nlon) return;
  const size_t pl = (size_t)t.nlat * t.nlon, o = (size_t)j * t.nlon + i;
  const double m[3] = {scale * M[o], scale * M[pl + o], scale * M[2 * pl + o]};
  tz_jacobian(t, Y, j, i, [&](int vo, int vi, int jj, int ii, double coef) {
    if (m[vo] != 0.0) atomicAdd(&G[vi * pl + (size_t)jj * t.nlon + ii], coef * m[vo]);
  });
}

__global__ void tz_lincomb_kernel(double* out, const double* a, const double* b, const double* c, double ca,
                                  double cb, double cc, long long n) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    out[k] = ca * a[k] + cb * b[k] + (c ? cc * c[k] : 0.0);
}

// x0 = xb + sigma_v w (diagonal B) or grad = w + sigma_v lam
__global__ void tz_scale_add_kernel(double* out, const double* a, const double* b, const double* sigma, long long plane) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < 3 * plane;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = a[k] + sigma[k / plane] * b[k];
}

// Observation misfits of the whole trajectory (obs sorted by level): forcing
// lam (H x - y) / sigma_o^2 per observation and J_o = lam/2 sum (H x - y)^2 /
// sigma_o^2, one block, fixed-order reduction.
__global__ void tz_obs_misfit_kernel(const double* traj, long long n, const int* level, const int* var,
                                     const double* fi, const double* fj, const double* y, const double* so,
                                     int nlon, int nlat, double lam, double* force, double* Jo) {
  __shared__ double sh[1024 / 32];
  double acc = 0.0;
  const size_t pl = (size_t)nlat * nlon;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    const int i0 = (int)floor(fi[k]), j0 = (int)floor(fj[k]);
    const double di = fi[k] - i0, dj = fj[k] - j0;
    const int i1 = (i0 + 1) % nlon;
    const double* x = traj + ((size_t)level[k] * 3 + var[k]) * pl;
    double hx = (1.0 - dj) * (1.0 - di) * x[(size_t)j0 * nlon + i0];
    if (di != 0.0) hx += (1.0 - dj) * di * x[(size_t)j0 * nlon + i1];
    if (dj != 0.0) {
      hx += dj * (1.0 - di) * x[(size_t)(j0 + 1) * nlon + i0];
      if (di != 0.0) hx += dj * di * x[(size_t)(j0 + 1) * nlon + i1];
    }
    const double d = hx - y[k], w = 1.0 / (so[k] * so[k]);
    force[k] = lam * w * d;
    acc += 0.5 * lam * w * d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    *Jo = s;
  }
}

// lam += H^T force for the observations [k0, k1) (one level)
__global__ void tz_obs_scatter_kernel(long long k0, long long k1, const int* var, const double* fi,
                                      const double* fj, const double* force, int nlon, int nlat, double* lam) {
  const size_t pl = (size_t)nlat * nlon;
  for (long long k = k0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; k < k1;
       k += (long long)gridDim.x * blockDim.x) {
    const int i0 = (int)floor(fi[k]), j0 = (int)floor(fj[k]);
    const double di = fi[k] - i0, dj = fj[k] - j0;
    const int i1 = (i0 + 1) % nlon;
    double* x = lam + (size_t)var[k] * pl;
    const double fk = force[k];
    atomicAdd(&x[(size_t)j0 * nlon + i0], (1.0 - dj) * (1.0 - di) * fk);
    if (di != 0.0) atomicAdd(&x[(size_t)j0 * nlon + i1], (1.0 - dj) * di * fk);
    if (dj != 0.0) {
      atomicAdd(&x[(size_t)(j0 + 1) * nlon + i0], dj * (1.0 - di) * fk);
      if (di != 0.0) atomicAdd(&x[(size_t)(j0 + 1) * nlon + i1], dj * di * fk);
    }
  }
}

// J_b = 1/2 w.w, one block, fixed order; J = J_b + J_o
__global__ void tz_finish_J_kernel(const double* w, long long n, const double* Jo, double* J) {
  __shared__ double sh[1024 / 32];
  double acc = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) acc += w[k] * w[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    *J = 0.5 * s + (Jo ? *Jo : 0.0);
  }
}

inline dim3 tz_grid(const TzArgs& t) { return dim3((t.nlon + 127) / 128, t.nlat); }
inline unsigned tz_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

cudaError_t launch_tz_stage(const TzArgs& t, const double* X, const double* Y, double* out, double cx, double cy,
                            cudaStream_t st) {
  tz_stage_kernel<<<tz_grid(t), 128, 0, st>>>(t, X, Y, out, cx, cy);
  return cudaGetLastError();
}
cudaError_t launch_tz_tl_stage(const TzArgs& t, const double* Y, const double* dX, const double* dY, double* dout,
                               double cx, double cy, cudaStream_t st) {
  tz_tl_stage_kernel<<<tz_grid(t), 128, 0, st>>>(t, Y, dX, dY, dout, cx, cy);
  return cudaGetLastError();
}
cudaError_t launch_tz_adj_scatter(const TzArgs& t, const double* Y, const double* M, double* G, double scale,
                                  cudaStream_t st) {
  tz_adj_scatter_kernel<<<tz_grid(t), 128, 0, st>>>(t, Y, M, G, scale);
  return cudaGetLastError();
}
cudaError_t launch_tz_lincomb(double* out, const double* a, const double* b, const double* c, double ca, double cb,
                              double cc, long long n, cudaStream_t st) {
  tz_lincomb_kernel<<<tz_blocks(n), 256, 0, st>>>(out, a, b, c, ca, cb, cc, n);
  return cudaGetLastError();
}
cudaError_t launch_tz_scale_add(double* out, const double* a, const double* b, const double* sigma, long long plane,
                                cudaStream_t st) {
  tz_scale_add_kernel<<<tz_blocks(3 * plane), 256, 0, st>>>(out, a, b, sigma, plane);
  return cudaGetLastError();
}
cudaError_t launch_tz_obs_misfit(const double* traj, long long n, const int* level, const int* var, const double* fi,
                                 const double* fj, const double* y, const double* so, int nlon, int nlat, double lam,
                                 double* force, double* Jo, cudaStream_t st) {
  tz_obs_misfit_kernel<<<1, 1024, 0, st>>>(traj, n, level, var, fi, fj, y, so, nlon, nlat, lam, force, Jo);
  return cudaGetLastError();
}
cudaError_t launch_tz_obs_scatter(long long k0, long long k1, const int* var, const double* fi, const double* fj,
                                  const double* force, int nlon, int nlat, double* lam, cudaStream_t st) {
  if (k1 <= k0) return cudaSuccess;
  tz_obs_scatter_kernel<<<tz_blocks(k1 - k0), 256, 0, st>>>(k0, k1, var, fi, fj, force, nlon, nlat, lam);
  return cudaGetLastError();
}
cudaError_t launch_tz_finish_J(const double* w, long long n, const double* Jo, double* J, cudaStream_t st) {
  tz_finish_J_kernel<<<1, 1024, 0, st>>>(w, n, Jo, J);
  return cudaGetLastError();
}

}  // namespace dd4dv
