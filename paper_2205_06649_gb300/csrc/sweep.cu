// Forward, adjoint and tangent-linear sweeps of the local shallow-water model
// over every subdomain's time window, batched in one launch each.
//
// Design (GB300, sm_103a): one thread-block cluster per subdomain.  The
// cluster's CTAs split the subdomain's box into horizontal stripes of rows;
// each CTA keeps its stripe of the state (plus one halo row on each side and
// a ghost column on each side) resident in shared memory for the whole time
// window.  Each RK3 stage is one cluster barrier phase: a CTA computes its
// edge rows first and stores them straight into its neighbours' halo rows
// through distributed shared memory, arrives at the cluster barrier, computes
// its interior rows while the barrier completes, and waits (the pushed halo
// exchange of phase_push).  The only HBM traffic of a step is the trajectory
// (and stage-state) store in the forward sweep and load in the adjoint sweep,
// ghost values of the frozen boundary trajectory (prefetched with cp.async on
// the FP32 path) and the sparse observation / overlap data.  FP32 buffers
// hold one 16-byte (h, u, v, 0) slot per point, FP64 buffers three planes.
// Clusters are ordered longest subdomain first (uneven sizes in one launch).
//
// Mathematics (paper arXiv 2205.06649):
//   model      Sec. 7 Eqs. EquU-EquH, centred differences, flux-form
//              continuity; SSP-RK3 time stepping
//   J terms    Sec. 3.3 Eq. eq:cost:parallel1 (observation misfit and overlap
//              penalty per level; the background term is in aux.cu)
//   adjoint    Alg. 6 (ADJ), the reversed product of step adjoints Eq. adjProd,
//              derived by hand from the discrete forward step
//   TLM        Alg. 6 (TLM), the linearised forward step.
#include "common.cuh"

#include <cooperative_groups.h>

#include <map>
#include <mutex>

namespace cg = cooperative_groups;

namespace dd4dv {

namespace {

// Shared-memory layout of one state buffer (R2 = R + 2 rows of W points,
// including the halo rows and ghost columns):
//   FP64: three planes [v][R2][W]; plane stride P = R2 W, column stride 1.
//   FP32: one 16-byte slot (h, u, v, 0) per point, [R2][W][4]; plane stride
//         P = 1, column stride 4, so a point's three values are one 128-bit
//         shared-memory access and a 5-point stencil is five of them.
// The FP64 sweeps are bound by the FP64 pipe, not by instruction issue, so
// they keep the denser planar layout.
template <typename T>
struct Lay {
  static constexpr bool kVec = sizeof(T) == 4;
  static constexpr int CS = kVec ? 4 : 1;   // column stride (elements)
  static constexpr int NS = kVec ? 4 : 3;   // elements per point in a buffer
};

template <typename T>
struct Geo {
  int s, rank, CL, R0, Rn, nx, ny, L, a, R2, W, P, flags;
  int RS;             // row stride (elements) = W * column stride
  int BUF;            // elements of one state buffer
  int Rprev, Rnext;   // own-row counts of the south / north neighbour CTA
  SubDesc d;
  T* gh;              // ghost cache: 3 slots of [6 R columns | 6 W rows] values
  int* gh_tag;        // level held by each slot (-1: none)
  T* tgb;             // shared buffer of prefetched overlap targets (FP32 sweeps), or nullptr
  int gh_len;         // values per slot
  // multipliers for division by nx, Rn, ny and the loaded row count nr
  // (mdiv below) in the per-point index mappings
  unsigned mnx, mRn, mny, mnr;
};

// Division by a per-CTA constant d >= 1 through a precomputed multiplier
// m = ceil(2^32 / d) (m = 0 encodes d = 1): floor(a / d) = floor(a m / 2^32)
// exactly whenever a * d < 2^32.  (With m = (2^32 + e) / d, 0 <= e < d, the
// product is a / d + a e / (d 2^32); the extra term is below 1 / d, the gap
// from a / d up to the next integer, when a e < 2^32.)  Every dividend here is
// an index into a CTA's shared-memory stripe, below 2^20, and every divisor
// is a row length or a row count: a * d stays below 2^31.
__host__ __device__ __forceinline__ unsigned magic_of(int d) {
  return d <= 1 ? 0u : (unsigned)(0xFFFFFFFFu / (unsigned)d + 1u);
}
__device__ __forceinline__ int mdiv(int a, unsigned m) {
  return m ? (int)__umulhi((unsigned)a, m) : a;
}

// Arithmetic with explicit rounding: the compiler neither contracts nor
// reorders these, so every inlined copy of the forward step (forward sweep,
// stage recomputation in the adjoint, checkpoint-segment recomputation,
// tangent-linear sweep) rounds identically and the copies agree bit for bit.
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ void split_rows(int ny, int CL, int rank, int& R0, int& Rn) {
  const int base = ny / CL, rem = ny % CL;
  R0 = rank * base + min(rank, rem);
  Rn = base + (rank < rem ? 1 : 0);
}

// Element index of point (rr, k) (own rows rr = 0 .. Rn-1, halo rows -1 and
// Rn; columns k = 0 .. nx-1, ghost columns -1 and nx), first variable; the
// variable v sits at + v P.
template <typename T>
__device__ __forceinline__ int pidx(const Geo<T>& g, int rr, int k) {
  return ((rr + 1) * g.W + k + 1) * Lay<T>::CS;
}
template <typename T>
__device__ __forceinline__ int off(const Geo<T>& g, int v, int rr, int k) {
  return pidx(g, rr, k) + v * g.P;
}

// The three values (h, u, v) of the point at element index o.
template <typename T>
__device__ __forceinline__ void ld3(const T* Z, int o, int P, T& h, T& u, T& v) {
  if constexpr (Lay<T>::kVec) {
    const float4 x = *reinterpret_cast<const float4*>(Z + o);
    h = x.x;
    u = x.y;
    v = x.z;
  } else {
    h = Z[o];
    u = Z[o + P];
    v = Z[o + 2 * P];
  }
}
template <typename T>
__device__ __forceinline__ void st3(T* Z, int o, int P, T h, T u, T v) {
  if constexpr (Lay<T>::kVec) {
    *reinterpret_cast<float4*>(Z + o) = make_float4(h, u, v, 0.0f);
  } else {
    Z[o] = h;
    Z[o + P] = u;
    Z[o + 2 * P] = v;
  }
}

// Per-row constants staged in shared memory for rows rr = -1 .. Rn (index
// i = rr + 1), as two 8-value records per row so that a point reads its row's
// constants with two (FP32) or four (FP64) 16-byte loads:
//   fw[8 i ..]: A, f, tau, B/c, g A, c of row i+1, c of row i-1, 0
//               (tendencies and tangent-linear tendencies)
//   bw[8 i ..]: A, f, tau, g A, B c, 1/c of row i+1, 1/c of row i-1, 2 tau
//               (adjoint tendencies)
// Wall ghost rows take the edge row's cos (mirror).
template <typename T>
struct RowSmem {
  T *fw, *bw;
};

template <typename T>
__device__ __forceinline__ void load_rec8(const T* p, T (&r)[8]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    const float4 y = *reinterpret_cast<const float4*>(p + 4);
    r[0] = x.x; r[1] = x.y; r[2] = x.z; r[3] = x.w;
    r[4] = y.x; r[5] = y.y; r[6] = y.z; r[7] = y.w;
  } else {
    for (int q = 0; q < 4; ++q) {
      const double2 x = *reinterpret_cast<const double2*>(p + 2 * q);
      r[2 * q] = x.x;
      r[2 * q + 1] = x.y;
    }
  }
}

template <typename T>
__device__ void load_rows(const SweepArgs<T>& a, const Geo<T>& g, RowSmem<T>& rs) {
  for (int i = threadIdx.x; i < g.Rn + 2; i += blockDim.x) {
    const int j = g.d.j0 + g.R0 + i - 1;
    const int jc = min(max(j, 0), a.nlat - 1);       // wall ghost rows mirror cos
    const int jn = min(max(j + 1, 0), a.nlat - 1);
    const int js = min(max(j - 1, 0), a.nlat - 1);
    const RowConst rc = a.rows[jc];
    const double cn = a.rows[jn].c, cs = a.rows[js].c;
    T* f = rs.fw + 8 * i;
    f[0] = (T)rc.A;
    f[1] = (T)rc.f;
    f[2] = (T)rc.tau;
    f[3] = (T)rc.BinvC;
    f[4] = (T)rc.gA;
    f[5] = (T)cn;
    f[6] = (T)cs;
    f[7] = (T)0;
    T* b = rs.bw + 8 * i;
    b[0] = (T)rc.A;
    b[1] = (T)rc.f;
    b[2] = (T)rc.tau;
    b[3] = (T)rc.gA;
    b[4] = (T)(a.Bth * rc.c);
    b[5] = (T)(1.0 / cn);
    b[6] = (T)(1.0 / cs);
    b[7] = (T)(2.0 * rc.tau);
  }
}

// Buffer kinds for halo / ghost completion.
enum { K_STATE = 0, K_ADJ = 1, K_DELTA = 2 };

// Boundary-trajectory value for variable v at global (j, i) blended between
// levels nA and nB with weights wA, wB (read from HBM).
template <typename T>
__device__ __forceinline__ T bnd_val(const SweepArgs<T>& a, int nA, int nB, T wA, T wB, int v, int j,
                                     int i) {
  const size_t plane = (size_t)a.nlat * a.nlon;
  const size_t o = ((size_t)v * a.nlat + j) * a.nlon + i;
  const T xa = a.bnd[(size_t)nA * 3 * plane + o];
  if (wB == (T)0) return xa;
  const T xb = a.bnd[(size_t)nB * 3 * plane + o];
  return xfma(wA, xa, xmul(wB, xb));
}

// ---- ghost cache --------------------------------------------------------
// The ghost values a CTA needs at one level -- the west/east columns of its
// own rows when the box has frozen lateral edges, the south/north rows when
// its stripe touches a frozen box edge -- are copied into a slot of a 3-level
// shared-memory ring with cp.async one step before they are used, so that the
// completion after each stage reads shared memory instead of waiting on HBM.
// Slot of level n: n mod 3; a lookup whose level is not in its slot falls back
// to HBM (results never depend on the cache).  The copies join the caller's
// next cp.async commit group.
// Slot layout: columns [side][var][R], then rows [side][var][W].

__device__ __forceinline__ void cp_async_4or8(void* dst, const void* src, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// All but the most recently committed group complete.
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T>
__device__ void ghost_prefetch(const SweepArgs<T>& a, const Geo<T>& g, int n) {
  if constexpr (sizeof(T) == 8) return;   // FP64 path: no cache (registers, ALU-bound)
  if (g.gh_len == 0 || n < 0 || n > a.nsteps) return;
  const int slot = n % 3;
  T* dst = g.gh + (size_t)slot * g.gh_len;
  const size_t plane = (size_t)a.nlat * a.nlon;
  const T* src = a.bnd + (size_t)n * 3 * plane;
  const int R = g.R2 - 2;
  if (!(g.flags & F_PERIODIC)) {
    const int iw = (g.d.i0 - 1 + a.nlon) % a.nlon, ie = (g.d.i0 + g.nx) % a.nlon;
    for (int idx = threadIdx.x; idx < 6 * g.Rn; idx += blockDim.x) {
      const int q = mdiv(idx, g.mRn);   // side * 3 + v
      const int side = q / 3;
      const int v = q - 3 * side, rr = idx - q * g.Rn;
      const int j = g.d.j0 + g.R0 + rr;
      cp_async_4or8(dst + (side * 3 + v) * R + rr,
                    src + ((size_t)v * a.nlat + j) * a.nlon + (side ? ie : iw), (int)sizeof(T));
    }
  }
  const bool south = g.rank == 0 && !(g.flags & F_SWALL);
  const bool north = g.rank == g.CL - 1 && !(g.flags & F_NWALL);
  if (south || north) {
    for (int idx = threadIdx.x; idx < 6 * g.nx; idx += blockDim.x) {
      const int q = mdiv(idx, g.mnx);   // side * 3 + v
      const int side = q / 3;
      if ((side == 0 && !south) || (side == 1 && !north)) continue;
      const int v = q - 3 * side, k = idx - q * g.nx;
      const int j = side ? g.d.j0 + g.ny : g.d.j0 - 1;
      cp_async_4or8(dst + 6 * R + (side * 3 + v) * g.W + k,
                    src + ((size_t)v * a.nlat + j) * a.nlon + (g.d.i0 + k) % a.nlon, (int)sizeof(T));
    }
  }
  if (threadIdx.x == 0) g.gh_tag[slot] = n;
}

// Source of the ghost values of one phase: the boundary trajectory blended
// between levels nA and nB (wA x(nA) + wB x(nB)).  Resolved once per phase:
// when both levels sit in the ghost cache, ca / cb point at their slots and
// every lookup is one or two shared-memory loads; otherwise (FP64 path, or a
// level not cached) the values are read from HBM.  Both give identical
// values.
template <typename T>
struct GhostSrc {
  const T* ca;
  const T* cb;   // nullptr when wB = 0
  int nA, nB;
  T wA, wB;
  bool cached;
};

template <typename T>
__device__ __forceinline__ GhostSrc<T> ghost_src(const Geo<T>& g, int nA, int nB, T wA, T wB) {
  GhostSrc<T> s{nullptr, nullptr, nA, nB, wA, wB, false};
  if constexpr (sizeof(T) == 4) {
    if (g.gh_len > 0 && nA >= 0 && nB >= 0) {
      const int sA = nA % 3, sB = nB % 3;
      if (g.gh_tag[sA] == nA && (wB == (T)0 || g.gh_tag[sB] == nB)) {
        s.cached = true;
        s.ca = g.gh + (size_t)sA * g.gh_len;
        s.cb = (wB == (T)0) ? nullptr : g.gh + (size_t)sB * g.gh_len;
      }
    }
  }
  return s;
}

// Ghost column of own row rr (side 0 = west, 1 = east) and ghost row value at
// column k (side 0 = south, 1 = north).
template <typename T>
__device__ __forceinline__ T gh_col(const SweepArgs<T>& a, const Geo<T>& g, const GhostSrc<T>& s, int side,
                                    int v, int rr) {
  if (s.cached) {
    const int o = (side * 3 + v) * (g.R2 - 2) + rr;
    const T xa = s.ca[o];
    return s.cb ? xfma(s.wA, xa, xmul(s.wB, s.cb[o])) : xa;
  }
  const int i = side == 0 ? (g.d.i0 - 1 + a.nlon) % a.nlon : (g.d.i0 + g.nx) % a.nlon;
  return bnd_val(a, s.nA, s.nB, s.wA, s.wB, v, g.d.j0 + g.R0 + rr, i);
}

template <typename T>
__device__ __forceinline__ T gh_row(const SweepArgs<T>& a, const Geo<T>& g, const GhostSrc<T>& s, int side,
                                    int v, int k) {
  if (s.cached) {
    const int o = 6 * (g.R2 - 2) + (side * 3 + v) * g.W + k;
    const T xa = s.ca[o];
    return s.cb ? xfma(s.wA, xa, xmul(s.wB, s.cb[o])) : xa;
  }
  return bnd_val(a, s.nA, s.nB, s.wA, s.wB, v, side ? g.d.j0 + g.ny : g.d.j0 - 1, (g.d.i0 + k) % a.nlon);
}

// Value of halo row `side` (0 south, 1 north) at column k of a stripe that
// has no neighbour CTA on that side: the wall mirror (h, u, -v) of the edge
// row, the frozen boundary trajectory blended between levels nA and nB, or
// zero (adjoint buffers at walls; adjoint and tangent-linear buffers at frozen
// edges).
template <typename T>
__device__ __forceinline__ void edge_row_val(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int kind,
                                             int side, int k, const GhostSrc<T>& gs, T& h, T& u, T& v) {
  const bool wall = side ? (g.flags & F_NWALL) : (g.flags & F_SWALL);
  if (wall) {
    if (kind == K_ADJ) {
      h = u = v = (T)0;
      return;
    }
    ld3(X, pidx(g, side ? g.Rn - 1 : 0, k), g.P, h, u, v);
    v = -v;
  } else if (kind == K_STATE) {
    h = gh_row(a, g, gs, side, 0, k);
    u = gh_row(a, g, gs, side, 1, k);
    v = gh_row(a, g, gs, side, 2, k);
  } else {
    h = u = v = (T)0;
  }
}

// Value of ghost column `side` (0 west, 1 east) of own row rr: the periodic
// wrap, the frozen boundary trajectory, or zero.
template <typename T>
__device__ __forceinline__ void ghost_col_val(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int kind,
                                              int side, int rr, const GhostSrc<T>& gs, T& h, T& u, T& v) {
  if (g.flags & F_PERIODIC) {
    ld3(X, pidx(g, rr, side ? 0 : g.nx - 1), g.P, h, u, v);
  } else if (kind == K_STATE) {
    h = gh_col(a, g, gs, side, 0, rr);
    u = gh_col(a, g, gs, side, 1, rr);
    v = gh_col(a, g, gs, side, 2, rr);
  } else {
    h = u = v = (T)0;
  }
}

// Complete a buffer whose own rows were just written by this CTA: cluster
// barrier, halo rows from the neighbour CTAs (DSMEM) or from the box-edge rule
// (wall mirror, frozen boundary trajectory, or zero), ghost columns of the own
// rows (periodic wrap, boundary trajectory, or zero), CTA barrier.
template <typename T>
__device__ void complete_buf(cg::cluster_group& cl, const SweepArgs<T>& a, const Geo<T>& g, T* X,
                             int kind, int nA, int nB, T wA, T wB) {
  if constexpr (sizeof(T) == 4) cp_async_wait_all();   // this thread's ghost copies land first
  cl.sync();
  const int nx = g.nx;
  const T* south_nb = (g.rank > 0) ? cl.map_shared_rank(X, g.rank - 1) : nullptr;
  const T* north_nb = (g.rank < g.CL - 1) ? cl.map_shared_rank(X, g.rank + 1) : nullptr;
  const GhostSrc<T> gs = ghost_src(g, nA, nB, wA, wB);
  // halo rows
  for (int idx = threadIdx.x; idx < 2 * nx; idx += blockDim.x) {
    const int side = idx >= nx ? 1 : 0;
    const int k = idx - side * nx;
    const T* nb = side ? north_nb : south_nb;
    T h, u, v;
    if (nb) {
      ld3(nb, pidx(g, side ? 0 : g.Rprev - 1, k), g.P, h, u, v);
    } else {
      edge_row_val(a, g, X, kind, side, k, gs, h, u, v);
    }
    st3(X, pidx(g, side ? g.Rn : -1, k), g.P, h, u, v);
  }
  // ghost columns of own rows
  for (int idx = threadIdx.x; idx < 2 * g.Rn; idx += blockDim.x) {
    const int side = idx >= g.Rn ? 1 : 0;
    const int rr = idx - side * g.Rn;
    T h, u, v;
    ghost_col_val(a, g, X, kind, side, rr, gs, h, u, v);
    st3(X, pidx(g, rr, side ? nx : -1), g.P, h, u, v);
  }
  __syncthreads();
}

// Box-edge halo rows (stripes at the box edges only) and ghost columns of a
// state buffer X whose own rows are in place; ghosts from the boundary
// trajectory blended between levels nA and nB.
template <typename T>
__device__ __forceinline__ void state_edges(const SweepArgs<T>& a, const Geo<T>& g, T* X, int j,
                                            const GhostSrc<T>& gs) {
  const int nx = g.nx;
  T h, u, v;
  if (j < 2 * nx) {
    const int side = j >= nx ? 1 : 0;
    const int k = j - side * nx;
    if (side ? g.rank != g.CL - 1 : g.rank != 0) return;   // interior halo: loaded
    edge_row_val(a, g, X, K_STATE, side, k, gs, h, u, v);
    st3(X, pidx(g, side ? g.Rn : -1, k), g.P, h, u, v);
  } else {
    j -= 2 * nx;
    const int side = j >= g.Rn ? 1 : 0;
    const int rr = j - side * g.Rn;
    ghost_col_val(a, g, X, K_STATE, side, rr, gs, h, u, v);
    st3(X, pidx(g, rr, side ? nx : -1), g.P, h, u, v);
  }
}

// Load one stored state (own rows and interior halo rows straight from HBM,
// box-edge halos by rule, ghost columns of own rows) whose ghosts come from
// the boundary trajectory blended between levels nA and nB.  src points at the
// [3][ny][nxp] block.  Ends with a CTA barrier.
template <typename T>
__device__ void load_state(const SweepArgs<T>& a, const Geo<T>& g, T* X, const T* src, int nA, int nB,
                           T wA, T wB) {
  const int nx = g.nx;
  const int r_lo = (g.rank > 0) ? -1 : 0;
  const int r_hi = (g.rank < g.CL - 1) ? g.Rn + 1 : g.Rn;
  const int nr = r_hi - r_lo;
  const size_t pl = (size_t)g.ny * g.d.nxp;
  for (int idx = threadIdx.x; idx < nr * nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);
    const int rr = q + r_lo, k = idx - q * nx;
    const T* s = src + (size_t)(g.R0 + rr) * g.d.nxp + k;
    st3(X, pidx(g, rr, k), g.P, s[0], s[pl], s[2 * pl]);
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();
  __syncthreads();
  const GhostSrc<T> gs = ghost_src(g, nA, nB, wA, wB);
  for (int j = threadIdx.x; j < 2 * nx + 2 * g.Rn; j += blockDim.x) state_edges(a, g, X, j, gs);
  __syncthreads();
}

// Load NS stored states at once (one pass, one barrier pair) so that their
// global-load latencies overlap.  Same rules as load_state.
template <typename T, int NS>
__device__ void load_states(const SweepArgs<T>& a, const Geo<T>& g, T* const* X, const T* const* src,
                            const int* nA, const int* nB, const T* wA, const T* wB) {
  const int nx = g.nx;
  const int r_lo = (g.rank > 0) ? -1 : 0;
  const int r_hi = (g.rank < g.CL - 1) ? g.Rn + 1 : g.Rn;
  const int nr = r_hi - r_lo;
  const size_t pl = (size_t)g.ny * g.d.nxp;
  for (int idx = threadIdx.x; idx < nr * nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);
    const int rr = q + r_lo, k = idx - q * nx;
    const size_t go = (size_t)(g.R0 + rr) * g.d.nxp + k;
    const int o = pidx(g, rr, k);
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      const T* s = src[b] + go;
      st3(X[b], o, g.P, s[0], s[pl], s[2 * pl]);
    }
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();
  __syncthreads();
  GhostSrc<T> gs[NS];
#pragma unroll
  for (int b = 0; b < NS; ++b) gs[b] = ghost_src(g, nA[b], nB[b], wA[b], wB[b]);
  for (int j = threadIdx.x; j < 2 * nx + 2 * g.Rn; j += blockDim.x) {
#pragma unroll
    for (int b = 0; b < NS; ++b) state_edges(a, g, X[b], j, gs[b]);
  }
  __syncthreads();
}

// Level l of the stored trajectory, ghosts at boundary level n.
template <typename T>
__device__ __forceinline__ void load_level(const SweepArgs<T>& a, const Geo<T>& g, T* X, int l, int n) {
  load_state(a, g, X, a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp, n, n, (T)1, (T)0);
}

template <typename T>
__device__ __forceinline__ T* stage_ptr(const SweepArgs<T>& a, const Geo<T>& g, int l, int which) {
  return a.stg + g.d.stg_off + ((size_t)l * 2 + which) * 3 * g.ny * g.d.nxp;
}

// The five stencil points of element index o in a buffer with plane stride
// P, column stride CS and row stride RS: centre, east, west, north, south.
template <typename T>
struct Pt5 {
  T h, u, v, hE, uE, vE, hW, uW, vW, hN, uN, vN, hS, uS, vS;
};
template <typename T>
__device__ __forceinline__ void load5(const T* Z, int o, int P, int CS, int RS, Pt5<T>& p) {
  ld3(Z, o, P, p.h, p.u, p.v);
  ld3(Z, o + CS, P, p.hE, p.uE, p.vE);
  ld3(Z, o - CS, P, p.hW, p.uW, p.vW);
  ld3(Z, o + RS, P, p.hN, p.uN, p.vN);
  ld3(Z, o - RS, P, p.hS, p.uS, p.vS);
}

// Tendencies F(Z) at one point (Sec. 7, centred differences):
//   F_u = -A u (uE-uW) - Bth v (uN-uS) + (f + tau u) v - gA (hE-hW)
//   F_v = -A u (vE-vW) - Bth v (vN-vS) - (f + tau u) u - gBth (hN-hS)
//   F_h = -A ((hu)_E - (hu)_W) - (Bth/c) ((h v c)_N - (h v c)_S)
// On the FP32 path h = h_ref + h' and the h_ref parts of the fluxes are
// formed from velocity differences.
template <typename T, bool DEV>
__device__ __forceinline__ void rhs_pt(const Pt5<T>& z, T A, T f, T tau, T BinvC, T gA, T cN, T cS, T Bth,
                                       T gBth, T href, T& Fh, T& Fu, T& Fv) {
  const T u = z.u, v = z.v;
  const T dUx = xsub(z.uE, z.uW), dUy = xsub(z.uN, z.uS);
  const T dVx = xsub(z.vE, z.vW), dVy = xsub(z.vN, z.vS);
  const T dHx = xsub(z.hE, z.hW), dHy = xsub(z.hN, z.hS);
  const T fu = xfma(tau, u, f);
  const T Au = xmul(A, u), Bv = xmul(Bth, v);
  Fu = xfma(fu, v, -xfma(Au, dUx, xfma(Bv, dUy, xmul(gA, dHx))));
  Fv = -xfma(Au, dVx, xfma(Bv, dVy, xfma(fu, u, xmul(gBth, dHy))));
  T flx = xfma(z.hE, z.uE, -xmul(z.hW, z.uW));
  T fly = xfma(xmul(z.hN, z.vN), cN, -xmul(xmul(z.hS, z.vS), cS));
  if (DEV) {
    flx = xfma(href, dUx, flx);
    fly = xfma(href, xfma(z.vN, cN, -xmul(z.vS, cS)), fly);
  }
  Fh = -xfma(A, flx, xmul(BinvC, fly));
}

// Adjoint of the tendencies: G = F'(Z)^T M at one point (derived by hand from
// rhs_pt; M holds zero at ghost points that carry no tendency).  Wall rows add
// the transposed ghost mirror (h, u, -v) of the edge row.
//   G_u = mu (tau v - A dU_x) - mv (A dV_x + f + 2 tau u) + A (muE uE - muW uW)
//         + A h (mhE - mhW) + Bth (muN vN - muS vS)
//   G_v = mu (f + tau u - Bth dU_y) - mv Bth dV_y + A (mvE uE - mvW uW)
//         + Bth (mvN vN - mvS vS) + (B c) h (mhN / cN - mhS / cS)
//   G_h = gA (muE - muW) + gBth (mvN - mvS) + A u (mhE - mhW)
//         + (B c) v (mhN / cN - mhS / cS)
// evaluated as 42 explicitly rounded operations, 21 of them fused
// multiply-adds.
template <typename T, bool DEV>
__device__ __forceinline__ void rhs_adj_pt(const Pt5<T>& z, const Pt5<T>& m, T A, T f, T tau, T gA, T BcC,
                                           T icN, T icS, T tau2, T Bth, T gBth, T href, int wall, T& Gh,
                                           T& Gu, T& Gv) {
  T h = z.h;
  if (DEV) h += href;
  const T u = z.u, v = z.v;
  const T mu = m.u, mv = m.v, mh = m.h;
  const T dUx = xsub(z.uE, z.uW), dVx = xsub(z.vE, z.vW);
  const T dUy = xsub(z.uN, z.uS), dVy = xsub(z.vN, z.vS);
  const T dmhEW = xsub(m.hE, m.hW);
  const T dmhNS = xfma(m.hN, icN, -xmul(m.hS, icS));
  Gh = xfma(xmul(BcC, v), dmhNS,
            xfma(xmul(A, u), dmhEW, xfma(gBth, xsub(m.vN, m.vS), xmul(gA, xsub(m.uE, m.uW)))));
  const T a1 = xfma(-A, dUx, xmul(tau, v));
  const T a2 = xfma(A, dVx, xfma(tau2, u, f));
  const T p1 = xfma(m.uE, z.uE, -xmul(m.uW, z.uW));
  const T p2 = xfma(m.uN, z.vN, -xmul(m.uS, z.vS));
  Gu = xfma(Bth, p2, xfma(xmul(A, h), dmhEW, xfma(A, p1, xfma(-mv, a2, xmul(mu, a1)))));
  const T b1 = xfma(-Bth, dUy, xfma(tau, u, f));
  const T q1 = xfma(m.vE, z.uE, -xmul(m.vW, z.uW));
  const T q2 = xfma(m.vN, z.vN, -xmul(m.vS, z.vS));
  Gv = xfma(xmul(BcC, h), dmhNS, xfma(Bth, q2, xfma(A, q1, xfma(-mv, xmul(Bth, dVy), xmul(mu, b1)))));
  if (wall == 1) {         // south wall: ghost row = (h, u, -v) of this row
    Gu = xfma(xmul(Bth, mu), v, Gu);
    Gv = xfma(-Bth, xfma(mv, v, xmul(h, mh)), Gv);
    Gh = xfma(gBth, mv, xfma(-Bth, xmul(v, mh), Gh));
  } else if (wall == 2) {  // north wall
    Gu = xfma(-xmul(Bth, mu), v, Gu);
    Gv = xfma(Bth, xfma(mv, v, xmul(h, mh)), Gv);
    Gh = xfma(Bth, xmul(v, mh), xfma(-gBth, mv, Gh));
  }
}

// Tangent-linear tendencies dF = F'(Z) dZ at one point.
template <typename T, bool DEV>
__device__ __forceinline__ void rhs_tl_pt(const Pt5<T>& z, const Pt5<T>& d, T A, T f, T tau, T BinvC, T gA,
                                          T cN, T cS, T Bth, T gBth, T href, T& dFh, T& dFu, T& dFv) {
  const T u = z.u, v = z.v;
  const T du = d.u, dv = d.v;
  const T uE = z.uE, uW = z.uW, uN = z.uN, uS = z.uS;
  const T vE = z.vE, vW = z.vW, vN = z.vN, vS = z.vS;
  T hE = z.hE, hW = z.hW, hN = z.hN, hS = z.hS;
  if (DEV) {
    hE += href; hW += href; hN += href; hS += href;
  }
  const T duE = d.uE, duW = d.uW, duN = d.uN, duS = d.uS;
  const T dvE = d.vE, dvW = d.vW, dvN = d.vN, dvS = d.vS;
  const T dhE = d.hE, dhW = d.hW, dhN = d.hN, dhS = d.hS;
  dFu = -A * (du * (uE - uW) + u * (duE - duW)) - Bth * (dv * (uN - uS) + v * (duN - duS)) +
        (f + tau * u) * dv + tau * du * v - gA * (dhE - dhW);
  dFv = -A * (du * (vE - vW) + u * (dvE - dvW)) - Bth * (dv * (vN - vS) + v * (dvN - dvS)) -
        (f + tau * u) * du - tau * du * u - gBth * (dhN - dhS);
  dFh = -A * ((dhE * uE + hE * duE) - (dhW * uW + hW * duW)) -
        BinvC * ((dhN * vN + hN * dvN) * cN - (dhS * vS + hS * dvS) * cS);
}

// The arithmetic of the transposed RK3 step at one point, shared by every
// adjoint sweep so that all of them round alike.  A stage adjoint
// mu_out = m + dt F'(z)^T m ...
template <typename T, bool DEV>
__device__ __forceinline__ void adj_stage_math(const Pt5<T>& z, const Pt5<T>& m, const T (&rc)[8], T dt, T Bth,
                                               T gBth, T href, int wall, T& v0, T& v1, T& v2) {
  T Gh, Gu, Gv;
  rhs_adj_pt<T, DEV>(z, m, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], rc[7], Bth, gBth, href, wall, Gh, Gu, Gv);
  v0 = xfma(dt, Gh, m.h);
  v1 = xfma(dt, Gu, m.u);
  v2 = xfma(dt, Gv, m.v);
}
// ... and lambda(n) = lambda'/3 + mu2/2 + (mu1 + dt F'(x)^T mu1)/6 from the
// stencil m of mu1, z of x, and lambda' = (ph, pu, pv), mu2 = (qh, qu, qv) at
// the point.
template <typename T, bool DEV>
__device__ __forceinline__ void adj_lambda_math(const Pt5<T>& z, const Pt5<T>& m, const T (&rc)[8], T dt, T Bth,
                                                T gBth, T href, int wall, T ph, T pu, T pv, T qh, T qu, T qv,
                                                T& v0, T& v1, T& v2) {
  const T c13 = (T)(1.0 / 3.0), c16 = (T)(1.0 / 6.0);
  T Gh, Gu, Gv;
  rhs_adj_pt<T, DEV>(z, m, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], rc[7], Bth, gBth, href, wall, Gh, Gu, Gv);
  v0 = xfma(c16, xfma(dt, Gh, m.h), xfma((T)0.5, qh, xmul(c13, ph)));
  v1 = xfma(c16, xfma(dt, Gu, m.u), xfma((T)0.5, qu, xmul(c13, pu)));
  v2 = xfma(c16, xfma(dt, Gv, m.v), xfma((T)0.5, qv, xmul(c13, pv)));
}

template <typename T>
__device__ __forceinline__ void block_reduce2(double& x, double& y, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    scratch[2 * wid] = x;
    scratch[2 * wid + 1] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0;
    for (int w = 0; w < nw; ++w) {
      sx += scratch[2 * w];
      sy += scratch[2 * w + 1];
    }
    x = sx;
    y = sy;
  }
}

// Overlap count at a local point: (covering subdomains) - 1.
template <typename T>
__device__ __forceinline__ int overlap_count(const Geo<T>& g, int l, int r, int k) {
  const SubDesc& d = g.d;
  const int cx = 1 + (k < d.wL) + (k >= d.nx - d.wR);
  const int cy = 1 + (r < d.wS) + (r >= d.ny - d.wN);
  const int ct = 1 + (l < d.tA) + (l > g.L - d.tB);
  return cx * cy * ct - 1;
}

// Observation misfit of the observations of level l whose lower corner row
// is one of this CTA's rows: J_o += 1/2 w d^2, obs_force = lambda w d.
// Observation term of one record with explicit rounding, so that every
// sweep kernel that evaluates it rounds alike: the bilinear value of the
// corner values x00, x01 (i + 1), x10 (j + 1), x11 (only the corners with
// non-zero weight are used), d = H x - y, J_o += 1/2 w d^2; returns the
// forcing lambda w d.
__device__ __forceinline__ double obs_term(const ObsRec& ob, double x00, double x01, double x10, double x11,
                                           double lam, double& Jo) {
  const double wj0 = __dsub_rn(1.0, ob.dj), wi0 = __dsub_rn(1.0, ob.di);
  double acc = __dmul_rn(__dmul_rn(wj0, wi0), x00);
  if (ob.di != 0.0) acc = __fma_rn(__dmul_rn(wj0, ob.di), x01, acc);
  if (ob.dj != 0.0) {
    acc = __fma_rn(__dmul_rn(ob.dj, wi0), x10, acc);
    if (ob.di != 0.0) acc = __fma_rn(__dmul_rn(ob.dj, ob.di), x11, acc);
  }
  const double d = __dsub_rn(acc, ob.y);
  Jo = __fma_rn(__dmul_rn(__dmul_rn(0.5, ob.w), d), d, Jo);
  return __dmul_rn(__dmul_rn(lam, ob.w), d);
}

// Overlap misfit of one point with overlap count c, explicitly rounded:
// part + c ((x0 - t0)^2 i0 + (x1 - t1)^2 i1 + (x2 - t2)^2 i2).
template <typename T>
__device__ __forceinline__ T overlap_term(T part, int c, T x0, T x1, T x2, T t0, T t1, T t2, T i0, T i1,
                                          T i2) {
  const T e0 = xsub(x0, t0), e1 = xsub(x1, t1), e2 = xsub(x2, t2);
  T sq = xmul(xmul(e0, e0), i0);
  sq = xfma(xmul(e1, e1), i1, sq);
  sq = xfma(xmul(e2, e2), i2, sq);
  return xfma((T)c, sq, part);
}

template <typename T>
__device__ void obs_level(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int l, double& Jo) {
  const int o0 = a.lvl_obs[g.d.obs_lvl + l], o1 = a.lvl_obs[g.d.obs_lvl + l + 1];
  // highest-numbered threads first (the low threads start the next phase's
  // edge rows)
  for (int o = o0 + (blockDim.x - 1 - threadIdx.x); o < o1; o += blockDim.x) {
    const ObsRec ob = a.obs[o];
    const int rr = ob.r0 - g.R0;
    if (rr < 0 || rr >= g.Rn) continue;
    const double x00 = (double)X[off(g, ob.var, rr, ob.k0)];
    const double x01 = ob.di != 0.0 ? (double)X[off(g, ob.var, rr, ob.k1)] : 0.0;
    const double x10 = ob.dj != 0.0 ? (double)X[off(g, ob.var, rr + 1, ob.k0)] : 0.0;
    const double x11 = (ob.dj != 0.0 && ob.di != 0.0) ? (double)X[off(g, ob.var, rr + 1, ob.k1)] : 0.0;
    a.obs_force[o] = obs_term(ob, x00, x01, x10, x11, a.lam, Jo);
  }
}

// Linearised observation forcing for Gauss-Newton products: with D the
// tangent-linear state at level l, obs_force = lambda w (H D) for the
// observations of level l whose lower corner row is one of this CTA's rows.
template <typename T>
__device__ void obs_level_lin(const SweepArgs<T>& a, const Geo<T>& g, const T* D, int l) {
  const int o0 = a.lvl_obs[g.d.obs_lvl + l], o1 = a.lvl_obs[g.d.obs_lvl + l + 1];
  for (int o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    const ObsRec ob = a.obs[o];
    const int rr = ob.r0 - g.R0;
    if (rr < 0 || rr >= g.Rn) continue;
    double acc = 0.0;
    const double wj0 = 1.0 - ob.dj, wi0 = 1.0 - ob.di;
    acc += (wj0 * wi0) * (double)D[off(g, ob.var, rr, ob.k0)];
    if (ob.di != 0.0) acc += (wj0 * ob.di) * (double)D[off(g, ob.var, rr, ob.k1)];
    if (ob.dj != 0.0) {
      acc += (ob.dj * wi0) * (double)D[off(g, ob.var, rr + 1, ob.k0)];
      if (ob.di != 0.0) acc += (ob.dj * ob.di) * (double)D[off(g, ob.var, rr + 1, ob.k1)];
    }
    a.obs_force[o] = a.lam * ob.w * acc;
  }
}

// Calls f(rr, k, c) for every own point (rr, k) of level l with overlap count
// c > 0, spread over the CTA's threads from the highest-numbered one down (the
// low threads start the next phase's edge rows).  At a level outside the time overlaps
// only the spatial bands have c > 0: rows r < wS and r >= ny - wN in full,
// and the columns k < wL and k >= nx - wR of the rows between; those points
// alone are visited.
template <typename T, typename F>
__device__ __forceinline__ void for_overlap_points(const Geo<T>& g, int l, F&& f) {
  const SubDesc& d = g.d;
  const int nx = g.nx;
  const bool any_t = (l < d.tA) || (l > g.L - d.tB);
  if (any_t || d.wL + d.wR >= nx) {
    for (int idx = blockDim.x - 1 - threadIdx.x; idx < g.Rn * nx; idx += blockDim.x) {
      const int rr = mdiv(idx, g.mnx), k = idx - rr * nx;
      const int c = overlap_count(g, l, g.R0 + rr, k);
      if (c) f(rr, k, c);
    }
    return;
  }
  // own rows [R0, R0 + Rn): full band rows at the low end (A rows) and at the
  // high end (C rows), the rest (B rows) with wL + wR band columns each
  const int A = max(0, min(g.Rn, d.wS - g.R0));
  const int C = max(0, min(g.Rn - A, g.R0 + g.Rn - (g.ny - d.wN)));
  const int B = g.Rn - A - C;
  const int wc = d.wL + d.wR;
  const int nA = A * nx, nC = C * nx, nB = B * wc;
  const unsigned mwc = magic_of(wc);
  for (int idx = blockDim.x - 1 - threadIdx.x; idx < nA + nC + nB; idx += blockDim.x) {
    int rr, k;
    if (idx < nA) {
      rr = mdiv(idx, g.mnx);
      k = idx - rr * nx;
    } else if (idx < nA + nC) {
      const int j = idx - nA;
      const int q = mdiv(j, g.mnx);
      rr = g.Rn - C + q;
      k = j - q * nx;
    } else {
      const int j = idx - nA - nC;
      const int q = mdiv(j, mwc);
      const int kk = j - q * wc;
      rr = A + q;
      k = kk < d.wL ? kk : nx - d.wR + (kk - d.wL);
    }
    const int c = overlap_count(g, l, g.R0 + rr, k);
    if (c) f(rr, k, c);
  }
}

// Overlap penalty at level l over own points: Jm2 += c sum_v (x - m)^2 / sb^2
// (twice the J_mu contribution; the caller halves the total, which is exact).
// The differences and this level's partial sum are formed in the state
// precision; the partial is added to the FP64 accumulator once per level (on
// the FP64 path this is all FP64).
template <typename T>
__device__ void overlap_level(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int l, double& Jm) {
  const SubDesc& d = g.d;
  const bool any_t = (l < d.tA) || (l > g.L - d.tB);
  const bool any_s = d.wL || d.wR || d.wS || d.wN;
  if (!any_t && !any_s) return;
  const T* tg = a.tgt + d.traj_off + (size_t)l * 3 * g.ny * d.nxp;
  const T i0 = a.isb2_s[0], i1 = a.isb2_s[1], i2 = a.isb2_s[2];
  const size_t pl = (size_t)g.ny * d.nxp;
  if (g.tgb) cp_async_wait_all();   // this thread's prefetched targets
  T part = (T)0;
  for_overlap_points(g, l, [&](int rr, int k, int c) {
    const int o = pidx(g, rr, k);
    T x0, x1, x2, t0, t1, t2;
    ld3(X, o, g.P, x0, x1, x2);
    if (g.tgb) {
      ld3(g.tgb, o, g.P, t0, t1, t2);
    } else {
      const size_t go = (size_t)(g.R0 + rr) * d.nxp + k;
      t0 = tg[go];
      t1 = tg[go + pl];
      t2 = tg[go + 2 * pl];
    }
    part = overlap_term(part, c, x0, x1, x2, t0, t1, t2, i0, i1, i2);
  });
  Jm += (double)part;
}

// Copies the overlap targets of level l at this CTA's overlap points into the
// shared target buffer (FP32 sweeps) with cp.async, a few phases before they
// are read.  overlap_level and add_forcing read each point on the thread that
// copied it (the same for_overlap_points mapping), so that thread's own
// cp.async wait is all the synchronisation they need; the adjoint's fused
// lambda(n) phase reads them on any thread, after a phase that waited for all
// copies and ended with a barrier.  The copies join the caller's next commit
// group.
template <typename T>
__device__ void prefetch_targets(const SweepArgs<T>& a, const Geo<T>& g, int l) {
  if (!g.tgb) return;
  const SubDesc& d = g.d;
  const bool any_t = (l < d.tA) || (l > g.L - d.tB);
  const bool any_s = d.wL || d.wR || d.wS || d.wN;
  if (!any_t && !any_s) return;
  const T* tg = a.tgt + d.traj_off + (size_t)l * 3 * g.ny * d.nxp;
  const size_t pl = (size_t)g.ny * d.nxp;
  for_overlap_points(g, l, [&](int rr, int k, int c) {
    const T* s = tg + (size_t)(g.R0 + rr) * d.nxp + k;
    T* dst = g.tgb + pidx(g, rr, k);
    cp_async_4or8(dst, s, (int)sizeof(T));
    cp_async_4or8(dst + g.P, s + pl, (int)sizeof(T));
    cp_async_4or8(dst + 2 * g.P, s + 2 * pl, (int)sizeof(T));
  });
}

template <typename T>
__device__ __forceinline__ bool setup_geo(const SweepArgs<T>& a, cg::cluster_group& cl, Geo<T>& g) {
  g.rank = cl.block_rank();
  g.CL = cl.num_blocks();
  const int cid = blockIdx.x / g.CL;
  if (cid >= a.n_sub) return false;
  g.s = a.order[cid];
  if (a.active && a.active[g.s] != a.active_value) return false;
  g.d = a.subs[g.s];
  g.nx = g.d.nx;
  g.ny = g.d.ny;
  g.a = g.d.a;
  g.L = g.d.b - g.d.a;
  g.flags = g.d.flags;
  if (g.ny < g.CL || g.nx + 2 > a.W) {   // uniform over the cluster
    if (threadIdx.x == 0 && g.rank == 0) atomicExch(a.err, 1);
    return false;
  }
  split_rows(g.ny, g.CL, g.rank, g.R0, g.Rn);
  int t;
  if (g.rank > 0) split_rows(g.ny, g.CL, g.rank - 1, t, g.Rprev); else g.Rprev = 0;
  if (g.rank < g.CL - 1) split_rows(g.ny, g.CL, g.rank + 1, t, g.Rnext); else g.Rnext = 0;
  g.R2 = a.R + 2;
  g.W = a.W;
  g.P = Lay<T>::kVec ? 1 : g.R2 * g.W;
  g.RS = g.W * Lay<T>::CS;
  g.BUF = Lay<T>::NS * g.R2 * g.W;
  if (g.rank != 0) g.flags &= ~F_SWALL;           // only the edge CTAs see the walls
  if (g.rank != g.CL - 1) g.flags &= ~F_NWALL;
  g.mnx = magic_of(g.nx);
  g.mRn = magic_of(g.Rn);
  g.mny = magic_of(g.ny);
  g.mnr = magic_of(g.Rn + (g.rank > 0) + (g.rank < g.CL - 1));
  return true;
}

// The arithmetic of one RK3 stage at one point, out = cx X + cy (Y + dt F(Y)),
// from the point's stencil y of Y, its row constants rc and its X values (read
// only when cx != 0).  Every sweep (forward, stage recomputation, checkpoint
// segments, tangent-linear, the deep-halo FP32 sweeps) calls this one
// function, so all of them round every stage identically.
template <typename T, bool DEV>
__device__ __forceinline__ void stage_math(const Pt5<T>& y, const T (&rc)[8], T dt, T Bth, T gBth, T href, T cx,
                                           T cy, T xh, T xu, T xv, T& o0, T& o1, T& o2) {
  T Fh, Fu, Fv;
  rhs_pt<T, DEV>(y, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth, href, Fh, Fu, Fv);
  o0 = xfma(dt, Fh, y.h);
  o1 = xfma(dt, Fu, y.u);
  o2 = xfma(dt, Fv, y.v);
  if (cy != (T)1) {
    o0 = xmul(cy, o0);
    o1 = xmul(cy, o1);
    o2 = xmul(cy, o2);
  }
  if (cx != (T)0) {
    o0 = xfma(cx, xh, o0);
    o1 = xfma(cx, xu, o1);
    o2 = xfma(cx, xv, o2);
  }
}

// One RK3 stage at own point (rr, k): out = cx X + cy (Y + dt F(Y)); the
// three new values are also returned.
template <typename T, bool DEV>
__device__ __forceinline__ void stage_point(const SweepArgs<T>& a, const Geo<T>& g, const RowSmem<T>& rs,
                                            T* out, const T* X, const T* Y, T cx, T cy, int rr, int k,
                                            T& o0, T& o1, T& o2) {
  const int P = g.P;
  const int o = pidx(g, rr, k);
  const int ri = rr + 1;
  T rc[8];
  load_rec8(rs.fw + 8 * ri, rc);
  Pt5<T> y;
  load5(Y, o, P, Lay<T>::CS, g.RS, y);
  T xh = (T)0, xu = (T)0, xv = (T)0;
  if (cx != (T)0) ld3(X, o, P, xh, xu, xv);
  stage_math<T, DEV>(y, rc, a.dt_s, a.Bth_s, a.gBth_s, a.href_s, cx, cy, xh, xu, xv, o0, o1, o2);
  st3(out, o, P, o0, o1, o2);
}

// One RK3 stage on own rows (halos completed afterwards by complete_buf).
// One point per thread per iteration (pairing points per thread for
// instruction-level parallelism measured slower on GB300: it doubles
// register pressure).
template <typename T, bool DEV>
__device__ void stage(const SweepArgs<T>& a, const Geo<T>& g, const RowSmem<T>& rs, T* out,
                      const T* X, const T* Y, T cx, T cy) {
  for (int idx = threadIdx.x; idx < g.Rn * g.nx; idx += blockDim.x) {
    const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
    T o0, o1, o2;
    stage_point<T, DEV>(a, g, rs, out, X, Y, cx, cy, rr, k, o0, o1, o2);
  }
}

// ---- pushed halo exchange -------------------------------------------------
// A phase that computes the own rows of buffer X can publish its halo data
// itself instead of having complete_buf pull it after a barrier:
//   1. fixed ghosts of X that do not depend on this phase (frozen boundary
//      values, zeros);
//   2. the edge rows 0 and Rn-1, each value also stored into the neighbour
//      CTA's halo row (distributed shared memory), into the wall mirror row,
//      or into the periodic ghost column;
//   3. cluster barrier arrive (release);
//   4. the interior rows, while the barrier completes;
//   5. CTA barrier, then cluster barrier wait (acquire).
// Ordering: a neighbour passes its wait only after this CTA's arrive, so it
// can be at most one phase ahead of this CTA's interior rows.  The buffer it
// then writes into is the next phase's output, whose halo rows no interior
// row of the current phase reads.  Halo rows of X are read only by edge
// rows, before the arrive.

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Step 1: box-edge halo rows without a neighbour CTA or a mirror, and
// ghost columns of a box that is not periodic.
template <typename T>
__device__ void fill_fixed(const SweepArgs<T>& a, const Geo<T>& g, T* X, int kind, int nA, int nB, T wA,
                           T wB) {
  const int nx = g.nx;
  const bool s_fixed = g.rank == 0 && (!(g.flags & F_SWALL) || kind == K_ADJ);
  const bool n_fixed = g.rank == g.CL - 1 && (!(g.flags & F_NWALL) || kind == K_ADJ);
  const bool cols = !(g.flags & F_PERIODIC);
  if (!s_fixed && !n_fixed && !cols) return;
  const GhostSrc<T> gs = ghost_src(g, nA, nB, wA, wB);
  // Edge-row points [0, 2 nx) then ghost-column points [2 nx, 2 nx + 2 Rn),
  // on the highest-numbered threads: the low threads compute the edge rows
  // and the most interior points of the phase.
  const int n = 2 * nx + 2 * g.Rn;
  for (int r = blockDim.x - 1 - threadIdx.x; r < n; r += blockDim.x) {
    T h, u, v;
    if (r < 2 * nx) {
      const int side = r >= nx ? 1 : 0;
      if (side ? !n_fixed : !s_fixed) continue;
      const int k = r - side * nx;
      edge_row_val(a, g, X, kind, side, k, gs, h, u, v);
      st3(X, pidx(g, side ? g.Rn : -1, k), g.P, h, u, v);
    } else {
      if (!cols) continue;
      const int j = r - 2 * nx;
      const int side = j >= g.Rn ? 1 : 0;
      const int rr = j - side * g.Rn;
      ghost_col_val(a, g, X, kind, side, rr, gs, h, u, v);
      st3(X, pidx(g, rr, side ? nx : -1), g.P, h, u, v);
    }
  }
}

// Step 2 for one point: its values (v0, v1, v2) go to the halo data that
// depends on them.
template <typename T>
__device__ __forceinline__ void publish(const Geo<T>& g, T* X, T* snb, T* nnb, int kind, int rr, int k, T v0,
                                        T v1, T v2) {
  if (rr == 0) {
    if (snb) {
      st3(snb, pidx(g, g.Rprev, k), g.P, v0, v1, v2);
    } else if ((g.flags & F_SWALL) && kind != K_ADJ) {
      st3(X, pidx(g, -1, k), g.P, v0, v1, -v2);
    }
  }
  if (rr == g.Rn - 1) {
    if (nnb) {
      st3(nnb, pidx(g, -1, k), g.P, v0, v1, v2);
    } else if ((g.flags & F_NWALL) && kind != K_ADJ) {
      st3(X, pidx(g, g.Rn, k), g.P, v0, v1, -v2);
    }
  }
  if (g.flags & F_PERIODIC) {
    if (k == 0) st3(X, pidx(g, rr, g.nx), g.P, v0, v1, v2);
    if (k == g.nx - 1) st3(X, pidx(g, rr, -1), g.P, v0, v1, v2);
  }
}

// Steps 1-5 with fn(rr, k, v0, v1, v2) computing and storing point (rr, k)
// of X and returning its values.
// pend = 1 leaves the most recent cp.async commit group in flight at the end
// of the phase (prefetches consumed in a later phase).
template <typename T, typename Fn>
__device__ void phase_push(cg::cluster_group& cl, const SweepArgs<T>& a, const Geo<T>& g, T* X, int kind,
                           int nA, int nB, T wA, T wB, Fn&& fn, int pend = 0) {
  fill_fixed(a, g, X, kind, nA, nB, wA, wB);
  T* snb = g.rank > 0 ? cl.map_shared_rank(X, g.rank - 1) : nullptr;
  T* nnb = g.rank < g.CL - 1 ? cl.map_shared_rank(X, g.rank + 1) : nullptr;
  const int nx = g.nx;
  const int ne = (g.Rn > 1 ? 2 : 1) * nx;
  for (int idx = threadIdx.x; idx < ne; idx += blockDim.x) {
    const int rr = idx < nx ? 0 : g.Rn - 1;
    const int k = idx < nx ? idx : idx - nx;
    T v0, v1, v2;
    fn(rr, k, v0, v1, v2);
    publish(g, X, snb, nnb, kind, rr, k, v0, v1, v2);
  }
  cluster_arrive_release();
  const int ni = (g.Rn > 2 ? g.Rn - 2 : 0) * nx;
  for (int idx = threadIdx.x; idx < ni; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);
    const int rr = 1 + q, k = idx - q * nx;
    T v0, v1, v2;
    fn(rr, k, v0, v1, v2);
    if ((g.flags & F_PERIODIC) && (k == 0 || k == nx - 1)) publish(g, X, snb, nnb, kind, rr, k, v0, v1, v2);
  }
  if constexpr (sizeof(T) == 4) {   // this thread's ghost copies land first
    if (pend)
      cp_async_wait_prev();
    else
      cp_async_wait_all();
  }
  __syncthreads();
  cluster_wait_acquire();
}

// RK3 stage with pushed halo exchange (replaces stage + complete_buf).
template <typename T, bool DEV>
__device__ __forceinline__ void stage_push(cg::cluster_group& cl, const SweepArgs<T>& a, const Geo<T>& g,
                                           const RowSmem<T>& rs, T* out, const T* X, const T* Y, T cx, T cy,
                                           int nA, int nB, T wA, T wB, int pend = 0) {
  phase_push(
      cl, a, g, out, K_STATE, nA, nB, wA, wB,
      [&](int rr, int k, T& v0, T& v1, T& v2) {
        stage_point<T, DEV>(a, g, rs, out, X, Y, cx, cy, rr, k, v0, v1, v2);
      },
      pend);
}

// Halo data of a buffer whose own rows are final (after forcing terms were
// added): fixed ghosts, edge rows pushed, periodic ghosts, full cluster
// barrier.
template <typename T>
__device__ void push_halos(cg::cluster_group& cl, const SweepArgs<T>& a, const Geo<T>& g, T* X, int kind) {
  fill_fixed(a, g, X, kind, 0, 0, (T)1, (T)0);
  T* snb = g.rank > 0 ? cl.map_shared_rank(X, g.rank - 1) : nullptr;
  T* nnb = g.rank < g.CL - 1 ? cl.map_shared_rank(X, g.rank + 1) : nullptr;
  const int nx = g.nx;
  const bool periodic = g.flags & F_PERIODIC;
  // edge rows (all columns), plus the two end columns of every row when periodic
  const int ne = (g.Rn > 1 ? 2 : 1) * nx;
  const int nper = periodic ? 2 * g.Rn : 0;
  for (int idx = threadIdx.x; idx < ne + nper; idx += blockDim.x) {
    int rr, k;
    if (idx < ne) {
      rr = idx < nx ? 0 : g.Rn - 1;
      k = idx < nx ? idx : idx - nx;
    } else {
      const int j = idx - ne;
      rr = j >> 1;
      k = (j & 1) ? nx - 1 : 0;
      if (rr == 0 || rr == g.Rn - 1) continue;   // done with the edge rows
    }
    T h, u, v;
    ld3(X, pidx(g, rr, k), g.P, h, u, v);
    publish(g, X, snb, nnb, kind, rr, k, h, u, v);
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();
  cl.sync();
}

template <typename T>
__device__ void store_block(const Geo<T>& g, const T* X, T* dst) {
  const size_t pl = (size_t)g.ny * g.d.nxp;
  for (int idx = threadIdx.x; idx < g.Rn * g.nx; idx += blockDim.x) {
    const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
    T h, u, v;
    ld3(X, pidx(g, rr, k), g.P, h, u, v);
    T* d = dst + (size_t)(g.R0 + rr) * g.d.nxp + k;
    d[0] = h;
    d[pl] = u;
    d[2 * pl] = v;
  }
}

template <typename T>
__device__ __forceinline__ void store_level(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int l) {
  store_block(g, X, a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp);
}

// The FP32 forward and adjoint sweeps (the ones with a ghost cache) also
// prefetch overlap targets into one more state-sized buffer, when the CTA's
// shared memory still fits the device's opt-in maximum with it (large boxes
// in few-CTA clusters read the targets from HBM instead, as the FP64 sweeps
// do).
template <typename T>
__host__ __device__ constexpr bool target_buffer(bool cache) {
  return cache && sizeof(T) == 4;
}
constexpr size_t kSmemOptinMax = 232448;   // 227 KB per CTA on sm_100 / sm_103

// Ghost-cache length per slot (FP32 forward / adjoint sweeps only).
template <typename T>
__host__ __device__ constexpr int ghost_len(bool cache, int R, int W) {
  return (cache && sizeof(T) == 4) ? 6 * R + 6 * W : 0;
}

template <typename T>
__device__ void carve(const SweepArgs<T>& a, const Geo<T>& g, int nbuf, T** bufs, RowSmem<T>& rs,
                      double** scratch, bool cache) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* p = reinterpret_cast<T*>(smem_raw);
  for (int b = 0; b < nbuf; ++b) {
    bufs[b] = p;
    p += g.BUF;
  }
  Geo<T>& gt = const_cast<Geo<T>&>(g);
  gt.tgb = nullptr;
  if (target_buffer<T>(cache) && a.tgb_on) {
    gt.tgb = p;
    p += g.BUF;
  }
  const int nr = a.R + 2;
  uintptr_t q = reinterpret_cast<uintptr_t>(p);
  q = (q + 15) & ~uintptr_t(15);   // 16-byte records
  rs.fw = reinterpret_cast<T*>(q);
  rs.bw = rs.fw + 8 * nr;
  p = rs.bw + 8 * nr;
  q = reinterpret_cast<uintptr_t>(p);
  q = (q + 15) & ~uintptr_t(15);
  *scratch = reinterpret_cast<double*>(q);
  q += 64 * sizeof(double);
  // ghost cache: 3 slots of 6 R + 6 W values, then 3 tags
  Geo<T>& gm = const_cast<Geo<T>&>(g);
  gm.gh_len = ghost_len<T>(cache, a.R, a.W);
  gm.gh = reinterpret_cast<T*>(q);
  gm.gh_tag = reinterpret_cast<int*>(q + 3 * (size_t)gm.gh_len * sizeof(T));
  if (threadIdx.x < 3) gm.gh_tag[threadIdx.x] = -1;
  __syncthreads();
}

template <typename T>
size_t smem_bytes_tg(int nbuf, int R, int W, bool cache, bool tg) {
  nbuf += tg ? 1 : 0;
  return (size_t)nbuf * Lay<T>::NS * (R + 2) * W * sizeof(T) + 16 + 16 * (size_t)(R + 2) * sizeof(T) + 16 +
         64 * sizeof(double) + 3 * (size_t)ghost_len<T>(cache, R, W) * sizeof(T) + 3 * sizeof(int) + 16;
}
// whether the sweep with nbuf state buffers carries the target buffer
template <typename T>
bool use_target_buffer(int nbuf, int R, int W, bool cache) {
  return target_buffer<T>(cache) && smem_bytes_tg<T>(nbuf, R, W, cache, true) <= kSmemOptinMax;
}
template <typename T>
size_t smem_bytes(int nbuf, int R, int W, bool cache) {
  return smem_bytes_tg<T>(nbuf, R, W, cache, use_target_buffer<T>(nbuf, R, W, cache));
}

// ---------------------------------------------------------------------------
// Forward sweep: x(a) (stored at level 0 by the init kernel) -> x(a+1..b),
// trajectory stored at every level, J_o and J_mu partial sums per CTA.
//
// TB = true: two state buffers instead of three.  x2 is written over x(n) in
// place (each point reads x(n) only at itself), and the last stage reads
// x(n) point by point from the trajectory level stored the step before
// (needs every level stored: ckpt 0).  Same arithmetic on the same values,
// so the same results; the smaller footprint fits two CTAs per SM where three
// buffers fit one.  The buffers swap roles every step.  Writing x2 over
// x(n) is safe under the pushed exchange: x(n)'s halo rows are read only by
// the first stage's edge rows, before this CTA's arrive, and a neighbour
// pushes x2 rows only after that arrive.
template <typename T, bool TB>
__global__ void __launch_bounds__(max_threads_forward<T>(), min_blocks_forward<T>()) fwd_kernel(SweepArgs<T> a) {
  constexpr bool DEV = sizeof(T) == 4;
  cg::cluster_group cl = cg::this_cluster();
  Geo<T> g;
  if (!setup_geo(a, cl, g)) return;
  T* buf[3];
  RowSmem<T> rs;
  double* scratch;
  carve(a, g, TB ? 2 : 3, buf, rs, &scratch, true);
  T* X = buf[0];
  T* S1 = buf[1];
  T* S2 = TB ? nullptr : buf[2];
  load_rows(a, g, rs);
  ghost_prefetch(a, g, g.a);
  if (g.L > 0) ghost_prefetch(a, g, g.a + 1);
  cp_async_commit();
  load_level(a, g, X, 0, g.a);   // includes a CTA barrier
  prefetch_targets(a, g, 0);
  cp_async_commit();
  double Jo = 0.0, Jm = 0.0;
  obs_level(a, g, X, 0, Jo);
  overlap_level(a, g, X, 0, Jm);
  for (int l = 0; l < g.L; ++l) {
    const int n = g.a + l;
    stage_push<T, DEV>(cl, a, g, rs, S1, X, X, (T)0, (T)1, n + 1, n + 1, (T)1, (T)0);
    // stores read the buffer with another thread mapping: after the barrier
    if (a.stg) store_block(g, S1, stage_ptr(a, g, l, 0));
    if constexpr (sizeof(T) == 8) {   // x1 alone: FP64 path only
      if (!a.stg && a.stg1 && g.d.stg1_off >= 0)
        store_block(g, S1, a.stg1 + g.d.stg1_off + (size_t)l * 3 * g.ny * g.d.nxp);
    }
    // after that barrier, level l's targets have been read and the ghost slot
    // of level n - 1 is free: prefetch the ghosts of the next step and the
    // targets of level l + 1, consumed after the third stage
    if (n + 2 <= g.d.b) ghost_prefetch(a, g, n + 2);
    prefetch_targets(a, g, l + 1);
    cp_async_commit();
    if constexpr (TB) {
      // x2 over x(n), then x(n+1) = 1/3 x(n) + 2/3 (x2 + dt F(x2)) into x1's
      // buffer with x(n) read from the stored level l
      stage_push<T, DEV>(cl, a, g, rs, X, X, S1, (T)0.75, (T)0.25, n, n + 1, (T)0.5, (T)0.5, 1);
      if (a.stg) store_block(g, X, stage_ptr(a, g, l, 1));
      const T* xs = a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp;
      const size_t pl = (size_t)g.ny * g.d.nxp;
      phase_push(cl, a, g, S1, K_STATE, n + 1, n + 1, (T)1, (T)0, [&](int rr, int k, T& o0, T& o1, T& o2) {
        const int o = pidx(g, rr, k);
        T rc[8];
        load_rec8(rs.fw + 8 * (rr + 1), rc);
        Pt5<T> y;
        load5(X, o, g.P, Lay<T>::CS, g.RS, y);
        const T* q = xs + (size_t)(g.R0 + rr) * g.d.nxp + k;
        stage_math<T, DEV>(y, rc, a.dt_s, a.Bth_s, a.gBth_s, a.href_s, (T)(1.0 / 3.0), (T)(2.0 / 3.0), q[0],
                           q[pl], q[2 * pl], o0, o1, o2);
        st3(S1, o, g.P, o0, o1, o2);
      });
      T* t = X;
      X = S1;
      S1 = t;
    } else {
      stage_push<T, DEV>(cl, a, g, rs, S2, X, S1, (T)0.75, (T)0.25, n, n + 1, (T)0.5, (T)0.5, 1);
      if (a.stg) store_block(g, S2, stage_ptr(a, g, l, 1));
      stage_push<T, DEV>(cl, a, g, rs, X, X, S2, (T)(1.0 / 3.0), (T)(2.0 / 3.0), n + 1, n + 1, (T)1, (T)0);
    }
    if (a.ckpt == 0 || (l + 1) % a.ckpt == 0) store_level(a, g, X, l + 1);
    obs_level(a, g, X, l + 1, Jo);
    overlap_level(a, g, X, l + 1, Jm);
  }
  Jm *= 0.5;
  block_reduce2<T>(Jo, Jm, scratch);
  if (threadIdx.x == 0) {
    a.part[((size_t)g.s * a.cl_max + g.rank) * 2 + 0] = Jo;
    a.part[((size_t)g.s * a.cl_max + g.rank) * 2 + 1] = Jm;
  }
  cl.sync();   // keep shared memory alive until every neighbour is done with it
}

// Overlap forcing mu c (x - m) / sb^2 of own point (rr, k) with overlap count
// c, added to (l0, l1, l2) with explicit rounding: the same arithmetic in
// add_forcing and in the fused lambda(n) phase of the adjoint sweep.  The
// targets m come from the shared target buffer when there is one (its
// copies have landed), else from HBM.
template <typename T>
__device__ __forceinline__ void overlap_force(const SweepArgs<T>& a, const Geo<T>& g, const T* X, const T* tg,
                                              int rr, int k, int c, T& l0, T& l1, T& l2) {
  const int o = pidx(g, rr, k);
  T x0, x1, x2, t0, t1, t2;
  ld3(X, o, g.P, x0, x1, x2);
  if (g.tgb) {
    ld3(g.tgb, o, g.P, t0, t1, t2);
  } else {
    const size_t pl = (size_t)g.ny * g.d.nxp;
    const size_t go = (size_t)(g.R0 + rr) * g.d.nxp + k;
    t0 = tg[go];
    t1 = tg[go + pl];
    t2 = tg[go + 2 * pl];
  }
  const T cc = (T)c;
  l0 = xfma(xmul(cc, a.musb2_s[0]), xsub(x0, t0), l0);
  l1 = xfma(xmul(cc, a.musb2_s[1]), xsub(x1, t1), l1);
  l2 = xfma(xmul(cc, a.musb2_s[2]), xsub(x2, t2), l2);
}

// Forcing of the adjoint at level l on own rows: observation scatter (H^T of
// lambda w d, fixed order per target) and overlap term mu c (x - m)/sb^2, or an
// external forcing y.  L holds the adjoint state, X the state at that level.
template <typename T>
__device__ void add_forcing(const SweepArgs<T>& a, const Geo<T>& g, T* Lb, const T* X, int l) {
  const SubDesc& d = g.d;
  if (a.yforce) {
    const double* y = a.yforce + d.ptraj_off + (size_t)l * 3 * g.ny * g.nx;
    for (int idx = threadIdx.x; idx < 3 * g.Rn * g.nx; idx += blockDim.x) {
      const int v = idx / (g.Rn * g.nx);
      const int rem = idx - v * g.Rn * g.nx;
      const int rr = rem / g.nx, k = rem - rr * g.nx;
      Lb[off(g, v, rr, k)] += (T)y[((size_t)v * g.ny + g.R0 + rr) * g.nx + k];
    }
    __syncthreads();
    return;
  }
  const bool any_t = (l < d.tA) || (l > g.L - d.tB);
  const bool any_s = d.wL || d.wR || d.wS || d.wN;
  if ((any_t || any_s) && a.mu != 0.0 && a.gn_dx) {   // Gauss-Newton product: mu c dx / sb^2
    const T* dx = a.gn_dx + d.traj_off + (size_t)l * 3 * g.ny * d.nxp;
    const T m0 = a.musb2_s[0], m1 = a.musb2_s[1], m2 = a.musb2_s[2];
    const size_t pl = (size_t)g.ny * d.nxp;
    for_overlap_points(g, l, [&](int rr, int k, int c) {
      const size_t go = (size_t)(g.R0 + rr) * d.nxp + k;
      const T cc = (T)c;
      const int o = pidx(g, rr, k);
      T l0, l1, l2;
      ld3(Lb, o, g.P, l0, l1, l2);
      st3(Lb, o, g.P, l0 + cc * m0 * dx[go], l1 + cc * m1 * dx[go + pl], l2 + cc * m2 * dx[go + 2 * pl]);
    });
  } else if ((any_t || any_s) && a.mu != 0.0) {
    const T* tg = a.tgt + d.traj_off + (size_t)l * 3 * g.ny * d.nxp;
    if (g.tgb) cp_async_wait_all();   // this thread's prefetched targets
    for_overlap_points(g, l, [&](int rr, int k, int c) {
      const int o = pidx(g, rr, k);
      T l0, l1, l2;
      ld3(Lb, o, g.P, l0, l1, l2);
      overlap_force(a, g, X, tg, rr, k, c, l0, l1, l2);
      st3(Lb, o, g.P, l0, l1, l2);
    });
  }
  __syncthreads();
  const int t0 = a.lvl_sc[d.sc_lvl + l], t1 = a.lvl_sc[d.sc_lvl + l + 1];
  const int plane = g.ny * g.nx;
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const int tg = a.sc_tgt[t];
    const int q = mdiv(tg, g.mnx);   // v * ny + r
    const int v = mdiv(q, g.mny);
    const int r = q - v * g.ny, k = tg - q * g.nx;
    const int rr = r - g.R0;
    if (rr < 0 || rr >= g.Rn) continue;
    double acc = 0.0;
    for (int c = a.sc_off[t]; c < a.sc_off[t + 1]; ++c) acc += a.sc_w[c] * a.obs_force[a.sc_obs[c]];
    Lb[off(g, v, rr, k)] += (T)acc;
  }
  __syncthreads();
}

// Adjoint sweep: lambda(b) = forcing(b); lambda(n) = M_n^T lambda(n+1) + forcing(n),
// the RK3 stages recomputed from the stored x(n).  Writes lambda(a) to lam_a.
//
// Buffer plans.  RL = false keeps x(n), x1, x2, lambda' and mu2 in five state
// buffers.  RL = true needs four: mu2 takes x(n)'s buffer once both stage
// states are formed, and x(n) is read again from HBM into x1's buffer after
// mu1 (x1's last use), for the lambda(n) phase and the overlap forcing; with
// stored stage states only x1 and x2 are loaded at the start of the step.
// Same arithmetic, same results, one more state read per step; the smaller
// footprint lets larger stripes or more CTAs per SM fit.  Writing mu2 into
// x(n)'s buffer is safe under the pushed exchange: a neighbour pushes mu2 rows
// into this CTA's halo only after this CTA arrived at the barrier of the
// phase before (its edge rows, the only readers of halo rows, are done), and
// the RL = true stored-stage step loads nothing into that buffer.
template <typename T, bool RL>
__global__ void __launch_bounds__(kStripeAdjThreads, 1) adj_kernel(SweepArgs<T> a) {
  constexpr bool DEV = sizeof(T) == 4;
  cg::cluster_group cl = cg::this_cluster();
  Geo<T> g;
  if (!setup_geo(a, cl, g)) return;
  T* buf[5];
  RowSmem<T> rs;
  double* scratch;
  carve(a, g, RL ? 4 : 5, buf, rs, &scratch, true);
  T* X = buf[0];
  T* X1 = buf[1];
  T* X2 = buf[2];   // also lambda_x1
  T* Lp = buf[3];
  T* L2 = RL ? buf[0] : buf[4];
  T* Xr = RL ? buf[1] : buf[0];   // x(n) in the lambda(n) phase
  load_rows(a, g, rs);
  ghost_prefetch(a, g, g.a + g.L);
  if (g.L > 0) ghost_prefetch(a, g, g.a + g.L - 1);
  cp_async_commit();
  // overlap targets prefetched for add_forcing (not for external forcing or
  // Gauss-Newton products, which take no targets)
  const bool pre_tg = g.tgb && a.mu != 0.0 && !a.gn_dx && !a.yforce;
  for (int i = threadIdx.x; i < g.BUF; i += blockDim.x) Lp[i] = (T)0;
  const T dt = a.dt_s, Bth = a.Bth_s, gBth = a.gBth_s, href = a.href_s;
  const int wall_s = (g.flags & F_SWALL) ? 1 : 0;
  const int wall_n = (g.flags & F_NWALL) ? 2 : 0;
  const size_t lvl_sz = (size_t)3 * g.ny * g.d.nxp;
  const int K = (a.ckpt > 0 && g.L > 0) ? a.ckpt : 0;
  T* segbuf = K ? a.seg + g.d.seg_off : nullptr;
  const int nseg = K ? (g.L + K - 1) / K : 1;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
  // levels [l0, l1] of this segment; without checkpoints one segment [0, L]
  const int l0 = K ? sgi * K : 0;
  const int l1 = K ? min(l0 + K, g.L) : g.L;
  // source of level l: the stored trajectory, or the recomputed segment
  auto level_src = [&](int l) -> const T* {
    if (!K || l == l0) return a.traj + g.d.traj_off + (size_t)l * lvl_sz;
    return segbuf + (size_t)(l - l0) * lvl_sz;
  };
  if (K) {
    // recompute x(l0+1 .. l1) from the checkpoint x(l0) into the segment buffer
    load_level(a, g, X, l0, g.a + l0);
    for (int l = l0; l < l1; ++l) {
      const int n = g.a + l;
      stage<T, DEV>(a, g, rs, X1, X, X, (T)0, (T)1);
      complete_buf(cl, a, g, X1, K_STATE, n + 1, n + 1, (T)1, (T)0);
      stage<T, DEV>(a, g, rs, X2, X, X1, (T)0.75, (T)0.25);
      complete_buf(cl, a, g, X2, K_STATE, n, n + 1, (T)0.5, (T)0.5);
      stage<T, DEV>(a, g, rs, X, X, X2, (T)(1.0 / 3.0), (T)(2.0 / 3.0));
      complete_buf(cl, a, g, X, K_STATE, n + 1, n + 1, (T)1, (T)0);
      store_block(g, X, segbuf + (size_t)(l + 1 - l0) * lvl_sz);
    }
    cl.sync();   // segment rows of every CTA written before any CTA reads its halo rows
  }
  if (sgi == nseg - 1) {
    // lambda(b) = forcing(b)
    load_state(a, g, X, level_src(g.L), g.a + g.L, g.a + g.L, (T)1, (T)0);
    if (pre_tg) prefetch_targets(a, g, g.L);
    cp_async_commit();
    add_forcing(a, g, Lp, X, g.L);
    complete_buf(cl, a, g, Lp, K_ADJ, 0, 0, (T)1, (T)0);
  }
  for (int l = l1 - 1; l >= l0; --l) {
    const int n = g.a + l;
    if (a.stg && !K && RL) {   // the stage states stored by the forward sweep
      T* bufs[2] = {X1, X2};
      const T* srcs[2] = {stage_ptr(a, g, l, 0), stage_ptr(a, g, l, 1)};
      const int nA[2] = {n + 1, n};
      const int nB[2] = {n + 1, n + 1};
      const T wA[2] = {(T)1, (T)0.5};
      const T wB[2] = {(T)0, (T)0.5};
      load_states<T, 2>(a, g, bufs, srcs, nA, nB, wA, wB);
    } else if (a.stg && !K) {   // x(n) and the stage states stored by the forward sweep
      T* bufs[3] = {X, X1, X2};
      const T* srcs[3] = {a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp,
                          stage_ptr(a, g, l, 0), stage_ptr(a, g, l, 1)};
      const int nA[3] = {n, n + 1, n};
      const int nB[3] = {n, n + 1, n + 1};
      const T wA[3] = {(T)1, (T)1, (T)0.5};
      const T wB[3] = {(T)0, (T)0, (T)0.5};
      load_states<T, 3>(a, g, bufs, srcs, nA, nB, wA, wB);
    } else if (sizeof(T) == 8 && !K && a.stg1 && g.d.stg1_off >= 0) {   // x(n) and the stored x1 (FP64)
      T* bufs[2] = {X, X1};
      const T* srcs[2] = {level_src(l), a.stg1 + g.d.stg1_off + (size_t)l * lvl_sz};
      const int nA[2] = {n, n + 1};
      const int nB[2] = {n, n + 1};
      const T wA[2] = {(T)1, (T)1};
      const T wB[2] = {(T)0, (T)0};
      load_states<T, 2>(a, g, bufs, srcs, nA, nB, wA, wB);
      stage_push<T, DEV>(cl, a, g, rs, X2, X, X1, (T)0.75, (T)0.25, n, n + 1, (T)0.5, (T)0.5);
    } else {       // recompute the stage states from x(n)
      load_state(a, g, X, level_src(l), n, n, (T)1, (T)0);
      stage_push<T, DEV>(cl, a, g, rs, X1, X, X, (T)0, (T)1, n + 1, n + 1, (T)1, (T)0);
      stage_push<T, DEV>(cl, a, g, rs, X2, X, X1, (T)0.75, (T)0.25, n, n + 1, (T)0.5, (T)0.5);
    }
    // after those barriers, the ghost slot of level n + 2 and the target
    // buffer are free: prefetch the ghosts of the next (earlier) step and the
    // targets of this level, consumed by add_forcing at the end of the step
    if (l > 0) ghost_prefetch(a, g, n - 1);
    if (pre_tg) prefetch_targets(a, g, l);
    cp_async_commit();
    const int P = g.P;
    constexpr int CS = Lay<T>::CS;
    // The transposed RK3 step with the stage adjoints scaled so that no stage
    // needs its own multiplication (G_k is linear in its argument):
    //   lambda_x2 = 2/3 mu2,  mu2 = lambda' + dt F'(x2)^T lambda'
    //   lambda_x1 = 1/6 mu1,  mu1 = mu2 + dt F'(x1)^T mu2
    //   lambda(n) = 1/3 lambda' + 3/4 lambda_x2 + lambda_x1 + dt F'(x)^T lambda_x1
    //             = 1/3 lambda' + 1/2 mu2 + 1/6 (mu1 + dt F'(x)^T mu1)
    // mu2 (into L2)
    phase_push(
        cl, a, g, L2, K_ADJ, 0, 0, (T)1, (T)0,
        [&](int rr, int k, T& v0, T& v1, T& v2) {
      const int o = pidx(g, rr, k), ri = rr + 1;
      const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
      T rc[8];
      load_rec8(rs.bw + 8 * ri, rc);
      Pt5<T> z, m;
      load5(X2, o, P, CS, g.RS, z);
      load5(Lp, o, P, CS, g.RS, m);
      adj_stage_math<T, DEV>(z, m, rc, dt, Bth, gBth, href, wall, v0, v1, v2);
      st3(L2, o, P, v0, v1, v2);
        },
        1);
    // mu1 (into X2's buffer)
    T* L1 = X2;
    phase_push(
        cl, a, g, L1, K_ADJ, 0, 0, (T)1, (T)0,
        [&](int rr, int k, T& v0, T& v1, T& v2) {
      const int o = pidx(g, rr, k), ri = rr + 1;
      const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
      T rc[8];
      load_rec8(rs.bw + 8 * ri, rc);
      Pt5<T> z, m;
      load5(X1, o, P, CS, g.RS, z);
      load5(L2, o, P, CS, g.RS, m);
      adj_stage_math<T, DEV>(z, m, rc, dt, Bth, gBth, href, wall, v0, v1, v2);
      st3(L1, o, P, v0, v1, v2);
        },
        0);   // the prefetched targets land before the next phase reads them
    // x(n) again, into x1's buffer (x1 is dead after mu1)
    if constexpr (RL) load_state(a, g, Xr, level_src(l), n, n, (T)1, (T)0);
    // lambda(n)
    const auto lam_n = [&](int rr, int k, T& v0, T& v1, T& v2) {
      const int o = pidx(g, rr, k), ri = rr + 1;
      const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
      T rc[8];
      load_rec8(rs.bw + 8 * ri, rc);
      Pt5<T> z, m;
      load5(Xr, o, P, CS, g.RS, z);
      load5(L1, o, P, CS, g.RS, m);
      T ph, pu, pv, qh, qu, qv;
      ld3(Lp, o, P, ph, pu, pv);
      ld3(L2, o, P, qh, qu, qv);
      adj_lambda_math<T, DEV>(z, m, rc, dt, Bth, gBth, href, wall, ph, pu, pv, qh, qu, qv, v0, v1, v2);
    };
    // With no external forcing, no Gauss-Newton product and no observation
    // at this level, lambda(n) takes its overlap forcing point by point and
    // pushes its halo in the same phase (the arithmetic of add_forcing,
    // without its passes and barriers).  Every CTA of the cluster takes the
    // same branch: the conditions belong to the subdomain.
    const SubDesc& d = g.d;
    const bool fuse = !a.yforce && !a.gn_dx && a.lvl_sc[d.sc_lvl + l] == a.lvl_sc[d.sc_lvl + l + 1];
    if (fuse) {
      const bool ovl = a.mu != 0.0 && ((l < d.tA) || (l > g.L - d.tB) || d.wL || d.wR || d.wS || d.wN);
      const T* tg = a.tgt + d.traj_off + (size_t)l * lvl_sz;
      phase_push(cl, a, g, Lp, K_ADJ, 0, 0, (T)1, (T)0, [&](int rr, int k, T& v0, T& v1, T& v2) {
        lam_n(rr, k, v0, v1, v2);
        if (ovl) {
          const int c = overlap_count(g, l, g.R0 + rr, k);
          if (c) overlap_force(a, g, Xr, tg, rr, k, c, v0, v1, v2);
        }
        st3(Lp, pidx(g, rr, k), P, v0, v1, v2);
      });
    } else {
      for (int idx = threadIdx.x; idx < g.Rn * g.nx; idx += blockDim.x) {
        const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
        T v0, v1, v2;
        lam_n(rr, k, v0, v1, v2);
        st3(Lp, pidx(g, rr, k), P, v0, v1, v2);
      }
      __syncthreads();
      add_forcing(a, g, Lp, Xr, l);
      push_halos(cl, a, g, Lp, K_ADJ);
    }
  }
  }
  // lambda(a) -> packed control layout (FP64)
  double* out = a.lam_a + g.d.ctrl_off;
  for (int idx = threadIdx.x; idx < 3 * g.Rn * g.nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // v * Rn + rr
    const int v = mdiv(q, g.mRn);
    const int rr = q - v * g.Rn, k = idx - q * g.nx;
    out[((size_t)v * g.ny + g.R0 + rr) * g.nx + k] = (double)Lp[off(g, v, rr, k)];
  }
  cl.sync();
}

// Tangent-linear sweep: x and dx advanced together; x stored to the
// trajectory, dx to the packed FP64 output and/or, for Gauss-Newton products,
// to gn_dx in the state precision with the linearised observation forcing.
template <typename T>
__device__ void load_delta0(const SweepArgs<T>& a, const Geo<T>& g, T* D) {
  const double* src = a.dx0 + g.d.ctrl_off;
  const int r_lo = (g.rank > 0) ? -1 : 0;
  const int r_hi = (g.rank < g.CL - 1) ? g.Rn + 1 : g.Rn;
  const int nr = r_hi - r_lo;
  for (int i = threadIdx.x; i < g.BUF; i += blockDim.x) D[i] = (T)0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < 3 * nr * g.nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // v * nr + (rr - r_lo)
    const int v = mdiv(q, g.mnr);
    const int rr = q - v * nr + r_lo;
    const int k = idx - q * g.nx;
    D[off(g, v, rr, k)] = (T)src[((size_t)v * g.ny + g.R0 + rr) * g.nx + k];
  }
  __syncthreads();
  if (g.flags & F_SWALL)
    for (int idx = threadIdx.x; idx < 3 * g.nx; idx += blockDim.x) {
      const int v = idx / g.nx, k = idx - v * g.nx;
      D[off(g, v, -1, k)] = (v == 2) ? -D[off(g, v, 0, k)] : D[off(g, v, 0, k)];
    }
  if (g.flags & F_NWALL)
    for (int idx = threadIdx.x; idx < 3 * g.nx; idx += blockDim.x) {
      const int v = idx / g.nx, k = idx - v * g.nx;
      D[off(g, v, g.Rn, k)] = (v == 2) ? -D[off(g, v, g.Rn - 1, k)] : D[off(g, v, g.Rn - 1, k)];
    }
  if (g.flags & F_PERIODIC)
    for (int idx = threadIdx.x; idx < 3 * g.Rn; idx += blockDim.x) {
      const int v = idx / g.Rn, rr = idx - v * g.Rn;
      D[off(g, v, rr, -1)] = D[off(g, v, rr, g.nx - 1)];
      D[off(g, v, rr, g.nx)] = D[off(g, v, rr, 0)];
    }
  __syncthreads();
}

template <typename T>
__device__ void store_delta(const SweepArgs<T>& a, const Geo<T>& g, const T* D, int l) {
  double* dst = a.dx_out + g.d.ptraj_off + (size_t)l * 3 * g.ny * g.nx;
  for (int idx = threadIdx.x; idx < 3 * g.Rn * g.nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // v * Rn + rr
    const int v = mdiv(q, g.mRn);
    const int rr = q - v * g.Rn, k = idx - q * g.nx;
    dst[((size_t)v * g.ny + g.R0 + rr) * g.nx + k] = (double)D[off(g, v, rr, k)];
  }
}

template <typename T, bool DEV>
__device__ void stage_tl(const SweepArgs<T>& a, const Geo<T>& g, const RowSmem<T>& rs, T* dout,
                         const T* DX, const T* Y, const T* DY, T cx, T cy) {
  const T dt = a.dt_s, Bth = a.Bth_s, gBth = a.gBth_s, href = a.href_s;
  for (int idx = threadIdx.x; idx < g.Rn * g.nx; idx += blockDim.x) {
    const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
    const int o = pidx(g, rr, k), ri = rr + 1;
    T Fh, Fu, Fv;
    T rc[8];
    load_rec8(rs.fw + 8 * ri, rc);
    Pt5<T> z, d;
    load5(Y, o, g.P, Lay<T>::CS, g.RS, z);
    load5(DY, o, g.P, Lay<T>::CS, g.RS, d);
    rhs_tl_pt<T, DEV>(z, d, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth, href, Fh, Fu, Fv);
    T xh, xu, xv;
    ld3(DX, o, g.P, xh, xu, xv);
    st3(dout, o, g.P, cx * xh + cy * (d.h + dt * Fh), cx * xu + cy * (d.u + dt * Fu),
        cx * xv + cy * (d.v + dt * Fv));
  }
}

template <typename T>
__global__ void __launch_bounds__(512) tlm_kernel(SweepArgs<T> a) {
  constexpr bool DEV = sizeof(T) == 4;
  cg::cluster_group cl = cg::this_cluster();
  Geo<T> g;
  if (!setup_geo(a, cl, g)) return;
  T* buf[6];
  RowSmem<T> rs;
  double* scratch;
  carve(a, g, 6, buf, rs, &scratch, false);
  T *X = buf[0], *S1 = buf[1], *S2 = buf[2], *D = buf[3], *D1 = buf[4], *D2 = buf[5];
  load_rows(a, g, rs);
  load_level(a, g, X, 0, g.a);
  load_delta0(a, g, D);
  if (a.dx_out) store_delta(a, g, D, 0);
  if (a.gn_dx) {
    store_block(g, D, a.gn_dx + g.d.traj_off);
    obs_level_lin(a, g, D, 0);
  }
  // Gauss-Newton products linearise about the trajectory and stage states the
  // last forward sweep stored: load them instead of recomputing them
  const bool lin_loaded = a.gn_dx && a.stg && a.ckpt == 0;
  for (int l = 0; l < g.L; ++l) {
    const int n = g.a + l;
    if (lin_loaded) {
      T* bufs[3] = {X, S1, S2};
      const T* srcs[3] = {a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp, stage_ptr(a, g, l, 0),
                          stage_ptr(a, g, l, 1)};
      const int nA[3] = {n, n + 1, n};
      const int nB[3] = {n, n + 1, n + 1};
      const T wA[3] = {(T)1, (T)1, (T)0.5};
      const T wB[3] = {(T)0, (T)0, (T)0.5};
      load_states<T, 3>(a, g, bufs, srcs, nA, nB, wA, wB);
      stage_tl<T, DEV>(a, g, rs, D1, D, X, D, (T)0, (T)1);
      complete_buf(cl, a, g, D1, K_DELTA, 0, 0, (T)1, (T)0);
      stage_tl<T, DEV>(a, g, rs, D2, D, S1, D1, (T)0.75, (T)0.25);
      complete_buf(cl, a, g, D2, K_DELTA, 0, 0, (T)1, (T)0);
      stage_tl<T, DEV>(a, g, rs, D, D, S2, D2, (T)(1.0 / 3.0), (T)(2.0 / 3.0));
      complete_buf(cl, a, g, D, K_DELTA, 0, 0, (T)1, (T)0);
      store_block(g, D, a.gn_dx + g.d.traj_off + (size_t)(l + 1) * 3 * g.ny * g.d.nxp);
      obs_level_lin(a, g, D, l + 1);
      continue;
    }
    stage_tl<T, DEV>(a, g, rs, D1, D, X, D, (T)0, (T)1);
    stage<T, DEV>(a, g, rs, S1, X, X, (T)0, (T)1);
    complete_buf(cl, a, g, S1, K_STATE, n + 1, n + 1, (T)1, (T)0);
    complete_buf(cl, a, g, D1, K_DELTA, 0, 0, (T)1, (T)0);
    stage_tl<T, DEV>(a, g, rs, D2, D, S1, D1, (T)0.75, (T)0.25);
    stage<T, DEV>(a, g, rs, S2, X, S1, (T)0.75, (T)0.25);
    complete_buf(cl, a, g, S2, K_STATE, n, n + 1, (T)0.5, (T)0.5);
    complete_buf(cl, a, g, D2, K_DELTA, 0, 0, (T)1, (T)0);
    stage_tl<T, DEV>(a, g, rs, D, D, S2, D2, (T)(1.0 / 3.0), (T)(2.0 / 3.0));
    stage<T, DEV>(a, g, rs, X, X, S2, (T)(1.0 / 3.0), (T)(2.0 / 3.0));
    complete_buf(cl, a, g, X, K_STATE, n + 1, n + 1, (T)1, (T)0);
    complete_buf(cl, a, g, D, K_DELTA, 0, 0, (T)1, (T)0);
    store_level(a, g, X, l + 1);
    if (a.dx_out) store_delta(a, g, D, l + 1);
    if (a.gn_dx) {
      store_block(g, D, a.gn_dx + g.d.traj_off + (size_t)(l + 1) * 3 * g.ny * g.d.nxp);
      obs_level_lin(a, g, D, l + 1);
    }
  }
  cl.sync();
}

// ===========================================================================
// Deep-halo FP32 sweeps: the throughput form of the FP32-state path.
//
// The stripe sweeps above exchange one halo row per RK3 stage, so a forward
// step has three cluster-barrier phases and an adjoint step three or four,
// each with a few points per thread.  Every such phase costs a roughly fixed
// latency (cluster barrier, memory fence, phase passes) whatever its work,
// and the FP32 sweeps, whose arithmetic is cheap, spend most of their time
// there.  The deep-halo sweeps keep kH = 3 halo rows on each side that has a
// neighbour CTA.  The first two stages of a step also compute the rows next to
// each neighbour's edge (four and two extra rows: the stencil of stage s + 1
// needs stage s one row further out), so a stripe needs its neighbours' values
// only once per step:
//   * after the last stage, a CTA stores its three edge rows of the new state
//     into its neighbours' exchange buffers HX (distributed shared memory) and
//     arrives at the cluster barrier (release); at the start of the next step
//     it waits (acquire) and copies its own HX into its halo rows;
//   * a second barrier phase, which a CTA arrives at once it has copied HX out
//     and waits on only before it stores into its neighbours' HX three stages
//     later, keeps a store from overwriting a buffer not yet copied out.
// The stage-state, trajectory and overlap work runs inside the stages from
// registers, with no separate passes.  Each point uses the same arithmetic
// (stage_math, adj_stage_math, adj_lambda_math) as the stripe sweeps, so both
// give the same values bit for bit.  Every stripe needs at least kH rows.
// Buffers: [R + 2 kH rows][W][4] FP32 slots (h, u, v, 0), rows -kH .. R + kH - 1.

constexpr int kH = 3;            // halo rows per side
constexpr int kMaxP = 4;         // own points per thread (register state of the last stage)
constexpr int kDeepThreads = 640;

struct G2 {
  int s, rank, CL, R0, Rn, nx, ny, L, a, W, flags, RS, R;
  bool hasS, hasN;                // neighbour CTA to the south / north
  SubDesc d;
  unsigned mnx;
  float* gh;                      // ghost cache: 3 slots of [6 (R + 4) column | 6 W row] values
  int* gh_tag;
  int gh_len;
};

__device__ __forceinline__ int p2(const G2& g, int rr, int k) { return ((rr + kH) * g.W + k + 1) * 4; }
// rows computed by stage st = 1, 2, 3 (kH - st rows beyond a neighbour edge)
__device__ __forceinline__ int lo_st(const G2& g, int st) { return g.hasS ? st - kH : 0; }
__device__ __forceinline__ int hi_st(const G2& g, int st) { return g.hasN ? g.Rn - 1 + kH - st : g.Rn - 1; }

__device__ __forceinline__ bool setup_g2(const SweepArgs<float>& a, cg::cluster_group& cl, G2& g) {
  g.rank = cl.block_rank();
  g.CL = cl.num_blocks();
  const int cid = blockIdx.x / g.CL;
  if (cid >= a.n_sub) return false;
  g.s = a.order[cid];
  if (a.active && a.active[g.s] != a.active_value) return false;
  g.d = a.subs[g.s];
  g.nx = g.d.nx;
  g.ny = g.d.ny;
  g.a = g.d.a;
  g.L = g.d.b - g.d.a;
  g.flags = g.d.flags;
  if (g.ny < kH * g.CL || g.nx + 2 > a.W || (g.ny + g.CL - 1) / g.CL > a.R ||
      (g.ny + g.CL - 1) / g.CL * g.nx > kMaxP * (int)blockDim.x) {   // uniform over the cluster
    if (threadIdx.x == 0 && g.rank == 0) atomicExch(a.err, 2);
    return false;
  }
  split_rows(g.ny, g.CL, g.rank, g.R0, g.Rn);
  g.R = a.R;
  g.W = a.W;
  g.RS = g.W * 4;
  g.hasS = g.rank > 0;
  g.hasN = g.rank < g.CL - 1;
  if (g.rank != 0) g.flags &= ~F_SWALL;
  if (g.rank != g.CL - 1) g.flags &= ~F_NWALL;
  g.mnx = magic_of(g.nx);
  return true;
}

// nbuf state buffers, the exchange buffer (2 kH rows of [W][4]), row constants
// of rows -kH .. R + kH - 1 (forward and adjoint records), reduction scratch,
// ghost cache.
__host__ __device__ constexpr size_t deep_buf_floats(int R, int W) { return (size_t)(R + 2 * kH) * W * 4; }
size_t smem_deep(int nbuf, int R, int W) {
  size_t b = (nbuf * deep_buf_floats(R, W) + (size_t)2 * kH * W * 4 + 16 * (size_t)(R + 2 * kH)) * sizeof(float);
  b = (b + 15) / 16 * 16 + 64 * sizeof(double);
  return b + 3 * (size_t)(6 * (R + 4) + 6 * W) * sizeof(float) + 3 * sizeof(int) + 16;
}

__device__ void carve2(G2& g, int nbuf, float** bufs, float** hx, float** fw, float** bw, double** scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* p = reinterpret_cast<float*>(smem_raw);
  for (int b = 0; b < nbuf; ++b) {
    bufs[b] = p;
    p += deep_buf_floats(g.R, g.W);
  }
  *hx = p;
  p += 2 * kH * g.W * 4;
  *fw = p;
  p += 8 * (g.R + 2 * kH);
  *bw = p;
  p += 8 * (g.R + 2 * kH);
  uintptr_t q = reinterpret_cast<uintptr_t>(p);
  q = (q + 15) & ~uintptr_t(15);
  *scratch = reinterpret_cast<double*>(q);
  q += 64 * sizeof(double);
  g.gh_len = 6 * (g.R + 4) + 6 * g.W;
  g.gh = reinterpret_cast<float*>(q);
  g.gh_tag = reinterpret_cast<int*>(q + 3 * (size_t)g.gh_len * sizeof(float));
  if (threadIdx.x < 3) g.gh_tag[threadIdx.x] = -1;
}

// Row constants (as load_rows) of rows -kH .. Rn + kH - 1.
__device__ void load_rows2(const SweepArgs<float>& a, const G2& g, float* fw, float* bw) {
  for (int i = threadIdx.x; i < g.Rn + 2 * kH; i += blockDim.x) {
    const int j = g.d.j0 + g.R0 + i - kH;
    const int jc = min(max(j, 0), a.nlat - 1);
    const int jn = min(max(j + 1, 0), a.nlat - 1);
    const int js = min(max(j - 1, 0), a.nlat - 1);
    const RowConst rc = a.rows[jc];
    const double cn = a.rows[jn].c, cs = a.rows[js].c;
    float* f = fw + 8 * i;
    f[0] = (float)rc.A;
    f[1] = (float)rc.f;
    f[2] = (float)rc.tau;
    f[3] = (float)rc.BinvC;
    f[4] = (float)rc.gA;
    f[5] = (float)cn;
    f[6] = (float)cs;
    f[7] = 0.0f;
    float* b = bw + 8 * i;
    b[0] = (float)rc.A;
    b[1] = (float)rc.f;
    b[2] = (float)rc.tau;
    b[3] = (float)rc.gA;
    b[4] = (float)(a.Bth * rc.c);
    b[5] = (float)(1.0 / cn);
    b[6] = (float)(1.0 / cs);
    b[7] = (float)(2.0 * rc.tau);
  }
}

// Ghost values of boundary level n into slot n % 3 (cp.async, joins the
// caller's next commit group): west / east columns (box not periodic) of the
// rows the first stage computes, and the south / north rows of a stripe at a
// frozen box edge.
__device__ void ghost_prefetch2(const SweepArgs<float>& a, const G2& g, int n) {
  if (n < 0 || n > a.nsteps) return;
  const int slot = n % 3;
  float* dst = g.gh + (size_t)slot * g.gh_len;
  const size_t plane = (size_t)a.nlat * a.nlon;
  const float* src = a.bnd + (size_t)n * 3 * plane;
  const int RC = g.R + 4;
  if (!(g.flags & F_PERIODIC)) {
    const int r0 = lo_st(g, 1), nr = hi_st(g, 1) - r0 + 1;
    const int iw = (g.d.i0 - 1 + a.nlon) % a.nlon, ie = (g.d.i0 + g.nx) % a.nlon;
    for (int idx = threadIdx.x; idx < 6 * nr; idx += blockDim.x) {
      const int q = idx / nr;   // side * 3 + v
      const int side = q / 3;
      const int v = q - 3 * side, rr = r0 + idx - q * nr;
      const int j = g.d.j0 + g.R0 + rr;
      cp_async_4or8(dst + q * RC + rr + 2, src + ((size_t)v * a.nlat + j) * a.nlon + (side ? ie : iw), 4);
    }
  }
  const bool south = g.rank == 0 && !(g.flags & F_SWALL);
  const bool north = g.rank == g.CL - 1 && !(g.flags & F_NWALL);
  if (south || north) {
    for (int idx = threadIdx.x; idx < 6 * g.nx; idx += blockDim.x) {
      const int q = mdiv(idx, g.mnx);
      const int side = q / 3;
      if ((side == 0 && !south) || (side == 1 && !north)) continue;
      const int v = q - 3 * side, k = idx - q * g.nx;
      const int j = side ? g.d.j0 + g.ny : g.d.j0 - 1;
      cp_async_4or8(dst + 6 * RC + q * g.W + k, src + ((size_t)v * a.nlat + j) * a.nlon + (g.d.i0 + k) % a.nlon,
                    4);
    }
  }
  if (threadIdx.x == 0) g.gh_tag[slot] = n;
}

// The boundary trajectory blended between levels nA and nB, from the ghost
// cache when both levels are there (else from HBM; same values).
struct GS2 {
  const float* ca;
  const float* cb;
  int nA, nB;
  float wA, wB;
};
__device__ __forceinline__ GS2 ghost_src2(const G2& g, int nA, int nB, float wA, float wB) {
  GS2 s{nullptr, nullptr, nA, nB, wA, wB};
  if (nA >= 0 && nB >= 0 && g.gh_tag[nA % 3] == nA && (wB == 0.0f || g.gh_tag[nB % 3] == nB)) {
    s.ca = g.gh + (size_t)(nA % 3) * g.gh_len;
    s.cb = (wB == 0.0f) ? nullptr : g.gh + (size_t)(nB % 3) * g.gh_len;
  }
  return s;
}
__device__ __forceinline__ float bnd_blend2(const SweepArgs<float>& a, const GS2& s, int v, int j, int i) {
  const size_t plane = (size_t)a.nlat * a.nlon;
  const size_t o = ((size_t)v * a.nlat + j) * a.nlon + i;
  const float xa = a.bnd[(size_t)s.nA * 3 * plane + o];
  if (s.wB == 0.0f) return xa;
  return xfma(s.wA, xa, xmul(s.wB, a.bnd[(size_t)s.nB * 3 * plane + o]));
}
__device__ __forceinline__ float gh_col2(const SweepArgs<float>& a, const G2& g, const GS2& s, int side, int v,
                                         int rr) {
  if (s.ca) {
    const int o = (side * 3 + v) * (g.R + 4) + rr + 2;
    const float xa = s.ca[o];
    return s.cb ? xfma(s.wA, xa, xmul(s.wB, s.cb[o])) : xa;
  }
  const int i = side == 0 ? (g.d.i0 - 1 + a.nlon) % a.nlon : (g.d.i0 + g.nx) % a.nlon;
  return bnd_blend2(a, s, v, g.d.j0 + g.R0 + rr, i);
}
__device__ __forceinline__ float gh_row2(const SweepArgs<float>& a, const G2& g, const GS2& s, int side, int v,
                                         int k) {
  if (s.ca) {
    const int o = 6 * (g.R + 4) + (side * 3 + v) * g.W + k;
    const float xa = s.ca[o];
    return s.cb ? xfma(s.wA, xa, xmul(s.wB, s.cb[o])) : xa;
  }
  return bnd_blend2(a, s, v, side ? g.d.j0 + g.ny : g.d.j0 - 1, (g.d.i0 + k) % a.nlon);
}

// Ghost cells of buffer Z that do not depend on its values, for stencil
// centres on rows [lo, hi]: at a frozen box edge the boundary trajectory
// (state buffers) or zero (adjoint buffers, which are also zero at walls);
// ghost columns when the box is not periodic.  Highest-numbered threads first.
__device__ void fill_fixed2(const SweepArgs<float>& a, const G2& g, float* Z, int lo, int hi, const GS2& gs,
                            bool adj) {
  const bool cols = !(g.flags & F_PERIODIC);
  const bool srow = g.rank == 0 && (adj || !(g.flags & F_SWALL));
  const bool nrow = g.rank == g.CL - 1 && (adj || !(g.flags & F_NWALL));
  const int nr = hi - lo + 1;
  const int n = 2 * g.nx + (cols ? 2 * nr : 0);
  for (int idx = blockDim.x - 1 - threadIdx.x; idx < n; idx += blockDim.x) {
    float h = 0.0f, u = 0.0f, v = 0.0f;
    if (idx < 2 * g.nx) {
      const int side = idx >= g.nx ? 1 : 0;
      if (side ? !nrow : !srow) continue;
      const int k = idx - side * g.nx;
      if (!adj) {
        h = gh_row2(a, g, gs, side, 0, k);
        u = gh_row2(a, g, gs, side, 1, k);
        v = gh_row2(a, g, gs, side, 2, k);
      }
      st3(Z, p2(g, side ? g.Rn : -1, k), 1, h, u, v);
    } else {
      const int j = idx - 2 * g.nx;
      const int side = j >= nr ? 1 : 0;
      const int rr = lo + j - side * nr;
      if (!adj) {
        h = gh_col2(a, g, gs, side, 0, rr);
        u = gh_col2(a, g, gs, side, 1, rr);
        v = gh_col2(a, g, gs, side, 2, rr);
      }
      st3(Z, p2(g, rr, side ? g.nx : -1), 1, h, u, v);
    }
  }
}

// Halo data a computed point (rr, k) of Z publishes in its own buffer: the
// periodic ghost columns and, for state buffers, the wall mirror row.
__device__ __forceinline__ void publish2(const G2& g, float* Z, bool state, int rr, int k, float v0, float v1,
                                         float v2) {
  if (g.flags & F_PERIODIC) {
    if (k == 0) st3(Z, p2(g, rr, g.nx), 1, v0, v1, v2);
    if (k == g.nx - 1) st3(Z, p2(g, rr, -1), 1, v0, v1, v2);
  }
  if (state) {
    if (rr == 0 && (g.flags & F_SWALL)) st3(Z, p2(g, -1, k), 1, v0, v1, -v2);
    if (rr == g.Rn - 1 && (g.flags & F_NWALL)) st3(Z, p2(g, g.Rn, k), 1, v0, v1, -v2);
  }
}

// Stores point (rr, k) of a buffer's new edge rows into the neighbours'
// exchange buffers (their halo rows -kH .. -1 and Rn .. Rn + kH - 1).
__device__ __forceinline__ void push2(const G2& g, float* hxS, float* hxN, int rr, int k, float v0, float v1,
                                      float v2) {
  if (hxS && rr < kH) *reinterpret_cast<float4*>(hxS + ((kH + rr) * g.W + k) * 4) = make_float4(v0, v1, v2, 0.0f);
  if (hxN && rr >= g.Rn - kH)
    *reinterpret_cast<float4*>(hxN + ((rr - (g.Rn - kH)) * g.W + k) * 4) = make_float4(v0, v1, v2, 0.0f);
}

// Halo rows of Z from this CTA's exchange buffer (with their periodic ghost
// columns).
__device__ void copy_hx2(const G2& g, const float* HX, float* Z) {
  const int nrow = (g.hasS ? kH : 0) + (g.hasN ? kH : 0);
  for (int idx = threadIdx.x; idx < nrow * g.nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);
    const int k = idx - q * g.nx;
    const int hr = g.hasS ? q : q + kH;
    const int rr = hr < kH ? hr - kH : g.Rn + hr - kH;
    const float4 v = *reinterpret_cast<const float4*>(HX + (hr * g.W + k) * 4);
    *reinterpret_cast<float4*>(Z + p2(g, rr, k)) = v;
    if (g.flags & F_PERIODIC) {
      if (k == 0) *reinterpret_cast<float4*>(Z + p2(g, rr, g.nx)) = v;
      if (k == g.nx - 1) *reinterpret_cast<float4*>(Z + p2(g, rr, -1)) = v;
    }
  }
}

// Rows [lo, hi] of a stored [3][ny][nxp] block into Z with cp.async (the
// caller commits and waits), their periodic ghost columns too, and at a wall
// the mirror row (read directly).  A warp's 4-byte copies into 16-byte slots
// would hit every bank four times; each group of eight lanes starts at a
// different slot component instead (four copies per point, the unused fourth
// component taking h), which spreads every copy instruction over all banks.
__device__ void load_rows_async2(const G2& g, float* Z, const float* src, int lo, int hi) {
  const size_t pl = (size_t)g.ny * g.d.nxp;
  const int n = (hi - lo + 1) * g.nx;
  const bool per = g.flags & F_PERIODIC;
  const int rot = (threadIdx.x >> 3) & 3;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);
    const int rr = lo + q, k = idx - q * g.nx;
    const float* s = src + (size_t)(g.R0 + rr) * g.d.nxp + k;
    float* d = Z + p2(g, rr, k);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int v = (c + rot) & 3;
      cp_async_4or8(d + v, s + (size_t)(v < 3 ? v : 0) * pl, 4);
    }
    if (per && (k == 0 || k == g.nx - 1)) {
      float* e = Z + p2(g, rr, k == 0 ? g.nx : -1);
      cp_async_4or8(e, s, 4);
      cp_async_4or8(e + 1, s + pl, 4);
      cp_async_4or8(e + 2, s + 2 * pl, 4);
    }
    if ((rr == 0 && (g.flags & F_SWALL)) || (rr == g.Rn - 1 && (g.flags & F_NWALL)))
      st3(Z, p2(g, rr == 0 ? -1 : g.Rn, k), 1, s[0], s[pl], -s[2 * pl]);
  }
}

// Rows a stored state must cover for stencil centres [lo, hi]: one row more
// on each side that has a neighbour (the box edge rows come from the rules).
__device__ __forceinline__ int load_lo2(const G2& g, int lo) { return g.hasS ? lo - 1 : 0; }
__device__ __forceinline__ int load_hi2(const G2& g, int hi) { return g.hasN ? hi + 1 : g.Rn - 1; }

__device__ __forceinline__ int overlap_count2(const G2& g, int l, int r, int k) {
  const SubDesc& d = g.d;
  const int cx = 1 + (k < d.wL) + (k >= d.nx - d.wR);
  const int cy = 1 + (r < d.wS) + (r >= d.ny - d.wN);
  const int ct = 1 + (l < d.tA) + (l > g.L - d.tB);
  return cx * cy * ct - 1;
}
__device__ __forceinline__ bool level_overlaps2(const G2& g, int l) {
  const SubDesc& d = g.d;
  return (l < d.tA) || (l > g.L - d.tB) || d.wL || d.wR || d.wS || d.wN;
}

// Overlap counts and targets of level l at this thread's own points (points
// t + i T of the own rows, i < kMaxP), loaded ahead of their use.
__device__ __forceinline__ void prefetch_own_targets2(const SweepArgs<float>& a, const G2& g, int l, int (&cv)[kMaxP],
                                                      float (&tv)[kMaxP][3]) {
  const bool any = a.mu != 0.0 && level_overlaps2(g, l);
  const size_t pl = (size_t)g.ny * g.d.nxp;
  const float* tg = a.tgt + g.d.traj_off + (size_t)l * 3 * pl;
#pragma unroll
  for (int i = 0; i < kMaxP; ++i) {
    cv[i] = 0;
    tv[i][0] = tv[i][1] = tv[i][2] = 0.0f;
    const int idx = threadIdx.x + i * blockDim.x;
    if (any && idx < g.Rn * g.nx) {
      const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
      const int c = overlap_count2(g, l, g.R0 + rr, k);
      cv[i] = c;
      if (c) {
        const float* t = tg + (size_t)(g.R0 + rr) * g.d.nxp + k;
        tv[i][0] = t[0];
        tv[i][1] = t[pl];
        tv[i][2] = t[2 * pl];
      }
    }
  }
}

// Observation misfit of level l (as obs_level): J_o += 1/2 w d^2, obs_force.
__device__ void obs_level2(const SweepArgs<float>& a, const G2& g, const float* X, int l, double& Jo) {
  const int o0 = a.lvl_obs[g.d.obs_lvl + l], o1 = a.lvl_obs[g.d.obs_lvl + l + 1];
  for (int o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    const ObsRec ob = a.obs[o];
    const int rr = ob.r0 - g.R0;
    if (rr < 0 || rr >= g.Rn) continue;
    const double x00 = (double)X[p2(g, rr, ob.k0) + ob.var];
    const double x01 = ob.di != 0.0 ? (double)X[p2(g, rr, ob.k1) + ob.var] : 0.0;
    const double x10 = ob.dj != 0.0 ? (double)X[p2(g, rr + 1, ob.k0) + ob.var] : 0.0;
    const double x11 = (ob.dj != 0.0 && ob.di != 0.0) ? (double)X[p2(g, rr + 1, ob.k1) + ob.var] : 0.0;
    a.obs_force[o] = obs_term(ob, x00, x01, x10, x11, a.lam, Jo);
  }
}

// One forward stage st on rows [lo_st, hi_st]: out = cx X + cy (Y + dt F(Y));
// own rows also go to the stage buffer hbm (when given).
template <int ST>
__device__ __forceinline__ void stage_rows2(const SweepArgs<float>& a, const G2& g, const float* fw, float* out,
                                            const float* X, const float* Y, float cx, float cy, float* hbm) {
  const int lo = lo_st(g, ST), hi = hi_st(g, ST);
  const int n = (hi - lo + 1) * g.nx;
  const size_t pl = (size_t)g.ny * g.d.nxp;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);
    const int rr = lo + q, k = idx - q * g.nx;
    const int o = p2(g, rr, k);
    float rc[8];
    load_rec8(fw + 8 * (rr + kH), rc);
    Pt5<float> y;
    load5(Y, o, 1, 4, g.RS, y);
    float xh = 0.0f, xu = 0.0f, xv = 0.0f;
    if (cx != 0.0f) ld3(X, o, 1, xh, xu, xv);
    float o0, o1, o2;
    stage_math<float, true>(y, rc, a.dt_s, a.Bth_s, a.gBth_s, a.href_s, cx, cy, xh, xu, xv, o0, o1, o2);
    st3(out, o, 1, o0, o1, o2);
    publish2(g, out, true, rr, k, o0, o1, o2);
    if (hbm && rr >= 0 && rr < g.Rn) {
      float* d = hbm + (size_t)(g.R0 + rr) * g.d.nxp + k;
      d[0] = o0;
      d[pl] = o1;
      d[2 * pl] = o2;
    }
  }
}

__device__ __forceinline__ float* stage_ptr2(const SweepArgs<float>& a, const SubDesc& d, int l, int which) {
  return a.stg + d.stg_off + ((size_t)l * 2 + which) * 3 * d.ny * d.nxp;
}
// All but the two (one) most recently committed cp.async groups complete.
__device__ __forceinline__ void cp_async_wait_prev2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one2() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}

// Forward sweep, deep-halo form (same results as fwd_kernel<float>).
__global__ void __launch_bounds__(kDeepThreads, 1) fwd_deep_kernel(SweepArgs<float> a) {
  cg::cluster_group cl = cg::this_cluster();
  G2 g;
  if (!setup_g2(a, cl, g)) return;
  float* buf[3];
  float *HX, *fw, *bw;
  double* scratch;
  carve2(g, 3, buf, &HX, &fw, &bw, &scratch);
  float* X = buf[0];
  float* S1 = buf[1];
  float* S2 = buf[2];
  float* hxS = g.hasS ? cl.map_shared_rank(HX, g.rank - 1) : nullptr;
  float* hxN = g.hasN ? cl.map_shared_rank(HX, g.rank + 1) : nullptr;
  load_rows2(a, g, fw, bw);
  __syncthreads();   // ghost tags initialised
  ghost_prefetch2(a, g, g.a);
  if (g.L > 0) ghost_prefetch2(a, g, g.a + 1);
  const size_t pl = (size_t)g.ny * g.d.nxp;
  const size_t lvl = 3 * pl;
  // x(a) (written by the initial-state kernel): own rows and the halo rows of stage 1
  load_rows_async2(g, X, a.traj + g.d.traj_off, load_lo2(g, lo_st(g, 1)), load_hi2(g, hi_st(g, 1)));
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  fill_fixed2(a, g, X, lo_st(g, 1), hi_st(g, 1), ghost_src2(g, g.a, g.a, 1.0f, 0.0f), false);
  __syncthreads();
  double Jo = 0.0, Jm = 0.0;
  obs_level2(a, g, X, 0, Jo);
  {
    int cv[kMaxP];
    float tv[kMaxP][3];
    prefetch_own_targets2(a, g, 0, cv, tv);
    const float i0 = a.isb2_s[0], i1 = a.isb2_s[1], i2 = a.isb2_s[2];
    float part = 0.0f;
#pragma unroll
    for (int i = 0; i < kMaxP; ++i) {
      const int idx = threadIdx.x + i * blockDim.x;
      if (cv[i]) {
        const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
        float x0, x1, x2;
        ld3(X, p2(g, rr, k), 1, x0, x1, x2);
        part = overlap_term(part, cv[i], x0, x1, x2, tv[i][0], tv[i][1], tv[i][2], i0, i1, i2);
      }
    }
    Jm += (double)part;
  }
  const float c13 = (float)(1.0 / 3.0), c23 = (float)(2.0 / 3.0);
  for (int l = 0; l < g.L; ++l) {
    const int n = g.a + l;
    if (l > 0) {
      cluster_wait_acquire();   // neighbours' edge rows of x(n) are in HX
      copy_hx2(g, HX, X);
      cp_async_wait_all();      // ghost levels n, n + 1
      __syncthreads();
      fill_fixed2(a, g, X, lo_st(g, 1), hi_st(g, 1), ghost_src2(g, n, n, 1.0f, 0.0f), false);
      __syncthreads();
      obs_level2(a, g, X, l, Jo);
    }
    cluster_arrive_relaxed();   // this CTA has copied its exchange buffer out
    if (n + 2 <= g.d.b) ghost_prefetch2(a, g, n + 2);
    cp_async_commit();
    int cv[kMaxP];
    float tv[kMaxP][3];
    prefetch_own_targets2(a, g, l + 1, cv, tv);
    // stage 1: x1 = x + dt F(x)
    fill_fixed2(a, g, S1, lo_st(g, 2), hi_st(g, 2), ghost_src2(g, n + 1, n + 1, 1.0f, 0.0f), false);
    stage_rows2<1>(a, g, fw, S1, X, X, 0.0f, 1.0f, a.stg ? stage_ptr2(a, g.d, l, 0) : nullptr);
    __syncthreads();
    // stage 2: x2 = 3/4 x + 1/4 (x1 + dt F(x1))
    fill_fixed2(a, g, S2, 0, g.Rn - 1, ghost_src2(g, n, n + 1, 0.5f, 0.5f), false);
    stage_rows2<2>(a, g, fw, S2, X, S1, 0.75f, 0.25f, a.stg ? stage_ptr2(a, g.d, l, 1) : nullptr);
    __syncthreads();
    cluster_wait_acquire();   // neighbours have copied their exchange buffers out
    // stage 3: x(n+1) = 1/3 x + 2/3 (x2 + dt F(x2)) on own rows, in place;
    // edge rows into the neighbours' exchange buffers; overlap term of level l + 1
    const float i0 = a.isb2_s[0], i1 = a.isb2_s[1], i2 = a.isb2_s[2];
    float part = 0.0f;
#pragma unroll
    for (int i = 0; i < kMaxP; ++i) {
      const int idx = threadIdx.x + i * blockDim.x;
      if (idx < g.Rn * g.nx) {
        const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
        const int o = p2(g, rr, k);
        float rc[8];
        load_rec8(fw + 8 * (rr + kH), rc);
        Pt5<float> y;
        load5(S2, o, 1, 4, g.RS, y);
        float xh, xu, xv;
        ld3(X, o, 1, xh, xu, xv);
        float o0, o1, o2;
        stage_math<float, true>(y, rc, a.dt_s, a.Bth_s, a.gBth_s, a.href_s, c13, c23, xh, xu, xv, o0, o1, o2);
        st3(X, o, 1, o0, o1, o2);
        publish2(g, X, true, rr, k, o0, o1, o2);
        push2(g, hxS, hxN, rr, k, o0, o1, o2);
        if (cv[i]) {
          part = overlap_term(part, cv[i], o0, o1, o2, tv[i][0], tv[i][1], tv[i][2], i0, i1, i2);
        }
      }
    }
    Jm += (double)part;
    cluster_arrive_release();   // x(n+1) edge rows are in the neighbours' exchange buffers
    if (a.ckpt == 0 || (l + 1) % a.ckpt == 0) {
      float* dst = a.traj + g.d.traj_off + (size_t)(l + 1) * lvl;
#pragma unroll
      for (int i = 0; i < kMaxP; ++i) {
        const int idx = threadIdx.x + i * blockDim.x;
        if (idx < g.Rn * g.nx) {
          const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
          float h, u, v;
          ld3(X, p2(g, rr, k), 1, h, u, v);   // written by this thread
          float* d = dst + (size_t)(g.R0 + rr) * g.d.nxp + k;
          d[0] = h;
          d[pl] = u;
          d[2 * pl] = v;
        }
      }
    }
  }
  if (g.L > 0) {
    cluster_wait_acquire();
    copy_hx2(g, HX, X);
    __syncthreads();
    obs_level2(a, g, X, g.L, Jo);
  }
  Jm *= 0.5;
  block_reduce2<float>(Jo, Jm, scratch);
  if (threadIdx.x == 0) {
    a.part[((size_t)g.s * a.cl_max + g.rank) * 2 + 0] = Jo;
    a.part[((size_t)g.s * a.cl_max + g.rank) * 2 + 1] = Jm;
  }
}

// Adjoint forcing on own rows at level l that follows the overlap term: the
// observation scatter (H^T of lambda w d, fixed order per target), as in
// add_forcing.
__device__ void scatter2(const SweepArgs<float>& a, const G2& g, float* Lb, int l) {
  const int t0 = a.lvl_sc[g.d.sc_lvl + l], t1 = a.lvl_sc[g.d.sc_lvl + l + 1];
  const unsigned mny = magic_of(g.ny);
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const int tg = a.sc_tgt[t];
    const int q = mdiv(tg, g.mnx);   // v * ny + r
    const int v = mdiv(q, mny);
    const int r = q - v * g.ny, k = tg - q * g.nx;
    const int rr = r - g.R0;
    if (rr < 0 || rr >= g.Rn) continue;
    double acc = 0.0;
    for (int c = a.sc_off[t]; c < a.sc_off[t + 1]; ++c) acc += a.sc_w[c] * a.obs_force[a.sc_obs[c]];
    Lb[p2(g, rr, k) + v] += (float)acc;
  }
}

// Overlap forcing mu c (x - m) / sb^2 added to (l0, l1, l2), the arithmetic of
// overlap_force with the targets given.
__device__ __forceinline__ void overlap_force2(const SweepArgs<float>& a, float x0, float x1, float x2,
                                               const float (&t)[3], int c, float& l0, float& l1, float& l2) {
  const float cc = (float)c;
  l0 = xfma(xmul(cc, a.musb2_s[0]), xsub(x0, t[0]), l0);
  l1 = xfma(xmul(cc, a.musb2_s[1]), xsub(x1, t[1]), l1);
  l2 = xfma(xmul(cc, a.musb2_s[2]), xsub(x2, t[2]), l2);
}

// Adjoint sweep, deep-halo form, with stage states stored by the forward
// sweep (same results as adj_kernel<float> in that mode).
__global__ void __launch_bounds__(kDeepThreads, 1) adj_deep_kernel(SweepArgs<float> a) {
  cg::cluster_group cl = cg::this_cluster();
  G2 g;
  if (!setup_g2(a, cl, g)) return;
  float* buf[5];
  float *HX, *fw, *bw;
  double* scratch;
  carve2(g, 5, buf, &HX, &fw, &bw, &scratch);
  float* X = buf[0];
  float* X1 = buf[1];
  float* X2 = buf[2];   // x2, then mu1
  float* Lp = buf[3];   // lambda(n+1), then lambda(n)
  float* L2 = buf[4];   // mu2
  float* hxS = g.hasS ? cl.map_shared_rank(HX, g.rank - 1) : nullptr;
  float* hxN = g.hasN ? cl.map_shared_rank(HX, g.rank + 1) : nullptr;
  load_rows2(a, g, fw, bw);
  // adjoint buffers start at zero: their box-edge ghost rows and the ghost
  // columns of a non-periodic box stay zero
  const int BUF = (int)deep_buf_floats(g.R, g.W);
  for (int i = threadIdx.x; i < BUF; i += blockDim.x) {
    Lp[i] = 0.0f;
    L2[i] = 0.0f;
  }
  __syncthreads();   // ghost tags initialised
  ghost_prefetch2(a, g, g.a + g.L);
  if (g.L > 0) ghost_prefetch2(a, g, g.a + g.L - 1);
  cp_async_commit();
  const size_t pl = (size_t)g.ny * g.d.nxp;
  const size_t lvl = 3 * pl;
  const float dt = a.dt_s, Bth = a.Bth_s, gBth = a.gBth_s, href = a.href_s;
  // lambda(b) = forcing(b) on own rows
  load_rows_async2(g, X, a.traj + g.d.traj_off + (size_t)g.L * lvl, 0, g.Rn - 1);
  cp_async_commit();
  int cv[kMaxP];
  float tv[kMaxP][3];
  prefetch_own_targets2(a, g, g.L, cv, tv);
  cp_async_wait_all();
  __syncthreads();
  cl.sync();   // every CTA of the cluster runs before any exchange-buffer store
#pragma unroll
  for (int i = 0; i < kMaxP; ++i) {
    const int idx = threadIdx.x + i * blockDim.x;
    if (cv[i]) {
      const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
      const int o = p2(g, rr, k);
      float x0, x1, x2, l0, l1, l2;
      ld3(X, o, 1, x0, x1, x2);
      ld3(Lp, o, 1, l0, l1, l2);
      overlap_force2(a, x0, x1, x2, tv[i], cv[i], l0, l1, l2);
      st3(Lp, o, 1, l0, l1, l2);
    }
  }
  __syncthreads();
  scatter2(a, g, Lp, g.L);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kMaxP; ++i) {
    const int idx = threadIdx.x + i * blockDim.x;
    if (idx < g.Rn * g.nx) {
      const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
      float v0, v1, v2;
      ld3(Lp, p2(g, rr, k), 1, v0, v1, v2);
      publish2(g, Lp, false, rr, k, v0, v1, v2);
      push2(g, hxS, hxN, rr, k, v0, v1, v2);
    }
  }
  cluster_arrive_release();
  const int wall_s = (g.flags & F_SWALL) ? 1 : 0;
  const int wall_n = (g.flags & F_NWALL) ? 2 : 0;
  for (int l = g.L - 1; l >= 0; --l) {
    const int n = g.a + l;
    cluster_wait_acquire();   // lambda(n+1) edge rows in HX; the previous step's phases are done
    if (l > 0) ghost_prefetch2(a, g, n - 1);
    cp_async_commit();
    const float* trl = a.traj + g.d.traj_off + (size_t)l * lvl;
    const float* s1 = a.stg + g.d.stg_off + ((size_t)l * 2 + 0) * lvl;
    const float* s2 = a.stg + g.d.stg_off + ((size_t)l * 2 + 1) * lvl;
    load_rows_async2(g, X2, s2, load_lo2(g, lo_st(g, 1)), load_hi2(g, hi_st(g, 1)));
    cp_async_commit();
    load_rows_async2(g, X1, s1, load_lo2(g, lo_st(g, 2)), load_hi2(g, hi_st(g, 2)));
    cp_async_commit();
    load_rows_async2(g, X, trl, load_lo2(g, lo_st(g, 3)), load_hi2(g, hi_st(g, 3)));
    cp_async_commit();
    copy_hx2(g, HX, Lp);
    prefetch_own_targets2(a, g, l, cv, tv);
    fill_fixed2(a, g, X2, lo_st(g, 1), hi_st(g, 1), ghost_src2(g, n, n + 1, 0.5f, 0.5f), false);
    fill_fixed2(a, g, X1, lo_st(g, 2), hi_st(g, 2), ghost_src2(g, n + 1, n + 1, 1.0f, 0.0f), false);
    fill_fixed2(a, g, X, 0, g.Rn - 1, ghost_src2(g, n, n, 1.0f, 0.0f), false);
    cp_async_wait_prev2();   // ghost level n - 1 and x2 have landed (x1, x may still be in flight)
    __syncthreads();
    cluster_arrive_relaxed();   // this CTA has copied its exchange buffer out
    // mu2 = lambda' + dt F'(x2)^T lambda'
    {
      const int lo = lo_st(g, 1), hi = hi_st(g, 1);
      for (int idx = threadIdx.x; idx < (hi - lo + 1) * g.nx; idx += blockDim.x) {
        const int q = mdiv(idx, g.mnx);
        const int rr = lo + q, k = idx - q * g.nx;
        const int o = p2(g, rr, k);
        const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
        float rc[8];
        load_rec8(bw + 8 * (rr + kH), rc);
        Pt5<float> z, m;
        load5(X2, o, 1, 4, g.RS, z);
        load5(Lp, o, 1, 4, g.RS, m);
        float v0, v1, v2;
        adj_stage_math<float, true>(z, m, rc, dt, Bth, gBth, href, wall, v0, v1, v2);
        st3(L2, o, 1, v0, v1, v2);
        publish2(g, L2, false, rr, k, v0, v1, v2);
      }
    }
    cp_async_wait_one2();   // x1 has landed
    __syncthreads();
    // mu1 = mu2 + dt F'(x1)^T mu2, into x2's buffer, whose ghosts become adjoint zeros
    {
      fill_fixed2(a, g, X2, 0, g.Rn - 1, ghost_src2(g, n, n, 1.0f, 0.0f), true);
      const int lo = lo_st(g, 2), hi = hi_st(g, 2);
      for (int idx = threadIdx.x; idx < (hi - lo + 1) * g.nx; idx += blockDim.x) {
        const int q = mdiv(idx, g.mnx);
        const int rr = lo + q, k = idx - q * g.nx;
        const int o = p2(g, rr, k);
        const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
        float rc[8];
        load_rec8(bw + 8 * (rr + kH), rc);
        Pt5<float> z, m;
        load5(X1, o, 1, 4, g.RS, z);
        load5(L2, o, 1, 4, g.RS, m);
        float v0, v1, v2;
        adj_stage_math<float, true>(z, m, rc, dt, Bth, gBth, href, wall, v0, v1, v2);
        st3(X2, o, 1, v0, v1, v2);
        publish2(g, X2, false, rr, k, v0, v1, v2);
      }
    }
    cp_async_wait_all();   // x has landed
    __syncthreads();
    cluster_wait_acquire();   // neighbours have copied their exchange buffers out
    // lambda(n) on own rows, in place, with the overlap forcing of level l;
    // without observations at this level the edge rows go to the neighbours here
    const bool obs_here = a.lvl_sc[g.d.sc_lvl + l] != a.lvl_sc[g.d.sc_lvl + l + 1];
#pragma unroll
    for (int i = 0; i < kMaxP; ++i) {
      const int idx = threadIdx.x + i * blockDim.x;
      if (idx < g.Rn * g.nx) {
        const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
        const int o = p2(g, rr, k);
        const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
        float rc[8];
        load_rec8(bw + 8 * (rr + kH), rc);
        Pt5<float> z, m;
        load5(X, o, 1, 4, g.RS, z);
        load5(X2, o, 1, 4, g.RS, m);
        float ph, pu, pv, qh, qu, qv;
        ld3(Lp, o, 1, ph, pu, pv);
        ld3(L2, o, 1, qh, qu, qv);
        float v0, v1, v2;
        adj_lambda_math<float, true>(z, m, rc, dt, Bth, gBth, href, wall, ph, pu, pv, qh, qu, qv, v0, v1, v2);
        if (cv[i]) overlap_force2(a, z.h, z.u, z.v, tv[i], cv[i], v0, v1, v2);
        st3(Lp, o, 1, v0, v1, v2);
        if (!obs_here) {
          publish2(g, Lp, false, rr, k, v0, v1, v2);
          push2(g, hxS, hxN, rr, k, v0, v1, v2);
        }
      }
    }
    if (obs_here) {
      __syncthreads();
      scatter2(a, g, Lp, l);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kMaxP; ++i) {
        const int idx = threadIdx.x + i * blockDim.x;
        if (idx < g.Rn * g.nx) {
          const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
          float v0, v1, v2;
          ld3(Lp, p2(g, rr, k), 1, v0, v1, v2);
          publish2(g, Lp, false, rr, k, v0, v1, v2);
          push2(g, hxS, hxN, rr, k, v0, v1, v2);
        }
      }
    }
    cluster_arrive_release();   // lambda(n) edge rows are in the neighbours' exchange buffers
  }
  cluster_wait_acquire();
  // lambda(a) -> packed control layout (FP64)
  double* out = a.lam_a + g.d.ctrl_off;
  for (int idx = threadIdx.x; idx < 3 * g.Rn * g.nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // v * Rn + rr
    const int v = q / g.Rn;
    const int rr = q - v * g.Rn, k = idx - q * g.nx;
    out[((size_t)v * g.ny + g.R0 + rr) * g.nx + k] = (double)Lp[p2(g, rr, k) + v];
  }
}

// The dynamic shared-memory attribute is a cap: it is set once per kernel and
// device to the device's opt-in maximum, together with permission for
// non-portable (16-CTA) clusters, so that no attribute call is made again
// (none lands inside a stream capture).
template <typename K>
cudaError_t raise_attributes(K kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, bool> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  bool& ok = done[{reinterpret_cast<const void*>(kernel), dev}];
  if (ok) return cudaSuccess;
  int cap = 0;
  e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  ok = true;
  return cudaSuccess;
}

template <typename T, typename K>
cudaError_t launch_cluster(K kernel, const SweepArgs<T>& a, int cl, int nthreads, size_t smem,
                           cudaStream_t st) {
  cudaError_t e = raise_attributes(kernel);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_sub * cl), 1, 1);
  cfg.blockDim = dim3((unsigned)nthreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

}  // namespace

template <typename T> size_t smem_forward(int R, int W) { return smem_bytes<T>(3, R, W, true); }
template <typename T> size_t smem_forward2(int R, int W) { return smem_bytes<T>(2, R, W, true); }
template <typename T> size_t smem_adjoint(int R, int W) { return smem_bytes<T>(5, R, W, true); }
template <typename T> size_t smem_adjoint_rl(int R, int W) { return smem_bytes<T>(4, R, W, true); }
template <typename T> size_t smem_tlm(int R, int W) { return smem_bytes<T>(6, R, W, false); }

// Clusters of the stripe adjoint (five buffers where they fit, else four)
// that can be resident at once with cl CTAs per subdomain and nthreads
// threads per CTA: a cluster must sit inside one GPC, so the count depends on
// how the GPCs' SMs divide by cl, not only on the CTAs per SM (0 when the
// shape cannot run).
template <typename T>
int active_clusters_adjoint(int R, int W, int cl, int nthreads) {
  const bool five = smem_adjoint<T>(R, W) <= kSmemOptinMax;
  const size_t smem = five ? smem_adjoint<T>(R, W) : smem_adjoint_rl<T>(R, W);
  if (smem > kSmemOptinMax || nthreads > kStripeAdjThreads) return 0;
  cudaError_t e = five ? raise_attributes(adj_kernel<T, false>) : raise_attributes(adj_kernel<T, true>);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cl, 1, 1);
  cfg.blockDim = dim3((unsigned)nthreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = five ? cudaOccupancyMaxActiveClusters(&n, adj_kernel<T, false>, &cfg)
           : cudaOccupancyMaxActiveClusters(&n, adj_kernel<T, true>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Whether the deep-halo FP32 sweep with nbuf state buffers can run a launch:
// every stripe has at least kH rows, a thread holds at most kMaxP own points,
// the threads fit its register budget and its shared memory fits.
template <typename T>
bool deep_fits(const SweepArgs<T>& a, int cl, int nthreads, int nbuf) {
  if (sizeof(T) != 4 || a.variant != 0 || cl < 1 || a.stg1) return false;
  if (a.min_ny < kH * cl || nthreads > kDeepThreads || nthreads < 64 || nthreads % 32) return false;
  if ((long long)a.R * (a.W - 2) > (long long)kMaxP * nthreads) return false;
  return smem_deep(nbuf, a.R, a.W) <= kSmemOptinMax;
}

// Forward variant 2 selects the two-buffer stripe forward (kind 4), which
// needs every trajectory level stored (ckpt 0); otherwise it acts as
// variant 1.
template <typename T>
int forward_kind(const SweepArgs<T>& a, int cl, int nthreads) {
  if (a.variant == 2 && a.ckpt == 0 && nthreads <= max_threads_forward<T>() &&
      smem_forward2<T>(a.R, a.W) <= kSmemOptinMax)
    return 4;
  if (deep_fits(a, cl, nthreads, 3)) return 2;
  if (nthreads > max_threads_forward<T>() || smem_forward<T>(a.R, a.W) > kSmemOptinMax) return 0;
  return 1;
}
// The deep-halo adjoint covers evaluations with stored stage states (no
// checkpoints, no external or Gauss-Newton forcing).  Variant 2 selects the
// stripe adjoint with four state buffers (x(n) reloaded; kind 3); the other
// variants fall back to it where five buffers do not fit.
template <typename T>
int adjoint_kind(const SweepArgs<T>& a, int cl, int nthreads) {
  const bool rl_fits = nthreads <= kStripeAdjThreads && smem_adjoint_rl<T>(a.R, a.W) <= kSmemOptinMax;
  if (a.variant == 2) return rl_fits ? 3 : 0;
  if (a.stg && a.ckpt == 0 && !a.yforce && !a.gn_dx && deep_fits(a, cl, nthreads, 5)) return 2;
  if (nthreads <= kStripeAdjThreads && smem_adjoint<T>(a.R, a.W) <= kSmemOptinMax) return 1;
  return rl_fits ? 3 : 0;
}

template <typename T>
cudaError_t launch_forward(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (forward_kind(a, cl, nthreads) == 2)
      return launch_cluster(fwd_deep_kernel, a, cl, nthreads, smem_deep(3, a.R, a.W), st);
  }
  SweepArgs<T> b = a;
  if (forward_kind(a, cl, nthreads) == 4) {
    b.tgb_on = use_target_buffer<T>(2, a.R, a.W, true) ? 1 : 0;
    return launch_cluster(fwd_kernel<T, true>, b, cl, nthreads, smem_forward2<T>(a.R, a.W), st);
  }
  b.tgb_on = use_target_buffer<T>(3, a.R, a.W, true) ? 1 : 0;
  return launch_cluster(fwd_kernel<T, false>, b, cl, nthreads, smem_forward<T>(a.R, a.W), st);
}
template <typename T>
cudaError_t launch_adjoint(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st) {
  const int kind = adjoint_kind(a, cl, nthreads);
  if constexpr (sizeof(T) == 4) {
    if (kind == 2) return launch_cluster(adj_deep_kernel, a, cl, nthreads, smem_deep(5, a.R, a.W), st);
  }
  SweepArgs<T> b = a;
  if (kind == 3) {
    b.tgb_on = use_target_buffer<T>(4, a.R, a.W, true) ? 1 : 0;
    return launch_cluster(adj_kernel<T, true>, b, cl, nthreads, smem_adjoint_rl<T>(a.R, a.W), st);
  }
  b.tgb_on = use_target_buffer<T>(5, a.R, a.W, true) ? 1 : 0;
  return launch_cluster(adj_kernel<T, false>, b, cl, nthreads, smem_adjoint<T>(a.R, a.W), st);
}
// The tangent-linear kernel is compiled for at most 512 threads (its loops
// are strided, so any CTA size gives the same result).
template <typename T>
cudaError_t launch_tlm(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st) {
  return launch_cluster(tlm_kernel<T>, a, cl, std::min(nthreads, 512), smem_tlm<T>(a.R, a.W), st);
}

#define DD4DV_INST(T)                                                                        \
  template int forward_kind<T>(const SweepArgs<T>&, int, int);                               \
  template int adjoint_kind<T>(const SweepArgs<T>&, int, int);                               \
  template size_t smem_forward<T>(int, int);                                                 \
  template size_t smem_adjoint<T>(int, int);                                                 \
  template size_t smem_adjoint_rl<T>(int, int);                                              \
  template size_t smem_tlm<T>(int, int);                                                     \
  template int active_clusters_adjoint<T>(int, int, int, int);                               \
  template cudaError_t launch_forward<T>(const SweepArgs<T>&, int, int, cudaStream_t);       \
  template cudaError_t launch_adjoint<T>(const SweepArgs<T>&, int, int, cudaStream_t);       \
  template cudaError_t launch_tlm<T>(const SweepArgs<T>&, int, int, cudaStream_t);
DD4DV_INST(double)
DD4DV_INST(float)
#undef DD4DV_INST

}  // namespace dd4dv
