// Forward, adjoint and tangent-linear sweeps of the local shallow-water model
// over every subdomain's time window, batched in one launch each.
//
// Design (GB300, sm_103a): one thread-block cluster per subdomain.  The
// cluster's CTAs split the subdomain's box into horizontal stripes of rows;
// each CTA keeps its stripe of the state (plus one halo row on each side and
// a ghost column on each side) resident in shared memory for the whole time
// window.  After every RK3 stage the CTAs barrier on the cluster and read
// their neighbours' edge rows through distributed shared memory
// (ld.shared::cluster via cooperative_groups::cluster_group::map_shared_rank),
// so the only HBM traffic of a step is the trajectory store (forward), the
// trajectory load (adjoint), ghost values of the frozen boundary trajectory
// and the sparse observation / overlap data.  Clusters are ordered longest
// subdomain first (uneven sizes in one launch).
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

template <typename T>
struct Geo {
  int s, rank, CL, R0, Rn, nx, ny, L, a, R2, W, P, flags;
  int Rprev, Rnext;   // own-row counts of the south / north neighbour CTA
  SubDesc d;
  T* gh;              // ghost cache: 3 slots of [6 R columns | 6 W rows] values
  int* gh_tag;        // level held by each slot (-1: none)
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

__device__ __forceinline__ void split_rows(int ny, int CL, int rank, int& R0, int& Rn) {
  const int base = ny / CL, rem = ny % CL;
  R0 = rank * base + min(rank, rem);
  Rn = base + (rank < rem ? 1 : 0);
}

template <typename T>
__device__ __forceinline__ int off(const Geo<T>& g, int v, int rr, int k) {
  return (v * g.R2 + rr + 1) * g.W + k + 1;
}

// Per-row constants staged in shared memory for rows rr = -1 .. Rn (index
// i = rr + 1), as two 8-value records per row so that a point reads its row's
// constants with two (FP32) or four (FP64) 16-byte loads:
//   fw[8 i ..]: A, f, tau, B/c, g A, c of row i+1, c of row i-1, 0
//               (tendencies and tangent-linear tendencies)
//   bw[8 i ..]: A, f, tau, g A, B c, 1/c of row i+1, 1/c of row i-1, 0
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
    b[7] = (T)0;
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
  return wA * xa + wB * xb;
}

// ---- ghost cache --------------------------------------------------------
// The ghost values a CTA needs at one level -- the west/east columns of its
// own rows when the box has frozen lateral edges, the south/north rows when
// its stripe touches a frozen box edge -- are copied into a slot of a 3-level
// shared-memory ring with cp.async one step before they are used, so that the
// completion after each stage reads shared memory instead of waiting on HBM.
// Slot of level n: n mod 3; a lookup whose level is not in its slot falls back
// to HBM (results never depend on the cache).
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
  cp_async_commit();
  if (threadIdx.x == 0) g.gh_tag[slot] = n;
}

// Ghost column of own row rr (side 0 = west, 1 = east) and ghost row value at
// column k (side 0 = south, 1 = north), blended between levels nA and nB.
template <typename T>
__device__ __forceinline__ T gh_col(const SweepArgs<T>& a, const Geo<T>& g, int nA, int nB, T wA, T wB,
                                    int side, int v, int rr) {
  if constexpr (sizeof(T) == 8) {
    const int i = side == 0 ? (g.d.i0 - 1 + a.nlon) % a.nlon : (g.d.i0 + g.nx) % a.nlon;
    return bnd_val(a, nA, nB, wA, wB, v, g.d.j0 + g.R0 + rr, i);
  }
  const int R = g.R2 - 2;
  const int sA = nA % 3, sB = nB % 3;
  if (g.gh_tag[sA] == nA && (wB == (T)0 || g.gh_tag[sB] == nB)) {
    const int o = (side * 3 + v) * R + rr;
    const T xa = g.gh[(size_t)sA * g.gh_len + o];
    if (wB == (T)0) return xa;
    return wA * xa + wB * g.gh[(size_t)sB * g.gh_len + o];
  }
  const int i = side == 0 ? (g.d.i0 - 1 + a.nlon) % a.nlon : (g.d.i0 + g.nx) % a.nlon;
  return bnd_val(a, nA, nB, wA, wB, v, g.d.j0 + g.R0 + rr, i);
}

template <typename T>
__device__ __forceinline__ T gh_row(const SweepArgs<T>& a, const Geo<T>& g, int nA, int nB, T wA, T wB,
                                    int side, int v, int k) {
  if constexpr (sizeof(T) == 8)
    return bnd_val(a, nA, nB, wA, wB, v, side ? g.d.j0 + g.ny : g.d.j0 - 1, (g.d.i0 + k) % a.nlon);
  const int R = g.R2 - 2;
  const int sA = nA % 3, sB = nB % 3;
  if (g.gh_tag[sA] == nA && (wB == (T)0 || g.gh_tag[sB] == nB)) {
    const int o = 6 * R + (side * 3 + v) * g.W + k;
    const T xa = g.gh[(size_t)sA * g.gh_len + o];
    if (wB == (T)0) return xa;
    return wA * xa + wB * g.gh[(size_t)sB * g.gh_len + o];
  }
  return bnd_val(a, nA, nB, wA, wB, v, side ? g.d.j0 + g.ny : g.d.j0 - 1, (g.d.i0 + k) % a.nlon);
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
  const bool periodic = g.flags & F_PERIODIC;
  // halo rows
  const T* south_nb = (g.rank > 0) ? cl.map_shared_rank(X, g.rank - 1) : nullptr;
  const T* north_nb = (g.rank < g.CL - 1) ? cl.map_shared_rank(X, g.rank + 1) : nullptr;
  for (int idx = threadIdx.x; idx < 2 * 3 * nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // side * 3 + v
    const int side = q / 3;
    const int v = q - 3 * side;
    const int k = idx - q * nx;
    T val;
    if (side == 0) {   // south halo rr = -1
      if (south_nb) {
        val = south_nb[off(g, v, g.Rprev - 1, k)];
      } else if (g.flags & F_SWALL) {
        val = (kind == K_ADJ) ? (T)0 : ((v == 2) ? -X[off(g, v, 0, k)] : X[off(g, v, 0, k)]);
      } else {
        val = (kind == K_STATE)
                  ? gh_row(a, g, nA, nB, wA, wB, 0, v, k)
                  : (T)0;
      }
      X[off(g, v, -1, k)] = val;
    } else {           // north halo rr = Rn
      if (north_nb) {
        val = north_nb[off(g, v, 0, k)];
      } else if (g.flags & F_NWALL) {
        val = (kind == K_ADJ) ? (T)0
                              : ((v == 2) ? -X[off(g, v, g.Rn - 1, k)] : X[off(g, v, g.Rn - 1, k)]);
      } else {
        val = (kind == K_STATE)
                  ? gh_row(a, g, nA, nB, wA, wB, 1, v, k)
                  : (T)0;
      }
      X[off(g, v, g.Rn, k)] = val;
    }
  }
  // ghost columns of own rows
  for (int idx = threadIdx.x; idx < 2 * 3 * g.Rn; idx += blockDim.x) {
    const int q = mdiv(idx, g.mRn);   // side * 3 + v
    const int side = q / 3;
    const int v = q - 3 * side;
    const int rr = idx - q * g.Rn;
    T val;
    if (periodic) {
      val = side == 0 ? X[off(g, v, rr, nx - 1)] : X[off(g, v, rr, 0)];
    } else if (kind == K_STATE) {
      val = gh_col(a, g, nA, nB, wA, wB, side, v, rr);
    } else {
      val = (T)0;
    }
    X[off(g, v, rr, side == 0 ? -1 : nx)] = val;
  }
  __syncthreads();
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
  for (int idx = threadIdx.x; idx < 3 * nr * nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // v * nr + (rr - r_lo)
    const int v = mdiv(q, g.mnr);
    const int rr = q - v * nr + r_lo;
    const int k = idx - q * nx;
    X[off(g, v, rr, k)] = src[((size_t)v * g.ny + g.R0 + rr) * g.d.nxp + k];
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();
  __syncthreads();
  const bool periodic = g.flags & F_PERIODIC;
  if (g.rank == 0) {
    for (int idx = threadIdx.x; idx < 3 * nx; idx += blockDim.x) {
      const int v = mdiv(idx, g.mnx), k = idx - v * nx;
      X[off(g, v, -1, k)] = (g.flags & F_SWALL)
                                ? ((v == 2) ? -X[off(g, v, 0, k)] : X[off(g, v, 0, k)])
                                : gh_row(a, g, nA, nB, wA, wB, 0, v, k);
    }
  }
  if (g.rank == g.CL - 1) {
    for (int idx = threadIdx.x; idx < 3 * nx; idx += blockDim.x) {
      const int v = mdiv(idx, g.mnx), k = idx - v * nx;
      X[off(g, v, g.Rn, k)] =
          (g.flags & F_NWALL)
              ? ((v == 2) ? -X[off(g, v, g.Rn - 1, k)] : X[off(g, v, g.Rn - 1, k)])
              : gh_row(a, g, nA, nB, wA, wB, 1, v, k);
    }
  }
  for (int idx = threadIdx.x; idx < 2 * 3 * g.Rn; idx += blockDim.x) {
    const int q = mdiv(idx, g.mRn);   // side * 3 + v
    const int side = q / 3;
    const int v = q - 3 * side;
    const int rr = idx - q * g.Rn;
    T val;
    if (periodic) {
      val = side == 0 ? X[off(g, v, rr, nx - 1)] : X[off(g, v, rr, 0)];
    } else {
      val = gh_col(a, g, nA, nB, wA, wB, side, v, rr);
    }
    X[off(g, v, rr, side == 0 ? -1 : nx)] = val;
  }
  __syncthreads();
}

// Load up to three stored states at once (one pass, one barrier pair) so that
// their global-load latencies overlap.  Same rules as load_state.
template <typename T>
__device__ void load_states3(const SweepArgs<T>& a, const Geo<T>& g, T* const* X, const T* const* src,
                             const int* nA, const int* nB, const T* wA, const T* wB) {
  const int nx = g.nx;
  const int r_lo = (g.rank > 0) ? -1 : 0;
  const int r_hi = (g.rank < g.CL - 1) ? g.Rn + 1 : g.Rn;
  const int nr = r_hi - r_lo;
  const int per = 3 * nr * nx;
  for (int idx = threadIdx.x; idx < 3 * per; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // (b * 3 + v) * nr + (rr - r_lo)
    const int bv = mdiv(q, g.mnr);
    const int b = bv / 3, v = bv - 3 * b;
    const int rr = q - bv * nr + r_lo;
    const int k = idx - q * nx;
    X[b][off(g, v, rr, k)] = src[b][((size_t)v * g.ny + g.R0 + rr) * g.d.nxp + k];
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();
  __syncthreads();
  const bool periodic = g.flags & F_PERIODIC;
  const int ne = 2 * 3 * nx;      // box-edge halo rows (both sides, all vars)
  const int nc = 2 * 3 * g.Rn;    // ghost columns of own rows
  const unsigned mb = magic_of(ne + nc);
  for (int idx = threadIdx.x; idx < 3 * (ne + nc); idx += blockDim.x) {
    const int b = mdiv(idx, mb);
    int j = idx - b * (ne + nc);
    T* Y = X[b];
    if (j < ne) {
      const int q = mdiv(j, g.mnx);   // side * 3 + v
      const int side = q / 3;
      const int v = q - 3 * side, k = j - q * nx;
      if (side == 0 && g.rank == 0) {
        Y[off(g, v, -1, k)] = (g.flags & F_SWALL)
                                  ? ((v == 2) ? -Y[off(g, v, 0, k)] : Y[off(g, v, 0, k)])
                                  : gh_row(a, g, nA[b], nB[b], wA[b], wB[b], 0, v, k);
      } else if (side == 1 && g.rank == g.CL - 1) {
        Y[off(g, v, g.Rn, k)] =
            (g.flags & F_NWALL)
                ? ((v == 2) ? -Y[off(g, v, g.Rn - 1, k)] : Y[off(g, v, g.Rn - 1, k)])
                : gh_row(a, g, nA[b], nB[b], wA[b], wB[b], 1, v, k);
      }
    } else {
      j -= ne;
      const int q = mdiv(j, g.mRn);   // side * 3 + v
      const int side = q / 3;
      const int v = q - 3 * side;
      const int rr = j - q * g.Rn;
      T val;
      if (periodic) {
        val = side == 0 ? Y[off(g, v, rr, nx - 1)] : Y[off(g, v, rr, 0)];
      } else {
        val = gh_col(a, g, nA[b], nB[b], wA[b], wB[b], side, v, rr);
      }
      Y[off(g, v, rr, side == 0 ? -1 : nx)] = val;
    }
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

// Tendencies F(Z) at one point (Sec. 7, centred differences):
//   F_u = -A u (uE-uW) - Bth v (uN-uS) + (f + tau u) v - gA (hE-hW)
//   F_v = -A u (vE-vW) - Bth v (vN-vS) - (f + tau u) u - gBth (hN-hS)
//   F_h = -A ((hu)_E - (hu)_W) - (Bth/c) ((h v c)_N - (h v c)_S)
// On the FP32 path h = h_ref + h' and the h_ref parts of the fluxes are
// formed from velocity differences.
template <typename T, bool DEV>
__device__ __forceinline__ void rhs_pt(const T* Z, int o, int P, int W, T A, T f, T tau, T BinvC,
                                       T gA, T cN, T cS, T Bth, T gBth, T href, T& Fh, T& Fu,
                                       T& Fv) {
  const T* H = Z;
  const T* U = Z + P;
  const T* V = Z + 2 * P;
  const T u = U[o], v = V[o];
  const T uE = U[o + 1], uW = U[o - 1], uN = U[o + W], uS = U[o - W];
  const T vE = V[o + 1], vW = V[o - 1], vN = V[o + W], vS = V[o - W];
  const T hE = H[o + 1], hW = H[o - 1], hN = H[o + W], hS = H[o - W];
  const T fu = f + tau * u;
  Fu = -A * u * (uE - uW) - Bth * v * (uN - uS) + fu * v - gA * (hE - hW);
  Fv = -A * u * (vE - vW) - Bth * v * (vN - vS) - fu * u - gBth * (hN - hS);
  T flx = hE * uE - hW * uW;
  T fly = hN * vN * cN - hS * vS * cS;
  if (DEV) {
    flx += href * (uE - uW);
    fly += href * (vN * cN - vS * cS);
  }
  Fh = -A * flx - BinvC * fly;
}

// Adjoint of the tendencies: G = F'(Z)^T M at one point (derived by hand from
// rhs_pt; M holds zero at ghost points that carry no tendency).  Wall rows add
// the transposed ghost mirror (h, u, -v) of the edge row.
template <typename T, bool DEV>
__device__ __forceinline__ void rhs_adj_pt(const T* Z, const T* M, int o, int P, int W, T A, T f,
                                           T tau, T gA, T BcC, T icN, T icS, T Bth, T gBth, T href,
                                           int wall, T& Gh, T& Gu, T& Gv) {
  const T* H = Z;
  const T* U = Z + P;
  const T* V = Z + 2 * P;
  const T* mH = M;
  const T* mU = M + P;
  const T* mV = M + 2 * P;
  T h = H[o];
  if (DEV) h += href;
  const T u = U[o], v = V[o];
  const T uE = U[o + 1], uW = U[o - 1], uN = U[o + W], uS = U[o - W];
  const T vE = V[o + 1], vW = V[o - 1], vN = V[o + W], vS = V[o - W];
  const T mu = mU[o], mv = mV[o], mh = mH[o];
  const T muE = mU[o + 1], muW = mU[o - 1], muN = mU[o + W], muS = mU[o - W];
  const T mvE = mV[o + 1], mvW = mV[o - 1], mvN = mV[o + W], mvS = mV[o - W];
  const T mhE = mH[o + 1], mhW = mH[o - 1], mhN = mH[o + W], mhS = mH[o - W];
  const T dmhEW = mhE - mhW;
  const T dmhNS = mhN * icN - mhS * icS;
  Gu = mu * (tau * v - A * (uE - uW)) - mv * (A * (vE - vW) + f + (T)2 * tau * u) +
       A * (muE * uE - muW * uW) + A * h * dmhEW + Bth * (muN * vN - muS * vS);
  Gv = mu * (f + tau * u - Bth * (uN - uS)) - mv * (Bth * (vN - vS)) + A * (mvE * uE - mvW * uW) +
       Bth * (mvN * vN - mvS * vS) + BcC * h * dmhNS;
  Gh = gA * (muE - muW) + gBth * (mvN - mvS) + A * u * dmhEW + BcC * v * dmhNS;
  if (wall == 1) {         // south wall: ghost row = (h, u, -v) of this row
    Gu += Bth * mu * v;
    Gv -= Bth * (mv * v + h * mh);
    Gh += gBth * mv - Bth * v * mh;
  } else if (wall == 2) {  // north wall
    Gu -= Bth * mu * v;
    Gv += Bth * (mv * v + h * mh);
    Gh += Bth * v * mh - gBth * mv;
  }
}

// Tangent-linear tendencies dF = F'(Z) dZ at one point.
template <typename T, bool DEV>
__device__ __forceinline__ void rhs_tl_pt(const T* Z, const T* D, int o, int P, int W, T A, T f,
                                          T tau, T BinvC, T gA, T cN, T cS, T Bth, T gBth, T href,
                                          T& dFh, T& dFu, T& dFv) {
  const T* H = Z;
  const T* U = Z + P;
  const T* V = Z + 2 * P;
  const T* dH = D;
  const T* dU = D + P;
  const T* dV = D + 2 * P;
  const T u = U[o], v = V[o];
  const T du = dU[o], dv = dV[o];
  const T uE = U[o + 1], uW = U[o - 1], uN = U[o + W], uS = U[o - W];
  const T vE = V[o + 1], vW = V[o - 1], vN = V[o + W], vS = V[o - W];
  T hE = H[o + 1], hW = H[o - 1], hN = H[o + W], hS = H[o - W];
  if (DEV) {
    hE += href; hW += href; hN += href; hS += href;
  }
  const T duE = dU[o + 1], duW = dU[o - 1], duN = dU[o + W], duS = dU[o - W];
  const T dvE = dV[o + 1], dvW = dV[o - 1], dvN = dV[o + W], dvS = dV[o - W];
  const T dhE = dH[o + 1], dhW = dH[o - 1], dhN = dH[o + W], dhS = dH[o - W];
  dFu = -A * (du * (uE - uW) + u * (duE - duW)) - Bth * (dv * (uN - uS) + v * (duN - duS)) +
        (f + tau * u) * dv + tau * du * v - gA * (dhE - dhW);
  dFv = -A * (du * (vE - vW) + u * (dvE - dvW)) - Bth * (dv * (vN - vS) + v * (dvN - dvS)) -
        (f + tau * u) * du - tau * du * u - gBth * (dhN - dhS);
  dFh = -A * ((dhE * uE + hE * duE) - (dhW * uW + hW * duW)) -
        BinvC * ((dhN * vN + hN * dvN) * cN - (dhS * vS + hS * dvS) * cS);
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
template <typename T>
__device__ void obs_level(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int l, double& Jo) {
  const int o0 = a.lvl_obs[g.d.obs_lvl + l], o1 = a.lvl_obs[g.d.obs_lvl + l + 1];
  for (int o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    const ObsRec ob = a.obs[o];
    const int rr = ob.r0 - g.R0;
    if (rr < 0 || rr >= g.Rn) continue;
    const T* P = X + ob.var * g.P;
    double acc = 0.0;
    const double wj0 = 1.0 - ob.dj, wi0 = 1.0 - ob.di;
    acc += (wj0 * wi0) * (double)P[(rr + 1) * g.W + ob.k0 + 1];
    if (ob.di != 0.0) acc += (wj0 * ob.di) * (double)P[(rr + 1) * g.W + ob.k1 + 1];
    if (ob.dj != 0.0) {
      acc += (ob.dj * wi0) * (double)P[(rr + 2) * g.W + ob.k0 + 1];
      if (ob.di != 0.0) acc += (ob.dj * ob.di) * (double)P[(rr + 2) * g.W + ob.k1 + 1];
    }
    const double d = acc - ob.y;
    Jo += 0.5 * ob.w * d * d;
    a.obs_force[o] = a.lam * ob.w * d;
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
    const T* P = D + ob.var * g.P;
    double acc = 0.0;
    const double wj0 = 1.0 - ob.dj, wi0 = 1.0 - ob.di;
    acc += (wj0 * wi0) * (double)P[(rr + 1) * g.W + ob.k0 + 1];
    if (ob.di != 0.0) acc += (wj0 * ob.di) * (double)P[(rr + 1) * g.W + ob.k1 + 1];
    if (ob.dj != 0.0) {
      acc += (ob.dj * wi0) * (double)P[(rr + 2) * g.W + ob.k0 + 1];
      if (ob.di != 0.0) acc += (ob.dj * ob.di) * (double)P[(rr + 2) * g.W + ob.k1 + 1];
    }
    a.obs_force[o] = a.lam * ob.w * acc;
  }
}

// Calls f(rr, k, c) for every own point (rr, k) of level l with overlap count
// c > 0, spread over the CTA's threads.  At a level outside the time overlaps
// only the spatial bands have c > 0: rows r < wS and r >= ny - wN in full,
// and the columns k < wL and k >= nx - wR of the rows between; those points
// alone are visited.
template <typename T, typename F>
__device__ __forceinline__ void for_overlap_points(const Geo<T>& g, int l, F&& f) {
  const SubDesc& d = g.d;
  const int nx = g.nx;
  const bool any_t = (l < d.tA) || (l > g.L - d.tB);
  if (any_t || d.wL + d.wR >= nx) {
    for (int idx = threadIdx.x; idx < g.Rn * nx; idx += blockDim.x) {
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
  for (int idx = threadIdx.x; idx < nA + nC + nB; idx += blockDim.x) {
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
  T part = (T)0;
  for_overlap_points(g, l, [&](int rr, int k, int c) {
    const size_t go = (size_t)(g.R0 + rr) * d.nxp + k;
    const T e0 = X[off(g, 0, rr, k)] - tg[go];
    const T e1 = X[off(g, 1, rr, k)] - tg[go + pl];
    const T e2 = X[off(g, 2, rr, k)] - tg[go + 2 * pl];
    part += (T)c * (e0 * e0 * i0 + e1 * e1 * i1 + e2 * e2 * i2);
  });
  Jm += (double)part;
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
  g.P = g.R2 * g.W;
  if (g.rank != 0) g.flags &= ~F_SWALL;           // only the edge CTAs see the walls
  if (g.rank != g.CL - 1) g.flags &= ~F_NWALL;
  g.mnx = magic_of(g.nx);
  g.mRn = magic_of(g.Rn);
  g.mny = magic_of(g.ny);
  g.mnr = magic_of(g.Rn + (g.rank > 0) + (g.rank < g.CL - 1));
  return true;
}

// One RK3 stage at own point (rr, k): out = cx X + cy (Y + dt F(Y)); the
// three new values are also returned.
template <typename T, bool DEV>
__device__ __forceinline__ void stage_point(const SweepArgs<T>& a, const Geo<T>& g, const RowSmem<T>& rs,
                                            T* out, const T* X, const T* Y, T cx, T cy, int rr, int k,
                                            T& o0, T& o1, T& o2) {
  const T dt = a.dt_s, Bth = a.Bth_s, gBth = a.gBth_s, href = a.href_s;
  const int P = g.P;
  const int o = (rr + 1) * g.W + k + 1;
  const int ri = rr + 1;
  T Fh, Fu, Fv;
  T rc[8];
  load_rec8(rs.fw + 8 * ri, rc);
  rhs_pt<T, DEV>(Y, o, P, g.W, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth, href, Fh, Fu, Fv);
  if (cx == (T)0) {
    o0 = cy * (Y[o] + dt * Fh);
    o1 = cy * (Y[o + P] + dt * Fu);
    o2 = cy * (Y[o + 2 * P] + dt * Fv);
  } else {
    o0 = cx * X[o] + cy * (Y[o] + dt * Fh);
    o1 = cx * X[o + P] + cy * (Y[o + P] + dt * Fu);
    o2 = cx * X[o + 2 * P] + cy * (Y[o + 2 * P] + dt * Fv);
  }
  out[o] = o0;
  out[o + P] = o1;
  out[o + 2 * P] = o2;
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
  if (s_fixed || n_fixed) {
    for (int idx = threadIdx.x; idx < 2 * 3 * nx; idx += blockDim.x) {
      const int q = mdiv(idx, g.mnx);   // side * 3 + v
      const int side = q / 3;
      if (side == 0 ? !s_fixed : !n_fixed) continue;
      const int v = q - 3 * side, k = idx - q * nx;
      const bool wall = (side == 0) ? (g.flags & F_SWALL) : (g.flags & F_NWALL);
      X[off(g, v, side == 0 ? -1 : g.Rn, k)] =
          (kind == K_STATE && !wall) ? gh_row(a, g, nA, nB, wA, wB, side, v, k) : (T)0;
    }
  }
  if (!(g.flags & F_PERIODIC)) {
    for (int idx = threadIdx.x; idx < 2 * 3 * g.Rn; idx += blockDim.x) {
      const int q = mdiv(idx, g.mRn);   // side * 3 + v
      const int side = q / 3;
      const int v = q - 3 * side, rr = idx - q * g.Rn;
      X[off(g, v, rr, side == 0 ? -1 : nx)] = (kind == K_STATE) ? gh_col(a, g, nA, nB, wA, wB, side, v, rr) : (T)0;
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
      snb[off(g, 0, g.Rprev, k)] = v0;
      snb[off(g, 1, g.Rprev, k)] = v1;
      snb[off(g, 2, g.Rprev, k)] = v2;
    } else if ((g.flags & F_SWALL) && kind != K_ADJ) {
      X[off(g, 0, -1, k)] = v0;
      X[off(g, 1, -1, k)] = v1;
      X[off(g, 2, -1, k)] = -v2;
    }
  }
  if (rr == g.Rn - 1) {
    if (nnb) {
      nnb[off(g, 0, -1, k)] = v0;
      nnb[off(g, 1, -1, k)] = v1;
      nnb[off(g, 2, -1, k)] = v2;
    } else if ((g.flags & F_NWALL) && kind != K_ADJ) {
      X[off(g, 0, g.Rn, k)] = v0;
      X[off(g, 1, g.Rn, k)] = v1;
      X[off(g, 2, g.Rn, k)] = -v2;
    }
  }
  if (g.flags & F_PERIODIC) {
    if (k == 0) {
      X[off(g, 0, rr, g.nx)] = v0;
      X[off(g, 1, rr, g.nx)] = v1;
      X[off(g, 2, rr, g.nx)] = v2;
    }
    if (k == g.nx - 1) {
      X[off(g, 0, rr, -1)] = v0;
      X[off(g, 1, rr, -1)] = v1;
      X[off(g, 2, rr, -1)] = v2;
    }
  }
}

// Steps 1-5 with fn(rr, k, v0, v1, v2) computing and storing point (rr, k)
// of X and returning its values.
template <typename T, typename Fn>
__device__ void phase_push(cg::cluster_group& cl, const SweepArgs<T>& a, const Geo<T>& g, T* X, int kind,
                           int nA, int nB, T wA, T wB, Fn&& fn) {
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
  if constexpr (sizeof(T) == 4) cp_async_wait_all();   // this thread's ghost copies land first
  __syncthreads();
  cluster_wait_acquire();
}

// RK3 stage with pushed halo exchange (replaces stage + complete_buf).
template <typename T, bool DEV>
__device__ __forceinline__ void stage_push(cg::cluster_group& cl, const SweepArgs<T>& a, const Geo<T>& g,
                                           const RowSmem<T>& rs, T* out, const T* X, const T* Y, T cx, T cy,
                                           int nA, int nB, T wA, T wB) {
  phase_push(cl, a, g, out, K_STATE, nA, nB, wA, wB, [&](int rr, int k, T& v0, T& v1, T& v2) {
    stage_point<T, DEV>(a, g, rs, out, X, Y, cx, cy, rr, k, v0, v1, v2);
  });
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
    publish(g, X, snb, nnb, kind, rr, k, X[off(g, 0, rr, k)], X[off(g, 1, rr, k)], X[off(g, 2, rr, k)]);
  }
  if constexpr (sizeof(T) == 4) cp_async_wait_all();
  cl.sync();
}

template <typename T>
__device__ void store_block(const Geo<T>& g, const T* X, T* dst) {
  for (int idx = threadIdx.x; idx < 3 * g.Rn * g.nx; idx += blockDim.x) {
    const int q = mdiv(idx, g.mnx);   // v * Rn + rr
    const int v = mdiv(q, g.mRn);
    const int rr = q - v * g.Rn, k = idx - q * g.nx;
    dst[((size_t)v * g.ny + g.R0 + rr) * g.d.nxp + k] = X[off(g, v, rr, k)];
  }
}

template <typename T>
__device__ __forceinline__ void store_level(const SweepArgs<T>& a, const Geo<T>& g, const T* X, int l) {
  store_block(g, X, a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp);
}

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
    p += 3 * g.P;
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
size_t smem_bytes(int nbuf, int R, int W, bool cache) {
  return (size_t)nbuf * 3 * (R + 2) * W * sizeof(T) + 16 + 16 * (size_t)(R + 2) * sizeof(T) + 16 +
         64 * sizeof(double) + 3 * (size_t)ghost_len<T>(cache, R, W) * sizeof(T) + 3 * sizeof(int) + 16;
}

// ---------------------------------------------------------------------------
// Forward sweep: x(a) (stored at level 0 by the init kernel) -> x(a+1..b),
// trajectory stored at every level, J_o and J_mu partial sums per CTA.
template <typename T>
__global__ void __launch_bounds__(512, 2) fwd_kernel(SweepArgs<T> a) {
  constexpr bool DEV = sizeof(T) == 4;
  cg::cluster_group cl = cg::this_cluster();
  Geo<T> g;
  if (!setup_geo(a, cl, g)) return;
  T* buf[3];
  RowSmem<T> rs;
  double* scratch;
  carve(a, g, 3, buf, rs, &scratch, true);
  T* X = buf[0];
  T* S1 = buf[1];
  T* S2 = buf[2];
  load_rows(a, g, rs);
  ghost_prefetch(a, g, g.a);
  if (g.L > 0) ghost_prefetch(a, g, g.a + 1);
  load_level(a, g, X, 0, g.a);   // includes a CTA barrier
  double Jo = 0.0, Jm = 0.0;
  obs_level(a, g, X, 0, Jo);
  overlap_level(a, g, X, 0, Jm);
  for (int l = 0; l < g.L; ++l) {
    const int n = g.a + l;
    if (n + 2 <= g.d.b) ghost_prefetch(a, g, n + 2);   // used by the next step
    stage_push<T, DEV>(cl, a, g, rs, S1, X, X, (T)0, (T)1, n + 1, n + 1, (T)1, (T)0);
    // stores read the buffer with another thread mapping: after the barrier
    if (a.stg) store_block(g, S1, stage_ptr(a, g, l, 0));
    stage_push<T, DEV>(cl, a, g, rs, S2, X, S1, (T)0.75, (T)0.25, n, n + 1, (T)0.5, (T)0.5);
    if (a.stg) store_block(g, S2, stage_ptr(a, g, l, 1));
    stage_push<T, DEV>(cl, a, g, rs, X, X, S2, (T)(1.0 / 3.0), (T)(2.0 / 3.0), n + 1, n + 1, (T)1, (T)0);
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
      Lb[off(g, 0, rr, k)] += cc * m0 * dx[go];
      Lb[off(g, 1, rr, k)] += cc * m1 * dx[go + pl];
      Lb[off(g, 2, rr, k)] += cc * m2 * dx[go + 2 * pl];
    });
  } else if ((any_t || any_s) && a.mu != 0.0) {
    const T* tg = a.tgt + d.traj_off + (size_t)l * 3 * g.ny * d.nxp;
    const T m0 = a.musb2_s[0], m1 = a.musb2_s[1], m2 = a.musb2_s[2];
    const size_t pl = (size_t)g.ny * d.nxp;
    for_overlap_points(g, l, [&](int rr, int k, int c) {
      const size_t go = (size_t)(g.R0 + rr) * d.nxp + k;
      const T cc = (T)c;
      Lb[off(g, 0, rr, k)] += cc * m0 * (X[off(g, 0, rr, k)] - tg[go]);
      Lb[off(g, 1, rr, k)] += cc * m1 * (X[off(g, 1, rr, k)] - tg[go + pl]);
      Lb[off(g, 2, rr, k)] += cc * m2 * (X[off(g, 2, rr, k)] - tg[go + 2 * pl]);
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
template <typename T>
__global__ void __launch_bounds__(512, 2) adj_kernel(SweepArgs<T> a) {
  constexpr bool DEV = sizeof(T) == 4;
  cg::cluster_group cl = cg::this_cluster();
  Geo<T> g;
  if (!setup_geo(a, cl, g)) return;
  T* buf[5];
  RowSmem<T> rs;
  double* scratch;
  carve(a, g, 5, buf, rs, &scratch, true);
  T* X = buf[0];
  T* X1 = buf[1];
  T* X2 = buf[2];   // also lambda_x1
  T* Lp = buf[3];
  T* L2 = buf[4];
  load_rows(a, g, rs);
  ghost_prefetch(a, g, g.a + g.L);
  if (g.L > 0) ghost_prefetch(a, g, g.a + g.L - 1);
  for (int i = threadIdx.x; i < 3 * g.P; i += blockDim.x) Lp[i] = (T)0;
  const T dt = a.dt_s, Bth = a.Bth_s, gBth = a.gBth_s, href = a.href_s;
  const T c23 = (T)(2.0 / 3.0), c13 = (T)(1.0 / 3.0);
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
    add_forcing(a, g, Lp, X, g.L);
    complete_buf(cl, a, g, Lp, K_ADJ, 0, 0, (T)1, (T)0);
  }
  for (int l = l1 - 1; l >= l0; --l) {
    const int n = g.a + l;
    if (l > 0) ghost_prefetch(a, g, n - 1);   // used by the next (earlier) step
    if (a.stg && !K) {   // x(n) and the stage states stored by the forward sweep
      T* bufs[3] = {X, X1, X2};
      const T* srcs[3] = {a.traj + g.d.traj_off + (size_t)l * 3 * g.ny * g.d.nxp,
                          stage_ptr(a, g, l, 0), stage_ptr(a, g, l, 1)};
      const int nA[3] = {n, n + 1, n};
      const int nB[3] = {n, n + 1, n + 1};
      const T wA[3] = {(T)1, (T)1, (T)0.5};
      const T wB[3] = {(T)0, (T)0, (T)0.5};
      load_states3(a, g, bufs, srcs, nA, nB, wA, wB);
    } else {       // recompute the stage states from x(n)
      load_state(a, g, X, level_src(l), n, n, (T)1, (T)0);
      stage_push<T, DEV>(cl, a, g, rs, X1, X, X, (T)0, (T)1, n + 1, n + 1, (T)1, (T)0);
      stage_push<T, DEV>(cl, a, g, rs, X2, X, X1, (T)0.75, (T)0.25, n, n + 1, (T)0.5, (T)0.5);
    }
    const int P = g.P;
    // lambda_x2 = 2/3 lambda' + 2/3 dt F'(x2)^T lambda'
    phase_push(cl, a, g, L2, K_ADJ, 0, 0, (T)1, (T)0, [&](int rr, int k, T& v0, T& v1, T& v2) {
      const int o = (rr + 1) * g.W + k + 1, ri = rr + 1;
      const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
      T Gh, Gu, Gv;
      T rc[8];
      load_rec8(rs.bw + 8 * ri, rc);
      rhs_adj_pt<T, DEV>(X2, Lp, o, P, g.W, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth,
                         href, wall, Gh, Gu, Gv);
      v0 = c23 * (Lp[o] + dt * Gh);
      v1 = c23 * (Lp[o + P] + dt * Gu);
      v2 = c23 * (Lp[o + 2 * P] + dt * Gv);
      L2[o] = v0;
      L2[o + P] = v1;
      L2[o + 2 * P] = v2;
    });
    // lambda_x1 = 1/4 lambda_x2 + 1/4 dt F'(x1)^T lambda_x2   (into X2's buffer)
    T* L1 = X2;
    phase_push(cl, a, g, L1, K_ADJ, 0, 0, (T)1, (T)0, [&](int rr, int k, T& v0, T& v1, T& v2) {
      const int o = (rr + 1) * g.W + k + 1, ri = rr + 1;
      const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
      T Gh, Gu, Gv;
      T rc[8];
      load_rec8(rs.bw + 8 * ri, rc);
      rhs_adj_pt<T, DEV>(X1, L2, o, P, g.W, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth,
                         href, wall, Gh, Gu, Gv);
      v0 = (T)0.25 * (L2[o] + dt * Gh);
      v1 = (T)0.25 * (L2[o + P] + dt * Gu);
      v2 = (T)0.25 * (L2[o + 2 * P] + dt * Gv);
      L1[o] = v0;
      L1[o + P] = v1;
      L1[o + 2 * P] = v2;
    });
    // lambda(n) = 1/3 lambda' + 3/4 lambda_x2 + lambda_x1 + dt F'(x)^T lambda_x1
    for (int idx = threadIdx.x; idx < g.Rn * g.nx; idx += blockDim.x) {
      const int rr = mdiv(idx, g.mnx), k = idx - rr * g.nx;
      const int o = (rr + 1) * g.W + k + 1, ri = rr + 1;
      const int wall = (rr == 0 ? wall_s : 0) | (rr == g.Rn - 1 ? wall_n : 0);
      T Gh, Gu, Gv;
      T rc[8];
      load_rec8(rs.bw + 8 * ri, rc);
      rhs_adj_pt<T, DEV>(X, L1, o, P, g.W, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth,
                         href, wall, Gh, Gu, Gv);
      Lp[o] = c13 * Lp[o] + (T)0.75 * L2[o] + L1[o] + dt * Gh;
      Lp[o + P] = c13 * Lp[o + P] + (T)0.75 * L2[o + P] + L1[o + P] + dt * Gu;
      Lp[o + 2 * P] = c13 * Lp[o + 2 * P] + (T)0.75 * L2[o + 2 * P] + L1[o + 2 * P] + dt * Gv;
    }
    __syncthreads();
    add_forcing(a, g, Lp, X, l);
    push_halos(cl, a, g, Lp, K_ADJ);
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
  for (int i = threadIdx.x; i < 3 * g.P; i += blockDim.x) D[i] = (T)0;
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
    const int o = (rr + 1) * g.W + k + 1, ri = rr + 1;
    T Fh, Fu, Fv;
    T rc[8];
    load_rec8(rs.fw + 8 * ri, rc);
    rhs_tl_pt<T, DEV>(Y, DY, o, g.P, g.W, rc[0], rc[1], rc[2], rc[3], rc[4], rc[5], rc[6], Bth, gBth, href, Fh,
                      Fu, Fv);
    dout[o] = cx * DX[o] + cy * (DY[o] + dt * Fh);
    dout[o + g.P] = cx * DX[o + g.P] + cy * (DY[o + g.P] + dt * Fu);
    dout[o + 2 * g.P] = cx * DX[o + 2 * g.P] + cy * (DY[o + 2 * g.P] + dt * Fv);
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
      load_states3(a, g, bufs, srcs, nA, nB, wA, wB);
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
template <typename T> size_t smem_adjoint(int R, int W) { return smem_bytes<T>(5, R, W, true); }
template <typename T> size_t smem_tlm(int R, int W) { return smem_bytes<T>(6, R, W, false); }

template <typename T>
int occupancy_adjoint(int R, int W, int nthreads) {
  const size_t smem = smem_adjoint<T>(R, W);
  if (raise_attributes(adj_kernel<T>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adj_kernel<T>, nthreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
cudaError_t launch_forward(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st) {
  return launch_cluster(fwd_kernel<T>, a, cl, nthreads, smem_forward<T>(a.R, a.W), st);
}
template <typename T>
cudaError_t launch_adjoint(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st) {
  return launch_cluster(adj_kernel<T>, a, cl, nthreads, smem_adjoint<T>(a.R, a.W), st);
}
template <typename T>
cudaError_t launch_tlm(const SweepArgs<T>& a, int cl, int nthreads, cudaStream_t st) {
  return launch_cluster(tlm_kernel<T>, a, cl, nthreads, smem_tlm<T>(a.R, a.W), st);
}

#define DD4DV_INST(T)                                                                        \
  template size_t smem_forward<T>(int, int);                                                 \
  template size_t smem_adjoint<T>(int, int);                                                 \
  template size_t smem_tlm<T>(int, int);                                                     \
  template int occupancy_adjoint<T>(int, int, int);                                          \
  template cudaError_t launch_forward<T>(const SweepArgs<T>&, int, int, cudaStream_t);       \
  template cudaError_t launch_adjoint<T>(const SweepArgs<T>&, int, int, cudaStream_t);       \
  template cudaError_t launch_tlm<T>(const SweepArgs<T>&, int, int, cudaStream_t);
DD4DV_INST(double)
DD4DV_INST(float)
#undef DD4DV_INST

}  // namespace dd4dv
