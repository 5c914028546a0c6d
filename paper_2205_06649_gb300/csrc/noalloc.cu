// dd4dv_forward_noalloc: the global model run of dd4dv_forward for callers
// that cannot allocate device memory.
//
// Who needs this: a caller whose device memory is owned by someone else --
// a framework whose caching allocator has already reserved the free memory,
// code that must not allocate after start-up (real-time or certified
// pipelines), or a host thread that must not make the implicit device-wide
// synchronisation that cudaMalloc/cudaFree can cause.  dd4dv_create allocates
// the context's buffers with cudaMalloc, so such a caller cannot use
// dd4dv_forward.  This entry point needs no context and calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// Its scratch (the two intermediate RK3 stage states and the per-row grid
// constants) lives in one file-scope __device__ array of fixed size that
// every GPU which loads this library keeps until the process exits.  The
// device address of that array is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current; that
// first call should therefore come before any stream capture.  The address is
// kept for the life of the process, so a device reset (cudaDeviceReset)
// after that first call is not supported.  The grid constants are computed
// by a kernel on the caller's stream, so a call only enqueues work: it makes
// no host copy and no stream or device synchronisation.  All calls on a
// device share the array: two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be ordered by the
// caller.  Every scratch word a call reads was written earlier by the same
// call, so nothing has to be cleared between calls.
#include "dd4dvar.h"
#include "common.cuh"

#include <cmath>
#include <mutex>
#include <string>

namespace dd4dv {
namespace {

constexpr long long kMaxStateDoubles = 3LL * 512 * 256;   // one state of up to 512 x 256 points
constexpr int kMaxRows = 1024;                            // latitude rows
constexpr long long kRowDoubles = (long long)kMaxRows * (sizeof(RowConst) / sizeof(double));
constexpr long long kScratchDoubles = 2 * kMaxStateDoubles + kRowDoubles;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set-up on the
// first call per device).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Per-row constants of the global grid (Sec. 7), one thread per latitude
// row: cell-centre latitude theta_j = lat_min + (j + 1/2) dtheta and
// A = 1/(2 a cos dlambda), f = 2 Omega sin, tau = tan / a, Bth / cos, g A.
// The products and sums are rounded one by one (no contraction), as the
// host computes them for dd4dv_create.
__global__ void noalloc_rows_kernel(RowConst* rows, int nlon, int nlat, double lat_min_deg,
                                    double lat_max_deg, double radius, double gravity, double omega) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlat) return;
  const double pi = 3.14159265358979323846;
  const double dlam = __ddiv_rn(__dmul_rn(2.0, pi), (double)nlon);
  const double dth = __ddiv_rn(__ddiv_rn(__dmul_rn(__dsub_rn(lat_max_deg, lat_min_deg), pi), 180.0),
                               (double)nlat);
  const double th0 = __ddiv_rn(__dmul_rn(lat_min_deg, pi), 180.0);
  const double Bth = __ddiv_rn(1.0, __dmul_rn(__dmul_rn(2.0, radius), dth));
  const double th = __dadd_rn(th0, __dmul_rn(__dadd_rn((double)j, 0.5), dth));
  RowConst r;
  r.c = cos(th);
  r.A = __ddiv_rn(1.0, __dmul_rn(__dmul_rn(__dmul_rn(2.0, radius), r.c), dlam));
  r.f = __dmul_rn(__dmul_rn(2.0, omega), sin(th));
  r.tau = __ddiv_rn(tan(th), radius);
  r.BinvC = __ddiv_rn(Bth, r.c);
  r.gA = __dmul_rn(gravity, r.A);
  rows[j] = r;
}

}  // namespace
}  // namespace dd4dv

namespace dd4dv {
// Sets the message that dd4dv_last_error(NULL) returns (defined in api.cu).
void set_global_error(const std::string& msg);
}

using namespace dd4dv;

extern "C" dd4dv_status dd4dv_forward_noalloc(const dd4dv_model* model, const double* x0, double* traj,
                                              void* cuda_stream) {
  auto bad = [](dd4dv_status st, const std::string& msg) {
    set_global_error(msg);
    return st;
  };
  if (!model || !x0 || !traj) return bad(DD4DV_EINVAL, "dd4dv_forward_noalloc: NULL argument");
  const dd4dv_model& m = *model;
  if (m.nlon < 3 || m.nlat < 2 || !(m.dt > 0.0) || m.nsteps < 0 || !(m.radius > 0.0) ||
      !(m.gravity > 0.0) || !(m.lat_max_deg > m.lat_min_deg) || m.lat_min_deg <= -90.0 ||
      m.lat_max_deg >= 90.0 || !std::isfinite(m.omega))
    return bad(DD4DV_EINVAL, "dd4dv_forward_noalloc: invalid model parameters");
  const long long G = 3LL * m.nlat * m.nlon;
  if (G > kMaxStateDoubles || m.nlat > kMaxRows)
    return bad(DD4DV_EINVAL, "dd4dv_forward_noalloc: grid larger than the static scratch limit "
                             "(3*nlat*nlon <= 393216 doubles, nlat <= 1024)");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return bad(DD4DV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  double* s1 = scratch;
  double* s2 = scratch + kMaxStateDoubles;
  RowConst* rows_d = reinterpret_cast<RowConst*>(scratch + 2 * kMaxStateDoubles);

  // per-row constants of the grid (Sec. 7), computed on the device into the
  // scratch array; the two scalars the stages take are formed here
  const double pi = 3.14159265358979323846;
  const double dth = (m.lat_max_deg - m.lat_min_deg) * pi / 180.0 / m.nlat;
  const double Bth = 1.0 / (2.0 * m.radius * dth);
  const double gBth = m.gravity * Bth;
  noalloc_rows_kernel<<<(m.nlat + 127) / 128, 128, 0, st>>>(rows_d, m.nlon, m.nlat, m.lat_min_deg,
                                                           m.lat_max_deg, m.radius, m.gravity, m.omega);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(traj, x0, G * sizeof(double), cudaMemcpyDeviceToDevice, st);
  for (int n = 0; n < m.nsteps && e == cudaSuccess; ++n) {
    const double* x = traj + (size_t)n * G;
    double* nx = traj + (size_t)(n + 1) * G;
    e = launch_global_stage(x, x, s1, 0.0, 1.0, rows_d, Bth, gBth, m.dt, m.nlon, m.nlat, st);
    if (e == cudaSuccess)
      e = launch_global_stage(x, s1, s2, 0.75, 0.25, rows_d, Bth, gBth, m.dt, m.nlon, m.nlat, st);
    if (e == cudaSuccess)
      e = launch_global_stage(x, s2, nx, 1.0 / 3.0, 2.0 / 3.0, rows_d, Bth, gBth, m.dt, m.nlon,
                              m.nlat, st);
  }
  if (e != cudaSuccess) return bad(DD4DV_ECUDA, std::string("dd4dv_forward_noalloc: ") + cudaGetErrorString(e));
  set_global_error("");
  return DD4DV_OK;
}
