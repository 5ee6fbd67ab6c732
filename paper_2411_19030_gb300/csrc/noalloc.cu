// noalloc.cu -- ptg_sensitivities_noalloc: the sensitivity reduction (a6) without any
// device allocation, for callers that are not allowed to allocate.
//
// Its per-chunk partial sums live in one file-scope __device__ array of fixed size
// (PTG_NOALLOC_SCRATCH_DOUBLES doubles).  Every GPU that loads this library holds that
// array for the lifetime of the process.  The host never dereferences the array's name:
// in host code it is only a stand-in for the device symbol, so its device address is looked
// up once per device with cudaGetSymbolAddress and passed to the kernel.
//
// The per-element accumulation (sens_element_sum) and the chunk reduction are the ones of
// ptg_sensitivities; only the source of dk/drho and dc/drho differs (evaluated from rho here,
// read from the op's workspace there).
#include <algorithm>
#include <cstdio>
#include <mutex>
#include "ptg_device.cuh"
#include "ptg_internal.h"
#include "trace.h"

namespace {

constexpr long long kScratchDoubles = PTG_NOALLOC_SCRATCH_DOUBLES;
constexpr int kMaxDevices = 64;
constexpr int kMaxChunks = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Partial sums over a contiguous chunk of time steps of
//   lambda_j,e^T ( dk_e Ke T_j,e + dc_e/dt Me (T_j - T_{j-1})_e )   (sens_element_sum),
// with dk_e and dc_e evaluated from rho (Eq. 2.5-2.6 differentiated) inside the kernel, so
// the call needs no coefficient workspace.  A value of rho outside [0, 1] (or NaN) is taken
// as 0, as the assembly does (which also records the error in its op's status word).
__global__ void sens_noalloc_kernel(int nx, int ny, double h, double dt, ptg_material m, const double* __restrict__ rho,
                                    const double* __restrict__ lam, int j0, int j1, const double* __restrict__ T,
                                    int hist_j0, int steps_per_chunk, double* __restrict__ partial) {
  const int Ne = nx * ny, nn = nx + 1, Nn = nn * (ny + 1);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ne) return;
  const int chunk = blockIdx.y;
  const int ja = j0 + chunk * steps_per_chunk;
  const int jb = min(j1, ja + steps_per_chunk - 1);
  const int ey = e / nx, ex = e % nx;
  double r = rho[e];
  if (!(r >= 0.0 && r <= 1.0)) r = 0.0;
  const bool has_dc = m.c0 != m.cmin;
  const double dke = (m.k0 == m.kmin) ? 0.0 : m.pk * (m.k0 - m.kmin) * pow(r, m.pk - 1.0);
  const double dce = has_dc ? m.pc * (m.c0 - m.cmin) * pow(r, m.pc - 1.0) / dt : 0.0;
  const double acc = ja <= jb ? ptg::sens_element_sum(ey * nn + ex, nn, Nn, h * h / 36.0, dke, dce, has_dc, lam, j0,
                                                      T, hist_j0, ja, jb)
                              : 0.0;
  partial[(size_t)chunk * Ne + e] = acc;
}

// Device address of the scratch array for the current device, looked up once per device and
// kept for the life of the process (so the entry point must not be used after a
// cudaDeviceReset of that device, which reloads the module).
cudaError_t scratch_for_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

int ptg_sensitivities_noalloc(int nx, int ny, double h, int Nt, double dt, const ptg_material* mat,
                              const double* rho_d, const double* lam_hist, int j0, int j1, const double* T_hist,
                              int hist_j0, int hist_rows, double* grad_d, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!mat || !rho_d || !lam_hist || !T_hist || !grad_d) return PTG_EINVAL;
  if (nx < 1 || ny < 1 || Nt < 1 || !(h > 0.0) || !(dt > 0.0)) return PTG_EINVAL;
  if (j0 < 1 || j1 < j0 || j1 > Nt) return PTG_EINVAL;
  if (j0 - 1 < hist_j0 || j1 >= hist_j0 + hist_rows) return PTG_EINVAL;
  // the material rules of ptg_op_create: positive conductivities and capacities
  if (!(mat->k0 > 0.0) || !(mat->kmin > 0.0) || !(mat->c0 > 0.0) || !(mat->cmin > 0.0)) {
    ptg::set_last_error("ptg_sensitivities_noalloc: k0, kmin, c0 and cmin must be positive");
    return PTG_EINVAL;
  }
  const long long Ne = (long long)nx * ny;
  if (Ne > kScratchDoubles) {
    char msg[200];
    std::snprintf(msg, sizeof(msg), "ptg_sensitivities_noalloc: %lld elements exceed the %lld-double scratch array",
                  Ne, kScratchDoubles);
    ptg::set_last_error(msg);
    return PTG_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_device(&scratch);
  if (e != cudaSuccess) {
    ptg::set_last_error(cudaGetErrorString(e));
    return PTG_ECUDA;
  }
  const int nsteps = j1 - j0 + 1;
  int nchunks = (int)std::min<long long>(kMaxChunks, kScratchDoubles / Ne);
  nchunks = std::max(1, std::min(nchunks, nsteps));
  const int spc = (nsteps + nchunks - 1) / nchunks;
  const int used = (nsteps + spc - 1) / spc;
  dim3 grid((unsigned)((Ne + 255) / 256), (unsigned)used);
  sens_noalloc_kernel<<<grid, 256, 0, stream>>>(nx, ny, h, dt, *mat, rho_d, lam_hist, j0, j1, T_hist, hist_j0, spc,
                                                scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = ptg::launch_sens_reduce((int)Ne, used, 1.0 / Nt, scratch, grad_d, stream);
  if (e != cudaSuccess) {
    ptg::set_last_error(cudaGetErrorString(e));
    return PTG_ECUDA;
  }
  return PTG_OK;
}

}  // extern "C"
