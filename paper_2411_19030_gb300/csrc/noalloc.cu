// noalloc.cu -- ptg_sensitivities_noalloc: the sensitivity reduction (a6) without any
// device allocation, for callers that are not allowed to allocate.
//
// Its per-chunk partial sums live in one file-scope __device__ array of fixed size
// (PTG_NOALLOC_SCRATCH_DOUBLES doubles).  Every GPU that loads this library holds that
// array for the lifetime of the process.  The host never dereferences the array's name:
// in host code it is only a stand-in for the device symbol, so its device address is looked
// up once per device with cudaGetSymbolAddress and passed to the kernel.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include "ptg_internal.h"

namespace {

constexpr long long kScratchDoubles = PTG_NOALLOC_SCRATCH_DOUBLES;
constexpr int kMaxDevices = 64;
constexpr int kMaxChunks = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Partial sums over a contiguous chunk of time steps of
//   lambda_j,e^T ( dk_e Ke T_j,e + dc_e/dt Me (T_j - T_{j-1})_e ),
// with dk_e and dc_e evaluated from rho (Eq. 2.5-2.6 differentiated) inside the kernel, so
// the call needs no coefficient workspace.
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
  const int g0 = ey * nn + ex;
  const double r = rho[e];
  const double dke = (m.k0 == m.kmin) ? 0.0 : m.pk * (m.k0 - m.kmin) * pow(r, m.pk - 1.0);
  const double dce = (m.c0 == m.cmin) ? 0.0 : m.pc * (m.c0 - m.cmin) * pow(r, m.pc - 1.0) / dt;
  const double h2 = h * h / 36.0;
  double acc = 0.0;
  if (ja <= jb) {
    const double* Tp = T + (size_t)(ja - 1 - hist_j0) * Nn;
    double psw = Tp[g0], pse = Tp[g0 + 1], pne = Tp[g0 + nn + 1], pnw = Tp[g0 + nn];
    for (int j = ja; j <= jb; ++j) {
      const double* Tj = T + (size_t)(j - hist_j0) * Nn;
      const double* Lj = lam + (size_t)(j - j0) * Nn;
      const double tsw = Tj[g0], tse = Tj[g0 + 1], tne = Tj[g0 + nn + 1], tnw = Tj[g0 + nn];
      const double lsw = Lj[g0], lse = Lj[g0 + 1], lne = Lj[g0 + nn + 1], lnw = Lj[g0 + nn];
      // Ke = (1/6)[4 -1 -2 -1; -1 4 -1 -2; -2 -1 4 -1; -1 -2 -1 4], local order SW, SE, NE, NW
      const double ksw = 4.0 * tsw - tse - 2.0 * tne - tnw;
      const double kse = -tsw + 4.0 * tse - tne - 2.0 * tnw;
      const double kne = -2.0 * tsw - tse + 4.0 * tne - tnw;
      const double knw = -tsw - 2.0 * tse - tne + 4.0 * tnw;
      double term = dke * (lsw * ksw + lse * kse + lne * kne + lnw * knw) / 6.0;
      if (dce != 0.0) {
        // Me = (h^2/36)[4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4]
        const double dsw = tsw - psw, dse = tse - pse, dne = tne - pne, dnw = tnw - pnw;
        const double msw = 4.0 * dsw + 2.0 * dse + dne + 2.0 * dnw;
        const double mse = 2.0 * dsw + 4.0 * dse + 2.0 * dne + dnw;
        const double mne = dsw + 2.0 * dse + 4.0 * dne + 2.0 * dnw;
        const double mnw = 2.0 * dsw + dse + 2.0 * dne + 4.0 * dnw;
        term += dce * (lsw * msw + lse * mse + lne * mne + lnw * mnw) * h2;
      }
      acc += term;
      psw = tsw; pse = tse; pne = tne; pnw = tnw;
    }
  }
  partial[(size_t)chunk * Ne + e] = acc;
}

// grad_e += -(1/Nt) * (sum of the chunk partials in chunk order)
__global__ void sens_noalloc_reduce_kernel(int Ne, int nchunks, double inv_nt, const double* __restrict__ partial,
                                           double* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ne) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(size_t)c * Ne + e];
  grad[e] -= inv_nt * s;
}

// Device address of the scratch array for the current device (looked up once per device).
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
  if (!mat || !rho_d || !lam_hist || !T_hist || !grad_d) return PTG_EINVAL;
  if (nx < 1 || ny < 1 || Nt < 1 || !(h > 0.0) || !(dt > 0.0)) return PTG_EINVAL;
  if (j0 < 1 || j1 < j0 || j1 > Nt) return PTG_EINVAL;
  if (j0 - 1 < hist_j0 || j1 >= hist_j0 + hist_rows) return PTG_EINVAL;
  const long long Ne = (long long)nx * ny;
  if (Ne > kScratchDoubles) {
    char msg[200];
    std::snprintf(msg, sizeof(msg), "ptg_sensitivities_noalloc: %lld elements exceed the %lld-double scratch array",
                  Ne, kScratchDoubles);
    ptg::set_last_error(msg);
    return PTG_EINVAL;
  }
  double* scratch = nullptr;
  if (scratch_for_device(&scratch) != cudaSuccess) {
    ptg::set_last_error(cudaGetErrorString(cudaGetLastError()));
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
  if (cudaGetLastError() != cudaSuccess) return PTG_ECUDA;
  sens_noalloc_reduce_kernel<<<(unsigned)((Ne + 255) / 256), 256, 0, stream>>>((int)Ne, used, 1.0 / Nt, scratch,
                                                                              grad_d);
  if (cudaGetLastError() != cudaSuccess) return PTG_ECUDA;
  return PTG_OK;
}

}  // extern "C"
