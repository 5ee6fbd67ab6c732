// design.cu -- the design parametrisation of Sec. 2.1 on the device: the density filter H
// (a weighted average over the elements within r_fil of each element centre, cone weights
// w = r_fil - distance, rows normalised), the threshold projection P, the area fraction of
// Sec. 3, and the chain rule d/dchi = H^T (P'(H chi) * d/drho).  All FP64.
#include <cmath>
#include <cstdint>
#include <new>
#include "ptg_internal.h"
#include "trace.h"

struct ptg_design {
  int device = 0;
  int nx = 0, ny = 0, Ne = 0, R = 0;
  double h = 0, r_fil = 0, beta = 0, eta = 0;
  double* wts = nullptr;     // [(2R+1)^2] cone weights of the offsets (0 outside the disc)
  double* rowsum = nullptr;  // [Ne] sum of the weights of each element's in-grid neighbours
  double* partial = nullptr; // [kVolBlocks] partial sums of the area fraction
};

namespace ptg {
namespace {

constexpr int kVolBlocks = 256;

// row sums of H's weights (the normalisation)
__global__ void rowsum_kernel(int nx, int ny, int R, const double* __restrict__ wts, double* __restrict__ S) {
  const int Ne = nx * ny, side = 2 * R + 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ne; e += gridDim.x * blockDim.x) {
    const int ey = e / nx, ex = e - ey * nx;
    double s = 0.0;
    for (int dy = -R; dy <= R; ++dy) {
      const int jy = ey + dy;
      if (jy < 0 || jy >= ny) continue;
      for (int dx = -R; dx <= R; ++dx) {
        const int jx = ex + dx;
        if (jx < 0 || jx >= nx) continue;
        s += wts[(dy + R) * side + dx + R];
      }
    }
    S[e] = s;
  }
}

// chi_fil = H chi, rho = P(chi_fil), dproj = P'(chi_fil)
__global__ void forward_kernel(int nx, int ny, int R, const double* __restrict__ wts, const double* __restrict__ S,
                               double beta, double eta, const double* __restrict__ chi, double* __restrict__ rho,
                               double* __restrict__ dproj) {
  const int Ne = nx * ny, side = 2 * R + 1;
  const double den = tanh(beta * (1.0 - eta)) + tanh(beta * eta);
  const double t_eta = tanh(beta * eta);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ne; e += gridDim.x * blockDim.x) {
    const int ey = e / nx, ex = e - ey * nx;
    double s = 0.0;
    for (int dy = -R; dy <= R; ++dy) {
      const int jy = ey + dy;
      if (jy < 0 || jy >= ny) continue;
      const double* wrow = wts + (dy + R) * side + R;
      const double* crow = chi + jy * nx;
      for (int dx = -R; dx <= R; ++dx) {
        const int jx = ex + dx;
        if (jx < 0 || jx >= nx) continue;
        s = fma(wrow[dx], crow[jx], s);
      }
    }
    const double xf = s / S[e];
    const double t = tanh(beta * (xf - eta));
    rho[e] = (t + t_eta) / den;
    dproj[e] = beta * (1.0 - t * t) / den;
  }
}

// out_j = sum_i H_ij dproj_i y_i = sum over neighbours i of j of w_ij dproj_i y_i / S_i (the
// weights are symmetric); y == nullptr stands for the constant 1/Ne (area-fraction gradient)
__global__ void backward_kernel(int nx, int ny, int R, const double* __restrict__ wts, const double* __restrict__ S,
                                const double* __restrict__ dproj, const double* __restrict__ y,
                                double* __restrict__ out) {
  const int Ne = nx * ny, side = 2 * R + 1;
  const double inv_ne = 1.0 / (double)Ne;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ne; e += gridDim.x * blockDim.x) {
    const int ey = e / nx, ex = e - ey * nx;
    double s = 0.0;
    for (int dy = -R; dy <= R; ++dy) {
      const int iy = ey + dy;
      if (iy < 0 || iy >= ny) continue;
      const double* wrow = wts + (dy + R) * side + R;
      for (int dx = -R; dx <= R; ++dx) {
        const int ix = ex + dx;
        if (ix < 0 || ix >= nx) continue;
        const int i = iy * nx + ix;
        const double yi = y ? y[i] : inv_ne;
        s = fma(wrow[dx], dproj[i] * yi / S[i], s);
      }
    }
    out[e] = s;
  }
}

// mean(rho): fixed-order block sums, then one block sums the partials in order
__global__ void volume_partial_kernel(int Ne, const double* __restrict__ rho, double* __restrict__ partial) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ne; e += gridDim.x * blockDim.x) s += rho[e];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void volume_final_kernel(int Ne, int nb, const double* __restrict__ partial, double* __restrict__ out) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[b];
  *out = s / (double)Ne;
}

}  // namespace
}  // namespace ptg

using namespace ptg;

extern "C" {

int ptg_design_create(int nx, int ny, double h, double r_fil, double beta, double eta, int device,
                      ptg_design** out) {
  PTG_TRACE(__func__);
  if (!out) return PTG_EINVAL;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || !(h > 0.0) || !(r_fil > 0.0) || !(beta > 0.0) ||
      !(eta > 0.0 && eta < 1.0))
    return PTG_EINVAL;
  const int R = (int)std::ceil(r_fil / h);
  if (R > 64) return PTG_EINVAL;          // a filter wider than 129 x 129 elements
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return PTG_ECUDA;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  ptg_design* d = new (std::nothrow) ptg_design();
  if (!d) return PTG_ENOMEM;
  d->device = device;
  d->nx = nx;
  d->ny = ny;
  d->Ne = nx * ny;
  d->R = R;
  d->h = h;
  d->r_fil = r_fil;
  d->beta = beta;
  d->eta = eta;
  const int side = 2 * R + 1;
  double* w = new (std::nothrow) double[side * side];
  cudaError_t e = w ? cudaSuccess : cudaErrorMemoryAllocation;
  if (w)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        const double v = r_fil - h * std::sqrt((double)(dx * dx + dy * dy));
        w[(dy + R) * side + dx + R] = v > 0.0 ? v : 0.0;
      }
  if (e == cudaSuccess) e = cudaMalloc(&d->wts, sizeof(double) * side * side);
  if (e == cudaSuccess) e = cudaMalloc(&d->rowsum, sizeof(double) * d->Ne);
  if (e == cudaSuccess) e = cudaMalloc(&d->partial, sizeof(double) * kVolBlocks);
  if (e == cudaSuccess) e = cudaMemcpy(d->wts, w, sizeof(double) * side * side, cudaMemcpyHostToDevice);
  delete[] w;
  if (e == cudaSuccess) {
    rowsum_kernel<<<(d->Ne + 255) / 256, 256>>>(nx, ny, R, d->wts, d->rowsum);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ptg_design_destroy(d);
    return e == cudaErrorMemoryAllocation ? PTG_ENOMEM : PTG_ECUDA;
  }
  *out = d;
  return PTG_OK;
}

void ptg_design_destroy(ptg_design* d) {
  if (!d) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);
  cudaFree(d->wts);
  cudaFree(d->rowsum);
  cudaFree(d->partial);
  cudaSetDevice(prev);
  delete d;
}

static int grid_for(int n) { return (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096; }

int ptg_design_forward(ptg_design* d, const double* chi_d, double* rho_d, double* dproj_d, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!d || !chi_d || !rho_d || !dproj_d) return PTG_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);
  forward_kernel<<<grid_for(d->Ne), 256, 0, stream>>>(d->nx, d->ny, d->R, d->wts, d->rowsum, d->beta, d->eta, chi_d,
                                                       rho_d, dproj_d);
  cudaError_t e = cudaGetLastError();
  cudaSetDevice(prev);
  return e == cudaSuccess ? PTG_OK : PTG_ECUDA;
}

int ptg_design_backward(ptg_design* d, const double* dproj_d, const double* df_drho_d, double* df_dchi_d,
                        cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!d || !dproj_d || !df_dchi_d) return PTG_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);
  backward_kernel<<<grid_for(d->Ne), 256, 0, stream>>>(d->nx, d->ny, d->R, d->wts, d->rowsum, dproj_d, df_drho_d,
                                                        df_dchi_d);
  cudaError_t e = cudaGetLastError();
  cudaSetDevice(prev);
  return e == cudaSuccess ? PTG_OK : PTG_ECUDA;
}

int ptg_design_volume(ptg_design* d, const double* rho_d, double* vol_d, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!d || !rho_d || !vol_d) return PTG_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);
  volume_partial_kernel<<<kVolBlocks, 256, 0, stream>>>(d->Ne, rho_d, d->partial);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    volume_final_kernel<<<1, 1, 0, stream>>>(d->Ne, kVolBlocks, d->partial, vol_d);
    e = cudaGetLastError();
  }
  cudaSetDevice(prev);
  return e == cudaSuccess ? PTG_OK : PTG_ECUDA;
}

}  // extern "C"
