// mesh.cu -- coarse propagators on the mesh of spacing 2h, the remedy for the sequential
// coarse sweep that the paper proposes (Sec. 7.3).  The coarse solves run in the same stepper on
// a second op whose grid has nx/2 x ny/2 elements (coarse design = mean of the four children).
// These kernels are the fine-mesh parts around them:
//   R  injection of fine nodal states to the coarse nodes,
//   P^T restriction of the adjoint source scale T^(p-1) (bilinear weights, as a load),
//   P  bilinear prolongation of coarse results, fused with the Parareal correction
//      (+ F - G_old), the history row and the fine-mesh p-norm of the prolongated state,
//   the theta recurrences and the g increments (Eq. 4.7) of G on the fine mesh.
// Row arguments (MeshRows) address row r of a stack of node or element vectors as
// base + (row0 + r * step) * n, so one kernel serves shifted and time-reversed sweeps.
#include "mesh.h"
#include "ptg_device.cuh"

namespace ptg {

namespace {

__device__ __forceinline__ const double* row_of(const MeshRows& a, int r, long long n) {
  return a.p ? a.p + (a.row0 + (long long)r * a.step) * n : nullptr;
}
__device__ __forceinline__ double* row_of(const MeshRowsW& a, int r, long long n) {
  return a.p ? a.p + (a.row0 + (long long)r * a.step) * n : nullptr;
}

__global__ void design_kernel(int nx, int ny, const double* __restrict__ rho, double* __restrict__ rhoH) {
  const int nxH = nx / 2, NeH = nxH * (ny / 2);
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= NeH) return;
  const int EY = E / nxH, EX = E - EY * nxH;
  const int e = 2 * EY * nx + 2 * EX;
  rhoH[E] = 0.25 * ((rho[e] + rho[e + 1]) + (rho[e + nx] + rho[e + nx + 1]));
}

// out[r] = R in[r]: the value at fine node (2I, 2J) for coarse node (I, J), 0 at coarse sinks.
__global__ void inject_kernel(int nx, int ny, MeshRows in, MeshRowsW out, const uint8_t* __restrict__ dirH) {
  const int nxH = nx / 2, nnH = nxH + 1, NnH = nnH * (ny / 2 + 1), Nn = (nx + 1) * (ny + 1);
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (I >= NnH) return;
  const int J = I / nnH, X = I - J * nnH;
  const double* src = row_of(in, r, Nn);
  double* dst = row_of(out, r, NnH);
  dst[I] = dirH[I] ? 0.0 : src[2 * J * (nx + 1) + 2 * X];
}

// out[r] = P^T (scale T[r]^(p-1)) on the coarse nodes (0 at coarse sinks); T is 0 at fine sinks,
// whose rows of P are zero.  scale = Theta^(1-p)/Ne (power mean) or p/Ne (modified objective).
__global__ void source_kernel(int nx, int ny, MeshRows T, MeshRowsW out, const double* __restrict__ Theta, double p,
                              int p_int, int objective, const uint8_t* __restrict__ dirF,
                              const uint8_t* __restrict__ dirH) {
  const int nn = nx + 1, nxH = nx / 2, nnH = nxH + 1, NnH = nnH * (ny / 2 + 1), Nn = nn * (ny + 1);
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (I >= NnH) return;
  double* dst = row_of(out, r, NnH);
  if (dirH[I]) {
    dst[I] = 0.0;
    return;
  }
  const double Ne = (double)nx * (double)ny;
  const double scale = (objective == PTG_OBJ_MODIFIED ? p : pow(*Theta, 1.0 - p)) / Ne;
  const double* t = row_of(T, r, Nn);
  const int J = I / nnH, X = I - J * nnH;
  double acc = 0.0;
  for (int dy = -1; dy <= 1; ++dy) {
    const int iy = 2 * J + dy;
    if (iy < 0 || iy > ny) continue;
    const double wy = dy == 0 ? 1.0 : 0.5;
    for (int dx = -1; dx <= 1; ++dx) {
      const int ix = 2 * X + dx;
      if (ix < 0 || ix > nx) continue;
      const int g = iy * nn + ix;
      if (dirF[g]) continue;
      acc += (wy * (dx == 0 ? 1.0 : 0.5)) * (scale * ipow(t[g], p_int - 1));
    }
  }
  dst[I] = acc;
}

// Per fine node i of row r:  v = (P c)_i with c = c1 - c2 + c3 (coarse rows; c2, c3 optional),
//   out[r][i] = v + (f1 - f2)_i   (f1, f2 optional),  out2[r][i] = v (optional),
//   hist[r][i] = out[r][i] (optional),  and the block's partial sum of v^p.
__global__ void prolong_kernel(int nx, int ny, MeshRows c1, MeshRows c2, MeshRows c3, MeshRows f1, MeshRows f2,
                               MeshRowsW out, MeshRowsW out2, MeshRowsW hist, const uint8_t* __restrict__ dirF,
                               const uint8_t* __restrict__ dirH, int p_int, double* __restrict__ pn_partial) {
  const int nn = nx + 1, Nn = nn * (ny + 1), nnH = nx / 2 + 1, NnH = nnH * (ny / 2 + 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  double vp = 0.0;
  if (i < Nn) {
    const double *a = row_of(c1, r, NnH), *b = row_of(c2, r, NnH), *c = row_of(c3, r, NnH);
    const int iy = i / nn, ix = i - iy * nn;
    double v = 0.0;
    if (!dirF[i]) {
      const int J0 = iy / 2, X0 = ix / 2;
      const int ny2 = (iy & 1) ? 2 : 1, nx2 = (ix & 1) ? 2 : 1;
      const double w = (ny2 == 2 ? 0.5 : 1.0) * (nx2 == 2 ? 0.5 : 1.0);
      for (int jy = 0; jy < ny2; ++jy) {
        for (int jx = 0; jx < nx2; ++jx) {
          const int I = (J0 + jy) * nnH + X0 + jx;
          if (dirH[I]) continue;
          double cv = a[I];
          if (b) cv = cv - b[I];
          if (c) cv = cv + c[I];
          v += w * cv;
        }
      }
    }
    double o = v;
    const double *fa = row_of(f1, r, Nn), *fb = row_of(f2, r, Nn);
    if (fa) o = v + (fb ? fa[i] - fb[i] : fa[i]);
    row_of(out, r, Nn)[i] = o;
    if (double* o2 = row_of(out2, r, Nn)) o2[i] = v;
    if (double* hh = row_of(hist, r, Nn)) hh[i] = o;
    vp = ipow(v, p_int);
  }
  // block sum in a fixed order: warp butterfly, then warp 0 over the warp sums
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) vp += __shfl_xor_sync(0xffffffffu, vp, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = vp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    pn_partial[(size_t)r * gridDim.x + blockIdx.x] = s;
  }
}

__device__ __forceinline__ double g_theta(double theta, double pn, double inv_norm, double p, int p_int, int objective) {
  const double inc = pn * inv_norm;
  return objective == PTG_OBJ_MODIFIED ? theta + inc : pow(ipow(theta, p_int) + inc, 1.0 / p);
}

// theta of G on independent states: out[s] = G_theta(theta_in[s], pn[s]) (pn summed in block order).
__global__ void theta_old_kernel(int nrows, int nb, const double* __restrict__ partial,
                                 const double* __restrict__ theta_in, double* __restrict__ theta_out, double inv_norm,
                                 double p, int p_int, int objective) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nrows) return;
  double pn = 0.0;
  for (int b = 0; b < nb; ++b) pn += partial[(size_t)s * nb + b];
  theta_out[s] = g_theta(theta_in[s], pn, inv_norm, p, p_int, objective);
}

// The primal correction of theta, in order: X[s+1] = G_theta(X[s], pn[s]) + F[s] - G[s].
__global__ void theta_chain_kernel(int ntau, int nb, const double* __restrict__ partial, const double* __restrict__ F,
                                   const double* __restrict__ G, double* __restrict__ X, double inv_norm, double p,
                                   int p_int, int objective) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double theta = X[0];
  for (int s = 0; s < ntau; ++s) {
    double pn = 0.0;
    for (int b = 0; b < nb; ++b) pn += partial[(size_t)s * nb + b];
    theta = (g_theta(theta, pn, inv_norm, p, p_int, objective) + F[s]) - G[s];
    X[s + 1] = theta;
  }
}

// dg[r][e] = -(1/Ntau) lambda_r,e^T (dk_e Ke T_k,e + dc_e/dtau Me (T_k - T_{k-M})_e)   (Eq. 4.7)
// with k = M s + 1 for s = s_of(r) and T_{k-M} read as T_0 for s = 0.
__global__ void dg_kernel(int nx, int ny, double h, double dtau, int has_dc, const double* __restrict__ dk,
                          const double* __restrict__ dc, MeshRows lam, const double* __restrict__ T_hist, int M,
                          int s0, int s_step, double inv_ntau, double* __restrict__ dg) {
  const int Ne = nx * ny, nn = nx + 1, Nn = nn * (ny + 1);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (e >= Ne) return;
  const int s = s0 + r * s_step;
  const int k = M * s + 1, km = k - M > 0 ? k - M : 0;
  const double* Tk = T_hist + (size_t)k * Nn;
  const double* Tm = T_hist + (size_t)km * Nn;
  const double* L = row_of(lam, r, Nn);
  const int ey = e / nx, ex = e - ey * nx, g0 = ey * nn + ex;
  const double lsw = L[g0], lse = L[g0 + 1], lne = L[g0 + nn + 1], lnw = L[g0 + nn];
  const double tsw = Tk[g0], tse = Tk[g0 + 1], tne = Tk[g0 + nn + 1], tnw = Tk[g0 + nn];
  // unit-coefficient Ke = (1/6)[[4,-1,-2,-1],[-1,4,-1,-2],[-2,-1,4,-1],[-1,-2,-1,4]] (SW, SE, NE, NW)
  double term = dk[e] * ((lsw * (4.0 * tsw - tse - 2.0 * tne - tnw) + lse * (-tsw + 4.0 * tse - tne - 2.0 * tnw) +
                          lne * (-2.0 * tsw - tse + 4.0 * tne - tnw) + lnw * (-tsw - 2.0 * tse - tne + 4.0 * tnw)) /
                         6.0);
  if (has_dc) {
    // Me = h^2/36 [[4,2,1,2],[2,4,2,1],[1,2,4,2],[2,1,2,4]]
    const double dsw = tsw - Tm[g0], dse = tse - Tm[g0 + 1], dne = tne - Tm[g0 + nn + 1], dnw = tnw - Tm[g0 + nn];
    const double cterm = (lsw * (4.0 * dsw + 2.0 * dse + dne + 2.0 * dnw) + lse * (2.0 * dsw + 4.0 * dse + 2.0 * dne + dnw) +
                          lne * (dsw + 2.0 * dse + 4.0 * dne + 2.0 * dnw) + lnw * (2.0 * dsw + dse + 2.0 * dne + 4.0 * dnw)) *
                         (h * h / 36.0);
    term += dc[e] * cterm / dtau;
  }
  dg[(size_t)r * Ne + e] = -(term * inv_ntau);
}

// G_old's g: out[s] = in[s + 1] + dg[s].
__global__ void g_old_kernel(int Ne, int ntau, const double* __restrict__ g_in, const double* __restrict__ dg,
                             double* __restrict__ g_out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)Ne * ntau) return;
  const int s = (int)(t / Ne), e = (int)(t - (long long)s * Ne);
  g_out[t] = g_in[(size_t)(s + 1) * Ne + e] + dg[t];
}

// The reverse correction of g, per element: X[Ntau] = 0 and, for s = Ntau-1 .. 0,
// X[s] = (X[s+1] + dg[s]) + F[s] - G[s]; dg rows are in the order s = Ntau-1 .. 0.
__global__ void g_chain_kernel(int Ne, int ntau, const double* __restrict__ dg_rev, const double* __restrict__ F,
                               const double* __restrict__ G, double* __restrict__ X) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ne) return;
  double g = 0.0;
  X[(size_t)ntau * Ne + e] = 0.0;
  for (int r = 0; r < ntau; ++r) {
    const int s = ntau - 1 - r;
    g = ((g + dg_rev[(size_t)r * Ne + e]) + F[(size_t)s * Ne + e]) - G[(size_t)s * Ne + e];
    X[(size_t)s * Ne + e] = g;
  }
}

}  // namespace

int mesh_blocks(int Nn) { return (Nn + kMeshThreads - 1) / kMeshThreads; }

cudaError_t mesh_design(int nx, int ny, const double* rho, double* rhoH, cudaStream_t st) {
  const int NeH = (nx / 2) * (ny / 2);
  design_kernel<<<(NeH + 255) / 256, 256, 0, st>>>(nx, ny, rho, rhoH);
  return cudaGetLastError();
}

cudaError_t mesh_inject(int nx, int ny, MeshRows in, MeshRowsW out, int nrows, const uint8_t* dirH, cudaStream_t st) {
  const int NnH = (nx / 2 + 1) * (ny / 2 + 1);
  inject_kernel<<<dim3((NnH + 255) / 256, nrows), 256, 0, st>>>(nx, ny, in, out, dirH);
  return cudaGetLastError();
}

cudaError_t mesh_source(int nx, int ny, MeshRows T, MeshRowsW out, int nrows, const double* Theta, double p, int p_int,
                        int objective, const uint8_t* dirF, const uint8_t* dirH, cudaStream_t st) {
  const int NnH = (nx / 2 + 1) * (ny / 2 + 1);
  source_kernel<<<dim3((NnH + 255) / 256, nrows), 256, 0, st>>>(nx, ny, T, out, Theta, p, p_int, objective, dirF, dirH);
  return cudaGetLastError();
}

cudaError_t mesh_prolong(int nx, int ny, MeshRows c1, MeshRows c2, MeshRows c3, MeshRows f1, MeshRows f2,
                         MeshRowsW out, MeshRowsW out2, MeshRowsW hist, int nrows, const uint8_t* dirF,
                         const uint8_t* dirH, int p_int, double* pn_partial, cudaStream_t st) {
  const int Nn = (nx + 1) * (ny + 1);
  prolong_kernel<<<dim3(mesh_blocks(Nn), nrows), kMeshThreads, 0, st>>>(nx, ny, c1, c2, c3, f1, f2, out, out2, hist,
                                                                         dirF, dirH, p_int, pn_partial);
  return cudaGetLastError();
}

cudaError_t mesh_theta_old(int nrows, int nb, const double* partial, const double* theta_in, double* theta_out,
                           double inv_norm, double p, int p_int, int objective, cudaStream_t st) {
  theta_old_kernel<<<(nrows + 127) / 128, 128, 0, st>>>(nrows, nb, partial, theta_in, theta_out, inv_norm, p, p_int,
                                                        objective);
  return cudaGetLastError();
}

cudaError_t mesh_theta_chain(int ntau, int nb, const double* partial, const double* F, const double* G, double* X,
                             double inv_norm, double p, int p_int, int objective, cudaStream_t st) {
  theta_chain_kernel<<<1, 32, 0, st>>>(ntau, nb, partial, F, G, X, inv_norm, p, p_int, objective);
  return cudaGetLastError();
}

cudaError_t mesh_dg(int nx, int ny, double h, double dtau, int has_dc, const double* dk, const double* dc, MeshRows lam,
                    const double* T_hist, int M, int s0, int s_step, int nrows, double inv_ntau, double* dg,
                    cudaStream_t st) {
  const int Ne = nx * ny;
  dg_kernel<<<dim3((Ne + 255) / 256, nrows), 256, 0, st>>>(nx, ny, h, dtau, has_dc, dk, dc, lam, T_hist, M, s0, s_step,
                                                           inv_ntau, dg);
  return cudaGetLastError();
}

cudaError_t mesh_g_old(int Ne, int ntau, const double* g_in, const double* dg, double* g_out, cudaStream_t st) {
  const long long n = (long long)Ne * ntau;
  g_old_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Ne, ntau, g_in, dg, g_out);
  return cudaGetLastError();
}

cudaError_t mesh_g_chain(int Ne, int ntau, const double* dg_rev, const double* F, const double* G, double* X,
                         cudaStream_t st) {
  g_chain_kernel<<<(Ne + 255) / 256, 256, 0, st>>>(Ne, ntau, dg_rev, F, G, X);
  return cudaGetLastError();
}

}  // namespace ptg
