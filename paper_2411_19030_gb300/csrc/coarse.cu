// coarse.cu -- set-up of the two-level preconditioner of the coarse-step solves.
//
// The solves with C/dtau + K (the coarse propagators G and the sequential correction sweep)
// are the worst conditioned of the pass.  Their FP32 CG is preconditioned additively with
//     M^-1 = D^-1 + P Ac^-1 P^T
// where D is the diagonal and P the piecewise-constant prolongation from aggregates of nodes:
// node (iy, ix) belongs to aggregate (ay, ax) with ay = min(iy / m, nay - 1) and
// ax = min(((ix + 1) / 4) / (m / 4), nax - 1), so that every aligned group of 4 nodes of the
// stepper (nodes 4g-1 .. 4g+2 of a row) lies in one aggregate; nax = (nx + 1) / m and
// nay = (ny + 1) / m aggregates per direction (at least 1), the last ones absorbing the
// remainder.  Ac = P^T A P restricted to the free nodes.  This file builds Ac in FP64,
// factors its band (half-bandwidth nax + 1) as L D L^T in FP32 and forms the dense inverse in
// FP32 (symmetrised, rows padded to a multiple of 4), which the stepper reads row-wise.
#include <cstdint>
#include "ptg_internal.h"

namespace ptg {

// One CTA per aggregate a = (ay, ax); the threads stride over its nodes.  For a free node i
// the 9-point row of A is split by the aggregate of each free neighbour j (one of the 3 x 3
// aggregates around a): Ac[a][b] = sum over i in a, j in b of A_ij.  Fixed-order block sums.
__global__ void galerkin_kernel(int nx, int ny, int W, int m, int nax, int nay, NodeWeights A,
                                const uint8_t* __restrict__ dirichlet, double* __restrict__ Ac) {
  const int a = blockIdx.x;
  const int ax = a % nax, ay = a / nax;
  const int nc = nax * nay;
  const int m4 = m / 4;
  // node extent of the aggregate
  const int y0 = ay * m, y1 = (ay == nay - 1) ? ny : ay * m + m - 1;
  const int x0 = max(0, ax * m - 1), x1 = (ax == nax - 1) ? nx : ax * m + m - 2;
  const int wx = x1 - x0 + 1, cnt = wx * (y1 - y0 + 1);
  auto agg_y = [&](int iy) { return min(iy / m, nay - 1); };
  auto agg_x = [&](int ix) { return min(((ix + 1) >> 2) / m4, nax - 1); };
  auto free_node = [&](int iy, int ix) {
    return iy >= 0 && iy <= ny && ix >= 0 && ix <= nx && !dirichlet[iy * (nx + 1) + ix];
  };
  __shared__ double part[9][32];
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int iy = y0 + t / wx, ix = x0 + t % wx;
    if (!free_node(iy, ix)) continue;
    const int go = (iy + 1) * W + ix + 1;
    // (offset, weight) of the 9 neighbours: C, E, W, N, S, NE, SW, NW, SE
    const int dyv[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
    const int dxv[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
    const double wv[9] = {A.C[go], A.E[go], A.E[go - 1], A.N[go], A.N[go - W],
                          A.NE[go], A.NE[go - W - 1], A.NW[go], A.NW[go - W + 1]};
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      const int jy = iy + dyv[n], jx = ix + dxv[n];
      if (!free_node(jy, jx)) continue;
      const int k = (agg_y(jy) - ay + 1) * 3 + (agg_x(jx) - ax + 1);
#pragma unroll
      for (int kk = 0; kk < 9; ++kk)
        if (kk == k) acc[kk] += wv[n];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double s = acc[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    const int k = threadIdx.x;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += part[k][w];
    const int bx = ax + k % 3 - 1, by = ay + k / 3 - 1;
    if (bx >= 0 && bx < nax && by >= 0 && by < nay) Ac[(size_t)a * nc + by * nax + bx] = s;
  }
}

// Band LDL^T of Ac (half-bandwidth b <= kCoarseMaxAgg + 1 < 32) in FP32 by one warp (the
// aggregated coarse matrix is well conditioned: the mass term C/dtau bounds its smallest
// eigenvalue away from zero, so FP32 factors give the inverse to about 1e-7 relative, ample
// for a preconditioner).  The working band sits in shared memory:
// w[i * (b+1) + (i - j)] = A[i][j] for i - b <= j <= i.  Step k: lane l owns row i = k+1+l of
// the trailing window and subtracts A[i][k] A[j][k] / D[k] from A[i][j], k < j <= i, taking
// A[j][k] from lane j-k-1 by shuffle.  Output, in `band`: the unit lower factor L[i][j] at the
// same positions and 1/D[i] in the diagonal slot.  A pivot D[k] <= 0 (an aggregate made only
// of Dirichlet nodes has an empty row) is replaced by 1 so that the preconditioner stays
// defined.
__global__ void band_ldlt_kernel(int nc, int b, const double* __restrict__ Ac, float* __restrict__ band) {
  extern __shared__ float w[];
  const int bw = b + 1;
  const int lane = threadIdx.x;
  for (int t = lane; t < nc * bw; t += 32) {
    const int i = t / bw, d = t - i * bw;
    w[t] = (i - d >= 0) ? (float)Ac[(size_t)i * nc + (i - d)] : 0.f;
  }
  __syncwarp();
  for (int k = 0; k < nc; ++k) {
    float dk = w[k * bw];
    if (!(dk > 0.f)) dk = 1.f;
    const float r = 1.0f / dk;
    const int i = k + 1 + lane;
    const bool mine = lane < b && i < nc;
    const float aik = mine ? w[i * bw + (i - k)] : 0.f;
    if (lane == 0) band[k * bw] = r;
    if (mine) band[i * bw + (i - k)] = aik * r;
    const float sik = aik * r;
    for (int jj = 0; jj < b; ++jj) {      // j = k+1+jj
      const float ajk = __shfl_sync(0xffffffffu, aik, jj);
      if (mine && jj <= lane) w[i * bw + (lane - jj)] -= sik * ajk;
    }
    __syncwarp();
  }
}

// Columns of Ac^-1 from the LDL^T factor: one lane per column, 32 columns per CTA, the
// substitutions L y = e_c, z = D^-1 y, L^T x = z in FP32 (the inverse is only a
// preconditioner and is stored in FP32).  X[i * nc + c] is the compact result.  The band
// loops run over a fixed kBandMax terms with out-of-band terms reading a zero, so that the
// loads of a row are issued together.
constexpr int kBandMax = kCoarseMaxAgg + 1;
__global__ void band_inverse_kernel(int nc, int b, const float* __restrict__ band, float* __restrict__ X) {
  extern __shared__ float fsm[];
  constexpr int bw = kBandMax + 1;
  float* L = fsm;                       // [nc][bw], zero beyond the band
  float* y = fsm + nc * bw;             // [nc + kBandMax][32], rows -kBandMax..-1 and beyond stay 0
  for (int t = threadIdx.x; t < nc * bw; t += blockDim.x) {
    const int i = t / bw, d = t - i * bw;
    L[t] = (d <= b && i - d >= 0) ? band[i * (b + 1) + d] : 0.f;
  }
  for (int t = threadIdx.x; t < (nc + kBandMax) * 32; t += blockDim.x) y[t] = 0.f;
  __syncthreads();
  float* yv = y + kBandMax * 32;        // yv[i * 32 + lane], i = -kBandMax .. nc-1
  const int lane = threadIdx.x;
  const int c = blockIdx.x * 32 + lane;
  const bool live = c < nc;
  for (int i = 0; i < nc; ++i) {        // L y = e_c
    float s0 = (live && i == c) ? 1.f : 0.f, s1 = 0.f;
#pragma unroll
    for (int d = 1; d <= kBandMax; d += 2) {
      s0 = fmaf(-L[i * bw + d], yv[(i - d) * 32 + lane], s0);
      if (d + 1 <= kBandMax) s1 = fmaf(-L[i * bw + d + 1], yv[(i - d - 1) * 32 + lane], s1);
    }
    yv[i * 32 + lane] = s0 + s1;
    __syncwarp();
  }
  for (int i = 0; i < nc; ++i) yv[i * 32 + lane] *= L[i * bw];   // z = D^-1 y
  __syncwarp();
  for (int i = nc - 1; i >= 0; --i) {   // L^T x = z; rows j > nc-1 read L = 0 via the guard
    float s0 = yv[i * 32 + lane], s1 = 0.f;
#pragma unroll
    for (int d = 1; d <= kBandMax; d += 2) {
      const int j = i + d;
      if (j < nc) s0 = fmaf(-L[j * bw + d], yv[j * 32 + lane], s0);
      if (d + 1 <= kBandMax && j + 1 < nc) s1 = fmaf(-L[(j + 1) * bw + d + 1], yv[(j + 1) * 32 + lane], s1);
    }
    yv[i * 32 + lane] = s0 + s1;
    __syncwarp();
  }
  if (live)
    for (int i = 0; i < nc; ++i) X[(size_t)i * nc + c] = yv[i * 32 + lane];
}

// Ainv in the padded layout (index ay * naxp + ax, ncp = nay * naxp), symmetrised:
// Ainv[P][Q] = (X[p][q] + X[q][p]) / 2, zero where P or Q is a padding index.
__global__ void pack_inverse_kernel(int nax, int nay, const float* __restrict__ X, float* __restrict__ Ainv) {
  const int naxp = coarse_row_stride(nax), ncp = nay * naxp, nc = nax * nay;
  const int Pi = blockIdx.y, Q = blockIdx.x * blockDim.x + threadIdx.x;
  if (Q >= ncp) return;
  const int py = Pi / naxp, px = Pi - py * naxp, qy = Q / naxp, qx = Q - qy * naxp;
  float v = 0.f;
  if (px < nax && qx < nax) {
    const int p = py * nax + px, q = qy * nax + qx;
    v = 0.5f * (X[(size_t)p * nc + q] + X[(size_t)q * nc + p]);
  }
  Ainv[(size_t)Pi * ncp + Q] = v;
}

// ---------------------------------------------------------------------------- three levels
// The 2h level of the three-level cycle: node (I, J), I = 0..nx1, J = 0..ny1 (nx = 2 nx1,
// ny = 2 ny1) sits on fine node (2I, 2J); P1 interpolates bilinearly, so the fine node
// (2I + di, 2J + dj), |di|, |dj| <= 1, takes the weight w(di) w(dj) of 2h node (I, J), with
// w(0) = 1 and w(+-1) = 1/2; rows of P1 at Dirichlet fine nodes are zero.  A1 = P1^T A P1 is a
// 9-point operator; one thread per (2h node a, neighbour b) sums P1(i, a) A(i, j) P1(j, b) over
// the free fine nodes i in the support of a and their free fine neighbours j (fixed order).
// A 2h node whose support holds no free fine node gets the identity row.
__device__ __forceinline__ double p1_weight(int d) { return d == 0 ? 1.0 : 0.5; }

__global__ void galerkin_l1_kernel(int nx, int ny, int W, NodeWeights A, const uint8_t* __restrict__ dirichlet,
                                   int nx1, int ny1, double* __restrict__ A1) {
  const int n1 = (nx1 + 1) * (ny1 + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * n1) return;
  const int k = t / n1, a = t - k * n1;
  const int I = a % (nx1 + 1), J = a / (nx1 + 1);
  const int dI = k % 3 - 1, dJ = k / 3 - 1;
  const int Ib = I + dI, Jb = J + dJ;
  double sum = 0.0;
  auto free_node = [&](int iy, int ix) {
    return iy >= 0 && iy <= ny && ix >= 0 && ix <= nx && !dirichlet[iy * (nx + 1) + ix];
  };
  if (Ib >= 0 && Ib <= nx1 && Jb >= 0 && Jb <= ny1) {
    for (int dj = -1; dj <= 1; ++dj) {
      for (int di = -1; di <= 1; ++di) {
        const int iy = 2 * J + dj, ix = 2 * I + di;
        if (!free_node(iy, ix)) continue;
        const double wa = p1_weight(di) * p1_weight(dj);
        const int go = (iy + 1) * W + ix + 1;
        // the 9 couplings of fine node i: C, E, W, N, S, NE, SW, NW, SE
        const int dyv[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
        const int dxv[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
        const double wv[9] = {A.C[go], A.E[go], A.E[go - 1], A.N[go], A.N[go - W],
                              A.NE[go], A.NE[go - W - 1], A.NW[go], A.NW[go - W + 1]};
        for (int n = 0; n < 9; ++n) {
          const int jy = iy + dyv[n], jx = ix + dxv[n];
          if (!free_node(jy, jx)) continue;
          const int ox = jx - 2 * Ib, oy = jy - 2 * Jb;
          if (ox < -1 || ox > 1 || oy < -1 || oy > 1) continue;
          sum += wa * wv[n] * (p1_weight(ox) * p1_weight(oy));
        }
      }
    }
  }
  if (k == 4 && !(sum > 0.0)) sum = 1.0;   // no free fine node in the support
  A1[(size_t)k * n1 + a] = sum;
}

// A2 = P2^T A1 P2 for aggregates of m x m 2h nodes (nax x nay, the last of a direction
// absorbing the remainder): one CTA per aggregate a, fixed-order block sums into the dense
// [nc][nc] FP64 matrix (as galerkin_kernel on the fine grid).
__global__ void galerkin_l2_kernel(int nx1, int ny1, int m, int nax, int nay, const double* __restrict__ A1,
                                   double* __restrict__ Ac) {
  const int a = blockIdx.x;
  const int ax = a % nax, ay = a / nax;
  const int nc = nax * nay, n1 = (nx1 + 1) * (ny1 + 1);
  const int y0 = ay * m, y1 = (ay == nay - 1) ? ny1 : ay * m + m - 1;
  const int x0 = ax * m, x1 = (ax == nax - 1) ? nx1 : ax * m + m - 1;
  const int wx = x1 - x0 + 1, cnt = wx * (y1 - y0 + 1);
  __shared__ double part[9][32];
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int J = y0 + t / wx, I = x0 + t % wx;
    const int i = J * (nx1 + 1) + I;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int Jb = J + k / 3 - 1, Ib = I + k % 3 - 1;
      if (Jb < 0 || Jb > ny1 || Ib < 0 || Ib > nx1) continue;
      const int kk = (l3_agg(Jb, m, nay) - ay + 1) * 3 + (l3_agg(Ib, m, nax) - ax + 1);
      const double v = A1[(size_t)k * n1 + i];
#pragma unroll
      for (int q = 0; q < 9; ++q)
        if (q == kk) acc[q] += v;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    const int k = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += part[k][w];
    const int bx = ax + k % 3 - 1, by = ay + k / 3 - 1;
    if (bx >= 0 && bx < nax && by >= 0 && by < nay) Ac[(size_t)a * nc + by * nax + bx] = v;
  }
}

cudaError_t launch_threelevel_setup(int nx, int ny, int W, const NodeWeights& A, const uint8_t* dirichlet, int m,
                                    double* A1, double* Ac, float* band, float* X, float* Ainv, cudaStream_t stream) {
  const int nx1 = nx / 2, ny1 = ny / 2, n1 = (nx1 + 1) * (ny1 + 1);
  const int nax = coarse_aggregates(nx1, m), nay = coarse_aggregates(ny1, m);   // (n1 + 1) / m 2h nodes
  const int nc = nax * nay, ncp = coarse_row_stride(nax) * nay;
  const int b = nax + 1;
  galerkin_l1_kernel<<<(9 * n1 + 255) / 256, 256, 0, stream>>>(nx, ny, W, A, dirichlet, nx1, ny1, A1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(Ac, 0, sizeof(double) * nc * nc, stream)) != cudaSuccess) return e;
  galerkin_l2_kernel<<<nc, 128, 0, stream>>>(nx1, ny1, m, nax, nay, A1, Ac);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t ldlt_smem = sizeof(float) * nc * (b + 1);
  const size_t inv_smem = sizeof(float) * (nc * (kBandMax + 1) + (nc + kBandMax) * 32);
  if ((e = configure_kernel((const void*)band_ldlt_kernel, ldlt_smem, false)) != cudaSuccess) return e;
  if ((e = configure_kernel((const void*)band_inverse_kernel, inv_smem, false)) != cudaSuccess) return e;
  band_ldlt_kernel<<<1, 32, ldlt_smem, stream>>>(nc, b, Ac, band);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  band_inverse_kernel<<<(nc + 31) / 32, 32, inv_smem, stream>>>(nc, b, band, X);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  pack_inverse_kernel<<<dim3((ncp + 127) / 128, ncp), 128, 0, stream>>>(nax, nay, X, Ainv);
  return cudaGetLastError();
}

cudaError_t launch_coarse_setup(int nx, int ny, int W, int m, const NodeWeights& A, const uint8_t* dirichlet,
                                double* Ac, float* band, float* X, float* Ainv, cudaStream_t stream) {
  const int nax = coarse_aggregates(nx, m), nay = coarse_aggregates(ny, m);
  const int nc = nax * nay, ncp = coarse_row_stride(nax) * nay;
  const int b = nax + 1;
  cudaError_t e = cudaMemsetAsync(Ac, 0, sizeof(double) * nc * nc, stream);
  if (e != cudaSuccess) return e;
  galerkin_kernel<<<nc, 256, 0, stream>>>(nx, ny, W, m, nax, nay, A, dirichlet, Ac);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t ldlt_smem = sizeof(float) * nc * (b + 1);
  const size_t inv_smem = sizeof(float) * (nc * (kBandMax + 1) + (nc + kBandMax) * 32);
  if ((e = configure_kernel((const void*)band_ldlt_kernel, ldlt_smem, false)) != cudaSuccess) return e;
  if ((e = configure_kernel((const void*)band_inverse_kernel, inv_smem, false)) != cudaSuccess) return e;
  band_ldlt_kernel<<<1, 32, ldlt_smem, stream>>>(nc, b, Ac, band);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  band_inverse_kernel<<<(nc + 31) / 32, 32, inv_smem, stream>>>(nc, b, band, X);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  pack_inverse_kernel<<<dim3((ncp + 127) / 128, ncp), 128, 0, stream>>>(nax, nay, X, Ainv);
  return cudaGetLastError();
}

}  // namespace ptg
