// mg.cu -- the geometric multigrid hierarchy of the coarse-step operator C/dtau + K, the
// preconditioner of the streamed coarse-step solves (stream.cuh).
//
// Level 0 is the solve's own grid (nx x ny elements); level l+1 keeps the nodes (2I, 2J) of
// level l (nx and ny halve) and carries the Galerkin operator A_{l+1} = P^T A_l P of bilinear
// interpolation P (a fine node takes the mean of the coarse nodes around it: weights 1, 1/2,
// 1/4).  Rows of P at nodes that are not unknowns (Dirichlet nodes on level 0, nodes without
// support below) are zero, so those nodes drop out of every level.  For the Q1 element matrices
// of Sec. 2.2 on a uniform grid, P^T A_h P is the same element operator on the 2h grid, so the
// bounds on the eigenvalues of D^-1 A, and with them the Jacobi damping, carry over to every
// level.  Every level is stored as FP32 per-node weights in the padded node layout of the fine
// arrays (centre, east, north, north-east, north-west; the other four couplings are those of the
// neighbour on the other side) plus omega/diag (0 off the unknowns).
#include <algorithm>
#include "ptg_internal.h"

namespace ptg {

namespace {

// coupling of node i = (x, y) of a level to its neighbour (x + c, y + d), |c|, |d| <= 1, from the
// five stored weights
__device__ __forceinline__ double coupling(const float* __restrict__ w, long long plen, int W, int loc, int c, int d) {
  const float* C = w;
  const float* E = w + plen;
  const float* N = w + 2 * plen;
  const float* NE = w + 3 * plen;
  const float* NW = w + 4 * plen;
  if (d == 0) return c == 0 ? C[loc] : (c == 1 ? E[loc] : E[loc - 1]);
  if (c == 0) return d == 1 ? N[loc] : N[loc - W];
  if (c == d) return d == 1 ? NE[loc] : NE[loc - W - 1];
  return d == 1 ? NW[loc] : NW[loc - W + 1];   // (-1, 1): own NW; (1, -1): NW of the SE neighbour
}

__device__ __forceinline__ double hat(int a) { return a == 0 ? 1.0 : 0.5; }   // |a| <= 1

// Level 0: FP32 copy of the FP64 node weights; omega/diag on the unknowns.  One thread per
// padded entry (rows -1 .. ny + 1); entries outside the grid are zero.
__global__ void mg_level0_kernel(NodeWeights A, const uint8_t* __restrict__ dirichlet, int nx, int ny, int W,
                                 float* __restrict__ w, long long plen, float omega) {
  const int n = (ny + 3) * W;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int iy = t / W - 1, ix = t % W - 1;
    const bool in = ix >= 0 && ix <= nx && iy >= 0 && iy <= ny;
    const int loc = t;
    float c = 0.f, e = 0.f, no = 0.f, ne = 0.f, nw = 0.f, wd = 0.f;
    if (in) {
      c = (float)A.C[loc];
      e = (float)A.E[loc];
      no = (float)A.N[loc];
      ne = (float)A.NE[loc];
      nw = (float)A.NW[loc];
      if (!dirichlet[iy * (nx + 1) + ix] && A.C[loc] > 0.0) wd = (float)(omega / A.C[loc]);
    }
    w[loc] = c;
    w[plen + loc] = e;
    w[2 * plen + loc] = no;
    w[3 * plen + loc] = ne;
    w[4 * plen + loc] = nw;
    w[5 * plen + loc] = wd;
  }
}

// Level l -> l+1: the five stored weights of every coarse node (I, J) are the entries
// (P^T A P)[(I,J), (I,J) + o] for o = (0,0), (1,0), (0,1), (1,1), (-1,1): the sum over the fine
// nodes i around (2I, 2J) and their neighbours k around (2I, 2J) + 2o of P[i,(I,J)] A[i,k]
// P[k,(I,J)+o], over unknowns only (omega/diag of the fine level nonzero).  FP64 sums.
__global__ void mg_galerkin_kernel(const float* __restrict__ wf, long long plf, int nxf, int nyf, int Wf,
                                   float* __restrict__ wc, long long plc, int nxc, int nyc, int Wc, float omega) {
  const float* wdf = wf + 5 * plf;
  const int n = (nyc + 3) * Wc;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int J = t / Wc - 1, I = t % Wc - 1;
    double out[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (I >= 0 && I <= nxc && J >= 0 && J <= nyc) {
      const int offs[5][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}, {-1, 1}};
      for (int o = 0; o < 5; ++o) {
        const int K = I + offs[o][0], L = J + offs[o][1];
        if (K < 0 || K > nxc || L < 0 || L > nyc) continue;
        double s = 0.0;
        for (int b = -1; b <= 1; ++b) {
          const int y = 2 * J + b;
          if (y < 0 || y > nyf) continue;
          for (int a = -1; a <= 1; ++a) {
            const int x = 2 * I + a;
            if (x < 0 || x > nxf) continue;
            const int li = (y + 1) * Wf + x + 1;
            if (wdf[li] == 0.f) continue;
            const double pi = hat(a) * hat(b);
            for (int d = -1; d <= 1; ++d) {
              const int ky = y + d, kb = ky - 2 * L;
              if (ky < 0 || ky > nyf || kb < -1 || kb > 1) continue;
              for (int c = -1; c <= 1; ++c) {
                const int kx = x + c, ka = kx - 2 * K;
                if (kx < 0 || kx > nxf || ka < -1 || ka > 1) continue;
                if (wdf[(ky + 1) * Wf + kx + 1] == 0.f) continue;
                s += pi * coupling(wf, plf, Wf, li, c, d) * (hat(ka) * hat(kb));
              }
            }
          }
        }
        out[o] = s;
      }
    }
    for (int o = 0; o < 5; ++o) wc[o * plc + t] = (float)out[o];
    wc[5 * plc + t] = out[0] > 0.0 ? (float)(omega / out[0]) : 0.f;
  }
}

}  // namespace

int mg_level_count(int nx, int ny) {
  int L = 1;
  while (L < kMgMaxLevels && nx % 2 == 0 && ny % 2 == 0 && std::min(nx, ny) > kMgMinCells) {
    nx /= 2;
    ny /= 2;
    ++L;
  }
  return L;
}

long long mg_layout(int nx, int ny, MgLevel* lv, int L, long long* ws_floats) {
  long long woff = 0, voff = 0;
  for (int l = 0; l < L; ++l) {
    MgLevel& m = lv[l];
    m.nx = nx;
    m.ny = ny;
    m.W = padded_width(nx);
    m.plen = (long long)(ny + 3) * m.W + 2 * kSlack;
    m.woff = woff;
    m.voff = voff;
    woff += 6 * m.plen;
    voff += (l == 0 ? 2 : 4) * m.plen;
    nx /= 2;
    ny /= 2;
  }
  *ws_floats = voff;
  return woff;
}

cudaError_t launch_mg_setup(NodeWeights A, const uint8_t* dirichlet, const MgLevel* lv, int L, float* w,
                            cudaStream_t stream) {
  const MgLevel& l0 = lv[0];
  const int threads = 256;
  auto blocks = [&](long long n) { return (int)std::min<long long>((n + threads - 1) / threads, 4096); };
  mg_level0_kernel<<<blocks((long long)(l0.ny + 3) * l0.W), threads, 0, stream>>>(
      A, dirichlet, l0.nx, l0.ny, l0.W, w + l0.woff + kSlack, l0.plen, kMgOmega);
  for (int l = 0; l + 1 < L; ++l) {
    const MgLevel& f = lv[l];
    const MgLevel& c = lv[l + 1];
    mg_galerkin_kernel<<<blocks((long long)(c.ny + 3) * c.W), threads, 0, stream>>>(
        w + f.woff + kSlack, f.plen, f.nx, f.ny, f.W, w + c.woff + kSlack, c.plen, c.nx, c.ny, c.W, kMgOmega);
  }
  return cudaGetLastError();
}


}  // namespace ptg
