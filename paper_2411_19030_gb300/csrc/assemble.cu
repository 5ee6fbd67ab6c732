// assemble.cu -- a1 (SIMP coefficients and element weights) and a6 (sensitivity reduction).
#include <algorithm>
#include <cstdint>
#include "ptg_device.cuh"
#include "ptg_internal.h"

namespace ptg {

struct NodeOut {
  double* p[15];
};

__device__ __forceinline__ void assemble_error(DevStats* st, int code) {
  if (atomicCAS(&st->status, 0, code) == 0) {
    st->fail_kind = 1;
    st->fail_step = -1;
  }
}

// a1, Sec. 2.1 Eq. 2.5-2.6 and Sec. 2.2: one thread per element of the padded element grid
// (rows ey = -1..ny, columns ex = -1..W-2, row-major with stride W).  Interior elements get
// the SIMP coefficients and the (D, S, T) weights of C/dt + K and C/dtau + K; the padding
// gets zeros.  wEf / wEc each hold three arrays (D, S, T) spaced PE apart.
__global__ void assemble_elements(int nx, int ny, int W, int PE, double h, ptg_material m, double dt, double dtau,
                                  const double* __restrict__ rho, double* __restrict__ k_out,
                                  double* __restrict__ c_out, double* __restrict__ dk_out, double* __restrict__ dc_out,
                                  double* __restrict__ wEf, double* __restrict__ wEc, DevStats* st) {
  const int pe = blockIdx.x * blockDim.x + threadIdx.x;
  if (pe >= (ny + 2) * W) return;
  const int ey = pe / W - 1, ex = pe % W - 1;
  double wf[3] = {0.0, 0.0, 0.0}, wc[3] = {0.0, 0.0, 0.0};
  if (ey >= 0 && ey < ny && ex >= 0 && ex < nx) {
    const int e = ey * nx + ex;
    double r = rho[e];
    if (!(r >= 0.0 && r <= 1.0)) {        // also catches NaN
      assemble_error(st, PTG_EINVAL);
      r = 0.0;
    }
    const double kk = m.kmin + (m.k0 - m.kmin) * pow(r, m.pk);
    const double cc = m.cmin + (m.c0 - m.cmin) * pow(r, m.pc);
    const double dk = (m.k0 == m.kmin) ? 0.0 : m.pk * (m.k0 - m.kmin) * pow(r, m.pk - 1.0);
    const double dc = (m.c0 == m.cmin) ? 0.0 : m.pc * (m.c0 - m.cmin) * pow(r, m.pc - 1.0);
    k_out[e] = kk;
    c_out[e] = cc;
    dk_out[e] = dk;
    dc_out[e] = dc;
    const double mm = cc * h * h / 36.0;   // consistent mass: Me = (h^2/36)[4 2 1 2; ...]
    // K_e = (k/6)[4 -1 -2 -1; ...]: D = 4k/6, S = -k/6, T = -2k/6
    const double kd = 4.0 * kk / 6.0, ks = -kk / 6.0, kt = -2.0 * kk / 6.0;
    const double mf = mm / dt, mc = mm / dtau;
    wf[0] = kd + 4.0 * mf;
    wf[1] = ks + 2.0 * mf;
    wf[2] = kt + mf;
    wc[0] = kd + 4.0 * mc;
    wc[1] = ks + 2.0 * mc;
    wc[2] = kt + mc;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    wEf[i * PE + pe] = wf[i];
    wEc[i * PE + pe] = wc[i];
  }
}

// Per-node FP64 weights of C/dt + K, C/dtau + K and C: one thread per node of the padded node
// grid (rows iy = -1..ny+1, stride W).  For a node with elements a = (iy-1, ix-1),
// b = (iy-1, ix), c = (iy, ix-1), d = (iy, ix):
//   centre = (Da + Db) + (Dc + Dd),  east = Sb + Sd,  north = Sc + Sd,  north-east = Td,
//   north-west = Tc  (the other four couplings are those of the neighbours).
// node[0..4]: C/dt + K, node[5..9]: C/dtau + K, node[10..14]: C, each (C, E, N, NE, NW).
__global__ void assemble_nodes(int nx, int ny, int W, int PE, double h, const double* __restrict__ wEf,
                               const double* __restrict__ wEc, const double* __restrict__ c_elem,
                               NodeOut out) {
  const int pn = blockIdx.x * blockDim.x + threadIdx.x;
  if (pn >= (ny + 3) * W) return;
  const int iy = pn / W - 1, ix = pn % W - 1;
  double v[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) v[i] = 0.0;
  if (iy >= 0 && iy <= ny && ix >= 0 && ix <= nx) {
    // padded element index of element (ey, ex) is (ey + 1) * W + ex + 1
    const int ea = iy * W + ix, eb = iy * W + ix + 1, ec = (iy + 1) * W + ix, ed = (iy + 1) * W + ix + 1;
    const double* wsrc[2] = {wEf, wEc};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const double* D = wsrc[t];
      const double* S = wsrc[t] + PE;
      const double* T = wsrc[t] + 2 * PE;
      v[5 * t + 0] = (D[ea] + D[eb]) + (D[ec] + D[ed]);
      v[5 * t + 1] = S[eb] + S[ed];
      v[5 * t + 2] = S[ec] + S[ed];
      v[5 * t + 3] = T[ed];
      v[5 * t + 4] = T[ec];
    }
    const double h2 = h * h / 36.0;
    auto me = [&](int ey, int ex) { return (ey >= 0 && ey < ny && ex >= 0 && ex < nx) ? c_elem[ey * nx + ex] * h2 : 0.0; };
    const double ma = me(iy - 1, ix - 1), mb = me(iy - 1, ix), mc = me(iy, ix - 1), md = me(iy, ix);
    v[10] = 4.0 * ((ma + mb) + (mc + md));
    v[11] = 2.0 * (mb + md);
    v[12] = 2.0 * (mc + md);
    v[13] = md;
    v[14] = mc;
  }
#pragma unroll
  for (int i = 0; i < 15; ++i) out.p[i][pn] = v[i];
}

// Unit-time load vector f_i = sum_e q_e int N_i = sum over the elements around node i of
// q_e h^2 / 4 (Sec. 2.2, element-wise constant q); zero on Dirichlet nodes.
__global__ void load_kernel(int nx, int ny, double h, const double* __restrict__ q_elem,
                            const uint8_t* __restrict__ dirichlet, double* __restrict__ fload) {
  const int nn = nx + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn * (ny + 1)) return;
  const int iy = i / nn, ix = i % nn;
  double s = 0.0;
  for (int dy = -1; dy <= 0; ++dy)
    for (int dx = -1; dx <= 0; ++dx) {
      const int ey = iy + dy, ex = ix + dx;
      if (ey >= 0 && ey < ny && ex >= 0 && ex < nx) s += q_elem[ey * nx + ex];
    }
  fload[i] = dirichlet[i] ? 0.0 : s * h * h / 4.0;
}

cudaError_t launch_assemble(int nx, int ny, double h, const ptg_material& m, double dt, double dtau, const double* rho,
                            const double* q_elem, const uint8_t* dirichlet, const AssembleOut& out, DevStats* st,
                            cudaStream_t stream) {
  const int W = padded_width(nx);
  const int PEe = (ny + 2) * W + 2 * kSlack;        // spacing of the D, S, T element arrays
  const int ne_pad = (ny + 2) * W;
  assemble_elements<<<(ne_pad + 255) / 256, 256, 0, stream>>>(nx, ny, W, PEe, h, m, dt, dtau, rho, out.k, out.c, out.dk,
                                                             out.dc, out.wEf, out.wEc, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  NodeOut no;
  for (int i = 0; i < 15; ++i) no.p[i] = out.node[i];
  const int nn_pad = (ny + 3) * W;
  assemble_nodes<<<(nn_pad + 255) / 256, 256, 0, stream>>>(nx, ny, W, PEe, h, out.wEf, out.wEc, out.c, no);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int Nn = (nx + 1) * (ny + 1);
  load_kernel<<<(Nn + 255) / 256, 256, 0, stream>>>(nx, ny, h, q_elem, dirichlet, out.fload);
  return cudaGetLastError();
}

// a6, Eq. 4.7: per element e and time chunk, sum over j of
//   lambda_j,e^T ( dk_e Ke T_j,e + dc_e/dt Me (T_j - T_{j-1})_e )   (sens_element_sum).
// One thread per element; blockIdx.y selects a contiguous chunk of time steps.
__global__ void sens_kernel(int nx, int ny, double h, double dt, int has_dc, const double* __restrict__ dk,
                            const double* __restrict__ dc, const double* __restrict__ lam, int j0, int j1,
                            const double* __restrict__ T, int hist_j0, int steps_per_chunk,
                            double* __restrict__ partial) {
  const int Ne = nx * ny, nn = nx + 1, Nn = nn * (ny + 1);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ne) return;
  const int chunk = blockIdx.y;
  const int ja = j0 + chunk * steps_per_chunk;
  const int jb = min(j1, ja + steps_per_chunk - 1);
  const int ey = e / nx, ex = e % nx;
  const double dke = dk[e], dce = has_dc ? dc[e] / dt : 0.0;
  const double acc = ja <= jb ? sens_element_sum(ey * nn + ex, nn, Nn, h * h / 36.0, dke, dce, has_dc != 0, lam, j0,
                                                 T, hist_j0, ja, jb)
                              : 0.0;
  partial[(size_t)chunk * Ne + e] = acc;
}

// grad_e += -(1/Nt) sum over chunks (fixed order) of the partial sums.
__global__ void sens_reduce_kernel(int Ne, int nchunks, double inv_nt, const double* __restrict__ partial,
                                   double* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ne) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(size_t)c * Ne + e];
  grad[e] -= inv_nt * s;
}

// Sec. 7.1: Theta = Theta~^(1/p) and the factor Theta^(1-p)/p of the gradient (one thread;
// the factor goes to scratch so that Theta may alias Theta~), then grad = factor * grad~.
__global__ void modified_objective_scalar_kernel(double p, const double* __restrict__ Theta_mod, double* Theta,
                                                 double* __restrict__ scratch) {
  const double Tm = *Theta_mod;
  const double T = pow(Tm, 1.0 / p);
  scratch[0] = pow(T, 1.0 - p) / p;
  *Theta = T;
}

__global__ void modified_objective_grad_kernel(int Ne, const double* __restrict__ scratch, const double* grad_mod,
                                               double* grad) {
  const double f = scratch[0];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ne; e += gridDim.x * blockDim.x) grad[e] = f * grad_mod[e];
}

cudaError_t launch_objective_from_modified(int Ne, double p, const double* Theta_mod, const double* grad_mod,
                                          double* Theta, double* grad, double* scratch, cudaStream_t stream) {
  modified_objective_scalar_kernel<<<1, 1, 0, stream>>>(p, Theta_mod, Theta, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int blocks = (Ne + 255) / 256 < 1216 ? (Ne + 255) / 256 : 1216;
  modified_objective_grad_kernel<<<blocks, 256, 0, stream>>>(Ne, scratch, grad_mod, grad);
  return cudaGetLastError();
}

cudaError_t launch_sensitivities(int nx, int ny, int Nt, double h, double dt, int has_dc, const double* dk,
                                 const double* dc, const double* lam, int j0, int j1, const double* T, int hist_j0,
                                 double* partial, int nchunks, double* grad, cudaStream_t stream) {
  const int Ne = nx * ny;
  const int nsteps = j1 - j0 + 1;
  const int spc = (nsteps + nchunks - 1) / nchunks;
  const int used = (nsteps + spc - 1) / spc;
  dim3 grid((Ne + 255) / 256, used);
  sens_kernel<<<grid, 256, 0, stream>>>(nx, ny, h, dt, has_dc, dk, dc, lam, j0, j1, T, hist_j0, spc, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sens_reduce_kernel<<<(Ne + 255) / 256, 256, 0, stream>>>(Ne, used, 1.0 / Nt, partial, grad);
  return cudaGetLastError();
}

// G_adj = H + c S on rows [0, n_l) of a lambda block and [0, n_g) of a g block, with the
// adjoint source scale c of Eq. 4.6 (Theta^(1-p)/Ne, or p/Ne for the modified objective of
// Sec. 7.1) read from the device scalar Theta.
__global__ void adjoint_combine_kernel(long long n_l, long long n_g, const double* __restrict__ Theta, double p,
                                       int Ne, int modified, const double* __restrict__ H_l,
                                       const double* __restrict__ H_g, const double* __restrict__ S_l,
                                       const double* __restrict__ S_g, double* __restrict__ G_l,
                                       double* __restrict__ G_g) {
  const double c = (modified ? p : pow(*Theta, 1.0 - p)) / (double)Ne;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_l + n_g; i += stride) {
    if (i < n_l)
      G_l[i] = fma(c, S_l[i], H_l[i]);
    else
      G_g[i - n_l] = fma(c, S_g[i - n_l], H_g[i - n_l]);
  }
}

cudaError_t launch_adjoint_combine(long long n_l, long long n_g, const double* Theta, double p, int Ne, int modified,
                                   const double* H_l, const double* H_g, const double* S_l, const double* S_g,
                                   double* G_l, double* G_g, cudaStream_t stream) {
  const long long n = n_l + n_g;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4 * 152);
  adjoint_combine_kernel<<<blocks, 256, 0, stream>>>(n_l, n_g, Theta, p, Ne, modified, H_l, H_g, S_l, S_g, G_l, G_g);
  return cudaGetLastError();
}

// FP32 element weights and the inverse diagonal for the streamed fine propagators (see
// ptg_internal.h).  Node entry i of the padded layout (slack included) is row i / W - 1 after the
// kSlack leading entries.
__global__ void stream_weights_kernel(int PE, int PN, const double* __restrict__ wE, const double* __restrict__ C,
                                      const uint8_t* __restrict__ dirichlet, int nx, int ny, int W,
                                      float* __restrict__ w32, float* __restrict__ w32_inv,
                                      double* __restrict__ w64_inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * PE) w32[i] = (float)wE[i];
  if (i < PN) {
    const int k = i - kSlack;
    const int iy = k >= 0 ? k / W - 1 : -2, ix = k >= 0 ? k % W - 1 : -2;
    const bool unknown = iy >= 0 && iy <= ny && ix >= 0 && ix <= nx && dirichlet[iy * (nx + 1) + ix] == 0;
    const double inv = unknown ? 1.0 / C[i] : 0.0;
    w32_inv[i] = (float)inv;
    w64_inv[i] = inv;
  }
}

cudaError_t launch_stream_weights(int PE, int PN, const double* wE, const double* C_node, const uint8_t* dirichlet,
                                  int nx, int ny, int W, float* w32, float* w32_inv, double* w64_inv,
                                  cudaStream_t stream) {
  const int n = 3 * PE > PN ? 3 * PE : PN;
  stream_weights_kernel<<<(n + 255) / 256, 256, 0, stream>>>(PE, PN, wE, C_node, dirichlet, nx, ny, W, w32, w32_inv,
                                                             w64_inv);
  return cudaGetLastError();
}

cudaError_t launch_sens_reduce(int Ne, int nchunks, double inv_nt, const double* partial, double* grad,
                               cudaStream_t stream) {
  sens_reduce_kernel<<<(Ne + 255) / 256, 256, 0, stream>>>(Ne, nchunks, inv_nt, partial, grad);
  return cudaGetLastError();
}

}  // namespace ptg
