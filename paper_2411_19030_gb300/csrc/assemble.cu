// assemble.cu -- a1 (SIMP coefficients and element weights) and a6 (sensitivity reduction).
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
//   lambda_j,e^T ( dk_e Ke T_j,e + dc_e/dt Me (T_j - T_{j-1})_e ).
// One thread per element; blockIdx.y selects a contiguous chunk of time steps.  T_{j-1} is
// carried in registers from the previous step, so each step reads lambda_j and T_j once.
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
  const int g0 = ey * nn + ex;
  const double h2 = h * h / 36.0;
  const double dke = dk[e], dce = has_dc ? dc[e] / dt : 0.0;
  double acc = 0.0;
  if (ja <= jb) {
    const double* Tp = T + (size_t)(ja - 1 - hist_j0) * Nn;
    double psw = Tp[g0], pse = Tp[g0 + 1], pne = Tp[g0 + nn + 1], pnw = Tp[g0 + nn];
    for (int j = ja; j <= jb; ++j) {
      const double* Tj = T + (size_t)(j - hist_j0) * Nn;
      const double* Lj = lam + (size_t)(j - j0) * Nn;
      const double tsw = Tj[g0], tse = Tj[g0 + 1], tne = Tj[g0 + nn + 1], tnw = Tj[g0 + nn];
      const double lsw = Lj[g0], lse = Lj[g0 + 1], lne = Lj[g0 + nn + 1], lnw = Lj[g0 + nn];
      const double ksw = 4.0 * tsw - tse - 2.0 * tne - tnw;
      const double kse = -tsw + 4.0 * tse - tne - 2.0 * tnw;
      const double kne = -2.0 * tsw - tse + 4.0 * tne - tnw;
      const double knw = -tsw - 2.0 * tse - tne + 4.0 * tnw;
      double term = dke * (lsw * ksw + lse * kse + lne * kne + lnw * knw) / 6.0;
      if (has_dc) {
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

}  // namespace ptg
