// stepper.cuh -- the cluster time stepper: every backward-Euler solve of the pass.
//
// One thread-block cluster owns one independent time-stepping system (one Parareal slice,
// one coarse step, or the sequential correction sweep).  Its CTAs split the node rows into
// slabs held on chip (ptg_device.cuh); each thread owns NG aligned groups of 4 consecutive
// nodes of a row.  Each solve of (C/dt + K) x = b (Eq. 2.7 / 4.4) is a Jacobi-preconditioned
// CG in precision Real inside an FP64 residual loop:
//     r = b - A x            (FP64, per-node FP64 weights: 9 FMAs per node)
//     while ||r|| > rtol ||b||:   CG on A d = r / ||r||  (Real),  x += ||r|| d,  r = b - A x
// With Real = double the first CG already meets the tolerance (plain FP64 PCG on the same
// per-node weights); with Real = float the CG uses FP32 element weights held in shared memory
// and this is iterative refinement with FP64 residuals.  CG carries q = A p by the recurrence
// q_{k+1} = A z_{k+1} + beta q_k, so each iteration has two cluster reductions and the halo
// exchange of z, the only stencil operand, rides on the second one.
//
// Task kinds (StepParams::kind), one task per cluster:
//   FINE_PRI    Alg. 1 repeated M times from u_s (or chained over slices), history written.
//   COARSE_PRI  Alg. 1 with dt -> dtau, Nt -> Ntau, one step ending at t_{M(s+1)}.
//   CORRECT_PRI Eq. 4.9 forward sweep: u_{s+1} = G(u_s) + F[s] - G_old[s].
//   FINE_ADJ    Alg. 2 repeated M times from v_{s+1} (or chained), g accumulated.
//   COARSE_ADJ  Alg. 2 with dt -> dtau, Nt -> Ntau, n+1 -> n+M, n-1 -> n-M.
//   CORRECT_ADJ Eq. 4.14 reverse sweep: v_s = G(v_{s+1}) + F[s] - G_old[s], v_Ntau = 0.
#pragma once
#include <type_traits>
#include "comm.cuh"
#include "ptg_device.cuh"
#include "ptg_internal.h"

namespace ptg {

template <class Real, int NG, class Comm>
struct Stepper {
  static constexpr bool kMixed = std::is_same<Real, float>::value;

  const StepParams& P;
  Comm& comm;
  Slab sb;
  // shared memory (each pointer at the first non-slack entry)
  double* x64;      // FP64 state, rows -1..R
  double* b64;      // FP64 right-hand side, rows 0..R-1
  Real* zbuf;       // CG stencil operand, rows -1..R
  Real* dinv;       // Jacobi inverse diagonal, rows 0..R-1 (0 on Dirichlet and pad nodes)
  float* wd = nullptr;  // FP32 element weights (D, S, T), element rows r0-1..r0+R-1 (FP32 CG, V-cycle)
  float* ws = nullptr;
  float* wt = nullptr;
  // per-thread groups: loc0[k] = offset of the group's first node in the halo buffers, -1 if none
  int loc0[NG];
  unsigned fmask = 0;   // bit 4k+j: node j of group k is an unknown (free, not a pad)
  NodeWeights A;    // per-node FP64 weights of the current operator
  double step_dt = 0.0;
  double inv_dt = 0.0;
  int gshift = 0;   // offset from a halo-buffer node to the same node of the global padded arrays
  double* ax64;     // A x64 from the last residual evaluation, rows 0..R-1 (reused by the next step;
                    // null when the plan leaves it out, P.keep_ax == 0)
  bool ax_valid = false;
  // two-level preconditioner of the coarse-step solves: see coarse_restrict_push
  bool tl = false;
  bool tl_loaded = false;
  int aj0 = 0, naj = 0;      // this CTA's aggregate rows [aj0, aj0 + naj)
  float* tl_ainv = nullptr;  // rows of Ainv for the CTA's aggregates, [naj * naxp][ncp]
  float* tl_slot = nullptr;  // restricted partials of every rank, [cs][ncp]
  float* tl_qc = nullptr;    // restricted vector summed over the covering ranks, [ncp]
  float* tl_ec = nullptr;    // coarse correction Ac^-1 P^T r on the CTA's aggregates, [naj * naxp]
  float* tl_gs = nullptr;    // group sums of the vector being restricted, [R * G]
  int* tl_gagg = nullptr;    // local aggregate (row-major in [naj][nax]) of every group, [R * G]
  int* tl_cov = nullptr;     // first / last rank covering each aggregate row, [nay][2]
  // V(1,1) two-grid cycle (P.tl_vc), see vcycle; aj0 / naj then cover the halo rows too
  bool vc = false;
  int ajo0 = 0, najo = 0;    // aggregate rows of the owned rows (the restriction's partials)
  Real* vqh = nullptr;       // q on the halo rows -1 and R (the neighbours' edge rows), [2][W]
  Real* vrh = nullptr;       // r on the halo rows -1 and R, [2][W]
  float* vy = nullptr;       // y = S r, then u = y + P ec, rows -1..R
  float* vsd = nullptr;      // S = omega D^-1, rows -1..R (0 off the unknowns)
  float* ve0 = nullptr;      // slab-local smoothing (P.tl_nu >= 2): ping-pong iterates, rows -1..R,
  float* ve1 = nullptr;      // halo rows kept at zero
  // three-level cycle (P.tl_l3, see vcycle3): the 2h rows [J0, J0 + R1) of this CTA (R1b: those
  // of the CTA below), padded 2h row width W1, stride own1s of the owned-row 2h arrays
  bool l3 = false;
  int J0 = 0, R1 = 0, R1b = 0, W1 = 0, own1s = 0;
  float* vw = nullptr;       // fine residual w0 = r - A e0, rows -1..R
  float* b1x = nullptr;      // 2h rows -1..R1: e1 = S1 r1 (halo rows from the neighbours)
  float* b1u = nullptr;      //                 u1 = e1 + P2 ec (owned and halo rows, computed here)
  float* b1z = nullptr;      //                 z1 = u1 + S1 (r1 - A1 u1) (halo rows from the neighbours)
  float* s1a = nullptr;      //                 slab-local smoothing iterates (halo rows kept at zero)
  float* s1b = nullptr;
  float* r1 = nullptr;       // owned 2h rows: restricted residual r1 = P1^T w0 (then r1 - A1 u1)
  float* a1w = nullptr;      // [9][own1s] A1 weights of the owned 2h nodes, k = (dJ + 1) * 3 + (dI + 1)
  float* s1d = nullptr;      // omega / diag(A1) of the owned 2h nodes
  float* l3_items = nullptr; // partial sums of the 2h residual per aggregate of the owned rows

  __device__ Stepper(const StepParams& P_, Comm& comm_, unsigned char* dyn) : P(P_), comm(comm_) {
    sb.nx = P.nx;
    sb.ny = P.ny;
    sb.cs = P.cs;
    sb.rank = comm.rank();
    slab_rows(P.ny + 1, P.cs, sb.rank, sb.r0, sb.R);
    sb.W = P.W;
    sb.G = P.W / kGroup;
    sb.ngroups = sb.R * sb.G;
    const int W = sb.W;
    const int halo = (P.rmax + 2) * W + 2 * kSlack;
    const int own = P.rmax * W + 2 * kSlack;
    const int elems = (P.rmax + 1) * W + 2 * kSlack;
    unsigned char* p = dyn;
    double* x64b = reinterpret_cast<double*>(p);  p += sizeof(double) * halo;
    double* b64b = reinterpret_cast<double*>(p);  p += sizeof(double) * own;
    double* axb = reinterpret_cast<double*>(p);   p += P.keep_ax ? sizeof(double) * own : 0;
    Real* zb = reinterpret_cast<Real*>(p);        p += sizeof(Real) * halo;
    Real* db = reinterpret_cast<Real*>(p);        p += sizeof(Real) * own;
    float* eb = reinterpret_cast<float*>(p);
    for (int i = threadIdx.x; i < halo; i += blockDim.x) {
      x64b[i] = 0.0;
      zb[i] = Real(0);
    }
    for (int i = threadIdx.x; i < own; i += blockDim.x) {
      b64b[i] = 0.0;
      if (P.keep_ax) axb[i] = 0.0;
      db[i] = Real(0);
    }
    if constexpr (kMixed) {
      for (int i = threadIdx.x; i < 3 * elems; i += blockDim.x) eb[i] = 0.f;
    }
    {
      if (P.tl_naj > 0) {
        const int naxp = coarse_row_stride(P.nax), ncp = naxp * P.nay;
        const int groups = P.rmax * (W / kGroup);
        // after the element weights (FP32 CG only); 16-byte aligned: every earlier array is a
        // multiple of 4 words
        float* t = eb + (kMixed ? 3 * elems : 0);
        tl_ainv = t;  t += P.tl_naj * naxp * ncp;
        tl_slot = t;  t += P.wide ? 0 : P.cs * ncp;   // grid-wide: the partials are in global memory
        tl_qc = t;    t += ncp;
        tl_ec = t;    t += P.tl_naj * naxp;
        if (P.tl_vc) {
          // every array a multiple of 4 words, so each starts 16-byte aligned
          constexpr int rw = (int)(sizeof(Real) / 4);
          float* v0 = t;
          vqh = reinterpret_cast<Real*>(t);  t += 2 * W * rw;
          vrh = reinterpret_cast<Real*>(t);  t += 2 * W * rw;
          vy = t + kSlack;   t += halo;
          vsd = t + kSlack;  t += halo;
          if (P.tl_nu >= 2) {
            ve0 = t + kSlack;  t += halo;
            ve1 = t + kSlack;  t += halo;
          }
          if constexpr (!kMixed) {
            wd = t + kSlack;
            ws = t + elems + kSlack;
            wt = t + 2 * elems + kSlack;
            t += 3 * elems;
          }
          for (float* z = v0 + threadIdx.x; z < t; z += blockDim.x) *z = 0.f;
        }
        if (P.tl_l3) {
          float* l0 = t;
          vw = t + kSlack;  t += halo;
          W1 = P.l3_W1;
          const int halo1 = (P.l3_r1max + 2) * W1 + 2 * kSlack;
          own1s = P.l3_r1max * W1 + 2 * kSlack;
          b1x = t + kSlack;  t += halo1;
          b1u = t + kSlack;  t += halo1;
          b1z = t + kSlack;  t += halo1;
          s1a = t + kSlack;  t += halo1;
          s1b = t + kSlack;  t += halo1;
          r1 = t + kSlack - W1;  t += own1s;     // r1[lr1 * W1 + I + 1]: owned rows from lr1 = 0
          a1w = t + kSlack - W1; t += 9 * own1s;
          s1d = t + kSlack - W1; t += own1s;
          l3_items = t;      t += P.tl_naj * naxp;
          for (float* z = l0 + threadIdx.x; z < t; z += blockDim.x) *z = 0.f;
          tl_cov = reinterpret_cast<int*>(t);
          l1_rows_of_slab(sb.r0, sb.R, J0, R1);
          if (sb.rank > 0) {
            int r0b, Rb, J0b;
            slab_rows(P.ny + 1, P.cs, sb.rank - 1, r0b, Rb);
            l1_rows_of_slab(r0b, Rb, J0b, R1b);
          }
          const int ny1 = P.l3_ny1;
          aj0 = l3_agg(J0 > 0 ? J0 - 1 : 0, P.cm, P.nay);
          naj = l3_agg(J0 + R1 <= ny1 ? J0 + R1 : ny1, P.cm, P.nay) - aj0 + 1;
          ajo0 = l3_agg(J0, P.cm, P.nay);
          najo = l3_agg(J0 + R1 - 1, P.cm, P.nay) - ajo0 + 1;
          for (int J = threadIdx.x; J < P.nay; J += blockDim.x) {
            int lo = -1, hi = -1;
            for (int q = 0; q < P.cs; ++q) {
              int r0q, Rq, J0q, R1q;
              slab_rows(P.ny + 1, P.cs, q, r0q, Rq);
              l1_rows_of_slab(r0q, Rq, J0q, R1q);
              if (R1q > 0 && J >= l3_agg(J0q, P.cm, P.nay) && J <= l3_agg(J0q + R1q - 1, P.cm, P.nay)) {
                if (lo < 0) lo = q;
                hi = q;
              }
            }
            tl_cov[2 * J] = lo;
            tl_cov[2 * J + 1] = hi;
          }
        } else {
        tl_gs = t;    t += groups;
        tl_gagg = reinterpret_cast<int*>(t);  t += P.tl_vc ? groups + 2 * (W / kGroup) : groups;
        tl_cov = reinterpret_cast<int*>(t);
        int ajhi, ajo1;
        coarse_rows_of_slab(sb.r0, sb.R, P.cm, P.nay, ajo0, ajo1);
        najo = ajo1 - ajo0 + 1;
        if (P.tl_vc) {
          coarse_rows_of_halo_slab(sb.r0, sb.R, P.ny, P.cm, P.nay, aj0, ajhi);
          // rows -1..R: group gi of row gi / G - 1 (no aggregate outside the grid)
          for (int gi = threadIdx.x; gi < (sb.R + 2) * sb.G; gi += blockDim.x) {
            const int lr = gi / sb.G - 1, g = gi - (lr + 1) * sb.G, row = sb.r0 + lr;
            tl_gagg[gi] = (row < 0 || row > P.ny)
                              ? -1
                              : (coarse_agg_y(row, P.cm, P.nay) - aj0) * naxp + coarse_agg_x(g, P.cm, P.nax);
          }
        } else {
          aj0 = ajo0;
          ajhi = ajo1;
          for (int gi = threadIdx.x; gi < sb.ngroups; gi += blockDim.x) {
            const int lr = gi / sb.G, g = gi - lr * sb.G;
            tl_gagg[gi] = (coarse_agg_y(sb.r0 + lr, P.cm, P.nay) - aj0) * naxp + coarse_agg_x(g, P.cm, P.nax);
          }
        }
        naj = ajhi - aj0 + 1;
        for (int J = threadIdx.x; J < P.nay; J += blockDim.x) {
          int lo = -1, hi = -1;
          for (int q = 0; q < P.cs; ++q) {
            int r0q, Rq, a, bq;
            slab_rows(P.ny + 1, P.cs, q, r0q, Rq);
            coarse_rows_of_slab(r0q, Rq, P.cm, P.nay, a, bq);
            if (J >= a && J <= bq) {
              if (lo < 0) lo = q;
              hi = q;
            }
          }
          tl_cov[2 * J] = lo;
          tl_cov[2 * J + 1] = hi;
        }
        }
      }
    }
    x64 = x64b + kSlack;
    b64 = b64b + kSlack - W;   // b64[loc] for loc in own rows (loc >= W)
    ax64 = P.keep_ax ? axb + kSlack - W : nullptr;
    zbuf = zb + kSlack;
    dinv = db + kSlack - W;    // dinv[loc] likewise
    if constexpr (kMixed) {
      wd = eb + kSlack;
      ws = eb + elems + kSlack;
      wt = eb + 2 * elems + kSlack;
    }
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int gi = threadIdx.x + k * blockDim.x;
      loc0[k] = -1;
      if (gi < sb.ngroups) {
        const int lr = gi / sb.G, g = gi - lr * sb.G;
        loc0[k] = (lr + 1) * W + kGroup * g;
      }
    }
    gshift = sb.r0 * W;
  }

  // global node index of node j of a group, or -1 for a pad node
  __device__ __forceinline__ int gnode(int l0, int j) const {
    const int lr = l0 / sb.W - 1;
    const int ix = (l0 - (lr + 1) * sb.W) + j - 1;
    return (ix >= 0 && ix <= P.nx) ? (sb.r0 + lr) * (P.nx + 1) + ix : -1;
  }

  template <class T, int NV, int NX = 0, class Post = NoPost>
  __device__ __forceinline__ void allreduce(T (&v)[NV + NX], Post post = Post()) {
    comm.template allreduce<T, NV, NX, Post>(v, sb.cs, post);
  }

  // Select the operator C/dt + K (fine) or C/dtau + K (coarse): per-node FP64 weights for the
  // residual (and the FP64 CG), FP32 element weights in shared memory for the FP32 CG, and
  // the Jacobi inverse diagonal (zero on Dirichlet and pad nodes).
  __device__ void set_operator(bool coarse) {
    A = coarse ? P.A_coarse : P.A_fine;
    step_dt = coarse ? P.dtau : P.dt;
    inv_dt = 1.0 / step_dt;
    ax_valid = false;
    tl = coarse && P.tl_naj > 0 && P.Ainv != nullptr;
    vc = tl && P.tl_vc;
    l3 = vc && P.tl_l3;
    if (tl && !tl_loaded) {        // rows of the aggregate rows aj0 .. aj0+naj-1 of Ainv, 16-byte copies
      const int naxp = coarse_row_stride(P.nax), ncp = naxp * P.nay;
      const int n4 = naj * naxp * ncp / 4;
      const float4* src = reinterpret_cast<const float4*>(P.Ainv + (size_t)aj0 * naxp * ncp);
      float4* dst = reinterpret_cast<float4*>(tl_ainv);
      for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = src[i];
      tl_loaded = true;
    }
    const int W = sb.W;
    __syncthreads();
    if (kMixed || vc) {
      const double* wE = coarse ? P.wE_coarse : P.wE_fine;
      const int PE = (P.ny + 2) * W + 2 * kSlack;      // one element array incl. slack
      const int n = (sb.R + 1) * W;
      const double* src = wE + sb.r0 * W;               // padded element row r0 = element row r0 - 1
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        wd[i] = (float)src[i];
        ws[i] = (float)src[PE + i];
        wt[i] = (float)src[2 * PE + i];
      }
    }
    fmask = 0;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const int g = gnode(l0, j);
        Real v = Real(0);
        if (g >= 0 && P.dirichlet[g] == 0) {
          v = Real(1) / (Real)A.C[l0 + gshift + j];
          fmask |= 1u << (kGroup * k + j);
        }
        dinv[l0 + j] = v;
      }
    }
    if (l3) {
      // the 2h stencil and omega / diag of the owned 2h nodes (FP32)
      const int n1 = P.l3_nx1 + 1, nn1 = n1 * (P.l3_ny1 + 1);
      for (int t = threadIdx.x; t < R1 * n1; t += blockDim.x) {
        const int lr1 = t / n1, I = t - lr1 * n1, o = lr1 * W1 + I + 1;
        const int g = (J0 + lr1) * n1 + I;
#pragma unroll
        for (int k = 0; k < 9; ++k) a1w[k * own1s + o] = (float)P.A1[(size_t)k * nn1 + g];
        s1d[o] = (float)((double)P.tl_omega / P.A1[(size_t)4 * nn1 + g]);
      }
    }
    if (vc) {
      // S = omega / diag on rows -1..R; 0 on Dirichlet, pad and out-of-grid nodes
      for (int i = threadIdx.x; i < (sb.R + 2) * W; i += blockDim.x) {
        const int lr = i / W - 1, ix = i - (lr + 1) * W - 1, row = sb.r0 + lr;
        float v = 0.f;
        if (row >= 0 && row <= P.ny && ix >= 0 && ix <= P.nx && P.dirichlet[row * (P.nx + 1) + ix] == 0)
          v = (float)((double)P.tl_omega / A.C[i + gshift]);
        vsd[i] = v;
      }
    }
    __syncthreads();
  }

  __device__ __forceinline__ bool unknown(int k, int j) const { return (fmask >> (kGroup * k + j)) & 1u; }

  // Load a node vector from global memory into x64: owned rows and both halo rows
  // (Dirichlet nodes forced to zero).  Ends with __syncthreads.
  __device__ void load_x64(const double* __restrict__ src) {
    ax_valid = false;
    __syncthreads();
    const int nn = P.nx + 1;
    const int rows = sb.R + 2;
    for (int t = threadIdx.x; t < rows * nn; t += blockDim.x) {
      const int row = t / nn, ix = t - row * nn;
      const int g = sb.r0 - 1 + row;
      if (g >= 0 && g <= P.ny) {
        const int gi = g * nn + ix;
        x64[row * sb.W + ix + 1] = P.dirichlet[gi] ? 0.0 : src[gi];
      }
    }
    __syncthreads();
  }

  __device__ void zero_x64() {
    ax_valid = false;
    __syncthreads();
    for (int i = threadIdx.x; i < (P.rmax + 2) * sb.W; i += blockDim.x) x64[i] = 0.0;
    __syncthreads();
  }

  // Correction sweeps: the start of a step is G_old plus the polynomial extrapolation of the
  // sweep's increments G(x^new) - G(x^old) through the last m of them (1 <= m <= 3):
  //   x64 = G + inc,  inc = d0 (m = 1), 2 d0 - d1 (m = 2), 3 (d0 - d1) + d2 (m = 3),
  // with d_i = X_i - Fm[i] the increment of the i-th step before, which by the correction itself
  // is the corrected state X_i that step produced minus the fine result Fm[i] of its slice; X_0
  // is x64 (the state the step propagates), X_1, X_2 node vectors of earlier corrected states.
  // On the owned and both halo rows: every CTA evaluates the same expression on the same
  // operands (x64's halos are exact), so the halos stay exact.  Ends with __syncthreads.
  __device__ void load_x64_increment(const double* __restrict__ G, int m, const double* const* Fm,
                                     const double* const* X) {
    ax_valid = false;
    __syncthreads();
    const int nn = P.nx + 1;
    const int rows = sb.R + 2;
    for (int t = threadIdx.x; t < rows * nn; t += blockDim.x) {
      const int row = t / nn, ix = t - row * nn;
      const int g = sb.r0 - 1 + row;
      if (g >= 0 && g <= P.ny) {
        const int gi = g * nn + ix;
        double& x = x64[row * sb.W + ix + 1];
        const double d0 = x - Fm[0][gi];
        double inc = d0;
        if (m == 2) inc = fma(2.0, d0, -(X[1][gi] - Fm[1][gi]));
        if (m == 3) inc = fma(3.0, d0 - (X[1][gi] - Fm[1][gi]), X[2][gi] - Fm[2][gi]);
        x = P.dirichlet[gi] ? 0.0 : G[gi] + inc;
      }
    }
    __syncthreads();
  }

  // Polynomial extrapolation in time of the initial guess: with x64 = x_1 (the last state) and
  // X[i-2] = x_i, i = 2..n, the states of the n previous equidistant steps (global node vectors),
  // x64 becomes the value at the next step of the polynomial of degree n-1 through them,
  //   n = 2: 2 x_1 - x_2;  n = 3: 3 x_1 - 3 x_2 + x_3;  n = 4: 4 x_1 - 6 x_2 + 4 x_3 - x_4,
  // on the owned rows and both halo rows.  x64's halo rows hold the neighbours' x_1, so every
  // CTA evaluates the same expression on the same operands and the halos stay exact: no
  // exchange is needed.  If wr is given, x_1 is first saved there on the owned rows (the
  // slice's ring of states; wr is none of the X).  Ends with __syncthreads.
  __device__ void extrapolate_x64(int n, const double* const* X, double* __restrict__ wr) {
    ax_valid = false;
    __syncthreads();
    const int nn = P.nx + 1;
    const int rows = sb.R + 2;
    for (int t = threadIdx.x; t < rows * nn; t += blockDim.x) {
      const int row = t / nn, ix = t - row * nn;
      const int g = sb.r0 - 1 + row;
      if (g >= 0 && g <= P.ny) {
        const int gi = g * nn + ix;
        double& x = x64[row * sb.W + ix + 1];
        const double x1 = x;
        if (wr && row >= 1 && row <= sb.R) wr[gi] = x1;
        if (n < 2) continue;
        double v;
        if (n == 2) {
          v = fma(2.0, x1, -X[0][gi]);
        } else if (n == 3) {
          v = fma(3.0, x1 - X[0][gi], X[1][gi]);
        } else {
          v = fma(4.0, x1 + X[1][gi], -fma(6.0, X[0][gi], X[2][gi]));
        }
        x = P.dirichlet[gi] ? 0.0 : v;
      }
    }
    __syncthreads();
  }

  // Store the owned nodes of x64 to a global node vector.
  __device__ void store_x64(double* __restrict__ dst) const {
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const int g = gnode(l0, j);
        if (g >= 0) dst[g] = x64[l0 + j];
      }
    }
  }

  // Refresh every CTA's halo rows of a buffer from the neighbours' owned rows.
  template <class T>
  __device__ void exchange(T* buf) {
    __syncthreads();
    comm.push_halos(buf, sb);
    comm.sync();
  }
  __device__ void exchange_x64() { exchange(x64); }

  // b64 = (C/dt) x64 + src, with src(global node) supplied per owned free node.
  template <class Src>
  __device__ void build_rhs(Src src) {
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      double y[4];
      stencil_node64<double>(x64, l0, P.mass, l0 + gshift, sb.W, y);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const bool free_node = dinv[l0 + j] != Real(0);
        b64[l0 + j] = free_node ? fma(y[j], inv_dt, src(gnode(l0, j))) : 0.0;
      }
    }
  }

  // r64 = b - A x64 on the owned groups (0 off the unknowns); returns the local sum of r^2.
  __device__ __forceinline__ double residual(double (&r64)[NG][4]) const {
    double rr = 0.0;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) r64[k][j] = 0.0;
      if (l0 < 0) continue;
      double y[4];
      stencil_node64<double>(x64, l0, A, l0 + gshift, sb.W, y);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        if (ax64) ax64[l0 + j] = y[j];
        if (unknown(k, j)) {
          r64[k][j] = b64[l0 + j] - y[j];
          rr = fma(r64[k][j], r64[k][j], rr);
        }
      }
    }
    return rr;
  }

  // r64 = b - (A x64 saved by the last residual evaluation); valid while x64 is unchanged.
  __device__ __forceinline__ double residual_saved(double (&r64)[NG][4]) const {
    double rr = 0.0;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) r64[k][j] = 0.0;
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        if (unknown(k, j)) {
          r64[k][j] = b64[l0 + j] - ax64[l0 + j];
          rr = fma(r64[k][j], r64[k][j], rr);
        }
      }
    }
    return rr;
  }

  __device__ __forceinline__ void apply_A(const Real* z, int l0, Real (&w)[4]) const {
    if constexpr (kMixed) {
      stencil_elem32(z, wd, ws, wt, l0, sb.W, w);
    } else {
      double y[4];
      stencil_node64<double>(z, l0, A, l0 + gshift, sb.W, y);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[j] = y[j];
    }
  }

  // Two-level preconditioner M^-1 = D^-1 + P Ac^-1 P^T of the coarse-step solves (CG in either
  // precision; the coarse part is applied in FP32, the FP64 residual loop around the CG fixes
  // the accuracy); P is piecewise constant on aggregates of m x m nodes aligned to the 4-node groups, so the
  // restriction P^T v is a sum of group sums and the prolongation adds one value per group.
  // Every CTA sends its partial sums for the aggregates its slab touches to every CTA of the
  // cluster (16-byte stores of 4 aggregates); the next cluster barrier (the one of the
  // following all-reduce) makes them visible.  coarse_gather then adds, chunk by chunk, the
  // partials of the covering ranks in rank order and multiplies by the CTA's rows of Ac^-1.
  // In the CG loop the coarse correction follows r by the same recurrence as r,
  // ec -= alpha Ac^-1 P^T q, so restricting q needs no cluster barrier of its own.
  template <class T>
  __device__ void coarse_restrict_push(const T (&v)[NG][4]) {
    const int G = sb.G, m4 = P.cm / 4, nax = P.nax, naxp = coarse_row_stride(nax), ncp = naxp * P.nay;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      if (loc0[k] < 0) continue;
      tl_gs[threadIdx.x + k * blockDim.x] = (float)((v[k][0] + v[k][1]) + (v[k][2] + v[k][3]));
    }
    __syncthreads();
    // 4 lanes per local aggregate (16 lanes per chunk of 4 aggregates), each summing every
    // 4th node row; padding aggregates (ax >= nax) sum to 0
    const int items = najo * naxp, padded = ((4 * items + 31) / 32) * 32;
    const int rlast = sb.r0 + sb.R - 1;
    const int lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < padded; t += blockDim.x) {
      const int item = t >> 2, part = t & 3;
      const int ajl = item / naxp, ax = item - ajl * naxp;
      const int ay = ajo0 + ajl;
      float acc = 0.f;
      if (item < items && ax < nax) {
        const int y0 = max(ay * P.cm, sb.r0), y1 = min(ay == P.nay - 1 ? P.ny : ay * P.cm + P.cm - 1, rlast);
        const int g0 = ax * m4, g1 = ax == nax - 1 ? G - 1 : g0 + m4 - 1;
        for (int iy = y0 + part; iy <= y1; iy += 4) {
          const float* row = tl_gs + (iy - sb.r0) * G;
          for (int g = g0; g <= g1; ++g) acc += row[g];
        }
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      // the 16 lanes of a chunk: lane (c, p) holds aggregate c's sum; collect all four
      const int base = lane & 16;
      float4 chunk;
      chunk.x = __shfl_sync(0xffffffffu, acc, base + 0);
      chunk.y = __shfl_sync(0xffffffffu, acc, base + 4);
      chunk.z = __shfl_sync(0xffffffffu, acc, base + 8);
      chunk.w = __shfl_sync(0xffffffffu, acc, base + 12);
      const int item0 = (t & ~15) >> 2;              // first aggregate of the chunk
      if (item0 < items) {
        const int ajl0 = item0 / naxp, ax0 = item0 - ajl0 * naxp;
        const int dst = sb.rank * ncp + (ajo0 + ajl0) * naxp + ax0;
        comm.publish_tl(tl_slot, dst, chunk, lane & 15, sb.cs);
      }
    }
  }

  // After the cluster barrier that follows coarse_restrict_push: qc = sum over the covering
  // ranks of the partials (in rank order), then ec = Ac^-1 qc (first == true) or
  // ec -= alpha Ac^-1 qc on the CTA's aggregate rows (8 lanes per row of Ac^-1, 16-byte loads).
  __device__ void coarse_gather(bool first, float alpha) {
    const int naxp = coarse_row_stride(P.nax), ncp = naxp * P.nay;
    const float* slots = comm.tl_slots(tl_slot);
    for (int L4 = threadIdx.x; L4 < ncp / 4; L4 += blockDim.x) {
      const int J = (4 * L4) / naxp;            // a 16-byte chunk lies in one aggregate row
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int q = tl_cov[2 * J]; q <= tl_cov[2 * J + 1]; ++q) {
        const float4 u = comm.tl_load4(slots, q * ncp + 4 * L4);
        acc.x += u.x; acc.y += u.y; acc.z += u.z; acc.w += u.w;
      }
      reinterpret_cast<float4*>(tl_qc)[L4] = acc;
    }
    __syncthreads();
    const int nrows = naj * naxp, n4 = ncp / 4;
    const int padded = ((8 * nrows + 31) / 32) * 32;
    const float4* q4 = reinterpret_cast<const float4*>(tl_qc);
    for (int t = threadIdx.x; t < padded; t += blockDim.x) {
      const int row = t >> 3, part = t & 7;
      float acc = 0.f;
      if (row < nrows) {
        const float4* a4 = reinterpret_cast<const float4*>(tl_ainv + (size_t)row * ncp);
        float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
#pragma unroll 4
        for (int L = part; L < n4; L += 8) {
          const float4 a = a4[L], r = q4[L];
          ax = fmaf(a.x, r.x, ax);
          ay = fmaf(a.y, r.y, ay);
          az = fmaf(a.z, r.z, az);
          aw = fmaf(a.w, r.w, aw);
        }
        acc = (ax + ay) + (az + aw);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      if (part == 0 && row < nrows) tl_ec[row] = first ? acc : fmaf(-alpha, acc, tl_ec[row]);
    }
    __syncthreads();
  }

  // z = D^-1 r + P ec on the owned nodes (0 off the unknowns), written to zbuf; returns the
  // local part of (r, z).
  __device__ Real prolong_precondition(const Real (&r)[NG][4]) {
    Real rz = Real(0);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      const Real e = (Real)tl_ec[tl_gagg[threadIdx.x + k * blockDim.x]];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const Real di = dinv[l0 + j];
        const Real z = unknown(k, j) ? fma(di, r[k][j], e) : Real(0);
        zbuf[l0 + j] = z;
        rz = fma(r[k][j], z, rz);
      }
    }
    return rz;
  }

  // The owned edge rows (0 and R-1) of a per-thread vector into the neighbours' two-row buffer
  // `edge` ([0]: the row below the slab, [1]: the row above), straight from registers;
  // visible after the next barrier.
  __device__ void put_edges(Real* edge, const Real (&v)[NG][4]) {
    comm.begin_edges();
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      const int lr = l0 / sb.W - 1;
      if (lr == 0 || lr == sb.R - 1) comm.put_edge(edge, lr, l0 - (lr + 1) * sb.W, v[k], sb);
    }
    comm.end_edges(edge, sb);
  }

  // offset in a rows -1..R buffer of entry i of the two halo rows ([0, W): row -1, [W, 2W): row R)
  __device__ __forceinline__ int halo_offset(int i) const { return i < sb.W ? i : (sb.R + 1) * sb.W + (i - sb.W); }

  // V(1,1) two-grid cycle z = M^-1 r in FP32 over the owned rows and the two halo rows:
  //   y = S r,  ec = Ac^-1 P^T (r - A y),  u = y + P ec (in place of y),  z = u + S (r - A u),
  // with the damped-Jacobi smoother S = omega D^-1 and A applied with the FP32 element weights,
  // so that I - M^-1 A = (I - S A)(I - P Ac^-1 P^T A)(I - S A) (symmetric).  The halo rows of r
  // (vrh) follow the owners' CG recurrence bit for bit, and every CTA computes ec for the
  // aggregate rows its halo rows touch from the same restricted vector, so y and u on a halo
  // row equal the owner's values: M^-1 is one operator across the CTAs.  One cluster barrier
  // (the restricted partials).  z goes to zbuf on the owned rows; returns the local (r, z).
  __device__ Real vcycle(const Real (&r)[NG][4]) {
    const int W = sb.W, G = sb.G;
    float rf[NG][4];   // r in FP32, converted once (FP64 conversions run on the FP64 pipe)
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) rf[k][j] = (float)r[k][j];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) vy[l0 + j] = vsd[l0 + j] * rf[k][j];
    }
    for (int i = threadIdx.x; i < 2 * W; i += blockDim.x) {
      const int l = halo_offset(i);
      vy[l] = vsd[l] * (float)vrh[i];
    }
    __syncthreads();
    float w[NG][4];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = 0.f;
      if (l0 < 0) continue;
      float t[4];
      stencil_elem32(vy, wd, ws, wt, l0, W, t);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = unknown(k, j) ? rf[k][j] - t[j] : 0.f;
    }
    coarse_restrict_push(w);
    comm.sync();
    coarse_gather(true, 0.f);
    for (int gi = threadIdx.x; gi < (sb.R + 2) * G; gi += blockDim.x) {
      const int a = tl_gagg[gi];
      const float e = a >= 0 ? tl_ec[a] : 0.f;
      const int l = (gi / G) * W + kGroup * (gi % G);   // row gi / G - 1, group gi % G
#pragma unroll
      for (int j = 0; j < kGroup; ++j) vy[l + j] = vsd[l + j] != 0.f ? vy[l + j] + e : 0.f;
    }
    __syncthreads();
    Real rz = Real(0);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      float t[4];
      stencil_elem32(vy, wd, ws, wt, l0, W, t);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const float z = unknown(k, j) ? fmaf(vsd[l0 + j], rf[k][j] - t[j], vy[l0 + j]) : 0.f;
        zbuf[l0 + j] = (Real)z;
        rz = fma(r[k][j], (Real)z, rz);
      }
    }
    return rz;
  }

  // Slab-local damped-Jacobi smoothing of A e = s: P.tl_nu steps from e = 0 over the owned rows
  // with the halo rows held at zero (the slab's diagonal block A_s of A), in FP32, the iterate
  // ping-ponging between two buffers; e returned in registers.  The result is a fixed polynomial
  // in D^-1 A_s times D^-1, a symmetric operator, so the cycle that uses it stays symmetric; it
  // needs no communication.
  __device__ void smooth_local(const float (&s)[NG][4], float (&e)[NG][4]) {
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) e[k][j] = l0 >= 0 ? vsd[l0 + j] * s[k][j] : 0.f;
    }
    for (int it = 1; it < P.tl_nu; ++it) {
      float* buf = (it & 1) ? ve0 : ve1;
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int l0 = loc0[k];
        if (l0 < 0) continue;
#pragma unroll
        for (int j = 0; j < kGroup; ++j) buf[l0 + j] = e[k][j];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int l0 = loc0[k];
        if (l0 < 0) continue;
        float t[4];
        stencil_elem32(buf, wd, ws, wt, l0, sb.W, t);
#pragma unroll
        for (int j = 0; j < kGroup; ++j) e[k][j] = fmaf(vsd[l0 + j], s[k][j] - t[j], e[k][j]);
      }
    }
  }

  // Two-grid cycle with the slab-local smoother S_s of smooth_local before and after the coarse
  // correction: e1 = S_s r;  ec = Ac^-1 P^T (r - A e1);  u = e1 + P ec;  z = u + S_s (r - A u),
  // so that I - M^-1 A = (I - S_s A)(I - P Ac^-1 P^T A)(I - S_s A).  e1's edge rows are
  // exchanged (a cluster barrier) before the residual; u on the halo rows is then the owner's
  // value (e1 from the owner, ec computed from the same restricted vector).  Two cluster
  // barriers.  z goes to zbuf on the owned rows; returns the local (r, z).
  __device__ Real vcycle_local(const Real (&r)[NG][4]) {
    const int W = sb.W, G = sb.G;
    float rf[NG][4], e[NG][4], w[NG][4];
#pragma unroll
    for (int k = 0; k < NG; ++k)
#pragma unroll
      for (int j = 0; j < kGroup; ++j) rf[k][j] = (float)r[k][j];
    smooth_local(rf, e);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) vy[l0 + j] = e[k][j];
    }
    exchange(vy);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = 0.f;
      if (l0 < 0) continue;
      float t[4];
      stencil_elem32(vy, wd, ws, wt, l0, W, t);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = unknown(k, j) ? rf[k][j] - t[j] : 0.f;
    }
    coarse_restrict_push(w);
    comm.sync();
    coarse_gather(true, 0.f);
    for (int gi = threadIdx.x; gi < (sb.R + 2) * G; gi += blockDim.x) {
      const int a = tl_gagg[gi];
      const float ea = a >= 0 ? tl_ec[a] : 0.f;
      const int l = (gi / G) * W + kGroup * (gi % G);   // row gi / G - 1, group gi % G
#pragma unroll
      for (int j = 0; j < kGroup; ++j) vy[l + j] = vsd[l + j] != 0.f ? vy[l + j] + ea : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      float t[4];
      stencil_elem32(vy, wd, ws, wt, l0, W, t);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = unknown(k, j) ? (float)r[k][j] - t[j] : 0.f;
    }
    smooth_local(w, e);
    Real rz = Real(0);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const float z = vy[l0 + j] + e[k][j];
        zbuf[l0 + j] = (Real)z;
        rz = fma(r[k][j], (Real)z, rz);
      }
    }
    return rz;
  }

  // ---------------------------------------------------------------- three-level cycle
  // 2h buffers: halo buffers (rows -1..R1) at (lr1 + 1) W1 + I + 1, owned-row arrays at lr1 W1 + I + 1
  __device__ __forceinline__ int h1(int lr1, int I) const { return (lr1 + 1) * W1 + I + 1; }
  __device__ __forceinline__ int o1(int lr1, int I) const { return lr1 * W1 + I + 1; }

  // (A1 x) at the owned 2h node (lr1, I) from a halo buffer x (zero outside the 2h grid)
  __device__ __forceinline__ float a1_apply(const float* __restrict__ x, int lr1, int I) const {
    const int c = h1(lr1, I), o = o1(lr1, I);
    float y = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) y = fmaf(a1w[k * own1s + o], x[c + (k / 3 - 1) * W1 + (k % 3 - 1)], y);
    return y;
  }

  // refresh the 2h halo rows of every CTA from the neighbours' owned rows
  __device__ void exchange_l1(float* buf) {
    __syncthreads();
    comm.push_halos_rows(buf, W1, R1, R1b, sb.rank, sb.cs);
    comm.sync();
  }

  // P.tl_nu damped-Jacobi steps of A1_s e = s from e = 0 on the owned 2h rows, with the 2h halo
  // rows held at zero (the diagonal block of A1 of this CTA's rows: a fixed polynomial in
  // S1 A1_s times S1, symmetric, no communication); e goes to the owned rows of `out`.
  __device__ void smooth_l1(const float* __restrict__ s, float* __restrict__ out) {
    const int n1 = P.l3_nx1 + 1, n = R1 * n1;
    float* cur = s1a;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int lr1 = t / n1, I = t - lr1 * n1;
      cur[h1(lr1, I)] = s1d[o1(lr1, I)] * s[o1(lr1, I)];
    }
    __syncthreads();
    for (int it = 1; it < P.tl_nu; ++it) {
      float* nxt = cur == s1a ? s1b : s1a;
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int lr1 = t / n1, I = t - lr1 * n1;
        nxt[h1(lr1, I)] = fmaf(s1d[o1(lr1, I)], s[o1(lr1, I)] - a1_apply(cur, lr1, I), cur[h1(lr1, I)]);
      }
      __syncthreads();
      cur = nxt;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int lr1 = t / n1, I = t - lr1 * n1;
      out[h1(lr1, I)] = cur[h1(lr1, I)];
    }
    __syncthreads();
  }

  // The 2h part of the three-level cycle, from the fine residual w0 in vw (halo rows exchanged):
  //   r1 = P1^T w0;  e1 = S1 r1;  ec = A2^-1 P2^T (r1 - A1 e1);  u1 = e1 + P2 ec;
  //   z1 = u1 + S1 (r1 - A1 u1) into b1z with its halo rows exchanged.
  __device__ __forceinline__ void l1_correct() {
    const int W = sb.W, n1 = P.l3_nx1 + 1, ny1 = P.l3_ny1;
    const int naxp = coarse_row_stride(P.nax), ncp = naxp * P.nay;
    // r1 = P1^T w0 on the owned 2h rows: fine rows 2J-1 .. 2J+1 lie in -1 .. R
    for (int t = threadIdx.x; t < R1 * n1; t += blockDim.x) {
      const int lr1 = t / n1, I = t - lr1 * n1;
      const int lr = 2 * (J0 + lr1) - sb.r0;
      const float* c = vw + (lr + 1) * W + 2 * I + 1;
      const float mid = fmaf(0.5f, c[-1] + c[1], c[0]);
      const float lo = fmaf(0.5f, c[-W - 1] + c[-W + 1], c[-W]);
      const float hi = fmaf(0.5f, c[W - 1] + c[W + 1], c[W]);
      r1[o1(lr1, I)] = fmaf(0.5f, lo + hi, mid);
    }
    __syncthreads();
    // 2h pre-smoothing e1 = S1 r1, exchanged
    smooth_l1(r1, b1x);
    exchange_l1(b1x);
    // 2h residual r1 - A1 e1 (in s1a's owned rows), summed per aggregate of the owned rows and
    // published to every CTA (16-byte chunks of 4 aggregates)
    for (int t = threadIdx.x; t < R1 * n1; t += blockDim.x) {
      const int lr1 = t / n1, I = t - lr1 * n1;
      s1a[h1(lr1, I)] = r1[o1(lr1, I)] - a1_apply(b1x, lr1, I);
    }
    __syncthreads();
    const int items = najo * naxp;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int ay = ajo0 + it / naxp, ax = it % naxp;
      float acc = 0.f;
      if (ax < P.nax) {
        const int ya = max(ay * P.cm, J0), yb = min(ay == P.nay - 1 ? ny1 : ay * P.cm + P.cm - 1, J0 + R1 - 1);
        const int xa = ax * P.cm, xb = ax == P.nax - 1 ? n1 - 1 : ax * P.cm + P.cm - 1;
        for (int J = ya; J <= yb; ++J)
          for (int I = xa; I <= xb; ++I) acc += s1a[h1(J - J0, I)];
      }
      l3_items[it] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (items / 4) * 16; t += blockDim.x) {
      const int c = t >> 4;
      const float4 chunk = reinterpret_cast<const float4*>(l3_items)[c];
      const int item0 = 4 * c, ajl0 = item0 / naxp, ax0 = item0 - ajl0 * naxp;
      comm.publish_tl(tl_slot, sb.rank * ncp + (ajo0 + ajl0) * naxp + ax0, chunk, t & 15, sb.cs);
    }
    comm.sync();
    coarse_gather(true, 0.f);
    // u1 = e1 + P2 ec on the owned and halo 2h rows
    for (int t = threadIdx.x; t < (R1 + 2) * n1; t += blockDim.x) {
      const int lr1 = t / n1 - 1, I = t - (lr1 + 1) * n1, J = J0 + lr1;
      if (J < 0 || J > ny1) continue;
      const float ec = tl_ec[(l3_agg(J, P.cm, P.nay) - aj0) * naxp + l3_agg(I, P.cm, P.nax)];
      b1u[h1(lr1, I)] = b1x[h1(lr1, I)] + ec;
    }
    __syncthreads();
    // 2h post-smoothing z1 = u1 + S1 (r1 - A1 u1), exchanged
    for (int t = threadIdx.x; t < R1 * n1; t += blockDim.x) {
      const int lr1 = t / n1, I = t - lr1 * n1;
      r1[o1(lr1, I)] -= a1_apply(b1u, lr1, I);
    }
    __syncthreads();
    smooth_l1(r1, b1z);
    for (int t = threadIdx.x; t < R1 * n1; t += blockDim.x) {
      const int lr1 = t / n1, I = t - lr1 * n1;
      b1z[h1(lr1, I)] += b1u[h1(lr1, I)];
    }
    exchange_l1(b1z);
  }

  // Three-level cycle z = M^-1 r in FP32 over the fine, 2h and aggregate levels:
  //   e0 = S0 r;  w0 = r - A e0;  r1 = P1^T w0;
  //   e1 = S1 r1;  ec = A2^-1 P2^T (r1 - A1 e1);  u1 = e1 + P2 ec;  z1 = u1 + S1 (r1 - A1 u1);
  //   u0 = e0 + P1 z1;  z = u0 + S0 (r - A u0),
  // S0, S1 the slab-local damped-Jacobi smoothers of smooth_local / smooth_l1, P1 bilinear from
  // the 2h nodes (2I, 2J), P2 piecewise constant on the aggregates, A1 = P1^T A P1,
  // A2 = P2^T A1 P2.  Each level's correction is the exact adjoint of its restriction and every
  // smoother is symmetric, so M^-1 is symmetric.  Values on halo rows equal the owners' (e0 and
  // e1 exchanged, ec from the same restricted vector in every CTA, z1 exchanged), so M^-1 is one
  // operator across the CTAs.  Five cluster barriers.  z goes to zbuf; returns the local (r, z).
  __device__ Real vcycle3(const Real (&r)[NG][4]) {
    const int W = sb.W;
    float e[NG][4], w[NG][4];
    // fine pre-smoothing e0 = S0 r, exchanged (r in FP32 in w)
#pragma unroll
    for (int k = 0; k < NG; ++k)
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = (float)r[k][j];
    smooth_local(w, e);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) vy[l0 + j] = e[k][j];
    }
    exchange(vy);
    // fine residual w0 = r - A e0 on the owned rows, exchanged
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      float t[4];
      stencil_elem32(vy, wd, ws, wt, l0, W, t);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) vw[l0 + j] = unknown(k, j) ? w[k][j] - t[j] : 0.f;
    }
    exchange(vw);
    l1_correct();
    // u0 = e0 + P1 z1 on the owned and halo fine rows (in vy); 0 off the unknowns
    for (int i = threadIdx.x; i < (sb.R + 2) * W; i += blockDim.x) {
      if (vsd[i] == 0.f) {
        vy[i] = 0.f;
        continue;
      }
      const int lr = i / W - 1, ix = i - (lr + 1) * W - 1, y = sb.r0 + lr;
      const int ja = y / 2 - J0, jb = (y + 1) / 2 - J0, ia = ix / 2, ib = (ix + 1) / 2;
      const float z = 0.25f * ((b1z[h1(ja, ia)] + b1z[h1(ja, ib)]) + (b1z[h1(jb, ia)] + b1z[h1(jb, ib)]));
      vy[i] += z;
    }
    __syncthreads();
    // fine post-smoothing z = u0 + S0 (r - A u0)
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = 0.f;
      if (l0 < 0) continue;
      float t[4];
      stencil_elem32(vy, wd, ws, wt, l0, W, t);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) w[k][j] = unknown(k, j) ? (float)r[k][j] - t[j] : 0.f;
    }
    smooth_local(w, e);
    Real rz = Real(0);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const float z = vy[l0 + j] + e[k][j];
        zbuf[l0 + j] = (Real)z;
        rz = fma(r[k][j], (Real)z, rz);
      }
    }
    return rz;
  }

  // Two damped-Jacobi steps on the slab's diagonal block A_s (the rows of the other slabs left
  // out): z = S r + S (r - A_s S r) = (2S - S A_s S) r, S = omega D^-1, a symmetric operator,
  // positive definite while omega lambda_max(D^-1 A_s) < 2 (at most 0.8 * 2.25).  FP32 CG only
  // (the FP32 element weights); the first step's iterate goes through zbuf, whose halo rows are
  // not read, so the neighbours may already be writing their new edge rows into them.  No
  // communication; two block barriers.  z goes to zbuf; returns the local (r, z).
  __device__ Real precond_local2(const Real (&r)[NG][4]) {
    if constexpr (!kMixed) {
      return Real(0);   // not used: FP64 CG has no FP32 element weights
    } else {
    const float om = P.tl_omega;
    float e[NG][4];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) e[k][j] = 0.f;
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        e[k][j] = om * (float)dinv[l0 + j] * (float)r[k][j];
        zbuf[l0 + j] = (Real)e[k][j];
      }
    }
    __syncthreads();
    float z[NG][4];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
#pragma unroll
      for (int j = 0; j < kGroup; ++j) z[k][j] = 0.f;
      if (l0 < 0) continue;
      const int lr = l0 / sb.W - 1;
      float t[4];
      stencil_elem32(zbuf, wd, ws, wt, l0, sb.W, t, lr == 0, lr == sb.R - 1);
#pragma unroll
      for (int j = 0; j < kGroup; ++j) z[k][j] = fmaf(om * (float)dinv[l0 + j], (float)r[k][j] - t[j], e[k][j]);
    }
    __syncthreads();
    Real rz = Real(0);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        zbuf[l0 + j] = (Real)z[k][j];
        rz = fma(r[k][j], (Real)z[k][j], rz);
      }
    }
    return rz;
    }
  }

  // Jacobi-preconditioned CG in precision Real on A d = r, where r (given per node) is the FP64
  // residual scaled to unit 2-norm; on return x64 += unscale * d.  Stops when ||r||^2 <= target2
  // (scaled units) or at the iteration limit; returns the iteration count.  All CG scalars and
  // dot products are in precision Real.
  __device__ int cg_correct(Real (&r)[NG][4], Real target2, double unscale) {
    // FP32 CG without a two-level form: the slab-local two-step preconditioner if asked for
    const bool local2 = kMixed && !tl && P.local_steps >= 2;
    Real d[NG][4], p[NG][4], q[NG][4];
    Real rz;
    {
      Real v[1] = {Real(0)};
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int l0 = loc0[k];
#pragma unroll
        for (int j = 0; j < kGroup; ++j) { d[k][j] = Real(0); p[k][j] = Real(0); q[k][j] = Real(0); }
        if (l0 < 0 || tl || local2) continue;
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
          const Real z = dinv[l0 + j] * r[k][j];
          zbuf[l0 + j] = z;
          v[0] = fma(r[k][j], z, v[0]);
        }
      }
      if (local2) {
        v[0] = precond_local2(r);
      } else if (l3) {
        v[0] = vcycle3(r);
      } else if (vc && P.tl_nu >= 2) {
        v[0] = vcycle_local(r);
      } else if (vc) {
        // r on the halo rows from the neighbours' owned edge rows
        put_edges(vrh, r);
        comm.sync();
        v[0] = vcycle(r);
      } else if (tl) {
        coarse_restrict_push(r);
        comm.sync();
        coarse_gather(true, 0.f);
        v[0] = prolong_precondition(r);
      }
      __syncthreads();
      comm.push_halos(zbuf, sb);
      allreduce<Real, 1>(v);
      rz = v[0];
    }
    int it = 0;
    Real beta = Real(0);
    bool done = !(Real(1) > target2);
    while (!done && it < P.itmax) {
      // q = A z + beta q, p = z + beta p, (p, q); alpha = rz / (p, q)
      Real pq[1] = {Real(0)};
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int l0 = loc0[k];
        if (l0 < 0) continue;
        Real w[4];
        apply_A(zbuf, l0, w);
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
          const Real wj = unknown(k, j) ? w[j] : Real(0);
          const Real z = zbuf[l0 + j];
          p[k][j] = fma(beta, p[k][j], z);
          q[k][j] = fma(beta, q[k][j], wj);
          pq[0] = fma(p[k][j], q[k][j], pq[0]);
        }
      }
      if (vc && !l3 && P.tl_nu < 2) {
        // q's owned edge rows to the neighbours, whose copies of r on their halo rows follow
        // the same recurrence (visible after the all-reduce's barrier)
        put_edges(vqh, q);
      } else if (tl && !vc) {
        coarse_restrict_push(q);             // visible after the all-reduce's cluster barrier
      }
      const Real rz_c = rz;
      allreduce<Real, 1>(pq, [rz_c](Real* t) { t[0] = rz_c / t[0]; });
      const Real alpha = pq[0];
      if (tl && !vc) coarse_gather(false, (float)alpha);
      // d += alpha p, r -= alpha q, z = D^-1 r; (r, z), (r, r) and beta = (r, z)_new / (r, z)
      Real v[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int l0 = loc0[k];
        if (l0 < 0) continue;
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
          d[k][j] = fma(alpha, p[k][j], d[k][j]);
          r[k][j] = fma(-alpha, q[k][j], r[k][j]);
          v[1] = fma(r[k][j], r[k][j], v[1]);
          if (!tl && !local2) {
            const Real z = dinv[l0 + j] * r[k][j];
            zbuf[l0 + j] = z;
            v[0] = fma(r[k][j], z, v[0]);
          }
        }
      }
      if (local2) {
        v[0] = precond_local2(r);
      } else if (l3) {
        v[0] = vcycle3(r);
      } else if (vc && P.tl_nu >= 2) {
        v[0] = vcycle_local(r);
      } else if (vc) {
        for (int i = threadIdx.x; i < 2 * sb.W; i += blockDim.x) vrh[i] = fma(-alpha, vqh[i], vrh[i]);
        v[0] = vcycle(r);
      } else if (tl) {
        v[0] = prolong_precondition(r);
      }
      __syncthreads();
      comm.push_halos(zbuf, sb);
      allreduce<Real, 2, 1>(v, [rz_c](Real* t) { t[2] = t[0] / rz_c; });
      ++it;
      if (!(v[1] > target2)) done = true;  // NaN keeps iterating until the limit
      beta = v[2];
      rz = v[0];
    }
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) x64[l0 + j] = fma((double)d[k][j], unscale, x64[l0 + j]);
    }
    return it;
  }

  // Solve (C/dt + K) x = b64 with x64 (owned + halos) as initial guess; on return x64 holds
  // the solution with valid halos in every CTA.  `step` is the fine index for error reports.
  // `reuse_ax`: x64 is the previous solution of the same operator, so the A x64 saved by that
  // solve's final residual check gives the first residual without another stencil.
  __device__ void solve(int step, bool reuse_ax = false) {
    double r64[NG][4];
    double bb_rr[2] = {0.0, 0.0};
    bb_rr[1] = (reuse_ax && ax_valid && ax64) ? residual_saved(r64) : residual(r64);
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) bb_rr[0] = fma(b64[l0 + j], b64[l0 + j], bb_rr[0]);
    }
    allreduce<double, 2>(bb_rr);
    const double bb = bb_rr[0];
    double rr = bb_rr[1];
    const double tol2 = P.rtol * P.rtol * bb;
    int sweeps = 0, its = 0;
    while (rr > tol2 && sweeps < P.refmax) {
      // scale the residual to unit norm so the Real-precision CG works on O(1) values
      const double nrm = sqrt(rr), scale = 1.0 / nrm;
      Real r[NG][4];
#pragma unroll
      for (int k = 0; k < NG; ++k)
#pragma unroll
        for (int j = 0; j < kGroup; ++j) r[k][j] = (Real)(r64[k][j] * scale);
      const Real target2 = (Real)fmax(P.inner_rtol * P.inner_rtol, 0.25 * tol2 / rr);
      its += cg_correct(r, target2, nrm);
      ++sweeps;
      exchange_x64();
      double v[1] = {residual(r64)};
      allreduce<double, 1>(v);
      rr = v[0];
    }
    ax_valid = true;
    if (threadIdx.x == 0 && sb.rank == 0) {
      atomicAdd(&P.stats->solves, 1ull);
      atomicAdd(&P.stats->cg_iters, (unsigned long long)its);
      atomicAdd(&P.stats->refinements, (unsigned long long)sweeps);
      atomicMax(&P.stats->max_cg_iters, (unsigned long long)its);
      atomicAdd(&P.stats->kind_solves[P.stats_kind], 1ull);
      atomicAdd(&P.stats->kind_cg_iters[P.stats_kind], (unsigned long long)its);
      atomicAdd(&P.stats->kind_refinements[P.stats_kind], (unsigned long long)sweeps);
      if (!(rr == rr) || !(bb == bb) || isinf(rr)) {
        record_error(P.stats, PTG_ENONFINITE, P.stats_kind, step);
      } else if (rr > tol2) {
        record_error(P.stats, PTG_ENOCONV, P.stats_kind, step);
      }
    }
  }

  // sum over owned free nodes of x64^p, reduced over the cluster (FP64)
  __device__ double pnorm_p() {
    double v[1] = {0.0};
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j)
        if (dinv[l0 + j] != Real(0)) v[0] += ipow(x64[l0 + j], P.p_int);
    }
    allreduce<double, 1>(v);
    return v[0];
  }

  // Element term of Eq. 4.7 for the owned elements:
  //   g[e] = gsrc[e] - (1/nnorm) * ( dk_e lambda_e^T Ke T_j,e + dc_e/dt lambda_e^T Me (T_j - T_jm)_e )
  //          (+ addF[e] - subG[e] when given)
  // lambda is x64 (valid halos), T_j / T_jm are full global node vectors.
  __device__ void accumulate_g(const double* __restrict__ Tj, const double* __restrict__ Tjm, double dt_step,
                               double nnorm, const double* __restrict__ gsrc, double* __restrict__ gdst,
                               const double* __restrict__ addF, const double* __restrict__ subG) const {
    const int nx = P.nx, nn = P.nx + 1;
    const int er = min(sb.R, P.ny - sb.r0);  // owned element rows ey in [r0, r0+er)
    const int nel = er > 0 ? er * nx : 0;
    const double h2 = P.h * P.h / 36.0;
    for (int t = threadIdx.x; t < nel; t += blockDim.x) {
      const int ler = t / nx, ex = t - ler * nx;
      const int ey = sb.r0 + ler;
      const int e = ey * nx + ex;
      const int l0 = (ler + 1) * sb.W + ex + 1;   // SW node in x64
      const double lsw = x64[l0], lse = x64[l0 + 1], lne = x64[l0 + sb.W + 1], lnw = x64[l0 + sb.W];
      const int g0 = ey * nn + ex;
      const double tsw = Tj[g0], tse = Tj[g0 + 1], tne = Tj[g0 + nn + 1], tnw = Tj[g0 + nn];
      // lambda^T Ke T, Ke = (1/6)[[4,-1,-2,-1],[-1,4,-1,-2],[-2,-1,4,-1],[-1,-2,-1,4]] (order SW,SE,NE,NW)
      const double ksw = 4.0 * tsw - tse - 2.0 * tne - tnw;
      const double kse = -tsw + 4.0 * tse - tne - 2.0 * tnw;
      const double kne = -2.0 * tsw - tse + 4.0 * tne - tnw;
      const double knw = -tsw - 2.0 * tse - tne + 4.0 * tnw;
      const double kterm = (lsw * ksw + lse * kse + lne * kne + lnw * knw) / 6.0;
      double term = P.dk[e] * kterm;
      if (P.has_dc) {
        const double dsw = tsw - Tjm[g0], dse = tse - Tjm[g0 + 1], dne = tne - Tjm[g0 + nn + 1], dnw = tnw - Tjm[g0 + nn];
        // lambda^T Me dT, Me = h^2/36 [[4,2,1,2],[2,4,2,1],[1,2,4,2],[2,1,2,4]]
        const double msw = 4.0 * dsw + 2.0 * dse + dne + 2.0 * dnw;
        const double mse = 2.0 * dsw + 4.0 * dse + 2.0 * dne + dnw;
        const double mne = dsw + 2.0 * dse + 4.0 * dne + 2.0 * dnw;
        const double mnw = 2.0 * dsw + dse + 2.0 * dne + 4.0 * dnw;
        const double cterm = (lsw * msw + lse * mse + lne * mne + lnw * mnw) * h2;
        term += P.dc[e] * cterm / dt_step;
      }
      double g = (gsrc ? gsrc[e] : 0.0) - term / nnorm;
      if (addF) g += addF[e] - subG[e];
      gdst[e] = g;
    }
  }

  __device__ __forceinline__ double* hist_row(int j) const {
    const int r = j - P.hist_j0;
    if (P.hist == nullptr || r < 0 || r >= P.hist_rows) return nullptr;
    return P.hist + (size_t)r * P.Nn;
  }

  // correction x64 = x64 + F - G on the owned nodes, written to X (and Y if given)
  __device__ void apply_correction(const double* __restrict__ Fs, const double* __restrict__ Gs, double* __restrict__ X,
                                   double* __restrict__ Y) {
    ax_valid = false;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) {
        const int g = gnode(l0, j);
        if (g < 0) continue;
        const double t = dinv[l0 + j] != Real(0) ? (x64[l0 + j] + Fs[g]) - Gs[g] : 0.0;
        x64[l0 + j] = t;
        X[g] = t;
        if (Y) Y[g] = t;
      }
    }
  }

  // Cumulative objective update with increment sp / N (N Ne the divisor, sp = ||T||_p^p / Ne
  // folded by the caller): the power mean of Sec. 4.4, or the plain sum of the modified
  // objective Theta~ = Theta^p (Sec. 7.1).
  __device__ __forceinline__ double accumulate_theta(double theta, double inc) const {
    return P.objective == PTG_OBJ_MODIFIED ? theta + inc : pow(ipow(theta, P.p_int) + inc, 1.0 / P.p);
  }
  // Factor of T^(p-1) in the adjoint source: Theta^(1-p)/Ne (Eq. 4.6) or p/Ne (Sec. 7.1).
  __device__ __forceinline__ double adjoint_scale(double Theta) const {
    return (P.objective == PTG_OBJ_MODIFIED ? P.p : pow(Theta, 1.0 - P.p)) / (double)P.Ne;
  }

  // Copy the own rows of a node field (stride Nn) from src to dst (and to hist if given).
  __device__ void copy_field(const double* src, double* dst, double* hist) {
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int l0 = loc0[k];
      if (l0 < 0) continue;
      for (int j = 0; j < kGroup; ++j) {
        const int g = gnode(l0, j);
        if (g < 0) continue;
        const double v = src[g];
        dst[g] = v;
        if (hist) hist[g] = v;
      }
    }
  }

  // ------------------------------------------------------------------ task bodies
  __device__ void fine_primal(int task) {
    const int sa = P.chained ? P.s0 : P.s0 + task;
    const int sb_end = P.chained ? P.s0 + P.ns : sa + 1;
    const int M = P.M;
    const double inv_norm = 1.0 / ((double)P.Nt * (double)P.Ne);
    set_operator(false);
    load_x64(P.in_field + (size_t)sa * P.Nn);
    double theta = P.in_aux[sa];
    if (P.chained) {                              // a sequential run also records its start
      if (double* row = hist_row(M * sa)) store_x64(row);
    }
    const int nring = P.extrap;
    double* ring = nring > 1 && P.prev_field ? P.prev_field + (size_t)task * nring * P.Nn : nullptr;
    int saved = 0;                                // states of this slice in the ring
    for (int s = sa; s < sb_end; ++s) {
      for (int j = M * s + 1; j <= M * (s + 1); ++j) {
        const double qj = P.q_time[j];
        build_rhs([&](int g) { return qj * P.fload[g]; });
        // initial guess: the polynomial extrapolation through T_{j-1} (in x64) .. T_{j-n}, kept in
        // a ring of P.extrap rows per task (T_k in row k mod P.extrap; step j writes row
        // (j-1) mod P.extrap and reads the others).  Each slice starts afresh, in a chained run
        // too, so that a slice recomputed alone from its start state (checkpointed
        // differentiation) repeats every solve bit for bit.
        if (ring) {
          if (j == M * s + 1) saved = 0;
          const int n = min(saved + 1, nring);
          const double* X[kMaxExtrap - 1];
          for (int i = 2; i <= n; ++i) X[i - 2] = ring + (size_t)((j - i) % nring) * P.Nn;
          extrapolate_x64(n, X, ring + (size_t)((j - 1) % nring) * P.Nn);
          ++saved;
          solve(j, false);
        } else {
          solve(j, true);
        }
        const double sp = pnorm_p();
        if (threadIdx.x == 0) theta = accumulate_theta(theta, sp * inv_norm);  // used by thread 0 only
        if (double* row = hist_row(j)) store_x64(row);
      }
      store_x64(P.out_field + (size_t)s * P.Nn);
      if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[s] = theta;
    }
  }

  __device__ void coarse_primal(int task) {
    const int s = P.s0 + task;
    set_operator(true);
    load_x64(P.in_field + (size_t)s * P.Nn);
    const double theta0 = P.in_aux[s];
    const int j = P.M * (s + 1);
    if (P.src_field) {                          // a given source per slice (coarse-mesh G)
      const double* src = P.src_field + (size_t)s * P.Nn;
      build_rhs([&](int g) { return src[g]; });
    } else {
      const double qj = P.q_time[j];
      build_rhs([&](int g) { return qj * P.fload[g]; });
    }
    if (P.guess_next) load_x64(P.in_field + (size_t)(s + 1) * P.Nn);   // start from the guess u_{s+1}
    solve(j);
    const double sp = pnorm_p();
    store_x64(P.out_field + (size_t)s * P.Nn);
    if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[s] = accumulate_theta(theta0, sp / ((double)P.Ntau * (double)P.Ne));
  }

  __device__ void correct_primal() {
    if (!P.plt) set_operator(true);
    double theta;
    if (P.in_field) {                           // u_0 taken from the guess states, copied to X[0]
      load_x64(P.in_field);
      store_x64(P.out_field);
      theta = P.in_aux[0];
      if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[0] = theta;
    } else {                                    // u_0 given in X[0]
      load_x64(P.out_field);
      theta = P.out_aux[0];
    }
    if (double* row = hist_row(0)) store_x64(row);
    if (P.plt) {                                // G = 0 (Sec. 7, Eq. 7.2): u_{s+1} = F(u_s^old)
      for (int s = 0; s < P.Ntau; ++s) {
        copy_field(P.F_field + (size_t)s * P.Nn, P.out_field + (size_t)(s + 1) * P.Nn, hist_row(P.M * (s + 1)));
        if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[s + 1] = P.F_aux[s];
      }
      return;
    }
    for (int s = 0; s < P.Ntau; ++s) {
      const int j = P.M * (s + 1);
      if (P.src_field) {                        // a given source per slice (coarse-mesh G)
        const double* src = P.src_field + (size_t)s * P.Nn;
        build_rhs([&](int g) { return src[g]; });
      } else {
        const double qj = P.q_time[j];
        build_rhs([&](int g) { return qj * P.fload[g]; });
      }
      // initial guess G(u_s^old) plus the extrapolation of the increments G(u^new) - G(u^old) of
      // the last min(extrap - 1, s) steps, the increment of step s-1-i being u_{s-i}^new - F[s-1-i]
      // by the correction itself (plain: G(u_s^old))
      const int m = min(P.extrap - 1, min(s, 3));
      if (m >= 1) {
        const double* Fm[3];
        const double* X[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < m; ++i) Fm[i] = P.F_field + (size_t)(s - 1 - i) * P.Nn;
        for (int i = 1; i < m; ++i) X[i] = P.out_field + (size_t)(s - i) * P.Nn;
        load_x64_increment(P.G_field + (size_t)s * P.Nn, m, Fm, X);
      } else {
        load_x64(P.G_field + (size_t)s * P.Nn);
      }
      solve(j);
      const double sp = pnorm_p();
      apply_correction(P.F_field + (size_t)s * P.Nn, P.G_field + (size_t)s * P.Nn,
                       P.out_field + (size_t)(s + 1) * P.Nn, hist_row(j));
      if (threadIdx.x == 0) {                    // theta is needed by thread 0 only
        const double theta_g = accumulate_theta(theta, sp / ((double)P.Ntau * (double)P.Ne));
        theta = (theta_g + P.F_aux[s]) - P.G_aux[s];
        if (sb.rank == 0) P.out_aux[s + 1] = theta;
      }
      exchange_x64();
    }
  }

  __device__ void fine_adjoint(int task) {
    const int s_lo = P.chained ? P.s0 : P.s0 + task;
    const int s_hi = P.chained ? P.s0 + P.ns - 1 : s_lo;
    const int M = P.M;
    const double Theta = *P.Theta;
    const double scale = adjoint_scale(Theta);
    set_operator(false);
    load_x64(P.in_field + (size_t)(s_hi + 1) * P.Nn);
    const double* gsrc = P.in_aux + (size_t)(s_hi + 1) * P.Ne;
    // initial guess: the extrapolation through lambda_{j+1} (in x64) .. lambda_{j+n}, kept in a
    // ring of P.extrap rows per task, lambda_k in row k mod P.extrap; step j writes row
    // (j+1) mod P.extrap and reads the n-1 <= P.extrap-1 others, so no CTA writes a row that a
    // neighbour reads in the same step
    const int nring = P.extrap;
    double* ring = nring > 1 && P.prev_field ? P.prev_field + (size_t)task * nring * P.Nn : nullptr;
    int saved = 0;   // states of this slice in the ring
    for (int s = s_hi; s >= s_lo; --s) {
      double* gdst = P.out_aux + (size_t)s * P.Ne;
      saved = 0;     // each slice starts afresh, as in the primal
      for (int j = M * (s + 1); j >= M * s + 1; --j) {
        const double* Tj = hist_row(j);
        const double* Tjm = hist_row(j - 1);
        if (Tj == nullptr || Tjm == nullptr) {   // host validation makes this unreachable
          if (threadIdx.x == 0 && sb.rank == 0) record_error(P.stats, PTG_EINVAL, P.stats_kind, j);
          return;
        }
        build_rhs([&](int g) { return scale * ipow(Tj[g], P.p_int - 1); });
        if (ring) {
          const int n = min(saved + 1, nring);
          const double* X[kMaxExtrap - 1];
          for (int i = 2; i <= n; ++i) X[i - 2] = ring + (size_t)((j + i) % nring) * P.Nn;
          extrapolate_x64(n, X, ring + (size_t)((j + 1) % nring) * P.Nn);
          ++saved;
          solve(j, false);
        } else {
          solve(j, true);
        }
        accumulate_g(Tj, Tjm, P.dt, (double)P.Nt, gsrc, gdst, nullptr, nullptr);
        gsrc = gdst;
        __syncthreads();
      }
      store_x64(P.out_field + (size_t)s * P.Nn);
    }
  }

  // G_adj of slice s; with P.src_mode 1 or 2 one of its two parts (G_adj is affine in the source
  // scale c of Eq. 4.6): 1 the solve and g update driven by v_{s+1} with c = 0, 2 those of the
  // unit source (c = 1) from lambda = 0 and g = 0.  The parts start from the state they
  // propagate (zero for part 2).
  __device__ void coarse_adjoint(int task) {
    const int s = P.s0 + task;
    const int kidx = P.M * s + 1;
    const int kprev = max(kidx - P.M, 0);
    const double scale = P.src_mode == 0 ? adjoint_scale(*P.Theta) : (P.src_mode == 1 ? 0.0 : 1.0);
    const double* Tk = P.hist + (size_t)kidx * P.Nn;
    const double* Tkm = P.hist + (size_t)kprev * P.Nn;
    set_operator(true);
    if (P.src_mode == 2)
      zero_x64();
    else
      load_x64(P.in_field + (size_t)(s + 1) * P.Nn);
    build_rhs([&](int g) { return scale * ipow(Tk[g], P.p_int - 1); });
    if (P.guess_next && P.src_mode == 0) load_x64(P.in_field + (size_t)s * P.Nn);   // start from the guess lambda_s
    solve(kidx);
    accumulate_g(Tk, Tkm, P.dtau, (double)P.Ntau, P.src_mode == 2 ? nullptr : P.in_aux + (size_t)(s + 1) * P.Ne,
                 P.out_aux + (size_t)s * P.Ne, nullptr, nullptr);
    store_x64(P.out_field + (size_t)s * P.Nn);
  }

  __device__ void correct_adjoint() {
    const double Theta = *P.Theta;
    const double scale = adjoint_scale(Theta);
    if (!P.plt) set_operator(true);
    // v_Ntau = 0
    {
      double* Xl = P.out_field + (size_t)P.Ntau * P.Nn;
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int l0 = loc0[k];
        if (l0 < 0) continue;
        for (int j = 0; j < kGroup; ++j) {
          const int g = gnode(l0, j);
          if (g >= 0) Xl[g] = 0.0;
        }
      }
      const int er = min(sb.R, P.ny - sb.r0);
      double* Xg = P.out_aux + (size_t)P.Ntau * P.Ne;
      for (int t = threadIdx.x; t < (er > 0 ? er * P.nx : 0); t += blockDim.x) Xg[sb.r0 * P.nx + t] = 0.0;
    }
    if (P.plt) {                                // G = 0 (Sec. 7, Eq. 7.2): v_s = F(v_{s+1}^old)
      const int er = min(sb.R, P.ny - sb.r0);
      for (int s = P.Ntau - 1; s >= 0; --s) {
        copy_field(P.F_field + (size_t)s * P.Nn, P.out_field + (size_t)s * P.Nn, nullptr);
        const double* Fg = P.F_aux + (size_t)s * P.Ne + sb.r0 * P.nx;
        double* Xg = P.out_aux + (size_t)s * P.Ne + sb.r0 * P.nx;
        for (int t = threadIdx.x; t < (er > 0 ? er * P.nx : 0); t += blockDim.x) Xg[t] = Fg[t];
      }
      return;
    }
    zero_x64();
    for (int s = P.Ntau - 1; s >= 0; --s) {
      const int kidx = P.M * s + 1;
      const int kprev = max(kidx - P.M, 0);
      const double* Tk = P.hist + (size_t)kidx * P.Nn;
      const double* Tkm = P.hist + (size_t)kprev * P.Nn;
      build_rhs([&](int g) { return scale * ipow(Tk[g], P.p_int - 1); });
      // initial guess G(v_{s+1}^old) plus the extrapolation of the increments of the last
      // min(extrap - 1, Ntau - 1 - s) steps, the increment of step s+1+i being
      // v_{s+1+i}^new - F[s+1+i] (plain: G(v_{s+1}^old))
      const int m = min(P.extrap - 1, min(P.Ntau - 1 - s, 3));
      if (m >= 1) {
        const double* Fm[3];
        const double* X[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < m; ++i) Fm[i] = P.F_field + (size_t)(s + 1 + i) * P.Nn;
        for (int i = 1; i < m; ++i) X[i] = P.out_field + (size_t)(s + 1 + i) * P.Nn;
        load_x64_increment(P.G_field + (size_t)s * P.Nn, m, Fm, X);
      } else {
        load_x64(P.G_field + (size_t)s * P.Nn);
      }
      solve(kidx);
      // g_s = g_{s+1} - (1/Ntau) term(lambda_G) + F_g[s] - G_g[s]
      accumulate_g(Tk, Tkm, P.dtau, (double)P.Ntau, P.out_aux + (size_t)(s + 1) * P.Ne, P.out_aux + (size_t)s * P.Ne,
                   P.F_aux + (size_t)s * P.Ne, P.G_aux + (size_t)s * P.Ne);
      comm.sync();                              // every CTA is done reading lambda_G halos
      apply_correction(P.F_field + (size_t)s * P.Nn, P.G_field + (size_t)s * P.Nn, P.out_field + (size_t)s * P.Nn,
                       nullptr);
      exchange_x64();
    }
  }
};

// One kernel per (precision, groups per thread, task kind); each kernel inlines a single task
// body, which keeps register pressure and compile time down.  Up to 512 threads per CTA (the
// plan picks the block size), at most 128 registers per thread.
constexpr int kStepMaxThreads = 512;

template <class Real, int NG, int KIND, class Comm>
__device__ __forceinline__ void run_task(Stepper<Real, NG, Comm>& st, int task) {
  if constexpr (KIND == KIND_FINE_PRI) st.fine_primal(task);
  if constexpr (KIND == KIND_COARSE_PRI) st.coarse_primal(task);
  if constexpr (KIND == KIND_CORRECT_PRI) st.correct_primal();
  if constexpr (KIND == KIND_FINE_ADJ) st.fine_adjoint(task);
  if constexpr (KIND == KIND_COARSE_ADJ) st.coarse_adjoint(task);
  if constexpr (KIND == KIND_CORRECT_ADJ) st.correct_adjoint();
}

template <class Real, int NG, int KIND>
__global__ void __launch_bounds__(kStepMaxThreads, 1) stepper_kernel(const __grid_constant__ StepParams P) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ RedSmem rs;
  ClusterComm comm(rs);
  Stepper<Real, NG, ClusterComm> st(P, comm, dyn_smem);
  // every CTA of the cluster has initialised its shared memory before any DSMEM traffic
  cluster_sync_all();
  run_task<Real, NG, KIND>(st, (int)(blockIdx.x / (unsigned)P.cs));
  // no CTA leaves while another may still read or write its shared memory
  cluster_sync_all();
}

// Systems spread over groups of CTAs of a cooperative launch: the grid holds gridDim.x / P.cs
// groups of P.cs CTAs (one slab each); group g runs tasks g, g + groups, ... < P.wide_tasks one
// after the other.  Halo rows, reduction partials and the two-level partials go through global
// memory (GridComm).  Used for one FP64 system over every SM, and for grids whose slabs do not
// fit the 16 CTAs of a cluster.
template <class Real, int NG, int KIND>
__global__ void __launch_bounds__(kStepMaxThreads, 1) stepper_wide_kernel(const __grid_constant__ StepParams P) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ RedSmem rs;
  GridComm comm(P, rs);
  const int ngroups = (int)gridDim.x / P.cs;
  for (int task = comm.gid; task < P.wide_tasks; task += ngroups) {
    Stepper<Real, NG, GridComm> st(P, comm, dyn_smem);
    run_task<Real, NG, KIND>(st, task);
    comm.sync();                               // the group's halo slots are free again
  }
}

// Persistent multi-design variant: `tasks` lists (design, task) pairs, largest designs first;
// every cluster claims the next pair from the work queue until the list is exhausted, and
// runs it with that design's parameters (table[design]).  All designs share the precision,
// the cluster size, the block size and NG; shared memory is carved per task for the design's
// geometry from the largest footprint that the launch reserves.
template <class Real, int NG, int KIND>
__global__ void __launch_bounds__(kStepMaxThreads, 1) stepper_batch_kernel(const StepParams* __restrict__ table,
                                                                       const int2* __restrict__ tasks, int ntasks,
                                                                       int* __restrict__ queue) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ RedSmem rs;
  __shared__ int s_task;
  ClusterComm comm(rs);
  const unsigned rank = comm.cl.block_rank();
  cluster_sync_all();                          // all CTAs running before any DSMEM store
  for (;;) {
    // rank 0 claims the next task and writes it into every CTA of the cluster; the barrier
    // publishes it (and orders it after the previous task's last shared-memory access)
    if (rank == 0 && threadIdx.x == 0) {
      const int t = atomicAdd(queue, 1);
      for (unsigned r = 0; r < comm.cl.num_blocks(); ++r) *comm.cl.map_shared_rank(&s_task, r) = t;
    }
    cluster_sync_all();
    const int t = s_task;                      // identical in every CTA: the loop is uniform
    if (t >= ntasks) break;
    const int2 tk = tasks[t];
    Stepper<Real, NG, ClusterComm> st(table[tk.x], comm, dyn_smem);
    cluster_sync_all();
    run_task<Real, NG, KIND>(st, tk.y);
    cluster_sync_all();
  }
}

}  // namespace ptg
