// stepper.cuh -- the cluster time stepper: every backward-Euler solve of the pass.
//
// One thread-block cluster owns one independent time-stepping system (one Parareal slice,
// one coarse step, or the sequential correction sweep).  Its CTAs split the node rows into
// slabs held on chip (ptg_device.cuh).  Each solve of (C/dt + K) x = b (Eq. 2.7 / 4.4) is a
// Jacobi-preconditioned CG in precision Real, wrapped in an FP64 residual loop:
//     r = b - A x            (FP64, from the FP64 element weights)
//     while ||r|| > rtol ||b||:   CG:  A d = r  (Real),  x += d,  r = b - A x
// With Real = double the first CG already meets the tolerance (plain FP64 PCG); with
// Real = float this is iterative refinement with FP64 residuals.  CG uses the recurrence
// q_{k+1} = A z_{k+1} + beta q_k (q = A p) so each iteration has two cluster reductions and
// the z halo exchange rides on the second one.
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
#include "ptg_device.cuh"
#include "ptg_internal.h"

namespace ptg {

__device__ __forceinline__ void record_error(DevStats* st, int code, int kind, int step) {
  if (atomicCAS(&st->status, 0, code) == 0) {
    st->fail_kind = 10 + kind;
    st->fail_step = step;
  }
}

template <class Real, int NPT>
struct Stepper {
  static constexpr bool kMixed = std::is_same<Real, float>::value;

  const StepParams& P;
  cg::cluster_group& cluster;
  RedSmem& rs;
  Slab sb;
  int phase = 0;
  // shared memory
  double* x64;      // FP64 state, own rows + halos
  double* b64;      // FP64 right-hand side, owned nodes (linear index)
  Real* zbuf;       // CG operand with halos
  Real* wd;         // element weights in CG precision
  Real* ws;
  Real* wt;
  // per-thread node slots: node i = threadIdx.x + k*blockDim.x of the slab
  int lrow[NPT];
  Real invd[NPT];
  unsigned freemask = 0;
  // current operator (FP64 element weights in global memory, offset to this slab)
  const double* gwd = nullptr;
  const double* gws = nullptr;
  const double* gwt = nullptr;
  double step_dt = 0.0;
  // per-solve counters (meaningful in thread 0)
  long long it_total = 0;

  __device__ Stepper(const StepParams& P_, cg::cluster_group& cl, RedSmem& rs_, unsigned char* dyn)
      : P(P_), cluster(cl), rs(rs_) {
    sb.nx = P.nx;
    sb.ny = P.ny;
    sb.cs = P.cs;
    sb.rank = (int)cluster.block_rank();
    slab_rows(P.ny + 1, P.cs, sb.rank, sb.r0, sb.R);
    sb.W = P.nx + 3;
    sb.EW = P.nx + 2;
    sb.nown = sb.R * (P.nx + 1);
    const int nodes_halo = (P.rmax + 2) * sb.W;
    const int elems = (P.rmax + 1) * sb.EW;
    x64 = reinterpret_cast<double*>(dyn);
    b64 = x64 + nodes_halo;
    zbuf = reinterpret_cast<Real*>(b64 + P.rmax * (P.nx + 1));
    wd = zbuf + nodes_halo;
    ws = wd + elems;
    wt = ws + elems;
    // zero every buffer: pads, halos outside the domain and unused rows stay zero
    for (int i = threadIdx.x; i < nodes_halo; i += blockDim.x) {
      x64[i] = 0.0;
      zbuf[i] = Real(0);
    }
    for (int i = threadIdx.x; i < P.rmax * (P.nx + 1); i += blockDim.x) b64[i] = 0.0;
    for (int i = threadIdx.x; i < elems; i += blockDim.x) {
      wd[i] = Real(0);
      ws[i] = Real(0);
      wt[i] = Real(0);
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      lrow[k] = i < sb.nown ? i / (P.nx + 1) : 0;
      if (i < sb.nown && P.dirichlet[sb.r0 * (P.nx + 1) + i] == 0) freemask |= 1u << k;
      invd[k] = Real(0);
    }
  }

  __device__ __forceinline__ bool own(int k, int& i) const {
    i = threadIdx.x + k * blockDim.x;
    return i < sb.nown;
  }
  __device__ __forceinline__ bool is_free(int k) const { return (freemask >> k) & 1u; }
  __device__ __forceinline__ int loc_of(int k, int i) const { return i + 2 * lrow[k] + sb.W + 1; }
  __device__ __forceinline__ int eloc_of(int k, int i) const { return i + lrow[k] + sb.EW + 1; }
  __device__ __forceinline__ int gnode(int i) const { return sb.r0 * (P.nx + 1) + i; }

  template <int NV>
  __device__ __forceinline__ void allreduce(double (&v)[NV]) {
    cluster_allreduce<NV>(v, rs, phase, cluster, sb.cs);
  }

  // Select the operator C/dt + K (fine) or C/dtau + K (coarse): copy its element weights
  // for this slab into shared memory in CG precision and form the Jacobi inverse diagonal.
  __device__ void set_operator(bool coarse) {
    const int PE = (P.ny + 2) * (P.nx + 2);
    const double* wA = coarse ? P.wA_coarse : P.wA_fine;
    step_dt = coarse ? P.dtau : P.dt;
    const int off = sb.r0 * sb.EW;  // padded element row r0 holds element row r0 - 1
    gwd = wA + off;
    gws = wA + PE + off;
    gwt = wA + 2 * PE + off;
    const int n = (sb.R + 1) * sb.EW;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      wd[i] = (Real)gwd[i];
      ws[i] = (Real)gws[i];
      wt[i] = (Real)gwt[i];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int i;
      if (own(k, i) && is_free(k)) {
        const int e = eloc_of(k, i);
        const Real dg = (wd[e - sb.EW - 1] + wd[e - sb.EW]) + (wd[e - 1] + wd[e]);
        invd[k] = Real(1) / dg;
      } else {
        invd[k] = Real(0);
      }
    }
  }

  // Load a node vector from global memory into x64: owned rows and both halo rows
  // (Dirichlet nodes forced to zero).  Ends with __syncthreads.
  __device__ void load_x64(const double* __restrict__ src) {
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
    __syncthreads();
    for (int i = threadIdx.x; i < (P.rmax + 2) * sb.W; i += blockDim.x) x64[i] = 0.0;
    __syncthreads();
  }

  // Store the owned rows of x64 to a global node vector.
  __device__ void store_x64(double* __restrict__ dst) const {
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int i;
      if (own(k, i)) dst[gnode(i)] = x64[loc_of(k, i)];
    }
  }

  // Refresh every CTA's halo rows of x64 from the neighbours' owned rows.
  __device__ void exchange_x64() {
    __syncthreads();
    push_halos(x64, sb, cluster);
    cluster_sync_all();
  }

  // b64 = (C/dt) x64 + src, with src supplied per owned node by the functor.
  template <class Src>
  __device__ void build_rhs(Src src) {
    const double inv_dt = 1.0 / step_dt;
    const double* gm = P.mass + sb.r0 * sb.EW;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int i;
      if (own(k, i)) {
        double b = 0.0;
        if (is_free(k)) b = mass9(x64, gm, loc_of(k, i), eloc_of(k, i), sb.W, sb.EW) * inv_dt + src(gnode(i));
        b64[i] = b;
      }
    }
  }

  // r = b - A x64 on owned free nodes (FP64).
  __device__ __forceinline__ double residual(int k, int i) const {
    double ax;
    if constexpr (kMixed) {
      ax = stencil9<double, double>(x64, gwd, gws, gwt, loc_of(k, i), eloc_of(k, i), sb.W, sb.EW);
    } else {
      ax = stencil9<double, Real>(x64, wd, ws, wt, loc_of(k, i), eloc_of(k, i), sb.W, sb.EW);
    }
    return b64[i] - ax;
  }

  // CG in precision Real on A d = r (r given per slot), d accumulated into x64.
  // Returns the iteration count.  Target: ||r_k||^2 <= target2.
  __device__ int cg_correct(Real (&r)[NPT], double rr0, double target2) {
    Real d[NPT], p[NPT], q[NPT];
    double rz;
    {
      double v[2] = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        d[k] = Real(0);
        p[k] = Real(0);
        q[k] = Real(0);
        if (own(k, i)) {
          const Real z = invd[k] * r[k];
          zbuf[loc_of(k, i)] = z;
          v[0] += (double)(r[k] * z);
        }
      }
      __syncthreads();
      push_halos(zbuf, sb, cluster);
      double w[1] = {v[0]};
      allreduce<1>(w);
      rz = w[0];
    }
    int it = 0;
    Real beta = Real(0);
    bool done = !(rr0 > target2);
    while (!done && it < P.itmax) {
      // q = A z + beta q, p = z + beta p, (p, q)
      double pq[1] = {0.0};
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        if (own(k, i)) {
          const int loc = loc_of(k, i);
          Real w = stencil9<Real, Real>(zbuf, wd, ws, wt, loc, eloc_of(k, i), sb.W, sb.EW);
          if (!is_free(k)) w = Real(0);
          const Real z = zbuf[loc];
          p[k] = fma(beta, p[k], z);
          q[k] = fma(beta, q[k], w);
          pq[0] += (double)(p[k] * q[k]);
        }
      }
      allreduce<1>(pq);
      const Real alpha = (Real)(rz / pq[0]);
      double v[2] = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        if (own(k, i)) {
          d[k] = fma(alpha, p[k], d[k]);
          r[k] = fma(-alpha, q[k], r[k]);
          const Real z = invd[k] * r[k];
          zbuf[loc_of(k, i)] = z;
          v[0] += (double)(r[k] * z);
          v[1] += (double)(r[k] * r[k]);
        }
      }
      __syncthreads();
      push_halos(zbuf, sb, cluster);
      allreduce<2>(v);
      ++it;
      if (!(v[1] > target2)) done = true;  // NaN keeps iterating until the limit
      beta = (Real)(v[0] / rz);
      rz = v[0];
    }
    // x64 += d on owned nodes
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int i;
      if (own(k, i)) x64[loc_of(k, i)] += (double)d[k];
    }
    return it;
  }

  // Solve (C/dt + K) x = b64 with x64 (owned + halos) as initial guess; on return x64 holds
  // the solution with valid halos in every CTA.  `step` is the fine index for error reports.
  __device__ void solve(int step) {
    double bb_rr[2] = {0.0, 0.0};
    Real r[NPT];
    double r64[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int i;
      r64[k] = 0.0;
      if (own(k, i) && is_free(k)) {
        r64[k] = residual(k, i);
        bb_rr[0] += b64[i] * b64[i];
        bb_rr[1] += r64[k] * r64[k];
      }
    }
    allreduce<2>(bb_rr);
    const double bb = bb_rr[0];
    double rr = bb_rr[1];
    const double tol2 = P.rtol * P.rtol * bb;
    int sweeps = 0, its = 0;
    while (rr > tol2 && sweeps < P.refmax) {
#pragma unroll
      for (int k = 0; k < NPT; ++k) r[k] = (Real)r64[k];
      const double target2 = fmax(P.inner_rtol * P.inner_rtol * rr, 0.25 * tol2);
      its += cg_correct(r, rr, target2);
      ++sweeps;
      exchange_x64();
      double v[1] = {0.0};
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        r64[k] = 0.0;
        if (own(k, i) && is_free(k)) {
          r64[k] = residual(k, i);
          v[0] += r64[k] * r64[k];
        }
      }
      allreduce<1>(v);
      rr = v[0];
    }
    if (threadIdx.x == 0 && sb.rank == 0) {
      atomicAdd(&P.stats->solves, 1ull);
      atomicAdd(&P.stats->cg_iters, (unsigned long long)its);
      atomicAdd(&P.stats->refinements, (unsigned long long)sweeps);
      atomicMax(&P.stats->max_cg_iters, (unsigned long long)its);
      if (!(rr == rr) || !(bb == bb) || isinf(rr)) {
        record_error(P.stats, PTG_ENONFINITE, P.kind, step);
      } else if (rr > tol2) {
        record_error(P.stats, PTG_ENOCONV, P.kind, step);
      }
    }
  }

  // sum over owned free nodes of x64^p, reduced over the cluster (FP64)
  __device__ double pnorm_p() {
    double v[1] = {0.0};
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int i;
      if (own(k, i) && is_free(k)) v[0] += ipow(x64[loc_of(k, i)], P.p_int);
    }
    allreduce<1>(v);
    return v[0];
  }

  // Element term of Eq. 4.7 for the owned elements:
  //   g[e] -= (1/nnorm) * ( dk_e lambda_e^T Ke T_j,e + dc_e/dt lambda_e^T Me (T_j - T_jm)_e )
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
      const int l0 = (ler + 1) * sb.W + ex + 1;   // SW in x64
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
      double g = gsrc[e] - term / nnorm;
      if (addF) g += addF[e] - subG[e];
      gdst[e] = g;
    }
  }

  __device__ __forceinline__ double* hist_row(int j) const {
    const int r = j - P.hist_j0;
    if (P.hist == nullptr || r < 0 || r >= P.hist_rows) return nullptr;
    return P.hist + (size_t)r * P.Nn;
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
    for (int s = sa; s < sb_end; ++s) {
      for (int j = M * s + 1; j <= M * (s + 1); ++j) {
        const double qj = P.q_time[j];
        build_rhs([&](int g) { return qj * P.fload[g]; });
        solve(j);
        const double sp = pnorm_p();
        theta = pow(ipow(theta, P.p_int) + sp * inv_norm, 1.0 / P.p);
        if (double* row = hist_row(j)) store_x64(row);
      }
      store_x64(P.out_field + (size_t)s * P.Nn);
      if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[s] = theta;
    }
  }

  __device__ void coarse_primal(int task) {
    const int s = task;
    set_operator(true);
    load_x64(P.in_field + (size_t)s * P.Nn);
    const double theta0 = P.in_aux[s];
    const int j = P.M * (s + 1);
    const double qj = P.q_time[j];
    build_rhs([&](int g) { return qj * P.fload[g]; });
    solve(j);
    const double sp = pnorm_p();
    const double theta = pow(ipow(theta0, P.p_int) + sp / ((double)P.Ntau * (double)P.Ne), 1.0 / P.p);
    store_x64(P.out_field + (size_t)s * P.Nn);
    if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[s] = theta;
  }

  __device__ void correct_primal() {
    set_operator(true);
    load_x64(P.out_field);                      // u_0
    double theta = P.out_aux[0];
    if (double* row = hist_row(0)) store_x64(row);
    for (int s = 0; s < P.Ntau; ++s) {
      const int j = P.M * (s + 1);
      const double qj = P.q_time[j];
      build_rhs([&](int g) { return qj * P.fload[g]; });
      load_x64(P.G_field + (size_t)s * P.Nn);   // initial guess G(u_s^old)
      solve(j);
      const double sp = pnorm_p();
      const double theta_g = pow(ipow(theta, P.p_int) + sp / ((double)P.Ntau * (double)P.Ne), 1.0 / P.p);
      const double* Fs = P.F_field + (size_t)s * P.Nn;
      const double* Gs = P.G_field + (size_t)s * P.Nn;
      double* Xn = P.out_field + (size_t)(s + 1) * P.Nn;
      double* hrow = hist_row(j);
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        if (own(k, i)) {
          const int g = gnode(i);
          const int loc = loc_of(k, i);
          const double t = is_free(k) ? (x64[loc] + Fs[g]) - Gs[g] : 0.0;
          x64[loc] = t;
          Xn[g] = t;
          if (hrow) hrow[g] = t;
        }
      }
      theta = (theta_g + P.F_aux[s]) - P.G_aux[s];
      if (threadIdx.x == 0 && sb.rank == 0) P.out_aux[s + 1] = theta;
      exchange_x64();
    }
  }

  __device__ void fine_adjoint(int task) {
    const int s_lo = P.chained ? P.s0 : P.s0 + task;
    const int s_hi = P.chained ? P.s0 + P.ns - 1 : s_lo;
    const int M = P.M;
    const double Theta = *P.Theta;
    const double scale = pow(Theta, 1.0 - P.p) / (double)P.Ne;
    set_operator(false);
    load_x64(P.in_field + (size_t)(s_hi + 1) * P.Nn);
    const double* gsrc = P.in_aux + (size_t)(s_hi + 1) * P.Ne;
    for (int s = s_hi; s >= s_lo; --s) {
      double* gdst = P.out_aux + (size_t)s * P.Ne;
      for (int j = M * (s + 1); j >= M * s + 1; --j) {
        const double* Tj = hist_row(j);
        const double* Tjm = hist_row(j - 1);
        if (Tj == nullptr || Tjm == nullptr) {   // host validation makes this unreachable
          if (threadIdx.x == 0 && sb.rank == 0) record_error(P.stats, PTG_EINVAL, P.kind, j);
          return;
        }
        build_rhs([&](int g) { return scale * ipow(Tj[g], P.p_int - 1); });
        solve(j);
        accumulate_g(Tj, Tjm, P.dt, (double)P.Nt, gsrc, gdst, nullptr, nullptr);
        gsrc = gdst;
        __syncthreads();
      }
      store_x64(P.out_field + (size_t)s * P.Nn);
    }
  }

  __device__ void coarse_adjoint(int task) {
    const int s = task;
    const int kidx = P.M * s + 1;
    const int kprev = max(kidx - P.M, 0);
    const double Theta = *P.Theta;
    const double scale = pow(Theta, 1.0 - P.p) / (double)P.Ne;
    const double* Tk = P.hist + (size_t)kidx * P.Nn;
    const double* Tkm = P.hist + (size_t)kprev * P.Nn;
    set_operator(true);
    load_x64(P.in_field + (size_t)(s + 1) * P.Nn);
    build_rhs([&](int g) { return scale * ipow(Tk[g], P.p_int - 1); });
    solve(kidx);
    accumulate_g(Tk, Tkm, P.dtau, (double)P.Ntau, P.in_aux + (size_t)(s + 1) * P.Ne, P.out_aux + (size_t)s * P.Ne,
                 nullptr, nullptr);
    store_x64(P.out_field + (size_t)s * P.Nn);
  }

  __device__ void correct_adjoint() {
    const double Theta = *P.Theta;
    const double scale = pow(Theta, 1.0 - P.p) / (double)P.Ne;
    set_operator(true);
    // v_Ntau = 0
    {
      double* Xl = P.out_field + (size_t)P.Ntau * P.Nn;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        if (own(k, i)) Xl[gnode(i)] = 0.0;
      }
      const int er = min(sb.R, P.ny - sb.r0);
      double* Xg = P.out_aux + (size_t)P.Ntau * P.Ne;
      for (int t = threadIdx.x; t < (er > 0 ? er * P.nx : 0); t += blockDim.x) Xg[sb.r0 * P.nx + t] = 0.0;
    }
    zero_x64();
    for (int s = P.Ntau - 1; s >= 0; --s) {
      const int kidx = P.M * s + 1;
      const int kprev = max(kidx - P.M, 0);
      const double* Tk = P.hist + (size_t)kidx * P.Nn;
      const double* Tkm = P.hist + (size_t)kprev * P.Nn;
      build_rhs([&](int g) { return scale * ipow(Tk[g], P.p_int - 1); });
      load_x64(P.G_field + (size_t)s * P.Nn);   // initial guess G(v_{s+1}^old)
      solve(kidx);
      // g_s = g_{s+1} - (1/Ntau) term(lambda_G) + F_g[s] - G_g[s]
      accumulate_g(Tk, Tkm, P.dtau, (double)P.Ntau, P.out_aux + (size_t)(s + 1) * P.Ne, P.out_aux + (size_t)s * P.Ne,
                   P.F_aux + (size_t)s * P.Ne, P.G_aux + (size_t)s * P.Ne);
      cluster_sync_all();                       // every CTA is done reading lambda_G halos
      const double* Fs = P.F_field + (size_t)s * P.Nn;
      const double* Gs = P.G_field + (size_t)s * P.Nn;
      double* Xn = P.out_field + (size_t)s * P.Nn;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        int i;
        if (own(k, i)) {
          const int g = gnode(i);
          const int loc = loc_of(k, i);
          const double t = is_free(k) ? (x64[loc] + Fs[g]) - Gs[g] : 0.0;
          x64[loc] = t;
          Xn[g] = t;
        }
      }
      exchange_x64();
    }
  }
};

// One kernel per (precision, slots per thread, threads per CTA, task kind): each kernel
// inlines a single task body, which keeps register pressure and compile time down.
// MINB = 2 CTAs per SM caps the kernel at 128 registers per thread for 256 threads.
template <class Real, int NPT, int NTHREADS, int KIND>
__global__ void __launch_bounds__(NTHREADS, (NTHREADS <= 256 ? 2 : 1)) stepper_kernel(const __grid_constant__ StepParams P) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ RedSmem rs;
  cg::cluster_group cluster = cg::this_cluster();
  Stepper<Real, NPT> st(P, cluster, rs, dyn_smem);
  // every CTA of the cluster has initialised its shared memory before any DSMEM traffic
  cluster_sync_all();
  const int task = (int)(blockIdx.x / (unsigned)P.cs);
  if constexpr (KIND == KIND_FINE_PRI) st.fine_primal(task);
  if constexpr (KIND == KIND_COARSE_PRI) st.coarse_primal(task);
  if constexpr (KIND == KIND_CORRECT_PRI) st.correct_primal();
  if constexpr (KIND == KIND_FINE_ADJ) st.fine_adjoint(task);
  if constexpr (KIND == KIND_COARSE_ADJ) st.coarse_adjoint(task);
  if constexpr (KIND == KIND_CORRECT_ADJ) st.correct_adjoint();
  // no CTA leaves while another may still read or write its shared memory
  cluster_sync_all();
}

}  // namespace ptg
