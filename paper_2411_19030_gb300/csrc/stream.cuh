// stream.cuh -- fine propagators (a2, a5) of large grids with the Krylov vectors in global memory.
//
// The cluster stepper keeps a system's CG vectors on chip, so at 512 x 512 a slice needs the
// shared memory and registers of about 50 SMs and only 3 of 128 slices run at once.  Here every
// slice is a group of G CTAs of one launch (G = 1 or 2 at 512 x 512, one or two per SM), and
// its vectors stream from HBM: x (FP64, two buffers: the state a step starts from and the one
// it solves for), the right-hand side b (FP64), and the CG vectors r, p, q, d (precision Real).
// All Ntau slices then advance together and the solves are bound by HBM bandwidth.
//
// Each step is the same as the stepper's (stepper.cuh): b = (C/dt) x_{j-1} + source, the start
// extrapolated through the slice's last states (the same ring of states per task), the FP64
// residual loop around a Jacobi-preconditioned CG in Real on A d = r / ||r||, then theta (primal)
// or the Eq. 4.7 element sums (adjoint).  Per CG iteration the group sums two sets of dot
// products (fixed order, identical in every CTA of the group: GridComm) and each CTA streams its
// rows: q = A z + beta q, p = z + beta p with z = D^-1 r formed on the fly from r, then
// d += alpha p, r -= alpha q; 44 bytes per node and iteration in FP32.  The FP32 operator
// (per-node weights C, E, N, NE, NW and 1/C, shared by every slice) stays in L2.
#pragma once
#include "comm.cuh"

namespace ptg {

template <class Real, int KIND>
struct Streamer {
  const StepParams& P;
  GridComm& comm;
  int rank = 0, r0 = 0, R = 0;   // this CTA's node rows [r0, r0 + R) of the group's system
  int nn = 0;                    // nodes per row (nx + 1)
  int cpr = 0;                   // 32-node chunks per row
  double *xa = nullptr, *xb = nullptr, *b = nullptr;   // group workspace, [Nn] each
  Real *r = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
  double step_dt = 0.0, inv_dt = 0.0;

  __device__ Streamer(const StepParams& P_, GridComm& comm_) : P(P_), comm(comm_) {
    rank = comm.rank();
    slab_rows(P.ny + 1, P.cs, rank, r0, R);
    nn = P.nx + 1;
    cpr = (nn + 31) / 32;
    const int grp = (int)blockIdx.x / P.cs;
    double* w64 = P.st_w64 + (size_t)grp * 3 * P.Nn;
    xa = w64;
    xb = w64 + P.Nn;
    b = w64 + 2 * (size_t)P.Nn;
    Real* wr = reinterpret_cast<Real*>(P.st_wr) + (size_t)grp * 4 * P.Nn;
    r = wr;
    p = wr + P.Nn;
    q = wr + 2 * (size_t)P.Nn;
    d = wr + 3 * (size_t)P.Nn;
    step_dt = P.dt;
    inv_dt = 1.0 / P.dt;
  }

  // Visit this CTA's nodes: warps take 32-node chunks of a row, f(g, iy, ix, go) for the nodes
  // inside the grid (g the node index, go its index in the padded weight arrays).
  template <class F>
  __device__ __forceinline__ void for_nodes(F f) const {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = warp; c < R * cpr; c += nwarps) {
      const int lr = c / cpr, ix = (c - lr * cpr) * 32 + lane;
      if (ix >= nn) continue;
      const int iy = r0 + lr;
      f(iy * nn + ix, iy, ix, (iy + 1) * P.W + ix + 1);
    }
  }

  __device__ __forceinline__ bool free_node(int g) const { return P.dirichlet[g] == 0; }

  // value of v at the node offset (dy, dx) from (iy, ix), 0 outside the grid
  template <class T>
  __device__ __forceinline__ T at(const T* __restrict__ v, int g, int iy, int ix, int dy, int dx) const {
    const int y = iy + dy, x = ix + dx;
    return (y >= 0 && y <= P.ny && x >= 0 && x <= P.nx) ? v[g + dy * nn + dx] : T(0);
  }

  // (A v)(g) with FP64 per-node weights W (padded layout)
  __device__ __forceinline__ double stencil64(const NodeWeights& A, const double* __restrict__ v, int g, int iy, int ix,
                                              int go) const {
    const int Wp = P.W;
    double y = A.C[go] * v[g];
    y = fma(A.E[go], at(v, g, iy, ix, 0, 1), y);
    y = fma(A.E[go - 1], at(v, g, iy, ix, 0, -1), y);
    y = fma(A.N[go], at(v, g, iy, ix, 1, 0), y);
    y = fma(A.N[go - Wp], at(v, g, iy, ix, -1, 0), y);
    y = fma(A.NE[go], at(v, g, iy, ix, 1, 1), y);
    y = fma(A.NE[go - Wp - 1], at(v, g, iy, ix, -1, -1), y);
    y = fma(A.NW[go], at(v, g, iy, ix, 1, -1), y);
    y = fma(A.NW[go - Wp + 1], at(v, g, iy, ix, -1, 1), y);
    return y;
  }

  // weight k (C, E, N, NE, NW) of C/dt + K at a padded node index, in the CG precision (the FP32
  // copies for FP32 CG, the FP64 weights for FP64 CG), and 1/C (0 off the unknowns)
  __device__ __forceinline__ Real wgt(int k, int idx) const {
    if constexpr (sizeof(Real) == 8) {
      const NodeWeights& A = P.A_fine;
      return (k == 0 ? A.C : k == 1 ? A.E : k == 2 ? A.N : k == 3 ? A.NE : A.NW)[idx];
    } else {
      return P.w32[k * P.w32_stride + idx];
    }
  }
  __device__ __forceinline__ Real winv(int idx) const {
    if constexpr (sizeof(Real) == 8)
      return P.w64_inv[idx];
    else
      return P.w32_inv[idx];
  }

  // z = D^-1 r at (g + offset), 0 outside the grid (the inverse diagonal is 0 off the unknowns)
  __device__ __forceinline__ Real zat(int g, int iy, int ix, int dy, int dx, int go) const {
    const int y = iy + dy, x = ix + dx;
    if (y < 0 || y > P.ny || x < 0 || x > P.nx) return Real(0);
    return winv(go + dy * P.W + dx) * r[g + dy * nn + dx];
  }

  // (A z)(g) in the CG precision, z = D^-1 r formed on the fly
  __device__ __forceinline__ Real stencil_z(int g, int iy, int ix, int go) const {
    const int Wp = P.W;
    Real y = wgt(0, go) * zat(g, iy, ix, 0, 0, go);
    y = fma(wgt(1, go), zat(g, iy, ix, 0, 1, go), y);
    y = fma(wgt(1, go - 1), zat(g, iy, ix, 0, -1, go), y);
    y = fma(wgt(2, go), zat(g, iy, ix, 1, 0, go), y);
    y = fma(wgt(2, go - Wp), zat(g, iy, ix, -1, 0, go), y);
    y = fma(wgt(3, go), zat(g, iy, ix, 1, 1, go), y);
    y = fma(wgt(3, go - Wp - 1), zat(g, iy, ix, -1, -1, go), y);
    y = fma(wgt(4, go), zat(g, iy, ix, 1, -1, go), y);
    y = fma(wgt(4, go - Wp + 1), zat(g, iy, ix, -1, 1, go), y);
    return y;
  }

  template <class T, int NV, int NX = 0, class Post = NoPost>
  __device__ __forceinline__ void allreduce(T (&v)[NV + NX], Post post = Post()) {
    comm.template allreduce<T, NV, NX, Post>(v, P.cs, post);
  }

  // r = b - A x (FP64, stored in Real unscaled); returns the local (b, b) and (r, r)
  __device__ void residual(const double* __restrict__ x, double& bb, double& rr) const {
    bb = 0.0;
    rr = 0.0;
    for_nodes([&](int g, int iy, int ix, int go) {
      double rv = 0.0;
      if (free_node(g)) {
        rv = b[g] - stencil64(P.A_fine, x, g, iy, ix, go);
        bb = fma(b[g], b[g], bb);
        rr = fma(rv, rv, rr);
      }
      r[g] = (Real)rv;
    });
  }

  // Solve (C/dt + K) x = b from the start in x (the group's rows of x, every row readable).
  __device__ void solve(double* __restrict__ x, int step) {
    double v2[2];
    residual(x, v2[0], v2[1]);
    allreduce<double, 2>(v2);
    const double bb = v2[0];
    double rr = v2[1];
    const double tol2 = P.rtol * P.rtol * bb;
    int sweeps = 0, its = 0;
    while (rr > tol2 && sweeps < P.refmax) {
      const double nrm = sqrt(rr);
      const Real scale = (Real)(1.0 / nrm);
      const Real target2 = (Real)fmax(P.inner_rtol * P.inner_rtol, 0.25 * tol2 / rr);
      // r /= ||r||, d = p = q = 0; (r, z)
      Real a[1] = {Real(0)};
      for_nodes([&](int g, int iy, int ix, int go) {
        const Real rv = r[g] * scale;
        r[g] = rv;
        d[g] = Real(0);
        p[g] = Real(0);
        q[g] = Real(0);
        a[0] = fma(rv, winv(go) * rv, a[0]);
      });
      allreduce<Real, 1>(a);
      Real rz = a[0], beta = Real(0);
      int it = 0;
      bool done = !(Real(1) > target2);
      while (!done && it < P.itmax) {
        // q = A z + beta q, p = z + beta p, (p, q); alpha = rz / (p, q)
        Real pq[1] = {Real(0)};
        for_nodes([&](int g, int iy, int ix, int go) {
          Real pv = Real(0), qv = Real(0);
          if (free_node(g)) {
            qv = fma(beta, q[g], stencil_z(g, iy, ix, go));
            pv = fma(beta, p[g], winv(go) * r[g]);
          }
          q[g] = qv;
          p[g] = pv;
          pq[0] = fma(pv, qv, pq[0]);
        });
        const Real rz_c = rz;
        allreduce<Real, 1>(pq, [rz_c](Real* t) { t[0] = rz_c / t[0]; });
        const Real alpha = pq[0];
        // d += alpha p, r -= alpha q; (r, z), (r, r), beta = (r, z)_new / (r, z)
        Real v[3] = {Real(0), Real(0), Real(0)};
        for_nodes([&](int g, int iy, int ix, int go) {
          d[g] = fma(alpha, p[g], d[g]);
          const Real rv = fma(-alpha, q[g], r[g]);
          r[g] = rv;
          v[0] = fma(rv, winv(go) * rv, v[0]);
          v[1] = fma(rv, rv, v[1]);
        });
        allreduce<Real, 2, 1>(v, [rz_c](Real* t) { t[2] = t[0] / rz_c; });
        ++it;
        if (!(v[1] > target2)) done = true;   // NaN keeps iterating until the limit
        beta = v[2];
        rz = v[0];
      }
      its += it;
      ++sweeps;
      // x += ||r|| d on the own rows, then the FP64 residual of the whole system
      for_nodes([&](int g, int iy, int ix, int go) {
        if (free_node(g)) x[g] = fma((double)d[g], nrm, x[g]);
      });
      comm.sync();
      residual(x, v2[0], v2[1]);
      double w1[1] = {v2[1]};
      allreduce<double, 1>(w1);
      rr = w1[0];
    }
    if (threadIdx.x == 0 && rank == 0) {
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

  __device__ __forceinline__ double* hist_row(int j) const {
    const int rr = j - P.hist_j0;
    if (P.hist == nullptr || rr < 0 || rr >= P.hist_rows) return nullptr;
    return P.hist + (size_t)rr * P.Nn;
  }

  __device__ __forceinline__ double accumulate_theta(double theta, double inc) const {
    return P.objective == PTG_OBJ_MODIFIED ? theta + inc : pow(ipow(theta, P.p_int) + inc, 1.0 / P.p);
  }
  __device__ __forceinline__ double adjoint_scale(double Theta) const {
    return (P.objective == PTG_OBJ_MODIFIED ? P.p : pow(Theta, 1.0 - P.p)) / (double)P.Ne;
  }

  // b = (C/dt) xp + src(g) on the own rows; xn = the start of the step: the extrapolation through
  // xp and the ring rows X[0..n-2] (n = 1: xp itself); the ring row wr receives xp.
  template <class Src>
  __device__ void begin_step(const double* __restrict__ xp, double* __restrict__ xn, int n, const double* const* X,
                             double* __restrict__ wr, Src src) {
    for_nodes([&](int g, int iy, int ix, int go) {
      const double x1 = xp[g];
      if (wr) wr[g] = x1;
      double bv = 0.0, xv = 0.0;
      if (free_node(g)) {
        bv = fma(stencil64(P.mass, xp, g, iy, ix, go), inv_dt, src(g));
        if (n <= 1)
          xv = x1;
        else if (n == 2)
          xv = fma(2.0, x1, -X[0][g]);
        else if (n == 3)
          xv = fma(3.0, x1 - X[0][g], X[1][g]);
        else
          xv = fma(4.0, x1 + X[1][g], -fma(6.0, X[0][g], X[2][g]));
      }
      b[g] = bv;
      xn[g] = xv;
    });
    comm.sync();
  }

  // copy a node vector of the system into the own rows of dst (Dirichlet nodes 0)
  __device__ void load(const double* __restrict__ src, double* __restrict__ dst) const {
    for_nodes([&](int g, int, int, int) { dst[g] = free_node(g) ? src[g] : 0.0; });
  }
  __device__ void store(const double* __restrict__ src, double* __restrict__ dst) const {
    if (!dst) return;
    for_nodes([&](int g, int, int, int) { dst[g] = src[g]; });
  }

  __device__ double pnorm_p(const double* __restrict__ x) {
    double v[1] = {0.0};
    for_nodes([&](int g, int, int, int) {
      if (free_node(g)) v[0] += ipow(x[g], P.p_int);
    });
    allreduce<double, 1>(v);
    return v[0];
  }

  // ------------------------------------------------------------------ task bodies
  __device__ void fine_primal(int task) {
    const int s = P.s0 + task;
    const int M = P.M;
    const double inv_norm = 1.0 / ((double)P.Nt * (double)P.Ne);
    double* x_prev = xa;
    double* x_cur = xb;
    load(P.in_field + (size_t)s * P.Nn, x_prev);
    comm.sync();
    double theta = P.in_aux[s];
    const int nring = P.extrap;
    double* ring = nring > 1 && P.prev_field ? P.prev_field + (size_t)task * nring * P.Nn : nullptr;
    int saved = 0;
    for (int j = M * s + 1; j <= M * (s + 1); ++j) {
      const double qj = P.q_time[j];
      const double* X[kMaxExtrap - 1];
      int n = 1;
      double* wr = nullptr;
      if (ring) {
        n = min(saved + 1, nring);
        for (int i = 2; i <= n; ++i) X[i - 2] = ring + (size_t)((j - i) % nring) * P.Nn;
        wr = ring + (size_t)((j - 1) % nring) * P.Nn;
        ++saved;
      }
      begin_step(x_prev, x_cur, n, X, wr, [&](int g) { return qj * P.fload[g]; });
      solve(x_cur, j);
      const double sp = pnorm_p(x_cur);
      if (threadIdx.x == 0) theta = accumulate_theta(theta, sp * inv_norm);
      store(x_cur, hist_row(j));
      double* t = x_prev;
      x_prev = x_cur;
      x_cur = t;
    }
    store(x_prev, P.out_field + (size_t)s * P.Nn);
    if (threadIdx.x == 0 && rank == 0) P.out_aux[s] = theta;
  }

  // Eq. 4.7 element sums of the own element rows (rows r0 .. r0 + R - 1 below ny)
  __device__ void accumulate_g(const double* __restrict__ lam, const double* __restrict__ Tj,
                               const double* __restrict__ Tjm, const double* __restrict__ gsrc,
                               double* __restrict__ gdst) const {
    const int nx = P.nx;
    const int er = min(R, P.ny - r0);
    const int nel = er > 0 ? er * nx : 0;
    const double h2 = P.h * P.h / 36.0;
    const double nnorm = (double)P.Nt;
    for (int t = threadIdx.x; t < nel; t += blockDim.x) {
      const int ler = t / nx, ex = t - ler * nx;
      const int ey = r0 + ler;
      const int e = ey * nx + ex;
      const int g0 = ey * nn + ex;
      const double lsw = lam[g0], lse = lam[g0 + 1], lne = lam[g0 + nn + 1], lnw = lam[g0 + nn];
      const double tsw = Tj[g0], tse = Tj[g0 + 1], tne = Tj[g0 + nn + 1], tnw = Tj[g0 + nn];
      const double ksw = 4.0 * tsw - tse - 2.0 * tne - tnw;
      const double kse = -tsw + 4.0 * tse - tne - 2.0 * tnw;
      const double kne = -2.0 * tsw - tse + 4.0 * tne - tnw;
      const double knw = -tsw - 2.0 * tse - tne + 4.0 * tnw;
      const double kterm = (lsw * ksw + lse * kse + lne * kne + lnw * knw) / 6.0;
      double term = P.dk[e] * kterm;
      if (P.has_dc) {
        const double dsw = tsw - Tjm[g0], dse = tse - Tjm[g0 + 1], dne = tne - Tjm[g0 + nn + 1],
                     dnw = tnw - Tjm[g0 + nn];
        const double msw = 4.0 * dsw + 2.0 * dse + dne + 2.0 * dnw;
        const double mse = 2.0 * dsw + 4.0 * dse + 2.0 * dne + dnw;
        const double mne = dsw + 2.0 * dse + 4.0 * dne + 2.0 * dnw;
        const double mnw = 2.0 * dsw + dse + 2.0 * dne + 4.0 * dnw;
        const double cterm = (lsw * msw + lse * mse + lne * mne + lnw * mnw) * h2;
        term += P.dc[e] * cterm / step_dt;
      }
      gdst[e] = gsrc[e] - term / nnorm;
    }
  }

  __device__ void fine_adjoint(int task) {
    const int s = P.s0 + task;
    const int M = P.M;
    const double scale = adjoint_scale(*P.Theta);
    double* x_prev = xa;
    double* x_cur = xb;
    load(P.in_field + (size_t)(s + 1) * P.Nn, x_prev);
    comm.sync();
    const double* gsrc = P.in_aux + (size_t)(s + 1) * P.Ne;
    double* gdst = P.out_aux + (size_t)s * P.Ne;
    const int nring = P.extrap;
    double* ring = nring > 1 && P.prev_field ? P.prev_field + (size_t)task * nring * P.Nn : nullptr;
    int saved = 0;
    for (int j = M * (s + 1); j >= M * s + 1; --j) {
      const double* Tj = hist_row(j);
      const double* Tjm = hist_row(j - 1);
      if (Tj == nullptr || Tjm == nullptr) {   // host validation makes this unreachable
        if (threadIdx.x == 0 && rank == 0) record_error(P.stats, PTG_EINVAL, P.stats_kind, j);
        return;
      }
      const double* X[kMaxExtrap - 1];
      int n = 1;
      double* wr = nullptr;
      if (ring) {
        n = min(saved + 1, nring);
        for (int i = 2; i <= n; ++i) X[i - 2] = ring + (size_t)((j + i) % nring) * P.Nn;
        wr = ring + (size_t)((j + 1) % nring) * P.Nn;
        ++saved;
      }
      begin_step(x_prev, x_cur, n, X, wr, [&](int g) { return scale * ipow(Tj[g], P.p_int - 1); });
      solve(x_cur, j);
      accumulate_g(x_cur, Tj, Tjm, gsrc, gdst);
      gsrc = gdst;
      double* t = x_prev;
      x_prev = x_cur;
      x_cur = t;
      __syncthreads();
    }
    store(x_prev, P.out_field + (size_t)s * P.Nn);
  }
};

}  // namespace ptg
