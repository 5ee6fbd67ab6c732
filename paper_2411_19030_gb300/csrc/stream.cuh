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
  int G4 = 0;                    // groups of 4 nodes per padded row (W / 4)
  // group workspace, padded node layout (node (iy, ix) at (iy + 1) W + ix + 1, the layout of the
  // per-node weights), zero off the unknowns
  double *xa = nullptr, *xb = nullptr, *b = nullptr;
  Real *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
  double step_dt = 0.0, inv_dt = 0.0;

  __device__ Streamer(const StepParams& P_, GridComm& comm_) : P(P_), comm(comm_) {
    rank = comm.rank();
    slab_rows(P.ny + 1, P.cs, rank, r0, R);
    nn = P.nx + 1;
    G4 = P.W / kGroup;
    const int grp = (int)blockIdx.x / P.cs;
    const size_t pv = (size_t)P.st_pv;                 // entries of one padded vector incl. slack
    double* w64 = P.st_w64 + (size_t)grp * 3 * pv + kSlack;
    xa = w64;
    xb = w64 + pv;
    b = w64 + 2 * pv;
    Real* wr = reinterpret_cast<Real*>(P.st_wr) + (size_t)grp * 5 * pv + kSlack;
    r = wr;
    z = wr + pv;
    p = wr + 2 * pv;
    q = wr + 3 * pv;
    d = wr + 4 * pv;
    step_dt = P.dt;
    inv_dt = 1.0 / P.dt;
  }

  // Visit this CTA's groups of 4 nodes (columns 4g-1 .. 4g+2 of an owned row): f(loc, iy, g) with
  // loc the padded index of the group's first node (16-byte aligned).
  template <class F>
  __device__ __forceinline__ void for_groups(F f) const {
    for (int t = threadIdx.x; t < R * G4; t += blockDim.x) {
      const int lr = t / G4, g = t - lr * G4, iy = r0 + lr;
      f((iy + 1) * P.W + kGroup * g, iy, g);
    }
  }

  // Two groups per loop trip (t and t + blockDim.x): f(loc[2], ok[2]) loads both groups' operands
  // before it computes, so each thread keeps twice the memory requests in flight.
  template <class F>
  __device__ __forceinline__ void for_group_pairs(F f) const {
    const int n = R * G4;
    for (int t0 = threadIdx.x; t0 < n; t0 += 2 * blockDim.x) {
      int loc[2];
      bool ok[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int t = t0 + u * (int)blockDim.x;
        ok[u] = t < n;
        const int lr = ok[u] ? t / G4 : 0, g = ok[u] ? t - lr * G4 : 0;
        loc[u] = (r0 + lr + 1) * P.W + kGroup * g;
      }
      f(loc, ok);
    }
  }

  // node index of column 4g-1+j of row iy, or -1 for a pad column
  __device__ __forceinline__ int gnode(int iy, int g, int j) const {
    const int ix = kGroup * g - 1 + j;
    return (ix >= 0 && ix <= P.nx) ? iy * nn + ix : -1;
  }

  // 1/C of the 4 nodes (0 off the unknowns) in the CG precision
  __device__ __forceinline__ void dinv4(int loc, Real (&v)[4]) const {
    if constexpr (sizeof(Real) == 8) {
      load4(P.w64_inv + loc, v);
    } else {
      const float4 c = *reinterpret_cast<const float4*>(P.w32_inv + loc);
      v[0] = c.x; v[1] = c.y; v[2] = c.z; v[3] = c.w;
    }
  }
  __device__ __forceinline__ void ld4(const Real* __restrict__ a, int loc, Real (&v)[4]) const {
    if constexpr (sizeof(Real) == 8) {
      load4(a + loc, v);
    } else {
      const float4 c = *reinterpret_cast<const float4*>(a + loc);
      v[0] = c.x; v[1] = c.y; v[2] = c.z; v[3] = c.w;
    }
  }
  __device__ __forceinline__ void st4(Real* __restrict__ a, int loc, const Real (&v)[4]) const {
    if constexpr (sizeof(Real) == 8) {
      *reinterpret_cast<double2*>(a + loc) = make_double2(v[0], v[1]);
      *reinterpret_cast<double2*>(a + loc + 2) = make_double2(v[2], v[3]);
    } else {
      *reinterpret_cast<float4*>(a + loc) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
  __device__ __forceinline__ void st4d(double* __restrict__ a, int loc, const double (&v)[4]) const {
    *reinterpret_cast<double2*>(a + loc) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(a + loc + 2) = make_double2(v[2], v[3]);
  }

  // (A z) on a group in the CG precision
  __device__ __forceinline__ void apply_z(int loc, Real (&w)[4]) const {
    if constexpr (sizeof(Real) == 8) {
      double y[4];
      stencil_node64<double>(z, loc, P.A_fine, loc, P.W, y);
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = y[j];
    } else {
      float y[4];
      stencil_elem32(z, P.w32, P.w32 + P.w32_stride, P.w32 + 2 * P.w32_stride, loc, P.W, y);
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = y[j];
    }
  }

  template <class T, int NV, int NX = 0, class Post = NoPost>
  __device__ __forceinline__ void allreduce(T (&v)[NV + NX], Post post = Post()) {
    comm.template allreduce<T, NV, NX, Post>(v, P.cs, post);
  }

  // r = b - A x (FP64, stored in the CG precision unscaled, 0 off the unknowns); the local
  // (b, b) and (r, r)
  __device__ void residual(const double* __restrict__ x, double& bb, double& rr) const {
    bb = 0.0;
    rr = 0.0;
    for_groups([&](int loc, int, int) {
      double y[4], bv[4];
      Real di[4], rv[4];
      stencil_node64<double>(x, loc, P.A_fine, loc, P.W, y);
      load4(b + loc, bv);
      dinv4(loc, di);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double t = di[j] != Real(0) ? bv[j] - y[j] : 0.0;
        bb = fma(bv[j], bv[j], bb);
        rr = fma(t, t, rr);
        rv[j] = (Real)t;
      }
      st4(r, loc, rv);
    });
  }

  // Solve (C/dt + K) x = b from the start in x (every row of x readable).
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
      // r /= ||r||, z = D^-1 r, d = p = q = 0; (r, z)
      Real a[1] = {Real(0)};
      for_groups([&](int loc, int, int) {
        Real rv[4], di[4], zv[4], zero[4] = {Real(0), Real(0), Real(0), Real(0)};
        ld4(r, loc, rv);
        dinv4(loc, di);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          rv[j] *= scale;
          zv[j] = di[j] * rv[j];
          a[0] = fma(rv[j], zv[j], a[0]);
        }
        st4(r, loc, rv);
        st4(z, loc, zv);
        st4(d, loc, zero);
        st4(p, loc, zero);
        st4(q, loc, zero);
      });
      allreduce<Real, 1>(a);
      Real rz = a[0], beta = Real(0);
      int it = 0;
      bool done = !(Real(1) > target2);
      while (!done && it < P.itmax) {
        // q = A z + beta q, p = z + beta p, (p, q); alpha = rz / (p, q)
        Real pq[1] = {Real(0)};
        for_groups([&](int loc, int, int) {
          Real w[4], qv[4], pv[4], zv[4], di[4];
          apply_z(loc, w);
          ld4(q, loc, qv);
          ld4(p, loc, pv);
          ld4(z, loc, zv);
          dinv4(loc, di);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            qv[j] = di[j] != Real(0) ? fma(beta, qv[j], w[j]) : Real(0);
            pv[j] = fma(beta, pv[j], zv[j]);
            pq[0] = fma(pv[j], qv[j], pq[0]);
          }
          st4(q, loc, qv);
          st4(p, loc, pv);
        });
        const Real rz_c = rz;
        allreduce<Real, 1>(pq, [rz_c](Real* t) { t[0] = rz_c / t[0]; });
        const Real alpha = pq[0];
        // d += alpha p, r -= alpha q, z = D^-1 r; (r, z), (r, r), beta = (r, z)_new / (r, z)
        Real v[3] = {Real(0), Real(0), Real(0)};
        for_group_pairs([&](const int (&loc)[2], const bool (&ok)[2]) {
          Real dv[2][4], pv[2][4], rv[2][4], qv[2][4], di[2][4];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!ok[u]) continue;
            ld4(d, loc[u], dv[u]);
            ld4(p, loc[u], pv[u]);
            ld4(r, loc[u], rv[u]);
            ld4(q, loc[u], qv[u]);
            dinv4(loc[u], di[u]);
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!ok[u]) continue;
            Real zv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              dv[u][j] = fma(alpha, pv[u][j], dv[u][j]);
              rv[u][j] = fma(-alpha, qv[u][j], rv[u][j]);
              zv[j] = di[u][j] * rv[u][j];
              v[0] = fma(rv[u][j], zv[j], v[0]);
              v[1] = fma(rv[u][j], rv[u][j], v[1]);
            }
            st4(d, loc[u], dv[u]);
            st4(r, loc[u], rv[u]);
            st4(z, loc[u], zv);
          }
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
      for_groups([&](int loc, int, int) {
        double xv[4];
        Real dv[4];
        load4(x + loc, xv);
        ld4(d, loc, dv);
#pragma unroll
        for (int j = 0; j < 4; ++j) xv[j] = fma((double)dv[j], nrm, xv[j]);
        st4d(x, loc, xv);
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

  // b = (C/dt) xp + src(node) on the own rows; xn = the start of the step: the extrapolation
  // through xp and the ring rows X[0..n-2] (n = 1: xp itself); the ring row wr receives xp.
  // The ring rows are node vectors ([Nn], unpadded).
  template <class Src>
  __device__ void begin_step(const double* __restrict__ xp, double* __restrict__ xn, int n, const double* const* X,
                             double* __restrict__ wr, Src src) {
    for_groups([&](int loc, int iy, int g) {
      double y[4], x1[4], bv[4], xv[4];
      stencil_node64<double>(xp, loc, P.mass, loc, P.W, y);
      load4(xp + loc, x1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        bv[j] = 0.0;
        xv[j] = 0.0;
        if (gi < 0) continue;
        if (wr) wr[gi] = x1[j];
        if (P.dirichlet[gi]) continue;
        bv[j] = fma(y[j], inv_dt, src(gi));
        if (n <= 1)
          xv[j] = x1[j];
        else if (n == 2)
          xv[j] = fma(2.0, x1[j], -X[0][gi]);
        else if (n == 3)
          xv[j] = fma(3.0, x1[j] - X[0][gi], X[1][gi]);
        else
          xv[j] = fma(4.0, x1[j] + X[1][gi], -fma(6.0, X[0][gi], X[2][gi]));
      }
      st4d(b, loc, bv);
      st4d(xn, loc, xv);
    });
    comm.sync();
  }

  // a node vector ([Nn]) into the own rows of a padded vector (0 off the unknowns), and back
  __device__ void load(const double* __restrict__ src, double* __restrict__ dst) const {
    for_groups([&](int loc, int iy, int g) {
      double v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        v[j] = (gi >= 0 && !P.dirichlet[gi]) ? src[gi] : 0.0;
      }
      st4d(dst, loc, v);
    });
  }
  __device__ void store(const double* __restrict__ src, double* __restrict__ dst) const {
    if (!dst) return;
    for_groups([&](int loc, int iy, int g) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        if (gi >= 0) dst[gi] = src[loc + j];
      }
    });
  }

  __device__ double pnorm_p(const double* __restrict__ x) {
    double v[1] = {0.0};
    for_groups([&](int loc, int iy, int g) {
      double xv[4];
      load4(x + loc, xv);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (gnode(iy, g, j) >= 0) v[0] += ipow(xv[j], P.p_int);   // 0 on Dirichlet nodes
    });
    allreduce<double, 1>(v);
    return v[0];
  }

  // Eq. 4.7 element sums of the own element rows (rows r0 .. r0 + R - 1 below ny); lam padded,
  // Tj and Tjm node vectors
  __device__ void accumulate_g(const double* __restrict__ lam, const double* __restrict__ Tj,
                               const double* __restrict__ Tjm, const double* __restrict__ gsrc,
                               double* __restrict__ gdst) const {
    const int nx = P.nx, Wp = P.W;
    const int er = min(R, P.ny - r0);
    const int nel = er > 0 ? er * nx : 0;
    const double h2 = P.h * P.h / 36.0;
    const double nnorm = (double)P.Nt;
    for (int t = threadIdx.x; t < nel; t += blockDim.x) {
      const int ler = t / nx, ex = t - ler * nx;
      const int ey = r0 + ler;
      const int e = ey * nx + ex;
      const int g0 = ey * nn + ex;
      const int l0 = (ey + 1) * Wp + ex + 1;
      const double lsw = lam[l0], lse = lam[l0 + 1], lne = lam[l0 + Wp + 1], lnw = lam[l0 + Wp];
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
