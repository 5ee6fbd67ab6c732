// stream.cuh -- propagators of large grids with the Krylov vectors in global memory: the fine
// propagators (a2, a5), and the coarse propagators (a3) and correction sweeps (a4) with FP64 CG;
// each CG preconditioned by Jacobi or by a geometric multigrid V-cycle in FP32 of its step's
// operator (see "multigrid" below).
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
  static constexpr bool kCoarse = KIND == KIND_COARSE_PRI || KIND == KIND_COARSE_ADJ || KIND == KIND_CORRECT_PRI ||
                                  KIND == KIND_CORRECT_ADJ;
  NodeWeights A64;               // the operator of the kind's step: C/dt + K or C/dtau + K
  float* mgws = nullptr;         // the group's multigrid workspace

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
    step_dt = kCoarse ? P.dtau : P.dt;
    inv_dt = 1.0 / step_dt;
    A64 = kCoarse ? P.A_coarse : P.A_fine;
    if (P.mg_levels > 0) mgws = P.mg_ws + (size_t)grp * P.mg_ws_stride;
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

  // (A z) on a group in the CG precision (FP32 coarse-step operator: the multigrid's level 0)
  __device__ __forceinline__ void apply_z(int loc, Real (&w)[4]) const {
    if constexpr (sizeof(Real) == 8) {
      double y[4];
      stencil_node64<double>(z, loc, A64, loc, P.W, y);
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = y[j];
    } else if constexpr (kCoarse) {
      float zl[6], zm[6], zh[6];
      load_window(z, loc - P.W, zl);
      load_window(z, loc, zm);
      load_window(z, loc + P.W, zh);
      lstencil(0, loc, zl, zm, zh, w);
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

  // ------------------------------------------------------------------ multigrid
  // z = M^-1 r by one V(nu, nu)-cycle over the levels of mg.cu, all in FP32:
  //   level l < L-1: u = S^nu f (damped Jacobi from zero), res = f - A u, f_{l+1} = P^T res,
  //                  e_{l+1} from the level below, u += P e_{l+1}, e = S^nu applied from u;
  //   level L-1:     e = mg_coarse_steps damped-Jacobi steps from zero,
  // with f = r on level 0 and e = z there.  Pre- and post-smoothing are the same symmetric
  // steps and restriction is the transpose of prolongation, so M^-1 is symmetric (and positive
  // definite: omega lambda_max(D^-1 A) < 2), as CG needs.  Levels with few rows run on the
  // group's first CTA alone with block barriers; a barrier between passes on two such levels is
  // a block barrier, every other one the group's barrier.
  __device__ __forceinline__ const float* lw(int l, int a) const {
    return P.mg_w + P.mg[l].woff + (size_t)a * P.mg[l].plen + kSlack;
  }
  __device__ __forceinline__ float* lv(int l, int a) const {
    return mgws + P.mg[l].voff + (size_t)a * P.mg[l].plen + kSlack;
  }
  __device__ __forceinline__ bool solo(int l) const { return P.cs == 1 || P.mg[l].ny + 1 <= P.mg_solo_rows; }
  __device__ __forceinline__ void xsync(int a, int b) {
    if (solo(a) && solo(b))
      __syncthreads();
    else
      comm.sync();
  }
  // f(loc) for this CTA's groups of 4 nodes of level l
  template <class F>
  __device__ __forceinline__ void for_lgroups(int l, F f) const {
    int r0l = 0, Rl = 0;
    if (solo(l)) {
      Rl = rank == 0 ? P.mg[l].ny + 1 : 0;
    } else {
      slab_rows(P.mg[l].ny + 1, P.cs, rank, r0l, Rl);
    }
    const int Wl = P.mg[l].W, G4l = Wl / kGroup;
    for (int t = threadIdx.x; t < Rl * G4l; t += blockDim.x) {
      const int lr = t / G4l, g = t - lr * G4l;
      f((r0l + lr + 1) * Wl + kGroup * g);
    }
  }
  __device__ __forceinline__ void ld4f(const float* __restrict__ a, int loc, float (&v)[4]) const {
    const float4 c = *reinterpret_cast<const float4*>(a + loc);
    v[0] = c.x; v[1] = c.y; v[2] = c.z; v[3] = c.w;
  }
  __device__ __forceinline__ void st4f(float* __restrict__ a, int loc, const float (&v)[4]) const {
    *reinterpret_cast<float4*>(a + loc) = make_float4(v[0], v[1], v[2], v[3]);
  }
  // y = A_l v on a group from v's windows on the rows below, at and above it (FP32 node weights)
  template <class T>
  __device__ __forceinline__ void lstencil(int l, int loc, const float (&vl)[6], const float (&vm)[6],
                                           const float (&vh)[6], T (&y)[4]) const {
    const int Wl = P.mg[l].W;
    const float *C = lw(l, 0), *E = lw(l, 1), *N = lw(l, 2), *NE = lw(l, 3), *NW = lw(l, 4);
    float c4[4], n4[4], nb[4], ne4[4], nw4[4], e5[5];
    ld4f(C, loc, c4);
    ld4f(N, loc, n4);
    ld4f(N, loc - Wl, nb);
    ld4f(NE, loc, ne4);
    ld4f(NW, loc, nw4);
    load_ewindow(E, loc, e5);
    const float* neb = NE + loc - Wl - 1;   // NE weights of the row below, shifted left
    const float* nwb = NW + loc - Wl + 1;   // NW weights of the row below, shifted right
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float a = c4[j] * vm[j + 1];
      a = fmaf(e5[j + 1], vm[j + 2], a);
      a = fmaf(e5[j], vm[j], a);
      a = fmaf(n4[j], vh[j + 1], a);
      a = fmaf(nb[j], vl[j + 1], a);
      a = fmaf(ne4[j], vh[j + 2], a);
      a = fmaf(neb[j], vl[j], a);
      a = fmaf(nw4[j], vh[j], a);
      a = fmaf(nwb[j], vl[j + 2], a);
      y[j] = (T)a;
    }
  }
  template <class T>
  __device__ __forceinline__ void lwindows(const T* __restrict__ v, int loc, int Wl, float (&a)[6], float (&b)[6],
                                           float (&c)[6]) const {
    T t[6];
    load_window(v, loc - Wl, t);
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = (float)t[i];
    load_window(v, loc, t);
#pragma unroll
    for (int i = 0; i < 6; ++i) b[i] = (float)t[i];
    load_window(v, loc + Wl, t);
#pragma unroll
    for (int i = 0; i < 6; ++i) c[i] = (float)t[i];
  }
  // Pre-smoothing of level l from zero on f: nu = 1: u = S f = omega D^-1 f and res = f - A u in
  // one pass (u of the neighbours formed from their f); nu = 2: u = S f + S (f - A S f) in one
  // pass, then res = f - A u after a barrier.  res is 0 off the unknowns.
  template <class T>
  __device__ void mg_pre(int l, const T* __restrict__ f) {
    const int Wl = P.mg[l].W;
    const float* wd = lw(l, 5);
    float* u = lv(l, l == 0 ? 0 : 1);
    float* res = lv(l, l == 0 ? 1 : 2);
    for_lgroups(l, [&](int loc) {
      float fl[6], fm[6], fh[6], dl[6], dm[6], dh[6], y[4], uo[4], ro[4], fc[4];
      lwindows(f, loc, Wl, fl, fm, fh);
      lwindows(wd, loc, Wl, dl, dm, dh);
#pragma unroll
      for (int j = 0; j < 4; ++j) fc[j] = fm[j + 1];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        fl[i] *= dl[i];   // u = S f on the window (fl.. now hold u)
        fm[i] *= dm[i];
        fh[i] *= dh[i];
      }
      lstencil(l, loc, fl, fm, fh, y);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float rj = dm[j + 1] != 0.f ? fc[j] - y[j] : 0.f;
        uo[j] = fm[j + 1];
        if (P.mg_nu >= 2) uo[j] = fmaf(dm[j + 1], rj, uo[j]);
        ro[j] = rj;
      }
      st4f(u, loc, uo);
      if (P.mg_nu < 2) st4f(res, loc, ro);
    });
    if (P.mg_nu >= 2) {
      xsync(l, l);
      for_lgroups(l, [&](int loc) {
        float ul[6], um[6], uh[6], y[4], ro[4], dv[4];
        T fv[4];
        lwindows(u, loc, Wl, ul, um, uh);
        lstencil(l, loc, ul, um, uh, y);
        ld4f(wd, loc, dv);
        ldv(f, loc, fv);
#pragma unroll
        for (int j = 0; j < 4; ++j) ro[j] = dv[j] != 0.f ? (float)fv[j] - y[j] : 0.f;
        st4f(res, loc, ro);
      });
    }
  }
  template <class T>
  __device__ __forceinline__ void ldv(const T* __restrict__ a, int loc, T (&v)[4]) const {
    if constexpr (sizeof(T) == 8) {
      load4(a + loc, v);
    } else {
      ld4f(a, loc, v);
    }
  }
  // f_{l+1} = P^T res_l on the nodes of level l+1 (0 off its unknowns)
  __device__ void mg_restrict(int l) {
    const int c = l + 1, Wf = P.mg[l].W, nxc = P.mg[c].nx;
    const float* res = lv(l, l == 0 ? 1 : 2);
    const float* wdc = lw(c, 5);
    float* fc = lv(c, 0);
    const int Wc = P.mg[c].W;
    for_lgroups(c, [&](int loc) {
      const int J = loc / Wc - 1, I0 = loc - (J + 1) * Wc - 1;
      float dv[4], o[4];
      ld4f(wdc, loc, dv);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int I = I0 + j;
        float acc = 0.f;
        if (dv[j] != 0.f && I >= 0 && I <= nxc) {
          const float* r0 = res + (2 * J + 1) * Wf + 2 * I + 1;   // fine node (2I, 2J)
#pragma unroll
          for (int b = -1; b <= 1; ++b) {
            const float* rr = r0 + b * Wf;
            const float row = fmaf(0.5f, rr[-1] + rr[1], rr[0]);
            acc = fmaf(b == 0 ? 1.f : 0.5f, row, acc);
          }
        }
        o[j] = acc;
      }
      st4f(fc, loc, o);
    });
  }
  // coarsest level: e = mg_coarse_steps damped-Jacobi steps from zero, the last into e
  __device__ void mg_coarsest(int l) {
    const int Wl = P.mg[l].W, n = P.mg_coarse_steps;
    const float* f = lv(l, 0);
    const float* wd = lw(l, 5);
    float* bufs[2] = {lv(l, 3), lv(l, 1)};   // step k writes bufs[(n - k) % 2]: the last lands in e
    for (int k = 1; k <= n; ++k) {
      float* dst = bufs[(n - k) & 1];
      const float* src = bufs[(n - k + 1) & 1];
      for_lgroups(l, [&](int loc) {
        float fv[4], dv[4], o[4];
        ld4f(f, loc, fv);
        ld4f(wd, loc, dv);
        if (k == 1) {
#pragma unroll
          for (int j = 0; j < 4; ++j) o[j] = dv[j] * fv[j];
        } else {
          float vl[6], vm[6], vh[6], y[4];
          lwindows(src, loc, Wl, vl, vm, vh);
          lstencil(l, loc, vl, vm, vh, y);
#pragma unroll
          for (int j = 0; j < 4; ++j) o[j] = fmaf(dv[j], fv[j] - y[j], vm[j + 1]);
        }
        st4f(dst, loc, o);
      });
      xsync(l, l);
    }
  }
  // u_l += P e_{l+1} on the unknowns of level l
  __device__ void mg_prolong(int l) {
    const int c = l + 1, Wl = P.mg[l].W, Wc = P.mg[c].W;
    const float* ec = lv(c, 3);
    const float* wd = lw(l, 5);
    float* u = lv(l, l == 0 ? 0 : 1);
    for_lgroups(l, [&](int loc) {
      const int y = loc / Wl - 1, x0 = loc - (y + 1) * Wl - 1;
      float dv[4], uv[4];
      ld4f(wd, loc, dv);
      ld4f(u, loc, uv);
      const int Ja = y >> 1, Jb = (y + 1) >> 1;   // y even: Ja = Jb = y / 2
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int x = x0 + j;
        if (dv[j] == 0.f) continue;               // also every pad column
        const int Ia = x >> 1, Ib = (x + 1) >> 1;
        const float* ra = ec + (Ja + 1) * Wc + 1;
        const float* rb = ec + (Jb + 1) * Wc + 1;
        const float v = 0.25f * ((ra[Ia] + ra[Ib]) + (rb[Ia] + rb[Ib]));
        uv[j] += v;
      }
      st4f(u, loc, uv);
    });
  }
  // Post-smoothing of level l from u: nu steps out = v + S (f - A v); level 0 writes z in the CG
  // precision and returns the local (r, z); nu = 2 goes through res.
  template <class T>
  __device__ Real mg_post(int l, const T* __restrict__ f) {
    const int Wl = P.mg[l].W;
    const float* wd = lw(l, 5);
    float* u = lv(l, l == 0 ? 0 : 1);
    float* tmp = lv(l, l == 0 ? 1 : 2);
    Real rz = Real(0);
    for (int step = 0; step < P.mg_nu; ++step) {
      const bool last = step == P.mg_nu - 1;
      const float* src = step == 0 ? u : tmp;
      if (step > 0) xsync(l, l);
      for_lgroups(l, [&](int loc) {
        float vl[6], vm[6], vh[6], y[4], dv[4], o[4];
        T fv[4];
        lwindows(src, loc, Wl, vl, vm, vh);
        lstencil(l, loc, vl, vm, vh, y);
        ld4f(wd, loc, dv);
        ldv(f, loc, fv);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = fmaf(dv[j], (float)fv[j] - y[j], vm[j + 1]);
        if (!last) {
          st4f(tmp, loc, o);
        } else if (l == 0) {
          Real zv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            zv[j] = (Real)o[j];
            rz = fma((Real)fv[j], zv[j], rz);
          }
          st4(z, loc, zv);
        } else {
          st4f(lv(l, 3), loc, o);
        }
      });
    }
    return rz;
  }
  // nu = 1: the prolongation and the post-smoothing step in one pass, out = u' + S (f - A u') with
  // u' = u + P e_{l+1} formed on the window from u and the coarse e (no barrier between them);
  // level 0 writes z in the CG precision and returns the local (r, z)
  template <class T>
  __device__ Real mg_prolong_post(int l, const T* __restrict__ f) {
    const int c = l + 1, Wl = P.mg[l].W, Wc = P.mg[c].W;
    const float* ec = lv(c, 3);
    const float* wd = lw(l, 5);
    const float* u = lv(l, l == 0 ? 0 : 1);
    const float *C = lw(l, 0), *E = lw(l, 1), *N = lw(l, 2), *NE = lw(l, 3), *NW = lw(l, 4);
    Real rz = Real(0);
    for_lgroups(l, [&](int loc) {
      const int y = loc / Wl - 1, x0 = loc - (y + 1) * Wl - 1;   // first node of the group
      // A u' accumulated row by row (rows y-1, y, y+1) from the window of u' = u + P e_{l+1};
      // x0 = 4g - 1 is odd, so window column i (node x0 - 1 + i) lies between coarse columns
      // cx0 + i/2 and cx0 + (i+1)/2 (equal for even i)
      const int cx0 = (x0 - 1) >> 1;
      float acc[4] = {0.f, 0.f, 0.f, 0.f}, uc[4];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int row = loc + (r - 1) * Wl;
        float v[6], d[6];
        load_window(u, row, v);
        load_window(wd, row, d);
        const int yy = y - 1 + r, Ja = yy >> 1, Jb = (yy + 1) >> 1;
        const float* ra = ec + (Ja + 1) * Wc + 1 + cx0;
        const float* rb = ec + (Jb + 1) * Wc + 1 + cx0;
        float ca[4], cb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ca[q] = ra[q];
          cb[q] = rb[q];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const int Ia = i >> 1, Ib = (i + 1) >> 1;
          const float pv = 0.25f * ((ca[Ia] + ca[Ib]) + (cb[Ia] + cb[Ib]));
          if (d[i] != 0.f) v[i] += pv;
        }
        if (r == 0) {          // the row below: N of the node below, NE of the SW, NW of the SE node
          float nb[4];
          ld4f(N, loc - Wl, nb);
          const float* neb = NE + loc - Wl - 1;
          const float* nwb = NW + loc - Wl + 1;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            acc[j] = fmaf(nb[j], v[j + 1], fmaf(neb[j], v[j], fmaf(nwb[j], v[j + 2], acc[j])));
        } else if (r == 1) {   // the node's row: C, E of the node, E of the west neighbour
          float c4[4], e5[5];
          ld4f(C, loc, c4);
          load_ewindow(E, loc, e5);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[j] = fmaf(c4[j], v[j + 1], fmaf(e5[j + 1], v[j + 2], fmaf(e5[j], v[j], acc[j])));
            uc[j] = v[j + 1];
          }
        } else {               // the row above: the node's N, NE, NW
          float n4[4], ne4[4], nw4[4];
          ld4f(N, loc, n4);
          ld4f(NE, loc, ne4);
          ld4f(NW, loc, nw4);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            acc[j] = fmaf(n4[j], v[j + 1], fmaf(ne4[j], v[j + 2], fmaf(nw4[j], v[j], acc[j])));
        }
      }
      float dv[4], o[4];
      T fv[4];
      ld4f(wd, loc, dv);
      ldv(f, loc, fv);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = fmaf(dv[j], (float)fv[j] - acc[j], uc[j]);
      if (l == 0) {
        Real zv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          zv[j] = (Real)o[j];
          rz = fma((Real)fv[j], zv[j], rz);
        }
        st4(z, loc, zv);
      } else {
        st4f(lv(l, 3), loc, o);
      }
    });
    return rz;
  }

  // z = M^-1 r from r (every row of r visible); returns the local (r, z).  z is visible to the
  // group after the next group barrier.
  __device__ Real vcycle() {
    const int L = P.mg_levels;
    for (int l = 0; l < L - 1; ++l) {
      if (l == 0)
        mg_pre(0, r);
      else
        mg_pre(l, (const float*)lv(l, 0));
      xsync(l, l + 1);
      mg_restrict(l);
      xsync(l + 1, l + 1);
    }
    mg_coarsest(L - 1);                 // ends with a barrier
    Real rz = Real(0);
    for (int l = L - 2; l >= 0; --l) {
      if (l < L - 2) xsync(l + 1, l);   // e_{l+1} of the level above is visible
      else if (!(solo(l + 1) && solo(l))) comm.sync();
      if (P.mg_nu == 1 && P.mg_fuse) {
        if (l == 0)
          rz = mg_prolong_post(0, r);
        else
          mg_prolong_post(l, (const float*)lv(l, 0));
        continue;
      }
      mg_prolong(l);
      xsync(l, l);
      if (l == 0)
        rz = mg_post(0, r);
      else
        mg_post(l, (const float*)lv(l, 0));
    }
    return rz;
  }

  // r = b - A x (FP64, stored in the CG precision unscaled, 0 off the unknowns); the local
  // (b, b) and (r, r)
  __device__ void residual(const double* __restrict__ x, double& bb, double& rr) const {
    bb = 0.0;
    rr = 0.0;
    for_groups([&](int loc, int, int) {
      double y[4], bv[4];
      Real di[4], rv[4];
      stencil_node64<double>(x, loc, A64, loc, P.W, y);
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
      // r /= ||r||, z = M^-1 r, d = p = q = 0; (r, z)
      const bool mg = P.mg_levels > 0;
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
        if (!mg) st4(z, loc, zv);
        st4(d, loc, zero);
        st4(p, loc, zero);
        st4(q, loc, zero);
      });
      if (mg) {
        comm.sync();
        a[0] = vcycle();
      }
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
              if (!mg) v[0] = fma(rv[u][j], zv[j], v[0]);
              v[1] = fma(rv[u][j], rv[u][j], v[1]);
            }
            st4(d, loc[u], dv[u]);
            st4(r, loc[u], rv[u]);
            if (!mg) st4(z, loc[u], zv);
          }
        });
        if (mg) {
          comm.sync();
          v[0] = vcycle();
        }
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
  // (the gsrc row is 0 if null; addF - subG is added if given)
  __device__ void accumulate_g(const double* __restrict__ lam, const double* __restrict__ Tj,
                               const double* __restrict__ Tjm, const double* __restrict__ gsrc,
                               double* __restrict__ gdst, double nnorm, const double* __restrict__ addF = nullptr,
                               const double* __restrict__ subG = nullptr) const {
    const int nx = P.nx, Wp = P.W;
    const int er = min(R, P.ny - r0);
    const int nel = er > 0 ? er * nx : 0;
    const double h2 = P.h * P.h / 36.0;
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
      double gv = (gsrc ? gsrc[e] : 0.0) - term / nnorm;
      if (addF) gv += addF[e] - subG[e];
      gdst[e] = gv;
    }
  }

  // b = (C/dt) xp + src(node) on the own rows (xp padded, every row visible), 0 off the unknowns
  template <class Src>
  __device__ void build_rhs(const double* __restrict__ xp, Src src) {
    for_groups([&](int loc, int iy, int g) {
      double y[4], bv[4];
      stencil_node64<double>(xp, loc, P.mass, loc, P.W, y);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        bv[j] = (gi < 0 || P.dirichlet[gi]) ? 0.0 : fma(y[j], inv_dt, src(gi));
      }
      st4d(b, loc, bv);
    });
  }
  // x = Gs + inc on the own rows, 0 off the unknowns: the start G(u^old) plus the polynomial
  // extrapolation of the last m (1..3) increments of the correction sweep (as the stepper's
  // load_x64_increment): d_i = X_i - Fm[i], X_0 = xc (padded, the state the step propagates),
  // X_1, X_2 node vectors of earlier corrected states; inc = d0, 2 d0 - d1 or 3 (d0 - d1) + d2
  __device__ void load_increment(const double* __restrict__ Gs, int m, const double* const* Fm,
                                 const double* const* X, const double* __restrict__ xc,
                                 double* __restrict__ x) const {
    for_groups([&](int loc, int iy, int g) {
      double v[4], c[4];
      load4(xc + loc, c);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        if (gi < 0 || P.dirichlet[gi]) {
          v[j] = 0.0;
          continue;
        }
        const double d0 = c[j] - Fm[0][gi];
        double inc = d0;
        if (m == 2) inc = fma(2.0, d0, -(X[1][gi] - Fm[1][gi]));
        if (m == 3) inc = fma(3.0, d0 - (X[1][gi] - Fm[1][gi]), X[2][gi] - Fm[2][gi]);
        v[j] = Gs[gi] + inc;
      }
      st4d(x, loc, v);
    });
  }
  // Parareal correction (Eq. 4.9 / 4.14): x = xs + Fs - Gs on the own rows into the padded x and
  // the node vectors X (and Y if given); 0 off the unknowns
  __device__ void correction(const double* __restrict__ xs, const double* __restrict__ Fs,
                             const double* __restrict__ Gs, double* __restrict__ x, double* __restrict__ X,
                             double* __restrict__ Y) const {
    for_groups([&](int loc, int iy, int g) {
      double v[4], c[4];
      load4(xs + loc, c);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        v[j] = (gi >= 0 && !P.dirichlet[gi]) ? (c[j] + Fs[gi]) - Gs[gi] : 0.0;
        if (gi >= 0) {
          X[gi] = v[j];
          if (Y) Y[gi] = v[j];
        }
      }
      st4d(x, loc, v);
    });
  }
  __device__ void zero_padded(double* __restrict__ x) const {
    for_groups([&](int loc, int, int) {
      const double zero[4] = {0.0, 0.0, 0.0, 0.0};
      st4d(x, loc, zero);
    });
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
      accumulate_g(x_cur, Tj, Tjm, gsrc, gdst, (double)P.Nt);
      gsrc = gdst;
      double* t = x_prev;
      x_prev = x_cur;
      x_cur = t;
      __syncthreads();
    }
    store(x_prev, P.out_field + (size_t)s * P.Nn);
  }

  // G_pri of slice s (one step of size dtau from u_s, started from the guess u_{s+1})
  __device__ void coarse_primal(int task) {
    const int s = P.s0 + task;
    const int j = P.M * (s + 1);
    load(P.in_field + (size_t)s * P.Nn, xa);
    comm.sync();
    if (P.src_field) {
      const double* src = P.src_field + (size_t)s * P.Nn;
      build_rhs(xa, [&](int g) { return src[g]; });
    } else {
      const double qj = P.q_time[j];
      build_rhs(xa, [&](int g) { return qj * P.fload[g]; });
    }
    load(P.in_field + (size_t)(P.guess_next ? s + 1 : s) * P.Nn, xb);
    comm.sync();
    solve(xb, j);
    const double sp = pnorm_p(xb);
    store(xb, P.out_field + (size_t)s * P.Nn);
    if (threadIdx.x == 0 && rank == 0)
      P.out_aux[s] = accumulate_theta(P.in_aux[s], sp / ((double)P.Ntau * (double)P.Ne));
  }

  // G_adj of slice s; src_mode 1 / 2 one of its two Theta-free parts (as the stepper)
  __device__ void coarse_adjoint(int task) {
    const int s = P.s0 + task;
    const int kidx = P.M * s + 1;
    const int kprev = max(kidx - P.M, 0);
    const double scale = P.src_mode == 0 ? adjoint_scale(*P.Theta) : (P.src_mode == 1 ? 0.0 : 1.0);
    const double* Tk = P.hist + (size_t)kidx * P.Nn;
    const double* Tkm = P.hist + (size_t)kprev * P.Nn;
    if (P.src_mode == 2)
      zero_padded(xa);
    else
      load(P.in_field + (size_t)(s + 1) * P.Nn, xa);
    comm.sync();
    build_rhs(xa, [&](int g) { return scale * ipow(Tk[g], P.p_int - 1); });
    if (P.guess_next && P.src_mode == 0)
      load(P.in_field + (size_t)s * P.Nn, xb);
    else if (P.src_mode == 2)
      zero_padded(xb);
    else
      load(P.in_field + (size_t)(s + 1) * P.Nn, xb);
    comm.sync();
    solve(xb, kidx);
    accumulate_g(xb, Tk, Tkm, P.src_mode == 2 ? nullptr : P.in_aux + (size_t)(s + 1) * P.Ne,
                 P.out_aux + (size_t)s * P.Ne, (double)P.Ntau);
    store(xb, P.out_field + (size_t)s * P.Nn);
  }

  // Eq. 4.9 forward correction sweep (one task): u_{s+1} = G(u_s) + F[s] - G_old[s]
  __device__ void correct_primal() {
    double theta;
    if (P.in_field) {                           // u_0 taken from the guess states, copied to X[0]
      load(P.in_field, xa);
      theta = P.in_aux[0];
      comm.sync();
      store(xa, P.out_field);
      if (threadIdx.x == 0 && rank == 0) P.out_aux[0] = theta;
    } else {
      load(P.out_field, xa);
      theta = P.out_aux[0];
    }
    store(xa, hist_row(0));
    if (P.plt) {                                // G = 0 (Sec. 7, Eq. 7.2): u_{s+1} = F(u_s^old)
      for (int s = 0; s < P.Ntau; ++s) {
        load(P.F_field + (size_t)s * P.Nn, xb);
        store(xb, P.out_field + (size_t)(s + 1) * P.Nn);
        store(xb, hist_row(P.M * (s + 1)));
        if (threadIdx.x == 0 && rank == 0) P.out_aux[s + 1] = P.F_aux[s];
      }
      return;
    }
    comm.sync();
    for (int s = 0; s < P.Ntau; ++s) {
      const int j = P.M * (s + 1);
      if (P.src_field) {
        const double* src = P.src_field + (size_t)s * P.Nn;
        build_rhs(xa, [&](int g) { return src[g]; });
      } else {
        const double qj = P.q_time[j];
        build_rhs(xa, [&](int g) { return qj * P.fload[g]; });
      }
      // start G(u_s^old) plus the extrapolated increments of the last min(extrap - 1, s) steps
      const int m = min(P.extrap - 1, min(s, 3));
      if (m >= 1) {
        const double* Fm[3];
        const double* X[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < m; ++i) Fm[i] = P.F_field + (size_t)(s - 1 - i) * P.Nn;
        for (int i = 1; i < m; ++i) X[i] = P.out_field + (size_t)(s - i) * P.Nn;
        load_increment(P.G_field + (size_t)s * P.Nn, m, Fm, X, xa, xb);
      } else {
        load(P.G_field + (size_t)s * P.Nn, xb);
      }
      comm.sync();
      solve(xb, j);
      const double sp = pnorm_p(xb);
      correction(xb, P.F_field + (size_t)s * P.Nn, P.G_field + (size_t)s * P.Nn, xa,
                 P.out_field + (size_t)(s + 1) * P.Nn, hist_row(j));
      if (threadIdx.x == 0) {
        const double theta_g = accumulate_theta(theta, sp / ((double)P.Ntau * (double)P.Ne));
        theta = (theta_g + P.F_aux[s]) - P.G_aux[s];
        if (rank == 0) P.out_aux[s + 1] = theta;
      }
      comm.sync();
    }
  }

  // Eq. 4.14 reverse correction sweep (one task): v_s = G(v_{s+1}) + F[s] - G_old[s], v_Ntau = 0
  __device__ void correct_adjoint() {
    const double scale = adjoint_scale(*P.Theta);
    const int er = min(R, P.ny - r0);
    const int ne_own = er > 0 ? er * P.nx : 0;
    double* Xl = P.out_field + (size_t)P.Ntau * P.Nn;
    for_groups([&](int loc, int iy, int g) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = gnode(iy, g, j);
        if (gi >= 0) Xl[gi] = 0.0;
      }
    });
    double* Xg = P.out_aux + (size_t)P.Ntau * P.Ne + (size_t)r0 * P.nx;
    for (int t = threadIdx.x; t < ne_own; t += blockDim.x) Xg[t] = 0.0;
    if (P.plt) {                                // G = 0: v_s = F(v_{s+1}^old)
      for (int s = P.Ntau - 1; s >= 0; --s) {
        load(P.F_field + (size_t)s * P.Nn, xb);
        store(xb, P.out_field + (size_t)s * P.Nn);
        const double* Fg = P.F_aux + (size_t)s * P.Ne + (size_t)r0 * P.nx;
        double* Og = P.out_aux + (size_t)s * P.Ne + (size_t)r0 * P.nx;
        for (int t = threadIdx.x; t < ne_own; t += blockDim.x) Og[t] = Fg[t];
      }
      return;
    }
    zero_padded(xa);
    comm.sync();
    for (int s = P.Ntau - 1; s >= 0; --s) {
      const int kidx = P.M * s + 1;
      const int kprev = max(kidx - P.M, 0);
      const double* Tk = P.hist + (size_t)kidx * P.Nn;
      const double* Tkm = P.hist + (size_t)kprev * P.Nn;
      build_rhs(xa, [&](int g) { return scale * ipow(Tk[g], P.p_int - 1); });
      // start G(v_{s+1}^old) plus the extrapolated increments of the last min(extrap - 1,
      // Ntau - 1 - s) steps
      const int m = min(P.extrap - 1, min(P.Ntau - 1 - s, 3));
      if (m >= 1) {
        const double* Fm[3];
        const double* X[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < m; ++i) Fm[i] = P.F_field + (size_t)(s + 1 + i) * P.Nn;
        for (int i = 1; i < m; ++i) X[i] = P.out_field + (size_t)(s + 1 + i) * P.Nn;
        load_increment(P.G_field + (size_t)s * P.Nn, m, Fm, X, xa, xb);
      } else {
        load(P.G_field + (size_t)s * P.Nn, xb);
      }
      comm.sync();
      solve(xb, kidx);
      // g_s = g_{s+1} - (1/Ntau) term(lambda_G) + F_g[s] - G_g[s]
      accumulate_g(xb, Tk, Tkm, P.out_aux + (size_t)(s + 1) * P.Ne, P.out_aux + (size_t)s * P.Ne,
                   (double)P.Ntau, P.F_aux + (size_t)s * P.Ne, P.G_aux + (size_t)s * P.Ne);
      correction(xb, P.F_field + (size_t)s * P.Nn, P.G_field + (size_t)s * P.Nn, xa,
                 P.out_field + (size_t)s * P.Nn, nullptr);
      comm.sync();
    }
  }
};

constexpr int kStreamThreads = 512;   // one CTA per SM, 128 registers per thread

// ngroups groups of P.cs CTAs; group g runs tasks g, g + ngroups, ... < P.wide_tasks (the
// correction sweeps are one task).
template <class Real, int KIND>
__global__ void __launch_bounds__(kStreamThreads, 1) stream_kernel(const __grid_constant__ StepParams P) {
  __shared__ RedSmem rs;
  GridComm comm(P, rs);
  Streamer<Real, KIND> st(P, comm);
  const int ngroups = (int)gridDim.x / P.cs;
  for (int task = comm.gid; task < P.wide_tasks; task += ngroups) {
    if constexpr (KIND == KIND_FINE_PRI) st.fine_primal(task);
    if constexpr (KIND == KIND_FINE_ADJ) st.fine_adjoint(task);
    if constexpr (KIND == KIND_COARSE_PRI) st.coarse_primal(task);
    if constexpr (KIND == KIND_COARSE_ADJ) st.coarse_adjoint(task);
    if constexpr (KIND == KIND_CORRECT_PRI) st.correct_primal();
    if constexpr (KIND == KIND_CORRECT_ADJ) st.correct_adjoint();
    comm.sync();                           // the group's workspace is free for its next task
  }
}

// The kernels of one task kind (FP32 and FP64 CG), instantiated in stream_inst.cu.
using StreamKernel = void (*)(const StepParams);
struct StreamKernels {
  StreamKernel f32, f64;
};
StreamKernels stream_select_0();
StreamKernels stream_select_1();
StreamKernels stream_select_2();
StreamKernels stream_select_3();
StreamKernels stream_select_4();
StreamKernels stream_select_5();

}  // namespace ptg
