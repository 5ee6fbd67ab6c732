// ptg_device.cuh -- device-side building blocks of the cluster time stepper.
//
// Layout (one thread-block cluster per independent time-stepping system):
//   * The (ny+1) node rows of the grid are split into CS horizontal slabs, one per CTA of
//     the cluster.  CTA `rank` owns node rows [r0, r0+R).
//   * Every grid-shaped buffer uses the padded row layout of ptg_internal.h: columns
//     ix = -1 .. W-2 at offsets ix+1 with W = roundup(nx+3, 4), zeros outside the domain,
//     kSlack entries of zero slack before and after.  Node buffers that a stencil reads hold
//     local rows lr = -1..R (one halo row on each side, filled by the neighbouring CTAs
//     through distributed shared memory stores); element buffers hold element rows r0-1 ..
//     r0+R-1.  Each thread works on aligned groups of 4 consecutive nodes of a row, so a
//     9-point stencil is a handful of 16-byte loads and needs no boundary branches.
//
// Operator (Sec. 2.2): for the bilinear square element with local node order SW, SE, NE,
// NW the matrix a*Ke + b*Me has only three distinct entries: a diagonal D, an edge-neighbour
// S and an opposite-corner T.  For C/dt + K with conductivity k_e and capacity c_e:
//   D = 4k/6 + 4m,  S = -k/6 + 2m,  T = -2k/6 + m,  m = c_e h^2 / (36 dt).
// Summing the four elements around a node gives the 9-point stencil used below.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include "ptg_internal.h"

namespace ptg {
namespace cg = cooperative_groups;

constexpr int kMaxCluster = 16;
constexpr int kMaxWarps = 32;

// First device-side error wins: status code, the task kind and the time index.
__device__ __forceinline__ void record_error(DevStats* st, int code, int kind, int step) {
  if (atomicCAS(&st->status, 0, code) == 0) {
    st->fail_kind = 10 + kind;
    st->fail_step = step;
  }
}

// ---------------------------------------------------------------------------- cluster sync
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Shared scratch for reductions (static shared memory of the stepper kernel).
template <class T>
struct RedBank {
  T slot[2][kMaxCluster][4];  // [phase][source rank][value]
  T warp[kMaxWarps][4];       // per-warp partials of this CTA
  T bcast[8];                 // finalised values (double path)
};
struct RedSmem {
  RedBank<float> f;
  RedBank<double> d;
};
template <class T> __device__ __forceinline__ RedBank<T>& bank(RedSmem& rs);
template <> __device__ __forceinline__ RedBank<float>& bank<float>(RedSmem& rs) { return rs.f; }
template <> __device__ __forceinline__ RedBank<double>& bank<double>(RedSmem& rs) { return rs.d; }

struct NoPost {
  template <class T>
  __device__ __forceinline__ void operator()(T*) const {}
};

// Cluster-wide all-reduce of the first NV entries of v (NV <= 4), followed by `post`, which may
// transform them and fill the NX extra entries v[NV..NV+NX) (for example CG step lengths from
// the dot products).  Every thread of every CTA of the cluster must call it the same number of
// times; the result is bitwise identical in every thread of every CTA: the warp butterfly
// combines the same pairs in every lane, lanes of warp 0 sum the warp partials in warp order,
// and every CTA writes its partial into every CTA's slot array.  In float every warp sums the
// slots with a second butterfly (lane r holds rank r) and applies `post` itself.  In double
// (1/58 of the float rate on this chip) thread 0 sums them in rank order, applies `post` and
// broadcasts through shared memory.
// One __syncthreads and one cluster barrier per call (two __syncthreads in double); the
// cluster barrier also publishes every DSMEM store made before the call.
template <class T, int NV, int NX = 0, class Post = NoPost>
__device__ __forceinline__ void cluster_allreduce(T (&v)[NV + NX], RedSmem& rs, int& phase,
                                                  cg::cluster_group& cluster, int cs, Post post = Post()) {
  RedBank<T>& rb = bank<T>(rs);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) rb.warp[warp][i] = v[i];
  }
  __syncthreads();
  if (warp == 0 && lane < cs) {
    T s[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      s[i] = rb.warp[0][i];
      for (int w = 1; w < nwarps; ++w) s[i] += rb.warp[w][i];
    }
    T* dst = cluster.map_shared_rank(&rb.slot[phase][0][0], (unsigned)lane);
    const int me = (int)cluster.block_rank();
#pragma unroll
    for (int i = 0; i < NV; ++i) dst[me * 4 + i] = s[i];
  }
  cluster_sync_all();
  if constexpr (sizeof(T) == 4) {
    // lane r loads rank r's partial; the same butterfly in every warp of every CTA
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      T t = lane < cs ? rb.slot[phase][lane][i] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[i] = t;
    }
    post(v);
  } else {
    if (threadIdx.x == 0) {
      T t[NV + NX];
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        t[i] = rb.slot[phase][0][i];
        for (int r = 1; r < cs; ++r) t[i] += rb.slot[phase][r][i];
      }
#pragma unroll
      for (int i = NV; i < NV + NX; ++i) t[i] = T(0);
      post(t);
#pragma unroll
      for (int i = 0; i < NV + NX; ++i) rb.bcast[i] = t[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV + NX; ++i) v[i] = rb.bcast[i];
  }
  phase ^= 1;
}

// ---------------------------------------------------------------------------- slab geometry
struct Slab {
  int nx, ny;      // elements per side
  int cs, rank;    // cluster size, this CTA's rank
  int r0, R;       // first owned node row, owned rows
  int W, G;        // padded row width and groups of 4 nodes per row
  int ngroups;     // owned groups R*G
};

__device__ __forceinline__ void slab_rows(int rows_total, int cs, int rank, int& r0, int& R) {
  const int base = rows_total / cs, rem = rows_total % cs;
  r0 = rank * base + (rank < rem ? rank : rem);
  R = base + (rank < rem ? 1 : 0);
}

// Copy this CTA's first and last owned rows of a halo buffer (`buf` points at row -1, row lr at
// buf + (lr+1)*W) into the halo rows of the CTAs above and below with 16-byte DSMEM stores.
// Visibility comes from the next cluster barrier.
template <class T>
__device__ __forceinline__ void push_halos(T* buf, const Slab& sb, cg::cluster_group& cluster) {
  constexpr int V = 16 / sizeof(T);           // elements per 16-byte store
  const int nv = sb.W / V;
  if (sb.rank > 0) {
    int r0n, Rn;
    slab_rows(sb.ny + 1, sb.cs, sb.rank - 1, r0n, Rn);
    T* dst = cluster.map_shared_rank(buf, (unsigned)(sb.rank - 1));
    const uint4* s = reinterpret_cast<const uint4*>(buf + 1 * sb.W);                  // own row lr = 0
    uint4* d = reinterpret_cast<uint4*>(dst + (Rn + 1) * sb.W);                       // its halo row lr = Rn
    for (int i = threadIdx.x; i < nv; i += blockDim.x) d[i] = s[i];
  }
  if (sb.rank < sb.cs - 1) {
    T* dst = cluster.map_shared_rank(buf, (unsigned)(sb.rank + 1));
    const uint4* s = reinterpret_cast<const uint4*>(buf + sb.R * sb.W);               // own row lr = R-1
    uint4* d = reinterpret_cast<uint4*>(dst);                                        // its halo row lr = -1
    for (int i = threadIdx.x; i < nv; i += blockDim.x) d[i] = s[i];
  }
}

// x^(p-1) and x^p for an even integer p >= 2 by repeated squaring (exact operation order is
// fixed so every CTA and every run computes the same value).
__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0, b = x;
  while (e > 0) {
    if (e & 1) r *= b;
    b *= b;
    e >>= 1;
  }
  return r;
}

// ---------------------------------------------------------------------------- stencils
// 6-entry window of a row around a group: w[0] = offset b-1, w[1..4] = b..b+3, w[5] = b+4
// (b a multiple of 4).  One 16-byte load for the centre in float, two in double.
template <class T>
__device__ __forceinline__ void load_window(const T* __restrict__ x, int b, T (&w)[6]) {
  w[0] = x[b - 1];
  if constexpr (sizeof(T) == 4) {
    const float4 c = *reinterpret_cast<const float4*>(x + b);
    w[1] = c.x; w[2] = c.y; w[3] = c.z; w[4] = c.w;
  } else {
    const double2 c0 = *reinterpret_cast<const double2*>(x + b);
    const double2 c1 = *reinterpret_cast<const double2*>(x + b + 2);
    w[1] = c0.x; w[2] = c0.y; w[3] = c1.x; w[4] = c1.y;
  }
  w[5] = x[b + 4];
}

// 5-entry window of an element row: e[0] = offset b-1, e[1..4] = b..b+3 (b a multiple of 4).
__device__ __forceinline__ void load_ewindow(const float* __restrict__ w, int b, float (&e)[5]) {
  e[0] = w[b - 1];
  const float4 c = *reinterpret_cast<const float4*>(w + b);
  e[1] = c.x; e[2] = c.y; e[3] = c.z; e[4] = c.w;
}

__device__ __forceinline__ void load4(const double* __restrict__ p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// y = A x for the 4 nodes of a group, FP64 per-node weights (global memory).
// x: node buffer (rows -1..R); loc0: offset of the group's first node in x;
// go: offset of the same node in the padded global node arrays; W: row width.
template <class T>
__device__ __forceinline__ void stencil_node64(const T* __restrict__ x, int loc0, const NodeWeights& nw, int go, int W,
                                               double (&y)[4]) {
  T xl[6], xm[6], xh[6];
  load_window(x, loc0 - W, xl);
  load_window(x, loc0, xm);
  load_window(x, loc0 + W, xh);
  double C[4], No[4], Nb[4], NEo[4], NWo[4];
  load4(nw.C + go, C);
  load4(nw.N + go, No);
  load4(nw.N + go - W, Nb);
  load4(nw.NE + go, NEo);
  load4(nw.NW + go, NWo);
  double E[5];
  E[0] = nw.E[go - 1];
  {
    double e4[4];
    load4(nw.E + go, e4);
    E[1] = e4[0]; E[2] = e4[1]; E[3] = e4[2]; E[4] = e4[3];
  }
  const double* neb = nw.NE + go - W - 1;      // NE weights of the row below, shifted left
  const double* nwb = nw.NW + go - W + 1;      // NW weights of the row below, shifted right
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    double a = C[j] * (double)xm[j + 1];
    a = fma(E[j + 1], (double)xm[j + 2], a);   // east
    a = fma(E[j], (double)xm[j], a);           // west  = east weight of the west neighbour
    a = fma(No[j], (double)xh[j + 1], a);      // north
    a = fma(Nb[j], (double)xl[j + 1], a);      // south = north weight of the south neighbour
    a = fma(NEo[j], (double)xh[j + 2], a);     // north-east
    a = fma(neb[j], (double)xl[j], a);         // south-west = NE weight of the SW neighbour
    a = fma(NWo[j], (double)xh[j], a);         // north-west
    a = fma(nwb[j], (double)xl[j + 2], a);     // south-east = NW weight of the SE neighbour
    y[j] = a;
  }
}

// y = A z for the 4 nodes of a group, FP32 element weights (D, S, T) in shared memory.
// For the node at window position c = j+1: elements a, b below-left / below-right and c, d
// above-left / above-right, i.e. element windows lower[j], lower[j+1], upper[j], upper[j+1].
// no_lo / no_hi: the node row below / above is left out (taken as zero), which applies the
// slab's diagonal block of the operator on its first / last row.
__device__ __forceinline__ void stencil_elem32(const float* __restrict__ z, const float* __restrict__ wd,
                                               const float* __restrict__ ws, const float* __restrict__ wt, int loc0,
                                               int W, float (&y)[4], bool no_lo = false, bool no_hi = false) {
  float zl[6], zm[6], zh[6];
  if (no_lo) {
#pragma unroll
    for (int i = 0; i < 6; ++i) zl[i] = 0.f;
  } else {
    load_window(z, loc0 - W, zl);
  }
  load_window(z, loc0, zm);
  if (no_hi) {
#pragma unroll
    for (int i = 0; i < 6; ++i) zh[i] = 0.f;
  } else {
    load_window(z, loc0 + W, zh);
  }
  float dl[5], sl[5], tl[5], du[5], su[5], tu[5];
  const int el = loc0 - W, eu = loc0;   // element windows share the node buffers' row offsets
  load_ewindow(wd, el, dl);
  load_ewindow(ws, el, sl);
  load_ewindow(wt, el, tl);
  load_ewindow(wd, eu, du);
  load_ewindow(ws, eu, su);
  load_ewindow(wt, eu, tu);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float Da = dl[j], Db = dl[j + 1], Dc = du[j], Dd = du[j + 1];
    const float Sa = sl[j], Sb = sl[j + 1], Sc = su[j], Sd = su[j + 1];
    float a = ((Da + Db) + (Dc + Dd)) * zm[j + 1];
    a = fmaf(Sa + Sc, zm[j], a);           // west:  shared by a, c
    a = fmaf(Sb + Sd, zm[j + 2], a);       // east:  shared by b, d
    a = fmaf(Sa + Sb, zl[j + 1], a);       // south: shared by a, b
    a = fmaf(Sc + Sd, zh[j + 1], a);       // north: shared by c, d
    a = fmaf(tl[j], zl[j], a);             // south-west corner of a
    a = fmaf(tl[j + 1], zl[j + 2], a);     // south-east corner of b
    a = fmaf(tu[j], zh[j], a);             // north-west corner of c
    a = fmaf(tu[j + 1], zh[j + 2], a);     // north-east corner of d
    y[j] = a;
  }
}

// Eq. 4.7, one element over the contiguous steps ja..jb (ja <= jb): the sum over j of
//   lambda_j,e^T ( dke Ke T_j,e + dce Me (T_j - T_{j-1})_e ),
// with dce already divided by the step size and Me = (h^2/36)[4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4],
// Ke = (1/6)[4 -1 -2 -1; -1 4 -1 -2; -2 -1 4 -1; -1 -2 -1 4] in the local order SW, SE, NE, NW.
// g0 is the element's SW node, nn = nx + 1, Nn the node count; lambda_j is row j - j0 of lam and
// T_j row j - hist_j0 of T.  T_{j-1} is carried in registers, so each step reads lambda_j and T_j
// once.  The capacity term is evaluated only when has_dc is set.
__device__ __forceinline__ double sens_element_sum(int g0, int nn, int Nn, double h2, double dke, double dce,
                                                   bool has_dc, const double* __restrict__ lam, int j0,
                                                   const double* __restrict__ T, int hist_j0, int ja, int jb) {
  double acc = 0.0;
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
  return acc;
}

}  // namespace ptg
