// ptg_device.cuh -- device-side building blocks of the cluster time stepper.
//
// Layout (one thread-block cluster per independent time-stepping system):
//   * The (ny+1) node rows of the grid are split into CS horizontal slabs, one per CTA of
//     the cluster.  CTA `rank` owns node rows [r0, r0+R).
//   * Node vectors that a stencil reads live in shared memory with one halo row above and
//     below and one zero pad column on each side: local row lr in [-1, R], column ix in
//     [-1, nx+1], index loc = (lr+1)*W + (ix+1) with W = nx+3.  Halo rows are filled by the
//     neighbouring CTAs through distributed shared memory (DSMEM) stores.
//   * Element weights of the 9-point operator live in shared memory for element rows
//     [r0-1, r0+R-1] and columns [-1, nx], index eloc = (ler+1)*EW + (ex+1), EW = nx+2,
//     with zeros outside the domain, so the stencil needs no boundary branches.
//
// Operator (Sec. 2.2): for the bilinear square element with local node order SW, SE, NE,
// NW the matrix a*Ke + b*Me has only three distinct entries: a diagonal D, an edge-neighbour
// S and an opposite-corner T.  For C/dt + K with conductivity k_e and capacity c_e:
//   D = 4k/6 + 4m,  S = -k/6 + 2m,  T = -2k/6 + m,  m = c_e h^2 / (36 dt).
// Summing the four elements around a node gives the 9-point stencil used below.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>

namespace ptg {
namespace cg = cooperative_groups;

constexpr int kMaxCluster = 16;
constexpr int kMaxWarps = 32;

// ---------------------------------------------------------------------------- cluster sync
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Shared scratch for reductions (static shared memory of the stepper kernel).
struct RedSmem {
  double slot[2][kMaxCluster][4];  // [phase][source rank][value]
  double warp[kMaxWarps][4];       // per-warp partials of this CTA
};

// Cluster-wide all-reduce of NV doubles.  Every thread of every CTA of the cluster must
// call it (the same number of times).  The result is bitwise identical in every thread of
// every CTA: the warp butterfly combines the same pairs in every lane, the CTA partials are
// written by each CTA into every CTA's slot array, and every thread sums the slots in rank
// order.  One __syncthreads and one cluster barrier per call.
template <int NV>
__device__ __forceinline__ void cluster_allreduce(double (&v)[NV], RedSmem& rs, int& phase,
                                                  cg::cluster_group& cluster, int cs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) rs.warp[warp][i] = v[i];
  }
  __syncthreads();
  if (warp == 0) {
    double s[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      s[i] = lane < nwarps ? rs.warp[lane][i] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
    }
    if (lane < cs) {
      double* dst = cluster.map_shared_rank(&rs.slot[phase][0][0], (unsigned)lane);
      const int me = (int)cluster.block_rank();
#pragma unroll
      for (int i = 0; i < NV; ++i) dst[me * 4 + i] = s[i];
    }
  }
  cluster_sync_all();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (int r = 0; r < cs; ++r) t += rs.slot[phase][r][i];
    v[i] = t;
  }
  phase ^= 1;
}

// ---------------------------------------------------------------------------- slab geometry
struct Slab {
  int nx, ny;      // elements per side
  int cs, rank;    // cluster size, this CTA's rank
  int r0, R;       // first owned node row, owned rows
  int W, EW;       // smem row strides of node and element buffers
  int nown;        // owned nodes R*(nx+1)
};

__device__ __forceinline__ void slab_rows(int rows_total, int cs, int rank, int& r0, int& R) {
  const int base = rows_total / cs, rem = rows_total % cs;
  r0 = rank * base + (rank < rem ? rank : rem);
  R = base + (rank < rem ? 1 : 0);
}

// Push this CTA's first and last owned rows of `buf` into the halo rows of the CTAs above
// and below (DSMEM stores).  Visibility comes from the next cluster barrier.
template <class T>
__device__ __forceinline__ void push_halos(T* buf, const Slab& sb, cg::cluster_group& cluster) {
  const int nn = sb.nx + 1;
  if (sb.rank > 0) {
    int r0n, Rn;
    slab_rows(sb.ny + 1, sb.cs, sb.rank - 1, r0n, Rn);
    T* dst = cluster.map_shared_rank(buf, (unsigned)(sb.rank - 1));
    const T* src = buf + 1 * sb.W + 1;              // own row lr = 0
    T* d = dst + (Rn + 1) * sb.W + 1;              // neighbour's halo row lr = Rn
    for (int ix = threadIdx.x; ix < nn; ix += blockDim.x) d[ix] = src[ix];
  }
  if (sb.rank < sb.cs - 1) {
    T* dst = cluster.map_shared_rank(buf, (unsigned)(sb.rank + 1));
    const T* src = buf + sb.R * sb.W + 1;           // own row lr = R-1
    T* d = dst + 0 * sb.W + 1;                      // neighbour's halo row lr = -1
    for (int ix = threadIdx.x; ix < nn; ix += blockDim.x) d[ix] = src[ix];
  }
}

// ---------------------------------------------------------------------------- stencils
// y = sum over the 4 elements around the node of (D, S, T)-weighted node values.
// wd/ws/wt point at element (ler = -1, ex = -1) of a padded element array with row stride EW.
template <class T, class W_>
__device__ __forceinline__ T stencil9(const T* __restrict__ x, const W_* __restrict__ wd, const W_* __restrict__ ws,
                                      const W_* __restrict__ wt, int loc, int eloc, int W, int EW) {
  // elements around node (lr, ix): a = (lr-1, ix-1), b = (lr-1, ix), c = (lr, ix-1), d = (lr, ix)
  const int ea = eloc - EW - 1, eb = eloc - EW, ec = eloc - 1, ed = eloc;
  const T Da = (T)wd[ea], Db = (T)wd[eb], Dc = (T)wd[ec], Dd = (T)wd[ed];
  const T Sa = (T)ws[ea], Sb = (T)ws[eb], Sc = (T)ws[ec], Sd = (T)ws[ed];
  const T Ta = (T)wt[ea], Tb = (T)wt[eb], Tc = (T)wt[ec], Td = (T)wt[ed];
  T y = ((Da + Db) + (Dc + Dd)) * x[loc];
  y = fma(Sa + Sc, x[loc - 1], y);        // west:  shared by a, c
  y = fma(Sb + Sd, x[loc + 1], y);        // east:  shared by b, d
  y = fma(Sa + Sb, x[loc - W], y);        // south: shared by a, b
  y = fma(Sc + Sd, x[loc + W], y);        // north: shared by c, d
  y = fma(Ta, x[loc - W - 1], y);         // south-west corner of a
  y = fma(Tb, x[loc - W + 1], y);         // south-east corner of b
  y = fma(Tc, x[loc + W - 1], y);         // north-west corner of c
  y = fma(Td, x[loc + W + 1], y);         // north-east corner of d
  return y;
}

// Consistent-mass apply with element weights m_e (= c_e h^2/36): per element (4, 2, 1) pattern.
__device__ __forceinline__ double mass9(const double* __restrict__ x, const double* __restrict__ m, int loc, int eloc,
                                        int W, int EW) {
  const int ea = eloc - EW - 1, eb = eloc - EW, ec = eloc - 1, ed = eloc;
  const double ma = m[ea], mb = m[eb], mc = m[ec], md = m[ed];
  double y = 4.0 * ((ma + mb) + (mc + md)) * x[loc];
  y = fma(2.0 * (ma + mc), x[loc - 1], y);
  y = fma(2.0 * (mb + md), x[loc + 1], y);
  y = fma(2.0 * (ma + mb), x[loc - W], y);
  y = fma(2.0 * (mc + md), x[loc + W], y);
  y = fma(ma, x[loc - W - 1], y);
  y = fma(mb, x[loc - W + 1], y);
  y = fma(mc, x[loc + W - 1], y);
  y = fma(md, x[loc + W + 1], y);
  return y;
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

}  // namespace ptg
