// comm.cuh -- how the CTAs that share one linear system talk to each other.
//
// The stepper (stepper.cuh) needs four collective operations: an all-reduce of a few
// scalars, the exchange of the first and last owned node rows with the neighbouring slabs
// (halo rows), a barrier, and the broadcast of the two-level preconditioner's restricted
// partials.  Two implementations:
//
//   ClusterComm  one thread-block cluster (up to 16 CTAs): distributed shared memory stores
//                and the hardware cluster barrier.  Used wherever several independent
//                systems run side by side (one cluster each).
//   GridComm     groups of G CTAs of one cooperative launch (up to kMaxGrid CTAs in all, one
//                per SM), each group running one system at a time: global memory and a
//                counting barrier per group.  Used for a single system whose solves are bound
//                by the FP64 pipe (1/58 of the FP32 rate on this chip), spread over every SM
//                instead of one cluster, and for grids whose slabs do not fit 16 CTAs.
//
// Both produce bitwise identical reductions in every CTA (fixed summation orders).
#pragma once
#include "ptg_device.cuh"

namespace ptg {

constexpr long kGridSpinLimit = 1L << 20; // polls of a grid barrier before it reports PTG_ETIMEOUT

// ---------------------------------------------------------------------------- cluster
struct ClusterComm {
  cg::cluster_group cl;
  RedSmem& rs;
  int phase = 0;

  __device__ ClusterComm(RedSmem& rs_) : cl(cg::this_cluster()), rs(rs_) {}
  __device__ int rank() const { return (int)cl.block_rank(); }
  __device__ void sync() { cluster_sync_all(); }

  template <class T, int NV, int NX, class Post>
  __device__ void allreduce(T (&v)[NV + NX], int cs, Post post) {
    cluster_allreduce<T, NV, NX, Post>(v, rs, phase, cl, cs, post);
  }
  // own first / last rows into the neighbours' halo rows; visible after the next barrier
  template <class T>
  __device__ void push_halos(T* buf, const Slab& sb) {
    ptg::push_halos(buf, sb, cl);
  }
  // The same for a buffer on the 2h level of the three-level cycle: rows of W1 floats, R1 owned
  // rows here, R1b owned rows in the CTA below (whose halo row lr = R1b receives row 0).
  __device__ void push_halos_rows(float* buf, int W1, int R1, int R1b, int rank, int cs) {
    const int nv = W1 / 4;
    if (rank > 0) {
      float* dst = cl.map_shared_rank(buf, (unsigned)(rank - 1));
      const uint4* s = reinterpret_cast<const uint4*>(buf + 1 * W1);
      uint4* d = reinterpret_cast<uint4*>(dst + (R1b + 1) * W1);
      for (int i = threadIdx.x; i < nv; i += blockDim.x) d[i] = s[i];
    }
    if (rank < cs - 1) {
      float* dst = cl.map_shared_rank(buf, (unsigned)(rank + 1));
      const uint4* s = reinterpret_cast<const uint4*>(buf + R1 * W1);
      uint4* d = reinterpret_cast<uint4*>(dst);
      for (int i = threadIdx.x; i < nv; i += blockDim.x) d[i] = s[i];
    }
  }
  // Edge rows sent straight from registers: the thread holding columns [col, col+4) of the
  // owned row lr (0 or R-1) stores them into the neighbour's two-row buffer `edge` ([0]: the
  // row below that CTA's slab, [1]: the row above); visible after the next barrier.
  __device__ void begin_edges() {}
  template <class T>
  __device__ void put_edge(T* edge, int lr, int col, const T (&v)[4], const Slab& sb) {
    if (lr == 0 && sb.rank > 0) {
      T* d = cl.map_shared_rank(edge, (unsigned)(sb.rank - 1)) + sb.W + col;
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = v[j];
    }
    if (lr == sb.R - 1 && sb.rank < sb.cs - 1) {
      T* d = cl.map_shared_rank(edge, (unsigned)(sb.rank + 1)) + col;
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = v[j];
    }
  }
  template <class T>
  __device__ void end_edges(T*, const Slab&) {}
  // a 16-byte chunk of restricted partials, written at offset dst of every rank's slot array;
  // the 16 lanes `sub` = 0..15 of a half-warp share the destinations
  __device__ void publish_tl(float* slot, int dst, const float4& chunk, int sub, int cs) {
    for (int q = sub; q < cs; q += 16) *reinterpret_cast<float4*>(cl.map_shared_rank(slot + dst, (unsigned)q)) = chunk;
  }
  __device__ const float* tl_slots(const float* local) const { return local; }
  __device__ float4 tl_load4(const float* slots, int idx) const {
    return *reinterpret_cast<const float4*>(slots + idx);
  }
};

// ---------------------------------------------------------------------------- grid
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The CTAs of a cooperative launch form groups of G = P.cs consecutive CTAs; each group runs
// one system at a time.  Reduction partials, halo rows and two-level partials are indexed by
// the global block index (every group owns its range); the barrier has one set of counters per
// group.
struct GridComm {
  const StepParams& P;
  RedSmem& rs;
  int phase = 0;
  const int G;                   // CTAs of the group
  const int gid;                 // group index
  const int base;                // first block of the group
  // halo rows published by push_halos and pulled in after the next barrier; pushes alternate
  // between two slot sets, so a CTA that has passed a barrier never overwrites slots that a
  // slower CTA of the group may still be pulling from the push before it
  unsigned char* pending_lo = nullptr;   // where the row below the slab goes (null: nothing pending)
  unsigned char* pending_hi = nullptr;   // where the row above goes
  int pending_bytes = 0;         // bytes of one row
  int hset = 0;                  // slot set of the latest push
  unsigned epoch = 0;            // barriers this CTA has passed in the launch

  __device__ GridComm(const StepParams& P_, RedSmem& rs_)
      : P(P_), rs(rs_), G(P_.cs), gid((int)blockIdx.x / P_.cs), base(((int)blockIdx.x / P_.cs) * P_.cs) {}
  __device__ int rank() const { return (int)blockIdx.x - base; }

  // Counting barrier over the CTAs of the group (co-resident: cooperative launch).  The group's
  // arrival count (zeroed before the launch) only grows: thread 0 of each CTA adds 1 with release
  // semantics, which publishes the CTA's global writes ordered before it by the block barrier, and
  // polls with acquire loads until the count reaches G times the barriers passed, which makes
  // every other CTA's writes before its arrival visible.  One global round trip after the last
  // arrival; no reset.  A wait that reaches P.wait_limit polls (kGridSpinLimit if not positive)
  // records PTG_ETIMEOUT and returns; once any CTA has recorded it (the group's broken flag,
  // P.g_bar[4 gid + 2]), every later wait returns at once, so a broken launch ends quickly with
  // the error instead of waiting out every barrier.
  __device__ void barrier() {
    __syncthreads();
    if (G == 1) {                // a group of one CTA: the block barrier orders its global accesses
      pull_halos();
      return;
    }
    if (threadIdx.x == 0) {
      unsigned* count = P.g_bar + 4 * gid;
      unsigned* broken = count + 2;
      ++epoch;
      const unsigned target = epoch * (unsigned)G;
      __threadfence();
      red_release_add_gpu(count, 1u);
      const long long limit = P.wait_limit > 0 ? P.wait_limit : (long long)kGridSpinLimit;
      long long spins = 0;
      while ((int)(ld_acquire_gpu(count) - target) < 0) {
        if ((++spins & 255) == 0 && ld_acquire_gpu(broken) != 0u) break;
        if (spins >= limit) {
          record_error(P.stats, PTG_ETIMEOUT, P.stats_kind, -1);
          atomicExch(broken, 1u);
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    pull_halos();
  }
  __device__ void sync() { barrier(); }

  template <class T, int NV, int NX, class Post>
  __device__ void allreduce(T (&v)[NV + NX], int /*cs*/, Post post) {
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
    double* slots = P.g_red + (size_t)phase * kMaxGrid * 4;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        T s = rb.warp[0][i];
        for (int w = 1; w < nwarps; ++w) s += rb.warp[w][i];
        slots[(int)blockIdx.x * 4 + i] = (double)s;  // exact for T = float too
      }
    }
    barrier();
    if constexpr (sizeof(T) == 4) {
      // every warp: lane-strided sums over the ranks, then the same butterfly
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        T t = T(0);
        for (int r = lane; r < G; r += 32) t += (T)__ldcg(slots + (base + r) * 4 + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        v[i] = t;
      }
      post(v);
    } else {
      // warp 0 sums (lane-strided, then the butterfly), thread 0 applies `post` and
      // broadcasts: one lane of FP64 work for the divisions instead of every thread
      if (warp == 0) {
        T t[NV + NX];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          T a = T(0);
          for (int r = lane; r < G; r += 32) a += (T)__ldcg(slots + (base + r) * 4 + i);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          t[i] = a;
        }
        if (lane == 0) {
#pragma unroll
          for (int i = NV; i < NV + NX; ++i) t[i] = T(0);
          post(t);
#pragma unroll
          for (int i = 0; i < NV + NX; ++i) rb.bcast[i] = t[i];
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < NV + NX; ++i) v[i] = rb.bcast[i];
    }
    phase ^= 1;
  }

  __device__ size_t halo_slot(int set, int block) const {
    return ((size_t)set * kMaxGrid + (size_t)block) * 2 * (size_t)P.g_halo_row_bytes;
  }
  // Publish the own first and last rows (local rows 0 and R-1 of buf, which points at row -1)
  // to this CTA's two global halo slots of the next set; the neighbours pull them after the
  // next barrier.
  template <class T>
  __device__ void push_halos(T* buf, const Slab& sb) {
    const int nb = sb.W * (int)sizeof(T);           // bytes per row, a multiple of 16
    hset ^= 1;
    unsigned char* out = reinterpret_cast<unsigned char*>(P.g_halo) + halo_slot(hset, (int)blockIdx.x);
    const uint4* s0 = reinterpret_cast<const uint4*>(buf + 1 * sb.W);
    const uint4* s1 = reinterpret_cast<const uint4*>(buf + sb.R * sb.W);
    uint4* d0 = reinterpret_cast<uint4*>(out);
    uint4* d1 = reinterpret_cast<uint4*>(out + P.g_halo_row_bytes);
    for (int i = threadIdx.x; i < nb / 16; i += blockDim.x) {
      d0[i] = s0[i];
      d1[i] = s1[i];
    }
    __threadfence();                                // each writer orders its own stores
    pending_lo = reinterpret_cast<unsigned char*>(buf);
    pending_hi = reinterpret_cast<unsigned char*>(buf + (sb.R + 1) * sb.W);
    pending_bytes = nb;
  }
  // 2h-level rows (see ClusterComm::push_halos_rows) through the global halo slots.
  __device__ void push_halos_rows(float* buf, int W1, int R1, int /*R1b*/, int /*rank*/, int /*cs*/) {
    const int nb = W1 * (int)sizeof(float);
    hset ^= 1;
    unsigned char* out = reinterpret_cast<unsigned char*>(P.g_halo) + halo_slot(hset, (int)blockIdx.x);
    const uint4* s0 = reinterpret_cast<const uint4*>(buf + 1 * W1);
    const uint4* s1 = reinterpret_cast<const uint4*>(buf + R1 * W1);
    uint4* d0 = reinterpret_cast<uint4*>(out);
    uint4* d1 = reinterpret_cast<uint4*>(out + P.g_halo_row_bytes);
    for (int i = threadIdx.x; i < nb / 16; i += blockDim.x) {
      d0[i] = s0[i];
      d1[i] = s1[i];
    }
    __threadfence();
    pending_lo = reinterpret_cast<unsigned char*>(buf);
    pending_hi = reinterpret_cast<unsigned char*>(buf + (R1 + 1) * W1);
    pending_bytes = nb;
  }
  // Edge rows from registers (see ClusterComm::put_edge): into this CTA's slots of the next set.
  __device__ void begin_edges() { hset ^= 1; }
  template <class T>
  __device__ void put_edge(T*, int lr, int col, const T (&v)[4], const Slab& sb) {
    unsigned char* out = reinterpret_cast<unsigned char*>(P.g_halo) + halo_slot(hset, (int)blockIdx.x);
    if (lr == 0) {
      T* d = reinterpret_cast<T*>(out) + col;
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = v[j];
    }
    if (lr == sb.R - 1) {
      T* d = reinterpret_cast<T*>(out + P.g_halo_row_bytes) + col;
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = v[j];
    }
    __threadfence();                                // each writer orders its own stores
  }
  template <class T>
  __device__ void end_edges(T* edge, const Slab& sb) {
    pending_lo = reinterpret_cast<unsigned char*>(edge);
    pending_hi = reinterpret_cast<unsigned char*>(edge + sb.W);
    pending_bytes = sb.W * (int)sizeof(T);
  }
  // After a barrier: the neighbours' last / first rows into the local halo rows -1 and R.
  __device__ void pull_halos() {
    if (!pending_lo) return;
    const unsigned char* hb = reinterpret_cast<const unsigned char*>(P.g_halo);
    const size_t rb = P.g_halo_row_bytes;
    const int n16 = pending_bytes / 16;
    uint4* lo = reinterpret_cast<uint4*>(pending_lo);   // row -1
    uint4* hi = reinterpret_cast<uint4*>(pending_hi);   // row R
    const int r = rank(), b = (int)blockIdx.x;
    if (r > 0) {
      const uint4* src = reinterpret_cast<const uint4*>(hb + halo_slot(hset, b - 1) + rb);
      for (int i = threadIdx.x; i < n16; i += blockDim.x) lo[i] = __ldcg(src + i);
    }
    if (r < G - 1) {
      const uint4* src = reinterpret_cast<const uint4*>(hb + halo_slot(hset, b + 1));
      for (int i = threadIdx.x; i < n16; i += blockDim.x) hi[i] = __ldcg(src + i);
    }
    pending_lo = pending_hi = nullptr;
    __syncthreads();
  }

  // the partials live in one global array read by every CTA of the group after the barrier
  // (dst is rank-relative; the group's range starts at its first block)
  __device__ void publish_tl(float* /*slot*/, int dst, const float4& chunk, int sub, int /*cs*/) {
    if (sub == 0) {
      *reinterpret_cast<float4*>(P.g_tl + (size_t)base * tl_ncp() + dst) = chunk;
      __threadfence();
    }
  }
  __device__ int tl_ncp() const { return coarse_row_stride(P.nax) * P.nay; }
  __device__ const float* tl_slots(const float* /*local*/) const { return P.g_tl + (size_t)base * tl_ncp(); }
  __device__ float4 tl_load4(const float* slots, int idx) const {
    return __ldcg(reinterpret_cast<const float4*>(slots + idx));
  }
};

}  // namespace ptg
