// stream.cu -- kernels and launch of the streamed fine propagators (stream.cuh).
#include "stream.cuh"

namespace ptg {

constexpr int kStreamThreads = 512;   // one CTA per SM, 128 registers per thread

// ngroups groups of P.cs CTAs; group g runs tasks g, g + ngroups, ... < P.wide_tasks.
template <class Real, int KIND>
__global__ void __launch_bounds__(kStreamThreads, 1) stream_kernel(const __grid_constant__ StepParams P) {
  __shared__ RedSmem rs;
  GridComm comm(P, rs);
  Streamer<Real, KIND> st(P, comm);
  const int ngroups = (int)gridDim.x / P.cs;
  for (int task = comm.gid; task < P.wide_tasks; task += ngroups) {
    if constexpr (KIND == KIND_FINE_PRI)
      st.fine_primal(task);
    else
      st.fine_adjoint(task);
    comm.sync();                           // the group's workspace is free for its next task
  }
}

cudaError_t launch_stream(const StepParams& P, int precision, int ngroups, int nthreads, cudaStream_t stream) {
  using K = void (*)(const StepParams);
  K k = nullptr;
  const bool f32 = precision == PTG_FP32_REFINE;
  if (P.kind == KIND_FINE_PRI) k = f32 ? &stream_kernel<float, KIND_FINE_PRI> : &stream_kernel<double, KIND_FINE_PRI>;
  if (P.kind == KIND_FINE_ADJ) k = f32 ? &stream_kernel<float, KIND_FINE_ADJ> : &stream_kernel<double, KIND_FINE_ADJ>;
  if (!k || ngroups < 1 || ngroups * P.cs > kMaxGrid) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(P.g_bar, 0, 4 * sizeof(unsigned) * ngroups, stream);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3((unsigned)(ngroups * P.cs), 1, 1);
  cfg.blockDim = dim3((unsigned)(nthreads < kStreamThreads ? nthreads : kStreamThreads), 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, P);
}

}  // namespace ptg
