// stream.cu -- launch of the streamed propagators (stream.cuh); the kernels are instantiated
// per task kind in stream_inst.cu.
#include "stream.cuh"

namespace ptg {

cudaError_t launch_stream(const StepParams& P, int precision, int ngroups, int nthreads, cudaStream_t stream) {
  StreamKernels ks{nullptr, nullptr};
  switch (P.kind) {
    case KIND_FINE_PRI: ks = stream_select_0(); break;
    case KIND_COARSE_PRI: ks = stream_select_1(); break;
    case KIND_CORRECT_PRI: ks = stream_select_2(); break;
    case KIND_FINE_ADJ: ks = stream_select_3(); break;
    case KIND_COARSE_ADJ: ks = stream_select_4(); break;
    case KIND_CORRECT_ADJ: ks = stream_select_5(); break;
    default: break;
  }
  const StreamKernel k = precision == PTG_FP32_REFINE ? ks.f32 : ks.f64;
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
