// stream_inst.cu -- instantiates the streamed propagator kernels of one task kind (PTG_KIND =
// 0..5) in FP32 and FP64 CG; compiled once per kind so the kernels build in parallel.
#include "stream.cuh"

#ifndef PTG_KIND
#error "define PTG_KIND (0..5)"
#endif

#define PTG_CAT2(a, b) a##_##b
#define PTG_STREAM_SELECT(kind) PTG_CAT2(stream_select, kind)

namespace ptg {

StreamKernels PTG_STREAM_SELECT(PTG_KIND)() {
  return StreamKernels{&stream_kernel<float, PTG_KIND>, &stream_kernel<double, PTG_KIND>};
}

}  // namespace ptg
