// stepper_inst.cu -- instantiates the cluster stepper for one precision and one task kind.
// Compiled once per (PTG_REAL, PTG_KIND) pair so the kernels build in parallel:
//   PTG_REAL = float (FP32 CG + FP64 refinement) or double (FP64 CG); PTG_KIND = 0..5.
#include "stepper.cuh"
#include "stepper_launch.cuh"

#ifndef PTG_REAL
#error "define PTG_REAL (float or double)"
#endif
#ifndef PTG_KIND
#error "define PTG_KIND (0..5)"
#endif
#ifndef PTG_TAG
#error "define PTG_TAG (f32 or f64)"
#endif

#define PTG_CAT3(a, b, c) a##_##b##_##c
#define PTG_SELECT_NAME(tag, kind) PTG_CAT3(stepper_select, tag, kind)

namespace ptg {

// The grid-wide (grouped) variant exists for every kind and precision, for up to 3 groups
// per thread.
template <int NG>
StepKernel wide_kernel() {
  if constexpr (NG <= 3) return &stepper_wide_kernel<PTG_REAL, NG, PTG_KIND>;
  else return nullptr;
}

StepKernels PTG_SELECT_NAME(PTG_TAG, PTG_KIND)(int ng) {
#define PTG_PAIR(NG_)                                                                                   \
  StepKernels{&stepper_kernel<PTG_REAL, NG_, PTG_KIND>, &stepper_batch_kernel<PTG_REAL, NG_, PTG_KIND>, \
              wide_kernel<NG_>()}
  switch (ng) {
    case 1: return PTG_PAIR(1);
    case 2: return PTG_PAIR(2);
    case 3: return PTG_PAIR(3);
    case 4: return PTG_PAIR(4);
    case 5: return PTG_PAIR(5);
    case 6: return PTG_PAIR(6);
    default: return StepKernels{nullptr, nullptr, nullptr};
  }
#undef PTG_PAIR
}

}  // namespace ptg
