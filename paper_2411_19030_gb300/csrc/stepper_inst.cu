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

StepKernel PTG_SELECT_NAME(PTG_TAG, PTG_KIND)(int ng) {
  switch (ng) {
    case 1: return &stepper_kernel<PTG_REAL, 1, PTG_KIND>;
    case 2: return &stepper_kernel<PTG_REAL, 2, PTG_KIND>;
    case 3: return &stepper_kernel<PTG_REAL, 3, PTG_KIND>;
    case 4: return &stepper_kernel<PTG_REAL, 4, PTG_KIND>;
    case 5: return &stepper_kernel<PTG_REAL, 5, PTG_KIND>;
    case 6: return &stepper_kernel<PTG_REAL, 6, PTG_KIND>;
    default: return nullptr;
  }
}

}  // namespace ptg
