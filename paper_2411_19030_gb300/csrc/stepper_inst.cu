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

StepKernel PTG_SELECT_NAME(PTG_TAG, PTG_KIND)(int npt, int nthreads) {
#define PTG_TRY(NT_, NPT_) \
  if (npt == NPT_ && nthreads == NT_) return &stepper_kernel<PTG_REAL, NPT_, NT_, PTG_KIND>;
  PTG_TRY(256, 2)
  PTG_TRY(256, 4)
  PTG_TRY(256, 6)
  PTG_TRY(256, 10)
  PTG_TRY(256, 12)
  PTG_TRY(512, 10)
#undef PTG_TRY
  return nullptr;
}

}  // namespace ptg
