// stepper_launch.cuh -- kernel table and launch helpers of the cluster stepper.
#pragma once
#include "ptg_internal.h"

namespace ptg {

using StepKernel = void (*)(const StepParams);

// Threads per CTA and node slots per thread supported by the build.
// (the list is repeated in stepper_inst.cu, which instantiates the kernels)
struct StepConfig {
  int nthreads, npt;
};
constexpr StepConfig kStepConfigs[] = {{256, 2}, {256, 4}, {256, 6}, {256, 10}, {256, 12}, {512, 10}};
constexpr int kNumStepConfigs = sizeof(kStepConfigs) / sizeof(kStepConfigs[0]);

// Defined by the per-(precision, kind) translation units.
#define PTG_DECLARE_SELECT(P, K) StepKernel stepper_select_##P##_##K(int npt, int nthreads);
PTG_DECLARE_SELECT(f32, 0) PTG_DECLARE_SELECT(f32, 1) PTG_DECLARE_SELECT(f32, 2)
PTG_DECLARE_SELECT(f32, 3) PTG_DECLARE_SELECT(f32, 4) PTG_DECLARE_SELECT(f32, 5)
PTG_DECLARE_SELECT(f64, 0) PTG_DECLARE_SELECT(f64, 1) PTG_DECLARE_SELECT(f64, 2)
PTG_DECLARE_SELECT(f64, 3) PTG_DECLARE_SELECT(f64, 4) PTG_DECLARE_SELECT(f64, 5)
#undef PTG_DECLARE_SELECT

inline StepKernel stepper_kernel_for(int precision, int kind, int npt, int nthreads) {
  const bool f32 = precision == PTG_FP32_REFINE;
  switch (kind) {
    case 0: return f32 ? stepper_select_f32_0(npt, nthreads) : stepper_select_f64_0(npt, nthreads);
    case 1: return f32 ? stepper_select_f32_1(npt, nthreads) : stepper_select_f64_1(npt, nthreads);
    case 2: return f32 ? stepper_select_f32_2(npt, nthreads) : stepper_select_f64_2(npt, nthreads);
    case 3: return f32 ? stepper_select_f32_3(npt, nthreads) : stepper_select_f64_3(npt, nthreads);
    case 4: return f32 ? stepper_select_f32_4(npt, nthreads) : stepper_select_f64_4(npt, nthreads);
    case 5: return f32 ? stepper_select_f32_5(npt, nthreads) : stepper_select_f64_5(npt, nthreads);
    default: return nullptr;
  }
}

}  // namespace ptg
