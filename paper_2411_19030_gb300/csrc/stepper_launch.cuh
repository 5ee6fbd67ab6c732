// stepper_launch.cuh -- kernel table of the cluster stepper.
#pragma once
#include "ptg_internal.h"

namespace ptg {

using StepKernel = void (*)(const StepParams);
using BatchKernel = void (*)(const StepParams*, const int2*, int, int*);
struct StepKernels {
  StepKernel single;
  BatchKernel batch;
  StepKernel wide;      // grid-wide variant (FP64, single-task kinds, NG <= 3), else null
};

// Groups of 4 nodes per thread (NG) supported by the build; a CTA has up to 512 threads, so
// it holds up to 2048 * NG nodes.  (stepper_inst.cu instantiates the same list.)
constexpr int kStepNG[] = {1, 2, 3, 4, 5, 6};
constexpr int kNumStepNG = sizeof(kStepNG) / sizeof(kStepNG[0]);
constexpr int kStepMaxThreadsHost = 512;

// Defined by the per-(precision, kind) translation units.
#define PTG_DECLARE_SELECT(P, K) StepKernels stepper_select_##P##_##K(int ng);
PTG_DECLARE_SELECT(f32, 0) PTG_DECLARE_SELECT(f32, 1) PTG_DECLARE_SELECT(f32, 2)
PTG_DECLARE_SELECT(f32, 3) PTG_DECLARE_SELECT(f32, 4) PTG_DECLARE_SELECT(f32, 5)
PTG_DECLARE_SELECT(f64, 0) PTG_DECLARE_SELECT(f64, 1) PTG_DECLARE_SELECT(f64, 2)
PTG_DECLARE_SELECT(f64, 3) PTG_DECLARE_SELECT(f64, 4) PTG_DECLARE_SELECT(f64, 5)
#undef PTG_DECLARE_SELECT

inline StepKernels stepper_kernels_for(int precision, int kind, int ng) {
  const bool f32 = precision == PTG_FP32_REFINE;
  switch (kind) {
    case 0: return f32 ? stepper_select_f32_0(ng) : stepper_select_f64_0(ng);
    case 1: return f32 ? stepper_select_f32_1(ng) : stepper_select_f64_1(ng);
    case 2: return f32 ? stepper_select_f32_2(ng) : stepper_select_f64_2(ng);
    case 3: return f32 ? stepper_select_f32_3(ng) : stepper_select_f64_3(ng);
    case 4: return f32 ? stepper_select_f32_4(ng) : stepper_select_f64_4(ng);
    case 5: return f32 ? stepper_select_f32_5(ng) : stepper_select_f64_5(ng);
    default: return StepKernels{nullptr, nullptr, nullptr};
  }
}
inline StepKernel stepper_kernel_for(int precision, int kind, int ng) { return stepper_kernels_for(precision, kind, ng).single; }

}  // namespace ptg
