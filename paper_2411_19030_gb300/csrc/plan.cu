// plan.cu -- launch of the cluster stepper and occupancy queries for plan selection.
#include "stepper_launch.cuh"

namespace ptg {

static cudaError_t configure(StepKernel k, int cs, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cs > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

static void cluster_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int nclusters, int cs, int nthreads,
                           size_t smem, cudaStream_t stream) {
  cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * cs), 1, 1);
  cfg.blockDim = dim3((unsigned)nthreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

cudaError_t launch_stepper(const StepParams& P, const Plan& plan, int precision, int ntasks, cudaStream_t stream) {
  StepKernel k = stepper_kernel_for(precision, P.kind, plan.ng);
  if (!k) return cudaErrorInvalidConfiguration;
  cudaError_t e = configure(k, plan.cs, plan.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(cfg, attr, ntasks, plan.cs, plan.nthreads, plan.smem, stream);
  return cudaLaunchKernelEx(&cfg, k, P);
}

cudaError_t query_stepper_plan(int nx, int ny, int precision, int kind, int cs, int ng, int nthreads, Plan* plan) {
  StepKernel k = stepper_kernel_for(precision, kind, ng);
  if (!k || nthreads < 32 || nthreads > kStepMaxThreadsHost || nthreads % 32) return cudaErrorInvalidConfiguration;
  plan->cs = cs;
  plan->nthreads = nthreads;
  plan->ng = ng;
  plan->rmax = (ny + 1 + cs - 1) / cs;
  plan->smem = stepper_smem_bytes(nx, plan->rmax, precision == PTG_FP32_REFINE ? 4 : 8);
  plan->max_active_clusters = 0;
  if (plan->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = configure(k, cs, plan->smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(cfg, attr, 64, cs, nthreads, plan->smem, 0);
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
  plan->max_active_clusters = n;
  return e;
}

}  // namespace ptg
