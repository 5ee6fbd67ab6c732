// plan.cu -- launches of the cluster stepper (single task set and persistent multi-design) and
// occupancy queries for plan selection.
#include <map>
#include <mutex>
#include <unordered_map>
#include "stepper_launch.cuh"

namespace ptg {

// Function attributes are set once per (device, kernel) (and raised when a larger shared-memory
// footprint is requested), so launches made after a warm-up call no attribute API and can be
// captured into a CUDA graph.
cudaError_t configure_kernel(const void* k, size_t smem, bool cluster) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({dev, k});
  if (it != done.end() && it->second >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  done[{dev, k}] = smem;
  return cudaSuccess;
}

static cudaError_t configure(const void* k, int cs, size_t smem) {
  (void)cs;
  return configure_kernel(k, smem, true);
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
  if (plan.wide) {
    // one system over a cooperative grid: every CTA must be resident (the grid barrier waits
    // for all of them); the barrier's count and generation start at zero
    StepKernel k = stepper_kernels_for(precision, P.kind, plan.ng).wide;
    const int ngroups = plan.max_active_clusters < ntasks ? plan.max_active_clusters : ntasks;
    if (!k || ngroups < 1 || ngroups * plan.cs > kMaxGrid || P.wide_tasks != ntasks) return cudaErrorInvalidConfiguration;
    cudaError_t e = configure_kernel((const void*)k, plan.smem, false);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(P.g_bar, 0, 4 * sizeof(unsigned) * ngroups, stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(ngroups * plan.cs), 1, 1);
    cfg.blockDim = dim3((unsigned)plan.nthreads, 1, 1);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, P);
  }
  StepKernel k = stepper_kernel_for(precision, P.kind, plan.ng);
  if (!k) return cudaErrorInvalidConfiguration;
  cudaError_t e = configure((const void*)k, plan.cs, plan.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(cfg, attr, ntasks, plan.cs, plan.nthreads, plan.smem, stream);
  return cudaLaunchKernelEx(&cfg, k, P);
}

cudaError_t launch_stepper_batch(int precision, int kind, const Plan& plan, const StepParams* table, const int2* tasks,
                                 int ntasks, int* queue, int nclusters, cudaStream_t stream) {
  BatchKernel k = stepper_kernels_for(precision, kind, plan.ng).batch;
  if (!k) return cudaErrorInvalidConfiguration;
  cudaError_t e = configure((const void*)k, plan.cs, plan.smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(cfg, attr, nclusters, plan.cs, plan.nthreads, plan.smem, stream);
  return cudaLaunchKernelEx(&cfg, k, table, tasks, ntasks, queue);
}

static cudaError_t occupancy(const void* k, int cs, int nthreads, size_t smem, int* out) {
  cudaError_t e = configure(k, cs, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(cfg, attr, 64, cs, nthreads, smem, 0);
  return cudaOccupancyMaxActiveClusters(out, k, &cfg);
}

cudaError_t query_stepper_plan(int nx, int ny, int precision, int kind, int cs, int ng, int nthreads, size_t extra_smem,
                               Plan* plan, bool keep_ax) {
  StepKernel k = stepper_kernel_for(precision, kind, ng);
  if (!k || nthreads < 32 || nthreads > kStepMaxThreadsHost || nthreads % 32) return cudaErrorInvalidConfiguration;
  plan->cs = cs;
  plan->nthreads = nthreads;
  plan->ng = ng;
  plan->rmax = (ny + 1 + cs - 1) / cs;
  plan->smem = stepper_smem_bytes(nx, plan->rmax, precision == PTG_FP32_REFINE ? 4 : 8, keep_ax) + extra_smem;
  plan->keep_ax = keep_ax;
  plan->max_active_clusters = 0;
  if (plan->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  int n = 0;
  cudaError_t e = occupancy((const void*)k, cs, nthreads, plan->smem, &n);
  plan->max_active_clusters = n;
  return e;
}

cudaError_t query_wide_plan(int nx, int ny, int precision, int kind, int ntasks, bool spread,
                            size_t (*extra_smem)(const void*, int), const void* ctx, Plan* plan, bool keep_ax) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int rows = ny + 1;
  const int cap = nsm < kMaxGrid ? nsm : kMaxGrid;
  const int gw = padded_width(nx) / kGroup;
  // candidate CTA counts per group: spread -> as many as possible; else the fewest that fit
  int gfirst, glast, gstep;
  if (spread) {
    gfirst = cap < rows / 2 ? cap : rows / 2;
    glast = 2;
    gstep = -1;
  } else {
    gfirst = 2;
    glast = cap;
    gstep = 1;
  }
  for (int G = gfirst; spread ? G >= glast : G <= glast; G += gstep) {
    const int rmax = (rows + G - 1) / G;
    if (rmax < 2) continue;
    const int groups = rmax * gw;
    for (int ng = 1; ng <= 3; ++ng) {
      StepKernel k = stepper_kernels_for(precision, kind, ng).wide;
      if (!k) return cudaErrorInvalidConfiguration;
      const int nthreads = ((groups + ng - 1) / ng + 31) / 32 * 32;
      if (nthreads > kStepMaxThreadsHost) continue;
      const size_t smem = stepper_smem_bytes(nx, rmax, precision == PTG_FP32_REFINE ? 4 : 8, keep_ax) + extra_smem(ctx, G);
      if (smem > 227 * 1024) continue;
      e = configure_kernel((const void*)k, smem, false);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nthreads, smem);
      if (e != cudaSuccess) return e;
      const int resident = per_sm * nsm < kMaxGrid ? per_sm * nsm : kMaxGrid;
      if (per_sm < 1 || G > resident) continue;
      int ngroups = resident / G;
      if (ngroups > ntasks) ngroups = ntasks;
      plan->cs = G;
      plan->nthreads = nthreads;
      plan->ng = ng;
      plan->rmax = rmax;
      plan->smem = smem;
      plan->max_active_clusters = ngroups;
      plan->wide = true;
      plan->keep_ax = keep_ax;
      return cudaSuccess;
    }
  }
  return cudaErrorInvalidConfiguration;
}

cudaError_t query_batch_occupancy(int precision, int kind, int cs, int ng, int nthreads, size_t smem, int* nclusters) {
  BatchKernel k = stepper_kernels_for(precision, kind, ng).batch;
  if (!k || nthreads < 32 || nthreads > kStepMaxThreadsHost || nthreads % 32 || smem > 227 * 1024)
    return cudaErrorInvalidConfiguration;
  return occupancy((const void*)k, cs, nthreads, smem, nclusters);
}

}  // namespace ptg
