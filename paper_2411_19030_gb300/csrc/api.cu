// api.cu -- the C ABI (include/ptg.h): op lifecycle, argument checks, plan choice, launches.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>
#include "mesh.h"
#include "ptg_internal.h"
#include "stepper_launch.cuh"
#include "launch_check.h"
#include "trace.h"

using namespace ptg;

struct ptg_op {
  int device = 0;
  ptg_grid g{};
  ptg_material mat{};
  ptg_time tm{};
  ptg_solve sv{};
  int Nn = 0, Ne = 0, M = 0, p_int = 0, has_dc = 0;
  double dtau = 0.0;
  int W = 0;               // padded row width
  // two-level preconditioner of the coarse-step solves (FP32 CG); tl_m == 0: disabled
  int tl_m = 0, tl_nax = 0, tl_nay = 0;
  int tl_vc = 0;   // 1: the two-grid cycle instead of the additive form
  int tl_nu = 1;   // its smoothing steps (see StepParams::tl_nu)
  int tl_nu3 = 1;  // the three-level cycle's smoothing steps on each smoothed level
  double* tl_Ac = nullptr;
  float *tl_band = nullptr, *tl_X = nullptr, *tl_Ainv = nullptr;
  // three-level cycle (ptg_solve.twolevel = PTG_TWOLEVEL_THREELEVEL, even nx and ny): the 2h
  // level and the aggregates of tl3_m x tl3_m of its nodes; tl3_m == 0: not set up
  int tl3_m = 0, tl3_nax = 0, tl3_nay = 0;
  double *tl3_A1 = nullptr, *tl3_Ac = nullptr;
  float *tl3_band = nullptr, *tl3_X = nullptr, *tl3_Ainv = nullptr;
  // streamed fine propagators (ptg_solve.fine_stream, stream.cuh): FP32 weights of C/dt + K and
  // 1/C ([6][PN]), the FP64 1/C ([PN]), and the workspace of st_groups concurrent slices
  float* w32 = nullptr;         // [3][PEe] FP32 element weights (D, S, T) of C/dt + K
  float* w32_inv = nullptr;     // [PN] FP32 1/C
  double* w64_inv = nullptr;    // [PN] FP64 1/C
  double* st_w64 = nullptr;     // [st_groups][3][PN] (x, x, b), padded node layout
  void* st_wr = nullptr;        // [st_groups][5][PN] (r, z, p, q, d) of the FP64 CG kinds
  void* st_wr32 = nullptr;      // the same for the FP32 CG kinds: the two layouts never share
                                // memory, whose padding rows must stay zero for both
  int st_groups = 0;            // 0: the op has no streaming workspace; the workspace holds
                                // st_groups + 1 groups, the last one the correction sweeps'
  // streamed coarse-step solves (ptg_solve.coarse_stream, mg.cu): the multigrid hierarchy of
  // C/dtau + K and its workspace (st_groups + 1 groups); mg_L == 0: the coarse kinds stay on chip
  int mg_L = 0;
  MgLevel mg_lv[kMgMaxLevels] = {};
  float* mg_w = nullptr;
  float* mg_wf = nullptr;       // the same hierarchy of C/dt + K for the streamed fine propagators
  int mg_Lf = 0;                // its levels (0: the fine kinds stream with Jacobi)
  float* mg_ws = nullptr;
  long long mg_ws_stride = 0;
  int mg_solo = 0, mg_csteps = 0, mg_fuse = -1;   // ptg_op_set_multigrid (0 / -1: the defaults)
  double* sw_red = nullptr;     // the correction sweeps' reduction partials and barrier, so that the
  unsigned* sw_bar = nullptr;   // adjoint coarse parts may run beside the forward sweep
  // device workspace
  double *k = nullptr, *c = nullptr, *dk = nullptr, *dc = nullptr;
  double* wE = nullptr;     // [2][3][PEe]: element (D, S, T) weights for dt and dtau (padded)
  double* nodew = nullptr;  // [15][PN]: per-node weights of C/dt + K, C/dtau + K and C (padded)
  double* fload = nullptr;
  double *q_elem = nullptr, *q_time = nullptr;
  uint8_t* dirichlet = nullptr;
  double* sens_partial = nullptr;
  double* lam_prev = nullptr;  // [n Ntau][Nn] ring of the last n states of each fine task (primal or adjoint)
  double* scratch = nullptr;   // [2] small device scalars
  // grid-wide launches (one system over every SM): reduction partials, barrier, halo rows,
  // two-level partials
  double* g_red = nullptr;
  unsigned* g_bar = nullptr;
  long long wait_limit = 0;  // polls of a grid barrier before PTG_ETIMEOUT (0: the kernel's default)
  void* g_halo = nullptr;
  float* g_tl = nullptr;
  int sens_chunks = 0;
  DevStats* stats = nullptr;
  // coarse propagators on the mesh of spacing 2h (ptg_solve.coarse_mesh): the op of that mesh
  // (its coarse kinds run the coarse steps) and the transfer workspace
  ptg_op* mesh = nullptr;
  double* mesh_rho = nullptr;    // [NeH] coarse design
  double* mesh_XH = nullptr;     // [Ntau+1][NnH] coarse states of a correction sweep
  double* mesh_FH = nullptr;     // [Ntau][NnH] injected F (or the states a coarse sweep starts from)
  double* mesh_GH = nullptr;     // [Ntau][NnH] injected G_old
  double* mesh_SH = nullptr;     // [Ntau][NnH] restricted adjoint sources
  double* mesh_YH = nullptr;     // [Ntau][NnH] results of independent coarse steps
  double* mesh_zero = nullptr;   // [Ntau+1] zeros (theta and F/G theta slots of the coarse op)
  double* mesh_aux = nullptr;    // [Ntau+1] theta outputs of the coarse op (not used)
  double* mesh_pn = nullptr;     // [Ntau][blocks] p-norm partials of the prolongated states
  double* mesh_lam = nullptr;    // [Ntau][Nn] prolongated adjoint states of G
  double* mesh_dg = nullptr;     // [Ntau][Ne] g increments of G
  cudaStream_t last_stream = nullptr;
  // the first failed launch check of the debug build (launch_check.h): PTG_EBOUNDS, the task
  // kind and the check's site; reported by ptg_get_stats when the device status is clear
  int dbg_status = 0, dbg_kind = 0, dbg_site = 0;
  std::mutex mu;
  std::map<std::tuple<int, int, int>, Plan> plans;   // (precision, kind, ntasks) -> plan
  std::map<int, Plan> plan_override;                   // kind -> forced plan
};

namespace {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
  return PTG_ECUDA;
}

#define PTG_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool coarse_kind(int kind) {
  return kind == KIND_COARSE_PRI || kind == KIND_CORRECT_PRI || kind == KIND_COARSE_ADJ || kind == KIND_CORRECT_ADJ;
}

// Precision of the kernels of a task kind: PTG_FP32_REFINE keeps the coarse-step solves
// (G and the correction sweeps) in FP64 and runs only the fine-step CG in FP32;
// PTG_FP32_REFINE_ALL runs every CG in FP32.  Returns PTG_FP64 or PTG_FP32_REFINE (the two
// kernel instantiations).
int kind_precision(int solve_precision, int kind) {
  if (solve_precision == PTG_FP64) return PTG_FP64;
  if (solve_precision == PTG_FP32_REFINE_ALL) return PTG_FP32_REFINE;
  return coarse_kind(kind) ? PTG_FP64 : PTG_FP32_REFINE;
}

// Two-level forms a plan may use, strongest last: tl_mode caps the op's choice (an op set up
// for the V-cycle runs the additive form under a plan capped at TL_ADDITIVE, e.g. when the
// V-cycle's buffers do not fit).
enum TlMode : int { TL_NONE = 0, TL_ADDITIVE = 1, TL_VCYCLE = 2, TL_VCYCLE3 = 3 };
bool uses_vcycle(const ptg_op* op, int tl_mode) { return tl_mode >= TL_VCYCLE && op->tl_vc; }
bool uses_three(const ptg_op* op, int tl_mode) { return tl_mode >= TL_VCYCLE3 && op->tl3_m > 0; }
int strongest_mode(const ptg_op* op) {
  if (op->tl_m == 0) return TL_NONE;
  if (op->tl3_m > 0) return TL_VCYCLE3;
  return op->tl_vc ? TL_VCYCLE : TL_ADDITIVE;
}

// Three-level cycle: the aggregate rows reserved per CTA for cluster size cs (those touched by
// the CTA's 2h rows and its two 2h halo rows), 0 if a slab has fewer than two fine rows (then
// some CTA would own no 2h row) or the mode does not apply; r1max the most 2h rows of a CTA.
int threelevel_rows(const ptg_op* op, int kind, int cs, int tl_mode, int* r1max = nullptr) {
  if (!uses_three(op, tl_mode) || !coarse_kind(kind)) return 0;
  const int rows = op->g.ny + 1, base = rows / cs, rem = rows % cs;
  const int ny1 = op->g.ny / 2;
  int best = 0, rmx = 0;
  for (int q = 0; q < cs; ++q) {
    const int r0 = q * base + (q < rem ? q : rem), R = base + (q < rem ? 1 : 0);
    if (R < 2) return 0;
    int J0, R1;
    l1_rows_of_slab(r0, R, J0, R1);
    const int lo = l3_agg(J0 > 0 ? J0 - 1 : 0, op->tl3_m, op->tl3_nay);
    const int hi = l3_agg(J0 + R1 <= ny1 ? J0 + R1 : ny1, op->tl3_m, op->tl3_nay);
    best = std::max(best, hi - lo + 1);
    rmx = std::max(rmx, R1);
  }
  if (r1max) *r1max = rmx;
  return best;
}

// Aggregate rows reserved per CTA for cluster size cs (the largest over the ranks; with the
// V-cycle the rows its halo rows touch too), 0 if the two-level preconditioner is off for this
// op, kind or plan.
int twolevel_rows(const ptg_op* op, int precision, int kind, int cs, int tl_mode = TL_VCYCLE) {
  (void)precision;
  if (tl_mode == TL_NONE || op->tl_m == 0 || !coarse_kind(kind)) return 0;
  if (tl_mode >= TL_VCYCLE3) return threelevel_rows(op, kind, cs, tl_mode);
  const bool vc = uses_vcycle(op, tl_mode);
  int best = 0;
  for (int q = 0; q < cs; ++q) {
    int r0, R, lo, hi;
    const int rows = op->g.ny + 1, base = rows / cs, rem = rows % cs;
    r0 = q * base + (q < rem ? q : rem);
    R = base + (q < rem ? 1 : 0);
    if (vc)
      coarse_rows_of_halo_slab(r0, R, op->g.ny, op->tl_m, op->tl_nay, lo, hi);
    else
      coarse_rows_of_slab(r0, R, op->tl_m, op->tl_nay, lo, hi);
    best = std::max(best, hi - lo + 1);
  }
  return best;
}

// precision: the kernel's (PTG_FP64 or PTG_FP32_REFINE)
size_t twolevel_bytes(const ptg_op* op, int precision, int kind, int cs, int tl_mode, bool slots = true) {
  const int ncj = twolevel_rows(op, precision, kind, cs, tl_mode);
  if (ncj == 0) return 0;
  const int rmax = (op->g.ny + 1 + cs - 1) / cs;
  if (tl_mode >= TL_VCYCLE3) {
    int r1max = 0;
    threelevel_rows(op, kind, cs, tl_mode, &r1max);
    return threelevel_smem_bytes(op->W, rmax, cs, padded_width(op->g.nx / 2), r1max, op->tl3_nax, op->tl3_nay, ncj,
                                 slots, precision == PTG_FP64 ? 8 : 4, op->tl_nu3);
  }
  return twolevel_smem_bytes(op->W, rmax, cs, op->tl_nax, op->tl_nay, ncj, slots, uses_vcycle(op, tl_mode),
                             precision == PTG_FP64 ? 8 : 4, op->tl_nu);
}

// Damping of the V-cycle's Jacobi smoother: the largest eigenvalue of D^-1 A lies between 1.5
// (conduction-dominated) and 2.25 (capacity-dominated: the consistent Q1 mass matrix), so
// omega lambda_max stays below 1.8 < 2 for every step size.
constexpr float kVcycleOmega = 0.8f;
// Default preconditioner of FP32 CG solves without a two-level form (ptg_solve.local_steps = 0):
// Jacobi on cluster launches, the two slab-local steps on cooperative-grid launches (run()).  The two slab-local steps cut the fine-step CG iterations (128 x 128 pass: 34 -> 27
// primal, 31 -> 24.5 adjoint) but cost more than they save there (fine kernels 7.6 + 8.5 ->
// 8.6 + 9.4 ms); on high-contrast 512 x 512 designs they pay (one-shot design iteration 13.2 ->
// 11.5 s).
constexpr int kLocalSteps = 1;
// Default smoothing steps of the V-cycle (ptg_solve.smooth_steps = 0): four slab-local Jacobi
// steps before and after the coarse correction.  Measured on the 128 x 128 one-shot pass
// (FP64 coarse-step CG): 1 global step 66.1 ms; 2, 3, 4, 6 local steps 59.2, 56.5, 55.9,
// 56.8 ms, the CG iterations per correction solve falling from 34 to 26, 23, 21, 19.
constexpr int kVcycleSmoothSteps = 4;
// Default smoothing steps of the three-level cycle on both its smoothed levels: a numpy model of
// the 128 x 128 coarse-step operator (slab-local Jacobi on 16 slabs, aggregates of 4 x 4 2h nodes)
// needs 13 PCG iterations with 3 or 4 steps, 14 with 2 on one level, 15 with 2 on both.
constexpr int kThreeLevelSmoothSteps = 3;

// Node count from which a single FP64 system runs grid-wide (see choose_plan).
constexpr int kWideMinNodes = 40000;
// Node count from which the coarse-step solves stream by default (multigrid-preconditioned FP64 CG
// with the vectors in HBM): 192 x 192 (37 249 nodes) and up.  On chip, a 192 x 192 one-shot pass
// took longer than a 256 x 256 one with the same slices (214 against 187 ms at 64 slices).
constexpr int kCoarseStreamMinNodes = 30000;
// Streamed coarse-step solves (stream.cuh, mg.cu): node rows per CTA of a correction sweep's
// group, the multigrid's smoothing steps, the damped-Jacobi steps on its coarsest level (at most
// 9 x 9 nodes) where no dense inverse applies, and the levels with at most kMgSoloRows node rows, which the group's first CTA
// runs alone (block barriers instead of the group's).
constexpr int kSweepRowsPerCta = 2;
constexpr int kMgNu = 1;
constexpr int kMgCoarseSteps = 10;
constexpr int kMgSoloRows = 33;
constexpr int kMgFuse = 1;

// two-level bytes of a grid-wide launch of G CTAs (the partials live in global memory)
struct WideCtx {
  const ptg_op* op;
  int precision, kind, tl_mode;
};
size_t wide_twolevel_bytes(const void* ctx, int G) {
  const WideCtx* c = static_cast<const WideCtx*>(ctx);
  return twolevel_bytes(c->op, c->precision, c->kind, G, c->tl_mode, false);
}

// Inner tolerance of an FP64 CG with the additive two-level preconditioner.  Its coarse
// correction is applied in FP32 and carried by the CG recurrence, so its rounding is relative
// to the residual the CG started from.  Once the CG has reduced its residual by much more than
// 1e-4 that rounding dominates the coarse correction and the CG stalls (measured: 2000 instead
// of 61 iterations per solve at 1e-5 on a near-binary design).  So each CG stops at a 1e-4
// reduction (or the op's looser inner_rtol) and the FP64 residual loop restarts it from the
// exact residual.  The two-grid cycle is recomputed from r at every iteration and carries no
// such error, so its FP64 CG runs to the final tolerance in one go (measured on the 128 x 128
// pass: one refinement sweep per solve instead of two, 53.8 instead of 55.9 ms, and no stall
// on near-binary designs).
constexpr double kTwoLevelInnerFp64 = 1e-4;

void twolevel_params(const ptg_op* op, int precision, StepParams& P, int tl_mode) {
  P.tl_naj = twolevel_rows(op, precision, P.kind, P.cs, tl_mode);
  P.tl_vc = P.tl_naj > 0 && uses_vcycle(op, tl_mode);
  P.tl_omega = kVcycleOmega;
  P.tl_nu = op->tl_nu;
  // local_steps 3 (multigrid) applies to streamed fine propagators only: the default elsewhere
  const int ls = op->sv.local_steps == 3 ? 0 : op->sv.local_steps;
  P.local_steps = ls > 0 ? ls : kLocalSteps;
  // FP32 CG: the op's inner tolerance; FP64 CG: to the final tolerance in one go, or in
  // kTwoLevelInnerFp64 steps with the additive two-level preconditioner
  if (precision == PTG_FP64)
    P.inner_rtol = P.tl_naj > 0 && !P.tl_vc ? std::max(kTwoLevelInnerFp64, op->sv.inner_rtol) : 0.0;
  if (P.tl_naj == 0) return;
  if (tl_mode >= TL_VCYCLE3) {
    // the V-cycle's fine buffers plus the 2h level; the aggregate level is on the 2h grid
    P.tl_vc = 1;
    P.tl_l3 = 1;
    P.tl_nu = op->tl_nu3;
    P.l3_nx1 = op->g.nx / 2;
    P.l3_ny1 = op->g.ny / 2;
    P.l3_W1 = padded_width(P.l3_nx1);
    threelevel_rows(op, P.kind, P.cs, tl_mode, &P.l3_r1max);
    P.A1 = op->tl3_A1;
    P.Ainv = op->tl3_Ainv;
    P.cm = op->tl3_m;
    P.nax = op->tl3_nax;
    P.nay = op->tl3_nay;
    P.inner_rtol = precision == PTG_FP64 ? 0.0 : P.inner_rtol;
    return;
  }
  P.Ainv = op->tl_Ainv;
  P.cm = op->tl_m;
  P.nax = op->tl_nax;
  P.nay = op->tl_nay;
}

// Best plan for `ntasks` concurrent clusters with or without the two-level preconditioner:
// fewest waves, then the shortest per-thread work (ng), then the largest cluster.  Returns
// the number of waves, or -1 if nothing fits.
long best_plan(ptg_op* op, int precision, int kind, int ntasks, int tl_mode, Plan* out, bool keep_ax = true) {
  const int nx = op->g.nx, ny = op->g.ny;
  const int G = op->W / kGroup;
  long best_waves = -1;
  for (int cs : {16, 8, 4, 2, 1}) {
    const int rmax = (ny + 1 + cs - 1) / cs;
    if (rmax < 2) continue;
    const int groups = rmax * G;
    for (int ng : kStepNG) {
      const int nthreads = ((groups + ng - 1) / ng + 31) / 32 * 32;
      if (nthreads > kStepMaxThreadsHost) continue;
      Plan p;
      cudaError_t e = query_stepper_plan(nx, ny, precision, kind, cs, ng, nthreads,
                                         twolevel_bytes(op, precision, kind, cs, tl_mode), &p, keep_ax);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (p.max_active_clusters <= 0) continue;
      const long waves = (ntasks + p.max_active_clusters - 1) / p.max_active_clusters;
      if (best_waves < 0 || waves < best_waves || (waves == best_waves && ng < out->ng)) {
        p.twolevel = twolevel_rows(op, precision, kind, cs, tl_mode) > 0;
        p.vc = p.twolevel && uses_vcycle(op, tl_mode);
        p.l3 = p.twolevel && uses_three(op, tl_mode);
        *out = p;
        best_waves = waves;
      }
    }
  }
  return best_waves;
}

// Choose the plan of a task kind for `ntasks` concurrent clusters.  The two-level
// preconditioner (coarse kinds) cuts the CG iterations about threefold for a shared-memory
// cost; with FP32 CG it is used unless its plan needs more waves than Jacobi's, with FP64 CG
// whenever it fits.
int choose_plan(ptg_op* op, int precision, int kind, int ntasks, Plan* out) {
  std::lock_guard<std::mutex> lk(op->mu);
  auto ov = op->plan_override.find(kind);
  if (ov != op->plan_override.end()) {
    *out = ov->second;
    return PTG_OK;
  }
  auto key = std::make_tuple(precision, kind, ntasks);
  auto it = op->plans.find(key);
  if (it != op->plans.end()) {
    *out = it->second;
    return PTG_OK;
  }
  // Coarse-step solves (a3 and a4) of ops with a multigrid hierarchy (ptg_solve.coarse_stream):
  // streamed, FP64 CG with the V-cycle of mg.cu.  Batched coarse kinds: G = SMs / slices CTAs per
  // slice, every slice at once; a correction sweep (one system): one group of a CTA per
  // kSweepRowsPerCta node rows, at most one per SM.
  if (coarse_kind(kind) && op->mg_L > 0 && op->st_groups > 0) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm = std::min(nsm, kMaxGrid);
    const bool sweep = kind == KIND_CORRECT_PRI || kind == KIND_CORRECT_ADJ;
    int G = sweep ? (op->g.ny + 1) / kSweepRowsPerCta : nsm / ntasks;
    G = std::max(1, std::min({G, nsm, std::max(1, (op->g.ny + 1) / 2)}));
    Plan sp;
    sp.cs = G;
    sp.nthreads = 512;
    sp.ng = 1;
    sp.rmax = (op->g.ny + 1 + G - 1) / G;
    sp.smem = 0;
    sp.max_active_clusters = sweep ? 1 : std::max(1, std::min({ntasks, nsm / G, op->st_groups}));
    sp.stream = true;
    op->plans[key] = sp;
    *out = sp;
    return PTG_OK;
  }
  // Fine kinds of the parallel schedule (ntasks >= 2 slices at once) on the streamed propagator
  // (ptg_solve.fine_stream).  One CTA of 512 threads per SM; G = SMs / slices CTAs per slice (at
  // least 2 node rows each), all slices at once.
  if ((kind == KIND_FINE_PRI || kind == KIND_FINE_ADJ) && op->st_groups > 0 && ntasks >= 2 &&
      op->sv.fine_stream != 1) {
    // fine_stream 0: streamed where no cluster holds a slice (the grouped launches of large
    // grids run only a few slices at a time: at 512 x 512, 3 of 128); measured there the one-shot
    // design iteration takes 4.4-4.8 s streamed against 7.6-9.0 s on chip.  Where clusters fit
    // (256 x 256) both take the same time and the on-chip path stays.
    bool want = op->sv.fine_stream == 2;
    if (!want && op->sv.fine_stream == 0) {
      Plan c;
      long w = best_plan(op, precision, kind, ntasks, TL_NONE, &c);
      if (w < 0) w = best_plan(op, precision, kind, ntasks, TL_NONE, &c, false);
      want = w < 0;
    }
    if (want) {
      int dev = 0, nsm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      nsm = std::min(nsm, kMaxGrid);
      int G = std::max(1, nsm / ntasks);
      G = std::min(G, std::max(1, (op->g.ny + 1) / 2));
      Plan sp;
      sp.cs = G;
      sp.nthreads = 512;
      sp.ng = 1;
      sp.rmax = (op->g.ny + 1 + G - 1) / G;
      sp.smem = 0;
      sp.max_active_clusters = std::max(1, std::min({ntasks, nsm / G, op->st_groups}));
      sp.stream = true;
      op->plans[key] = sp;
      *out = sp;
      return PTG_OK;
    }
  }
  // One FP64 system: a cluster runs its CG on 16 SMs, bound by their FP64 pipes; a grid-wide
  // launch spreads the FP64 work over every SM, but each of its reductions costs a few
  // microseconds of global-memory round trips against about one for a cluster.  Measured on
  // GB300 the cluster wins at 128 x 128; the grid wins once the per-iteration FP64 work of 16
  // SMs dominates (kWideMinNodes).  Grids whose slabs do not fit 16 CTAs (512 x 512) run in
  // groups of CTAs of one cooperative launch.  grid_wide: 0 never, 1 by these rules, 2 always.
  // The strongest two-level form whose plan fits (and, for FP32 CG, adds no wave over
  // Jacobi's: FP64 CG on GB300 is bound by the FP64 pipe, so the cut in iterations outweighs
  // extra waves; FP32 CG is bound by latency).
  // A plan may leave out the saved A x of the last residual (one more FP64 stencil per step) when
  // that lets a two-level form, or any plan at all, fit.
  Plan jac, two;
  long wj = best_plan(op, precision, kind, ntasks, TL_NONE, &jac);
  if (wj < 0) wj = best_plan(op, precision, kind, ntasks, TL_NONE, &jac, false);
  long wt = -1;
  if (twolevel_rows(op, precision, kind, 1) > 0) {
    for (int mode = strongest_mode(op); mode > TL_NONE && wt < 0; --mode) {
      for (bool keep_ax : {true, false}) {
        Plan c;
        const long w = best_plan(op, precision, kind, ntasks, mode, &c, keep_ax);
        if (w >= 0 && (wj < 0 || w <= wj || precision == PTG_FP64)) {
          two = c;
          wt = w;
          break;
        }
      }
    }
  }
  const bool spread = ntasks == 1 && precision == PTG_FP64;
  const bool no_cluster = wj < 0 && wt < 0;
  const bool want_wide = op->sv.grid_wide == 2 ||
                         (op->sv.grid_wide == 1 && (no_cluster || (spread && op->Nn >= kWideMinNodes)));
  if (want_wide) {
    // one FP64 system over every SM (spread), or groups of the fewest CTAs whose slabs fit,
    // with the strongest two-level form that fits.  Groups leave out the saved A x: smaller
    // slabs per CTA mean fewer CTAs per group and more systems at a time.
    for (int mode = std::min(strongest_mode(op), (int)TL_VCYCLE); mode >= TL_NONE; --mode) {   // no 3-level on grids
      for (bool keep_ax : {spread, !spread}) {
        Plan w;
        WideCtx ctx{op, precision, kind, mode};
        if (query_wide_plan(op->g.nx, op->g.ny, precision, kind, ntasks, spread, wide_twolevel_bytes, &ctx, &w,
                            keep_ax) == cudaSuccess) {
          w.twolevel = twolevel_rows(op, precision, kind, w.cs, mode) > 0;
          w.vc = w.twolevel && uses_vcycle(op, mode);
          op->plans[key] = w;
          *out = w;
          return PTG_OK;
        }
        cudaGetLastError();
      }
    }
  }
  if (no_cluster) {
    std::snprintf(g_last_error, sizeof(g_last_error), "no launch plan fits a %dx%d grid", op->g.nx, op->g.ny);
    return PTG_EINVAL;
  }
  const Plan best = wt >= 0 ? two : jac;
  op->plans[key] = best;
  *out = best;
  return PTG_OK;
}

// States the initial guess of a fine step is extrapolated through (ptg_solve.initial_guess).
// Measured in FP64 Jacobi CG to 1e-10 on the 128 x 128 case (dt = 1/1024): 36 iterations per
// step from the last state, 21 linear, 14 quadratic, 8 cubic.
constexpr int kInitialGuessDefault = 4;
int guess_states(const ptg_solve& sv) { return sv.initial_guess > 0 ? sv.initial_guess : kInitialGuessDefault; }

void base_params(const ptg_op* op, StepParams& P) {
  std::memset(&P, 0, sizeof(P));
  P.nx = op->g.nx;
  P.ny = op->g.ny;
  P.Nn = op->Nn;
  P.Ne = op->Ne;
  P.Nt = op->tm.Nt;
  P.Ntau = op->tm.Ntau;
  P.M = op->M;
  P.p_int = op->p_int;
  P.h = op->g.h;
  P.dt = op->tm.dt;
  P.dtau = op->dtau;
  P.p = op->tm.p;
  P.has_dc = op->has_dc;
  P.rtol = op->sv.rtol;
  P.inner_rtol = op->sv.inner_rtol;   // used by the FP32 CG kernels only
  P.itmax = op->sv.cg_iters_max;
  P.refmax = op->sv.refine_max;
  P.W = op->W;
  const size_t PEe = (size_t)(op->g.ny + 2) * op->W + 2 * kSlack;
  const size_t PN = (size_t)(op->g.ny + 3) * op->W + 2 * kSlack;
  P.wE_fine = op->wE + kSlack;
  P.wE_coarse = op->wE + 3 * PEe + kSlack;
  auto nw = [&](int base) {
    NodeWeights w;
    w.C = op->nodew + (base + 0) * PN + kSlack;
    w.E = op->nodew + (base + 1) * PN + kSlack;
    w.N = op->nodew + (base + 2) * PN + kSlack;
    w.NE = op->nodew + (base + 3) * PN + kSlack;
    w.NW = op->nodew + (base + 4) * PN + kSlack;
    return w;
  };
  P.A_fine = nw(0);
  P.A_coarse = nw(5);
  P.mass = nw(10);
  if (op->w32) {
    P.w32 = op->w32 + kSlack;
    P.w32_stride = (int)PEe;
    P.w32_inv = op->w32_inv + kSlack;
    P.w64_inv = op->w64_inv + kSlack;
    P.st_pv = (long long)PN;
  }
  P.dk = op->dk;
  P.dc = op->dc;
  P.fload = op->fload;
  P.q_time = op->q_time;
  P.dirichlet = op->dirichlet;
  P.stats = op->stats;
  P.objective = op->tm.objective;
  P.hist_rows = 0;
  P.keep_ax = 1;
  P.extrap = guess_states(op->sv);
  P.guess_next = P.extrap > 1;
  P.prev_field = op->lam_prev;
}

#ifdef PTG_DEBUG
static_assert(kCheckMaxLevels == kMgMaxLevels && kCheckSlack == kSlack, "launch_check.h constants");

// The debug build's launch checks (launch_check.h): PTG_OK, or PTG_EBOUNDS with the first failed
// check recorded on the op (the launch is then skipped).
int debug_check(ptg_op* op, const StepParams& P, const Plan& plan, int ntasks) {
  LaunchFacts f;
  f.kind = P.kind;
  f.s0 = P.s0;
  f.ns = P.ns;
  f.chained = P.chained;
  f.ntasks = ntasks;
  f.Ntau = op->tm.Ntau;
  f.M = op->M;
  f.plt = P.plt;
  f.has_hist = P.hist != nullptr;
  f.hist_j0 = P.hist_j0;
  f.hist_rows = P.hist_rows;
  f.ny = op->g.ny;
  f.W = op->W;
  f.cs = plan.cs;
  f.rmax = plan.rmax;
  f.streamed = plan.stream;
  f.wide = plan.wide;
  f.groups = plan.max_active_clusters;
  f.st_groups = op->st_groups;
  f.st_pv = P.st_pv;
  f.mg_levels = plan.stream ? P.mg_levels : 0;
  for (int l = 0; l < f.mg_levels && l < kCheckMaxLevels; ++l) {
    f.mg_voff[l] = P.mg[l].voff;
    f.mg_plen[l] = P.mg[l].plen;
  }
  f.mg_ws_stride = P.mg_ws_stride;
  const int site = launch_check_site(f);
  if (site == kSiteNone) return PTG_OK;
  if (op->dbg_status == 0) {
    op->dbg_status = PTG_EBOUNDS;
    op->dbg_kind = 30 + P.stats_kind;
    op->dbg_site = site;
  }
  return PTG_EBOUNDS;
}
#endif

int run(ptg_op* op, StepParams& P, int ntasks, cudaStream_t stream, int stats_kind = -1) {
  P.stats_kind = stats_kind >= 0 ? stats_kind : P.kind;
  Plan plan;
  const int prec = kind_precision(op->sv.precision, P.kind);
  int rc = choose_plan(op, prec, P.kind, ntasks, &plan);
  if (rc != PTG_OK) return rc;
  P.cs = plan.cs;
  P.rmax = plan.rmax;
  if (plan.stream) {
    if (P.chained) return PTG_EINVAL;            // a chained run is one task: never planned so
    P.wide = 1;
    P.wide_tasks = ntasks;
    P.g_red = op->g_red;
    P.g_bar = op->g_bar;
    P.wait_limit = op->wait_limit;
    P.st_w64 = op->st_w64;
    P.st_wr = prec == PTG_FP64 ? op->st_wr : op->st_wr32;
    const size_t rbytes = prec == PTG_FP64 ? sizeof(double) : sizeof(float);
    if (!P.st_wr) return PTG_EINVAL;           // (allocated for every precision a streamed kind uses)
    twolevel_params(op, prec, P, TL_NONE);
    const int L = coarse_kind(P.kind) ? op->mg_L : op->mg_Lf;
    if (L > 0) {
      P.mg_levels = L;
      P.mg_nu = kMgNu;
      P.mg_coarse_steps = op->mg_csteps > 0 ? op->mg_csteps : kMgCoarseSteps;
      P.mg_solo_rows = op->mg_solo > 0 ? op->mg_solo : kMgSoloRows;
      P.mg_fuse = op->mg_fuse >= 0 ? op->mg_fuse : kMgFuse;
      for (int l = 0; l < L; ++l) P.mg[l] = op->mg_lv[l];
      P.mg_w = coarse_kind(P.kind) ? op->mg_w : op->mg_wf;
      P.mg_ws = op->mg_ws;
      P.mg_ws_stride = op->mg_ws_stride;
      if (P.kind == KIND_CORRECT_PRI || P.kind == KIND_CORRECT_ADJ) {
        // the sweep's own group of the workspace, partials and barrier
        const size_t g = (size_t)op->st_groups;
        P.st_w64 = op->st_w64 + g * 3 * (size_t)P.st_pv;
        P.st_wr = static_cast<char*>(P.st_wr) + g * 5 * (size_t)P.st_pv * rbytes;
        P.mg_ws = op->mg_ws + g * (size_t)op->mg_ws_stride;
        P.g_red = op->sw_red;
        P.g_bar = op->sw_bar;
      }
    }
#ifdef PTG_DEBUG
    if (const int rc = debug_check(op, P, plan, ntasks)) return rc;
#endif
    op->last_stream = stream;
    PTG_CUDA(launch_stream(P, prec, plan.max_active_clusters, plan.nthreads, stream));
    return PTG_OK;
  }
  if (plan.wide) {
    P.wide = 1;
    P.wide_tasks = ntasks;
    P.g_red = op->g_red;
    P.g_bar = op->g_bar;
    P.wait_limit = op->wait_limit;
    P.g_halo = op->g_halo;
    P.g_halo_row_bytes = op->W * (int)sizeof(double);
    P.g_tl = op->g_tl;
  }
  twolevel_params(op, prec, P,
                  plan.twolevel && !P.plt ? (plan.l3 ? TL_VCYCLE3 : (plan.vc ? TL_VCYCLE : TL_ADDITIVE)) : TL_NONE);
  P.keep_ax = plan.keep_ax ? 1 : 0;
  // on cooperative-grid launches every reduction is a global-memory round trip of several
  // microseconds, so the default trades two slab-local sweeps for fewer CG iterations there
  if ((op->sv.local_steps == 0 || op->sv.local_steps == 3) && plan.wide) P.local_steps = 2;
#ifdef PTG_DEBUG
  if (const int rc = debug_check(op, P, plan, ntasks)) return rc;
#endif
  op->last_stream = stream;
  PTG_CUDA(launch_stepper(P, plan, prec, ntasks, stream));
  return PTG_OK;
}

bool window_covers(int j0, int rows, int lo, int hi) { return lo >= j0 && hi < j0 + rows; }

void ptg_op_free(ptg_op* op);

void free_all(ptg_op* op) {
  void* ptrs[] = {op->k, op->c, op->dk, op->dc, op->wE, op->nodew, op->fload,
                  op->q_elem, op->q_time, op->dirichlet, op->sens_partial, op->lam_prev, op->scratch, op->stats,
                  op->g_red, op->g_bar, op->g_halo, op->g_tl,
                  op->tl_Ac, op->tl_band, op->tl_X, op->tl_Ainv,
                  op->tl3_A1, op->tl3_Ac, op->tl3_band, op->tl3_X, op->tl3_Ainv,
                  op->w32, op->w32_inv, op->w64_inv, op->st_w64, op->st_wr, op->st_wr32, op->mg_w, op->mg_wf, op->mg_ws, op->sw_red,
                  op->sw_bar,
                  op->mesh_rho, op->mesh_XH, op->mesh_FH, op->mesh_GH, op->mesh_SH, op->mesh_YH,
                  op->mesh_zero, op->mesh_aux, op->mesh_pn, op->mesh_lam, op->mesh_dg};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (op->mesh) ptg_op_free(op->mesh);
  op->mesh = nullptr;
}

void ptg_op_free(ptg_op* op) {
  free_all(op);
  delete op;
}

// Launch coarse-kind tasks of the 2h-mesh op on behalf of the fine op: the solver counters
// and errors go to the fine op's status word under the fine kind they stand for.
int mesh_run(ptg_op* op, StepParams& P, int ntasks, int stats_kind, cudaStream_t st) {
  P.stats = op->stats;
  op->mesh->last_stream = st;
  return run(op->mesh, P, ntasks, st, stats_kind);
}

// G_pri / G_adj of every slice on the 2h mesh (Sec. 7.3 future work; the readings are those of
// the oracle's coarse_mesh module): R the states, one coarse step each on the 2h-mesh op, P
// the results; theta from the fine-mesh p-norm of P x, g from the fine-mesh sensitivity term of
// P z (Eq. 4.7).
int mesh_coarse_sweep(ptg_op* op, int direction, const double* X_field, const double* X_aux, const double* T_hist,
                      const double* Theta_d, double* G_field, double* G_aux, cudaStream_t st) {
  ptg_op* H = op->mesh;
  const int nx = op->g.nx, ny = op->g.ny, Ne = op->Ne, Ntau = op->tm.Ntau, M = op->M;
  const uint8_t *dirF = op->dirichlet, *dirH = H->dirichlet;
  const MeshRows none = mrows(nullptr);
  const MeshRowsW nonew = mrowsw(nullptr);
  StepParams P;
  base_params(H, P);
  P.kind = KIND_COARSE_PRI;
  P.s0 = 0;
  P.ns = Ntau;
  P.in_field = op->mesh_FH;
  P.in_aux = op->mesh_zero;
  P.guess_next = 0;                       // the injected states hold no u_{s+1}
  P.out_field = op->mesh_YH;
  P.out_aux = op->mesh_aux;
  if (direction == PTG_PRIMAL) {
    PTG_CUDA(mesh_inject(nx, ny, mrows(X_field), mrowsw(op->mesh_FH), Ntau, dirH, st));
    int rc = mesh_run(op, P, Ntau, KIND_COARSE_PRI, st);
    if (rc != PTG_OK) return rc;
    PTG_CUDA(mesh_prolong(nx, ny, mrows(op->mesh_YH), none, none, none, none, mrowsw(G_field), nonew, nonew, Ntau,
                          dirF, dirH, op->p_int, op->mesh_pn, st));
    PTG_CUDA(mesh_theta_old(Ntau, mesh_blocks(op->Nn), op->mesh_pn, X_aux, G_aux, 1.0 / ((double)Ntau * Ne), op->tm.p,
                            op->p_int, op->tm.objective, st));
  } else {
    // lambda_{s+1}^old and the source of step k = M s + 1
    PTG_CUDA(mesh_inject(nx, ny, mrows(X_field, 1), mrowsw(op->mesh_FH), Ntau, dirH, st));
    PTG_CUDA(mesh_source(nx, ny, mrows(T_hist, 1, M), mrowsw(op->mesh_SH), Ntau, Theta_d, op->tm.p, op->p_int,
                         op->tm.objective, dirF, dirH, st));
    P.src_field = op->mesh_SH;
    int rc = mesh_run(op, P, Ntau, KIND_COARSE_ADJ, st);
    if (rc != PTG_OK) return rc;
    PTG_CUDA(mesh_prolong(nx, ny, mrows(op->mesh_YH), none, none, none, none, mrowsw(G_field), nonew, nonew, Ntau,
                          dirF, dirH, op->p_int, op->mesh_pn, st));
    PTG_CUDA(mesh_dg(nx, ny, op->g.h, op->dtau, op->has_dc, op->dk, op->dc, mrows(G_field), T_hist, M, 0, 1, Ntau,
                     1.0 / Ntau, op->mesh_dg, st));
    PTG_CUDA(mesh_g_old(Ne, Ntau, X_aux, op->mesh_dg, G_aux, st));
  }
  return PTG_OK;
}

// The 2h-mesh op of a fine op (ptg_solve.coarse_mesh): nx/2 x ny/2 elements of side 2h, the
// fine op's materials, precision and solver settings, one step of dtau per slice (Nt = Ntau,
// M = 1, the load at t_{M(s+1)}), sink nodes where the fine node is a sink, element sources
// averaged over the four children; and the transfer workspace.
int create_mesh(ptg_op* op, const uint8_t* dirichlet_h, const double* q_elem_h, const double* q_time_h) {
  const int nx = op->g.nx, ny = op->g.ny, nxH = nx / 2, nyH = ny / 2, Ntau = op->tm.Ntau, M = op->M;
  const int NnH = (nxH + 1) * (nyH + 1), NeH = nxH * nyH;
  ptg_grid gH{nxH, nyH, 2.0 * op->g.h};
  ptg_time tH = op->tm;
  tH.Nt = Ntau;
  tH.Ntau = Ntau;
  tH.dt = op->dtau;
  ptg_solve sH = op->sv;
  sH.coarse_mesh = 0;
  sH.initial_guess = 1;   // it runs coarse kinds only, and from injected states that hold no u_{s+1}
  std::vector<uint8_t> dH(NnH);
  for (int J = 0; J <= nyH; ++J)
    for (int I = 0; I <= nxH; ++I) dH[J * (nxH + 1) + I] = dirichlet_h[2 * J * (nx + 1) + 2 * I];
  std::vector<double> qH(NeH), qtH(Ntau + 1);
  for (int EY = 0; EY < nyH; ++EY)
    for (int EX = 0; EX < nxH; ++EX) {
      auto q = [&](int ey, int ex) { return q_elem_h ? q_elem_h[ey * nx + ex] : 1.0; };
      qH[EY * nxH + EX] = 0.25 * ((q(2 * EY, 2 * EX) + q(2 * EY, 2 * EX + 1)) +
                                  (q(2 * EY + 1, 2 * EX) + q(2 * EY + 1, 2 * EX + 1)));
    }
  for (int j = 0; j <= Ntau; ++j) qtH[j] = q_time_h ? q_time_h[(size_t)M * j] : 1.0;
  int rc = ptg_op_create(&gH, &op->mat, &tH, &sH, dH.data(), qH.data(), qtH.data(), op->device, &op->mesh);
  if (rc != PTG_OK) return rc;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  };
  const size_t nb = (size_t)mesh_blocks(op->Nn);
  A(&op->mesh_rho, (size_t)NeH * sizeof(double));
  A(&op->mesh_XH, (size_t)(Ntau + 1) * NnH * sizeof(double));
  A(&op->mesh_FH, (size_t)Ntau * NnH * sizeof(double));
  A(&op->mesh_GH, (size_t)Ntau * NnH * sizeof(double));
  A(&op->mesh_SH, (size_t)Ntau * NnH * sizeof(double));
  A(&op->mesh_YH, (size_t)Ntau * NnH * sizeof(double));
  A(&op->mesh_zero, (size_t)(Ntau + 1) * sizeof(double));
  A(&op->mesh_aux, (size_t)(Ntau + 1) * sizeof(double));
  A(&op->mesh_pn, (size_t)Ntau * nb * sizeof(double));
  A(&op->mesh_lam, (size_t)Ntau * op->Nn * sizeof(double));
  A(&op->mesh_dg, (size_t)Ntau * op->Ne * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(op->mesh_zero, 0, (size_t)(Ntau + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(op->mesh_aux, 0, (size_t)(Ntau + 1) * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "coarse mesh workspace");
  return PTG_OK;
}

// The correction sweeps with the 2h-mesh G.  With w_s = F_s - G_s (fine) the corrected state
// is u_{s+1} = P x_{s+1} + w_s, where x_{s+1} is the coarse step from R u_s; and R u_{s+1} =
// x_{s+1} + R w_s, so the 2h-mesh op's own correction sweep on R F and R G_old (same
// recurrence, on the coarse mesh) yields R u_{s+1}, hence x_{s+1} = R u_{s+1} - R F_s + R G_s.
// Only the coarse solves are sequential; prolongation, history rows, theta and g follow in
// parallel over the slices (the theta and g recurrences are scalar / per element).
int mesh_correct(ptg_op* op, int direction, const double* F_field, const double* F_aux, const double* G_field,
                 const double* G_aux, double* X_field, double* X_aux, double* T_hist, const double* Theta_d,
                 cudaStream_t st) {
  ptg_op* H = op->mesh;
  const int nx = op->g.nx, ny = op->g.ny, Nn = op->Nn, NnH = H->Nn, Ne = op->Ne, Ntau = op->tm.Ntau, M = op->M;
  const uint8_t *dirF = op->dirichlet, *dirH = H->dirichlet;
  const MeshRows none = mrows(nullptr);
  const MeshRowsW nonew = mrowsw(nullptr);
  StepParams P;
  base_params(H, P);
  P.kind = KIND_CORRECT_PRI;
  P.s0 = 0;
  P.ns = Ntau;
  P.in_field = nullptr;                   // x_0 given in row 0 of the coarse states
  P.out_field = op->mesh_XH;
  P.out_aux = op->mesh_aux;
  P.F_field = op->mesh_FH;
  P.F_aux = op->mesh_zero;
  P.G_field = op->mesh_GH;
  P.G_aux = op->mesh_zero;
  if (direction == PTG_PRIMAL) {
    PTG_CUDA(mesh_inject(nx, ny, mrows(F_field), mrowsw(op->mesh_FH), Ntau, dirH, st));
    PTG_CUDA(mesh_inject(nx, ny, mrows(G_field), mrowsw(op->mesh_GH), Ntau, dirH, st));
    PTG_CUDA(mesh_inject(nx, ny, mrows(X_field), mrowsw(op->mesh_XH), 1, dirH, st));
    int rc = mesh_run(op, P, 1, KIND_CORRECT_PRI, st);
    if (rc != PTG_OK) return rc;
    if (T_hist) PTG_CUDA(cudaMemcpyAsync(T_hist, X_field, (size_t)Nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    PTG_CUDA(mesh_prolong(nx, ny, mrows(op->mesh_XH, 1), mrows(op->mesh_FH), mrows(op->mesh_GH), mrows(F_field),
                          mrows(G_field), mrowsw(X_field, 1), nonew, T_hist ? mrowsw(T_hist, M, M) : nonew, Ntau,
                          dirF, dirH, op->p_int, op->mesh_pn, st));
    PTG_CUDA(mesh_theta_chain(Ntau, mesh_blocks(Nn), op->mesh_pn, F_aux, G_aux, X_aux, 1.0 / ((double)Ntau * Ne),
                              op->tm.p, op->p_int, op->tm.objective, st));
  } else {
    // time-reversed on the coarse mesh: coarse row r stands for slice s = Ntau - 1 - r
    PTG_CUDA(cudaMemsetAsync(X_field + (size_t)Ntau * Nn, 0, (size_t)Nn * sizeof(double), st));
    PTG_CUDA(cudaMemsetAsync(op->mesh_XH, 0, (size_t)NnH * sizeof(double), st));
    PTG_CUDA(mesh_inject(nx, ny, mrows(F_field, Ntau - 1, -1), mrowsw(op->mesh_FH), Ntau, dirH, st));
    PTG_CUDA(mesh_inject(nx, ny, mrows(G_field, Ntau - 1, -1), mrowsw(op->mesh_GH), Ntau, dirH, st));
    PTG_CUDA(mesh_source(nx, ny, mrows(T_hist, (long long)M * (Ntau - 1) + 1, -M), mrowsw(op->mesh_SH), Ntau, Theta_d,
                         op->tm.p, op->p_int, op->tm.objective, dirF, dirH, st));
    P.src_field = op->mesh_SH;
    int rc = mesh_run(op, P, 1, KIND_CORRECT_ADJ, st);
    if (rc != PTG_OK) return rc;
    PTG_CUDA(mesh_prolong(nx, ny, mrows(op->mesh_XH, 1), mrows(op->mesh_FH), mrows(op->mesh_GH),
                          mrows(F_field, Ntau - 1, -1), mrows(G_field, Ntau - 1, -1), mrowsw(X_field, Ntau - 1, -1),
                          mrowsw(op->mesh_lam), nonew, Ntau, dirF, dirH, op->p_int, op->mesh_pn, st));
    PTG_CUDA(mesh_dg(nx, ny, op->g.h, op->dtau, op->has_dc, op->dk, op->dc, mrows(op->mesh_lam), T_hist, M, Ntau - 1,
                     -1, Ntau, 1.0 / Ntau, op->mesh_dg, st));
    PTG_CUDA(mesh_g_chain(Ne, Ntau, op->mesh_dg, F_aux, G_aux, X_aux, st));
  }
  return PTG_OK;
}

}  // namespace

namespace ptg {
// Lets other translation units of the library report a message through ptg_last_error.
void set_last_error(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace ptg

extern "C" {

const char* ptg_version(void) {
#ifdef PTG_DEBUG
  return "ptg 0.1 sm_103a debug";
#else
  return PTG_TRACE_ENABLED ? "ptg 0.1 sm_103a nvtx" : "ptg 0.1 sm_103a";
#endif
}

const char* ptg_last_error(void) { return g_last_error; }

int ptg_op_create(const ptg_grid* grid, const ptg_material* mat, const ptg_time* time, const ptg_solve* solve,
                  const uint8_t* dirichlet_h, const double* q_elem_h, const double* q_time_h, int device,
                  ptg_op** out) {
  PTG_TRACE(__func__);
  if (!out) return PTG_EINVAL;
  *out = nullptr;
  if (!grid || !mat || !time || !solve || !dirichlet_h) return PTG_EINVAL;
  if (grid->nx < 2 || grid->ny < 2 || grid->nx > 4096 || grid->ny > 4096 || !(grid->h > 0.0)) return PTG_EINVAL;
  if (time->Nt < 1 || time->Ntau < 1 || time->Nt % time->Ntau != 0 || !(time->dt > 0.0)) return PTG_EINVAL;
  const double p = time->p;
  if (!(p >= 2.0 && p <= 64.0) || p != (double)(int)p || ((int)p) % 2 != 0) return PTG_EINVAL;
  if (time->objective != PTG_OBJ_POWER_MEAN && time->objective != PTG_OBJ_MODIFIED) return PTG_EINVAL;
  if (solve->precision != PTG_FP64 && solve->precision != PTG_FP32_REFINE && solve->precision != PTG_FP32_REFINE_ALL)
    return PTG_EINVAL;
  if (solve->twolevel < PTG_TWOLEVEL_NONE || solve->twolevel > PTG_TWOLEVEL_THREELEVEL) return PTG_EINVAL;
  if (solve->fine_stream < 0 || solve->fine_stream > 2) return PTG_EINVAL;
  if (solve->coarse_stream < 0 || solve->coarse_stream > 2) return PTG_EINVAL;
  if (solve->smooth_steps < 0 || solve->smooth_steps > 16) return PTG_EINVAL;
  if (solve->coarse_mesh != 0 && solve->coarse_mesh != 1) return PTG_EINVAL;
  if (solve->local_steps < 0 || solve->local_steps > 3) return PTG_EINVAL;
  if (solve->initial_guess < 0 || solve->initial_guess > kMaxExtrap) return PTG_EINVAL;
  if (solve->coarse_mesh && (grid->nx % 2 || grid->ny % 2 || grid->nx < 4 || grid->ny < 4)) return PTG_EINVAL;
  if (!(solve->rtol > 0.0) || solve->cg_iters_max < 1 || solve->refine_max < 1 || !(solve->inner_rtol >= 0.0))
    return PTG_EINVAL;
  if (!(mat->k0 > 0.0) || !(mat->kmin > 0.0) || !(mat->c0 > 0.0) || !(mat->cmin > 0.0)) return PTG_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    std::snprintf(g_last_error, sizeof(g_last_error), "no CUDA device %d", device);
    return PTG_ECUDA;
  }
  DeviceGuard dg(device);
  ptg_op* op = new (std::nothrow) ptg_op();
  if (!op) return PTG_ENOMEM;
  op->device = device;
  op->g = *grid;
  op->mat = *mat;
  op->tm = *time;
  op->sv = *solve;
  op->Nn = (grid->nx + 1) * (grid->ny + 1);
  op->Ne = grid->nx * grid->ny;
  op->M = time->Nt / time->Ntau;
  op->dtau = op->M * time->dt;
  op->p_int = (int)p;
  op->has_dc = mat->c0 != mat->cmin;
  op->W = padded_width(grid->nx);
  const size_t PEe = (size_t)(grid->ny + 2) * op->W + 2 * kSlack;
  const size_t PN = (size_t)(grid->ny + 3) * op->W + 2 * kSlack;
  const int blocks_e = (op->Ne + 255) / 256;
  op->sens_chunks = std::max(1, std::min(64, (4 * 152 + blocks_e - 1) / blocks_e));
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
  };
  A(&op->k, op->Ne * sizeof(double));
  A(&op->c, op->Ne * sizeof(double));
  A(&op->dk, op->Ne * sizeof(double));
  A(&op->dc, op->Ne * sizeof(double));
  A(&op->wE, 6 * PEe * sizeof(double));
  A(&op->nodew, 15 * PN * sizeof(double));
  A(&op->fload, op->Nn * sizeof(double));
  A(&op->q_elem, op->Ne * sizeof(double));
  A(&op->q_time, (time->Nt + 1) * sizeof(double));
  A(&op->dirichlet, op->Nn);
  A(&op->sens_partial, (size_t)op->sens_chunks * op->Ne * sizeof(double));
  if (guess_states(*solve) > 1)
    A(&op->lam_prev, (size_t)guess_states(*solve) * time->Ntau * op->Nn * sizeof(double));
  // two-level preconditioner: aggregates of m x m nodes, m the smallest multiple of 4 giving
  // at most kCoarseMaxAgg aggregates per direction
  if (solve->twolevel) {
    int m = 4;
    while ((grid->nx + 1) / m > kCoarseMaxAgg || (grid->ny + 1) / m > kCoarseMaxAgg) m += 4;
    op->tl_m = m;
    op->tl_vc = solve->twolevel == PTG_TWOLEVEL_VCYCLE || solve->twolevel == PTG_TWOLEVEL_THREELEVEL;
    op->tl_nu = solve->smooth_steps > 0 ? solve->smooth_steps : kVcycleSmoothSteps;
    op->tl_nu3 = solve->smooth_steps > 0 ? solve->smooth_steps : kThreeLevelSmoothSteps;
    op->tl_nax = coarse_aggregates(grid->nx, m);
    op->tl_nay = coarse_aggregates(grid->ny, m);
    const size_t nc = (size_t)op->tl_nax * op->tl_nay;
    A(&op->tl_Ac, nc * nc * sizeof(double));
    A(&op->tl_band, nc * (op->tl_nax + 2) * sizeof(float));
    const size_t ncp = (size_t)coarse_row_stride(op->tl_nax) * op->tl_nay;
    A(&op->tl_X, nc * nc * sizeof(float));
    A(&op->tl_Ainv, ncp * ncp * sizeof(float));
    A(&op->g_tl, (size_t)kMaxGrid * ncp * sizeof(float));
    // the three-level cycle needs the 2h grid (even nx, ny) with at least 4 x 4 of its nodes;
    // aggregates of m x m 2h nodes, m the smallest size giving at most kCoarseMaxAgg per direction
    if (solve->twolevel == PTG_TWOLEVEL_THREELEVEL && grid->nx % 2 == 0 && grid->ny % 2 == 0 && grid->nx >= 6 &&
        grid->ny >= 6) {
      const int nx1 = grid->nx / 2, ny1 = grid->ny / 2;
      int m3 = 2;
      while ((nx1 + 1) / m3 > kCoarseMaxAgg || (ny1 + 1) / m3 > kCoarseMaxAgg) ++m3;
      op->tl3_m = m3;
      op->tl3_nax = coarse_aggregates(nx1, m3);
      op->tl3_nay = coarse_aggregates(ny1, m3);
      const size_t nc3 = (size_t)op->tl3_nax * op->tl3_nay;
      const size_t ncp3 = (size_t)coarse_row_stride(op->tl3_nax) * op->tl3_nay;
      A(&op->tl3_A1, (size_t)9 * (nx1 + 1) * (ny1 + 1) * sizeof(double));
      A(&op->tl3_Ac, nc3 * nc3 * sizeof(double));
      A(&op->tl3_band, nc3 * (op->tl3_nax + 2) * sizeof(float));
      A(&op->tl3_X, nc3 * nc3 * sizeof(float));
      A(&op->tl3_Ainv, ncp3 * ncp3 * sizeof(float));
    }
  }
  // streamed coarse-step solves: coarse_stream = 2 where the grid coarsens at least once, or 0 on
  // grids of kCoarseStreamMinNodes nodes or more with at least three levels
  const int mgL = mg_level_count(grid->nx, grid->ny);
  if ((solve->coarse_stream == 2 && mgL >= 2) ||
      (solve->coarse_stream == 0 && op->Nn >= kCoarseStreamMinNodes && mgL >= 3))
    op->mg_L = mgL;
  // streamed fine propagators: fine_stream = 2, or 0 on grids of kWideMinNodes nodes or more
  // (the plan streams only where no cluster holds a slice); their CG preconditioned by the
  // multigrid cycle of C/dt + K with local_steps = 3 (at least two levels), or by default with at
  // least three levels
  const bool fine_st = solve->fine_stream == 2 || (solve->fine_stream == 0 && op->Nn >= kWideMinNodes);
  if (fine_st && ((solve->local_steps == 3 && mgL >= 2) || (solve->local_steps == 0 && mgL >= 3))) op->mg_Lf = mgL;
  if (fine_st || op->mg_L > 0) {
    int dev_sm = 0;
    cudaDeviceGetAttribute(&dev_sm, cudaDevAttrMultiProcessorCount, device);
    op->st_groups = std::max(1, std::min(time->Ntau, std::min(dev_sm, kMaxGrid)));
    const size_t ng = (size_t)op->st_groups + 1;
    const size_t PNs = (size_t)(grid->ny + 3) * op->W + 2 * kSlack;
    const size_t PEs = (size_t)(grid->ny + 2) * op->W + 2 * kSlack;
    // CG vectors in the precision of each streamed kind's CG
    const int pf = kind_precision(solve->precision, KIND_FINE_PRI), pc = kind_precision(solve->precision, KIND_COARSE_PRI);
    const bool f64 = (fine_st && pf == PTG_FP64) || (op->mg_L > 0 && pc == PTG_FP64);
    const bool f32 = (fine_st && pf != PTG_FP64) || (op->mg_L > 0 && pc != PTG_FP64);
    A(&op->w32, 3 * PEs * sizeof(float));
    A(&op->w32_inv, PNs * sizeof(float));
    A(&op->w64_inv, PNs * sizeof(double));
    A(&op->st_w64, ng * 3 * PNs * sizeof(double));
    if (f64) A(&op->st_wr, ng * 5 * PNs * sizeof(double));
    if (f32) A(&op->st_wr32, ng * 5 * PNs * sizeof(float));
    // the padded vectors are zero outside the unknowns; only unknowns are ever written
    if (e == cudaSuccess) e = cudaMemset(op->st_w64, 0, ng * 3 * PNs * sizeof(double));
    if (e == cudaSuccess && f64) e = cudaMemset(op->st_wr, 0, ng * 5 * PNs * sizeof(double));
    if (e == cudaSuccess && f32) e = cudaMemset(op->st_wr32, 0, ng * 5 * PNs * sizeof(float));
    if (op->mg_L > 0 || op->mg_Lf > 0) {
      long long wsf = 0;
      const long long wf = mg_layout(grid->nx, grid->ny, op->mg_lv, std::max(op->mg_L, op->mg_Lf), &wsf);
      op->mg_ws_stride = wsf;
      A(&op->mg_ws, ng * (size_t)wsf * sizeof(float));
      A(&op->sw_red, 2 * kMaxGrid * 4 * sizeof(double));
      A(&op->sw_bar, 4 * sizeof(unsigned));
      // rows and columns outside each level's grid and the slack stay zero
      if (e == cudaSuccess) e = cudaMemset(op->mg_ws, 0, ng * (size_t)wsf * sizeof(float));
      for (float** w : {op->mg_L > 0 ? &op->mg_w : nullptr, op->mg_Lf > 0 ? &op->mg_wf : nullptr}) {
        if (!w) continue;
        A(w, (size_t)wf * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(*w, 0, (size_t)wf * sizeof(float));
      }
    }
  }
  A(&op->scratch, 2 * sizeof(double));
  A(&op->g_red, 2 * kMaxGrid * 4 * sizeof(double));
  A(&op->g_bar, 4 * kMaxGrid * sizeof(unsigned));
  A(&op->g_halo, (size_t)2 * kMaxGrid * 2 * op->W * sizeof(double));
  A(&op->stats, sizeof(DevStats));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(op);
    delete op;
    return PTG_ENOMEM;
  }
  double* tmp = new (std::nothrow) double[std::max(op->Ne, time->Nt + 1)];
  if (!tmp) {
    free_all(op);
    delete op;
    return PTG_ENOMEM;
  }
  for (int i = 0; i < op->Ne; ++i) tmp[i] = q_elem_h ? q_elem_h[i] : 1.0;
  e = cudaMemcpy(op->q_elem, tmp, op->Ne * sizeof(double), cudaMemcpyHostToDevice);
  for (int i = 0; i <= time->Nt; ++i) tmp[i] = q_time_h ? q_time_h[i] : 1.0;
  if (e == cudaSuccess) e = cudaMemcpy(op->q_time, tmp, (time->Nt + 1) * sizeof(double), cudaMemcpyHostToDevice);
  delete[] tmp;
  if (e == cudaSuccess) e = cudaMemcpy(op->dirichlet, dirichlet_h, op->Nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(op->stats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(op->fload, 0, op->Nn * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(op->wE, 0, 6 * PEe * sizeof(double));          // slack stays zero
  if (e == cudaSuccess) e = cudaMemset(op->nodew, 0, 15 * PN * sizeof(double));
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "ptg_op_create");
    free_all(op);
    delete op;
    return rc;
  }
  // the grid must fit one cluster for every kind and precision this op may run
  Plan probe;
  for (int kind = 0; kind < 6; ++kind) {
    int rc = choose_plan(op, kind_precision(op->sv.precision, kind), kind, 1, &probe);
    if (rc != PTG_OK) {
      free_all(op);
      delete op;
      return rc;
    }
  }
  if (solve->coarse_mesh) {
    int rc = create_mesh(op, dirichlet_h, q_elem_h, q_time_h);
    if (rc != PTG_OK) {
      free_all(op);
      delete op;
      return rc;
    }
  }
  *out = op;
  return PTG_OK;
}

void ptg_op_destroy(ptg_op* op) {
  if (!op) return;
  DeviceGuard dg(op->device);
  cudaDeviceSynchronize();
  ptg_op_free(op);
}

int ptg_op_sizes(const ptg_op* op, int* Nn, int* Ne, int* Nt, int* Ntau, int* M) {
  if (!op) return PTG_EINVAL;
  if (Nn) *Nn = op->Nn;
  if (Ne) *Ne = op->Ne;
  if (Nt) *Nt = op->tm.Nt;
  if (Ntau) *Ntau = op->tm.Ntau;
  if (M) *M = op->M;
  return PTG_OK;
}

int ptg_op_set_plan(ptg_op* op, int kind, int cs, int ng) {
  if (!op || kind < 0 || kind > 5) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  std::lock_guard<std::mutex> lk(op->mu);
  if (cs == 0) {
    op->plan_override.erase(kind);
    return PTG_OK;
  }
  if ((kind == KIND_CORRECT_PRI || kind == KIND_CORRECT_ADJ) && op->mg_L > 0 && op->st_groups > 0) {
    // a streamed correction sweep: one group of cs CTAs (at most one per SM, >= 2 rows each)
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cs < 1 || cs > std::min(nsm, kMaxGrid) || cs > (op->g.ny + 1) / 2) return PTG_EINVAL;
    Plan sp;
    sp.cs = cs;
    sp.nthreads = 512;
    sp.ng = 1;
    sp.rmax = (op->g.ny + 1 + cs - 1) / cs;
    sp.max_active_clusters = 1;
    sp.stream = true;
    op->plan_override[kind] = sp;
    return PTG_OK;
  }
  if (cs != 1 && cs != 2 && cs != 4 && cs != 8 && cs != 16) return PTG_EINVAL;
  const int rmax = (op->g.ny + 1 + cs - 1) / cs;
  if (rmax < 2) return PTG_EINVAL;
  const int groups = rmax * (op->W / kGroup);
  if (ng < 1 || ng > kStepNG[kNumStepNG - 1]) return PTG_EINVAL;
  const int nthreads = ((groups + ng - 1) / ng + 31) / 32 * 32;
  if (nthreads > kStepMaxThreadsHost) return PTG_EINVAL;
  // with the strongest two-level form where it applies and fits, else with Jacobi
  for (int mode = strongest_mode(op); mode >= TL_NONE; --mode) {
    const int prec = kind_precision(op->sv.precision, kind);
    if (mode > TL_NONE && twolevel_rows(op, prec, kind, cs, mode) == 0) continue;
    for (bool keep_ax : {true, false}) {
      Plan p;
      cudaError_t e = query_stepper_plan(op->g.nx, op->g.ny, prec, kind, cs, ng, nthreads,
                                         twolevel_bytes(op, prec, kind, cs, mode), &p, keep_ax);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (p.max_active_clusters <= 0) continue;
      p.twolevel = mode > TL_NONE;
      p.vc = uses_vcycle(op, mode);
      p.l3 = uses_three(op, mode);
      op->plan_override[kind] = p;
      return PTG_OK;
    }
  }
  return PTG_EINVAL;
}

int ptg_op_set_multigrid(ptg_op* op, int solo_rows, int coarse_steps, int fused) {
  if (!op || solo_rows < 0 || coarse_steps < 0 || coarse_steps > 64 || fused < -1 || fused > 1) return PTG_EINVAL;
  op->mg_solo = solo_rows;
  op->mg_csteps = coarse_steps;
  op->mg_fuse = fused;
  return PTG_OK;
}

int ptg_op_get_plan(ptg_op* op, int kind, int ntasks, int* cs, int* nthreads, int* ng, int* max_active_clusters) {
  if (!op || kind < 0 || kind > 5 || ntasks < 1) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  Plan p;
  int rc = choose_plan(op, kind_precision(op->sv.precision, kind), kind, ntasks, &p);
  if (rc != PTG_OK) return rc;
  if (cs) *cs = p.cs;
  if (nthreads) *nthreads = p.nthreads;
  if (ng) *ng = p.ng;
  if (max_active_clusters) *max_active_clusters = p.max_active_clusters;
  return PTG_OK;
}

int ptg_fe_assemble_operator(ptg_op* op, const double* rho_d, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !rho_d) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  op->last_stream = stream;
  AssembleOut out;
  out.k = op->k;
  out.c = op->c;
  out.dk = op->dk;
  out.dc = op->dc;
  const size_t PEe = (size_t)(op->g.ny + 2) * op->W + 2 * kSlack;
  const size_t PN = (size_t)(op->g.ny + 3) * op->W + 2 * kSlack;
  out.wEf = op->wE + kSlack;
  out.wEc = op->wE + 3 * PEe + kSlack;
  for (int i = 0; i < 15; ++i) out.node[i] = op->nodew + i * PN + kSlack;
  out.fload = op->fload;
  PTG_CUDA(launch_assemble(op->g.nx, op->g.ny, op->g.h, op->mat, op->tm.dt, op->dtau, rho_d, op->q_elem,
                           op->dirichlet, out, op->stats, stream));
  if (op->w32)
    PTG_CUDA(launch_stream_weights((int)PEe, (int)PN, op->wE, op->nodew, op->dirichlet, op->g.nx, op->g.ny, op->W,
                                   op->w32, op->w32_inv, op->w64_inv, stream));
  if (op->mg_L > 0) {
    NodeWeights Ac{out.node[5], out.node[6], out.node[7], out.node[8], out.node[9]};
    PTG_CUDA(launch_mg_setup(Ac, op->dirichlet, op->mg_lv, op->mg_L, op->mg_w, stream));
  }
  if (op->mg_Lf > 0) {
    NodeWeights Af{out.node[0], out.node[1], out.node[2], out.node[3], out.node[4]};
    PTG_CUDA(launch_mg_setup(Af, op->dirichlet, op->mg_lv, op->mg_Lf, op->mg_wf, stream));
  }
  if (op->tl_m) {
    NodeWeights Ac;
    Ac.C = out.node[5];
    Ac.E = out.node[6];
    Ac.N = out.node[7];
    Ac.NE = out.node[8];
    Ac.NW = out.node[9];
    PTG_CUDA(launch_coarse_setup(op->g.nx, op->g.ny, op->W, op->tl_m, Ac, op->dirichlet, op->tl_Ac, op->tl_band,
                                 op->tl_X, op->tl_Ainv, stream));
    if (op->tl3_m > 0)
      PTG_CUDA(launch_threelevel_setup(op->g.nx, op->g.ny, op->W, Ac, op->dirichlet, op->tl3_m, op->tl3_A1,
                                       op->tl3_Ac, op->tl3_band, op->tl3_X, op->tl3_Ainv, stream));
  }
  if (op->mesh) {                // the 2h-mesh op on the averaged design
    PTG_CUDA(mesh_design(op->g.nx, op->g.ny, rho_d, op->mesh_rho, stream));
    return ptg_fe_assemble_operator(op->mesh, op->mesh_rho, stream);
  }
  return PTG_OK;
}

int ptg_fine_propagate_slices(ptg_op* op, int schedule, int s0, int ns, const double* U_T, const double* U_theta,
                              double* T_hist, int hist_j0, int hist_rows, double* F_T, double* F_theta,
                              cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !U_T || !U_theta || !F_T || !F_theta) return PTG_EINVAL;
  if (schedule != PTG_SLICES_PARALLEL && schedule != PTG_SLICES_CHAINED) return PTG_EINVAL;
  if (s0 < 0 || ns < 1 || s0 + ns > op->tm.Ntau) return PTG_EINVAL;
  if (T_hist && !window_covers(hist_j0, hist_rows, op->M * s0 + 1, op->M * (s0 + ns))) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  StepParams P;
  base_params(op, P);
  P.kind = KIND_FINE_PRI;
  P.s0 = s0;
  P.ns = ns;
  P.chained = schedule == PTG_SLICES_CHAINED;
  P.in_field = U_T;
  P.in_aux = U_theta;
  P.out_field = F_T;
  P.out_aux = F_theta;
  P.hist = T_hist;
  P.hist_j0 = hist_j0;
  P.hist_rows = T_hist ? hist_rows : 0;
  return run(op, P, P.chained ? 1 : ns, stream);
}

int ptg_coarse_sweep(ptg_op* op, int direction, const double* X_field, const double* X_aux, const double* T_hist,
                     const double* Theta_d, double* G_field, double* G_aux, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op) return PTG_EINVAL;
  return ptg_coarse_sweep_slices(op, direction, 0, op->tm.Ntau, X_field, X_aux, T_hist, Theta_d, G_field, G_aux,
                                 stream);
}

int ptg_coarse_sweep_slices(ptg_op* op, int direction, int s0, int ns, const double* X_field, const double* X_aux,
                            const double* T_hist, const double* Theta_d, double* G_field, double* G_aux,
                            cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !X_field || !X_aux || !G_field || !G_aux) return PTG_EINVAL;
  if (direction != PTG_PRIMAL && direction != PTG_ADJOINT) return PTG_EINVAL;
  if (direction == PTG_ADJOINT && (!T_hist || !Theta_d)) return PTG_EINVAL;
  if (s0 < 0 || ns < 1 || s0 + ns > op->tm.Ntau) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  if (op->mesh) {
    if (s0 != 0 || ns != op->tm.Ntau) return PTG_EINVAL;   // the 2h-mesh G runs every slice
    op->last_stream = stream;
    return mesh_coarse_sweep(op, direction, X_field, X_aux, T_hist, Theta_d, G_field, G_aux, stream);
  }
  StepParams P;
  base_params(op, P);
  P.kind = direction == PTG_PRIMAL ? KIND_COARSE_PRI : KIND_COARSE_ADJ;
  P.s0 = s0;
  P.ns = ns;
  P.in_field = X_field;
  P.in_aux = X_aux;
  P.out_field = G_field;
  P.out_aux = G_aux;
  P.hist = const_cast<double*>(T_hist);
  P.hist_j0 = 0;
  P.hist_rows = T_hist ? op->tm.Nt + 1 : 0;
  P.Theta = Theta_d;
  return run(op, P, ns, stream);
}

int ptg_coarse_adjoint_split(ptg_op* op, int s0, int ns, const double* V_lam, const double* V_g, const double* T_hist,
                             double* H_lam, double* H_g, double* S_lam, double* S_g, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !V_lam || !V_g || !T_hist || !H_lam || !H_g || !S_lam || !S_g) return PTG_EINVAL;
  if (s0 < 0 || ns < 1 || s0 + ns > op->tm.Ntau) return PTG_EINVAL;
  if (op->mesh) return PTG_EINVAL;                       // the 2h-mesh G has its own adjoint path
  DeviceGuard dg(op->device);
  for (int part = 1; part <= 2; ++part) {
    StepParams P;
    base_params(op, P);
    P.kind = KIND_COARSE_ADJ;
    P.s0 = s0;
    P.ns = ns;
    P.src_mode = part;
    P.in_field = V_lam;
    P.in_aux = V_g;
    P.out_field = part == 1 ? H_lam : S_lam;
    P.out_aux = part == 1 ? H_g : S_g;
    P.hist = const_cast<double*>(T_hist);
    P.hist_j0 = 0;
    P.hist_rows = op->tm.Nt + 1;
    P.Theta = nullptr;
    const int rc = run(op, P, ns, stream);
    if (rc != PTG_OK) return rc;
  }
  return PTG_OK;
}

int ptg_op_overlap_ok(ptg_op* op, int* ok) {
  if (!op || !ok) return PTG_EINVAL;
  *ok = 0;
  if (op->M < 2 || op->mesh) return PTG_OK;
  DeviceGuard dg(op->device);
  Plan pc, pa;
  int rc = choose_plan(op, kind_precision(op->sv.precision, KIND_CORRECT_PRI), KIND_CORRECT_PRI, 1, &pc);
  if (rc == PTG_OK)
    rc = choose_plan(op, kind_precision(op->sv.precision, KIND_COARSE_ADJ), KIND_COARSE_ADJ, op->tm.Ntau, &pa);
  if (rc != PTG_OK) return rc;
  // a streamed sweep has its own workspace, partials and barrier; a streamed G_adj shares the op's
  // grid partials with cooperative-grid stepper plans, and its workspace and partials with a
  // streamed F_adj, which must then wait for it (2)
  if (!((!pc.wide || pc.stream) && !pa.wide)) return PTG_OK;
  *ok = 1;
  if (pa.stream) {
    Plan pf;
    rc = choose_plan(op, kind_precision(op->sv.precision, KIND_FINE_ADJ), KIND_FINE_ADJ, op->tm.Ntau, &pf);
    if (rc != PTG_OK) return rc;
    if (pf.stream || pf.wide) *ok = 2;
  }
  return PTG_OK;
}

int ptg_coarse_adjoint_combine(ptg_op* op, int s0, int ns, const double* Theta_d, const double* H_lam,
                               const double* H_g, const double* S_lam, const double* S_g, double* G_lam, double* G_g,
                               cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !Theta_d || !H_lam || !H_g || !S_lam || !S_g || !G_lam || !G_g) return PTG_EINVAL;
  if (s0 < 0 || ns < 1 || s0 + ns > op->tm.Ntau) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  const long long Nn = op->Nn, Ne = (long long)op->g.nx * op->g.ny;
  const long long ol = (long long)s0 * Nn, og = (long long)s0 * Ne;
  op->last_stream = stream;
  PTG_CUDA(launch_adjoint_combine((long long)ns * Nn, (long long)ns * Ne, Theta_d, op->tm.p, (int)Ne,
                                  op->tm.objective == PTG_OBJ_MODIFIED, H_lam + ol, H_g + og, S_lam + ol, S_g + og,
                                  G_lam + ol, G_g + og, stream));
  return PTG_OK;
}

int ptg_parareal_correct(ptg_op* op, int direction, const double* F_field, const double* F_aux, const double* G_field,
                         const double* G_aux, double* X_field, double* X_aux, double* T_hist, const double* Theta_d,
                         cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !F_field || !F_aux || !X_field || !X_aux) return PTG_EINVAL;
  if ((G_field == nullptr) != (G_aux == nullptr)) return PTG_EINVAL;   // both NULL: PLT (G = 0)
  if (direction != PTG_PRIMAL && direction != PTG_ADJOINT) return PTG_EINVAL;
  if (direction == PTG_ADJOINT && (!T_hist || !Theta_d)) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  if (op->mesh && G_field) {
    op->last_stream = stream;
    return mesh_correct(op, direction, F_field, F_aux, G_field, G_aux, X_field, X_aux, T_hist, Theta_d, stream);
  }
  StepParams P;
  base_params(op, P);
  P.kind = direction == PTG_PRIMAL ? KIND_CORRECT_PRI : KIND_CORRECT_ADJ;
  P.s0 = 0;
  P.ns = op->tm.Ntau;
  P.F_field = F_field;
  P.F_aux = F_aux;
  P.G_field = G_field;
  P.G_aux = G_aux;
  P.plt = G_field == nullptr;
  P.out_field = X_field;
  P.out_aux = X_aux;
  P.hist = T_hist;
  P.hist_j0 = 0;
  P.hist_rows = T_hist ? op->tm.Nt + 1 : 0;
  P.Theta = Theta_d;
  return run(op, P, 1, stream);
}

int ptg_objective_from_modified(ptg_op* op, const double* Theta_mod_d, const double* grad_mod_d, double* Theta_d,
                                double* grad_d, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !Theta_mod_d || !grad_mod_d || !Theta_d || !grad_d) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  op->last_stream = stream;
  PTG_CUDA(launch_objective_from_modified(op->Ne, op->tm.p, Theta_mod_d, grad_mod_d, Theta_d, grad_d, op->scratch,
                                          stream));
  return PTG_OK;
}

int ptg_adjoint_sweep(ptg_op* op, int schedule, int s0, int ns, const double* T_hist, int hist_j0, int hist_rows,
                      const double* Theta_d, const double* V_lam, const double* V_g, double* F_lam, double* F_g,
                      cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !T_hist || !Theta_d || !V_lam || !V_g || !F_lam || !F_g) return PTG_EINVAL;
  if (schedule != PTG_SLICES_PARALLEL && schedule != PTG_SLICES_CHAINED) return PTG_EINVAL;
  if (s0 < 0 || ns < 1 || s0 + ns > op->tm.Ntau) return PTG_EINVAL;
  if (!window_covers(hist_j0, hist_rows, op->M * s0, op->M * (s0 + ns))) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  StepParams P;
  base_params(op, P);
  P.kind = KIND_FINE_ADJ;
  P.s0 = s0;
  P.ns = ns;
  P.chained = schedule == PTG_SLICES_CHAINED;
  P.in_field = V_lam;
  P.in_aux = V_g;
  P.out_field = F_lam;
  P.out_aux = F_g;
  P.hist = const_cast<double*>(T_hist);
  P.hist_j0 = hist_j0;
  P.hist_rows = hist_rows;
  P.Theta = Theta_d;
  return run(op, P, P.chained ? 1 : ns, stream);
}

int ptg_sensitivities(ptg_op* op, const double* lam_hist, int j0, int j1, const double* T_hist, int hist_j0,
                      int hist_rows, double* grad_d, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op || !lam_hist || !T_hist || !grad_d) return PTG_EINVAL;
  if (j0 < 1 || j1 < j0 || j1 > op->tm.Nt) return PTG_EINVAL;
  if (!window_covers(hist_j0, hist_rows, j0 - 1, j1)) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  op->last_stream = stream;
  PTG_CUDA(launch_sensitivities(op->g.nx, op->g.ny, op->tm.Nt, op->g.h, op->tm.dt, op->has_dc, op->dk, op->dc,
                                lam_hist, j0, j1, T_hist, hist_j0, op->sens_partial, op->sens_chunks, grad_d, stream));
  return PTG_OK;
}

int ptg_get_stats(ptg_op* op, ptg_stats* out) {
  if (!op || !out) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  DevStats s;
  PTG_CUDA(cudaStreamSynchronize(op->last_stream));
  PTG_CUDA(cudaMemcpy(&s, op->stats, sizeof(s), cudaMemcpyDeviceToHost));
  out->status = s.status;
  out->fail_kind = s.fail_kind;
  out->fail_step = s.fail_step;
  if (s.status == PTG_OK && op->dbg_status != PTG_OK) {
    out->status = op->dbg_status;
    out->fail_kind = op->dbg_kind;
    out->fail_step = op->dbg_site;
  }
  out->reserved = 0;
  out->solves = (long long)s.solves;
  out->cg_iters = (long long)s.cg_iters;
  out->refinements = (long long)s.refinements;
  out->max_cg_iters = (long long)s.max_cg_iters;
  for (int k = 0; k < 6; ++k) {
    out->kind_solves[k] = (long long)s.kind_solves[k];
    out->kind_cg_iters[k] = (long long)s.kind_cg_iters[k];
    out->kind_refinements[k] = (long long)s.kind_refinements[k];
  }
  return PTG_OK;
}

int ptg_op_set_wait_limit(ptg_op* op, long long polls) {
  if (!op || polls < 0) return PTG_EINVAL;
  std::lock_guard<std::mutex> lk(op->mu);
  op->wait_limit = polls;
  return PTG_OK;
}

int ptg_reset_stats(ptg_op* op, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!op) return PTG_EINVAL;
  DeviceGuard dg(op->device);
  op->last_stream = stream;
  op->dbg_status = op->dbg_kind = op->dbg_site = 0;
  PTG_CUDA(cudaMemsetAsync(op->stats, 0, sizeof(DevStats), stream));
  return PTG_OK;
}

}  // extern "C"

// =========================================================================== batches
// Several designs (ops, possibly of different grid sizes) advanced together: one persistent
// multi-design launch per phase of the pass, every cluster taking (design, task) pairs from a
// work queue, largest designs first.

namespace {

// 0..5: one-shot kinds; 6: sequential primal; 7: sequential adjoint; 8, 9: primal and adjoint
// corrections of the PLT variant (G = 0)
constexpr int kPhases = 10;

struct BatchBuf {
  double *T_hist, *U_T, *U_th, *V_l, *V_g, *U_T_new, *U_th_new, *V_l_new, *V_g_new;
  double *F_T, *F_th, *G_T, *G_th, *F_l, *F_g, *G_l, *G_g, *rho;
  double* lam_prev;   // [n Ntau][Nn] fine-step initial guesses (null when the op starts plainly)
};

struct PhasePlan {
  Plan plan;
  int nclusters = 0;
  int ntasks = 0;
  StepParams* table = nullptr;   // device, one per design
  int2* tasks = nullptr;         // device
  bool ready = false;
};

int phase_kind(int ph) {
  if (ph < 6) return ph;
  if (ph == 6) return KIND_FINE_PRI;
  if (ph == 7) return KIND_FINE_ADJ;
  return ph == 8 ? KIND_CORRECT_PRI : KIND_CORRECT_ADJ;
}

}  // namespace

struct ptg_batch {
  int device = 0;
  int precision = 0;
  std::vector<ptg_op*> ops;
  // designs whose op streams its coarse-step solves (ptg_solve.coarse_stream): the passes run
  // them through the op's own launches on the batch's buffers, not in the persistent launches,
  // whose geometry is then sized by the other designs
  std::vector<char> own;
  // their correction sweeps run side by side, each on a group of kBatchSweepCtas CTAs, on
  // streams forked from and joined to the caller's stream
  std::vector<cudaStream_t> side;
  int nsweep_side = 0;           // side streams the streamed sweeps use (as many as fit the chip)
  cudaEvent_t fork = nullptr, fork2 = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<BatchBuf> bufs;
  std::vector<void*> allocs;
  std::vector<int> order;        // design indices, largest first
  PhasePlan ph[kPhases];
  int* queue = nullptr;          // [kPhases]
  std::mutex mu;
};

namespace {

void batch_free(ptg_batch* b) {
  for (void* p : b->allocs)
    if (p) cudaFree(p);
  b->allocs.clear();
  for (cudaStream_t s : b->side)
    if (s) cudaStreamDestroy(s);
  b->side.clear();
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  b->join.clear();
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->fork2) cudaEventDestroy(b->fork2);
  b->fork = b->fork2 = nullptr;
  for (auto& p : b->ph) {
    if (p.table) cudaFree(p.table);
    if (p.tasks) cudaFree(p.tasks);
    p.table = nullptr;
    p.tasks = nullptr;
  }
  if (b->queue) cudaFree(b->queue);
  b->queue = nullptr;
}

// Design d runs in the persistent launch of phase ph (the sequential phases take every design).
bool in_launch(const ptg_batch* b, int d, int ph) { return ph == 6 || ph == 7 || !b->own[d]; }

// Per-design parameters of one phase with cluster size cs.
StepParams phase_params(const ptg_batch* b, int d, int ph, int cs, int tl_mode, bool keep_ax) {
  const ptg_op* op = b->ops[d];
  const BatchBuf& B = b->bufs[d];
  StepParams P;
  base_params(op, P);
  P.cs = cs;
  P.rmax = (op->g.ny + 1 + cs - 1) / cs;
  P.kind = phase_kind(ph);
  P.stats_kind = P.kind;
  P.keep_ax = keep_ax ? 1 : 0;
  P.prev_field = B.lam_prev;   // the batch's own workspace: an op may appear twice
  P.s0 = 0;
  P.ns = op->tm.Ntau;
  P.hist = B.T_hist;
  P.hist_j0 = 0;
  P.hist_rows = op->tm.Nt + 1;
  twolevel_params(op, kind_precision(b->precision, P.kind), P, tl_mode);
  const int Ntau = op->tm.Ntau;
  switch (ph) {
    case 0:  P.in_field = B.U_T; P.in_aux = B.U_th; P.out_field = B.F_T; P.out_aux = B.F_th; break;
    case 1:  P.in_field = B.U_T; P.in_aux = B.U_th; P.out_field = B.G_T; P.out_aux = B.G_th; break;
    case 2:
      P.in_field = B.U_T; P.in_aux = B.U_th; P.out_field = B.U_T_new; P.out_aux = B.U_th_new;
      P.F_field = B.F_T; P.F_aux = B.F_th; P.G_field = B.G_T; P.G_aux = B.G_th;
      break;
    case 3:
      P.in_field = B.V_l; P.in_aux = B.V_g; P.out_field = B.F_l; P.out_aux = B.F_g; P.Theta = B.U_th_new + Ntau;
      break;
    case 4:
      P.in_field = B.V_l; P.in_aux = B.V_g; P.out_field = B.G_l; P.out_aux = B.G_g; P.Theta = B.U_th_new + Ntau;
      break;
    case 5:
      P.out_field = B.V_l_new; P.out_aux = B.V_g_new; P.F_field = B.F_l; P.F_aux = B.F_g; P.G_field = B.G_l;
      P.G_aux = B.G_g; P.Theta = B.U_th_new + Ntau;
      break;
    case 6:   // sequential primal: u_0 in U[0], checkpoints into U[1..]
      P.chained = 1; P.in_field = B.U_T; P.in_aux = B.U_th; P.out_field = B.U_T + op->Nn; P.out_aux = B.U_th + 1;
      break;
    case 7:   // sequential adjoint: v_Ntau = 0 in V[Ntau], checkpoints into V[0..Ntau-1]
      P.chained = 1; P.in_field = B.V_l; P.in_aux = B.V_g; P.out_field = B.V_l; P.out_aux = B.V_g;
      P.Theta = B.U_th + Ntau;
      break;
    case 8:   // PLT primal correction: U_new[s+1] = F[s]
      P.plt = 1; P.in_field = B.U_T; P.in_aux = B.U_th; P.out_field = B.U_T_new; P.out_aux = B.U_th_new;
      P.F_field = B.F_T; P.F_aux = B.F_th;
      break;
    case 9:   // PLT adjoint correction: V_new[s] = F[s]
      P.plt = 1; P.out_field = B.V_l_new; P.out_aux = B.V_g_new; P.F_field = B.F_l; P.F_aux = B.F_g;
      P.Theta = B.U_th_new + Ntau;
      break;
  }
  return P;
}

// Tasks of a phase: (design, slice) for the parallel kinds, (design, 0) for the sweeps and the
// chained runs, largest designs first.
std::vector<int2> phase_tasks(const ptg_batch* b, int ph) {
  std::vector<int2> t;
  const bool per_slice = ph == 0 || ph == 1 || ph == 3 || ph == 4;
  for (int d : b->order) {
    if (!in_launch(b, d, ph)) continue;
    const int n = per_slice ? b->ops[d]->tm.Ntau : 1;
    for (int s = 0; s < n; ++s) t.push_back(make_int2(d, s));
  }
  return t;
}

// Install a plan for a phase: validate it for every design, upload the parameter table and
// the task list, and size the persistent grid.  tl_mode: the strongest two-level form the
// designs may use where it applies.
int batch_install(ptg_batch* b, int ph, int cs, int ng, int nthreads, int tl_mode, bool keep_ax = true) {
  const int kind = phase_kind(ph);
  const int prec = kind_precision(b->precision, kind);
  size_t smem = 0;
  for (int d = 0; d < (int)b->ops.size(); ++d) {
    if (!in_launch(b, d, ph)) continue;
    const ptg_op* op = b->ops[d];
    const int rmax = (op->g.ny + 1 + cs - 1) / cs;
    if (rmax < 2) return PTG_EINVAL;
    const int groups = rmax * (op->W / kGroup);
    if (groups > ng * nthreads) return PTG_EINVAL;
    smem = std::max(smem, stepper_smem_bytes(op->g.nx, rmax, prec == PTG_FP32_REFINE ? 4 : 8, keep_ax) +
                              twolevel_bytes(op, prec, kind, cs, tl_mode));
  }
  int nclusters = 0;
  if (query_batch_occupancy(prec, kind, cs, ng, nthreads, smem, &nclusters) != cudaSuccess || nclusters <= 0) {
    cudaGetLastError();
    return PTG_EINVAL;
  }
  std::vector<StepParams> table;
  for (int d = 0; d < (int)b->ops.size(); ++d) table.push_back(phase_params(b, d, ph, cs, tl_mode, keep_ax));
  std::vector<int2> tasks = phase_tasks(b, ph);
  PhasePlan& pp = b->ph[ph];
  if (!pp.table) PTG_CUDA(cudaMalloc(&pp.table, sizeof(StepParams) * table.size()));
  if (!pp.tasks) PTG_CUDA(cudaMalloc(&pp.tasks, sizeof(int2) * tasks.size()));
  PTG_CUDA(cudaMemcpy(pp.table, table.data(), sizeof(StepParams) * table.size(), cudaMemcpyHostToDevice));
  PTG_CUDA(cudaMemcpy(pp.tasks, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice));
  pp.plan.cs = cs;
  pp.plan.ng = ng;
  pp.plan.nthreads = nthreads;
  pp.plan.smem = smem;
  pp.plan.max_active_clusters = nclusters;
  pp.plan.twolevel = tl_mode > TL_NONE;
  pp.plan.vc = tl_mode >= TL_VCYCLE;
  pp.plan.keep_ax = keep_ax;
  pp.ntasks = (int)tasks.size();
  pp.nclusters = std::min(nclusters, pp.ntasks);
  pp.ready = true;
  return PTG_OK;
}

// Default plan of a phase: fewest waves, then the fewest groups per thread, then the largest
// cluster; the two-level preconditioner unless it needs more waves (the autotuner may replace
// the plan).
long batch_best(ptg_batch* b, int ph, int tl_mode, int ntasks, int* best_cs, int* best_ng, int* best_nt,
                bool keep_ax = true) {
  long best_waves = -1;
  const int prec = kind_precision(b->precision, phase_kind(ph));
  for (int cs : {16, 8, 4, 2}) {
    for (int ng : kStepNG) {
      int nt = 32;
      bool ok = true;
      size_t smem = 0;
      for (int d = 0; d < (int)b->ops.size(); ++d) {
        if (!in_launch(b, d, ph)) continue;
        const ptg_op* op = b->ops[d];
        const int rmax = (op->g.ny + 1 + cs - 1) / cs;
        if (rmax < 2) { ok = false; break; }
        const int groups = rmax * (op->W / kGroup);
        nt = std::max(nt, ((groups + ng - 1) / ng + 31) / 32 * 32);
        smem = std::max(smem, stepper_smem_bytes(op->g.nx, rmax, prec == PTG_FP32_REFINE ? 4 : 8, keep_ax) +
                                  twolevel_bytes(op, prec, phase_kind(ph), cs, tl_mode));
      }
      if (!ok || nt > kStepMaxThreadsHost) continue;
      int ncl = 0;
      if (query_batch_occupancy(prec, phase_kind(ph), cs, ng, nt, smem, &ncl) != cudaSuccess || ncl <= 0) {
        cudaGetLastError();
        continue;
      }
      const long waves = (ntasks + ncl - 1) / ncl;
      if (best_waves < 0 || waves < best_waves || (waves == best_waves && ng < *best_ng)) {
        best_waves = waves;
        *best_cs = cs;
        *best_ng = ng;
        *best_nt = nt;
      }
    }
  }
  return best_waves;
}

// The strongest two-level form of any design of the batch for a phase (TL_NONE: none applies).
int batch_twolevel_mode(const ptg_batch* b, int ph) {
  if (ph >= 8) return TL_NONE;   // the PLT corrections solve nothing
  int mode = TL_NONE;
  for (int d = 0; d < (int)b->ops.size(); ++d)
    if (in_launch(b, d, ph) && twolevel_rows(b->ops[d], b->precision, phase_kind(ph), 1) > 0)
      mode = std::max(mode, strongest_mode(b->ops[d]));
  return std::min(mode, (int)TL_VCYCLE);   // batches run at most the two-grid cycle
}

int batch_default(ptg_batch* b, int ph) {
  const int ntasks = (int)phase_tasks(b, ph).size();
  int jc = 0, jg = 0, jt = 0;
  bool jkeep = true;
  long wj = batch_best(b, ph, TL_NONE, ntasks, &jc, &jg, &jt);
  if (wj < 0) {
    jkeep = false;
    wj = batch_best(b, ph, TL_NONE, ntasks, &jc, &jg, &jt, false);
  }
  const bool fp64 = kind_precision(b->precision, phase_kind(ph)) == PTG_FP64;
  // the strongest two-level form that fits, leaving out the saved A x if that makes it fit
  for (int mode = batch_twolevel_mode(b, ph); mode > TL_NONE; --mode) {
    for (bool keep_ax : {true, false}) {
      int tc = 0, tg = 0, tt = 0;
      const long wt = batch_best(b, ph, mode, ntasks, &tc, &tg, &tt, keep_ax);
      if (wt >= 0 && (wj < 0 || wt <= wj || fp64)) return batch_install(b, ph, tc, tg, tt, mode, keep_ax);
    }
  }
  if (wj < 0) return PTG_EINVAL;
  return batch_install(b, ph, jc, jg, jt, TL_NONE, jkeep);
}

// CTAs of the group of a batched design's streamed correction sweep: nine such sweeps fill the
// chip side by side (measured at 256 x 256: 71 ms for 64 steps on 16 CTAs, against 45 ms alone
// on 128 CTAs, one after the other).
constexpr int kBatchSweepCtas = 16;
constexpr int kBatchSideStreams = 24;
// Designs of this many nodes or more take their own path in a batch even with on-chip solves:
// the persistent launch's geometry is sized by its largest design, and their own cluster
// launches run beside it.  Measured on the 48-design workload: 1.98 s per batched pass with
// 15000 (128 x 128 and larger on their own path), 2.12 s with 30000, 2.60 s with only the
// streamed designs on it; 9000 gained nothing over 15000.
constexpr int kBatchOwnMinNodes = 15000;

// Phase ph of design d through its op's own launches (the per-op entry points on the batch's
// buffers), as a single-design pass runs it.
int batch_own_phase(ptg_batch* b, int d, int ph, cudaStream_t st) {
  ptg_op* op = b->ops[d];
  const BatchBuf& B = b->bufs[d];
  const int Ntau = op->tm.Ntau, Nt = op->tm.Nt;
  const double* Theta = B.U_th_new + Ntau;
  switch (ph) {
    case 0:
      return ptg_fine_propagate_slices(op, PTG_SLICES_PARALLEL, 0, Ntau, B.U_T, B.U_th, B.T_hist, 0, Nt + 1, B.F_T,
                                       B.F_th, st);
    case 1: return ptg_coarse_sweep(op, PTG_PRIMAL, B.U_T, B.U_th, nullptr, nullptr, B.G_T, B.G_th, st);
    case 2:
    case 8:   // u_0 of the corrected states, then the sweep (G = 0 for PLT)
      PTG_CUDA(cudaMemcpyAsync(B.U_T_new, B.U_T, (size_t)op->Nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
      PTG_CUDA(cudaMemcpyAsync(B.U_th_new, B.U_th, sizeof(double), cudaMemcpyDeviceToDevice, st));
      return ptg_parareal_correct(op, PTG_PRIMAL, B.F_T, B.F_th, ph == 8 ? nullptr : B.G_T, ph == 8 ? nullptr : B.G_th,
                                  B.U_T_new, B.U_th_new, B.T_hist, nullptr, st);
    case 3:
      return ptg_adjoint_sweep(op, PTG_SLICES_PARALLEL, 0, Ntau, B.T_hist, 0, Nt + 1, Theta, B.V_l, B.V_g, B.F_l,
                               B.F_g, st);
    case 4: return ptg_coarse_sweep(op, PTG_ADJOINT, B.V_l, B.V_g, B.T_hist, Theta, B.G_l, B.G_g, st);
    case 5:
    case 9:
      return ptg_parareal_correct(op, PTG_ADJOINT, B.F_l, B.F_g, ph == 9 ? nullptr : B.G_l, ph == 9 ? nullptr : B.G_g,
                                  B.V_l_new, B.V_g_new, B.T_hist, Theta, st);
    default: return PTG_EINVAL;
  }
}

// A design's own launches of phase ph are cluster launches (no cooperative grid): they can run
// beside the persistent launch, which they need not be co-resident with.
bool own_beside(ptg_batch* b, int d, int ph) {
  if (ph == 8 || ph == 9) return true;   // the PLT corrections: copies
  ptg_op* op = b->ops[d];
  const int kind = phase_kind(ph);
  const int ntasks = (kind == KIND_CORRECT_PRI || kind == KIND_CORRECT_ADJ) ? 1 : op->tm.Ntau;
  Plan p;
  return choose_plan(op, kind_precision(op->sv.precision, kind), kind, ntasks, &p) == PTG_OK && !p.stream && !p.wide;
}

// Phase ph: the persistent launch of the designs in it on `stream`; the designs on their own path
// (a) with cluster launches beside it on the side streams, forked before it, and (b) with
// streamed launches after it: correction sweeps side by side on the side streams (each on a
// group of kBatchSweepCtas CTAs, a plan override of its op for that launch only), the rest one
// after the other on `stream`.  Every side stream used joins `stream` at the end.
#if PTG_TRACE_ENABLED
const char* const kPhaseTrace[kPhases] = {"fine primal",  "coarse primal",      "primal correction",
                                          "fine adjoint", "coarse adjoint",     "adjoint correction",
                                          "sequential primal", "sequential adjoint", "primal copy (G = 0)",
                                          "adjoint copy (G = 0)"};
#endif

int batch_run(ptg_batch* b, int ph, cudaStream_t stream) {
#if PTG_TRACE_ENABLED
  PTG_TRACE(kPhaseTrace[ph]);
#endif
  std::vector<int> beside, after;
  for (int d : b->order) {
    if (in_launch(b, d, ph)) continue;
    (!b->side.empty() && own_beside(b, d, ph) ? beside : after).push_back(d);
  }
  const int nside = (int)b->side.size();
  std::vector<char> used(nside, 0);
  if (!beside.empty()) {
    PTG_CUDA(cudaEventRecord(b->fork, stream));
    for (size_t i = 0; i < beside.size(); ++i) {
      const int k = (int)(i % nside);
      if (!used[k]) PTG_CUDA(cudaStreamWaitEvent(b->side[k], b->fork, 0));
      used[k] = 1;
      int rc = batch_own_phase(b, beside[i], ph, b->side[k]);
      if (rc != PTG_OK) return rc;
    }
  }
  {
    std::lock_guard<std::mutex> lk(b->mu);
    if (!phase_tasks(b, ph).empty()) {
      if (!b->ph[ph].ready) {
        int rc = batch_default(b, ph);
        if (rc != PTG_OK) return rc;
      }
      const PhasePlan& pp = b->ph[ph];
      PTG_CUDA(launch_stepper_batch(kind_precision(b->precision, phase_kind(ph)), phase_kind(ph), pp.plan, pp.table,
                                    pp.tasks, pp.ntasks, b->queue + ph, pp.nclusters, stream));
    }
  }
  const bool sweep = ph == 2 || ph == 5;
  if (sweep && after.size() >= 2 && b->nsweep_side > 0) {
    PTG_CUDA(cudaEventRecord(b->fork2, stream));
    const int kind = phase_kind(ph);
    for (size_t i = 0; i < after.size(); ++i) {
      const int k = (int)(i % b->nsweep_side);
      PTG_CUDA(cudaStreamWaitEvent(b->side[k], b->fork2, 0));
      used[k] = 1;
      ptg_op* op = b->ops[after[i]];
      Plan saved;
      bool had = false;
      {
        std::lock_guard<std::mutex> lk(op->mu);
        auto it = op->plan_override.find(kind);
        had = it != op->plan_override.end();
        if (had) saved = it->second;
        Plan sp;
        sp.cs = std::max(1, std::min(kBatchSweepCtas, (op->g.ny + 1) / 2));
        sp.nthreads = 512;
        sp.ng = 1;
        sp.rmax = (op->g.ny + 1 + sp.cs - 1) / sp.cs;
        sp.max_active_clusters = 1;
        sp.stream = true;
        op->plan_override[kind] = sp;
      }
      const int rc = batch_own_phase(b, after[i], ph, b->side[k]);
      {
        std::lock_guard<std::mutex> lk(op->mu);
        if (had)
          op->plan_override[kind] = saved;
        else
          op->plan_override.erase(kind);
      }
      if (rc != PTG_OK) return rc;
    }
  } else {
    for (int d : after) {
      int rc = batch_own_phase(b, d, ph, stream);
      if (rc != PTG_OK) return rc;
    }
  }
  for (int k = 0; k < nside; ++k) {
    if (!used[k]) continue;
    PTG_CUDA(cudaEventRecord(b->join[k], b->side[k]));
    PTG_CUDA(cudaStreamWaitEvent(stream, b->join[k], 0));
  }
  for (ptg_op* op : b->ops) op->last_stream = stream;
  return PTG_OK;
}

}  // namespace

extern "C" {

int ptg_batch_create(ptg_op* const* ops, int nops, ptg_batch** out) {
  PTG_TRACE(__func__);
  if (!out) return PTG_EINVAL;
  *out = nullptr;
  if (!ops || nops < 1) return PTG_EINVAL;
  for (int d = 0; d < nops; ++d) {
    if (!ops[d]) return PTG_EINVAL;
    if (ops[d]->device != ops[0]->device || ops[d]->sv.precision != ops[0]->sv.precision) return PTG_EINVAL;
    if (ops[d]->mesh) return PTG_EINVAL;   // the persistent batch kernels run fine-mesh G only
  }
  DeviceGuard dg(ops[0]->device);
  ptg_batch* b = new (std::nothrow) ptg_batch();
  if (!b) return PTG_ENOMEM;
  b->device = ops[0]->device;
  b->precision = ops[0]->sv.precision;
  b->ops.assign(ops, ops + nops);
  int nown = 0;
  for (ptg_op* op : b->ops) {
    const bool own = op->mg_L > 0 || op->Nn >= kBatchOwnMinNodes;
    b->own.push_back(own ? 1 : 0);
    nown += own ? 1 : 0;
  }
  // an op that holds two designs would run two of its launches at once on its one workspace:
  // no side streams
  for (int x = 0; x < nops; ++x)
    for (int y = x + 1; y < nops; ++y)
      if (b->own[x] && ops[x] == ops[y]) nown = 0;
  cudaError_t e = cudaSuccess;
  auto A = [&](double** p, size_t n) {
    *p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void**)p, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, n * sizeof(double));
    b->allocs.push_back(*p);
  };
  for (ptg_op* op : b->ops) {
    const size_t Nn = op->Nn, Ne = op->Ne, Nt = op->tm.Nt, T = op->tm.Ntau;
    BatchBuf B;
    A(&B.T_hist, (Nt + 1) * Nn);
    A(&B.U_T, (T + 1) * Nn); A(&B.U_th, T + 1); A(&B.V_l, (T + 1) * Nn); A(&B.V_g, (T + 1) * Ne);
    A(&B.U_T_new, (T + 1) * Nn); A(&B.U_th_new, T + 1); A(&B.V_l_new, (T + 1) * Nn); A(&B.V_g_new, (T + 1) * Ne);
    A(&B.F_T, T * Nn); A(&B.F_th, T); A(&B.G_T, T * Nn); A(&B.G_th, T);
    A(&B.F_l, T * Nn); A(&B.F_g, T * Ne); A(&B.G_l, T * Nn); A(&B.G_g, T * Ne);
    A(&B.rho, Ne);
    B.lam_prev = nullptr;
    if (guess_states(op->sv) > 1) A(&B.lam_prev, guess_states(op->sv) * T * Nn);
    b->bufs.push_back(B);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->queue, kPhases * sizeof(int));
  if (nown >= 1) {
    // side streams: up to kBatchSideStreams for the cluster launches beside the persistent
    // launch; the first SMs / kBatchSweepCtas of them carry the streamed sweeps side by side
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    const int nside = std::max(1, std::min(nown, kBatchSideStreams));
    b->nsweep_side = std::max(1, std::min(nside, nsm / kBatchSweepCtas));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming);
    for (int k = 0; k < nside && e == cudaSuccess; ++k) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->side.push_back(st);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->join.push_back(ev);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return PTG_ENOMEM;
  }
  b->order.resize(nops);
  for (int d = 0; d < nops; ++d) b->order[d] = d;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    const long wx = (long)b->ops[x]->Nn * b->ops[x]->tm.Nt, wy = (long)b->ops[y]->Nn * b->ops[y]->tm.Nt;
    return wx > wy;
  });
  *out = b;
  return PTG_OK;
}

void ptg_batch_destroy(ptg_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  cudaDeviceSynchronize();
  batch_free(b);
  delete b;
}

int ptg_batch_buffers(ptg_batch* b, int d, ptg_pass_buffers* out) {
  if (!b || !out || d < 0 || d >= (int)b->ops.size()) return PTG_EINVAL;
  const BatchBuf& B = b->bufs[d];
  out->T_hist = B.T_hist;
  out->U_T = B.U_T; out->U_theta = B.U_th; out->V_lam = B.V_l; out->V_g = B.V_g;
  out->U_T_new = B.U_T_new; out->U_theta_new = B.U_th_new; out->V_lam_new = B.V_l_new; out->V_g_new = B.V_g_new;
  out->F_T = B.F_T; out->F_theta = B.F_th; out->G_T = B.G_T; out->G_theta = B.G_th;
  out->F_lam = B.F_l; out->F_g = B.F_g; out->G_lam = B.G_l; out->G_g = B.G_g;
  out->rho = B.rho;
  return PTG_OK;
}

int ptg_batch_assemble(ptg_batch* b, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!b) return PTG_EINVAL;
  for (int d = 0; d < (int)b->ops.size(); ++d) {
    int rc = ptg_fe_assemble_operator(b->ops[d], b->bufs[d].rho, stream);
    if (rc != PTG_OK) return rc;
  }
  return PTG_OK;
}

int ptg_batch_sequential_pass(ptg_batch* b, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!b) return PTG_EINVAL;
  DeviceGuard dg(b->device);
  int rc = batch_run(b, 6, stream);
  if (rc == PTG_OK) rc = batch_run(b, 7, stream);
  return rc;
}

int ptg_batch_oneshot_pass(ptg_batch* b, int variant, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!b || (variant != PTG_PARAREAL && variant != PTG_PLT)) return PTG_EINVAL;
  DeviceGuard dg(b->device);
  static const int parareal[] = {0, 1, 2, 3, 4, 5};
  static const int plt[] = {0, 8, 3, 9};
  const int* phases = variant == PTG_PLT ? plt : parareal;
  const int n = variant == PTG_PLT ? 4 : 6;
  for (int i = 0; i < n; ++i) {
    int rc = batch_run(b, phases[i], stream);
    if (rc != PTG_OK) return rc;
  }
  return PTG_OK;
}

int ptg_batch_commit(ptg_batch* b, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!b) return PTG_EINVAL;
  DeviceGuard dg(b->device);
  for (int d = 0; d < (int)b->ops.size(); ++d) {
    const ptg_op* op = b->ops[d];
    const BatchBuf& B = b->bufs[d];
    const size_t T1 = op->tm.Ntau + 1;
    PTG_CUDA(cudaMemcpyAsync(B.U_T, B.U_T_new, T1 * op->Nn * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    PTG_CUDA(cudaMemcpyAsync(B.U_th, B.U_th_new, T1 * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    PTG_CUDA(cudaMemcpyAsync(B.V_l, B.V_l_new, T1 * op->Nn * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    PTG_CUDA(cudaMemcpyAsync(B.V_g, B.V_g_new, T1 * op->Ne * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  }
  return PTG_OK;
}

int ptg_batch_run_phase(ptg_batch* b, int phase, cudaStream_t stream) {
  PTG_TRACE(__func__);
  if (!b || phase < 0 || phase >= kPhases) return PTG_EINVAL;
  DeviceGuard dg(b->device);
  return batch_run(b, phase, stream);
}

int ptg_batch_set_plan(ptg_batch* b, int phase, int cs, int ng, int nthreads) {
  if (!b || phase < 0 || phase >= kPhases) return PTG_EINVAL;
  if (cs != 2 && cs != 4 && cs != 8 && cs != 16) return PTG_EINVAL;
  if (ng < 1 || ng > kStepNG[kNumStepNG - 1] || nthreads < 32 || nthreads > kStepMaxThreadsHost || nthreads % 32)
    return PTG_EINVAL;
  DeviceGuard dg(b->device);
  std::lock_guard<std::mutex> lk(b->mu);
  // with the strongest two-level form where it applies and fits, else with Jacobi
  for (int mode = batch_twolevel_mode(b, phase); mode > TL_NONE; --mode)
    for (bool keep_ax : {true, false})
      if (batch_install(b, phase, cs, ng, nthreads, mode, keep_ax) == PTG_OK) return PTG_OK;
  if (batch_install(b, phase, cs, ng, nthreads, TL_NONE) == PTG_OK) return PTG_OK;
  return batch_install(b, phase, cs, ng, nthreads, TL_NONE, false);
}

int ptg_batch_design_path(ptg_batch* b, int design, int* own) {
  if (!b || !own || design < 0 || design >= (int)b->ops.size()) return PTG_EINVAL;
  *own = b->own[design] ? 1 : 0;
  return PTG_OK;
}

int ptg_batch_get_plan(ptg_batch* b, int phase, int* cs, int* ng, int* nthreads, int* nclusters) {
  if (!b || phase < 0 || phase >= kPhases) return PTG_EINVAL;
  DeviceGuard dg(b->device);
  std::lock_guard<std::mutex> lk(b->mu);
  if (!b->ph[phase].ready) {
    int rc = batch_default(b, phase);
    if (rc != PTG_OK) return rc;
  }
  const PhasePlan& pp = b->ph[phase];
  if (cs) *cs = pp.plan.cs;
  if (ng) *ng = pp.plan.ng;
  if (nthreads) *nthreads = pp.plan.nthreads;
  if (nclusters) *nclusters = pp.nclusters;
  return PTG_OK;
}

}  // extern "C"
