// ptg_internal.h -- structures shared by the host ABI layer and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ptg.h"

namespace ptg {

// Task kinds of the cluster stepper (one task per thread-block cluster).
enum Kind : int {
  KIND_FINE_PRI = 0,     // a2: F_pri of one slice (or all slices chained)
  KIND_COARSE_PRI = 1,   // a3: G_pri of one slice
  KIND_CORRECT_PRI = 2,  // a4: forward correction sweep (single task)
  KIND_FINE_ADJ = 3,     // a5: F_adj of one slice (or all slices chained)
  KIND_COARSE_ADJ = 4,   // a3: G_adj of one slice
  KIND_CORRECT_ADJ = 5,  // a4: reverse correction sweep (single task)
};

// Device status word and counters (one per op).
struct DevStats {
  int status;      // first error code recorded
  int fail_kind;
  int fail_step;
  int pad;
  unsigned long long solves;
  unsigned long long cg_iters;
  unsigned long long refinements;
  unsigned long long max_cg_iters;
  unsigned long long kind_solves[6];       // per task kind (Kind)
  unsigned long long kind_cg_iters[6];
  unsigned long long kind_refinements[6];
};

// Padded row layout shared by every grid-shaped array of the stepper (host and device):
// a row holds columns ix = -1 .. W-2 at offsets ix+1, W = roundup(nx + 3, 4), so rows are
// 16-byte aligned and split into W/4 aligned groups of 4 nodes; out-of-domain entries are 0.
// Every such array starts kSlack entries after its base so that a group's neighbours
// (offsets -1 and +4) are always inside the allocation.
constexpr int kGroup = 4;
constexpr int kSlack = 4;
constexpr int kMaxExtrap = 4;   // most states an extrapolated initial guess goes through
inline __host__ __device__ int padded_width(int nx) { return ((nx + 3 + kGroup - 1) / kGroup) * kGroup; }

// Per-node FP64 weights of a symmetric 9-point operator (padded node grid, rows iy = -1..ny+1):
// centre, east, north, north-east and north-west couplings of each node; the west, south,
// south-west and south-east couplings are the east/north/north-east/north-west weights of the
// neighbour on the other side.
struct NodeWeights {
  const double* C;
  const double* E;
  const double* N;
  const double* NE;
  const double* NW;
};

// Geometric multigrid hierarchy of the coarse-step operator (mg.cu): level l has nx, ny
// elements (halved per level), the padded width W, arrays of plen floats each (slack included),
// its six weight arrays (C, E, N, NE, NW, omega/diag) at woff in the op's weight buffer, and its
// vectors at voff in a group's workspace (level 0: u, res; coarser: f, u, res, e).
constexpr int kMgMaxLevels = 10;
constexpr int kMgMinCells = 8;       // a level with min(nx, ny) <= 8 is the coarsest
constexpr float kMgOmega = 0.8f;     // Jacobi damping: omega lambda_max(D^-1 A) <= 1.8 on every level
struct MgLevel {
  int nx, ny, W, pad;
  long long plen, woff, voff;
};

// Everything one stepper launch needs (passed by value in parameter space).
struct StepParams {
  // problem
  int nx, ny, Nn, Ne, Nt, Ntau, M;
  int W;                     // padded row width
  int p_int;                 // even integer power-mean exponent
  double h, dt, dtau, p;
  int has_dc;                // capacity depends on rho (dC/drho != 0)
  // launch geometry
  int cs;                    // cluster size
  int rmax;                  // max owned rows of a CTA
  // task
  int kind;
  int s0, ns;                // slice range
  int chained;               // PTG_SLICES_CHAINED for fine tasks
  // solver
  double rtol, inner_rtol;
  int itmax, refmax;
  // op data (device, FP64, padded layouts; pointers at the first non-slack entry)
  const double* wE_fine;     // [3][(ny+2) W] element (D, S, T) weights of C/dt + K
  const double* wE_coarse;   // [3][(ny+2) W] element (D, S, T) weights of C/dtau + K
  NodeWeights A_fine;        // per-node weights of C/dt + K
  NodeWeights A_coarse;      // per-node weights of C/dtau + K
  NodeWeights mass;          // per-node weights of C
  const double* dk;          // [Ne]
  const double* dc;          // [Ne]
  const double* fload;       // [Nn] unit-time load, zero on Dirichlet nodes
  const double* q_time;      // [Nt+1]
  const uint8_t* dirichlet;  // [Nn]
  // state I/O (meaning depends on kind; see the stepper)
  const double* in_field;
  const double* in_aux;
  double* out_field;
  double* out_aux;
  const double* F_field;
  const double* F_aux;
  const double* G_field;
  const double* G_aux;
  double* hist;              // history window (row r = time hist_j0 + r) or null
  int hist_j0, hist_rows;
  const double* Theta;       // device scalar (adjoint kinds)
  DevStats* stats;
  int stats_kind;            // task kind under which the solver counters and errors are recorded
  const double* src_field;   // coarse kinds: [Ntau][Nn] right-hand-side source per slice instead of q_j f
  int objective;             // PTG_OBJ_POWER_MEAN or PTG_OBJ_MODIFIED
  int plt;                   // correction kinds: coarse propagators identically zero (copy F)
  int src_mode;              // coarse adjoint: 0 source scale Theta^(1-p)/Ne (or p/Ne); 1 no source (the part
                             // driven by the state); 2 unit source scale from zero lambda and zero g
  // two-level preconditioner of the coarse-step solves (Ainv == null: Jacobi)
  const float* Ainv;         // [ncp][ncp] inverse of the Galerkin coarse matrix (padded layout)
  int cm, nax, nay;          // aggregate size m and aggregate counts per direction
  int tl_naj;                // aggregate rows reserved per CTA (0: two-level disabled for this launch)
  int tl_vc;                 // 1: V(1,1) two-grid cycle with damped-Jacobi smoothing; 0: additive D^-1 + P Ac^-1 P^T
  float tl_omega;            // damping of the V-cycle's Jacobi smoother
  int local_steps;           // FP32 CG without two-level: 1 Jacobi, 2 two slab-local damped-Jacobi steps
  int keep_ax;               // 1: keep A x of the last residual (saves one FP64 stencil per step), 8 B per node
  int extrap;                // fine kinds: start each CG from the extrapolation through the slice's
                             // last `extrap` states (1: the last state alone; up to kMaxExtrap)
  int guess_next;            // coarse kinds: start each CG from the guess state at the slice's other end
  double* prev_field;        // fine kinds with extrap > 1: [extrap tasks][Nn] ring of each task's last
                             // states (or null: every step starts from the last state)
  int tl_nu;                 // V-cycle smoothing: <= 1 one global Jacobi step before and after; k >= 2 k
                             // slab-local steps before and after
  // three-level cycle (P.tl_l3): the V-cycle's coarse correction becomes a two-grid cycle of its
  // own on the 2h level (node (I, J) at fine node (2I, 2J), operator A1 = P1^T A P1 with bilinear
  // P1), whose coarse level is the aggregates of m x m 2h nodes (cm, nax, nay, Ainv, tl_naj then
  // describe that aggregation)
  int tl_l3;
  int l3_nx1, l3_ny1;        // 2h nodes per direction minus one (nx / 2, ny / 2)
  int l3_W1;                 // padded row width of the 2h buffers
  int l3_r1max;              // most 2h rows owned by a CTA of the launch
  const double* A1;          // [9][(ny1 + 1) (nx1 + 1)] 2h stencil, k = (dJ + 1) * 3 + (dI + 1)
  // streamed fine propagators (stream.cuh): per group of P.cs CTAs, three FP64 vectors (x, x, b)
  // and five CG vectors (r, z, p, q, d) in the kernel's precision, each st_pv entries in the padded
  // node layout with its slack; the FP32 element weights (D, S, T) of C/dt + K, w32_stride floats
  // apart in the padded element layout; 1/C (0 off the unknowns) in FP32 and FP64, padded node layout
  double* st_w64;
  void* st_wr;
  long long st_pv;
  const float* w32;
  int w32_stride;
  const float* w32_inv;
  const double* w64_inv;
  // one system over a whole cooperative grid (GridComm): global scratch of the op
  int wide;                  // 1: launched as stepper_wide_kernel, groups of cs CTAs
  int wide_tasks;            // tasks of a grid-wide launch (group g runs g, g + groups, ...)
  double* g_red;             // [2][kMaxGrid][4] reduction partials
  unsigned* g_bar;           // [4 per group] barrier: arrival count, unused, broken flag (zeroed per launch)
  long long wait_limit;      // polls of a grid barrier before it reports PTG_ETIMEOUT (<= 0: kGridSpinLimit)
  void* g_halo;              // [2 sets][kMaxGrid][2] rows of g_halo_row_bytes: first / last owned row
  int g_halo_row_bytes;      // W * 8 (a row of doubles; float rows use the first half)
  float* g_tl;               // [kMaxGrid][ncp] restricted partials of the two-level preconditioner
  // streamed coarse-step solves (stream.cuh): FP64 CG preconditioned by one V(nu, nu)-cycle of the
  // multigrid hierarchy (mg_levels = 0: Jacobi); mg_ws + group * mg_ws_stride is a group's
  // workspace; levels with at most mg_solo_rows node rows run on the group's first CTA alone
  int mg_levels;
  int mg_nu;                 // damped-Jacobi steps before and after the coarse correction
  int mg_coarse_steps;       // damped-Jacobi steps on the coarsest level (from zero)
  int mg_solo_rows;
  int mg_fuse;               // nu = 1: prolongation and post-smoothing in one pass (one barrier less
                             // per level)
  MgLevel mg[kMgMaxLevels];
  const float* mg_w;
  float* mg_ws;
  long long mg_ws_stride;
};

// Two-level preconditioner of the coarse-step solves: aggregates of m x m nodes (m a multiple
// of 4, so every aligned group of 4 nodes lies in one aggregate), at most kCoarseMaxAgg per
// direction; the last aggregate of a direction absorbs the remainder.
constexpr int kCoarseMaxAgg = 16;
inline __host__ __device__ int coarse_aggregates(int n_elems, int m) {
  const int a = (n_elems + 1) / m;
  return a < 1 ? 1 : a;
}
// aggregate row of node row iy
inline __host__ __device__ int coarse_agg_y(int iy, int m, int nay) {
  const int a = iy / m;
  return a < nay - 1 ? a : nay - 1;
}
// aggregate column of the group g (nodes 4g-1 .. 4g+2)
inline __host__ __device__ int coarse_agg_x(int g, int m, int nax) {
  const int a = g / (m / 4);
  return a < nax - 1 ? a : nax - 1;
}
// aggregate rows [jlo, jhi] touched by the node rows r0 .. r0+R-1 of a slab
inline __host__ __device__ void coarse_rows_of_slab(int r0, int R, int m, int nay, int& jlo, int& jhi) {
  jlo = coarse_agg_y(r0, m, nay);
  jhi = coarse_agg_y(r0 + R - 1, m, nay);
}
// aggregate rows touched by the slab and its two halo rows (node rows r0-1 .. r0+R inside
// 0 .. ny): the V-cycle prolongs the coarse correction onto the halo rows as well
inline __host__ __device__ void coarse_rows_of_halo_slab(int r0, int R, int ny, int m, int nay, int& jlo, int& jhi) {
  jlo = coarse_agg_y(r0 > 0 ? r0 - 1 : 0, m, nay);
  jhi = coarse_agg_y(r0 + R <= ny ? r0 + R : ny, m, nay);
}
// Coarse vectors index aggregate (ay, ax) as L = ay * naxp + ax with naxp = nax rounded up to
// a multiple of 4 (16-byte chunks never straddle two aggregate rows); ncp = nay * naxp is the
// padded length of a coarse vector and of a row of the dense inverse (zero in the padding).
inline __host__ __device__ int coarse_row_stride(int nax) { return (nax + 3) / 4 * 4; }

// Shared-memory bytes of the two-level preconditioner for one CTA (naj aggregate rows); the
// partials of every rank sit in shared memory for a cluster (slots = true), in global memory
// for a grid-wide launch.  The V-cycle (vc) adds its smoother buffers over the slab and its
// halo rows, the halo rows of q and r in the CG precision (real_bytes), and FP32 element
// weights where the CG runs in FP64 (the FP32 CG has them already).
inline size_t twolevel_smem_bytes(int W, int rmax, int cs, int nax, int nay, int naj, bool slots = true,
                                  bool vc = false, int real_bytes = 4, int nu = 1) {
  const size_t naxp = (size_t)coarse_row_stride(nax), ncp = naxp * nay;
  const size_t G = (size_t)(W / kGroup);
  const size_t groups = (size_t)rmax * G;
  const size_t halo = (size_t)(rmax + 2) * W + 2 * kSlack;   // a buffer over rows -1..R
  const size_t elems = (size_t)(rmax + 1) * W + 2 * kSlack;  // element rows -1..R-1
  size_t b = 0;
  b += (size_t)naj * naxp * ncp * 4;        // rows of Ainv for the CTA's aggregates
  if (slots) b += (size_t)cs * ncp * 4;     // restricted partials of every rank
  b += ncp * 4;                             // their sum over the covering ranks
  b += (size_t)naj * naxp * 4;              // coarse correction of the CTA's aggregates
  if (vc) {
    b += 4 * (size_t)W * real_bytes;        // q and r on the two halo rows
    b += 2 * halo * 4;                      // the smoother iterate (y, then u) and omega D^-1
    if (real_bytes == 8) b += 3 * elems * 4;  // FP32 (D, S, T) element weights
    if (nu >= 2) b += 2 * halo * 4;         // the slab-local smoother's two iterates
  }
  b += groups * 4;                          // group sums of the restricted vector
  b += (vc ? groups + 2 * G : groups) * 4;  // aggregate of every group (V-cycle: halo rows too)
  b += (size_t)nay * 2 * 4;                 // covering rank range per aggregate row
  return (b + 15) & ~size_t(15);
}

// Three-level cycle: the 2h rows J owned by the slab of fine rows r0 .. r0+R-1 are those with
// r0 <= 2J < r0 + R, i.e. J0 = ceil(r0 / 2) .. ceil((r0 + R) / 2) - 1 (R >= 2 gives at least one).
inline __host__ __device__ void l1_rows_of_slab(int r0, int R, int& J0, int& R1) {
  J0 = (r0 + 1) / 2;
  R1 = (r0 + R + 1) / 2 - J0;
}
// aggregate of 2h node index I (or J) among na aggregates of m nodes (the last absorbs the rest)
inline __host__ __device__ int l3_agg(int I, int m, int na) {
  const int a = I / m;
  return a < na - 1 ? a : na - 1;
}
// Shared-memory bytes of the three-level cycle for one CTA: the aggregate level as in
// twolevel_smem_bytes (naj aggregate rows, partials of every rank for a cluster), the fine
// V-cycle buffers, the fine residual with halos, and on the 2h level (r1max owned rows of W1
// entries): five buffers with halo rows, the restricted residual, nine stencil weights and
// omega / diag per owned node, and the per-aggregate partial sums.
inline size_t threelevel_smem_bytes(int W, int rmax, int cs, int W1, int r1max, int nax, int nay, int naj,
                                    bool slots, int real_bytes, int nu) {
  const size_t naxp = (size_t)coarse_row_stride(nax), ncp = naxp * nay;
  const size_t halo = (size_t)(rmax + 2) * W + 2 * kSlack;
  const size_t elems = (size_t)(rmax + 1) * W + 2 * kSlack;
  const size_t halo1 = (size_t)(r1max + 2) * W1 + 2 * kSlack;
  const size_t own1 = (size_t)r1max * W1 + 2 * kSlack;
  size_t b = 0;
  b += (size_t)naj * naxp * ncp * 4;        // rows of Ainv for the CTA's aggregates
  if (slots) b += (size_t)cs * ncp * 4;     // restricted partials of every rank
  b += ncp * 4;                             // their sum over the covering ranks
  b += (size_t)naj * naxp * 4;              // coarse correction of the CTA's aggregates
  b += 4 * (size_t)W * real_bytes;          // (the V-cycle's halo rows of q and r, unused here)
  b += 2 * halo * 4;                        // fine smoother iterate and omega D^-1
  if (real_bytes == 8) b += 3 * elems * 4;  // FP32 (D, S, T) element weights
  if (nu >= 2) b += 2 * halo * 4;           // the slab-local smoother's two iterates
  b += halo * 4;                            // fine residual with halo rows
  b += 5 * halo1 * 4;                       // 2h: e1, u1, z1, two smoother iterates
  b += 11 * own1 * 4;                       // 2h: restricted residual, 9 weights, omega / diag
  b += (size_t)naj * naxp * 4;              // per-aggregate partial sums
  b += (size_t)nay * 2 * 4;                 // covering rank range per aggregate row
  return (b + 15) & ~size_t(15);
}

// Shared-memory footprint (bytes) of one CTA of the stepper.
inline size_t stepper_smem_bytes(int nx, int rmax, int real_bytes, bool keep_ax = true) {
  const size_t W = (size_t)padded_width(nx);
  const size_t halo = (size_t)(rmax + 2) * W + 2 * kSlack;   // rows -1..R
  const size_t own = (size_t)rmax * W + 2 * kSlack;          // rows 0..R-1
  const size_t elems = (size_t)(rmax + 1) * W + 2 * kSlack;  // element rows -1..R-1
  size_t b = 0;
  b += halo * sizeof(double);                  // x64: FP64 state with halos
  b += own * sizeof(double);                   // b64: FP64 right-hand side
  if (keep_ax) b += own * sizeof(double);      // ax64: A x of the last residual evaluation (optional)
  b += halo * real_bytes;                      // zbuf: CG stencil operand with halos
  b += own * real_bytes;                       // dinv: Jacobi inverse diagonal (0 off the unknowns)
  if (real_bytes == 4) b += 3 * elems * 4;     // (D, S, T) element weights for the FP32 CG
  return (b + 15) & ~size_t(15);
}

// Host entry points of the kernel translation units.
struct Plan {
  int cs = 0, nthreads = 0, ng = 0, rmax = 0;
  size_t smem = 0;
  int max_active_clusters = 0;
  bool twolevel = false;     // coarse kinds: two-level preconditioner (its shared memory is in smem)
  bool vc = false;           // ... in the V(1,1) cycle form (else additive)
  bool l3 = false;           // ... as the three-level cycle
  bool keep_ax = true;       // the saved A x of the last residual is in smem
  bool wide = false;         // one task over a cooperative grid of cs CTAs (GridComm), no clusters
  bool stream = false;       // fine kinds: the streamed propagator (stream.cuh), cs CTAs per slice
};

// CTAs of a grid-wide launch at most (>= the SM count of the chip).
constexpr int kMaxGrid = 160;

cudaError_t launch_stepper(const StepParams& P, const Plan& plan, int precision, int ntasks, cudaStream_t stream);
cudaError_t launch_stepper_batch(int precision, int kind, const Plan& plan, const StepParams* table, const int2* tasks,
                                 int ntasks, int* queue, int nclusters, cudaStream_t stream);
cudaError_t query_batch_occupancy(int precision, int kind, int cs, int ng, int nthreads, size_t smem, int* nclusters);
cudaError_t launch_coarse_setup(int nx, int ny, int W, int m, const NodeWeights& A, const uint8_t* dirichlet,
                                double* Ac, float* band, float* X, float* Ainv, cudaStream_t stream);
// Three-level set-up from the coarse-step operator's node weights: the 2h Galerkin stencil A1
// ([9][(ny/2 + 1)(nx/2 + 1)]), then the aggregates of m x m 2h nodes: A2 = P2^T A1 P2 (dense FP64
// in Ac), its band LDL^T and dense inverse in FP32, packed as for the fine aggregates.
cudaError_t launch_threelevel_setup(int nx, int ny, int W, const NodeWeights& A, const uint8_t* dirichlet, int m,
                                    double* A1, double* Ac, float* band, float* X, float* Ainv, cudaStream_t stream);
// Raise a kernel's dynamic shared-memory limit (and allow non-portable cluster sizes) once per
// device; later calls with no larger footprint make no attribute call.
cudaError_t configure_kernel(const void* k, size_t smem, bool cluster);
cudaError_t query_stepper_plan(int nx, int ny, int precision, int kind, int cs, int ng, int nthreads, size_t extra_smem,
                               Plan* plan, bool keep_ax = true);
// Plan of the grid-wide variant.  spread: one system over as many CTAs as there are SMs (rmax
// >= 2 rows each); otherwise the fewest CTAs per group whose slabs fit, and as many groups as
// fit the chip (plan.max_active_clusters = groups, at most ntasks).  extra_smem(G) gives the
// two-level bytes for G CTAs.  cudaErrorInvalidConfiguration if nothing fits.
cudaError_t query_wide_plan(int nx, int ny, int precision, int kind, int ntasks, bool spread,
                            size_t (*extra_smem)(const void*, int), const void* ctx, Plan* plan, bool keep_ax = true);

// Device arrays written by the assembly (see ptg_op in api.cu for their shapes).
struct AssembleOut {
  double *k, *c, *dk, *dc;            // [Ne]
  double *wEf, *wEc;                  // [3][(ny+2) W] element (D, S, T) weights
  double* node[15];                   // per-node weights: A_fine C,E,N,NE,NW; A_coarse ...; mass ...
  double* fload;                      // [Nn]
};
cudaError_t launch_assemble(int nx, int ny, double h, const ptg_material& m, double dt, double dtau, const double* rho,
                            const double* q_elem, const uint8_t* dirichlet, const AssembleOut& out, DevStats* st,
                            cudaStream_t stream);

cudaError_t launch_objective_from_modified(int Ne, double p, const double* Theta_mod, const double* grad_mod,
                                          double* Theta, double* grad, double* scratch, cudaStream_t stream);
cudaError_t launch_sensitivities(int nx, int ny, int Nt, double h, double dt, int has_dc, const double* dk,
                                 const double* dc, const double* lam, int j0, int j1, const double* T, int hist_j0,
                                 double* partial, int nchunks, double* grad, cudaStream_t stream);

// For the streamed fine propagators: FP32 copies of the 3 x PE FP64 element weights (D, S, T) of
// C/dt + K (slack included), and 1/C in FP32 and FP64 (0 off the unknowns) on the PN entries of
// the padded node layout (slack included; C the node weight array with its slack).
cudaError_t launch_stream_weights(int PE, int PN, const double* wE, const double* C_node, const uint8_t* dirichlet,
                                  int nx, int ny, int W, float* w32, float* w32_inv, double* w64_inv,
                                  cudaStream_t stream);
cudaError_t launch_stream(const StepParams& P, int precision, int ngroups, int nthreads, cudaStream_t stream);
// Multigrid hierarchy: the number of levels of an nx x ny grid (1: no coarsening), the layout of
// L levels (returns the floats of the weight buffer; *ws_floats the floats of one group's
// workspace), and the set-up of every level's weights from the FP64 node weights A (buffer
// zeroed beforehand: the slack and the rows outside the grid stay zero).
int mg_level_count(int nx, int ny);
long long mg_layout(int nx, int ny, MgLevel* lv, int L, long long* ws_floats);
cudaError_t launch_mg_setup(NodeWeights A, const uint8_t* dirichlet, const MgLevel* lv, int L, float* w,
                            cudaStream_t stream);
// G_l = H_l + c S_l ([n_l]) and G_g = H_g + c S_g ([n_g]), c the adjoint source scale of Theta
cudaError_t launch_adjoint_combine(long long n_l, long long n_g, const double* Theta, double p, int Ne, int modified,
                                   const double* H_l, const double* H_g, const double* S_l, const double* S_g,
                                   double* G_l, double* G_g, cudaStream_t stream);
// grad[e] -= inv_nt * (sum of partial[c][e] over c = 0..nchunks-1, in that order)
cudaError_t launch_sens_reduce(int Ne, int nchunks, double inv_nt, const double* partial, double* grad,
                               cudaStream_t stream);

void set_last_error(const char* msg);

}  // namespace ptg
