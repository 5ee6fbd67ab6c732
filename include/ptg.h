/*
 * ptg.h -- C ABI of the GB300 (sm_103a) one-shot Parareal topology-optimisation pass
 * for transient heat conduction (Appel & Alexandersen, arXiv 2411.19030).
 *
 * The library computes, for one design rho, the per-design-iteration state / adjoint /
 * sensitivity pass of the paper's one-shot Parareal method (Algorithm 3):
 *
 *   a1  ptg_fe_assemble_operator   SIMP coefficients and element weights      Sec. 2.1-2.2, Eq. 2.5-2.7
 *   a2  ptg_fine_propagate_slices  F_pri of every slice (modified Parareal)   Alg. 1, Sec. 4.3-4.4
 *   a3  ptg_coarse_sweep           G_pri / G_adj of every slice (batched)     Alg. 1-2 substitutions, Sec. 4.4
 *   a4  ptg_parareal_correct       sequential correction sweep                Eq. 4.9 (forward), Eq. 4.14 (reverse)
 *   a5  ptg_adjoint_sweep          F_adj of every slice                        Alg. 2, Sec. 4.4
 *   a6  ptg_sensitivities          sum_j lambda_j^T dR_j/drho_e reduction      Eq. 4.7
 *
 * Discretisation (Sec. 2.2): nx*ny square bilinear elements of side h, depth 1; nodes
 * row-major (node = iy*(nx+1) + ix), elements row-major (e = ey*nx + ex); element-wise
 * constant k, c, q; backward Euler  C (T_j - T_{j-1})/dt + K T_j = q_j; Dirichlet nodes
 * (T = lambda = 0) are removed from the unknowns.  Objective (Eq. 2.11):
 *   Theta = ( sum_{j=1..Nt} ||T_j||_p^p / (Nt Ne) )^(1/p),  p even.
 * Parareal indexing (Sec. 4.2-4.4): M = Nt/Ntau, slice s = 0..Ntau-1 spans fine steps
 * j = M s + 1 .. M (s+1); primal states u_n = (T_{Mn}, theta_{Mn}); adjoint states
 * v_n = (lambda_{Mn+1}, g_{Mn+1}) with v_Ntau = 0.
 *
 * Conventions for every call
 *  - Ownership: the caller owns every array argument (device memory unless stated,
 *    contiguous, FP64, row-major with the shapes given).  The library owns only the
 *    opaque ptg_op and the device workspace it allocates in ptg_op_create.
 *  - Execution: every compute call is asynchronous on `stream` (a cudaStream_t; 0 is the
 *    legacy default stream) and performs no host synchronisation.  Calls on one op must
 *    not overlap on the GPU (they share the op's workspace).
 *  - Errors: every call returns PTG_OK or a negative code.  Argument errors are detected
 *    on the host before anything is launched (PTG_EINVAL).  Conditions found on the
 *    device (non-finite or out-of-range design values, a solve that hit its iteration
 *    limit, a non-finite solution) are recorded in the op's device status word and
 *    reported by ptg_get_stats, which synchronises the stream.  No call traps or aborts.
 *  - No C++ exception crosses this boundary.  Calls on distinct ops are independent.
 */
#ifndef PTG_H
#define PTG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define PTG_OK          0
#define PTG_EINVAL     -1   /* invalid argument (host check) or invalid design value (device) */
#define PTG_ENOCONV    -2   /* a linear solve stopped at its iteration limit */
#define PTG_ENONFINITE -3   /* a non-finite value appeared in a solution or an objective */
#define PTG_ETIMEOUT   -4   /* a bounded device wait gave up */
#define PTG_ECUDA      -5   /* a CUDA runtime call failed (see ptg_last_error) */
#define PTG_ENOMEM     -6   /* device allocation failed */
#define PTG_EBOUNDS    -7   /* debug build (libptg_debug.so) only: a launch check found an index range
                                outside the op's allocations; the launch was skipped */

/* precision of the fine-propagator CG (Sec. 2.2 solves; precision pattern of the port) */
#define PTG_FP64            0  /* CG and every accumulation in FP64 */
#define PTG_FP32_REFINE     1  /* fine-step solves: CG in FP32 on the FP64 residual, refined in FP64;
                                  coarse-step solves (G and the correction sweeps): FP64 CG */
#define PTG_FP32_REFINE_ALL 2  /* every solve as the fine-step solves of PTG_FP32_REFINE */

/* slice scheduling of ptg_fine_propagate_slices / ptg_adjoint_sweep */
#define PTG_SLICES_PARALLEL 0  /* every slice starts from its own given state (Parareal F) */
#define PTG_SLICES_CHAINED  1  /* one sequential run: slice s starts where slice s-1 ended */

#define PTG_PRIMAL   1
#define PTG_ADJOINT -1

/* objectives (ptg_time.objective) */
#define PTG_OBJ_POWER_MEAN 0   /* Theta of Eq. 2.11 with the cumulative power mean of Sec. 4.4 */
#define PTG_OBJ_MODIFIED   1   /* Theta~ = Theta^p of Sec. 7.1: cumulative plain sum, adjoint source p/Ne T^(p-1) */

/* ------------------------------------------------------------------ problem description */
typedef struct {
    int nx, ny;        /* elements per side, each >= 2 */
    double h;          /* element side; the domain is [0, nx h] x [0, ny h] with depth 1 */
} ptg_grid;

typedef struct {       /* SIMP interpolation, Eq. 2.5-2.6 */
    double k0, kmin, pk;   /* k = kmin + (k0 - kmin) rho^pk */
    double c0, cmin, pc;   /* c = cmin + (c0 - cmin) rho^pc */
} ptg_material;

typedef struct {
    int Nt;            /* fine steps, t_j = j dt */
    int Ntau;          /* Parareal slices; must divide Nt (Sec. 4.2) */
    double dt;         /* fine step; the coarse step is dtau = (Nt/Ntau) dt */
    double p;          /* power-mean exponent, an even integer >= 2 (Eq. 2.11) */
    int objective;     /* PTG_OBJ_POWER_MEAN or PTG_OBJ_MODIFIED; every theta / g quantity of the
                          passes then refers to that objective */
} ptg_time;

#define PTG_TWOLEVEL_NONE 0
#define PTG_TWOLEVEL_ADDITIVE 1
#define PTG_TWOLEVEL_VCYCLE 2
#define PTG_TWOLEVEL_THREELEVEL 3

typedef struct {
    int precision;     /* PTG_FP64, PTG_FP32_REFINE or PTG_FP32_REFINE_ALL */
    double rtol;       /* stop when ||b - A x||_2 <= rtol ||b||_2 (FP64 residual) */
    double inner_rtol; /* relative residual reduction of each FP32 CG (FP32 solves only) */
    int cg_iters_max;  /* iteration limit of one CG */
    int refine_max;    /* limit of refinement sweeps of one solve */
    int twolevel;      /* preconditioner of the CG of the coarse-step solves (C/dtau + K), with
                          P piecewise constant on aggregates of m x m nodes (m the smallest
                          multiple of 4 giving <= 16 aggregates per direction), Ac = P^T A P
                          and its inverse applied in FP32:
                          PTG_TWOLEVEL_NONE      Jacobi everywhere;
                          PTG_TWOLEVEL_ADDITIVE  D^-1 + P Ac^-1 P^T;
                          PTG_TWOLEVEL_VCYCLE    a symmetric two-grid cycle: damped-Jacobi
                                                 smoothing S (omega = 0.8, smooth_steps), the
                                                 coarse correction of the residual, S again, i.e.
                                                 I - M^-1 A = (I - S A)(I - P Ac^-1 P^T A)(I - S A),
                                                 applied in FP32.
                          PTG_TWOLEVEL_THREELEVEL the same cycle with its coarse correction
                                                 replaced by a two-grid cycle on the 2h level:
                                                 P1 bilinear from the nodes (2I, 2J), A1 =
                                                 P1^T A P1 (9-point), damped-Jacobi smoothing
                                                 on the CTA's 2h rows (smooth_steps), and the
                                                 aggregates of m x m 2h nodes (m giving <= 16
                                                 per direction) with their dense inverse below
                                                 it; symmetric, in FP32.  Needs even nx, ny and
                                                 a one-cluster launch with >= 2 fine rows per
                                                 CTA; elsewhere (odd grids, cooperative-grid
                                                 launches, batches) the two-grid cycle.
                          Other values: PTG_EINVAL. */
    int grid_wide;     /* systems may run on groups of CTAs of one cooperative launch, talking
                          through global memory, instead of one 16-CTA cluster each: a single
                          FP64 system (correction sweeps, chained runs) over every SM, other
                          kinds in groups of the fewest CTAs whose slabs fit.  0 never; 1 for a
                          single FP64 system on >= 40000 nodes and whenever no cluster plan fits
                          (grids beyond about 300 x 300); 2 always. */
    int smooth_steps;  /* PTG_TWOLEVEL_VCYCLE smoothing, before and after the coarse correction:
                          1: one damped-Jacobi step on the whole grid; k in 2..16: k damped-Jacobi
                          steps on each CTA's slab alone (the slab's diagonal block of A, no
                          communication).  0: the library's default.  Other values: PTG_EINVAL. */
    int coarse_mesh;   /* 1: the coarse propagators G_pri and G_adj take their step of dtau on the
                          mesh of spacing 2h (the remedy for the sequential coarse sweep proposed
                          as future work in Sec. 7.3): nx/2 x ny/2 elements whose density is the
                          mean of their four children, states restricted by injection and
                          prolongated by bilinear interpolation, the adjoint source restricted by
                          the transpose of the interpolation; theta and g increments of G from the
                          prolongated state on the fine mesh.  F, the corrections, the history and
                          every output stay on the fine mesh.  Needs even nx, ny >= 4 (else
                          PTG_EINVAL); the batch entry points reject such ops.  0: G on the fine
                          mesh (Sec. 4.4). */
    int local_steps;   /* preconditioner of the FP32 CG solves that use no two-level form (the fine
                          steps): 1 Jacobi; 2 two damped-Jacobi steps (omega = 0.8) on each CTA's
                          slab alone, z = (2S - S A_s S) r with S = omega D^-1 and A_s the slab's
                          diagonal block of A (symmetric, no communication); 3 on the streamed
                          fine propagators (fine_stream) of grids that coarsen at least once: the
                          multigrid V(1,1)-cycle of coarse_stream, built on C/dt + K (elsewhere as
                          0); 0 the library's default: the multigrid cycle on streamed fine
                          propagators of grids with at least three levels, else 1 on cluster
                          launches and 2 on cooperative-grid launches (whose reductions go through
                          global memory).  Other values: PTG_EINVAL. */
    int initial_guess; /* where each CG of a time step starts (only iteration counts change):
                          1 plain: a fine step from the state it steps from, a batched coarse step
                          (ptg_coarse_sweep) from the state it propagates;
                          n in 2..4 predicted: a fine step from the polynomial extrapolation
                          through the last n states of its slice (n = 2: 2 x_{j-1} - x_{j-2};
                          fewer in the first steps of every slice, chained runs included, so a
                          slice recomputed alone repeats its solves bit for bit; the states are
                          kept in a workspace of the op, n rows per slice), a
                          batched coarse step from the guess state at the other end of its slice
                          (u_{s+1} for G_pri, lambda_{Ms+1} for G_adj), which the previous
                          one-shot iteration left close to the answer, and a correction-sweep
                          step (ptg_parareal_correct) from G_old[s] plus the polynomial
                          extrapolation, through the increments G(x^new) - G(x^old) of the last
                          n - 1 steps of the sweep (fewer at its start), of the next one; the
                          increment of a step is the corrected state it produced minus the fine
                          result of its slice, e.g. u_s - F[s-1] (primal) or v_{s+1} - F[s+1]
                          (adjoint);
                          0 the library's default (4).  Other values: PTG_EINVAL. */
    int fine_stream;   /* fine propagators of the parallel schedule (a2, a5): 2 with the Krylov vectors
                          in global memory, one group of CTAs per slice and every slice at once
                          (the FP32 operator stays in L2); 1 on chip (one thread-block cluster,
                          or a cooperative group, per slice with its vectors on chip); 0 the
                          library's choice: streamed where no cluster holds a slice (grids of
                          roughly 300 x 300 and more), on chip elsewhere.  Other values:
                          PTG_EINVAL. */
    int coarse_stream; /* coarse-step solves (G_pri, G_adj and the correction sweeps, a3 and a4) with
                          the Krylov vectors in global memory: FP64 CG (FP32 under
                          PTG_FP32_REFINE_ALL) preconditioned by one V(1,1)-cycle of geometric
                          multigrid in FP32: level l+1 the nodes (2I, 2J) of level l down to a
                          grid of at most 8 elements across (while nx and ny stay even), Galerkin
                          operators P^T A P of bilinear interpolation P, damped-Jacobi smoothing
                          (omega = 0.8), ten damped-Jacobi steps on the coarsest level; symmetric.
                          The batched coarse propagators run every slice at once, one group of
                          CTAs per slice; a correction sweep runs as one group of about one CTA
                          per two node rows (at most one per SM).  2 wherever the grid coarsens
                          at least once; 1 never (the on-chip stepper with ptg_solve.twolevel);
                          0 the library's choice: grids of 30000 nodes or more with at least
                          three levels.  Other values: PTG_EINVAL. */
} ptg_solve;

typedef struct {
    int status;             /* PTG_OK or the first device-side error code recorded */
    int fail_kind;          /* who recorded status: 1 assemble; 10 + task kind for the stepper
                               (10 fine primal, 11 coarse primal, 12 correct primal,
                                13 fine adjoint, 14 coarse adjoint, 15 correct adjoint);
                               30 + task kind for a launch check of the debug build */
    int fail_step;          /* fine time index j of the failing step (or -1); for PTG_EBOUNDS
                               the failed check: 1 slices, 2 history rows, 3 streamed groups,
                               4 streamed workspace, 5 multigrid levels, 6 row ownership */
    int reserved;
    long long solves;       /* linear solves since the last reset */
    long long cg_iters;     /* CG iterations since the last reset */
    long long refinements;  /* refinement sweeps (FP32_REFINE) since the last reset */
    long long max_cg_iters; /* largest CG iteration count of one solve */
    long long kind_solves[6];      /* the same counters per stepper task kind (see ptg_op_get_plan) */
    long long kind_cg_iters[6];
    long long kind_refinements[6];
} ptg_stats;

typedef struct ptg_op ptg_op;   /* opaque: operator coefficients, launch plan, workspace */

/* Library version string ("ptg <major>.<minor> sm_103a"; the build with NVTX ranges, libptg_nvtx.so,
 * appends " nvtx", the debug build, libptg_debug.so, " debug").  The NVTX build wraps every call
 * that enqueues GPU work in an NVTX range of the domain "ptg" named after the call, and each batch
 * phase in a nested range.  The debug build checks, before every launch of an op's task kinds,
 * that the index ranges the launch will touch (slices, history rows, workspace groups, multigrid
 * levels, node rows) lie inside the op's allocations; a failed check skips the launch, the call
 * returns PTG_EBOUNDS, and ptg_get_stats reports it with the check in fail_step. */
const char* ptg_version(void);

/* Text of the last CUDA error seen by this thread's calls (static storage). */
const char* ptg_last_error(void);

/*
 * Create an operator for one problem (Sec. 2-3).  Allocates the device workspace and
 * chooses the launch plan; assembles nothing yet.
 *   dirichlet_h  HOST uint8 [Nn]: 1 marks a Dirichlet node (T = 0, Eq. 2.1c), copied.
 *   q_elem_h     HOST FP64 [Ne] element source density, or NULL for q_e = 1; copied.
 *   q_time_h     HOST FP64 [Nt+1] time factor of the source at t_0..t_Nt, or NULL for 1;
 *                the load vector at t_j is q_time[j] * sum_e q_e int N_i (copied).
 *   device       CUDA device ordinal the op lives on.
 * Errors: PTG_EINVAL (Ntau does not divide Nt, p not even, sizes out of range, grid too
 * large for one thread-block cluster), PTG_ENOMEM, PTG_ECUDA.  *out is NULL on error.
 */
int ptg_op_create(const ptg_grid* grid, const ptg_material* mat, const ptg_time* time,
                  const ptg_solve* solve, const uint8_t* dirichlet_h, const double* q_elem_h,
                  const double* q_time_h, int device, ptg_op** out);

/* Release the op and its workspace (waits for the device).  NULL is ignored. */
void ptg_op_destroy(ptg_op* op);

/* Sizes of the op: Nn, Ne, Nt, Ntau, M (any pointer may be NULL). */
int ptg_op_sizes(const ptg_op* op, int* Nn, int* Ne, int* Nt, int* Ntau, int* M);

/* Tuning of the multigrid cycle of the streamed solves (ptg_solve.coarse_stream, local_steps = 3)
 * for the launches that follow: solo_rows, levels with at most this many node rows run on the
 * first CTA of a group alone (block barriers instead of the group's); coarse_steps, damped-Jacobi
 * steps on the coarsest level (1..64); fused, 1 prolongation and post-smoothing in one pass, 0 in
 * two.  0 (solo_rows, coarse_steps) and -1 (fused) restore the library's defaults (33, 10, 1).
 * Results change only within the solver tolerance.  PTG_EINVAL on other values. */
int ptg_op_set_multigrid(ptg_op* op, int solo_rows, int coarse_steps, int fused);

/*
 * Launch plan of the cluster stepper.  Every solve runs on one thread-block cluster of
 * `cs` CTAs (1, 2, 4, 8 or 16) that split the node rows; each CTA has `nthreads` threads
 * (a multiple of 32, at most 512), each holding `ng` aligned groups of 4 nodes (1..6).  kind: 0 fine primal,
 * 1 coarse primal, 2 primal correction, 3 fine adjoint, 4 coarse adjoint, 5 adjoint correction.
 * ptg_op_get_plan reports the plan used for `ntasks` concurrent clusters (chosen for the
 * fewest waves, then the largest cluster).  ptg_op_set_plan forces a plan for a kind
 * (cs = 0 removes the override); PTG_EINVAL if the plan does not fit the grid or device.  For a
 * streamed correction sweep (ptg_solve.coarse_stream) cs is the number of CTAs of its group
 * (1 .. SMs, at least two node rows each) and ng is ignored.
 */
int ptg_op_get_plan(ptg_op* op, int kind, int ntasks, int* cs, int* nthreads, int* ng, int* max_active_clusters);
int ptg_op_set_plan(ptg_op* op, int kind, int cs, int ng);

/*
 * a1 -- Sec. 2.1-2.2, Eq. 2.5-2.6: evaluate the SIMP coefficients k_e, c_e, dk_e/drho,
 * dc_e/drho of the design rho_d (device FP64 [Ne], rho in [0,1]) and the element weights
 * of C/dt + K and C/dtau + K used by every solve.  The op keeps the results until the
 * next call.  A value of rho outside [0,1] or non-finite records PTG_EINVAL on the
 * device.  Must precede every other compute call for that design.
 */
int ptg_fe_assemble_operator(ptg_op* op, const double* rho_d, cudaStream_t stream);

/*
 * a2 -- Alg. 1 and Sec. 4.3: the fine primal propagator F_pri of slices s0..s0+ns-1.
 *   schedule   PTG_SLICES_PARALLEL: slice s starts from (U_T[s], U_theta[s]) and all
 *              slices run concurrently (the parallel part of Parareal).
 *              PTG_SLICES_CHAINED: one sequential run from (U_T[s0], U_theta[s0]); slice s
 *              starts from the end of slice s-1 (sequential time stepping, the initialisation of Alg. 3).
 *   U_T        [Ntau+1][Nn], U_theta [Ntau+1]: start states (only rows s0.. are read).
 *   T_hist     history window or NULL: row r holds T_{hist_j0 + r}, hist_rows rows.  Every
 *              computed T_j, j = M s + 1 .. M (s+1), is written to its row (the last one
 *              is the uncorrected slice end).  Rows outside the window are not written;
 *              the window must cover every written row or PTG_EINVAL is returned.
 *   F_T        [Ntau][Nn], F_theta [Ntau]: slice-end states (T_{M(s+1)}, theta_{M(s+1)}).
 */
int ptg_fine_propagate_slices(ptg_op* op, int schedule, int s0, int ns,
                              const double* U_T, const double* U_theta,
                              double* T_hist, int hist_j0, int hist_rows,
                              double* F_T, double* F_theta, cudaStream_t stream);

/*
 * a3 -- Sec. 4.4: the coarse propagators of slices s = 0..Ntau-1, evaluated for all slices
 * concurrently, on the guess states X (the G(u_n^k) terms of the correction).
 *   direction PTG_PRIMAL: G_pri(s, u_s) = one step of size dtau ending at t_{M(s+1)} with the
 *             load q_{M(s+1)}, and theta += ||T||_p^p/(Ntau Ne) in the power-mean recursion.
 *             X_field = U_T [Ntau+1][Nn], X_aux = U_theta [Ntau+1]; outputs
 *             G_field [Ntau][Nn], G_aux [Ntau].  T_hist and Theta_d are unused (may be NULL).
 *   direction PTG_ADJOINT: G_adj(s, v_{s+1}) = one reverse step of size dtau solving for
 *             lambda_k, k = M s + 1, from lambda_{k+M}, with the source Theta^(1-p)/Ne T_k^(p-1)
 *             and g -= (1/Ntau) lambda^T(dC/drho (T_k - T_{k-M})/dtau + dK/drho T_k), where
 *             T_{k-M} is read as T_0 for s = 0.  X_field = V_lam [Ntau+1][Nn],
 *             X_aux = V_g [Ntau+1][Ne] (rows s+1 are read); outputs G_field [Ntau][Nn],
 *             G_aux [Ntau][Ne].  T_hist is the full history [Nt+1][Nn]; Theta_d points to Theta.
 *   Every row of X_field is read (the start of one step, the initial guess of another: see
 *   ptg_solve.initial_guess), so G_field must not overlap X_field.
 */
int ptg_coarse_sweep(ptg_op* op, int direction, const double* X_field, const double* X_aux,
                     const double* T_hist, const double* Theta_d,
                     double* G_field, double* G_aux, cudaStream_t stream);

/*
 * a3 on the slices s0 .. s0+ns-1 only (Sec. 4.2: the coarse propagators of different slices are
 * independent), e.g. one process's share when the slices are split over several GPUs.  Arrays
 * and their meaning as for ptg_coarse_sweep (full Ntau-row shapes); only rows s0 .. s0+ns-1 of
 * G_field / G_aux are written, and only the rows of X_field, X_aux and T_hist that those slices
 * read must be valid: X rows s and s+1, and for the adjoint T_hist rows M s + 1 and M(s-1) + 1
 * (row 0 for s = 0).  0 <= s0, 1 <= ns, s0 + ns <= Ntau, else PTG_EINVAL; ops whose coarse
 * propagators run on the 2h mesh accept only the whole range.
 */
int ptg_coarse_sweep_slices(ptg_op* op, int direction, int s0, int ns, const double* X_field, const double* X_aux,
                            const double* T_hist, const double* Theta_d, double* G_field, double* G_aux,
                            cudaStream_t stream);

/*
 * a3, adjoint direction, in two parts that need no Theta.  The adjoint source of Eq. 4.6 is
 * c T_k^(p-1) with c = Theta^(1-p)/Ne (p/Ne for PTG_OBJ_MODIFIED), and the solve and the g update
 * of G_adj are affine in c, so G_adj(s, v_{s+1}) = H[s] + c S[s] with
 *   H[s] = G_adj(s, v_{s+1}) with the source left out (c = 0), started from lambda_{k+M},
 *   S[s] = G_adj(s, 0) with c = 1 (lambda = 0 and g = 0 in), started from zero,
 * each solved to the op's tolerance.  Slices s0 .. s0+ns-1; arrays as for ptg_coarse_sweep
 * (H_lam, S_lam [Ntau][Nn]; H_g, S_g [Ntau][Ne]; only rows s0 .. s0+ns-1 written).  The parts read
 * only the history rows M s + 1 and M(s-1) + 1 (row 0 for s = 0), which ptg_fine_propagate_slices
 * writes and, for M > 1, the forward correction sweep does not, so they can run before Theta is
 * known: beside ptg_parareal_correct(PTG_PRIMAL) of the same op on another stream, when
 * ptg_op_overlap_ok allows it.  That is the one exception to the rule that calls on one op do not
 * overlap: a streamed sweep (ptg_solve.coarse_stream) keeps a workspace of its own, and parts on
 * cluster launches touch no op workspace but the counters.  Ops with the 2h-mesh coarse
 * propagators: PTG_EINVAL.
 * ptg_coarse_adjoint_combine then forms G_lam = H_lam + c S_lam and G_g = H_g + c S_g on the same
 * rows, with c from the device scalar Theta_d.
 */
int ptg_coarse_adjoint_split(ptg_op* op, int s0, int ns, const double* V_lam, const double* V_g, const double* T_hist,
                             double* H_lam, double* H_g, double* S_lam, double* S_g, cudaStream_t stream);
int ptg_coarse_adjoint_combine(ptg_op* op, int s0, int ns, const double* Theta_d, const double* H_lam,
                               const double* H_g, const double* S_lam, const double* S_g, double* G_lam, double* G_g,
                               cudaStream_t stream);
/* Whether ptg_coarse_adjoint_split may run beside ptg_parareal_correct(PTG_PRIMAL) of this op:
 * M > 1, coarse propagators on the fine mesh, the forward sweep on a cluster or streamed, and the
 * batched coarse adjoint (Ntau tasks) on clusters or streamed (cooperative-grid stepper plans
 * share the op's grid workspace).  *ok = 1: the parts may also overlap ptg_adjoint_sweep;
 * *ok = 2: streamed parts share their workspace with the fine adjoint propagator, which must
 * start after them; *ok = 0: no overlap. */
int ptg_op_overlap_ok(ptg_op* op, int* ok);

/*
 * a4 -- Eq. 4.9 / 4.14: the sequential correction sweep of one Parareal iteration.
 *   G_field == G_aux == NULL selects the PLT variant of Sec. 7 (coarse propagators identically
 *   zero, Eq. 7.1-7.2): u_{s+1} = F[s] and v_s = F[s], a copy with no solve.
 *   PTG_PRIMAL: X_new[0] (U_T[0], U_theta[0]) holds u_0 on entry; for s = 0..Ntau-1,
 *      u_{s+1} = G_pri(s, u_s) + F[s] - G_old[s], and the corrected T_{M(s+1)} is written to
 *      T_hist row M(s+1) (T_hist may be NULL).  Theta = X_aux[Ntau] afterwards.
 *   PTG_ADJOINT: v_Ntau = 0 is written; for s = Ntau-1..0,
 *      v_s = G_adj(s, v_{s+1}) + F[s] - G_old[s]; the gradient is X_aux row 0 (g_1).
 *      T_hist (full, read only) and Theta_d are required.
 *   F_field/F_aux are the fine results of a2/a5 and G_field/G_aux the coarse results of a3
 *   on the same guess; X_field/X_aux have the state shapes of ptg_coarse_sweep.
 */
int ptg_parareal_correct(ptg_op* op, int direction,
                         const double* F_field, const double* F_aux,
                         const double* G_field, const double* G_aux,
                         double* X_field, double* X_aux,
                         double* T_hist, const double* Theta_d, cudaStream_t stream);

/*
 * Sec. 7.1: the power-mean objective and its gradient from the modified objective's,
 *   Theta = Theta~^(1/p),  grad_e = Theta^(1-p)/p grad~_e,  e = 0..Ne-1.
 * Theta_mod_d, Theta_d: device scalars; grad_mod_d, grad_d: [Ne] device arrays.  The outputs
 * may alias the inputs.  Theta~ must be positive (a zero objective has no power-mean gradient).
 */
int ptg_objective_from_modified(ptg_op* op, const double* Theta_mod_d, const double* grad_mod_d,
                                double* Theta_d, double* grad_d, cudaStream_t stream);

/*
 * a5 -- Alg. 2 and Sec. 4.4: the fine adjoint propagator F_adj of slices s0..s0+ns-1, each
 * from v_{s+1} = (V_lam[s+1], V_g[s+1]) backwards through j = M(s+1) .. M s + 1:
 *   solve (C/dt + K) lambda_j = C/dt lambda_{j+1} + Theta^(1-p)/Ne T_j^(p-1),
 *   g_j = g_{j+1} - (1/Nt) lambda_j^T (dC/drho (T_j - T_{j-1})/dt + dK/drho T_j).
 *   schedule  PTG_SLICES_PARALLEL (all slices concurrently from their own v_{s+1}) or
 *             PTG_SLICES_CHAINED (one reverse sequential run from v_{s0+ns}).
 *   T_hist    history window: row r holds T_{hist_j0 + r}; rows M s .. M(s+1) of every slice
 *             processed must lie inside it (else PTG_EINVAL).
 *   Theta_d   device pointer to Theta (the corrected theta_Nt of the same pass).
 *   F_lam [Ntau][Nn], F_g [Ntau][Ne]: slice-end states (lambda_{Ms+1}, g_{Ms+1}).
 */
int ptg_adjoint_sweep(ptg_op* op, int schedule, int s0, int ns,
                      const double* T_hist, int hist_j0, int hist_rows, const double* Theta_d,
                      const double* V_lam, const double* V_g,
                      double* F_lam, double* F_g, cudaStream_t stream);

/*
 * a6 -- Eq. 4.7: grad_e += -(1/Nt) sum_{j=j0..j1} lambda_j^T (dc_e Me (T_j - T_{j-1})/dt
 *                                                           + dk_e Ke T_j)|_e
 * for every element e, from an adjoint history lam_hist [j1-j0+1][Nn] (row r = lambda_{j0+r})
 * and a temperature window T_hist (row r = T_{hist_j0+r}) that covers j0-1 .. j1.
 * 1 <= j0 <= j1 <= Nt.  grad_d [Ne] is accumulated into (not overwritten).
 */
int ptg_sensitivities(ptg_op* op, const double* lam_hist, int j0, int j1,
                      const double* T_hist, int hist_j0, int hist_rows,
                      double* grad_d, cudaStream_t stream);

/*
 * ptg_sensitivities_noalloc -- the reduction of ptg_sensitivities without any device
 * allocation.  The paper has no counterpart: this entry point exists for callers that are
 * not allowed to allocate device memory themselves -- code whose device memory is owned by
 * another allocator (a framework's caching pool, an application with a fixed memory
 * budget), and timed loops in which cudaMalloc/cudaFree would synchronise the device.
 * ptg_op_create allocates a workspace; this call needs no op and no workspace.
 *   Inputs as for ptg_sensitivities, with the problem given explicitly: grid (nx, ny, h),
 *   Nt and dt, the SIMP material and the design rho_d (device FP64 [Ne]), from which the
 *   kernel evaluates dk/drho and dc/drho itself.  grad_d [Ne] is accumulated into.
 *   Scratch: the per-chunk partial sums use one static device array of
 *   PTG_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB) that every GPU loading this library keeps
 *   until the process exits.  Grids with nx*ny > PTG_NOALLOC_SCRATCH_DOUBLES are rejected
 *   with PTG_EINVAL before anything is launched.  Every call shares that array and leaves
 *   its partial sums behind; each call overwrites every entry it reads, so nothing needs
 *   clearing, but calls that overlap on the GPU (other streams, other threads) race on it
 *   and must be serialised by the caller.
 *   Set-up: the first call on a device (that device current) looks up the array's device
 *   address once and keeps it; make that first call before any stream capture begins, and do
 *   not call this entry point after a cudaDeviceReset of that device.
 *   Materials: k0, kmin, c0, cmin must be positive (as for ptg_op_create; else PTG_EINVAL).
 *   The design must lie in [0, 1]; a value outside (or NaN) is taken as 0, as
 *   ptg_fe_assemble_operator does (which also reports it), and is not reported here.
 * Returns PTG_OK, PTG_EINVAL (arguments, size) or PTG_ECUDA.
 */
#define PTG_NOALLOC_SCRATCH_DOUBLES (1 << 21)
int ptg_sensitivities_noalloc(int nx, int ny, double h, int Nt, double dt, const ptg_material* mat,
                              const double* rho_d, const double* lam_hist, int j0, int j1,
                              const double* T_hist, int hist_j0, int hist_rows,
                              double* grad_d, cudaStream_t stream);

/* ------------------------------------------------------------------ batches of designs
 * A batch advances several designs (ops of the same precision on the same device, grid sizes
 * may differ) together: each phase of a pass is ONE persistent launch in which every
 * thread-block cluster takes (design, slice) tasks from a work queue, largest designs first.
 * The batch owns each design's pass buffers (ptg_pass_buffers); the caller fills rho (and,
 * if it wants, the warm start) through the pointers returned by ptg_batch_buffers.
 * Phases: 0 fine primal, 1 coarse primal, 2 primal correction, 3 fine adjoint, 4 coarse
 * adjoint, 5 adjoint correction (the one-shot pass, the iteration body of Alg. 3); 6 sequential primal,
 * 7 sequential adjoint (the initialisation of Alg. 3, writing the warm start U/V); 8 and 9 the
 * primal and adjoint corrections of the PLT variant (G = 0, Sec. 7).
 * A large design takes no part in the persistent launches of phases 0-5, 8 and 9: one whose op
 * streams its coarse-step solves (ptg_solve.coarse_stream), or one of 15000 nodes or more.
 * Each of those phases runs it through its op's own entry points on the batch's buffers, as a
 * single-design pass does.  Its cluster launches run beside the persistent launch; its
 * streamed launches follow it, the correction sweeps of several designs side by side (groups
 * of 16 CTAs).  The side launches run on streams forked from and joined to `stream`.
 * ptg_batch_design_path reports which designs take that path.
 * Every call is asynchronous on `stream`; after a first call of each phase (which uploads the
 * plan) the launch sequence can be captured into a CUDA graph.
 */
typedef struct {
    double *T_hist;                              /* [Nt+1][Nn] */
    double *U_T, *U_theta, *V_lam, *V_g;         /* warm start: [Ntau+1][Nn], [Ntau+1], [Ntau+1][Nn], [Ntau+1][Ne] */
    double *U_T_new, *U_theta_new, *V_lam_new, *V_g_new;   /* result of the one-shot pass, same shapes */
    double *F_T, *F_theta, *G_T, *G_theta;       /* slice results of the primal: [Ntau][Nn], [Ntau] */
    double *F_lam, *F_g, *G_lam, *G_g;           /* slice results of the adjoint: [Ntau][Nn], [Ntau][Ne] */
    double *rho;                                 /* [Ne] the design, read by ptg_batch_assemble */
} ptg_pass_buffers;

typedef struct ptg_batch ptg_batch;

/* ptg_batch_create: a batch of nops >= 1 ops (the same device and precision; ops with the 2h-mesh
 * coarse propagators are refused), each one design.  An op may hold several designs; if such an
 * op takes the designs' own path, the batch runs without side streams.  The batch allocates and
 * owns every design's pass buffers, zeroed; the ops
 * stay the caller's and must outlive the batch.  PTG_EINVAL on such arguments, PTG_ENOMEM when
 * device memory runs out (nothing is left allocated).  ptg_batch_destroy synchronises the device
 * and frees the buffers.  ptg_batch_buffers: the device pointers of design `design`'s buffers,
 * valid until ptg_batch_destroy; PTG_EINVAL for a design out of range. */
int ptg_batch_create(ptg_op* const* ops, int nops, ptg_batch** out);
void ptg_batch_destroy(ptg_batch* b);
int ptg_batch_buffers(ptg_batch* b, int design, ptg_pass_buffers* out);
/* a1 for every design from its buffers' rho. */
int ptg_batch_assemble(ptg_batch* b, cudaStream_t stream);
/* The initialisation of Alg. 3 for every design: sequential primal and adjoint, writing U/V and T_hist;
 * Theta = U_theta[Ntau], gradient = V_g row 0. */
int ptg_batch_sequential_pass(ptg_batch* b, cudaStream_t stream);
/* The iteration body of Alg. 3 for every design from the warm start U/V: writes *_new and T_hist;
 * Theta = U_theta_new[Ntau], gradient = V_g_new row 0.  variant PTG_PARAREAL, or PTG_PLT for
 * coarse propagators identically zero (Sec. 7: the corrections copy F, G_* are not written). */
#define PTG_PARAREAL 0
#define PTG_PLT      1
int ptg_batch_oneshot_pass(ptg_batch* b, int variant, cudaStream_t stream);
/* Copy the one-shot result (*_new) into the warm start for the next design iteration. */
int ptg_batch_commit(ptg_batch* b, cudaStream_t stream);
/* One phase alone (its inputs must be current), e.g. to time it. */
int ptg_batch_run_phase(ptg_batch* b, int phase, cudaStream_t stream);
/* Plan of a phase's persistent launch: cluster size (2..16), groups per thread (1..6), threads per
 * CTA (32..512, multiple of 32); PTG_EINVAL if it does not fit every design of the launch or the
 * device. */
int ptg_batch_set_plan(ptg_batch* b, int phase, int cs, int ng, int nthreads);
/* The plan of a phase's persistent launch (the default one is chosen and installed on first use)
 * and the number of clusters it launches; NULL outputs are skipped.  PTG_EINVAL for a phase out of
 * range. */
int ptg_batch_get_plan(ptg_batch* b, int phase, int* cs, int* ng, int* nthreads, int* nclusters);
/* *own = 1 if design d runs the pass phases through its op's own launches, 0 if in the
 * persistent launches. */
int ptg_batch_design_path(ptg_batch* b, int design, int* own);

/*
 * Design parametrisation (Sec. 2.1) and area constraint (Sec. 3), on the device, FP64.
 *   chi_fil = H chi: weighted average over the elements whose centres lie within r_fil of the
 *             element's centre, cone weights r_fil - distance, each row normalised;
 *   rho     = P(chi_fil) = (tanh(beta (chi_fil - eta)) + tanh(beta eta)) /
 *                          (tanh(beta (1 - eta)) + tanh(beta eta)),  dproj = P'(chi_fil).
 * ptg_design_forward: chi [Ne] -> rho [Ne], dproj [Ne].
 * ptg_design_backward: df_dchi = H^T (dproj * df_drho) [Ne] (the chain rule of a function of
 *             rho); df_drho == NULL stands for the constant 1/Ne (the area-fraction gradient).
 * ptg_design_volume: *vol_d = mean(rho) (the area fraction on the uniform grid).
 * Element arrays are row-major (ey, ex), caller-owned device memory; calls are asynchronous.
 * r_fil must be positive and at most 64 h; 0 < eta < 1; beta > 0; 1 <= nx, ny <= 4096; a valid
 * device.  PTG_EINVAL otherwise (and for NULL arrays), PTG_ENOMEM or PTG_ECUDA from the set-up.
 */
typedef struct ptg_design ptg_design;
int ptg_design_create(int nx, int ny, double h, double r_fil, double beta, double eta, int device,
                      ptg_design** out);
void ptg_design_destroy(ptg_design* d);
int ptg_design_forward(ptg_design* d, const double* chi_d, double* rho_d, double* dproj_d, cudaStream_t stream);
int ptg_design_backward(ptg_design* d, const double* dproj_d, const double* df_drho_d, double* df_dchi_d,
                        cudaStream_t stream);
int ptg_design_volume(ptg_design* d, const double* rho_d, double* vol_d, cudaStream_t stream);

/*
 * The design update of Alg. 3 on the host: the Method of Moving Asymptotes (Svanberg 1987) for
 * min f0(x) s.t. f1(x) <= 0 and x_min <= x <= x_max (the paper's large-beta variant is not
 * given; this is the plain method).  Moving asymptotes (shrink 0.7 on oscillation, expand 1.2
 * on monotone progress), move limit `move`, convex separable models, and the single-multiplier
 * dual solved by bisection.  ptg_mma_update takes host arrays of length n (x, df0, df1) and
 * writes the next iterate to x_new (host); it keeps the last two iterates and asymptotes.
 * PTG_EINVAL for n < 1, x_max <= x_min, move <= 0 or NULL arrays; PTG_ENOMEM from create.
 */
typedef struct ptg_mma ptg_mma;
int ptg_mma_create(int n, double x_min, double x_max, double move, ptg_mma** out);
void ptg_mma_destroy(ptg_mma* m);
int ptg_mma_update(ptg_mma* m, const double* x, double f0, const double* df0, double f1, const double* df1,
                   double* x_new);
/* The state MMA carries between updates (to save and resume a design loop): the update count k
 * and, as host arrays of length n, the last two iterates x1 (newest) and x2 and the last
 * asymptotes L, U.  set_state restores exactly what get_state returned. */
int ptg_mma_get_state(const ptg_mma* m, long long* k, double* x1, double* x2, double* L, double* U);
int ptg_mma_set_state(ptg_mma* m, long long k, const double* x1, const double* x2, const double* L, const double* U);

/* Copy the device status and counters into *out (synchronises the op's last stream). */
int ptg_get_stats(ptg_op* op, ptg_stats* out);

/*
 * Bound of the device-side waits of this op's cooperative-grid launches (ptg_solve.grid_wide):
 * a CTA that has polled a grid barrier `polls` times without the release records PTG_ETIMEOUT
 * in the status word and stops waiting, and so does every later wait of that launch, so the
 * launch ends with the error and meaningless results instead of hanging.  0 restores the
 * default (2^20 polls, never reached by a correct co-resident launch); a small value makes the
 * waits give up early (failure-detection tests).  Negative: PTG_EINVAL.  Applies to launches
 * made after the call.
 */
int ptg_op_set_wait_limit(ptg_op* op, long long polls);

/* Clear the device status word and the counters (asynchronous on stream). */
int ptg_reset_stats(ptg_op* op, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PTG_H */
