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
};

// Everything one stepper launch needs (passed by value in parameter space).
struct StepParams {
  // problem
  int nx, ny, Nn, Ne, Nt, Ntau, M;
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
  // op data (device, FP64)
  const double* wA_fine;     // [3][(ny+2)(nx+2)] padded (D, S, T) of C/dt + K
  const double* wA_coarse;   // [3][(ny+2)(nx+2)] padded (D, S, T) of C/dtau + K
  const double* mass;        // [(ny+2)(nx+2)] padded c_e h^2/36
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
};

// Shared-memory footprint (bytes) of one CTA of the stepper for a given plan.
inline size_t stepper_smem_bytes(int nx, int rmax, int real_bytes, int nthreads) {
  const size_t W = (size_t)nx + 3, EW = (size_t)nx + 2;
  const size_t nodes_halo = (size_t)(rmax + 2) * W;
  const size_t elems = (size_t)(rmax + 1) * EW;
  const size_t nown_cap = (size_t)rmax * (nx + 1);
  size_t b = 0;
  b += nodes_halo * sizeof(double);            // x64: FP64 state with halos
  b += nown_cap * sizeof(double);              // b64: FP64 right-hand side of owned nodes
  b += nodes_halo * real_bytes;                // zbuf: preconditioned residual with halos
  b += 3 * elems * real_bytes;                 // (D, S, T) element weights in CG precision
  b = (b + 15) & ~size_t(15);
  (void)nthreads;
  return b;
}

// Host entry points of the kernel translation units.
struct Plan {
  int cs = 0, nthreads = 0, npt = 0, rmax = 0;
  size_t smem = 0;
  int max_active_clusters = 0;
};

cudaError_t launch_stepper(const StepParams& P, const Plan& plan, int precision, int ntasks, cudaStream_t stream);
cudaError_t query_stepper_plan(int nx, int ny, int precision, int kind, int cs, int nthreads, int npt, Plan* plan);

cudaError_t launch_assemble(int nx, int ny, double h, const ptg_material& m, double dt, double dtau, const double* rho,
                            const double* q_elem, const uint8_t* dirichlet, double* k, double* c, double* dk, double* dc,
                            double* wAf, double* wAc, double* mass, double* fload, DevStats* st, cudaStream_t stream);

cudaError_t launch_sensitivities(int nx, int ny, int Nt, double h, double dt, int has_dc, const double* dk,
                                 const double* dc, const double* lam, int j0, int j1, const double* T, int hist_j0,
                                 double* partial, int nchunks, double* grad, cudaStream_t stream);

void set_last_error(const char* msg);

}  // namespace ptg
