// mesh.h -- host launchers of the coarse-mesh transfer kernels (mesh.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ptg {

// Row r of a stack of vectors of length n lives at p + (row0 + r * step) * n (step may be
// negative or zero); p == nullptr marks an absent operand.
struct MeshRows {
  const double* p;
  long long row0, step;
};
struct MeshRowsW {
  double* p;
  long long row0, step;
};
inline MeshRows mrows(const double* p, long long row0 = 0, long long step = 1) { return MeshRows{p, row0, step}; }
inline MeshRowsW mrowsw(double* p, long long row0 = 0, long long step = 1) { return MeshRowsW{p, row0, step}; }

constexpr int kMeshThreads = 256;
int mesh_blocks(int Nn);   // blocks of the prolongation (the p-norm partials per row)

cudaError_t mesh_design(int nx, int ny, const double* rho, double* rhoH, cudaStream_t st);
cudaError_t mesh_inject(int nx, int ny, MeshRows in, MeshRowsW out, int nrows, const uint8_t* dirH, cudaStream_t st);
cudaError_t mesh_source(int nx, int ny, MeshRows T, MeshRowsW out, int nrows, const double* Theta, double p, int p_int,
                        int objective, const uint8_t* dirF, const uint8_t* dirH, cudaStream_t st);
cudaError_t mesh_prolong(int nx, int ny, MeshRows c1, MeshRows c2, MeshRows c3, MeshRows f1, MeshRows f2,
                         MeshRowsW out, MeshRowsW out2, MeshRowsW hist, int nrows, const uint8_t* dirF,
                         const uint8_t* dirH, int p_int, double* pn_partial, cudaStream_t st);
cudaError_t mesh_theta_old(int nrows, int nb, const double* partial, const double* theta_in, double* theta_out,
                           double inv_norm, double p, int p_int, int objective, cudaStream_t st);
cudaError_t mesh_theta_chain(int ntau, int nb, const double* partial, const double* F, const double* G, double* X,
                             double inv_norm, double p, int p_int, int objective, cudaStream_t st);
cudaError_t mesh_dg(int nx, int ny, double h, double dtau, int has_dc, const double* dk, const double* dc, MeshRows lam,
                    const double* T_hist, int M, int s0, int s_step, int nrows, double inv_ntau, double* dg,
                    cudaStream_t st);
cudaError_t mesh_g_old(int Ne, int ntau, const double* g_in, const double* dg, double* g_out, cudaStream_t st);
cudaError_t mesh_g_chain(int Ne, int ntau, const double* dg_rev, const double* F, const double* G, double* X,
                         cudaStream_t st);

}  // namespace ptg
