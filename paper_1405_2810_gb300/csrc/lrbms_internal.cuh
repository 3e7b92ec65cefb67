// Internal device-side layout of a resident simulation and the kernel
// launchers shared between the translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lrbms {

constexpr int kMaxM = 16;         // largest number of mobility profiles
constexpr int kCellTile = 2048;   // cells per tile of the per-cell kernels
constexpr int kCellThreads = 256;
constexpr int kFaceThreads = 256;

// Status words (same values as lrbms_status).
constexpr int kStOk = 0;
constexpr int kStNotSpd = -4;
constexpr int kStNonFinite = -5;

// Everything a kernel needs about one simulation. Lives in device memory,
// one entry per slot; all pointers point into the context's arena.
struct SimDev {
  // grid and coarse grid
  int nx, ny, Sx, Sy, cx, cy;
  int n_cells, n_sub, n_cf, nb, nxf, n_faces;
  int M, N, max_NE;
  int n_tiles;      // ceil(n_cells / kCellTile)
  int n_blocks;     // n_sub + n_cf assembled blocks
  int relperm, swapped, prof_mode, dt_mode;
  double hx, hy, vol, c_pen, Lf, inv_eta_w, inv_eta_o, cfl, dt_fixed, dt_max;
  double lam0, lam1;  // lambda(0), lambda(1)

  // problem data
  const double* perm;
  const double* poro;
  const uint8_t* prof_idx;  // prof_mode 0
  const double* prof;       // prof_mode 1: [M][n_cells]
  const double* Gpinv;      // [M*M]
  const int8_t* bc_type;    // [nb]
  const double* p_D;
  const double* v_N;
  const double* s_D;

  // reduced basis and components
  const int* NE;            // [n_sub]
  const int* xoff;          // [n_sub+1]
  const long long* phi_off; // [n_sub]
  const double* Phi;
  const float* Phi32;       // mixed precision copy (or null)
  const long long* aoff;    // [n_blocks+1] offsets of assembled blocks
  const double* comp;       // block b at (M+1)*aoff[b]: [M+1][size_b]
  const float* comp32;
  const double* rhs;        // subdomain E at (M+1)*xoff[E]: [M+1][N_E]

  // block Cholesky factor (envelope of the lexicographic subdomain order)
  const long long* loff;    // [n_sub+1] row panel k: [N_k][W_k], W_k = xoff[k+1]-xoff[jlo_k]
  const long long* ioff;    // [n_sub+1] inverse of diagonal block k: [N_k][N_k]

  // state and work arrays
  double* s;        // [2][n_cells] ping-pong; current = steps & 1
  double* p;        // [3][n_cells]
  double* F;        // [n_faces]
  double* x;        // [N]
  double* b;        // [N]
  double* y;        // [2N] substitution work (forward result, then backward result)
  double* rv;       // [N] refinement residual
  double* dv;       // [N] refinement correction
  double* A;        // [aoff[n_blocks]]
  double* L;        // [loff[n_sub]]
  double* Linv;     // [ioff[n_sub]]
  double* fit_part; // [n_tiles][kMaxM]
  double* cfl_part; // [n_tiles]
  double* mass_part;// [n_tiles]
  double* scal;     // [0] t, [1] dt, [2] cumulative boundary outflow volume,
                    // [3] boundary outflow rate of the last step
  double* theta;    // [M]
  int* status;      // [1]
  int* steps;       // [1]
};

__host__ __device__ inline int jlo_of(int k, int Sx) { return k - Sx > 0 ? k - Sx : 0; }

// Launchers (all enqueue on `st`; `active` lists slot indices, device array).
void launch_fit(const SimDev* sims, const int* active, int n_active, int max_tiles,
                cudaStream_t st);
void launch_assemble(const SimDev* sims, const int* active, int n_active, int max_blocks,
                     int mixed, cudaStream_t st);
void launch_chol_solve(const SimDev* sims, const int* active, int n_active, int mode, int iters,
                       cudaStream_t st);
void launch_reconstruct(const SimDev* sims, const int* active, int n_active, int max_sub,
                        int mixed, cudaStream_t st);
void launch_flux(const SimDev* sims, const int* active, int n_active, int max_faces,
                 cudaStream_t st);
void launch_cfl(const SimDev* sims, const int* active, int n_active, int max_tiles,
                cudaStream_t st);
void launch_transport(const SimDev* sims, const int* active, int n_active, int max_tiles,
                      cudaStream_t st);
void launch_finalize(const SimDev* sims, const int* active, int n_active, cudaStream_t st);
void launch_to_float(const double* src, float* dst, size_t n, cudaStream_t st);
void launch_sat_io(const SimDev* sims, const int* active, int n_active, const double* const* src,
                   double* const* dst, cudaStream_t st);

}  // namespace lrbms
