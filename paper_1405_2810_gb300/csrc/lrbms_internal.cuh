// Internal device-side layout of a resident simulation and the kernel
// launchers shared between the translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lrbms {

constexpr int kMaxM = 16;         // largest number of mobility profiles
constexpr int kCellTile = 2048;   // most cells per tile of the per-cell kernels (tiles are whole rows)
constexpr int kMaxNx = 8192;      // widest fine grid (a tile row and its faces sit in shared memory)
constexpr int kCellThreads = 256;
constexpr int kFaceThreads = 256;

// Status words (same values as lrbms_status).
constexpr int kStOk = 0;
constexpr int kStNotSpd = -4;
constexpr int kStNonFinite = -5;
constexpr int kStTimeout = -6;
constexpr int kStCfl = -8;

// Everything a kernel needs about one simulation. Lives in device memory,
// one entry per slot; all pointers point into the context's arena.
struct SimDev {
  // grid and coarse grid
  int nx, ny, Sx, Sy, cx, cy;
  int n_cells, n_sub, n_cf, nb, nxf, n_faces;
  int M, N, max_NE;
  int panel_words;  // max over block rows of N_k * (padded W_k): shared-memory panel of the solve
  int max_w;        // widest block row W_k of the solve
  int tile_rows;    // grid rows per tile: max(1, kCellTile / nx)
  int n_tiles;      // ceil(ny / tile_rows)
  int n_blocks;     // n_sub + n_cf assembled blocks
  int relperm, swapped, prof_mode, dt_mode;
  int refactor_period;  // steps one FP32 factor serves (mixed solver)
  int refactor_stages;  // steps over which the next FP32 factor is built (1: all at once)
  int vel_mode;         // mobility of the velocity: 0 lambda(s^n), 1 fitted (needs theta of the step)
  int transport;        // 0: P0 finite volume upwind; 1: P1 DG with the slope limiter
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
  const long long* loff;    // [n_sub+1] panel k stored transposed: [W_k][N_k], W_k = xoff[k+1]-xoff[jlo_k];
                            // offsets are multiples of 4 elements (16-byte aligned copies)
  const long long* ioff;    // [n_sub+1] inverse of diagonal block k, [N_k][N_k], then its transpose;
                            // same alignment
  const unsigned long long* sched;  // copy schedule of the substitutions (launch_sched)

  // per-step cell data and load-time coefficients
  double* lam;      // [2][n_cells] lambda(s^n), ping-pong like s
  double* fw;       // [2][n_cells] f_w(s^n), ping-pong like s
  double* inv_pv;   // [n_cells] 1 / (phi_e |e|)
  double* fcoef;    // [3][n_faces] per-face coefficients of the flux (k_prepare)
  double* fwD;      // [nb] f_w(s_D) of every boundary face (k_prepare)

  // state and work arrays
  double* s;        // [2][n_cells] ping-pong; current = steps & 1 (cell means)
  double* sslope;   // [2][2][n_cells] P1-DG slopes c1, c2 per half (transport 1; else null)
  double* sunl;     // [2][n_cells] unlimited slopes of the next step (transport 1; else null)
  double* p;        // [3][n_cells]
  double* F;        // [n_faces]
  double* x;        // [N]
  double* xp;       // [N] previous step's solution (initial guess of the mixed solver)
  double* xpp;      // [N] the solution before that
  double* b;        // [N]
  double* y;        // [2N] substitution work (forward result, then backward result)
  double* rv;       // [N] refinement residual
  double* dv;       // [N] refinement correction (conjugate gradients: preconditioned residual)
  double* pv;       // [N] conjugate gradients: search direction (mixed solver)
  double* qv;       // [N] conjugate gradients: A times the search direction
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
  int* fit_ready;   // [1] lambda, f_w and the fit sums of the current s are computed
  int* inject;      // [1] test hook: non-zero withholds one copy of the next substitution (may be null)
  int* info;        // [8] solve bookkeeping (kernels_solve.cu, kInfo*); may be null
};

__host__ __device__ inline int jlo_of(int k, int Sx) { return k - Sx > 0 ? k - Sx : 0; }

constexpr int kSolveWarps = 4;  // warps of the CTA that solves one reduced system
// 64-bit words of the substitution copy schedule: kSolveWarps + 1 list starts,
// then the warps' lists, together at most n_sub (4 Sx + 16) chunk descriptors.
// Per block row and direction: the leader's two chunks, and the other warps'
// C columns of a panel row of n2 <= 32 elements in pieces of pc columns, at
// most C / pc + 3 pieces. A FIFO holds at least panel_words / 4 + 965
// elements and pc n2 >= FIFO / 2 - 36, while C <= 32 Sx and C n2 <=
// panel_words: C / pc < min(8, 2.2 Sx), so at most 2 (5 + min(8, 2.2 Sx))
// chunks per block row.
inline size_t sched_words(int n_sub, int Sx) {
  return kSolveWarps + 1 + (size_t)n_sub * (4 * (size_t)Sx + 16);
}

// Launchers (all enqueue on `st`; `active` lists slot indices, device array).
// Load-time coefficients of one simulation (device pointer to its SimDev).
void launch_prepare(const SimDev* sim, int n_items, cudaStream_t st);
void launch_fit(const SimDev* sims, const int* active, int n_active, int max_tiles,
                cudaStream_t st);
void launch_assemble(const SimDev* sims, const int* active, int n_active, int max_blocks,
                     int mixed, cudaStream_t st, int threads = 128);
constexpr int kMaxNE = 32;  // local basis sizes 1..32 (one warp lane per row)
constexpr size_t kMaxSolveSmem = 220 * 1024;  // leaves room for static shared memory
// Shape maxima over the simulations of one solve launch.
struct SolveShape {
  int n_sub, panel_words, max_w, N;
};
// Shared memory of the solve kernels for elements of `elem` bytes.
size_t solve_smem_bytes(int n_sub, int panel_words, int max_w, int N, size_t elem);
// Shared-memory panel size (elements) and widest block row of the reduced
// solve for basis sizes NE with prefix sums xoff (lengths n_sub, n_sub + 1).
// In shared memory every block of a row starts on a multiple of 4 columns and
// a row may carry up to 4 columns of stride padding.
inline void solve_panel_sizes(int n_sub, int Sx, const int* NE, const int* xoff, int* panel_words,
                              int* max_w) {
  int pw = 0, mw = 0;
  for (int k = 0; k < n_sub; ++k) {
    const int W = xoff[k + 1] - xoff[jlo_of(k, Sx)];
    int Wp = 0;
    for (int i = jlo_of(k, Sx); i <= k; ++i) Wp += (NE[i] + 3) & ~3;
    if (NE[k] * (Wp + 4) > pw) pw = NE[k] * (Wp + 4);
    if (W > mw) mw = W;
  }
  *panel_words = pw;
  *max_w = mw;
}
// Offsets of the factor panels and diagonal inverses (multiples of 4 elements;
// block k holds L_kk^-1 and then (L_kk^-1)^T).
__host__ __device__ inline void solve_offsets(int n_sub, int Sx, const int* NE, const int* xoff, long long* loff,
                                              long long* ioff) {
  loff[0] = 0;
  ioff[0] = 0;
  for (int k = 0; k < n_sub; ++k) {
    const long long w = (long long)NE[k] * (xoff[k + 1] - xoff[jlo_of(k, Sx)]);
    loff[k + 1] = loff[k] + ((w + 3) & ~3LL);
    ioff[k + 1] = ioff[k] + 2 * (((long long)NE[k] * NE[k] + 3) & ~3LL);  // inverse and its transpose
  }
}
// mode 0: FP64 factor; mode 1: FP32 factor (FP64 for simulations whose FP32
// factorisation meets a non-positive pivot). Both refine with FP64 residuals.
cudaError_t launch_chol_solve(const SimDev* sims, const int* active, int n_active, int mode, int iters,
                              const SolveShape& sh, cudaStream_t st);
// The mixed solver's FP32 factorisation step alone (k_factor32), after prepare_chol_solve.
cudaError_t launch_factor32(const SimDev* sims, const int* active, int n_active, const SolveShape& sh,
                            cudaStream_t st);
// Shared-memory attributes of the solve kernels for a launch shape; call
// before launch_chol_solve (and outside a stream capture).
cudaError_t prepare_chol_solve(int mode, const SolveShape& sh);
// Substitution copy schedule of one simulation (device pointer to its SimDev,
// whose NE, xoff, loff, ioff and sched are set).
void launch_sched(const SimDev* sim, cudaStream_t st);
// FP64 solve of the fine systems of the offline builder (one-cell blocks).
cudaError_t launch_fine_solve(const SimDev* sims, const int* active, int n_active, cudaStream_t st);
void launch_reconstruct(const SimDev* sims, const int* active, int n_active, int max_sub,
                        int mixed, cudaStream_t st, int threads = 256);
// Face fluxes and per-tile CFL maxima; smem = flux_cfl_smem of the widest tile.
void launch_flux_cfl(const SimDev* sims, const int* active, int n_active, int max_tiles, size_t smem,
                     cudaStream_t st);
cudaError_t prepare_flux_cfl(size_t smem);
inline size_t flux_cfl_smem(int nx, int ny, int tile_rows) {
  const int nr = tile_rows < ny ? tile_rows : ny;
  return 8 * ((size_t)nr * (nx + 1) + (size_t)(nr + 1) * nx);
}
void launch_transport(const SimDev* sims, const int* active, int n_active, int max_tiles,
                      cudaStream_t st);
// P1-DG transport and the slope limiter (simulations with transport 1 only).
void launch_transport_dg(const SimDev* sims, const int* active, int n_active, int max_tiles,
                         cudaStream_t st);
void launch_finalize(const SimDev* sims, const int* active, int n_active, cudaStream_t st,
                     int* status_out = nullptr);
void launch_to_float(const double* src, float* dst, size_t n, cudaStream_t st);
// Saturations in (src: also lambda, f_w and the fit sums of the new state)
// and out, per active simulation; max_tiles: the largest n_tiles among them.
void launch_sat_io(const SimDev* sims, const int* active, int n_active, int max_tiles, const double* const* src,
                   double* const* dst, cudaStream_t st);

}  // namespace lrbms
