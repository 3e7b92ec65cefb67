// Reduced system of Eq. reducedSystem: assembly and solve.
//
// assemble: theta = G^+ r (normal equations of Eq. leastSquaresFit from the
//   fixed-order sum of the fit partials), then every block
//   A_b = c_b + sum_q theta_q (b_q)_b and every subdomain right-hand side
//   b_E = e_E + sum_q theta_q (d_q)_E, streamed from the component arrays.
// chol_solve: one CTA per simulation. The matrix is symmetric positive
//   definite with a 5-point block pattern over the Sx x Sy subdomains; in
//   lexicographic subdomain order its Cholesky factor lives in the envelope
//   j in [k - Sx, k] of every block row k. Block row k of L is kept as a dense
//   N_k x W_k panel (left-looking: L_kj = (A_kj - sum_i L_ki L_ji^T) L_jj^-T,
//   L_kk = chol(A_kk - sum_i L_ki L_ki^T)); the inverse of every diagonal block
//   is kept to turn the triangular solves into small products. Forward and
//   backward substitution follow, then iterative refinement with an FP64
//   residual r = b - A x. The factor is kept in FP64 (mode 0) or FP32 (mode 1:
//   FP32 factor and substitutions, FP64 residual and update, which converges to
//   the FP64 solution when cond(A) eps_32 < 1).
#include "lrbms_internal.cuh"

namespace lrbms {

namespace {

// theta = G^+ (sum over tiles of the fit partials), by warp 0; w[0] = 1.
__device__ void compute_weights(const SimDev& S, double* w, double* rsh, bool store) {
  const int M = S.M;
  if (threadIdx.x < 32) {
    const int q = threadIdx.x;
    if (q < M) {
      double r = 0.0;
      for (int t = 0; t < S.n_tiles; ++t) r += S.fit_part[(size_t)t * kMaxM + q];
      rsh[q] = r;
    }
    __syncwarp();
    if (q < M) {
      double th = 0.0;
      for (int j = 0; j < M; ++j) th = fma(S.Gpinv[q * M + j], rsh[j], th);
      w[1 + q] = th;
      if (store) S.theta[q] = th;
    }
    if (q == 0) w[0] = 1.0;
  }
  __syncthreads();
}

__global__ void k_assemble(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int bidx = blockIdx.x;
  if (bidx >= S.n_blocks + S.n_sub || S.status[0] != kStOk) return;
  __shared__ double w[kMaxM + 1];
  __shared__ double rsh[kMaxM];
  compute_weights(S, w, rsh, bidx == 0);
  const int Q = S.M + 1;
  if (bidx < S.n_blocks) {
    const long long o = S.aoff[bidx];
    const int size = (int)(S.aoff[bidx + 1] - o);
    const double* c = S.comp + (size_t)Q * o;
    for (int i = threadIdx.x; i < size; i += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc = fma(w[q], c[(size_t)q * size + i], acc);
      S.A[o + i] = acc;
    }
  } else {
    const int E = bidx - S.n_blocks;
    const int NE = S.NE[E], x0 = S.xoff[E];
    const double* c = S.rhs + (size_t)Q * x0;
    for (int i = threadIdx.x; i < NE; i += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc = fma(w[q], c[(size_t)q * NE + i], acc);
      S.b[x0 + i] = acc;
    }
  }
}

// Mixed precision: FP32 components, FP32 products accumulated in FP32.
__global__ void k_assemble32(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int bidx = blockIdx.x;
  if (bidx >= S.n_blocks + S.n_sub || S.status[0] != kStOk) return;
  __shared__ double w[kMaxM + 1];
  __shared__ double rsh[kMaxM];
  compute_weights(S, w, rsh, bidx == 0);
  float wf[kMaxM + 1];
  const int Q = S.M + 1;
#pragma unroll
  for (int q = 0; q < kMaxM + 1; ++q) wf[q] = q < Q ? (float)w[q] : 0.0f;
  if (bidx < S.n_blocks) {
    const long long o = S.aoff[bidx];
    const int size = (int)(S.aoff[bidx + 1] - o);
    const float* c = S.comp32 + (size_t)Q * o;
    for (int i = threadIdx.x; i < size; i += blockDim.x) {
      float acc = 0.0f;
      for (int q = 0; q < Q; ++q) acc = fmaf(wf[q], c[(size_t)q * size + i], acc);
      S.A[o + i] = (double)acc;
    }
  } else {
    const int E = bidx - S.n_blocks;
    const int NE = S.NE[E], x0 = S.xoff[E];
    const double* c = S.rhs + (size_t)Q * x0;
    for (int i = threadIdx.x; i < NE; i += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc = fma(w[q], c[(size_t)q * NE + i], acc);
      S.b[x0 + i] = acc;
    }
  }
}

// Index of the assembled coupling block between subdomain k and its left
// (dir 0) or lower (dir 1) neighbour; -1 if none.
__device__ __forceinline__ int coupling_block(const SimDev& S, int k, int dir) {
  const int I = k % S.Sx, J = k / S.Sx;
  if (dir == 0) return I > 0 ? S.n_sub + J * (S.Sx - 1) + (I - 1) : -1;
  return J > 0 ? S.n_sub + S.Sy * (S.Sx - 1) + (J - 1) * S.Sx + I : -1;
}
// ... and with its right (dir 2) or upper (dir 3) neighbour.
__device__ __forceinline__ int coupling_block_up(const SimDev& S, int k, int dir) {
  const int I = k % S.Sx, J = k / S.Sx;
  if (dir == 2) return I < S.Sx - 1 ? S.n_sub + J * (S.Sx - 1) + I : -1;
  return J < S.Sy - 1 ? S.n_sub + S.Sy * (S.Sx - 1) + J * S.Sx + I : -1;
}

// Sum over a group of G lanes (G a power of two dividing 32, groups aligned
// inside warps); every lane of the warp must call it.
template <typename T>
__device__ __forceinline__ T group_sum(T v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Envelope block Cholesky of the assembled A (FP64) with factor storage T.
// Returns false if a pivot is not positive (or not finite).
template <typename T>
__device__ bool factor(const SimDev& S, T* Lst, T* Linv, T* tmp) {
  const int nsub = S.n_sub, Sx = S.Sx;
  __shared__ int bad;
  __shared__ T dsh;
  if (threadIdx.x == 0) bad = 0;
  for (int k = 0; k < nsub; ++k) {
    const int jl = jlo_of(k, Sx);
    const int base = S.xoff[jl];
    const int W = S.xoff[k + 1] - base;
    const int Nk = S.NE[k];
    T* R = Lst + S.loff[k];
    for (int i = threadIdx.x; i < Nk * W; i += blockDim.x) R[i] = T(0);
    __syncthreads();
    {
      const double* Akk = S.A + S.aoff[k];
      const int cd = S.xoff[k] - base;
      for (int i = threadIdx.x; i < Nk * Nk; i += blockDim.x) {
        const int r = i / Nk, c = i - r * Nk;
        R[r * W + cd + c] = (T)Akk[i];
      }
      for (int dir = 0; dir < 2; ++dir) {
        const int bblk = coupling_block(S, k, dir);
        if (bblk < 0) continue;
        const int j = dir == 0 ? k - 1 : k - Sx;
        const int Nj = S.NE[j];
        const double* Ab = S.A + S.aoff[bblk];  // [N_j][N_k] = A_{j,k}
        const int cj = S.xoff[j] - base;
        for (int i = threadIdx.x; i < Nk * Nj; i += blockDim.x) {
          const int r = i / Nj, c = i - r * Nj;  // A_{k,j}[r][c] = A_{j,k}[c][r]
          R[r * W + cj + c] = (T)Ab[c * Nk + r];
        }
      }
    }
    __syncthreads();
    for (int j = jl; j <= k; ++j) {
      const int Nj = S.NE[j];
      const int c0 = S.xoff[j] - base;
      const int jlj = jlo_of(j, Sx);
      const int Wj = S.xoff[j + 1] - S.xoff[jlj];
      const T* Lj = Lst + S.loff[j];
      const int offj = base - S.xoff[jlj];
      const int len = c0;
      if (len > 0) {
        // R[:, c0:c0+Nj] -= R[:, 0:len] L_j[:, offj:offj+len]^T, each output a
        // dot product split over a group of G lanes when outputs are few
        const int n_out = Nk * Nj;
        int G = 1;
        while (G < 32 && 2 * G * n_out <= (int)blockDim.x && G < len) G *= 2;
        const int lg = threadIdx.x & (G - 1), grp = threadIdx.x / G, n_grp = blockDim.x / G;
        for (int o0 = 0; o0 < n_out; o0 += n_grp) {
          const int o = o0 + grp;
          const int r = o / Nj, c = o - r * Nj;
          const bool live = o < n_out && !(j == k && c > r);
          T acc = T(0);
          if (live) {
            const T* a = R + (size_t)r * W;
            const T* bb = Lj + (size_t)c * Wj + offj;
            for (int t = lg; t < len; t += G) acc = fma(a[t], bb[t], acc);
          }
          if (G > 1) acc = group_sum(acc, G);
          if (live && lg == 0) R[r * W + c0 + c] -= acc;
        }
        __syncthreads();
      }
      if (j < k) {
        const T* Li = Linv + S.ioff[j];
        for (int i = threadIdx.x; i < Nk * Nj; i += blockDim.x) {
          const int r = i / Nj, c = i - r * Nj;
          T acc = T(0);
          for (int t = 0; t <= c; ++t) acc = fma(R[r * W + c0 + t], Li[c * Nj + t], acc);
          tmp[i] = acc;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < Nk * Nj; i += blockDim.x) {
          const int r = i / Nj, c = i - r * Nj;
          R[r * W + c0 + c] = tmp[i];
        }
        __syncthreads();
      } else {
        for (int c = 0; c < Nk; ++c) {
          if (threadIdx.x == 0) {
            const T d = R[c * W + c0 + c];
            if (!(d > T(0)) || !isfinite((double)d)) bad = 1;
            dsh = sqrt(d);
            R[c * W + c0 + c] = dsh;
          }
          __syncthreads();
          if (bad) return false;
          for (int r = c + 1 + threadIdx.x; r < Nk; r += blockDim.x) R[r * W + c0 + c] /= dsh;
          __syncthreads();
          const int m = Nk - c - 1;
          for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
            const int r = c + 1 + i / m, t = c + 1 + i % m;
            if (t <= r) R[r * W + c0 + t] -= R[r * W + c0 + c] * R[t * W + c0 + c];
          }
          __syncthreads();
        }
        // zero the strict upper triangle and invert the diagonal block
        for (int i = threadIdx.x; i < Nk * Nk; i += blockDim.x) {
          const int r = i / Nk, c = i - r * Nk;
          if (c > r) R[r * W + c0 + c] = T(0);
        }
        __syncthreads();
        T* Li = Linv + S.ioff[k];
        for (int col = threadIdx.x; col < Nk; col += blockDim.x) {
          for (int r = 0; r < Nk; ++r) {
            if (r < col) {
              Li[r * Nk + col] = T(0);
              continue;
            }
            T sum = (r == col) ? T(1) : T(0);
            for (int t = col; t < r; ++t) sum -= R[r * W + c0 + t] * Li[t * Nk + col];
            Li[r * Nk + col] = sum / R[r * W + c0 + r];
          }
        }
        __syncthreads();
      }
    }
  }
  return true;
}

// Solve L L^T out = in with factor storage T (arithmetic in T); y is work.
template <typename T>
__device__ void substitute(const SimDev& S, const T* Lst, const T* Linv, const double* in,
                           double* out, T* y, T* t) {
  const int nsub = S.n_sub, Sx = S.Sx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < nsub; ++k) {
    const int jl = jlo_of(k, Sx);
    const int base = S.xoff[jl];
    const int W = S.xoff[k + 1] - base;
    const int Nk = S.NE[k];
    const int off = W - Nk;
    const T* R = Lst + S.loff[k];
    for (int r = warp; r < Nk; r += nw) {
      T acc = T(0);
      for (int g = lane; g < off; g += 32) acc = fma(R[(size_t)r * W + g], y[base + g], acc);
      acc = group_sum(acc, 32);
      if (lane == 0) t[r] = (T)in[S.xoff[k] + r] - acc;
    }
    __syncthreads();
    const T* Li = Linv + S.ioff[k];
    for (int r = threadIdx.x; r < Nk; r += blockDim.x) {
      T acc = T(0);
      for (int c = 0; c <= r; ++c) acc = fma(Li[r * Nk + c], t[c], acc);
      y[S.xoff[k] + r] = acc;
    }
    __syncthreads();
  }
  // backward: the second half of y holds the solution in T
  T* z = y + S.N;
  for (int k = nsub - 1; k >= 0; --k) {
    const int Nk = S.NE[k];
    const int kmax = min(k + Sx, nsub - 1);
    for (int c = warp; c < Nk; c += nw) {
      T acc = T(0);
      for (int kk = k + 1; kk <= kmax; ++kk) {
        const int jl2 = jlo_of(kk, Sx);
        const int W2 = S.xoff[kk + 1] - S.xoff[jl2];
        const int col = S.xoff[k] - S.xoff[jl2] + c;
        const T* R2 = Lst + S.loff[kk];
        const int N2 = S.NE[kk];
        for (int r = lane; r < N2; r += 32) acc = fma(R2[(size_t)r * W2 + col], z[S.xoff[kk] + r], acc);
      }
      acc = group_sum(acc, 32);
      if (lane == 0) t[c] = y[S.xoff[k] + c] - acc;
    }
    __syncthreads();
    const T* Li = Linv + S.ioff[k];
    for (int c = threadIdx.x; c < Nk; c += blockDim.x) {
      T acc = T(0);
      for (int r = c; r < Nk; ++r) acc = fma(Li[r * Nk + c], t[r], acc);
      z[S.xoff[k] + c] = acc;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < S.N; i += blockDim.x) out[i] = (double)z[i];
  __syncthreads();
}

// r = b - A x with the block-sparse assembled A, in FP64.
__device__ void residual(const SimDev& S, const double* x, const double* b, double* r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int E = 0; E < S.n_sub; ++E) {
    const int NE = S.NE[E], x0 = S.xoff[E];
    for (int i = warp; i < NE; i += nw) {
      double acc = 0.0;
      const double* Ad = S.A + S.aoff[E];
      for (int c = lane; c < NE; c += 32) acc = fma(Ad[i * NE + c], x[x0 + c], acc);
      for (int dir = 0; dir < 2; ++dir) {  // neighbours earlier in the order: A_{E,j} = blk^T
        const int bb = coupling_block(S, E, dir);
        if (bb < 0) continue;
        const int j = dir == 0 ? E - 1 : E - S.Sx;
        const int Nj = S.NE[j];
        const double* Ab = S.A + S.aoff[bb];  // [N_j][N_E]
        for (int c = lane; c < Nj; c += 32) acc = fma(Ab[c * NE + i], x[S.xoff[j] + c], acc);
      }
      for (int dir = 2; dir < 4; ++dir) {  // neighbours later in the order: A_{E,j} = blk
        const int bb = coupling_block_up(S, E, dir);
        if (bb < 0) continue;
        const int j = dir == 2 ? E + 1 : E + S.Sx;
        const int Nj = S.NE[j];
        const double* Ab = S.A + S.aoff[bb];  // [N_E][N_j]
        for (int c = lane; c < Nj; c += 32) acc = fma(Ab[i * Nj + c], x[S.xoff[j] + c], acc);
      }
      acc = group_sum(acc, 32);
      if (lane == 0) r[x0 + i] = b[x0 + i] - acc;
    }
  }
  __syncthreads();
}

// x = (L L^T)^-1 b, then `iters` refinement steps x += (L L^T)^-1 (b - A x)
// with the residual in FP64.
template <typename T>
__device__ void solve_refine(const SimDev& S, const T* Lst, const T* Linv, int iters, T* sm) {
  T* y = reinterpret_cast<T*>(S.y);  // [2N] of T (the y array holds 2N doubles)
  substitute<T>(S, Lst, Linv, S.b, S.x, y, sm);
  for (int it = 0; it < iters; ++it) {
    residual(S, S.x, S.b, S.rv);
    substitute<T>(S, Lst, Linv, S.rv, S.dv, y, sm);
    for (int i = threadIdx.x; i < S.N; i += blockDim.x) S.x[i] += S.dv[i];
    __syncthreads();
  }
}

// mode 0: FP64 factor, `iters` refinement steps.
// mode 1: FP32 factor with FP64 residuals (`iters` steps); a simulation whose
//         FP32 factorisation meets a non-positive pivot is factorised in FP64.
__global__ void k_chol_solve(const SimDev* __restrict__ sims, const int* __restrict__ active,
                             int mode, int iters) {
  const SimDev& S = sims[active[blockIdx.x]];
  if (S.status[0] != kStOk) return;
  extern __shared__ double sm[];
  if (mode == 1) {
    float* Lf = reinterpret_cast<float*>(S.L);
    float* Lif = reinterpret_cast<float*>(S.Linv);
    if (factor<float>(S, Lf, Lif, reinterpret_cast<float*>(sm))) {
      solve_refine<float>(S, Lf, Lif, iters, reinterpret_cast<float*>(sm));
      return;
    }
    __syncthreads();
  }
  if (!factor<double>(S, S.L, S.Linv, sm)) {
    if (threadIdx.x == 0) S.status[0] = kStNotSpd;
    return;
  }
  solve_refine<double>(S, S.L, S.Linv, mode == 1 ? iters : iters, sm);
}

// ---------------------------------------------------------------- static scratch
// Reduced solve for callers that must not allocate device memory: the factor
// panels, diagonal inverses, work vectors and offset tables live in this
// file-scope array, which every GPU that loads the library holds until exit.
constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Offset tables from the basis sizes (one thread; n_sub is modest).
__global__ void k_noalloc_tables(SimDev S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int* NE = const_cast<int*>(S.NE);
  int* xoff = const_cast<int*>(S.xoff);
  long long* aoff = const_cast<long long*>(S.aoff);
  long long* loff = const_cast<long long*>(S.loff);
  long long* ioff = const_cast<long long*>(S.ioff);
  xoff[0] = 0;
  for (int E = 0; E < S.n_sub; ++E) xoff[E + 1] = xoff[E] + NE[E];
  aoff[0] = 0;
  for (int E = 0; E < S.n_sub; ++E) aoff[E + 1] = aoff[E] + (long long)NE[E] * NE[E];
  int b = S.n_sub;
  for (int J = 0; J < S.Sy; ++J)
    for (int I = 0; I + 1 < S.Sx; ++I, ++b) aoff[b + 1] = aoff[b] + (long long)NE[J * S.Sx + I] * NE[J * S.Sx + I + 1];
  for (int J = 0; J + 1 < S.Sy; ++J)
    for (int I = 0; I < S.Sx; ++I, ++b) aoff[b + 1] = aoff[b] + (long long)NE[J * S.Sx + I] * NE[(J + 1) * S.Sx + I];
  loff[0] = 0;
  ioff[0] = 0;
  for (int k = 0; k < S.n_sub; ++k) {
    loff[k + 1] = loff[k] + (long long)NE[k] * (xoff[k + 1] - xoff[jlo_of(k, S.Sx)]);
    ioff[k + 1] = ioff[k] + (long long)NE[k] * NE[k];
  }
  S.status[0] = kStOk;
}

__global__ void k_chol_solve_static(SimDev S, int mode, int iters) {
  extern __shared__ double sm[];
  if (mode == 1) {
    float* Lf = reinterpret_cast<float*>(S.L);
    float* Lif = reinterpret_cast<float*>(S.Linv);
    if (factor<float>(S, Lf, Lif, reinterpret_cast<float*>(sm))) {
      solve_refine<float>(S, Lf, Lif, iters, reinterpret_cast<float*>(sm));
      return;
    }
    __syncthreads();
  }
  if (!factor<double>(S, S.L, S.Linv, sm)) {
    if (threadIdx.x == 0) S.status[0] = kStNotSpd;
    return;
  }
  solve_refine<double>(S, S.L, S.Linv, iters, sm);
}

}  // namespace

void launch_assemble(const SimDev* sims, const int* active, int n_active, int max_blocks,
                     int mixed, cudaStream_t st) {
  if (mixed)
    k_assemble32<<<dim3(max_blocks, n_active), 128, 0, st>>>(sims, active);
  else
    k_assemble<<<dim3(max_blocks, n_active), 128, 0, st>>>(sims, active);
}

void launch_chol_solve(const SimDev* sims, const int* active, int n_active, int mode, int iters,
                       cudaStream_t st) {
  const size_t smem = 64 * 64 * sizeof(double);  // max_NE <= 64 (checked at load)
  k_chol_solve<<<n_active, 256, smem, st>>>(sims, active, mode, iters);
}

}  // namespace lrbms

// ---------------------------------------------------------------- C ABI
#include "lrbms.h"

namespace {
constexpr int kMaxDevices = 64;
unsigned char* g_noalloc_dev[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int lrbms_solve_noalloc(int Sx, int Sy, const int* N_E, const double* A, const double* rhs,
                                   double* x, int solver, int refine_iters, void* stream) {
  using namespace lrbms;
  if (Sx < 1 || Sy < 1 || !N_E || !A || !rhs || !x || refine_iters < 0 || refine_iters > 16 ||
      (solver != LRBMS_SOLVE_FP64 && solver != LRBMS_SOLVE_MIXED))
    return LRBMS_E_ARG;
  const int n_sub = Sx * Sy;
  const int n_cf = Sy * (Sx - 1) + (Sy - 1) * Sx;
  // sizes from the caller's (host) basis sizes; no host or device allocation
  long long N = 0, l_tot = 0, i_tot = 0;
  for (int E = 0; E < n_sub; ++E) {
    if (N_E[E] < 1 || N_E[E] > 64) return LRBMS_E_ARG;
    N += N_E[E];
    i_tot += (long long)N_E[E] * N_E[E];
  }
  {
    long long x0 = 0;  // running prefix for the envelope widths
    for (int k = 0; k < n_sub; ++k) {
      const int jl = jlo_of(k, Sx);
      long long base = 0;
      for (int j = 0; j < jl; ++j) base += N_E[j];
      x0 += N_E[k];
      l_tot += (long long)N_E[k] * (x0 - base);
    }
  }
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t off = 0;
  const size_t o_NE = off; off = up(off + 4 * (size_t)n_sub);
  const size_t o_xoff = off; off = up(off + 4 * (size_t)(n_sub + 1));
  const size_t o_aoff = off; off = up(off + 8 * (size_t)(n_sub + n_cf + 1));
  const size_t o_loff = off; off = up(off + 8 * (size_t)(n_sub + 1));
  const size_t o_ioff = off; off = up(off + 8 * (size_t)(n_sub + 1));
  const size_t o_status = off; off = up(off + 4);
  const size_t o_L = off; off = up(off + 8 * (size_t)l_tot);
  const size_t o_Li = off; off = up(off + 8 * (size_t)i_tot);
  const size_t o_y = off; off = up(off + 16 * (size_t)N);
  const size_t o_rv = off; off = up(off + 8 * (size_t)N);
  const size_t o_dv = off; off = up(off + 8 * (size_t)N);
  if (off > kNoAllocBytes) return LRBMS_E_BUDGET;  // system larger than the static scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LRBMS_E_CUDA;
  if (!g_noalloc_dev[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LRBMS_E_CUDA;
    g_noalloc_dev[dev] = static_cast<unsigned char*>(ptr);
  }
  unsigned char* base = g_noalloc_dev[dev];
  cudaStream_t st = (cudaStream_t)stream;
  SimDev S{};
  S.Sx = Sx; S.Sy = Sy; S.n_sub = n_sub; S.n_cf = n_cf; S.n_blocks = n_sub + n_cf; S.N = (int)N;
  S.NE = (const int*)(base + o_NE); S.xoff = (const int*)(base + o_xoff);
  S.aoff = (const long long*)(base + o_aoff); S.loff = (const long long*)(base + o_loff);
  S.ioff = (const long long*)(base + o_ioff); S.status = (int*)(base + o_status);
  S.L = (double*)(base + o_L); S.Linv = (double*)(base + o_Li); S.y = (double*)(base + o_y);
  S.rv = (double*)(base + o_rv); S.dv = (double*)(base + o_dv);
  S.A = const_cast<double*>(A); S.b = const_cast<double*>(rhs); S.x = x;
  if (cudaMemcpyAsync(base + o_NE, N_E, 4 * (size_t)n_sub, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LRBMS_E_CUDA;
  k_noalloc_tables<<<1, 1, 0, st>>>(S);
  const int mode = solver == LRBMS_SOLVE_MIXED ? 1 : 0;
  const int iters = refine_iters > 0 ? refine_iters : (mode == 1 ? 4 : 1);
  k_chol_solve_static<<<1, 256, 64 * 64 * sizeof(double), st>>>(S, mode, iters);
  if (cudaGetLastError() != cudaSuccess) return LRBMS_E_CUDA;
  int status = 0;
  if (cudaMemcpyAsync(&status, base + o_status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LRBMS_E_CUDA;
  return status == 0 ? LRBMS_OK : LRBMS_E_NOT_SPD;
}
