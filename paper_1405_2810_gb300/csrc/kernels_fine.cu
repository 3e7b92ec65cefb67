// FP64 envelope block Cholesky for the fine SWIP-DG systems of the offline
// builder (Section 3.2 on one-cell blocks: three unknowns per block, Sx = nx).
// Left-looking over block rows with row panels [N_k][W_k] in global memory,
// the inverse of every diagonal block kept for the substitutions, and one
// step of iterative refinement with an FP64 residual. One CTA per system.
#include "lrbms_internal.cuh"

namespace lrbms {

namespace {

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
__global__ void k_fine_solve(const SimDev* __restrict__ sims, const int* __restrict__ active,
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

}  // namespace

cudaError_t launch_fine_solve(const SimDev* sims, const int* active, int n_active, cudaStream_t st) {
  k_fine_solve<<<n_active, 256, 64 * 64 * sizeof(double), st>>>(sims, active, 0, 1);
  return cudaGetLastError();
}

}  // namespace lrbms
