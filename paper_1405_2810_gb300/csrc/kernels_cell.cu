// Per-cell and per-face kernels of the LRBMS online step:
//   prepare    (at load) per-face coefficients of Definition 2 and 1/(phi|e|)
//   fit        lambda(s^n) and f_w(s^n) per cell, and the partial sums of the
//              normal equations of Eq. leastSquaresFit (only after the
//              saturation was set from outside: otherwise the transport
//              kernel of the previous step has computed them)
//   reconstruct p_E = Phi_E x_E (Algorithm 3, step 5(b))
//   flux_cfl   face fluxes of Definition 2 (Eq. velocityDG) with mobility
//              lambda(s^n), and per tile the maximum of outflow_e / (phi|e|)
//              (the inverse of the CFL bound)
//   transport  explicit upwind update of Definition 3 with P0 saturation, then
//              lambda, f_w and the fit sums of the new saturation
//   finalize   time, cumulative boundary outflow and step counter
// Tiles are blocks of whole grid rows (tile_rows rows, at most kCellTile
// cells). Every reduction uses this fixed partition and a fixed order, so a
// simulation's results do not depend on which other simulations share the
// launch.
#include "lrbms_internal.cuh"

#include <cfloat>

namespace lrbms {

namespace {

__device__ __forceinline__ const double* cur_s(const SimDev& S) {
  return S.s + (size_t)(S.steps[0] & 1) * S.n_cells;
}
__device__ __forceinline__ double* next_s(const SimDev& S) {
  return S.s + (size_t)((S.steps[0] + 1) & 1) * S.n_cells;
}
// lambda and f_w of the current saturation, and of the next one (ping-pong
// like the saturation).
__device__ __forceinline__ size_t cur_half(const SimDev& S) { return (size_t)(S.steps[0] & 1) * S.n_cells; }
__device__ __forceinline__ size_t next_half(const SimDev& S) { return (size_t)((S.steps[0] + 1) & 1) * S.n_cells; }

// max(v, 0) for a double by its sign bit (integer pipe; the FP64 pipe of
// this part is narrow). A NaN with a clear sign bit passes through.
__device__ __forceinline__ double pos_part(double v) { return __double_as_longlong(v) > 0 ? v : 0.0; }

// First and one-past-last cell of a tile (blocks of whole rows).
__device__ __forceinline__ void tile_range(const SimDev& S, int tile, int& e0, int& e1) {
  const int j0 = tile * S.tile_rows;
  e0 = j0 * S.nx;
  e1 = min(j0 + S.tile_rows, S.ny) * S.nx;
}

// Eq. brooksCorey: lambda_w = k_rw/eta_w, lambda_o = k_ro/eta_o.
__device__ __forceinline__ void phase_mob(const SimDev& S, double s, double& lw, double& lo) {
  if (S.relperm == 0) {
    lw = s * s * S.inv_eta_w;
    lo = (1.0 - s) * (1.0 - s) * S.inv_eta_o;
  } else {
    lw = s * S.inv_eta_w;
    lo = (1.0 - s) * S.inv_eta_o;
  }
}
// Eq. frationalFlow.
__device__ __forceinline__ double frac_flow(const SimDev& S, double s) {
  double lw, lo;
  phase_mob(S, s, lw, lo);
  return lw / (lw + lo);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Fixed-order block sum of one value per thread; result valid in thread 0.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) r += red[i];
  return r;
}
__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) r = fmax(r, red[i]);
  return r;
}

// ------------------------------------------------------------------ prepare
// Per-face coefficients of Definition 2 (they depend on the permeability
// only): interior faces F = -(c0 lambda_1 dp_1 + c1 lambda_2 dp_2) + c2 [p],
// with c0 = |f| (2/h_n) tau_1 kappa_1, c1 = |f| (2/h_n) tau_2 kappa_2 (mean
// weights of reading R3) and c2 = sigma_f (|f| sigma_f / h_f = sigma_f in 2D);
// Dirichlet faces: c0 = |f| (2/h_n) kappa_e, c2 = c_pen kappa_e, c1 = p_D;
// Neumann faces: c0 = c2 = 0, c1 = |f| v_N. Per cell: 1/(phi_e |e|).
__global__ void k_prepare(const SimDev* __restrict__ sp) {
  const SimDev& S = *sp;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  for (int e = i0; e < S.n_cells; e += stride) S.inv_pv[e] = 1.0 / (S.poro[e] * S.vol);
  const int nx = S.nx, ny = S.ny, nf = S.n_faces;
  for (int f = i0; f < nf; f += stride) {
    int e1 = -1, e2 = -1, bidx = -1;
    double flen, dscale;
    if (f < S.nxf) {
      const int j = f / (nx + 1), i = f - j * (nx + 1);
      if (i > 0) e1 = j * nx + i - 1;
      if (i < nx) e2 = j * nx + i;
      if (i == 0) bidx = j;
      if (i == nx) bidx = ny + j;
      flen = S.hy;
      dscale = 2.0 / S.hx;
    } else {
      const int g = f - S.nxf;
      const int j = g / nx, i = g - j * nx;
      if (j > 0) e1 = (j - 1) * nx + i;
      if (j < ny) e2 = j * nx + i;
      if (j == 0) bidx = 2 * ny + i;
      if (j == ny) bidx = 2 * ny + nx + i;
      flen = S.hx;
      dscale = 2.0 / S.hy;
    }
    double c0, c1, c2;
    if (e1 >= 0 && e2 >= 0) {
      const double k1 = S.perm[e1], k2 = S.perm[e2];
      const double ks = k1 + k2;
      const double t1 = (S.swapped ? k2 : k1) / ks;
      const double t2 = (S.swapped ? k1 : k2) / ks;
      c0 = flen * dscale * t1 * k1;
      c1 = flen * dscale * t2 * k2;
      c2 = S.c_pen * 2.0 * k1 * k2 / ks;
    } else {
      const int e = (e1 >= 0) ? e1 : e2;
      if (S.bc_type[bidx] == 1) {
        const double ke = S.perm[e];
        c0 = flen * dscale * ke;
        c1 = S.p_D[bidx];
        c2 = S.c_pen * ke;
      } else {
        c0 = 0.0;
        c1 = flen * S.v_N[bidx];
        c2 = 0.0;
      }
    }
    S.fcoef[f] = c0;
    S.fcoef[(size_t)nf + f] = c1;
    S.fcoef[2 * (size_t)nf + f] = c2;
  }
  for (int b = i0; b < S.nb; b += stride) S.fwD[b] = frac_flow(S, S.s_D[b]);
}

// ------------------------------------------------------------------ fit
// lambda(s_e) and f_w(s_e) (stored for the flux and transport kernels) and the
// contribution of cell e to r_q = sum_e Lambda^q_e lambda(s_e). With the
// threshold profiles of Algorithm 2 (Lambda^q_e = lambda(1) if q >= k_e else
// lambda(0)) the cells are binned by k_e and r follows from the bin sums.
__device__ __forceinline__ void fit_cell(const SimDev& S, double s, int e, double* lam_out, double* fw_out,
                                         double (&acc)[kMaxM]) {
  double lw, lo;
  phase_mob(S, s, lw, lo);
  const double lam = lw + lo;
  lam_out[e] = lam;
  fw_out[e] = lw / lam;  // Eq. frationalFlow
  if (S.prof_mode == 0) {
    switch (S.prof_idx[e] - 1) {  // one add: the cell's bin
#define LRBMS_BIN(q) \
  case q:            \
    acc[q] += lam;   \
    break;
      LRBMS_BIN(0) LRBMS_BIN(1) LRBMS_BIN(2) LRBMS_BIN(3) LRBMS_BIN(4) LRBMS_BIN(5) LRBMS_BIN(6)
      LRBMS_BIN(7) LRBMS_BIN(8) LRBMS_BIN(9) LRBMS_BIN(10) LRBMS_BIN(11) LRBMS_BIN(12) LRBMS_BIN(13)
      LRBMS_BIN(14) LRBMS_BIN(15)
#undef LRBMS_BIN
      default: break;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kMaxM; ++q)
      if (q < S.M) acc[q] += S.prof[(size_t)q * S.n_cells + e] * lam;
  }
}

// Block sums of the tile's fit contributions -> fit_part[tile]: every warp
// reduces its M bins by shuffles (the accumulators stay in registers: every
// index is a compile-time constant), then thread q adds the warps' partial
// sums of bin q in warp order (fixed order, one barrier).
__device__ void fit_store(const SimDev& S, const double (&acc)[kMaxM], int tile) {
  __shared__ double red[kCellThreads / 32][kMaxM];
  __shared__ double tot[kMaxM];
  const int M = S.M, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kMaxM; ++q) {
    if (q < M) {
      const double v = warp_sum(acc[q]);
      if (lane == 0) red[w][q] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double v = 0.0;
    for (int i = 0; i < nw; ++i) v += red[i][threadIdx.x];
    tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    const int q = threadIdx.x;  // 0-based profile q+1
    double r;
    if (S.prof_mode == 0) {
      // bins tot[k-1] hold sum of lambda over cells with index k
      r = 0.0;
      for (int k = 1; k <= M; ++k) r += tot[k - 1] * ((q + 1 >= k) ? S.lam1 : S.lam0);
    } else {
      r = tot[q];
    }
    S.fit_part[(size_t)tile * kMaxM + q] = r;
  }
}

// Fit of the current saturation; skipped when the previous step's transport
// kernel has already computed it (fit_ready).
__global__ void k_fit(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int tile = blockIdx.x;
  if (tile >= S.n_tiles || S.status[0] != kStOk || S.fit_ready[0]) return;
  const double* s = cur_s(S);
  double acc[kMaxM];
#pragma unroll
  for (int q = 0; q < kMaxM; ++q) acc[q] = 0.0;
  int e0, e1;
  tile_range(S, tile, e0, e1);
  double* lam = S.lam + cur_half(S);
  double* fw = S.fw + cur_half(S);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) fit_cell(S, s[e], e, lam, fw, acc);
  fit_store(S, acc, tile);
}

// ------------------------------------------------------------------ reconstruct
__global__ void k_reconstruct(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int E = blockIdx.x;
  if (E >= S.n_sub || S.status[0] != kStOk) return;
  extern __shared__ double xs[];
  const int NE = S.NE[E];
  const int x0 = S.xoff[E];
  for (int i = threadIdx.x; i < NE; i += blockDim.x) xs[i] = S.x[x0 + i];
  __syncthreads();
  const int cells = S.cx * S.cy;
  const int rows = 3 * cells;
  const double* Phi = S.Phi + S.phi_off[E];
  const int I = E % S.Sx, J = E / S.Sx;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < NE; ++i) acc = fma(Phi[(size_t)i * rows + r], xs[i], acc);
    const int k = r / cells, c = r - k * cells;
    const int li = c % S.cx, lj = c / S.cx;
    const int ge = (J * S.cy + lj) * S.nx + I * S.cx + li;
    S.p[(size_t)k * S.n_cells + ge] = acc;
  }
}

__global__ void k_reconstruct32(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int E = blockIdx.x;
  if (E >= S.n_sub || S.status[0] != kStOk) return;
  extern __shared__ double xsd[];
  float* xs = reinterpret_cast<float*>(xsd);
  const int NE = S.NE[E];
  const int x0 = S.xoff[E];
  for (int i = threadIdx.x; i < NE; i += blockDim.x) xs[i] = (float)S.x[x0 + i];
  __syncthreads();
  const int cells = S.cx * S.cy;
  const int rows = 3 * cells;
  const float* Phi = S.Phi32 + S.phi_off[E];
  const int I = E % S.Sx, J = E / S.Sx;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    float acc = 0.0f;
    for (int i = 0; i < NE; ++i) acc = fmaf(Phi[(size_t)i * rows + r], xs[i], acc);
    const int k = r / cells, c = r - k * cells;
    const int li = c % S.cx, lj = c / S.cx;
    const int ge = (J * S.cy + lj) * S.nx + I * S.cx + li;
    S.p[(size_t)k * S.n_cells + ge] = (double)acc;
  }
}

// ------------------------------------------------------------------ flux
// Definition 2 for P1 pressure and P0 coefficients: the normal gradient is
// constant per cell and the jump is linear along the face, so with the
// coefficients of k_prepare
//   F = -(c0 lambda_1 dp_1 + c1 lambda_2 dp_2) + c2 [p](midpoint),
// dp the normal-direction dof of each cell (the gradient times h_n / 2).
// Mobility of a cell in Definition 2: lambda(s^n) of the cell (reading R7),
// or the fitted mobility sum_q theta_q Lambda^q_e of the reduced system
// (variant; from a per-profile-index table for threshold profiles).
struct MobState {
  const double* lam;
  __device__ __forceinline__ double operator[](int e) const { return lam[e]; }
};
struct MobFitIndexed {
  const uint8_t* k;
  const double* tab;  // [kMaxM + 1]: fitted mobility of a cell whose first lambda(1) index is k
  __device__ __forceinline__ double operator[](int e) const { return tab[k[e]]; }
};
struct MobFitDense {
  const double* prof;
  const double* theta;  // shared copy
  int M, n;
  __device__ __forceinline__ double operator[](int e) const {
    double v = 0.0;
    for (int q = 0; q < M; ++q) v = fma(theta[q], prof[(size_t)q * n + e], v);
    return v;
  }
};

template <typename Mob>
__device__ __forceinline__ double face_flux(const SimDev& S, const Mob& lam, int f) {
  const double* p0 = S.p;
  const int nx = S.nx, ny = S.ny, nf = S.n_faces;
  int e1 = -1, e2 = -1, bidx = -1;
  bool xface;
  if (f < S.nxf) {
    xface = true;
    const int j = f / (nx + 1), i = f - j * (nx + 1);
    if (i > 0) e1 = j * nx + i - 1;
    if (i < nx) e2 = j * nx + i;
    if (i == 0) bidx = j;
    if (i == nx) bidx = ny + j;
  } else {
    xface = false;
    const int g = f - S.nxf;
    const int j = g / nx, i = g - j * nx;
    if (j > 0) e1 = (j - 1) * nx + i;
    if (j < ny) e2 = j * nx + i;
    if (j == 0) bidx = 2 * ny + i;
    if (j == ny) bidx = 2 * ny + nx + i;
  }
  const double* pt = S.p + (xface ? 1 : 2) * (size_t)S.n_cells;  // normal-direction dof
  const double c0 = S.fcoef[f], c1 = S.fcoef[(size_t)nf + f], c2 = S.fcoef[2 * (size_t)nf + f];
  if (e1 >= 0 && e2 >= 0) {
    const double jump = (p0[e1] + pt[e1]) - (p0[e2] - pt[e2]);
    return -(c0 * lam[e1] * pt[e1] + c1 * lam[e2] * pt[e2]) + c2 * jump;
  }
  const int e = (e1 >= 0) ? e1 : e2;
  const double sgn = (e1 >= 0) ? 1.0 : -1.0;  // outward normal along +axis?
  double Fout;
  if (S.bc_type[bidx] == 1) {
    const double pmid = p0[e] + sgn * pt[e];
    Fout = -c0 * lam[e] * (sgn * pt[e]) + c2 * (pmid - c1);
  } else {
    Fout = c1;
  }
  return sgn * Fout;
}

// Fluxes of every face that touches the tile's rows, staged in shared memory
// ([nr][nx+1] x-faces, then [nr+1][nx] y-faces); the faces the tile owns (its
// x-faces and the y-faces above its rows, plus the bottom boundary for the
// first tile) are written to F, each face by exactly one tile (the y-faces
// below a tile are computed again, bitwise the same, by the tile above them).
// Then per cell outflow_e / (phi_e |e|) and its tile maximum (cfl_part).
template <typename Mob>
__device__ void tile_fluxes(const SimDev& S, const Mob& lam, double* fsh, int j0, int nfx, int nfy) {
  const int nx = S.nx;
  for (int t = threadIdx.x; t < nfx + nfy; t += blockDim.x) {
    int f;
    bool own;
    if (t < nfx) {
      f = j0 * (nx + 1) + t;
      own = true;
    } else {
      const int u = t - nfx, r = u / nx;
      f = S.nxf + j0 * nx + u;
      own = r > 0 || j0 == 0;
    }
    const double F = face_flux(S, lam, f);
    fsh[t] = F;
    if (own) S.F[f] = F;
  }
}

__global__ void k_flux_cfl(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int tile = blockIdx.x;
  if (tile >= S.n_tiles || S.status[0] != kStOk) return;
  extern __shared__ double fsh[];
  const int nx = S.nx;
  const int j0 = tile * S.tile_rows, nr = min(S.tile_rows, S.ny - j0);
  const int nfx = nr * (nx + 1), nfy = (nr + 1) * nx;
  if (S.vel_mode == 0) {
    tile_fluxes(S, MobState{S.lam + cur_half(S)}, fsh, j0, nfx, nfy);
  } else {
    __shared__ double th[kMaxM], tab[kMaxM + 1];
    if (threadIdx.x < S.M) th[threadIdx.x] = S.theta[threadIdx.x];
    __syncthreads();
    if (S.prof_mode == 0) {
      // index k: Lambda^q = lambda(0) for q < k, lambda(1) for q >= k (1-based)
      if (threadIdx.x >= 1 && threadIdx.x <= S.M) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int q = 1; q <= S.M; ++q) v = fma(th[q - 1], q >= k ? S.lam1 : S.lam0, v);
        tab[k] = v;
      }
      __syncthreads();
      tile_fluxes(S, MobFitIndexed{S.prof_idx, tab}, fsh, j0, nfx, nfy);
    } else {
      tile_fluxes(S, MobFitDense{S.prof, th, S.M, S.n_cells}, fsh, j0, nfx, nfy);
    }
  }
  __syncthreads();
  const double* Fx = fsh;
  const double* Fy = fsh + nfx;
  double m = 0.0;
  for (int c = threadIdx.x; c < nr * nx; c += blockDim.x) {
    const int r = c / nx, i = c - r * nx;
    const double out = pos_part(-Fx[r * (nx + 1) + i]) + pos_part(Fx[r * (nx + 1) + i + 1]) +
                       pos_part(-Fy[r * nx + i]) + pos_part(Fy[(r + 1) * nx + i]);
    m = fmax(m, out * S.inv_pv[j0 * nx + c]);
  }
  __shared__ double red[32];
  const double rmax = block_max(m, red);
  if (threadIdx.x == 0) S.cfl_part[tile] = rmax;
}

// Outward fluxes of cell (i,j): left face -F, right +F, bottom -F, top +F.
__device__ __forceinline__ void cell_faces(const SimDev& S, int e, int& fl, int& fr, int& fb,
                                           int& ft) {
  const int nx = S.nx;
  const int j = e / nx, i = e - j * nx;
  fl = j * (nx + 1) + i;
  fr = fl + 1;
  fb = S.nxf + j * nx + i;
  ft = fb + nx;
}

// Reading R12: dt = cfl min_e phi_e|e| / (L_f outflow_e) = cfl / (L_f max_e outflow_e / (phi_e|e|)),
// divided by 2k + 1 = 3 for the piecewise-linear DG transport.
__device__ __forceinline__ double step_dt(const SimDev& S) {
  if (S.dt_mode == 1) return S.dt_fixed;
  double m = 0.0;
  for (int t = 0; t < S.n_tiles; ++t) m = fmax(m, S.cfl_part[t]);
  double dt = (m > 0.0) ? S.cfl / (S.Lf * m) : DBL_MAX;
  if (S.transport == 1 && dt < DBL_MAX) dt /= 3.0;
  if (S.dt_max > 0.0) dt = fmin(dt, S.dt_max);
  return dt;
}

// ------------------------------------------------------------------ transport
// Face term G_f = F_f f_w(s_up) with s_up from the face's own upwind rule
// (s|e1 if F >= 0, else s|e2; s_D on boundary inflow). Both cells of an
// interior face evaluate G_f from identical operands, so it cancels exactly
// in the total water volume.
// F >= 0 by the bit pattern (integer pipe): +0 and -0 count as >= 0; a NaN
// flux makes the new saturation non-finite either way.
__device__ __forceinline__ bool nonneg(double F) {
  const long long b = __double_as_longlong(F);
  return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool finite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ double face_term_interior(const double* fw, double F, int e1, int e2) {
  return F * (nonneg(F) ? fw[e1] : fw[e2]);
}
// Boundary face b with outward flux Fo: the cell's own f_w on outflow,
// f_w(s_D) (computed at load) on inflow.
__device__ __forceinline__ double face_term_boundary(const SimDev& S, const double* fw, double Fo, int e, int b) {
  return Fo * (nonneg(Fo) ? fw[e] : S.fwD[b]);
}

// A fixed step beyond the CFL bound with CFL number 1 (dt L_f outflow_e /
// (phi_e |e|) > 1 in some cell) is refused: the simulation is frozen with
// status kStCfl before its saturation changes.
__device__ __forceinline__ bool fixed_step_breaks_cfl(const SimDev& S) {
  if (S.dt_mode != 1 || !(S.Lf > 0.0)) return false;
  double m = 0.0;
  for (int t = 0; t < S.n_tiles; ++t) m = fmax(m, S.cfl_part[t]);
  return S.dt_fixed * S.Lf * m * (S.transport == 1 ? 3.0 : 1.0) > 1.0;
}

__global__ void k_transport(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int tile = blockIdx.x;
  if (tile >= S.n_tiles || S.status[0] != kStOk || S.transport != 0) return;
  __shared__ double dt_sh;
  __shared__ int cfl_bad;
  if (threadIdx.x == 0) {
    dt_sh = step_dt(S);
    cfl_bad = fixed_step_breaks_cfl(S);
    if (cfl_bad && tile == 0) S.status[0] = kStCfl;
  }
  __syncthreads();
  if (cfl_bad) return;
  const double dt = dt_sh;
  const double* s = cur_s(S);
  double* sn = next_s(S);
  const int nx = S.nx, ny = S.ny;
  int e0, e1;
  tile_range(S, tile, e0, e1);
  double bout = 0.0;
  bool bad = !(dt > 0.0 && dt < DBL_MAX);
  const double* fw = S.fw + cur_half(S);
  double* lam_n = S.lam + next_half(S);
  double* fw_n = S.fw + next_half(S);
  double acc[kMaxM];
#pragma unroll
  for (int q = 0; q < kMaxM; ++q) acc[q] = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int j = e / nx, i = e - j * nx;
    int fl, fr, fb, ft;
    cell_faces(S, e, fl, fr, fb, ft);
    double net = 0.0, g;
    // left face: this cell is e2; outward flux -F
    if (i > 0) {
      net -= face_term_interior(fw, S.F[fl], e - 1, e);
    } else {
      g = face_term_boundary(S, fw, -S.F[fl], e, j);
      net += g;
      bout += g;
    }
    if (i < nx - 1) {
      net += face_term_interior(fw, S.F[fr], e, e + 1);
    } else {
      g = face_term_boundary(S, fw, S.F[fr], e, ny + j);
      net += g;
      bout += g;
    }
    if (j > 0) {
      net -= face_term_interior(fw, S.F[fb], e - nx, e);
    } else {
      g = face_term_boundary(S, fw, -S.F[fb], e, 2 * ny + i);
      net += g;
      bout += g;
    }
    if (j < ny - 1) {
      net += face_term_interior(fw, S.F[ft], e, e + nx);
    } else {
      g = face_term_boundary(S, fw, S.F[ft], e, 2 * ny + nx + i);
      net += g;
      bout += g;
    }
    const double v = s[e] - dt * S.inv_pv[e] * net;
    if (!finite_bits(v)) bad = true;
    sn[e] = v;
    fit_cell(S, v, e, lam_n, fw_n, acc);  // the next step's fit (Eq. leastSquaresFit)
  }
  __shared__ double red[32];
  const double tot = block_sum(bout, red);
  const int anybad = __syncthreads_or(bad ? 1 : 0);
  if (threadIdx.x == 0) {
    S.mass_part[tile] = tot;
    if (anybad) S.status[0] = kStNonFinite;
  }
  fit_store(S, acc, tile);
}


// ------------------------------------------------------------------ P1-DG transport
// Definition 3 with k = 1 (Eq. saturationDG, explicit Euler, gravity and
// sources zero, the saturation penalty dropped as for k = 0): per cell the
// mean c0 (in s) and the slopes c1, c2 of s_h = c0 + c1 psi1 + c2 psi2 in the
// pressure's local basis (in sslope); the velocity is the lowest-order
// Raviart-Thomas field of the face fluxes, u_x = (F_l (1 - r) + F_r (1 + r)) /
// (2 hy), u_y = (F_b (1 - t) + F_t (1 + t)) / (2 hx) in the cell's reference
// coordinates r, t; 3 x 3 Gauss points in the cell and 3 on each face. Both
// cells of a face evaluate its upwind values from the same operands, so the
// face terms of the means cancel exactly in the total water volume.
__constant__ double kGX[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};  // Gauss-Legendre nodes sqrt(3/5)
__constant__ double kGW[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};

// s_h at tangential coordinate q on side 0 (left), 1 (right), 2 (bottom), 3 (top)
__device__ __forceinline__ double dg_trace(double c0, double c1, double c2, int side, double q) {
  switch (side) {
    case 0: return c0 - c1 + c2 * q;
    case 1: return c0 + c1 + c2 * q;
    case 2: return c0 + c1 * q - c2;
    default: return c0 + c1 * q + c2;
  }
}

__device__ __forceinline__ size_t slope_half(const SimDev& S, int parity) {
  return (size_t)(parity & 1) * 2 * S.n_cells;
}

__global__ void k_transport_dg(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int tile = blockIdx.x;
  if (tile >= S.n_tiles || S.status[0] != kStOk || S.transport != 1) return;
  __shared__ double dt_sh;
  __shared__ int cfl_bad;
  if (threadIdx.x == 0) {
    dt_sh = step_dt(S);
    cfl_bad = fixed_step_breaks_cfl(S);
    if (cfl_bad && tile == 0) S.status[0] = kStCfl;
  }
  __syncthreads();
  if (cfl_bad) return;
  const double dt = dt_sh;
  const int n = S.n_cells, nx = S.nx, ny = S.ny;
  const double* s = cur_s(S);
  double* sn = next_s(S);
  const double* sl = S.sslope + slope_half(S, S.steps[0]);
  double* unl = S.sunl;  // [2][n] unlimited slopes of s^{n+1}
  double* lam_n = S.lam + next_half(S);
  double* fw_n = S.fw + next_half(S);
  const double hx = S.hx, hy = S.hy, vol = S.vol;
  int e0, e1;
  tile_range(S, tile, e0, e1);
  double bout = 0.0;
  bool bad = !(dt > 0.0 && dt < DBL_MAX);
  double acc[kMaxM];
#pragma unroll
  for (int q = 0; q < kMaxM; ++q) acc[q] = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int j = e / nx, i = e - j * nx;
    const double c0 = s[e], c1 = sl[e], c2 = sl[n + e];
    int fl, fr, fb, ft;
    cell_faces(S, e, fl, fr, fb, ft);
    const double Fs[4] = {S.F[fl], S.F[fr], S.F[fb], S.F[ft]};
    double R0 = 0.0, R1 = 0.0, R2 = 0.0;
    // volume term: f(s) u . grad psi_j with grad psi1 = (2/hx, 0), grad psi2 = (0, 2/hy)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double ux = (Fs[0] * (1.0 - kGX[a]) + Fs[1] * (1.0 + kGX[a])) / (2.0 * hy);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double uy = (Fs[2] * (1.0 - kGX[b]) + Fs[3] * (1.0 + kGX[b])) / (2.0 * hx);
        const double w = kGW[a] * kGW[b] * vol / 4.0;
        const double f = frac_flow(S, c0 + c1 * kGX[a] + c2 * kGX[b]);
        R1 += w * f * ux * (2.0 / hx);
        R2 += w * f * uy * (2.0 / hy);
      }
    }
    // face terms: -int_f (u . n_out) f(s_up) psi_j ds
#pragma unroll
    for (int side = 0; side < 4; ++side) {
      const double sgn = (side & 1) ? 1.0 : -1.0;
      const double Fout = sgn * Fs[side];
      int nb = -1, bidx = -1;
      if (side == 0) { if (i > 0) nb = e - 1; else bidx = j; }
      if (side == 1) { if (i < nx - 1) nb = e + 1; else bidx = ny + j; }
      if (side == 2) { if (j > 0) nb = e - nx; else bidx = 2 * ny + i; }
      if (side == 3) { if (j < ny - 1) nb = e + nx; else bidx = 2 * ny + nx + i; }
      const bool own_up = sgn > 0.0 ? (Fout >= 0.0) : (Fout > 0.0);
      double gsum = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double own = dg_trace(c0, c1, c2, side, kGX[q]);
        double up;
        if (nb >= 0) {
          up = own_up ? own : dg_trace(s[nb], sl[nb], sl[n + nb], side ^ 1, kGX[q]);
        } else {
          up = (Fout >= 0.0) ? own : S.s_D[bidx];
        }
        const double g = kGW[q] * frac_flow(S, up);
        const double p1 = side < 2 ? sgn : kGX[q];
        const double p2 = side < 2 ? kGX[q] : sgn;
        R0 -= Fout * 0.5 * g;
        R1 -= Fout * 0.5 * g * p1;
        R2 -= Fout * 0.5 * g * p2;
        gsum += g;
      }
      if (nb < 0) bout += Fout * 0.5 * gsum;
    }
    const double pv = S.poro[e] * vol;
    const double c0n = c0 + dt * R0 / pv;
    const double c1n = c1 + dt * R1 / (pv / 3.0);
    const double c2n = c2 + dt * R2 / (pv / 3.0);
    if (!isfinite(c0n) || !isfinite(c1n) || !isfinite(c2n)) bad = true;
    sn[e] = c0n;
    unl[e] = c1n;
    unl[n + e] = c2n;
    fit_cell(S, c0n, e, lam_n, fw_n, acc);  // the next step's fit, at the cell means
  }
  __shared__ double red[32];
  const double tot = block_sum(bout, red);
  const int anybad = __syncthreads_or(bad ? 1 : 0);
  if (threadIdx.x == 0) {
    S.mass_part[tile] = tot;
    if (anybad) S.status[0] = kStNonFinite;
  }
  fit_store(S, acc, tile);
}

// m_i of the limiter (Section 3.4) from g_i and d_i, the three cases as printed.
__device__ __forceinline__ double gradient_scale(double g, double d) {
  if (g * d < 0.0 && fabs(g) > 1e-8 && fabs(d) > 1e-8) return 0.0;
  if (g * d > 0.0 && fabs(g) > fabs(d) && fabs(g) > 1e-8 && fabs(d) > 1e-8) return d / g;
  return 1.0;
}

// The limiter of Section 3.4 (Eq. limiterMain) on s^{n+1}: shock detector on
// the upstream faces (|int_f [s] ds| / (0.08 d sqrt(h_e) |e|), d = 2, h_e =
// diam(e), s_D on an inflow boundary face), flagged if > 1 or if s_h leaves
// [0, 1] at a vertex; a flagged cell keeps its mean and scales its slopes by
// min_i m_i over its face neighbours. Reads the unlimited slopes of every
// cell (sunl) and writes the limited ones, so cells never see a limited
// neighbour.
__global__ void k_limit_dg(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int tile = blockIdx.x;
  if (tile >= S.n_tiles || S.status[0] != kStOk || S.transport != 1) return;
  const int n = S.n_cells, nx = S.nx, ny = S.ny;
  const double* sn = next_s(S);
  const double* unl = S.sunl;
  double* sl_n = S.sslope + slope_half(S, S.steps[0] + 1);
  const double scale = 1.0 / (0.08 * 2.0 * sqrt(sqrt(S.hx * S.hx + S.hy * S.hy)) * S.vol);
  int e0, e1;
  tile_range(S, tile, e0, e1);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int j = e / nx, i = e - j * nx;
    const double c0 = sn[e], c1 = unl[e], c2 = unl[n + e];
    int fl, fr, fb, ft;
    cell_faces(S, e, fl, fr, fb, ft);
    const double Fs[4] = {S.F[fl], S.F[fr], S.F[fb], S.F[ft]};
    int nbs[4];
    double eta = 0.0;
#pragma unroll
    for (int side = 0; side < 4; ++side) {
      const double sgn = (side & 1) ? 1.0 : -1.0;
      int nb = -1, bidx = -1;
      if (side == 0) { if (i > 0) nb = e - 1; else bidx = j; }
      if (side == 1) { if (i < nx - 1) nb = e + 1; else bidx = ny + j; }
      if (side == 2) { if (j > 0) nb = e - nx; else bidx = 2 * ny + i; }
      if (side == 3) { if (j < ny - 1) nb = e + nx; else bidx = 2 * ny + nx + i; }
      nbs[side] = nb;
      if (sgn * Fs[side] < 0.0) {  // upstream face
        const double own = dg_trace(c0, c1, c2, side, 0.0);
        const double other = nb >= 0 ? dg_trace(sn[nb], unl[nb], unl[n + nb], side ^ 1, 0.0) : S.s_D[bidx];
        eta += fabs((side < 2 ? S.hy : S.hx) * (own - other));
      }
    }
    eta *= scale;
    bool flag = eta > 1.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double sv = c0 + ((v & 1) ? c1 : -c1) + ((v & 2) ? c2 : -c2);
      flag |= sv < 0.0 || sv > 1.0;
    }
    double alpha = 1.0;
    if (flag) {
#pragma unroll
      for (int side = 0; side < 4; ++side) {
        const int nb = nbs[side];
        if (nb < 0) continue;
        const double g = ((side & 1) ? 2.0 : -2.0) * (side < 2 ? c1 : c2);
        alpha = fmin(alpha, gradient_scale(g, sn[nb] - c0));
      }
    }
    sl_n[e] = flag ? alpha * c1 : c1;
    sl_n[n + e] = flag ? alpha * c2 : c2;
  }
}

// ------------------------------------------------------------------ finalize
// status_out (optional) receives every listed simulation's status word, in
// list order, so that the host reads the batch's statuses with one copy.
__global__ void k_finalize(const SimDev* __restrict__ sims, const int* __restrict__ active,
                           int n_active, int* __restrict__ status_out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_active) return;
  const SimDev& S = sims[active[a]];
  const int st = S.status[0];
  if (status_out) status_out[a] = st;
  if (st != kStOk) return;
  const double dt = step_dt(S);
  double out = 0.0;
  for (int t = 0; t < S.n_tiles; ++t) out += S.mass_part[t];
  S.scal[0] += dt;
  S.scal[1] = dt;
  S.scal[2] += dt * out;
  S.scal[3] = out;
  S.steps[0] += 1;
  S.fit_ready[0] = 1;  // k_transport computed lambda, f_w and the fit sums of s^{n+1}
}

// Saturation exchange with caller memory (pinned host or device pointers).
// The saturation of the next step read from caller memory (pinned host or
// device, through unified addressing), tile by tile, together with what the
// step's fit needs of it (lambda, f_w and the fit sums of Eq.
// leastSquaresFit, as k_fit computes them), so that the step's k_fit skips.
__global__ void k_sat_in(const SimDev* __restrict__ sims, const int* __restrict__ active,
                         const double* const* __restrict__ src) {
  const SimDev& S = sims[active[blockIdx.y]];
  const double* in = src[blockIdx.y];
  const int tile = blockIdx.x;
  if (!in || tile >= S.n_tiles) return;
  double* s = S.s + (size_t)(S.steps[0] & 1) * S.n_cells;
  int e0, e1;
  tile_range(S, tile, e0, e1);
  if (S.status[0] != kStOk) {  // frozen: the state is still replaced, nothing is fitted
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) s[e] = in[e];
    if (tile == 0 && threadIdx.x == 0) S.fit_ready[0] = 0;
    return;
  }
  double acc[kMaxM];
#pragma unroll
  for (int q = 0; q < kMaxM; ++q) acc[q] = 0.0;
  double* lam = S.lam + cur_half(S);
  double* fw = S.fw + cur_half(S);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double v = in[e];
    s[e] = v;
    fit_cell(S, v, e, lam, fw, acc);
  }
  fit_store(S, acc, tile);
  if (tile == 0 && threadIdx.x == 0) S.fit_ready[0] = 1;  // every tile is done when the kernel ends
}
__global__ void k_sat_out(const SimDev* __restrict__ sims, const int* __restrict__ active,
                          double* const* __restrict__ dst) {
  const SimDev& S = sims[active[blockIdx.y]];
  double* out = dst[blockIdx.y];
  if (!out) return;
  const double* s = S.s + (size_t)(S.steps[0] & 1) * S.n_cells;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.n_cells; e += gridDim.x * blockDim.x)
    out[e] = s[e];
}

__global__ void k_to_float(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

}  // namespace

void launch_to_float(const double* src, float* dst, size_t n, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_to_float<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n);
}

void launch_sat_io(const SimDev* sims, const int* active, int n_active, int max_tiles, const double* const* src,
                   double* const* dst, cudaStream_t st) {
  if (src) k_sat_in<<<dim3(max_tiles, n_active), kCellThreads, 0, st>>>(sims, active, src);
  if (dst) k_sat_out<<<dim3(16, n_active), 256, 0, st>>>(sims, active, dst);
}

void launch_prepare(const SimDev* sim, int n_items, cudaStream_t st) {
  int blocks = (n_items + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_prepare<<<blocks, 256, 0, st>>>(sim);
}
void launch_fit(const SimDev* sims, const int* active, int n_active, int max_tiles,
                cudaStream_t st) {
  k_fit<<<dim3(max_tiles, n_active), kCellThreads, 0, st>>>(sims, active);
}
// threads: CTA size; every size computes each pressure dof the same way.
void launch_reconstruct(const SimDev* sims, const int* active, int n_active, int max_sub,
                        int mixed, cudaStream_t st, int threads) {
  const size_t smem = 64 * sizeof(double);  // max_NE <= 64 (checked at load)
  if (mixed)
    k_reconstruct32<<<dim3(max_sub, n_active), threads, smem, st>>>(sims, active);
  else
    k_reconstruct<<<dim3(max_sub, n_active), threads, smem, st>>>(sims, active);
}
void launch_flux_cfl(const SimDev* sims, const int* active, int n_active, int max_tiles, size_t smem,
                     cudaStream_t st) {
  k_flux_cfl<<<dim3(max_tiles, n_active), kFaceThreads, smem, st>>>(sims, active);
}
cudaError_t prepare_flux_cfl(size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)k_flux_cfl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
void launch_transport(const SimDev* sims, const int* active, int n_active, int max_tiles,
                      cudaStream_t st) {
  k_transport<<<dim3(max_tiles, n_active), kCellThreads, 0, st>>>(sims, active);
}
void launch_transport_dg(const SimDev* sims, const int* active, int n_active, int max_tiles,
                         cudaStream_t st) {
  k_transport_dg<<<dim3(max_tiles, n_active), kCellThreads, 0, st>>>(sims, active);
  k_limit_dg<<<dim3(max_tiles, n_active), kCellThreads, 0, st>>>(sims, active);
}
void launch_finalize(const SimDev* sims, const int* active, int n_active, cudaStream_t st, int* status_out) {
  k_finalize<<<(n_active + 127) / 128, 128, 0, st>>>(sims, active, n_active, status_out);
}

}  // namespace lrbms
