// Offline phase on the GPU: Algorithm 2 (initial pressure and velocity,
// time-of-flight, mobility profiles, snapshots and local Gram-Schmidt; the
// greedy selection is replaced by a caller-given list of snapshot parameters)
// followed by the offline/online decomposition of Section 4.4.
//
// The fine SWIP-DG system (Section 3.2) of a P1 pressure on one-cell blocks
// has exactly the 5-point block pattern the online solver factorises, so every
// fine solve here runs through the same envelope block Cholesky
// on a "fine" system with Sx = nx, Sy = ny and three unknowns per block
// (launch_fine_solve).
//
// Local SWIP matrices use closed forms for rectangles: on a face with
// tangential coordinate t in [-1,1], the P1 traces are alpha + beta t, so
// int_f (alpha_a + beta_a t)(alpha_b + beta_b t) = |f| (alpha_a alpha_b +
// beta_a beta_b / 3) and int_f t = 0; volume terms are
// gamma kappa |e| diag(0, 4/hx^2, 4/hy^2).
#include "lrbms.h"
#include "lrbms_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace lrbms {

// Fine-grid data of one problem being built.
struct FineDev {
  int nx, ny, Sx, Sy, cx, cy, n_cells, nxf, n_faces, nb, M, relperm, swapped;
  double hx, hy, vol, c_pen, inv_eta_w, inv_eta_o, lam0, lam1;
  const double* perm;
  const double* poro;
  const int8_t* bc_type;
  const double* p_D;
  const double* v_N;
  const double* s_D;
  const double* s0;
  uint8_t* prof_idx;
  const double* prof;  // [M][n_cells] dense profiles (saturation-snapshot variant), or null
};

// One fine system to assemble: mobility gamma per cell given by
//   mode 0: lambda(s0), mode 1: sum_q mu_q Lambda^q, mode 2: Lambda^q (q = prof)
// and the terms selected by `parts` (bit 0 penalty + Dirichlet-penalty and
// Neumann right-hand side, bit 1 volume + consistency + Dirichlet-consistency
// right-hand side).
struct SysJob {
  int prob, mode, parts, q;
  const double* mu;  // [M]
  double* D;         // [n_cells][9] diagonal blocks
  double* O;         // blocks per interior face in coarse-face order [9] (row e1, col e2)
  double* r;         // [n_cells][3]
};

namespace {

__device__ __forceinline__ double mob_total(const FineDev& f, double s) {
  if (f.relperm == 0) return s * s * f.inv_eta_w + (1.0 - s) * (1.0 - s) * f.inv_eta_o;
  return s * f.inv_eta_w + (1.0 - s) * f.inv_eta_o;
}

__device__ __forceinline__ double job_gamma(const FineDev& f, const SysJob& J, int e) {
  if (J.mode == 0) return mob_total(f, f.s0[e]);
  if (f.prof) {
    if (J.mode == 2) return f.prof[(size_t)J.q * f.n_cells + e];
    double g = 0.0;
    for (int q = 0; q < f.M; ++q) g += J.mu[q] * f.prof[(size_t)q * f.n_cells + e];
    return g;
  }
  const int k = f.prof_idx[e];
  if (J.mode == 2) return (J.q + 1 >= k) ? f.lam1 : f.lam0;
  double g = 0.0;
  for (int q = 0; q < f.M; ++q) g += J.mu[q] * ((q + 1 >= k) ? f.lam1 : f.lam0);
  return g;
}

// Trace coefficients on a face of a cell: value = alpha + beta t.
// side = +1: the face at the cell's + end along `axis`, -1: at its - end.
__device__ __forceinline__ void traces(int axis, int side, double* al, double* be) {
  al[0] = 1.0; be[0] = 0.0;
  if (axis == 0) {
    al[1] = side; be[1] = 0.0;
    al[2] = 0.0; be[2] = 1.0;
  } else {
    al[1] = 0.0; be[1] = 1.0;
    al[2] = side; be[2] = 0.0;
  }
}

// Normal derivative (along +axis) of each local basis function.
__device__ __forceinline__ void dnormal(const FineDev& f, int axis, double* g) {
  g[0] = 0.0;
  g[1] = axis == 0 ? 2.0 / f.hx : 0.0;
  g[2] = axis == 1 ? 2.0 / f.hy : 0.0;
}

// 6x6 local matrix of an interior face (rows/cols 0..2: e1, 3..5: e2), normal
// +axis from e1 to e2: penalty sigma/h int [.][.], consistency and symmetry
// -int {gamma kappa grad . n}[.] (reading R1 sign), weights tau (reading R3).
__device__ void interior_face_matrix(const FineDev& f, int axis, double k1, double g1, double k2,
                                     double g2, int parts, double* Mx) {
  const double flen = axis == 0 ? f.hy : f.hx;
  double a1[3], b1[3], a2[3], b2[3], dn[3];
  traces(axis, +1, a1, b1);
  traces(axis, -1, a2, b2);
  dnormal(f, axis, dn);
  double al[6], be[6], mn[6];
  const double t1 = (f.swapped ? k2 : k1) / (k1 + k2), t2 = (f.swapped ? k1 : k2) / (k1 + k2);
  for (int k = 0; k < 3; ++k) {
    al[k] = a1[k]; be[k] = b1[k]; mn[k] = t1 * g1 * k1 * dn[k];
    al[3 + k] = -a2[k]; be[3 + k] = -b2[k]; mn[3 + k] = t2 * g2 * k2 * dn[k];
  }
  const double sig = f.c_pen * 2.0 * k1 * k2 / (k1 + k2);  // sigma/h_f * |f| = sigma (h_f = |f|)
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double v = 0.0;
      if (parts & 1) v += sig * (al[a] * al[b] + be[a] * be[b] / 3.0);
      if (parts & 2) v -= flen * (al[a] * mn[b] + mn[a] * al[b]);
      Mx[a * 6 + b] = v;
    }
}

// Boundary face of cell e on side `side` along `axis` (outward normal
// side * e_axis): 3x3 matrix and right-hand side.
__device__ void boundary_face(const FineDev& f, int axis, int side, int b, double ke, double ge,
                              int parts, double* Mx, double* rv) {
  const double flen = axis == 0 ? f.hy : f.hx;
  double al[3], be[3], dn[3], mn[3];
  traces(axis, side, al, be);
  dnormal(f, axis, dn);
  for (int k = 0; k < 3; ++k) mn[k] = ge * ke * side * dn[k];
  for (int k = 0; k < 9; ++k) Mx[k] = 0.0;
  for (int k = 0; k < 3; ++k) rv[k] = 0.0;
  if (f.bc_type[b] == 1) {
    const double sig = f.c_pen * ke;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        if (parts & 1) v += sig * (al[a] * al[c] + be[a] * be[c] / 3.0);
        if (parts & 2) v -= flen * (al[a] * mn[c] + mn[a] * al[c]);
        Mx[a * 3 + c] = v;
      }
    for (int a = 0; a < 3; ++a) {
      if (parts & 1) rv[a] += sig * al[a] * f.p_D[b];
      if (parts & 2) rv[a] -= flen * mn[a] * f.p_D[b];
    }
  } else if (parts & 1) {
    for (int a = 0; a < 3; ++a) rv[a] -= flen * al[a] * f.v_N[b];
  }
}

__device__ __forceinline__ int coarse_face_of_fine(const FineDev& f, int face) {
  // interior fine face -> index among interior faces in "coarse-face" order of
  // the one-cell-block system (x-interfaces J*(nx-1)+I, then y-interfaces)
  if (face < f.nxf) {
    const int j = face / (f.nx + 1), i = face - j * (f.nx + 1);
    return j * (f.nx - 1) + (i - 1);
  }
  const int g = face - f.nxf;
  const int j = g / f.nx, i = g - j * f.nx;
  return f.ny * (f.nx - 1) + (j - 1) * f.nx + i;
}

__global__ void k_fine_system(const FineDev* __restrict__ fds, const SysJob* __restrict__ jobs) {
  const SysJob J = jobs[blockIdx.y];
  const FineDev& f = fds[J.prob];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double Mx[36], rv[3];
  if (t < f.n_cells) {
    const int e = t, j = e / f.nx, i = e - j * f.nx;
    const double ke = f.perm[e], ge = job_gamma(f, J, e);
    double D[9], r[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 9; ++k) D[k] = 0.0;
    if (J.parts & 2) {
      D[4] = ge * ke * f.vol * 4.0 / (f.hx * f.hx);
      D[8] = ge * ke * f.vol * 4.0 / (f.hy * f.hy);
    }
    // four faces: (axis, side, neighbour or boundary index)
    for (int s4 = 0; s4 < 4; ++s4) {
      const int axis = s4 >> 1, side = (s4 & 1) ? +1 : -1;
      int nb = -1, bidx = -1;
      if (axis == 0) {
        if (side < 0) { if (i > 0) nb = e - 1; else bidx = j; }
        else { if (i < f.nx - 1) nb = e + 1; else bidx = f.ny + j; }
      } else {
        if (side < 0) { if (j > 0) nb = e - f.nx; else bidx = 2 * f.ny + i; }
        else { if (j < f.ny - 1) nb = e + f.nx; else bidx = 2 * f.ny + f.nx + i; }
      }
      if (nb >= 0) {
        const double kn = f.perm[nb], gn = job_gamma(f, J, nb);
        if (side > 0) {  // this cell is e1
          interior_face_matrix(f, axis, ke, ge, kn, gn, J.parts, Mx);
          for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) D[a * 3 + c] += Mx[a * 6 + c];
        } else {         // this cell is e2
          interior_face_matrix(f, axis, kn, gn, ke, ge, J.parts, Mx);
          for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) D[a * 3 + c] += Mx[(3 + a) * 6 + 3 + c];
        }
      } else {
        boundary_face(f, axis, side, bidx, ke, ge, J.parts, Mx, rv);
        for (int k = 0; k < 9; ++k) D[k] += Mx[k];
        for (int k = 0; k < 3; ++k) r[k] += rv[k];
      }
    }
    for (int k = 0; k < 9; ++k) J.D[(size_t)e * 9 + k] = D[k];
    for (int k = 0; k < 3; ++k) J.r[(size_t)e * 3 + k] = r[k];
  }
  if (t < f.n_faces) {
    const int face = t;
    int e1 = -1, e2 = -1, axis;
    if (face < f.nxf) {
      axis = 0;
      const int j = face / (f.nx + 1), i = face - j * (f.nx + 1);
      if (i > 0 && i < f.nx) { e1 = j * f.nx + i - 1; e2 = e1 + 1; }
    } else {
      axis = 1;
      const int g = face - f.nxf;
      const int j = g / f.nx, i = g - j * f.nx;
      if (j > 0 && j < f.ny) { e1 = (j - 1) * f.nx + i; e2 = e1 + f.nx; }
    }
    if (e1 >= 0) {
      interior_face_matrix(f, axis, f.perm[e1], job_gamma(f, J, e1), f.perm[e2],
                           job_gamma(f, J, e2), J.parts, Mx);
      double* O = J.O + (size_t)coarse_face_of_fine(f, face) * 9;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) O[a * 3 + c] = Mx[a * 6 + 3 + c];
    }
  }
}

// Face fluxes of Definition 2 from a cell-major P1 pressure x[e*3+k], with
// the mobility lambda(s0) (Algorithm 2, step 1(a)).
__global__ void k_fine_flux(const FineDev* __restrict__ fds, const double* const* __restrict__ xs,
                            double* const* __restrict__ Fs) {
  const FineDev& f = fds[blockIdx.y];
  const double* x = xs[blockIdx.y];
  double* F = Fs[blockIdx.y];
  const int face = blockIdx.x * blockDim.x + threadIdx.x;
  if (face >= f.n_faces) return;
  int e1 = -1, e2 = -1, bidx = -1, axis;
  if (face < f.nxf) {
    axis = 0;
    const int j = face / (f.nx + 1), i = face - j * (f.nx + 1);
    if (i > 0) e1 = j * f.nx + i - 1;
    if (i < f.nx) e2 = j * f.nx + i;
    if (i == 0) bidx = j;
    if (i == f.nx) bidx = f.ny + j;
  } else {
    axis = 1;
    const int g = face - f.nxf;
    const int j = g / f.nx, i = g - j * f.nx;
    if (j > 0) e1 = (j - 1) * f.nx + i;
    if (j < f.ny) e2 = j * f.nx + i;
    if (j == 0) bidx = 2 * f.ny + i;
    if (j == f.ny) bidx = 2 * f.ny + f.nx + i;
  }
  const double flen = axis == 0 ? f.hy : f.hx;
  const double dsc = axis == 0 ? 2.0 / f.hx : 2.0 / f.hy;
  const int kt = 1 + axis;  // basis function varying along the normal
  double val;
  if (e1 >= 0 && e2 >= 0) {
    const double k1 = f.perm[e1], k2 = f.perm[e2];
    const double t1 = (f.swapped ? k2 : k1) / (k1 + k2), t2 = (f.swapped ? k1 : k2) / (k1 + k2);
    const double g1 = mob_total(f, f.s0[e1]), g2 = mob_total(f, f.s0[e2]);
    const double mean = t1 * g1 * k1 * dsc * x[e1 * 3 + kt] + t2 * g2 * k2 * dsc * x[e2 * 3 + kt];
    const double jump = (x[e1 * 3] + x[e1 * 3 + kt]) - (x[e2 * 3] - x[e2 * 3 + kt]);
    val = -flen * mean + f.c_pen * 2.0 * k1 * k2 / (k1 + k2) * jump;
  } else {
    const int e = e1 >= 0 ? e1 : e2;
    const double sg = e1 >= 0 ? 1.0 : -1.0;
    double out;
    if (f.bc_type[bidx] == 1) {
      const double ke = f.perm[e], ge = mob_total(f, f.s0[e]);
      out = -flen * ge * ke * sg * dsc * x[e * 3 + kt] +
            f.c_pen * ke * (x[e * 3] + sg * x[e * 3 + kt] - f.p_D[bidx]);
    } else {
      out = flen * f.v_N[bidx];
    }
    val = sg * out;
  }
  F[face] = val;
}

// CFL bound of the initial velocity: min_e phi|e| / outflow_e (as a positive
// double, so the bit pattern orders like the value).
__global__ void k_fine_cfl(const FineDev* __restrict__ fds, double* const* __restrict__ Fs,
                           unsigned long long* out) {
  const FineDev& f = fds[blockIdx.y];
  const double* F = Fs[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.n_cells) return;
  const int j = e / f.nx, i = e - j * f.nx;
  const int fl = j * (f.nx + 1) + i, fb = f.nxf + j * f.nx + i;
  const double o = fmax(-F[fl], 0.0) + fmax(F[fl + 1], 0.0) + fmax(-F[fb], 0.0) + fmax(F[fb + f.nx], 0.0);
  if (o > 0.0) atomicMin(out + blockIdx.y, __double_as_longlong(f.poro[e] * f.vol / o));
}

// One Jacobi sweep of the upwind time-of-flight equations (Eq. timeOfFlight
// with constant test functions): tau_e = (phi|e| + sum_in |F| tau_up) / sum_out F.
__global__ void k_tof_sweep(const FineDev* __restrict__ fds, double* const* __restrict__ Fs,
                            double* const* __restrict__ tin, double* const* __restrict__ tout,
                            int* changed) {
  const FineDev& f = fds[blockIdx.y];
  const double* F = Fs[blockIdx.y];
  const double* a = tin[blockIdx.y];
  double* b = tout[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.n_cells) return;
  const int j = e / f.nx, i = e - j * f.nx;
  const int fl = j * (f.nx + 1) + i, fb = f.nxf + j * f.nx + i;
  const double fo[4] = {-F[fl], F[fl + 1], -F[fb], F[fb + f.nx]};
  const int nbr[4] = {i > 0 ? e - 1 : -1, i < f.nx - 1 ? e + 1 : -1, j > 0 ? e - f.nx : -1,
                      j < f.ny - 1 ? e + f.nx : -1};
  double out = 0.0, src = f.poro[e] * f.vol;
  for (int k = 0; k < 4; ++k) {
    if (fo[k] >= 0.0) out += fo[k];
    else if (nbr[k] >= 0) src += -fo[k] * a[nbr[k]];
  }
  const double v = out > 0.0 ? src / out : DBL_MAX;
  if (v != a[e]) *changed = 1;
  b[e] = v;
}

// Profile index (Algorithm 2, step 1(c)): first q in 2..M-1 with
// tau <= (q-1) T/(M-2), else M; and a histogram of the indices.
// Dense profiles of the saturation-snapshot variant (Section 6): the
// saturations s_q [M][n_cells] are replaced in place by lambda(s_q).
__global__ void k_sat_profiles(const FineDev* __restrict__ fds, int prob, double* __restrict__ P) {
  const FineDev& f = fds[prob];
  const size_t n = (size_t)f.M * f.n_cells;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    P[i] = mob_total(f, P[i]);
}

__global__ void k_profiles(FineDev* fds, double* const* __restrict__ taus, const double* T,
                           unsigned int* hist) {
  FineDev& f = fds[blockIdx.y];
  const double* tau = taus[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= f.n_cells) return;
  int k = f.M;
  for (int q = 2; q <= f.M - 1; ++q)
    if (tau[e] <= (q - 1) * T[blockIdx.y] / (f.M - 2)) {
      k = q;
      break;
    }
  f.prof_idx[e] = (uint8_t)k;
  atomicAdd(hist + blockIdx.y * (kMaxM + 1) + k, 1u);
}

__device__ double block_reduce_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  __syncthreads();
  return r;
}

// Local bases (Algorithm 2, step 2(e)): for subdomain E, the normalised unit
// function, then each snapshot restricted to E, orthonormalised by two passes
// of modified Gram-Schmidt in L2(E) (weights |e| (1, 1/3, 1/3)) and rejected
// when its remaining norm is below 1e-10 of its original norm; stops at N_E.
// Output layout: [N_E][3 cells_E], row k*cells_E + c.
// The fine solution x [n_cells][3] of system blockIdx.y into the pressure
// field p [3][n_cells] of its resident simulation.
struct SoaJob {
  const double* x;
  double* p;
  int n_cells;
};
__global__ void k_fine_to_soa(const SoaJob* __restrict__ jobs) {
  const SoaJob J = jobs[blockIdx.y];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J.n_cells; e += gridDim.x * blockDim.x) {
    J.p[e] = J.x[3 * e];
    J.p[(size_t)J.n_cells + e] = J.x[3 * e + 1];
    J.p[2 * (size_t)J.n_cells + e] = J.x[3 * e + 2];
  }
}

struct GsJob {
  int prob, E, NE, n_snap;
  const double* const* snaps;  // cell-major fine pressures
  double* Phi;                 // output for this subdomain
  int* got;                    // number of functions produced
  int have0;                   // functions already in Phi (0: start with the unit function)
};

__global__ void k_gram_schmidt(const FineDev* __restrict__ fds, const GsJob* __restrict__ jobs) {
  const GsJob J = jobs[blockIdx.x];
  const FineDev& f = fds[J.prob];
  const int cells = f.cx * f.cy, rows = 3 * cells;
  const int I = J.E % f.Sx, Jy = J.E / f.Sx;
  extern __shared__ double v[];  // rows
  __shared__ double red[32];
  const double w3[3] = {f.vol, f.vol / 3.0, f.vol / 3.0};
  int have = J.have0;
  for (int cand = have > 0 ? 0 : -1; cand < J.n_snap && have < J.NE; ++cand) {
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const int k = r / cells, c = r - k * cells;
      if (cand < 0) {
        v[r] = (k == 0) ? 1.0 : 0.0;
      } else {
        const int li = c % f.cx, lj = c / f.cx;
        const int ge = (Jy * f.cy + lj) * f.nx + I * f.cx + li;
        v[r] = J.snaps[cand][ge * 3 + k];
      }
    }
    __syncthreads();
    double n0 = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) n0 += w3[r / cells] * v[r] * v[r];
    n0 = sqrt(block_reduce_sum(n0, red));
    if (!(n0 > 0.0)) continue;
    for (int pass = 0; pass < 2; ++pass)
      for (int b = 0; b < have; ++b) {
        const double* ph = J.Phi + (size_t)b * rows;
        double d = 0.0;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) d += w3[r / cells] * ph[r] * v[r];
        d = block_reduce_sum(d, red);
        for (int r = threadIdx.x; r < rows; r += blockDim.x) v[r] -= d * ph[r];
        __syncthreads();
      }
    double nw = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) nw += w3[r / cells] * v[r] * v[r];
    nw = sqrt(block_reduce_sum(nw, red));
    if (!(nw >= 1e-10 * n0)) continue;
    double* out = J.Phi + (size_t)have * rows;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) out[r] = v[r] / nw;
    __syncthreads();
    ++have;
  }
  if (threadIdx.x == 0) *J.got = have;
}

// Projection (Section 4.4) of the fine component q (0: penalty terms, q >= 1:
// volume + consistency with Lambda^q) onto the local bases, for one
// assembled block (diagonal block of E, or coarse face (E-, E+)) or one
// subdomain right-hand side. Fine blocks: D [n_cells][9], O per interior fine
// face [9] (row e1, col e2), r [n_cells][3].
struct ProjJob {
  int prob, kind, E, Ep, q;  // kind 0: diagonal block E, 1: coarse face (E, Ep), 2: rhs of E
  int NE, NEp;
  const double* D;
  const double* O;
  const double* r;
  const double* PhiE;   // [NE][rows]
  const double* PhiEp;  // [NEp][rows]
  double* out;          // block [NE][NEp] or vector [NE]
};

__device__ __forceinline__ int gcell(const FineDev& f, int E, int c) {
  const int I = E % f.Sx, J = E / f.Sx, li = c % f.cx, lj = c / f.cx;
  return (J * f.cy + lj) * f.nx + I * f.cx + li;
}

__global__ void k_project(const FineDev* __restrict__ fds, const ProjJob* __restrict__ jobs) {
  const ProjJob P = jobs[blockIdx.x];
  const FineDev& f = fds[P.prob];
  const int cells = f.cx * f.cy, rows = 3 * cells;
  if (P.kind == 2) {
    for (int i = threadIdx.x; i < P.NE; i += blockDim.x) {
      double acc = 0.0;
      const double* ph = P.PhiE + (size_t)i * rows;
      for (int c = 0; c < cells; ++c) {
        const double* rr = P.r + (size_t)gcell(f, P.E, c) * 3;
        for (int k = 0; k < 3; ++k) acc += ph[k * cells + c] * rr[k];
      }
      P.out[i] = acc;
    }
    return;
  }
  const int NJ = P.kind == 0 ? P.NE : P.NEp;
  for (int idx = threadIdx.x; idx < P.NE * NJ; idx += blockDim.x) {
    const int i = idx / NJ, jj = idx - i * NJ;
    const double* pi = P.PhiE + (size_t)i * rows;
    double acc = 0.0;
    if (P.kind == 0) {
      const double* pj = P.PhiE + (size_t)jj * rows;
      for (int c = 0; c < cells; ++c) {
        const double* D = P.D + (size_t)gcell(f, P.E, c) * 9;
        for (int k = 0; k < 3; ++k) {
          const double t = D[k * 3] * pj[c] + D[k * 3 + 1] * pj[cells + c] + D[k * 3 + 2] * pj[2 * cells + c];
          acc += pi[k * cells + c] * t;
        }
      }
      // interior fine faces inside E: both orientations of the coupling block
      for (int c = 0; c < cells; ++c) {
        const int li = c % f.cx, lj = c / f.cx;
        const int e = gcell(f, P.E, c);
        for (int dir = 0; dir < 2; ++dir) {
          if (dir == 0 && li + 1 >= f.cx) continue;
          if (dir == 1 && lj + 1 >= f.cy) continue;
          const int c2 = dir == 0 ? c + 1 : c + f.cx;
          const int ei = e % f.nx, ej = e / f.nx;
          const int cf = dir == 0 ? ej * (f.nx - 1) + ei : f.ny * (f.nx - 1) + ej * f.nx + ei;
          const double* O = P.O + (size_t)cf * 9;
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
              const double o = O[k * 3 + l];
              acc += o * (pi[k * cells + c] * pj[l * cells + c2] + pi[l * cells + c2] * pj[k * cells + c]);
            }
        }
      }
    } else {
      const double* pj = P.PhiEp + (size_t)jj * rows;
      const bool xdir = (P.Ep == P.E + 1);
      const int n = xdir ? f.cy : f.cx;
      for (int t = 0; t < n; ++t) {
        // cell c1 in E on the interface, c2 its neighbour in Ep
        const int c1 = xdir ? t * f.cx + (f.cx - 1) : (f.cy - 1) * f.cx + t;
        const int c2 = xdir ? t * f.cx : t;
        const int e = gcell(f, P.E, c1);
        const int ei = e % f.nx, ej = e / f.nx;
        const int cf = xdir ? ej * (f.nx - 1) + ei : f.ny * (f.nx - 1) + ej * f.nx + ei;
        const double* O = P.O + (size_t)cf * 9;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) acc += pi[k * cells + c1] * O[k * 3 + l] * pj[l * cells + c2];
      }
    }
    P.out[(size_t)i * NJ + jj] = acc;
  }
}

// Rotated copy: Phi_E Q_E, Q_E^T B Q_E' per component, Q_E^T r_E.
struct RotJob {
  int kind, NE, NEp, rows, Q1;  // kind 0: basis of E, 1: block (E, E'), 2: rhs of E
  const double* QE;
  const double* QEp;
  const double* src;
  double* dst;
};

__global__ void k_rotate(const RotJob* __restrict__ jobs) {
  const RotJob R = jobs[blockIdx.x];
  if (R.kind == 0) {
    for (int idx = threadIdx.x; idx < R.NE * R.rows; idx += blockDim.x) {
      const int j = idx / R.rows, r = idx - j * R.rows;
      double acc = 0.0;
      for (int i = 0; i < R.NE; ++i) acc += R.src[(size_t)i * R.rows + r] * R.QE[i * R.NE + j];
      R.dst[idx] = acc;
    }
  } else if (R.kind == 1) {
    const int sz = R.NE * R.NEp;
    for (int q = 0; q < R.Q1; ++q) {
      const double* B = R.src + (size_t)q * sz;
      double* out = R.dst + (size_t)q * sz;
      for (int idx = threadIdx.x; idx < sz; idx += blockDim.x) {
        const int a = idx / R.NEp, b = idx - a * R.NEp;
        double acc = 0.0;
        for (int i = 0; i < R.NE; ++i) {
          double t = 0.0;
          for (int j = 0; j < R.NEp; ++j) t += B[i * R.NEp + j] * R.QEp[j * R.NEp + b];
          acc += R.QE[i * R.NE + a] * t;
        }
        out[idx] = acc;
      }
    }
  } else {
    for (int q = 0; q < R.Q1; ++q)
      for (int a = threadIdx.x; a < R.NE; a += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < R.NE; ++i) acc += R.QE[i * R.NE + a] * R.src[(size_t)q * R.NE + i];
        R.dst[(size_t)q * R.NE + a] = acc;
      }
  }
}

}  // namespace

// ----------------------------------------------------------------- host side
namespace {


// ---- greedy basis selection (Algorithm 2, step 2): training systems
// A_t = c + sum_q mu_tq b_q, rhs_t = e + sum_q mu_tq d_q of the current local
// bases, their reduced solutions, and the true error of Section 6 in the
// energy norm of the fine SWIP matrix at mu_bar.
struct GreedyDev {
  int n_sub, n_blocks, M, nx, ny, cells, n_int;
  const int* NE;            // [n_sub] current sizes
  const int* xoff;          // [n_sub + 1]
  const long long* aoff;    // [n_blocks + 1]
  const long long* phioff;  // [n_sub] (cap layout)
  const double* comp;       // block b at (M+1) aoff[b]: [M+1][size_b]
  const double* rhs;        // subdomain E at (M+1) xoff[E]: [M+1][N_E]
  const double* Phi;
  const double* mu;         // [n_tr][M]
  double* A;                // [n_tr][aoff[n_blocks]]
  double* b;                // [n_tr][N]
  const double* x;          // [n_tr][N]
  const double* const* snaps;  // [n_tr] cell-major fine pressures
  double* diff;             // [n_tr][3 n_cells]
  const double* Dbar;       // [n_cells][9]  fine matrix at mu_bar
  const double* Obar;       // [n_int][9]
  double* part;             // [n_tr][gridDim.x] energy partial sums
  long long a_tot;
  int N;
};

__global__ void k_greedy_assemble(const GreedyDev* __restrict__ gp) {
  const GreedyDev& G = *gp;
  const int t = blockIdx.y, bidx = blockIdx.x;
  const int Q = G.M + 1;
  __shared__ double w[kMaxM + 1];
  if (threadIdx.x == 0) w[0] = 1.0;
  if (threadIdx.x < G.M) w[1 + threadIdx.x] = G.mu[(size_t)t * G.M + threadIdx.x];
  __syncthreads();
  if (bidx < G.n_blocks) {
    const long long o = G.aoff[bidx];
    const int size = (int)(G.aoff[bidx + 1] - o);
    const double* c = G.comp + (size_t)Q * o;
    for (int i = threadIdx.x; i < size; i += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc = fma(w[q], c[(size_t)q * size + i], acc);
      G.A[(size_t)t * G.a_tot + o + i] = acc;
    }
  } else if (bidx < G.n_blocks + G.n_sub) {
    const int E = bidx - G.n_blocks, NE = G.NE[E], x0 = G.xoff[E];
    const double* c = G.rhs + (size_t)Q * x0;
    for (int i = threadIdx.x; i < NE; i += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc = fma(w[q], c[(size_t)q * NE + i], acc);
      G.b[(size_t)t * G.N + x0 + i] = acc;
    }
  }
}

// diff_t = (sum_i x_ti phi_i) - p_h(mu_t), cell-major, for every training t
__global__ void k_greedy_diff(const FineDev* __restrict__ fds, const GreedyDev* __restrict__ gp, int prob) {
  const GreedyDev& G = *gp;
  const FineDev& f = fds[prob];
  const int t = blockIdx.y, n_cells = G.nx * G.ny, cells = G.cells, rows = 3 * cells;
  const double* x = G.x + (size_t)t * G.N;
  const double* snap = G.snaps[t];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_cells; e += gridDim.x * blockDim.x) {
    const int i = e % G.nx, j = e / G.nx;
    const int E = (j / f.cy) * f.Sx + (i / f.cx);
    const int c = (j % f.cy) * f.cx + (i % f.cx);
    const double* Ph = G.Phi + G.phioff[E];
    const int NE = G.NE[E], x0 = G.xoff[E];
    for (int k = 0; k < 3; ++k) {
      double v = 0.0;
      for (int a = 0; a < NE; ++a) v = fma(Ph[(size_t)a * rows + k * cells + c], x[x0 + a], v);
      G.diff[((size_t)t * n_cells + e) * 3 + k] = v - snap[e * 3 + k];
    }
  }
}

// Partial sums of diff^T Kbar diff per CTA (fixed partition): the cell's
// diagonal block, and twice its coupling to the right and upper neighbours
// (the matrix is symmetric; each interior face block is stored once, row e1).
__global__ void k_greedy_energy(const GreedyDev* __restrict__ gp) {
  const GreedyDev& G = *gp;
  const int t = blockIdx.y, nx = G.nx, ny = G.ny, n_cells = nx * ny;
  const double* d = G.diff + (size_t)t * n_cells * 3;
  __shared__ double red[32];
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_cells; e += gridDim.x * blockDim.x) {
    const int i = e % nx, j = e / nx;
    const double* v = d + (size_t)e * 3;
    const double* D = G.Dbar + (size_t)e * 9;
    for (int k = 0; k < 3; ++k) acc += v[k] * (D[k * 3] * v[0] + D[k * 3 + 1] * v[1] + D[k * 3 + 2] * v[2]);
    if (i + 1 < nx) {
      const double* O = G.Obar + (size_t)(j * (nx - 1) + i) * 9;
      const double* u = d + (size_t)(e + 1) * 3;
      for (int k = 0; k < 3; ++k) acc += 2.0 * v[k] * (O[k * 3] * u[0] + O[k * 3 + 1] * u[1] + O[k * 3 + 2] * u[2]);
    }
    if (j + 1 < ny) {
      const double* O = G.Obar + (size_t)(ny * (nx - 1) + j * nx + i) * 9;
      const double* u = d + (size_t)(e + nx) * 3;
      for (int k = 0; k < 3; ++k) acc += 2.0 * v[k] * (O[k * 3] * u[0] + O[k * 3 + 1] * u[1] + O[k * 3 + 2] * u[2]);
    }
  }
  const double r = block_reduce_sum(acc, red);
  if (threadIdx.x == 0) G.part[(size_t)t * gridDim.x + blockIdx.x] = r;
}

// ---- compression (Algorithm 2, step 3): principal components, without
// centring, of the restrictions psi_1..psi_n of the snapshots the greedy
// selected, in L2(E), one CTA per subdomain:
//  1. X = Q R by two passes of modified Gram-Schmidt in L2(E) (Q
//     L2(E)-orthonormal; a column whose remaining norm is at most 1e-13 of its
//     own norm adds no row to R, k <= n rows in all);
//  2. the singular value decomposition of the k x n matrix R by one-sided
//     (Hestenes) Jacobi rotations of the k columns of R^T, accumulated in the
//     k x k matrix W: R^T W has orthogonal columns of norms sigma_j, so the
//     left singular vectors of X in L2(E) are Q W. Each warp rotates one pair
//     of columns; the pairs of a round (circle schedule) are disjoint;
//  3. energies l_j = sigma_j^2 in descending order, singular values at most
//     n eps_64 sigma_1 counted as 0, and the fewest r modes (r at most the
//     cap) whose discarded energy is at most eps_pca^2 of the total.
// Scratch per subdomain: Q [n][rows], Rt [n][n] (row b of R at Rt + b n),
// W [n][n] (column j at W + j n). Output: [r][rows], row k*cells + c.
constexpr int kMaxPcaSnap = 256;
struct PcaJob {
  int prob, E, n, cap;
  const double* const* snaps;  // cell-major fine pressures
  const int* idx;              // [n] selected snapshots
  double* Q;
  double* Rt;
  double* W;
  double* out;
  int* got;
  double eps;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_pca(const FineDev* __restrict__ fds, const PcaJob* __restrict__ jobs) {
  const PcaJob J = jobs[blockIdx.x];
  const FineDev& f = fds[J.prob];
  const int cells = f.cx * f.cy, rows = 3 * cells, n = J.n;
  const int I = J.E % f.Sx, Jy = J.E / f.Sx;
  extern __shared__ double v[];  // rows
  __shared__ double red[32];
  __shared__ double sig[kMaxPcaSnap];
  __shared__ int order[kMaxPcaSnap];
  __shared__ int s_rot, s_r;
  const double w3[3] = {f.vol, f.vol / 3.0, f.vol / 3.0};
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) J.Rt[i] = 0.0, J.W[i] = 0.0;
  __syncthreads();
  // 1. QR
  int k = 0;
  for (int j = 0; j < n; ++j) {
    const double* sn = J.snaps[J.idx[j]];
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const int kk = r / cells, c = r - kk * cells;
      const int ge = (Jy * f.cy + c / f.cx) * f.nx + I * f.cx + c % f.cx;
      v[r] = sn[ge * 3 + kk];
    }
    __syncthreads();
    double n0 = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) n0 += w3[r / cells] * v[r] * v[r];
    n0 = sqrt(block_reduce_sum(n0, red));
    if (!(n0 > 0.0)) continue;
    for (int pass = 0; pass < 2; ++pass)
      for (int b = 0; b < k; ++b) {
        const double* qb = J.Q + (size_t)b * rows;
        double d = 0.0;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) d += w3[r / cells] * qb[r] * v[r];
        d = block_reduce_sum(d, red);
        for (int r = threadIdx.x; r < rows; r += blockDim.x) v[r] -= d * qb[r];
        if (threadIdx.x == 0) J.Rt[(size_t)b * n + j] += d;
        __syncthreads();
      }
    double nw = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) nw += w3[r / cells] * v[r] * v[r];
    nw = sqrt(block_reduce_sum(nw, red));
    if (!(nw > 1e-13 * n0)) continue;
    double* qk = J.Q + (size_t)k * rows;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) qk[r] = v[r] / nw;
    if (threadIdx.x == 0) J.Rt[(size_t)k * n + j] = nw;
    __syncthreads();
    ++k;
  }
  // 2. one-sided Jacobi on the k columns of R^T (column b = row b of R)
  for (int i = threadIdx.x; i < k; i += blockDim.x) J.W[(size_t)i * n + i] = 1.0;
  __syncthreads();
  const int kp = k + (k & 1), n_warps = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int sweep = 0; sweep < 60 && k > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < kp - 1; ++round) {
      for (int pi = warp; pi < kp / 2; pi += n_warps) {
        int a, b;
        if (pi == 0) {
          a = 0, b = 1 + round;
        } else {
          a = 1 + (round + pi) % (kp - 1);
          b = 1 + (round - pi + (kp - 1)) % (kp - 1);
        }
        if (a >= k || b >= k) continue;
        double* ra = J.Rt + (size_t)a * n;
        double* rb = J.Rt + (size_t)b * n;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < n; i += 32) al += ra[i] * ra[i], be += rb[i] * rb[i], ga += ra[i] * rb[i];
        al = warp_sum(al), be = warp_sum(be), ga = warp_sum(ga);
        if (!(fabs(ga) > 1e-15 * sqrt(al * be))) continue;
        const double ze = (be - al) / (2.0 * ga);
        const double tt = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1.0 + ze * ze));
        const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        for (int i = lane; i < n; i += 32) {
          const double x = ra[i], y = rb[i];
          ra[i] = cs * x - sn * y, rb[i] = sn * x + cs * y;
        }
        double* wa = J.W + (size_t)a * n;
        double* wb = J.W + (size_t)b * n;
        for (int i = lane; i < k; i += 32) {
          const double x = wa[i], y = wb[i];
          wa[i] = cs * x - sn * y, wb[i] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  // 3. singular values, order and the number of modes
  for (int b = warp; b < k; b += n_warps) {
    const double* rb = J.Rt + (size_t)b * n;
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) s2 += rb[i] * rb[i];
    s2 = warp_sum(s2);
    if (lane == 0) sig[b] = sqrt(s2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < k; ++b) order[b] = b;
    for (int b = 1; b < k; ++b) {  // insertion sort, descending
      const int o = order[b];
      int c = b;
      while (c > 0 && sig[order[c - 1]] < sig[o]) order[c] = order[c - 1], --c;
      order[c] = o;
    }
    const double floor_s = k > 0 ? n * 2.220446049250313e-16 * sig[order[0]] : 0.0;
    double total = 0.0;
    for (int b = k - 1; b >= 0; --b) {
      const double s = sig[order[b]] > floor_s ? sig[order[b]] : 0.0;
      total += s * s;
    }
    // tail(r) = sum of the energies from position r on
    int r = 1;
    while (r < k && r < J.cap) {
      const double sr = sig[order[r]] > floor_s ? sig[order[r]] : 0.0;
      if (!(sr > 0.0)) break;
      double tail = 0.0;
      for (int b = k - 1; b >= r; --b) {
        const double s = sig[order[b]] > floor_s ? sig[order[b]] : 0.0;
        tail += s * s;
      }
      if (!(tail > J.eps * J.eps * total)) break;
      ++r;
    }
    s_r = k > 0 ? r : 0;
    *J.got = s_r;
  }
  __syncthreads();
  // modes Q W e_order[j]
  const int r = s_r;
  for (int j = 0; j < r; ++j) {
    const double* wj = J.W + (size_t)order[j] * n;
    double* o = J.out + (size_t)j * rows;
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
      double acc = 0.0;
      for (int b = 0; b < k; ++b) acc = fma(J.Q[(size_t)b * rows + row], wj[b], acc);
      o[row] = acc;
    }
  }
}

struct DevBuf {
  std::vector<void*> ptrs;
  ~DevBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return (T*)p;
  }
};

// Max over [0,1] of f_w'(s) by dense sampling of a central difference and a
// local golden-section refinement.
double max_fw_slope(double ew, double eo, int law) {
  auto fw = [&](double s) {
    const double lw = (law == 0 ? s * s : s) / ew;
    const double lo = (law == 0 ? (1 - s) * (1 - s) : (1 - s)) / eo;
    return lw / (lw + lo);
  };
  auto d = [&](double s) {
    const double h = 1e-7, a = std::max(0.0, s - h), b = std::min(1.0, s + h);
    return (fw(b) - fw(a)) / (b - a);
  };
  const int n = 200000;
  int best = 0;
  double bv = -1;
  for (int i = 0; i <= n; ++i) {
    const double v = d((double)i / n);
    if (v > bv) bv = v, best = i;
  }
  double lo = std::max(0, best - 1) / (double)n, hi = std::min(n, best + 1) / (double)n;
  const double gr = (std::sqrt(5.0) - 1) / 2;
  for (int it = 0; it < 80; ++it) {
    const double c = hi - gr * (hi - lo), e = lo + gr * (hi - lo);
    if (d(c) > d(e)) hi = e; else lo = c;
  }
  return std::max(bv, d(0.5 * (lo + hi)));
}

// Minimum-norm pseudo-inverse of a symmetric M x M matrix (cyclic Jacobi
// eigen-decomposition; eigenvalues below 1e-12 of the largest dropped).
void sym_pinv(int M, const std::vector<double>& G, std::vector<double>& out) {
  std::vector<double> A = G, V(M * M, 0.0);
  for (int i = 0; i < M; ++i) V[i * M + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < M; ++p)
      for (int q = p + 1; q < M; ++q) off += A[p * M + q] * A[p * M + q];
    if (off < 1e-300) break;
    for (int p = 0; p < M; ++p)
      for (int q = p + 1; q < M; ++q) {
        const double apq = A[p * M + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (A[q * M + q] - A[p * M + p]) / (2 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1));
        const double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < M; ++k) {
          const double akp = A[k * M + p], akq = A[k * M + q];
          A[k * M + p] = c * akp - s * akq;
          A[k * M + q] = s * akp + c * akq;
        }
        for (int k = 0; k < M; ++k) {
          const double apk = A[p * M + k], aqk = A[q * M + k];
          A[p * M + k] = c * apk - s * aqk;
          A[q * M + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < M; ++k) {
          const double vkp = V[k * M + p], vkq = V[k * M + q];
          V[k * M + p] = c * vkp - s * vkq;
          V[k * M + q] = s * vkp + c * vkq;
        }
      }
  }
  double wmax = 0;
  for (int i = 0; i < M; ++i) wmax = std::max(wmax, A[i * M + i]);
  out.assign(M * M, 0.0);
  for (int k = 0; k < M; ++k) {
    const double w = A[k * M + k];
    if (!(w > 1e-12 * wmax)) continue;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) out[i * M + j] += V[i * M + k] * V[j * M + k] / w;
  }
}

}  // namespace

// Fine-system solves through the online solver: one "simulation" per system
// with one-cell blocks.
struct FineSolver {
  int nx, ny;
  int n_cells, n_int;
  std::vector<SimDev> sims;
  SimDev* d_sims = nullptr;
  int* d_active = nullptr;
  DevBuf* buf;
  // shared metadata
  int *NE = nullptr, *xoff = nullptr;
  long long *aoff = nullptr, *loff = nullptr, *ioff = nullptr;

  bool init(DevBuf& b, int nx_, int ny_, int count, cudaStream_t st) {
    buf = &b;
    nx = nx_; ny = ny_;
    n_cells = nx * ny;
    n_int = ny * (nx - 1) + (ny - 1) * nx;
    const int n_blocks = n_cells + n_int;
    std::vector<int> ne(n_cells, 3), xo(n_cells + 1);
    for (int e = 0; e <= n_cells; ++e) xo[e] = 3 * e;
    std::vector<long long> ao(n_blocks + 1), lo(n_cells + 1), io(n_cells + 1);
    for (int k = 0; k <= n_blocks; ++k) ao[k] = 9LL * k;
    lo[0] = 0; io[0] = 0;
    for (int k = 0; k < n_cells; ++k) {
      const int jl = jlo_of(k, nx);
      lo[k + 1] = lo[k] + 3LL * (xo[k + 1] - xo[jl]);
      io[k + 1] = io[k] + 9;
    }
    NE = b.get<int>(n_cells); xoff = b.get<int>(n_cells + 1);
    aoff = b.get<long long>(n_blocks + 1); loff = b.get<long long>(n_cells + 1);
    ioff = b.get<long long>(n_cells + 1);
    if (!NE || !xoff || !aoff || !loff || !ioff) return false;
    cudaMemcpyAsync(NE, ne.data(), 4 * ne.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(xoff, xo.data(), 4 * xo.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(aoff, ao.data(), 8 * ao.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(loff, lo.data(), 8 * lo.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ioff, io.data(), 8 * io.size(), cudaMemcpyHostToDevice, st);
    sims.resize(count);
    for (int s = 0; s < count; ++s) {
      SimDev d{};
      d.nx = nx; d.ny = ny; d.Sx = nx; d.Sy = ny; d.n_sub = n_cells; d.n_cf = n_int;
      d.n_blocks = n_blocks; d.N = 3 * n_cells; d.max_NE = 3;
      d.NE = NE; d.xoff = xoff; d.aoff = aoff; d.loff = loff; d.ioff = ioff;
      d.A = b.get<double>(9 * (size_t)n_blocks);
      d.b = b.get<double>(3 * (size_t)n_cells);
      d.x = b.get<double>(3 * (size_t)n_cells);
      d.y = b.get<double>(6 * (size_t)n_cells);
      d.rv = b.get<double>(3 * (size_t)n_cells);
      d.dv = b.get<double>(3 * (size_t)n_cells);
      d.L = b.get<double>((size_t)lo[n_cells]);
      d.Linv = b.get<double>(9 * (size_t)n_cells);
      d.status = b.get<int>(1);
      if (!d.A || !d.b || !d.x || !d.y || !d.rv || !d.dv || !d.L || !d.Linv || !d.status) return false;
      cudaMemsetAsync(d.status, 0, 4, st);
      sims[s] = d;
    }
    d_sims = b.get<SimDev>(count);
    d_active = b.get<int>(count);
    if (!d_sims || !d_active) return false;
    std::vector<int> act(count);
    for (int s = 0; s < count; ++s) act[s] = s;
    cudaMemcpyAsync(d_sims, sims.data(), sizeof(SimDev) * count, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_active, act.data(), 4 * count, cudaMemcpyHostToDevice, st);
    return cudaStreamSynchronize(st) == cudaSuccess;
  }
};

}  // namespace lrbms

using namespace lrbms;

// Defined in lrbms_api.cu.
extern "C" cudaStream_t lrbms_internal_stream(lrbms_ctx* ctx);
extern "C" int lrbms_internal_fail(lrbms_ctx* ctx, int code, const char* msg);
extern "C" int lrbms_internal_sim(lrbms_ctx* ctx, int id, lrbms::SimDev* out);
extern "C" lrbms::SimDev* lrbms_internal_dsims(lrbms_ctx* ctx);
extern "C" cudaStream_t lrbms_internal_admit_stream(lrbms_ctx* ctx);
extern "C" bool lrbms_internal_in_last_batch(lrbms_ctx* ctx, int id);
extern "C" void lrbms_internal_count(lrbms_ctx* ctx, long long n);
extern "C" int lrbms_internal_share_factor(lrbms_ctx* ctx, int src, int dst);

#define BCK(call)                                                              \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return lrbms_internal_fail(ctx, LRBMS_E_CUDA, (std::string(#call) + ": " + \
                                                     cudaGetErrorString(e_)).c_str()); \
  } while (0)


// Algorithm 2, step 2 for one problem: starting from the unit function of
// every subdomain, solve the reduced system of every training parameter mu_t
// (FP64 block Cholesky, batched), measure the true error of Section 6,
// ||p_N(mu_t) - p_h(mu_t)|| in the energy norm of the fine SWIP matrix at
// mu_bar (the oracle's reading), and extend every subdomain below its cap by
// the Gram-Schmidt orthonormalised restriction of the worst-approximated
// snapshot, until the worst error is at most the tolerance, every cap is
// reached or no subdomain grows. NE: caps on entry, sizes on return; Phi and
// phioff: the compacted bases.
template <typename RunSystems>
static int greedy_bases(lrbms_ctx* ctx, DevBuf& B, cudaStream_t st, const FineDev* d_fd, const FineDev& f, int p,
                        const lrbms_build_opts& O, const double* dmu, const double* const* dsnap, std::vector<int>& NE,
                        double*& Phi, std::vector<long long>& phioff, const std::vector<int>& cfm,
                        const std::vector<int>& cfp, int n_int, RunSystems& run_systems) {
  const int n_sub = f.Sx * f.Sy, n_cf = (int)cfm.size(), n_blocks = n_sub + n_cf, M = O.M, Q = M + 1;
  const int cells = f.cx * f.cy, rows = 3 * cells, n_cells = f.n_cells, n_tr = O.n_snap;
  const std::vector<int> cap = NE;
  // capacities of the growing system (caps)
  long long a_cap = 0;
  int N_cap = 0;
  for (int E = 0; E < n_sub; ++E) a_cap += (long long)cap[E] * cap[E], N_cap += cap[E];
  for (int c = 0; c < n_cf; ++c) a_cap += (long long)cap[cfm[c]] * cap[cfp[c]];
  std::vector<int> xcap(n_sub + 1, 0);
  for (int E = 0; E < n_sub; ++E) xcap[E + 1] = xcap[E] + cap[E];
  std::vector<long long> lcap(n_sub + 1), icap(n_sub + 1);
  solve_offsets(n_sub, f.Sx, cap.data(), xcap.data(), lcap.data(), icap.data());
  // fine component blocks (Section 4.4) and the energy-norm matrix at mu_bar
  std::vector<double*> D(Q), Ob(Q), R(Q);
  std::vector<SysJob> jobs(Q + 1);
  for (int q = 0; q < Q; ++q) {
    D[q] = B.get<double>(9 * (size_t)n_cells);
    Ob[q] = B.get<double>(9 * (size_t)std::max(n_int, 1));
    R[q] = B.get<double>(3 * (size_t)n_cells);
    if (!D[q] || !Ob[q] || !R[q]) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "greedy component blocks");
    jobs[q] = q == 0 ? SysJob{p, 2, 1, 0, nullptr, D[q], Ob[q], R[q]} : SysJob{p, 2, 2, q - 1, nullptr, D[q], Ob[q], R[q]};
  }
  double* dmubar = B.get<double>(M);
  double* Dbar = B.get<double>(9 * (size_t)n_cells);
  double* Obar = B.get<double>(9 * (size_t)std::max(n_int, 1));
  double* rbar = B.get<double>(3 * (size_t)n_cells);
  if (!dmubar || !Dbar || !Obar || !rbar) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "greedy energy matrix");
  std::vector<double> mubar(M, 1.0 / M);
  if (O.mu_bar) BCK(cudaMemcpy(mubar.data(), O.mu_bar, 8 * (size_t)M, cudaMemcpyDefault));
  BCK(cudaMemcpyAsync(dmubar, mubar.data(), 8 * (size_t)M, cudaMemcpyHostToDevice, st));
  jobs[Q] = SysJob{p, 1, 3, 0, dmubar, Dbar, Obar, rbar};
  if (int rc = run_systems(jobs)) return lrbms_internal_fail(ctx, rc, "greedy assembly");
  // buffers
  double* comp = B.get<double>((size_t)Q * a_cap);
  double* rhs = B.get<double>((size_t)Q * N_cap);
  double* A = B.get<double>((size_t)n_tr * a_cap);
  double* bv = B.get<double>((size_t)n_tr * N_cap);
  double* xv = B.get<double>((size_t)n_tr * N_cap);
  double* yv = B.get<double>((size_t)n_tr * 2 * N_cap);
  double* rv = B.get<double>((size_t)n_tr * N_cap);
  double* dv = B.get<double>((size_t)n_tr * N_cap);
  double* Lv = B.get<double>((size_t)n_tr * lcap[n_sub]);
  double* Li = B.get<double>((size_t)n_tr * icap[n_sub]);
  int* stv = B.get<int>(n_tr);
  double* diff = B.get<double>((size_t)n_tr * 3 * n_cells);
  int* dNE = B.get<int>(n_sub);
  int* dxoff = B.get<int>(n_sub + 1);
  long long* daoff = B.get<long long>(n_blocks + 1);
  long long* dloff = B.get<long long>(n_sub + 1);
  long long* dioff = B.get<long long>(n_sub + 1);
  long long* dphioff = B.get<long long>(n_sub);
  unsigned long long* dsched = B.get<unsigned long long>(sched_words(n_sub, f.Sx));
  int* dgot = B.get<int>(n_sub);
  int* dact = B.get<int>(n_tr);
  SimDev* dsims = B.get<SimDev>(n_tr);
  GreedyDev* dG = B.get<GreedyDev>(1);
  constexpr int kEnergyBlocks = 64;
  double* dpart = B.get<double>((size_t)n_tr * kEnergyBlocks);
  GsJob* dgs = B.get<GsJob>(n_sub);
  if (!comp || !rhs || !A || !bv || !xv || !yv || !rv || !dv || !Lv || !Li || !stv || !diff || !dNE || !dxoff ||
      !daoff || !dloff || !dioff || !dphioff || !dsched || !dgot || !dact || !dsims || !dG || !dpart || !dgs)
    return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "greedy buffers");
  BCK(cudaMemcpyAsync(dphioff, phioff.data(), 8 * (size_t)n_sub, cudaMemcpyHostToDevice, st));
  {
    std::vector<int> act(n_tr);
    for (int t = 0; t < n_tr; ++t) act[t] = t;
    BCK(cudaMemcpyAsync(dact, act.data(), 4 * (size_t)n_tr, cudaMemcpyHostToDevice, st));
  }
  // unit functions
  std::vector<int> cur(n_sub, 0);
  {
    std::vector<GsJob> gj(n_sub);
    for (int E = 0; E < n_sub; ++E) gj[E] = GsJob{p, E, 1, 0, dsnap, Phi + phioff[E], dgot + E, 0};
    BCK(cudaMemcpyAsync(dgs, gj.data(), sizeof(GsJob) * n_sub, cudaMemcpyHostToDevice, st));
    k_gram_schmidt<<<(unsigned)n_sub, 256, 8 * (size_t)rows, st>>>(d_fd, dgs);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(cur.data(), dgot, 4 * (size_t)n_sub, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
  }
  std::vector<double> hist;
  std::vector<int> chosen;  // the snapshot set Psi of step 2(d)
  std::vector<double> part((size_t)n_tr * kEnergyBlocks);
  for (int it = 0; it < 200; ++it) {
    // layout of the current system
    std::vector<int> xoff(n_sub + 1, 0);
    for (int E = 0; E < n_sub; ++E) xoff[E + 1] = xoff[E] + cur[E];
    std::vector<long long> aoff(n_blocks + 1, 0);
    for (int E = 0; E < n_sub; ++E) aoff[E + 1] = aoff[E] + (long long)cur[E] * cur[E];
    for (int c = 0; c < n_cf; ++c) aoff[n_sub + c + 1] = aoff[n_sub + c] + (long long)cur[cfm[c]] * cur[cfp[c]];
    std::vector<long long> loff(n_sub + 1), ioff(n_sub + 1);
    solve_offsets(n_sub, f.Sx, cur.data(), xoff.data(), loff.data(), ioff.data());
    int panel_words = 0, max_w = 0;
    solve_panel_sizes(n_sub, f.Sx, cur.data(), xoff.data(), &panel_words, &max_w);
    const int N = xoff[n_sub];
    if (solve_smem_bytes(n_sub, panel_words, max_w, N, sizeof(double)) > kMaxSolveSmem)
      return lrbms_internal_fail(ctx, LRBMS_E_FORMAT, "greedy: reduced system too large for the on-chip solve");
    BCK(cudaMemcpyAsync(dNE, cur.data(), 4 * (size_t)n_sub, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(dxoff, xoff.data(), 4 * (size_t)(n_sub + 1), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(daoff, aoff.data(), 8 * (size_t)(n_blocks + 1), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(dloff, loff.data(), 8 * (size_t)(n_sub + 1), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(dioff, ioff.data(), 8 * (size_t)(n_sub + 1), cudaMemcpyHostToDevice, st));
    // components of the current bases (Section 4.4)
    std::vector<ProjJob> pj;
    for (int q = 0; q < Q; ++q) {
      for (int E = 0; E < n_sub; ++E) {
        const double* PE = Phi + phioff[E];
        const size_t sz = (size_t)cur[E] * cur[E];
        pj.push_back(ProjJob{p, 0, E, E, q, cur[E], cur[E], D[q], Ob[q], R[q], PE, PE,
                             comp + (size_t)Q * aoff[E] + q * sz});
        pj.push_back(ProjJob{p, 2, E, E, q, cur[E], 0, D[q], Ob[q], R[q], PE, PE,
                             rhs + (size_t)Q * xoff[E] + (size_t)q * cur[E]});
      }
      for (int c = 0; c < n_cf; ++c) {
        const int Em = cfm[c], Ep = cfp[c];
        const size_t sz = (size_t)cur[Em] * cur[Ep];
        pj.push_back(ProjJob{p, 1, Em, Ep, q, cur[Em], cur[Ep], D[q], Ob[q], R[q], Phi + phioff[Em],
                             Phi + phioff[Ep], comp + (size_t)Q * aoff[n_sub + c] + q * sz});
      }
    }
    ProjJob* dpj = B.get<ProjJob>(pj.size());
    if (!dpj) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "greedy projection jobs");
    BCK(cudaMemcpyAsync(dpj, pj.data(), sizeof(ProjJob) * pj.size(), cudaMemcpyHostToDevice, st));
    k_project<<<(unsigned)pj.size(), 256, 0, st>>>(d_fd, dpj);
    BCK(cudaGetLastError());
    // training systems and their solves
    GreedyDev G{n_sub, n_blocks, M, f.nx, f.ny, cells, n_int, dNE, dxoff, daoff, dphioff, comp, rhs, Phi, dmu,
                A, bv, xv, dsnap, diff, Dbar, Obar, dpart, aoff[n_blocks], N};
    BCK(cudaMemcpyAsync(dG, &G, sizeof(G), cudaMemcpyHostToDevice, st));
    k_greedy_assemble<<<dim3(n_blocks + n_sub, n_tr), 128, 0, st>>>(dG);
    BCK(cudaGetLastError());
    std::vector<SimDev> sims(n_tr);
    for (int t = 0; t < n_tr; ++t) {
      SimDev d{};
      d.Sx = f.Sx; d.Sy = f.Sy; d.n_sub = n_sub; d.n_cf = n_cf; d.n_blocks = n_blocks; d.N = N;
      d.panel_words = panel_words; d.max_w = max_w;
      d.NE = dNE; d.xoff = dxoff; d.aoff = daoff; d.loff = dloff; d.ioff = dioff; d.sched = dsched;
      d.A = A + (size_t)t * aoff[n_blocks]; d.b = bv + (size_t)t * N; d.x = xv + (size_t)t * N;
      d.y = yv + (size_t)t * 2 * N; d.rv = rv + (size_t)t * N; d.dv = dv + (size_t)t * N;
      d.L = Lv + (size_t)t * loff[n_sub]; d.Linv = Li + (size_t)t * ioff[n_sub]; d.status = stv + t;
      sims[t] = d;
    }
    BCK(cudaMemsetAsync(stv, 0, 4 * (size_t)n_tr, st));
    BCK(cudaMemcpyAsync(dsims, sims.data(), sizeof(SimDev) * n_tr, cudaMemcpyHostToDevice, st));
    launch_sched(dsims, st);
    const SolveShape sh{n_sub, panel_words, max_w, N};
    BCK(prepare_chol_solve(0, sh));
    BCK(launch_chol_solve(dsims, dact, n_tr, 0, 1, sh, st));
    std::vector<int> sst(n_tr);
    BCK(cudaMemcpyAsync(sst.data(), stv, 4 * (size_t)n_tr, cudaMemcpyDeviceToHost, st));
    // error fields and energy norms
    k_greedy_diff<<<dim3(std::min(152, (n_cells + 255) / 256), n_tr), 256, 0, st>>>(d_fd, dG, p);
    k_greedy_energy<<<dim3(kEnergyBlocks, n_tr), 256, 0, st>>>(dG);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(part.data(), dpart, 8 * part.size(), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    for (int t = 0; t < n_tr; ++t)
      if (sst[t]) return lrbms_internal_fail(ctx, LRBMS_E_NOT_SPD, "greedy: a training system was not positive definite");
    int kmax = 0;
    double emax = -1.0;
    for (int t = 0; t < n_tr; ++t) {
      double e2 = 0.0;
      for (int b = 0; b < kEnergyBlocks; ++b) e2 += part[(size_t)t * kEnergyBlocks + b];
      const double e = std::sqrt(std::max(e2, 0.0));
      if (e > emax) emax = e, kmax = t;
    }
    hist.push_back(emax);
    int tot = 0, tot_cap = 0;
    for (int E = 0; E < n_sub; ++E) tot += cur[E], tot_cap += cap[E];
    if (emax <= O.greedy_tol || tot >= tot_cap) break;
    chosen.push_back(kmax);
    // extend every subdomain below its cap by the worst-approximated snapshot
    std::vector<GsJob> gj;
    for (int E = 0; E < n_sub; ++E)
      if (cur[E] < cap[E]) gj.push_back(GsJob{p, E, cur[E] + 1, 1, dsnap + kmax, Phi + phioff[E], dgot + E, cur[E]});
    BCK(cudaMemcpyAsync(dgot, cur.data(), 4 * (size_t)n_sub, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(dgs, gj.data(), sizeof(GsJob) * gj.size(), cudaMemcpyHostToDevice, st));
    k_gram_schmidt<<<(unsigned)gj.size(), 256, 8 * (size_t)rows, st>>>(d_fd, dgs);
    BCK(cudaGetLastError());
    std::vector<int> got(n_sub);
    BCK(cudaMemcpyAsync(got.data(), dgot, 4 * (size_t)n_sub, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    bool grew = false;
    for (int E = 0; E < n_sub; ++E) grew |= got[E] > cur[E];
    cur = got;
    if (!grew) break;
  }
  if (O.pca_eps > 0.0 && !chosen.empty()) {
    // step 3: the bases become the principal components of the selected
    // snapshots' restrictions (written over the cap layout of Phi)
    const int n = (int)chosen.size();
    if (n > kMaxPcaSnap) return lrbms_internal_fail(ctx, LRBMS_E_FORMAT, "compression: more than 256 snapshots");
    double* Qs = B.get<double>((size_t)n_sub * n * rows);
    double* Rts = B.get<double>((size_t)n_sub * n * n);
    double* Ws = B.get<double>((size_t)n_sub * n * n);
    int* didx = B.get<int>(n);
    PcaJob* dpj = B.get<PcaJob>(n_sub);
    if (!Qs || !Rts || !Ws || !didx || !dpj) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "compression buffers");
    std::vector<PcaJob> jobs_pca(n_sub);
    for (int E = 0; E < n_sub; ++E)
      jobs_pca[E] = PcaJob{p, E, n, cap[E], dsnap, didx, Qs + (size_t)E * n * rows, Rts + (size_t)E * n * n,
                           Ws + (size_t)E * n * n, Phi + phioff[E], dgot + E, O.pca_eps};
    BCK(cudaMemcpyAsync(didx, chosen.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(dpj, jobs_pca.data(), sizeof(PcaJob) * n_sub, cudaMemcpyHostToDevice, st));
    k_pca<<<(unsigned)n_sub, 256, 8 * (size_t)rows, st>>>(d_fd, dpj);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(cur.data(), dgot, 4 * (size_t)n_sub, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    for (int E = 0; E < n_sub; ++E)
      if (cur[E] < 1) return lrbms_internal_fail(ctx, LRBMS_E_FORMAT, "compression: a subdomain kept no mode");
  }
  if (O.history) {
    const int nh = std::min((int)hist.size(), O.max_history);
    BCK(cudaMemcpy(O.history, hist.data(), 8 * (size_t)nh, cudaMemcpyDefault));
  }
  if (O.n_history) *O.n_history = (int)hist.size();
  // compact the bases to their sizes
  std::vector<long long> off2(n_sub + 1, 0);
  for (int E = 0; E < n_sub; ++E) off2[E + 1] = off2[E] + (long long)cur[E] * rows;
  double* P2 = B.get<double>((size_t)off2[n_sub]);
  if (!P2) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "basis buffers");
  for (int E = 0; E < n_sub; ++E)
    BCK(cudaMemcpyAsync(P2 + off2[E], Phi + phioff[E], 8 * (size_t)(off2[E + 1] - off2[E]), cudaMemcpyDeviceToDevice,
                        st));
  BCK(cudaStreamSynchronize(st));
  Phi = P2;
  phioff = off2;
  NE = cur;
  return LRBMS_OK;
}

extern "C" int lrbms_offline_build(lrbms_ctx* ctx, int n_prob, const lrbms_problem* probs,
                                   const lrbms_build_opts* opts, int n_copies,
                                   const double* const* rot, int* sim_ids, int* achieved) {
  if (!ctx || n_prob < 1 || !probs || !opts || n_copies < 1 || !sim_ids)
    return lrbms_internal_fail(ctx, LRBMS_E_ARG, "bad arguments");
  cudaStream_t st = lrbms_internal_stream(ctx);
  const lrbms_problem& p0 = probs[0];
  const int nx = p0.nx, ny = p0.ny, Sx = p0.Sx, Sy = p0.Sy;
  for (int p = 0; p < n_prob; ++p) {
    const lrbms_problem& P = probs[p];
    const lrbms_build_opts& O = opts[p];
    if (P.nx != nx || P.ny != ny || P.Sx != Sx || P.Sy != Sy)
      return lrbms_internal_fail(ctx, LRBMS_E_ARG, "all problems of one build must share the grids");
    if (nx < 2 || ny < 2 || nx % Sx || ny % Sy)
      return lrbms_internal_fail(ctx, LRBMS_E_ARG, "grid must be at least 2x2 and match the subdomains");
    if (O.M < 3 || O.M > kMaxM || O.n_snap < 0 || (O.n_snap && !O.mu) || !O.N_E || (O.n_steps_T < 1 && !O.prof_s) ||
        !(O.c_pen > 0))
      return lrbms_internal_fail(ctx, LRBMS_E_ARG, "bad build options");
  }
  const int n_cells = nx * ny, cx = nx / Sx, cy = ny / Sy, cells = cx * cy, n_sub = Sx * Sy;
  const int nxf = (nx + 1) * ny, n_faces = nxf + nx * (ny + 1), nb = 2 * nx + 2 * ny;
  const int n_int = ny * (nx - 1) + (ny - 1) * nx;
  const int n_cf = Sy * (Sx - 1) + (Sy - 1) * Sx;
  DevBuf B;

  // ---- problem data on the device
  std::vector<FineDev> fd(n_prob);
  for (int p = 0; p < n_prob; ++p) {
    const lrbms_problem& P = probs[p];
    FineDev& f = fd[p];
    f.nx = nx; f.ny = ny; f.Sx = Sx; f.Sy = Sy; f.cx = cx; f.cy = cy; f.n_cells = n_cells;
    f.nxf = nxf; f.n_faces = n_faces; f.nb = nb; f.M = opts[p].M; f.relperm = P.relperm;
    f.swapped = P.mean_weights; f.hx = P.Lx / nx; f.hy = P.Ly / ny; f.vol = f.hx * f.hy;
    f.c_pen = opts[p].c_pen; f.inv_eta_w = 1.0 / P.eta_w; f.inv_eta_o = 1.0 / P.eta_o;
    f.lam0 = f.inv_eta_o; f.lam1 = f.inv_eta_w;
    double* perm = B.get<double>(n_cells); double* poro = B.get<double>(n_cells);
    double* s0 = B.get<double>(n_cells);
    int8_t* bct = B.get<int8_t>(nb);
    double* pD = B.get<double>(nb); double* vN = B.get<double>(nb); double* sD = B.get<double>(nb);
    uint8_t* pidx = B.get<uint8_t>(n_cells);
    if (!perm || !poro || !s0 || !bct || !pD || !vN || !sD || !pidx)
      return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the offline build");
    BCK(cudaMemcpyAsync(perm, P.perm, 8 * (size_t)n_cells, cudaMemcpyDefault, st));
    BCK(cudaMemcpyAsync(poro, P.poro, 8 * (size_t)n_cells, cudaMemcpyDefault, st));
    BCK(cudaMemcpyAsync(s0, P.s0, 8 * (size_t)n_cells, cudaMemcpyDefault, st));
    BCK(cudaMemcpyAsync(bct, P.bc_type, nb, cudaMemcpyDefault, st));
    BCK(cudaMemcpyAsync(pD, P.p_D, 8 * (size_t)nb, cudaMemcpyDefault, st));
    BCK(cudaMemcpyAsync(vN, P.v_N, 8 * (size_t)nb, cudaMemcpyDefault, st));
    BCK(cudaMemcpyAsync(sD, P.s_D, 8 * (size_t)nb, cudaMemcpyDefault, st));
    f.perm = perm; f.poro = poro; f.s0 = s0; f.bc_type = bct; f.p_D = pD; f.v_N = vN; f.s_D = sD;
    f.prof_idx = pidx;
    f.prof = nullptr;
    if (opts[p].prof_s) {  // saturation snapshots: lambda(s_q) after the FineDev table is on the device
      double* pr = B.get<double>((size_t)f.M * n_cells);
      if (!pr) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the profiles");
      BCK(cudaMemcpyAsync(pr, opts[p].prof_s, 8 * (size_t)f.M * n_cells, cudaMemcpyDefault, st));
      f.prof = pr;
    }
  }
  FineDev* d_fd = B.get<FineDev>(n_prob);
  if (!d_fd) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the offline build");
  BCK(cudaMemcpyAsync(d_fd, fd.data(), sizeof(FineDev) * n_prob, cudaMemcpyHostToDevice, st));
  for (int p = 0; p < n_prob; ++p)
    if (fd[p].prof) {
      k_sat_profiles<<<152, 256, 0, st>>>(d_fd, p, const_cast<double*>(fd[p].prof));
      BCK(cudaGetLastError());
    }

  auto run_systems = [&](std::vector<SysJob>& jobs) -> int {
    SysJob* dj = B.get<SysJob>(jobs.size());
    if (!dj) return LRBMS_E_BUDGET;
    if (cudaMemcpyAsync(dj, jobs.data(), sizeof(SysJob) * jobs.size(), cudaMemcpyHostToDevice, st)) return LRBMS_E_CUDA;
    const int n = std::max(n_cells, n_faces);
    k_fine_system<<<dim3((n + 127) / 128, (unsigned)jobs.size()), 128, 0, st>>>(d_fd, dj);
    return cudaGetLastError() == cudaSuccess ? 0 : LRBMS_E_CUDA;
  };

  // ---- step 1(a): initial pressure with lambda(s0)
  FineSolver init;
  if (!init.init(B, nx, ny, n_prob, st))
    return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the initial fine solves");
  {
    std::vector<SysJob> jobs(n_prob);
    for (int p = 0; p < n_prob; ++p)
      jobs[p] = SysJob{p, 0, 3, 0, nullptr, init.sims[p].A, init.sims[p].A + 9 * (size_t)n_cells,
                       init.sims[p].b};
    if (int rc = run_systems(jobs)) return lrbms_internal_fail(ctx, rc, "fine assembly");
    BCK(launch_fine_solve(init.d_sims, init.d_active, n_prob, st));
  }
  // ---- velocity, time-of-flight and profiles (steps 1(b), 1(c))
  std::vector<double*> hF(n_prob), hta(n_prob), htb(n_prob);
  std::vector<const double*> hx(n_prob);
  for (int p = 0; p < n_prob; ++p) {
    hF[p] = B.get<double>(n_faces); hta[p] = B.get<double>(n_cells); htb[p] = B.get<double>(n_cells);
    if (!hF[p] || !hta[p] || !htb[p]) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "tof buffers");
    hx[p] = init.sims[p].x;
    BCK(cudaMemsetAsync(hta[p], 0, 8 * (size_t)n_cells, st));
  }
  double** dF = B.get<double*>(n_prob); double** dta = B.get<double*>(n_prob);
  double** dtb = B.get<double*>(n_prob); const double** dx = (const double**)B.get<double*>(n_prob);
  unsigned long long* dcfl = B.get<unsigned long long>(n_prob);
  int* dchg = B.get<int>(1);
  unsigned int* dhist = B.get<unsigned int>(n_prob * (kMaxM + 1));
  double* dT = B.get<double>(n_prob);
  if (!dF || !dta || !dtb || !dx || !dcfl || !dchg || !dhist || !dT)
    return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "tof buffers");
  BCK(cudaMemcpyAsync(dF, hF.data(), sizeof(double*) * n_prob, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(dta, hta.data(), sizeof(double*) * n_prob, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(dtb, htb.data(), sizeof(double*) * n_prob, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(dx, hx.data(), sizeof(double*) * n_prob, cudaMemcpyHostToDevice, st));
  {
    std::vector<unsigned long long> inf(n_prob);
    const double big = DBL_MAX;
    for (auto& v : inf) std::memcpy(&v, &big, 8);
    BCK(cudaMemcpyAsync(dcfl, inf.data(), 8 * (size_t)n_prob, cudaMemcpyHostToDevice, st));
  }
  BCK(cudaMemsetAsync(dhist, 0, 4 * (size_t)n_prob * (kMaxM + 1), st));
  k_fine_flux<<<dim3((n_faces + 255) / 256, n_prob), 256, 0, st>>>(d_fd, dx, dF);
  k_fine_cfl<<<dim3((n_cells + 255) / 256, n_prob), 256, 0, st>>>(d_fd, dF, dcfl);
  {
    const int max_sweeps = 16 * (nx + ny) + 64;
    int sweep = 0;
    for (; sweep < max_sweeps; sweep += 2) {
      BCK(cudaMemsetAsync(dchg, 0, 4, st));
      k_tof_sweep<<<dim3((n_cells + 255) / 256, n_prob), 256, 0, st>>>(d_fd, dF, dta, dtb, dchg);
      k_tof_sweep<<<dim3((n_cells + 255) / 256, n_prob), 256, 0, st>>>(d_fd, dF, dtb, dta, dchg);
      if (sweep % 32 == 30 || sweep + 2 >= max_sweeps) {
        int chg = 1;
        BCK(cudaMemcpyAsync(&chg, dchg, 4, cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        if (!chg) break;
      }
    }
  }
  std::vector<unsigned long long> cflbits(n_prob);
  BCK(cudaMemcpyAsync(cflbits.data(), dcfl, 8 * (size_t)n_prob, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  std::vector<double> T(n_prob), Lf(n_prob);
  for (int p = 0; p < n_prob; ++p) {
    double m;
    std::memcpy(&m, &cflbits[p], 8);
    Lf[p] = max_fw_slope(probs[p].eta_w, probs[p].eta_o, probs[p].relperm);
    const double dt0 = probs[p].cfl * m / Lf[p];
    T[p] = opts[p].n_steps_T * dt0;
  }
  BCK(cudaMemcpyAsync(dT, T.data(), 8 * (size_t)n_prob, cudaMemcpyHostToDevice, st));
  k_profiles<<<dim3((n_cells + 255) / 256, n_prob), 256, 0, st>>>(d_fd, dta, dT, dhist);
  std::vector<unsigned int> hist(n_prob * (kMaxM + 1));
  BCK(cudaMemcpyAsync(hist.data(), dhist, 4 * hist.size(), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  // G = P P^T from the histogram of profile indices, then its pseudo-inverse
  std::vector<std::vector<double>> Gp(n_prob);
  for (int p = 0; p < n_prob; ++p) {
    const int M = opts[p].M;
    std::vector<double> G(M * M, 0.0);
    if (fd[p].prof) {  // dense profiles: G = P P^T summed over the cells in order
      std::vector<double> P((size_t)M * n_cells);
      BCK(cudaMemcpy(P.data(), fd[p].prof, 8 * P.size(), cudaMemcpyDeviceToHost));
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
          double g = 0.0;
          for (int e = 0; e < n_cells; ++e) g += P[(size_t)a * n_cells + e] * P[(size_t)b * n_cells + e];
          G[a * M + b] = g;
        }
      sym_pinv(M, G, Gp[p]);
      continue;
    }
    for (int k = 1; k <= M; ++k) {
      const double n = hist[p * (kMaxM + 1) + k];
      if (n == 0) continue;
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b)
          G[a * M + b] += n * ((a + 1 >= k) ? fd[p].lam1 : fd[p].lam0) * ((b + 1 >= k) ? fd[p].lam1 : fd[p].lam0);
    }
    sym_pinv(M, G, Gp[p]);
  }

  // ---- snapshots (step 2(c)) for all problems at once
  std::vector<int> snap_off(n_prob + 1, 0);
  for (int p = 0; p < n_prob; ++p) snap_off[p + 1] = snap_off[p] + opts[p].n_snap;
  const int n_snap_tot = snap_off[n_prob];
  FineSolver snaps;
  std::vector<double*> dmu(n_prob);
  if (n_snap_tot) {
    if (!snaps.init(B, nx, ny, n_snap_tot, st))
      return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the snapshot solves");
    std::vector<SysJob> jobs;
    for (int p = 0; p < n_prob; ++p) {
      dmu[p] = B.get<double>((size_t)opts[p].n_snap * opts[p].M);
      BCK(cudaMemcpyAsync(dmu[p], opts[p].mu, 8 * (size_t)opts[p].n_snap * opts[p].M, cudaMemcpyDefault, st));
      for (int k = 0; k < opts[p].n_snap; ++k) {
        const SimDev& d = snaps.sims[snap_off[p] + k];
        jobs.push_back(SysJob{p, 1, 3, 0, dmu[p] + (size_t)k * opts[p].M, d.A, d.A + 9 * (size_t)n_cells, d.b});
      }
    }
    if (int rc = run_systems(jobs)) return lrbms_internal_fail(ctx, rc, "snapshot assembly");
    BCK(launch_fine_solve(snaps.d_sims, snaps.d_active, n_snap_tot, st));
  }

  // ---- local bases (step 2(e))
  std::vector<std::vector<int>> NE(n_prob, std::vector<int>(n_sub));
  std::vector<std::vector<long long>> phioff(n_prob, std::vector<long long>(n_sub + 1, 0));
  std::vector<double*> Phi(n_prob);
  int* dgot = B.get<int>((size_t)n_prob * n_sub);
  std::vector<GsJob> gjobs;
  std::vector<const double*> snap_ptrs(std::max(n_snap_tot, 1));
  for (int s = 0; s < n_snap_tot; ++s) snap_ptrs[s] = snaps.sims[s].x;
  const double** dsnap = (const double**)B.get<double*>(std::max(n_snap_tot, 1));
  BCK(cudaMemcpyAsync(dsnap, snap_ptrs.data(), sizeof(double*) * snap_ptrs.size(), cudaMemcpyHostToDevice, st));
  std::vector<int> cfm(n_cf), cfp(n_cf);
  {
    int fidx = 0;
    for (int J = 0; J < Sy; ++J)
      for (int I = 0; I + 1 < Sx; ++I, ++fidx) cfm[fidx] = J * Sx + I, cfp[fidx] = J * Sx + I + 1;
    for (int J = 0; J + 1 < Sy; ++J)
      for (int I = 0; I < Sx; ++I, ++fidx) cfm[fidx] = J * Sx + I, cfp[fidx] = (J + 1) * Sx + I;
  }
  for (int p = 0; p < n_prob; ++p) {
    BCK(cudaMemcpy(NE[p].data(), opts[p].N_E, 4 * (size_t)n_sub, cudaMemcpyDefault));
    for (int E = 0; E < n_sub; ++E) {
      if (NE[p][E] < 1 || NE[p][E] > kMaxNE || NE[p][E] > 3 * cells)
        return lrbms_internal_fail(ctx, LRBMS_E_ARG, "local basis sizes must be in 1..min(32, 3 cells_E)");
      phioff[p][E + 1] = phioff[p][E] + (long long)NE[p][E] * 3 * cells;
    }
    Phi[p] = B.get<double>((size_t)phioff[p][n_sub]);
    if (!Phi[p]) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "basis buffers");
    if (opts[p].greedy) {
      // Algorithm 2, step 2: greedy selection over the training set opts.mu
      // (caps N_E per subdomain); the bases come out compacted to their sizes
      std::vector<int> cur;
      const int rc = greedy_bases(ctx, B, st, d_fd, fd[p], p, opts[p], dmu[p], dsnap + snap_off[p], NE[p], Phi[p],
                                  phioff[p], cfm, cfp, n_int, run_systems);
      if (rc) return rc;
      continue;
    }
    for (int E = 0; E < n_sub; ++E)
      gjobs.push_back(GsJob{p, E, NE[p][E], opts[p].n_snap, dsnap + snap_off[p], Phi[p] + phioff[p][E],
                            dgot + p * n_sub + E, 0});
  }
  {
    if (!gjobs.empty()) {
      GsJob* dj = B.get<GsJob>(gjobs.size());
      BCK(cudaMemcpyAsync(dj, gjobs.data(), sizeof(GsJob) * gjobs.size(), cudaMemcpyHostToDevice, st));
      k_gram_schmidt<<<(unsigned)gjobs.size(), 256, 8 * (size_t)3 * cells, st>>>(d_fd, dj);
      BCK(cudaGetLastError());
    }
    std::vector<int> got((size_t)n_prob * n_sub);
    BCK(cudaMemcpyAsync(got.data(), dgot, 4 * got.size(), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    for (int p = 0; p < n_prob; ++p) {
      if (opts[p].greedy) continue;  // sizes already final
      bool fewer = false;
      for (int E = 0; E < n_sub; ++E)
        if (got[p * n_sub + E] != NE[p][E]) {
          if (!opts[p].allow_fewer)
            return lrbms_internal_fail(ctx, LRBMS_E_FORMAT,
                                       "too few independent snapshots for the requested local basis size");
          fewer = true;
        }
      if (!fewer) continue;
      // keep the functions obtained: compact the bases to the achieved sizes
      std::vector<long long> off2(n_sub + 1, 0);
      for (int E = 0; E < n_sub; ++E) off2[E + 1] = off2[E] + (long long)got[p * n_sub + E] * 3 * cells;
      double* P2 = B.get<double>((size_t)off2[n_sub]);
      if (!P2) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "basis buffers");
      for (int E = 0; E < n_sub; ++E) {
        BCK(cudaMemcpyAsync(P2 + off2[E], Phi[p] + phioff[p][E], 8 * (size_t)(off2[E + 1] - off2[E]),
                            cudaMemcpyDeviceToDevice, st));
        NE[p][E] = got[p * n_sub + E];
      }
      Phi[p] = P2;
      phioff[p] = off2;
    }
    if (achieved) {
      for (int p = 0; p < n_prob; ++p)
        for (int E = 0; E < n_sub; ++E) achieved[p * n_sub + E] = NE[p][E];
    }
  }

  // ---- components (Section 4.4): fine blocks per component, then projection
  std::vector<std::vector<int>> xoff(n_prob, std::vector<int>(n_sub + 1, 0));
  std::vector<std::vector<long long>> aoff(n_prob, std::vector<long long>(n_sub + n_cf + 1, 0));
  std::vector<double*> comp(n_prob), rhs(n_prob);
  for (int p = 0; p < n_prob; ++p) {
    const int Q = opts[p].M + 1;
    for (int E = 0; E < n_sub; ++E) xoff[p][E + 1] = xoff[p][E] + NE[p][E];
    for (int E = 0; E < n_sub; ++E) aoff[p][E + 1] = aoff[p][E] + (long long)NE[p][E] * NE[p][E];
    for (int c = 0; c < n_cf; ++c)
      aoff[p][n_sub + c + 1] = aoff[p][n_sub + c] + (long long)NE[p][cfm[c]] * NE[p][cfp[c]];
    comp[p] = B.get<double>((size_t)Q * aoff[p][n_sub + n_cf]);
    rhs[p] = B.get<double>((size_t)Q * xoff[p][n_sub]);
    if (!comp[p] || !rhs[p]) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "component buffers");
  }
  {
    // fine blocks of every component of every problem (reused buffers per problem)
    for (int p = 0; p < n_prob; ++p) {
      const int Q = opts[p].M + 1;
      std::vector<SysJob> jobs(Q);
      std::vector<double*> D(Q), O(Q), R(Q);
      for (int q = 0; q < Q; ++q) {
        D[q] = B.get<double>(9 * (size_t)n_cells);
        O[q] = B.get<double>(9 * (size_t)std::max(n_int, 1));
        R[q] = B.get<double>(3 * (size_t)n_cells);
        if (!D[q] || !O[q] || !R[q]) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "fine component blocks");
        jobs[q] = q == 0 ? SysJob{p, 2, 1, 0, nullptr, D[q], O[q], R[q]}
                         : SysJob{p, 2, 2, q - 1, nullptr, D[q], O[q], R[q]};
      }
      if (int rc = run_systems(jobs)) return lrbms_internal_fail(ctx, rc, "component assembly");
      std::vector<ProjJob> pj;
      for (int q = 0; q < Q; ++q) {
        for (int E = 0; E < n_sub; ++E) {
          const double* PE = Phi[p] + phioff[p][E];
          const size_t sz = (size_t)NE[p][E] * NE[p][E];
          pj.push_back(ProjJob{p, 0, E, E, q, NE[p][E], NE[p][E], D[q], O[q], R[q], PE, PE,
                               comp[p] + (size_t)Q * aoff[p][E] + q * sz});
          pj.push_back(ProjJob{p, 2, E, E, q, NE[p][E], 0, D[q], O[q], R[q], PE, PE,
                               rhs[p] + (size_t)Q * xoff[p][E] + (size_t)q * NE[p][E]});
        }
        for (int c = 0; c < n_cf; ++c) {
          const int Em = cfm[c], Ep = cfp[c];
          const size_t sz = (size_t)NE[p][Em] * NE[p][Ep];
          pj.push_back(ProjJob{p, 1, Em, Ep, q, NE[p][Em], NE[p][Ep], D[q], O[q], R[q],
                               Phi[p] + phioff[p][Em], Phi[p] + phioff[p][Ep],
                               comp[p] + (size_t)Q * aoff[p][n_sub + c] + q * sz});
        }
      }
      ProjJob* dj = B.get<ProjJob>(pj.size());
      if (!dj) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "projection jobs");
      BCK(cudaMemcpyAsync(dj, pj.data(), sizeof(ProjJob) * pj.size(), cudaMemcpyHostToDevice, st));
      k_project<<<(unsigned)pj.size(), 256, 0, st>>>(d_fd, dj);
      BCK(cudaGetLastError());
      BCK(cudaStreamSynchronize(st));
    }
  }
  for (int s = 0; s < n_snap_tot; ++s) {
    int stv = 0;
    BCK(cudaMemcpy(&stv, snaps.sims[s].status, 4, cudaMemcpyDeviceToHost));
    if (stv) return lrbms_internal_fail(ctx, LRBMS_E_NOT_SPD, "a fine snapshot system was not positive definite");
  }
  for (int p = 0; p < n_prob; ++p) {
    int stv = 0;
    BCK(cudaMemcpy(&stv, init.sims[p].status, 4, cudaMemcpyDeviceToHost));
    if (stv) return lrbms_internal_fail(ctx, LRBMS_E_NOT_SPD, "the initial fine system was not positive definite");
  }

  // ---- admit n_copies simulations per problem (optionally with rotated bases)
  for (int p = 0; p < n_prob; ++p) {
    const int Q = opts[p].M + 1;
    std::vector<long long> qoff(n_sub + 1, 0);
    for (int E = 0; E < n_sub; ++E) qoff[E + 1] = qoff[E] + (long long)NE[p][E] * NE[p][E];
    double* rPhi = B.get<double>((size_t)phioff[p][n_sub]);
    double* rcomp = B.get<double>((size_t)Q * aoff[p][n_sub + n_cf]);
    double* rrhs = B.get<double>((size_t)Q * xoff[p][n_sub]);
    double* dQ = B.get<double>((size_t)qoff[n_sub]);
    int* dne = B.get<int>(n_sub);
    if (!rPhi || !rcomp || !rrhs || !dQ || !dne) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "copy buffers");
    BCK(cudaMemcpyAsync(dne, NE[p].data(), 4 * (size_t)n_sub, cudaMemcpyHostToDevice, st));
    double* dGp = B.get<double>(opts[p].M * opts[p].M);
    BCK(cudaMemcpyAsync(dGp, Gp[p].data(), 8 * Gp[p].size(), cudaMemcpyHostToDevice, st));
    for (int r = 0; r < n_copies; ++r) {
      const double* Qh = rot ? rot[p * n_copies + r] : nullptr;
      const double *uPhi = Phi[p], *ucomp = comp[p], *urhs = rhs[p];
      if (Qh) {
        BCK(cudaMemcpyAsync(dQ, Qh, 8 * (size_t)qoff[n_sub], cudaMemcpyDefault, st));
        std::vector<RotJob> rj;
        for (int E = 0; E < n_sub; ++E) {
          rj.push_back(RotJob{0, NE[p][E], NE[p][E], 3 * cells, Q, dQ + qoff[E], dQ + qoff[E],
                              Phi[p] + phioff[p][E], rPhi + phioff[p][E]});
          rj.push_back(RotJob{1, NE[p][E], NE[p][E], 0, Q, dQ + qoff[E], dQ + qoff[E],
                              comp[p] + (size_t)Q * aoff[p][E], rcomp + (size_t)Q * aoff[p][E]});
          rj.push_back(RotJob{2, NE[p][E], NE[p][E], 0, Q, dQ + qoff[E], dQ + qoff[E],
                              rhs[p] + (size_t)Q * xoff[p][E], rrhs + (size_t)Q * xoff[p][E]});
        }
        for (int c = 0; c < n_cf; ++c)
          rj.push_back(RotJob{1, NE[p][cfm[c]], NE[p][cfp[c]], 0, Q, dQ + qoff[cfm[c]], dQ + qoff[cfp[c]],
                              comp[p] + (size_t)Q * aoff[p][n_sub + c], rcomp + (size_t)Q * aoff[p][n_sub + c]});
        RotJob* dj = B.get<RotJob>(rj.size());
        if (!dj) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "rotation jobs");
        BCK(cudaMemcpyAsync(dj, rj.data(), sizeof(RotJob) * rj.size(), cudaMemcpyHostToDevice, st));
        k_rotate<<<(unsigned)rj.size(), 256, 0, st>>>(dj);
        BCK(cudaGetLastError());
        uPhi = rPhi; ucomp = rcomp; urhs = rrhs;
      }
      lrbms_offline off{};
      off.M = opts[p].M;
      off.N_E = dne;
      off.prof_idx = fd[p].prof ? nullptr : fd[p].prof_idx;
      off.prof = fd[p].prof;
      off.Gpinv = dGp;
      off.Phi = uPhi;
      off.Dblk = ucomp;
      off.Fblk = n_cf ? ucomp + (size_t)Q * aoff[p][n_sub] : nullptr;
      off.rhs = urhs;
      off.c_pen = opts[p].c_pen;
      off.Lf = Lf[p];
      BCK(cudaStreamSynchronize(st));
      const int rc = lrbms_offline_load(ctx, &probs[p], &off, &sim_ids[p * n_copies + r]);
      if (rc) return rc;
    }
  }
  BCK(cudaStreamSynchronize(st));
  return LRBMS_OK;
}

extern "C" int lrbms_clone(lrbms_ctx* ctx, int src, const double* rot, int* sim_id) {
  if (!ctx || !sim_id) return lrbms_internal_fail(ctx, LRBMS_E_ARG, "bad arguments");
  SimDev d;
  if (lrbms_internal_sim(ctx, src, &d)) return lrbms_internal_fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  // The copy runs on the admission stream. A source in the batch of the last
  // step may still be changing: wait for the context stream first; any other
  // source is at rest, and the copy overlaps the steps in flight.
  if (lrbms_internal_in_last_batch(ctx, src)) BCK(cudaStreamSynchronize(lrbms_internal_stream(ctx)));
  cudaStream_t st = lrbms_internal_admit_stream(ctx);
  BCK(cudaStreamSynchronize(st));
  const int n_sub = d.n_sub, n_cf = d.n_cf, Q = d.M + 1, cells = d.cx * d.cy;
  std::vector<int> NE(n_sub), xoff(n_sub + 1);
  std::vector<long long> aoff(d.n_blocks + 1), phioff(n_sub);
  BCK(cudaMemcpy(NE.data(), d.NE, 4 * (size_t)n_sub, cudaMemcpyDeviceToHost));
  BCK(cudaMemcpy(xoff.data(), d.xoff, 4 * (size_t)(n_sub + 1), cudaMemcpyDeviceToHost));
  BCK(cudaMemcpy(aoff.data(), d.aoff, 8 * (size_t)(d.n_blocks + 1), cudaMemcpyDeviceToHost));
  BCK(cudaMemcpy(phioff.data(), d.phi_off, 8 * (size_t)n_sub, cudaMemcpyDeviceToHost));
  std::vector<int> cfm(n_cf), cfp(n_cf);
  {
    int f = 0;
    for (int J = 0; J < d.Sy; ++J)
      for (int I = 0; I + 1 < d.Sx; ++I, ++f) cfm[f] = J * d.Sx + I, cfp[f] = J * d.Sx + I + 1;
    for (int J = 0; J + 1 < d.Sy; ++J)
      for (int I = 0; I < d.Sx; ++I, ++f) cfm[f] = J * d.Sx + I, cfp[f] = (J + 1) * d.Sx + I;
  }
  std::vector<long long> qoff(n_sub + 1, 0);
  for (int E = 0; E < n_sub; ++E) qoff[E + 1] = qoff[E] + (long long)NE[E] * NE[E];
  const long long phi_tot = phioff[n_sub - 1] + (long long)NE[n_sub - 1] * 3 * cells;
  int steps = 0;
  BCK(cudaMemcpy(&steps, d.steps, 4, cudaMemcpyDeviceToHost));
  // An unrotated copy is loaded straight from the source's arrays and its
  // current saturation (the source is at rest): no scratch buffers, whose
  // cudaMalloc and cudaFree would wait for the steps in flight on the other
  // streams.
  const double* s0 = d.s + (size_t)(steps & 1) * d.n_cells;
  const double *uPhi = d.Phi, *ucomp = d.comp, *urhs = d.rhs;
  DevBuf B;
  if (rot) {
    double* rPhi = B.get<double>((size_t)phi_tot);
    double* rcomp = B.get<double>((size_t)Q * aoff[d.n_blocks]);
    double* rrhs = B.get<double>((size_t)Q * xoff[n_sub]);
    double* dQ = B.get<double>((size_t)qoff[n_sub]);
    double* s0buf = B.get<double>((size_t)d.n_cells);
    if (!rPhi || !rcomp || !rrhs || !dQ || !s0buf) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "clone buffers");
    BCK(cudaMemcpyAsync(s0buf, s0, 8 * (size_t)d.n_cells, cudaMemcpyDeviceToDevice, st));
    s0 = s0buf;
    BCK(cudaMemcpyAsync(dQ, rot, 8 * (size_t)qoff[n_sub], cudaMemcpyDefault, st));
    std::vector<RotJob> rj;
    for (int E = 0; E < n_sub; ++E) {
      rj.push_back(RotJob{0, NE[E], NE[E], 3 * cells, Q, dQ + qoff[E], dQ + qoff[E], d.Phi + phioff[E], rPhi + phioff[E]});
      rj.push_back(RotJob{1, NE[E], NE[E], 0, Q, dQ + qoff[E], dQ + qoff[E], d.comp + (size_t)Q * aoff[E],
                          rcomp + (size_t)Q * aoff[E]});
      rj.push_back(RotJob{2, NE[E], NE[E], 0, Q, dQ + qoff[E], dQ + qoff[E], d.rhs + (size_t)Q * xoff[E],
                          rrhs + (size_t)Q * xoff[E]});
    }
    for (int c = 0; c < n_cf; ++c)
      rj.push_back(RotJob{1, NE[cfm[c]], NE[cfp[c]], 0, Q, dQ + qoff[cfm[c]], dQ + qoff[cfp[c]],
                          d.comp + (size_t)Q * aoff[n_sub + c], rcomp + (size_t)Q * aoff[n_sub + c]});
    RotJob* dj = B.get<RotJob>(rj.size());
    if (!dj) return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "rotation jobs");
    BCK(cudaMemcpyAsync(dj, rj.data(), sizeof(RotJob) * rj.size(), cudaMemcpyHostToDevice, st));
    k_rotate<<<(unsigned)rj.size(), 256, 0, st>>>(dj);
    BCK(cudaGetLastError());
    uPhi = rPhi; ucomp = rcomp; urhs = rrhs;
  }
  lrbms_problem pr{};
  pr.nx = d.nx; pr.ny = d.ny; pr.Sx = d.Sx; pr.Sy = d.Sy;
  pr.Lx = d.hx * d.nx; pr.Ly = d.hy * d.ny;
  pr.perm = d.perm; pr.poro = d.poro; pr.eta_w = 1.0 / d.inv_eta_w; pr.eta_o = 1.0 / d.inv_eta_o;
  pr.relperm = d.relperm; pr.bc_type = d.bc_type; pr.p_D = d.p_D; pr.v_N = d.v_N; pr.s_D = d.s_D;
  pr.s0 = s0; pr.cfl = d.cfl; pr.dt_mode = d.dt_mode; pr.dt_fixed = d.dt_fixed; pr.dt_max = d.dt_max;
  pr.mean_weights = d.swapped;
  pr.velocity = d.vel_mode;
  pr.transport = d.transport;
  lrbms_offline off{};
  off.M = d.M; off.N_E = d.NE; off.prof_idx = d.prof_idx; off.prof = d.prof; off.Gpinv = d.Gpinv;
  off.Phi = uPhi; off.Dblk = ucomp; off.Fblk = n_cf ? ucomp + (size_t)Q * aoff[n_sub] : nullptr;
  off.rhs = urhs; off.c_pen = d.c_pen; off.Lf = d.Lf;
  BCK(cudaStreamSynchronize(st));
  const int rc = lrbms_offline_load(ctx, &pr, &off, sim_id);
  if (rc != LRBMS_OK) return rc;
  // Same basis and state as a source that has not stepped: the same matrix,
  // so the new simulation can start with the source's FP32 factor.
  if (!rot && steps == 0) return lrbms_internal_share_factor(ctx, src, *sim_id);
  return LRBMS_OK;
}

// Algorithm 1 (the high-dimensional IMPES scheme) on resident simulations:
// per step the fine SWIP-DG pressure system of Definition 1 with lambda(s^n)
// is assembled and solved in FP64 (one envelope block Cholesky per system,
// one-cell blocks), and the fine pressure then goes through the same flux
// (Definition 2), CFL and upwind transport (Definition 3) kernels as the
// reduced step.
extern "C" int lrbms_fine_step(lrbms_ctx* ctx, int n_sims, const int* ids, int n_steps, int* status) {
  if (!ctx || n_sims < 1 || !ids || n_steps < 0) return lrbms_internal_fail(ctx, LRBMS_E_ARG, "bad arguments");
  cudaStream_t st = lrbms_internal_stream(ctx);
  std::vector<SimDev> sd(n_sims);
  for (int i = 0; i < n_sims; ++i) {
    if (lrbms_internal_sim(ctx, ids[i], &sd[i])) return lrbms_internal_fail(ctx, LRBMS_E_STATE, "unknown simulation id");
    if (sd[i].nx != sd[0].nx || sd[i].ny != sd[0].ny)
      return lrbms_internal_fail(ctx, LRBMS_E_ARG, "the simulations of one fine step must share the fine grid");
    if (sd[i].vel_mode != 0)
      return lrbms_internal_fail(ctx, LRBMS_E_ARG, "the fine scheme uses lambda(s^n): velocity must be STATE");
    if (sd[i].nx < 2 || sd[i].ny < 2) return lrbms_internal_fail(ctx, LRBMS_E_ARG, "fine grid must be at least 2x2");
  }
  const int nx = sd[0].nx, ny = sd[0].ny, n_cells = nx * ny;
  DevBuf B;
  FineSolver fs;
  if (!fs.init(B, nx, ny, n_sims, st))
    return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the fine systems");
  std::vector<FineDev> fd(n_sims);
  int max_tiles = 0;
  bool any_dg = false;
  size_t flux_smem = 0;
  for (int i = 0; i < n_sims; ++i) {
    const SimDev& d = sd[i];
    any_dg |= d.transport == 1;
    FineDev& f = fd[i];
    f.nx = nx; f.ny = ny; f.Sx = d.Sx; f.Sy = d.Sy; f.cx = d.cx; f.cy = d.cy; f.n_cells = n_cells;
    f.nxf = d.nxf; f.n_faces = d.n_faces; f.nb = d.nb; f.M = d.M; f.relperm = d.relperm; f.swapped = d.swapped;
    f.hx = d.hx; f.hy = d.hy; f.vol = d.vol; f.c_pen = d.c_pen; f.inv_eta_w = d.inv_eta_w; f.inv_eta_o = d.inv_eta_o;
    f.lam0 = d.lam0; f.lam1 = d.lam1;
    f.perm = d.perm; f.poro = d.poro; f.bc_type = d.bc_type; f.p_D = d.p_D; f.v_N = d.v_N; f.s_D = d.s_D;
    f.prof_idx = nullptr;
    max_tiles = std::max(max_tiles, d.n_tiles);
    flux_smem = std::max(flux_smem, flux_cfl_smem(d.nx, d.ny, d.tile_rows));
  }
  FineDev* d_fd = B.get<FineDev>(n_sims);
  SysJob* d_jobs = B.get<SysJob>(n_sims);
  SoaJob* d_soa = B.get<SoaJob>(n_sims);
  int* d_act = B.get<int>(n_sims);
  if (!d_fd || !d_jobs || !d_soa || !d_act)
    return lrbms_internal_fail(ctx, LRBMS_E_BUDGET, "device memory for the fine systems");
  std::vector<SysJob> jobs(n_sims);
  std::vector<SoaJob> soa(n_sims);
  for (int i = 0; i < n_sims; ++i) {
    jobs[i] = SysJob{i, 0, 3, 0, nullptr, fs.sims[i].A, fs.sims[i].A + 9 * (size_t)n_cells, fs.sims[i].b};
    soa[i] = SoaJob{fs.sims[i].x, sd[i].p, n_cells};
  }
  BCK(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(SysJob) * n_sims, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(d_soa, soa.data(), sizeof(SoaJob) * n_sims, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(d_act, ids, sizeof(int) * n_sims, cudaMemcpyHostToDevice, st));
  BCK(prepare_flux_cfl(flux_smem));
  SimDev* d_sims = lrbms_internal_dsims(ctx);
  std::vector<int> sst(n_sims, 0), steps(n_sims, 0);
  for (int k = 0; k < n_steps; ++k) {
    // the current saturation of each simulation (ping-pong by its step count)
    BCK(cudaStreamSynchronize(st));
    for (int i = 0; i < n_sims; ++i) {
      BCK(cudaMemcpy(&steps[i], sd[i].steps, 4, cudaMemcpyDeviceToHost));
      fd[i].s0 = sd[i].s + (size_t)(steps[i] & 1) * n_cells;
      BCK(cudaMemsetAsync(sd[i].fit_ready, 0, 4, st));  // lambda, f_w of s^n for flux and transport
    }
    BCK(cudaMemcpyAsync(d_fd, fd.data(), sizeof(FineDev) * n_sims, cudaMemcpyHostToDevice, st));
    const int n = std::max(n_cells, sd[0].n_faces);
    k_fine_system<<<dim3((n + 127) / 128, (unsigned)n_sims), 128, 0, st>>>(d_fd, d_jobs);
    BCK(launch_fine_solve(fs.d_sims, fs.d_active, n_sims, st));
    k_fine_to_soa<<<dim3((n_cells + 255) / 256 < 152 ? (n_cells + 255) / 256 : 152, (unsigned)n_sims), 256, 0, st>>>(
        d_soa);
    BCK(cudaGetLastError());
    // a fine system that is not positive definite freezes its simulation
    BCK(cudaStreamSynchronize(st));
    for (int i = 0; i < n_sims; ++i) {
      int fst = 0;
      BCK(cudaMemcpy(&fst, fs.sims[i].status, 4, cudaMemcpyDeviceToHost));
      if (fst != 0) BCK(cudaMemcpy(sd[i].status, &fst, 4, cudaMemcpyHostToDevice));
    }
    launch_fit(d_sims, d_act, n_sims, max_tiles, st);
    launch_flux_cfl(d_sims, d_act, n_sims, max_tiles, flux_smem, st);
    launch_transport(d_sims, d_act, n_sims, max_tiles, st);
    if (any_dg) launch_transport_dg(d_sims, d_act, n_sims, max_tiles, st);
    launch_finalize(d_sims, d_act, n_sims, st);
    BCK(cudaGetLastError());
    lrbms_internal_count(ctx, any_dg ? 10 : 8);
  }
  BCK(cudaStreamSynchronize(st));
  if (status)
    for (int i = 0; i < n_sims; ++i) BCK(cudaMemcpy(&status[i], sd[i].status, 4, cudaMemcpyDeviceToHost));
  return LRBMS_OK;
}
