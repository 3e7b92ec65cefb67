// Reduced system of Eq. reducedSystem: assembly and solve.
//
// assemble: theta = G^+ r (normal equations of Eq. leastSquaresFit from the
//   fixed-order sum of the fit partials), then every block
//   A_b = c_b + sum_q theta_q (b_q)_b and every subdomain right-hand side
//   b_E = e_E + sum_q theta_q (d_q)_E, streamed from the component arrays.
// chol_solve: one CTA of four warps per simulation. The matrix is symmetric positive
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

// Eq. leastSquaresFit: theta = G^+ r, r_q the sum over tiles (in tile order)
// of the fit partials; one warp per simulation, once per step, before the
// assembly's CTAs read it.
__global__ void k_theta(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.x]];
  if (S.status[0] != kStOk) return;
  __shared__ double rsh[kMaxM];
  const int M = S.M, q = threadIdx.x;
  if (q < M) {
    double r = 0.0;
    for (int t = 0; t < S.n_tiles; ++t) r += S.fit_part[(size_t)t * kMaxM + q];
    rsh[q] = r;
  }
  __syncwarp();
  if (q < M) {
    double th = 0.0;
    for (int j = 0; j < M; ++j) th = fma(S.Gpinv[q * M + j], rsh[j], th);
    S.theta[q] = th;
  }
}

// Eq. reducedSystem: A = c + sum_q theta_q b_q and rhs = e + sum_q theta_q d_q,
// the components stored as Q = M + 1 consecutive arrays per block (weight 1,
// then theta). One CTA per block of A or per subdomain's rhs.
__device__ __forceinline__ void load_weights(const SimDev& S, double* w) {
  if (threadIdx.x <= S.M) w[threadIdx.x] = threadIdx.x == 0 ? 1.0 : S.theta[threadIdx.x - 1];
  __syncthreads();
}

__global__ void k_assemble(const SimDev* __restrict__ sims, const int* __restrict__ active) {
  const SimDev& S = sims[active[blockIdx.y]];
  const int bidx = blockIdx.x;
  if (bidx >= S.n_blocks + S.n_sub || S.status[0] != kStOk) return;
  __shared__ double w[kMaxM + 1];
  load_weights(S, w);
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
  load_weights(S, w);
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

// ---------------------------------------------------------------- bulk-copy ring
// Chunks of the factor (a block of a panel, or a diagonal inverse) are copied
// from global to shared memory by cp.async.bulk, each completing on the "full"
// mbarrier of its slot; consumers release a slot on its "empty" mbarrier
// before the producer (lane 0 of warp 0) refills it. The copies of the next
// chunks run while the CTA computes on the current one. Every wait is bounded.
constexpr int kNW = kSolveWarps;             // warps per simulation
constexpr int kThreads = 32 * kNW;
constexpr int kRing = 4;                     // slots of the factorisation ring
constexpr int kSlot = kMaxNE * kMaxNE + 8;   // elements per slot: one 32 x 32 block + alignment slack
constexpr int kMaxSlots = 32;                // slots (and full/empty mbarrier pairs) at most
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  #pragma unroll 1
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) break;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
}

// Ring state (all threads walk the same chunk stream): chunk n lives in slot
// n % nslot; ph holds the parity awaited next on each full barrier. Producer
// state, meaningful in warp 0: eph, the parity awaited next on each empty
// barrier; used, the barriers filled before; fpar, the number of fills of each
// barrier mod 2. Barrier s always pairs with slot s of the current ring.
template <typename T>
struct Ring {
  T* base;
  uint64_t* full;
  uint64_t* empty;
  int* dl;  // per slot: element offset of the chunk within its aligned copy
  int nslot;
  unsigned issued, consumed;
  unsigned ph, eph, used, fpar;
  bool ok;
};

// Producer (called by warp 0; lane 0 copies): the copy of `count` elements
// starting at element `off` of `src` (src 16-byte aligned) starts at the
// 16-byte boundary at or below `off` and its size is rounded up to 16 bytes.
// A slot filled before is refilled once its empty barrier has completed.
template <typename T>
__device__ __forceinline__ void ring_issue(Ring<T>& r, const T* src, long long off, int count, int lane) {
  constexpr int kA = 16 / (int)sizeof(T);
  const int d = (int)(off & (kA - 1));
  const uint32_t bytes = (uint32_t)(((d + count) * (int)sizeof(T) + 15) & ~15);
  const int s = (int)(r.issued % (unsigned)r.nslot);
  if (r.used & (1u << s)) {  // after a timed-out wait, no further waits (fail fast)
    if (lane == 0 && r.ok && !mbar_wait(&r.empty[s], (r.eph >> s) & 1u)) r.ok = false;
    r.eph ^= 1u << s;
  }
  r.used |= 1u << s;
  r.fpar ^= 1u << s;
  if (lane == 0) {
    r.dl[s] = d;  // published to the waiting threads by the arrive (release) below
    mbar_expect_tx(&r.full[s], bytes);
    bulk_g2s(r.base + (size_t)s * kSlot, src + (off - d), bytes, &r.full[s]);
  }
  ++r.issued;
}

// Consumer: wait for the next chunk; returns its first element.
template <typename T>
__device__ __forceinline__ const T* ring_wait(Ring<T>& r) {
  const int s = (int)(r.consumed % (unsigned)r.nslot);
  if (r.ok && !mbar_wait(&r.full[s], (r.ph >> s) & 1u)) r.ok = false;  // fail fast after a timeout
  r.ph ^= 1u << s;
  return r.base + (size_t)s * kSlot + r.dl[s];
}
// Consumer done with the chunk (after ring_wait): `count` arrivals on its
// empty barrier (kNW consumers of 1, or one consumer of kNW).
template <typename T>
__device__ __forceinline__ void ring_release(Ring<T>& r, int lane, uint32_t count) {
  const int s = (int)(r.consumed % (unsigned)r.nslot);
  __syncwarp();
  if (lane == 0) mbar_arrive(&r.empty[s], count);
  ++r.consumed;
}
// A chunk consumed by another warp.
template <typename T>
__device__ __forceinline__ void ring_skip(Ring<T>& r) {
  const int s = (int)(r.consumed % (unsigned)r.nslot);
  r.ph ^= 1u << s;
  ++r.consumed;
}

// Error paths: bounded wait by the producer (lane 0 of the leader warp) for
// the last fill of every barrier, so that no copy is in flight when the CTA exits.
__device__ __forceinline__ int vwarp();
template <typename T>
__device__ void ring_drain(const Ring<T>& r) {
  if ((threadIdx.x & 31) == 0 && vwarp() == 0)
    #pragma unroll 1
    for (int s = 0; s < kMaxSlots; ++s)
      if (r.used & (1u << s)) mbar_wait(&r.full[s], ((~r.fpar) >> s) & 1u);
}

// ---------------------------------------------------------------- per-CTA shared memory
struct SolveMeta {
  int* NE;
  int* xoff;
  long long* loff;
  long long* ioff;
};

__host__ __device__ inline size_t meta_bytes(int n_sub) {
  return ((size_t)4 * (2 * n_sub + 1) + 15) / 16 * 16 + (size_t)16 * (n_sub + 1);
}
__host__ __device__ inline size_t round4(size_t v) { return (v + 3) & ~(size_t)3; }
constexpr size_t kBarBytes = 8 * kMaxSlots * 2 + 8 * kMaxSlots + 16;  // full, empty, dl, epos, flags
// Offset tables, barriers, slot offsets, FIFO entry starts and flags, per-warp partial vectors
// [kNW][32], the panel R of the current block row (padded columns), the
// factorisation ring, the substitution vectors [2N] and [32].
__host__ __device__ inline size_t warp_smem_bytes(int n_sub, int panel_words, int N, size_t elem) {
  return meta_bytes(n_sub) + kBarBytes +
         elem * (32 * kNW + round4(panel_words) + (size_t)kRing * kSlot + round4(2 * (size_t)N) + 32);
}

template <typename T>
struct CtaSmem {
  SolveMeta mt;
  uint64_t* full;   // [kMaxSlots]
  uint64_t* empty;  // [kMaxSlots]
  int* dl;          // [kMaxSlots]
  int* epos;        // [kMaxSlots] entry starts of the substitution FIFOs
  int* flag;        // [0] non-positive pivot, [1] copy timeout
  T* part;          // [kNW][32]
  T* R;             // [panel_words]
  T* ring;          // [kRing][kSlot]
  T* yz;            // [2N]
  T* tv;            // [32]
  int n_sub_slots;  // slots of the substitution ring, which spans R and the factor ring
  unsigned ph;      // ring state carried between the factorisation and the substitutions
  unsigned eph, used, fpar;
};

template <typename T>
__device__ CtaSmem<T> cta_carve_and_load(const SimDev& S, unsigned char* b) {
  CtaSmem<T> m;
  const int ns = S.n_sub;
  m.mt.NE = reinterpret_cast<int*>(b);
  m.mt.xoff = m.mt.NE + ns;
  const size_t o = ((size_t)4 * (2 * ns + 1) + 15) / 16 * 16;
  m.mt.loff = reinterpret_cast<long long*>(b + o);
  m.mt.ioff = m.mt.loff + (ns + 1);
  unsigned char* bb = b + meta_bytes(ns);
  m.full = reinterpret_cast<uint64_t*>(bb);
  m.empty = m.full + kMaxSlots;
  m.dl = reinterpret_cast<int*>(m.empty + kMaxSlots);
  m.epos = m.dl + kMaxSlots;
  m.flag = m.epos + kMaxSlots;
  T* t = reinterpret_cast<T*>(bb + kBarBytes);
  const size_t rw = round4((size_t)S.panel_words);
  m.part = t;
  m.R = t + 32 * kNW;
  m.ring = m.R + rw;
  m.yz = m.ring + (size_t)kRing * kSlot;
  m.tv = m.yz + round4(2 * (size_t)S.N);
  const size_t nss = (rw + (size_t)kRing * kSlot) / kSlot;
  m.n_sub_slots = nss > (size_t)kMaxSlots ? kMaxSlots : (int)nss;
  m.ph = m.eph = m.used = m.fpar = 0;
  #pragma unroll 1
  for (int i = threadIdx.x; i < ns; i += kThreads) m.mt.NE[i] = S.NE[i];
  #pragma unroll 1
  for (int i = threadIdx.x; i <= ns; i += kThreads) {
    m.mt.xoff[i] = S.xoff[i];
    m.mt.loff[i] = S.loff[i];
    m.mt.ioff[i] = S.ioff[i];
  }
  if (threadIdx.x == 0) {
    #pragma unroll 1
    for (int i = 0; i < kMaxSlots; ++i) {
      mbar_init(&m.full[i], 1);
      mbar_init(&m.empty[i], kNW);
    }
    m.flag[0] = 0;
    m.flag[1] = 0;
    m.flag[2] = 0;  // block rows of cfactor_mma: all
    m.flag[3] = ns;
    fence_mbar_init();
  }
  __syncthreads();
  return m;
}

// Role of the warp within its CTA: the leader (role 0: producer, diagonal
// factorisations, inverse steps) rotates with the CTA index, so that the
// leaders of the CTAs sharing an SM sit on different SM sub-partitions.
__device__ __forceinline__ int vwarp() {
  return (int)(((threadIdx.x >> 5) + kNW - blockIdx.x % kNW) % kNW);
}

// Invalidate the mbarriers (before the shared memory is carved again).
__device__ void cta_release_barriers(uint64_t* full) {
  __syncthreads();
  if (threadIdx.x == 0)
    #pragma unroll 1
    for (int i = 0; i < 2 * kMaxSlots; ++i) mbar_inval(&full[i]);
  __syncthreads();
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ float vget(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2& v, int i) { return i == 0 ? v.x : v.y; }

// Padded width of block row k in R: sum over its envelope of round4(N_i).
__device__ __forceinline__ int padded_width(const SolveMeta& mt, int jl, int k) {
  int w = 0;
  #pragma unroll 1
  for (int i = jl; i <= k; ++i) w += (mt.NE[i] + 3) & ~3;
  return w;
}
// Row stride of R for padded width Wc: 16-byte aligned rows whose starts fall
// on 16 (mod 32) bytes when Wc * sizeof(T) is a multiple of 32, so that a
// column read by lanes over rows spreads over 8 bank groups.
template <typename T>
__device__ __forceinline__ int row_stride(int Wc) {
  return ((Wc * (int)sizeof(T)) & 31) == 0 ? Wc + 16 / (int)sizeof(T) : Wc;
}

// Row-GEMM on one warp, lane = output column c (< ncols):
//   C[r][c] (set: =, else -=) sum_{t < 4 NV} A[r][t] B[t][c],  r < nrows,
// A rows in shared memory (16-byte aligned, zero beyond the true inner size),
// B element (t, c) at Bp[t * bst + c * bsc] for t < nt (zero for t >= nt).
// Four rows per pass for independent accumulation chains; with `set` C may
// alias A (every row is read by all lanes before it is written). Not inlined:
// one copy per unroll depth keeps the kernel's instruction footprint small
// when several CTAs share an SM.
template <typename T, int NV>
__device__ __noinline__ void rowgemm_nv(const T* __restrict__ A, int lda, T* C, int ldc, int nrows, const T* Bp,
                                        int bst, int bsc, int nt, int ncols, int lane, bool set) {
  using V = typename Vec16<T>::type;
  constexpr int kV = Vec16<T>::n;
  constexpr int NT = 4 * NV;
  T b[NT];
  const bool act = lane < ncols;
#pragma unroll
  for (int t = 0; t < NT; ++t) b[t] = (act && t < nt) ? Bp[t * bst + lane * bsc] : T(0);
#pragma unroll 1
  for (int r = 0; r < nrows; r += 4) {  // rows past nrows repeat the last row and are not written
    T acc[4][2];
    int ri[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[i][0] = acc[i][1] = T(0);
      ri[i] = min(r + i, nrows - 1);
    }
#pragma unroll
    for (int v = 0; v < NT / kV; ++v) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const V x = reinterpret_cast<const V*>(A + ri[i] * lda)[v];
#pragma unroll
        for (int e = 0; e < kV; ++e) acc[i][e & 1] = fma(vget(x, e), b[v * kV + e], acc[i][e & 1]);
      }
    }
    if (set) __syncwarp();
    if (act) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (r + i < nrows) {
          T* c = C + (r + i) * ldc + lane;
          *c = (set ? T(0) : *c) - (acc[i][0] + acc[i][1]) * (set ? T(-1) : T(1));
        }
      }
    }
  }
  __syncwarp();
}

template <typename T>
__device__ __forceinline__ void rowgemm(const T* A, int lda, T* C, int ldc, int nrows, const T* Bp, int bst,
                                        int bsc, int nt, int ncols, int lane, bool set) {
  if (nrows <= 0) return;
  switch ((nt + 3) >> 2) {
    case 1: rowgemm_nv<T, 1>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    case 2: rowgemm_nv<T, 2>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    case 3: rowgemm_nv<T, 3>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    case 4: rowgemm_nv<T, 4>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    case 5: rowgemm_nv<T, 5>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    case 6: rowgemm_nv<T, 6>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    case 7: rowgemm_nv<T, 7>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
    default: rowgemm_nv<T, 8>(A, lda, C, ldc, nrows, Bp, bst, bsc, nt, ncols, lane, set); break;
  }
}

// Chunk sequence of the factorisation of block row k: for every j in
// [jlo_k, k): the transposed inverse of L_jj, then L_{j'j} for j' in (j, k)
// (rows of the transposed panel j' at the columns of block j).
struct FactorSeq {
  int k, j, jp;
  __device__ bool done() const { return j >= k; }
  __device__ void next() {
    if (++jp >= k) {
      ++j;
      jp = j;
    }
  }
};

template <typename T>
__device__ __forceinline__ void factor_issue(Ring<T>& r, FactorSeq& q, const SolveMeta& mt, int Sx, const T* LT,
                                             const T* Linv, int lane) {
  const int Nj = mt.NE[q.j];
  if (q.jp == q.j) {
    ring_issue<T>(r, Linv, mt.ioff[q.j] + ((Nj * Nj + 3) & ~3), Nj * Nj, lane);
  } else {
    const int Njp = mt.NE[q.jp];
    const long long off = mt.loff[q.jp] + (long long)(mt.xoff[q.j] - mt.xoff[jlo_of(q.jp, Sx)]) * Njp;
    ring_issue<T>(r, LT, off, Nj * Njp, lane);
  }
  q.next();
}

// Cholesky factor and inverse of the N x N diagonal block Rd (shared memory,
// row stride ld) by one warp, so that no CTA barrier is needed (the other
// warps write the row's panel back meanwhile). The lower triangle is copied
// to the work area W with the odd row stride N | 1 (a column is read without
// bank conflicts). Right-looking factorisation, lane = row: column c is
// scaled by 1/sqrt(D[c][c]), then D[i][t] -= l_i l_t for c < t <= i (the
// loop runs over every t > c; the entries above the diagonal it also
// touches are never read). Inverse Y = L^-1 row by row, lane = column:
// Y[i][j] = (delta_ij - sum_{t < i} L[i][t] Y[t][j]) / L[i][i], over a
// zero-filled Y. Writes L^-1 to Li [N][N] and its transpose after it, and
// the transpose also to the panel's diagonal slot LTd (L itself is never
// read again: products use the inverse), where the forward substitution
// fetches it in the same copy as the block to its left.
// Returns true (in every lane) on a non-positive or non-finite pivot.
template <typename T>
__device__ __noinline__ bool diag_block_warp(const T* Rd, int ld, int N, T* W, T* LTd, T* Li) {
  const int lane = threadIdx.x & 31;
  const int ldd = N | 1;
  T* D = W;
  T* Y = W + ((N * ldd + 3) & ~3);
  T* dinv = Y + ((N * N + 3) & ~3);  // [32] 1 / L[c][c]
#pragma unroll 1
  for (int i = 0; i < N; ++i)
    if (lane <= i) D[i * ldd + lane] = Rd[i * ld + lane];
#pragma unroll 1
  for (int e = lane; e < N * N; e += 32) Y[e] = T(0);
  __syncwarp();
  bool bad = false;
#pragma unroll 1
  for (int c = 0; c < N; ++c) {
    T piv = D[c * ldd + c];
    if (!(piv > T(0)) || !isfinite(piv)) {
      bad = true;
      piv = T(1);
    }
    const T d = sqrt(piv);
    const T inv = T(1) / d;
    T li = T(0);
    if (lane > c && lane < N) {
      li = D[lane * ldd + c] * inv;
      D[lane * ldd + c] = li;
    }
    __syncwarp();
    if (lane == 0) {
      D[c * ldd + c] = d;
      dinv[c] = inv;
    }
    if (lane < N) {
      T* Di = D + lane * ldd;
      int t = c + 1;
#pragma unroll 1
      for (; t + 3 < N; t += 4) {
        const T l0 = D[t * ldd + c], l1 = D[(t + 1) * ldd + c], l2 = D[(t + 2) * ldd + c], l3 = D[(t + 3) * ldd + c];
        const T d0 = Di[t], d1 = Di[t + 1], d2 = Di[t + 2], d3 = Di[t + 3];
        Di[t] = fma(-li, l0, d0);
        Di[t + 1] = fma(-li, l1, d1);
        Di[t + 2] = fma(-li, l2, d2);
        Di[t + 3] = fma(-li, l3, d3);
      }
#pragma unroll 1
      for (; t < N; ++t) Di[t] = fma(-li, D[t * ldd + c], Di[t]);
    }
    __syncwarp();
  }
  // inverse, lane = column j (Y[t][j] = 0 for t < j)
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    const T* Dr = D + i * ldd;
    T s0 = (lane == i) ? T(1) : T(0), s1 = T(0);
    int t = 0;
#pragma unroll 1
    for (; t + 1 < i; t += 2) {
      s0 = fma(-Dr[t], Y[t * N + lane], s0);
      s1 = fma(-Dr[t + 1], Y[(t + 1) * N + lane], s1);
    }
    if (t < i) s0 = fma(-Dr[t], Y[t * N + lane], s0);
    if (lane <= i) Y[i * N + lane] = (s0 + s1) * dinv[i];
    __syncwarp();
  }
  T* LiT = Li + ((N * N + 3) & ~3);
  if (lane < N) {
#pragma unroll 1
    for (int c = 0; c < N; ++c) {
      const T y = Y[c * N + lane];  // row c of L^-1 (zero right of the diagonal)
      Li[c * N + lane] = y;
      LiT[lane * N + c] = y;
      LTd[lane * N + c] = y;  // the panel's diagonal slot holds L^-1 in LiT's layout (see fwd_pair)
    }
  }
  return __any_sync(0xffffffffu, bad);
}

// Own rows [r0, r0 + nr) of the block-row panel R (row stride Wp) <- the
// assembled blocks of A in block row k (diagonal, left and lower neighbours;
// FP64 rounded to T), zero elsewhere and in the padding columns.
template <typename T>
__device__ void fill_rows(const SimDev& S, const SolveMeta& mt, T* R, int k, int jl, int Wp, int r0, int nr, int lane) {
  const int nsub = S.n_sub, Sx = S.Sx, Nk = mt.NE[k], r1 = r0 + nr;
  const int I = k % Sx, J = k / Sx;
  int pc = 0;
  #pragma unroll 1
  for (int i = jl; i <= k; ++i) {
    const int Ni = mt.NE[i], Np = (Ni + 3) & ~3;
    const double* blk = nullptr;
    if (i == k) blk = S.A + S.aoff[k];
    else if (I > 0 && i == k - 1) blk = S.A + S.aoff[nsub + J * (Sx - 1) + (I - 1)];        // [N_i][N_k]
    else if (J > 0 && i == k - Sx) blk = S.A + S.aoff[nsub + S.Sy * (Sx - 1) + (J - 1) * Sx + I];  // [N_i][N_k]
    if (i == k) {  // lanes over columns
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (u < nr && lane < Nk) ? blk[(r0 + u) * Nk + lane] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u < nr && lane < Np) R[(r0 + u) * Wp + pc + lane] = (T)v[u];
    } else if (blk) {  // A_{k,i}[r][c] = blk[c][r]: lanes over own rows read coalesced
      #pragma unroll 1
      for (int c0 = 0; c0 < Np; c0 += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (c0 + u < Ni && lane < nr) ? blk[(c0 + u) * Nk + r0 + lane] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < Np && lane < nr) R[(r0 + lane) * Wp + pc + c0 + u] = (T)v[u];
      }
    } else {
      #pragma unroll 1
      for (int r = r0; r < r1; ++r)
        if (lane < Np) R[r * Wp + pc + lane] = T(0);
    }
    pc += Np;
  }
  __syncwarp();
}

// Envelope block Cholesky of the assembled A (FP64) with factor storage T, by
// the kNW warps of one CTA, each owning a contiguous range of the rows of the
// current block row. Block row k is formed in R and processed right-looking:
// for each block j of the envelope, X_j = R_j L_jj^-T is finalised (L_kj =
// X_j), then the later off-diagonal blocks j' of the row are updated, R_j' -=
// X_j L_{j'j}^T (lane = column of j'); these steps touch only the warp's own
// rows. After a CTA barrier the diagonal block is updated with all X_j; the
// leader warp computes L_kk = chol(R_kk) and its inverse (diag_block_warp)
// while the other warps write the row's panel back.
// Panels are stored transposed, LT_k [W_k][N_k]; block k of the inverses holds
// L_kk^-1 and its transpose. Returns kFacOk, kFacPivot on a non-positive (or
// non-finite) pivot, or kFacTimeout if a copy did not complete.
constexpr int kFacOk = 0, kFacPivot = 1, kFacTimeout = 2;

template <typename T>
__device__ int cfactor(const SimDev& S, T* LT, T* Linv, CtaSmem<T>& m) {
  const SolveMeta& mt = m.mt;
  const int nsub = S.n_sub, Sx = S.Sx;
  const int lane = threadIdx.x & 31, w = vwarp();
  T* R = m.R;
  Ring<T> rg{m.ring, m.full, m.empty, m.dl, kRing, 0u, 0u, m.ph, m.eph, m.used, m.fpar, true};
  #pragma unroll 1
  for (int k = 0; k < nsub; ++k) {
    const int jl = jlo_of(k, Sx);
    const int base = mt.xoff[jl];
    const int Nk = mt.NE[k];
    const int Wc = padded_width(mt, jl, k);
    const int Wp = row_stride<T>(Wc);
    const int pck = Wc - ((Nk + 3) & ~3);
    const int r0 = (w * Nk) / kNW, r1 = ((w + 1) * Nk) / kNW, nr = r1 - r0;
    // every chunk of this row refers to rows written (and fenced) before it
    FactorSeq q{k, jl, jl};
    if (w == 0)
      while (!q.done() && (int)(rg.issued - rg.consumed) < rg.nslot) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
    fill_rows<T>(S, mt, R, k, jl, Wp, r0, nr, lane);
    __syncwarp();
    T* LTk = LT + mt.loff[k];
    T* Rw = R + r0 * Wp;
    int pcj = 0;
    #pragma unroll 1
    for (int j = jl; j < k; ++j) {
      const int Nj = mt.NE[j];
      const int Njp4 = (Nj + 3) & ~3;
      {  // X_j = R_j L_jj^-T on own rows (in place); B = (L_jj^-1)^T
        const T* LiT = ring_wait<T>(rg);
        rowgemm<T>(Rw + pcj, Wp, Rw + pcj, Wp, nr, LiT, Nj, 1, Nj, Nj, lane, true);
        ring_release<T>(rg, lane, 1);
        if (w == 0 && !q.done()) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
      }
      // R_j' -= X_j L_{j'j}^T for j' in (j, k), own rows
      int pcjp = pcj + Njp4;
      #pragma unroll 1
      for (int jp = j + 1; jp < k; ++jp) {
        const int Njp = mt.NE[jp];
        const T* Lc = ring_wait<T>(rg);  // [t][c'] = L_{j'j}[c'][t]
        rowgemm<T>(Rw + pcj, Wp, Rw + pcjp, Wp, nr, Lc, Njp, 1, Nj, Njp, lane, false);
        ring_release<T>(rg, lane, 1);
        if (w == 0 && !q.done()) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
        pcjp += (Njp + 3) & ~3;
      }
      pcj += Njp4;
    }
    __syncthreads();  // every X_j of the row is final
    {  // R_kk -= sum_j X_j X_j^T on own rows; B[t][c] = X_j[c][t]
      int pc = 0;
      #pragma unroll 1
      for (int j = jl; j < k; ++j) {
        const int Nj = mt.NE[j];
        rowgemm<T>(Rw + pc, Wp, Rw + pck, Wp, nr, R + pc, 1, Wp, Nj, Nk, lane, false);
        pc += (Nj + 3) & ~3;
      }
    }
    __syncthreads();
    if (w == 0) {  // diagonal block by the leader (its work area: the factor ring, idle between rows)
      const bool badp = diag_block_warp<T>(R + pck, Wp, Nk, m.ring, LTk + (size_t)(mt.xoff[k] - base) * Nk,
                                           Linv + mt.ioff[k]);
      if (badp && lane == 0) m.flag[0] = 1;
    } else {  // meanwhile L_kj = X_j into the transposed panel (lanes over rows: coalesced)
      int pc = 0;
      #pragma unroll 1
      for (int j = jl; j < k; ++j) {
        const int Nj = mt.NE[j], gj = mt.xoff[j] - base;
        if (lane < Nk)
          #pragma unroll 1
          for (int c = w - 1; c < Nj; c += kNW - 1) LTk[(size_t)(gj + c) * Nk + lane] = R[lane * Wp + pc + c];
        pc += (Nj + 3) & ~3;
      }
    }
    if (!rg.ok) m.flag[1] = 1;
    fence_proxy_async();  // the next rows copy these panels with the async proxy
    __syncthreads();
    if (m.flag[0] | m.flag[1]) {
      const int code = m.flag[1] ? kFacTimeout : kFacPivot;
      ring_drain<T>(rg);
      m.ph = rg.ph;
      m.eph = rg.eph;
      m.used = rg.used;
      m.fpar = rg.fpar;
      __syncthreads();
      return code;
    }
  }
  m.ph = rg.ph;
  m.eph = rg.eph;
  m.used = rg.used;
  m.fpar = rg.fpar;
  return kFacOk;
}

// ---------------------------------------------------------------- tensor-core block products
// FP32 block products of the factorisation on the tensor cores: mma.sync
// m16n8k8 with TF32 operands split into high and low parts, three products
// per term (a_lo b_hi + a_hi b_lo + a_hi b_hi, FP32 accumulation), which
// keeps the products at FP32 accuracy.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp: C[r][c] (set: =, else -=) sum_{t < K} A[r][t] B(t, c) for TM
// consecutive 16-row tiles from mt0 (rows r < M) and all c < N (N, K <= 32);
// A row-major (lda), B(t, c) at B[t * ldbk + c * ldbn], C row-major (ldc).
// B's fragments are loaded and split once per k-step and serve every tile.
// Every tile's rows are read for all t before any is written, so with `set`
// C may alias A. Each accumulator takes its terms in the same order for any
// TM (k-steps ascending; per k-step a_lo b_hi, a_hi b_lo, a_hi b_hi).
template <int TM>
__device__ __forceinline__ void mma_tiles(const float* A, int lda, float* C, int ldc, int M, int N, int K,
                                          const float* B, int ldbk, int ldbn, int mt0, bool set) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  float acc[TM][4][4];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[m][i][0] = acc[m][i][1] = acc[m][i][2] = acc[m][i][3] = 0.f;
#pragma unroll 1
  for (int kt = 0; kt * 8 < K; ++kt) {
    const int k0 = kt * 8 + tq, k1 = k0 + 4;
    uint32_t bh[4][2], bl[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int n = nt * 8 + g;
      const float b0 = (nt * 8 < N && k0 < K && n < N) ? B[k0 * ldbk + n * ldbn] : 0.f;
      const float b1 = (nt * 8 < N && k1 < K && n < N) ? B[k1 * ldbk + n * ldbn] : 0.f;
      split_tf32(b0, bh[nt][0], bl[nt][0]);
      split_tf32(b1, bh[nt][1], bl[nt][1]);
    }
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      const int r0 = (mt0 + m) * 16 + g, r1 = r0 + 8;
      float av[4];
      av[0] = (r0 < M && k0 < K) ? A[r0 * lda + k0] : 0.f;
      av[1] = (r1 < M && k0 < K) ? A[r1 * lda + k0] : 0.f;
      av[2] = (r0 < M && k1 < K) ? A[r0 * lda + k1] : 0.f;
      av[3] = (r1 < M && k1 < K) ? A[r1 * lda + k1] : 0.f;
      uint32_t ah[4], al[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) split_tf32(av[i], ah[i], al[i]);
      // term by term over the independent accumulators (small terms first)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        if (nt * 8 < N) mma_tf32(acc[m][nt], al, bh[nt]);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        if (nt * 8 < N) mma_tf32(acc[m][nt], ah, bl[nt]);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
        if (nt * 8 < N) mma_tf32(acc[m][nt], ah, bh[nt]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int r0 = (mt0 + m) * 16 + g, r1 = r0 + 8;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt * 8 < N) {
        const int c0 = nt * 8 + 2 * tq, c1 = c0 + 1;
        if (r0 < M && c0 < N) C[r0 * ldc + c0] = set ? acc[m][nt][0] : C[r0 * ldc + c0] - acc[m][nt][0];
        if (r0 < M && c1 < N) C[r0 * ldc + c1] = set ? acc[m][nt][1] : C[r0 * ldc + c1] - acc[m][nt][1];
        if (r1 < M && c0 < N) C[r1 * ldc + c0] = set ? acc[m][nt][2] : C[r1 * ldc + c0] - acc[m][nt][2];
        if (r1 < M && c1 < N) C[r1 * ldc + c1] = set ? acc[m][nt][3] : C[r1 * ldc + c1] - acc[m][nt][3];
      }
    }
  }
  __syncwarp();
}

// One warp: the 16-row tiles [m0, m1) of C (set: =, else -=) A B, rows
// r < M (M <= 32), as mma_tiles; two tiles share B's fragments.
__device__ __noinline__ void mma_block(const float* A, int lda, float* C, int ldc, int M, int N, int K,
                                       const float* B, int ldbk, int ldbn, int m0, int m1, bool set) {
  const int me = min(m1, (M + 15) >> 4);
  if (me - m0 >= 2)
    mma_tiles<2>(A, lda, C, ldc, M, N, K, B, ldbk, ldbn, m0, set);
  else if (me - m0 == 1)
    mma_tiles<1>(A, lda, C, ldc, M, N, K, B, ldbk, ldbn, m0, set);
}

// FP32 envelope block Cholesky with the block products on the tensor cores,
// by the CTA. Block row k is formed in R and processed right-looking in one
// barrier-separated phase per block j of the envelope (X_j = R_j L_jj^-T =
// L_kj final at its start): R_j' -= X_j L_{j'j}^T for j' in (j, k), each
// block product by one warp in turn; X_{j+1} by the warp that applied the
// update into block j+1; R_kk -= X_j X_j^T. Every warp waits for every chunk of the ring before it
// releases it (whether it used it or not), so no warp releases a slot ahead
// of the chunk's user. The diagonal block is factored by the leader warp as in
// cfactor. Same results contract as cfactor. Only block rows [m.flag[2],
// m.flag[3]) are computed (cta_carve_and_load sets all rows); the rows
// before m.flag[2] must already be in LT and Linv. The range is read from
// shared memory, so that it takes no register through the row loop.
__device__ int cfactor_mma(const SimDev& S, float* LT, float* Linv, CtaSmem<float>& m) {
  using T = float;
  const SolveMeta& mt = m.mt;
  const int Sx = S.Sx;
  const volatile int* rows = m.flag + 2;
  const int lane = threadIdx.x & 31, w = vwarp();
  T* R = m.R;
  Ring<T> rg{m.ring, m.full, m.empty, m.dl, kRing, 0u, 0u, m.ph, m.eph, m.used, m.fpar, true};
#pragma unroll 1
  for (int k = rows[0]; k < rows[1]; ++k) {
    const int jl = jlo_of(k, Sx);
    const int base = mt.xoff[jl];
    const int Nk = mt.NE[k];
    const int Wc = padded_width(mt, jl, k);
    const int Wp = row_stride<T>(Wc);
    const int pck = Wc - ((Nk + 3) & ~3);
    const int r0 = (w * Nk) / kNW, r1 = ((w + 1) * Nk) / kNW, nr = r1 - r0;
    const int mtn = (Nk + 15) >> 4;
    FactorSeq q{k, jl, jl};
    if (w == 0)
      while (!q.done() && (int)(rg.issued - rg.consumed) < rg.nslot) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
    fill_rows<T>(S, mt, R, k, jl, Wp, r0, nr, lane);
    __syncthreads();
    T* LTk = LT + mt.loff[k];
    if (jl < k) {  // X_jl = R_jl L_jl,jl^-T, its 16-row tiles on different warps
      const int N0 = mt.NE[jl];
      const T* LiT = ring_wait<T>(rg);
      if (w < mtn) mma_block(R, Wp, R, Wp, Nk, N0, N0, LiT, N0, 1, w, w + 1, true);
      ring_release<T>(rg, lane, 1);
      if (w == 0 && !q.done()) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
      __syncthreads();
    }
    int pcj = 0;
#pragma unroll 1
    for (int j = jl; j < k; ++j) {
      // phase j: X_j is final. Tasks in chunk order: R_j' -= X_j L_{j'j}^T for
      // j' = j+1 .. k-1, then X_{j+1} = R_{j+1} L^-T (by the warp that applied
      // the update into block j+1), then R_kk -= X_j X_j^T. One barrier per phase.
      const int Nj = mt.NE[j];
      const int Njp4 = (Nj + 3) & ~3;
      const int crit = (j - jl) % kNW;  // owner of block j+1's update and of X_{j+1}
      int task = 0;
      int pcjp = pcj + Njp4;
#pragma unroll 1
      for (int jp = j + 1; jp < k; ++jp) {
        const int Njp = mt.NE[jp];
        const T* Lc = ring_wait<T>(rg);
        if ((crit + task++) % kNW == w) mma_block(R + pcj, Wp, R + pcjp, Wp, Nk, Njp, Nj, Lc, Njp, 1, 0, 2, false);
        ring_release<T>(rg, lane, 1);
        if (w == 0 && !q.done()) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
        pcjp += (Njp + 3) & ~3;
      }
      if (j + 1 < k) {  // X_{j+1}
        const int N1 = mt.NE[j + 1];
        const T* LiT = ring_wait<T>(rg);
        if (w == crit) mma_block(R + pcj + Njp4, Wp, R + pcj + Njp4, Wp, Nk, N1, N1, LiT, N1, 1, 0, 2, true);
        ring_release<T>(rg, lane, 1);
        if (w == 0 && !q.done()) factor_issue<T>(rg, q, mt, Sx, LT, Linv, lane);
      }
      // R_kk -= X_j X_j^T; B(t, c) = X_j[c][t]
      if ((crit + task++) % kNW == w) mma_block(R + pcj, Wp, R + pck, Wp, Nk, Nk, Nj, R + pcj, 1, Wp, 0, 2, false);
      __syncthreads();
      pcj += Njp4;
    }
    if (w == 0) {  // diagonal block by the leader (its work area: the factor ring, idle between rows)
      const bool badp = diag_block_warp<T>(R + pck, Wp, Nk, m.ring, LTk + (size_t)(mt.xoff[k] - base) * Nk,
                                           Linv + mt.ioff[k]);
      if (badp && lane == 0) m.flag[0] = 1;
    } else {  // meanwhile L_kj = X_j into the transposed panel (lanes over rows: coalesced)
      int pc = 0;
#pragma unroll 1
      for (int j = jl; j < k; ++j) {
        const int Nj = mt.NE[j], gj = mt.xoff[j] - base;
        if (lane < Nk)
#pragma unroll 1
          for (int c = w - 1; c < Nj; c += kNW - 1) LTk[(size_t)(gj + c) * Nk + lane] = R[lane * Wp + pc + c];
        pc += (Nj + 3) & ~3;
      }
    }
    if (!rg.ok) m.flag[1] = 1;
    fence_proxy_async();  // the next rows copy these panels with the async proxy
    __syncthreads();
    if (m.flag[0] | m.flag[1]) {
      const int code = m.flag[1] ? kFacTimeout : kFacPivot;
      ring_drain<T>(rg);
      m.ph = rg.ph;
      m.eph = rg.eph;
      m.used = rg.used;
      m.fpar = rg.fpar;
      __syncthreads();
      return code;
    }
  }
  m.ph = rg.ph;
  m.eph = rg.eph;
  m.used = rg.used;
  m.fpar = rg.fpar;
  return kFacOk;
}

// ---------------------------------------------------------------- substitutions
// Forward and backward substitution, pipelined over the block rows with one
// CTA barrier per row. Forward, step k: the leader finishes row k (the other
// warps' partial sums for it, the block L_{k,k-1}, then y_k = L_kk^-1 t_k:
// the critical path) while the other warps form row k+1's sums over blocks
// jlo(k+1)..k-1. Backward, step k (descending): the leader applies the
// contribution of row k+1 to row k and z_k = L_kk^-T (y_k - p_k); the other
// warps apply the contributions of row k+1 to their columns of rows j < k
// (p_j += L_{k+1 j}^T z_{k+1}). Every warp streams its own chunks through
// its own region of shared memory (a FIFO of variable-size bulk copies with
// kEnt full barriers), so no warp waits for another to release a slot.
constexpr int kEnt = kMaxSlots / kNW;  // chunks in flight per warp

template <typename T>
struct WRing {
  T* base;          // the warp's region [cap]
  int cap;          // elements (multiple of 4)
  int b0;           // first barrier of the warp
  uint64_t* full;   // all barriers
  int* eoff;        // per barrier: element offset of the chunk's data in the region
  int* epos;        // per barrier: start of the entry in the region
  int pos, tpos;    // next allocation; start of the oldest live entry
  unsigned issued, consumed;
  unsigned ph, used, fpar;
  bool ok;
};

// Issue a chunk if it fits (lane 0 copies); returns false if the region is full.
// withhold: account for the chunk but do not copy it (the test hook of the
// bounded waits: its full barrier never completes).
template <typename T>
__device__ __forceinline__ bool wring_try_issue(WRing<T>& r, const T* src, long long off, int count, int lane,
                                                bool withhold = false) {
  constexpr int kA = 16 / (int)sizeof(T);
  if ((int)(r.issued - r.consumed) >= kEnt) return false;
  const int d = (int)(off & (kA - 1));
  const int need = (d + count + 3) & ~3;  // elements, 16-byte multiple
  int at;
  if (r.issued == r.consumed) {
    at = 0;
    r.tpos = 0;
  } else if (r.pos > r.tpos) {
    if (r.pos + need <= r.cap) at = r.pos;
    else if (need <= r.tpos) at = 0;
    else return false;
  } else {  // wrapped: free space is [pos, tpos)
    if (r.pos + need <= r.tpos) at = r.pos;
    else return false;
  }
  const int e = (int)(r.issued % (unsigned)kEnt);
  const int b = r.b0 + e;
  r.used |= 1u << b;
  r.fpar ^= 1u << b;
  if (lane == 0) {
    r.eoff[b] = at + d;
    r.epos[b] = at;
    if (!withhold) {
      mbar_expect_tx(&r.full[b], (uint32_t)(need * (int)sizeof(T)));
      bulk_g2s(r.base + at, src + (off - d), (uint32_t)(need * (int)sizeof(T)), &r.full[b]);
    }
  }
  r.pos = at + need;
  ++r.issued;
  return true;
}

template <typename T>
__device__ __forceinline__ const T* wring_wait(WRing<T>& r) {
  const int b = r.b0 + (int)(r.consumed % (unsigned)kEnt);
  if (r.ok && !mbar_wait(&r.full[b], (r.ph >> b) & 1u)) r.ok = false;  // fail fast after a timeout
  r.ph ^= 1u << b;
  return r.base + r.eoff[b];
}

template <typename T>
__device__ __forceinline__ void wring_release(WRing<T>& r) {
  __syncwarp();
  ++r.consumed;
  if (r.consumed == r.issued) r.tpos = r.pos;
  else r.tpos = r.epos[r.b0 + (int)(r.consumed % (unsigned)kEnt)];
}

// The chunks of the substitutions, per warp in consumption order. Block row
// k (forward k = 0, 1, ..., then backward k = nsub-1, ..., 0) gives
//  - the leader: the coupling block to the previous row (forward: panel k at
//    block k-1) or to the next row (backward: panel k+1 at block k), then the
//    diagonal inverse of row k;
//  - warp w >= 1: its share of the C_k = xoff[k] - xoff[jlo(k+1)] columns of
//    panel k+1 before block k (blocks jlo(k+1)..k-1, adjacent in the
//    transposed panel), columns [C_k (w-1)/(kNW-1), C_k w/(kNW-1)), copied in
//    pieces of at most pc columns, so that one copy usually carries all of a
//    warp's blocks of the row. The forward pass uses them for row k+1's sum
//    over those blocks, the backward pass for their update by z_{k+1}.
// Each warp keeps kPartWords elements at the start of its FIFO region for
// the forward partial sums (two rows of 32).
constexpr int kPartWords = 64;
__host__ __device__ inline int fifo_cap(int panel_words) {
  return ((int)((round4((size_t)panel_words) + (size_t)kRing * kSlot) / kNW) & ~3) - kPartWords;
}
// Most columns of a piece for a row of n2 elements: half the FIFO, at least one column.
__host__ __device__ inline int piece_cols(int panel_words, int n2) {
  const int c = (fifo_cap(panel_words) / 2 - 4) / n2;
  return c > 1 ? c : 1;
}
// The leader's forward chunk of row k: the coupling block L_{k,k-1} and the
// panel's diagonal slot (L_kk^-1, transposed) are adjacent in panel k, so one
// copy carries both when they fit half a FIFO (always for k = 0, the slot
// alone); otherwise the inverse comes from the inverse array.
__host__ __device__ inline bool fwd_pair(int panel_words, int nprev, int nk) {
  return (nprev + nk) * nk + 3 <= fifo_cap(panel_words) / 2;
}
__device__ __forceinline__ void warp_share(const SolveMeta& mt, int Sx, int nsub, int w, int k, int* c0, int* c1) {
  if (w == 0 || k + 1 >= nsub) {
    *c0 = *c1 = 0;
    return;
  }
  const int C = mt.xoff[k] - mt.xoff[jlo_of(k + 1, Sx)];
  *c0 = (int)((long long)C * (w - 1) / (kNW - 1));
  *c1 = (int)((long long)C * w / (kNW - 1));
}

// Chunk descriptor of the copy schedule: element offset (bits 0-39) into the
// panels, or into the diagonal inverses if bit 63 is set; element count in
// bits 40-55.
constexpr unsigned long long kDescOffMask = (1ull << 40) - 1;
constexpr unsigned long long kDescInverse = 1ull << 63;
__device__ __forceinline__ unsigned long long sdesc(long long off, int cnt, bool inv) {
  return (unsigned long long)off | ((unsigned long long)cnt << 40) | (inv ? kDescInverse : 0ull);
}

// The copy schedule of a simulation, by one thread: the word layout is that
// of sched_words (list starts relative to the buffer, then the lists); the
// order is the consumption order of csubstitute, forward then backward. The
// schedule depends only on the basis sizes, so it is built once at load.
__device__ void build_sched(const SimDev& S, unsigned long long* out) {
  const SolveMeta mt{const_cast<int*>(S.NE), const_cast<int*>(S.xoff), const_cast<long long*>(S.loff),
                     const_cast<long long*>(S.ioff)};
  const int nsub = S.n_sub, Sx = S.Sx;
  unsigned long long n = kNW + 1;
  #pragma unroll 1
  for (int w = 0; w < kNW; ++w) {
    out[w] = n;
    #pragma unroll 1
    for (int dir = 1; dir >= -1; dir -= 2) {
      #pragma unroll 1
      for (int k = dir > 0 ? 0 : nsub - 1; dir > 0 ? k < nsub : k >= 0; k += dir) {
        const int Nk = mt.NE[k];
        if (w == 0) {
          const int Np = k >= 1 ? mt.NE[k - 1] : 0;
          if (dir > 0 && fwd_pair(S.panel_words, Np, Nk)) {  // panel k at block k-1 and the diagonal slot
            out[n++] = sdesc(mt.loff[k] + (long long)(mt.xoff[k] - Np - mt.xoff[jlo_of(k, Sx)]) * Nk, (Np + Nk) * Nk,
                             false);
            continue;
          }
          if (dir > 0 && k >= 1)  // panel k at block k-1: [g][c]
            out[n++] = sdesc(mt.loff[k] + (long long)(mt.xoff[k - 1] - mt.xoff[jlo_of(k, Sx)]) * Nk, Np * Nk, false);
          if (dir < 0 && k <= nsub - 2)  // panel k+1 at block k
            out[n++] = sdesc(mt.loff[k + 1] + (long long)(mt.xoff[k] - mt.xoff[jlo_of(k + 1, Sx)]) * mt.NE[k + 1],
                             Nk * mt.NE[k + 1], false);
          out[n++] = sdesc(mt.ioff[k] + (dir > 0 ? ((Nk * Nk + 3) & ~3) : 0), Nk * Nk, true);
          continue;
        }
        int c0, c1;
        warp_share(mt, Sx, nsub, w, k, &c0, &c1);
        if (c1 <= c0) continue;
        const int N2 = mt.NE[k + 1], pc = piece_cols(S.panel_words, N2);
        #pragma unroll 1
        for (int c = c0; c < c1; c += pc)
          out[n++] = sdesc(mt.loff[k + 1] + (long long)c * N2, (c1 - c < pc ? c1 - c : pc) * N2, false);
      }
    }
  }
  out[kNW] = n;
}

__global__ void k_sched(const SimDev* __restrict__ sp) {
  if (threadIdx.x == 0 && blockIdx.x == 0) build_sched(*sp, const_cast<unsigned long long*>(sp->sched));
}

// The warp's copy schedule, 32 descriptors at a time in registers (lane l
// holds descriptor base + l in cur and base + 32 + l in nxt).
struct SFeed {
  const unsigned long long* d;
  int n, next, base;
  unsigned long long cur, nxt;
  int withhold;  // chunk whose copy is withheld (test hook), or -1
};

__device__ __forceinline__ SFeed sfeed_open(const unsigned long long* sched, int w, int lane) {
  SFeed f;
  const long long s0 = (long long)sched[w], s1 = (long long)sched[w + 1];
  f.d = sched + s0;
  f.n = (int)(s1 - s0);
  f.next = 0;
  f.base = 0;
  f.cur = lane < f.n ? f.d[lane] : 0ull;
  f.nxt = 32 + lane < f.n ? f.d[32 + lane] : 0ull;
  f.withhold = -1;
  return f;
}

// Issue the warp's next chunks while they fit.
template <typename T>
__device__ __forceinline__ void srefill(WRing<T>& r, SFeed& f, const T* LT, const T* Linv, int lane) {
  #pragma unroll 1
  while (f.next < f.n) {
    if (f.next - f.base == 32) {
      f.cur = f.nxt;
      f.base += 32;
      const int j = f.base + 32 + lane;
      f.nxt = j < f.n ? f.d[j] : 0ull;
    }
    const unsigned long long dsc = __shfl_sync(0xffffffffu, f.cur, f.next - f.base);
    const T* src = (dsc & kDescInverse) ? Linv : LT;
    if (!wring_try_issue<T>(r, src, (long long)(dsc & kDescOffMask), (int)((dsc >> 40) & 0xffff), lane,
                            f.next == f.withhold))
      return;
    ++f.next;
  }
}

// sum_{g < K} P[g ld] v[g] (P already offset to the lane's column), four
// independent chains so that the shared-memory loads overlap.
template <typename T>
__device__ __forceinline__ T dot_col(const T* P, int ld, const T* v, int K) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int g = 0;
#pragma unroll 2
  for (; g + 3 < K; g += 4) {
    a0 = fma(P[g * ld], v[g], a0);
    a1 = fma(P[(g + 1) * ld], v[g + 1], a1);
    a2 = fma(P[(g + 2) * ld], v[g + 2], a2);
    a3 = fma(P[(g + 3) * ld], v[g + 3], a3);
  }
  if (g < K) {
    a0 = fma(P[g * ld], v[g], a0);
    if (g + 1 < K) a1 = fma(P[(g + 1) * ld], v[g + 1], a1);
    if (g + 2 < K) a2 = fma(P[(g + 2) * ld], v[g + 2], a2);
  }
  return (a0 + a1) + (a2 + a3);
}

// sum_{c < K} Pr[c] v[c] over the lane's own row Pr, starting at column c0
// and wrapping (lanes start at different columns: rows of even length K
// would otherwise fall into the same shared-memory banks); four chains.
template <typename T>
__device__ __forceinline__ T dot_row(const T* Pr, const T* v, int K, int c0) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int c = c0, u = 0;
#pragma unroll 2
  for (; u + 3 < K; u += 4) {
    const int c1 = c + 1 == K ? 0 : c + 1;
    const int c2 = c1 + 1 == K ? 0 : c1 + 1;
    const int c3 = c2 + 1 == K ? 0 : c2 + 1;
    a0 = fma(Pr[c], v[c], a0);
    a1 = fma(Pr[c1], v[c1], a1);
    a2 = fma(Pr[c2], v[c2], a2);
    a3 = fma(Pr[c3], v[c3], a3);
    c = c3 + 1 == K ? 0 : c3 + 1;
  }
  if (u < K) {
    const int c1 = c + 1 == K ? 0 : c + 1;
    const int c2 = c1 + 1 == K ? 0 : c1 + 1;
    a0 = fma(Pr[c], v[c], a0);
    if (u + 1 < K) a1 = fma(Pr[c1], v[c1], a1);
    if (u + 2 < K) a2 = fma(Pr[c2], v[c2], a2);
  }
  return (a0 + a1) + (a2 + a3);
}

// Wait for the warp's next chunk. Chunks are issued while they fit, at the
// start of each pass and at the end of each block row; a chunk not issued
// yet (the FIFO was full at the last refill) is issued here first, which it
// always can be: everything before it has been consumed and released.
template <typename T>
__device__ __forceinline__ const T* swait(WRing<T>& r, SFeed& f, const T* LT, const T* Linv, int lane) {
  if (r.consumed == r.issued) srefill<T>(r, f, LT, Linv, lane);
  return wring_wait<T>(r);
}

// Solve L L^T out = in with the transposed panels (arithmetic in T) by the
// CTA; y and z live in shared memory. Returns false if a copy did not complete.
template <typename T>
__device__ bool csubstitute(const SimDev& S, const T* LT, const T* Linv, const double* in, double* out,
                            CtaSmem<T>& m) {
  const SolveMeta& mt = m.mt;
  const int nsub = S.n_sub, Sx = S.Sx, N = S.N;
  const int lane = threadIdx.x & 31, w = vwarp();
  T* y = m.yz;
  T* z = y + N;
  T* tv = m.tv;
  // warp w's region of the panel and ring area: kPartWords partial-sum
  // elements (forward pass, two rows of 32), then its FIFO of chunks
  const int region = fifo_cap(S.panel_words) + kPartWords;
  T* part = m.R + (size_t)w * region;
  WRing<T> rg{part + kPartWords, fifo_cap(S.panel_words), w * kEnt, m.full, m.dl, m.epos, 0, 0, 0u, 0u, m.ph,
              m.used, m.fpar, true};
  #pragma unroll 1
  for (int i = threadIdx.x; i < N; i += kThreads) {
    y[i] = (T)in[i];
    z[i] = T(0);
  }
  SFeed fd = sfeed_open(S.sched, w, lane);
  // Test hook of the bounded waits: the leader withholds the last chunk of its
  // list. Every earlier chunk has been awaited by then, so when that one wait
  // runs out no copy is left in flight.
  if (w == 0 && S.inject && S.inject[0] != 0) fd.withhold = fd.n - 1;
  srefill<T>(rg, fd, LT, Linv, lane);
  __syncthreads();
  // forward, y_k = L_kk^-1 (in_k - sum_{j<k} L_kj y_j): at step k the leader
  // finishes row k with the partial sums the other warps formed for it at
  // step k-1 and the block L_{k,k-1}; meanwhile the other warps form row
  // k+1's sums over blocks jlo(k+1)..k-1 (y of those blocks is known)
  #pragma unroll 1
  for (int k = 0; k < nsub; ++k) {
    const int Nk = mt.NE[k], xk = mt.xoff[k];
    if (w == 0) {
      T t = (lane < Nk) ? y[xk + lane] : T(0);
      const int Nj = k >= 1 ? mt.NE[k - 1] : 0;
      const bool pair = fwd_pair(S.panel_words, Nj, Nk);
      const T* P = (k >= 1 || pair) ? swait<T>(rg, fd, LT, Linv, lane) : nullptr;  // [g][c] (and the slot)
      if (k >= 1) {
        const int h = (k & 1) * 32 + lane;
        if (lane < Nk) t -= (m.R[(size_t)region + h] + m.R[2 * (size_t)region + h]) + m.R[3 * (size_t)region + h];
        if (lane < Nk) t -= dot_col<T>(P + lane, Nk, y + mt.xoff[k - 1], Nj);
      }
      if (lane < Nk) tv[lane] = t;
      __syncwarp();
      const T* LiT = pair ? P + Nj * Nk : nullptr;
      if (!pair) {
        if (k >= 1) wring_release<T>(rg);
        LiT = swait<T>(rg, fd, LT, Linv, lane);
      }
      // y_k[c] = sum_{t <= c} Linv[c][t] tv[t] (the stored inverse holds its zeros)
      const T yk = lane < Nk ? dot_col<T>(LiT + lane, Nk, tv, Nk) : T(0);
      wring_release<T>(rg);
      if (lane < Nk) y[xk + lane] = yk;
    } else if (k + 1 < nsub) {
      int c0, c1;
      warp_share(mt, Sx, nsub, w, k, &c0, &c1);
      const int N2 = mt.NE[k + 1], pc = piece_cols(S.panel_words, N2);
      const T* yb = y + mt.xoff[jlo_of(k + 1, Sx)];
      T acc = T(0);
      #pragma unroll 1
      for (int c = c0; c < c1; c += pc) {
        const T* P = swait<T>(rg, fd, LT, Linv, lane);  // columns c.. of panel k+1, [c][g]
        if (lane < N2) acc += dot_col<T>(P + lane, N2, yb + c, min(pc, c1 - c));
        wring_release<T>(rg);
      }
      if (lane < N2) part[((k + 1) & 1) * 32 + lane] = acc;  // zero for an empty share
    }
    srefill<T>(rg, fd, LT, Linv, lane);
    __syncthreads();
  }
  // backward, z_k = L_kk^-T (y_k - sum_{k'>k} L_k'k^T z_k'): at step k, with
  // z_{k+1} known, the leader applies L_{k+1,k}^T z_{k+1} to row k and
  // finishes it, the other warps apply L_{k+1,j}^T z_{k+1} to their columns of
  // blocks jlo(k+1)..k-1 (the feed runs on into the backward chunks)
  srefill<T>(rg, fd, LT, Linv, lane);
  #pragma unroll 1
  for (int k = nsub - 1; k >= 0; --k) {
    const int Nk = mt.NE[k], xk = mt.xoff[k];
    if (w == 0) {
      if (k <= nsub - 2) {  // p_k += L_{k+1,k}^T z_{k+1}
        const int N2 = mt.NE[k + 1];
        const T* P = swait<T>(rg, fd, LT, Linv, lane);  // [g][c]: g in block k, c in block k+1
        const T* zn = z + mt.xoff[k + 1];
        if (lane < Nk) z[xk + lane] += dot_row<T>(P + lane * N2, zn, N2, (N2 & 1) ? 0 : lane % N2);
        wring_release<T>(rg);
      }
      const T* Li = swait<T>(rg, fd, LT, Linv, lane);
      if (lane < Nk) tv[lane] = y[xk + lane] - z[xk + lane];
      __syncwarp();
      // z_k[c] = sum_{r >= c} Linv[r][c] tv[r] (zeros stored above the diagonal)
      const T zc = lane < Nk ? dot_col<T>(Li + lane, Nk, tv, Nk) : T(0);
      wring_release<T>(rg);
      if (lane < Nk) z[xk + lane] = zc;
    } else if (k + 1 < nsub) {
      int c0, c1;
      warp_share(mt, Sx, nsub, w, k, &c0, &c1);
      const int N2 = mt.NE[k + 1], pc = piece_cols(S.panel_words, N2);
      const T* zn = z + mt.xoff[k + 1];
      T* zb = z + mt.xoff[jlo_of(k + 1, Sx)];
      #pragma unroll 1
      for (int c = c0; c < c1; c += pc) {
        const int nc = min(pc, c1 - c);
        const T* P = swait<T>(rg, fd, LT, Linv, lane);  // columns c.. of panel k+1, [c][g]
        #pragma unroll 1
        for (int u = lane; u < nc; u += 32) zb[c + u] += dot_row<T>(P + u * N2, zn, N2, (N2 & 1) ? 0 : u % N2);
        wring_release<T>(rg);
      }
    }
    srefill<T>(rg, fd, LT, Linv, lane);
    __syncthreads();
  }
  #pragma unroll 1
  for (int i = threadIdx.x; i < N; i += kThreads) out[i] = (double)z[i];
  if (!rg.ok) m.flag[1] = 1;
  m.ph = rg.ph;
  m.used = rg.used;
  m.fpar = rg.fpar;
  __syncthreads();
  if (m.flag[1]) {
    if (lane == 0)  // bounded wait for the warp's copies still in flight
      #pragma unroll 1
      for (int b = rg.b0; b < rg.b0 + kEnt; ++b)
        if (rg.used & (1u << b)) mbar_wait(&rg.full[b], ((~rg.fpar) >> b) & 1u);
    if (threadIdx.x == 0 && S.inject) S.inject[0] = 0;  // the hook fires once
    __syncthreads();
    return false;
  }
  return true;
}

// acc += sum_{c < n} a[c * sa] xs[c * sx] with four chains (FP64).
__device__ __noinline__ double dot_strided(const double* __restrict__ a, int sa, const double* xs, int sx, int n,
                                           double acc) {
  double a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = 0;
  #pragma unroll 1
  for (; c + 3 < n; c += 4) {
    acc = fma(a[c * sa], xs[c * sx], acc);
    a1 = fma(a[(c + 1) * sa], xs[(c + 1) * sx], a1);
    a2 = fma(a[(c + 2) * sa], xs[(c + 2) * sx], a2);
    a3 = fma(a[(c + 3) * sa], xs[(c + 3) * sx], a3);
  }
  #pragma unroll 1
  for (; c < n; ++c) acc = fma(a[c * sa], xs[c * sx], acc);
  return (acc + a1) + (a2 + a3);
}

// r = b - A x (r = A x when b is null) with the block-sparse assembled A, in
// FP64, by the CTA; x is staged in the shared work area xs [N]. One thread
// per row (rows g = threadIdx.x, + kThreads, ...; the row's subdomain by
// binary search in xoff), so that every lane of a warp issues its FP64 FMAs
// (rows of neighbouring subdomains share a warp): GB300's FP64 pipe bounds
// this product. Row i of subdomain E sums, in this order, its diagonal block
// (read down column i: the block is symmetric, and column i's elements are
// consecutive across the threads of consecutive rows), the left and lower
// couplings (stored [N_j][N_E]: column i, consecutive across rows) and the
// right and upper ones (stored [N_E][N_j]: row i).
__device__ void cresidual(const SimDev& S, const SolveMeta& mt, const double* x, const double* b, double* r,
                          double* xs) {
  const int Sx = S.Sx, Sy = S.Sy, nsub = S.n_sub;
  #pragma unroll 1
  for (int i = threadIdx.x; i < S.N; i += kThreads) xs[i] = x[i];
  __syncthreads();
  #pragma unroll 1
  for (int g = threadIdx.x; g < S.N; g += kThreads) {
    int lo = 0, hi = nsub;  // xoff[lo] <= g < xoff[hi]
    #pragma unroll 1
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (mt.xoff[mid] <= g) lo = mid;
      else hi = mid;
    }
    const int E = lo, NE = mt.NE[E], i = g - mt.xoff[E];
    const int I = E % Sx, J = E / Sx;
    double acc = dot_strided(S.A + S.aoff[E] + i, NE, xs + mt.xoff[E], 1, NE, 0.0);
    if (I > 0) {
      const int j = E - 1;
      acc = dot_strided(S.A + S.aoff[nsub + J * (Sx - 1) + (I - 1)] + i, NE, xs + mt.xoff[j], 1, mt.NE[j], acc);
    }
    if (J > 0) {
      const int j = E - Sx;
      acc = dot_strided(S.A + S.aoff[nsub + Sy * (Sx - 1) + (J - 1) * Sx + I] + i, NE, xs + mt.xoff[j], 1, mt.NE[j],
                        acc);
    }
    if (I < Sx - 1) {
      const int j = E + 1, Nj = mt.NE[j];
      acc = dot_strided(S.A + S.aoff[nsub + J * (Sx - 1) + I] + (size_t)i * Nj, 1, xs + mt.xoff[j], 1, Nj, acc);
    }
    if (J < Sy - 1) {
      const int j = E + Sx, Nj = mt.NE[j];
      acc = dot_strided(S.A + S.aoff[nsub + Sy * (Sx - 1) + J * Sx + I] + (size_t)i * Nj, 1, xs + mt.xoff[j], 1, Nj,
                        acc);
    }
    r[g] = b ? b[g] - acc : acc;
  }
  __syncthreads();
}

// max over the CTA of v (every thread passes its partial); red: [kNW] doubles.
__device__ __forceinline__ double cta_max(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = red[0];
#pragma unroll
  for (int u = 1; u < kNW; ++u) r = fmax(r, red[u]);
  __syncthreads();
  return r;
}

// sum over the CTA of v in a fixed order (bitwise reproducible); red: [kNW] doubles.
__device__ __forceinline__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = red[0];
#pragma unroll
  for (int u = 1; u < kNW; ++u) r += red[u];
  __syncthreads();
  return r;
}

// x = (L L^T)^-1 b, then up to `iters` refinement steps x += (L L^T)^-1 (b - A x)
// with the residual in FP64 (max norms throughout; ||dv_0|| := ||x_0||). The
// refinement stops
//  - converged: once the next correction, predicted from the contraction of
//    the last two, ||dv_k|| min(1, ||dv_k|| / ||dv_{k-1}||), is below
//    kRefineTol ||x||;
//  - at the rounding floor: once a correction no longer halves and is below
//    kFloorTol ||x||;
//  - stalled: a correction that no longer halves above that level (the
//    factor is too inexact for this matrix; the FP32 kernel then hands the
//    simulation to the FP64 one).
// Returns kRefOk, kRefStalled or kRefTimeout (a copy did not complete). The
// warm-started mixed solve uses csolve_pcg instead.
// Per-simulation solve bookkeeping (S.info, ints): [0] correction passes of
// the last solve, [1] FP64 redos, [2] FP32 factorisations, [3] refactorings
// forced by a stale factor that did not converge, [4] correction passes,
// [5] reduced solves (all since load), [6] the FP32 factor's state: 0 none,
// a >= 1 computed a - 1 steps ago, [7] refactor at the next step, [8] the
// FP32 buffer holding the current factor (0 or 1), [9] 1 if the current
// factor was built in stages.
constexpr int kInfoPasses = 0, kInfoRedo64 = 1, kInfoFactors = 2, kInfoStaleRetry = 3, kInfoPassSum = 4,
              kInfoSolves = 5, kInfoAge = 6, kInfoRefactor = 7, kInfoBuf = 8, kInfoStaged = 9;
constexpr double kRefineTol = 1e-12;
// The conjugate gradients stop tighter: their error is not the rounding noise
// of a direct solve but a systematic remainder, which a 50-step trajectory of
// a 32x32 case carried to 1.5e-10 relative (6x the disagreement of two FP64
// direct solvers) at 1e-12.
constexpr double kCgTol = 2.5e-13;
constexpr double kFloorTol = 1e-8;
constexpr int kRefOk = 0, kRefStalled = 1, kRefTimeout = 2, kRefNotConverged = 3;

template <typename T>
__device__ int csolve_refine(const SimDev& S, const T* Lst, const T* Linv, int iters, CtaSmem<T>& m) {
  double* red = reinterpret_cast<double*>(m.part);  // [kNW] doubles (part is free between passes)
  double prev = 0.0;
  int steps = 0, rc = kRefOk;
  // pass 0 solves for x, pass it >= 1 for the correction dv of refinement
  // step it (one substitution call site keeps the kernel's code small)
#pragma unroll 1
  for (int it = 0; it <= iters; ++it) {
    const bool corr = it > 0;
    if (corr) cresidual(S, m.mt, S.x, S.b, S.rv, reinterpret_cast<double*>(m.yz));
    if (!csubstitute<T>(S, Lst, Linv, corr ? S.rv : S.b, corr ? S.dv : S.x, m)) return kRefTimeout;
    double mdv = 0.0, mx = 0.0;
#pragma unroll 1
    for (int i = threadIdx.x; i < S.N; i += kThreads) {
      double xi = S.x[i];
      if (corr) {
        xi += S.dv[i];
        S.x[i] = xi;
        mdv = fmax(mdv, fabs(S.dv[i]));
      }
      mx = fmax(mx, fabs(xi));
    }
    mdv = cta_max(mdv, red);
    mx = cta_max(mx, red);
    if (!corr) {
      prev = mx;
      continue;
    }
    steps = it;
    const double pred = mdv * fmin(1.0, mdv / prev);
    if (!(pred > kRefineTol * mx)) {  // converged (also on 0/0)
      rc = kRefOk;
      break;
    }
    if (mdv > 0.5 * prev) {
      rc = mdv > kFloorTol * mx ? kRefStalled : kRefOk;
      break;
    }
    prev = mdv;
  }
  if (threadIdx.x == 0 && S.info) {
    S.info[kInfoPasses] = steps;
    S.info[kInfoPassSum] += steps + 1;  // every substitution pass
  }
  return rc;
}

// Warm-started preconditioned conjugate gradients in FP64 with the FP32
// Cholesky factor L L^T (of this step or an earlier one) as the
// preconditioner: from the guess x, r = b - A x; then per pass
// z = (L L^T)^-1 r, rho = r.z, p = z + (rho / rho_prev) p (p = z first),
// q = A p, alpha = rho / p.q, x += alpha p, r -= alpha q. A changes between
// steps only through the fitted mobility coefficients, so the spectrum of
// (L L^T)^-1 A stays clustered near 1 and the iteration needs fewer passes
// than plain refinement (x += (L L^T)^-1 (b - A x)), most of all with a
// stale factor. Stops like csolve_refine, at kCgTol (the correction alpha p
// in max norm, predicted from the last two; the first accepted only if itself
// below kCgTol ||x||) after at most iters + 1 passes. Returns kRefOk,
// kRefTimeout, kRefStalled (p.q or r.z not positive: the preconditioned
// operator is not positive definite in this precision) or kRefNotConverged.
// Work vectors: S.rv (r), S.dv (z), S.pv (p), S.qv (q).
template <typename T>
__device__ int csolve_pcg(const SimDev& S, const T* Lst, const T* Linv, int iters, CtaSmem<T>& m) {
  double* red = reinterpret_cast<double*>(m.part);  // [kNW] doubles (part is free between passes)
  double* xs = reinterpret_cast<double*>(m.yz);
  cresidual(S, m.mt, S.x, S.b, S.rv, xs);
  double rho = 0.0, prev = 0.0;
  int steps = 0, rc = kRefNotConverged;
#pragma unroll 1
  for (int it = 0; it <= iters; ++it) {
    if (!csubstitute<T>(S, Lst, Linv, S.rv, S.dv, m)) return kRefTimeout;
    double acc = 0.0;
#pragma unroll 1
    for (int i = threadIdx.x; i < S.N; i += kThreads) acc = fma(S.rv[i], S.dv[i], acc);
    const double rn = cta_sum(acc, red);
    if (!(rn > 0.0)) {  // r = 0: x is exact; otherwise not positive definite
      rc = rn == 0.0 ? kRefOk : kRefStalled;
      break;
    }
    const double beta = it == 0 ? 0.0 : rn / rho;
    rho = rn;
#pragma unroll 1
    for (int i = threadIdx.x; i < S.N; i += kThreads) S.pv[i] = it == 0 ? S.dv[i] : fma(beta, S.pv[i], S.dv[i]);
    __syncthreads();
    cresidual(S, m.mt, S.pv, nullptr, S.qv, xs);
    acc = 0.0;
#pragma unroll 1
    for (int i = threadIdx.x; i < S.N; i += kThreads) acc = fma(S.pv[i], S.qv[i], acc);
    const double pq = cta_sum(acc, red);
    steps = it + 1;
    if (!(pq > 0.0) || !(pq < INFINITY)) {
      rc = kRefStalled;
      break;
    }
    const double al = rho / pq;
    double mdv = 0.0, mx = 0.0;
#pragma unroll 1
    for (int i = threadIdx.x; i < S.N; i += kThreads) {
      const double d = al * S.pv[i];
      const double xi = S.x[i] + d;
      S.x[i] = xi;
      S.rv[i] = fma(-al, S.qv[i], S.rv[i]);
      mdv = fmax(mdv, fabs(d));
      mx = fmax(mx, fabs(xi));
    }
    mdv = cta_max(mdv, red);
    mx = cta_max(mx, red);
    const double pred = it == 0 ? mdv : mdv * fmin(1.0, mdv / prev);
    if (!(pred > kCgTol * mx)) {
      rc = kRefOk;
      break;
    }
    prev = mdv;
  }
  if (threadIdx.x == 0 && S.info) {
    S.info[kInfoPasses] = steps;
    S.info[kInfoPassSum] += steps;
  }
  return rc;
}

constexpr int kStRetry64 = 1;  // transient status: redo this simulation's solve in FP64
constexpr int kStRetry32 = 2;  // transient status: refactor in FP32 now and solve again

// The FP32 factor of an earlier step serves as the preconditioner of the
// conjugate gradients (A changes only through the fitted mobility
// coefficients, so the factor of a nearby step still clusters the spectrum
// near 1) for refactor_period steps; then
// the simulation refactors. Simulations loaded together therefore refactor on
// the same steps, which keeps the refinement passes of a launch even (a
// launch lasts as long as its slowest simulation). A step that needs more than
// kRefactorPasses passes also refactors at the next step. The warm solve
// gets at most kStalePasses passes (or refine_iters + 1 if more);
// a stale factor that has not converged by then, or stalls, is recomputed at
// once (kStRetry32); a fresh one hands the solve to FP64.
constexpr int kRefactorPasses = 10;
constexpr int kStalePasses = 12;

// Staged refactorisation (refactor_stages R > 1): the next factor is built
// in the idle FP32 buffer over the last R steps of the current one's period,
// a contiguous range of about n_sub / R block rows per step, each row from
// that step's matrix (the lower triangular result with a positive diagonal
// is still a symmetric positive definite preconditioner). The build's last
// stage runs when the current factor expires (age refactor_period + 1) and
// the solve of that step already uses the new factor. So no step pays a whole
// factorisation; the price is a factor whose early rows are up to R - 1 steps
// older. A fresh factor (age 0, or a refactorisation forced by a slow or
// failed solve) is still computed whole, in the current buffer.
struct FactorPlan {
  int k0, k1;  // block rows to compute (k1 <= k0: none)
  int buf;     // FP32 buffer written
  bool whole, last_stage;
};

__host__ __device__ __forceinline__ FactorPlan factor_plan(const SimDev& S, const volatile int* info) {
  const int age = info[kInfoAge], P = S.refactor_period, R = S.refactor_stages;
  const int cur = info[kInfoBuf] & 1;
  FactorPlan p{0, 0, cur, false, false};
  if (age == 0 || info[kInfoRefactor] != 0 || (R <= 1 && age > P)) {
    p.k1 = S.n_sub;
    p.whole = true;
    return p;
  }
  if (R <= 1) return p;
  const int st = age - (P - R + 2);  // stage of the build in progress
  if (st < 0) return p;
  if (st >= R) {  // past the period without a completed build: whole, now
    p.k1 = S.n_sub;
    p.whole = true;
    return p;
  }
  p.k0 = (int)((long long)S.n_sub * st / R);
  p.k1 = (int)((long long)S.n_sub * (st + 1) / R);
  p.buf = cur ^ 1;
  p.last_stage = st == R - 1;
  return p;
}

// The two FP32 factor buffers of the mixed solver share the FP64 factor's
// storage (8 bytes per element): buffer 1 starts after buffer 0's elements.
__device__ __forceinline__ float* fac32_lt(const SimDev& S, const SolveMeta& mt, int buf) {
  return reinterpret_cast<float*>(S.L) + (buf ? mt.loff[S.n_sub] : 0);
}
__device__ __forceinline__ float* fac32_inv(const SimDev& S, const SolveMeta& mt, int buf) {
  return reinterpret_cast<float*>(S.Linv) + (buf ? mt.ioff[S.n_sub] : 0);
}

// Initial guess of the warm solve: the quadratic extrapolation
// 3 x^n - 3 x^{n-1} + x^{n-2} of the last three solutions once there are
// three, the linear 2 x^n - x^{n-1} once there are two (xp and xpp keep the
// two before x^n). A CPU emulation at the 8x8-subdomain bench shape put the
// guess's median error at 3e-6 (quadratic) against 1.6e-5 (linear), and the
// conjugate gradients at 3.3 against 3.9 passes.
__device__ void extrapolate_guess(const SimDev& S) {
  const int ns = S.info[kInfoSolves];
  #pragma unroll 1
  for (int i = threadIdx.x; i < S.N; i += kThreads) {
    const double xn = S.x[i], x1 = S.xp[i];
    if (ns >= 3) S.x[i] = 3.0 * (xn - x1) + S.xpp[i];
    else if (ns >= 2) S.x[i] = 2.0 * xn - x1;
    S.xpp[i] = x1;
    S.xp[i] = xn;
  }
  __syncthreads();
}

// FP32 factorisation of the simulations that need one this step (no factor
// yet, or marked by the last step's refinement). A non-positive pivot hands
// the simulation to the FP64 kernel.
__global__ void __launch_bounds__(kThreads, 4) k_factor32(const SimDev* __restrict__ sims,
                                                          const int* __restrict__ active, int n_active) {
  const int a = blockIdx.x;
  if (a >= n_active) return;
  const SimDev& S = sims[active[a]];
  if (S.status[0] != kStOk) return;
  int buf;
  {
    const FactorPlan p = factor_plan(S, S.info);
    if (p.k1 <= p.k0 && !p.last_stage) return;
    buf = p.buf;
  }
  extern __shared__ double sm[];
  unsigned char* b = reinterpret_cast<unsigned char*>(sm);
  CtaSmem<float> m = cta_carve_and_load<float>(S, b);
  if (threadIdx.x == 0) {
    const FactorPlan p = factor_plan(S, S.info);
    m.flag[2] = p.k0;  // block rows of this step (an empty range computes nothing)
    m.flag[3] = p.k1;
  }
  __syncthreads();
  const int f = cfactor_mma(S, fac32_lt(S, m.mt, buf), fac32_inv(S, m.mt, buf), m);
  if (threadIdx.x == 0) {
    // S.info is unchanged until here: the plan is read again (volatile: not
    // kept in registers through the factorisation).
    const FactorPlan p = factor_plan(S, S.info);
    if (p.whole) {
      if (f == kFacOk) {
        S.info[kInfoFactors] += 1;
        S.info[kInfoAge] = 1;
        S.info[kInfoRefactor] = 0;
        S.info[kInfoStaged] = 0;
      } else {
        S.info[kInfoAge] = 0;
        S.status[0] = f == kFacPivot ? kStRetry64 : kStTimeout;
      }
    } else if (f == kFacTimeout) {
      S.status[0] = kStTimeout;
    } else if (f == kFacPivot) {
      S.info[kInfoRefactor] = 1;  // abandon the build: a whole factorisation at the next step
    } else if (p.last_stage) {  // the build is complete: it serves from this step's solve on
      S.info[kInfoBuf] = p.buf;
      S.info[kInfoFactors] += 1;
      S.info[kInfoAge] = 1;
      S.info[kInfoStaged] = 1;
    }
  }
}

// Warm-started refinement with the current FP32 factor (fresh or stale).
__global__ void __launch_bounds__(kThreads, 4) k_refine32(const SimDev* __restrict__ sims,
                                                          const int* __restrict__ active, int n_active, int iters) {
  const int a = blockIdx.x;
  if (a >= n_active) return;
  const SimDev& S = sims[active[a]];
  if (S.status[0] != kStOk) return;
  extern __shared__ double sm[];
  unsigned char* b = reinterpret_cast<unsigned char*>(sm);
  CtaSmem<float> m = cta_carve_and_load<float>(S, b);
  const bool fresh = S.info[kInfoAge] == 1 && S.info[kInfoStaged] == 0;  // a staged build counts as stale
  const int budget = max(iters, kStalePasses - 1);
  extrapolate_guess(S);
  const int cur = S.info[kInfoBuf] & 1;
  const int r = csolve_pcg<float>(S, fac32_lt(S, m.mt, cur), fac32_inv(S, m.mt, cur), budget, m);
  if (threadIdx.x == 0) {
    if (r == kRefOk) {
      S.info[kInfoSolves] += 1;
      S.info[kInfoAge] += 1;
      if (S.info[kInfoPasses] > kRefactorPasses) S.info[kInfoRefactor] = 1;
    } else if (r == kRefTimeout) {
      S.status[0] = kStTimeout;
    } else {
      S.status[0] = fresh ? kStRetry64 : kStRetry32;
    }
  }
}

// A stale factor that did not converge: refactor in FP32 now and solve from
// scratch (cold start); a failure there hands the simulation to FP64.
__global__ void __launch_bounds__(kThreads) k_retry32(const SimDev* __restrict__ sims,
                                                      const int* __restrict__ active, int n_active, int iters) {
  const int a = blockIdx.x;
  if (a >= n_active) return;
  const SimDev& S = sims[active[a]];
  if (S.status[0] != kStRetry32) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    S.status[0] = kStOk;
    S.info[kInfoStaleRetry] += 1;
  }
  extern __shared__ double sm[];
  unsigned char* b = reinterpret_cast<unsigned char*>(sm);
  CtaSmem<float> m = cta_carve_and_load<float>(S, b);
  const int cur = S.info[kInfoBuf] & 1;
  float* Lf = fac32_lt(S, m.mt, cur);
  float* Lif = fac32_inv(S, m.mt, cur);
  const int f = cfactor_mma(S, Lf, Lif, m);
  if (f != kFacOk) {
    if (threadIdx.x == 0) {
      S.info[kInfoAge] = 0;
      S.status[0] = f == kFacPivot ? kStRetry64 : kStTimeout;
    }
    return;
  }
  const int r = csolve_refine<float>(S, Lf, Lif, iters, m);
  if (threadIdx.x == 0) {
    S.info[kInfoFactors] += 1;
    S.info[kInfoAge] = 2;  // computed this step, and served it
    S.info[kInfoRefactor] = 0;
    S.info[kInfoStaged] = 0;
    if (r == kRefTimeout) S.status[0] = kStTimeout;
    else if (r != kRefOk) S.status[0] = kStRetry64;
    else S.info[kInfoSolves] += 1;
  }
}

// FP64 factor. only_retry: process only the simulations marked by the FP32 kernel.
__global__ void __launch_bounds__(kThreads) k_csolve64(const SimDev* __restrict__ sims,
                                                       const int* __restrict__ active, int n_active, int iters,
                                                       int only_retry) {
  const int a = blockIdx.x;
  if (a >= n_active) return;
  const SimDev& S = sims[active[a]];
  const int st = S.status[0];
  if (only_retry ? st != kStRetry64 : st != kStOk) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    S.status[0] = kStOk;
    if (only_retry && S.info) {
      S.info[kInfoRedo64] += 1;
      S.info[kInfoAge] = 0;  // the FP64 factor overwrites the FP32 one
      S.info[kInfoRefactor] = 0;
    }
  }
  extern __shared__ double sm[];
  unsigned char* b = reinterpret_cast<unsigned char*>(sm);
  CtaSmem<double> m = cta_carve_and_load<double>(S, b);
  const int f = cfactor<double>(S, S.L, S.Linv, m);
  if (f != kFacOk) {
    if (threadIdx.x == 0) S.status[0] = f == kFacPivot ? kStNotSpd : kStTimeout;
    return;
  }
  const int r = csolve_refine<double>(S, S.L, S.Linv, iters, m);
  if (threadIdx.x == 0) {
    if (r == kRefTimeout) S.status[0] = kStTimeout;
    else if (S.info) S.info[kInfoSolves] += 1;
  }
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
  #pragma unroll 1
  for (int E = 0; E < S.n_sub; ++E) xoff[E + 1] = xoff[E] + NE[E];
  aoff[0] = 0;
  #pragma unroll 1
  for (int E = 0; E < S.n_sub; ++E) aoff[E + 1] = aoff[E] + (long long)NE[E] * NE[E];
  int b = S.n_sub;
  #pragma unroll 1
  for (int J = 0; J < S.Sy; ++J)
    #pragma unroll 1
    for (int I = 0; I + 1 < S.Sx; ++I, ++b) aoff[b + 1] = aoff[b] + (long long)NE[J * S.Sx + I] * NE[J * S.Sx + I + 1];
  #pragma unroll 1
  for (int J = 0; J + 1 < S.Sy; ++J)
    #pragma unroll 1
    for (int I = 0; I < S.Sx; ++I, ++b) aoff[b + 1] = aoff[b] + (long long)NE[J * S.Sx + I] * NE[(J + 1) * S.Sx + I];
  loff[0] = 0;
  ioff[0] = 0;
  solve_offsets(S.n_sub, S.Sx, NE, xoff, loff, ioff);
  build_sched(S, const_cast<unsigned long long*>(S.sched));
  S.status[0] = kStOk;
}

// A solution with a NaN or Inf entry (from a non-finite right-hand side) is
// reported as such rather than as a converged solve.
__device__ void mark_nonfinite_solution(const SimDev& S) {
  bool bad = false;
  #pragma unroll 1
  for (int i = threadIdx.x; i < S.N; i += kThreads) bad |= !isfinite(S.x[i]);
  if (__syncthreads_or(bad ? 1 : 0) && threadIdx.x == 0 && S.status[0] == kStOk) S.status[0] = kStNonFinite;
}

__global__ void __launch_bounds__(kThreads) k_csolve_static(SimDev S, int mode, int iters) {
  extern __shared__ double sm[];
  unsigned char* b = reinterpret_cast<unsigned char*>(sm);
  if (mode == 1) {
    float* Lf = reinterpret_cast<float*>(S.L);
    float* Lif = reinterpret_cast<float*>(S.Linv);
    CtaSmem<float> mf = cta_carve_and_load<float>(S, b);
    const int f = cfactor_mma(S, Lf, Lif, mf);
    if (f == kFacOk) {
      const int r = csolve_refine<float>(S, Lf, Lif, iters, mf);
      if (r == kRefTimeout && threadIdx.x == 0) S.status[0] = kStTimeout;
      if (r != kRefStalled) {
        __syncthreads();
        mark_nonfinite_solution(S);
        return;
      }
    }
    if (f == kFacTimeout) {
      if (threadIdx.x == 0) S.status[0] = kStTimeout;
      return;
    }
    cta_release_barriers(mf.full);
  }
  CtaSmem<double> md = cta_carve_and_load<double>(S, b);
  const int f = cfactor<double>(S, S.L, S.Linv, md);
  if (f != kFacOk) {
    if (threadIdx.x == 0) S.status[0] = f == kFacPivot ? kStNotSpd : kStTimeout;
    return;
  }
  if (csolve_refine<double>(S, S.L, S.Linv, iters, md) == kRefTimeout && threadIdx.x == 0) S.status[0] = kStTimeout;
  __syncthreads();
  mark_nonfinite_solution(S);
}

}  // namespace

// threads: CTA size (a multiple of 32, at least 32); every size computes each
// entry of A and b the same way, so the choice does not change the result.
void launch_assemble(const SimDev* sims, const int* active, int n_active, int max_blocks,
                     int mixed, cudaStream_t st, int threads) {
  k_theta<<<n_active, 32, 0, st>>>(sims, active);
  if (mixed)
    k_assemble32<<<dim3(max_blocks, n_active), threads, 0, st>>>(sims, active);
  else
    k_assemble<<<dim3(max_blocks, n_active), threads, 0, st>>>(sims, active);
}

void launch_sched(const SimDev* sim, cudaStream_t st) { k_sched<<<1, 32, 0, st>>>(sim); }

size_t solve_smem_bytes(int n_sub, int panel_words, int max_w, int N, size_t elem) {
  (void)max_w;
  return warp_smem_bytes(n_sub, panel_words, N, elem);
}

static cudaError_t set_smem(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Dynamic shared-memory limits of the solve kernels for a launch shape (set
// before a launch, and before a stream capture of one).
cudaError_t prepare_chol_solve(int mode, const SolveShape& sh) {
  cudaError_t e;
  if (mode == 1) {
    const size_t s32 = warp_smem_bytes(sh.n_sub, sh.panel_words, sh.N, sizeof(float));
    if ((e = set_smem((const void*)k_factor32, s32)) != cudaSuccess) return e;
    if ((e = set_smem((const void*)k_refine32, s32)) != cudaSuccess) return e;
    if ((e = set_smem((const void*)k_retry32, s32)) != cudaSuccess) return e;
  }
  const size_t s64 = warp_smem_bytes(sh.n_sub, sh.panel_words, sh.N, sizeof(double));
  return set_smem((const void*)k_csolve64, s64);
}

// One CTA of kNW warps per simulation; the CTAs spread over the SMs, as many
// per SM as their shared memory allows (attributes from prepare_chol_solve).
cudaError_t launch_factor32(const SimDev* sims, const int* active, int n_active, const SolveShape& sh,
                            cudaStream_t st) {
  if (n_active <= 0) return cudaSuccess;
  const size_t s32 = warp_smem_bytes(sh.n_sub, sh.panel_words, sh.N, sizeof(float));
  k_factor32<<<n_active, kThreads, s32, st>>>(sims, active, n_active);
  return cudaGetLastError();
}

cudaError_t launch_chol_solve(const SimDev* sims, const int* active, int n_active, int mode, int iters,
                              const SolveShape& sh, cudaStream_t st) {
  if (n_active <= 0) return cudaSuccess;
  if (mode == 1) {
    const size_t s32 = warp_smem_bytes(sh.n_sub, sh.panel_words, sh.N, sizeof(float));
    k_factor32<<<n_active, kThreads, s32, st>>>(sims, active, n_active);
    k_refine32<<<n_active, kThreads, s32, st>>>(sims, active, n_active, iters);
    k_retry32<<<n_active, kThreads, s32, st>>>(sims, active, n_active, iters);
  }
  const size_t s64 = warp_smem_bytes(sh.n_sub, sh.panel_words, sh.N, sizeof(double));
  k_csolve64<<<n_active, kThreads, s64, st>>>(sims, active, n_active, iters, mode == 1 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace lrbms

// ---------------------------------------------------------------- C ABI
#include "lrbms.h"

namespace {
constexpr int kMaxDevices = 64;
constexpr int kNoAllocMaxSub = 4096;
unsigned char* g_noalloc_dev[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int lrbms_test_factor_plan(int n_sub, int refactor_period, int refactor_stages, const int* info,
                                      int* out) {
  if (n_sub < 1 || refactor_period < 1 || refactor_stages < 1 || refactor_stages > refactor_period || !info || !out)
    return LRBMS_E_ARG;
  lrbms::SimDev S{};
  S.n_sub = n_sub;
  S.refactor_period = refactor_period;
  S.refactor_stages = refactor_stages;
  const lrbms::FactorPlan p = lrbms::factor_plan(S, info);
  out[0] = p.k0;
  out[1] = p.k1;
  out[2] = p.buf;
  out[3] = p.whole ? 1 : 0;
  out[4] = p.last_stage ? 1 : 0;
  return LRBMS_OK;
}

extern "C" int lrbms_solve_noalloc(int Sx, int Sy, const int* N_E, const double* A, const double* rhs,
                                   double* x, int solver, int refine_iters, void* stream) {
  using namespace lrbms;
  (void)cudaGetLastError();  // an error left pending by earlier work is not this call's
  if (Sx < 1 || Sy < 1 || !N_E || !A || !rhs || !x || refine_iters < 0 || refine_iters > 16 ||
      (solver != LRBMS_SOLVE_FP64 && solver != LRBMS_SOLVE_MIXED))
    return LRBMS_E_ARG;
  // the kernels dereference A, rhs and x on the device: host pointers are refused
  for (const void* p : {(const void*)A, (const void*)rhs, (const void*)x}) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      (void)cudaGetLastError();
      return LRBMS_E_ARG;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return LRBMS_E_ARG;
  }
  const int n_sub = Sx * Sy;
  const int n_cf = Sy * (Sx - 1) + (Sy - 1) * Sx;
  // sizes from the caller's (host) basis sizes; no host or device allocation
  long long N = 0, l_tot = 0, i_tot = 0;
  for (int E = 0; E < n_sub; ++E) {
    if (N_E[E] < 1 || N_E[E] > kMaxNE) return LRBMS_E_ARG;
    N += N_E[E];
    i_tot += 2 * (long long)round4((size_t)N_E[E] * N_E[E]);
  }
  // prefix sums on the stack (no allocation); n_sub is capped for this reason
  if (n_sub > kNoAllocMaxSub) return LRBMS_E_BUDGET;
  int xo[kNoAllocMaxSub + 1];
  xo[0] = 0;
  for (int E = 0; E < n_sub; ++E) xo[E + 1] = xo[E] + N_E[E];
  for (int k = 0; k < n_sub; ++k) l_tot += (long long)round4((size_t)N_E[k] * (xo[k + 1] - xo[jlo_of(k, Sx)]));
  int panel_words = 0, max_w = 0;
  solve_panel_sizes(n_sub, Sx, N_E, xo, &panel_words, &max_w);
  if (solve_smem_bytes(n_sub, panel_words, max_w, (int)N, sizeof(double)) > kMaxSolveSmem) return LRBMS_E_BUDGET;
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
  const size_t o_sched = off; off = up(off + 8 * sched_words(n_sub, Sx));
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
  S.sched = (const unsigned long long*)(base + o_sched);
  S.A = const_cast<double*>(A); S.b = const_cast<double*>(rhs); S.x = x;
  S.panel_words = panel_words;
  S.max_w = max_w;
  if (cudaMemcpyAsync(base + o_NE, N_E, 4 * (size_t)n_sub, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LRBMS_E_CUDA;
  k_noalloc_tables<<<1, 1, 0, st>>>(S);
  const int mode = solver == LRBMS_SOLVE_MIXED ? 1 : 0;
  const int iters = refine_iters > 0 ? refine_iters : (mode == 1 ? 6 : 1);
  const size_t smem = solve_smem_bytes(n_sub, panel_words, max_w, (int)N, sizeof(double));
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_csolve_static, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return LRBMS_E_BUDGET;
  k_csolve_static<<<1, kThreads, smem, st>>>(S, mode, iters);
  if (cudaGetLastError() != cudaSuccess) return LRBMS_E_CUDA;
  int status = 0;
  if (cudaMemcpyAsync(&status, base + o_status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LRBMS_E_CUDA;
  if (status == kStOk) return LRBMS_OK;
  if (status == kStTimeout) return LRBMS_E_TIMEOUT;
  if (status == kStNonFinite) return LRBMS_E_NONFINITE;
  return LRBMS_E_NOT_SPD;
}
