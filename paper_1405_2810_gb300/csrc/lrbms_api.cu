// Host side of the C ABI declared in include/lrbms.h: context, device-memory
// arena, slot table of resident simulations, offline-data loader and the
// driver that enqueues the kernels of one online step (Algorithm 3, step 5)
// for a batch of simulations.
#include "lrbms.h"
#include "lrbms_internal.cuh"

#include <algorithm>
#include <cmath>
#include <iterator>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

using lrbms::SimDev;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over one cudaMalloc'd arena; free blocks are merged.
class Arena {
 public:
  cudaError_t init(size_t cap) {
    cap_ = align_up(cap);
    cudaError_t e = cudaMalloc(&base_, cap_);
    if (e != cudaSuccess) {
      base_ = nullptr;
      return e;
    }
    free_[0] = cap_;
    return cudaSuccess;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  // Returns offset or SIZE_MAX.
  size_t alloc(size_t n) {
    n = align_up(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        size_t off = it->first, rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        used_ += n;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void free(size_t off, size_t n) {
    n = align_up(n);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return base_; }
  size_t used() const { return used_; }
  size_t cap() const { return cap_; }

 private:
  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Slot {
  bool used = false;
  bool prefactored = false;  // at rest, holding the FP32 factor of its current matrix
  size_t off = 0, bytes = 0;
  SimDev d{};
};

}  // namespace

struct lrbms_ctx {
  int device = 0;
  int precision = LRBMS_FP64;
  int solver = LRBMS_SOLVE_FP64;
  int refine_iters = 1;
  int refactor_period = 8;
  int refactor_stages = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t admit_stream = nullptr;  // admission copies and kernels (overlap the steps)
  int* d_status = nullptr;              // [max_slots] statuses of the last step, in list order
  int* h_status = nullptr;              // pinned copy
  int last_n = 0;                       // simulations of the last lrbms_step
  Arena arena;
  std::vector<Slot> slots;
  SimDev* d_sims = nullptr;
  int* d_active = nullptr;    // [max_slots + 1]: the step's list, then the admission stream's one entry
  std::vector<int> last_active;
  const double** d_io = nullptr;  // [2 * max_slots] saturation exchange pointers
  std::string err;
  long long launches = 0;
  // profiling of live steps
  int prof_cap = 0, prof_n = 0;
  std::vector<cudaEvent_t> prof_ev;
  // one online step of the current batch, captured as a CUDA graph; valid
  // while the batch (active list) and its launch shape stay the same
  cudaGraphExec_t graph = nullptr;
  std::vector<long long> graph_key;
  int graph_kernels = 0;
  // autotuned CTA sizes of assembly and reconstruction per shape class
  // (basis-size class, cells per subdomain, component precision)
  std::map<std::vector<int>, std::pair<int, int>> tuned;
};

namespace {

int fail(lrbms_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
int cuda_fail(lrbms_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LRBMS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

struct Layout {
  size_t total = 0;
  size_t add(size_t bytes) {
    size_t o = total;
    total = align_up(total + bytes);
    return o;
  }
};

bool valid_sim(lrbms_ctx* ctx, int id) {
  return ctx && id >= 0 && id < (int)ctx->slots.size() && ctx->slots[id].used;
}

}  // namespace

extern "C" {

int lrbms_create(lrbms_ctx** out, const lrbms_config* cfg) {
  if (!out || !cfg) return LRBMS_E_ARG;
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->hbm_budget == 0 || cfg->refine_iters < 0 || cfg->refine_iters > 16 ||
      cfg->refactor_period < 0 || cfg->refactor_period > 1000 || cfg->refactor_stages < 0 ||
      cfg->refactor_stages > (cfg->refactor_period > 0 ? cfg->refactor_period : 8) ||
      (cfg->precision != LRBMS_FP64 && cfg->precision != LRBMS_MIXED) ||
      (cfg->solver != LRBMS_SOLVE_FP64 && cfg->solver != LRBMS_SOLVE_MIXED))
    return LRBMS_E_ARG;
  lrbms_ctx* ctx = new lrbms_ctx();
  ctx->device = cfg->device;
  ctx->precision = cfg->precision;
  ctx->solver = cfg->solver;
  ctx->refine_iters = cfg->refine_iters > 0 ? cfg->refine_iters : (cfg->solver == LRBMS_SOLVE_MIXED ? 6 : 1);
  ctx->refactor_period = cfg->refactor_period > 0 ? cfg->refactor_period : 8;  // measured best at 512 sims
  ctx->refactor_stages = cfg->refactor_stages > 0 ? cfg->refactor_stages : 1;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    delete ctx;
    return LRBMS_E_CUDA;
  }
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return LRBMS_E_CUDA;
    }
    ctx->own_stream = true;
  }
  if (ctx->arena.init(cfg->hbm_budget) != cudaSuccess ||
      cudaMalloc(&ctx->d_sims, sizeof(SimDev) * cfg->max_slots) != cudaSuccess ||
      cudaMalloc(&ctx->d_active, sizeof(int) * (cfg->max_slots + 1)) != cudaSuccess ||
      cudaMalloc(&ctx->d_io, sizeof(double*) * 2 * cfg->max_slots) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(int) * cfg->max_slots) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(int) * cfg->max_slots) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->admit_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->arena.release();
    if (ctx->d_sims) cudaFree(ctx->d_sims);
    if (ctx->d_active) cudaFree(ctx->d_active);
    if (ctx->d_io) cudaFree(ctx->d_io);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return LRBMS_E_CUDA;
  }
  ctx->slots.resize(cfg->max_slots);
  *out = ctx;
  return LRBMS_OK;
}

int lrbms_destroy(lrbms_ctx* ctx) {
  if (!ctx) return LRBMS_E_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  ctx->arena.release();
  cudaFree(ctx->d_sims);
  cudaFree(ctx->d_active);
  cudaFree(ctx->d_io);
  cudaStreamSynchronize(ctx->admit_stream);
  cudaStreamDestroy(ctx->admit_stream);
  cudaFree(ctx->d_status);
  cudaFreeHost(ctx->h_status);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return LRBMS_OK;
}

const char* lrbms_last_error(const lrbms_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

cudaStream_t lrbms_internal_stream(lrbms_ctx* ctx) { return ctx->stream; }
cudaStream_t lrbms_internal_admit_stream(lrbms_ctx* ctx) { return ctx->admit_stream; }
bool lrbms_internal_in_last_batch(lrbms_ctx* ctx, int id) {
  return std::find(ctx->last_active.begin(), ctx->last_active.end(), id) != ctx->last_active.end();
}
int lrbms_internal_sim(lrbms_ctx* ctx, int id, SimDev* out) {
  if (!valid_sim(ctx, id)) return LRBMS_E_STATE;
  *out = ctx->slots[id].d;
  return LRBMS_OK;
}
int lrbms_internal_fail(lrbms_ctx* ctx, int code, const char* msg) { return fail(ctx, code, msg); }

// Warm admission (mixed solver). A resting simulation that has not stepped
// gets the FP32 factor of its current matrix once, on the admission stream:
// the fit, theta, the assembly and a whole factorisation of that one
// simulation, exactly as its own first step would compute them (that step
// then finds a factor of age 1 and reuses it). The factor and the solver
// state are copied into dst, a new simulation with the same basis and state
// (so the same matrix), whose first step then reuses them too: the results
// are bitwise those of a cold start, without the first step's whole
// factorisation. If the factorisation fails, src is restored and nothing
// is copied (both factor at their first step).
int lrbms_internal_share_factor(lrbms_ctx* ctx, int src, int dst) {
  if (ctx->solver != LRBMS_SOLVE_MIXED || !valid_sim(ctx, src) || !valid_sim(ctx, dst) || src == dst)
    return LRBMS_OK;
  Slot& ss = ctx->slots[src];
  const SimDev& d = ss.d;
  const SimDev& t = ctx->slots[dst].d;
  if (t.n_sub != d.n_sub || t.N != d.N || t.panel_words != d.panel_words) return LRBMS_OK;
  cudaStream_t st = ctx->admit_stream;
  int* act = ctx->d_active + ctx->slots.size();
  if (!ss.prefactored) {
    CK(cudaMemcpyAsync(act, &src, sizeof(int), cudaMemcpyHostToDevice, st));
    lrbms::launch_fit(ctx->d_sims, act, 1, d.n_tiles, st);
    lrbms::launch_assemble(ctx->d_sims, act, 1, d.n_blocks + d.n_sub, ctx->precision == LRBMS_MIXED, st, 128);
    const lrbms::SolveShape sh{d.n_sub, d.panel_words, d.max_w, d.N};
    CK(lrbms::prepare_chol_solve(ctx->solver, sh));
    CK(lrbms::launch_factor32(ctx->d_sims, act, 1, sh, st));
    ctx->launches += 4;
    int status = -1, age = -1;
    CK(cudaMemcpyAsync(&status, d.status, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&age, d.info + 6, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (status != LRBMS_OK || age != 1) {  // undo: src factors at its own first step
      CK(cudaMemsetAsync(d.status, 0, 4, st));
      CK(cudaMemsetAsync(d.info, 0, 4 * 12, st));
      CK(cudaStreamSynchronize(st));
      return LRBMS_OK;
    }
    ss.prefactored = true;
  }
  long long ends[2] = {0, 0};  // loff[n_sub], ioff[n_sub]
  CK(cudaMemcpyAsync(&ends[0], d.loff + d.n_sub, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ends[1], d.ioff + d.n_sub, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpyAsync(t.L, d.L, 8 * (size_t)ends[0], cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(t.Linv, d.Linv, 8 * (size_t)ends[1], cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(t.info, d.info, 4 * 12, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->slots[dst].prefactored = true;
  return LRBMS_OK;
}
SimDev* lrbms_internal_dsims(lrbms_ctx* ctx) { return ctx->d_sims; }
void lrbms_internal_count(lrbms_ctx* ctx, long long n) { ctx->launches += n; }

long long lrbms_launch_count(const lrbms_ctx* ctx) { return ctx ? ctx->launches : 0; }

int lrbms_memory(lrbms_ctx* ctx, size_t* used, size_t* capacity) {
  if (!ctx) return LRBMS_E_ARG;
  if (used) *used = ctx->arena.used();
  if (capacity) *capacity = ctx->arena.cap();
  return LRBMS_OK;
}

int lrbms_sync(lrbms_ctx* ctx) {
  if (!ctx) return LRBMS_E_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  return LRBMS_OK;
}

int lrbms_offline_load(lrbms_ctx* ctx, const lrbms_problem* pr, const lrbms_offline* off,
                       int* sim_id) {
  if (!ctx || !pr || !off || !sim_id) return fail(ctx, LRBMS_E_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  const int nx = pr->nx, ny = pr->ny, Sx = pr->Sx, Sy = pr->Sy, M = off->M;
  if (nx < 1 || ny < 1 || Sx < 1 || Sy < 1 || nx % Sx || ny % Sy)
    return fail(ctx, LRBMS_E_ARG, "grid sizes must be positive and nx%Sx == ny%Sy == 0");
  if (!(pr->Lx > 0) || !(pr->Ly > 0) || !(pr->eta_w > 0) || !(pr->eta_o > 0))
    return fail(ctx, LRBMS_E_ARG, "domain lengths and viscosities must be positive");
  if (M < 1 || M > lrbms::kMaxM) return fail(ctx, LRBMS_E_ARG, "M must be in 1..16");
  if (!pr->perm || !pr->poro || !pr->bc_type || !pr->p_D || !pr->v_N || !pr->s_D || !pr->s0)
    return fail(ctx, LRBMS_E_ARG, "missing problem array");
  if (!off->N_E || !off->Gpinv || !off->Phi || !off->Dblk || !off->rhs || (!off->Fblk && Sx * Sy > 1))
    return fail(ctx, LRBMS_E_ARG, "missing offline array");
  if ((off->prof_idx == nullptr) == (off->prof == nullptr))
    return fail(ctx, LRBMS_E_ARG, "exactly one of prof_idx and prof must be given");
  if (pr->dt_mode == LRBMS_DT_CFL && !(pr->cfl > 0 && off->Lf > 0))
    return fail(ctx, LRBMS_E_ARG, "CFL step needs cfl > 0 and Lf > 0");
  if (pr->transport != LRBMS_TRANSPORT_FV && pr->transport != LRBMS_TRANSPORT_DG1)
    return fail(ctx, LRBMS_E_ARG, "transport must be LRBMS_TRANSPORT_FV or LRBMS_TRANSPORT_DG1");
  if (pr->velocity != LRBMS_VELOCITY_STATE && pr->velocity != LRBMS_VELOCITY_FITTED)
    return fail(ctx, LRBMS_E_ARG, "velocity must be LRBMS_VELOCITY_STATE or LRBMS_VELOCITY_FITTED");
  if (pr->dt_mode == LRBMS_DT_FIXED && !(pr->dt_fixed > 0))
    return fail(ctx, LRBMS_E_ARG, "fixed step needs dt_fixed > 0");
  int slot = -1;
  for (int i = 0; i < (int)ctx->slots.size(); ++i)
    if (!ctx->slots[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) return fail(ctx, LRBMS_E_BUDGET, "slot table full");

  const int n_cells = nx * ny, n_sub = Sx * Sy, cx = nx / Sx, cy = ny / Sy, cells = cx * cy;
  const int n_cf = Sy * (Sx - 1) + (Sy - 1) * Sx, nb = 2 * nx + 2 * ny;
  const int nxf = (nx + 1) * ny, n_faces = nxf + nx * (ny + 1);
  const int n_blocks = n_sub + n_cf;
  // host copies of the basis sizes (may be a device pointer)
  std::vector<int> NE(n_sub);
  CK(cudaMemcpy(NE.data(), off->N_E, sizeof(int) * n_sub, cudaMemcpyDefault));
  int max_NE = 0;
  for (int E = 0; E < n_sub; ++E) {
    if (NE[E] < 1 || NE[E] > lrbms::kMaxNE || NE[E] > 3 * cells)
      return fail(ctx, LRBMS_E_FORMAT, "local basis sizes must be in 1..min(32, 3*cells_E)");
    max_NE = NE[E] > max_NE ? NE[E] : max_NE;
  }
  std::vector<int> xoff(n_sub + 1, 0);
  for (int E = 0; E < n_sub; ++E) xoff[E + 1] = xoff[E] + NE[E];
  const int N = xoff[n_sub];
  std::vector<long long> phi_off(n_sub);
  long long phi_tot = 0;
  for (int E = 0; E < n_sub; ++E) {
    phi_off[E] = phi_tot;
    phi_tot += (long long)NE[E] * 3 * cells;
  }
  std::vector<int> cf_m(n_cf), cf_p(n_cf);
  {
    int f = 0;
    for (int J = 0; J < Sy; ++J)
      for (int I = 0; I + 1 < Sx; ++I, ++f) cf_m[f] = J * Sx + I, cf_p[f] = J * Sx + I + 1;
    for (int J = 0; J + 1 < Sy; ++J)
      for (int I = 0; I < Sx; ++I, ++f) cf_m[f] = J * Sx + I, cf_p[f] = (J + 1) * Sx + I;
  }
  std::vector<long long> aoff(n_blocks + 1, 0);
  for (int E = 0; E < n_sub; ++E) aoff[E + 1] = aoff[E] + (long long)NE[E] * NE[E];
  for (int f = 0; f < n_cf; ++f)
    aoff[n_sub + f + 1] = aoff[n_sub + f] + (long long)NE[cf_m[f]] * NE[cf_p[f]];
  const long long a_tot = aoff[n_blocks];
  const long long d_tot = aoff[n_sub];  // diagonal blocks
  std::vector<long long> loff(n_sub + 1, 0), ioff(n_sub + 1, 0);
  lrbms::solve_offsets(n_sub, Sx, NE.data(), xoff.data(), loff.data(), ioff.data());
  int panel_words = 0, max_w = 0;
  lrbms::solve_panel_sizes(n_sub, Sx, NE.data(), xoff.data(), &panel_words, &max_w);
  if (lrbms::solve_smem_bytes(n_sub, panel_words, max_w, N, sizeof(double)) > lrbms::kMaxSolveSmem)
    return fail(ctx, LRBMS_E_FORMAT, "reduced system too large for the on-chip solve (shared memory)");
  if (nx > lrbms::kMaxNx) return fail(ctx, LRBMS_E_ARG, "nx must be at most 8192");
  const int tile_rows = std::max(1, lrbms::kCellTile / nx);
  const int n_tiles = (ny + tile_rows - 1) / tile_rows;
  const bool mixed = ctx->precision == LRBMS_MIXED;
  const size_t Q = (size_t)M + 1;

  Layout L;
  const size_t o_perm = L.add(8 * (size_t)n_cells), o_poro = L.add(8 * (size_t)n_cells);
  const size_t o_pidx = off->prof_idx ? L.add(n_cells) : 0;
  const size_t o_prof = off->prof ? L.add(8 * (size_t)M * n_cells) : 0;
  const size_t o_gp = L.add(8 * (size_t)M * M);
  const size_t o_bct = L.add(nb), o_pD = L.add(8 * (size_t)nb), o_vN = L.add(8 * (size_t)nb),
               o_sD = L.add(8 * (size_t)nb);
  const size_t o_NE = L.add(4 * (size_t)n_sub), o_xoff = L.add(4 * (size_t)(n_sub + 1));
  const size_t o_phioff = L.add(8 * (size_t)n_sub), o_aoff = L.add(8 * (size_t)(n_blocks + 1));
  const size_t o_loff = L.add(8 * (size_t)(n_sub + 1)), o_ioff = L.add(8 * (size_t)(n_sub + 1));
  const size_t o_phi = L.add(8 * (size_t)phi_tot);
  const size_t o_comp = L.add(8 * Q * (size_t)a_tot);
  const size_t o_rhs = L.add(8 * Q * (size_t)N);
  const size_t o_phi32 = mixed ? L.add(4 * (size_t)phi_tot) : 0;
  const size_t o_comp32 = mixed ? L.add(4 * Q * (size_t)a_tot) : 0;
  const size_t o_s = L.add(16 * (size_t)n_cells), o_p = L.add(24 * (size_t)n_cells);
  const bool dg = pr->transport == LRBMS_TRANSPORT_DG1;
  const size_t o_slope = dg ? L.add(32 * (size_t)n_cells) : 0, o_unl = dg ? L.add(16 * (size_t)n_cells) : 0;
  const size_t o_F = L.add(8 * (size_t)n_faces);
  const size_t o_lam = L.add(16 * (size_t)n_cells), o_fw = L.add(16 * (size_t)n_cells),
               o_ipv = L.add(8 * (size_t)n_cells), o_fc = L.add(24 * (size_t)n_faces), o_fwD = L.add(8 * (size_t)nb);
  const size_t o_x = L.add(8 * (size_t)N), o_xp = L.add(8 * (size_t)N), o_xpp = L.add(8 * (size_t)N),
               o_b = L.add(8 * (size_t)N),
               o_y = L.add(16 * (size_t)N),
               o_rv = L.add(8 * (size_t)N), o_dv = L.add(8 * (size_t)N), o_pv = L.add(8 * (size_t)N),
               o_qv = L.add(8 * (size_t)N);
  const size_t o_A = L.add(8 * (size_t)a_tot);
  const size_t o_L = L.add(8 * (size_t)loff[n_sub]), o_Li = L.add(8 * (size_t)ioff[n_sub]);
  const size_t o_fitp = L.add(8 * (size_t)n_tiles * lrbms::kMaxM);
  const size_t o_cflp = L.add(8 * (size_t)n_tiles), o_massp = L.add(8 * (size_t)n_tiles);
  const size_t o_scal = L.add(8 * 4), o_theta = L.add(8 * lrbms::kMaxM);
  const size_t o_status = L.add(4), o_steps = L.add(4), o_info = L.add(4 * 12), o_fitr = L.add(4),
               o_inj = L.add(4);
  const size_t o_sched = L.add(8 * lrbms::sched_words(n_sub, Sx));
  (void)d_tot;

  const size_t aoffset = ctx->arena.alloc(L.total);
  if (aoffset == SIZE_MAX) return fail(ctx, LRBMS_E_BUDGET, "device-memory budget exhausted");
  char* base = ctx->arena.base() + aoffset;
  auto P = [&](size_t o) { return (void*)(base + o); };

  SimDev d{};
  d.nx = nx; d.ny = ny; d.Sx = Sx; d.Sy = Sy; d.cx = cx; d.cy = cy;
  d.n_cells = n_cells; d.n_sub = n_sub; d.n_cf = n_cf; d.nb = nb; d.nxf = nxf; d.n_faces = n_faces;
  d.M = M; d.N = N; d.max_NE = max_NE; d.n_tiles = n_tiles; d.tile_rows = tile_rows; d.n_blocks = n_blocks;
  d.panel_words = panel_words;
  d.max_w = max_w;
  d.relperm = pr->relperm; d.swapped = pr->mean_weights; d.prof_mode = off->prof_idx ? 0 : 1;
  d.vel_mode = pr->velocity;
  d.transport = pr->transport;
  d.dt_mode = pr->dt_mode;
  d.hx = pr->Lx / nx; d.hy = pr->Ly / ny; d.vol = d.hx * d.hy; d.c_pen = off->c_pen; d.Lf = off->Lf;
  d.inv_eta_w = 1.0 / pr->eta_w; d.inv_eta_o = 1.0 / pr->eta_o; d.cfl = pr->cfl;
  d.dt_fixed = pr->dt_fixed; d.dt_max = pr->dt_max;
  // lambda(0) and lambda(1) for both relative permeability laws (k_rw(0)=0,
  // k_rw(1)=1, k_ro(0)=1, k_ro(1)=0)
  d.lam0 = d.inv_eta_o;
  d.lam1 = d.inv_eta_w;
  d.perm = (const double*)P(o_perm); d.poro = (const double*)P(o_poro);
  d.prof_idx = off->prof_idx ? (const uint8_t*)P(o_pidx) : nullptr;
  d.prof = off->prof ? (const double*)P(o_prof) : nullptr;
  d.Gpinv = (const double*)P(o_gp);
  d.bc_type = (const int8_t*)P(o_bct); d.p_D = (const double*)P(o_pD);
  d.v_N = (const double*)P(o_vN); d.s_D = (const double*)P(o_sD);
  d.NE = (const int*)P(o_NE); d.xoff = (const int*)P(o_xoff);
  d.phi_off = (const long long*)P(o_phioff); d.aoff = (const long long*)P(o_aoff);
  d.loff = (const long long*)P(o_loff); d.ioff = (const long long*)P(o_ioff);
  d.Phi = (const double*)P(o_phi); d.comp = (const double*)P(o_comp); d.rhs = (const double*)P(o_rhs);
  d.Phi32 = mixed ? (const float*)P(o_phi32) : nullptr;
  d.comp32 = mixed ? (const float*)P(o_comp32) : nullptr;
  d.s = (double*)P(o_s); d.p = (double*)P(o_p); d.F = (double*)P(o_F);
  d.sslope = dg ? (double*)P(o_slope) : nullptr;
  d.sunl = dg ? (double*)P(o_unl) : nullptr;
  d.x = (double*)P(o_x); d.xp = (double*)P(o_xp); d.xpp = (double*)P(o_xpp); d.b = (double*)P(o_b); d.y = (double*)P(o_y);
  d.refactor_period = ctx->refactor_period;
  d.refactor_stages = ctx->refactor_stages;
  d.rv = (double*)P(o_rv); d.dv = (double*)P(o_dv); d.pv = (double*)P(o_pv); d.qv = (double*)P(o_qv);
  d.A = (double*)P(o_A); d.L = (double*)P(o_L); d.Linv = (double*)P(o_Li);
  d.fit_part = (double*)P(o_fitp); d.cfl_part = (double*)P(o_cflp); d.mass_part = (double*)P(o_massp);
  d.scal = (double*)P(o_scal); d.theta = (double*)P(o_theta);
  d.status = (int*)P(o_status); d.steps = (int*)P(o_steps); d.info = (int*)P(o_info);
  d.fit_ready = (int*)P(o_fitr);
  d.inject = (int*)P(o_inj);
  d.sched = (const unsigned long long*)P(o_sched);
  d.lam = (double*)P(o_lam); d.fw = (double*)P(o_fw); d.inv_pv = (double*)P(o_ipv); d.fcoef = (double*)P(o_fc);
  d.fwD = (double*)P(o_fwD);

  // the admission stream: the copies and kernels of a new simulation overlap
  // the steps that run meanwhile on the context stream
  cudaStream_t st = ctx->admit_stream;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
  };
  const size_t nc8 = 8 * (size_t)n_cells;
  CK(cp(P(o_perm), pr->perm, nc8));
  CK(cp(P(o_poro), pr->poro, nc8));
  if (off->prof_idx) CK(cp(P(o_pidx), off->prof_idx, n_cells));
  if (off->prof) CK(cp(P(o_prof), off->prof, nc8 * M));
  CK(cp(P(o_gp), off->Gpinv, 8 * (size_t)M * M));
  CK(cp(P(o_bct), pr->bc_type, nb));
  CK(cp(P(o_pD), pr->p_D, 8 * (size_t)nb));
  CK(cp(P(o_vN), pr->v_N, 8 * (size_t)nb));
  CK(cp(P(o_sD), pr->s_D, 8 * (size_t)nb));
  CK(cp(P(o_phi), off->Phi, 8 * (size_t)phi_tot));
  CK(cp(P(o_comp), off->Dblk, 8 * Q * (size_t)aoff[n_sub]));
  if (n_cf) CK(cp((char*)P(o_comp) + 8 * Q * aoff[n_sub], off->Fblk, 8 * Q * (size_t)(a_tot - aoff[n_sub])));
  CK(cp(P(o_rhs), off->rhs, 8 * Q * (size_t)N));
  CK(cp(P(o_s), pr->s0, nc8));
  // metadata from host vectors (pageable: staged before the call returns)
  CK(cp(P(o_NE), NE.data(), 4 * (size_t)n_sub));
  CK(cp(P(o_xoff), xoff.data(), 4 * (size_t)(n_sub + 1)));
  CK(cp(P(o_phioff), phi_off.data(), 8 * (size_t)n_sub));
  CK(cp(P(o_aoff), aoff.data(), 8 * (size_t)(n_blocks + 1)));
  CK(cp(P(o_loff), loff.data(), 8 * (size_t)(n_sub + 1)));
  CK(cp(P(o_ioff), ioff.data(), 8 * (size_t)(n_sub + 1)));
  CK(cudaMemsetAsync(P(o_scal), 0, 8 * 4, st));
  CK(cudaMemsetAsync(P(o_theta), 0, 8 * lrbms::kMaxM, st));
  CK(cudaMemsetAsync(P(o_status), 0, 4, st));
  CK(cudaMemsetAsync(P(o_steps), 0, 4, st));
  CK(cudaMemsetAsync(P(o_info), 0, 4 * 12, st));
  CK(cudaMemsetAsync(P(o_fitr), 0, 4, st));
  CK(cudaMemsetAsync(P(o_inj), 0, 4, st));
  if (dg) CK(cudaMemsetAsync(P(o_slope), 0, 32 * (size_t)n_cells, st));  // s0 piecewise constant
  CK(cudaMemsetAsync(P(o_p), 0, 24 * (size_t)n_cells, st));
  CK(cudaMemsetAsync(P(o_F), 0, 8 * (size_t)n_faces, st));
  CK(cudaMemsetAsync(P(o_x), 0, 8 * (size_t)N, st));
  CK(cudaMemsetAsync(P(o_xp), 0, 8 * (size_t)N, st));
  CK(cudaMemsetAsync(P(o_xpp), 0, 8 * (size_t)N, st));
  if (mixed) {
    lrbms::launch_to_float((const double*)P(o_phi), (float*)P(o_phi32), phi_tot, st);
    lrbms::launch_to_float((const double*)P(o_comp), (float*)P(o_comp32), Q * a_tot, st);
    ctx->launches += 2;
  }
  CK(cp(ctx->d_sims + slot, &d, sizeof(SimDev)));
  lrbms::launch_prepare(ctx->d_sims + slot, std::max(n_cells, n_faces), st);
  lrbms::launch_sched(ctx->d_sims + slot, st);
  ctx->launches += 2;
  CK(cudaStreamSynchronize(st));  // caller buffers may be freed on return
  CK(cudaGetLastError());
  Slot& s = ctx->slots[slot];
  s.used = true;
  s.off = aoffset;
  s.bytes = L.total;
  s.d = d;
  *sim_id = slot;
  return LRBMS_OK;
}

int lrbms_release(lrbms_ctx* ctx, int id) {
  if (!valid_sim(ctx, id)) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  CK(cudaStreamSynchronize(ctx->stream));
  Slot& s = ctx->slots[id];
  ctx->arena.free(s.off, s.bytes);
  s = Slot();
  ctx->last_active.clear();
  return LRBMS_OK;
}

int lrbms_step(lrbms_ctx* ctx, int n_sims, const int* ids, int n_steps, int* status) {
  if (!ctx || n_sims < 1 || !ids || n_steps < 0) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  if (n_sims > (int)ctx->slots.size()) return fail(ctx, LRBMS_E_ARG, "too many simulations");
  CK(cudaSetDevice(ctx->device));
  std::vector<int> act(ids, ids + n_sims);
  int max_tiles = 0, max_blocks = 0, max_sub = 0;
  bool any_dg = false;
  size_t flux_smem = 0;
  lrbms::SolveShape sh{0, 0, 0, 0};
  for (int id : act) {
    if (!valid_sim(ctx, id)) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
    ctx->slots[id].prefactored = false;  // it leaves the state its factor was computed for
    const SimDev& d = ctx->slots[id].d;
    sh.n_sub = std::max(sh.n_sub, d.n_sub);
    sh.panel_words = std::max(sh.panel_words, d.panel_words);
    sh.max_w = std::max(sh.max_w, d.max_w);
    sh.N = std::max(sh.N, d.N);
    max_tiles = std::max(max_tiles, d.n_tiles);
    max_blocks = std::max(max_blocks, d.n_blocks + d.n_sub);
    max_sub = std::max(max_sub, d.n_sub);
    flux_smem = std::max(flux_smem, lrbms::flux_cfl_smem(d.nx, d.ny, d.tile_rows));
    any_dg |= d.transport == LRBMS_TRANSPORT_DG1;
  }
  cudaStream_t st = ctx->stream;
  if (act != ctx->last_active) {
    CK(cudaMemcpyAsync(ctx->d_active, act.data(), sizeof(int) * n_sims, cudaMemcpyHostToDevice, st));
    ctx->last_active = act;
  }
  const int mixed = ctx->precision == LRBMS_MIXED;
  const int per_step = 7 + (ctx->solver == LRBMS_SOLVE_MIXED ? 4 : 1)  // mixed solve: factor (where
                       + (any_dg ? 2 : 0);                             // needed), refine, retry, FP64 redo
  CK(lrbms::prepare_chol_solve(ctx->solver, sh));  // kernel attributes, outside any capture
  CK(lrbms::prepare_flux_cfl(flux_smem));
  // Autotuner: the first step of a new shape class times every CTA size of
  // the two streaming contractions on the live data (both kernels are pure
  // functions of their inputs, which the step then recomputes) and keeps the
  // fastest; every size gives the same result.
  int ne_max = 0, cells_max = 0;
  for (int id : act) {
    ne_max = std::max(ne_max, ctx->slots[id].d.max_NE);
    cells_max = std::max(cells_max, ctx->slots[id].d.cx * ctx->slots[id].d.cy);
  }
  const std::vector<int> tkey{(ne_max + 7) / 8, cells_max, mixed};
  auto tit = ctx->tuned.find(tkey);
  if (tit == ctx->tuned.end() && n_steps > 0) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto best_of = [&](const std::vector<int>& sizes, int kernels, auto&& launch) -> int {
      int best = sizes[0];
      float best_ms = 1e30f;
      for (int t : sizes) {
        launch(t);  // warm-up
        cudaEventRecord(e0, st);
        launch(t);
        launch(t);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ctx->launches += 3 * kernels;
        if (ms < best_ms) best_ms = ms, best = t;
      }
      return best;
    };
    const int ta = best_of({64, 128, 256, 512}, 2, [&](int t) {  // theta, then the assembly
      lrbms::launch_assemble(ctx->d_sims, ctx->d_active, n_sims, max_blocks, mixed, st, t);
    });
    const int tr = best_of({128, 256, 512, 1024}, 1, [&](int t) {
      lrbms::launch_reconstruct(ctx->d_sims, ctx->d_active, n_sims, max_sub, mixed, st, t);
    });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    tit = ctx->tuned.emplace(tkey, std::make_pair(ta, tr)).first;
  }
  const int t_asm = tit == ctx->tuned.end() ? 128 : tit->second.first;
  const int t_rec = tit == ctx->tuned.end() ? 256 : tit->second.second;
  // The kernels of one step, in order; ev (optional) gets an event before the
  // first phase and after every phase.
  auto enqueue_step = [&](cudaEvent_t* ev) -> cudaError_t {
    auto mark = [&](int i) {
      if (ev) cudaEventRecord(ev[i], st);
    };
    mark(0);
    lrbms::launch_fit(ctx->d_sims, ctx->d_active, n_sims, max_tiles, st);
    mark(1);
    lrbms::launch_assemble(ctx->d_sims, ctx->d_active, n_sims, max_blocks, mixed, st, t_asm);
    mark(2);
    cudaError_t e = lrbms::launch_chol_solve(ctx->d_sims, ctx->d_active, n_sims, ctx->solver, ctx->refine_iters,
                                             sh, st);
    if (e != cudaSuccess) return e;
    mark(3);
    lrbms::launch_reconstruct(ctx->d_sims, ctx->d_active, n_sims, max_sub, mixed, st, t_rec);
    mark(4);
    lrbms::launch_flux_cfl(ctx->d_sims, ctx->d_active, n_sims, max_tiles, flux_smem, st);
    mark(5);
    lrbms::launch_transport(ctx->d_sims, ctx->d_active, n_sims, max_tiles, st);
    if (any_dg) lrbms::launch_transport_dg(ctx->d_sims, ctx->d_active, n_sims, max_tiles, st);
    mark(6);
    lrbms::launch_finalize(ctx->d_sims, ctx->d_active, n_sims, st, ctx->d_status);
    mark(7);
    return cudaGetLastError();
  };
  int k = 0;
  // Profiled steps launch kernel by kernel (events between the phases).
  for (; k < n_steps && ctx->prof_n < ctx->prof_cap; ++k) {
    CK(enqueue_step(&ctx->prof_ev[(size_t)ctx->prof_n++ * (LRBMS_N_PHASES + 1)]));
    ctx->launches += per_step;
  }
  if (k < n_steps) {
    // The other steps replay one captured graph of the step's kernels.
    std::vector<long long> key(act.begin(), act.end());
    for (long long v : {(long long)sh.n_sub, (long long)sh.panel_words, (long long)sh.max_w, (long long)sh.N,
                        (long long)max_tiles, (long long)max_blocks, (long long)max_sub, (long long)flux_smem,
                        (long long)t_asm, (long long)t_rec, (long long)any_dg})
      key.push_back(v);
    if (!ctx->graph || key != ctx->graph_key) {
      if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
      ctx->graph = nullptr;
      ctx->graph_key.clear();
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const cudaError_t e1 = enqueue_step(nullptr);
        const cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
            cudaGraphInstantiate(&ctx->graph, g, 0) == cudaSuccess) {
          ctx->graph_key = key;
          ctx->graph_kernels = per_step;
        } else {
          ctx->graph = nullptr;
        }
        if (g) cudaGraphDestroy(g);
      }
      (void)cudaGetLastError();  // a stream that cannot be captured: launch directly below
    }
    for (; k < n_steps; ++k) {
      if (ctx->graph) {
        CK(cudaGraphLaunch(ctx->graph, st));
      } else {
        CK(enqueue_step(nullptr));
      }
      ctx->launches += per_step;
    }
  }
  CK(cudaGetLastError());
  if (n_steps == 0) {  // a status query: read the status words themselves
    if (status) {
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i < n_sims; ++i)
        CK(cudaMemcpy(&status[i], ctx->slots[act[i]].d.status, sizeof(int), cudaMemcpyDeviceToHost));
    }
    return LRBMS_OK;
  }
  ctx->last_n = n_sims;
  if (status) return lrbms_step_status(ctx, n_sims, status);
  return LRBMS_OK;
}

int lrbms_step_status(lrbms_ctx* ctx, int n_sims, int* status) {
  if (!ctx || !status || n_sims < 1 || n_sims > ctx->last_n) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  if (ctx->last_active.empty() || (int)ctx->last_active.size() < n_sims)
    return fail(ctx, LRBMS_E_STATE, "no step to report");
  // one copy of the statuses k_finalize gathered in list order
  CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int) * n_sims, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(status, ctx->h_status, sizeof(int) * n_sims);
  return LRBMS_OK;
}

int lrbms_step_io(lrbms_ctx* ctx, int n_sims, const int* ids, int n_steps, const double* const* s_in,
                  double* const* s_out, int* status) {
  if (!ctx || n_sims < 1 || !ids) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  if (n_sims > (int)ctx->slots.size()) return fail(ctx, LRBMS_E_ARG, "too many simulations");
  for (int i = 0; i < n_sims; ++i)
    if (!valid_sim(ctx, ids[i])) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  std::vector<int> act(ids, ids + n_sims);
  if (act != ctx->last_active) {
    CK(cudaMemcpyAsync(ctx->d_active, act.data(), sizeof(int) * n_sims, cudaMemcpyHostToDevice, st));
    ctx->last_active = act;
  }
  const size_t ms = ctx->slots.size();
  std::vector<const double*> ptrs(2 * ms, nullptr);
  for (int i = 0; i < n_sims; ++i) {
    ptrs[i] = s_in ? s_in[i] : nullptr;
    ptrs[ms + i] = s_out ? (const double*)s_out[i] : nullptr;
  }
  CK(cudaMemcpyAsync(ctx->d_io, ptrs.data(), sizeof(double*) * 2 * ms, cudaMemcpyHostToDevice, st));
  int max_tiles = 1;
  for (int i = 0; i < n_sims; ++i) max_tiles = std::max(max_tiles, ctx->slots[ids[i]].d.n_tiles);
  if (s_in) {
    lrbms::launch_sat_io(ctx->d_sims, ctx->d_active, n_sims, max_tiles, ctx->d_io, nullptr, st);
    ctx->launches += 1;
  }
  int rc = lrbms_step(ctx, n_sims, ids, n_steps, nullptr);
  if (rc) return rc;
  if (s_out) {
    lrbms::launch_sat_io(ctx->d_sims, ctx->d_active, n_sims, max_tiles, nullptr, (double* const*)(ctx->d_io + ms),
                         st);
    ctx->launches += 1;
  }
  CK(cudaGetLastError());
  if (status && n_steps > 0) return lrbms_step_status(ctx, n_sims, status);
  CK(cudaStreamSynchronize(st));
  if (status)
    for (int i = 0; i < n_sims; ++i)
      CK(cudaMemcpy(&status[i], ctx->slots[ids[i]].d.status, sizeof(int), cudaMemcpyDeviceToHost));
  return LRBMS_OK;
}

int lrbms_profile_start(lrbms_ctx* ctx, int max_steps) {
  if (!ctx || max_steps < 0) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t need = (size_t)max_steps * (LRBMS_N_PHASES + 1);
  while (ctx->prof_ev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ctx->prof_ev.push_back(e);
  }
  ctx->prof_cap = max_steps;
  ctx->prof_n = 0;
  return LRBMS_OK;
}

int lrbms_profile_read(lrbms_ctx* ctx, double* phase_ms, double* step_ms, int* n_recorded) {
  if (!ctx) return LRBMS_E_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  const int n = ctx->prof_n;
  if (n_recorded) *n_recorded = n;
  std::vector<double> acc(LRBMS_N_PHASES, 0.0);
  for (int k = 0; k < n; ++k) {
    cudaEvent_t* ev = &ctx->prof_ev[(size_t)k * (LRBMS_N_PHASES + 1)];
    for (int ph = 0; ph < LRBMS_N_PHASES; ++ph) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, ev[ph], ev[ph + 1]));
      acc[ph] += t;
    }
    if (step_ms) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, ev[0], ev[LRBMS_N_PHASES]));
      step_ms[k] = t;
    }
  }
  if (phase_ms)
    for (int ph = 0; ph < LRBMS_N_PHASES; ++ph) phase_ms[ph] = n ? acc[ph] / n : 0.0;
  ctx->prof_cap = 0;
  return LRBMS_OK;
}

size_t lrbms_field_bytes(lrbms_ctx* ctx, int id, int field) {
  if (!valid_sim(ctx, id)) return 0;
  const SimDev& d = ctx->slots[id].d;
  switch (field) {
    case LRBMS_FIELD_THETA: return 8 * (size_t)d.M;
    case LRBMS_FIELD_A: {
      // sum of block sizes: computed from the host copy of the layout
      size_t n = 0;
      std::vector<long long> a(d.n_blocks + 1);
      if (cudaMemcpy(a.data(), d.aoff, 8 * a.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
      n = (size_t)a[d.n_blocks];
      return 8 * n;
    }
    case LRBMS_FIELD_RHS:
    case LRBMS_FIELD_X: return 8 * (size_t)d.N;
    case LRBMS_FIELD_P: return 24 * (size_t)d.n_cells;
    case LRBMS_FIELD_FLUX: return 8 * (size_t)d.n_faces;
    case LRBMS_FIELD_S: return 8 * (size_t)d.n_cells;
    case LRBMS_FIELD_DT: return 8;
    case LRBMS_FIELD_STATUS: return 4;
    case LRBMS_FIELD_SOLVE_INFO: return 24;
    case LRBMS_FIELD_SLOPES: return 16 * (size_t)d.n_cells;
    case LRBMS_FIELD_PHI: return 24 * (size_t)d.N * d.cx * d.cy;
    default: return 0;
  }
}

int lrbms_get_field(lrbms_ctx* ctx, int id, int field, void* dst, size_t bytes) {
  if (!valid_sim(ctx, id)) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  if (!dst || bytes != lrbms_field_bytes(ctx, id, field))
    return fail(ctx, LRBMS_E_ARG, "destination size does not match the field");
  CK(cudaStreamSynchronize(ctx->stream));
  const SimDev& d = ctx->slots[id].d;
  const void* src = nullptr;
  int steps = 0;
  switch (field) {
    case LRBMS_FIELD_THETA: src = d.theta; break;
    case LRBMS_FIELD_A: src = d.A; break;
    case LRBMS_FIELD_RHS: src = d.b; break;
    case LRBMS_FIELD_X: src = d.x; break;
    case LRBMS_FIELD_P: src = d.p; break;
    case LRBMS_FIELD_FLUX: src = d.F; break;
    case LRBMS_FIELD_S:
      CK(cudaMemcpy(&steps, d.steps, 4, cudaMemcpyDeviceToHost));
      src = d.s + (size_t)(steps & 1) * d.n_cells;
      break;
    case LRBMS_FIELD_DT: src = d.scal + 1; break;
    case LRBMS_FIELD_STATUS: src = d.status; break;
    case LRBMS_FIELD_SOLVE_INFO: src = d.info; break;
    case LRBMS_FIELD_PHI: src = d.Phi; break;
    case LRBMS_FIELD_SLOPES:
      if (!d.sslope) {  // piecewise-constant transport: no slopes (dst may be host memory)
        const std::vector<double> zeros(bytes / sizeof(double), 0.0);
        CK(cudaMemcpy(dst, zeros.data(), bytes, cudaMemcpyDefault));
        return LRBMS_OK;
      }
      CK(cudaMemcpy(&steps, d.steps, 4, cudaMemcpyDeviceToHost));
      src = d.sslope + (size_t)(steps & 1) * 2 * d.n_cells;
      break;
    default: return fail(ctx, LRBMS_E_ARG, "unknown field");
  }
  CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
  return LRBMS_OK;
}

int lrbms_get_state(lrbms_ctx* ctx, int id, double* s, double* t, double* mass_out) {
  if (!valid_sim(ctx, id)) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  const SimDev& d = ctx->slots[id].d;
  if (s) {
    int rc = lrbms_get_field(ctx, id, LRBMS_FIELD_S, s, 8 * (size_t)d.n_cells);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  double sc[4];
  CK(cudaMemcpy(sc, d.scal, sizeof(sc), cudaMemcpyDeviceToHost));
  if (t) *t = sc[0];
  if (mass_out) *mass_out = sc[2];
  return LRBMS_OK;
}

int lrbms_tuned_threads(lrbms_ctx* ctx, int n_sims, const int* ids, int* assemble, int* reconstruct) {
  if (!ctx || n_sims < 1 || !ids) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  int ne_max = 0, cells_max = 0;
  for (int i = 0; i < n_sims; ++i) {
    if (!valid_sim(ctx, ids[i])) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
    ne_max = std::max(ne_max, ctx->slots[ids[i]].d.max_NE);
    cells_max = std::max(cells_max, ctx->slots[ids[i]].d.cx * ctx->slots[ids[i]].d.cy);
  }
  auto it = ctx->tuned.find(std::vector<int>{(ne_max + 7) / 8, cells_max, ctx->precision == LRBMS_MIXED});
  if (it == ctx->tuned.end()) return fail(ctx, LRBMS_E_STATE, "this shape class has not been tuned yet");
  if (assemble) *assemble = it->second.first;
  if (reconstruct) *reconstruct = it->second.second;
  return LRBMS_OK;
}

int lrbms_test_withhold_copy(lrbms_ctx* ctx, int id) {
  if (!valid_sim(ctx, id)) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  CK(cudaStreamSynchronize(ctx->stream));
  const int one = 1;
  CK(cudaMemcpy(ctx->slots[id].d.inject, &one, sizeof(int), cudaMemcpyHostToDevice));
  return LRBMS_OK;
}

int lrbms_set_saturation(lrbms_ctx* ctx, int id, const double* s) {
  if (!valid_sim(ctx, id) || !s) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  const SimDev& d = ctx->slots[id].d;
  CK(cudaStreamSynchronize(ctx->stream));
  int steps = 0;
  CK(cudaMemcpy(&steps, d.steps, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(d.s + (size_t)(steps & 1) * d.n_cells, s, 8 * (size_t)d.n_cells, cudaMemcpyDefault));
  CK(cudaMemset(d.fit_ready, 0, 4));  // the next step fits the new saturation
  if (ctx->slots[id].prefactored) {   // the factor of the old state no longer matches
    CK(cudaMemset(d.info, 0, 4 * 12));
    ctx->slots[id].prefactored = false;
  }
  if (d.sslope) CK(cudaMemset(d.sslope + (size_t)(steps & 1) * 2 * d.n_cells, 0, 16 * (size_t)d.n_cells));
  return LRBMS_OK;
}

int lrbms_set_slopes(lrbms_ctx* ctx, int id, const double* slopes) {
  if (!valid_sim(ctx, id) || !slopes) return fail(ctx, LRBMS_E_ARG, "bad arguments");
  const SimDev& d = ctx->slots[id].d;
  if (!d.sslope) return fail(ctx, LRBMS_E_ARG, "the simulation uses the piecewise-constant transport");
  CK(cudaStreamSynchronize(ctx->stream));
  int steps = 0;
  CK(cudaMemcpy(&steps, d.steps, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(d.sslope + (size_t)(steps & 1) * 2 * d.n_cells, slopes, 16 * (size_t)d.n_cells,
                cudaMemcpyDefault));
  return LRBMS_OK;
}

int lrbms_run(lrbms_ctx* ctx, int id, int n_steps, double* s_out, double* p_out, double* flux_out) {
  if (!valid_sim(ctx, id)) return fail(ctx, LRBMS_E_STATE, "unknown simulation id");
  int st = 0;
  int rc = lrbms_step(ctx, 1, &id, n_steps, &st);
  if (rc) return rc;
  const SimDev& d = ctx->slots[id].d;
  if (s_out && (rc = lrbms_get_field(ctx, id, LRBMS_FIELD_S, s_out, 8 * (size_t)d.n_cells))) return rc;
  if (p_out && (rc = lrbms_get_field(ctx, id, LRBMS_FIELD_P, p_out, 24 * (size_t)d.n_cells))) return rc;
  if (flux_out && (rc = lrbms_get_field(ctx, id, LRBMS_FIELD_FLUX, flux_out, 8 * (size_t)d.n_faces)))
    return rc;
  if (st != LRBMS_OK) return fail(ctx, st, "simulation stopped with a non-zero status");
  return LRBMS_OK;
}

}  // extern "C"
