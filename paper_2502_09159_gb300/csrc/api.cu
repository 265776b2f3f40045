// C ABI of libstmg: handle, setup uploads, hot-path entry points, the hp space-time
// V-cycle (Alg. 1 with the subroutines of App. B) and FGMRES per slab.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "levels.h"

using namespace stmg;

namespace {

template <typename T>
struct PrecDev {
  T* inv = nullptr;   // per-patch inverses, interleaved layout
  T* b = nullptr;     // V-cycle right-hand side of this level
  T* x = nullptr;     // V-cycle iterate of this level
  T* r = nullptr;     // residual work vector
  T* x2 = nullptr;    // FP32, 2D: the iterate after the prolongation fused into the residual
  ApplyParams<T> ap{};
  ApplyRegParams<T> rp{};   // tables of the register-resident 2D operator (apply variant 3)
  TransferParams<T> tp{};   // transfer between this level and the next coarser one
  bool has_inv = false;
  // FP32 V-cycle with half-precision inverses: FP16 rows scaled to [-1, 1], FP32 row scales
  __half* invh = nullptr;
  float* rsc = nullptr;
  bool half = false;
};

struct LevelDev {
  LevelHost H;
  int* dofs = nullptr;
  PrecDev<double> d;
  PrecDev<float> f;
  double* G = nullptr;      // coarsest level: bordered inverse, column-major
  double* Gacc = nullptr;   // coarsest level with D > 1024: FP64 accumulator of the tiled GEMV
  float* Gf = nullptr;      // coarsest level: G rounded to FP32, for the FP32 V-cycle
  int streaming = 0;        // read the inverses with evict-first loads
  int sweep_var[2] = {1, 1};  // per precision: 1 = block per patch group, 2 = TMA-pipelined, 3 = pipelined block
  int ppb[2] = {1, 1};        // per precision: patches per block of the block sweeps
  int unroll[2] = {8, 8};     // per precision: chunks per load round of the block sweeps (4 or 8)
  template <typename T> PrecDev<T>& pd();
};
template <> PrecDev<double>& LevelDev::pd<double>() { return d; }
template <> PrecDev<float>& LevelDev::pd<float>() { return f; }

struct ProfPair { int cat; cudaEvent_t a, b; };
constexpr int PROF_VCYCLE = STMG_PROF_N;   // internal: whole V-cycles (MG w/o smoother = this - smoother)

}  // namespace

struct stmg_handle {
  stmg_config cfg{};
  std::vector<LevelDev> L;
  cudaStream_t st = nullptr;      // caller's stream (nullptr: legacy default stream)
  cudaStream_t gst = nullptr;     // internal stream that launches the captured V-cycles
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double tau = 0.0;
  // FGMRES storage
  double *V = nullptr, *Z = nullptr, *w = nullptr, *hcol = nullptr, *tmp = nullptr, *partial = nullptr;
  double *bnorm = nullptr, *xhost_b = nullptr, *xhost_x = nullptr;
  int m_alloc = 0;
  double* hc_host = nullptr;      // pinned: the Arnoldi column of H of each iteration
  int* err_host = nullptr;        // pinned: the device error flag after each iteration
  cudaEvent_t ev_it[2] = {nullptr, nullptr};   // ends of the (at most two) iterations in flight
  int* d_err = nullptr;           // device flag raised by bounded waits that expired
  double* dot_part = nullptr;     // per-block partial sums of stmg_dot (allocated on first use)
  unsigned* cgs_bar = nullptr;    // grid barrier of the cooperative CGS2 step (count, generation)
  double* cgs_part = nullptr;     // its partial sums
  int cgs_blocks = 0;             // co-resident blocks of that launch (0: use the split kernels)
  int inject_wait_fault = 0;      // testing hook: arm the next grid barrier so that it cannot complete
  int n_sm = 1;
  ForcingParams fp{};
  MassParams mp{};
  // instrumentation
  int prof = 0;
  std::vector<ProfPair> pending;        // eager pairs not yet read
  std::vector<ProfPair> graph_pairs[2]; // pairs recorded inside the captured V-cycles
  std::vector<cudaEvent_t> all_events;
  double prof_ms[STMG_PROF_N + 1] = {};
  long long prof_n[STMG_PROF_N + 1] = {};
  long long launches = 0;
  long long graph_kernels[2] = {0, 0};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_pending[2] = {false, false};
  std::vector<cudaEvent_t> free_events;
  bool capturing = false;
  void* noalloc = nullptr;        // device address of stmg_smooth_noalloc's fixed array (this device)
  // persistent multigrid kernel (levels mgp_first.. coarsest in one launch), per precision
  void* mgp_desc[2] = {nullptr, nullptr};   // device array of MGLevelDesc<T>
  int mgp_first[2] = {0, 0};                // first level of the persistent part (0: not used)
  int mgp_eligible[2] = {0, 0};             // first level from which it could run (0: none)
  int mgp_blocks[2] = {0, 0};                // grid of the persistent kernel
  int mgp_bpsm[2] = {0, 0};                  // resident blocks per SM it may use
  unsigned* mgp_bar = nullptr;              // its grid barrier (count, generation)
  // stmg_march_host: double-buffered device inputs / solutions, a copy stream and its events
  double *mh_in[2] = {nullptr, nullptr}, *mh_x[2] = {nullptr, nullptr}, *mh_b = nullptr, *mh_t = nullptr;
  cudaStream_t cst = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
};

// Device address of the fixed array of stmg_smooth_noalloc on the current device (defined
// at the end of this file); looked up once per device, at handle creation.
static int noalloc_scratch_address(void** out);

// ------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------
#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      std::fprintf(stderr, "stmg: %s failed: %s (%s:%d)\n", #call,                  \
                   cudaGetErrorString(e_), __FILE__, __LINE__);                    \
      return e_ == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA;       \
    }                                                                              \
  } while (0)

#define CKS(call)                      \
  do {                                 \
    int s_ = (call);                   \
    if (s_ != STMG_OK) return s_;      \
  } while (0)

static cudaEvent_t new_event(stmg_handle* h) {
  if (!h->capturing && !h->free_events.empty()) {
    cudaEvent_t e = h->free_events.back();
    h->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  h->all_events.push_back(e);
  return e;
}

static void rec(stmg_handle* h, cudaEvent_t e, cudaStream_t s) {
  if (h->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

// profiling bracket: level 1 records only STMG_PROF_FINE_SWEEP, level 2 everything
struct Prof {
  stmg_handle* h; int cat; cudaStream_t s; cudaEvent_t a = nullptr, b = nullptr; int which;
  Prof(stmg_handle* h_, int cat_, cudaStream_t s_, int which_ = -1) : h(h_), cat(cat_), s(s_), which(which_) {
    const int need = cat == STMG_PROF_FINE_SWEEP ? 1 : 2;
    if (h->prof >= need) {
      a = new_event(h); b = new_event(h);
      if (a && b) rec(h, a, s);
    }
  }
  ~Prof() {
    if (a && b) {
      rec(h, b, s);
      if (h->capturing) h->graph_pairs[which].push_back({cat, a, b});
      else h->pending.push_back({cat, a, b});
    }
  }
};

static void harvest(stmg_handle* h, std::vector<ProfPair>& v, bool keep) {
  for (auto& p : v) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->prof_ms[p.cat] += ms;
      h->prof_n[p.cat] += 1;
      if (p.cat == STMG_PROF_FINE_SWEEP) { h->prof_ms[STMG_PROF_SMOOTHER] += ms; h->prof_n[STMG_PROF_SMOOTHER] += 1; }
    }
    if (!keep) { h->free_events.push_back(p.a); h->free_events.push_back(p.b); }
  }
  if (!keep) v.clear();
}

// read every completed profiling pair (call after the stream has been synchronised)
static void harvest_all(stmg_handle* h) {
  harvest(h, h->pending, false);
  for (int w = 0; w < 2; ++w)
    if (h->graph_pending[w]) { harvest(h, h->graph_pairs[w], true); h->graph_pending[w] = false; }
}

template <typename T> constexpr int prec_of();
template <> constexpr int prec_of<double>() { return STMG_FP64; }
template <> constexpr int prec_of<float>() { return STMG_FP32; }

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

template <typename T>
static void fill_apply_params(const LevelHost& H, ApplyParams<T>* p, int variant) {
  std::memset(p, 0, sizeof(*p));
  p->n = H.n; p->G = H.G; p->kt = H.kt; p->npm = H.npm;
  p->n_nodes = H.n_nodes; p->n_vel = H.n_vel; p->n_pres = H.n_pres;
  const int np = H.np;
  for (int i = 0; i < np * np; ++i) { p->M1[i] = (T)H.t1.M1[i]; p->K1[i] = (T)H.t1.K1[i]; }
  for (int i = 0; i < (H.r + 1) * np; ++i) { p->G1[i] = (T)H.t1.G1[i]; p->N1[i] = (T)H.t1.N1[i]; }
  for (int a = 0; a < H.kt; ++a) {
    for (int b = 0; b < H.kt; ++b) p->Kt[a * MAXKT + b] = (T)H.tt.K[a * H.kt + b];
    p->beta[a] = (T)(H.tt.M[a] * H.nu * std::pow(H.h, H.dim - 2));
    p->bscale[a] = (T)(-H.tt.M[a] * std::pow(H.h, H.dim - 1));
  }
  p->hd = (T)std::pow(H.h, H.dim);
  for (int m = 0; m < H.npm; ++m)
    for (int d = 0; d < 3; ++d) p->modes[m][d] = (signed char)H.modes[m][d];
  // cells per block: enough lines for ~128-256 threads, shared memory <= 64 KB
  const int lines = H.kt * H.dim * ipow(np, H.dim - 1);
  int cpb = std::max(1, 192 / lines);
  while (cpb > 1 && apply_smem_bytes<T>(H.dim, np, H.kt, H.npm, cpb) > 64 * 1024) --cpb;
  cpb = std::min(cpb, H.n_cells);
  p->cpb = cpb;
  p->variant = 1;
  p->tcx = p->tcy = std::min(4, H.n);
  while (p->tcx > 1 && apply2d_smem_bytes<T>(np, H.kt, H.npm, p->tcx, p->tcy) > 96 * 1024) p->tcx = p->tcy = p->tcx / 2;
  if (H.dim == 2 && variant != 1) p->variant = 2;   // node-centred form (2D levels)
}

template <typename T>
static void fill_apply_reg_params(const LevelHost& H, ApplyRegParams<T>* p) {
  std::memset(p, 0, sizeof(*p));
  p->n = H.n; p->G = H.G; p->kt = H.kt; p->npm = H.npm;
  p->n_nodes = H.n_nodes; p->n_vel = H.n_vel; p->n_pres = H.n_pres;
  const int np = H.np;
  for (int i = 0; i < np * np; ++i) { p->M1[i] = (T)H.t1.M1[i]; p->K1[i] = (T)H.t1.K1[i]; }
  if (H.dim == 2)
    for (int d = 0; d < 2; ++d)
      for (int e = 0; e <= H.r; ++e)
        for (int i = 0; i < np; ++i) {
          p->FX[d][e * np + i] = (T)(d == 0 ? H.t1.G1 : H.t1.N1)[e * np + i];
          p->FY[d][e * np + i] = (T)(d == 1 ? H.t1.G1 : H.t1.N1)[e * np + i];
        }
  for (int a = 0; a < H.kt; ++a) {
    for (int b = 0; b < H.kt; ++b) p->Kt[a * MAXKT + b] = (T)H.tt.K[a * H.kt + b];
    p->beta[a] = (T)(H.tt.M[a] * H.nu * std::pow(H.h, H.dim - 2));
    p->bscale[a] = (T)(-H.tt.M[a] * std::pow(H.h, H.dim - 1));
  }
  p->hd = (T)std::pow(H.h, H.dim);
}

template <typename T>
static void fill_transfer_params(const LevelHost& F, const LevelHost& C, TransferParams<T>* p) {
  std::memset(p, 0, sizeof(*p));
  p->dim = F.dim;
  p->h_type = F.n == 2 * C.n ? 1 : 0;
  p->nc = C.n; p->nf = F.n; p->npc = C.np; p->npf = F.np;
  p->ns = p->h_type ? 2 * (F.np - 1) + 1 : F.np;
  p->Gc = C.G; p->Gf = F.G; p->ktc = C.kt; p->ktf = F.kt; p->npmc = C.npm; p->npmf = F.npm;
  p->nnc = C.n_nodes; p->nnf = F.n_nodes; p->nvc = C.n_vel; p->nvf = F.n_vel;
  p->npc_tot = C.n_pres; p->npf_tot = F.n_pres;
  p->rc = C.r;
  p->variant = 1;
  for (int s = 0; s < p->ns; ++s) {
    double xi;
    if (p->h_type) {
      int child = std::min(s / (F.np - 1), 1);
      int loc = s - child * (F.np - 1);
      xi = 0.5 * (child + F.t1.xi[loc]);
    } else {
      xi = F.t1.xi[s];
    }
    for (int j = 0; j < C.np; ++j) {
      double v = lagrange_eval(C.t1.xi, C.np, j, xi);
      for (int jj = 0; jj < C.np; ++jj)
        if (std::fabs(xi - C.t1.xi[jj]) < 1e-14) v = (jj == j) ? 1.0 : 0.0;
      p->P1[s * MAXNP + j] = (T)v;
    }
  }
  // phi_ac^coarse at the fine Radau points.  The system's span has F.nsub = m C.nsub
  // subintervals on the fine level (m = 1: p in time per subinterval; m = 2: h in time);
  // fine subinterval jf lies in coarse subinterval jf / m, and its local Radau coordinate s
  // maps to xi = (2 (jf - m jc) + s + 1) / m - 1 there (right ends belong to their own
  // coarse subinterval: DG functions are evaluated from the left at interval ends).
  const int mt = F.nsub / C.nsub;
  for (int af = 0; af < F.kt; ++af)
    for (int ac = 0; ac < C.kt; ++ac) {
      const int jf = af / F.tt.k1, bf = af % F.tt.k1, jc = ac / C.tt.k1, bc = ac % C.tt.k1;
      double v = 0.0;
      if (jf / mt == jc) {
        const double xi = (2.0 * (jf - mt * jc) + F.tt.nodes1[bf] + 1.0) / mt - 1.0;
        v = lagrange_eval(C.tt.nodes1, C.tt.k1, bc, xi);
        for (int jj = 0; jj < C.tt.k1; ++jj)
          if (std::fabs(xi - C.tt.nodes1[jj]) < 1e-14) v = (jj == bc) ? 1.0 : 0.0;
      }
      p->Pt[af * MAXKT + ac] = (T)v;
    }
  // E[o][i' * (rc+1) + i] = int_0^1 L_i((o + xi)/2) L_i'(xi) dxi
  double gx[16], gw[16];
  const int nq = C.r + 2;
  gauss_legendre(nq, gx, gw);
  for (int o = 0; o < 2; ++o)
    for (int ip = 0; ip <= C.r; ++ip)
      for (int i = 0; i <= C.r; ++i) {
        double s = 0.0;
        for (int q = 0; q < nq; ++q) {
          const double xi = 0.5 * (gx[q] + 1.0), w = 0.5 * gw[q];
          s += w * legendre_unit(i, 0.5 * (o + xi)) * legendre_unit(ip, xi);
        }
        p->E[o][ip * (C.r + 1) + i] = (T)(std::fabs(s) < 1e-15 ? 0.0 : s);
      }
  for (int m = 0; m < C.npm; ++m) for (int d = 0; d < 3; ++d) p->modes_c[m][d] = (signed char)C.modes[m][d];
  for (int m = 0; m < F.npm; ++m) for (int d = 0; d < 3; ++d) p->modes_f[m][d] = (signed char)F.modes[m][d];
  p->cpb = 1;
  while (p->cpb < 8 && transfer_smem<T>(*p, 0) * 2 <= 48 * 1024 && transfer_smem<T>(*p, 1) * 2 <= 48 * 1024)
    p->cpb *= 2;
  const int ncd = F.dim == 2 ? C.n * C.n : C.n * C.n * C.n;
  if (p->cpb > ncd) p->cpb = ncd;
}

template <typename T>
static int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA;
  }
  return STMG_OK;
}

// with_inverses = false sets up only the operator and the work vectors (the finest level
// always has FP64 operator data: FGMRES applies S in FP64 whatever the V-cycle precision)
// the operator kernels enumerate the pressure modes at compile time (mode_exp)
static bool modes_in_kernel_order(const LevelHost& H) {
  if ((int)H.modes.size() != H.npm) return false;
  for (int m = 0; m < H.npm; ++m)
    for (int k = 0; k < H.dim; ++k)
      if (H.modes[m][k] != mode_exp(H.dim, H.r, m, k)) return false;
  return true;
}

// the register-resident operator forms index the 2D pressure modes by mode_index
static bool modes_graded_2d(const LevelHost& H) {
  if (H.dim != 2 || (int)H.modes.size() != H.npm) return false;
  for (int m = 0; m < H.npm; ++m)
    if (mode_index(H.modes[m][0], H.modes[m][1]) != m) return false;
  return true;
}
template <typename T>
static bool reg_form_ok(const LevelHost& H) {
  return H.dim == 2 && modes_graded_2d(H) && apply2d_reg_supported<T>(H.np, H.kt, H.npm);
}
template <typename T>
static bool pair_form_ok(const LevelHost& H) {
  return reg_form_ok<T>(H) && apply2d_pair_supported<T>(H.np, H.kt, H.npm);
}

template <typename T>
static int setup_precision(stmg_handle* h, LevelDev& lv, const double* d_cls, const int* d_cls_of,
                           bool with_inverses = true) {
  PrecDev<T>& P = lv.pd<T>();
  const LevelHost& H = lv.H;
  fill_apply_params<T>(H, &P.ap, h->cfg.apply_variant);
  fill_apply_reg_params<T>(H, &P.rp);
  const int av = h->cfg.apply_variant;
  if (pair_form_ok<T>(H) && av == 4)
    P.ap.variant = 4;                    // its pair-split form, on request
  else if (reg_form_ok<T>(H) && (av == 0 || av == 3 || av == 4))
    P.ap.variant = 3;                    // register-resident form where the cell tile fits
  if (P.ap.variant >= 3) P.ap.cpb = 64;  // threads per block of the register forms (tuned later)
  CKS(dalloc(&P.b, H.size));
  CKS(dalloc(&P.x, H.size));
  CKS(dalloc(&P.r, H.size));
  if (std::is_same<T, float>::value && H.dim == 2) CKS(dalloc(&P.x2, H.size));
  if (H.smoother >= 0 && with_inverses) {
    // omega / valence per dof (FP64), folded into the rows of every stored inverse
    std::vector<double> w(H.size, 0.0);
    for (long long i = 0; i < H.size; ++i)
      if (H.valence[i] > 0) w[i] = h->cfg.omega / H.valence[i];
    double* d_w = nullptr;
    CKS(dalloc(&d_w, H.size));
    CK(cudaMemcpy(d_w, w.data(), sizeof(double) * H.size, cudaMemcpyHostToDevice));
    int s = STMG_OK;
    if (std::is_same<T, float>::value && h->cfg.half_inverses) {
      const int Bh = (H.B + 7) / 8 * 8;
      s = dalloc(&P.invh, (size_t)H.n_patches * H.B * Bh);
      if (s == STMG_OK) s = dalloc(&P.rsc, (size_t)H.n_patches * H.B);
      if (s == STMG_OK && launch_replicate_inverses_half(d_cls, d_cls_of, lv.dofs, d_w, P.invh, P.rsc, H.n_patches,
                                                         H.B, Bh, h->st) != cudaSuccess)
        s = STMG_ERR_CUDA;
      P.half = true;
    } else {
      s = dalloc(&P.inv, (size_t)H.n_patches * H.B * H.Bc);
      if (s == STMG_OK && launch_replicate_inverses<T>(d_cls, d_cls_of, lv.dofs, d_w, P.inv, H.n_patches, H.B,
                                                       H.Bc, h->st) != cudaSuccess)
        s = STMG_ERR_CUDA;
    }
    cudaStreamSynchronize(h->st);
    cudaFree(d_w);
    if (s != STMG_OK) return s;
    P.has_inv = true;
  }
  return STMG_OK;
}

static void free_level(LevelDev& lv) {
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(lv.dofs); f(lv.G); f(lv.Gacc); f(lv.Gf);
  f(lv.d.inv); f(lv.d.b); f(lv.d.x); f(lv.d.r); f(lv.f.invh); f(lv.f.rsc);
  f(lv.f.inv); f(lv.f.b); f(lv.f.x); f(lv.f.r); f(lv.f.x2); f(lv.d.x2);
  lv = LevelDev();
}

// ------------------------------------------------------------------------------------
// level operations (enqueue on stream s)
// ------------------------------------------------------------------------------------
template <typename T>
static int op_apply(stmg_handle* h, int l, const T* x, const T* b, T* y, int mode, cudaStream_t s) {
  LevelDev& lv = h->L[l];
  const ApplyParams<T>& ap = lv.pd<T>().ap;
  if (ap.variant == 2) {                 // writes every entry of y
    CK(launch_apply2d<T>(lv.H.np, ap, x, b, y, mode, s));
  } else if (ap.variant == 3) {          // scatter-adds every row
    CK(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)lv.H.size, s));
    CK(launch_apply2d_reg<T>(lv.H.np, lv.pd<T>().rp, x, b, y, mode, ap.cpb >= 16 ? ap.cpb : 64, s));
  } else if (ap.variant == 4) {          // scatter-adds every row
    CK(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)lv.H.size, s));
    CK(launch_apply2d_pair<T>(lv.H.np, lv.pd<T>().rp, x, b, y, mode, s));
  } else {
    CK(cudaMemsetAsync(y, 0, sizeof(T) * lv.H.size, s));
    CK(launch_apply<T>(lv.H.dim, lv.H.np, ap, x, b, y, mode, s));
  }
  h->launches += 1;
  return STMG_OK;
}

template <typename T>
static int op_sweep(stmg_handle* h, int l, const T* res, T* x, cudaStream_t s) {
  LevelDev& lv = h->L[l];
  PrecDev<T>& P = lv.pd<T>();
  if (!P.has_inv) return STMG_ERR_ARG;
  Prof pr(h, l == 0 ? STMG_PROF_FINE_SWEEP : STMG_PROF_SMOOTHER, s, prec_of<T>());
  const int w = prec_of<T>();
  if (P.half)
    CK(launch_vanka_sweep_half(lv.dofs, P.invh, P.rsc, (const float*)res, (float*)x, lv.H.n_patches, lv.H.B,
                               (lv.H.B + 7) / 8 * 8, lv.ppb[w], lv.streaming, s));
  else if (lv.sweep_var[w] == 2 && tma_sweep_supported<T>(lv.H.B))
    CK(launch_vanka_sweep_tma<T>(lv.dofs, P.inv, res, x, lv.H.n_patches, lv.H.B, lv.H.Bc, h->n_sm,
                                 lv.streaming, h->d_err, s));
  else if (lv.sweep_var[w] == 3 && pipe_sweep_supported<T>(lv.H.B, lv.ppb[w]))
    CK(launch_vanka_sweep_pipe<T>(lv.dofs, P.inv, res, x, lv.H.n_patches, lv.H.B, lv.H.Bc, lv.ppb[w], lv.unroll[w],
                                  lv.streaming, s));
  else
    CK(launch_vanka_sweep<T>(lv.dofs, P.inv, res, x, lv.H.n_patches, lv.H.B, lv.H.Bc, lv.ppb[w], lv.unroll[w],
                             lv.streaming, s));
  h->launches += 1;
  return STMG_OK;
}

// b_c = P^T r_f; with zc != NULL also zc = 0 (the coarse iterate), by the gather form in the
// same launch, else by a zero-fill
template <typename T>
static int op_restrict(stmg_handle* h, int l, const T* rf, T* bc, cudaStream_t s, T* zc = nullptr) {
  LevelDev& lc = h->L[l + 1];
  const TransferParams<T>& tp = h->L[l].pd<T>().tp;
  const bool gather = tp.variant == 2 && transfer_gather_supported(tp);
  if (!gather) {                                  // the gather form writes all of b_c (and zc)
    CK(cudaMemsetAsync(bc, 0, sizeof(T) * lc.H.size, s));
    if (zc) CK(cudaMemsetAsync(zc, 0, sizeof(T) * lc.H.size, s));
  }
  CK(launch_restrict<T>(tp, rf, bc, gather ? zc : nullptr, s));
  h->launches += 1;
  return STMG_OK;
}

template <typename T>
static int op_prolongate_add(stmg_handle* h, int l, const T* yc, T* xf, cudaStream_t s) {
  CK(launch_prolongate<T>(h->L[l].pd<T>().tp, yc, xf, s));
  h->launches += 1;
  return STMG_OK;
}

template <typename T>
static int op_coarse(stmg_handle* h, const T* b, T* x, cudaStream_t s) {
  LevelDev& lv = h->L.back();
  const int D = (int)lv.H.size;
  const bool g32 = std::is_same<T, float>::value && lv.Gf;   // FP32 V-cycle: the FP32 copy of G
  if (lv.Gacc) {
    if (g32) CK((launch_coarse_tiled<float, float>(D, lv.Gf, (const float*)b, (float*)x, lv.Gacc, s)));
    else CK((launch_coarse_tiled<T, double>(D, lv.G, b, x, lv.Gacc, s)));
    h->launches += 2;
  } else {
    if (g32) CK((launch_coarse<float, float>(D, lv.Gf, (const float*)b, (float*)x, s)));
    else CK((launch_coarse<T, double>(D, lv.G, b, x, s)));
    h->launches += 1;
  }
  return STMG_OK;
}

// ------------------------------------------------------------------------------------
// Launch-parameter tuner: per level and precision, time each candidate launch shape with
// CUDA events (3 warm-up launches, then up to three trials of 5 launches, the fastest
// trial counting, on the level's own work vectors, whose contents are irrelevant to the
// timing) and keep the fastest.  The clocks are brought up first: after the host-side
// setup the GPU may be idle, and a clock that is still ramping favours whichever
// candidate is timed last.
//   sweep      block sweep with 1, 2, 4, 8 patches per block, or the TMA-pipelined sweep
//   apply      1 ... 32 cells per block (shared memory <= 100 KB)
//   transfers  1 ... 32 coarse cells per block for restriction + prolongation
// ------------------------------------------------------------------------------------
// Device time of one candidate: five back-to-back launches captured in a CUDA graph on the
// internal stream (so the host's launch overhead, larger than a small level's kernel, does
// not enter), the graph replayed three times after a warm-up, the fastest replay counting.
// The launches that precede the capture run eagerly, outside capture (kernel attributes).
template <typename F>
static int time_it(stmg_handle* h, F&& fn, float* ms) {
  cudaEvent_t a = new_event(h), b = new_event(h);
  if (!a || !b) return STMG_ERR_CUDA;
  cudaStream_t saved = h->st;
  const int saved_prof = h->prof;
  h->prof = 0;
  h->st = h->gst;
  int st = STMG_OK;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  auto run = [&]() -> int {
    for (int i = 0; i < 2; ++i) CKS(fn());
    CK(cudaStreamSynchronize(h->gst));
    CK(cudaStreamBeginCapture(h->gst, cudaStreamCaptureModeRelaxed));
    int s = STMG_OK;
    for (int i = 0; i < 5 && s == STMG_OK; ++i) s = fn();
    cudaError_t e = cudaStreamEndCapture(h->gst, &g);
    CKS(s);
    CK(e);
    CK(cudaGraphInstantiate(&ge, g, 0));
    CK(cudaGraphLaunch(ge, h->gst));
    float best = 1e30f;
    for (int trial = 0; trial < 3; ++trial) {
      CK(cudaEventRecord(a, h->gst));
      CK(cudaGraphLaunch(ge, h->gst));
      CK(cudaEventRecord(b, h->gst));
      CK(cudaEventSynchronize(b));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, a, b));
      if (t < best) best = t;
      if (t > 5.f) break;                  // long launches: one trial is stable
    }
    *ms = best;
    return STMG_OK;
  };
  st = run();
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (st != STMG_OK) cudaGetLastError();
  h->st = saved;
  h->prof = saved_prof;
  h->free_events.push_back(a);
  h->free_events.push_back(b);
  return st;
}

// level 0's residual, repeated until about 20 ms of device time has passed
template <typename T>
static int warm_clocks_t(stmg_handle* h) {
  PrecDev<T>& P = h->L[0].pd<T>();
  float total = 0.f, ms = 0.f;
  for (int it = 0; it < 64 && total < 20.f; ++it) {
    CKS(time_it(h, [&]() { return op_apply<T>(h, 0, P.x, P.b, P.r, RESIDUAL, h->st); }, &ms));
    total += 1.6f * ms;                  // at least 8 launches of at least ms / 5 each
  }
  return STMG_OK;
}

static int warm_clocks(stmg_handle* h) {
  const long long saved = h->launches;
  int st = STMG_OK;
  if (h->L[0].pd<float>().b) st = warm_clocks_t<float>(h);
  else if (h->L[0].pd<double>().b) st = warm_clocks_t<double>(h);
  h->launches = saved;
  return st;
}

template <typename T>
static int autotune_level(stmg_handle* h, int l) {
  LevelDev& lv = h->L[l];
  PrecDev<T>& P = lv.pd<T>();
  if (!P.b) return STMG_OK;
  const int w = prec_of<T>();
  const size_t bytes = sizeof(T) * lv.H.size;
  CK(cudaMemsetAsync(P.b, 0, bytes, h->st));
  CK(cudaMemsetAsync(P.x, 0, bytes, h->st));
  CK(cudaMemsetAsync(P.r, 0, bytes, h->st));
  const long long saved = h->launches;
  const bool last = l + 1 == (int)h->L.size();
  float best = 1e30f, ms = 0.f;
  if (!last && P.has_inv) {
    int best_var = 1, best_ppb = lv.ppb[w], best_unroll = lv.unroll[w];
    const int only = h->cfg.sweep_variant;             // 0: free choice, 1 / 2 / 3: fixed variant
    for (int ppb = 1; ppb <= 8 && (only == 0 || only == 1); ppb *= 2) {
      if (ppb > 1 && ppb * lv.H.B > 1024) break;
      for (int u = 4; u <= 8; u += 4) {
        lv.sweep_var[w] = 1;
        lv.ppb[w] = ppb;
        lv.unroll[w] = u;
        CKS(time_it(h, [&]() { return op_sweep<T>(h, l, P.r, P.x, h->st); }, &ms));
        if (ms < best) { best = ms; best_var = 1; best_ppb = ppb; best_unroll = u; }
      }
    }
    if ((only == 0 || only == 2) && !P.half && tma_sweep_supported<T>(lv.H.B)) {
      lv.sweep_var[w] = 2;
      CKS(time_it(h, [&]() { return op_sweep<T>(h, l, P.r, P.x, h->st); }, &ms));
      if (ms < best) { best = ms; best_var = 2; }
    }
    for (int ppb = 1; ppb <= 8 && (only == 0 || only == 3) && !P.half; ppb *= 2) {
      if (!pipe_sweep_supported<T>(lv.H.B, ppb)) break;
      for (int u = 4; u <= 8; u += 4) {
        lv.sweep_var[w] = 3;
        lv.ppb[w] = ppb;
        lv.unroll[w] = u;
        CKS(time_it(h, [&]() { return op_sweep<T>(h, l, P.r, P.x, h->st); }, &ms));
        if (ms < best) { best = ms; best_var = 3; best_ppb = ppb; best_unroll = u; }
      }
    }
    lv.sweep_var[w] = best_var;
    lv.ppb[w] = best_ppb;
    lv.unroll[w] = best_unroll;
  }
  {
    best = 1e30f;
    int best_cpb = P.ap.cpb, best_var = 1, best_tx = P.ap.tcx, best_ty = P.ap.tcy;
    const int fixed = lv.H.dim == 2 ? h->cfg.apply_variant : 1;   // 0: free choice, 1 / 2: fixed variant
    P.ap.variant = 1;
    for (int cpb = 1; cpb <= 32 && cpb <= lv.H.n_cells && (fixed == 0 || fixed == 1); cpb *= 2) {
      if (apply_smem_bytes<T>(lv.H.dim, lv.H.np, lv.H.kt, lv.H.npm, cpb) > 100 * 1024) break;
      P.ap.cpb = cpb;
      CKS(time_it(h, [&]() { return op_apply<T>(h, l, P.x, P.b, P.r, RESIDUAL, h->st); }, &ms));
      if (ms < best) { best = ms; best_cpb = cpb; }
    }
    if (lv.H.dim == 2 && (fixed == 0 || fixed == 2)) {   // node-centred form: tiles of tx x ty cells
      static const int tiles[][2] = {{2, 2}, {4, 2}, {4, 4}, {8, 4}, {8, 8}, {16, 8}};
      P.ap.variant = 2;
      for (const auto& t : tiles) {
        if (t[0] > 2 * lv.H.n || t[1] > 2 * lv.H.n) continue;
        if (apply2d_smem_bytes<T>(lv.H.np, lv.H.kt, lv.H.npm, t[0], t[1]) > 100 * 1024) continue;
        P.ap.tcx = std::min(t[0], lv.H.n);
        P.ap.tcy = std::min(t[1], lv.H.n);
        CKS(time_it(h, [&]() { return op_apply<T>(h, l, P.x, P.b, P.r, RESIDUAL, h->st); }, &ms));
        if (ms < best) { best = ms; best_var = 2; best_tx = P.ap.tcx; best_ty = P.ap.tcy; }
      }
    }
    const bool pair = pair_form_ok<T>(lv.H);
    if ((fixed == 0 || fixed == 3 || (fixed == 4 && !pair)) && reg_form_ok<T>(lv.H)) {
      // register-resident form: 64 threads per block, or the block size that gives every
      // SM the same number of items (k or k + 1 blocks per SM)
      P.ap.variant = 3;
      const long long items = (long long)lv.H.n * lv.H.n * lv.H.kt * 2;
      const long long per = (items + 64LL * h->n_sm - 1) / (64LL * h->n_sm);   // blocks per SM at 64
      int sizes[3] = {64, (int)((items + h->n_sm * per - 1) / (h->n_sm * per)),
                      (int)((items + h->n_sm * (per + 1) - 1) / (h->n_sm * (per + 1)))};
      for (int bs : sizes) {
        if (bs < 16 || bs > 64) continue;
        P.ap.cpb = bs;                   // the block size of this form
        CKS(time_it(h, [&]() { return op_apply<T>(h, l, P.x, P.b, P.r, RESIDUAL, h->st); }, &ms));
        if (ms < best) { best = ms; best_var = 3; best_cpb = bs; }
      }
    }
    if ((fixed == 0 || fixed == 4) && pair) {
      P.ap.variant = 4;                  // its pair-split form
      CKS(time_it(h, [&]() { return op_apply<T>(h, l, P.x, P.b, P.r, RESIDUAL, h->st); }, &ms));
      if (ms < best) { best = ms; best_var = 4; }
    }
    P.ap.cpb = best_cpb;
    P.ap.variant = best_var;
    P.ap.tcx = best_tx;
    P.ap.tcy = best_ty;
  }
  if (!last && h->L[l + 1].pd<T>().b) {
    PrecDev<T>& C = h->L[l + 1].pd<T>();
    const int ncd = lv.H.dim == 2 ? h->L[l + 1].H.n * h->L[l + 1].H.n : h->L[l + 1].H.n * h->L[l + 1].H.n * h->L[l + 1].H.n;
    best = 1e30f;
    int best_cpb = P.tp.cpb, best_var = P.tp.variant;
    const int fixed = h->cfg.transfer_variant;        // 0: free choice, 1 / 2: fixed variant
    auto pair = [&]() {
      CKS(op_restrict<T>(h, l, P.r, C.b, h->st));
      return op_prolongate_add<T>(h, l, C.x, P.x, h->st);
    };
    if (fixed != 2 || !transfer_gather_supported(P.tp)) {
      P.tp.variant = 1;
      for (int cpb = 1; cpb <= 32 && cpb <= ncd; cpb *= 2) {
        P.tp.cpb = cpb;
        if (transfer_smem<T>(P.tp, 0) > 100 * 1024 || transfer_smem<T>(P.tp, 1) > 100 * 1024) break;
        CKS(time_it(h, pair, &ms));
        if (ms < best) { best = ms; best_cpb = cpb; best_var = 1; }
      }
    }
    if (fixed != 1 && transfer_gather_supported(P.tp)) {
      P.tp.variant = 2;
      CKS(time_it(h, pair, &ms));
      if (ms < best) { best = ms; best_var = 2; }
    }
    P.tp.cpb = best_cpb;
    P.tp.variant = best_var;
  }
  h->launches = saved;
  return STMG_OK;
}

template <typename T>
static int vcycle_level(stmg_handle* h, int l, cudaStream_t s);

// ------------------------------------------------------------------------------------
// Persistent multigrid kernel: which levels it can run, its level descriptors, and where
// the tuner lets it start.
// ------------------------------------------------------------------------------------
template <typename T>
static bool mgp_level_ok(const stmg_handle* h, int i) {
  const LevelDev& lv = h->L[i];
  const LevelHost& H = lv.H;
  const PrecDev<T>& P = const_cast<LevelDev&>(lv).pd<T>();
  const bool coarsest = i + 1 == (int)h->L.size();
  if (H.dim != 2 || !P.b) return false;
  if (coarsest) return H.size <= 1 << 15;              // FP64 bordered inverse of the coarsest level
  if (H.np != 3 || H.kt > 4 || H.npm != 3 || !P.has_inv || P.half || H.B > 256) return false;
  const TransferParams<T>& tp = P.tp;
  return tp.dim == 2 && tp.npf == 3 && tp.npc == 3 && 2 * tp.ktf <= 256 && tp.ktc <= tp.ktf;
}

template <typename T>
static int mgp_setup(stmg_handle* h) {
  const int w = prec_of<T>();
  const int L = (int)h->L.size();
  h->mgp_first[w] = h->mgp_eligible[w] = 0;
  if (L < 3 || !h->L[0].pd<T>().b) return STMG_OK;
  int first = L - 1;                                    // lowest level from which every level is covered
  while (first > 1 && mgp_level_ok<T>(h, first - 1)) --first;
  if (!mgp_level_ok<T>(h, L - 1) || first > L - 2) return STMG_OK;   // needs at least one smoothed level
  if (!h->mgp_bar) {
    CKS(dalloc(&h->mgp_bar, 2));
    CK(cudaMemset(h->mgp_bar, 0, 2 * sizeof(unsigned)));
  }
  h->mgp_bpsm[w] = mg_persist_blocks<T>(h->n_sm);
  h->mgp_blocks[w] = h->n_sm * h->mgp_bpsm[w];
  if (h->mgp_blocks[w] < 1) return STMG_OK;
  LevelDev& lc = h->L[L - 1];
  if (!lc.Gacc) {
    CKS(dalloc(&lc.Gacc, lc.H.size));
    CK(cudaMemset(lc.Gacc, 0, sizeof(double) * lc.H.size));
  }
  std::vector<MGLevelDesc<T>> d(L - first);
  for (int i = first; i < L; ++i) {
    LevelDev& lv = h->L[i];
    PrecDev<T>& P = lv.pd<T>();
    MGLevelDesc<T>& e = d[i - first];
    std::memset(&e, 0, sizeof(e));
    e.rp = P.rp;
    e.tp = P.tp;
    e.b = P.b; e.x = P.x; e.r = P.r;
    e.dofs = lv.dofs;
    e.inv = P.inv;
    e.n_patches = lv.H.n_patches;
    e.size = lv.H.size;
    e.B = lv.H.B; e.Bc = lv.H.Bc;
    e.ppb = lv.H.B > 0 ? std::max(1, 256 / lv.H.B) : 1;
    e.kt = lv.H.kt;
    e.ht = P.tp.h_type;
    if (i == L - 1) { e.G = lv.G; e.acc = lv.Gacc; e.D = (int)lv.H.size; }
  }
  if (h->mgp_desc[w]) cudaFree(h->mgp_desc[w]);
  h->mgp_desc[w] = nullptr;
  MGLevelDesc<T>* dd = nullptr;
  CKS(dalloc(&dd, d.size()));
  h->mgp_desc[w] = dd;
  CK(cudaMemcpy(dd, d.data(), sizeof(MGLevelDesc<T>) * d.size(), cudaMemcpyHostToDevice));
  h->mgp_eligible[w] = first;
  // the descriptor array starts at level `first`; a later start uses its tail
  return STMG_OK;
}

// Device time of one V-cycle of precision T (zero-guess iterate not reset between the
// timed repetitions: the cost does not depend on the values).
template <typename T>
static int time_vcycle(stmg_handle* h, float* ms) {
  return time_it(h, [&]() { return vcycle_level<T>(h, 0, h->st); }, ms);
}

// Where the persistent kernel starts (or whether it runs at all): per precision, the
// fastest V-cycle among "one kernel per operation" and every admissible first level.
template <typename T>
static int mgp_choose(stmg_handle* h) {
  const int w = prec_of<T>();
  const int first = h->mgp_eligible[w];
  h->mgp_first[w] = 0;
  if (first < 1 || h->cfg.persistent == 0) return STMG_OK;
  if (h->cfg.persistent == 2 || !h->cfg.autotune) { h->mgp_first[w] = first; return STMG_OK; }
  float best = 1e30f, ms = 0.f;
  int best_first = 0, best_blocks = h->mgp_blocks[w];
  const int L = (int)h->L.size();
  for (int f = 0; f <= L - 2; ++f) {
    if (f != 0 && f < first) continue;
    for (int bps = 1; bps <= h->mgp_bpsm[w]; ++bps) {   // grid: 1 or 2 blocks per SM (barrier cost vs width)
      if (f == 0 && bps > 1) break;
      h->mgp_first[w] = f;
      h->mgp_blocks[w] = h->n_sm * bps;
      CKS(time_vcycle<T>(h, &ms));
      if (ms < best) { best = ms; best_first = f; best_blocks = h->mgp_blocks[w]; }
    }
  }
  h->mgp_first[w] = best_first;
  h->mgp_blocks[w] = best_blocks;
  return STMG_OK;
}

static int autotune_impl(stmg_handle* h) {
  CKS(warm_clocks(h));
  for (size_t l = 0; l < h->L.size(); ++l) {
    CKS(autotune_level<double>(h, (int)l));
    CKS(autotune_level<float>(h, (int)l));
  }
  {
    const long long saved = h->launches;
    CKS(mgp_setup<double>(h));
    CKS(mgp_setup<float>(h));
    CKS(mgp_choose<double>(h));
    CKS(mgp_choose<float>(h));
    h->launches = saved;
  }
  for (auto& g : h->graph) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  h->graph_pairs[0].clear(); h->graph_pairs[1].clear();
  if (h->st) CK(cudaStreamSynchronize(h->st)); else CK(cudaDeviceSynchronize());
  return STMG_OK;
}

// Whether level l's post-smoothing residual takes the coarser level's correction through
// the fused kernel (prolongation and residual in one launch, the result in x2): FP32, a 2D
// register-resident level with a transfer shape the fused kernel covers, not inside the
// persistent multigrid kernel.
template <typename T>
static bool fused_up(const stmg_handle* h, int l) {
  if (!std::is_same<T, float>::value || !h->cfg.fuse_transfers || h->cfg.nu2 < 1) return false;
  if (l + 1 >= (int)h->L.size()) return false;
  const int w = prec_of<T>();
  if (h->mgp_first[w] > 0 && l >= h->mgp_first[w]) return false;
  const LevelDev& lv = h->L[l];
  const PrecDev<float>& P = lv.f;
  return P.x2 && reg_form_ok<float>(lv.H) &&
         apply2d_reg_pro_supported(lv.H.np, lv.H.kt, lv.H.npm, P.tp.npc, P.tp.h_type, P.tp.ktc);
}

// Whether level l's descent computes its residual and restricts it in one launch: FP32,
// the same levels and transfer shapes as fused_up, with presmoothing.
template <typename T>
static bool fused_down(const stmg_handle* h, int l) {
  if (!std::is_same<T, float>::value || !h->cfg.fuse_transfers || h->cfg.nu1 < 1) return false;
  if (l + 1 >= (int)h->L.size()) return false;
  const int w = prec_of<T>();
  if (h->mgp_first[w] > 0 && l >= h->mgp_first[w]) return false;
  const LevelDev& lv = h->L[l];
  const PrecDev<float>& P = lv.f;
  return reg_form_ok<float>(lv.H) &&
         apply2d_reg_pro_supported(lv.H.np, lv.H.kt, lv.H.npm, P.tp.npc, P.tp.h_type, P.tp.ktc);
}

// where level l's V-cycle leaves its iterate
template <typename T>
static T* final_x(stmg_handle* h, int l) {
  PrecDev<T>& P = h->L[l].pd<T>();
  return fused_up<T>(h, l) ? P.x2 : P.x;
}

// V-cycle on level l: input L[l].b, output final_x(l) from the zero initial guess, Alg. 1.
// L[l].x must be zero on entry: on the finest level the caller zeroes it (with the
// conversion of the right-hand side), on the coarser ones the restriction does.
template <typename T>
static int vcycle_level(stmg_handle* h, int l, cudaStream_t s) {
  LevelDev& lv = h->L[l];
  if (l == 0) {
    // the coarser right-hand sides that the fused restrictions accumulate into, zeroed
    // together in one launch (every V-cycle enters here at the finest level)
    ZeroList z{};
    for (int i = 0; i + 1 < (int)h->L.size() && z.count < ZeroList::MAX; ++i)
      if (fused_down<T>(h, i)) {
        z.p[z.count] = (float*)h->L[i + 1].f.b;
        z.n[z.count] = h->L[i + 1].H.size;
        ++z.count;
      }
    if (z.count > 0) {
      CK(launch_zero_many(z, s));
      h->launches += 1;
    }
  }
  PrecDev<T>& P = lv.pd<T>();
  const int w = prec_of<T>();
  if (h->mgp_first[w] > 0 && l == h->mgp_first[w]) {   // this level and all coarser ones in one launch
    CK(launch_mg_persist<T>(reinterpret_cast<const MGLevelDesc<T>*>(h->mgp_desc[w]) + (l - h->mgp_eligible[w]),
                            (int)h->L.size() - l,
                            h->cfg.nu1, h->cfg.nu2, h->mgp_bar, h->d_err, h->mgp_blocks[w], s));
    h->launches += 1;
    return STMG_OK;
  }
  if (l == (int)h->L.size() - 1) return op_coarse<T>(h, P.b, P.x, s);
  for (int it = 0; it < h->cfg.nu1; ++it) {          // presmoothing (Eq. Alg:VGMGPre)
    if (it == 0) {
      CKS(op_sweep<T>(h, l, P.b, P.x, s));           // x = 0: the residual is b
    } else {
      CKS(op_apply<T>(h, l, P.x, P.b, P.r, RESIDUAL, s));
      CKS(op_sweep<T>(h, l, P.r, P.x, s));
    }
  }
  PrecDev<T>& C = h->L[l + 1].pd<T>();
  if (fused_down<T>(h, l)) {
    // steps 1-3 of Alg. 4 / 5 in one launch: C.b = P^T (b - S x), C.x = 0
    LevelDev& lf = h->L[l];
    if (l >= ZeroList::MAX) CK(cudaMemsetAsync(C.b, 0, sizeof(T) * (size_t)h->L[l + 1].H.size, s));
    CK(launch_apply2d_reg_rst(lf.H.np, lf.f.rp, lf.f.tp, (const float*)P.x, (const float*)P.b, (float*)C.b,
                              (float*)C.x, lf.f.ap.variant == 3 && lf.f.ap.cpb >= 16 ? lf.f.ap.cpb : 64, s));
    h->launches += 1;
  } else {
    const T* res = P.b;
    if (h->cfg.nu1 > 0) {                            // step 1 of Alg. 4 / 5
      CKS(op_apply<T>(h, l, P.x, P.b, P.r, RESIDUAL, s));
      res = P.r;
    }
    CKS(op_restrict<T>(h, l, res, C.b, s, C.x));     // step 2/3 of Alg. 4 / 5; C.x = 0
  }
  CKS(vcycle_level<T>(h, l + 1, s));
  const T* ec = final_x<T>(h, l + 1);
  T* xu = P.x;
  int it0 = 0;
  if (fused_up<T>(h, l)) {
    // x2 = x + P ec and r = b - S x2 in one launch (Alg. 6 / 7 and the first
    // postsmoothing residual); the postsmoothing then updates x2
    LevelDev& lf = h->L[l];
    CK(cudaMemsetAsync(P.r, 0, sizeof(T) * (size_t)lf.H.size, s));
    CK(launch_apply2d_reg_pro(lf.H.np, lf.f.rp, lf.f.tp, (const float*)P.x, (const float*)ec, (const float*)P.b,
                              (float*)P.r, (float*)P.x2, lf.f.ap.variant == 3 && lf.f.ap.cpb >= 16 ? lf.f.ap.cpb : 64,
                              s));
    h->launches += 1;
    xu = P.x2;
    CKS(op_sweep<T>(h, l, P.r, xu, s));
    it0 = 1;
  } else {
    CKS(op_prolongate_add<T>(h, l, ec, P.x, s));     // Alg. 6 / 7
  }
  for (int it = it0; it < h->cfg.nu2; ++it) {        // postsmoothing (Eq. Alg:VGMGPost)
    CKS(op_apply<T>(h, l, xu, P.b, P.r, RESIDUAL, s));
    CKS(op_sweep<T>(h, l, P.r, xu, s));
  }
  return STMG_OK;
}

// Run the V-cycle on the finest level's fixed buffers, through a CUDA graph if enabled.
template <typename T>
static int run_vcycle(stmg_handle* h) {
  const int w = prec_of<T>();
  if (!h->cfg.use_graphs) return vcycle_level<T>(h, 0, h->st);
  if (!h->graph[w]) {
    // warm-up run (sets kernel attributes outside capture), then capture on gst
    CK(cudaEventRecord(h->ev_fork, h->st));
    CK(cudaStreamWaitEvent(h->gst, h->ev_fork, 0));
    CKS(vcycle_level<T>(h, 0, h->gst));
    CK(cudaStreamSynchronize(h->gst));
    harvest(h, h->pending, false);
    const long long before = h->launches;
    CK(cudaStreamBeginCapture(h->gst, cudaStreamCaptureModeRelaxed));
    h->capturing = true;
    int s = vcycle_level<T>(h, 0, h->gst);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->gst, &g);
    if (s != STMG_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return STMG_ERR_CUDA;
    e = cudaGraphInstantiate(&h->graph[w], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->graph[w] = nullptr; return STMG_ERR_CUDA; }
    h->graph_kernels[w] = h->launches - before;
    h->launches = before;
    CK(cudaEventRecord(h->ev_join, h->gst));
    CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    return STMG_OK;   // the warm-up run already produced this V-cycle's output
  }
  CK(cudaEventRecord(h->ev_fork, h->st));
  CK(cudaStreamWaitEvent(h->gst, h->ev_fork, 0));
  CK(cudaGraphLaunch(h->graph[w], h->gst));
  h->launches += h->graph_kernels[w];
  CK(cudaEventRecord(h->ev_join, h->gst));
  CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
  if (h->prof && !h->graph_pairs[w].empty()) h->graph_pending[w] = true;
  return STMG_OK;
}

// z = M v (FP64 in and out) with the V-cycle in precision prec
// ready: the FP32 V-cycle's b (= (float) v) and zero x are already in place (written by
// the Arnoldi step that produced v)
static int precondition(stmg_handle* h, int prec, const double* v, double* z, bool ready = false) {
  LevelDev& l0 = h->L[0];
  const long long D = l0.H.size;
  Prof pr(h, PROF_VCYCLE, h->st);
  if (prec == STMG_FP64) {
    if (!l0.d.b) return STMG_ERR_ARG;
    CK((launch_convert_zero<double, double>(D, v, l0.d.b, l0.d.x, h->st)));   // b = v, x = 0
    CKS(run_vcycle<double>(h));
    CK(cudaMemcpyAsync(z, l0.d.x, sizeof(double) * D, cudaMemcpyDeviceToDevice, h->st));
    h->launches += 1;
  } else {
    if (!l0.f.b) return STMG_ERR_ARG;
    if (!ready) {
      CK((launch_convert_zero<double, float>(D, v, l0.f.b, l0.f.x, h->st)));  // b = (float) v, x = 0
      h->launches += 1;
    }
    CKS(run_vcycle<float>(h));
    CK((launch_convert<float, double>(D, final_x<float>(h, 0), z, h->st)));
    h->launches += 1;
  }
  return STMG_OK;
}

// ||x||_2 into dev_out[0] (device), via the multidot reduction
static int dev_norm(stmg_handle* h, const double* x, long long n, double* dev_out) {
  const int nb = multidot_blocks(n);
  CK(launch_multidot(n, 1, x, n, x, h->partial, nb, h->st));
  CK(launch_reduce_partials(1, nb, h->partial, dev_out, 0, h->st));
  CK(launch_sqrt_inplace(dev_out, h->st));
  h->launches += 3;
  return STMG_OK;
}

static int ensure_krylov(stmg_handle* h, int m) {
  if (h->m_alloc >= m) return STMG_OK;
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(h->V); f(h->Z); f(h->w); f(h->hcol); f(h->tmp); f(h->partial); f(h->bnorm);
  h->V = h->Z = h->w = h->hcol = h->tmp = h->partial = h->bnorm = nullptr;
  const long long D = h->L[0].H.size;
  CKS(dalloc(&h->V, (size_t)(m + 1) * D));
  CKS(dalloc(&h->Z, (size_t)m * D));
  CKS(dalloc(&h->w, D));
  CKS(dalloc(&h->hcol, m + 2));
  CKS(dalloc(&h->tmp, m + 2));
  CKS(dalloc(&h->partial, (size_t)304 * (m + 2)));
  if (h->cgs_blocks > 0) {
    if (h->cgs_part) cudaFree(h->cgs_part);
    h->cgs_part = nullptr;
    CKS(dalloc(&h->cgs_part, (size_t)cgs2_scratch(h->cgs_blocks)));
  }
  CKS(dalloc(&h->bnorm, 4));
  if (h->hc_host) cudaFreeHost(h->hc_host);
  if (h->err_host) cudaFreeHost(h->err_host);
  h->hc_host = nullptr;
  h->err_host = nullptr;
  CK(cudaMallocHost((void**)&h->hc_host, sizeof(double) * (size_t)(m + 1) * (m + 2)));
  CK(cudaMallocHost((void**)&h->err_host, sizeof(int) * (size_t)(m + 1)));
  for (int i = 0; i < 2; ++i)
    if (!h->ev_it[i]) CK(cudaEventCreateWithFlags(&h->ev_it[i], cudaEventDisableTiming));
  h->m_alloc = m;
  return STMG_OK;
}

static CellsParams cells_params(const LevelHost& H) {
  CellsParams p{};
  p.dim = H.dim; p.n = H.n; p.r1 = H.r + 1; p.np = H.np; p.G = H.G; p.kt = H.kt; p.npm = H.npm;
  p.Pn = H.dim == 2 ? H.np * H.np : H.np * H.np * H.np;
  p.C = H.kt * (H.dim * p.Pn + H.npm);
  p.n_nodes = H.n_nodes; p.nv = H.n_vel; p.npr = H.n_pres; p.size = H.size; p.n_cells = H.n_cells;
  // the previous system's last subinterval polynomial at the next system's Radau points:
  // subinterval j of the next system lies at s + 2 (j + 1) on its reference interval
  const int k1 = H.tt.k1, last = H.nsub - 1;
  for (int a = 0; a < H.kt; ++a)
    for (int bb = 0; bb < H.kt; ++bb) {
      const int ja = a / k1, jb = bb / k1;
      p.E[a * H.kt + bb] = jb == last ? lagrange_eval(H.tt.nodes1, k1, bb % k1, H.tt.nodes1[a % k1] + 2.0 * (ja + 1))
                                      : 0.0;
    }
  return p;
}

static int solve_impl(stmg_handle* h, const double* b, double* x, stmg_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  const int m = h->cfg.gmres_max_iter;
  const double tol = h->cfg.rel_tol;
  const int prec = h->cfg.precond_precision;
  CKS(ensure_krylov(h, m));
  LevelDev& l0 = h->L[0];
  const long long D = l0.H.size;
  cudaStream_t s = h->st;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
  double hv[2];
  info->iterations = 0; info->rel_residual = 0.0; info->status = STMG_OK; info->seconds = 0.0;
  if (h->cgs_bar) CK(cudaMemsetAsync(h->cgs_bar, 0, 2 * sizeof(unsigned), s));
  if (h->inject_wait_fault && h->cgs_bar) {
    // an arrival count far above the block count: no block is ever the last to arrive
    CK(cudaMemsetAsync(h->cgs_bar, 0x7f, sizeof(unsigned), s));
    h->inject_wait_fault = 0;
  }
  CKS(dev_norm(h, b, D, h->bnorm));
  // the boundary rows of S are the identity: x_D = b_D exactly.  The V-cycle's corrections
  // vanish on boundary dofs, so FGMRES keeps x_D where it starts; start it there.
  CK(launch_copy_boundary(cells_params(l0.H), b, x, s));
  h->launches += 1;
  {
    Prof pr(h, STMG_PROF_OPERATOR, s);
    CKS(op_apply<double>(h, 0, x, b, h->V, RESIDUAL, s));
  }
  CKS(dev_norm(h, h->V, D, h->bnorm + 1));
  CK(cudaMemcpyAsync(hv, h->bnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  harvest_all(h);
  const double bn = hv[0], beta = hv[1];
  if (!std::isfinite(bn) || !std::isfinite(beta)) { info->status = STMG_ERR_NONFINITE; return info->status; }
  if (bn == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * D, s));
    CK(cudaStreamSynchronize(s));
    return STMG_OK;
  }
  if (beta <= tol * bn) {
    info->rel_residual = beta / bn;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return STMG_OK;
  }
  CK(launch_scale(D, 1.0 / beta, h->V, h->V, s));
  h->launches += 1;
  g[0] = beta;
  // One FGMRES iteration on the device: precondition v_j, apply S, Arnoldi step (which
  // writes v_{j+1}); then its column of H and the error flag are copied to pinned host
  // slots and an event marks the end.  Nothing on the device waits for the host, so while
  // the host reads iteration j the device can already run iteration j + 1: it is
  // enqueued before the host waits whenever the residual history does not predict that
  // iteration j converges (the residual estimate falls by a steady factor per iteration;
  // a wrong "not yet" costs one iteration of device work that is discarded, a wrong
  // "converged" one host round trip).  With profiling on, iterations are not overlapped.
  // ready32[jj]: the Arnoldi step that produced v_jj also wrote the FP32 V-cycle's inputs
  std::vector<char> ready32(m + 1, 0);
  const bool fuse32 = prec == STMG_FP32 && l0.f.b;
  auto enqueue_iteration = [&](int jj) -> int {
    double* vj = h->V + (size_t)jj * D;
    double* zj = h->Z + (size_t)jj * D;
    CKS(precondition(h, prec, vj, zj, ready32[jj] != 0));
    {
      Prof pr(h, STMG_PROF_OPERATOR, s);
      CKS(op_apply<double>(h, 0, zj, nullptr, h->w, APPLY, s));
    }
    if (h->cgs_blocks > 0 && jj + 1 <= cgs2_max_vectors()) {
      Prof pr(h, STMG_PROF_OTHER, s);
      // CGS2 and the normalisation of the next basis vector in one cooperative launch
      bool wrote = false;
      CK(launch_cgs2(D, jj + 1, h->V, D, h->w, h->cgs_part, h->hcol, h->V + (size_t)(jj + 1) * D,
                     fuse32 ? l0.f.b : nullptr, fuse32 ? l0.f.x : nullptr, &wrote, h->cgs_bar, h->d_err,
                     h->cgs_blocks, h->cfg.arnoldi_form == 0, s));
      ready32[jj + 1] = wrote ? 1 : 0;
      h->launches += 1;
    } else {
      Prof pr(h, STMG_PROF_OTHER, s);
      const int nb = multidot_blocks(D);
      // CGS2: h = V^T w, w -= V h, twice; h accumulated in hcol
      CK(launch_multidot(D, jj + 1, h->V, D, h->w, h->partial, nb, s));
      CK(launch_reduce_partials(jj + 1, nb, h->partial, h->hcol, 0, s));
      CK(launch_multiaxpy(D, jj + 1, h->V, D, h->hcol, -1.0, h->w, s));
      CK(launch_multidot(D, jj + 1, h->V, D, h->w, h->partial, nb, s));
      CK(launch_reduce_partials(jj + 1, nb, h->partial, h->tmp, 0, s));
      CK(launch_multiaxpy(D, jj + 1, h->V, D, h->tmp, -1.0, h->w, s));
      CK(launch_reduce_partials(jj + 1, nb, h->partial, h->hcol, 1, s));
      CKS(dev_norm(h, h->w, D, h->hcol + jj + 1));
      CK(launch_scale_by_inverse(D, h->hcol + jj + 1, h->w, h->V + (size_t)(jj + 1) * D, s));
      h->launches += 8;
    }
    CK(cudaMemcpyAsync(h->hc_host + (size_t)jj * (m + 2), h->hcol, sizeof(double) * (jj + 2), cudaMemcpyDeviceToHost,
                       s));
    CK(cudaMemcpyAsync(h->err_host + jj, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->ev_it[jj & 1], s));
    return STMG_OK;
  };
  const bool overlap = h->prof == 0;
  std::vector<double> rest(m + 1, 0.0);           // residual estimate after i iterations
  rest[0] = beta;
  int j = 0, status = STMG_ERR_NOT_CONVERGED;
  CKS(enqueue_iteration(0));
  for (j = 0; j < m; ++j) {
    bool ahead = false;
    if (overlap && j + 1 < m) {
      // predicted residual after iteration j: the last reduction factor applied once more
      const double pred = j >= 1 ? rest[j] * (rest[j] / rest[j - 1]) : rest[j];
      if (!(pred <= 4.0 * tol * bn)) {
        CKS(enqueue_iteration(j + 1));
        ahead = true;
      }
    }
    CK(cudaEventSynchronize(h->ev_it[j & 1]));
    harvest_all(h);
    const double* hc = h->hc_host + (size_t)j * (m + 2);
    if (h->err_host[j]) {             // a bounded wait expired (grid barrier or TMA pipeline)
      CK(cudaStreamSynchronize(s));   // the iteration enqueued ahead finishes first
      CK(cudaMemset(h->d_err, 0, sizeof(int)));
      if (h->cgs_bar) CK(cudaMemset(h->cgs_bar, 0, 2 * sizeof(unsigned)));
      if (h->mgp_bar) CK(cudaMemset(h->mgp_bar, 0, 2 * sizeof(unsigned)));
      info->status = STMG_ERR_TIMEOUT;
      info->iterations = j + 1;
      return STMG_ERR_TIMEOUT;
    }
    for (int i = 0; i <= j + 1; ++i) {
      if (!std::isfinite(hc[i])) {
        CK(cudaStreamSynchronize(s));
        info->status = STMG_ERR_NONFINITE; info->iterations = j + 1; return info->status;
      }
      H[(size_t)i * m + j] = hc[i];
    }
    for (int i = 0; i < j; ++i) {     // previous Givens rotations
      const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
      H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
      H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
    }
    const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
    const double den = std::hypot(a, c);
    if (den == 0.0) { status = STMG_ERR_BREAKDOWN; break; }
    cs[j] = a / den; sn[j] = c / den;
    H[(size_t)j * m + j] = den;
    H[(size_t)(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    rest[j + 1] = std::fabs(g[j + 1]);
    if (std::fabs(g[j + 1]) <= tol * bn) { status = STMG_OK; ++j; break; }
    if (c == 0.0) { status = STMG_OK; ++j; break; }   // lucky breakdown: exact solution
    if (!ahead && j + 1 < m) CKS(enqueue_iteration(j + 1));
  }
  const int kdim = j < m ? j : m;
  // back substitution H y = g, then x += Z y
  std::vector<double> y(kdim, 0.0);
  for (int i = kdim - 1; i >= 0; --i) {
    double t = g[i];
    for (int q = i + 1; q < kdim; ++q) t -= H[(size_t)i * m + q] * y[q];
    y[i] = t / H[(size_t)i * m + i];
  }
  CK(cudaMemcpyAsync(h->tmp, y.data(), sizeof(double) * kdim, cudaMemcpyHostToDevice, s));
  CK(launch_multiaxpy(D, kdim, h->Z, D, h->tmp, 1.0, x, s));
  h->launches += 1;
  {
    Prof pr(h, STMG_PROF_OPERATOR, s);
    CKS(op_apply<double>(h, 0, x, b, h->w, RESIDUAL, s));
  }
  CKS(dev_norm(h, h->w, D, h->bnorm + 2));
  CK(cudaMemcpyAsync(hv, h->bnorm + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  int derr = 0;
  CK(cudaMemcpyAsync(&derr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  harvest_all(h);
  if (derr) {
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    if (h->cgs_bar) CK(cudaMemset(h->cgs_bar, 0, 2 * sizeof(unsigned)));
    if (h->mgp_bar) CK(cudaMemset(h->mgp_bar, 0, 2 * sizeof(unsigned)));
    info->status = STMG_ERR_TIMEOUT;
    return STMG_ERR_TIMEOUT;
  }
  info->iterations = kdim;
  info->rel_residual = hv[0] / bn;
  if (!std::isfinite(info->rel_residual)) status = STMG_ERR_NONFINITE;
  else if (info->rel_residual <= tol * (1.0 + 1e-3)) status = STMG_OK;
  else if (status == STMG_OK) status = STMG_ERR_NOT_CONVERGED;
  info->status = status;
  info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

template <typename T>
static int smooth_t(stmg_handle* h, int lvl, const T* b, T* x, int steps) {
  PrecDev<T>& P = h->L[lvl].pd<T>();
  for (int s = 0; s < steps; ++s) {
    CKS(op_apply<T>(h, lvl, x, b, P.r, RESIDUAL, h->st));
    CKS(op_sweep<T>(h, lvl, P.r, x, h->st));
  }
  return STMG_OK;
}

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" {

const char* stmg_status_string(int s) {
  switch (s) {
    case STMG_OK: return "ok";
    case STMG_ERR_ARG: return "invalid argument";
    case STMG_ERR_OOM: return "out of memory";
    case STMG_ERR_NOT_CONVERGED: return "not converged";
    case STMG_ERR_BREAKDOWN: return "Arnoldi breakdown";
    case STMG_ERR_NONFINITE: return "non-finite value";
    case STMG_ERR_CUDA: return "CUDA error";
    case STMG_ERR_UNIMPLEMENTED: return "not implemented for these parameters";
    case STMG_ERR_SINGULAR: return "singular patch or coarse matrix";
    case STMG_ERR_TOO_LARGE: return "level larger than the fixed scratch of stmg_smooth_noalloc";
    case STMG_ERR_TIMEOUT: return "a bounded device-side wait expired";
    default: return "unknown status";
  }
}

int stmg_default_config(stmg_config* c) {
  if (!c) return STMG_ERR_ARG;
  std::memset(c, 0, sizeof(*c));
  c->dim = 2; c->n_cells = 8; c->r = 1; c->k = 1;
  c->nu = 1.0; c->T = 1.0; c->n_slabs = 4;
  c->n_levels = 0;
  for (int i = 0; i < STMG_MAX_LEVELS; ++i) c->smoother[i] = STMG_CELL;
  c->omega = 0.7; c->nu1 = 1; c->nu2 = 1;
  c->precond_precision = STMG_FP64;
  c->precisions = 3;
  c->gmres_max_iter = 200;
  c->rel_tol = 1e-8;
  c->use_graphs = 1;
  c->sweep_variant = 0;
  c->autotune = 1;
  c->coarse_n = 1;
  c->k_min = 1;
  c->n_sub = 1;
  c->half_inverses = 0;
  c->transfer_variant = 0;
  c->apply_variant = 0;
  c->persistent = 1;
  c->time_h = 0;
  c->arnoldi_form = 0;
  c->fuse_transfers = 1;
  for (int i = 0; i < STMG_MAX_LEVELS; ++i) c->level_nsub[i] = 0;
  return STMG_OK;
}

// ------------------------------------------------------------------------------------
// Tuning cache.  With the environment variable STMG_TUNE_CACHE naming a file, stmg_create
// writes the launch shapes the tuner chose there, and a later stmg_create of the same
// configuration (same levels, precisions and options) reads them instead of timing the
// candidates again: a process running under a profiler, whose timings are distorted, then
// runs the shapes that were chosen without it.  One text line per configuration.
// ------------------------------------------------------------------------------------
static std::string tune_key(const stmg_handle* h) {
  const stmg_config& c = h->cfg;
  std::string k = "v1 d" + std::to_string(c.dim) + " p" + std::to_string(c.precisions) + " h" +
                  std::to_string(c.half_inverses) + " sv" + std::to_string(c.sweep_variant) + " av" +
                  std::to_string(c.apply_variant) + " tv" + std::to_string(c.transfer_variant) + " pe" +
                  std::to_string(c.persistent) + " nu" + std::to_string(c.nu1) + std::to_string(c.nu2) + " fu" +
                  std::to_string(c.fuse_transfers);
  for (const auto& L : h->L)
    k += " L" + std::to_string(L.H.n) + "." + std::to_string(L.H.r) + "." + std::to_string(L.H.k) + "." +
         std::to_string(L.H.nsub) + "." + std::to_string(L.H.smoother);
  return k;
}

static void tune_cache_save(const stmg_handle* h, const char* path) {
  std::string line = tune_key(h) + " |";
  for (const auto& L : h->L) {
    for (int w = 0; w < 2; ++w) {
      const int tv = w == 0 ? L.d.tp.variant : L.f.tp.variant, tc = w == 0 ? L.d.tp.cpb : L.f.tp.cpb;
      const ApplyParams<double>& ad = L.d.ap;
      const ApplyParams<float>& af = L.f.ap;
      const int av = w == 0 ? ad.variant : af.variant, ac = w == 0 ? ad.cpb : af.cpb;
      const int tx = w == 0 ? ad.tcx : af.tcx, ty = w == 0 ? ad.tcy : af.tcy;
      line += " " + std::to_string(L.sweep_var[w]) + "," + std::to_string(L.ppb[w]) + "," + std::to_string(L.unroll[w]) +
              "," + std::to_string(av) + "," + std::to_string(ac) + "," + std::to_string(tx) + "," + std::to_string(ty) +
              "," + std::to_string(tv) + "," + std::to_string(tc);
    }
  }
  for (int w = 0; w < 2; ++w) line += " m" + std::to_string(h->mgp_first[w]) + "," + std::to_string(h->mgp_blocks[w]);
  // keep the other configurations' lines
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(path, "r")) {
    char buf[8192];
    const std::string key = tune_key(h) + " |";
    while (std::fgets(buf, sizeof(buf), f)) {
      std::string l(buf);
      if (l.compare(0, key.size(), key) != 0) keep.push_back(l);
    }
    std::fclose(f);
  }
  if (FILE* f = std::fopen(path, "w")) {
    for (const auto& l : keep) std::fputs(l.c_str(), f);
    std::fputs((line + "\n").c_str(), f);
    std::fclose(f);
  }
}

static bool tune_cache_load(stmg_handle* h, const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  const std::string key = tune_key(h) + " |";
  char buf[8192];
  std::string found;
  while (std::fgets(buf, sizeof(buf), f)) {
    std::string l(buf);
    if (l.compare(0, key.size(), key) == 0) found = l.substr(key.size());
  }
  std::fclose(f);
  if (found.empty()) return false;
  const char* p = found.c_str();
  for (auto& L : h->L) {
    for (int w = 0; w < 2; ++w) {
      int v[9];
      int used = 0;
      if (std::sscanf(p, " %d,%d,%d,%d,%d,%d,%d,%d,%d%n", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7], &v[8],
                      &used) != 9)
        return false;
      p += used;
      L.sweep_var[w] = v[0]; L.ppb[w] = v[1]; L.unroll[w] = v[2];
      if (w == 0) { L.d.ap.variant = v[3]; L.d.ap.cpb = v[4]; L.d.ap.tcx = v[5]; L.d.ap.tcy = v[6]; L.d.tp.variant = v[7]; L.d.tp.cpb = v[8]; }
      else { L.f.ap.variant = v[3]; L.f.ap.cpb = v[4]; L.f.ap.tcx = v[5]; L.f.ap.tcy = v[6]; L.f.tp.variant = v[7]; L.f.tp.cpb = v[8]; }
    }
  }
  // the persistent kernel's descriptors are built as after tuning; its start and grid as cached
  if (mgp_setup<double>(h) != STMG_OK || mgp_setup<float>(h) != STMG_OK) return false;
  for (int w = 0; w < 2; ++w) {
    int first = 0, blocks = 0, used = 0;
    if (std::sscanf(p, " m%d,%d%n", &first, &blocks, &used) != 2) return false;
    p += used;
    h->mgp_first[w] = h->mgp_eligible[w] > 0 ? first : 0;
    if (blocks > 0) h->mgp_blocks[w] = blocks;
  }
  return true;
}

static int create_impl(const stmg_config* cfg, stmg_handle* h) {
  h->cfg = *cfg;
  const stmg_config& c = h->cfg;
  if (c.dim != 2 && c.dim != 3) return STMG_ERR_ARG;
  if (c.n_cells < 1 || c.r < 1 || c.k < 0 || c.n_slabs < 1 || !(c.T > 0) || !(c.nu > 0)) return STMG_ERR_ARG;
  if (c.r > 4 || c.k > 3) return STMG_ERR_UNIMPLEMENTED;
  if (c.n_sub < 1) return STMG_ERR_ARG;
  if (c.n_sub * (c.k + 1) > MAXKT) return STMG_ERR_UNIMPLEMENTED;
  if (c.gmres_max_iter < 1 || !(c.rel_tol > 0) || c.nu1 < 0 || c.nu2 < 0) return STMG_ERR_ARG;
  if ((c.precisions & 3) == 0) return STMG_ERR_ARG;
  if (c.sweep_variant < 0 || c.sweep_variant > 3) return STMG_ERR_ARG;
  if (c.transfer_variant < 0 || c.transfer_variant > 2) return STMG_ERR_ARG;
  if (c.apply_variant < 0 || c.apply_variant > 4) return STMG_ERR_ARG;
  if (c.persistent < 0 || c.persistent > 2) return STMG_ERR_ARG;
  if (c.precond_precision != STMG_FP64 && c.precond_precision != STMG_FP32) return STMG_ERR_ARG;
  if (!(c.precisions & (1 << c.precond_precision))) return STMG_ERR_ARG;
  h->tau = c.T / ((double)c.n_slabs * c.n_sub);
  if (c.time_h < 0 || c.time_h > 1) return STMG_ERR_ARG;
  if (c.arnoldi_form < 0 || c.arnoldi_form > 1) return STMG_ERR_ARG;
  if (c.fuse_transfers < 0 || c.fuse_transfers > 1) return STMG_ERR_ARG;
  // levels (n, r, k, nsub) fine -> coarse; a level of fewer subintervals covers the same
  // system time span T / n_slabs with longer ones (h-coarsening in time, App. A)
  std::vector<std::array<int, 4>> lv;
  if (c.n_levels == 0) {
    if (c.n_cells & (c.n_cells - 1)) return STMG_ERR_ARG;   // default rule needs n = 2^c
    if (c.coarse_n < 1 || c.coarse_n > c.n_cells || (c.coarse_n & (c.coarse_n - 1))) return STMG_ERR_ARG;
    if (c.k_min < 1) return STMG_ERR_ARG;
    const auto dh = default_hierarchy(c.n_cells, c.r, c.k, c.coarse_n, c.k_min);
    int ns = c.n_sub;
    if (c.time_h) {                      // halve the subintervals on the finest space level first
      while (ns > 1 && ns % 2 == 0) {
        lv.push_back({dh[0][0], dh[0][1], dh[0][2], ns});
        ns /= 2;
      }
    }
    for (const auto& l : dh) lv.push_back({l[0], l[1], l[2], ns});
  } else {
    if (c.n_levels > STMG_MAX_LEVELS) return STMG_ERR_ARG;
    for (int i = 0; i < c.n_levels; ++i)
      lv.push_back({c.level_n[i], c.level_r[i], c.level_k[i], c.level_nsub[i] > 0 ? c.level_nsub[i] : c.n_sub});
    if (lv[0][0] != c.n_cells || lv[0][1] != c.r || lv[0][2] != c.k || lv[0][3] != c.n_sub) return STMG_ERR_ARG;
  }
  if (lv.size() > STMG_MAX_LEVELS) return STMG_ERR_ARG;
  for (size_t i = 0; i < lv.size(); ++i) {
    if (lv[i][1] < 1 || lv[i][1] > 4 || lv[i][2] < 0 || lv[i][2] > 3 || lv[i][0] < 1 || lv[i][3] < 1) return STMG_ERR_ARG;
    if (lv[i][3] * (lv[i][2] + 1) > MAXKT) return STMG_ERR_UNIMPLEMENTED;
    if (i + 1 < lv.size()) {
      const auto &f = lv[i], &cc = lv[i + 1];
      const bool hstep = f[0] == 2 * cc[0], same = f[0] == cc[0];
      if (!(hstep || same) || cc[1] > f[1] || cc[2] > f[2]) return STMG_ERR_ARG;
      if (cc[3] > f[3] || f[3] % cc[3] != 0) return STMG_ERR_ARG;    // coarser temporal mesh nested in the finer
    }
  }
  h->L.resize(lv.size());
  try {
    const double span = c.T / c.n_slabs;
    for (size_t i = 0; i < lv.size(); ++i) {
      LevelDev& L = h->L[i];
      init_level_geometry(&L.H, c.dim, lv[i][0], lv[i][1], lv[i][2], span / lv[i][3], c.nu, lv[i][3]);
      if (!modes_in_kernel_order(L.H)) return STMG_ERR_ARG;   // host tables and kernels out of step
    }
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  CK(cudaStreamCreateWithFlags(&h->gst, cudaStreamNonBlocking));
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
    CKS(dalloc(&h->d_err, 1));
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    // stmg_smooth_noalloc's array: its module (and the array's device memory) is loaded
    // here, at set-up, so that the no-alloc call itself never triggers a load
    CKS(noalloc_scratch_address(&h->noalloc));
    h->cgs_blocks = cgs2_blocks(h->n_sm);
    if (h->cgs_blocks > 0) {
      CKS(dalloc(&h->cgs_bar, 2));
      CK(cudaMemset(h->cgs_bar, 0, 2 * sizeof(unsigned)));
    }
  }
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  for (size_t i = 0; i < h->L.size(); ++i) {
    LevelDev& L = h->L[i];
    LevelHost& H = L.H;
    const bool coarsest = i + 1 == h->L.size();
    double* d_cls = nullptr;
    int* d_cls_of = nullptr;
    if (!coarsest) {
      const int kind = c.smoother[i] == STMG_VSP ? STMG_VSP : STMG_CELL;
      build_patches(&H, kind);
      if (!build_class_inverses(&H)) return STMG_ERR_SINGULAR;
      CKS(dalloc(&L.dofs, H.dofs.size()));
      CK(cudaMemcpy(L.dofs, H.dofs.data(), sizeof(int) * H.dofs.size(), cudaMemcpyHostToDevice));
      CKS(dalloc(&d_cls, H.class_inv.size()));
      CK(cudaMemcpy(d_cls, H.class_inv.data(), sizeof(double) * H.class_inv.size(), cudaMemcpyHostToDevice));
      CKS(dalloc(&d_cls_of, H.patch_class.size()));
      CK(cudaMemcpy(d_cls_of, H.patch_class.data(), sizeof(int) * H.patch_class.size(), cudaMemcpyHostToDevice));
      const double inv_bytes = (double)H.n_patches * H.B * H.Bc * 4.0;
      L.streaming = inv_bytes > 48e6 ? 1 : 0;
      for (int w = 0; w < 2; ++w) {
        L.ppb[w] = std::max(1, std::min(8, 1024 / H.B));
        L.sweep_var[w] = c.sweep_variant == 2 ? 2 : 1;
        if (c.sweep_variant == 3) {
          L.ppb[w] = std::max(1, std::min(4, 512 / H.B));
          L.sweep_var[w] = 3;
        }
      }
    } else {
      std::vector<double> Gcm;
      if (!build_coarse_inverse(&H, &Gcm)) return STMG_ERR_SINGULAR;
      CKS(dalloc(&L.G, Gcm.size()));
      CK(cudaMemcpy(L.G, Gcm.data(), sizeof(double) * Gcm.size(), cudaMemcpyHostToDevice));
      if (c.precisions & 2) {        // the FP32 V-cycle's copy: half the bytes, FP32 products
        std::vector<float> Gf(Gcm.begin(), Gcm.end());
        CKS(dalloc(&L.Gf, Gf.size()));
        CK(cudaMemcpy(L.Gf, Gf.data(), sizeof(float) * Gf.size(), cudaMemcpyHostToDevice));
      }
      if (H.size > 1024) {
        CKS(dalloc(&L.Gacc, H.size));
        CK(cudaMemset(L.Gacc, 0, sizeof(double) * H.size));   // the tiled product keeps it zero between solves
      }
    }
    int st = STMG_OK;
    if (c.precisions & 1) st = setup_precision<double>(h, L, d_cls, d_cls_of);
    else if (i == 0) st = setup_precision<double>(h, L, d_cls, d_cls_of, false);
    if (st == STMG_OK && (c.precisions & 2)) st = setup_precision<float>(h, L, d_cls, d_cls_of);
    cudaStreamSynchronize(h->st);
    if (d_cls) cudaFree(d_cls);
    if (d_cls_of) cudaFree(d_cls_of);
    // keep the host copies small: drop the per-class index lists and dense inverses
    H.class_idx.clear(); H.class_idx.shrink_to_fit();
    H.class_dir.clear(); H.class_dir.shrink_to_fit();
    H.class_inv.clear(); H.class_inv.shrink_to_fit();
    if (st != STMG_OK) return st;
  }
  for (size_t i = 0; i + 1 < h->L.size(); ++i) {
    fill_transfer_params<double>(h->L[i].H, h->L[i + 1].H, &h->L[i].d.tp);
    fill_transfer_params<float>(h->L[i].H, h->L[i + 1].H, &h->L[i].f.tp);
    if (c.transfer_variant == 2) {
      if (transfer_gather_supported(h->L[i].d.tp)) h->L[i].d.tp.variant = 2;
      if (transfer_gather_supported(h->L[i].f.tp)) h->L[i].f.tp.variant = 2;
    }
  }
  const char* cache = std::getenv("STMG_TUNE_CACHE");
  if (c.autotune && cache && *cache && tune_cache_load(h, cache)) {
    // launch shapes of an earlier tuning of the same configuration (profiling runs)
  } else if (c.autotune) {
    CKS(autotune_impl(h));
    if (cache && *cache) tune_cache_save(h, cache);
  } else {
    CKS(mgp_setup<double>(h));
    CKS(mgp_setup<float>(h));
    CKS(mgp_choose<double>(h));
    CKS(mgp_choose<float>(h));
  }
  // finest-level helpers: slab coupling and forcing
  const LevelHost& F = h->L[0].H;
  MassParams& mp = h->mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.dim = F.dim; mp.n = F.n; mp.G = F.G; mp.np = F.np; mp.kt = F.kt;
  mp.n_nodes = F.n_nodes; mp.n_vel = F.n_vel;
  for (int i = 0; i < F.np * F.np; ++i) mp.M1[i] = F.t1.M1[i];
  mp.hd = std::pow(F.h, F.dim);
  for (int a = 0; a < F.kt; ++a) mp.phi_left[a] = F.tt.phi_left[a];
  ForcingParams& fp = h->fp;
  std::memset(&fp, 0, sizeof(fp));
  fp.dim = F.dim; fp.n = F.n; fp.G = F.G; fp.np = F.np; fp.nq = F.r + 4; fp.kt = F.kt;
  fp.n_nodes = F.n_nodes; fp.n_vel = F.n_vel;
  double gx[16], gw[16];
  gauss_legendre(fp.nq, gx, gw);
  for (int q = 0; q < fp.nq; ++q) {
    const double xq = 0.5 * (gx[q] + 1.0);
    fp.wq[q] = 0.5 * gw[q] * F.h;
    for (int p = 0; p < F.np; ++p) fp.phiq[p * fp.nq + q] = lagrange_eval(F.t1.xi, F.np, p, xq);
  }
  for (int a = 0; a < F.kt; ++a) fp.scale[a] = 0.5 * h->tau * F.tt.weights[a];
  CK(cudaDeviceSynchronize());
  return STMG_OK;
}

int stmg_create(const stmg_config* cfg, stmg_handle** out) {
  if (!cfg || !out) return STMG_ERR_ARG;
  *out = nullptr;
  stmg_handle* h = new (std::nothrow) stmg_handle();
  if (!h) return STMG_ERR_OOM;
  int s;
  try {
    s = create_impl(cfg, h);
  } catch (const std::bad_alloc&) {
    s = STMG_ERR_OOM;
  } catch (...) {
    s = STMG_ERR_ARG;
  }
  if (s != STMG_OK) { stmg_destroy(h); return s; }
  *out = h;
  return STMG_OK;
}

void stmg_destroy(stmg_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
  if (h->gst) cudaStreamSynchronize(h->gst);
  for (auto& g : h->graph) if (g) cudaGraphExecDestroy(g);
  for (auto& L : h->L) free_level(L);
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(h->V); f(h->Z); f(h->w); f(h->hcol); f(h->tmp); f(h->partial); f(h->bnorm);
  f(h->xhost_b); f(h->xhost_x); f(h->d_err); f(h->dot_part); f(h->cgs_bar); f(h->cgs_part);
  if (h->hc_host) cudaFreeHost(h->hc_host);
  if (h->err_host) cudaFreeHost(h->err_host);
  for (auto e : h->ev_it)
    if (e) cudaEventDestroy(e);
  if (h->cst) cudaStreamSynchronize(h->cst);
  for (int i = 0; i < 2; ++i) {
    f(h->mh_in[i]); f(h->mh_x[i]);
    if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
    if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
  }
  f(h->mh_b); f(h->mh_t);
  f(h->mgp_desc[0]); f(h->mgp_desc[1]); f(h->mgp_bar);
  if (h->cst) cudaStreamDestroy(h->cst);
  for (auto e : h->all_events) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->gst) cudaStreamDestroy(h->gst);
  delete h;
}

int stmg_set_stream(stmg_handle* h, void* stream) {
  if (!h) return STMG_ERR_ARG;
  h->st = reinterpret_cast<cudaStream_t>(stream);
  return STMG_OK;
}

int stmg_num_levels(const stmg_handle* h, int* n) {
  if (!h || !n) return STMG_ERR_ARG;
  *n = (int)h->L.size();
  return STMG_OK;
}

int stmg_level_info(const stmg_handle* h, int lvl, stmg_level_info_t* info) {
  if (!h || !info || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  const LevelDev& L = h->L[lvl];
  const LevelHost& H = L.H;
  std::memset(info, 0, sizeof(*info));
  info->n = H.n; info->r = H.r; info->k = H.k;
  info->n_sub = H.nsub;
  info->size = H.size; info->n_vel = H.n_vel; info->n_pres = H.n_pres;
  info->smoother = H.smoother;
  info->patch_size = H.B;
  info->n_patches = H.n_patches;
  info->n_patch_classes = (int)H.class_rep.size();
  if (L.d.has_inv) info->inverse_bytes[0] = (long long)H.n_patches * H.B * H.Bc * 8;
  if (L.f.has_inv)
    info->inverse_bytes[1] = L.f.half ? (long long)H.n_patches * H.B * ((H.B + 7) / 8 * 8) * 2 + H.n_patches * H.B * 4
                                      : (long long)H.n_patches * H.B * H.Bc * 4;
  for (int w = 0; w < 2; ++w) {
    info->sweep_variant[w] = L.sweep_var[w];
    info->patches_per_block[w] = L.ppb[w];
  }
  info->apply_cells_per_block[0] = L.d.ap.cpb;
  info->apply_cells_per_block[1] = L.f.ap.cpb;
  info->transfer_cells_per_block[0] = L.d.tp.variant == 2 ? 0 : L.d.tp.cpb;
  info->transfer_cells_per_block[1] = L.f.tp.variant == 2 ? 0 : L.f.tp.cpb;
  info->streaming = L.streaming;
  info->apply_variant[0] = L.d.ap.variant;
  info->apply_variant[1] = L.f.ap.variant;
  info->apply_tile[0][0] = L.d.ap.tcx; info->apply_tile[0][1] = L.d.ap.tcy;
  info->apply_tile[1][0] = L.f.ap.tcx; info->apply_tile[1][1] = L.f.ap.tcy;
  for (int w = 0; w < 2; ++w) info->persistent[w] = h->mgp_first[w] > 0 && lvl >= h->mgp_first[w] ? 1 : 0;
  for (int w = 0; w < 2; ++w) info->sweep_unroll[w] = L.unroll[w];
  return STMG_OK;
}

static bool prec_ok(const stmg_handle* h, int lvl, int prec) {
  if (!h || lvl < 0 || lvl >= (int)h->L.size()) return false;
  if (prec == STMG_FP64) return h->L[lvl].d.b != nullptr;
  if (prec == STMG_FP32) return h->L[lvl].f.b != nullptr;
  return false;
}

int stmg_apply(stmg_handle* h, int lvl, int prec, const void* x, void* y) {
  if (!prec_ok(h, lvl, prec) || !x || !y) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return op_apply<double>(h, lvl, (const double*)x, nullptr, (double*)y, APPLY, h->st);
  return op_apply<float>(h, lvl, (const float*)x, nullptr, (float*)y, APPLY, h->st);
}

int stmg_apply_transpose(stmg_handle* h, int lvl, int prec, const void* x, void* y) {
  if (!prec_ok(h, lvl, prec) || !x || !y || x == y) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return op_apply<double>(h, lvl, (const double*)x, nullptr, (double*)y, APPLY_T, h->st);
  return op_apply<float>(h, lvl, (const float*)x, nullptr, (float*)y, APPLY_T, h->st);
}

int stmg_residual(stmg_handle* h, int lvl, int prec, const void* b, const void* x, void* r) {
  if (!prec_ok(h, lvl, prec) || !x || !b || !r) return STMG_ERR_ARG;
  if (prec == STMG_FP64)
    return op_apply<double>(h, lvl, (const double*)x, (const double*)b, (double*)r, RESIDUAL, h->st);
  return op_apply<float>(h, lvl, (const float*)x, (const float*)b, (float*)r, RESIDUAL, h->st);
}

int stmg_smooth(stmg_handle* h, int lvl, int prec, const void* b, void* x, int steps) {
  if (!prec_ok(h, lvl, prec) || !b || !x || steps < 0 || lvl == (int)h->L.size() - 1) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return smooth_t<double>(h, lvl, (const double*)b, (double*)x, steps);
  return smooth_t<float>(h, lvl, (const float*)b, (float*)x, steps);
}

int stmg_vanka_sweep(stmg_handle* h, int lvl, int prec, const void* res, void* x) {
  if (!prec_ok(h, lvl, prec) || !res || !x || lvl == (int)h->L.size() - 1) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return op_sweep<double>(h, lvl, (const double*)res, (double*)x, h->st);
  return op_sweep<float>(h, lvl, (const float*)res, (float*)x, h->st);
}

int stmg_restrict(stmg_handle* h, int lvl, int prec, const void* rf, void* bc) {
  if (!prec_ok(h, lvl, prec) || lvl + 1 >= (int)h->L.size() || !rf || !bc) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return op_restrict<double>(h, lvl, (const double*)rf, (double*)bc, h->st);
  return op_restrict<float>(h, lvl, (const float*)rf, (float*)bc, h->st);
}

int stmg_prolongate_add(stmg_handle* h, int lvl, int prec, const void* yc, void* xf) {
  if (!prec_ok(h, lvl, prec) || lvl + 1 >= (int)h->L.size() || !yc || !xf) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return op_prolongate_add<double>(h, lvl, (const double*)yc, (double*)xf, h->st);
  return op_prolongate_add<float>(h, lvl, (const float*)yc, (float*)xf, h->st);
}

int stmg_coarse_solve(stmg_handle* h, int prec, const void* b, void* x) {
  if (!h || !b || !x || !prec_ok(h, (int)h->L.size() - 1, prec)) return STMG_ERR_ARG;
  if (prec == STMG_FP64) return op_coarse<double>(h, (const double*)b, (double*)x, h->st);
  return op_coarse<float>(h, (const float*)b, (float*)x, h->st);
}

int stmg_vcycle(stmg_handle* h, int prec, const double* b, double* x) {
  if (!h || !b || !x || !prec_ok(h, 0, prec)) return STMG_ERR_ARG;
  if (!(h->cfg.precisions & (1 << prec))) return STMG_ERR_ARG;   // that V-cycle was not set up
  return precondition(h, prec, b, x);
}

int stmg_dirichlet_lift(stmg_handle* h, const double* g, const double* b, double* y) {
  if (!h || !g || !b || !y || y == g || y == b || !prec_ok(h, 0, STMG_FP64)) return STMG_ERR_ARG;
  return op_apply<double>(h, 0, g, b, y, LIFT, h->st);
}

int stmg_slab_rhs(stmg_handle* h, const double* F, const double* x_prev, double* b) {
  if (!h || !F || !b) return STMG_ERR_ARG;
  const LevelHost& H = h->L[0].H;
  CK(cudaMemcpyAsync(b, F, sizeof(double) * H.size, cudaMemcpyDeviceToDevice, h->st));
  if (x_prev) {
    CK(launch_mass_coupling(h->mp, x_prev + (size_t)(H.kt - 1) * H.n_vel, b, h->st));
    h->launches += 1;
  }
  return STMG_OK;
}

int stmg_solve_slab(stmg_handle* h, const double* b, double* x, stmg_solve_info* info) {
  if (!h || !b || !x || !info) return STMG_ERR_ARG;
  return solve_impl(h, b, x, info);
}

int stmg_solve_slab_host(stmg_handle* h, const double* bh, double* xh, stmg_solve_info* info) {
  if (!h || !bh || !xh || !info) return STMG_ERR_ARG;
  const long long D = h->L[0].H.size;
  if (!h->xhost_b) {
    CKS(dalloc(&h->xhost_b, D));
    CKS(dalloc(&h->xhost_x, D));
  }
  CK(cudaMemcpyAsync(h->xhost_b, bh, sizeof(double) * D, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->xhost_x, xh, sizeof(double) * D, cudaMemcpyHostToDevice, h->st));
  int s = solve_impl(h, h->xhost_b, h->xhost_x, info);
  CK(cudaMemcpyAsync(xh, h->xhost_x, sizeof(double) * D, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return s;
}

// Time marching with host buffers.  Slab s's input is copied in on the copy stream while
// slab s-1 is solved (two device input buffers), and slab s's solution is copied out on
// the copy stream while slab s+1 is solved (two device solution buffers); the solves
// themselves run on the handle's stream and synchronise it, so the copies overlap them.
static int march_host_impl(stmg_handle* h, int n_slabs, int kind, const double* in_h, double* x_h,
                           stmg_solve_info* infos) {
  const LevelHost& H = h->L[0].H;
  const long long D = H.size;
  const size_t bytes = sizeof(double) * D;
  if (!h->cst) {
    CK(cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CK(cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming));
    }
  }
  for (int i = 0; i < 2; ++i) {
    if (!h->mh_in[i]) CKS(dalloc(&h->mh_in[i], D));
    if (!h->mh_x[i]) CKS(dalloc(&h->mh_x[i], D));
  }
  if (!h->mh_b) CKS(dalloc(&h->mh_b, D));
  if (!h->mh_t) CKS(dalloc(&h->mh_t, D));
  cudaStream_t s = h->st;
  // the copy stream starts after everything already queued on the handle's stream
  CK(cudaEventRecord(h->ev_out[0], s));
  CK(cudaStreamWaitEvent(h->cst, h->ev_out[0], 0));
  CK(cudaMemcpyAsync(h->mh_in[0], in_h, bytes, cudaMemcpyHostToDevice, h->cst));
  CK(cudaEventRecord(h->ev_in[0], h->cst));
  CK(cudaEventRecord(h->ev_out[1], h->cst));
  int status = STMG_OK;
  for (int sl = 0; sl < n_slabs; ++sl) {
    const int cur = sl & 1, nxt = cur ^ 1;
    if (sl + 1 < n_slabs) {
      // mh_in[nxt] was last read by slab sl-1's right-hand side, which the (synchronous)
      // solve of slab sl-1 has completed
      CK(cudaMemcpyAsync(h->mh_in[nxt], in_h + (size_t)(sl + 1) * D, bytes, cudaMemcpyHostToDevice, h->cst));
      CK(cudaEventRecord(h->ev_in[nxt], h->cst));
    }
    CK(cudaStreamWaitEvent(s, h->ev_in[cur], 0));
    const double* x_prev = sl > 0 ? h->mh_x[nxt] : nullptr;
    if (kind == STMG_MARCH_FORCING) {
      CKS(stmg_slab_rhs(h, h->mh_in[cur], x_prev, h->mh_b));
    } else {
      CK(cudaMemsetAsync(h->mh_t, 0, bytes, s));
      if (x_prev) {
        CK(launch_mass_coupling(h->mp, x_prev + (size_t)(H.kt - 1) * H.n_vel, h->mh_t, s));
        h->launches += 1;
      }
      CKS(op_apply<double>(h, 0, h->mh_in[cur], h->mh_t, h->mh_b, LIFT, s));
    }
    // mh_x[cur] held slab sl-2's solution: its copy to the host must have finished
    CK(cudaStreamWaitEvent(s, h->ev_out[cur], 0));
    CK(cudaMemsetAsync(h->mh_x[cur], 0, bytes, s));
    stmg_solve_info info{};
    const int st = solve_impl(h, h->mh_b, h->mh_x[cur], &info);
    if (infos) infos[sl] = info;
    if (st != STMG_OK) { status = st; break; }
    CK(cudaMemcpyAsync(x_h + (size_t)sl * D, h->mh_x[cur], bytes, cudaMemcpyDeviceToHost, h->cst));
    CK(cudaEventRecord(h->ev_out[cur], h->cst));
  }
  CK(cudaStreamSynchronize(h->cst));
  return status;
}

int stmg_march_host(stmg_handle* h, int n_slabs, int kind, const double* in_host, double* x_host,
                    stmg_solve_info* infos) {
  if (!h || n_slabs < 1 || !in_host || !x_host) return STMG_ERR_ARG;
  if (kind != STMG_MARCH_FORCING && kind != STMG_MARCH_BOUNDARY) return STMG_ERR_ARG;
  return march_host_impl(h, n_slabs, kind, in_host, x_host, infos);
}

int stmg_forcing_npoints(const stmg_handle* h, int* nq) {
  if (!h || !nq) return STMG_ERR_ARG;
  *nq = ipow(h->fp.nq, h->fp.dim);
  return STMG_OK;
}

int stmg_forcing_points(stmg_handle* h, double* xq) {
  if (!h || !xq) return STMG_ERR_ARG;
  const LevelHost& F = h->L[0].H;
  const int nq = h->fp.nq, dim = F.dim, nqc = ipow(nq, dim);
  double gx[16], gw[16];
  gauss_legendre(nq, gx, gw);
  std::vector<double> pts((size_t)F.n_cells * nqc * dim);
  for (long long c = 0; c < F.n_cells; ++c) {
    const int cc[3] = {(int)(c % F.n), (int)((c / F.n) % F.n), dim == 3 ? (int)(c / ((long long)F.n * F.n)) : 0};
    for (int q = 0; q < nqc; ++q) {
      const int qi[3] = {q % nq, (q / nq) % nq, q / (nq * nq)};
      for (int d = 0; d < dim; ++d)
        pts[((size_t)c * nqc + q) * dim + d] = (cc[d] + 0.5 * (gx[qi[d]] + 1.0)) * F.h;
    }
  }
  CK(cudaMemcpy(xq, pts.data(), sizeof(double) * pts.size(), cudaMemcpyHostToDevice));
  return STMG_OK;
}

int stmg_slab_times(const stmg_handle* h, int slab, double* t) {
  if (!h || !t || slab < 0) return STMG_ERR_ARG;
  const LevelHost& F = h->L[0].H;
  for (int a = 0; a < F.kt; ++a)
    t[a] = (double)slab * F.nsub * h->tau + 0.5 * h->tau * (F.tt.nodes[a] + 1.0);
  return STMG_OK;
}

int stmg_assemble_forcing(stmg_handle* h, const double* fq, double* F) {
  if (!h || !fq || !F) return STMG_ERR_ARG;
  CK(cudaMemsetAsync(F, 0, sizeof(double) * h->L[0].H.size, h->st));
  CK(launch_forcing(h->fp, fq, F, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_set_profiling(stmg_handle* h, int on) {
  if (!h || on < 0 || on > 2) return STMG_ERR_ARG;
  if (on != h->prof) {
    for (auto& g : h->graph) if (g) { cudaGraphExecDestroy(g); g = nullptr; }   // recapture with/without events
    h->graph_pairs[0].clear(); h->graph_pairs[1].clear();
  }
  h->prof = on;
  return STMG_OK;
}

int stmg_get_profile(stmg_handle* h, double* ms, long long* n, int reset) {
  if (!h) return STMG_ERR_ARG;
  if (h->st) CK(cudaStreamSynchronize(h->st)); else CK(cudaDeviceSynchronize());
  CK(cudaStreamSynchronize(h->gst));
  harvest_all(h);
  for (int i = 0; i < STMG_PROF_N; ++i) {
    if (ms) ms[i] = h->prof_ms[i];
    if (n) n[i] = h->prof_n[i];
  }
  if (ms) ms[STMG_PROF_MG_OTHER] = h->prof_ms[PROF_VCYCLE] - h->prof_ms[STMG_PROF_SMOOTHER];
  if (n) n[STMG_PROF_MG_OTHER] = h->prof_n[PROF_VCYCLE];
  if (reset) {
    std::memset(h->prof_ms, 0, sizeof(h->prof_ms));
    std::memset(h->prof_n, 0, sizeof(h->prof_n));
  }
  return STMG_OK;
}

int stmg_inject_wait_fault(stmg_handle* h) {
  if (!h) return STMG_ERR_ARG;
  if (!h->cgs_bar) return STMG_ERR_UNIMPLEMENTED;
  h->inject_wait_fault = 1;
  return STMG_OK;
}

long long stmg_kernel_launches(const stmg_handle* h) { return h ? h->launches : 0; }

int stmg_autotune(stmg_handle* h) {
  if (!h) return STMG_ERR_ARG;
  return autotune_impl(h);
}

int stmg_device_status(stmg_handle* h) {
  if (!h) return STMG_ERR_ARG;
  if (h->st) CK(cudaStreamSynchronize(h->st)); else CK(cudaDeviceSynchronize());
  CK(cudaStreamSynchronize(h->gst));
  int derr = 0;
  CK(cudaMemcpy(&derr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr) {
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    if (h->mgp_bar) CK(cudaMemset(h->mgp_bar, 0, 2 * sizeof(unsigned)));
    return STMG_ERR_TIMEOUT;
  }
  return STMG_OK;
}

// ---- cell tensors and temporal extrapolation ---------------------------------------


int stmg_cells_channels(const stmg_handle* h, int lvl, int* C) {
  if (!h || !C || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  *C = cells_params(h->L[lvl].H).C;
  return STMG_OK;
}

int stmg_cells_gather(stmg_handle* h, int lvl, const double* x, const double* base, const float* inv_scale,
                      float* cells) {
  if (!h || !x || !cells || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  const CellsParams p = cells_params(h->L[lvl].H);
  CK(launch_cells_gather(p, x, base, inv_scale, cells, p.C, 0, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_cells_gather_strided(stmg_handle* h, int lvl, const double* x, const double* base, const float* inv_scale,
                              float* cells, long long row_stride, int channel_offset) {
  if (!h || !x || !cells || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  const CellsParams p = cells_params(h->L[lvl].H);
  if (channel_offset < 0 || row_stride < channel_offset + p.C) return STMG_ERR_ARG;
  CK(launch_cells_gather(p, x, base, inv_scale, cells, row_stride, channel_offset, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_cells_scatter_add(stmg_handle* h, int lvl, const float* cells, const float* scale, double* x) {
  if (!h || !x || !cells || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  CK(launch_cells_scatter_add(cells_params(h->L[lvl].H), cells, scale, x, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_cells_gather_adjoint(stmg_handle* h, int lvl, const double* x, const float* scale, float* cells) {
  if (!h || !x || !cells || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  CK(launch_cells_gather_adjoint(cells_params(h->L[lvl].H), x, scale, cells, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_dot(stmg_handle* h, long long n, const double* x, const double* y, double* out) {
  if (!h || !x || !y || !out || n < 1) return STMG_ERR_ARG;
  if (!h->dot_part) CKS(dalloc(&h->dot_part, (size_t)dot_blocks()));
  CK(launch_dot(n, x, y, h->dot_part, out, h->st));
  h->launches += 2;
  return STMG_OK;
}

int stmg_extrapolate(stmg_handle* h, int lvl, const double* x_prev, double* x_next) {
  if (!h || !x_prev || !x_next || x_prev == x_next || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  CK(launch_extrapolate(cells_params(h->L[lvl].H), x_prev, x_next, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_remove_pressure_mean(stmg_handle* h, int lvl, double* x) {
  if (!h || !x || lvl < 0 || lvl >= (int)h->L.size()) return STMG_ERR_ARG;
  CK(launch_remove_pressure_mean(cells_params(h->L[lvl].H), x, h->st));
  h->launches += 1;
  return STMG_OK;
}

int stmg_sweep_bytes(const stmg_handle* h, int lvl, int prec, double* bytes) {
  if (!h || !bytes || lvl < 0 || lvl + 1 >= (int)h->L.size()) return STMG_ERR_ARG;
  const LevelHost& H = h->L[lvl].H;
  const double s = prec == STMG_FP64 ? 8.0 : 4.0;
  // inverses (valence weights folded in) + patch index table + gathered residual +
  // read-modify-write of x; half-precision inverses: 2 bytes per entry plus a row scale
  const double invb = (prec == STMG_FP32 && h->L[lvl].f.half)
                          ? (double)H.n_patches * H.B * ((H.B + 7) / 8 * 8) * 2.0 + (double)H.n_patches * H.B * 4.0
                          : (double)H.n_patches * H.B * H.Bc * s;
  *bytes = invb + (double)H.n_patches * H.B * 4.0 + 3.0 * H.size * s;
  return STMG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Smoothing step without device allocation.
//
// stmg_smooth keeps its residual in a work vector that stmg_create allocated with
// cudaMalloc.  Some callers must not have device memory allocated on their behalf while
// they run (for example a process whose device memory is handed out entirely by its own
// pool allocator, or a time-critical loop that cannot absorb the implicit synchronisation
// of cudaMalloc/cudaFree).  stmg_smooth_noalloc does the same smoothing step with the
// residual held in the library's own fixed device array below, so the call itself
// allocates nothing.
//
// The array lives in this file's module.  With lazy module loading (the CUDA default) the
// module, and with it the array's STMG_NOALLOC_MAX_ENTRIES * 8 bytes of device memory, is
// loaded by the first use of the symbol on a device; that first use is the address lookup
// in stmg_create, so the memory is taken when the first handle is created on a device and
// held until the process exits.  A failure there (no device memory left) is reported by
// stmg_create as STMG_ERR_OOM.
// ------------------------------------------------------------------------------------
static __device__ __align__(256) double stmg_noalloc_scratch[STMG_NOALLOC_MAX_ENTRIES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};   // device address of the array, per device (under the mutex)

template <typename T>
int smooth_noalloc_t(stmg_handle* h, int lvl, const T* b, T* x, int steps, T* res) {
  for (int s = 0; s < steps; ++s) {
    CKS(op_apply<T>(h, lvl, x, b, res, RESIDUAL, h->st));   // overwrites res: r = b - S x
    CKS(op_sweep<T>(h, lvl, res, x, h->st));
  }
  return STMG_OK;
}
}  // namespace

// `stmg_noalloc_scratch` named in host code is only a host-side stand-in; its device
// address has to come from cudaGetSymbolAddress with the device current.  Looked up once
// per device (the first stmg_create on it), cached under a mutex.
static int noalloc_scratch_address(void** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return STMG_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, stmg_noalloc_scratch));   // cudaErrorMemoryAllocation -> STMG_ERR_OOM
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return STMG_OK;
}

extern "C" int stmg_smooth_noalloc(stmg_handle* h, int lvl, int prec, const void* b, void* x, int steps) {
  if (!prec_ok(h, lvl, prec) || !b || !x || steps < 0 || lvl == (int)h->L.size() - 1) return STMG_ERR_ARG;
  if (h->L[lvl].H.size > (long long)STMG_NOALLOC_MAX_ENTRIES) return STMG_ERR_TOO_LARGE;
  if (!h->noalloc) return STMG_ERR_CUDA;
  if (prec == STMG_FP64)
    return smooth_noalloc_t<double>(h, lvl, (const double*)b, (double*)x, steps, (double*)h->noalloc);
  return smooth_noalloc_t<float>(h, lvl, (const float*)b, (float*)x, steps, (float*)h->noalloc);
}
