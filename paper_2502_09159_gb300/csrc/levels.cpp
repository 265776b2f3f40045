// Host setup of the multigrid levels: hierarchy (Alg. 2/3), patch index sets (cell and
// vertex-star patches, remark after Eq. vanka), patch matrices R_T S R_T^T assembled
// from element contributions, their inversion (Gauss-Jordan, partial pivoting, FP64),
// and the bordered coarsest-level inverse.
#include "levels.h"

#include <algorithm>
#include <cmath>
#include <sched.h>

#include <atomic>
#include <condition_variable>
#include <mutex>
#include <cstring>
#include <map>
#include <stdexcept>
#include <thread>
#include <unordered_map>

namespace stmg {

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }
static int binom(int n, int k) { long long r = 1; for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i; return (int)r; }

std::vector<std::array<int, 3>> default_hierarchy(int n, int r, int k, int coarse_n, int k_min) {
  // space: (n, r), (n, r/2), ..., (n, 1), then (n/2, 1), ..., (coarse_n, 1); coarse_n is the
  // coarsest mesh of Alg. 2 (its h_0 = 1 / coarse_n)
  std::vector<std::array<int, 2>> space;
  for (int rr = r; rr >= 1; rr /= 2) space.push_back({n, rr});
  for (int nn = n / 2; nn >= coarse_n && nn >= 1; nn /= 2) space.push_back({nn, 1});
  // time: k, k/2, ..., 1, then 1 again (the geometric loop of Alg. 2 re-adds the last
  // pair); k = 0 stays 0.  Both lists are aligned at the coarse end, the shorter one is
  // padded at the fine end with its finest entry (Alg. 3, P4).
  // k_min: lowest temporal degree of the polynomial loop (Alg. 2's r_0 applied in time; the
  // paper's runs use 1); k_min >= k keeps DG(k) on every level.
  std::vector<int> time;
  const int kmin = k_min < 1 ? 1 : k_min;
  if (k == 0) time.push_back(0);
  else {
    int kk = k;
    time.push_back(kk);
    while (kk / 2 >= kmin) { kk /= 2; time.push_back(kk); }
    time.push_back(kk);
  }
  const size_t L = std::max(space.size(), time.size());
  while (space.size() < L) space.insert(space.begin(), space.front());
  while (time.size() < L) time.insert(time.begin(), time.front());
  std::vector<std::array<int, 3>> out;
  for (size_t i = 0; i < L; ++i) out.push_back({space[i][0], space[i][1], time[i]});
  return out;
}

void init_level_geometry(LevelHost* L, int dim, int n, int r, int k, double tau, double nu, int nsub) {
  L->dim = dim; L->n = n; L->r = r; L->k = k; L->kt = nsub * (k + 1); L->nsub = nsub;
  L->np = r + 2; L->G = (r + 1) * n + 1;
  L->nq = ipow(L->np, dim);
  L->h = 1.0 / n; L->tau = tau; L->nu = nu;
  pressure_modes(dim, r, &L->modes);
  L->npm = (int)L->modes.size();
  if (L->npm != binom(r + dim, dim)) throw std::runtime_error("pressure modes");
  L->n_cells = ipow(n, dim);
  L->n_nodes = 1; for (int d = 0; d < dim; ++d) L->n_nodes *= L->G;
  L->n_vel = (long long)dim * L->n_nodes;
  L->n_pres = (long long)L->n_cells * L->npm;
  L->size = (long long)L->kt * (L->n_vel + L->n_pres);
  L->t1 = make_tables_1d(r);
  L->tt = make_time_tables(k, tau, nsub);
  // element matrices on a cell of size h (Kronecker products of the 1D tables)
  const int np = L->np, nq = L->nq;
  L->Me.assign((size_t)nq * nq, 0.0);
  L->Ae.assign((size_t)nq * nq, 0.0);
  L->Be.assign((size_t)dim * L->npm * nq, 0.0);
  std::vector<std::array<int, 3>> loc(nq);
  for (int p = 0; p < nq; ++p) loc[p] = {p % np, (p / np) % np, dim == 3 ? p / (np * np) : 0};
  const double h = L->h;
  for (int p = 0; p < nq; ++p)
    for (int q = 0; q < nq; ++q) {
      double m = std::pow(h, dim), a = 0.0;
      for (int d = 0; d < dim; ++d) m *= L->t1.M1[loc[p][d] * np + loc[q][d]];
      for (int dd = 0; dd < dim; ++dd) {
        double t = std::pow(h, dim - 2);
        for (int d = 0; d < dim; ++d)
          t *= (d == dd ? L->t1.K1 : L->t1.M1)[loc[p][d] * np + loc[q][d]];
        a += t;
      }
      L->Me[(size_t)p * nq + q] = m;
      L->Ae[(size_t)p * nq + q] = a;
    }
  for (int c = 0; c < dim; ++c)
    for (int m = 0; m < L->npm; ++m)
      for (int p = 0; p < nq; ++p) {
        double v = std::pow(h, dim - 1);
        for (int d = 0; d < dim; ++d) v *= (d == c ? L->t1.G1 : L->t1.N1)[L->modes[m][d] * np + loc[p][d]];
        L->Be[((size_t)c * L->npm + m) * nq + p] = v;
      }
}

// ------------------------------------------------------------------------------------
// patches
// ------------------------------------------------------------------------------------
static bool node_dirichlet(const LevelHost& L, const int* g) {
  for (int d = 0; d < L.dim; ++d)
    if (g[d] == 0 || g[d] == L.G - 1) return true;
  return false;
}

static long long node_index(const LevelHost& L, const int* g) {
  long long idx = 0, s = 1;
  for (int d = 0; d < L.dim; ++d) { idx += g[d] * s; s *= L.G; }
  return idx;
}

// Fill the patch of cells [clo, chi] (per dim, inclusive) with velocity nodes of the
// closure box and all pressure modes of the cells; returns global slab indices, with
// a parallel Dirichlet flag.
static void box_patch(const LevelHost& L, const int* clo, const int* chi, std::vector<long long>* idx,
                      std::vector<char>* dir) {
  const int dim = L.dim, R1 = L.r + 1;
  int nlo[3] = {0, 0, 0}, nhi[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) { nlo[d] = clo[d] * R1; nhi[d] = (chi[d] + 1) * R1; }
  idx->clear();
  dir->clear();
  for (int a = 0; a < L.kt; ++a)
    for (int comp = 0; comp < dim; ++comp)
      for (int gz = nlo[2]; gz <= nhi[2]; ++gz)
        for (int gy = nlo[1]; gy <= nhi[1]; ++gy)
          for (int gx = nlo[0]; gx <= nhi[0]; ++gx) {
            int g[3] = {gx, gy, gz};
            idx->push_back(a * L.n_vel + comp * L.n_nodes + node_index(L, g));
            dir->push_back(node_dirichlet(L, g) ? 1 : 0);
          }
  const long long poff = (long long)L.kt * L.n_vel;
  for (int a = 0; a < L.kt; ++a)
    for (int cz = clo[2]; cz <= chi[2]; ++cz)
      for (int cy = clo[1]; cy <= chi[1]; ++cy)
        for (int cx = clo[0]; cx <= chi[0]; ++cx) {
          const long long cell = cx + (long long)L.n * (cy + (long long)L.n * cz);
          for (int m = 0; m < L.npm; ++m) {
            idx->push_back(poff + a * L.n_pres + cell * L.npm + m);
            dir->push_back(0);
          }
        }
}

void build_patches(LevelHost* L, int kind) {
  const int dim = L->dim, n = L->n;
  L->smoother = kind;
  std::vector<long long> idx;
  std::vector<char> dir;
  std::map<long long, int> class_of_key;
  int per[3] = {1, 1, 1};
  for (int d = 0; d < dim; ++d) per[d] = kind == STMG_CELL ? n : n + 1;
  L->n_patches = (long long)per[0] * per[1] * per[2];
  // first pass: B_max
  int Bmax = 0;
  if (kind == STMG_CELL) {
    Bmax = L->kt * (dim * L->nq + L->npm);
  } else {
    const int side = 2 * (L->r + 1) + 1;
    int nside = n >= 2 ? side : L->np;
    Bmax = L->kt * (dim * ipow(nside, dim) + ipow(n >= 2 ? 2 : 1, dim) * L->npm);
  }
  L->B = Bmax;
  L->Bc = (Bmax + 3) / 4 * 4;
  L->dofs.assign((size_t)L->n_patches * Bmax, -2);
  L->patch_class.assign(L->n_patches, 0);
  L->class_rep.clear();
  L->class_B.clear();
  for (long long p = 0; p < L->n_patches; ++p) {
    int c[3] = {(int)(p % per[0]), (int)((p / per[0]) % per[1]), (int)(p / ((long long)per[0] * per[1]))};
    int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
    long long key = 0;
    for (int d = 0; d < dim; ++d) {
      if (kind == STMG_CELL) {
        clo[d] = chi[d] = c[d];
        // which neighbours exist: c-1, c+1
        key |= (long long)((c[d] > 0) | ((c[d] < n - 1) << 1)) << (4 * d);
      } else {
        clo[d] = std::max(c[d] - 1, 0);
        chi[d] = std::min(c[d], n - 1);
        int bits = 0;
        for (int o = -2; o <= 1; ++o) if (c[d] + o >= 0 && c[d] + o <= n - 1) bits |= 1 << (o + 2);
        key |= (long long)bits << (4 * d);
      }
    }
    box_patch(*L, clo, chi, &idx, &dir);
    if ((int)idx.size() > Bmax) throw std::runtime_error("patch larger than B_max");
    for (size_t i = 0; i < idx.size(); ++i) L->dofs[(size_t)p * Bmax + i] = dir[i] ? -1 : (int)idx[i];
    auto it = class_of_key.find(key);
    if (it == class_of_key.end()) {
      const int cid = (int)L->class_rep.size();
      class_of_key[key] = cid;
      L->class_rep.push_back(p);
      L->class_B.push_back((int)idx.size());
      L->class_idx.push_back(idx);
      L->class_dir.push_back(dir);
      L->patch_class[p] = cid;
    } else {
      L->patch_class[p] = it->second;
    }
  }
  // valence of every slab dof (number of patches containing it)
  L->valence.assign(L->size, 0);
  for (size_t e = 0; e < L->dofs.size(); ++e)
    if (L->dofs[e] >= 0) L->valence[L->dofs[e]]++;
}

// S restricted to the index set idx (global slab indices), boundary rows/cols identity.
void assemble_submatrix(const LevelHost& L, const std::vector<long long>& idx, const std::vector<char>& dir,
                        std::vector<double>* S) {
  const int B = (int)idx.size(), dim = L.dim, np = L.np, nq = L.nq, kt = L.kt, npm = L.npm, n = L.n;
  S->assign((size_t)B * B, 0.0);
  std::unordered_map<long long, int> pos;
  pos.reserve(B * 2);
  for (int i = 0; i < B; ++i) pos[idx[i]] = i;
  // node bounding box of the set
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
  bool any_vel = false;
  std::vector<long long> cells_with_p;
  const long long poff = (long long)kt * L.n_vel;
  for (int i = 0; i < B; ++i) {
    if (idx[i] < poff) {
      long long g = idx[i] % L.n_vel % L.n_nodes;
      for (int d = 0; d < dim; ++d) { int gd = (int)(g % L.G); g /= L.G; lo[d] = std::min(lo[d], gd); hi[d] = std::max(hi[d], gd); }
      any_vel = true;
    }
  }
  int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    if (any_vel) { clo[d] = std::max(0, lo[d] / (L.r + 1) - 1); chi[d] = std::min(n - 1, hi[d] / (L.r + 1)); }
    else { clo[d] = 0; chi[d] = n - 1; }
  }
  std::vector<int> vpos((size_t)kt * dim * nq), ppos((size_t)kt * npm);
  const double* Kt = L.tt.K;
  for (int cz = clo[2]; cz <= chi[2]; ++cz)
    for (int cy = clo[1]; cy <= chi[1]; ++cy)
      for (int cx = clo[0]; cx <= chi[0]; ++cx) {
        const int cc[3] = {cx, cy, cz};
        const long long cell = cx + (long long)n * (cy + (long long)n * cz);
        bool any = false;
        for (int p = 0; p < nq; ++p) {
          int g[3] = {cc[0] * (np - 1) + p % np, cc[1] * (np - 1) + (p / np) % np,
                      dim == 3 ? cc[2] * (np - 1) + p / (np * np) : 0};
          const long long gn = node_index(L, g);
          for (int a = 0; a < kt; ++a)
            for (int comp = 0; comp < dim; ++comp) {
              auto it = pos.find(a * L.n_vel + comp * L.n_nodes + gn);
              const int v = it == pos.end() ? -1 : it->second;
              vpos[((size_t)a * dim + comp) * nq + p] = v;
              any = any || v >= 0;
            }
        }
        bool anyp = false;
        for (int a = 0; a < kt; ++a)
          for (int m = 0; m < npm; ++m) {
            auto it = pos.find(poff + a * L.n_pres + cell * npm + m);
            ppos[a * npm + m] = it == pos.end() ? -1 : it->second;
            anyp = anyp || ppos[a * npm + m] >= 0;
          }
        if (!any && !anyp) continue;
        for (int comp = 0; comp < dim; ++comp)
          for (int p = 0; p < nq; ++p)
            for (int q = 0; q < nq; ++q) {
              const double me = L.Me[(size_t)p * nq + q], ae = L.Ae[(size_t)p * nq + q];
              for (int a = 0; a < kt; ++a) {
                const int ip = vpos[((size_t)a * dim + comp) * nq + p];
                if (ip < 0) continue;
                for (int b = 0; b < kt; ++b) {
                  const int iq = vpos[((size_t)b * dim + comp) * nq + q];
                  if (iq < 0) continue;
                  double v = Kt[a * kt + b] * me;
                  if (a == b) v += L.tt.M[a] * L.nu * ae;
                  (*S)[(size_t)ip * B + iq] += v;
                }
              }
            }
        for (int a = 0; a < kt; ++a)
          for (int m = 0; m < npm; ++m) {
            const int im = ppos[a * npm + m];
            if (im < 0) continue;
            for (int comp = 0; comp < dim; ++comp)
              for (int p = 0; p < nq; ++p) {
                const int ip = vpos[((size_t)a * dim + comp) * nq + p];
                if (ip < 0) continue;
                const double v = -L.tt.M[a] * L.Be[((size_t)comp * npm + m) * nq + p];
                (*S)[(size_t)ip * B + im] += v;
                (*S)[(size_t)im * B + ip] += v;
              }
          }
      }
  for (int i = 0; i < B; ++i)
    if (dir[i]) {
      for (int j = 0; j < B; ++j) { (*S)[(size_t)i * B + j] = 0.0; (*S)[(size_t)j * B + i] = 0.0; }
      (*S)[(size_t)i * B + i] = 1.0;
    }
}

// CPUs this process may run on (its affinity mask), at least 1.
static int usable_cpus() {
  cpu_set_t set;
  CPU_ZERO(&set);
  if (sched_getaffinity(0, sizeof(set), &set) == 0) return std::max(1, CPU_COUNT(&set));
  return (int)std::max(1u, std::thread::hardware_concurrency());
}

// Barrier for the threads of one blocked inversion: a waiting thread spins for a short
// while (cheap when every thread has a core), then sleeps on a condition variable (so
// that threads without a core of their own do not hold up the ones still working).
class HybridBarrier {
 public:
  explicit HybridBarrier(int n) : n_(n) {}
  void wait() {
    const unsigned g = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
      count_.store(0, std::memory_order_relaxed);
      {
        std::lock_guard<std::mutex> lk(mu_);
        gen_.fetch_add(1, std::memory_order_acq_rel);
      }
      cv_.notify_all();
      return;
    }
    for (int spins = 0; spins < 4000; ++spins)
      if (gen_.load(std::memory_order_acquire) != g) return;
    std::unique_lock<std::mutex> lk(mu_);
    cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != g; });
  }

 private:
  const int n_;
  std::atomic<int> count_{0};
  std::atomic<unsigned> gen_{0};
  std::mutex mu_;
  std::condition_variable cv_;
};

// r[j] += sum_k a[k] T[k][j] and s[j] += sum_k b[k] T[k][j] for j in [j0, j1) (two
// rows of the matrix at once; T row-major with row length n).  Rows of T are taken four
// at a time: each loaded T element serves eight multiply-adds, each r[j], s[j] is loaded
// and stored once per four.
static void rank_update2(double* __restrict r, double* __restrict s, const double* a, const double* b,
                         const double* __restrict T, long long n, int kb, int j0, int j1) {
  int k = 0;
  for (; k + 4 <= kb; k += 4) {
    const double a0 = a[k], a1 = a[k + 1], a2 = a[k + 2], a3 = a[k + 3];
    const double b0 = b[k], b1 = b[k + 1], b2 = b[k + 2], b3 = b[k + 3];
    const double* __restrict t0 = T + (size_t)k * n;
    const double* __restrict t1 = t0 + n;
    const double* __restrict t2 = t1 + n;
    const double* __restrict t3 = t2 + n;
    for (int j = j0; j < j1; ++j) {
      const double u0 = t0[j], u1 = t1[j], u2 = t2[j], u3 = t3[j];
      r[j] += a0 * u0 + a1 * u1 + a2 * u2 + a3 * u3;
      s[j] += b0 * u0 + b1 * u1 + b2 * u2 + b3 * u3;
    }
  }
  for (; k < kb; ++k) {
    const double ak = a[k], bk = b[k];
    const double* __restrict tk = T + (size_t)k * n;
    for (int j = j0; j < j1; ++j) {
      r[j] += ak * tk[j];
      s[j] += bk * tk[j];
    }
  }
}

// The same for one row.
static void rank_update1(double* __restrict r, const double* a, const double* __restrict T, long long n, int kb,
                         int j0, int j1) {
  int k = 0;
  for (; k + 4 <= kb; k += 4) {
    const double a0 = a[k], a1 = a[k + 1], a2 = a[k + 2], a3 = a[k + 3];
    if (a0 == 0.0 && a1 == 0.0 && a2 == 0.0 && a3 == 0.0) continue;
    const double* __restrict t0 = T + (size_t)k * n;
    const double* __restrict t1 = t0 + n;
    const double* __restrict t2 = t1 + n;
    const double* __restrict t3 = t2 + n;
    for (int j = j0; j < j1; ++j) r[j] += a0 * t0[j] + a1 * t1[j] + a2 * t2[j] + a3 * t3[j];
  }
  for (; k < kb; ++k) {
    const double ak = a[k];
    if (ak == 0.0) continue;
    const double* __restrict tk = T + (size_t)k * n;
    for (int j = j0; j < j1; ++j) r[j] += ak * tk[j];
  }
}

// Blocked in-place Gauss-Jordan with partial pivoting, for the large dense matrices of
// coarse levels and 3D patches.  The columns are taken in panels of NB.  Inside a panel
// the elimination steps update only the panel's columns (every row, pivot search and row
// interchanges as in the scalar method).  With P the panel's pivot rows, K its columns,
// R the other columns and E the pivot block before the panel, the NB steps together map
// [P,K] -> E^-1, [others,K] -> -[others,K] E^-1, and, what is left to do afterwards,
// [P,R] -> E^-1 [P,R] and [others,R] -> [others,R] - [others,K] E^-1 [P,R]: one rank-NB
// update of every row with T = the old [P,R] (steps of Gauss-Jordan on a set of pivots
// compose into this block step).  Each matrix row is then streamed once per panel
// instead of once per column.  One thread eliminates the panel (n x NB values, cache
// resident); the rank-NB update, nearly all of the arithmetic, is split over nth threads
// by contiguous row ranges, so the threads meet three times per panel.
static bool invert_gauss_jordan_blocked(double* A, int n, int nth) {
  constexpr int NB = 32, JB = 256;
  nth = std::max(1, std::min(nth, n / 32));
  std::vector<int> piv(n);
  double amax = 0.0;
  for (size_t i = 0; i < (size_t)n * n; ++i) amax = std::max(amax, std::fabs(A[i]));
  std::vector<double> T((size_t)NB * n), W((size_t)n * NB);
  HybridBarrier bar(nth);
  std::atomic<bool> ok{true};
  // the panel's columns [c0, c1) of every row are eliminated in W (n x kb, contiguous:
  // the column walks of the pivot search and the updates stay within a few MB instead of
  // touching one page per matrix row); a row interchange swaps the rows' W parts and the
  // rest of the rows in A
  auto panel = [&](int c0, int c1) {
    const int kb = c1 - c0;
    for (int i = 0; i < n; ++i) std::memcpy(&W[(size_t)i * kb], A + (size_t)i * n + c0, sizeof(double) * kb);
    bool good = true;
    for (int c = c0; c < c1 && good; ++c) {
      const int lc = c - c0;
      // pivot: the first row (in order) of largest magnitude in column c among rows >= c
      int p = c;
      double best = std::fabs(W[(size_t)c * kb + lc]);
      for (int i = c + 1; i < n; ++i) {
        const double v = std::fabs(W[(size_t)i * kb + lc]);
        if (v > best) { best = v; p = i; }
      }
      if (!(best > 1e-14 * amax)) { good = false; break; }
      piv[c] = p;
      if (p != c) {
        for (int j = 0; j < kb; ++j) std::swap(W[(size_t)c * kb + j], W[(size_t)p * kb + j]);
        for (int j = 0; j < c0; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
        for (int j = c1; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
      }
      double* rc = &W[(size_t)c * kb];
      const double inv = 1.0 / rc[lc];
      rc[lc] = 1.0;
      for (int j = 0; j < kb; ++j) rc[j] *= inv;
      for (int i = 0; i < n; ++i) {
        if (i == c) continue;
        double* ri = &W[(size_t)i * kb];
        const double f = ri[lc];
        if (f == 0.0) continue;
        ri[lc] = 0.0;
        for (int j = 0; j < kb; ++j) ri[j] -= f * rc[j];
      }
    }
    for (int i = 0; i < n; ++i) std::memcpy(A + (size_t)i * n + c0, &W[(size_t)i * kb], sizeof(double) * kb);
    return good;
  };
  auto worker = [&](int t) {
    const int lo = (int)((long long)n * t / nth), hi = (int)((long long)n * (t + 1) / nth);
    double a[NB], b[NB];
    for (int c0 = 0; c0 < n; c0 += NB) {
      const int kb = std::min(NB, n - c0), c1 = c0 + kb;
      if (t == 0 && !panel(c0, c1)) ok.store(false);
      bar.wait();                               // the panel is complete in every row
      if (!ok.load()) return;
      for (int q = t; q < kb; q += nth) {       // T = old [P,R]; [P,R] = 0 (gets E^-1 T below)
        double* rp = A + (size_t)(c0 + q) * n;
        double* tq = T.data() + (size_t)q * n;
        for (int j = 0; j < c0; ++j) { tq[j] = rp[j]; rp[j] = 0.0; }
        for (int j = c1; j < n; ++j) { tq[j] = rp[j]; rp[j] = 0.0; }
      }
      bar.wait();
      // columns in chunks of JB: the chunk of T (kb x JB, 64 KB) stays in the core's
      // cache while the thread's rows pass through it
      for (int j0 = 0; j0 < n; j0 += JB) {
        const int j1 = std::min(n, j0 + JB);
        const int ja = std::min(j1, c0), jb = std::max(j0, c1);   // the chunk without the panel
        if (ja <= j0 && jb >= j1) continue;
        int i = lo;
        for (; i + 2 <= hi; i += 2) {
          double* ri = A + (size_t)i * n;
          double* rs = ri + n;
          for (int q = 0; q < kb; ++q) { a[q] = ri[c0 + q]; b[q] = rs[c0 + q]; }
          if (ja > j0) rank_update2(ri, rs, a, b, T.data(), n, kb, j0, ja);
          if (jb < j1) rank_update2(ri, rs, a, b, T.data(), n, kb, jb, j1);
        }
        if (i < hi) {
          double* ri = A + (size_t)i * n;
          for (int q = 0; q < kb; ++q) a[q] = ri[c0 + q];
          if (ja > j0) rank_update1(ri, a, T.data(), n, kb, j0, ja);
          if (jb < j1) rank_update1(ri, a, T.data(), n, kb, jb, j1);
        }
      }
      bar.wait();                               // every row is up to date for the next panel
    }
  };
  // the helper threads wait at a gate until all of them exist: if one cannot be created,
  // the others are sent home before they reach a barrier and the work runs on one thread
  std::atomic<int> gate{0};                   // 0 wait, 1 run, -1 cancelled
  std::vector<std::thread> th;
  try {
    for (int t = 1; t < nth; ++t)
      th.emplace_back([&, t]() {
        while (gate.load(std::memory_order_acquire) == 0) std::this_thread::yield();
        if (gate.load(std::memory_order_acquire) > 0) worker(t);
      });
  } catch (const std::exception&) {
    gate.store(-1, std::memory_order_release);
    for (auto& x : th) x.join();
    return invert_gauss_jordan_blocked(A, n, 1);
  }
  gate.store(1, std::memory_order_release);
  worker(0);
  for (auto& x : th) x.join();
  if (!ok.load()) return false;
  for (int c = n - 1; c >= 0; --c)
    if (piv[c] != c)
      for (int i = 0; i < n; ++i) std::swap(A[(size_t)i * n + c], A[(size_t)i * n + piv[c]]);
  return true;
}

// In-place inverse of the row-major n x n matrix A (Gauss-Jordan, partial pivoting).
// nth: threads for the blocked form (n >= 256); 0 = the CPUs the process may use, at
// most 32.
bool invert_gauss_jordan(double* A, int n, int nth) {
  if (n >= 256) {
    if (nth <= 0) nth = std::min(32, usable_cpus());
    return invert_gauss_jordan_blocked(A, n, nth);
  }
  std::vector<int> piv(n);
  std::vector<double> row(n);
  double amax = 0.0;
  for (size_t i = 0; i < (size_t)n * n; ++i) amax = std::max(amax, std::fabs(A[i]));
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = std::fabs(A[(size_t)c * n + c]);
    for (int i = c + 1; i < n; ++i) {
      const double v = std::fabs(A[(size_t)i * n + c]);
      if (v > best) { best = v; p = i; }
    }
    if (!(best > 1e-14 * amax)) return false;
    piv[c] = p;
    if (p != c)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
    const double inv = 1.0 / A[(size_t)c * n + c];
    A[(size_t)c * n + c] = 1.0;
    double* rc = A + (size_t)c * n;
    for (int j = 0; j < n; ++j) rc[j] *= inv;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      double* ri = A + (size_t)i * n;
      const double f = ri[c];
      if (f == 0.0) continue;
      ri[c] = 0.0;
      for (int j = 0; j < n; ++j) ri[j] -= f * rc[j];
    }
  }
  // undo the row interchanges as column interchanges, last first
  for (int c = n - 1; c >= 0; --c)
    if (piv[c] != c)
      for (int i = 0; i < n; ++i) std::swap(A[(size_t)i * n + c], A[(size_t)i * n + piv[c]]);
  return true;
}

bool build_class_inverses(LevelHost* L) {
  const int nc = (int)L->class_rep.size(), B = L->B;
  // classes run in parallel; a large inverse gets the threads the classes leave free
  const unsigned hw = (unsigned)usable_cpus();
  const unsigned nth = std::max(1u, std::min(16u, hw));
  const int inner = nc <= 1 ? 0 : std::max(1, (int)(hw / std::min<unsigned>(nth, (unsigned)nc)));
  L->class_inv.assign((size_t)nc * B * B, 0.0);
  std::vector<int> ok(nc, 1);
  const long long poff = (long long)L->kt * L->n_vel;
  auto work = [&](int c) {
    std::vector<double> S;
    const std::vector<long long>& idx = L->class_idx[c];
    assemble_submatrix(*L, idx, L->class_dir[c], &S);
    const int b = L->class_B[c];
    // a patch holding every cell's pressure (the centre vertex star of a 2x2 mesh) is
    // surrounded by boundary dofs only: singular in the pressure constant of every
    // temporal dof; invert it bordered like the coarsest level (zero-mean correction)
    std::vector<int> mode0;
    for (int i = 0; i < b; ++i)
      if (idx[i] >= poff && (idx[i] - poff) % L->n_pres % L->npm == 0) mode0.push_back(i);
    if ((long long)mode0.size() == (long long)L->kt * L->n_cells) {
      const int kt = L->kt, bb = b + kt;
      std::vector<double> A((size_t)bb * bb, 0.0);
      for (int i = 0; i < b; ++i) std::memcpy(&A[(size_t)i * bb], &S[(size_t)i * b], sizeof(double) * b);
      for (int i : mode0) {
        const int a = (int)((idx[i] - poff) / L->n_pres);
        A[(size_t)i * bb + b + a] = 1.0;
        A[(size_t)(b + a) * bb + i] = 1.0;
      }
      if (!invert_gauss_jordan(A.data(), bb, inner)) { ok[c] = 0; return; }
      for (int i = 0; i < b; ++i)
        std::memcpy(&L->class_inv[((size_t)c * B + i) * B], &A[(size_t)i * bb], sizeof(double) * b);
      return;
    }
    if (!invert_gauss_jordan(S.data(), b, inner)) { ok[c] = 0; return; }
    for (int i = 0; i < b; ++i)
      std::memcpy(&L->class_inv[((size_t)c * B + i) * B], &S[(size_t)i * b], sizeof(double) * b);
  };
  if (nc <= 1 || nth <= 1) {
    for (int c = 0; c < nc; ++c) work(c);
  } else {
    std::vector<std::thread> th;
    unsigned started = 0;
    try {
      for (unsigned t = 0; t < nth; ++t) {
        th.emplace_back([&, t]() { for (int c = (int)t; c < nc; c += (int)nth) work(c); });
        ++started;
      }
    } catch (const std::exception&) {
      // a thread could not be created: its classes run here after the others
    }
    for (auto& t : th) t.join();
    for (unsigned t = started; t < nth; ++t)
      for (int c = (int)t; c < nc; c += (int)nth) work(c);
  }
  for (int c = 0; c < nc; ++c) if (!ok[c]) return false;
  return true;
}

bool build_coarse_inverse(LevelHost* L, std::vector<double>* Gcm) {
  // all dofs of the level, in slab order
  std::vector<long long> idx(L->size);
  std::vector<char> dir(L->size, 0);
  for (long long i = 0; i < L->size; ++i) idx[i] = i;
  for (int a = 0; a < L->kt; ++a)
    for (int comp = 0; comp < L->dim; ++comp)
      for (long long g = 0; g < L->n_nodes; ++g) {
        int gg[3] = {0, 0, 0};
        long long t = g;
        for (int d = 0; d < L->dim; ++d) { gg[d] = (int)(t % L->G); t /= L->G; }
        if (node_dirichlet(*L, gg)) dir[a * L->n_vel + comp * L->n_nodes + g] = 1;
      }
  std::vector<double> S;
  assemble_submatrix(*L, idx, dir, &S);
  const int D = (int)L->size, kt = L->kt, Db = D + kt;
  std::vector<double> A((size_t)Db * Db, 0.0);
  for (int i = 0; i < D; ++i) std::memcpy(&A[(size_t)i * Db], &S[(size_t)i * D], sizeof(double) * D);
  const long long poff = (long long)kt * L->n_vel;
  for (int a = 0; a < kt; ++a)
    for (long long c = 0; c < L->n_cells; ++c) {
      const long long i = poff + a * L->n_pres + c * L->npm;   // mode 0 = the constant
      A[(size_t)i * Db + D + a] = 1.0;
      A[(size_t)(D + a) * Db + i] = 1.0;
    }
  if (!invert_gauss_jordan(A.data(), Db)) return false;
  Gcm->assign((size_t)D * D, 0.0);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) (*Gcm)[(size_t)j * D + i] = A[(size_t)i * Db + j];   // column-major
  return true;
}

}  // namespace stmg
