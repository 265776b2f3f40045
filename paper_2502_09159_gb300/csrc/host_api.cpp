// Host-only entry points of libstmg: the setup numerics without a GPU (hierarchy, 1D and
// temporal tables, patch index sets and patch inverses, the coarse bordered inverse).
// They let a CPU-only process inspect exactly what stmg_create would upload.
#include <cstring>
#include <exception>
#include <vector>

#include "internal.h"
#include "levels.h"
#include "stmg.h"

using namespace stmg;

extern "C" {

int stmg_host_default_hierarchy(int n, int r, int k, int coarse_n, int k_min, int* levels, int* count) {
  if (!levels || !count || n < 1 || r < 1 || k < 0 || coarse_n < 1 || k_min < 1) return STMG_ERR_ARG;
  auto lv = default_hierarchy(n, r, k, coarse_n, k_min);
  if ((int)lv.size() > STMG_MAX_LEVELS) return STMG_ERR_ARG;
  for (size_t i = 0; i < lv.size(); ++i)
    for (int j = 0; j < 3; ++j) levels[3 * i + j] = lv[i][j];
  *count = (int)lv.size();
  return STMG_OK;
}

int stmg_host_tables_1d(int r, double* xi, double* M1, double* K1, double* G1, double* N1) {
  if (r < 1 || r > 4) return STMG_ERR_ARG;
  try {
    Tables1D t = make_tables_1d(r);
    const int np = r + 2;
    if (xi) std::memcpy(xi, t.xi, sizeof(double) * np);
    if (M1) std::memcpy(M1, t.M1, sizeof(double) * np * np);
    if (K1) std::memcpy(K1, t.K1, sizeof(double) * np * np);
    if (G1) std::memcpy(G1, t.G1, sizeof(double) * (r + 1) * np);
    if (N1) std::memcpy(N1, t.N1, sizeof(double) * (r + 1) * np);
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  return STMG_OK;
}

int stmg_host_time_tables(int k, double tau, double* nodes, double* weights, double* K, double* Mdiag,
                          double* phi_left) {
  if (k < 0 || k > 3 || !(tau > 0)) return STMG_ERR_ARG;
  try {
    TimeTables t = make_time_tables(k, tau);
    const int kt = k + 1;
    if (nodes) std::memcpy(nodes, t.nodes, sizeof(double) * kt);
    if (weights) std::memcpy(weights, t.weights, sizeof(double) * kt);
    if (K) std::memcpy(K, t.K, sizeof(double) * kt * kt);
    if (Mdiag) std::memcpy(Mdiag, t.M, sizeof(double) * kt);
    if (phi_left) std::memcpy(phi_left, t.phi_left, sizeof(double) * kt);
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  return STMG_OK;
}

// Patch `patch` of kind STMG_CELL / STMG_VSP on the level (dim, n, r, k): its dof list
// (slab indices; -1 boundary, -2 padding; length *B) and its FP64 inverse (row-major
// *B x *B, padding rows/columns zero).  Pass dofs = inv = NULL to query *B and the
// number of patches / classes.
int stmg_host_patch(int dim, int n, int r, int k, double nu, double tau, int kind, long long patch, int* dofs,
                    double* inv, int* B, long long* n_patches, int* n_classes) {
  if ((dim != 2 && dim != 3) || n < 1 || r < 1 || r > 4 || k < 0 || k > 3 || !B) return STMG_ERR_ARG;
  try {
    LevelHost L;
    init_level_geometry(&L, dim, n, r, k, tau, nu);
    build_patches(&L, kind == STMG_VSP ? STMG_VSP : STMG_CELL);
    *B = L.B;
    if (n_patches) *n_patches = L.n_patches;
    if (n_classes) *n_classes = (int)L.class_rep.size();
    if (!dofs && !inv) return STMG_OK;
    if (patch < 0 || patch >= L.n_patches) return STMG_ERR_ARG;
    if (dofs) std::memcpy(dofs, &L.dofs[(size_t)patch * L.B], sizeof(int) * L.B);
    if (inv) {
      if (!build_class_inverses(&L)) return STMG_ERR_SINGULAR;
      const int c = L.patch_class[patch];
      std::memcpy(inv, &L.class_inv[(size_t)c * L.B * L.B], sizeof(double) * L.B * L.B);
    }
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  return STMG_OK;
}

// Valence (number of patches containing each slab dof) of the level's patches.
int stmg_host_valence(int dim, int n, int r, int k, int kind, int* valence, long long* size) {
  if ((dim != 2 && dim != 3) || n < 1 || r < 1 || r > 4 || k < 0 || k > 3 || !size) return STMG_ERR_ARG;
  try {
    LevelHost L;
    init_level_geometry(&L, dim, n, r, k, 1.0, 1.0);
    *size = L.size;
    if (!valence) return STMG_OK;
    build_patches(&L, kind == STMG_VSP ? STMG_VSP : STMG_CELL);
    std::memcpy(valence, L.valence.data(), sizeof(int) * L.size);
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  return STMG_OK;
}

// Bordered coarse inverse G (column-major D x D) of the level (dim, n, r, k).
int stmg_host_coarse_inverse(int dim, int n, int r, int k, double nu, double tau, double* G, long long* D) {
  if ((dim != 2 && dim != 3) || n < 1 || r < 1 || r > 4 || k < 0 || k > 3 || !D) return STMG_ERR_ARG;
  try {
    LevelHost L;
    init_level_geometry(&L, dim, n, r, k, tau, nu);
    *D = L.size;
    if (!G) return STMG_OK;
    if (L.size > 6000) return STMG_ERR_ARG;
    std::vector<double> Gcm;
    if (!build_coarse_inverse(&L, &Gcm)) return STMG_ERR_SINGULAR;
    std::memcpy(G, Gcm.data(), sizeof(double) * Gcm.size());
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  return STMG_OK;
}

// In-place inverse of a row-major n x n matrix by the routine that inverts the patch
// matrices and the coarse bordered matrix.
int stmg_host_invert(double* A, int n, int threads) {
  if (!A || n < 1 || threads < 0) return STMG_ERR_ARG;
  try {
    if (!invert_gauss_jordan(A, n, threads)) return STMG_ERR_SINGULAR;
  } catch (const std::exception&) {
    return STMG_ERR_OOM;
  }
  return STMG_OK;
}

}  // extern "C"
