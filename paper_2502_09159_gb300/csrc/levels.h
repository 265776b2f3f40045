// Host-side level data of libstmg (built once in stmg_create, then uploaded).
#pragma once

#include <array>
#include <vector>

#include "internal.h"

namespace stmg {

struct LevelHost {
  int dim = 2, n = 1, r = 1, k = 0, kt = 1, nsub = 1, np = 3, nq = 9, G = 3, npm = 3, n_cells = 1;
  long long n_nodes = 0, n_vel = 0, n_pres = 0, size = 0;
  double h = 1.0, tau = 1.0, nu = 1.0;
  Tables1D t1;
  TimeTables tt;
  std::vector<std::array<int, 3>> modes;
  std::vector<double> Me, Ae, Be;          // element matrices [nq*nq], [nq*nq], [dim][npm][nq]
  // patches (all levels but the coarsest)
  int smoother = -1, B = 0, Bc = 0;
  long long n_patches = 0;
  std::vector<int> dofs;                   // [n_patches][B]: slab index, -1 boundary, -2 padding
  std::vector<int> patch_class;            // [n_patches]
  std::vector<long long> class_rep;        // representative patch per class
  std::vector<int> class_B;                // actual patch size per class
  std::vector<std::vector<long long>> class_idx;
  std::vector<std::vector<char>> class_dir;
  std::vector<double> class_inv;           // [n_classes][B][B] row-major FP64
  std::vector<int> valence;                // [size]
};

std::vector<std::array<int, 3>> default_hierarchy(int n, int r, int k, int coarse_n = 1, int k_min = 1);
void init_level_geometry(LevelHost* L, int dim, int n, int r, int k, double tau, double nu, int nsub = 1);
void build_patches(LevelHost* L, int kind);
void assemble_submatrix(const LevelHost& L, const std::vector<long long>& idx, const std::vector<char>& dir,
                        std::vector<double>* S);
bool invert_gauss_jordan(double* A, int n, int nth = 0);
bool build_class_inverses(LevelHost* L);
bool build_coarse_inverse(LevelHost* L, std::vector<double>* Gcm);

}  // namespace stmg
