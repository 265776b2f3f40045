// Matrix-free slab operator on 2D levels, register-resident form (Sec. 4.5, Eq. InAlg /
// DefDtauh).
//
// One thread per (cell, temporal dof a), threads of a warp on consecutive cells of one cell
// row and the same a, so that the loads of a warp are unit-stride runs and every read of
// the parameter bank (the 1D factors, K_tau, the mode tables) is uniform across the warp.
// Per velocity component the thread holds the cell's NP x NP node values in registers and
// applies, with compile-time loop bounds and indices throughout:
//   u~     = sum_b K_tau[a,b] u_b                                  (time combination)
//   cont_m += sum_q CB_d[m][q] u_a[q]                              (continuity rows)
//   A1     = h^d (M1 along y) u~ + beta_a (K1 along y) u_a,  A2 = (M1 along y) u_a
//   y_q    = (M1 along x) A1 + beta_a (K1 along x) A2 + bscale_a sum_m CB_d[m][q] p_a[m]
// with CB_d[m][q] = F(mode m, x, ix) F(mode m, y, iy), F = G1 = int L ell' in the direction
// of component d and N1 = int L ell in the other one (the B_h^T / B_h factors of the
// Legendre pressure modes).  The velocity rows are scatter-added (nodes on cell faces
// belong to two or four cells; y zero-filled before the launch), the cell's pressure rows
// are stored.  Boundary rows are the identity, written by the cell that owns the node;
// boundary columns read as 0.  LIFT reads only the boundary values of x and no pressure;
// APPLY_T transposes K_tau.  About 35 multiply-adds per dof, no shared memory, no barrier.
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

template <typename T, int NP, int KT>
__global__ void __launch_bounds__(64) k_apply2d_reg(const ApplyRegParams<T> P, const T* __restrict__ x,
                                                     const T* __restrict__ b, T* __restrict__ y, int mode) {
  constexpr int E = NP - 1, NQ = NP * NP;
  constexpr int NPM = NP * (NP - 1) / 2;            // C(r + 2, 2) pressure modes, r = NP - 2
  const int n = P.n, G = P.G;
  const long long ncells = (long long)n * n;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncells * KT) return;
  const int a = (int)(t / ncells);
  const long long c = t - (long long)a * ncells;
  const int cx = (int)(c % n), cy = (int)(c / n);
  const long long nvel = P.n_vel, nnod = P.n_nodes;
  const long long poff = (long long)KT * nvel;
  const bool res = mode == RESIDUAL || mode == LIFT;
  const bool lift = mode == LIFT;
  const bool tr = mode == APPLY_T;
  const long long base = (long long)(cy * E) * G + cx * E;      // global index of the cell's node (0, 0)
  // boundary lines of the cell's nodes (the mesh boundary crosses a cell only at its outer lines)
  const bool bx0 = cx == 0, bx1 = cx == n - 1, by0 = cy == 0, by1 = cy == n - 1;

  T p[NPM];
#pragma unroll
  for (int m = 0; m < NPM; ++m) p[m] = lift ? T(0) : x[poff + (long long)a * P.n_pres + c * NPM + m];
  T cont[NPM];
#pragma unroll
  for (int m = 0; m < NPM; ++m) cont[m] = 0;
  T kt_row[KT];
#pragma unroll
  for (int bb = 0; bb < KT; ++bb) kt_row[bb] = tr ? P.Kt[bb * MAXKT + a] : P.Kt[a * MAXKT + bb];
  const T beta = P.beta[a], bsc = P.bscale[a], hd = P.hd;

#pragma unroll
  for (int d = 0; d < 2; ++d) {
    T ut[NQ], ua[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { ut[q] = 0; ua[q] = 0; }
#pragma unroll
    for (int bb = 0; bb < KT; ++bb) {
      const T* xb = x + bb * nvel + d * nnod + base;
#pragma unroll
      for (int iy = 0; iy < NP; ++iy) {
        const bool dy = (iy == 0 && by0) || (iy == E && by1);
#pragma unroll
        for (int ix = 0; ix < NP; ++ix) {
          const bool dir = dy || (ix == 0 && bx0) || (ix == E && bx1);
          const bool take = lift ? dir : !dir;
          const T v = take ? xb[iy * G + ix] : T(0);
          ut[iy * NP + ix] += kt_row[bb] * v;
          if (bb == a) ua[iy * NP + ix] = v;
        }
      }
    }
    // continuity rows of this component
#pragma unroll
    for (int m = 0; m < NPM; ++m) {
      T s = 0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += P.CB[d][m][q] * ua[q];
      cont[m] += s;
    }
    // y-pass: A1 = hd M1y ut + beta K1y ua, A2 = M1y ua (column by column)
    T A1[NQ], A2[NQ];
#pragma unroll
    for (int ix = 0; ix < NP; ++ix) {
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T m1 = 0, k1 = 0, m2 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          m1 += P.M1[i * NP + j] * ut[j * NP + ix];
          k1 += P.K1[i * NP + j] * ua[j * NP + ix];
          m2 += P.M1[i * NP + j] * ua[j * NP + ix];
        }
        A1[i * NP + ix] = hd * m1 + beta * k1;
        A2[i * NP + ix] = m2;
      }
    }
    // x-pass, pressure gradient, scatter (row by row)
    T* yd = y + a * nvel + d * nnod + base;
    const T* bd = b + a * nvel + d * nnod + base;
    const T* xd = x + a * nvel + d * nnod + base;
#pragma unroll
    for (int iy = 0; iy < NP; ++iy) {
      const bool dy = (iy == 0 && by0) || (iy == E && by1);
      const bool oy = iy < E || by1;                      // this cell owns the node row (for boundary rows)
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const bool dir = dy || (i == 0 && bx0) || (i == E && bx1);
        const bool own = oy && (i < E || bx1);
        const long long off = (long long)iy * G + i;
        if (dir) {
          if (own) {
            const T xv = xd[off];
            yd[off] = mode == RESIDUAL ? bd[off] - xv : xv;   // identity row, written by its owner only
          }
          continue;
        }
        T m1 = 0, k1 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          m1 += P.M1[i * NP + j] * A1[iy * NP + j];
          k1 += P.K1[i * NP + j] * A2[iy * NP + j];
        }
        T bt = 0;
#pragma unroll
        for (int m = 0; m < NPM; ++m) bt += P.CB[d][m][iy * NP + i] * p[m];
        T v = m1 + beta * k1 + bsc * bt;
        if (res) v = own ? bd[off] - v : -v;               // b enters once, through the owner
        atomicAdd(yd + off, v);
      }
    }
  }
  // pressure rows of the cell
#pragma unroll
  for (int m = 0; m < NPM; ++m) {
    const long long gi = poff + (long long)a * P.n_pres + c * NPM + m;
    const T v = bsc * cont[m];
    y[gi] = res ? b[gi] - v : v;
  }
}

template <typename T, int NP, int KT>
static cudaError_t launch_apply2d_reg_t(const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode,
                                        cudaStream_t st) {
  const long long tot = (long long)p.n * p.n * KT;
  const unsigned blocks = (unsigned)((tot + 63) / 64);      // small blocks: the finest levels have few cells
  k_apply2d_reg<T, NP, KT><<<blocks, 64, 0, st>>>(p, x, b, y, mode);
  return cudaGetLastError();
}

// the shapes whose cell tile fits the registers (FP32 up to Q5, FP64 up to Q3)
template <typename T>
bool apply2d_reg_supported(int np, int kt, int npm) {
  const int np_max = sizeof(T) == 4 ? 5 : 4;
  return np >= 3 && np <= np_max && kt >= 1 && kt <= 4 && npm == np * (np - 1) / 2;
}

template <typename T>
cudaError_t launch_apply2d_reg(int np, const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode,
                               cudaStream_t st) {
#define STMG_R2(N, K) \
  if (np == N && p.kt == K) return launch_apply2d_reg_t<T, N, K>(p, x, b, y, mode, st);
  if (!apply2d_reg_supported<T>(np, p.kt, p.npm)) return cudaErrorInvalidValue;
  STMG_R2(3, 1) STMG_R2(3, 2) STMG_R2(3, 3) STMG_R2(3, 4)
  STMG_R2(4, 1) STMG_R2(4, 2) STMG_R2(4, 3) STMG_R2(4, 4)
  if constexpr (sizeof(T) == 4) {
    STMG_R2(5, 1) STMG_R2(5, 2) STMG_R2(5, 3) STMG_R2(5, 4)
  }
#undef STMG_R2
  return cudaErrorInvalidValue;
}

template cudaError_t launch_apply2d_reg<double>(int, const ApplyRegParams<double>&, const double*, const double*,
                                                double*, int, cudaStream_t);
template cudaError_t launch_apply2d_reg<float>(int, const ApplyRegParams<float>&, const float*, const float*, float*,
                                               int, cudaStream_t);
template bool apply2d_reg_supported<double>(int, int, int);
template bool apply2d_reg_supported<float>(int, int, int);

}  // namespace stmg
