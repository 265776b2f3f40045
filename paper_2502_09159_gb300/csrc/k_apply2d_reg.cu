// Matrix-free slab operator on 2D levels, register-resident form (Sec. 4.5, Eq. InAlg /
// DefDtauh).
//
// One thread per (cell, temporal dof a, velocity component d), threads of a warp on
// consecutive cells of one (a, d), so that the loads of a warp are unit-stride runs and
// every read of the parameter bank (the 1D factors, K_tau, the mode tables) is uniform
// across the warp.  The thread holds the cell's NP x NP node values of its component in
// registers and applies, with compile-time loop bounds and indices throughout:
//   u~     = sum_b K_tau[a,b] u_b                                  (time combination)
//   cont_m += sum_q F_x(m, ix) F_y(m, iy) u_a[q]                   (continuity rows)
//   A1     = h^d (M1 along y) u~ + beta_a (K1 along y) u_a,  A2 = (M1 along y) u_a
//   y_q    = (M1 along x) A1 + beta_a (K1 along x) A2 + bscale_a sum_m F_x(m, ix) F_y(m, iy) p_a[m]
// with F = G1 = int L ell' in the direction of component d and N1 = int L ell in the other
// one (the B_h^T / B_h factors of the Legendre pressure modes), both B_h terms
// sum-factorised over the modes (ex, ey): first along one direction, then the other.  Every row is scatter-added (nodes on cell faces belong to two
// or four cells, a cell's pressure rows get one share per component; y zero-filled before
// the launch).  Boundary rows are the identity, added by the cell that owns the node;
// boundary columns read as 0.  LIFT reads only the boundary values of x and no pressure;
// APPLY_T transposes K_tau.  About 35 multiply-adds per dof, no shared memory, no barrier.
#include <cuda_runtime.h>

#include "internal.h"
#include "mg_device.cuh"

namespace stmg {

template <typename T, int NP, int KT>
__global__ void __launch_bounds__(64) k_apply2d_reg(const ApplyRegParams<T> P, const T* __restrict__ x,
                                                    const T* __restrict__ b, T* __restrict__ y, int mode) {
  apply2d_reg_thread<T, NP, KT, false>(P, x, b, y, mode, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename T, int NP, int KT>
static cudaError_t launch_apply2d_reg_t(const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode, int bs,
                                        cudaStream_t st) {
  const long long tot = (long long)p.n * p.n * KT * 2;      // (cell, temporal dof, component)
  // small blocks (the finest levels have few cells); bs < 64 spreads the items evenly
  // over the SMs when 64 does not divide them into equal shares
  const int threads = bs >= 1 && bs <= 64 ? bs : 64;
  const unsigned blocks = (unsigned)((tot + threads - 1) / threads);
  k_apply2d_reg<T, NP, KT><<<blocks, threads, 0, st>>>(p, x, b, y, mode);
  return cudaGetLastError();
}

// the shapes whose cell tile fits the registers (FP32 up to Q5, FP64 up to Q3)
template <typename T>
bool apply2d_reg_supported(int np, int kt, int npm) {
  const int np_max = sizeof(T) == 4 ? 5 : 4;
  return np >= 3 && np <= np_max && kt >= 1 && kt <= 4 && npm == np * (np - 1) / 2;
}

template <typename T>
cudaError_t launch_apply2d_reg(int np, const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode, int bs,
                               cudaStream_t st) {
#define STMG_R2(N, K) \
  if (np == N && p.kt == K) return launch_apply2d_reg_t<T, N, K>(p, x, b, y, mode, bs, st);
  if (!apply2d_reg_supported<T>(np, p.kt, p.npm)) return cudaErrorInvalidValue;
  STMG_R2(3, 1) STMG_R2(3, 2) STMG_R2(3, 3) STMG_R2(3, 4)
  STMG_R2(4, 1) STMG_R2(4, 2) STMG_R2(4, 3) STMG_R2(4, 4)
  if constexpr (sizeof(T) == 4) {
    STMG_R2(5, 1) STMG_R2(5, 2) STMG_R2(5, 3) STMG_R2(5, 4)
  }
#undef STMG_R2
  return cudaErrorInvalidValue;
}

// residual with the coarser level's correction prolongated on the fly (single precision):
// x2 = x + P ec, r = b - S x2 (y = r zero on entry); the transfer shapes of the gather form
// with a register-resident fine level: Q3 <- Q2 on one mesh, Q2 <- Q2 on one mesh or on
// the mesh of half the cells
template <int NP, int KT, int NPC, int HT>
__global__ void __launch_bounds__(64) k_apply2d_reg_pro(const ApplyRegParams<float> P, const TransferParams<float> Q,
                                                        const float* __restrict__ x, const float* __restrict__ ec,
                                                        const float* __restrict__ b, float* __restrict__ y,
                                                        float* __restrict__ x2) {
  apply2d_reg_thread<float, NP, KT, false, NPC, HT>(P, x, b, y, RESIDUAL, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                                                    &Q, ec, x2);
}

// residual restricted to the coarser level in the same launch (single precision):
// bc = P^T (b - S x) (bc zero on entry), xc = 0 at every coarse dof; same shapes
template <int NP, int KT, int NPC, int HT>
__global__ void __launch_bounds__(64) k_apply2d_reg_rst(const ApplyRegParams<float> P, const TransferParams<float> Q,
                                                        const float* __restrict__ x, const float* __restrict__ b,
                                                        float* __restrict__ bc, float* __restrict__ xc) {
  apply2d_reg_thread<float, NP, KT, false, NPC, HT, true>(P, x, b, nullptr, RESIDUAL,
                                                          blockIdx.x * (long long)blockDim.x + threadIdx.x, &Q, nullptr,
                                                          nullptr, bc, xc);
}

cudaError_t launch_apply2d_reg_rst(int np, const ApplyRegParams<float>& p, const TransferParams<float>& q,
                                   const float* x, const float* b, float* bc, float* xc, int bs, cudaStream_t st) {
  if (!apply2d_reg_pro_supported(np, p.kt, p.npm, q.npc, q.h_type, q.ktc)) return cudaErrorInvalidValue;
  const long long tot = (long long)p.n * p.n * p.kt * 2;
  const int threads = bs >= 1 && bs <= 64 ? bs : 64;
  const unsigned blocks = (unsigned)((tot + threads - 1) / threads);
#define STMG_RST(N, K, C, H)                                                                            \
  if (np == N && p.kt == K && q.npc == C && q.h_type == H) {                                            \
    k_apply2d_reg_rst<N, K, C, H><<<blocks, threads, 0, st>>>(p, q, x, b, bc, xc);                    \
    return cudaGetLastError();                                                                           \
  }
#define STMG_RST_K(N, C, H) STMG_RST(N, 1, C, H) STMG_RST(N, 2, C, H) STMG_RST(N, 3, C, H) STMG_RST(N, 4, C, H)
  STMG_RST_K(4, 3, 0) STMG_RST_K(3, 3, 0) STMG_RST_K(3, 3, 1)
#undef STMG_RST_K
#undef STMG_RST
  return cudaErrorInvalidValue;
}

bool apply2d_reg_pro_supported(int np, int kt, int npm, int npc, int ht, int ktc) {
  if (!apply2d_reg_supported<float>(np, kt, npm) || ktc > kt) return false;
  return (np == 4 && npc == 3 && ht == 0) || (np == 3 && npc == 3 && (ht == 0 || ht == 1));
}

cudaError_t launch_apply2d_reg_pro(int np, const ApplyRegParams<float>& p, const TransferParams<float>& q,
                                   const float* x, const float* ec, const float* b, float* y, float* x2, int bs,
                                   cudaStream_t st) {
  if (!apply2d_reg_pro_supported(np, p.kt, p.npm, q.npc, q.h_type, q.ktc)) return cudaErrorInvalidValue;
  const long long tot = (long long)p.n * p.n * p.kt * 2;
  const int threads = bs >= 1 && bs <= 64 ? bs : 64;
  const unsigned blocks = (unsigned)((tot + threads - 1) / threads);
#define STMG_PRO(N, K, C, H)                                                                            \
  if (np == N && p.kt == K && q.npc == C && q.h_type == H) {                                            \
    k_apply2d_reg_pro<N, K, C, H><<<blocks, threads, 0, st>>>(p, q, x, ec, b, y, x2);                 \
    return cudaGetLastError();                                                                           \
  }
#define STMG_PRO_K(N, C, H) STMG_PRO(N, 1, C, H) STMG_PRO(N, 2, C, H) STMG_PRO(N, 3, C, H) STMG_PRO(N, 4, C, H)
  STMG_PRO_K(4, 3, 0) STMG_PRO_K(3, 3, 0) STMG_PRO_K(3, 3, 1)
#undef STMG_PRO_K
#undef STMG_PRO
  return cudaErrorInvalidValue;
}

// pair-split form: two lanes per (cell, temporal dof, component), NP even (Q3 in 2D)
template <typename T, int NP, int KT>
__global__ void __launch_bounds__(32) k_apply2d_pair(const ApplyRegParams<T> P, const T* __restrict__ x,
                                                     const T* __restrict__ b, T* __restrict__ y, int mode) {
  apply2d_pair_thread<T, NP, KT, false>(P, x, b, y, mode, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <typename T, int NP, int KT>
static cudaError_t launch_apply2d_pair_t(const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode,
                                         cudaStream_t st) {
  const long long tot = (long long)p.n * p.n * KT * 2 * 2;  // (cell, temporal dof, component, column half)
  // one-warp blocks (every lane reaches the shuffles): on a level of few cells the warps
  // then spread over the SMs in units of one warp, not two
  const unsigned blocks = (unsigned)((tot + 31) / 32);
  k_apply2d_pair<T, NP, KT><<<blocks, 32, 0, st>>>(p, x, b, y, mode);
  return cudaGetLastError();
}

template <typename T>
bool apply2d_pair_supported(int np, int kt, int npm) {
  return np == 4 && kt >= 1 && kt <= 4 && npm == np * (np - 1) / 2;
}

template <typename T>
cudaError_t launch_apply2d_pair(int np, const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode,
                                cudaStream_t st) {
  if (!apply2d_pair_supported<T>(np, p.kt, p.npm)) return cudaErrorInvalidValue;
  switch (p.kt) {
    case 1: return launch_apply2d_pair_t<T, 4, 1>(p, x, b, y, mode, st);
    case 2: return launch_apply2d_pair_t<T, 4, 2>(p, x, b, y, mode, st);
    case 3: return launch_apply2d_pair_t<T, 4, 3>(p, x, b, y, mode, st);
    default: return launch_apply2d_pair_t<T, 4, 4>(p, x, b, y, mode, st);
  }
}

template cudaError_t launch_apply2d_pair<double>(int, const ApplyRegParams<double>&, const double*, const double*,
                                                 double*, int, cudaStream_t);
template cudaError_t launch_apply2d_pair<float>(int, const ApplyRegParams<float>&, const float*, const float*,
                                                float*, int, cudaStream_t);
template bool apply2d_pair_supported<double>(int, int, int);
template bool apply2d_pair_supported<float>(int, int, int);

template cudaError_t launch_apply2d_reg<double>(int, const ApplyRegParams<double>&, const double*, const double*,
                                                double*, int, int, cudaStream_t);
template cudaError_t launch_apply2d_reg<float>(int, const ApplyRegParams<float>&, const float*, const float*, float*,
                                               int, int, cudaStream_t);
template bool apply2d_reg_supported<double>(int, int, int);
template bool apply2d_reg_supported<float>(int, int, int);

}  // namespace stmg
