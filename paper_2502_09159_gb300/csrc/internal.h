// Internal declarations of libstmg: level data, kernel parameter blocks and launchers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <array>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "stmg.h"

namespace stmg {

constexpr int MAXNP = 6;    // velocity nodes per direction per cell (r <= 4)
constexpr int MAXKT = 8;    // temporal dofs per system: n_sub (k + 1) <= 8
constexpr int MAXPM = 35;   // pressure modes per cell, C(4+3, 3)
constexpr int MAXNS = 2 * (MAXNP - 1) + 1;  // fine nodes per direction under one coarse cell

// ------------------------------------------------------------------------------------
// host-side numerics (setup.cpp)
// ------------------------------------------------------------------------------------
struct Tables1D {                 // one spatial degree on the reference interval [0,1]
  int np = 0;                     // r + 2 velocity nodes
  int r = 0;
  double xi[MAXNP];               // Gauss-Lobatto nodes
  double M1[MAXNP * MAXNP];       // int ell_i ell_j
  double K1[MAXNP * MAXNP];       // int ell_i' ell_j'
  double G1[MAXNP * MAXNP];       // [i * np + p] = int L_i ell_p'   (i <= r)
  double N1[MAXNP * MAXNP];       // [i * np + p] = int L_i ell_p
};

struct TimeTables {               // DG(k) with the right Radau Lagrange basis on n_sub subintervals
  int kt = 0;                     // n_sub (k + 1) temporal dofs, subinterval by subinterval
  int k1 = 0, nsub = 1;           // k + 1, subintervals per system
  double nodes1[MAXKT];           // Radau points of one subinterval on [-1, 1]
  double nodes[MAXKT], weights[MAXKT];   // nodes of subinterval j shifted by 2 j
  double K[MAXKT * MAXKT];        // [a * kt + b]: block-bidiagonal (K1 on, -C1 below the diagonal)
  double M[MAXKT];                // diagonal of the temporal mass, includes tau/2
  double phi_left[MAXKT];         // phi_a(t_{n-1}^+) on the first subinterval, 0 on the others
};

Tables1D make_tables_1d(int r);
TimeTables make_time_tables(int k, double tau, int nsub = 1);
void pressure_modes(int dim, int r, std::vector<std::array<int, 3>>* out);
void gauss_legendre(int n, double* x, double* w);            // on [-1, 1]
double lagrange_eval(const double* nodes, int n, int j, double t);
double legendre_unit(int i, double xi);                       // sqrt(2i+1) P_i(2 xi - 1)

// ------------------------------------------------------------------------------------
// kernel parameter blocks (passed by value; tables converted to the kernel type)
// ------------------------------------------------------------------------------------
template <typename T>
struct ApplyParams {
  int n, G, kt, npm, cpb;
  int variant;                    // 1: per-cell kernel (k_apply), 2: node-centred 2D kernel (k_apply2d),
                                  // 3: register-resident 2D kernel, 4: its pair-split form (k_apply2d_reg)
  int tcx, tcy;                   // variant 2: cells per block in x and y
  long long n_nodes, n_vel, n_pres;
  T M1[MAXNP * MAXNP], K1[MAXNP * MAXNP], G1[MAXNP * MAXNP], N1[MAXNP * MAXNP];
  T Kt[MAXKT * MAXKT];
  T hd;                           // h^d (mass scaling)
  T beta[MAXKT];                  // M_tau[a] nu h^(d-2) (Laplacian scaling)
  T bscale[MAXKT];                // -M_tau[a] h^(d-1)   (divergence scaling)
  signed char modes[MAXPM][3];
};

// register-resident 2D operator (k_apply2d_reg.cu): tables in the parameter bank
constexpr int MAXPM2 = 15;  // pressure modes per cell in 2D, C(4+2, 2)
// index of the 2D pressure mode (ex, ey) in a cell's mode list, ordered by degree
// s = ex + ey, then by ey: m = s (s + 1) / 2 + ey (the order of the host's mode tables;
// the register-resident operators rely on it)
__host__ __device__ constexpr int mode_index(int ex, int ey) { return (ex + ey) * (ex + ey + 1) / 2 + ey; }

// exponent k (0: x, 1: y, 2: z) of pressure mode m of degree <= r in the host's mode
// order: degree s ascending; in 2D (s - j, j) with j ascending, in 3D (s - l - j, j, l)
// with l, then j ascending.  Called with compile-time arguments it folds to a constant.
__host__ __device__ constexpr int mode_exp(int dim, int r, int m, int k) {
  int idx = 0;
  for (int s = 0; s <= r; ++s) {
    if (dim == 2) {
      for (int j = 0; j <= s; ++j, ++idx)
        if (idx == m) return k == 0 ? s - j : (k == 1 ? j : 0);
    } else {
      for (int l = 0; l <= s; ++l)
        for (int j = 0; j <= s - l; ++j, ++idx)
          if (idx == m) return k == 0 ? s - l - j : (k == 1 ? j : l);
    }
  }
  return 0;
}

template <typename T>
struct ApplyRegParams {
  int n, G, kt, npm;
  long long n_nodes, n_vel, n_pres;
  T M1[MAXNP * MAXNP], K1[MAXNP * MAXNP];
  // B_h factors of the 2D Legendre pressure modes (ex, ey) of degree ex + ey <= r, by
  // velocity component d: FX[d][ex * np + ix] along x, FY[d][ey * np + iy] along y
  // (G1 = int L ell' in the direction of d, N1 = int L ell in the other one)
  T FX[2][MAXNP * MAXNP], FY[2][MAXNP * MAXNP];
  T Kt[MAXKT * MAXKT];
  T hd, beta[MAXKT], bscale[MAXKT];
};

template <typename T>
struct TransferParams {
  int dim, h_type;                // h_type: 1 = n -> 2n in space, 0 = same mesh
  int nc, nf, npc, npf, ns;       // coarse / fine cells per dir, nodes per cell, span nodes
  int Gc, Gf, ktc, ktf, npmc, npmf, cpb;
  long long nnc, nnf, nvc, nvf, npc_tot, npf_tot;   // nodes, velocity dofs, pressure dofs
  T P1[MAXNS * MAXNP];            // [s * npc + j] = ell_j^coarse(position of fine node s)
  T Pt[MAXKT * MAXKT];            // [af * ktc + ac] = phi_ac^coarse(t_af^fine)
  T E[2][MAXNP * MAXNP];          // h-type pressure: E[o][i' * (rc+1) + i]
  signed char modes_c[MAXPM][3], modes_f[MAXPM][3];
  int rc;                         // coarse pressure degree
  int variant;                    // 1: per coarse cell (shared memory), 2: gather form (2D)
};

// one level of the persistent multigrid kernel (k_mg_persist.cu), in device memory
template <typename T>
struct MGLevelDesc {
  ApplyRegParams<T> rp;           // operator tables of the level (residual)
  TransferParams<T> tp;           // transfer to the next coarser level (gather form, Q2 -> Q2)
  T *b, *x, *r;                   // the level's V-cycle vectors
  const int* dofs;                // patch table [n_patches][B]
  const T* inv;                   // per-patch inverses, interleaved layout [patch][chunk][row][VW]
  long long n_patches, size;      // patches; D of the level
  int B, Bc, ppb, kt, ht;         // patch size, padded columns, patches per block, k + 1, h-type of tp
  const double* G;                // coarsest level: FP64 bordered inverse, column-major D x D
  double* acc;                    // coarsest level: FP64 accumulator (zero between uses)
  int D;
};

struct ForcingParams {
  int dim, n, G, np, nq, kt, cpb;
  long long n_nodes, n_vel;
  double phiq[MAXNP * 10];        // [p * nq + q] = ell_p(xq)
  double wq[10];                  // Gauss weights on [0,1] times h
  double scale[MAXKT];            // tau/2 w_a
};

struct MassParams {
  int dim, n, G, np, kt, cpb;
  long long n_nodes, n_vel;
  double M1[MAXNP * MAXNP];
  double hd;
  double phi_left[MAXKT];
};

struct CellsParams {              // level geometry for the cell-tensor maps
  int dim, n, r1, np, G, kt, npm, C, Pn;   // r1 = r + 1, Pn = np^dim nodes per cell
  long long n_nodes, nv, npr, size, n_cells;
  double E[MAXKT * MAXKT];        // [a * kt + b] = phi_b(s_a + 2): temporal extrapolation
};

// ------------------------------------------------------------------------------------
// launchers (return cudaError_t of the launch); all asynchronous on `st`
// ------------------------------------------------------------------------------------
enum ApplyMode { APPLY = 0, RESIDUAL = 1, LIFT = 2, APPLY_T = 3 };

template <typename T>
cudaError_t launch_apply(int dim, int np, const ApplyParams<T>& p, const T* x, const T* b, T* y,
                         int mode, cudaStream_t st);
template <typename T>
size_t apply_smem_bytes(int dim, int np, int kt, int npm, int cpb);
// register-resident form on 2D levels (k_apply2d_reg.cu), kt <= 4: y must be zero on entry
// (every row is scatter-added); bs threads per block (1..64, else 64)
template <typename T>
cudaError_t launch_apply2d_reg(int np, const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode, int bs,
                               cudaStream_t st);
template <typename T>
bool apply2d_reg_supported(int np, int kt, int npm);
// the register-resident residual with the coarser level's correction prolongated on the
// fly (single precision): x2 = x + P ec, y = b - S x2 (y zero on entry); q = the transfer
// between the two levels (fine level = this one)
bool apply2d_reg_pro_supported(int np, int kt, int npm, int npc, int ht, int ktc);
cudaError_t launch_apply2d_reg_pro(int np, const ApplyRegParams<float>& p, const TransferParams<float>& q,
                                   const float* x, const float* ec, const float* b, float* y, float* x2, int bs,
                                   cudaStream_t st);
// the register-resident residual restricted to the coarser level in the same launch
// (single precision): bc = P^T (b - S x) (bc zero on entry), xc = 0; the shapes of
// apply2d_reg_pro_supported
cudaError_t launch_apply2d_reg_rst(int np, const ApplyRegParams<float>& p, const TransferParams<float>& q,
                                   const float* x, const float* b, float* bc, float* xc, int bs, cudaStream_t st);
// its pair-split form (two lanes per cell item, Q3 only), y zero on entry as well
template <typename T>
cudaError_t launch_apply2d_pair(int np, const ApplyRegParams<T>& p, const T* x, const T* b, T* y, int mode,
                                cudaStream_t st);
template <typename T>
bool apply2d_pair_supported(int np, int kt, int npm);
// node-centred form on 2D levels (k_apply2d.cu): writes every entry of y, no zero-fill needed
template <typename T>
cudaError_t launch_apply2d(int np, const ApplyParams<T>& p, const T* x, const T* b, T* y, int mode, cudaStream_t st);
template <typename T>
size_t apply2d_smem_bytes(int np, int kt, int npm, int tcx, int tcy);

// block sweep: rounds of `unroll` (4 or 8) column chunks per load burst
template <typename T>
cudaError_t launch_vanka_sweep(const int* dofs, const T* inv, const T* res, T* x, long long n_patches, int B,
                               int Bc, int ppb, int unroll, int streaming, cudaStream_t st);
// pipelined block sweep (first loads before the gather, double-buffered rounds of `unroll`
// = 4 or 8 chunks); needs ppb * B <= 512
template <typename T>
cudaError_t launch_vanka_sweep_pipe(const int* dofs, const T* inv, const T* res, T* x, long long n_patches, int B,
                                    int Bc, int ppb, int unroll, int streaming, cudaStream_t st);
template <typename T>
bool pipe_sweep_supported(int B, int ppb);
constexpr int TMA_NCW = 4;   // consumer warps of the TMA-pipelined sweep (+1 producer warp)
// half-precision inverses with FP32 row scales for the FP32 V-cycle (k_vanka.cu)
cudaError_t launch_replicate_inverses_half(const double* cls, const int* cls_of_patch, const int* dofs, const double* w,
                                           __half* inv, float* rscale, long long n_patches, int B, int Bh,
                                           cudaStream_t st);
cudaError_t launch_vanka_sweep_half(const int* dofs, const __half* inv, const float* rscale, const float* res, float* x,
                                    long long n_patches, int B, int Bh, int ppb, int streaming, cudaStream_t st);
template <typename T>
cudaError_t launch_vanka_sweep_tma(const int* dofs, const T* inv, const T* res, T* x, long long n_patches, int B,
                                   int Bc, int n_sm, int streaming, int* err, cudaStream_t st);
template <typename T>
bool tma_sweep_supported(int B);
template <typename T>
cudaError_t launch_replicate_inverses(const double* cls, const int* cls_of_patch, const int* dofs,
                                      const double* w, T* inv, long long n_patches, int B, int Bc,
                                      cudaStream_t st);

template <typename T>
cudaError_t launch_prolongate(const TransferParams<T>& p, const T* yc, T* xf, cudaStream_t st);
// zc (may be NULL): the gather form also writes zeros to it (the coarse iterate of the
// V-cycle); the per-cell form leaves it alone
template <typename T>
cudaError_t launch_restrict(const TransferParams<T>& p, const T* rf, T* bc, T* zc, cudaStream_t st);
template <typename T>
size_t transfer_smem(const TransferParams<T>& p, int restrict_);
template <typename T>
bool transfer_gather_supported(const TransferParams<T>& p);   // the gather form has this shape

// coarse direct solve x = G b; G stored in FP64 or (FP32 V-cycle) FP32, products in G's type
template <typename T, typename M>
cudaError_t launch_coarse(int D, const M* Gcm, const T* b, T* x, cudaStream_t st);
template <typename T, typename M>
cudaError_t launch_coarse_tiled(int D, const M* Gcm, const T* b, T* x, double* acc, cudaStream_t st);

cudaError_t launch_mass_coupling(const MassParams& p, const double* vprev, double* b, cudaStream_t st);
cudaError_t launch_forcing(const ForcingParams& p, const double* fq, double* F, cudaStream_t st);

// all levels below the finest in one persistent launch (k_mg_persist.cu); levels[nl-1] is
// the coarsest; bar: 2 zeroed unsigned (grid barrier); err: device error flag
template <typename T>
cudaError_t launch_mg_persist(const MGLevelDesc<T>* levels, int nl, int nu1, int nu2, unsigned* bar, int* err,
                              int nblocks, cudaStream_t st);
template <typename T>
int mg_persist_blocks(int n_sm);   // resident blocks per SM (at most 2; 0: not available)

// vector kernels
template <typename Ti, typename To>
cudaError_t launch_convert(long long n, const Ti* in, To* out, cudaStream_t st);
// out = (To) in, zero = 0
template <typename Ti, typename To>
cudaError_t launch_convert_zero(long long n, const Ti* in, To* out, To* zero, cudaStream_t st);
cudaError_t launch_scale(long long n, double a, const double* x, double* y, cudaStream_t st);
cudaError_t launch_multidot(long long n, int nvec, const double* V, long long ld, const double* w,
                            double* partial, int nblocks, cudaStream_t st);
cudaError_t launch_reduce_partials(int nvec, int nblocks, const double* partial, double* out,
                                   int accumulate, cudaStream_t st);
// y += sign * sum_i coef[i] V[i], coef on the device
cudaError_t launch_multiaxpy(long long n, int nvec, const double* V, long long ld,
                             const double* coef, double sign, double* y, cudaStream_t st);
// y = a * x where a = 1 / dev_scalar[0] (normalisation without a host round trip)
cudaError_t launch_scale_by_inverse(long long n, const double* dev_scalar, const double* x,
                                    double* y, cudaStream_t st);
cudaError_t launch_sqrt_inplace(double* v, cudaStream_t st);

int multidot_blocks(long long n);
// one CGS2 Arnoldi step in a cooperative launch (see k_vec.cu); bar: 2 zeroed unsigned
// a few float vectors zeroed in one launch
struct ZeroList {
  static constexpr int MAX = 8;
  float* p[MAX];
  long long n[MAX];
  int count;
};
cudaError_t launch_zero_many(const ZeroList& z, cudaStream_t st);

// reg: take the register-resident form where it fits (nv <= 16, at most 2048 rows per block).
// vnext32, zero32 (optional): the register form also writes (float) vnext and zeroes
// zero32; *wrote32 says whether it did
cudaError_t launch_cgs2(long long n, int nv, const double* V, long long ld, double* w, double* partial, double* hcol,
                        double* vnext, float* vnext32, float* zero32, bool* wrote32, unsigned* bar, int* err,
                        int nblocks, bool reg, cudaStream_t st);
int cgs2_blocks(int n_sm);       // co-resident blocks to launch (0: not available)
int cgs2_max_vectors();
int cgs2_scratch(int nblocks);   // doubles of partial-sum scratch for nblocks

// cell tensors (k_cells.cu)
// cells[c * ld + offset + ch]; ld = C, offset = 0 for a plain [n_cells][C] tensor
cudaError_t launch_cells_gather(const CellsParams& p, const double* x, const double* base, const float* inv_scale,
                                float* cells, long long ld, int offset, cudaStream_t st);
cudaError_t launch_cells_scatter_add(const CellsParams& p, const float* cells, const float* scale, double* x,
                                     cudaStream_t st);
cudaError_t launch_cells_gather_adjoint(const CellsParams& p, const double* x, const float* scale, float* cells,
                                        cudaStream_t st);
cudaError_t launch_extrapolate(const CellsParams& p, const double* xp, double* xn, cudaStream_t st);
// x[g] = b[g] on every boundary velocity dof g
cudaError_t launch_copy_boundary(const CellsParams& p, const double* b, double* x, cudaStream_t st);
// out[0] = sum x_i y_i (deterministic: per-block partials, then a fixed-order sum); partial:
// scratch of at least dot_blocks() doubles
cudaError_t launch_dot(long long n, const double* x, const double* y, double* partial, double* out, cudaStream_t st);
int dot_blocks();
cudaError_t launch_remove_pressure_mean(const CellsParams& p, double* x, cudaStream_t st);

}  // namespace stmg
