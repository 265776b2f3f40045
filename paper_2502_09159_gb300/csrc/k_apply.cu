// Matrix-free space-time Stokes slab operator (Sec. 4.5, Eq. InAlg / DefDtauh).
//
// One thread block handles `cpb` consecutive cells.  Per cell and temporal dof a it
//   * gathers the velocity nodes (boundary nodes read as 0: identity columns) and the
//     pressure modes into shared memory,
//   * forms u~_a = sum_b K_tau[a,b] u_b (the time combination, Sec. 4.5),
//   * applies h^d (M1 (x) M1 (x) M1) u~_a + beta_a sum_dir (K1 in dir, M1 elsewhere) u_a by
//     sum factorisation, one thread per 1D line, 1D matrices from the parameter bank,
//   * adds the pressure gradient -M_tau[a] B^T p_a and forms the continuity rows
//     -M_tau[a] B u_a with the tensor-product 1D factors of the Legendre basis,
//   * scatter-adds the velocity rows (atomics; cells share nodes) and stores the
//     cell-local pressure rows.
// Boundary rows are the identity: the owner cell of each boundary node adds +x (apply)
// or b - x (residual).  The LIFT mode moves non-homogeneous boundary data to the right-
// hand side: y = b - S_{.,D} g on the interior rows (only the boundary values of g are
// read) and y = g on the boundary rows.  APPLY_T applies S^T: M_h, A_h and M_tau are
// symmetric and the two B blocks are each other's transposes, so S^T is S with the
// temporal matrix K_tau transposed.  On axis-aligned uniform cells every element operator is a sum
// of Kronecker products of the 1D matrices M1 = int ell ell, K1 = int ell' ell',
// G1 = int L ell', N1 = int L ell on [0,1]; the kernel applies those factors directly.
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

namespace {

template <int DIM, int NP>
struct Shape {
  static constexpr int NQ = DIM == 2 ? NP * NP : NP * NP * NP;
  static constexpr int NL = NQ / NP;
};

template <typename T, int DIM, int NP>
__device__ __forceinline__ void cell_coords(int c, int n, int* cc) {
  cc[0] = c % n;
  cc[1] = (c / n) % n;
  cc[2] = DIM == 3 ? c / (n * n) : 0;
}

}  // namespace

template <typename T, int DIM, int NP>
__global__ void __launch_bounds__(256) k_apply(const ApplyParams<T> P, const T* __restrict__ x,
                                               const T* __restrict__ b, T* __restrict__ y,
                                               int mode) {
  using S = Shape<DIM, NP>;
  constexpr int NQ = S::NQ, NL = S::NL;
  // pressure modes per cell, C(r + d, d) with r = NP - 2; the host checks that P.npm and
  // its mode table agree with this count and with mode_exp's order
  constexpr int NPM = DIM == 2 ? NP * (NP - 1) / 2 : (NP + 1) * NP * (NP - 1) / 6;
  const int kt = P.kt, npm = P.npm, n = P.n, G = P.G;
  const int ncells = DIM == 2 ? n * n : n * n * n;
  const int c0 = blockIdx.x * P.cpb;
  const int nc = min(P.cpb, ncells - c0);
  if (nc <= 0) return;
  const int VS = kt * DIM * NQ;          // velocity values of one cell
  const int cs = P.cpb * VS;             // stride between buffers
  extern __shared__ __align__(16) unsigned char smraw[];
  T* U = reinterpret_cast<T*>(smraw);    // gathered velocity           [cell][a][comp][node]
  T* UT = U + cs;                        // time-combined velocity
  T* A1 = UT + cs;                       // sum-factorisation temporaries
  T* A2 = A1 + cs;
  T* A3 = DIM == 3 ? A2 + cs : A2;
  T* YV = (DIM == 3 ? A3 : A2) + cs;     // velocity result
  T* PIN = YV + cs;                      // gathered pressure           [cell][a][m]
  T* YP = PIN + P.cpb * kt * npm;        // pressure result

  const long long nvel = P.n_vel, nnod = P.n_nodes;
  const long long poff = (long long)kt * nvel;

  // ---- gather ------------------------------------------------------------------------
  {
    const int tot = nc * VS;
    for (int w = threadIdx.x; w < tot; w += blockDim.x) {
      int t = w;
      const int ix = t % NP; t /= NP;
      const int cl = t % nc; t /= nc;
      const int iy = t % NP; t /= NP;
      int iz = 0;
      if (DIM == 3) { iz = t % NP; t /= NP; }
      const int comp = t % DIM;
      const int a = t / DIM;
      int cc[3];
      cell_coords<T, DIM, NP>(c0 + cl, n, cc);
      const int gx = cc[0] * (NP - 1) + ix, gy = cc[1] * (NP - 1) + iy, gz = cc[2] * (NP - 1) + iz;
      bool dir = gx == 0 || gx == G - 1 || gy == 0 || gy == G - 1;
      if (DIM == 3) dir = dir || gz == 0 || gz == G - 1;
      const long long g = gx + (long long)G * (gy + (long long)G * gz);
      const int node = ix + NP * (iy + NP * iz);
      // LIFT reads only the boundary values (the columns S_{.,D}); the other modes only
      // the interior ones (boundary columns are identity columns)
      const bool take = mode == LIFT ? dir : !dir;
      U[cl * VS + (a * DIM + comp) * NQ + node] = take ? x[a * nvel + comp * nnod + g] : T(0);
    }
    const int totp = nc * kt * npm;
    for (int w = threadIdx.x; w < totp; w += blockDim.x) {
      const int m = w % npm, t = w / npm, a = t % kt, cl = t / kt;
      PIN[(cl * kt + a) * npm + m] = mode == LIFT ? T(0) : x[poff + a * P.n_pres + (long long)(c0 + cl) * npm + m];
    }
  }
  __syncthreads();

  // ---- time combination u~_a = sum_b K[a,b] u_b and continuity rows -------------------
  {
    const int tot = nc * VS;
    for (int w = threadIdx.x; w < tot; w += blockDim.x) {
      const int node_comp = w % (DIM * NQ);
      const int t = w / (DIM * NQ);
      const int a = t % kt, cl = t / kt;
      const T* u = U + cl * VS + node_comp;
      T s = 0;
      const bool tr = mode == APPLY_T;         // S^T: the temporal matrix transposed
      for (int bb = 0; bb < kt; ++bb) s += P.Kt[tr ? bb * MAXKT + a : a * MAXKT + bb] * u[bb * DIM * NQ];
      UT[cl * VS + a * DIM * NQ + node_comp] = s;
    }
    const int totp = nc * kt * npm;
    for (int w = threadIdx.x; w < totp; w += blockDim.x) {
      const int m = w % npm, t = w / npm, a = t % kt, cl = t / kt;
      const int ex = P.modes[m][0], ey = P.modes[m][1], ez = P.modes[m][2];
      T s = 0;
      for (int comp = 0; comp < DIM; ++comp) {
        const T* u = U + cl * VS + (a * DIM + comp) * NQ;
        const T* Fx = (comp == 0 ? P.G1 : P.N1) + ex * NP;
        const T* Fy = (comp == 1 ? P.G1 : P.N1) + ey * NP;
        const T* Fz = (comp == 2 ? P.G1 : P.N1) + ez * NP;
        for (int iz = 0; iz < (DIM == 3 ? NP : 1); ++iz) {
          const T fz = DIM == 3 ? Fz[iz] : T(1);
          for (int iy = 0; iy < NP; ++iy) {
            T row = 0;
#pragma unroll
            for (int ix = 0; ix < NP; ++ix) row += Fx[ix] * u[ix + NP * (iy + NP * iz)];
            s += fz * Fy[iy] * row;
          }
        }
      }
      YP[(cl * kt + a) * npm + m] = P.bscale[a] * s;
    }
  }
  __syncthreads();

  const int nlines = nc * kt * DIM * NL;
  if (DIM == 2) {
    // y-pass: A1 = h^d M1y u~ + beta K1y u,  A2 = M1y u
    for (int w = threadIdx.x; w < nlines; w += blockDim.x) {
      const int ix = w % NP, t = w / NP;           // t = (cl * kt + a) * DIM + comp
      const int a = (t / DIM) % kt;
      const int base = t * NQ + ix;
      T u[NP], ut[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) { u[j] = U[base + j * NP]; ut[j] = UT[base + j * NP]; }
      const T be = P.beta[a];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T m1 = 0, k1 = 0, m2 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          m1 += P.M1[i * NP + j] * ut[j];
          k1 += P.K1[i * NP + j] * u[j];
          m2 += P.M1[i * NP + j] * u[j];
        }
        A1[base + i * NP] = P.hd * m1 + be * k1;
        A2[base + i * NP] = m2;
      }
    }
    __syncthreads();
    // x-pass: YV = M1x A1 + beta K1x A2 - M_tau B^T p
    for (int w = threadIdx.x; w < nlines; w += blockDim.x) {
      const int iy = w % NP, t = w / NP;
      const int comp = t % DIM, a = (t / DIM) % kt, cl = t / (DIM * kt);
      const int base = t * NQ + iy * NP;
      T t1[NP], t2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) { t1[j] = A1[base + j]; t2[j] = A2[base + j]; }
      const T be = P.beta[a];
      const T* p = PIN + (cl * kt + a) * npm;
      const T* Fy = comp == 1 ? P.G1 : P.N1;
      const T* Fx = comp == 0 ? P.G1 : P.N1;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T m1 = 0, k1 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          m1 += P.M1[i * NP + j] * t1[j];
          k1 += P.K1[i * NP + j] * t2[j];
        }
        T bt = 0;
#pragma unroll
        for (int m = 0; m < NPM; ++m)
          bt += Fx[mode_exp(2, NP - 2, m, 0) * NP + i] * Fy[mode_exp(2, NP - 2, m, 1) * NP + iy] * p[m];
        YV[base + i] = m1 + be * k1 + P.bscale[a] * bt;
      }
    }
  } else {
    // z-pass: A1 = M1z u~, A2 = M1z u, A3 = K1z u
    constexpr int SZ = NP * NP;
    for (int w = threadIdx.x; w < nlines; w += blockDim.x) {
      const int l = w % NL, t = w / NL;            // l = ix + NP iy
      const int base = t * NQ + l;
      T u[NP], ut[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) { u[j] = U[base + j * SZ]; ut[j] = UT[base + j * SZ]; }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          a1 += P.M1[i * NP + j] * ut[j];
          a2 += P.M1[i * NP + j] * u[j];
          a3 += P.K1[i * NP + j] * u[j];
        }
        A1[base + i * SZ] = a1;
        A2[base + i * SZ] = a2;
        A3[base + i * SZ] = a3;
      }
    }
    __syncthreads();
    // y-pass: U <- h^d M1y A1 + beta (K1y A2 + M1y A3),  UT <- M1y A2
    for (int w = threadIdx.x; w < nlines; w += blockDim.x) {
      const int l = w % NL, t = w / NL;            // l = ix + NP iz
      const int a = (t / DIM) % kt;
      const int ix = l % NP, iz = l / NP;
      const int base = t * NQ + ix + iz * SZ;
      T a1[NP], a2[NP], a3[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) { a1[j] = A1[base + j * NP]; a2[j] = A2[base + j * NP]; a3[j] = A3[base + j * NP]; }
      const T be = P.beta[a];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T m1 = 0, k2 = 0, m3 = 0, m2 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          m1 += P.M1[i * NP + j] * a1[j];
          k2 += P.K1[i * NP + j] * a2[j];
          m3 += P.M1[i * NP + j] * a3[j];
          m2 += P.M1[i * NP + j] * a2[j];
        }
        U[base + i * NP] = P.hd * m1 + be * (k2 + m3);
        UT[base + i * NP] = m2;
      }
    }
    __syncthreads();
    // x-pass: YV = M1x U + beta K1x UT - M_tau B^T p
    for (int w = threadIdx.x; w < nlines; w += blockDim.x) {
      const int l = w % NL, t = w / NL;            // l = iy + NP iz
      const int comp = t % DIM, a = (t / DIM) % kt, cl = t / (DIM * kt);
      const int iy = l % NP, iz = l / NP;
      const int base = t * NQ + l * NP;
      T c1[NP], c2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) { c1[j] = U[base + j]; c2[j] = UT[base + j]; }
      const T be = P.beta[a];
      const T* p = PIN + (cl * kt + a) * npm;
      const T* Fx = comp == 0 ? P.G1 : P.N1;
      const T* Fy = comp == 1 ? P.G1 : P.N1;
      const T* Fz = comp == 2 ? P.G1 : P.N1;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T m1 = 0, k1 = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          m1 += P.M1[i * NP + j] * c1[j];
          k1 += P.K1[i * NP + j] * c2[j];
        }
        T bt = 0;
#pragma unroll
        for (int m = 0; m < NPM; ++m)
          bt += Fx[mode_exp(3, NP - 2, m, 0) * NP + i] * Fy[mode_exp(3, NP - 2, m, 1) * NP + iy] *
                Fz[mode_exp(3, NP - 2, m, 2) * NP + iz] * p[m];
        YV[base + i] = m1 + be * k1 + P.bscale[a] * bt;
      }
    }
  }
  __syncthreads();

  // ---- scatter -----------------------------------------------------------------------
  {
    const int tot = nc * VS;
    const bool res = mode == RESIDUAL || mode == LIFT;
    for (int w = threadIdx.x; w < tot; w += blockDim.x) {
      int t = w;
      const int ix = t % NP; t /= NP;
      const int cl = t % nc; t /= nc;
      const int iy = t % NP; t /= NP;
      int iz = 0;
      if (DIM == 3) { iz = t % NP; t /= NP; }
      const int comp = t % DIM;
      const int a = t / DIM;
      int cc[3];
      cell_coords<T, DIM, NP>(c0 + cl, n, cc);
      const int gx = cc[0] * (NP - 1) + ix, gy = cc[1] * (NP - 1) + iy, gz = cc[2] * (NP - 1) + iz;
      bool dir = gx == 0 || gx == G - 1 || gy == 0 || gy == G - 1;
      bool own = (ix < NP - 1 || cc[0] == n - 1) && (iy < NP - 1 || cc[1] == n - 1);
      if (DIM == 3) {
        dir = dir || gz == 0 || gz == G - 1;
        own = own && (iz < NP - 1 || cc[2] == n - 1);
      }
      const long long gi = a * nvel + comp * nnod + gx + (long long)G * (gy + (long long)G * gz);
      T add = 0;
      if (!dir) {
        const T v = YV[cl * VS + (a * DIM + comp) * NQ + ix + NP * (iy + NP * iz)];
        add = res ? -v : v;
      }
      if (own) {
        if (dir) add += mode == LIFT ? x[gi] : (res ? b[gi] - x[gi] : x[gi]);
        else if (res) add += b[gi];
      } else if (dir) {
        continue;
      }
      atomicAdd(y + gi, add);
    }
    const int totp = nc * kt * npm;
    for (int w = threadIdx.x; w < totp; w += blockDim.x) {
      const int m = w % npm, t = w / npm, a = t % kt, cl = t / kt;
      const long long gi = poff + a * P.n_pres + (long long)(c0 + cl) * npm + m;
      const T v = YP[(cl * kt + a) * npm + m];
      y[gi] = res ? b[gi] - v : v;
    }
  }
}

template <typename T>
size_t apply_smem_bytes(int dim, int np, int kt, int npm, int cpb) {
  const int nq = dim == 2 ? np * np : np * np * np;
  const int nbuf = dim == 2 ? 5 : 6;
  return sizeof(T) * ((size_t)cpb * kt * dim * nq * nbuf + 2 * (size_t)cpb * kt * npm);
}

template <typename T, int DIM, int NP>
static cudaError_t launch_apply_t(const ApplyParams<T>& p, const T* x, const T* b, T* y, int mode,
                                  cudaStream_t st) {
  const int ncells = DIM == 2 ? p.n * p.n : p.n * p.n * p.n;
  const size_t smem = apply_smem_bytes<T>(DIM, NP, p.kt, p.npm, p.cpb);
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_apply<T, DIM, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int lines = p.cpb * p.kt * DIM * (DIM == 2 ? NP : NP * NP);
  int threads = ((lines + 31) / 32) * 32;
  threads = threads < 64 ? 64 : (threads > 256 ? 256 : threads);
  const int blocks = (ncells + p.cpb - 1) / p.cpb;
  k_apply<T, DIM, NP><<<blocks, threads, smem, st>>>(p, x, b, y, mode);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(int dim, int np, const ApplyParams<T>& p, const T* x, const T* b, T* y, int mode,
                         cudaStream_t st) {
#define STMG_APPLY_CASE(D, N) \
  if (dim == D && np == N) return launch_apply_t<T, D, N>(p, x, b, y, mode, st);
  STMG_APPLY_CASE(2, 3) STMG_APPLY_CASE(2, 4) STMG_APPLY_CASE(2, 5) STMG_APPLY_CASE(2, 6)
  STMG_APPLY_CASE(3, 3) STMG_APPLY_CASE(3, 4) STMG_APPLY_CASE(3, 5) STMG_APPLY_CASE(3, 6)
#undef STMG_APPLY_CASE
  return cudaErrorInvalidValue;
}

template cudaError_t launch_apply<double>(int, int, const ApplyParams<double>&, const double*, const double*,
                                          double*, int, cudaStream_t);
template cudaError_t launch_apply<float>(int, int, const ApplyParams<float>&, const float*, const float*, float*,
                                         int, cudaStream_t);
template size_t apply_smem_bytes<double>(int, int, int, int, int);
template size_t apply_smem_bytes<float>(int, int, int, int, int);

// ------------------------------------------------------------------------------------
// Slab coupling (Eq. InAlg right-hand side): b^v_a += phi_a(t_{n-1}^+) M_h v_prev
// ------------------------------------------------------------------------------------
__global__ void k_mass_coupling(const MassParams P, const double* __restrict__ v, double* __restrict__ b) {
  const int dim = P.dim, np = P.np, n = P.n, G = P.G;
  const int nq = dim == 2 ? np * np : np * np * np;
  const int ncells = dim == 2 ? n * n : n * n * n;
  const int c = blockIdx.x;
  if (c >= ncells) return;
  __shared__ double U[3 * 216], W[3 * 216];
  int cc[3] = {c % n, (c / n) % n, dim == 3 ? c / (n * n) : 0};
  const int tot = dim * nq;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int node = w % nq, comp = w / nq;
    const int ix = node % np, iy = (node / np) % np, iz = dim == 3 ? node / (np * np) : 0;
    const int gx = cc[0] * (np - 1) + ix, gy = cc[1] * (np - 1) + iy, gz = cc[2] * (np - 1) + iz;
    const long long g = gx + (long long)G * (gy + (long long)G * gz);
    U[w] = v[comp * P.n_nodes + g];              // boundary values included (Eq. InAlg: full M_h)
  }
  __syncthreads();
  // W = h^d (M1 (x) M1 (x) M1) U, direct tensor contraction (small, setup-like cost)
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int node = w % nq, comp = w / nq;
    const int ix = node % np, iy = (node / np) % np, iz = dim == 3 ? node / (np * np) : 0;
    double s = 0.0;
    for (int jz = 0; jz < (dim == 3 ? np : 1); ++jz) {
      const double fz = dim == 3 ? P.M1[iz * np + jz] : 1.0;
      for (int jy = 0; jy < np; ++jy) {
        double row = 0.0;
        for (int jx = 0; jx < np; ++jx) row += P.M1[ix * np + jx] * U[comp * nq + jx + np * (jy + np * jz)];
        s += fz * P.M1[iy * np + jy] * row;
      }
    }
    W[w] = P.hd * s;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < tot * P.kt; w += blockDim.x) {
    const int a = w / tot, r = w % tot;
    const int node = r % nq, comp = r / nq;
    const int ix = node % np, iy = (node / np) % np, iz = dim == 3 ? node / (np * np) : 0;
    const int gx = cc[0] * (np - 1) + ix, gy = cc[1] * (np - 1) + iy, gz = cc[2] * (np - 1) + iz;
    bool dir = gx == 0 || gx == G - 1 || gy == 0 || gy == G - 1 || (dim == 3 && (gz == 0 || gz == G - 1));
    if (dir) continue;
    const long long g = gx + (long long)G * (gy + (long long)G * gz);
    atomicAdd(b + a * P.n_vel + comp * P.n_nodes + g, P.phi_left[a] * W[r]);
  }
}

cudaError_t launch_mass_coupling(const MassParams& p, const double* vprev, double* b, cudaStream_t st) {
  const int ncells = p.dim == 2 ? p.n * p.n : p.n * p.n * p.n;
  k_mass_coupling<<<ncells, 128, 0, st>>>(p, vprev, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Forcing (Eq. DefFn): F^a_i = tau/2 w_a sum_q w_q f(x_q, t^a) . chi_i(x_q)
// The quadrature weight times the 1D basis value, W1[p][q] = w_q ell_p(x_q), is staged in
// shared memory, and the tensor-product sum is factorised: along x, then y (then z).
// ------------------------------------------------------------------------------------
__global__ void k_forcing(const ForcingParams P, const double* __restrict__ fq, double* __restrict__ F) {
  const int dim = P.dim, np = P.np, n = P.n, G = P.G, nq = P.nq;
  const int nnode = dim == 2 ? np * np : np * np * np;
  const int nqc = dim == 2 ? nq * nq : nq * nq * nq;
  const int ncells = dim == 2 ? n * n : n * n * n;
  const int c = blockIdx.x;
  if (c >= ncells) return;
  __shared__ double W1[MAXNP * 10];
  for (int e = threadIdx.x; e < np * nq; e += blockDim.x) W1[e] = P.wq[e % nq] * P.phiq[e];
  __syncthreads();
  int cc[3] = {c % n, (c / n) % n, dim == 3 ? c / (n * n) : 0};
  const int tot = P.kt * dim * nnode;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    const int node = w % nnode, t = w / nnode, comp = t % dim, a = t / dim;
    const int ix = node % np, iy = (node / np) % np, iz = dim == 3 ? node / (np * np) : 0;
    const int gx = cc[0] * (np - 1) + ix, gy = cc[1] * (np - 1) + iy, gz = cc[2] * (np - 1) + iz;
    bool dir = gx == 0 || gx == G - 1 || gy == 0 || gy == G - 1 || (dim == 3 && (gz == 0 || gz == G - 1));
    if (dir) continue;
    const double* f = fq + ((long long)a * ncells + c) * nqc * dim;
    const double* wx = W1 + ix * nq;
    const double* wy = W1 + iy * nq;
    const double* wz = W1 + iz * nq;
    double s = 0.0;
    for (int qz = 0; qz < (dim == 3 ? nq : 1); ++qz) {
      double sy = 0.0;
      for (int qy = 0; qy < nq; ++qy) {
        const double* fr = f + ((long long)(qz * nq + qy) * nq) * dim + comp;
        double sx = 0.0;
        for (int qx = 0; qx < nq; ++qx) sx += wx[qx] * fr[qx * dim];
        sy += wy[qy] * sx;
      }
      s += (dim == 3 ? wz[qz] : 1.0) * sy;
    }
    const long long g = gx + (long long)G * (gy + (long long)G * gz);
    atomicAdd(F + a * P.n_vel + comp * P.n_nodes + g, P.scale[a] * s);
  }
}

cudaError_t launch_forcing(const ForcingParams& p, const double* fq, double* F, cudaStream_t st) {
  const int ncells = p.dim == 2 ? p.n * p.n : p.n * p.n * p.n;
  k_forcing<<<ncells, 128, 0, st>>>(p, fq, F);
  return cudaGetLastError();
}

}  // namespace stmg
