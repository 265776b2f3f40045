// Matrix-free slab operator on 2D levels, node-centred form (Sec. 4.5, Eq. InAlg / DefDtauh).
//
// On the uniform mesh the assembled 1D matrices M_G and K_G (Gauss-Lobatto Lagrange basis
// of Q_{r+1}, G = (r+1) n + 1 nodes per direction) are banded: the row of a node interior
// to cell c holds row i of the element matrix (M1 or K1) over the NP = r+2 nodes of c, the
// row of a vertex between cells c-1 and c holds the last row of c-1's and the first row of
// c's element matrix.  The velocity block of S is a sum of Kronecker products of these
// matrices, applied here as two 1D passes ("stencils") over a tile of nodes:
//   y-pass:  A2_b = M_y u_b,  KU_b = K_y u_b                       (every temporal dof b)
//            A1_a = h^d sum_b K_tau[a,b] A2_b + beta_a KU_a           (time combination)
//   x-pass:  Y_a  = M_x A1_a + beta_a K_x A2_a - M_tau[a] h (B^T p_a)
// i.e. Y_a = h^d (M (x) M) sum_b K_tau[a,b] u_b + beta_a (M (x) K + K (x) M) u_a - ...,
// with beta_a = M_tau[a] nu h^(d-2).  The pressure gradient at a node sums, over the (up
// to four) cells holding it, the tensor-product factors (G1 or N1 per direction) of the
// Legendre modes times the cell's pressure; the continuity rows of a cell sum the same
// factors over the cell's nodes.
//
// One thread block owns a tile of tcx x tcy cells and writes every output entry of that
// tile exactly once: the velocity rows of the nodes [cx0 (NP-1), (cx0+tcx)(NP-1)) in each
// direction (the last tile of a row also the closing boundary node) and the pressure rows
// of its cells.  It reads the nodes of the tile and of one cell layer below and to the
// left (the stencils of the tile's first vertex line reach into those cells).  No atomics,
// and no zero-fill of y before the launch.
//
// Boundary velocity dofs: their columns are identity columns (read as 0), their rows are
// identity rows: y = x (APPLY, APPLY_T), b - x (RESIDUAL), g = x (LIFT).  LIFT reads only
// the boundary values of x (no pressure) and returns b - S_{.,D} g on the other rows.
// APPLY_T transposes K_tau (M_h, A_h, M_tau are symmetric; the B blocks are each other's
// transposes).
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

namespace {

// (A_G w)(g): w holds the values of global nodes I0, I0+1, ... at w[(node - I0) * stride];
// A1 is the NP x NP element matrix (row-major) in shared memory; n cells per direction.
template <typename T, int NP>
__device__ __forceinline__ T stencil(const T* __restrict__ A1, const T* __restrict__ w, int stride, int g, int I0,
                                     int n) {
  constexpr int E = NP - 1;
  const int c = g / E, i = g - c * E;
  T s = 0;
  if (i != 0) {
    const T* row = A1 + i * NP;
    const T* v = w + (c * E - I0) * stride;
#pragma unroll
    for (int j = 0; j < NP; ++j) s += row[j] * v[j * stride];
  } else {
    if (c < n) {
      const T* v = w + (c * E - I0) * stride;
#pragma unroll
      for (int j = 0; j < NP; ++j) s += A1[j] * v[j * stride];
    }
    if (c > 0) {
      const T* row = A1 + (NP - 1) * NP;
      const T* v = w + ((c - 1) * E - I0) * stride;
#pragma unroll
      for (int j = 0; j < NP; ++j) s += row[j] * v[j * stride];
    }
  }
  return s;
}

}  // namespace

// shared memory of one block (T elements), see the carve-up in the kernel
template <typename T>
size_t apply2d_smem_bytes(int np, int kt, int npm, int tcx, int tcy) {
  const int E = np - 1;
  const size_t nix = (size_t)(tcx + 1) * E + 1, niy = (size_t)(tcy + 1) * E + 1, noy = (size_t)tcy * E + 1;
  const size_t tables = 2 * np * np + 2 * (size_t)npm * np * np + (size_t)kt * kt;
  const size_t u = (size_t)kt * niy * nix;
  const size_t a12 = 2 * (size_t)kt * noy * nix;
  const size_t pp = (size_t)kt * (tcx + 1) * (tcy + 1) * npm;
  const size_t yp = (size_t)kt * tcx * tcy * npm;
  return sizeof(T) * (tables + u + a12 + pp + yp);
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_apply2d(const ApplyParams<T> P, const T* __restrict__ x,
                                                 const T* __restrict__ b, T* __restrict__ y, int mode) {
  constexpr int E = NP - 1, NQ = NP * NP;
  const int kt = P.kt, npm = P.npm, n = P.n, G = P.G, tcx = P.tcx, tcy = P.tcy;
  const int ntx = (n + tcx - 1) / tcx;
  const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
  const int cx0 = bx * tcx, cy0 = by * tcy;
  const int ncx = min(tcx, n - cx0), ncy = min(tcy, n - cy0);
  if (ncx <= 0 || ncy <= 0) return;
  // output node ranges [O0, O1) and input node ranges [I0, I1] per direction
  const int OX0 = cx0 * E, OX1 = cx0 + ncx == n ? G : (cx0 + ncx) * E;
  const int OY0 = cy0 * E, OY1 = cy0 + ncy == n ? G : (cy0 + ncy) * E;
  const int IX0 = max(cx0 - 1, 0) * E, IX1 = (cx0 + ncx) * E;
  const int IY0 = max(cy0 - 1, 0) * E, IY1 = (cy0 + ncy) * E;
  const int NOX = OX1 - OX0, NOY = OY1 - OY0, NIX = IX1 - IX0 + 1, NIY = IY1 - IY0 + 1;
  const int PCX0 = max(cx0 - 1, 0), PCY0 = max(cy0 - 1, 0);        // first cell of the pressure tile
  const int NPX = cx0 + ncx - PCX0, NPY = cy0 + ncy - PCY0;
  const long long nvel = P.n_vel, nnod = P.n_nodes, poff = (long long)kt * P.n_vel;
  const bool res = mode == RESIDUAL || mode == LIFT;

  extern __shared__ __align__(16) unsigned char smraw[];
  T* sM = reinterpret_cast<T*>(smraw);        // [NP][NP]
  T* sK = sM + NQ;                            // [NP][NP]
  T* sCB = sK + NQ;                           // [2][npm][NQ]: Fx(mode, ix) Fy(mode, iy), per component
  T* sKt = sCB + 2 * npm * NQ;                // [kt][kt] (transposed for APPLY_T)
  T* U = sKt + kt * kt;                       // [kt][NIY][NIX]  one velocity component
  const int sizeA = kt * NOY * NIX;
  T* A1 = U + kt * NIY * NIX;                 // [kt][NOY][NIX]
  T* A2 = A1 + sizeA;                         // [kt][NOY][NIX]
  T* PP = A2 + sizeA;                         // [kt][NPY * NPX][npm]
  T* YP = PP + kt * NPY * NPX * npm;          // [kt][ncy * ncx][npm]

  const int tid = threadIdx.x, bd = blockDim.x;
  for (int e = tid; e < NQ; e += bd) { sM[e] = P.M1[e]; sK[e] = P.K1[e]; }
  for (int e = tid; e < 2 * npm * NQ; e += bd) {
    const int comp = e / (npm * NQ), t = e - comp * npm * NQ, m = t / NQ, q = t - m * NQ;
    const int ix = q % NP, iy = q / NP;
    const T* Fx = comp == 0 ? P.G1 : P.N1;
    const T* Fy = comp == 1 ? P.G1 : P.N1;
    sCB[e] = Fx[P.modes[m][0] * NP + ix] * Fy[P.modes[m][1] * NP + iy];
  }
  for (int e = tid; e < kt * kt; e += bd) {
    const int a = e / kt, bb = e - a * kt;
    sKt[e] = mode == APPLY_T ? P.Kt[bb * MAXKT + a] : P.Kt[a * MAXKT + bb];
  }
  for (int e = tid; e < kt * NPY * NPX * npm; e += bd) {
    const int m = e % npm, t = e / npm, cl = t % (NPY * NPX), a = t / (NPY * NPX);
    const int cx = PCX0 + cl % NPX, cy = PCY0 + cl / NPX;
    PP[e] = mode == LIFT ? T(0) : x[poff + a * P.n_pres + ((long long)cy * n + cx) * npm + m];
  }
  for (int e = tid; e < kt * ncy * ncx * npm; e += bd) YP[e] = 0;

  for (int comp = 0; comp < 2; ++comp) {
    __syncthreads();        // tables ready / the previous component's passes are done with U, A1, A2
    // ---- gather the component's nodes (identity columns of the boundary read as 0)
    for (int e = tid; e < NIY * NIX; e += bd) {
      const int ly = e / NIX, lx = e - ly * NIX;
      const int gx = IX0 + lx, gy = IY0 + ly;
      const bool dir = gx == 0 || gx == G - 1 || gy == 0 || gy == G - 1;
      const bool take = mode == LIFT ? dir : !dir;
      const long long g = comp * nnod + (long long)gy * G + gx;
      for (int bb = 0; bb < kt; ++bb) U[bb * NIY * NIX + e] = take ? x[bb * nvel + g] : T(0);
    }
    __syncthreads();
    // ---- continuity rows of the tile's cells: YP[a][cell][m] += sum_nodes CB(m, node) u_a(node)
    for (int e = tid; e < kt * ncy * ncx * npm; e += bd) {
      const int m = e % npm, t = e / npm, cl = t % (ncy * ncx), a = t / (ncy * ncx);
      const int cx = cx0 + cl % ncx, cy = cy0 + cl / ncx;
      const T* u = U + a * NIY * NIX + (cy * E - IY0) * NIX + (cx * E - IX0);
      const T* cb = sCB + (comp * npm + m) * NQ;
      T s = 0;
#pragma unroll
      for (int iy = 0; iy < NP; ++iy)
#pragma unroll
        for (int ix = 0; ix < NP; ++ix) s += cb[iy * NP + ix] * u[iy * NIX + ix];
      YP[e] += s;
    }
    // ---- y-pass on the output rows, over all input columns
    for (int e = tid; e < NOY * NIX; e += bd) {
      const int oy = e / NIX, lx = e - oy * NIX;
      const int gy = OY0 + oy;
      T m2[MAXKT], k2[MAXKT];
#pragma unroll
      for (int bb = 0; bb < MAXKT; ++bb) {
        m2[bb] = 0; k2[bb] = 0;
        if (bb < kt) {
          const T* col = U + bb * NIY * NIX + lx;
          m2[bb] = stencil<T, NP>(sM, col, NIX, gy, IY0, n);
          k2[bb] = stencil<T, NP>(sK, col, NIX, gy, IY0, n);
        }
      }
#pragma unroll
      for (int a = 0; a < MAXKT; ++a) {
        if (a < kt) {
          T t = 0;
#pragma unroll
          for (int bb = 0; bb < MAXKT; ++bb)
            if (bb < kt) t += sKt[a * kt + bb] * m2[bb];
          A1[a * NOY * NIX + e] = P.hd * t + P.beta[a] * k2[a];
          A2[a * NOY * NIX + e] = m2[a];
        }
      }
    }
    __syncthreads();
    // ---- x-pass, pressure gradient, boundary rows; every output written once
    for (int e = tid; e < kt * NOY * NOX; e += bd) {
      const int t = e / NOX, ox = e - t * NOX, a = t / NOY, oy = t - a * NOY;
      const int gx = OX0 + ox, gy = OY0 + oy;
      const long long gi = a * nvel + comp * nnod + (long long)gy * G + gx;
      const bool dir = gx == 0 || gx == G - 1 || gy == 0 || gy == G - 1;
      if (dir) {
        y[gi] = mode == RESIDUAL ? b[gi] - x[gi] : x[gi];
        continue;
      }
      const T* r1 = A1 + (a * NOY + oy) * NIX;
      const T* r2 = A2 + (a * NOY + oy) * NIX;
      T v = stencil<T, NP>(sM, r1, 1, gx, IX0, n) + P.beta[a] * stencil<T, NP>(sK, r2, 1, gx, IX0, n);
      // pressure gradient: the cells holding node (gx, gy)
      const int cxa = gx / E, ixa = gx - cxa * E, cya = gy / E, iya = gy - cya * E;
      T bt = 0;
#pragma unroll
      for (int sy = 0; sy < 2; ++sy) {
        const int cy = cya - sy, iy = sy ? E : iya;
        if ((sy == 1 && iya != 0) || cy < 0 || cy >= n) continue;
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const int cx = cxa - sx, ix = sx ? E : ixa;
          if ((sx == 1 && ixa != 0) || cx < 0 || cx >= n) continue;
          const T* p = PP + (a * NPY * NPX + (cy - PCY0) * NPX + (cx - PCX0)) * npm;
          const T* cb = sCB + comp * npm * NQ + iy * NP + ix;
          for (int m = 0; m < npm; ++m) bt += cb[m * NQ] * p[m];
        }
      }
      v += P.bscale[a] * bt;
      y[gi] = res ? b[gi] - v : v;
    }
  }
  __syncthreads();
  // ---- pressure rows
  for (int e = tid; e < kt * ncy * ncx * npm; e += bd) {
    const int m = e % npm, t = e / npm, cl = t % (ncy * ncx), a = t / (ncy * ncx);
    const int cx = cx0 + cl % ncx, cy = cy0 + cl / ncx;
    const long long gi = poff + a * P.n_pres + ((long long)cy * n + cx) * npm + m;
    const T v = P.bscale[a] * YP[e];
    y[gi] = res ? b[gi] - v : v;
  }
}

template <typename T, int NP>
static cudaError_t launch_apply2d_t(const ApplyParams<T>& p, const T* x, const T* b, T* y, int mode,
                                    cudaStream_t st) {
  const size_t smem = apply2d_smem_bytes<T>(NP, p.kt, p.npm, p.tcx, p.tcy);
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_apply2d<T, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int ntx = (p.n + p.tcx - 1) / p.tcx, nty = (p.n + p.tcy - 1) / p.tcy;
  const int E = NP - 1;
  const int items = (p.tcy * E + 1) * ((p.tcx + 1) * E + 1);
  int threads = ((items + 31) / 32) * 32;
  threads = threads < 64 ? 64 : (threads > 256 ? 256 : threads);
  k_apply2d<T, NP><<<ntx * nty, threads, smem, st>>>(p, x, b, y, mode);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply2d(int np, const ApplyParams<T>& p, const T* x, const T* b, T* y, int mode,
                           cudaStream_t st) {
  if (p.tcx < 1 || p.tcy < 1) return cudaErrorInvalidValue;
  switch (np) {
    case 3: return launch_apply2d_t<T, 3>(p, x, b, y, mode, st);
    case 4: return launch_apply2d_t<T, 4>(p, x, b, y, mode, st);
    case 5: return launch_apply2d_t<T, 5>(p, x, b, y, mode, st);
    case 6: return launch_apply2d_t<T, 6>(p, x, b, y, mode, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_apply2d<double>(int, const ApplyParams<double>&, const double*, const double*, double*,
                                            int, cudaStream_t);
template cudaError_t launch_apply2d<float>(int, const ApplyParams<float>&, const float*, const float*, float*, int,
                                           cudaStream_t);
template size_t apply2d_smem_bytes<double>(int, int, int, int, int);
template size_t apply2d_smem_bytes<float>(int, int, int, int, int);

}  // namespace stmg
