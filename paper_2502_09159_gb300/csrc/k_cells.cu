// Cell tensors of slab vectors and the temporal extrapolation (learned initial guess).
//
// A cell tensor holds, per cell, every slab entry that belongs to the cell: the velocity
// values at its (r+2)^d nodes for each temporal dof and component, then its pressure
// modes for each temporal dof.  The gather copies shared nodes into every cell; the
// scatter averages the copies back, summing in increasing cell order (deterministic).
#include <cuda_runtime.h>

#include "internal.h"

namespace stmg {

static unsigned grid_of(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  const long long cap = 152LL * 32;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

__global__ void k_cells_gather(CellsParams p, const double* __restrict__ x, const double* __restrict__ base,
                               const float* __restrict__ inv_scale, float* __restrict__ cells, long long ld,
                               int offset) {
  const long long total = p.n_cells * p.C;
  const int nvch = p.kt * p.dim * p.Pn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / p.C;
    const int ch = (int)(e - c * p.C);
    long long g;
    if (ch < nvch) {
      const int a = ch / (p.dim * p.Pn);
      const int rem = ch - a * p.dim * p.Pn;
      const int comp = rem / p.Pn, node = rem - comp * p.Pn;
      const int lx = node % p.np, ly = (node / p.np) % p.np, lz = node / (p.np * p.np);
      const long long cx = c % p.n, cy = (c / p.n) % p.n, cz = c / ((long long)p.n * p.n);
      const long long gx = cx * p.r1 + lx, gy = cy * p.r1 + ly, gz = cz * p.r1 + lz;
      const long long gi = p.dim == 2 ? gx + p.G * gy : gx + p.G * (gy + p.G * gz);
      g = a * p.nv + comp * p.n_nodes + gi;
    } else {
      const int j = ch - nvch;
      const int a = j / p.npm, m = j - a * p.npm;
      g = p.kt * p.nv + a * p.npr + c * p.npm + m;
    }
    double v = x[g] - (base ? base[g] : 0.0);
    if (inv_scale) v *= (double)inv_scale[ch];
    cells[c * ld + offset + ch] = (float)v;
  }
}

cudaError_t launch_cells_gather(const CellsParams& p, const double* x, const double* base, const float* inv_scale,
                                float* cells, long long ld, int offset, cudaStream_t st) {
  k_cells_gather<<<grid_of(p.n_cells * p.C, 256), 256, 0, st>>>(p, x, base, inv_scale, cells, ld, offset);
  return cudaGetLastError();
}

// Cells containing global node index i along one direction, with the local index there:
// a node on a cell boundary belongs to the cell below (local r+1) and the one above
// (local 0), interior boundaries only.
__device__ __forceinline__ int cells_of_node(int i, int r1, int n, int* cell, int* loc) {
  const int q = i / r1, rm = i - q * r1;
  if (rm != 0) { cell[0] = q; loc[0] = rm; return 1; }
  int cnt = 0;
  if (q - 1 >= 0) { cell[cnt] = q - 1; loc[cnt] = r1; ++cnt; }
  if (q < n) { cell[cnt] = q; loc[cnt] = 0; ++cnt; }
  return cnt;
}

__global__ void k_cells_scatter_add(CellsParams p, const float* __restrict__ cells, const float* __restrict__ scale,
                                    double* __restrict__ x) {
  const long long vel = p.kt * p.nv;
  const int nvch = p.kt * p.dim * p.Pn;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < p.size;
       g += (long long)gridDim.x * blockDim.x) {
    if (g < vel) {
      const int a = (int)(g / p.nv);
      const long long rem = g - a * p.nv;
      const int comp = (int)(rem / p.n_nodes);
      const long long node = rem - comp * p.n_nodes;
      const int ix = (int)(node % p.G), iy = (int)((node / p.G) % p.G);
      const int iz = p.dim == 3 ? (int)(node / ((long long)p.G * p.G)) : 0;
      const int last = p.G - 1;
      if (ix == 0 || ix == last || iy == 0 || iy == last || (p.dim == 3 && (iz == 0 || iz == last))) continue;
      int cx[2], lx[2], cy[2], ly[2], cz[2] = {0, 0}, lz[2] = {0, 0};
      const int nx = cells_of_node(ix, p.r1, p.n, cx, lx);
      const int ny = cells_of_node(iy, p.r1, p.n, cy, ly);
      const int nz = p.dim == 3 ? cells_of_node(iz, p.r1, p.n, cz, lz) : 1;
      const int chb = (a * p.dim + comp) * p.Pn;
      double acc = 0.0;
      for (int zz = 0; zz < nz; ++zz)
        for (int yy = 0; yy < ny; ++yy)
          for (int xx = 0; xx < nx; ++xx) {
            const long long c = cx[xx] + (long long)p.n * (cy[yy] + (long long)p.n * cz[zz]);
            const int ch = chb + lx[xx] + p.np * (ly[yy] + p.np * lz[zz]);
            const double v = (double)cells[c * p.C + ch];
            acc = __dadd_rn(acc, scale ? __dmul_rn((double)scale[ch], v) : v);
          }
      x[g] += acc / (double)(nx * ny * nz);
    } else {
      const long long j = g - vel;
      const int a = (int)(j / p.npr);
      const long long rem = j - a * p.npr;
      const long long c = rem / p.npm;
      const int m = (int)(rem - c * p.npm);
      const int ch = nvch + a * p.npm + m;
      const double v = (double)cells[c * p.C + ch];
      x[g] += scale ? __dmul_rn((double)scale[ch], v) : v;
    }
  }
}

cudaError_t launch_cells_scatter_add(const CellsParams& p, const float* cells, const float* scale, double* x,
                                     cudaStream_t st) {
  k_cells_scatter_add<<<grid_of(p.size, 256), 256, 0, st>>>(p, cells, scale, x);
  return cudaGetLastError();
}

// Adjoint of the averaging scatter: every copy of a velocity dof g receives
// scale[ch] x[g] / (number of copies of g); boundary dofs give 0 (the scatter leaves them).
__global__ void k_cells_gather_adjoint(CellsParams p, const double* __restrict__ x, const float* __restrict__ scale,
                                       float* __restrict__ cells) {
  const long long total = p.n_cells * p.C;
  const int nvch = p.kt * p.dim * p.Pn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / p.C;
    const int ch = (int)(e - c * p.C);
    double v;
    if (ch < nvch) {
      const int a = ch / (p.dim * p.Pn);
      const int rem = ch - a * p.dim * p.Pn;
      const int comp = rem / p.Pn, node = rem - comp * p.Pn;
      const int lx = node % p.np, ly = (node / p.np) % p.np, lz = node / (p.np * p.np);
      const long long cx = c % p.n, cy = (c / p.n) % p.n, cz = c / ((long long)p.n * p.n);
      const long long gx = cx * p.r1 + lx, gy = cy * p.r1 + ly, gz = cz * p.r1 + lz;
      const long long last = p.G - 1;
      const bool dir = gx == 0 || gx == last || gy == 0 || gy == last || (p.dim == 3 && (gz == 0 || gz == last));
      // copies along one direction: 2 on an interior cell boundary, else 1
      auto copies = [&](long long gi, int li) { return (li == 0 || li == p.np - 1) && gi > 0 && gi < last ? 2 : 1; };
      int cnt = copies(gx, lx) * copies(gy, ly);
      if (p.dim == 3) cnt *= copies(gz, lz);
      const long long gi = p.dim == 2 ? gx + p.G * gy : gx + p.G * (gy + p.G * gz);
      v = dir ? 0.0 : x[a * p.nv + comp * p.n_nodes + gi] / (double)cnt;
    } else {
      const int j = ch - nvch;
      const int a = j / p.npm, m = j - a * p.npm;
      v = x[p.kt * p.nv + a * p.npr + c * p.npm + m];
    }
    if (scale) v *= (double)scale[ch];
    cells[e] = (float)v;
  }
}

cudaError_t launch_cells_gather_adjoint(const CellsParams& p, const double* x, const float* scale, float* cells,
                                        cudaStream_t st) {
  k_cells_gather_adjoint<<<grid_of(p.n_cells * p.C, 256), 256, 0, st>>>(p, x, scale, cells);
  return cudaGetLastError();
}

__global__ void k_copy_boundary(CellsParams p, const double* __restrict__ b, double* __restrict__ x) {
  const long long vel = p.kt * p.nv;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < vel; g += (long long)gridDim.x * blockDim.x) {
    const long long node = (g % p.nv) % p.n_nodes;
    const int ix = (int)(node % p.G), iy = (int)((node / p.G) % p.G);
    const int iz = p.dim == 3 ? (int)(node / ((long long)p.G * p.G)) : 0;
    const int last = p.G - 1;
    if (ix == 0 || ix == last || iy == 0 || iy == last || (p.dim == 3 && (iz == 0 || iz == last))) x[g] = b[g];
  }
}

cudaError_t launch_copy_boundary(const CellsParams& p, const double* b, double* x, cudaStream_t st) {
  k_copy_boundary<<<grid_of(p.kt * p.nv, 256), 256, 0, st>>>(p, b, x);
  return cudaGetLastError();
}

constexpr int DOT_BLOCKS = 304;

__global__ void __launch_bounds__(256) k_dot(long long n, const double* __restrict__ x, const double* __restrict__ y,
                                             double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_dot_finish(const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < DOT_BLOCKS; ++i) s += partial[i];
    out[0] = s;
  }
}

int dot_blocks() { return DOT_BLOCKS; }

cudaError_t launch_dot(long long n, const double* x, const double* y, double* partial, double* out, cudaStream_t st) {
  k_dot<<<DOT_BLOCKS, 256, 0, st>>>(n, x, y, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dot_finish<<<1, 32, 0, st>>>(partial, out);
  return cudaGetLastError();
}

__global__ void k_extrapolate(CellsParams p, const double* __restrict__ xp, double* __restrict__ xn) {
  const long long tot = p.nv + p.npr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const bool v = i < p.nv;
    const long long blk = v ? p.nv : p.npr;
    const long long off = v ? 0 : p.kt * p.nv;
    const long long j = v ? i : i - p.nv;
    double u[MAXKT];
    for (int b = 0; b < p.kt; ++b) u[b] = xp[off + b * blk + j];
    for (int a = 0; a < p.kt; ++a) {
      double s = 0.0;
      for (int b = 0; b < p.kt; ++b) s += p.E[a * p.kt + b] * u[b];
      xn[off + a * blk + j] = s;
    }
  }
}

cudaError_t launch_extrapolate(const CellsParams& p, const double* xp, double* xn, cudaStream_t st) {
  k_extrapolate<<<grid_of(p.nv + p.npr, 256), 256, 0, st>>>(p, xp, xn);
  return cudaGetLastError();
}

// one block per temporal dof: mean of the mode-0 coefficients, then subtract it
__global__ void __launch_bounds__(1024) k_remove_pmean(CellsParams p, double* __restrict__ x) {
  __shared__ double red[1024];
  double* P = x + p.kt * p.nv + blockIdx.x * p.npr;
  double s = 0.0;
  for (long long c = threadIdx.x; c < p.n_cells; c += blockDim.x) s += P[c * p.npm];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  const double mean = red[0] / (double)p.n_cells;
  for (long long c = threadIdx.x; c < p.n_cells; c += blockDim.x) P[c * p.npm] -= mean;
}

cudaError_t launch_remove_pressure_mean(const CellsParams& p, double* x, cudaStream_t st) {
  k_remove_pmean<<<p.kt, 1024, 0, st>>>(p, x);
  return cudaGetLastError();
}

}  // namespace stmg
