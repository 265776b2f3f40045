// Internal launchers of the learned-initial-guess network (k_net.cu).
#pragma once

#include <cuda_runtime.h>

namespace stmg {

// out[b][y][x][o] = act(bias[o] + sum W[o][ky][kx][c] in[index[b]][y+ky-1][x+kx-1][c]);
// bias, mask and index may be NULL; mask zeroes outputs where mask <= 0 (same shape as out);
// accumulate adds the result to out instead of overwriting it.
cudaError_t launch_conv3x3(const float* in, const int* index, const float* Wm, const float* bias, const float* mask,
                           float* out, int B, int H, int W, int Cin, int Cout, int relu, int accumulate,
                           cudaStream_t st);
// Wt[c][tap][o] = W[o][8 - tap][c]
cudaError_t launch_flip_transpose(const float* Wm, float* Wt, int Cin, int Cout, cudaStream_t st);
// dW (Cout x 9 Cin) and db (Cout, may be NULL) of sum G * conv(in); part: scratch of part_cap floats
cudaError_t launch_conv3x3_grads(const float* in, const int* index, const float* G, float* dW, float* db, int B,
                                 int H, int W, int Cin, int Cout, float* part, long long part_cap, cudaStream_t st);
cudaError_t launch_mse(const float* pred, const float* target, const int* index, long long per_sample, int batch,
                       float* grad, double* part, double* loss, cudaStream_t st);
int mse_partials();
cudaError_t launch_adam(long long n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st);
cudaError_t launch_channel_rms(long long rows, int C, const float* data, float* rms, float* inv, cudaStream_t st);
cudaError_t launch_tensor_rms(long long n, const float* data, float* rms, float* inv, cudaStream_t st);
cudaError_t launch_scale_channels(long long rows, int C, float* d, const float* s, cudaStream_t st);

}  // namespace stmg
