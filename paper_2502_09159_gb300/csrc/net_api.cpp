// C ABI of the learned-initial-guess network (include/stmg_net.h): buffers, parameter
// layout, the forward / backward sequence of layers and the training step.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "net_internal.h"
#include "stmg.h"
#include "stmg_net.h"

using namespace stmg;

struct stmg_net {
  int H = 0, W = 0, cin = 0, hid = 0, cout = 0, L = 0, maxb = 0, skip = 0;
  std::vector<int> ci, co;                  // channels in / out per layer
  std::vector<long long> woff, boff;        // offsets of W and bias in the flat vector
  long long soff = 0;                       // offset of the bypass weights (skip != 0)
  long long np = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  float* wt = nullptr;                      // flipped, transposed weights of one layer
  std::vector<float*> acts;                 // acts[l]: input of layer l (l >= 1)
  float* g[2] = {nullptr, nullptr};         // gradient ping-pong
  float *pred = nullptr, *gpred = nullptr;  // training step: prediction and its gradient
  float* part = nullptr;
  long long part_cap = 0;
  double* loss_part = nullptr;
  cudaStream_t st = nullptr;
  std::vector<void*> owned;
};

#define NCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      std::fprintf(stderr, "stmg_net: %s failed: %s\n", #call, cudaGetErrorString(e_));    \
      return e_ == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA;               \
    }                                                                                      \
  } while (0)

namespace {

int alloc(stmg_net* n, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA;
  n->owned.push_back(*p);
  return STMG_OK;
}

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based 64-bit generator
uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int init_params(stmg_net* n, uint64_t seed) {
  std::vector<float> h((size_t)n->np, 0.f);
  uint64_t s = seed;
  for (int l = 0; l + 1 < n->L; ++l) {       // last layer and bypass stay zero: a fresh network returns 0
    const double bound = std::sqrt(6.0 / (9.0 * n->ci[l]));
    const long long cnt = (long long)n->co[l] * 9 * n->ci[l];
    for (long long i = 0; i < cnt; ++i) {
      const double u = (double)(splitmix64(&s) >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
      h[(size_t)(n->woff[l] + i)] = (float)((2.0 * u - 1.0) * bound);
    }
  }
  NCK(cudaMemcpy(n->params, h.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice));
  NCK(cudaMemset(n->m, 0, sizeof(float) * n->np));
  NCK(cudaMemset(n->v, 0, sizeof(float) * n->np));
  NCK(cudaMemset(n->grads, 0, sizeof(float) * n->np));
  return STMG_OK;
}

const float* layer_in(const stmg_net* n, int l, const float* in) { return l == 0 ? in : n->acts[l]; }

int forward(stmg_net* n, int batch, const float* in, const int* index, float* out) {
  for (int l = 0; l < n->L; ++l) {
    const float* x = layer_in(n, l, in);
    float* y = l + 1 == n->L ? out : n->acts[l + 1];
    NCK(launch_conv3x3(x, l == 0 ? index : nullptr, n->params + n->woff[l], n->params + n->boff[l], nullptr, y,
                       batch, n->H, n->W, n->ci[l], n->co[l], l + 1 < n->L, 0, n->st));
  }
  if (n->skip)   // linear bypass from the input, added to the output
    NCK(launch_conv3x3(in, index, n->params + n->soff, nullptr, nullptr, out, batch, n->H, n->W, n->cin, n->cout, 0,
                       1, n->st));
  return STMG_OK;
}

int backward(stmg_net* n, int batch, const float* in, const int* index, const float* gout) {
  const float* G = gout;
  int cur = 0;
  if (n->skip)
    NCK(launch_conv3x3_grads(in, index, gout, n->grads + n->soff, nullptr, batch, n->H, n->W, n->cin, n->cout,
                             n->part, n->part_cap, n->st));
  for (int l = n->L - 1; l >= 0; --l) {
    const float* x = layer_in(n, l, in);
    NCK(launch_conv3x3_grads(x, l == 0 ? index : nullptr, G, n->grads + n->woff[l], n->grads + n->boff[l], batch,
                             n->H, n->W, n->ci[l], n->co[l], n->part, n->part_cap, n->st));
    if (l > 0) {
      // input gradient, masked by the ReLU that produced this layer's input
      NCK(launch_flip_transpose(n->params + n->woff[l], n->wt, n->ci[l], n->co[l], n->st));
      NCK(launch_conv3x3(G, nullptr, n->wt, nullptr, n->acts[l], n->g[cur], batch, n->H, n->W, n->co[l], n->ci[l], 0,
                         0, n->st));
      G = n->g[cur];
      cur ^= 1;
    }
  }
  return STMG_OK;
}

bool ok_batch(const stmg_net* n, int batch) { return n && batch >= 1 && batch <= n->maxb; }

}  // namespace

extern "C" {

int stmg_net_create(int H, int W, int c_in, int hidden, int c_out, int n_layers, int skip, int max_batch,
                    unsigned long long seed, stmg_net** out) {
  if (!out) return STMG_ERR_ARG;
  *out = nullptr;
  if (H < 1 || W < 1 || n_layers < 1 || n_layers > 16 || max_batch < 1) return STMG_ERR_ARG;
  if (c_in < 1 || c_in > 1024 || c_out < 1 || c_out > 1024 || (n_layers > 1 && (hidden < 1 || hidden > 1024)))
    return STMG_ERR_ARG;
  stmg_net* n = new stmg_net();
  n->H = H; n->W = W; n->cin = c_in; n->hid = hidden; n->cout = c_out; n->L = n_layers; n->maxb = max_batch;
  n->skip = skip ? 1 : 0;
  int maxc = 0, maxk = 0;
  for (int l = 0; l < n_layers; ++l) {
    const int a = l == 0 ? c_in : hidden, b = l + 1 == n_layers ? c_out : hidden;
    n->ci.push_back(a);
    n->co.push_back(b);
    n->woff.push_back(n->np);
    n->np += (long long)b * 9 * a;
    n->boff.push_back(n->np);
    n->np += b;
    maxc = std::max(maxc, std::max(a, b));
    maxk = std::max(maxk, b * 9 * a);
  }
  if (n->skip) {
    n->soff = n->np;
    n->np += (long long)c_out * 9 * c_in;
    maxk = std::max(maxk, c_out * 9 * c_in);
  }
  const long long pix = (long long)max_batch * H * W;
  n->part_cap = std::max((long long)64 * maxk, ((pix + 511) / 512) * (long long)maxc);
  int s = STMG_OK;
  auto A = [&](void** p, size_t bytes) { if (s == STMG_OK) s = alloc(n, p, bytes); };
  A((void**)&n->params, sizeof(float) * n->np);
  A((void**)&n->grads, sizeof(float) * n->np);
  A((void**)&n->m, sizeof(float) * n->np);
  A((void**)&n->v, sizeof(float) * n->np);
  A((void**)&n->wt, sizeof(float) * maxk);
  n->acts.assign(n_layers, nullptr);
  for (int l = 1; l < n_layers; ++l) A((void**)&n->acts[l], sizeof(float) * pix * hidden);
  if (n_layers > 1) {
    A((void**)&n->g[0], sizeof(float) * pix * hidden);
    A((void**)&n->g[1], sizeof(float) * pix * hidden);
  }
  A((void**)&n->pred, sizeof(float) * pix * c_out);
  A((void**)&n->gpred, sizeof(float) * pix * c_out);
  A((void**)&n->part, sizeof(float) * n->part_cap);
  A((void**)&n->loss_part, sizeof(double) * mse_partials());
  if (s == STMG_OK) s = init_params(n, seed);
  if (s != STMG_OK) {
    stmg_net_destroy(n);
    return s;
  }
  *out = n;
  return STMG_OK;
}

void stmg_net_destroy(stmg_net* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  for (void* p : n->owned) cudaFree(p);
  delete n;
}

int stmg_net_set_stream(stmg_net* n, void* stream) {
  if (!n) return STMG_ERR_ARG;
  n->st = (cudaStream_t)stream;
  return STMG_OK;
}

int stmg_net_num_params(const stmg_net* n, long long* np) {
  if (!n || !np) return STMG_ERR_ARG;
  *np = n->np;
  return STMG_OK;
}

int stmg_net_set_params(stmg_net* n, const float* p) {
  if (!n || !p) return STMG_ERR_ARG;
  NCK(cudaMemcpyAsync(n->params, p, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, n->st));
  NCK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->np, n->st));
  NCK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->np, n->st));
  return STMG_OK;
}

int stmg_net_get_params(const stmg_net* n, float* p) {
  if (!n || !p) return STMG_ERR_ARG;
  NCK(cudaMemcpyAsync(p, n->params, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, n->st));
  return STMG_OK;
}

int stmg_net_get_grads(const stmg_net* n, float* g) {
  if (!n || !g) return STMG_ERR_ARG;
  NCK(cudaMemcpyAsync(g, n->grads, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, n->st));
  return STMG_OK;
}

int stmg_net_forward(stmg_net* n, int batch, const float* in, const int* index, float* out) {
  if (!ok_batch(n, batch) || !in || !out || in == out) return STMG_ERR_ARG;
  return forward(n, batch, in, index, out);
}

int stmg_net_backward(stmg_net* n, int batch, const float* in, const int* index, const float* grad_out) {
  if (!ok_batch(n, batch) || !in || !grad_out) return STMG_ERR_ARG;
  return backward(n, batch, in, index, grad_out);
}

int stmg_net_mse(stmg_net* n, int batch, const float* pred, const float* target, const int* index, float* grad,
                 double* loss) {
  if (!ok_batch(n, batch) || !pred || !target) return STMG_ERR_ARG;
  NCK(launch_mse(pred, target, index, (long long)n->H * n->W * n->cout, batch, grad, n->loss_part, loss, n->st));
  return STMG_OK;
}

int stmg_net_adam(stmg_net* n, float lr, float beta1, float beta2, float eps, int step) {
  if (!n || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
    return STMG_ERR_ARG;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
  NCK(launch_adam(n->np, n->params, n->grads, n->m, n->v, lr, beta1, beta2, eps, c1, c2, n->st));
  return STMG_OK;
}

int stmg_net_train_step(stmg_net* n, int batch, const float* inputs, const float* targets, const int* index,
                        float lr, float beta1, float beta2, float eps, int step, double* loss) {
  if (!ok_batch(n, batch) || !inputs || !targets) return STMG_ERR_ARG;
  int s = forward(n, batch, inputs, index, n->pred);
  if (s != STMG_OK) return s;
  NCK(launch_mse(n->pred, targets, index, (long long)n->H * n->W * n->cout, batch, n->gpred, n->loss_part, loss,
                 n->st));
  s = backward(n, batch, inputs, index, n->gpred);
  if (s != STMG_OK) return s;
  return stmg_net_adam(n, lr, beta1, beta2, eps, step);
}

int stmg_channel_rms(long long rows, int C, const float* data, float* rms, float* inv_rms, void* stream) {
  if (rows < 1 || C < 1 || !data) return STMG_ERR_ARG;
  NCK(launch_channel_rms(rows, C, data, rms, inv_rms, (cudaStream_t)stream));
  return STMG_OK;
}

int stmg_tensor_rms(long long n, const float* data, float* rms, float* inv_rms, void* stream) {
  if (n < 1 || !data) return STMG_ERR_ARG;
  NCK(launch_tensor_rms(n, data, rms, inv_rms, (cudaStream_t)stream));
  return STMG_OK;
}

int stmg_scale_channels(long long rows, int C, float* data, const float* s, void* stream) {
  if (rows < 1 || C < 1 || !data || !s) return STMG_ERR_ARG;
  NCK(launch_scale_channels(rows, C, data, s, (cudaStream_t)stream));
  return STMG_OK;
}

}  // extern "C"
