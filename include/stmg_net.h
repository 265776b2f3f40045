/* libstmg: learned initial guess for the slab solves.
 *
 * The paper starts every slab solve from the data of the previous slab only through the
 * coupling term of Eq. InAlg; it has no learned initial guess.  These calls add one: a
 * small fully convolutional network maps the previous slab's solution, written as one
 * tensor row per cell, to a correction of the extrapolated DG(k) polynomial, and FGMRES
 * with the multigrid preconditioner still solves every slab to its tolerance from that
 * guess.
 *
 * Two groups of calls:
 *   - slab-vector <-> cell-tensor maps and the temporal extrapolation on a level of a
 *     multigrid handle, declared in stmg.h with the other handle calls (stmg_cells_*,
 *     stmg_extrapolate, stmg_remove_pressure_mean);
 *   - the network (this file): stmg_net_*.
 *
 * Tensors.  NHWC FP32, row-major: [batch][H][W][C], the cell (ix, iy) of an n x n mesh at
 * row iy, column ix (cells lexicographic with x fastest, as in the slab layout of stmg.h).
 *
 * Network.  n_layers 3x3 convolutions with zero padding, channels
 * c_in -> hidden -> ... -> hidden -> c_out, a bias per output channel and ReLU after every
 * layer except the last:
 *     y[b, i, j, o] = bias[o] + sum_{ky, kx, c} W[o, ky, kx, c] x[b, i + ky - 1, j + kx - 1, c]
 * With skip != 0 a linear bypass, one more 3x3 convolution (c_in -> c_out, no bias), maps
 * the input straight to the output and is added to the last layer's result: the hidden
 * layers are narrower than the cell tensors, and the bypass carries the part of the map
 * that is linear.
 * Parameters: one flat FP32 vector, layer after layer, each layer W[o][ky][kx][c] followed
 * by bias[o], then the bypass W[o][ky][kx][c]; stmg_net_num_params gives its length.
 * Initialisation: He-uniform weights (bound sqrt(6 / (9 c))) from a seeded splitmix64
 * stream, zero biases, and a zero last layer and bypass so that a fresh network returns 0
 * (the guess is then the extrapolation).
 * Loss: mean of (pred - target)^2 over all elements.  Optimiser: Adam (Kingma and Ba, 2015)
 * with bias correction.  All reductions run in a fixed order: results are deterministic.
 *
 * Ownership.  Array arguments are DEVICE pointers owned by the caller.  The network owns
 * its parameters, gradients, Adam moments, activations and scratch (allocated once in
 * stmg_net_create for up to max_batch samples).  `index` arguments (device int arrays of
 * length batch, may be NULL) select sample index[b] of a dataset of samples of the tensor
 * shape for batch entry b; NULL means the samples 0 .. batch-1 in order.
 *
 * Streams.  Calls are asynchronous on the stream set with stmg_net_set_stream (default:
 * the legacy default stream).  Status codes are those of stmg.h.
 */
#ifndef STMG_NET_H
#define STMG_NET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stmg_net stmg_net;

/* Create a network for H x W grids.  1 <= n_layers <= 16, channels in 1..1024,
   max_batch >= 1.  STMG_ERR_ARG on bad sizes, STMG_ERR_OOM if memory runs out. */
int  stmg_net_create(int H, int W, int c_in, int hidden, int c_out, int n_layers, int skip, int max_batch,
                     unsigned long long seed, stmg_net** out);
void stmg_net_destroy(stmg_net* net);
int  stmg_net_set_stream(stmg_net* net, void* cuda_stream);
int  stmg_net_num_params(const stmg_net* net, long long* n);

/* Copy the flat parameter vector in or out (device pointers, length num_params).
   set_params also clears the Adam moments. */
int  stmg_net_set_params(stmg_net* net, const float* params);
int  stmg_net_get_params(const stmg_net* net, float* params);
/* Gradient of the last stmg_net_backward / stmg_net_train_step (length num_params). */
int  stmg_net_get_grads(const stmg_net* net, float* grads);

/* out[batch][H][W][c_out] = network(in[index[b]]), in a dataset of [*][H][W][c_in]
   samples.  Keeps the activations for a following stmg_net_backward.  out must not
   alias in.  batch in 1..max_batch. */
int  stmg_net_forward(stmg_net* net, int batch, const float* in, const int* index, float* out);

/* Gradient of sum(grad_out * network(in)) with respect to the parameters, for the same
   (batch, in, index) as the preceding stmg_net_forward; overwrites the stored gradient. */
int  stmg_net_backward(stmg_net* net, int batch, const float* in, const int* index, const float* grad_out);

/* Mean squared error of pred[batch][H][W][c_out] against target[index[b]]: writes
   d loss / d pred to grad (may be NULL) and the loss to *loss (device double, may be
   NULL). */
int  stmg_net_mse(stmg_net* net, int batch, const float* pred, const float* target, const int* index,
                  float* grad, double* loss);

/* One Adam update of the parameters with the stored gradient; step >= 1 is the update
   number (bias correction). */
int  stmg_net_adam(stmg_net* net, float lr, float beta1, float beta2, float eps, int step);

/* forward + mse + backward + adam on one minibatch: inputs[index[b]] -> targets[index[b]].
   loss: device double (may be NULL) receives the minibatch loss before the update. */
int  stmg_net_train_step(stmg_net* net, int batch, const float* inputs, const float* targets,
                         const int* index, float lr, float beta1, float beta2, float eps, int step,
                         double* loss);

/* Per-channel statistics of data[rows][C] (FP32): rms[c] = sqrt(mean_rows data^2) and
   inv_rms[c] = 1 / rms[c] (0 where rms[c] is 0).  Either output may be NULL. */
int  stmg_channel_rms(long long rows, int C, const float* data, float* rms, float* inv_rms, void* cuda_stream);

/* Root mean square of all n entries of data (FP32) and its inverse (0 if the RMS is 0),
   written to rms[0] / inv_rms[0] (device; either may be NULL). */
int  stmg_tensor_rms(long long n, const float* data, float* rms, float* inv_rms, void* cuda_stream);

/* data[rows][C] *= s[c] in place. */
int  stmg_scale_channels(long long rows, int C, float* data, const float* s, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
