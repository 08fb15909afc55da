/*
 * libmuffin warm-start network -- a small 3D convolutional network that
 * predicts, from a dirty cube, a starting cube for Algorithm 1.
 *
 * The paper's own warm start is the two-step schedule of Sec. 4: the second
 * run of Algorithm 1 starts from the cube the first run produced.  This
 * network generalises that: trained on (dirty cube, state of Algorithm 1
 * after a number of passes) pairs, it predicts the cube X and, optionally,
 * the J+1 planes of the wavelet dual U; Algorithm 1 then runs on from the
 * predicted state (muffin_set_state with V = 0).  The paper has no network;
 * everything below is defined here.
 *
 * Network: six zero-padded 3x3x3 cross-correlations over (channel, row,
 * column) of the cube, 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> K feature maps
 * (1 <= K <= 8), a bias and a ReLU after each layer but the last.  Input
 * a0 = y / s with s = max |y| over the dirty cube.  Outputs: the cube
 * max(s * z[0], 0) and K-1 fields clamp(z[k], -1, 1), k >= 1.  Loss, for a
 * target cube t_x, target fields t_aux and output weights lam:
 *   (1/V) sum_p [lam_0 (z[0] - t_x/s)^2 + sum_{k>=1} lam_k (z[k] - t_aux[k-1])^2].
 * Training: Adam (Kingma and Ba, ICLR 2015, Algorithm 1; beta1 0.9, beta2
 * 0.999, eps 1e-8).
 *
 * Arithmetic: weights, activations and activation gradients are bfloat16,
 * every sum is accumulated in float32; master weights, their gradients and
 * Adam's moments are float32.  The 32 -> 32 layers and their gradients run on
 * the tensor cores.
 *
 * Parameters travel as one packed float32 vector: for each layer in order,
 * its weights [co][ci][3][3][3] (tap index (dz+1)*9 + (dy+1)*3 + (dx+1) for
 * the offset (dz, dy, dx) along (channel, row, column)) and then its biases
 * [co]; 111616 + 865 K values in all.
 *
 * Cubes: float32 [nz][ny][nx] (nz = spectral channels).  Fields: [nz][K-1]
 * [ny][nx] (the layout of U in include/muffin.h when K - 1 = J + 1).  Feature maps:
 * bfloat16 [nz][ny][nx][32] (features innermost), passed as void pointers to
 * 16-bit storage.  Pointers named d_* are device pointers, h_* host pointers;
 * the library never allocates: the caller provides workspaces.  Work goes on
 * the stream given at creation.  Every call returns a muffin_status
 * (include/muffin.h); muffin_net_last_error describes the last failure.
 */
#ifndef MUFFIN_NET_H
#define MUFFIN_NET_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct muffin_net muffin_net;

/* Number of packed float32 parameters with n_out output maps (0 if n_out is
 * outside [1, 8]); 112481 for n_out = 1. */
int muffin_net_num_params(int n_out);

/* Device workspace for a network with n_out output maps working on
 * nz x ny x nx cubes; training != 0 also holds every activation, the
 * gradients and Adam's moments.  0 if the sizes are invalid (each >= 1,
 * nz*ny*nx < 2^31 / 32, 1 <= n_out <= 8). */
size_t muffin_net_workspace_bytes(int nz, int ny, int nx, int n_out, int training);

/* Create a network context over a caller-owned workspace (>= the bytes
 * above, 256-byte aligned, valid until muffin_net_destroy).  h_out_weight:
 * host, n_out loss weights lam_k >= 0 (NULL: all 1).  The parameters start
 * at zero: call muffin_net_set_params. */
int muffin_net_create(muffin_net** net, int nz, int ny, int nx, int n_out, const float* h_out_weight,
                      int training, void* d_workspace, size_t ws_bytes, cudaStream_t stream);

/* Load packed float32 parameters (device, muffin_net_num_params(n_out)
 * values); resets Adam's moments and step count.  Asynchronous. */
int muffin_net_set_params(muffin_net* net, const float* d_theta);
/* Copy the current packed parameters out (device).  Asynchronous. */
int muffin_net_get_params(const muffin_net* net, float* d_theta);

/* Prediction of the starting state from the dirty cube d_dirty (float32
 * [nz][ny][nx], device): d_x = max(s * z[0], 0) (float32 [nz][ny][nx]) and,
 * if n_out > 1, d_aux = clamp(z[k], -1, 1) (float32 [nz][n_out-1][ny][nx];
 * may be NULL only when n_out == 1).  Synchronises the stream and returns
 * MUFFIN_ERR_TIMEOUT when a tensor-core wait gave up (the prediction is then
 * incomplete and must not be used); see muffin_net_check. */
int muffin_net_predict(muffin_net* net, const float* d_dirty, float* d_x, float* d_aux);

/* Loss at (d_dirty, d_target_x, d_target_aux) and its packed gradient
 * (device float32, muffin_net_num_params(n_out) values), without changing
 * the parameters.  d_target_x: float32 [nz][ny][nx]; d_target_aux: bfloat16
 * [nz][n_out-1][ny][nx] (NULL only when n_out == 1).  Training contexts only
 * (else MUFFIN_ERR_STATE).  h_loss (may be NULL) receives the loss; if given,
 * the call synchronises. */
int muffin_net_loss_grad(muffin_net* net, const float* d_dirty, const float* d_target_x,
                         const void* d_target_aux, float* d_grad, double* h_loss);

/* One Adam step on the pair at learning rate lr (finite, >= 0).  Training
 * contexts only.  d_loss (device, may be NULL) receives the loss of the pair
 * before the step, as a double.  Asynchronous: if a tensor-core wait of this
 * step (or of an unchecked earlier call on the device) gave up, the device
 * drops the parameter update instead of applying an incomplete gradient, and
 * the next muffin_net_check reports MUFFIN_ERR_TIMEOUT. */
int muffin_net_train_step(muffin_net* net, const float* d_dirty, const float* d_target_x,
                          const void* d_target_aux, float lr, double* d_loss);

const char* muffin_net_last_error(const muffin_net* net);  /* net may be NULL (create errors) */

/* Wait for the context's stream, then read and clear the device's count of
 * tensor-core waits that gave up (a wait that runs out of polls makes its
 * thread block record the give-up, drain its copies and MMAs in flight at the
 * full bound, skip its remaining tiles and free its tensor memory; the GPU
 * context stays usable).  Returns
 * MUFFIN_OK, or MUFFIN_ERR_TIMEOUT when the count was not zero (described by
 * muffin_net_last_error).  The count is per device, shared by all network
 * contexts and single-layer calls on it. */
int muffin_net_check(muffin_net* net);

/* Poll bound of the tensor-core pipeline waits on the current device (each
 * poll is one mbarrier try_wait, which may suspend for a bounded time);
 * polls < 0 restores the default 2^20.  0 makes every pipeline wait give up
 * at once (used by the tests of the give-up path).  Returns MUFFIN_OK or
 * MUFFIN_ERR_CUDA.  Takes effect for kernels launched afterwards. */
int muffin_net_set_wait_limit(long long polls);

/* Number of tensor-core waits of the 32 -> 32 layers on the current device
 * that gave up since the last call (a layer whose wait gives up leaves its
 * remaining output tiles unwritten); resets the count.  Synchronises the
 * device; -1 on a CUDA error. */
int muffin_net_wait_timeouts(void);
void muffin_net_destroy(muffin_net* net);

/* ---- single layers (the kernels the network is made of), for callers that
 * compose their own networks and for checking each kernel on its own ----
 * A 32 -> 32 layer on a [nz][ny][nx][32] bfloat16 map.  d_w: float32 weights
 * [32][32][3][3][3] as in the packed vector (rounded to bfloat16 inside).
 * d_scratch: device, >= muffin_conv3d_scratch_bytes(nz, ny, nx) bytes. */
size_t muffin_conv3d_scratch_bytes(int nz, int ny, int nx);

/* d_z = act(conv(d_a, W) + b): act = ReLU if relu != 0; d_b may be NULL
 * (no bias).  Output bfloat16 [nz][ny][nx][32]. */
int muffin_conv3d_forward(const void* d_a, const float* d_w, const float* d_b, int relu, void* d_z,
                          int nz, int ny, int nx, void* d_scratch, size_t scratch_bytes, cudaStream_t stream);

/* Gradient with respect to the layer input: d_da = m * conv^T(d_dz, W), where
 * m = (d_mask > 0) elementwise if d_mask != NULL (the ReLU of the previous
 * layer, given by its output), else 1.  All maps bfloat16 [nz][ny][nx][32]. */
int muffin_conv3d_backward_data(const void* d_dz, const float* d_w, const void* d_mask, void* d_da,
                                int nz, int ny, int nx, void* d_scratch, size_t scratch_bytes,
                                cudaStream_t stream);

/* Gradients with respect to the weights (d_dw, float32 [32][32][3][3][3])
 * and the biases (d_db, float32 [32], may be NULL) of a layer with input d_a
 * and output gradient d_dz (both bfloat16 [nz][ny][nx][32]). */
int muffin_conv3d_backward_weights(const void* d_a, const void* d_dz, float* d_dw, float* d_db,
                                   int nz, int ny, int nx, void* d_scratch, size_t scratch_bytes,
                                   cudaStream_t stream);

/* Description of the last failed single-layer call (process-wide). */
const char* muffin_conv3d_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MUFFIN_NET_H */
