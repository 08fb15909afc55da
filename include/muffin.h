/*
 * libmuffin -- GB300 (sm_103a) implementation of the primal-dual MUFFIN
 * iteration (Deguignet, Ferrari, Mary, Ferrari, "Distributed multi-frequency
 * image reconstruction for radio-interferometry", Sec. 3, Algorithm 1).
 *
 * Problem (Sec. 2, Eqs. 5-6), for a cube X = [x_1 .. x_L] of L channels of
 * N x N pixels:
 *     min_X  sum_l w_l/2 ||y_l - H_l x_l||^2 + 1_{R+}(X)
 *            + mu_s sum_l ||W_s x_l||_1 + mu_lambda sum_n ||W_lambda x^n||_1
 * with H_l the circular convolution by the PSF of channel l (Eq. 4), W_s the
 * isotropic undecimated wavelet transform (B3 spline, J detail planes plus the
 * coarse plane, periodic) and W_lambda the orthonormal DCT-II along channels.
 * W_s may instead be the union of eight orthonormal Daubechies wavelet bases
 * the paper compares it with (Sec. 4): W_s x = (1/sqrt 8)[Psi_1 x; ..; Psi_8 x],
 * Psi_p the J-level periodic 2D DWT with the filter of p vanishing moments
 * (minimum phase, by spectral factorisation), coefficients of each basis in
 * the Mallat layout of an N x N plane; then U is [L][8][N][N].
 *
 * Conventions shared by every entry point:
 *  - Cubes are float32, channel-major, row-major: element (l, y, x) of an
 *    [L][N][N] cube is at l*N*N + y*N + x.  Wavelet coefficients U are
 *    [L][J+1][N][N] (plane J is the coarse plane).
 *  - Pointers named d_* are DEVICE pointers, h_* HOST pointers.  The library
 *    never takes ownership of caller memory and never calls cudaMalloc: the
 *    caller allocates the workspace (muffin_workspace_bytes) and every buffer.
 *  - Work is enqueued on the stream given to muffin_init, asynchronously,
 *    except calls that write host outputs (they synchronise that stream).
 *  - Every call returns a muffin_status; on error, muffin_last_error() gives
 *    a one-line description.  A failed call leaves the state it found unless
 *    its description says otherwise.
 *  - Call order: muffin_init -> muffin_set_psf -> muffin_iterate /
 *    muffin_objective / ...; other orders return MUFFIN_ERR_STATE.
 */
#ifndef MUFFIN_H
#define MUFFIN_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct muffin_ctx muffin_ctx;

typedef enum {
  MUFFIN_OK = 0,
  MUFFIN_ERR_ARG = -1,        /* bad size, pointer or parameter */
  MUFFIN_ERR_CUDA = -2,       /* a CUDA call failed (message names it) */
  MUFFIN_ERR_NOMEM = -3,      /* workspace too small */
  MUFFIN_ERR_STATE = -4,      /* call out of order */
  MUFFIN_ERR_NONFINITE = -5,  /* NaN or Inf in an input or in the state */
  MUFFIN_ERR_TIMEOUT = -6     /* a bounded device wait gave up (muffin_objective, network calls) */
} muffin_status;

/* Parameters of Eqs. 5-6 and Algorithm 1. */
typedef struct {
  int nx, ny;            /* image size; nx == ny == N, N a power of two in [16, 1024] */
  int nchan;             /* L >= 1; L <= 512 */
  int nscales;           /* J >= 0 detail planes of W_s, 2^J < N */
  int iuwt_gen;          /* 1: w_j = c_j - c_{j+1};  2: w_j = c_j - H_j c_{j+1} (Sec. 4) */
  double mu_s;           /* spatial weight mu_s >= 0 (Eq. 6) */
  double mu_l;           /* spectral weight mu_lambda >= 0 (Eq. 6) */
  double tau;            /* primal step; <= 0: Condat's rule from power-iteration norms */
  double sigma;          /* dual step; <= 0: 1 (Sec. 4 uses sigma = 1) */
  double rho;            /* relaxation; <= 0: 1 */
  const double* h_chan_weight; /* host, L weights w_l = 1/sigma_l^2 of Eq. 5; NULL: all 1 */
  int fine_levels;       /* tiling split j1 of W_s (advanced); < 0: automatic */
  int power_iters;       /* power-method passes for each operator norm; <= 0: 40 */
  int dictionary;        /* W_s: 0 IUWT (above), 1 union of eight Daubechies bases (needs J >= 1;
                            iuwt_gen and fine_levels are then ignored) */
} muffin_params;

/* Bytes of device workspace a context with these parameters needs (0 if the
 * parameters are invalid; see muffin_check_params). */
size_t muffin_workspace_bytes(const muffin_params* p);

/* MUFFIN_OK if the parameters describe a problem this library can solve,
 * else MUFFIN_ERR_ARG with a reason in h_msg (may be NULL, >= 128 bytes). */
int muffin_check_params(const muffin_params* p, char* h_msg, size_t msg_len);

/* Create a context (Algorithm 1, "Initialize": X = U = V = 0).
 * d_dirty: [L][N][N] dirty cube y of Eq. 4, copied into the workspace (the
 * caller may free it afterwards).  d_workspace: caller-owned, at least
 * muffin_workspace_bytes(p) bytes, 256-byte aligned, valid until
 * muffin_destroy.  stream: where all work of this context is enqueued. */
int muffin_init(muffin_ctx** ctx, const muffin_params* p, const float* d_dirty, void* d_workspace,
                size_t ws_bytes, cudaStream_t stream);

/* Set the PSFs (Eq. 4): d_psf [L][N][N], channel l's PSF with its peak at
 * pixel (N/2, N/2).  Builds the Fourier multipliers of H_l^T H_l, the vector
 * H_l^T y_l, the operator norms by the power method and, if tau was left to
 * the library, the step sizes (Condat: 1/tau - sigma ||L||^2 > beta/2).
 * Synchronises the stream. */
int muffin_set_psf(muffin_ctx* ctx, const float* d_psf);

/* Run n_iter >= 0 passes of Algorithm 1 (Eqs. 8-14), asynchronously. */
int muffin_iterate(muffin_ctx* ctx, int n_iter);

/* Objective of Eqs. 5-6 at the current X (positivity holds by construction):
 * h_obj[0] = total; if h_terms != NULL it receives (data term, mu_s spatial
 * l1, mu_lambda spectral l1).  FP64 FFT and FP64 reductions.  Synchronises.
 * Returns MUFFIN_ERR_TIMEOUT if, since the last check, a thread block of a
 * pipelined (TMA) pass kernel -- the spectral step or the column filter --
 * gave up one of its bounded waits (its tiles were then not written; the
 * count is per device). */
int muffin_objective(muffin_ctx* ctx, double* h_obj, double* h_terms);

/* Current X out to / in from a device cube [L][N][N] (warm start: set X and
 * keep U, V). */
int muffin_get_cube(muffin_ctx* ctx, float* d_x);
int muffin_set_cube(muffin_ctx* ctx, const float* d_x);

/* Full state (X [L][N][N], U [L][J+1][N][N], V [L][N][N], pass count) out /
 * in, device buffers in the natural layout.  Restoring a saved state and
 * iterating gives the same cube as never having stopped. */
int muffin_get_state(muffin_ctx* ctx, float* d_x, float* d_u, float* d_v, long long* h_iter);
int muffin_set_state(muffin_ctx* ctx, const float* d_x, const float* d_u, const float* d_v, long long iter);

/* Change mu_s / mu_lambda (two-step calibration of Sec. 4: first mu_lambda
 * = 0, then mu_lambda > 0 from the same X).  Automatic step sizes are
 * recomputed; the state is kept. */
int muffin_set_mu(muffin_ctx* ctx, double mu_s, double mu_l);

/* Step sizes in use and the norms behind them: beta = max_l w_l ||H_l||^2 by
 * the power method, l_norm2 = mu_s^2 ||W_s||^2 + mu_lambda^2, beta_closed =
 * max_l w_l max_k |hhat_l(k)|^2 (exact, H_l is circulant).  Any pointer may
 * be NULL. */
int muffin_step_sizes(const muffin_ctx* ctx, double* tau, double* sigma, double* rho, double* beta,
                      double* l_norm2, double* beta_closed, double* ws_norm2);

/* Per-stage timing: run n_iter passes launching each kernel stage between
 * CUDA events on the context stream (no graph); h_ms[k] receives the summed
 * milliseconds of stage k for k < n_stages (see muffin_stage_name; with the
 * union of bases, stage 0 is its adjoint and stage 4 its analysis).
 * Synchronises. */
int muffin_iterate_timed(muffin_ctx* ctx, int n_iter, double* h_ms, int n_stages);
int muffin_num_stages(void);
const char* muffin_stage_name(int k);
/* Bytes one launch of stage k must move at least (each input read once, each
 * output written once) for this context; 0 if the stage does not run. */
double muffin_stage_bytes(const muffin_ctx* ctx, int k);
/* Number of kernels one pass of Algorithm 1 launches for this context. */
int muffin_kernels_per_iteration(const muffin_ctx* ctx);
/* Schedule of one pass (no change to what it computes): the gradient FFTs,
 * the primal step and the spatial analysis and adjoint run per group of
 * channels_per_group channels (0: the whole cube as one group), so that the
 * row spectra and the c_j1 / r_j1 hand-offs of a group stay in the L2 cache;
 * groups alternate between `branches` (1..3) concurrent branches of the
 * pass's CUDA graph, and the spectral step runs on its own branch once every
 * group's D is written.  Results are bitwise the same for every plan.
 * muffin_plan reports the plan in effect (groups never exceed the channel
 * count; branches never exceed the group count). */
int muffin_set_plan(muffin_ctx* ctx, int channels_per_group, int branches);
int muffin_plan(const muffin_ctx* ctx, int* channels_per_group, int* branches);

/* Wavelet tiling in use: levels j < *fine_levels run on halo tiles, the others
 * on class sub-images split over *cluster blocks (0: single-block streaming
 * kernel).  Either pointer may be NULL. */
int muffin_tiling(const muffin_ctx* ctx, int* fine_levels, int* cluster);

/* Threads per block of the vectorised wavelet kernels of the split in use
 * (256 or 512; each block size has its own work runs per thread), chosen by
 * the set-up autotuner with the split when fine_levels < 0.  Either pointer
 * may be NULL. */
int muffin_block_threads(const muffin_ctx* ctx, int* fine_threads, int* coarse_threads);

const char* muffin_last_error(const muffin_ctx* ctx);  /* ctx may be NULL (init errors) */

/* The Daubechies lowpass filter with p vanishing moments (1 <= p <= 8) that
 * the union of bases uses, h[0 .. 2p-1] (host, double), H(z) = sum_t h[t] z^-t,
 * minimum phase, sum h = sqrt 2.  Host computation only (no CUDA call);
 * returns 0, or -1 if p is out of range. */
int muffin_daubechies_filter(int p, double* h_out);

/* Batches of cubes of uneven sizes.  A batch captures one pass of Algorithm 1
 * of every context (each with its own sizes, PSFs, tiling and workspace) as
 * parallel branches of a single CUDA graph, so one graph launch per pass runs
 * all cubes concurrently on the GPU.  The contexts must have had
 * muffin_set_psf; they stay usable on their own.  Work is enqueued on stream:
 * order it with the contexts' own streams (use the same stream, or
 * synchronise).  A context changed after the batch was built (muffin_set_mu,
 * muffin_set_psf) is picked up by a new capture at the next iterate. */
typedef struct muffin_batch muffin_batch;
int muffin_batch_create(muffin_batch** batch, muffin_ctx* const* ctxs, int n, cudaStream_t stream);
int muffin_batch_iterate(muffin_batch* batch, int n_iter);
const char* muffin_batch_last_error(const muffin_batch* batch);  /* batch may be NULL (create errors) */

/* How a batch runs one pass (no change to what it computes):
 *   mode 0  parallel branches of one CUDA graph, every cube with its own
 *           kernels (the default);
 *   mode 1  one persistent cooperative kernel per pass over every cube: six
 *           stages of the pass (row FFTs, column filter, inverse rows with the
 *           primal step, spatial analysis, coarse levels, spatial adjoint with
 *           the spectral step), each a work list of (cube, channel, tile)
 *           items taken by the resident blocks in turn, separated by grid
 *           barriers.  Captured in the batch's graph like mode 0.  Needs
 *           generation-1 IUWT cubes with N in {128, 256, 512, 1024} and a
 *           wavelet split whose coarse sub-images are 32, 64 or 128 wide with
 *           at most 3 coarse levels, at most 8 cubes (else MUFFIN_ERR_ARG).
 * Every barrier wait of mode 1 gives up after a bounded number of polls
 * (muffin_batch_set_wait_limit; polls < 0 restores the default 2^22, each
 * poll sleeping about 128 ns): the blocks then skip the remaining stages and
 * the launch ends; muffin_batch_check (which synchronises) reports it as
 * MUFFIN_ERR_TIMEOUT and clears the flag.  The barrier words live in the first
 * context's workspace. */
int muffin_batch_set_mode(muffin_batch* batch, int mode);
int muffin_batch_mode(const muffin_batch* batch);
int muffin_batch_set_wait_limit(muffin_batch* batch, long long polls);
int muffin_batch_check(muffin_batch* batch);
void muffin_batch_destroy(muffin_batch* batch);

/* Spectral l1 sum  sum_n ||W_lambda x^n||_1  of a device cube d_x [nchan][n_pix]
 * (float32, channel-major), written as one double to d_out (device), for
 * callers that cannot allocate device memory at all: code inside a host
 * framework that owns every device byte through its own pool, a plugin handed
 * fixed buffers, or a memory-capped service.  The paper has no counterpart;
 * it is the third term of muffin_objective (divided by mu_lambda) computed by
 * the same kernel, with its scratch (per-block partial sums and DCT tables)
 * in one static device array of about 515 KiB that every GPU loading the
 * library holds until the process exits.  Limits: 1 <= n_pix <= 2^20,
 * 1 <= nchan <= 256; larger sizes return MUFFIN_ERR_ARG.  Calls no cudaMalloc
 * or cudaFree.  The first call on each device looks up the array's device
 * address.  Every call
 * shares the array and leaves its contents behind, so calls that overlap on
 * the GPU (other streams, other host threads) race: serialise them.
 * Asynchronous on stream; errors are described by muffin_noalloc_last_error. */
int muffin_spectral_l1_noalloc(const float* d_x, int n_pix, int nchan, double* d_out, cudaStream_t stream);
const char* muffin_noalloc_last_error(void);
void muffin_destroy(muffin_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MUFFIN_H */
