/*
 * bte_surrogate.h -- C ABI of the learned surrogate of the batched solver:
 * an ensemble of small MLPs that maps a drive / field / temperature point
 * x = (E_dc, E_omega, omega, B, mu) to y = (absorption, time-averaged drift
 * velocity), the two observables the solver reports per point (Sec. 2,
 * Eqs. v_dr_generic and absorption_def), trained on points the batched
 * solver computed, with the solver as fallback wherever the members
 * disagree.  The paper has no learned part; the network is the library's
 * own:
 *
 *   xh = 2 (x - x_lo) / (x_hi - x_lo) - 1
 *   h1 = silu(W1 xh + b1), h2 = silu(W2 h1 + b2), h3 = silu(W3 h2 + b3)
 *   y  = (W4 h3 + b4) * y_std + y_mean,       silu(z) = z / (1 + exp(-z))
 *
 * with hidden width 256.  Each member's parameters are packed as W1 [256][5],
 * b1 [256], W2 [256][256], b2 [256], W3 [256][256], b3 [256], W4 [2][256],
 * b4 [2] (133,634 FP32 values, row-major).  Training minimises
 * (1/(2B)) sum_b |yh_b - (t_b - y_mean)/y_std|^2 over minibatches of B
 * points with Adam; the 256 x 256 layers and their backward products run on
 * BF16 tensor cores with FP32 accumulation; the master weights, Adam moments,
 * the 5-input and 2-output layers and all reductions are FP32.
 *
 * Conventions: as in bte.h (status codes, bte_last_error, HOST pointers
 * unless a comment says "device", one host thread per handle at a time).
 * Work is queued on the handle's stream; every call with host outputs
 * synchronises it.
 */
#ifndef BTE_SURROGATE_H
#define BTE_SURROGATE_H

#include "bte.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bte_sur bte_sur;

typedef struct {
    int32_t members;        /* ensemble size, 1..64 (0: 8)                              */
    int32_t width;          /* hidden width; only 256 is supported (0: 256)              */
    int32_t batch_capacity; /* rows of activations held on the device: training
                               minibatch limit and inference chunk (multiple of 128,
                               0: 16384)                                                 */
    int32_t reserved;
    double x_lo[5], x_hi[5];/* input box used for normalisation (x_hi > x_lo)            */
    double y_mean[2];       /* output standardisation (y_std > 0)                        */
    double y_std[2];
    void* stream;           /* cudaStream_t, or NULL for a stream the handle creates     */
} bte_sur_config;

/* Creates an ensemble with all parameters zero; BTE_EINVAL for a bad config. */
BTE_API int bte_sur_create(const bte_sur_config* cfg, bte_sur** out);

/* Number of FP32 values of one packed member (133,634 at width 256). */
BTE_API int64_t bte_sur_param_count(const bte_sur* h);

/* Replaces every member's parameters from HOST p [members][param_count] and
 * resets the Adam state (moments 0, step count 0). */
BTE_API int bte_sur_set_params(bte_sur* h, const float* p);

/* Copies every member's FP32 parameters to HOST p [members][param_count]. */
BTE_API int bte_sur_get_params(bte_sur* h, float* p);

/* Uploads a training set: HOST x [n][5], y [n][2] (raw, unnormalised).  The
 * handle keeps its own device copy until the next call or bte_sur_destroy. */
BTE_API int bte_sur_set_data(bte_sur* h, const float* x, const float* y, int64_t n);

/* `steps` Adam steps on the uploaded set.  order is HOST
 * [steps][members][batch] of row indices into the set (each member sees its
 * own minibatches), lr HOST [steps] learning rates, batch <= batch_capacity.
 * Adam: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.  When loss
 * is not NULL it receives HOST [steps][members] minibatch losses. */
BTE_API int bte_sur_train(bte_sur* h, const int32_t* order, int32_t steps, int32_t batch,
                          const float* lr, double* loss);

/* Loss and gradient of every member on HOST x [n][5], t [n][2]
 * (n <= batch_capacity): grad HOST [members][param_count], loss HOST
 * [members] (either may be NULL).  Parameters are not changed. */
BTE_API int bte_sur_grad(bte_sur* h, const float* x, const float* t, int32_t n, float* grad,
                         double* loss);

/* Ensemble prediction of HOST x [n][5]: mean and population standard
 * deviation over members of the de-standardised outputs (HOST [n][2] each)
 * and, when mask is not NULL, mask[i] = 1 where max(std[i][0], std[i][1]) >
 * threshold (or is NaN), else 0.  Works in chunks of batch_capacity rows
 * over two device buffer sets: the copies of one chunk (on two internal
 * copy streams, created on the first call) overlap the inference of the
 * next; with page-locked host arrays the copies are fully asynchronous.
 * Returns when every output is written. */
BTE_API int bte_sur_predict(bte_sur* h, const float* x, int64_t n, float* mean, float* stdv,
                            uint8_t* mask, double threshold);

/* As bte_sur_predict with DEVICE arrays; queued on the handle's stream,
 * returns without waiting (mask may be NULL). */
BTE_API int bte_sur_predict_device(bte_sur* h, const float* x, int64_t n, float* mean,
                                   float* stdv, uint8_t* mask, double threshold);

/* Solver parameters of one surrogate point x = (E_dc, E_omega, omega, B, mu)
 * (omega > 0, mu > 0): phi_y in [-L, L] with L = 7/sqrt(mu) + 1.5 B,
 * m_points = clamp(2 ceil(L / 0.02) + 1, 201, 2001), n_max = clamp(ceil(12 +
 * 3 mu + 10 B), 20, 200), dt = 1e-3, ceil(16 omega / (2 pi)) + 1 periods with
 * the last one averaged (the exp(-t) transient is below 1.2e-7 after t = 16,
 * and one whole period of the periodic state gives the window average). */
BTE_API int bte_sur_protocol(const double* x, int32_t precision, bte_params* out);

/* Surrogate with solver fallback for HOST x [n][5] (double): predicts every
 * point, then solves the points whose ensemble std exceeds threshold with
 * bte_batch_run (parameters from bte_sur_protocol at `precision`, options
 * `opts` or NULL) and takes the solver's result there.  y HOST [n][2]
 * receives (absorption, v_dc); solved HOST [n] (may be NULL) 1 where the
 * solver ran; status HOST [n] (may be NULL) the solver's per-point status
 * (BTE_OK for predicted points).  Returns the worst solver status. */
BTE_API int bte_sur_hybrid(bte_sur* h, const double* x, int64_t n, double threshold,
                           int32_t precision, const bte_batch_opts* opts, double* y,
                           uint8_t* solved, int32_t* status);

/* Frees the handle and its device memory.  NULL is ignored. */
BTE_API void bte_sur_destroy(bte_sur* h);

#ifdef __cplusplus
}
#endif

#endif /* BTE_SURROGATE_H */
