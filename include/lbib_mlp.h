/* lbib_mlp.h -- C ABI of the learned surrogate: a multilayer perceptron
 * trained and evaluated on the GPU by the library's own kernels.
 *
 * The paper reports trajectories of the adhesion observables N_L, delta p and
 * r for a parameter sweep (particle aspect ratio, Ca, cell shape, ligand
 * density; Sec. 3.1, Figs. 5-9).  The surrogate maps such parameters and the
 * time t u_max / H to those observables; it has no counterpart in the paper.
 *
 * Network: n_hidden hidden layers of `width` units with GELU,
 *   a_0 = bf16(s_in * (x - c_in)),
 *   z_l = W_l a_{l-1} + b_l,  a_l = bf16(GELU(z_l))   (l = 1 .. n_hidden),
 *   y   = s_out * (W_out a_{n_hidden} + b_out) + c_out,
 * weights used in BF16 (FP32 master copies), products accumulated in FP32.
 * GELU in the tanh form of Hendrycks & Gimpel (Gaussian Error Linear Units,
 * 2016): GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), within
 * 5e-4 of z Phi(z) (Phi the standard normal distribution function); the tanh
 * is evaluated by the GPU's tanh approximation (relative error about 2^-11).
 * Training minimises the mean over the batch and the outputs of
 * ((y - t) / s_out)^2 (targets standardised by the same affine map) with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * All calls return lbib_status (include/lbib.h); messages through
 * lbib_last_error(NULL).  A context is used by one thread at a time.
 */
#ifndef LBIB_MLP_H
#define LBIB_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "lbib.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbib_mlp lbib_mlp;

typedef struct lbib_mlp_desc {
    int32_t n_in;        /* input features, 1 .. 32 */
    int32_t width;       /* hidden units, a multiple of 64, <= 1024 */
    int32_t n_hidden;    /* hidden layers, 1 .. 8 */
    int32_t n_out;       /* outputs, 1 .. 64 */
    int32_t max_batch;   /* largest batch a call may pass, >= 1 */
    int32_t device;      /* CUDA device ordinal */
    void* cuda_stream;   /* cudaStream_t to enqueue on (borrowed), or NULL for a private one */
    uint64_t seed;       /* weight initialisation (uniform +-sqrt(6 / (fan_in + fan_out)), biases 0) */
    const float* in_shift;   /* host, n_in values c_in (copied); NULL: zeros */
    const float* in_scale;   /* host, n_in values s_in (copied); NULL: ones */
    const float* out_shift;  /* host, n_out values c_out (copied); NULL: zeros */
    const float* out_scale;  /* host, n_out values s_out (copied); NULL: ones */
} lbib_mlp_desc;

/* Creates a network on desc->device; *out receives the handle. */
lbib_status lbib_mlp_create(const lbib_mlp_desc* desc, lbib_mlp** out);

/* Inference: x DEVICE [batch][n_in] floats, y DEVICE [batch][n_out] floats,
 * 1 <= batch <= max_batch; enqueued on the context stream (no wait). */
lbib_status lbib_mlp_forward(lbib_mlp* net, const float* x, int32_t batch, float* y);

/* One Adam step on the batch: x DEVICE [batch][n_in], t DEVICE [batch][n_out]
 * targets; lr the step size; loss DEVICE float (may be NULL) receives the
 * batch loss before the update.  Enqueued on the context stream. */
lbib_status lbib_mlp_train_step(lbib_mlp* net, const float* x, const float* t, int32_t batch, float lr,
                                float* loss);

/* Gradient of the batch loss with respect to every parameter, without an
 * update, copied to the HOST array grad of n >= lbib_mlp_param_count values
 * (layout as lbib_mlp_get_params); *loss (host, may be NULL) the loss.  Waits. */
lbib_status lbib_mlp_gradients(lbib_mlp* net, const float* x, const float* t, int32_t batch, float* grad, size_t n,
                               float* loss);

/* Data-parallel training (each rank holds a copy of the network; the ranks'
 * shards of one global batch have equal size).  The loss is a mean over the
 * batch, so the global batch's gradient is the mean of the shards' gradients:
 * every rank calls lbib_mlp_backward on its shard, the caller sums the arrays
 * across ranks (an all-reduce) and every rank calls lbib_mlp_apply_gradient
 * with scale = 1 / ranks, which leaves the copies identical.
 *
 * lbib_mlp_backward: gradient of the batch loss with respect to every
 * parameter, without an update, into the DEVICE array grad of
 * n >= lbib_mlp_param_count floats (layout as lbib_mlp_get_params); loss
 * DEVICE float (may be NULL) receives the batch loss.  Enqueued on the context
 * stream (no wait); the values equal lbib_mlp_gradients' bit for bit. */
lbib_status lbib_mlp_backward(lbib_mlp* net, const float* x, const float* t, int32_t batch, float* grad, size_t n,
                              float* loss);

/* One Adam step (as lbib_mlp_train_step's) with the gradient scale * grad in
 * place of a batch's own: grad DEVICE, n >= param_count floats, layout as
 * lbib_mlp_get_params; scale finite, lr > 0.  Enqueued on the context stream;
 * grad may be overwritten by the next call on the context only after this one
 * has run (stream order). */
lbib_status lbib_mlp_apply_gradient(lbib_mlp* net, const float* grad, size_t n, float scale, float lr);

/* Number of parameters: for each layer (hidden ones first, then the output
 * layer) its weights W [out][in] row-major, then its biases b [out]. */
lbib_status lbib_mlp_param_count(lbib_mlp* net, size_t* n);

/* FP32 master parameters to / from a HOST array of n >= param_count values
 * (set also resets the Adam moments and step count).  Wait for the stream. */
lbib_status lbib_mlp_get_params(lbib_mlp* net, float* params, size_t n);
lbib_status lbib_mlp_set_params(lbib_mlp* net, const float* params, size_t n);

/* Waits for the context stream and reads the tensor-core kernels' status
 * word: LBIB_ERR_TIMEOUT when one of their bounded waits gave up (that
 * call's products are incomplete).  From then on the network refuses work
 * (LBIB_ERR_TIMEOUT from forward, train_step, backward, apply_gradient and
 * gradients; gradients and get_params also check the word) until
 * lbib_mlp_set_params loads parameters again. */
lbib_status lbib_mlp_sync(lbib_mlp* net);
/* Fault injection for failure-detection tests (no counterpart in the paper;
 * nothing faults or hangs a GPU): kind LBIB_FAULT_WAIT_TIMEOUT sets, in
 * stream order, the status bit a bounded wait sets when it gives up. */
lbib_status lbib_mlp_inject_fault(lbib_mlp* net, int32_t kind);
/* Releases every resource of net (NULL is ignored). */
void lbib_mlp_destroy(lbib_mlp* net);

#ifdef __cplusplus
}
#endif

#endif /* LBIB_MLP_H */
