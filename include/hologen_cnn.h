/*
 * hologen_cnn.h -- C ABI of the learned warm start for GS: a small
 * encoder-decoder CNN that maps a target amplitude to a starting replay
 * phase, its training step, and the tensor-core convolution kernels it is
 * built from.
 *
 * The paper (HoloGen, arXiv:2008.12214) has no network: GS and its variants
 * (Section 3.2) start from a free replay phase, and this net only proposes
 * that phase; GS still iterates to its error as before.  Plain random-phase
 * GS stays the fallback and the measure of the net's value.
 *
 * Network (all 3x3 convolutions zero-padded and followed by ReLU):
 *   encoder levels 0..3 of widths 32, 64, 128, 256, two convolutions each,
 *   2x2 average pooling between levels; decoder levels 2, 1, 0: nearest 2x
 *   upsampling of the coarser output concatenated with the encoder output of
 *   the same level ([upsampled, skip] channel order), two convolutions;
 *   head: 1x1 convolution 32 -> 2 giving (c, s); phase = atan2(s, c).
 *   Input: T / max(T) per image.  1,946,338 parameters.
 * Loss per image (mean over the batch), wT = T^2 / sum T^2:
 *   L = sum_px wT |(c, s) - (cos phi, sin phi)|^2 / 2
 * with phi the label phase (the replay phase GS reaches): the net regresses
 * the label's phasor, which on the unit circle is 1 - cos(phase error).
 * Adam with beta1 0.9, beta2 0.999, eps 1e-8, bias corrected.
 *
 * Parameter vector (FP32, the order of every get/set call): for each 3x3
 * convolution in the order e0a e0b e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b
 * d0a d0b its weight [9][Cout][Cin] (tap t = 3 (dy+1) + (dx+1)) then its
 * bias [Cout]; then the head weight [2][32] and bias [2].
 *
 * Data: images are [batch][H][W] float in replay order (as in hologen.h);
 * H and W must be multiples of 8 with (H/8) * (W/8) >= 128 and each of
 * W/8, W/4, W/2, W either a multiple of 128 or a divisor of 128 (e.g. 128,
 * 256, 512, 1024).  Activations live in the net as BF16 [B][H][W][C]; the
 * convolutions accumulate in FP32 on the tensor cores.
 *
 * Buffers are DEVICE pointers; calls enqueue on the net's stream and return
 * (hg_cnn_sync waits and reports device-side errors).  Status codes are
 * those of hologen.h.
 */
#ifndef HOLOGEN_CNN_H
#define HOLOGEN_CNN_H

#include <stddef.h>
#include <stdint.h>

#include "hologen.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hg_cnn_s *hg_cnn;

#define HG_CNN_NPARAMS 1946338

/* Creates a net for images of height x width and batches up to max_batch,
 * with He-normal weights (std sqrt(2 / (9 Cin)), head std sqrt(1/32), zero
 * biases) drawn from `seed`, Adam state zero.  stream: cudaStream_t (NULL:
 * legacy default stream).  Errors: HG_ERR_INVALID_ARG, HG_ERR_UNSUPPORTED_SIZE
 * (shape rules above), HG_ERR_OOM, HG_ERR_CUDA. */
hg_status hg_cnn_create(hg_cnn *out, int height, int width, int max_batch, uint64_t seed, void *stream);
void hg_cnn_destroy(hg_cnn net);

/* Parameter vector in and out (HG_CNN_NPARAMS floats, device).  Setting
 * also refreshes the BF16 copies the convolutions read. */
hg_status hg_cnn_set_params(hg_cnn net, const float *params);
hg_status hg_cnn_get_params(hg_cnn net, float *params);
/* Training state for checkpoint / resume: `state` holds 3 x HG_CNN_NPARAMS
 * floats (device): the parameters, then Adam's first and second moments, in
 * the parameter order above; `step` is Adam's step count.  A net given the
 * state of another continues its training bit for bit. */
hg_status hg_cnn_get_state(hg_cnn net, float *state, int64_t *step);
hg_status hg_cnn_set_state(hg_cnn net, const float *state, int64_t step);
/* Gradient of the loss of the last hg_cnn_train_step / hg_cnn_gradients. */
hg_status hg_cnn_get_grads(hg_cnn net, float *grads);

/* Forward pass of `batch` targets [batch][H][W]: cs_out [batch][H][W][2]
 * (c, s) and/or phase_out [batch][H][W] = atan2(s, c) (+ the base phase, see
 * hg_cnn_set_base_phase), either may be NULL. */
hg_status hg_cnn_forward(hg_cnn net, const float *target, int batch, float *cs_out, float *phase_out);

/* Loss and gradients for (target, phase label) without updating the
 * parameters; loss_out: one double (device) or NULL. */
hg_status hg_cnn_gradients(hg_cnn net, const float *target, const float *phase_label, int batch,
                           double *loss_out);

/* One training step: loss and gradients, then one Adam update of every
 * parameter with learning rate lr (the step counter advances). */
hg_status hg_cnn_train_step(hg_cnn net, const float *target, const float *phase_label, int batch, float lr,
                            double *loss_out);

/* One Adam update of every parameter from the given gradient vector
 * (HG_CNN_NPARAMS floats, device or host, parameter order above) with
 * learning rate lr; the step counter advances and hg_cnn_get_grads then
 * returns these gradients.  With the gradients of hg_cnn_gradients this is
 * hg_cnn_train_step; data-parallel training averages each rank's gradients
 * over the ranks (an all-reduce) in between.  The paper has no network, so
 * no counterpart there.  Errors: HG_ERR_INVALID_ARG (NULL, lr <= 0),
 * HG_ERR_CUDA. */
hg_status hg_cnn_apply_grads(hg_cnn net, const float *grads, float lr);

/* A base phase phi_b [H][W] float radians (device or host pointer; NULL
 * removes it), the same for every image: with it the network models the
 * remainder of a label over the base, e^{i(phi - phi_b)}.  The loss of
 * hg_cnn_gradients / hg_cnn_train_step compares (c, s) with
 * e^{i(phi - phi_b)}, and hg_cnn_forward's phase_out is atan2(s, c) + phi_b
 * (not wrapped).  GS labels grown from one shared start phase keep a large
 * part of that start (Section 3.2's loop changes the replay phase only
 * partly), a fixed random field that a convolutional network cannot produce
 * from the target; with the start as the base, the network is asked only for
 * what GS added.  The paper has no network, so no counterpart there.  Copies
 * the field into the net's own device buffer (allocated at the first call)
 * and waits for the copy.  Errors: HG_ERR_INVALID_ARG (NULL net),
 * HG_ERR_OOM, HG_ERR_CUDA. */
hg_status hg_cnn_set_base_phase(hg_cnn net, const float *base);

/* Waits for the net's stream; HG_ERR_TIMEOUT if a bounded device wait gave
 * up, HG_ERR_INVALID_ARG if a target held a negative / NaN / infinite value,
 * HG_ERR_NUMERIC for an all-zero target. */
hg_status hg_cnn_sync(hg_cnn net);
/* Kernels the last call enqueued. */
int hg_cnn_launch_count(hg_cnn net);

/*
 * Layer-level tensor-core convolutions (the net's building blocks, exposed
 * for tests and measurement).  BF16 tensors are passed as raw 16-bit words;
 * layouts as in the net: activations [B][H][W][C], weights [9][Cout][Cin].
 * Cin and Cout multiples of 32; Cout <= 512 for the forward, <= 256 for the
 * weight gradient; W a multiple or divisor of 128 (forward) and of 64
 * (weight gradient), H such that whole tiles fit (H * W a multiple of 128).
 *
 * hg_conv3x3_forward  y = relu?(conv(x, w) + bias) [* (mask > 0)]; bias and
 *                     mask may be NULL.
 * hg_conv3x3_dgrad    dx = conv(dy, w_rot) [* (mask > 0)], the gradient wrt
 *                     x of sum(dy * conv(x, w)), given w_rot[t][ci][co] =
 *                     w[8 - t][co][ci] ([9][Cin][Cout]).
 * hg_conv3x3_wgrad    dw [9][Cout][Cin] = sum_px dy[p][co] x[p + shift_t][ci]
 *                     and db [Cout] = sum_px dy (may be NULL), FP32.
 *                     workspace: hg_conv3x3_wgrad_workspace(...) bytes of
 *                     device memory.
 * Errors: HG_ERR_INVALID_ARG, HG_ERR_UNSUPPORTED_SIZE, HG_ERR_CUDA; a timed
 * out device wait is reported by hg_conv_status.
 */
hg_status hg_conv3x3_forward(const uint16_t *x, int B, int H, int W, int Cin, const uint16_t *w, int Cout,
                             const float *bias, int relu, const uint16_t *mask, uint16_t *y, void *stream);
hg_status hg_conv3x3_dgrad(const uint16_t *dy, int B, int H, int W, int Cout, const uint16_t *w_rot, int Cin,
                           const uint16_t *mask, uint16_t *dx, void *stream);
size_t hg_conv3x3_wgrad_workspace(int B, int H, int W, int Cin, int Cout);
hg_status hg_conv3x3_wgrad(const uint16_t *x, const uint16_t *dy, int B, int H, int W, int Cin, int Cout,
                           float *dw, float *db, void *workspace, size_t workspace_bytes, void *stream);
/* Waits for `stream`; HG_ERR_TIMEOUT if a layer-level kernel's bounded wait
 * gave up since the last call (the flag is then cleared). */
hg_status hg_conv_status(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HOLOGEN_CNN_H */
