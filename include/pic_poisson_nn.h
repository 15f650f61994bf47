/*
 * pic_poisson_nn -- kernels of the learned warm start for the batched mode
 * solve: a small convolutional U-Net maps the mode residual of the
 * previous-step iterate, r_m = b_m - A_m phi_hat_(t-1),m, to an approximate
 * correction d_m ~ A_m^{-1} r_m, and the solve starts from
 * phi_hat_(t-1) + alpha d with the minimal-residual step alpha.  The paper
 * trains no network; this extension follows the project specification of a
 * learned initial guess, and the multigrid still iterates to the same
 * residual (the guess changes only the number of cycles).
 *
 * Tensors: NHWC BF16 (n = azimuthal mode, y = axial cell k, x = radial cell i,
 * channels contiguous), except where FP32 or the solver's FP64 mode layout
 * (see pic_poisson.h) is stated.  All pointers are caller-owned device memory;
 * every call is asynchronous on `stream` (a cudaStream_t) and returns a
 * PIC_POISSON_* status (EINVAL for bad sizes, ECUDA for launch failures; see
 * pic_poisson_last_error()).
 */
#ifndef PIC_POISSON_NN_H
#define PIC_POISSON_NN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * 3x3 convolution, stride 1, zero padding: out[n,y,x,co] = bias[co] +
 * sum_{tap, ci} w[tap][co][ci] in[n, y+dy, x+dx, ci] (tap = 3 (dy+1) + (dx+1)),
 * optional ReLU.  in: BF16 [n,h,w,cin], cin a multiple of 16; w: BF16
 * [9][cout][cin]; bias: FP32 [cout] or NULL; cout a multiple of 8, <= 128.
 * Writes out_bf16 (BF16 [n,h,w,cout]) and/or out_f32 (FP32, same shape).
 * Runs on the tcgen05 tensor cores (an implicit GEMM: 128 output pixels x
 * cout per tile, TMA-staged operands, FP32 accumulators in tensor memory)
 * when cout is a multiple of 16, w is a multiple of 128 or 16, 32 or 64, and
 * every tensor is 16-byte aligned; otherwise as pic_nn_conv3x3_mma_sync.
 */
int pic_nn_conv3x3(const void *in, int cin, const void *w, const float *bias, void *out_bf16, float *out_f32, int cout,
                   int n, int h, int wd, int relu, void *stream);
/* The same convolution on the legacy mma.sync m16n8k16 path (BF16 tensor
 * cores, FP32 accumulation; any w), for comparison and as the fallback. */
int pic_nn_conv3x3_mma_sync(const void *in, int cin, const void *w, const float *bias, void *out_bf16,
                            float *out_f32, int cout, int n, int h, int wd, int relu, void *stream);
/* Whether a bounded wait of the tcgen05 convolution ran out since the last
 * call: *status = 0 (none) or 1 + the role that gave up (0 TMA producer,
 * 1 MMA issuer, 2 epilogue, 3 / 4 the final drains); clears the flag.  Such a
 * kernel ends early and its output is not valid.  Synchronous. */
int pic_nn_conv_tc_status(int *status);

/* Weights of the data-gradient convolution: wt[8-tap][ci][co] = w[tap][co][ci]
 * (so d_in = conv3x3(d_out, wt) with cin' = cout, cout' = cin). */
int pic_nn_flip_weights(const void *w, int cout, int cin, void *wt, void *stream);

/* Scratch (floats) that pic_nn_conv3x3_wgrad needs for these sizes. */
size_t pic_nn_wgrad_scratch_floats(int cin, int cout, int n, int h, int wd);

/*
 * Weight and bias gradients of pic_nn_conv3x3: dw[tap][co][ci] =
 * sum_pixels dout[p][co] in[p + shift(tap)][ci], dbias[co] = sum_p dout[p][co]
 * (FP32, deterministic: per-chunk partials summed in chunk order).
 */
int pic_nn_conv3x3_wgrad(const void *in, int cin, const void *dout, int cout, int n, int h, int wd, float *dw,
                         float *dbias, float *scratch, size_t scratch_floats, void *stream);

/* dy = 0 where y <= 0 (ReLU backward, in place on dy; count elements). */
int pic_nn_relu_bwd(const void *y, void *dy, long count, void *stream);

/* 2x2 average pooling [n,h,w,c] -> [n,h/2,w/2,c] (backward = 1: its adjoint,
 * in = d_out [n,h/2,w/2,c], out = d_in [n,h,w,c]). */
int pic_nn_pool2(const void *in, void *out, int n, int h, int wd, int c, int backward, void *stream);

/* Nearest 2x upsampling [n,h,w,c] into channels [0,c) of out [n,2h,2w,cstride]
 * (backward = 1: sum over each 2x2 block from those channels into [n,h,w,c]). */
int pic_nn_up2(const void *in, void *out, int n, int h, int wd, int c, int cstride, int backward, void *stream);

/* dst[p, doff + ch] = src[p, soff + ch] for ch < c (channel concatenation / split). */
int pic_nn_copy_channels(const void *src, int sstride, int soff, void *dst, int dstride, int doff, long pixels, int c,
                         void *stream);

/* Mean-squared error of the first `used` of c FP32 channels against target
 * [pixels][used]; writes dpred (BF16 [pixels][c], zero on unused channels) and
 * the loss (one FP32, device).  scratch: ceil(pixels*c/256) floats. */
int pic_nn_mse(const float *pred, const float *target, long pixels, int c, int used, void *dpred, float *scratch,
               float *loss, void *stream);

/* Adam step on FP32 master weights w with gradient g and moments m, v (step
 * counted from 1); also writes the BF16 copy w_bf16 when non-NULL. */
int pic_nn_adam(float *w, const float *g, float *m, float *v, long count, float lr, float b1, float b2, float eps,
                int step, void *w_bf16, void *stream);

/* a += b, BF16, count elements (gradient accumulation at skip connections). */
int pic_nn_add(void *a, const void *b, long count, void *stream);

/* b = BF16(a), count elements. */
int pic_nn_to_bf16(const float *a, void *b, long count, void *stream);

/*
 * Network input from a complex FP64 mode-layout field x (nz, nr, nm): per
 * mode the RMS over the cells (rms, FP32 [nm]), and out = BF16 [nm, nz, nr, 16]
 * with channels Re x / rms, Im x / rms, shift (FP32 [nz][nr][nm] or NULL),
 * then zeros.  scratch: 256 * nm doubles.
 */
int pic_nn_pack_modes(const double *x, const float *shift, int nr, int nz, int nm, float *rms, double *scratch,
                      void *out, void *stream);

/* Training target of a complex FP64 mode-layout field x (nz, nr, nm): per
 * mode the RMS of |x| over the cells (rms, FP32 [nm]) and out = FP32
 * [nm, nz, nr, 2] = (Re x, Im x) * sqrt(2) / rms, each real component at
 * unit RMS.  scratch: 256 * nm doubles. */
int pic_nn_pack_target(const double *x, int nr, int nz, int nm, float *rms, double *scratch, float *out,
                       void *stream);
/* A training batch: xb[b] = X[idx[b]] (BF16 [pixels][16] per sample) with
 * channels 0-1 multiplied by sign[b], yb[b] = sign[b] * Y[idx[b]] (FP32
 * [pixels][2]); idx (int64) and sign (FP32, +-1) device arrays of batch entries. */
int pic_nn_gather_batch(const void *X, const float *Y, const long *idx, const float *sign, int batch, long pixels,
                        void *xb, float *yb, void *stream);
/* d (FP64 mode layout) = gain * rms[m] * (y[m,k,i,0] + i y[m,k,i,1]), y FP32 with c channels. */
int pic_nn_unpack_modes(const float *y, int c, const float *rms, float gain, int nr, int nz, int nm, double *d,
                        void *stream);

/* Mode-layout 2:1 restriction (sum of each 2x2 fine block) from (nr, nz) to
 * (nr/2, nz/2), and bilinear cell-centred prolongation back (zero on walls). */
int pic_nn_restrict2(const double *f, int nr, int nz, int nm, double *c, void *stream);
int pic_nn_prolong2(const double *c, int nr, int nz, int nm, double *f, void *stream);

/*
 * out = x + alpha d with alpha = sign <r, b> / <b, b> (Parseval-weighted over
 * the entries; alpha = 0 when <b, b> = 0); with b = -A d and sign = -1 this is
 * the step that minimises ||r - alpha A d||, so the result's residual is never
 * larger than r's.  *alpha (device, may be NULL) receives the step.
 * scratch: 1027 doubles.
 */
int pic_nn_minres_step(const double *x, const double *d, const double *r, const double *b, long entries, int nm,
                       int nt, double sign, double *scratch, double *out, double *alpha, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PIC_POISSON_NN_H */
