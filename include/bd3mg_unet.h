/*
 * bd3mg_unet.h -- C ABI of the learned warm start: a small 3D U-Net that maps
 * an observation y (and its per-depth blur width) to a start point x0 for the
 * block 3MG iteration of bd3mg.h.
 *
 * The paper has no learned component (its only initialisation is a random
 * start, Section 3.1); this network is the warm start asked of this library.
 * Its training targets are solutions of the penalised problem of Section 3.1
 * (Eq. "crit") computed by the 3MG iteration itself.
 *
 * Network (levels L, widths c[0..L-1], input channels cin):
 *   encoder level l: two 3x3x3 convolutions (zero padding) + bias + ReLU,
 *     preceded for l > 0 by 2x2x2 max pooling (ties: first maximum in
 *     (dz, dy, dx) order);
 *   decoder level l = L-2 .. 0: a 2x2x2 stride-2 transposed convolution + bias
 *     (no activation) from level l+1, concatenation [encoder level l output,
 *     upsampled] along channels, then two 3x3x3 convolutions + bias + ReLU;
 *   head: 1x1x1 convolution c[0] -> 1 + bias; the prediction is
 *     base + head(...) (residual output; base is normally y).
 * Inputs [B][D][H][W][cin] float32 (channels last, cin <= 16); D, H, W
 * multiples of 2^(L-1).  Requirements of this build: c[0] = 16, every c[l] a
 * multiple of 16 and <= 128, 1 <= L <= 6.
 *
 * Parameters are one flat float32 vector, layer by layer in the order
 *   enc0a, enc0b, enc1a, enc1b, ..., enc(L-1)a, enc(L-1)b,
 *   up(L-2), dec(L-2)a, dec(L-2)b, ..., up0, dec0a, dec0b, head,
 * each layer as its weight then its bias.  A 3x3x3 weight is [27][Cout][Cin]
 * with tap t = (dz*3 + dy)*3 + dx reading input voxel (z+dz-1, y+dy-1,
 * x+dx-1); an up weight is [8][Cout][Cin] with tap a = (az*2 + ay)*2 + ax
 * writing output voxel (2z+az, 2y+ay, 2x+ax); the head weight is [1][1][c0].
 *
 * Precision: FP32 master weights (Adam state FP32); BF16 weights, activations
 * and activation gradients; every contraction accumulates in FP32 on the
 * tcgen05 tensor cores (TMEM accumulators); the loss and its sums in FP64.
 *
 * Conventions follow bd3mg.h: statuses (bd3mg_status), errors are sticky per
 * object, work is ordered on the stream given at creation, calls that return
 * host values synchronise it, one host thread per object.  Device memory is
 * obtained with cudaMallocAsync on that stream.
 */
#ifndef BD3MG_UNET_H
#define BD3MG_UNET_H

#include <stddef.h>

#include "bd3mg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bd3mg_unet bd3mg_unet;

typedef struct {
    int levels;              /* L */
    int widths[8];           /* c[0..L-1] */
    int cin;                 /* input channels, 1..16 */
    double lr, beta1, beta2, eps;   /* Adam; 0 -> 1e-3, 0.9, 0.999, 1e-8 */
} bd3mg_unet_params;

/* Create a network with all parameters zero (set them with
 * bd3mg_unet_set_params).  stream: cudaStream_t as void*. */
bd3mg_status bd3mg_unet_create(const bd3mg_unet_params *p, void *stream, bd3mg_unet **out);

/* Number of float32 parameters of the flat vector. */
long long bd3mg_unet_param_count(bd3mg_unet *net);

/* Copy the flat FP32 parameters in (from HOST memory; resets Adam's moments
 * and step count) or out (to HOST memory). */
bd3mg_status bd3mg_unet_set_params(bd3mg_unet *net, const float *params);
bd3mg_status bd3mg_unet_get_params(bd3mg_unet *net, float *params);

/* Flat FP32 gradient of the last bd3mg_unet_train_step or
 * bd3mg_unet_loss_grad (HOST memory out). */
bd3mg_status bd3mg_unet_get_grads(bd3mg_unet *net, float *grads);

/* Forward pass: inp DEVICE [B][D][H][W][cin] float32, base DEVICE [B][D][H][W]
 * float32 or NULL (zero), pred DEVICE [B][D][H][W] float32 out.  Enqueued,
 * not synchronised. */
bd3mg_status bd3mg_unet_forward(bd3mg_unet *net, int B, int D, int H, int W, const float *inp, const float *base,
                                float *pred);

/* Forward, MSE loss mean((pred - target)^2) and the full backward pass (the
 * gradient is kept for bd3mg_unet_get_grads); no parameter update.  loss may be
 * NULL (then nothing is synchronised). */
bd3mg_status bd3mg_unet_loss_grad(bd3mg_unet *net, int B, int D, int H, int W, const float *inp, const float *base,
                                  const float *target, double *loss);

/* bd3mg_unet_loss_grad followed by one Adam step (bias-corrected moments) on
 * every parameter; the BF16 weights are refreshed from the FP32 masters. */
bd3mg_status bd3mg_unet_train_step(bd3mg_unet *net, int B, int D, int H, int W, const float *inp,
                                   const float *base, const float *target, double *loss);

/* Single tensor-core layers on DEVICE buffers (building blocks of the network,
 * exposed for testing).  x, dz, out: BF16 channels-last tensors over a
 * [B][D][H][W] grid with row strides ldx, ldz, ldo (elements, multiples of 8).
 * w: BF16 weights [27][cout][cin] (conv3) or [8][cout][cin] (up).
 *   bd3mg_unet_conv3: out = act(conv3(x) + bias) with act = ReLU if relu,
 *     then out *= (mask > 0) if mask (rows of ldm) is not NULL.
 *   bd3mg_unet_conv3_wgrad: dw[t][co][ci] = sum_v dz[v][co] x[v + s_t][ci]
 *     (FP32 out, DEVICE).
 *   bd3mg_unet_up: out (grid [B][2D][2H][2W]) = up(x) + bias.
 * cin, cout multiples of 16; cin <= 256, cout <= 128 (wgrad), cout <= 256.
 * Each call synchronises the stream and returns BD3MG_ETIMEOUT if one of the
 * kernel's bounded waits (TMA copies, MMA completion) ran out. */
bd3mg_status bd3mg_unet_conv3(int B, int D, int H, int W, const void *x, int ldx, int cin, const void *w, int cout,
                              const float *bias, int relu, const void *mask, int ldm, void *out, int ldo,
                              void *stream);
bd3mg_status bd3mg_unet_conv3_wgrad(int B, int D, int H, int W, const void *x, int ldx, int cin, const void *dz,
                                    int ldz, int cout, float *dw, void *stream);
bd3mg_status bd3mg_unet_up(int B, int D, int H, int W, const void *x, int ldx, int cin, const void *w, int cout,
                           const float *bias, void *out, int ldo, void *stream);

/* Process-wide choice of the 3x3x3 convolution kernel (not thread-safe; set it
 * before launching work).  1 (the default): a convolution whose operands fit
 * (cout a multiple of 16 up to 128, cin of 16, 32, 64 or 128 channels, the 27
 * taps' weights of cout output channels, or of cout / parts <= 64 in 2 or 4
 * launches, and a ring of four staged input slices, or of two where four do
 * not fit, within 224 KB of shared memory, x 16-byte aligned) runs
 * the TMA-staged kernel, which
 * marches along z, copies each input slice of an 8 x 16 column once and adds
 * it to the three outputs it feeds with one group of MMAs; the others run the
 * row-gather implicit GEMM.  0: the row-gather implicit GEMM for every
 * convolution.  Both add the taps of an output in the same order (z-tap, then
 * in-plane tap, then channel), so their outputs are the same bits.  Returns
 * the previous setting. */
int bd3mg_unet_set_tma_conv(int enable);

const char *bd3mg_unet_error_string(bd3mg_unet *net);
void bd3mg_unet_destroy(bd3mg_unet *net);

#ifdef __cplusplus
}
#endif

#endif /* BD3MG_UNET_H */
