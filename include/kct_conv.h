/*
 * kct_conv.h -- C ABI of the tensor-core 3D convolutions (sm_103a) used by the learned
 * warm start for CGLS (a 3D U-Net that maps the normalised backprojection A^T b / (A^T A 1) to
 * an initial guess). Not part of the projector: the paper has no learned component; it is
 * the reconstruction around the operator.
 *
 * Convolution: 3x3x3, stride 1, zero padding 1, no dilation.
 *   y[n][z][y][x][co] = bias[co] + sum_{t, ci} w[co][t][ci] * x[n][z+dz-1][y+dy-1][x+dx-1][ci],
 *   t = (dz * 3 + dy) * 3 + dx, out-of-range input voxels read as 0.
 * Number types: BF16 operands, FP32 accumulation (tcgen05.mma kind::f16), BF16 output.
 * Layouts (C-contiguous, device memory owned by the caller, 16-byte aligned):
 *   activations  [n][d][h][w][c]  bf16 (channels last)
 *   weights      [cout][27][cin]  bf16
 *   bias         [cout]           float32 (may be NULL)
 * Supported sizes: cin, cout in {16, 32, 48, 64, 96, 128}; w a multiple of 16; h a multiple
 * of 128 / min(w, 128) (the output tile is 128 voxels of one z-slice). Other sizes return
 * KCT_ERR_UNSUPPORTED before any launch.
 *
 * d_err: device int32 error word. A kernel whose bounded wait on a pipeline barrier runs
 * out sets it to 1 and returns (its output is then incomplete); the caller reads it.
 * Return values are kct_status codes (kct.h); kct_conv_last_error() gives the detail.
 * All calls enqueue on `stream` (a cudaStream_t as void*) and do not synchronise.
 */
#ifndef KCT_CONV_H
#define KCT_CONV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kct_conv_desc {
    int32_t n, d, h, w;   /* batch and spatial size (input and output) */
    int32_t cin, cout;    /* channels */
} kct_conv_desc;

/* Forward convolution y = conv(x, w) + bias, then max(., 0) if relu != 0. The input
 * gradient of a convolution is this call with the roles of cin and cout exchanged and the
 * weights flipped in the taps and transposed: w'[ci][26 - t][co] = w[co][t][ci]. */
int kct_conv3d_fwd(const kct_conv_desc *desc, const void *d_x, const void *d_w, const float *d_bias, void *d_y,
                   int32_t relu, int32_t *d_err, void *stream);

/* Weight gradient gw[co][t][ci] = sum_v g[v][co] * x[v + offset(t)][ci] (float32, overwritten).
 * Operands are channels-first copies, made by the caller:
 *   d_gt             g^T  [n][cout][d][h][w] bf16
 *   d_xt0/1/2        x^T shifted along x by -1, 0, +1: xt_k[n][ci][z][y][x] = x[n][z][y][x + k - 1][ci]
 *                    (0 outside), each [n][cin][d][h][w] bf16.
 * The sum over voxels is split across blocks and added with float atomics (the order of the
 * additions is not fixed). */
int kct_conv3d_wgrad(const kct_conv_desc *desc, const void *d_gt, const void *d_xt0, const void *d_xt1,
                     const void *d_xt2, float *d_gw, int32_t *d_err, void *stream);

/* Detail of the last failure on the calling thread. */
const char *kct_conv_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KCT_CONV_H */
