/*
 * unet.h - C ABI of the learned few-view correction in libbp: the kernels a
 * 3-D residual U-Net needs for training and inference on one GB300.
 *
 * The paper has no learned component; these calls serve the few-view
 * workload (a network maps a back-projection from 1/6 of the views to the
 * full-view FDK). Every convolution is a 3x3x3, stride 1, zero-padded
 * convolution computed as an implicit GEMM on the tensor cores with BF16
 * operands and FP32 accumulation.
 *
 * Convolutions run as implicit GEMMs on the tensor cores: tcgen05.mma with
 * TMEM accumulators and TMA-staged halo bricks where the layer fits that
 * kernel's tile (cnn_set_tensor_path below), mma.sync otherwise.
 *
 * Conventions
 *   - Activations are channels-last [N][D][H][W][cstride] tensors; a call
 *     reads or writes channels [coff, coff + C) of each voxel, so a
 *     concatenation is two writes into one tensor. Element types are stated
 *     per argument (BF16 = 16-bit bfloat, raw bits as uint16).
 *   - Conv weights are BF16 [Cout][27][Cin] (tap index (dz*3+dy)*3+dx,
 *     input channel fastest); biases FP32 [Cout]; weight gradients FP32
 *     [Cout][27][Cin] and bias gradients FP32 [Cout], accumulated (+=).
 *   - Cin and Cout of the tensor-core calls are multiples of 16; channel
 *     strides and offsets are multiples of 8. Device pointers are 16-byte
 *     aligned and owned by the caller. Calls are asynchronous on `stream`,
 *     never allocate, and return bp_status (bp.h) with the message in
 *     bp_last_error(NULL).
 */
#ifndef UNET_H
#define UNET_H

#include "bp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y[..., yoff + co] = act(b[co] + sum_{tap, ci} w[co][tap][ci] x[v + tap][xoff + ci])
 * with act = ReLU when relu != 0. y is BF16 (y_fp32 == 0) or FP32. */
bp_status cnn_conv3d_forward(const void *x, int x_cstride, int x_coff, const void *w,
                             const float *b, void *y, int y_cstride, int y_coff, int y_fp32,
                             int n, int d, int h, int wd, int cin, int cout, int relu,
                             void *stream);

/* A convolution followed by the 1x1x1 output head, for inference: the
 * activation act(b + conv(x)) is rounded to BF16 and projected in the
 * convolution's epilogue, so it is never written:
 *   out[v] = res[v] + head_b[0] + sum_co head_w[co] bf16(act(b[co] + conv(x)[v][co]))
 * (the result cnn_conv3d_forward followed by cnn_head1_forward gives, bit
 * for bit). head_w FP32 [cout], head_b FP32 [1] (device, may be NULL), res
 * and out FP32 [N][D][H][W] (res may be NULL). Only the persistent tcgen05
 * kernel has this epilogue (cnn_set_tensor_path mode 1, Cout 16 or 32,
 * width a multiple of 128, depth a multiple of 4, 27 Cin Cout x 2 bytes up
 * to 81 KB); other layers return BP_ERR_UNSUPPORTED and the caller runs
 * the two calls. */
bp_status cnn_conv3d_forward_head(const void *x, int x_cstride, int x_coff, const void *w,
                                  const float *b, const float *head_w, const float *head_b,
                                  const float *res, float *out, int n, int d, int h, int wd,
                                  int cin, int cout, int relu, void *stream);

/* Input gradient of the convolution: dx[..., dxoff + ci] = sum_{tap, co}
 * w[co][tap][ci] dy[v - tap][dyoff + co] (BF16 in, BF16 out, FP32
 * accumulation). wt is a caller-owned BF16 buffer of 27*cin*cout elements
 * that receives the flipped, transposed weights used for it. */
bp_status cnn_conv3d_dgrad(const void *dy, int dy_cstride, int dy_coff, const void *w, void *wt,
                           void *dx, int dx_cstride, int dx_coff, int n, int d, int h, int wd,
                           int cin, int cout, void *stream);

/* The input gradient of cnn_conv3d_dgrad for callers that cannot allocate
 * device memory: code running while a CUDA graph is being captured, where a
 * cudaMalloc would break the capture; a serving loop or an external runtime
 * that owns every allocation on the device and hands this library only the
 * tensors; or a process whose device memory is already fully reserved by a
 * pooling allocator. This call takes no weight buffer and allocates nothing
 * (no cudaMalloc, no cudaFree, no allocating library routine): the flipped,
 * transposed weights go to a static device array of the library, reserved
 * on every GPU that loads it until the process exits.
 *   Limit: 27 * cin * cout <= 442368 BF16 values (cin * cout <= 16384, e.g.
 *   128 x 128); larger layers get BP_ERR_INVALID_ARG and must use
 *   cnn_conv3d_dgrad.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and caches it for the life of the process; make
 *   that first call before any stream capture on that device. A device
 *   reset (cudaDeviceReset, or anything else that destroys the primary
 *   context) is not supported afterwards: the cached address would be stale.
 *   All calls share the one array. Each call overwrites every value it
 *   later reads, so what an earlier call left there is never used, but two
 *   calls whose work overlaps on the GPU (different streams without
 *   ordering) race on it.
 * There is no counterpart in the paper. Other arguments and the result are
 * those of cnn_conv3d_dgrad. */
bp_status cnn_conv3d_dgrad_noalloc(const void *dy, int dy_cstride, int dy_coff, const void *w,
                                   void *dx, int dx_cstride, int dx_coff, int n, int d, int h,
                                   int wd, int cin, int cout, void *stream);

/* Weight and bias gradients: dw[co][tap][ci] += sum_v dy[v][co] x[v + tap][ci],
 * db[co] += sum_v dy[v][co] (db may be NULL). x and dy BF16. */
bp_status cnn_conv3d_wgrad(const void *x, int x_cstride, int x_coff, const void *dy,
                           int dy_cstride, int dy_coff, float *dw, float *db, int n, int d,
                           int h, int wd, int cin, int cout, void *stream);

/* Output head: one-channel 3x3x3 convolution on the CUDA cores (FP32
 * accumulation): out[v] = res[v] + b[0] + sum_{tap, ci} w[tap][ci] x[v + tap][ci]
 * with x BF16 [N][D][H][W][cstride] (channels 0..cin-1), w FP32 [27][cin],
 * b FP32 [1] (device), res and out FP32 [N][D][H][W] (res may be NULL). */
bp_status cnn_head_forward(const void *x, int x_cstride, const float *w, const float *b,
                           const float *res, float *out, int n, int d, int h, int wd, int cin,
                           void *stream);

/* Head gradients for an FP32 output gradient g [N][D][H][W]:
 * dx[v][ci] = sum_tap w[tap][ci] g[v - tap] (BF16 [..][dx_cstride]),
 * dw[tap][ci] += sum_v g[v] x[v + tap][ci], db[0] += sum_v g[v]. */
bp_status cnn_head_backward(const void *x, int x_cstride, const float *w, const float *g,
                            void *dx, int dx_cstride, float *dw, float *db, int n, int d, int h,
                            int wd, int cin, void *stream);

/* 2x2x2 max pooling (BF16): y[N][D/2][H/2][W/2][c] over the channels
 * [xoff, xoff+c) of x; D, H, W even. Backward: dy is routed to the arg-max
 * of each window (first maximum in z, y, x order) and added to dx there
 * (the other seven positions keep their value), so a skip connection's
 * gradient already in dx is summed with the pooled branch's. */
bp_status cnn_maxpool2_forward(const void *x, int x_cstride, int x_coff, void *y, int n, int d,
                               int h, int wd, int c, void *stream);
bp_status cnn_maxpool2_backward(const void *x, int x_cstride, int x_coff, const void *dy,
                                void *dx, int dx_cstride, int dx_coff, int n, int d, int h,
                                int wd, int c, void *stream);

/* Nearest-neighbour 2x upsampling (BF16): y[2z+a][2y+b][2x+c] = x[z][y][x]
 * into channels [yoff, yoff+c) of y ([N][2D][2H][2W][y_cstride]).
 * Backward: dx[z][y][x] = sum of the 8 children of dy (FP32 sum, BF16 out). */
bp_status cnn_upsample2_forward(const void *x, void *y, int y_cstride, int y_coff, int n, int d,
                                int h, int wd, int c, void *stream);
bp_status cnn_upsample2_backward(const void *dy, int dy_cstride, int dy_coff, void *dx, int n,
                                 int d, int h, int wd, int c, void *stream);

/* ReLU backward in place: g[v][goff+c] = 0 where y[v][yoff+c] <= 0 (BF16). */
bp_status cnn_relu_backward(void *g, int g_cstride, int g_coff, const void *y, int y_cstride,
                            int y_coff, long long nvox, int c, void *stream);

/* FP32 [nvox] -> BF16 channels-last [nvox][cstride]: channel 0 = x, the
 * channels 1..cstride-1 are zeroed. */
bp_status cnn_pack_input(const float *x, void *y, int cstride, long long nvox, void *stream);

/* Input layer for a one-channel FP32 volume x [N][D][H][W] (the network's
 * first convolution; a GEMM over channels would spend 15/16 of its products
 * on zero channels):
 *   y[v][y_coff + co] = act(b[co] + sum_tap w[co][tap] * bf16(x[v + tap]))
 * x is rounded to BF16 (the network's activation type) before the products,
 * which accumulate in FP32; act = ReLU when relu != 0. With cout 16, wd a
 * multiple of 8 and x 16-byte aligned it runs on tcgen05, the three x taps
 * in K against banded weights and the bias carried in the sum as two BF16
 * parts (within 2^-16 of b); otherwise on mma.sync with K = the 27 taps,
 * summed from the bias (cnn_set_tensor_path(0) forces mma.sync). The two
 * differ by rounding order only. w is BF16 [cout][27] (tap index (dz*3+dy)*3+dx), b FP32 [cout]
 * (may be NULL), y BF16 [N][D][H][W][y_cstride]. cout is a multiple of 8 up
 * to 32, wd a multiple of 4, y_cstride and y_coff multiples of 8, y 16-byte
 * aligned; anything else returns BP_ERR_INVALID_ARG. */
bp_status cnn_stem_forward(const float *x, const void *w, const float *b, void *y, int y_cstride,
                           int y_coff, int n, int d, int h, int wd, int cout, int relu,
                           void *stream);

/* Its weight and bias gradients (FP32, accumulated):
 *   dw[co][tap] += sum_v dy[v][dy_coff + co] * bf16(x[v + tap]),
 *   db[co] += sum_v dy[v][dy_coff + co]   (db may be NULL)
 * dy BF16 [N][D][H][W][dy_cstride]; same limits on cout and the channel
 * layout as cnn_stem_forward (any wd). */
bp_status cnn_stem_wgrad(const float *x, const void *dy, int dy_cstride, int dy_coff, float *dw,
                         float *db, int n, int d, int h, int wd, int cout, void *stream);

/* The input layer and the 2 x 2 x 2 max pooling that follows it in one pass
 * (no counterpart in the paper, whose method has no network): y as
 * cnn_stem_forward writes it, and pooled[v'][co] = max over the eight voxels
 * of y[.][co] under v' (bit for bit cnn_maxpool2_forward on y), without
 * reading y back. pooled is BF16 [n][d/2][h/2][wd/2][cout] (dense, 16-byte
 * aligned); d and h even, other limits as cnn_stem_forward.
 * BP_ERR_INVALID_ARG on bad arguments. */
bp_status cnn_stem_pool_forward(const float *x, const void *w, const float *b, void *y, int y_cstride, int y_coff,
                                void *pooled, int n, int d, int h, int wd, int cout, int relu, void *stream);

/* Additive skip connection: nearest 2x upsampling of x (BF16
 * [N][D][H][W][c], dense) plus a skip tensor at the fine resolution:
 *   y[2z+a][2y+b][2x+c][y_coff + ch] =
 *       bf16(x[z][y][x][ch] + skip[2z+a][2y+b][2x+c][s_coff + ch])
 * (the two BF16 values summed in FP32, rounded once). d, h, wd are the
 * coarse dimensions. c, the strides and the offsets are multiples of 8 and
 * the pointers 16-byte aligned. Its gradient is cnn_upsample2_backward for
 * x and the output gradient itself for skip. */
bp_status cnn_upsample2_add_forward(const void *x, const void *skip, int s_cstride, int s_coff,
                                    void *y, int y_cstride, int y_coff, int n, int d, int h,
                                    int wd, int c, void *stream);

/* 1x1x1 output head (cin channels -> 1), the usual last layer of a U-Net:
 *   out[v] = res[v] + b[0] + sum_ci w[ci] x[v][ci]
 * x BF16 [nvox][x_cstride] (channels 0..cin-1), w FP32 [cin], b FP32 [1]
 * (device, may be NULL), res and out FP32 [nvox] (res may be NULL); FP32
 * products summed in channel order. cin a multiple of 8 up to 32,
 * x_cstride a multiple of 8, x 16-byte aligned. */
bp_status cnn_head1_forward(const void *x, int x_cstride, const float *w, const float *b,
                            const float *res, float *out, long long nvox, int cin, void *stream);

/* Its gradients for an FP32 output gradient g [nvox]:
 *   dx[v][ci] = bf16(w[ci] g[v])   (BF16 [nvox][dx_cstride], overwritten)
 *   dw[ci] += sum_v g[v] x[v][ci],  db[0] += sum_v g[v]   (FP32; db may be NULL)
 * Same layout limits as cnn_head1_forward. */
bp_status cnn_head1_backward(const void *x, int x_cstride, const float *w, const float *g, void *dx,
                             int dx_cstride, float *dw, float *db, long long nvox, int cin,
                             void *stream);

/* Inference of the network's last step when no convolution follows the
 * last skip (no counterpart in the paper, whose method has no network):
 * cnn_upsample2_add_forward into a temporary and cnn_head1_forward on it,
 * in one pass and bit for bit their result, the full-resolution sum never
 * written:
 *   a[v][ci] = bf16(up(x)[v][ci] + skip[v][ci]),
 *   out[v] = res[v] + b[0] + sum_ci w[ci] a[v][ci].
 * x BF16 [n][d][h][wd][c] (dense, coarse), skip BF16 [n][2d][2h][2wd]
 * [s_cstride] (channels s_coff ..), w FP32 [c], b FP32 [1] (may be NULL),
 * res and out FP32 [n][2d][2h][2wd] (res may be NULL). c a multiple of 8 up
 * to 32; s_cstride and s_coff multiples of 8; x and skip 16-byte aligned,
 * res and out 8-byte aligned. BP_ERR_INVALID_ARG on bad arguments. */
bp_status cnn_upsample2_add_head1_forward(const void *x, const void *skip, int s_cstride, int s_coff,
                                          const float *w, const float *b, const float *res, float *out, int n,
                                          int d, int h, int wd, int c, void *stream);

/* Mean-square error: g = 2 (p - t) / n (FP32), and sum (p - t)^2 added
 * into loss[0] (FP32, caller zeroes it). */
bp_status cnn_mse(const float *p, const float *t, float *g, float *loss, long long n, void *stream);

/* Adam step on n FP32 parameters with BF16 copies: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);
 * p16 (may be NULL) receives bf16(p). Then g is zeroed. */
bp_status cnn_adam(float *p, float *g, float *m, float *v, void *p16, long long n, float lr,
                   float b1, float b2, float eps, int t, void *stream);

/* Tuning and testing (no counterpart in the paper).
 *   cnn_set_tensor_path  process-wide choice of the kernel behind
 *                        cnn_conv3d_forward and cnn_conv3d_dgrad: 1 (default)
 *                        the tcgen05 kernels (TMEM accumulators, TMA-staged
 *                        bricks, one MMA per brick row shared by the output
 *                        rows it feeds) for every layer that fits their tile
 *                        (width a multiple of 128, depth a multiple of 4,
 *                        Cout 16 or 32, Cin a multiple of 16, 16-byte
 *                        aligned): the persistent one (one CTA per SM,
 *                        resident weights, two brick stages, two TMEM
 *                        accumulator sets) where all weights fit in shared
 *                        memory beside the stages (27 Cin Cout x 2 bytes up
 *                        to 81 KB), the per-tile one otherwise; 2: the
 *                        per-tile tcgen05 kernel only; 0: always the
 *                        mma.sync kernel.
 *   cnn_device_status    synchronise the stream, then read and clear the
 *                        device error word of the tensor-core kernels
 *                        (bounded waits): BP_OK, BP_ERR_TIMEOUT or BP_ERR_DEVICE. */
bp_status cnn_set_tensor_path(int mode);
bp_status cnn_device_status(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* UNET_H */
