/*
 * clb_nop.h -- C ABI of the learned warm start's kernels: a small
 * convolutional neural operator that predicts the steady (u, v, T) of a
 * porous cavity from its porosity field and (Ra, Da, Pr, sigma), used to
 * initialise the time march (clb_set_fields).  The paper has no learned
 * component; the time march it describes still decides the answer.
 *
 * Conventions: all pointers are device pointers; activations are BF16 in
 * NHWC layout (channels fastest); convolution weights are a BF16 matrix
 * [taps * cin][cout] (cout fastest), taps = 9 for a 3x3 convolution with
 * zero padding 1, 1 for a 1x1 convolution; biases, gradients of weights and
 * optimiser state are FP32.  Every call is asynchronous on `stream`
 * (cudaStream_t, NULL = legacy stream) and returns CLB_NOP_OK or an error;
 * shapes are checked on the host before any launch.  Products run on the
 * BF16 tensor cores with FP32 accumulation, on tcgen05 (accumulator in
 * TMEM): fed by TMA copies when the pixels tile into whole image rows and
 * the channel counts are multiples of 8 (for the forward pass: when the
 * transposed weights are given), otherwise from operands gathered through
 * registers when the gathered channel count is a multiple of 8 and the
 * operands are 16-byte aligned; the 1x1 convolution to 4 outputs runs on
 * CUDA cores; other shapes on an mma.sync implicit GEMM.  A TMA box that
 * extends past a tensor's last channel is much slower than one inside it:
 * channel counts of 32, or multiples of 64, keep every box inside.
 */
#ifndef CLB_NOP_H
#define CLB_NOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CLB_NOP_OK 0
#define CLB_NOP_ERR_ARG (-1)
#define CLB_NOP_ERR_CUDA (-2)
#define CLB_NOP_ERR_TIMEOUT (-3)

/* y[n,h,w,co] = act(bias[co] + sum_{tap,ci} x[n,h+dy,w+dx,ci] W[tap*cin+ci][co]);
 * act = ReLU if relu != 0; y is FP32 if y_f32 != 0, else BF16.  wt, if not
 * NULL, is W transposed ([cout][taps*cin], clb_nop_transpose) and enables
 * the tcgen05 path. */
int clb_nop_conv_fwd(const void* x, const void* w, const void* wt, const float* bias, void* y, int32_t y_f32,
                     int32_t relu, int32_t n, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                     void* stream);

/* dx[n,h,w,ci] = sum_{tap,co} dy[n,h-dy,w-dx,co] W[tap*cin+ci][co], then
 * zeroed where mask (the layer input, BF16) is <= 0 if mask != NULL. */
int clb_nop_conv_dgrad(const void* dy, const void* w, const void* mask, void* dx, int32_t n, int32_t h, int32_t wd,
                       int32_t cin, int32_t cout, int32_t taps, void* stream);

/* dw[tap*cin+ci][co] += sum_{n,h,w} x[n,h+dy,w+dx,ci] dy[n,h,w,co]  (FP32
 * atomics; clear dw first).  splitk >= 1 splits the pixel sum over that many
 * blocks; splitk <= 0 lets the library choose (about four blocks per SM). */
int clb_nop_conv_wgrad(const void* x, const void* dy, float* dw, int32_t n, int32_t h, int32_t wd, int32_t cin,
                       int32_t cout, int32_t taps, int32_t splitk, void* stream);

/* The weight gradient above and, in the same pass, the bias gradient
 * db[co] += sum_{n,h,w} dy[n,h,w,co] (FP32; clear db first; db NULL: weights
 * only).  On the tensor-core path the bias rides along as an extra row of
 * ones in the pixel operand (when taps * cin is not a multiple of 128). */
int clb_nop_conv_wgrad_bias(const void* x, const void* dy, float* dw, float* db, int32_t n, int32_t h, int32_t wd,
                            int32_t cin, int32_t cout, int32_t taps, int32_t splitk, void* stream);

/* db[c] += sum over npix pixels of dy[p][c]  (clear db first). */
int clb_nop_bias_grad(const void* dy, float* db, int64_t npix, int32_t c, void* stream);

/* 2x2 average pooling (h, w even): forward (n,h,w,c) -> (n,h/2,w/2,c);
 * backward takes dy (n,h/2,w/2,c) and writes dx (n,h,w,c). */
int clb_nop_pool2(const void* in, void* out, int32_t n, int32_t h, int32_t w, int32_t c, int32_t backward,
                  void* stream);

/* Nearest 2x upsampling: forward (n,h,w,c) -> (n,2h,2w,c); backward takes
 * dy (n,2h,2w,c) and writes dx (n,h,w,c) (sum of the four copies). */
int clb_nop_up2(const void* in, void* out, int32_t n, int32_t h, int32_t w, int32_t c, int32_t backward,
                void* stream);

/* Channel concatenation y = [a | b] over npix pixels; inverse != 0 splits y
 * back into a and b. */
int clb_nop_concat(void* a, void* b, void* y, int64_t npix, int32_t ca, int32_t cb, int32_t inverse, void* stream);

/* Channel-weighted mean squared error of n FP32 values laid out with nch
 * channels fastest (n a multiple of nch): *loss += sum_i w[i % nch]
 * (pred_i - target_i)^2 / n and grad_i = 2 w[i % nch] (pred_i - target_i) / n
 * in BF16; wch = NULL weighs every channel 1 (clear *loss first). */
int clb_nop_mse(const float* pred, const float* target, const float* wch, int32_t nch, void* grad, float* loss,
                int64_t n, void* stream);

/* One Adam step (bias-corrected, step count t >= 1) on FP32 weights w with
 * FP32 gradient g and moments m, v; wb (BF16 copy of w) refreshed if not NULL. */
int clb_nop_adam(float* w, const float* g, float* m, float* v, void* wb, int64_t n, float lr, float b1, float b2,
                 float eps, int32_t t, void* stream);

/* One tensor of a multi-tensor Adam step: FP32 weights w, gradient g,
 * moments m, v (n = rows * cols values, row-major [rows][cols]); wb (BF16
 * copy, same layout) and wbt (BF16 transposed copy [cols][rows]) are
 * refreshed when not NULL. */
typedef struct {
    float* w;
    const float* g;
    float* m;
    float* v;
    void* wb;
    void* wbt;
    int64_t n;
    int32_t rows, cols;
} clb_nop_adam_seg;

/* The Adam step of clb_nop_adam on nseg tensors in one launch per 32 of them
 * (segs: a host array, passed by value to the kernel). */
int clb_nop_adam_multi(const clb_nop_adam_seg* segs, int32_t nseg, float lr, float b1, float b2, float eps, int32_t t,
                       void* stream);

/* out = (d1 + d2) where a > 0, else 0 (d2, a may be NULL: no term / no mask). */
int clb_nop_add_mask(const void* d1, const void* d2, const void* a, void* out, int64_t n, void* stream);

/* y = BF16(x) for n values. */
int clb_nop_cast_bf16(const float* x, void* y, int64_t n, void* stream);

/* wt[c][r] = w[r][c] for a BF16 rows x cols matrix. */
int clb_nop_transpose(const void* w, void* wt, int32_t rows, int32_t cols, void* stream);

/* Synchronises `stream` and reports (and clears) the tcgen05 kernels'
 * time-out flag: CLB_NOP_ERR_TIMEOUT if a kernel gave up waiting for its
 * tensor-core operations (about 2 s) and skipped its output. */
int clb_nop_check(void* stream);

/* Failure-path self-test: one CTA takes TMEM, waits on an mbarrier that
 * nothing arrives at for at most limit_cycles SM clock cycles (1 ..
 * 4e9), then does what the tcgen05 kernels do when their tensor-core
 * operations do not complete in time: sets the time-out flag, skips its
 * output and frees the TMEM.  No tensor-core operation is issued and the
 * context stays usable; a following clb_nop_check returns
 * CLB_NOP_ERR_TIMEOUT (and clears the flag).  For tests of the failure
 * detection. */
int clb_nop_wait_selftest(int64_t limit_cycles, void* stream);

/* Clear `bytes` bytes at ptr. */
int clb_nop_zero(void* ptr, int64_t bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CLB_NOP_H */
