/*
 * surrogate.h -- C ABI of the kernels behind the learned sensitivity
 * surrogate: a small convolutional U-Net that maps a design rho and the
 * damping level to an estimate of the sensitivity map dW~/drho, so that an
 * optimizer can take cheap intermediate design steps between full
 * forward + adjoint runs (which stay the reference and check the steps).
 * The paper has no such component; its Sec. 1 notes that learned models need
 * large data sets, which the adjoint runs themselves provide here.
 *
 * All pointers are device pointers to FP32 data (loss: FP64) owned by the
 * caller; the functions allocate nothing and enqueue work on `stream` (a
 * cudaStream_t, NULL = legacy default stream).  Activations are stored
 * [C][B][H][W] (channel, batch, row, column), so a convolution is the GEMM
 * W[Cout][Cin k k] . col[Cin k k][B H W] and a channel concatenation is two
 * tensors placed one after the other.  Every function returns 0 on success,
 * 1 for invalid arguments, 3 if a CUDA launch failed.
 */
#ifndef FDTD_SURROGATE_H
#define FDTD_SURROGATE_H

#ifdef __cplusplus
extern "C" {
#endif

/* C[M][N] = alpha op(A) op(B) + beta C (row-major).  op(A) = A (M x K, lda)
 * or A^T (A stored K x M) when transA; op(B) = B (K x N, ldb) or B^T (B
 * stored N x K) when transB.  work: caller device scratch of work_elems
 * floats (may be NULL with work_elems = 0).  When the product has few output
 * tiles and a long K (weight gradients) it is split into K slices, as many
 * as the scratch holds at M x N floats each; each slice writes its partial
 * product there and the slices are summed in a fixed order, so results are
 * deterministic whatever the split.  Without scratch the product runs
 * unsplit (slower for weight gradients, same precision class). */
int nn_gemm(int transA, int transB, int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
            float beta, float *C, int ldc, float *work, long long work_elems, void *stream);

/* The same product with BF16 operands on the tensor cores and FP32
 * accumulation and output: each tile of A and B (FP32 in memory) is rounded
 * to BF16 (nearest even) as it is staged in shared memory, then C = alpha
 * op(A16) op(B16) + beta C with mma.sync (m16n8k16) and FP32 accumulators.
 * K splitting and the scratch as for nn_gemm. */
int nn_gemm_bf16(int transA, int transB, int M, int N, int K, float alpha, const float *A, int lda, const float *B,
                 int ldb, float beta, float *C, int ldc, float *work, long long work_elems, void *stream);

/* col[(c 9 + t)][(b H + y) W + x] = x[c][b][y + t/3 - 1][x + t%3 - 1], zero
 * outside the image (3 x 3 convolution, stride 1, padding 1). */
int nn_im2col3(const float *x, int C, int B, int H, int W, float *col, void *stream);

/* dx += the adjoint of nn_im2col3 applied to dcol. */
int nn_col2im3_add(const float *dcol, int C, int B, int H, int W, float *dx, void *stream);

/* y[c][p] = act(y[c][p] + bias[c]) for c < Cout, p < P; act = ReLU if relu. */
int nn_bias_act(float *y, const float *bias, int Cout, long long P, int relu, void *stream);

/* dy <- dy * (y > 0) if relu (y: the layer's output), then db[c] = sum_p dy[c][p]. */
int nn_act_bwd_bias(const float *y, float *dy, float *db, int Cout, long long P, int relu, void *stream);

/* 2 x 2 average pooling of `planes` planes of H x W (H, W even), and dx += its adjoint. */
int nn_pool2(const float *x, long long planes, int H, int W, float *y, void *stream);
int nn_pool2_bwd_add(const float *dy, long long planes, int H, int W, float *dx, void *stream);

/* 2x nearest upsampling of planes h x w to 2h x 2w, and dx += its adjoint. */
int nn_up2(const float *x, long long planes, int h, int w, float *y, void *stream);
int nn_up2_bwd_add(const float *dy, long long planes, int h, int w, float *dx, void *stream);

/* *loss = mean (y - t)^2 over n values (FP64), dy = 2 (y - t) / n. */
int nn_mse(const float *y, const float *t, long long n, float *dy, double *loss, void *stream);

/* Adam step `step` (>= 1) on n parameters: m, v are the moment buffers. */
int nn_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float beta1, float beta2, float eps,
            int step, void *stream);

/* x[0 .. n) = 0. */
int nn_zero(float *x, long long n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_SURROGATE_H */
