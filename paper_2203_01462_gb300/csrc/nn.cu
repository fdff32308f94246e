// Kernels of the learned sensitivity surrogate (a small conv U-Net): a tiled
// FP32 GEMM and a BF16 tensor-core GEMM (mma.sync, FP32 accumulation), im2col
// / col2im for 3x3 convolutions, bias + ReLU, 2x2 average pooling, 2x
// nearest upsampling, MSE loss and Adam.  Not part of the paper;
// the surrogate proposes intermediate design steps between adjoint runs.
//
// Activations use the layout [C][B][H][W]: a convolution is the product
// W[Cout][Cin K K] . col[Cin K K][B H W], and concatenating along channels is
// placing tensors next to each other in memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "../../include/surrogate.h"

namespace {

constexpr int TPB = 256;
inline int blocks_for(long long n, int cap = 152 * 16)
{
    long long b = (n + TPB - 1) / TPB;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

// C[M][N] = alpha op(A) op(B) + beta C, row-major.  op(A) is M x K (A stored
// K x M when TA), op(B) is K x N (B stored N x K when TB).  64 x 64 output
// tiles, 16-deep K slices in shared memory, 4 x 4 outputs per thread.
constexpr int GT = 64, GK = 16;

// Split K: blockIdx.z takes the K slice [z kc, (z + 1) kc); with more than
// one slice each slice writes alpha times its partial tile to part[z] (M x N,
// row-major) and k_splitk_sum adds the slices in order, so the result does
// not depend on which block finishes first.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, float alpha, const float *__restrict__ A, int lda,
                                              const float *__restrict__ B, int ldb, float beta, float *C, int ldc,
                                              int kc, float *part)
{
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4] = {};
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    for (int k0 = kb; k0 < ke; k0 += GK) {
        // 64 x 16 elements of each operand, 4 per thread.
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int mm, kk;
            if (TA) { kk = e / GT; mm = e % GT; }   // A stored K x M: consecutive m
            else { mm = e / GK; kk = e % GK; }      // A stored M x K: consecutive k
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.0f;
            if (gm < M && gk < ke) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][mm] = v;
            int nn2, kk2;
            if (TB) { nn2 = e / GK; kk2 = e % GK; }  // B stored N x K: consecutive k
            else { kk2 = e / GT; nn2 = e % GT; }     // B stored K x N: consecutive n
            const int gn = n0 + nn2, gk2 = k0 + kk2;
            float u = 0.0f;
            if (gn < N && gk2 < ke) u = TB ? B[(long long)gn * ldb + gk2] : B[(long long)gk2 * ldb + gn];
            Bs[kk2][nn2] = u;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            if (gridDim.z > 1) {
                part[((long long)blockIdx.z * M + gm) * N + gn] = alpha * acc[i][j];
            } else {
                float *c = C + (long long)gm * ldc + gn;
                *c = alpha * acc[i][j] + (beta != 0.0f ? beta * *c : 0.0f);
            }
        }
    }
}

// C = sum over s = 0 .. S-1 of part[s] (in that order) + beta C.
__global__ void k_splitk_sum(float *C, int ldc, const float *__restrict__ part, int M, int N, int S, float beta)
{
    const long long n = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float acc = part[e];
        for (int z = 1; z < S; ++z) acc += part[z * n + e];
        float *c = C + (e / N) * ldc + e % N;
        *c = acc + (beta != 0.0f ? beta * *c : 0.0f);
    }
}

// col[(c*9 + t)][(b*H + y)*W + x] = x[c][b][y + dy_t][x + dx_t] (zero padding).
// One thread per (c, pixel) writes the pixel's nine taps: the index
// arithmetic is done once, the nine stores of a warp are each contiguous.
__global__ void k_im2col3(const float *x, int C, int B, int H, int W, float *col)
{
    const int HW = H * W;
    const long long P = (long long)B * HW, n = (long long)C * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / P);
        const long long p = e - (long long)c * P;
        const int b = (int)(p / HW), rem = (int)(p - (long long)b * HW);
        const int yy = rem / W, xx = rem - yy * W;
        const float *src = x + ((long long)c * B + b) * HW;
        float *dst = col + (long long)c * 9 * P + p;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int sy = yy + t / 3 - 1, sx = xx + t % 3 - 1;
            dst[(long long)t * P] = (sy >= 0 && sy < H && sx >= 0 && sx < W) ? src[sy * W + sx] : 0.0f;
        }
    }
}

// Adjoint of im2col: dx[c][b][y][x] += sum over taps of dcol at the pixels
// that read it (gathered, so no atomics).
__global__ void k_col2im3(const float *col, int C, int B, int H, int W, float *dx)
{
    const long long P = (long long)B * H * W, n = (long long)C * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / P);
        const long long p = e % P;
        const int xx = (int)(p % W), yy = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
        float s = 0.0f;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            // pixel (oy, ox) read (yy, xx) through tap t when oy + t/3 - 1 = yy
            const int oy = yy - (t / 3 - 1), ox = xx - (t % 3 - 1);
            if (oy >= 0 && oy < H && ox >= 0 && ox < W)
                s += col[((long long)c * 9 + t) * P + ((long long)b * H + oy) * W + ox];
        }
        dx[e] += s;
    }
}

__global__ void k_bias_act(float *y, const float *bias, int Cout, long long P, int relu)
{
    const long long n = (long long)Cout * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float v = y[e] + bias[e / P];
        y[e] = relu && v < 0.0f ? 0.0f : v;
    }
}

// dy <- dy * (y > 0) where relu, then db[c] = sum over the row: one block
// of 1024 threads per row, 16-byte accesses when `vec` (P a multiple of 4,
// both arrays 16-byte aligned), a fixed summation order.
__global__ void __launch_bounds__(1024) k_relu_bwd_bias(const float *y, float *dy, float *db, long long P, int relu,
                                                        int vec)
{
    __shared__ float part[32];
    const int c = blockIdx.x;
    float s = 0.0f;
    const float *yr = y + (long long)c * P;
    float *dr = dy + (long long)c * P;
    if (vec) {
        const float4 *y4 = reinterpret_cast<const float4 *>(yr);
        float4 *d4 = reinterpret_cast<float4 *>(dr);
        for (long long p = threadIdx.x; p < P / 4; p += blockDim.x) {
            float4 g = d4[p];
            if (relu) {
                const float4 v = y4[p];
                if (!(v.x > 0.0f)) g.x = 0.0f;
                if (!(v.y > 0.0f)) g.y = 0.0f;
                if (!(v.z > 0.0f)) g.z = 0.0f;
                if (!(v.w > 0.0f)) g.w = 0.0f;
                d4[p] = g;
            }
            s += (g.x + g.y) + (g.z + g.w);
        }
    } else {
        for (long long p = threadIdx.x; p < P; p += blockDim.x) {
            float g = dr[p];
            if (relu && !(yr[p] > 0.0f)) g = 0.0f;
            dr[p] = g;
            s += g;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) db[c] = s;
    }
}

// 2 x 2 average pooling of planes [n][H][W] -> [n][H/2][W/2] and its adjoint.
__global__ void k_pool2(const float *x, long long planes, int H, int W, float *y)
{
    const int h = H / 2, w = W / 2;
    const long long n = planes * h * w;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long pl = e / ((long long)h * w);
        const int yy = (int)((e / w) % h), xx = (int)(e % w);
        const float *s = x + (pl * H + 2 * yy) * W + 2 * xx;
        y[e] = 0.25f * (s[0] + s[1] + s[W] + s[W + 1]);
    }
}

__global__ void k_pool2_bwd(const float *dy, long long planes, int H, int W, float *dx)
{
    const long long n = planes * H * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long pl = e / ((long long)H * W);
        const int yy = (int)((e / W) % H), xx = (int)(e % W);
        dx[e] += 0.25f * dy[(pl * (H / 2) + yy / 2) * (W / 2) + xx / 2];
    }
}

// 2x nearest upsampling of planes [n][h][w] -> [n][2h][2w] and its adjoint.
__global__ void k_up2(const float *x, long long planes, int h, int w, float *y)
{
    const int H = 2 * h, W = 2 * w;
    const long long n = planes * H * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long pl = e / ((long long)H * W);
        const int yy = (int)((e / W) % H), xx = (int)(e % W);
        y[e] = x[(pl * h + yy / 2) * w + xx / 2];
    }
}

__global__ void k_up2_bwd(const float *dy, long long planes, int h, int w, float *dx)
{
    const long long n = planes * h * w;
    const int W = 2 * w;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long pl = e / ((long long)h * w);
        const int yy = (int)((e / w) % h), xx = (int)(e % w);
        const float *s = dy + (pl * 2 * h + 2 * yy) * W + 2 * xx;
        dx[e] += s[0] + s[1] + s[W] + s[W + 1];
    }
}

// loss = mean (y - t)^2 (FP64 accumulation into *loss, which must start at 0);
// dy = 2 (y - t) / n.
__global__ void k_mse(const float *y, const float *t, long long n, float *dy, double *loss)
{
    double s = 0.0;
    const float inv = 2.0f / (float)n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = y[e] - t[e];
        dy[e] = inv * d;
        s += (double)d * (double)d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / (double)n);
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.0f - b1) * gg;
        const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

__global__ void k_zero_f(float *x, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        x[e] = 0.0f;
}

int status(cudaStream_t) { return cudaGetLastError() == cudaSuccess ? 0 : 3; }

}  // namespace

namespace {

// BF16 tensor-core GEMM (mma.sync m16n8k16, FP32 accumulation).  Block tile
// 64 (M) x 128 (N), K in slices of 32: each slice of op(A) and op(B) is read
// as FP32 from global memory (coalesced along whichever index is
// contiguous), rounded to BF16 (nearest even) and stored k-contiguous in
// shared memory, As[m][k] and Bs[n][k], rows padded to 40 elements so that
// the fragment loads of a warp hit 32 distinct banks.  Eight warps, 2 along
// M x 4 along N, each own a 32 x 32 sub-tile: 2 x 4 fragments of 16 x 8.
constexpr int BM = 64, BN = 128, BK = 32, BKP = BK + 8;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); }

// C = alpha op(A) op(B) + beta C as in k_gemm (split K over blockIdx.z).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_bf16(int M, int N, int K, float alpha, const float *__restrict__ A,
                                                   int lda, const float *__restrict__ B, int ldb, float beta,
                                                   float *C, int ldc, int kc, float *part)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][BKP];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BKP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 2, wn = warp & 3;
    const int g = lane >> 2, t = lane & 3;  // fragment row / column group
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][jn][r] = 0.0f;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            int mm, kk;
            if (TA) { kk = e / BM; mm = e % BM; }  // A stored K x M: consecutive m
            else { mm = e / BK; kk = e % BK; }     // A stored M x K: consecutive k
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.0f;
            if (gm < M && gk < ke) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[mm][kk] = __float2bfloat16_rn(v);
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            int nn, kk;
            if (TB) { nn = e / BK; kk = e % BK; }  // B stored N x K: consecutive k
            else { kk = e / BN; nn = e % BN; }     // B stored K x N: consecutive n
            const int gn = n0 + nn, gk = k0 + kk;
            float v = 0.0f;
            if (gn < N && gk < ke) v = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[nn][kk] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + g, c = ks + 2 * t;
                a[i][0] = lds32(&As[r][c]);
                a[i][1] = lds32(&As[r + 8][c]);
                a[i][2] = lds32(&As[r][c + 8]);
                a[i][3] = lds32(&As[r + 8][c + 8]);
            }
#pragma unroll
            for (int jn = 0; jn < 4; ++jn) {
                const int n = wn * 32 + jn * 8 + g, c = ks + 2 * t;
                b[jn][0] = lds32(&Bs[n][c]);
                b[jn][1] = lds32(&Bs[n][c + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int jn = 0; jn < 4; ++jn) mma_bf16(acc[i][jn], a[i], b[jn]);
        }
        __syncthreads();
    }
    // accumulator r of fragment (i, jn): row g (+8 for r >= 2), column 2t (+1 for odd r)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int gm = m0 + wm * 32 + i * 16 + g + (r >= 2 ? 8 : 0);
                const int gn = n0 + wn * 32 + jn * 8 + 2 * t + (r & 1);
                if (gm >= M || gn >= N) continue;
                if (gridDim.z > 1) {
                    part[((long long)blockIdx.z * M + gm) * N + gn] = alpha * acc[i][jn][r];
                } else {
                    float *c = C + (long long)gm * ldc + gn;
                    *c = alpha * acc[i][jn][r] + (beta != 0.0f ? beta * *c : 0.0f);
                }
            }
}

}  // namespace

extern "C" {

// K slices of one product: with few output tiles and a long K (weight
// gradients), enough slices to give every SM a couple of blocks, as many as
// the scratch (work_elems floats, M x N per slice) holds; kc receives the
// slice depth (a multiple of `step`).
static int splitk(int M, int N, int K, long long tiles, int step, long long work_elems, int *kc)
{
    long long splits = 1;
    if (tiles < 2 * 152 && K > 8 * step) {
        const long long want = (2 * 152 + tiles - 1) / tiles, most = (K + 4 * step - 1) / (4 * step);
        splits = want < most ? want : most;
    }
    const long long fit = work_elems / ((long long)M * N);
    if (splits > fit) splits = fit > 1 ? fit : 1;
    *kc = (int)(((K + splits - 1) / splits + step - 1) / step * step);
    return (K + *kc - 1) / *kc;
}

int nn_gemm(int transA, int transB, int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
            float beta, float *C, int ldc, float *work, long long work_elems, void *stream)
{
    if (M < 0 || N < 0 || K < 0 || !C || (K > 0 && (!A || !B)) || work_elems < 0 || (work_elems > 0 && !work))
        return 1;
    if (M == 0 || N == 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    int kc = 0;
    const int splits = splitk(M, N, K, (long long)((N + GT - 1) / GT) * ((M + GT - 1) / GT), GK, work_elems, &kc);
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, splits);
    if (!transA && !transB) k_gemm<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    else if (!transA && transB) k_gemm<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    else if (transA && !transB) k_gemm<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    else k_gemm<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    if (splits > 1) k_splitk_sum<<<blocks_for((long long)M * N), TPB, 0, st>>>(C, ldc, work, M, N, splits, beta);
    return status(st);
}

int nn_gemm_bf16(int transA, int transB, int M, int N, int K, float alpha, const float *A, int lda, const float *B,
                 int ldb, float beta, float *C, int ldc, float *work, long long work_elems, void *stream)
{
    if (M < 0 || N < 0 || K < 0 || !C || (K > 0 && (!A || !B)) || work_elems < 0 || (work_elems > 0 && !work))
        return 1;
    if (M == 0 || N == 0) return 0;
    if (K == 0) return nn_gemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work, work_elems, stream);
    cudaStream_t st = (cudaStream_t)stream;
    int kc = 0;
    const int splits = splitk(M, N, K, (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM), BK, work_elems, &kc);
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    if (!transA && !transB) k_gemm_bf16<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    else if (!transA && transB) k_gemm_bf16<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    else if (transA && !transB) k_gemm_bf16<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    else k_gemm_bf16<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kc, work);
    if (splits > 1) k_splitk_sum<<<blocks_for((long long)M * N), TPB, 0, st>>>(C, ldc, work, M, N, splits, beta);
    return status(st);
}

int nn_im2col3(const float *x, int C, int B, int H, int W, float *col, void *stream)
{
    if (!x || !col || C <= 0 || B <= 0 || H <= 0 || W <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_im2col3<<<blocks_for((long long)C * 9 * B * H * W), TPB, 0, st>>>(x, C, B, H, W, col);
    return status(st);
}

int nn_col2im3_add(const float *col, int C, int B, int H, int W, float *dx, void *stream)
{
    if (!col || !dx || C <= 0 || B <= 0 || H <= 0 || W <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_col2im3<<<blocks_for((long long)C * B * H * W), TPB, 0, st>>>(col, C, B, H, W, dx);
    return status(st);
}

int nn_bias_act(float *y, const float *bias, int Cout, long long P, int relu, void *stream)
{
    if (!y || !bias || Cout <= 0 || P <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_bias_act<<<blocks_for((long long)Cout * P), TPB, 0, st>>>(y, bias, Cout, P, relu);
    return status(st);
}

int nn_act_bwd_bias(const float *y, float *dy, float *db, int Cout, long long P, int relu, void *stream)
{
    if (!y || !dy || !db || Cout <= 0 || P <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    const int vec = (P & 3) == 0 && (((uintptr_t)y | (uintptr_t)dy) & 15) == 0;
    k_relu_bwd_bias<<<Cout, 1024, 0, st>>>(y, dy, db, P, relu, vec);
    return status(st);
}

int nn_pool2(const float *x, long long planes, int H, int W, float *y, void *stream)
{
    if (!x || !y || planes <= 0 || H < 2 || W < 2 || (H | W) & 1) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_pool2<<<blocks_for(planes * (H / 2) * (W / 2)), TPB, 0, st>>>(x, planes, H, W, y);
    return status(st);
}

int nn_pool2_bwd_add(const float *dy, long long planes, int H, int W, float *dx, void *stream)
{
    if (!dy || !dx || planes <= 0 || H < 2 || W < 2 || (H | W) & 1) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_pool2_bwd<<<blocks_for(planes * H * W), TPB, 0, st>>>(dy, planes, H, W, dx);
    return status(st);
}

int nn_up2(const float *x, long long planes, int h, int w, float *y, void *stream)
{
    if (!x || !y || planes <= 0 || h <= 0 || w <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_up2<<<blocks_for(planes * 4 * h * w), TPB, 0, st>>>(x, planes, h, w, y);
    return status(st);
}

int nn_up2_bwd_add(const float *dy, long long planes, int h, int w, float *dx, void *stream)
{
    if (!dy || !dx || planes <= 0 || h <= 0 || w <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_up2_bwd<<<blocks_for(planes * h * w), TPB, 0, st>>>(dy, planes, h, w, dx);
    return status(st);
}

int nn_mse(const float *y, const float *t, long long n, float *dy, double *loss, void *stream)
{
    if (!y || !t || !dy || !loss || n <= 0) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_zero_f<<<1, 32, 0, st>>>((float *)loss, 2);
    k_mse<<<blocks_for(n), TPB, 0, st>>>(y, t, n, dy, loss);
    return status(st);
}

int nn_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float beta1, float beta2, float eps,
            int step, void *stream)
{
    if (!p || !g || !m || !v || n <= 0 || step < 1) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<blocks_for(n), TPB, 0, st>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return status(st);
}

int nn_zero(float *x, long long n, void *stream)
{
    if (!x || n < 0) return 1;
    if (n == 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    k_zero_f<<<blocks_for(n), TPB, 0, st>>>(x, n);
    return status(st);
}

}  // extern "C"
